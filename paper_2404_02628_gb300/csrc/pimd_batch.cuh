// Batched replicas (uneven N, beta, xi): per-replica launch arguments kept in
// device memory, so that one launch of each step kernel covers every replica
// (blockIdx.z selects the replica).
#pragma once
#include "pimd_md.cuh"
#include "pimd_xdf.cuh"

struct RepArgs {
    BeadView bv;          // beads of the replica ([P][d][n_pad] slices of the batch arrays)
    ForceParams fp;       // k_s = P/beta^2 etc. of the replica
    MDParams mp;          // kT = 1/beta, Q of the replica
    XView xv;             // exchange workspace view (store mode, band width = nb: no helpers)
    FinalizeOut fo;       // endpoint-force output (f, part)
    double* part_spr;     // springs partials [gx_spr][P]
    double* part_pair;    // pair partials [gx_pair][P][2]
    double* part_md;      // kinetic/thermostat partials [gx_md][2]
    ScalarSources ss;     // scalar reduction sources -> out[SC_COUNT]
};

// Grid extents shared by all replicas of a batch (the largest replica's).
struct BatchGrid {
    int R, P, d, M;
    int mixed;
    int gx_spr, gx_pair, gx_md, gx_prep, gx_fin, gx_table, nb_max;
    int pair_t;       // pair-kernel block size (particles per block), 64/128/256
    int gx_pair_max;  // pair partial-sum blocks per slice allocated (for the smallest block)
    const int2* tiles;   // device: (replica, factor tile) of every replica with xi > 0
    int n_tiles;
    const int2* blocks;  // device: (replica, diagonal block) of every replica with xi > 0
    int n_blocks;
};

// Work list of the batched recursion and band sums, run as one persistent
// launch after the prep, factor-tile and block-operator kernels: each block
// claims the next item, waits (bounded) until the items its item depends on
// are done, runs it, and counts it done.  Recursion items (longest replicas
// first) come before all band items, and a band item depends only on the
// two recursion items of its replica, which were claimed by blocks already
// running: the launch needs no co-residency.
enum { BI_REC = 3, BI_BAND = 4 };
struct BatchItem {
    int type, r, a, b;  // kind, replica; recursion: a = direction; band: a = block, b = direction
};
struct BatchSched {
    const BatchItem* items;
    int n_items;
    int* next;        // next item to claim (zeroed before each launch)
    int* done;        // [R][4] finished recursion items at [r][3] (zeroed before each launch)
    const int* need;  // [R][4] recursion items of each replica at [r][3]
    int* err;
    int spin_limit;
};

// Springs and trap + pairs of every replica as (replica, slice, particle
// block) units taken grid-stride from a flat list: prefix[r] is the first unit
// of replica r (R + 1 entries), gx the partial-sum stride per slice.
struct ForceUnits {
    const int* prefix;
    int R, gx;
};

int batch_md_blocks(int nmax, int P, int d);
cudaError_t batch_launch_exchange_persistent(const RepArgs* ra, const BatchSched& sc, int blocks, cudaStream_t st);
cudaError_t batch_launch_force_units(const RepArgs* ra, const ForceUnits& fu, const BatchGrid& g, int blocks,
                                     cudaStream_t st);
cudaError_t batch_launch_finalize(const RepArgs* ra, const BatchGrid& g, cudaStream_t st);
cudaError_t batch_launch_prep_tables_ops(const RepArgs* ra, const BatchGrid& g, cudaStream_t st, ProfMarks* pm);
cudaError_t batch_launch_tables_ops(const RepArgs* ra, const BatchGrid& g, cudaStream_t st, ProfMarks* pm);
cudaError_t batch_launch_md(const RepArgs* ra, const BatchGrid& g, bool pre, cudaStream_t st);
cudaError_t batch_launch_forces(const RepArgs* ra, const BatchGrid& g, cudaStream_t st, ProfMarks* pm);
cudaError_t batch_launch_exchange(const RepArgs* ra, const BatchGrid& g, cudaStream_t st, ProfMarks* pm);
cudaError_t batch_launch_scalars(const RepArgs* ra, const BatchGrid& g, cudaStream_t st);
size_t xsolo_smem();
