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
};

int batch_md_blocks(int nmax, int P, int d);
cudaError_t batch_launch_md(const RepArgs* ra, const BatchGrid& g, bool pre, cudaStream_t st);
cudaError_t batch_launch_forces(const RepArgs* ra, const BatchGrid& g, cudaStream_t st, ProfMarks* pm);
cudaError_t batch_launch_exchange(const RepArgs* ra, const BatchGrid& g, cudaStream_t st, ProfMarks* pm);
cudaError_t batch_launch_scalars(const RepArgs* ra, const BatchGrid& g, cudaStream_t st);
size_t xsolo_smem();
