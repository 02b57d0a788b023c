// C ABI of the PIMD hot path (include/pimd.h): argument checks, workspace
// layout, kernel sequencing and the captured per-step CUDA graph.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>
#include <algorithm>

#include "../../include/pimd.h"
#include "pimd_exchange.cuh"
#include "pimd_md.cuh"
#include "pimd_batch.cuh"
#include "pimd_forcework.cuh"

namespace {

thread_local std::string g_global_error;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t total = 0;
    size_t add(size_t bytes)
    {
        size_t off = total;
        total = align256(total + bytes);
        return off;
    }
};

// Offsets of every workspace region.
struct ExchLayout {
    size_t Km, Ke, rho_m, rho_e, y_m, y_e, c_m, c_e, z_m, z_e, part_m, part_e, band_m, band_e, flags, err, lsum;
};

void exch_layout(Layout& L, ExchLayout& o, int N, int S, int store)
{
    const int nb = (N + 31) / 32, nbp = nb * 32;
    const long long ntiles = store ? (long long)nb * (nb + 1) / 2 : (long long)(2 * nb - 1);
    o.Km = L.add((size_t)ntiles * 1024 * sizeof(double));
    o.Ke = L.add((size_t)ntiles * 1024 * sizeof(int));
    o.rho_m = L.add(nbp * sizeof(double));
    o.rho_e = L.add(nbp * sizeof(int));
    o.y_m = L.add((nbp + 1) * sizeof(double));
    o.y_e = L.add((nbp + 1) * sizeof(int));
    o.c_m = L.add((nbp + 1) * sizeof(double));
    o.c_e = L.add((nbp + 1) * sizeof(int));
    o.z_m = L.add(nbp * sizeof(double));
    o.z_e = L.add(nbp * sizeof(int));
    o.part_m = L.add((size_t)2 * nb * S * 32 * 4 * sizeof(double));
    o.part_e = L.add((size_t)2 * nb * S * 32 * sizeof(int));
    o.band_m = L.add((size_t)2 * nb * 2 * 32 * 4 * sizeof(double));
    o.band_e = L.add((size_t)2 * nb * 2 * 32 * sizeof(int));
    o.flags = L.add((size_t)(2 * nb + 2 * nb * S) * sizeof(int));
    o.err = L.add(4 * sizeof(int));
    o.lsum = L.add((size_t)exch_prep_blocks(N) * 2 * sizeof(double));
}

ExchView exch_view(char* base, const ExchLayout& o, int N, int P, int d, double beta, double xi, int S, int store,
                   const double* a, const double* b, int lda, int ldb, int spin_limit, int n_help)
{
    ExchView v;
    memset(&v, 0, sizeof(v));
    v.N = N;
    v.nb = (N + 31) / 32;
    v.d = d;
    v.S = S;
    v.store = store;
    v.xi_zero = (xi == 0.0);
    v.kappa = P / (2.0 * beta);
    v.ks = P / (beta * beta);
    v.beta = beta;
    v.log_xi = (xi > 0.0) ? log(xi) : 0.0;
    v.a = a;
    v.b = b;
    v.lda = lda;
    v.ldb = ldb;
    v.Km = (double*)(base + o.Km);
    v.Ke = (int*)(base + o.Ke);
    v.rho_m = (double*)(base + o.rho_m);
    v.rho_e = (int*)(base + o.rho_e);
    v.y_m = (double*)(base + o.y_m);
    v.y_e = (int*)(base + o.y_e);
    v.c_m = (double*)(base + o.c_m);
    v.c_e = (int*)(base + o.c_e);
    v.z_m = (double*)(base + o.z_m);
    v.z_e = (int*)(base + o.z_e);
    v.part_m = (double*)(base + o.part_m);
    v.part_e = (int*)(base + o.part_e);
    v.band_m = (double*)(base + o.band_m);
    v.band_e = (int*)(base + o.band_e);
    v.flags = (int*)(base + o.flags);
    v.err = (int*)(base + o.err);
    v.lsum = (double*)(base + o.lsum);
    v.spin_limit = default_spin_limit(spin_limit);
    if (n_help < 2) n_help = 2;
    v.n_help_f = n_help / 2;
    v.n_help_b = n_help - v.n_help_f;
    return v;
}

int device_sms()
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return sms;
}

int default_helpers(const pimd_config& cfg)
{
    if (cfg.helper_ctas > 0) return cfg.helper_ctas;
    int sms = device_sms();
    return sms > 4 ? sms - 2 : 2;
}

constexpr int EX_STREAMS = 4;  // helper-partial streams per block the workspace holds
// streams a single system's double-float recursion uses before autotuning
// (at most EX_STREAMS; measured best or near it at N = 1600 and 10000)
constexpr int XDF_STREAMS_DEFAULT = 3;

// Workspace regions of the double-float exchange path.
struct XLayout {
    size_t ah, al, bh, bl, crh, crl, tab, lnn, M, G, Q, P, yh, yl, ye, ch, cl, ce, uh, ul,
        wh, wl,
        parth, partl, parte, bandh, bandl, bande, flags, err, lsum, lam;
};

// entries of an ln n table that covers every row index of an N-particle exchange part
static int ln_entries(int N) { return (N + 1 + 31) / 32 * 32; }

void xdf_layout(Layout& L, XLayout& o, int N, int S, int W, int store)
{
    const int nb = (N + 1 + 31) / 32, np = nb * 32;
    const long long nt = xdf_ntiles(nb, W, store);
    const size_t f = sizeof(float), i4 = sizeof(int);
    o.ah = L.add(3 * np * f);
    o.al = L.add(3 * np * f);
    o.bh = L.add(3 * np * f);
    o.bl = L.add(3 * np * f);
    o.crh = L.add(np * f);
    o.crl = L.add(np * f);
    o.tab = L.add(256 * sizeof(float2));
    o.lnn = L.add(np * sizeof(double));
    o.M = L.add((size_t)nt * sizeof(XTile));
    o.G = L.add((size_t)nb * sizeof(XTile));
    o.Q = L.add((size_t)nb * sizeof(XTile));
    o.P = L.add((size_t)nb * sizeof(XTile));
    o.yh = L.add(np * f);
    o.yl = L.add(np * f);
    o.ye = L.add(np * i4);
    o.ch = L.add(np * f);
    o.cl = L.add(np * f);
    o.ce = L.add(np * i4);
    o.uh = L.add(3 * np * f);
    o.ul = L.add(3 * np * f);
    o.wh = L.add(3 * np * f);
    o.wl = L.add(3 * np * f);
    o.parth = L.add((size_t)2 * nb * S * 32 * 4 * f);
    o.partl = L.add((size_t)2 * nb * S * 32 * 4 * f);
    o.parte = L.add((size_t)2 * nb * S * 32 * i4);
    o.bandh = L.add((size_t)4 * nb * 32 * 4 * f);  // band sums, then diagonal-tile sums
    o.bandl = L.add((size_t)4 * nb * 32 * 4 * f);
    o.bande = L.add((size_t)4 * nb * 32 * i4);
    o.flags = L.add((size_t)(2 * nb + 2 * nb * S + 1) * i4);  // chain, partial flags, band-item counter
    o.err = L.add(4 * i4);
    o.lsum = L.add((size_t)xdf_prep_blocks(np) * 2 * sizeof(double));
    o.lam = L.add(4 * sizeof(double));
}

XView xdf_view(char* base, const XLayout& o, int N, int P, int d, double beta, double xi, int S, int W, int store,
               const double* a, const double* b, int lda, int ldb, int spin_limit, int n_help)
{
    XView v;
    memset(&v, 0, sizeof v);
    v.N = N;
    v.nb = (N + 1 + 31) / 32;
    v.npad = v.nb * 32;
    v.d = d;
    v.S = S;
    v.W = W;
    v.store = store;
    v.xi_zero = (xi == 0.0);
    v.kappa = P / (2.0 * beta);
    v.ks = P / (beta * beta);
    v.beta = beta;
    v.log_xi = (xi > 0.0) ? log(xi) : 0.0;
    v.kap_h = (float)v.kappa;
    v.kap_l = (float)(v.kappa - (double)v.kap_h);
    v.a = a;
    v.b = b;
    v.lda = lda;
    v.ldb = ldb;
#define XP(name, T) v.name = (T*)(base + o.name)
    XP(ah, float); XP(al, float); XP(bh, float); XP(bl, float); XP(crh, float); XP(crl, float);
    v.tab = (const float2*)(base + o.tab);
    v.lnn = (const double*)(base + o.lnn);
    XP(M, XTile); XP(G, XTile); XP(Q, XTile); XP(P, XTile);
    XP(yh, float); XP(yl, float); XP(ye, int); XP(ch, float); XP(cl, float); XP(ce, int);
    XP(uh, float); XP(ul, float); XP(wh, float); XP(wl, float);
    XP(parth, float); XP(partl, float); XP(parte, int); XP(bandh, float); XP(bandl, float); XP(bande, int);
    XP(flags, int); XP(err, int); XP(lsum, double); XP(lam, double);
#undef XP
    v.spin_limit = default_spin_limit(spin_limit);
    if (n_help < 2) n_help = 2;
    v.n_help_f = n_help / 2;
    v.n_help_b = n_help - v.n_help_f;
    return v;
}

int cfg_band(const pimd_config& c) { return c.exch_band > 0 ? c.exch_band : 4; }

}  // namespace

struct pimd_ctx {
    int N, P, d;
    double beta, omega, g, s, xi, A;
    pimd_config cfg;
    std::string err;
    // bound state
    bool bound = false;
    pimd_buffers buf;
    cudaStream_t st = nullptr;
    cudaStream_t cap = nullptr;  // private stream used only to capture the step graph
    cudaGraphExec_t graph = nullptr;
    bool graph_failed = false;
    long long steps = 0;
    Layout L;
    int nsp = 1;                         // species with exchange recursions of their own (pimd_set_species)
    int sp_n[PIMD_MAXSP] = {}, sp_off[PIMD_MAXSP] = {};  // particles and first particle of each species
    ExchLayout exs[PIMD_MAXSP];
    XLayout xls[PIMD_MAXSP];
    bool use_df = true;
    size_t off_lnn, off_spr, off_pair, off_fin, off_md, off_sc, off_flag;
    int n_help;
    int pair_t = 128;  // pair-kernel block size (pimd_autotune)
    int n_force = 0;   // force-worker blocks folded into the recursion launch (0: separate kernels)
    int n_streams = XDF_STREAMS_DEFAULT;  // helper-partial streams per block of the recursion (1..EX_STREAMS)
    struct HostReport {  // pinned: device error word, non-finite flag and scalar slots, read in one round trip
        int err, flag;
        double sc[SC_COUNT];
    }* host_rep = nullptr;
    int fused_gx = 0;  // particle blocks per slice of the last folded force evaluation (0: not folded)
    ExchView xvs[PIMD_MAXSP];  // per species; species 0 holds the error word and exp table all share
    XView xds[PIMD_MAXSP];
    BeadView bv;
    ForceParams fp;
    MDParams mp;
    const char* slot_names[64] = {};
};

struct pimd_vb {
    int N, P, d;
    double beta, xi;
    int n_help;
    int store;       // 1: factor table stored (12 bytes per term), 0: recomputed where used
    Layout L;
    XLayout xl;
    size_t off_fin;
};

// Automatic table mode of the exchange-potential handle: store the N(N+1)/2
// factors up to N = 16383 (about 1.6 GB), recompute them above.
constexpr int VB_STORE_MAX_N = 16383;

static void vb_layout(pimd_vb* h)
{
    h->L = Layout();
    xdf_layout(h->L, h->xl, h->N, EX_STREAMS, 4, h->store);
    h->off_fin = h->L.add((size_t)xdf_finalize_blocks(h->N) * sizeof(double));
}

static pimd_status fail(pimd_t c, pimd_status s, const std::string& m)
{
    if (c) c->err = m;
    else g_global_error = m;
    return s;
}

static pimd_status cuda_fail(pimd_t c, cudaError_t e, const char* where)
{
    return fail(c, PIMD_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

extern "C" void pimd_default_config(pimd_config* cfg)
{
    if (!cfg) return;
    memset(cfg, 0, sizeof(*cfg));
    cfg->dt = 0.01;
    cfg->nhc_len = 4;
    cfg->nhc_Q = 0.0;
    cfg->mass = 1.0;
    cfg->precision = PIMD_PREC_FP64;
    cfg->amp_convention = PIMD_AMP_PAPER;
    cfg->table_mode = PIMD_TABLE_STORE;
    cfg->thermostat = 1;
    cfg->helper_ctas = 0;
    cfg->spin_limit = 0;
    cfg->exchange_arith = PIMD_XARITH_DF;
    cfg->exch_band = 0;
    cfg->nhc_fp32 = 0;
    cfg->batch_schedule = PIMD_BATCH_PERSISTENT;
}

extern "C" pimd_status pimd_create(int N, int P, int d, double beta, double omega, double g, double s, double xi,
                                   pimd_t* out)
{
    if (!out) return fail(nullptr, PIMD_EINVAL, "pimd_create: out is NULL");
    *out = nullptr;
    if (N < 1 || N > (1 << 22)) return fail(nullptr, PIMD_EINVAL, "pimd_create: N must be in [1, 4194304]");
    if (P < 2 || P > 65535) return fail(nullptr, PIMD_EINVAL, "pimd_create: P must be in [2, 65535]");
    if (d < 1 || d > 3) return fail(nullptr, PIMD_EINVAL, "pimd_create: d must be 1, 2 or 3");
    if (!(beta > 0.0) || !isfinite(beta)) return fail(nullptr, PIMD_EINVAL, "pimd_create: beta must be > 0");
    if (!(omega >= 0.0) || !isfinite(omega)) return fail(nullptr, PIMD_EINVAL, "pimd_create: omega must be >= 0");
    if (!isfinite(g)) return fail(nullptr, PIMD_EINVAL, "pimd_create: g must be finite");
    if (!(s > 0.0) || !isfinite(s)) return fail(nullptr, PIMD_EINVAL, "pimd_create: s must be > 0");
    if (!(xi >= 0.0 && xi <= 1.0)) return fail(nullptr, PIMD_EINVAL, "pimd_create: xi must be in [0, 1]");
    pimd_ctx* c = new pimd_ctx();
    c->N = N;
    c->P = P;
    c->d = d;
    c->beta = beta;
    c->omega = omega;
    c->g = g;
    c->s = s;
    c->xi = xi;
    pimd_default_config(&c->cfg);
    c->A = g / (M_PI * s * s);
    c->nsp = 1;
    c->sp_n[0] = N;
    c->sp_off[0] = 0;
    *out = c;
    return PIMD_OK;
}

extern "C" pimd_status pimd_set_species(pimd_t c, int n_species, const int* counts)
{
    if (!c || !counts) return fail(c, PIMD_EINVAL, "pimd_set_species: NULL argument");
    if (c->bound) return fail(c, PIMD_ESTATE, "pimd_set_species: context already bound");
    if (n_species < 1 || n_species > PIMD_MAXSP) return fail(c, PIMD_EINVAL, "pimd_set_species: n_species must be in [1, 4]");
    long long tot = 0;
    for (int sp = 0; sp < n_species; ++sp) {
        if (counts[sp] < 1) return fail(c, PIMD_EINVAL, "pimd_set_species: every species needs at least one particle");
        tot += counts[sp];
    }
    if (tot != c->N) return fail(c, PIMD_EINVAL, "pimd_set_species: counts must add up to N");
    c->nsp = n_species;
    int off = 0;
    for (int sp = 0; sp < n_species; ++sp) {
        c->sp_n[sp] = counts[sp];
        c->sp_off[sp] = off;
        off += counts[sp];
    }
    return PIMD_OK;
}

extern "C" pimd_status pimd_configure(pimd_t c, const pimd_config* cfg)
{
    if (!c || !cfg) return fail(c, PIMD_EINVAL, "pimd_configure: NULL argument");
    if (c->bound) return fail(c, PIMD_ESTATE, "pimd_configure: context already bound");
    if (!(cfg->dt > 0.0) || !isfinite(cfg->dt)) return fail(c, PIMD_EINVAL, "pimd_configure: dt must be > 0");
    if (cfg->nhc_len < 1 || cfg->nhc_len > 8) return fail(c, PIMD_EINVAL, "pimd_configure: nhc_len must be in [1, 8]");
    if (!(cfg->mass > 0.0)) return fail(c, PIMD_EINVAL, "pimd_configure: mass must be > 0");
    if (cfg->precision != PIMD_PREC_FP64 && cfg->precision != PIMD_PREC_MIXED)
        return fail(c, PIMD_EINVAL, "pimd_configure: unknown precision");
    if (cfg->amp_convention != PIMD_AMP_PAPER && cfg->amp_convention != PIMD_AMP_RAW)
        return fail(c, PIMD_EINVAL, "pimd_configure: unknown amp_convention");
    if (cfg->table_mode != PIMD_TABLE_STORE && cfg->table_mode != PIMD_TABLE_RECOMPUTE)
        return fail(c, PIMD_EINVAL, "pimd_configure: unknown table_mode");
    if (cfg->helper_ctas < 0 || cfg->spin_limit < 0) return fail(c, PIMD_EINVAL, "pimd_configure: negative count");
    if (cfg->exchange_arith != PIMD_XARITH_DF && cfg->exchange_arith != PIMD_XARITH_FP64)
        return fail(c, PIMD_EINVAL, "pimd_configure: unknown exchange_arith");
    if (cfg->exch_band != 0 && (cfg->exch_band < 2 || cfg->exch_band > XDF_MAXW))
        return fail(c, PIMD_EINVAL, "pimd_configure: exch_band must be 0 or in [2, 5]");
    c->cfg = *cfg;
    c->A = (cfg->amp_convention == PIMD_AMP_PAPER) ? c->g / (M_PI * c->s * c->s) : c->g;
    return PIMD_OK;
}

static void ctx_layout(pimd_ctx* c)
{
    c->L = Layout();
    c->use_df = c->cfg.exchange_arith == PIMD_XARITH_DF;
    // ln n for every species, first so that its offset never moves (the
    // autotuner re-lays the rest out for other band widths)
    c->off_lnn = c->L.add((size_t)ln_entries(c->N) * sizeof(double));
    for (int sp = 0; sp < c->nsp; ++sp) {
        if (c->use_df)
            xdf_layout(c->L, c->xls[sp], c->sp_n[sp], EX_STREAMS, cfg_band(c->cfg), c->cfg.table_mode == PIMD_TABLE_STORE);
        else
            exch_layout(c->L, c->exs[sp], c->sp_n[sp], EX_STREAMS, c->cfg.table_mode == PIMD_TABLE_STORE);
    }
    c->off_spr = c->L.add((size_t)springs_grid_x(c->N) * c->P * sizeof(double));
    c->off_pair = c->L.add((size_t)pair_grid_x(c->N, PAIR_T_MIN) * c->P * 2 * sizeof(double));
    // finalize partials of every species, one after the other
    c->off_fin = c->L.add((size_t)(std::max(exch_finalize_blocks(c->N), xdf_finalize_blocks(c->N)) + PIMD_MAXSP) *
                          sizeof(double));
    c->off_md = c->L.add((size_t)md_blocks(c->N, c->P, c->d) * 2 * sizeof(double));
    c->off_sc = c->L.add(SC_COUNT * sizeof(double));
    c->off_flag = c->L.add(4 * sizeof(int));
}

extern "C" pimd_status pimd_workspace_bytes(pimd_t c, int n_pad, size_t* bytes)
{
    if (!c || !bytes) return fail(c, PIMD_EINVAL, "pimd_workspace_bytes: NULL argument");
    if (n_pad < c->N || (n_pad & 31)) return fail(c, PIMD_EINVAL, "pimd_workspace_bytes: n_pad must be >= N and a multiple of 32");
    ctx_layout(c);
    *bytes = c->L.total;
    return PIMD_OK;
}

// Exchange views of the bound buffers under the current configuration: one
// per species, over that species' particles (beads 1 and P offset by its
// first particle).  Every species reports into species 0's error word and
// reads species 0's exp table.
static void ctx_views(pimd_ctx* c)
{
    const pimd_buffers* b = &c->buf;
    const int np = b->n_pad;
    for (int sp = 0; sp < c->nsp; ++sp) {
        const double* rP = b->r + (size_t)(c->P - 1) * c->d * np + c->sp_off[sp];
        const double* r1 = b->r + c->sp_off[sp];
        if (c->use_df) {
            c->xds[sp] = xdf_view((char*)b->work, c->xls[sp], c->sp_n[sp], c->P, c->d, c->beta, c->xi, c->n_streams,
                                  cfg_band(c->cfg), c->cfg.table_mode == PIMD_TABLE_STORE, rP, r1, np, np,
                                  c->cfg.spin_limit, c->n_help);
            if (sp > 0) {
                c->xds[sp].err = c->xds[0].err;
                c->xds[sp].tab = c->xds[0].tab;
            }
            c->xds[sp].lnn = (const double*)((char*)b->work + c->off_lnn);
        } else {
            c->xvs[sp] = exch_view((char*)b->work, c->exs[sp], c->sp_n[sp], c->P, c->d, c->beta, c->xi, EX_STREAMS,
                                   c->cfg.table_mode == PIMD_TABLE_STORE, rP, r1, np, np, c->cfg.spin_limit, c->n_help);
            if (sp > 0) c->xvs[sp].err = c->xvs[0].err;
        }
    }
}

// Finalize blocks of one species.
static int fin_blocks(const pimd_ctx* c, int n)
{
    return c->use_df ? xdf_finalize_blocks(n) : exch_finalize_blocks(n);
}

static pimd_status enqueue_forces(pimd_ctx* c, cudaStream_t st, double* f, bool exch, bool inter,
                                  ProfMarks* pm = nullptr)
{
    cudaError_t e;
    ForceParams fp = c->fp;
    fp.accumulate = 0;
    char* base = (char*)c->buf.work;
    c->fused_gx = 0;
    if (exch && inter && c->use_df && c->xi != 0.0 && c->n_force > 0 && c->nsp == 1) {
        // springs and trap + pairs run as force workers inside the recursion launch
        ForceWork fw;
        memset(&fw, 0, sizeof fw);
        fw.b = c->bv;
        fw.b.f = f;
        fw.fp = c->fp;
        fw.part_spr = (double*)(base + c->off_spr);
        fw.part_pair = (double*)(base + c->off_pair);
        fw.gx = (c->N + XDF_THREADS - 1) / XDF_THREADS;
        fw.counter = (int*)(base + c->off_flag) + 1;
        e = cudaMemsetAsync(fw.counter, 0, sizeof(int), st);
        if (e == cudaSuccess) e = xdf_launch_forward(c->xds[0], st, pm, &fw, c->n_force);
        if (e != cudaSuccess) return cuda_fail(c, e, "exchange recursion with force workers");
        FinalizeOut o;
        memset(&o, 0, sizeof(o));
        o.f = f;
        o.ldf = c->buf.n_pad;
        o.P = c->P;
        o.part = (double*)(base + c->off_fin);
        e = xdf_launch_adjoint(c->xds[0], o, st, pm);
        if (e != cudaSuccess) return cuda_fail(c, e, "exchange forces");
        c->fused_gx = fw.gx;
        return PIMD_OK;
    }
    if (exch) {
        e = launch_springs(c->bv, fp, f, (double*)(base + c->off_spr), st);
        prof_mark(pm, "springs", st);
        if (e != cudaSuccess) return cuda_fail(c, e, "springs kernel");
        fp.accumulate = 1;
    } else {
        e = launch_zero((double*)(base + c->off_spr), springs_grid_x(c->N) * c->P, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "zero kernel");
    }
    if (inter) {
        e = launch_pair(c->bv, fp, f, (double*)(base + c->off_pair), st, c->pair_t);
        prof_mark(pm, "pair", st);
        if (e != cudaSuccess) return cuda_fail(c, e, "pair kernel");
    } else {
        e = launch_zero((double*)(base + c->off_pair), (size_t)pair_grid_x(c->N, c->pair_t) * c->P * 2, st);
        if (e != cudaSuccess) return cuda_fail(c, e, "zero kernel");
    }
    if (exch) {
        // one exchange recursion per species, each over its own particles
        int fin_off = 0;
        for (int sp = 0; sp < c->nsp; ++sp) {
            FinalizeOut o;
            memset(&o, 0, sizeof(o));
            o.f = f + c->sp_off[sp];
            o.ldf = c->buf.n_pad;
            o.P = c->P;
            o.part = (double*)(base + c->off_fin) + fin_off;
            if (c->use_df) {
                e = xdf_launch_forward(c->xds[sp], st, pm);
                if (e != cudaSuccess) return cuda_fail(c, e, "exchange recursion");
                e = xdf_launch_adjoint(c->xds[sp], o, st, pm);
            } else {
                e = exch_launch_forward(c->xvs[sp], st, 1, pm);
                if (e != cudaSuccess) return cuda_fail(c, e, "exchange recursion");
                e = exch_launch_adjoint(c->xvs[sp], o, exch_finalize_blocks(c->sp_n[sp]), st, pm);
            }
            if (e != cudaSuccess) return cuda_fail(c, e, "exchange forces");
            fin_off += fin_blocks(c, c->sp_n[sp]);
        }
    }
    return PIMD_OK;
}

static pimd_status enqueue_scalars(pimd_ctx* c, cudaStream_t st)
{
    char* base = (char*)c->buf.work;
    cudaError_t e = launch_md_energy(c->bv, c->mp, (double*)(base + c->off_md), st);
    if (e != cudaSuccess) return cuda_fail(c, e, "energy kernel");
    ScalarSources s;
    memset(&s, 0, sizeof(s));
    s.springs = (double*)(base + c->off_spr);
    s.n_springs = (c->fused_gx ? c->fused_gx : springs_grid_x(c->N)) * c->P;
    s.nsp = c->nsp;
    s.n_fin = 0;
    for (int sp = 0; sp < c->nsp; ++sp) {
        s.lsum[sp] = c->use_df ? c->xds[sp].lsum : c->xvs[sp].lsum;
        s.n_lsum[sp] = c->use_df ? xdf_prep_blocks(c->xds[sp].npad) : exch_prep_blocks(c->sp_n[sp]);
        s.lam[sp] = c->use_df ? c->xds[sp].lam : nullptr;
        s.y_m[sp] = c->xvs[sp].y_m;
        s.y_e[sp] = c->xvs[sp].y_e;
        s.c_m[sp] = c->xvs[sp].c_m;
        s.c_e[sp] = c->xvs[sp].c_e;
        s.N[sp] = c->sp_n[sp];
        s.n_fin += fin_blocks(c, c->sp_n[sp]);
    }
    s.pair = (double*)(base + c->off_pair);
    s.n_pair = (c->fused_gx ? c->fused_gx : pair_grid_x(c->N, c->pair_t)) * c->P;
    s.fin = (double*)(base + c->off_fin);
    s.md = (double*)(base + c->off_md);
    s.n_md = md_blocks(c->N, c->P, c->d);
    s.xi_zero = (c->xi == 0.0);
    s.log_xi = (c->xi > 0.0) ? log(c->xi) : 0.0;
    s.out = (double*)(base + c->off_sc);
    e = launch_scalars(s, st);
    if (e != cudaSuccess) return cuda_fail(c, e, "scalar reduction");
    return PIMD_OK;
}

static pimd_status enqueue_step(pimd_ctx* c, cudaStream_t st, ProfMarks* pm = nullptr)
{
    cudaError_t e = launch_md_pre(c->bv, c->mp, st);
    prof_mark(pm, "md_pre", st);
    if (e != cudaSuccess) return cuda_fail(c, e, "md pre kernel");
    pimd_status s = enqueue_forces(c, st, c->buf.f, true, true, pm);
    if (s != PIMD_OK) return s;
    e = launch_md_post(c->bv, c->mp, st);
    prof_mark(pm, "md_post", st);
    if (e != cudaSuccess) return cuda_fail(c, e, "md post kernel");
    return PIMD_OK;
}

static pimd_status check_device_error(pimd_ctx* c)
{
    int h[2] = {0, 0};
    char* base = (char*)c->buf.work;
    cudaError_t e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronize");
    int* errp = c->use_df ? c->xds[0].err : c->xvs[0].err;
    e = cudaMemcpy(&h[0], errp, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "error word read");
    e = cudaMemcpy(&h[1], base + c->off_flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "flag read");
    if (h[0] != 0) {
        cudaMemsetAsync(errp, 0, sizeof(int), c->st);
        cudaStreamSynchronize(c->st);
        char msg[160];
        snprintf(msg, sizeof msg, "device wait gave up (code 0x%08x); increase spin_limit or check co-residency", h[0]);
        return fail(c, PIMD_ETIMEOUT, msg);
    }
    return PIMD_OK;
}

extern "C" pimd_status pimd_bind(pimd_t c, const pimd_buffers* b, void* stream)
{
    if (!c || !b) return fail(c, PIMD_EINVAL, "pimd_bind: NULL argument");
    if (c->bound) return fail(c, PIMD_ESTATE, "pimd_bind: already bound");
    if (!b->r || !b->p || !b->f || !b->work) return fail(c, PIMD_EINVAL, "pimd_bind: NULL buffer");
    if (c->cfg.thermostat && (!b->eta || !b->peta)) return fail(c, PIMD_EINVAL, "pimd_bind: thermostat buffers missing");
    if (b->n_pad < c->N || (b->n_pad & 31)) return fail(c, PIMD_EINVAL, "pimd_bind: n_pad must be >= N and a multiple of 32");
    if (((uintptr_t)b->work & 255) != 0) return fail(c, PIMD_EINVAL, "pimd_bind: workspace must be 256-byte aligned");
    ctx_layout(c);
    if (b->work_bytes < c->L.total) {
        char msg[160];
        snprintf(msg, sizeof msg, "pimd_bind: workspace too small (%zu < %zu bytes)", b->work_bytes, c->L.total);
        return fail(c, PIMD_ENOMEM, msg);
    }
    c->buf = *b;
    c->st = (cudaStream_t)stream;
    if (!c->host_rep) {
        void* hp = nullptr;
        cudaError_t e2 = cudaMallocHost(&hp, sizeof(pimd_ctx::HostReport));
        if (e2 != cudaSuccess) return cuda_fail(c, e2, "pimd_bind: pinned report buffer");
        c->host_rep = (pimd_ctx::HostReport*)hp;
    }
    c->n_help = default_helpers(c->cfg);
    c->n_force = 0;
    if (c->use_df && c->A != 0.0 && c->xi != 0.0 && c->nsp == 1) {
        // SMs the recursion's helpers do not need take the springs and pairs
        const int sms = device_sms(), nb = (c->N + 1 + 31) / 32;
        if (c->cfg.helper_ctas <= 0) c->n_help = std::max(4, std::min(sms - 2 - 8, nb));
        c->n_force = std::max(0, sms - 2 - c->n_help);
    }
    const int np = b->n_pad;
    ctx_views(c);
    c->bv.N = c->N;
    c->bv.P = c->P;
    c->bv.d = c->d;
    c->bv.ld = np;
    c->bv.r = b->r;
    c->bv.p = b->p;
    c->bv.f = b->f;
    c->bv.eta = b->eta;
    c->bv.peta = b->peta;
    c->bv.M = c->cfg.nhc_len;
    c->fp.ks = c->P / (c->beta * c->beta);
    c->fp.omega2 = c->omega * c->omega;
    c->fp.A = c->A;
    c->fp.inv_s2 = 1.0 / (c->s * c->s);
    c->fp.mixed = c->cfg.precision == PIMD_PREC_MIXED;
    c->fp.accumulate = 0;
    force_constants(c->fp, c->P);
    c->mp.dt = c->cfg.dt;
    c->mp.mass = c->cfg.mass;
    c->mp.kT = 1.0 / c->beta;
    c->mp.Q = c->cfg.nhc_Q > 0.0 ? c->cfg.nhc_Q : c->beta / c->P;
    c->mp.inv_mass = 1.0 / c->mp.mass;
    c->mp.inv_Q = 1.0 / c->mp.Q;
    c->mp.thermostat = c->cfg.thermostat;
    c->mp.nhc_fp32 = c->cfg.nhc_fp32 != 0;
    nhc_constants(c->mp);
    cudaError_t e;
    if (c->cfg.thermostat) {
        const size_t n = (size_t)c->cfg.nhc_len * c->P * c->d * np;
        e = cudaMemsetAsync(b->eta, 0, n * sizeof(double), c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->peta, 0, n * sizeof(double), c->st);
        if (e != cudaSuccess) return cuda_fail(c, e, "pimd_bind: thermostat reset");
    }
    e = cudaMemsetAsync(c->use_df ? c->xds[0].err : c->xvs[0].err, 0, 4 * sizeof(int), c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "pimd_bind: error word reset");
    if (c->use_df) {
        e = xdf_upload_table((float2*)c->xds[0].tab, c->st);
        if (e == cudaSuccess) e = xdf_fill_lntab((double*)c->xds[0].lnn, ln_entries(c->N), c->st);
        if (e != cudaSuccess) return cuda_fail(c, e, "pimd_bind: exp and log table upload");
    }
    e = cudaMemsetAsync((char*)b->work + c->off_flag, 0, 4 * sizeof(int), c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "pimd_bind: flag reset");
    c->bound = true;
    c->steps = 0;
    pimd_status s = enqueue_forces(c, c->st, b->f, true, true);
    if (s != PIMD_OK) {
        c->bound = false;
        return s;
    }
    return PIMD_OK;
}

extern "C" pimd_status pimd_forces(pimd_t c, double* V_out)
{
    if (!c) return fail(c, PIMD_EINVAL, "pimd_forces: NULL handle");
    if (!c->bound) return fail(c, PIMD_ESTATE, "pimd_forces: not bound");
    pimd_status s = enqueue_forces(c, c->st, c->buf.f, true, true);
    if (s != PIMD_OK) return s;
    if (V_out) {
        s = enqueue_scalars(c, c->st);
        if (s != PIMD_OK) return s;
        s = check_device_error(c);
        if (s != PIMD_OK) return s;
        double t[SC_COUNT];
        cudaError_t e = cudaMemcpy(t, (char*)c->buf.work + c->off_sc, sizeof t, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "pimd_forces: scalar read");
        const double Vxi = t[SC_EINT] + (t[SC_GLINK] - t[SC_LAMBDA]) / c->beta;
        *V_out = Vxi + t[SC_U] / c->P;
        if (!isfinite(*V_out)) return fail(c, PIMD_ENONFINITE, "pimd_forces: non-finite potential");
    }
    return PIMD_OK;
}

static pimd_status partial_forces(pimd_t c, double* f_out, double* out, bool exch, const char* name)
{
    if (!c || !f_out) return fail(c, PIMD_EINVAL, std::string(name) + ": NULL argument");
    if (!c->bound) return fail(c, PIMD_ESTATE, std::string(name) + ": not bound");
    if (!exch) {
        cudaError_t e = cudaMemsetAsync(f_out, 0, (size_t)c->P * c->d * c->buf.n_pad * sizeof(double), c->st);
        if (e != cudaSuccess) return cuda_fail(c, e, name);
    }
    pimd_status s = enqueue_forces(c, c->st, f_out, exch, !exch);
    if (s != PIMD_OK) return s;
    if (out) {
        s = enqueue_scalars(c, c->st);
        if (s != PIMD_OK) return s;
        s = check_device_error(c);
        if (s != PIMD_OK) return s;
        double t[SC_COUNT];
        cudaError_t e = cudaMemcpy(t, (char*)c->buf.work + c->off_sc, sizeof t, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, name);
        *out = exch ? t[SC_EINT] + (t[SC_GLINK] - t[SC_LAMBDA]) / c->beta : t[SC_U] / c->P;
    }
    return PIMD_OK;
}

extern "C" pimd_status pimd_exchange_forces(pimd_t c, double* f_out, double* V_out)
{
    return partial_forces(c, f_out, V_out, true, "pimd_exchange_forces");
}

extern "C" pimd_status pimd_interaction_forces(pimd_t c, double* f_out, double* U_out)
{
    return partial_forces(c, f_out, U_out, false, "pimd_interaction_forces");
}

extern "C" pimd_status pimd_step_eager(pimd_t c, int nsteps)
{
    if (!c) return fail(c, PIMD_EINVAL, "pimd_step_eager: NULL handle");
    if (!c->bound) return fail(c, PIMD_ESTATE, "pimd_step_eager: not bound");
    if (nsteps < 0) return fail(c, PIMD_EINVAL, "pimd_step_eager: nsteps < 0");
    for (int n = 0; n < nsteps; ++n) {
        pimd_status s = enqueue_step(c, c->st);
        if (s != PIMD_OK) return s;
    }
    c->steps += nsteps;
    return PIMD_OK;
}

static pimd_status build_graph(pimd_ctx* c)
{
    cudaError_t e;
    if (!c->cap) {
        e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(c, e, "graph stream");
    }
    e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c, e, "begin capture");
    pimd_status s = enqueue_step(c, c->cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->cap, &g);
    if (s != PIMD_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "end capture");
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph = nullptr;
        return cuda_fail(c, e, "graph instantiate");
    }
    return PIMD_OK;
}

extern "C" pimd_status pimd_step(pimd_t c, int nsteps)
{
    if (!c) return fail(c, PIMD_EINVAL, "pimd_step: NULL handle");
    if (!c->bound) return fail(c, PIMD_ESTATE, "pimd_step: not bound");
    if (nsteps < 0) return fail(c, PIMD_EINVAL, "pimd_step: nsteps < 0");
    if (!c->graph && !c->graph_failed) {
        if (build_graph(c) != PIMD_OK) {
            c->graph_failed = true;
            cudaGetLastError();
        }
    }
    if (!c->graph) return pimd_step_eager(c, nsteps);
    for (int n = 0; n < nsteps; ++n) {
        cudaError_t e = cudaGraphLaunch(c->graph, c->st);
        if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
    }
    c->steps += nsteps;
    return PIMD_OK;
}

extern "C" pimd_status pimd_step_profiled(pimd_t c, int nsteps, double* ms_out, int max_slots, int* n_slots)
{
    if (!c || !ms_out || !n_slots || max_slots < 1) return fail(c, PIMD_EINVAL, "pimd_step_profiled: bad argument");
    if (!c->bound) return fail(c, PIMD_ESTATE, "pimd_step_profiled: not bound");
    if (nsteps < 1) return fail(c, PIMD_EINVAL, "pimd_step_profiled: nsteps < 1");
    ProfMarks pm;
    memset(&pm, 0, sizeof pm);
    for (int i = 0; i < 64; ++i) {
        cudaError_t e = cudaEventCreate(&pm.ev[i]);
        if (e != cudaSuccess) {
            for (int k = 0; k < i; ++k) cudaEventDestroy(pm.ev[k]);
            return cuda_fail(c, e, "pimd_step_profiled: event create");
        }
    }
    for (int i = 0; i < max_slots; ++i) ms_out[i] = 0.0;
    pimd_status s = PIMD_OK;
    int nk = 0;
    for (int n = 0; n < nsteps && s == PIMD_OK; ++n) {
        pm.n = 0;
        prof_mark(&pm, "start", c->st);
        s = enqueue_step(c, c->st, &pm);
        if (s != PIMD_OK) break;
        cudaError_t e = cudaEventSynchronize(pm.ev[pm.n - 1]);
        if (e != cudaSuccess) {
            s = cuda_fail(c, e, "pimd_step_profiled: sync");
            break;
        }
        nk = pm.n - 1;
        for (int k = 1; k < pm.n && k - 1 < max_slots; ++k) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, pm.ev[k - 1], pm.ev[k]);
            ms_out[k - 1] += ms;
            c->slot_names[k - 1] = pm.name[k];
        }
    }
    for (int i = 0; i < 64; ++i) cudaEventDestroy(pm.ev[i]);
    if (s != PIMD_OK) return s;
    c->steps += nsteps;
    *n_slots = nk < max_slots ? nk : max_slots;
    return check_device_error(c);
}

// ---------------------------------------------------------------------------
// Autotuning: time the force evaluation (which leaves r and p untouched) for
// each candidate launch shape, keep the fastest, and remember the choice in
// an optional text cache keyed by device and problem.

static std::string device_key()
{
    int dev = 0;
    cudaDeviceProp pr;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return "unknown";
    std::string n = pr.name;
    for (char& ch : n)
        if (ch == ' ' || ch == '|') ch = '_';
    return n + "_sm" + std::to_string(pr.multiProcessorCount);
}

static bool cache_lookup(const char* path, const std::string& key, std::string& value)
{
    if (!path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof line, f)) {
        std::string l(line);
        while (!l.empty() && (l.back() == '\n' || l.back() == '\r')) l.pop_back();
        const size_t bar = l.find('|');
        if (bar != std::string::npos && l.substr(0, bar) == key) {
            value = l.substr(bar + 1);  // the last entry for a key wins
            found = true;
        }
    }
    fclose(f);
    return found;
}

static void cache_store(const char* path, const std::string& key, const std::string& value)
{
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s|%s\n", key.c_str(), value.c_str());
    fclose(f);
}

static int cache_field(const std::string& v, const char* name, int dflt)
{
    const std::string k = std::string(name) + "=";
    const size_t p = v.find(k);
    return p == std::string::npos ? dflt : atoi(v.c_str() + p + k.size());
}

template <class F>
static double time_ms(cudaStream_t st, int reps, F&& enqueue)
{
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return 1e30;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return 1e30;
    }
    enqueue();  // warm
    cudaEventRecord(a, st);
    for (int i = 0; i < reps; ++i) enqueue();
    cudaEventRecord(b, st);
    float ms = 1e30f;
    if (cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return (double)ms / reps;
}

static void drop_graph(pimd_ctx* c)
{
    if (c->graph) cudaGraphExecDestroy(c->graph);
    c->graph = nullptr;
    c->graph_failed = false;
}

// Bytes of the double-float exchange regions of every species for band width W.
static size_t xdf_footprint(const pimd_ctx* c, int W)
{
    Layout L;
    for (int sp = 0; sp < c->nsp; ++sp) {
        XLayout xl;
        xdf_layout(L, xl, c->sp_n[sp], EX_STREAMS, W, c->cfg.table_mode == PIMD_TABLE_STORE);
    }
    return L.total;
}

extern "C" pimd_status pimd_autotune(pimd_t c, const char* cache_path)
{
    if (!c) return fail(c, PIMD_EINVAL, "pimd_autotune: NULL handle");
    if (!c->bound) return fail(c, PIMD_ESTATE, "pimd_autotune: not bound");
    char kb[256];
    snprintf(kb, sizeof kb, "single N=%d P=%d d=%d prec=%d arith=%d table=%d xi0=%d g0=%d sp=%d", c->N, c->P, c->d,
             c->cfg.precision, c->cfg.exchange_arith, c->cfg.table_mode, c->xi == 0.0, c->A == 0.0, c->nsp);
    const std::string key = device_key() + " " + kb;
    std::string val;
    int bestW = cfg_band(c->cfg), bestT = c->pair_t, bestH = c->n_help, bestF = c->n_force, bestS = c->n_streams;
    const int sms = device_sms();
    const bool can_fold = c->use_df && c->A != 0.0 && c->xi != 0.0 && c->nsp == 1;
    if (cache_lookup(cache_path, key, val)) {
        bestW = cache_field(val, "W", bestW);
        bestT = cache_field(val, "pair_t", bestT);
        bestH = cache_field(val, "help", bestH);
        bestF = cache_field(val, "fold", bestF);
        bestS = cache_field(val, "S", bestS);
    } else {
        std::vector<int> Ws, Ts;
        if (c->use_df && c->xi != 0.0) {
            const size_t bound = xdf_footprint(c, cfg_band(c->cfg));
            for (int W = 2; W <= XDF_MAXW; ++W)
                if (xdf_footprint(c, W) <= bound) Ws.push_back(W);  // candidate fits the bound workspace
        }
        if (Ws.empty()) Ws.push_back(bestW);
        if (c->A != 0.0) Ts = {64, 128, 256};
        else Ts = {c->pair_t};
        // launch shapes: (pair block, helper blocks, force-worker blocks); the
        // folded shapes hand the SMs the helpers leave to springs and pairs
        struct Shape { int T, H, F; };
        std::vector<Shape> shapes;
        const int H_sep = default_helpers(c->cfg);
        for (int T : Ts) shapes.push_back({T, H_sep, 0});
        if (can_fold && sms > 16) {
            const int nb = (c->N + 1 + 31) / 32;
            std::vector<int> Hs;
            for (int H : {nb / 2, nb, (5 * nb) / 4, (3 * nb) / 2, (7 * nb) / 4, 2 * nb, (5 * nb) / 2, 3 * nb}) {
                H = std::max(4, std::min(sms - 2 - 8, H));
                if (std::find(Hs.begin(), Hs.end(), H) == Hs.end()) Hs.push_back(H);
            }
            for (int H : Hs) shapes.push_back({c->pair_t, H, sms - 2 - H});
        }
        // helper-partial streams per block of the double-float recursion
        std::vector<int> Ss;
        if (c->use_df && c->xi != 0.0) Ss = {2, 3, 4};
        else Ss = {c->n_streams};
        double best = 1e30;
        const int W0 = c->cfg.exch_band;
        for (int W : Ws)
            for (const Shape& sh : shapes)
                for (int S : Ss) {
                    c->cfg.exch_band = W;
                    c->pair_t = sh.T;
                    c->n_help = sh.H;
                    c->n_force = sh.F;
                    c->n_streams = S;
                    ctx_views(c);
                    pimd_status st = PIMD_OK;
                    const double ms = time_ms(c->st, 5, [&] {
                        if (st == PIMD_OK) st = enqueue_forces(c, c->st, c->buf.f, true, true);
                    });
                    if (st != PIMD_OK) return st;
                    if (ms < best) {
                        best = ms;
                        bestW = W;
                        bestT = sh.T;
                        bestH = sh.H;
                        bestF = sh.F;
                        bestS = S;
                    }
                }
        c->cfg.exch_band = W0;
        char vb[96];
        snprintf(vb, sizeof vb, "W=%d;pair_t=%d;help=%d;fold=%d;S=%d", bestW, bestT, bestH, bestF, bestS);
        cache_store(cache_path, key, vb);
    }
    if (bestW < 2 || bestW > XDF_MAXW || !pair_block_ok(bestT) || bestH < 2 || bestF < 0 || bestS < 1 ||
        bestS > EX_STREAMS ||
        (bestF > 0 && (!can_fold || 2 + bestH + bestF > sms)))
        return fail(c, PIMD_EINVAL, "pimd_autotune: bad cache entry");
    if (c->use_df && xdf_footprint(c, bestW) > xdf_footprint(c, cfg_band(c->cfg)))
        bestW = cfg_band(c->cfg);  // cached choice does not fit this workspace
    c->cfg.exch_band = bestW;
    c->pair_t = bestT;
    c->n_streams = bestS;
    c->n_help = bestH;
    c->n_force = bestF;
    ctx_layout(c);
    ctx_views(c);
    drop_graph(c);
    pimd_status s = enqueue_forces(c, c->st, c->buf.f, true, true);
    if (s != PIMD_OK) return s;
    return check_device_error(c);
}

extern "C" pimd_status pimd_tuning(pimd_t c, int* exch_band, int* pair_block, int* helpers, int* force_blocks,
                                   int* streams)
{
    if (!c || !exch_band || !pair_block) return fail(c, PIMD_EINVAL, "pimd_tuning: NULL argument");
    *exch_band = cfg_band(c->cfg);
    *pair_block = c->pair_t;
    if (helpers) *helpers = c->n_help;
    if (force_blocks) *force_blocks = c->n_force;
    if (streams) *streams = c->n_streams;
    return PIMD_OK;
}

extern "C" const char* pimd_profile_slot_name(pimd_t c, int slot)
{
    if (!c || slot < 0 || slot >= 64 || !c->slot_names[slot]) return "";
    return c->slot_names[slot];
}

// Estimators of one system from its scalar slots (primitive and virial
// readings; Sec. III spring terms, Sec. II U).  False if any is non-finite.
static bool fill_estimates(const double* t, int Pi, int Ni, int di, double beta, int thermostat, long long steps,
                           pimd_estimates* out)
{
    const double P = Pi, N = Ni, d = di;
    out->V_xi = t[SC_EINT] + (t[SC_GLINK] - t[SC_LAMBDA]) / beta;
    out->V_xi_bwd = t[SC_EINT] + (t[SC_GLINK] - t[SC_LAMBDA_B]) / beta;
    out->U_over_P = t[SC_U] / P;
    out->spring = t[SC_EINT] + t[SC_SPRING_X];
    out->virial = t[SC_VIRIAL];
    out->kinetic = t[SC_KIN];
    out->E_prim = 0.5 * P * d * N / beta - out->spring + out->U_over_P;
    out->E_vir = out->U_over_P + out->virial / (2.0 * P);
    out->H_conserved = out->kinetic + out->V_xi + out->U_over_P + (thermostat ? t[SC_THERMO] : 0.0);
    out->step = steps;
    const double* q = &out->E_prim;
    for (int i = 0; i < 9; ++i)
        if (!isfinite(q[i])) return false;
    return true;
}

extern "C" pimd_status pimd_estimators(pimd_t c, pimd_estimates* out)
{
    if (!c || !out) return fail(c, PIMD_EINVAL, "pimd_estimators: NULL argument");
    if (!c->bound) return fail(c, PIMD_ESTATE, "pimd_estimators: not bound");
    pimd_status s = enqueue_scalars(c, c->st);
    if (s != PIMD_OK) return s;
    char* base = (char*)c->buf.work;
    cudaError_t e = cudaMemsetAsync(base + c->off_flag, 0, sizeof(int), c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "pimd_estimators: flag reset");
    e = launch_nonfinite_scan(c->buf.f, c->N, c->P, c->d, c->buf.n_pad, (int*)(base + c->off_flag), c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "pimd_estimators: scan");
    // error word, flag and scalars in one round trip through the pinned buffer
    pimd_ctx::HostReport* hr = c->host_rep;
    int* errp = c->use_df ? c->xds[0].err : c->xvs[0].err;
    e = cudaMemcpyAsync(&hr->err, errp, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hr->flag, base + c->off_flag, sizeof(int), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hr->sc, base + c->off_sc, sizeof hr->sc, cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "pimd_estimators: read");
    if (hr->err != 0) {
        const int code = hr->err;
        cudaMemsetAsync(errp, 0, sizeof(int), c->st);
        cudaStreamSynchronize(c->st);
        char msg[160];
        snprintf(msg, sizeof msg, "device wait gave up (code 0x%08x); increase spin_limit or check co-residency", code);
        return fail(c, PIMD_ETIMEOUT, msg);
    }
    double t[SC_COUNT];
    memcpy(t, hr->sc, sizeof t);
    const int flag = hr->flag;
    if (!fill_estimates(t, c->P, c->N, c->d, c->beta, c->cfg.thermostat, c->steps, out))
        return fail(c, PIMD_ENONFINITE, "pimd_estimators: non-finite estimate");
    if (flag) return fail(c, PIMD_ENONFINITE, "pimd_estimators: non-finite force");
    return PIMD_OK;
}

extern "C" pimd_status pimd_state_bytes(pimd_t c, size_t* bytes)
{
    if (!c || !bytes) return fail(c, PIMD_EINVAL, "pimd_state_bytes: NULL argument");
    if (!c->bound) return fail(c, PIMD_ESTATE, "pimd_state_bytes: not bound");
    const size_t n = (size_t)c->P * c->d * c->buf.n_pad;
    const size_t m = c->cfg.thermostat ? (size_t)c->cfg.nhc_len * n : 0;
    *bytes = 64 + (3 * n + 2 * m) * sizeof(double);
    return PIMD_OK;
}

struct StateHeader {
    char magic[8];
    long long N, P, d, n_pad, M, steps, thermostat, pad;
};

extern "C" pimd_status pimd_get_state(pimd_t c, void* host, size_t bytes)
{
    size_t need = 0;
    pimd_status s = pimd_state_bytes(c, &need);
    if (s != PIMD_OK) return s;
    if (!host || bytes < need) return fail(c, PIMD_EINVAL, "pimd_get_state: buffer too small");
    const size_t n = (size_t)c->P * c->d * c->buf.n_pad;
    const size_t m = c->cfg.thermostat ? (size_t)c->cfg.nhc_len * n : 0;
    StateHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, "PIMDST1", 8);
    h.N = c->N;
    h.P = c->P;
    h.d = c->d;
    h.n_pad = c->buf.n_pad;
    h.M = c->cfg.nhc_len;
    h.steps = c->steps;
    h.thermostat = c->cfg.thermostat;
    char* out = (char*)host;
    memcpy(out, &h, sizeof h);
    double* q = (double*)(out + 64);
    cudaError_t e = cudaMemcpyAsync(q, c->buf.r, n * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(q + n, c->buf.p, n * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(q + 2 * n, c->buf.f, n * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess && m) e = cudaMemcpyAsync(q + 3 * n, c->buf.eta, m * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess && m) e = cudaMemcpyAsync(q + 3 * n + m, c->buf.peta, m * sizeof(double), cudaMemcpyDeviceToHost, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "pimd_get_state");
    return PIMD_OK;
}

extern "C" pimd_status pimd_set_state(pimd_t c, const void* host, size_t bytes)
{
    size_t need = 0;
    pimd_status s = pimd_state_bytes(c, &need);
    if (s != PIMD_OK) return s;
    if (!host || bytes < need) return fail(c, PIMD_EINVAL, "pimd_set_state: buffer too small");
    StateHeader h;
    memcpy(&h, host, sizeof h);
    if (memcmp(h.magic, "PIMDST1", 8) != 0 || h.N != c->N || h.P != c->P || h.d != c->d || h.n_pad != c->buf.n_pad ||
        h.M != c->cfg.nhc_len || h.thermostat != c->cfg.thermostat)
        return fail(c, PIMD_EINVAL, "pimd_set_state: blob does not match this context");
    const size_t n = (size_t)c->P * c->d * c->buf.n_pad;
    const size_t m = c->cfg.thermostat ? (size_t)c->cfg.nhc_len * n : 0;
    const double* q = (const double*)((const char*)host + 64);
    cudaError_t e = cudaMemcpyAsync(c->buf.r, q, n * sizeof(double), cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->buf.p, q + n, n * sizeof(double), cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->buf.f, q + 2 * n, n * sizeof(double), cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess && m) e = cudaMemcpyAsync(c->buf.eta, q + 3 * n, m * sizeof(double), cudaMemcpyHostToDevice, c->st);
    if (e == cudaSuccess && m) e = cudaMemcpyAsync(c->buf.peta, q + 3 * n + m, m * sizeof(double), cudaMemcpyHostToDevice, c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "pimd_set_state");
    c->steps = h.steps;
    return PIMD_OK;
}

extern "C" pimd_status pimd_density_accumulate(pimd_t c, int nbins, double r_max, double* hist)
{
    if (!c || !hist) return fail(c, PIMD_EINVAL, "pimd_density_accumulate: NULL argument");
    if (!c->bound) return fail(c, PIMD_ESTATE, "pimd_density_accumulate: not bound");
    if (nbins < 1 || nbins > DENSITY_MAX_BINS || !(r_max > 0.0) || !std::isfinite(r_max))
        return fail(c, PIMD_EINVAL, "pimd_density_accumulate: nbins in [1, 8192] and finite r_max > 0 required");
    cudaError_t e = launch_density(c->bv, nbins, r_max / nbins, hist, c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "pimd_density_accumulate");
    return PIMD_OK;
}

extern "C" pimd_status pimd_init_state(pimd_t c, unsigned long long seed)
{
    if (!c) return fail(c, PIMD_EINVAL, "pimd_init_state: NULL handle");
    if (!c->bound) return fail(c, PIMD_ESTATE, "pimd_init_state: not bound");
    cudaError_t e = launch_init_state(c->bv, sqrt(c->mp.mass * c->mp.kT), seed, c->st);
    if (e == cudaSuccess && c->cfg.thermostat) {
        const size_t n = (size_t)c->cfg.nhc_len * c->P * c->d * c->buf.n_pad;
        e = cudaMemsetAsync(c->buf.eta, 0, n * sizeof(double), c->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(c->buf.peta, 0, n * sizeof(double), c->st);
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "pimd_init_state");
    c->steps = 0;
    return enqueue_forces(c, c->st, c->buf.f, true, true);
}

cudaError_t launch_cycle_naive(const BeadView& b, double ks, double* E, int ldE, cudaStream_t st);

extern "C" pimd_status pimd_cycle_energies_naive(pimd_t c, double* E_out, int ldE)
{
    if (!c || !E_out) return fail(c, PIMD_EINVAL, "pimd_cycle_energies_naive: NULL argument");
    if (!c->bound) return fail(c, PIMD_ESTATE, "pimd_cycle_energies_naive: not bound");
    if (ldE < c->N) return fail(c, PIMD_EINVAL, "pimd_cycle_energies_naive: ldE < N");
    if (c->N > 65535) return fail(c, PIMD_EINVAL, "pimd_cycle_energies_naive: N > 65535");
    cudaError_t e = launch_cycle_naive(c->bv, c->P / (c->beta * c->beta), E_out, ldE, c->st);
    if (e != cudaSuccess) return cuda_fail(c, e, "pimd_cycle_energies_naive");
    return PIMD_OK;
}

extern "C" pimd_status pimd_sync(pimd_t c)
{
    if (!c) return fail(c, PIMD_EINVAL, "pimd_sync: NULL handle");
    if (!c->bound) return fail(c, PIMD_ESTATE, "pimd_sync: not bound");
    return check_device_error(c);
}

extern "C" const char* pimd_last_error(pimd_t c) { return c ? c->err.c_str() : g_global_error.c_str(); }
extern "C" const char* pimd_global_error(void) { return g_global_error.c_str(); }

extern "C" void pimd_destroy(pimd_t c)
{
    if (!c) return;
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->host_rep) cudaFreeHost(c->host_rep);
    delete c;
}

// ---------------------------------------------------------------------------
// Exchange potential alone (autograd).

extern "C" pimd_status pimd_vb_create(int N, int P, int d, double beta, double xi, pimd_vb_t* out)
{
    if (!out) return fail(nullptr, PIMD_EINVAL, "pimd_vb_create: out is NULL");
    *out = nullptr;
    if (N < 1 || N > (1 << 22) || P < 2 || d < 1 || d > 3 || !(beta > 0.0) || !(xi >= 0.0 && xi <= 1.0))
        return fail(nullptr, PIMD_EINVAL, "pimd_vb_create: bad argument");
    pimd_vb* h = new pimd_vb();
    h->N = N;
    h->P = P;
    h->d = d;
    h->beta = beta;
    h->xi = xi;
    pimd_config cfg;
    pimd_default_config(&cfg);
    h->n_help = default_helpers(cfg);
    h->store = N <= VB_STORE_MAX_N;
    vb_layout(h);
    *out = h;
    return PIMD_OK;
}

extern "C" pimd_status pimd_vb_set_table_mode(pimd_vb_t h, int table_mode)
{
    if (!h) return fail(nullptr, PIMD_EINVAL, "pimd_vb_set_table_mode: NULL handle");
    if (table_mode == PIMD_TABLE_STORE) h->store = 1;
    else if (table_mode == PIMD_TABLE_RECOMPUTE) h->store = 0;
    else if (table_mode == -1) h->store = h->N <= VB_STORE_MAX_N;
    else return fail(nullptr, PIMD_EINVAL, "pimd_vb_set_table_mode: unknown mode");
    vb_layout(h);
    return PIMD_OK;
}

extern "C" pimd_status pimd_vb_workspace_bytes(pimd_vb_t h, size_t* bytes)
{
    if (!h || !bytes) return fail(nullptr, PIMD_EINVAL, "pimd_vb_workspace_bytes: NULL argument");
    *bytes = h->L.total;
    return PIMD_OK;
}

static pimd_status vb_check(pimd_vb_t h, const double* r1, const double* rP, int ld, void* work, size_t bytes, const char* nm)
{
    if (!h || !r1 || !rP || !work) return fail(nullptr, PIMD_EINVAL, std::string(nm) + ": NULL argument");
    if (ld < h->N) return fail(nullptr, PIMD_EINVAL, std::string(nm) + ": ld < N");
    if (((uintptr_t)work & 255) != 0) return fail(nullptr, PIMD_EINVAL, std::string(nm) + ": workspace not 256-byte aligned");
    if (bytes < h->L.total) return fail(nullptr, PIMD_ENOMEM, std::string(nm) + ": workspace too small");
    return PIMD_OK;
}

extern "C" pimd_status pimd_vb_forward(pimd_vb_t h, const double* r1, const double* rP, int ld, void* work,
                                       size_t work_bytes, double* V_out, void* stream)
{
    pimd_status s = vb_check(h, r1, rP, ld, work, work_bytes, "pimd_vb_forward");
    if (s != PIMD_OK) return s;
    if (!V_out) return fail(nullptr, PIMD_EINVAL, "pimd_vb_forward: V_out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    XView v = xdf_view((char*)work, h->xl, h->N, h->P, h->d, h->beta, h->xi, EX_STREAMS, 4, h->store, rP, r1, ld, ld, 0,
                       h->n_help);
    cudaError_t e = cudaMemsetAsync(v.err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = xdf_upload_table((float2*)v.tab, st);
    if (e == cudaSuccess) e = xdf_fill_lntab((double*)v.lnn, v.npad, st);
    if (e == cudaSuccess) e = xdf_launch_forward(v, st, nullptr);
    if (e == cudaSuccess) e = xdf_launch_vb_value(v, V_out, st);
    if (e != cudaSuccess) return fail(nullptr, PIMD_ECUDA, std::string("pimd_vb_forward: ") + cudaGetErrorString(e));
    return PIMD_OK;
}

extern "C" pimd_status pimd_vb_backward(pimd_vb_t h, const double* r1, const double* rP, int ld, void* work,
                                        size_t work_bytes, const double* gV, double* g_r1, double* g_rP, void* stream)
{
    pimd_status s = vb_check(h, r1, rP, ld, work, work_bytes, "pimd_vb_backward");
    if (s != PIMD_OK) return s;
    if (!gV || !g_r1 || !g_rP) return fail(nullptr, PIMD_EINVAL, "pimd_vb_backward: NULL output");
    cudaStream_t st = (cudaStream_t)stream;
    XView v = xdf_view((char*)work, h->xl, h->N, h->P, h->d, h->beta, h->xi, EX_STREAMS, 4, h->store, rP, r1, ld, ld, 0,
                       h->n_help);
    FinalizeOut o;
    memset(&o, 0, sizeof(o));
    o.g1 = g_r1;
    o.gP = g_rP;
    o.ldg = ld;
    o.gscale = gV;
    o.P = h->P;
    o.part = (double*)((char*)work + h->off_fin);
    cudaError_t e = xdf_launch_adjoint(v, o, st, nullptr);
    if (e != cudaSuccess) return fail(nullptr, PIMD_ECUDA, std::string("pimd_vb_backward: ") + cudaGetErrorString(e));
    return PIMD_OK;
}

extern "C" pimd_status pimd_vb_sync(pimd_vb_t h, void* work, size_t work_bytes, void* stream)
{
    if (!h || !work) return fail(nullptr, PIMD_EINVAL, "pimd_vb_sync: NULL argument");
    if (((uintptr_t)work & 255) != 0) return fail(nullptr, PIMD_EINVAL, "pimd_vb_sync: workspace not 256-byte aligned");
    if (work_bytes < h->L.total) return fail(nullptr, PIMD_ENOMEM, "pimd_vb_sync: workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    int* errp = (int*)((char*)work + h->xl.err);
    cudaError_t e = cudaStreamSynchronize(st);
    int code = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&code, errp, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(nullptr, PIMD_ECUDA, std::string("pimd_vb_sync: ") + cudaGetErrorString(e));
    if (code != 0) {
        e = cudaMemsetAsync(errp, 0, sizeof(int), st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return fail(nullptr, PIMD_ECUDA, std::string("pimd_vb_sync: ") + cudaGetErrorString(e));
        char msg[160];
        snprintf(msg, sizeof msg, "pimd_vb_sync: a device wait gave up (code 0x%08x); the last values are NaN", code);
        return fail(nullptr, PIMD_ETIMEOUT, msg);
    }
    return PIMD_OK;
}

extern "C" void pimd_vb_destroy(pimd_vb_t h) { delete h; }

// ---------------------------------------------------------------------------
// Batched replicas (uneven N, beta, xi; shared P, d, omega, g, s and config):
// every step kernel is one launch over all replicas, the exchange recursion
// one block per replica and direction (xsolo), the step one CUDA graph.

namespace {
constexpr int BATCH_NMAX = 2047;  // xsolo keeps h of every block in shared memory
}

struct pimd_batch {
    int R, P, d;
    double omega, g, s, A;
    std::vector<int> N, npad;
    std::vector<double> beta, xi;
    pimd_config cfg;
    std::string err;
    bool bound = false;
    pimd_batch_buffers buf;
    cudaStream_t st = nullptr, cap = nullptr;
    cudaGraphExec_t graph = nullptr;
    bool graph_failed = false;
    long long steps = 0;
    std::vector<size_t> off;  // bead element offset of each replica (R + 1 entries)
    BatchGrid grid;
    Layout L;
    size_t off_args = 0, off_err = 0, off_sc = 0, off_tab = 0, off_flag = 0;
    std::vector<RepArgs> args;
    const char* slot_names[64] = {};
    // persistent schedule: work list, per-replica phase counts, force-unit prefix
    int sched = PIMD_BATCH_PERSISTENT;
    std::vector<BatchItem> items;
    std::vector<int> need, prefix;
    std::vector<int2> tiles, blocks;  // flat (replica, tile) and (replica, diagonal block) lists
    size_t off_items = 0, off_need = 0, off_cnt = 0, off_prefix = 0, off_tiles = 0, off_blocks = 0;
    std::vector<size_t> off_parts;  // per replica: springs and pair partial regions
    size_t parts_bytes = 0;
    cudaStream_t side = nullptr;    // second stream of the step (springs and pairs)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

// The persistent launch's work list (see BatchItem): the recursions longest
// replica first, then the band sums shortest replica first (their recursions
// end first); need[r][BI_REC] counts a replica's recursion items.  Also the
// flat (replica, tile) and (replica, diagonal block) lists of the factor-tile
// and block-operator kernels.
static void batch_items(pimd_batch* b)
{
    std::vector<int> order(b->R);
    for (int r = 0; r < b->R; ++r) order[r] = r;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->N[x] > b->N[y]; });
    auto nbof = [&](int r) { return (b->N[r] + 1 + 31) / 32; };
    b->items.clear();
    b->tiles.clear();
    b->blocks.clear();
    b->need.assign((size_t)b->R * 4, 0);
    for (int r : order) {
        if (b->xi[r] == 0.0) continue;  // no exchange recursion at xi = 0
        b->items.push_back({BI_REC, r, 0, 0});
        b->items.push_back({BI_REC, r, 1, 0});
        b->need[r * 4 + BI_REC] = 2;
        const long long nt = xdf_ntiles(nbof(r), nbof(r), 1);
        for (long long t = 0; t < nt; ++t) b->tiles.push_back(make_int2(r, (int)t));
        for (int J = 0; J < nbof(r); ++J) b->blocks.push_back(make_int2(r, J));
    }
    for (int q = b->R - 1; q >= 0; --q) {
        const int r = order[q];
        if (b->xi[r] == 0.0) continue;
        for (int J = 0; J < nbof(r); ++J)
            for (int dir = 0; dir < 2; ++dir) b->items.push_back({BI_BAND, r, J, dir});
    }
}

// First force unit of every replica for the current pair block (R + 1 entries).
static void batch_prefix(pimd_batch* b)
{
    b->prefix.assign(b->R + 1, 0);
    for (int r = 0; r < b->R; ++r)
        b->prefix[r + 1] = b->prefix[r] + b->P * pair_grid_x(b->N[r], b->grid.pair_t);
}

static pimd_status bfail(pimd_batch_t b, pimd_status s, const std::string& m)
{
    if (b) b->err = m;
    else g_global_error = m;
    return s;
}

static pimd_status bcuda(pimd_batch_t b, cudaError_t e, const char* where)
{
    return bfail(b, PIMD_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

extern "C" pimd_status pimd_batch_create(int R, const int* N, int P, int d, const double* beta, const double* xi,
                                         double omega, double g, double s, pimd_batch_t* out)
{
    if (!out) return bfail(nullptr, PIMD_EINVAL, "pimd_batch_create: out is NULL");
    *out = nullptr;
    if (R < 1 || R > 65535 || !N || !beta || !xi) return bfail(nullptr, PIMD_EINVAL, "pimd_batch_create: R in [1, 65535] and arrays required");
    if (P < 2 || P > 65535) return bfail(nullptr, PIMD_EINVAL, "pimd_batch_create: P must be in [2, 65535]");
    if (d < 1 || d > 3) return bfail(nullptr, PIMD_EINVAL, "pimd_batch_create: d must be 1, 2 or 3");
    if (!(omega >= 0.0) || !isfinite(omega) || !isfinite(g) || !(s > 0.0) || !isfinite(s))
        return bfail(nullptr, PIMD_EINVAL, "pimd_batch_create: omega >= 0, finite g and s > 0 required");
    for (int r = 0; r < R; ++r) {
        if (N[r] < 1 || N[r] > BATCH_NMAX) return bfail(nullptr, PIMD_EINVAL, "pimd_batch_create: each N must be in [1, 2047]");
        if (!(beta[r] > 0.0) || !isfinite(beta[r])) return bfail(nullptr, PIMD_EINVAL, "pimd_batch_create: each beta must be > 0");
        if (!(xi[r] >= 0.0 && xi[r] <= 1.0)) return bfail(nullptr, PIMD_EINVAL, "pimd_batch_create: each xi must be in [0, 1]");
    }
    pimd_batch* b = new pimd_batch();
    b->R = R;
    b->P = P;
    b->d = d;
    b->omega = omega;
    b->g = g;
    b->s = s;
    b->N.assign(N, N + R);
    b->beta.assign(beta, beta + R);
    b->xi.assign(xi, xi + R);
    b->npad.resize(R);
    b->off.resize(R + 1);
    b->off[0] = 0;
    for (int r = 0; r < R; ++r) {
        b->npad[r] = (N[r] + 31) / 32 * 32;
        b->off[r + 1] = b->off[r] + (size_t)P * d * b->npad[r];
    }
    pimd_default_config(&b->cfg);
    b->A = g / (M_PI * s * s);
    *out = b;
    return PIMD_OK;
}

extern "C" pimd_status pimd_batch_configure(pimd_batch_t b, const pimd_config* cfg)
{
    if (!b || !cfg) return bfail(b, PIMD_EINVAL, "pimd_batch_configure: NULL argument");
    if (b->bound) return bfail(b, PIMD_ESTATE, "pimd_batch_configure: already bound");
    if (!(cfg->dt > 0.0) || cfg->nhc_len < 1 || cfg->nhc_len > 8 || !(cfg->mass > 0.0))
        return bfail(b, PIMD_EINVAL, "pimd_batch_configure: dt > 0, nhc_len in [1, 8], mass > 0 required");
    if (cfg->precision != PIMD_PREC_FP64 && cfg->precision != PIMD_PREC_MIXED)
        return bfail(b, PIMD_EINVAL, "pimd_batch_configure: unknown precision");
    if (cfg->amp_convention != PIMD_AMP_PAPER && cfg->amp_convention != PIMD_AMP_RAW)
        return bfail(b, PIMD_EINVAL, "pimd_batch_configure: unknown amplitude convention");
    if (cfg->batch_schedule != PIMD_BATCH_PERSISTENT && cfg->batch_schedule != PIMD_BATCH_KERNELS)
        return bfail(b, PIMD_EINVAL, "pimd_batch_configure: unknown batch_schedule");
    b->cfg = *cfg;
    b->A = cfg->amp_convention == PIMD_AMP_RAW ? b->g : b->g / (M_PI * b->s * b->s);
    return PIMD_OK;
}

extern "C" pimd_status pimd_batch_layout(pimd_batch_t b, size_t* offsets)
{
    if (!b || !offsets) return bfail(b, PIMD_EINVAL, "pimd_batch_layout: NULL argument");
    for (int r = 0; r <= b->R; ++r) offsets[r] = b->off[r];
    return PIMD_OK;
}

// Workspace: per replica an exchange layout (store mode, band width nb) and
// its partial-sum arrays sized by the batch grid; then the RepArgs array, the
// scalar slots [R][SC_COUNT], one exp table and one error word.
static void batch_layout(pimd_batch* b, std::vector<XLayout>& xl, std::vector<size_t>& offs)
{
    int nmax = 0;
    for (int n : b->N) nmax = std::max(nmax, n);
    const int npmax = (nmax + 1 + 31) / 32 * 32, nbmax = npmax / 32;
    BatchGrid& g = b->grid;
    g.R = b->R;
    g.P = b->P;
    g.d = b->d;
    g.M = b->cfg.nhc_len;
    g.mixed = b->cfg.precision == PIMD_PREC_MIXED;
    g.gx_spr = springs_grid_x(nmax);
    if (!pair_block_ok(g.pair_t)) g.pair_t = 128;
    g.gx_pair = pair_grid_x(nmax, g.pair_t);
    g.gx_pair_max = pair_grid_x(nmax, PAIR_T_MIN);
    g.gx_md = batch_md_blocks((nmax + 31) / 32 * 32, b->P, b->d);
    g.gx_prep = xdf_prep_blocks(npmax);
    g.gx_fin = xdf_finalize_blocks(nmax);
    g.gx_table = (int)xdf_ntiles(nbmax, nbmax, 1);
    g.nb_max = nbmax;
    b->L = Layout();
    xl.resize(b->R);
    offs.resize((size_t)b->R * 5);
    for (int r = 0; r < b->R; ++r) {
        const int nb = (b->N[r] + 1 + 31) / 32;
        xdf_layout(b->L, xl[r], b->N[r], 1, nb, 1);
        offs[5 * r + 0] = b->L.add((size_t)std::max(g.gx_spr, g.gx_pair_max) * b->P * sizeof(double));
        offs[5 * r + 1] = b->L.add((size_t)g.gx_pair_max * b->P * 2 * sizeof(double));
        offs[5 * r + 2] = b->L.add((size_t)g.gx_fin * sizeof(double));
        offs[5 * r + 3] = b->L.add((size_t)g.gx_md * 2 * sizeof(double));
        offs[5 * r + 4] = b->L.add((size_t)g.gx_prep * 2 * sizeof(double));
    }
    b->off_args = b->L.add((size_t)b->R * sizeof(RepArgs));
    b->off_sc = b->L.add((size_t)b->R * SC_COUNT * sizeof(double));
    b->off_tab = b->L.add(256 * sizeof(float2));
    b->off_err = b->L.add(4 * sizeof(int));
    b->off_flag = b->L.add(4 * sizeof(int));
    batch_items(b);
    b->off_items = b->L.add(b->items.size() * sizeof(BatchItem));
    b->off_need = b->L.add((size_t)b->R * 4 * sizeof(int));
    b->off_cnt = b->L.add(((size_t)b->R * 4 + 1) * sizeof(int));
    b->off_prefix = b->L.add(((size_t)b->R + 1) * sizeof(int));
    b->off_tiles = b->L.add(b->tiles.size() * sizeof(int2));
    b->off_blocks = b->L.add(b->blocks.size() * sizeof(int2));
}

// Per-replica springs and pair partial sums: slots a schedule does not write
// must read zero, so they are cleared whenever the partial layout changes
// (bind, schedule or pair block).
static cudaError_t batch_clear_parts(pimd_batch* b)
{
    char* base = (char*)b->buf.work;
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < b->R && e == cudaSuccess; ++r) {
        e = cudaMemsetAsync(b->args[r].part_spr, 0,
                            (size_t)std::max(b->grid.gx_spr, b->grid.gx_pair_max) * b->P * sizeof(double), b->st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(b->args[r].part_pair, 0, (size_t)b->grid.gx_pair_max * b->P * 2 * sizeof(double), b->st);
    }
    (void)base;
    return e;
}

// Partial-sum counts of the scalar reduction for the current schedule and
// pair block, then uploads the replica arguments and the force-unit prefix.
static pimd_status batch_upload_args(pimd_batch* b);

extern "C" pimd_status pimd_batch_workspace_bytes(pimd_batch_t b, size_t* bytes)
{
    if (!b || !bytes) return bfail(b, PIMD_EINVAL, "pimd_batch_workspace_bytes: NULL argument");
    std::vector<XLayout> xl;
    std::vector<size_t> offs;
    batch_layout(b, xl, offs);
    *bytes = b->L.total;
    return PIMD_OK;
}

static pimd_status batch_enqueue_forces(pimd_batch* b, cudaStream_t st, ProfMarks* pm = nullptr)
{
    char* base = (char*)b->buf.work;
    const RepArgs* ra = (const RepArgs*)(base + b->off_args);
    cudaError_t e;
    if (b->sched == PIMD_BATCH_KERNELS) {
        e = batch_launch_forces(ra, b->grid, st, pm);
        if (e != cudaSuccess) return bcuda(b, e, "batch springs/pair kernels");
        e = batch_launch_exchange(ra, b->grid, st, pm);
        if (e != cudaSuccess) return bcuda(b, e, "batch exchange kernels");
        return PIMD_OK;
    }
    BatchSched sc;
    sc.items = (const BatchItem*)(base + b->off_items);
    sc.n_items = (int)b->items.size();
    sc.done = (int*)(base + b->off_cnt);
    sc.next = sc.done + (size_t)b->R * 4;
    sc.need = (const int*)(base + b->off_need);
    sc.err = (int*)(base + b->off_err);
    sc.spin_limit = default_spin_limit(b->cfg.spin_limit);
    ForceUnits fu;
    fu.prefix = (const int*)(base + b->off_prefix);
    fu.R = b->R;
    fu.gx = b->grid.gx_pair;
    const int sms = std::max(1, device_sms());
    // the side stream only when not profiling: per-kernel event times need one stream
    const bool fork = (pm == nullptr);
    if (fork) {
        e = cudaEventRecord(b->ev_fork, st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->side, b->ev_fork, 0);
        if (e != cudaSuccess) return bcuda(b, e, "batch fork");
    }
    e = batch_launch_prep_tables_ops(ra, b->grid, st, pm);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + b->off_cnt, 0, ((size_t)b->R * 4 + 1) * sizeof(int), st);
    if (e != cudaSuccess) return bcuda(b, e, "batch prep, factor tiles and block operators");
    // the recursion launch one block per SM, ahead of the force units in
    // issue order, so that its blocks find room beside them
    e = batch_launch_exchange_persistent(ra, sc, sms, st);
    prof_mark(pm, "batch_exch_persistent", st);
    if (e != cudaSuccess) return bcuda(b, e, "batch persistent exchange");
    e = batch_launch_force_units(ra, fu, b->grid, 4 * sms, fork ? b->side : st);
    prof_mark(pm, "batch_force_units", st);
    if (e != cudaSuccess) return bcuda(b, e, "batch force units");
    if (fork) {
        e = cudaEventRecord(b->ev_join, b->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->ev_join, 0);
        if (e != cudaSuccess) return bcuda(b, e, "batch join");
    }
    e = batch_launch_finalize(ra, b->grid, st);
    prof_mark(pm, "batch_exch_finalize", st);
    if (e != cudaSuccess) return bcuda(b, e, "batch endpoint forces");
    return PIMD_OK;
}

static pimd_status batch_enqueue_step(pimd_batch* b, cudaStream_t st, ProfMarks* pm = nullptr)
{
    const RepArgs* ra = (const RepArgs*)((char*)b->buf.work + b->off_args);
    cudaError_t e = batch_launch_md(ra, b->grid, true, st);
    prof_mark(pm, "batch_md_pre", st);
    if (e != cudaSuccess) return bcuda(b, e, "batch md pre kernel");
    pimd_status s = batch_enqueue_forces(b, st, pm);
    if (s != PIMD_OK) return s;
    e = batch_launch_md(ra, b->grid, false, st);
    prof_mark(pm, "batch_md_post", st);
    if (e != cudaSuccess) return bcuda(b, e, "batch md post kernel");
    return PIMD_OK;
}

static pimd_status batch_check_device(pimd_batch* b)
{
    cudaError_t e = cudaStreamSynchronize(b->st);
    if (e != cudaSuccess) return bcuda(b, e, "stream synchronize");
    int h = 0;
    int* errp = (int*)((char*)b->buf.work + b->off_err);
    e = cudaMemcpy(&h, errp, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "error word read");
    if (h != 0) {
        cudaMemsetAsync(errp, 0, sizeof(int), b->st);
        cudaStreamSynchronize(b->st);
        char msg[160];
        snprintf(msg, sizeof msg, "device wait gave up (code 0x%08x)", h);
        return bfail(b, PIMD_ETIMEOUT, msg);
    }
    return PIMD_OK;
}

extern "C" pimd_status pimd_batch_bind(pimd_batch_t b, const pimd_batch_buffers* bf, void* stream)
{
    if (!b || !bf) return bfail(b, PIMD_EINVAL, "pimd_batch_bind: NULL argument");
    if (b->bound) return bfail(b, PIMD_ESTATE, "pimd_batch_bind: already bound");
    if (!bf->r || !bf->p || !bf->f || !bf->work) return bfail(b, PIMD_EINVAL, "pimd_batch_bind: NULL buffer");
    if (b->cfg.thermostat && (!bf->eta || !bf->peta)) return bfail(b, PIMD_EINVAL, "pimd_batch_bind: thermostat buffers missing");
    if (((uintptr_t)bf->work & 255) != 0) return bfail(b, PIMD_EINVAL, "pimd_batch_bind: workspace must be 256-byte aligned");
    std::vector<XLayout> xl;
    std::vector<size_t> offs;
    batch_layout(b, xl, offs);
    if (bf->work_bytes < b->L.total) {
        char msg[160];
        snprintf(msg, sizeof msg, "pimd_batch_bind: workspace too small (%zu < %zu bytes)", bf->work_bytes, b->L.total);
        return bfail(b, PIMD_ENOMEM, msg);
    }
    b->buf = *bf;
    b->st = (cudaStream_t)stream;
    char* base = (char*)bf->work;
    const int M = b->cfg.nhc_len;
    b->args.assign(b->R, RepArgs());
    for (int r = 0; r < b->R; ++r) {
        RepArgs& a = b->args[r];
        memset(&a, 0, sizeof a);
        const int N = b->N[r], np = b->npad[r], P = b->P, d = b->d, nb = (N + 1 + 31) / 32;
        const double beta = b->beta[r];
        double* rr = bf->r + b->off[r];
        a.bv.N = N;
        a.bv.P = P;
        a.bv.d = d;
        a.bv.ld = np;
        a.bv.r = rr;
        a.bv.p = bf->p + b->off[r];
        a.bv.f = bf->f + b->off[r];
        a.bv.eta = bf->eta ? bf->eta + (size_t)M * b->off[r] : nullptr;
        a.bv.peta = bf->peta ? bf->peta + (size_t)M * b->off[r] : nullptr;
        a.bv.M = M;
        a.fp.ks = P / (beta * beta);
        a.fp.omega2 = b->omega * b->omega;
        a.fp.A = b->A;
        a.fp.inv_s2 = 1.0 / (b->s * b->s);
        a.fp.mixed = b->cfg.precision == PIMD_PREC_MIXED;
        force_constants(a.fp, P);
        a.mp.dt = b->cfg.dt;
        a.mp.mass = b->cfg.mass;
        a.mp.kT = 1.0 / beta;
        a.mp.Q = b->cfg.nhc_Q > 0.0 ? b->cfg.nhc_Q : beta / P;
        a.mp.inv_mass = 1.0 / a.mp.mass;
        a.mp.inv_Q = 1.0 / a.mp.Q;
        a.mp.thermostat = b->cfg.thermostat;
        a.mp.nhc_fp32 = b->cfg.nhc_fp32 != 0;
        nhc_constants(a.mp);
        a.xv = xdf_view(base, xl[r], N, P, d, beta, b->xi[r], 1, nb, 1, rr + (size_t)(P - 1) * d * np, rr, np, np,
                        b->cfg.spin_limit, 0);
        a.xv.err = (int*)(base + b->off_err);
        a.xv.tab = (const float2*)(base + b->off_tab);
        a.xv.lsum = (double*)(base + offs[5 * r + 4]);
        a.fo.f = a.bv.f;
        a.fo.ldf = np;
        a.fo.P = P;
        a.fo.part = (double*)(base + offs[5 * r + 2]);
        a.part_spr = (double*)(base + offs[5 * r + 0]);
        a.part_pair = (double*)(base + offs[5 * r + 1]);
        a.part_md = (double*)(base + offs[5 * r + 3]);
        ScalarSources& ss = a.ss;
        ss.springs = a.part_spr;
        ss.n_springs = b->grid.gx_spr * P;
        ss.nsp = 1;
        ss.lsum[0] = a.xv.lsum;
        ss.n_lsum[0] = b->grid.gx_prep;
        ss.pair = a.part_pair;
        ss.n_pair = b->grid.gx_pair * P;
        ss.fin = a.fo.part;
        ss.n_fin = b->grid.gx_fin;
        ss.md = a.part_md;
        ss.n_md = b->grid.gx_md;
        ss.N[0] = N;
        ss.xi_zero = b->xi[r] == 0.0;
        ss.log_xi = b->xi[r] > 0.0 ? log(b->xi[r]) : 0.0;
        ss.lam[0] = a.xv.lam;
        ss.out = (double*)(base + b->off_sc) + (size_t)r * SC_COUNT;
    }
    cudaError_t e = cudaSuccess;
    b->sched = b->cfg.batch_schedule;
    if (!b->side) e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (e == cudaSuccess && !b->ev_fork) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess && !b->ev_join) e = cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) return bcuda(b, e, "pimd_batch_bind: side stream");
    // the work list and phase counts never change after bind
    e = cudaMemcpy(base + b->off_items, b->items.data(), b->items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(base + b->off_need, b->need.data(), b->need.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !b->tiles.empty())
        e = cudaMemcpy(base + b->off_tiles, b->tiles.data(), b->tiles.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !b->blocks.empty())
        e = cudaMemcpy(base + b->off_blocks, b->blocks.data(), b->blocks.size() * sizeof(int2), cudaMemcpyHostToDevice);
    b->grid.tiles = (const int2*)(base + b->off_tiles);
    b->grid.n_tiles = (int)b->tiles.size();
    b->grid.blocks = (const int2*)(base + b->off_blocks);
    b->grid.n_blocks = (int)b->blocks.size();
    if (e != cudaSuccess) return bcuda(b, e, "pimd_batch_bind: work list");
    if (e == cudaSuccess && b->cfg.thermostat) {
        const size_t n = (size_t)M * b->off[b->R];
        e = cudaMemsetAsync(bf->eta, 0, n * sizeof(double), b->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(bf->peta, 0, n * sizeof(double), b->st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(base + b->off_err, 0, 8 * sizeof(int), b->st);
    if (e == cudaSuccess) e = xdf_upload_table((float2*)(base + b->off_tab), b->st);
    if (e != cudaSuccess) return bcuda(b, e, "pimd_batch_bind: setup");
    pimd_status us = batch_upload_args(b);
    if (us != PIMD_OK) return us;
    for (const auto& a : b->args)
        if (e == cudaSuccess) e = xdf_fill_lntab((double*)a.xv.lnn, a.xv.npad, b->st);
    if (e != cudaSuccess) return bcuda(b, e, "pimd_batch_bind: log tables");
    b->bound = true;
    b->steps = 0;
    pimd_status s = batch_enqueue_forces(b, b->st);
    if (s != PIMD_OK) {
        b->bound = false;
        return s;
    }
    return PIMD_OK;
}

extern "C" pimd_status pimd_batch_init_state(pimd_batch_t b, unsigned long long seed)
{
    if (!b) return bfail(b, PIMD_EINVAL, "pimd_batch_init_state: NULL handle");
    if (!b->bound) return bfail(b, PIMD_ESTATE, "pimd_batch_init_state: not bound");
    cudaError_t e = cudaSuccess;
    for (int r = 0; r < b->R && e == cudaSuccess; ++r)
        e = launch_init_state(b->args[r].bv, sqrt(b->args[r].mp.mass * b->args[r].mp.kT),
                              splitmix64_at(seed, (unsigned long long)r), b->st);
    if (e == cudaSuccess && b->cfg.thermostat) {
        const size_t n = (size_t)b->cfg.nhc_len * b->off[b->R];
        e = cudaMemsetAsync(b->buf.eta, 0, n * sizeof(double), b->st);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->buf.peta, 0, n * sizeof(double), b->st);
    }
    if (e != cudaSuccess) return bcuda(b, e, "pimd_batch_init_state");
    b->steps = 0;
    return batch_enqueue_forces(b, b->st);
}

extern "C" pimd_status pimd_batch_forces(pimd_batch_t b)
{
    if (!b) return bfail(b, PIMD_EINVAL, "pimd_batch_forces: NULL handle");
    if (!b->bound) return bfail(b, PIMD_ESTATE, "pimd_batch_forces: not bound");
    return batch_enqueue_forces(b, b->st);
}

extern "C" pimd_status pimd_batch_step_eager(pimd_batch_t b, int nsteps)
{
    if (!b) return bfail(b, PIMD_EINVAL, "pimd_batch_step_eager: NULL handle");
    if (!b->bound) return bfail(b, PIMD_ESTATE, "pimd_batch_step_eager: not bound");
    if (nsteps < 0) return bfail(b, PIMD_EINVAL, "pimd_batch_step_eager: nsteps < 0");
    for (int n = 0; n < nsteps; ++n) {
        pimd_status s = batch_enqueue_step(b, b->st);
        if (s != PIMD_OK) return s;
    }
    b->steps += nsteps;
    return PIMD_OK;
}

extern "C" pimd_status pimd_batch_capture_graph(pimd_batch_t b)
{
    if (!b) return bfail(b, PIMD_EINVAL, "pimd_batch_capture_graph: NULL handle");
    if (!b->bound) return bfail(b, PIMD_ESTATE, "pimd_batch_capture_graph: not bound");
    if (b->graph) return PIMD_OK;
    cudaError_t e;
    if (!b->cap) {
        e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bcuda(b, e, "graph stream");
    }
    e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(b, e, "begin capture");
    pimd_status s = batch_enqueue_step(b, b->cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->cap, &g);
    if (s != PIMD_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return bcuda(b, e, "end capture");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return bcuda(b, e, "graph instantiate");
    }
    return PIMD_OK;
}

extern "C" pimd_status pimd_batch_step(pimd_batch_t b, int nsteps)
{
    if (!b) return bfail(b, PIMD_EINVAL, "pimd_batch_step: NULL handle");
    if (!b->bound) return bfail(b, PIMD_ESTATE, "pimd_batch_step: not bound");
    if (nsteps < 0) return bfail(b, PIMD_EINVAL, "pimd_batch_step: nsteps < 0");
    if (!b->graph && !b->graph_failed) {
        if (pimd_batch_capture_graph(b) != PIMD_OK) {
            b->graph_failed = true;
            cudaGetLastError();
        }
    }
    if (!b->graph) return pimd_batch_step_eager(b, nsteps);
    for (int n = 0; n < nsteps; ++n) {
        cudaError_t e = cudaGraphLaunch(b->graph, b->st);
        if (e != cudaSuccess) return bcuda(b, e, "graph launch");
    }
    b->steps += nsteps;
    return PIMD_OK;
}

extern "C" pimd_status pimd_batch_step_profiled(pimd_batch_t b, int nsteps, double* ms_out, int max_slots, int* n_slots)
{
    if (!b || !ms_out || !n_slots || max_slots < 1) return bfail(b, PIMD_EINVAL, "pimd_batch_step_profiled: bad argument");
    if (!b->bound) return bfail(b, PIMD_ESTATE, "pimd_batch_step_profiled: not bound");
    ProfMarks pm;
    memset(&pm, 0, sizeof pm);
    for (int i = 0; i < 64; ++i)
        if (cudaEventCreate(&pm.ev[i]) != cudaSuccess) return bfail(b, PIMD_ECUDA, "event create");
    for (int i = 0; i < max_slots; ++i) ms_out[i] = 0.0;
    int slots = 0;
    pimd_status s = PIMD_OK;
    for (int n = 0; n < nsteps && s == PIMD_OK; ++n) {
        pm.n = 0;
        prof_mark(&pm, "start", b->st);
        s = batch_enqueue_step(b, b->st, &pm);
        cudaEventSynchronize(pm.ev[pm.n - 1]);
        slots = std::min(pm.n - 1, max_slots);
        for (int i = 0; i < slots; ++i) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, pm.ev[i], pm.ev[i + 1]);
            ms_out[i] += ms;
            b->slot_names[i] = pm.name[i + 1];
        }
    }
    for (int i = 0; i < 64; ++i) cudaEventDestroy(pm.ev[i]);
    b->steps += nsteps;
    *n_slots = slots;
    return s;
}

extern "C" const char* pimd_batch_profile_slot_name(pimd_batch_t b, int slot)
{
    if (!b || slot < 0 || slot >= 64 || !b->slot_names[slot]) return "";
    return b->slot_names[slot];
}

// Re-derives the grid-dependent fields of the replica arguments (after a
// tuning change) and uploads them.
static pimd_status batch_upload_args(pimd_batch* b)
{
    // springs partials: kernel layout (128-particle blocks) or force-unit layout
    // (pair-block units, stride gx_pair); pair partials stride gx_pair in both
    for (auto& a : b->args) {
        a.ss.n_springs = (b->sched == PIMD_BATCH_KERNELS ? b->grid.gx_spr : b->grid.gx_pair) * b->P;
        a.ss.n_pair = b->grid.gx_pair * b->P;
    }
    batch_prefix(b);
    char* base = (char*)b->buf.work;
    cudaError_t e = cudaMemcpyAsync(base + b->off_args, b->args.data(), b->args.size() * sizeof(RepArgs),
                                    cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + b->off_prefix, b->prefix.data(), b->prefix.size() * sizeof(int),
                            cudaMemcpyHostToDevice, b->st);
    if (e == cudaSuccess) e = batch_clear_parts(b);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
    return e == cudaSuccess ? PIMD_OK : bcuda(b, e, "batch argument upload");
}

static void batch_set_pair_t(pimd_batch* b, int T)
{
    int nmax = 0;
    for (int n : b->N) nmax = std::max(nmax, n);
    b->grid.pair_t = T;
    b->grid.gx_pair = pair_grid_x(nmax, T);
}

extern "C" pimd_status pimd_batch_tuning(pimd_batch_t b, int* pair_block)
{
    if (!b || !pair_block) return bfail(b, PIMD_EINVAL, "pimd_batch_tuning: NULL argument");
    *pair_block = pair_block_ok(b->grid.pair_t) ? b->grid.pair_t : 128;  // the layout's default before bind
    return PIMD_OK;
}

extern "C" pimd_status pimd_batch_schedule(pimd_batch_t b, int* schedule)
{
    if (!b || !schedule) return bfail(b, PIMD_EINVAL, "pimd_batch_schedule: NULL argument");
    *schedule = b->bound ? b->sched : b->cfg.batch_schedule;
    return PIMD_OK;
}

extern "C" pimd_status pimd_batch_autotune(pimd_batch_t b, const char* cache_path)
{
    if (!b) return bfail(b, PIMD_EINVAL, "pimd_batch_autotune: NULL handle");
    if (!b->bound) return bfail(b, PIMD_ESTATE, "pimd_batch_autotune: not bound");
    long long sumN = 0, sumN2 = 0;
    for (int n : b->N) {
        sumN += n;
        sumN2 += (long long)n * n;
    }
    char kb[256];
    snprintf(kb, sizeof kb, "batch R=%d sumN=%lld sumN2=%lld P=%d d=%d prec=%d g0=%d", b->R, sumN, sumN2, b->P, b->d,
             b->cfg.precision, b->A == 0.0);
    const std::string key = device_key() + " " + kb;
    std::string val;
    int bestT = b->grid.pair_t, bestS = b->sched;
    if (cache_lookup(cache_path, key, val)) {
        bestT = cache_field(val, "pair_t", bestT);
        bestS = cache_field(val, "sched", bestS);
    } else {
        double best = 1e30;
        std::vector<int> Ts = {64, 128, 256};
        if (b->A == 0.0) Ts = {bestT};
        for (int S : {PIMD_BATCH_PERSISTENT, PIMD_BATCH_KERNELS})
            for (int T : Ts) {
                b->sched = S;
                batch_set_pair_t(b, T);
                pimd_status st = batch_upload_args(b);
                if (st != PIMD_OK) return st;
                const double ms = time_ms(b->st, 3, [&] {
                    if (st == PIMD_OK) st = batch_enqueue_forces(b, b->st);
                });
                if (st != PIMD_OK) return st;
                if (ms < best) {
                    best = ms;
                    bestT = T;
                    bestS = S;
                }
            }
        char vb[64];
        snprintf(vb, sizeof vb, "pair_t=%d;sched=%d", bestT, bestS);
        cache_store(cache_path, key, vb);
    }
    if (!pair_block_ok(bestT) || (bestS != PIMD_BATCH_PERSISTENT && bestS != PIMD_BATCH_KERNELS))
        return bfail(b, PIMD_EINVAL, "pimd_batch_autotune: bad cache entry");
    b->sched = bestS;
    batch_set_pair_t(b, bestT);
    pimd_status s = batch_upload_args(b);
    if (s != PIMD_OK) return s;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->graph_failed = false;
    s = batch_enqueue_forces(b, b->st);
    if (s != PIMD_OK) return s;
    return batch_check_device(b);
}

extern "C" pimd_status pimd_batch_estimators(pimd_batch_t b, pimd_estimates* out)
{
    if (!b || !out) return bfail(b, PIMD_EINVAL, "pimd_batch_estimators: NULL argument");
    if (!b->bound) return bfail(b, PIMD_ESTATE, "pimd_batch_estimators: not bound");
    char* base = (char*)b->buf.work;
    const RepArgs* ra = (const RepArgs*)(base + b->off_args);
    cudaError_t e = batch_launch_scalars(ra, b->grid, b->st);
    if (e != cudaSuccess) return bcuda(b, e, "batch scalar reduction");
    int* flag = (int*)(base + b->off_flag);
    e = cudaMemsetAsync(flag, 0, sizeof(int), b->st);
    for (int r = 0; r < b->R && e == cudaSuccess; ++r)
        e = launch_nonfinite_scan(b->buf.f + b->off[r], b->N[r], b->P, b->d, b->npad[r], flag, b->st);
    if (e != cudaSuccess) return bcuda(b, e, "pimd_batch_estimators: scan");
    pimd_status s = batch_check_device(b);
    if (s != PIMD_OK) return s;
    std::vector<double> t((size_t)b->R * SC_COUNT);
    int hflag = 0;
    e = cudaMemcpy(t.data(), base + b->off_sc, t.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "pimd_batch_estimators: read");
    bool finite = true;
    for (int r = 0; r < b->R; ++r)
        finite &= fill_estimates(&t[(size_t)r * SC_COUNT], b->P, b->N[r], b->d, b->beta[r], b->cfg.thermostat, b->steps,
                                 &out[r]);
    if (!finite) return bfail(b, PIMD_ENONFINITE, "pimd_batch_estimators: non-finite estimate");
    if (hflag) return bfail(b, PIMD_ENONFINITE, "pimd_batch_estimators: non-finite force");
    return PIMD_OK;
}

extern "C" pimd_status pimd_batch_sync(pimd_batch_t b)
{
    if (!b) return bfail(b, PIMD_EINVAL, "pimd_batch_sync: NULL handle");
    if (!b->bound) return bfail(b, PIMD_ESTATE, "pimd_batch_sync: not bound");
    return batch_check_device(b);
}

extern "C" const char* pimd_batch_last_error(pimd_batch_t b) { return b ? b->err.c_str() : g_global_error.c_str(); }

extern "C" void pimd_batch_destroy(pimd_batch_t b)
{
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->ev_join) cudaEventDestroy(b->ev_join);
    delete b;
}

// ---------------------------------------------------------------------------
// Exchange potential with library-owned scratch, for callers that cannot
// allocate device memory (see pimd_vb_forward_noalloc in pimd.h).

#include <mutex>

#define PIMD_NOALLOC_MAX_N 1024
#define PIMD_NOALLOC_BYTES ((size_t)8 << 20)

// Fixed scratch for the whole recursion state of one call (factor table,
// chain vectors, flags, partial sums).  Every GPU that loads the library
// holds these 8 MiB until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PIMD_NOALLOC_BYTES];

static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[128];

// Device address of the scratch array on the current device.  The array's
// name in host code is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
static pimd_status noalloc_scratch(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, PIMD_ECUDA, std::string("pimd_vb_forward_noalloc: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 128) return fail(nullptr, PIMD_EINVAL, "pimd_vb_forward_noalloc: device index out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(nullptr, PIMD_ECUDA, std::string("pimd_vb_forward_noalloc: scratch address lookup failed: ") +
                                                 cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return PIMD_OK;
}

extern "C" pimd_status pimd_vb_forward_noalloc(int N, int P, int d, double beta, double xi, const double* r1,
                                               const double* rP, int ld, double* V_out, void* stream)
{
    if (N < 1 || N > PIMD_NOALLOC_MAX_N)
        return fail(nullptr, PIMD_EINVAL, "pimd_vb_forward_noalloc: N must be in [1, 1024] (fixed 8 MiB scratch)");
    if (P < 2 || d < 1 || d > 3 || !(beta > 0.0) || !(xi >= 0.0 && xi <= 1.0))
        return fail(nullptr, PIMD_EINVAL, "pimd_vb_forward_noalloc: bad argument");
    if (!r1 || !rP || !V_out || ld < N) return fail(nullptr, PIMD_EINVAL, "pimd_vb_forward_noalloc: NULL pointer or ld < N");
    Layout L;
    ExchLayout ex;
    exch_layout(L, ex, N, EX_STREAMS, 1);
    if (L.total > PIMD_NOALLOC_BYTES)
        return fail(nullptr, PIMD_EINVAL, "pimd_vb_forward_noalloc: N too large for the fixed scratch");
    void* base = nullptr;
    pimd_status s = noalloc_scratch(&base);
    if (s != PIMD_OK) return s;
    pimd_config cfg;
    pimd_default_config(&cfg);
    cudaStream_t st = (cudaStream_t)stream;
    ExchView v = exch_view((char*)base, ex, N, P, d, beta, xi, EX_STREAMS, 1, rP, r1, ld, ld, 0, default_helpers(cfg));
    cudaError_t e = cudaMemsetAsync(v.err, 0, sizeof(int), st);  // error word must start at zero
    if (e == cudaSuccess) e = exch_launch_forward(v, st, 1);      // also zeroes the chain flags
    if (e == cudaSuccess) e = exch_launch_vb_value(v, exch_prep_blocks(N), V_out, st);
    if (e != cudaSuccess) return fail(nullptr, PIMD_ECUDA, std::string("pimd_vb_forward_noalloc: ") + cudaGetErrorString(e));
    return PIMD_OK;
}
