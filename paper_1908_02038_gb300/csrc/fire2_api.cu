// Host side of the C ABI declared in include/fire2.h: handle management,
// buffer sizing, the neighbour-mode choice, and the CUDA graph that runs a
// whole FIRE 2.0 relaxation (Algorithm 2 + Algorithm 4) on the device with a
// conditional WHILE node, so no host synchronisation happens per iteration.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "fire2.h"
#include "fire2_device.cuh"
#include "fire2_grad.cuh"
#include "fire2_neb.cuh"
#include "fire2_tile.cuh"

using namespace fire2;

struct fire_batch_state;
void fire2_batch_free(fire_batch_state* b);
fire_status fire2_batch_create(fire_handle_t* h, int32_t n_sys, const int64_t* offsets,
                               fire_batch_state** out);

// Buffers of the differentiable form (allocated on first use).
struct GradState {
    int cap = 0, nb = 0;
    dvec4* x = nullptr;
    float4* xf = nullptr;
    uint32_t* nbr = nullptr;
    int* nnbr = nullptr;
    double *rho = nullptr, *F1 = nullptr, *F2 = nullptr, *drho = nullptr, *dq = nullptr;
    double* part = nullptr;        // 9 x nb block partials
    double* vec = nullptr;         // 4 work vectors of 3N (r, p, Ap, lambda)
    double* pcache = nullptr;      // HVP pair coefficients, 3 x cap x N (implicit gradient)
    size_t pcache_slots = 0;
    CgState* cs = nullptr;         // device scalars of the CG solve
    CgState* h_cs = nullptr;       // pinned copy
    double* h_part = nullptr;      // pinned copy of part
    DevState* st = nullptr;        // status word of the list build
};

// Nudged elastic band handles (fire_neb_init): the movable images are the
// handle's atoms, image k = atoms [k img_n, (k + 1) img_n).
struct NebState {
    int n_img = 0;
    double k = 0.0;
    int climb = 0;
    int nb = 1;                    // k_neb_sums blocks per image
    int nb_proj = 1;               // k_neb_project blocks
    dvec4* end = nullptr;          // 2 x img_n fixed end states
    double* eatom = nullptr;       // per-atom energies
    double* part = nullptr;        // kNebSums x n_img x nb
    double* coef = nullptr;        // 4 x n_img
    double* E = nullptr;           // n_img + 2
    int* climber = nullptr;
    double* d_path = nullptr;      // staging for the host-pointer call, (n_img + 2) x img_n x 3
    double* d_end_energy = nullptr;   // scratch for the end-state evaluations
    fire_handle* inner = nullptr;  // one-image handle for the end-state energies
};

static void neb_free(NebState* q) {
    if (!q) return;
    for (void* p : {(void*)q->end, (void*)q->eatom, (void*)q->part, (void*)q->coef, (void*)q->E,
                    (void*)q->climber, (void*)q->d_path, (void*)q->d_end_energy})
        if (p) cudaFree(p);
    if (q->inner) fire_destroy(q->inner);
    delete q;
}

struct fire_handle {
    int device = 0;
    fire_system_t sys{};
    fire_potential_t pot{};
    fire_params_t par{};
    PotC potc{};
    int n = 0;
    int cap = 0;         // allocated half-list capacity per atom
    int ncell_alloc = 0;
    Bufs b{};
    cudaStream_t stream = nullptr;   // default stream of host-pointer calls
    cudaStream_t cap0 = nullptr, cap1 = nullptr, cap2 = nullptr;  // private capture streams
    DevState* h_state = nullptr;     // pinned
    double* h_pos = nullptr;         // pinned staging, N x 3
    // cached relaxation graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    GeoC gkey{};
    bool has_graph = false;
    double budget_s = 3600.0;
    int exec_mode = FIRE_EXEC_GRAPH_WHILE;
    int chunk = 32;                  // iterations per graph launch, chunked mode
    int body_iters = 0;              // iterations per WHILE-body launch, graph mode (0: auto)
    cudaGraphExec_t exec_init = nullptr, exec_chunk = nullptr, exec_final = nullptr;
    fire_batch_state* batch = nullptr;   // set for handles made by fire_batch_init
    GradState grad;
    // tabulated pair functions: device copies and launch shapes
    float *tab_ffd = nullptr, *tab_fff = nullptr;
    float *tab_d32 = nullptr, *tab_f32 = nullptr;
    size_t smem_d = 0, smem_f = 0;
    int nb_tab_d = 0, nb_tab_f = 0;
    uint8_t* dofmask = nullptr;      // device copy of the frozen-DOF mask (n bytes)
    int img_n = 0;                   // atoms per image (n, except for NEB handles)
    bool verify = false;             // FP32-pair: stops on ftol confirmed in FP64
    int sms = 0;                     // SM count of the device
    int tile_mode = FIRE_TILES_AUTO; // shared-memory tiles of the FP64 half-list passes
    int stage_cap = 0;               // staged atoms per tile (0 = kStageMax)
    size_t loc_slots = 0;            // allocated nbr_loc entries
    int tile_alloc = 0;              // allocated tiles (tile_key, tile_ns)
    bool tile_attr = false;          // dynamic shared-memory limits of the tile kernels set
    NebState* neb = nullptr;
    std::string err;
};

namespace {

std::string g_init_err = "no error";

fire_status fail(fire_handle* h, fire_status code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    else g_init_err = buf;
    return code;
}

#define CK(h, call)                                                                      \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail((h), e_ == cudaErrorMemoryAllocation ? FIRE_ERR_NOMEM : FIRE_ERR_CUDA, \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

double cutoff(const fire_potential_t& p) {
    if (p.kind == FIRE_POT_SW) return p.sw_a * p.sigma;
    return p.kind == FIRE_POT_LJ ? p.rc_lj : p.rc;
}

// The FP64 form's tabulated RGL passes (fixed-point separations, double-float
// pair terms, k_density_ff / k_force_ff) ...
bool fixed64_form(const fire_potential_t& p) {
    return p.kind == FIRE_POT_RGL && p.precision == FIRE_PREC_FP64 && p.pair_eval == FIRE_PAIR_TABLE;
}
// ... on a half list with FP64 atomics (Newton's third law) or a full list.
bool fixed64_half(const fire_potential_t& p) {
    return fixed64_form(p) && p.newton != FIRE_NEWTON_OFF;
}
// Blocks of the double-float density pass: one thread per atom on blocks of
// kDensFF1Block (3 per SM at 40 registers: 0.289 against 0.312 ms with
// blocks of 128 on the 1M-atom box, 0.302 with 256, 0.357 with 1024),
// split lists on blocks of kForceBlock.
inline int dens_ff_block(int tpa) { return tpa == 1 ? kDensFF1Block : kForceBlock; }
inline int dens_ff_grid(int n, int tpa) {
    return (int)(((long long)n * tpa + dens_ff_block(tpa) - 1) / dens_ff_block(tpa));
}

// The pair passes that can split an atom's list over several threads: the
// FP64 table form and the FP32-pair form with exponentials.
bool tpa_form(const fire_potential_t& p) {
    return fixed64_form(p) || p.kind == FIRE_POT_LJ ||
           (p.kind == FIRE_POT_RGL && p.precision == FIRE_PREC_FP32_PAIR &&
            p.pair_eval == FIRE_PAIR_ANALYTIC);
}

constexpr int kMaxTpa = 32;
constexpr int kMaxHvpTpa = 8;   // the Hessian-vector product passes

// Threads per atom chosen when the caller sets none: the fewest (1, 2, 4, ...)
// that give a pair pass at least 1024 threads per SM in the FP64 forms, 512
// in the FP32-pair form, up to 8 for RGL and 32 for LJ.  Measured on GB300
// (152 SMs, us per iteration at 1 / 2 / 4 / 8 threads per atom): FP64 form
// 3,751 atoms 110 / 94 / 78 / 57, 29,931 atoms 116 / 104 / 93 / 90, 59,762
// atoms 135 / 126 / 119 / 122, 128,277 atoms 187 / 194 / 189 / 204, 997,450
// atoms 986 / 1031 / 1090 / 1307; FP32-pair form 29,931 atoms
// 108 / 81 / 73 / 78, 59,762 atoms 115 / 92 / 92 / 102, 997,450 atoms
// 652 / 680 / 753 / 963.  Beyond 8 (us per iteration at 8 / 16 / 32): the
// RGL passes gain nothing (3,960 atoms, FP64 form 46.4 / 46.7 / 50.3,
// FP32-pair form 45.8 / 48.9 / 54.3), while the LJ force pass, whose pair
// terms are FP64 arithmetic at 1/58 of the FP32 rate, spreads them over more
// SMs (255 atoms 30.7 / 28.0 / 25.8).  Later, with the current passes
// (us per iteration, 31,680 atoms): FP64 form 71.8 / 71.6 / 86.1 at
// 4 / 8 / 16, FP32-pair form 64.9 / 58.5 / 64.3 at 2 / 4 / 8.
int tpa_for(long long n, int sms, int per_sm, int cap = kMaxTpa) {
    int t = 1;
    while (t < cap && n * t < (long long)sms * per_sm) t *= 2;
    return t;
}
int auto_tpa(const fire_potential_t& p, long long n, int sms) {
    return tpa_for(n, sms, p.precision == FIRE_PREC_FP32_PAIR ? 512 : 1024,
                   p.kind == FIRE_POT_LJ ? kMaxTpa : 8);
}

// Whether the FP64 half-list passes of this geometry run on tiles: the FP64
// table form on a half list, cell mode, one system, and tiles asked for.
// FIRE_TILES_AUTO takes the untiled passes: on GB300 the tiled ones remove
// the FP64 additions and L2 atomics of the neighbour terms (FP64 pipe 62 % ->
// 3 %, L2 40 % -> 8 % in the force pass) but both passes are bound by the
// issue of their double-float arithmetic, and the tiles' staging, barriers
// and fixed-point splits cost more issue than they save (1M-atom box: force
// 0.49 ms against 0.41, density 0.38 against 0.29).
bool tiles_wanted(const fire_handle* h, const GeoC& g) {
    if (!fixed64_half(h->pot) || g.brute || h->neb || g.img_n != h->n) return false;
    return h->tile_mode == FIRE_TILES_ON;
}

// Neighbour geometry for a box.  The list radius is rc + skin, with the skin
// reduced where a periodic axis is shorter than 2 (rc + skin) so that the
// minimum image stays unique within the list radius.
GeoC make_geo(const fire_handle* h, const double box[3]) {
    GeoC g{};
    const double rc = cutoff(h->pot);
    double skin = h->pot.skin;
    for (int a = 0; a < 3; ++a)
        if (h->sys.periodic[a]) skin = std::min(skin, 0.5 * box[a] * (1.0 - 1e-12) - rc);
    skin = std::max(skin, 0.0);
    const double rl = rc + skin;
    g.rlist2 = rl * rl;
    g.half_skin2 = 0.25 * skin * skin;
    g.rc2f = (float)(rc * rc);
    g.brute = 0;
    for (int a = 0; a < 3; ++a) {
        g.L[a] = box[a];
        g.Linv[a] = 1.0 / box[a];
        g.per[a] = h->sys.periodic[a] ? 1 : 0;
        // a periodic axis needs 3 cells for a stencil without repeats; an
        // open axis takes any count (at least one), its cells clamped
        g.nc[a] = std::max((int)std::floor(box[a] / rl), g.per[a] ? 0 : 1);
        if (g.per[a] && g.nc[a] < 3) g.brute = 1;
    }
    if (g.brute)
        for (int a = 0; a < 3; ++a) g.nc[a] = 1;
    for (int a = 0; a < 3; ++a) g.cinv[a] = g.nc[a] / box[a];
    double lmax = 0.0;
    for (int a = 0; a < 3; ++a) {
        g.Lf[a] = (float)box[a];
        g.Linvf[a] = (float)(1.0 / box[a]);
        lmax = std::max(lmax, box[a]);
    }
    // FP32 positions carry absolute errors up to ~1.2e-7 of the coordinate
    // magnitude (positions stay within about one box length of the box)
    const double margin = 1e-3 * rc + 8.0 * 1.2e-7 * (2.0 * lmax);
    g.rlist2f = (float)((rl + margin) * (rl + margin));
    g.full = (h->pot.precision == FIRE_PREC_FP32_PAIR || h->pot.kind == FIRE_POT_SW ||
              (fixed64_form(h->pot) && !fixed64_half(h->pot))) ? 1 : 0;
    for (int a = 0; a < 3; ++a) {
        g.Lq[a] = (int)(unsigned)(unsigned long long)std::llrint(box[a] * h->b.qscale);
        g.Lq64[a] = std::llrint(std::ldexp(box[a], kFixedBits64));
    }
    g.img_n = h->img_n > 0 ? h->img_n : h->n;
    // bricks of cells: the tiles of the FP64 half-list passes (fire2_tile.cuh);
    // flat in z, the axis the half list cuts (a tile's stage then holds about
    // twice its own atoms); bricks of one cell, the plain cell order, otherwise
    for (int a = 0; a < 3; ++a) {
        g.bk[a] = 1;
        g.nbk[a] = g.nc[a];
    }
    if (tiles_wanted(h, g)) {
        for (int a = 0; a < 3; ++a) {
            g.bk[a] = std::min(kTileBrick[a], g.nc[a]);
            g.nbk[a] = ceil_div(g.nc[a], g.bk[a]);
        }
        g.tiled = 1;
        g.ntile = g.nbk[0] * g.nbk[1] * g.nbk[2];
        g.stage_cap = h->stage_cap > 0 ? h->stage_cap : kStageMax;
    }
    g.ncell_img = g.nbk[0] * g.nbk[1] * g.nbk[2] * g.bk[0] * g.bk[1] * g.bk[2];
    return g;
}

// Half-list capacity: 1.5x the expected upper-half-space count at the mean
// density, plus a margin; never more than N - 1.
int estimate_cap(const fire_handle* h, const GeoC& g) {
    const double vol = g.L[0] * g.L[1] * g.L[2];
    const double dens = g.img_n / vol;    // atoms of one image
    const double rl = std::sqrt(g.rlist2);
    const double half = 2.0 / 3.0 * M_PI * rl * rl * rl * dens;
    long long cap = (long long)std::ceil(1.5 * half * (g.full ? 2.0 : 1.0)) + 16;
    cap = std::min<long long>(cap, std::max(h->n - 1, 1));
    return (int)std::max<long long>(cap, 1);
}

bool same_geo(const GeoC& a, const GeoC& b) { return std::memcmp(&a, &b, sizeof(GeoC)) == 0; }

void drop_graph(fire_handle* h) {
    if (h->exec) cudaGraphExecDestroy(h->exec);
    if (h->graph) cudaGraphDestroy(h->graph);
    for (cudaGraphExec_t* e : {&h->exec_init, &h->exec_chunk, &h->exec_final})
        if (*e) cudaGraphExecDestroy(*e);
    h->exec_init = h->exec_chunk = h->exec_final = nullptr;
    h->exec = nullptr;
    h->graph = nullptr;
    h->has_graph = false;
}

// Blocks of the tile passes: kTileMinBlocks per SM (as many as the force
// pass's stage and registers allow), looping over the tiles; never more than
// the energy partials allocated for the density pass.
int tile_grid(const fire_handle* h, const GeoC& g) {
    const int nb_max = ceil_div((long long)h->n * kMaxTpa, kForceBlock);
    return std::max(1, std::min(std::min(g.ntile, kTileMinBlocks * h->sms), nb_max));
}

fire_status ensure_buffers(fire_handle* h, const GeoC& g, int cap) {
    if (cap > h->cap) {
        drop_graph(h);
        cudaFree(h->b.nbr);
        cudaFree(h->b.crep);
        cudaFree(h->b.cden);
        h->b.nbr = nullptr;
        h->b.crep = h->b.cden = nullptr;
        const size_t slots = (size_t)cap * h->n;
        CK(h, cudaMalloc(&h->b.nbr, slots * sizeof(uint32_t)));
        if (h->pot.kind == FIRE_POT_RGL && h->pot.precision == FIRE_PREC_FP64 &&
            !fixed64_form(h->pot)) {
            CK(h, cudaMalloc(&h->b.crep, slots * sizeof(double)));
            CK(h, cudaMalloc(&h->b.cden, slots * sizeof(double)));
        }
        h->cap = cap;
    }
    h->b.cap = h->cap;
    const int ncell = (h->n / g.img_n) * g.ncell_img;
    if (ncell > h->ncell_alloc) {
        drop_graph(h);
        cudaFree(h->b.cell_count);
        cudaFree(h->b.cell_start);
        h->b.cell_count = h->b.cell_start = nullptr;
        CK(h, cudaMalloc(&h->b.cell_count, (size_t)ncell * sizeof(int)));
        CK(h, cudaMalloc(&h->b.cell_start, ((size_t)ncell + 1) * sizeof(int)));
        h->ncell_alloc = ncell;
    }
    h->b.ncell = ncell;
    if (g.tiled) {
        const size_t slots = (size_t)h->cap * h->n;
        if (slots > h->loc_slots) {
            drop_graph(h);
            cudaFree(h->b.nbr_loc);
            h->b.nbr_loc = nullptr;
            h->loc_slots = 0;
            CK(h, cudaMalloc(&h->b.nbr_loc, slots * sizeof(uint16_t)));
            h->loc_slots = slots;
        }
        if (g.ntile > h->tile_alloc) {
            drop_graph(h);
            cudaFree(h->b.tile_key);
            cudaFree(h->b.tile_ns);
            h->b.tile_key = nullptr;
            h->b.tile_ns = nullptr;
            h->tile_alloc = 0;
            CK(h, cudaMalloc(&h->b.tile_key, (size_t)g.ntile * kStageMax * sizeof(uint32_t)));
            CK(h, cudaMalloc(&h->b.tile_ns, (size_t)g.ntile * sizeof(int)));
            h->tile_alloc = g.ntile;
        }
        if (!h->tile_attr) {
            CK(h, cudaFuncSetAttribute(k_density_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kDensTileSmem));
            CK(h, cudaFuncSetAttribute(k_force_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kForceTileSmem));
            // all of the unified L1 / shared storage as shared memory: the
            // resident blocks' stages need it
            CK(h, cudaFuncSetAttribute(k_density_tile,
                                       cudaFuncAttributePreferredSharedMemoryCarveout, 100));
            CK(h, cudaFuncSetAttribute(k_force_tile,
                                       cudaFuncAttributePreferredSharedMemoryCarveout, 100));
            h->tile_attr = true;
        }
    }
    // energy partials of the density (or only) pass, then the embedding's
    h->b.ne_dens = g.tiled ? tile_grid(h, g)
                 : fixed64_form(h->pot) ? dens_ff_grid(h->n, h->b.tpa) : h->b.nb_force;
    return FIRE_OK;
}

// --- launch helpers (used both for direct launches and for capture) -------

void launch_build(fire_handle* h, const GeoC& g, int force, cudaStream_t s) {
    const int n = h->n;
    if (!g.brute) {
        k_cell_zero<<<ceil_div(h->b.ncell, kElemBlock), kElemBlock, 0, s>>>(h->b, g, force);
        k_cell_count<<<ceil_div(n, kElemBlock), kElemBlock, 0, s>>>(h->b, g, force);
        k_cell_scan<<<1, 1024, 0, s>>>(h->b, g, force);
        k_cell_fill<<<ceil_div(n, kElemBlock), kElemBlock, 0, s>>>(h->b, g, force);
        k_cell_sort<<<ceil_div(h->b.ncell, kElemBlock), kElemBlock, 0, s>>>(h->b, g, force);
    }
    k_nbr_build<<<ceil_div(n, kForceBlock), kForceBlock, 0, s>>>(h->b, g, force);
    if (g.tiled)
        k_tile_build<<<std::max(1, std::min(g.ntile, 4 * h->sms)), kTileThreads, 0, s>>>(h->b, g,
                                                                                         force);
}

// The pair passes for the handle's threads per atom (b.tpa).  The density
// pass writes one energy partial per block: dens_ff_grid blocks.
template <bool HALF>
void density_ff(const Bufs& b, const PotC& P, const GeoC& g, cudaStream_t s) {
    const int nb = dens_ff_grid(b.n, b.tpa), bs = dens_ff_block(b.tpa);
    switch (b.tpa) {
    case 32: k_density_ff<HALF, 32><<<nb, bs, 0, s>>>(b, P, g); break;
    case 16: k_density_ff<HALF, 16><<<nb, bs, 0, s>>>(b, P, g); break;
    case 8: k_density_ff<HALF, 8><<<nb, bs, 0, s>>>(b, P, g); break;
    case 4: k_density_ff<HALF, 4><<<nb, bs, 0, s>>>(b, P, g); break;
    case 2: k_density_ff<HALF, 2><<<nb, bs, 0, s>>>(b, P, g); break;
    default: k_density_ff1<HALF><<<nb, bs, 0, s>>>(b, P, g);
    }
}
template <bool HALF>
void force_ff(const Bufs& b, const PotC& P, const GeoC& g, cudaStream_t s) {
    // one thread per atom: blocks of 512 (1M-atom box: 0.461 against 0.483 ms
    // with blocks of 128, at the same 1,024 threads per SM; 64 registers)
    constexpr int B1 = 512;
    const long long n = b.n;
    switch (b.tpa) {
    case 32: k_force_ff<HALF, 32, kForceBlock><<<ceil_div(n * 32, kForceBlock), kForceBlock, 0, s>>>(b, P, g); break;
    case 16: k_force_ff<HALF, 16, kForceBlock><<<ceil_div(n * 16, kForceBlock), kForceBlock, 0, s>>>(b, P, g); break;
    case 8: k_force_ff<HALF, 8, kForceBlock><<<ceil_div(n * 8, kForceBlock), kForceBlock, 0, s>>>(b, P, g); break;
    case 4: k_force_ff<HALF, 4, kForceBlock><<<ceil_div(n * 4, kForceBlock), kForceBlock, 0, s>>>(b, P, g); break;
    case 2: k_force_ff<HALF, 2, kForceBlock><<<ceil_div(n * 2, kForceBlock), kForceBlock, 0, s>>>(b, P, g); break;
    default: k_force_ff<HALF, 1, B1><<<ceil_div(n, B1), B1, 0, s>>>(b, P, g);
    }
}
void force_lj(const Bufs& b, const PotC& P, const GeoC& g, cudaStream_t s) {
    switch (b.tpa) {
    case 32: k_force_lj<32><<<b.nb_force, kForceBlock, 0, s>>>(b, P, g); break;
    case 16: k_force_lj<16><<<b.nb_force, kForceBlock, 0, s>>>(b, P, g); break;
    case 8: k_force_lj<8><<<b.nb_force, kForceBlock, 0, s>>>(b, P, g); break;
    case 4: k_force_lj<4><<<b.nb_force, kForceBlock, 0, s>>>(b, P, g); break;
    case 2: k_force_lj<2><<<b.nb_force, kForceBlock, 0, s>>>(b, P, g); break;
    default: k_force_lj<1><<<b.nb_force, kForceBlock, 0, s>>>(b, P, g);
    }
}
void density32(const Bufs& b, const PotC& P, const GeoC& g, cudaStream_t s) {
    switch (b.tpa) {
    case 32: k_density32<32><<<b.nb_force, kForceBlock, 0, s>>>(b, P, g); break;
    case 16: k_density32<16><<<b.nb_force, kForceBlock, 0, s>>>(b, P, g); break;
    case 8: k_density32<8><<<b.nb_force, kForceBlock, 0, s>>>(b, P, g); break;
    case 4: k_density32<4><<<b.nb_force, kForceBlock, 0, s>>>(b, P, g); break;
    case 2: k_density32<2><<<b.nb_force, kForceBlock, 0, s>>>(b, P, g); break;
    default: k_density32<1><<<b.nb_force, kForceBlock, 0, s>>>(b, P, g);
    }
}
void force32(const Bufs& b, const PotC& P, const GeoC& g, cudaStream_t s) {
    // one thread per atom on blocks of 512 (1M-atom box: 0.232 against
    // 0.239 ms with blocks of 128); the pass writes no per-block partials
    constexpr int B1 = 512;
    switch (b.tpa) {
    case 32: k_force32<32, kForceBlock><<<b.nb_force, kForceBlock, 0, s>>>(b, P, g); break;
    case 16: k_force32<16, kForceBlock><<<b.nb_force, kForceBlock, 0, s>>>(b, P, g); break;
    case 8: k_force32<8, kForceBlock><<<b.nb_force, kForceBlock, 0, s>>>(b, P, g); break;
    case 4: k_force32<4, kForceBlock><<<b.nb_force, kForceBlock, 0, s>>>(b, P, g); break;
    case 2: k_force32<2, kForceBlock><<<b.nb_force, kForceBlock, 0, s>>>(b, P, g); break;
    default: k_force32<1, B1><<<ceil_div(b.n, B1), B1, 0, s>>>(b, P, g);
    }
}

// The two passes of the cached Hessian-vector product, TPA threads per atom.
template <int TPA>
void hvp_cached_t(const GradBufs& b, const double* u, double* hu, const int* skip, int n,
                  cudaStream_t s) {
    const int nb = ceil_div((long long)n * TPA, kForceBlock);
    k_g_hvp1c<TPA><<<nb, kForceBlock, 0, s>>>(b, u, skip);
    k_g_hvp2c<TPA><<<nb, kForceBlock, 0, s>>>(b, u, hu, skip);
}
void hvp_cached(const GradBufs& b, const double* u, double* hu, const int* skip, int tpa, int n,
                cudaStream_t s) {
    switch (tpa) {
    case 8: hvp_cached_t<8>(b, u, hu, skip, n, s); break;
    case 4: hvp_cached_t<4>(b, u, hu, skip, n, s); break;
    case 2: hvp_cached_t<2>(b, u, hu, skip, n, s); break;
    default: hvp_cached_t<1>(b, u, hu, skip, n, s);
    }
}

// FP32-pair handles that confirm their stops: the FP64 passes on the same
// full list (they return at once unless a stop is being confirmed).
void launch_confirm(fire_handle* h, const GeoC& g, cudaStream_t s) {
    Bufs bv = h->b;
    bv.pass_role = 2;
    density_ff<false>(bv, h->potc, g, s);
    force_ff<false>(bv, h->potc, g, s);
}

// The force passes of one evaluation; with confirm_passes, also the FP64
// confirming passes of FP32-pair handles (the graph loop puts those under
// an IF node instead).
void launch_forces(fire_handle* h, const GeoC& g, cudaStream_t s, bool confirm_passes = true) {
    const int n = h->n;
    const bool tab = h->pot.kind == FIRE_POT_RGL && h->pot.pair_eval == FIRE_PAIR_TABLE;
    if (tab && h->pot.precision == FIRE_PREC_FP32_PAIR) {
        k_density32_tab<<<h->nb_tab_d, kTabBlock, h->smem_d, s>>>(h->b, h->potc, g);
        k_force32_tab<<<h->nb_tab_f, kTabBlock, h->smem_f, s>>>(h->b, h->potc, g);
    } else if (tab && fixed64_half(h->pot) && g.tiled) {
        const int nt = tile_grid(h, g);
        k_density_tile<<<nt, kTileThreads, kDensTileSmem, s>>>(h->b, h->potc, g);
        k_embed<<<h->b.nb_embed, kElemBlock, 0, s>>>(h->b);
        k_force_tile<<<nt, kTileThreads, kForceTileSmem, s>>>(h->b, h->potc, g);
    } else if (tab && fixed64_half(h->pot)) {
        density_ff<true>(h->b, h->potc, g, s);
        k_embed<<<h->b.nb_embed, kElemBlock, 0, s>>>(h->b);
        force_ff<true>(h->b, h->potc, g, s);
    } else if (tab) {
        density_ff<false>(h->b, h->potc, g, s);
        force_ff<false>(h->b, h->potc, g, s);
    } else if (h->pot.kind == FIRE_POT_RGL && h->pot.precision == FIRE_PREC_FP32_PAIR) {
        density32(h->b, h->potc, g, s);
        force32(h->b, h->potc, g, s);
    } else if (h->pot.kind == FIRE_POT_RGL) {
        k_density<<<h->b.nb_force, kForceBlock, 0, s>>>(h->b, h->potc, g);
        k_embed<<<h->b.nb_embed, kElemBlock, 0, s>>>(h->b);
        k_force_rgl<<<h->b.nb_force, kForceBlock, 0, s>>>(h->b, g);
    } else if (h->pot.kind == FIRE_POT_SW) {
        k_force_sw<<<h->b.nb_force, kForceBlock, 0, s>>>(h->b, h->potc, g);
    } else {
        force_lj(h->b, h->potc, g, s);
    }
    if (h->verify && confirm_passes) launch_confirm(h, g, s);
    (void)n;
}

// Device constants of a NEB handle's projection and reduction kernels.
NebC neb_consts(const fire_handle* h) {
    const NebState& q = *h->neb;
    NebC c;
    c.end = q.end;
    c.part = q.part;
    c.coef = q.coef;
    c.E = q.E;
    c.climber = q.climber;
    c.k = q.k;
    c.climb = q.climb;
    c.n_img = q.n_img;
    c.img_n = h->img_n;
    c.nb = q.nb;
    return c;
}

// The reductions and the control step (Algorithm 2) of one evaluation: one
// launch (k_reduce_ctl, whose last block runs the control), or for NEB
// handles two (k_neb_sums, whose last block sets the band's coefficients,
// and k_neb_project, which ends with the reductions of (F^NEB, v) and whose
// last block runs the control).
void launch_reduce_control(fire_handle* h, const GeoC& g, cudaStream_t s, int mode,
                           cudaGraphConditionalHandle hc, int has_handle) {
    if (h->neb) {
        const NebC c = neb_consts(h);
        k_neb_sums<<<dim3(c.nb, c.n_img), kNebBlock, (size_t)c.n_img * kNebSums * sizeof(double),
                     s>>>(h->b, g, c);
        k_neb_project<<<h->neb->nb_proj, kNebBlock, 0, s>>>(h->b, g, c, mode, hc, has_handle);
        return;
    }
    k_reduce_ctl<<<h->b.nb_red, kElemBlock, 0, s>>>(h->b, mode, hc, has_handle);
}

// Four blocks per SM, looping over the atoms (1M-atom box: 53 us against 55,
// 57 and 63 us at 8, 16 and 32 blocks per SM).
int update_grid(const fire_handle* h) {
    return std::max(1, std::min(ceil_div(h->n, kElemBlock), 4 * h->sms));
}

// The element-wise step; with dmax > 0 in two passes (see k_update_pre).
void launch_update(fire_handle* h, const GeoC& g, cudaStream_t s, cudaGraphConditionalHandle hif,
                   int has_if, cudaGraphConditionalHandle hconf = {}, int has_conf = 0) {
    const bool capped = h->par.dmax > 0.0;
    if (capped) k_update_pre<<<update_grid(h), kElemBlock, 0, s>>>(h->b);
    k_update<<<update_grid(h), kElemBlock, 0, s>>>(h->b, g, hif, has_if, capped ? 1 : 0,
                                                      hconf, has_conf);
}

// Appends a conditional node (WHILE or IF, one body) at the capture position
// of `s` and makes it the stream's only dependency; returns its body graph.
cudaError_t add_conditional(cudaStream_t s, cudaGraphConditionalHandle hc,
                            cudaGraphConditionalNodeType type, cudaGraph_t* body) {
    cudaStreamCaptureStatus cst;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &cst, nullptr, &cg, &deps, nullptr, &ndeps);
    cudaGraphNode_t cnode = nullptr;
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    std::memset(cp_raw, 0, sizeof cp_raw);
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = hc;
    cp.conditional.type = type;
    cp.conditional.size = 1;
    if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, cg, deps, nullptr, ndeps, &cp);
    if (e == cudaSuccess)
        e = cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1,
                                                cudaStreamSetCaptureDependencies);
    if (e == cudaSuccess) *body = cp.conditional.phGraph_out[0];
    return e;
}

// The device loop as one graph:
//   prepare, build, forces, reductions, control (initial evaluation)
//   WHILE (not stopped):
//     update (its last block sets the IF condition: displacement > skin/2)
//     IF (rebuild): cell binning + neighbour list
//     forces, reductions, control (sets the WHILE condition)
//   finalize
// Iterations per WHILE-body launch (build_graph; fire_set_exec_mode can set
// it).
constexpr int kLoopUnroll = 8;
constexpr int kMaxBodyIters = 64;

fire_status build_graph(fire_handle* h, const GeoC& g) {
    drop_graph(h);
    cudaGraph_t graph = nullptr;
    CK(h, cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle hw;
    cudaError_t e = cudaGraphConditionalHandleCreate(&hw, graph, 0, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(h, FIRE_ERR_CUDA, "cudaGraphConditionalHandleCreate: %s", cudaGetErrorString(e));
    }
    const int n = h->n;
    e = cudaStreamBeginCaptureToGraph(h->cap0, graph, nullptr, nullptr, 0,
                                      cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(h, FIRE_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
    }
    k_prepare<<<ceil_div(n, kElemBlock), kElemBlock, 0, h->cap0>>>(h->b);
    launch_build(h, g, 1, h->cap0);
    launch_forces(h, g, h->cap0);
    launch_reduce_control(h, g, h->cap0, CTL_INITIAL, hw, 1);

    cudaGraph_t body = nullptr;
    e = add_conditional(h->cap0, hw, cudaGraphCondTypeWhile, &body);
    // The WHILE body: kLoopUnroll iterations, as a body launch costs more
    // than the launches it saves (graph loop, one against eight iterations
    // per body: LJ 255 atoms 41.3 -> 33.4 us per iteration, RGL 3,957 atoms
    // 45.7 -> 42.6 us, 31,647 atoms 77.0 -> 75.0 us; the 1M-atom relaxation
    // 264.3 -> 262.5 ms).  Each iteration's cell-list chain and confirming
    // passes sit under IF nodes of their own (six gated launches cost more:
    // 3,960 atoms 45.6 -> 42.4 us, 61,875 atoms 105 -> 101 us); an
    // all-pairs build (one kernel) stays gated inside its kernel.  With one
    // iteration per body (fire_set_exec_mode) the same IF nodes sit in the
    // body.  Iterations past the stop return at once.
    const int unroll = h->body_iters > 0 ? h->body_iters : kLoopUnroll;
    if (e == cudaSuccess && unroll > 1) {
        e = cudaStreamBeginCaptureToGraph(h->cap1, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            const cudaGraphConditionalHandle none{};
            // an IF node of this body whose branch `fill` captures on cap2
            auto if_node = [&](cudaGraphConditionalHandle hc, auto fill) {
                cudaGraph_t bb = nullptr;
                cudaError_t r = add_conditional(h->cap1, hc, cudaGraphCondTypeIf, &bb);
                if (r == cudaSuccess)
                    r = cudaStreamBeginCaptureToGraph(h->cap2, bb, nullptr, nullptr, 0,
                                                      cudaStreamCaptureModeRelaxed);
                if (r == cudaSuccess) {
                    fill(h->cap2);
                    cudaGraph_t bb_out = nullptr;
                    r = cudaStreamEndCapture(h->cap2, &bb_out);
                }
                return r;
            };
            for (int u = 0; u < unroll && e == cudaSuccess; ++u) {
                // the cell-list chain (six kernels) and the FP64 confirming
                // passes under IF nodes of their own, set by this iteration's
                // update; an all-pairs build (one kernel) stays gated
                cudaGraphConditionalHandle hb = none, hc = none;
                const int has_b = g.brute ? 0 : 1, has_c = h->verify ? 1 : 0;
                if (has_b) e = cudaGraphConditionalHandleCreate(&hb, body, 0, cudaGraphCondAssignDefault);
                if (e == cudaSuccess && has_c)
                    e = cudaGraphConditionalHandleCreate(&hc, body, 0, cudaGraphCondAssignDefault);
                if (e != cudaSuccess) break;
                launch_update(h, g, h->cap1, hb, has_b, hc, has_c);
                if (has_b)
                    e = if_node(hb, [&](cudaStream_t s2) { launch_build(h, g, 1, s2); });
                else
                    launch_build(h, g, 0, h->cap1);
                if (e != cudaSuccess) break;
                launch_forces(h, g, h->cap1, !has_c);
                if (has_c) e = if_node(hc, [&](cudaStream_t s2) { launch_confirm(h, g, s2); });
                if (e != cudaSuccess) break;
                launch_reduce_control(h, g, h->cap1, CTL_LOOP, hw, 1);
            }
            cudaGraph_t body_out = nullptr;
            const cudaError_t e1 = cudaStreamEndCapture(h->cap1, &body_out);
            if (e == cudaSuccess) e = e1;
        }
    } else if (e == cudaSuccess) {
        cudaGraphConditionalHandle hif, hconf{};
        e = cudaGraphConditionalHandleCreate(&hif, body, 0, cudaGraphCondAssignDefault);
        if (e == cudaSuccess && h->verify)
            e = cudaGraphConditionalHandleCreate(&hconf, body, 0, cudaGraphCondAssignDefault);
        if (e == cudaSuccess)
            e = cudaStreamBeginCaptureToGraph(h->cap1, body, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeRelaxed);
        if (e == cudaSuccess) {
            launch_update(h, g, h->cap1, hif, 1, hconf, h->verify ? 1 : 0);
            cudaGraph_t build_body = nullptr;
            e = add_conditional(h->cap1, hif, cudaGraphCondTypeIf, &build_body);
            if (e == cudaSuccess)
                e = cudaStreamBeginCaptureToGraph(h->cap2, build_body, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) {
                launch_build(h, g, 1, h->cap2);
                cudaGraph_t bb_out = nullptr;
                e = cudaStreamEndCapture(h->cap2, &bb_out);
            }
            launch_forces(h, g, h->cap1, false);
            if (e == cudaSuccess && h->verify) {   // the confirming passes, only when due
                cudaGraph_t conf_body = nullptr;
                e = add_conditional(h->cap1, hconf, cudaGraphCondTypeIf, &conf_body);
                if (e == cudaSuccess)
                    e = cudaStreamBeginCaptureToGraph(h->cap2, conf_body, nullptr, nullptr, 0,
                                                      cudaStreamCaptureModeRelaxed);
                if (e == cudaSuccess) {
                    launch_confirm(h, g, h->cap2);
                    cudaGraph_t cb_out = nullptr;
                    e = cudaStreamEndCapture(h->cap2, &cb_out);
                }
            }
            launch_reduce_control(h, g, h->cap1, CTL_LOOP, hw, 1);
            cudaGraph_t body_out = nullptr;
            const cudaError_t e1 = cudaStreamEndCapture(h->cap1, &body_out);
            if (e == cudaSuccess) e = e1;
        }
    }
    k_finalize<<<ceil_div(n, kElemBlock), kElemBlock, 0, h->cap0>>>(h->b);
    cudaGraph_t out = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->cap0, &out);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(h, FIRE_ERR_CUDA, "graph capture failed: %s / %s", cudaGetErrorString(e),
                    cudaGetErrorString(e2));
    }
    e = cudaGraphInstantiate(&h->exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        h->exec = nullptr;
        return fail(h, FIRE_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    }
    h->graph = graph;
    h->gkey = g;
    h->has_graph = true;
    return FIRE_OK;
}

// Captures the kernels `fn` launches on cap0 into an executable plain graph.
template <typename Fn>
fire_status capture_plain(fire_handle* h, cudaGraphExec_t* out, Fn fn) {
    cudaError_t e = cudaStreamBeginCapture(h->cap0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return fail(h, FIRE_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
    fn(h->cap0);
    cudaGraph_t gr = nullptr;
    e = cudaStreamEndCapture(h->cap0, &gr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, FIRE_ERR_CUDA, "capture failed: %s", cudaGetErrorString(e));
    }
    e = cudaGraphInstantiate(out, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return fail(h, FIRE_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    return FIRE_OK;
}

// Chunked execution: three plain graphs (set-up, `chunk` loop bodies, write
// back); every body kernel returns at once when the state says "done", and
// the host reads that flag once per chunk.  Used where conditional graph
// nodes are not wanted (profilers cannot look inside them).
fire_status build_chunked(fire_handle* h, const GeoC& g) {
    drop_graph(h);
    const int n = h->n;
    const cudaGraphConditionalHandle none{};
    fire_status st = capture_plain(h, &h->exec_init, [&](cudaStream_t s) {
        k_prepare<<<ceil_div(n, kElemBlock), kElemBlock, 0, s>>>(h->b);
        launch_build(h, g, 1, s);
        launch_forces(h, g, s);
        launch_reduce_control(h, g, s, CTL_INITIAL, none, 0);
    });
    if (st == FIRE_OK)
        st = capture_plain(h, &h->exec_chunk, [&](cudaStream_t s) {
            for (int c = 0; c < h->chunk; ++c) {
                launch_update(h, g, s, none, 0);
                launch_build(h, g, 0, s);
                launch_forces(h, g, s);
                launch_reduce_control(h, g, s, CTL_LOOP, none, 0);
            }
        });
    if (st == FIRE_OK)
        st = capture_plain(h, &h->exec_final, [&](cudaStream_t s) {
            k_finalize<<<ceil_div(n, kElemBlock), kElemBlock, 0, s>>>(h->b);
        });
    if (st != FIRE_OK) {
        drop_graph(h);
        return st;
    }
    h->gkey = g;
    h->has_graph = true;
    return FIRE_OK;
}

fire_status check_box(fire_handle* h, const double box[3]) {
    if (!box) return fail(h, FIRE_ERR_ARG, "box is NULL");
    const double rc = cutoff(h->pot);
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 0.0) || !std::isfinite(box[a]))
            return fail(h, FIRE_ERR_ARG, "box[%d] = %g must be positive and finite", a, box[a]);
        if (h->sys.periodic[a] && box[a] < 2.0 * rc)
            return fail(h, FIRE_ERR_ARG,
                        "periodic box[%d] = %g is shorter than twice the cut-off %g", a, box[a], rc);
    }
    return FIRE_OK;
}

void init_state(fire_handle* h, double ftol, int64_t maxiter) {
    DevState& s = *h->h_state;
    std::memset(&s, 0, sizeof s);
    const fire_params_t& p = h->par;
    FireParamsD& q = s.prm;
    q.ftol = ftol;
    q.maxiter = maxiter;
    q.dt_start = p.dt_start;
    q.dtmax = p.tmax * p.dt_start;
    q.dtmin = p.tmin * p.dt_start;
    q.dtgrow = p.dtgrow;
    q.dtshrink = p.dtshrink;
    q.alpha0 = p.alpha0;
    q.alphashrink = p.alphashrink;
    q.mass = h->sys.mass;
    q.delaystep = p.delaystep;
    q.vdfmax = p.vdfmax;
    q.halfstepback = p.halfstepback;
    q.initialdelay = p.initialdelay;
    q.norm = p.norm;
    q.integrator = p.integrator;
    q.variant = p.variant;
    q.dmax = p.dmax;
    fire_scal_init(q, s.fs);
    s.budget_ns = (unsigned long long)(h->budget_s * 1e9);
    s.ftol_user = ftol;
    s.vstate = h->verify ? 1 : 0;
    s.vmode = h->verify ? h->par.confirm64 : 0;
    s.fsw = 3.0 * ftol;   // mode 2: the FP64 phase starts below 3 ftol
}

fire_status status_to_error(fire_handle* h, int st) {
    switch (st) {
        case ST_OK: return FIRE_OK;
        case ST_NONFINITE: return fail(h, FIRE_ERR_NONFINITE, "non-finite force, energy or velocity");
        case ST_NBR_OVERFLOW: return fail(h, FIRE_ERR_NBR_OVERFLOW, "neighbour list overflow");
        case ST_TIMEOUT: return fail(h, FIRE_ERR_TIMEOUT, "device loop exceeded its time budget");
        case ST_RANGE:
            return fail(h, FIRE_ERR_ARG, "positions lie more than one box length outside the box");
        case ST_CROWDED:
            return fail(h, FIRE_ERR_ARG,
                        "more than %d atoms within the Stillinger-Weber cut-off of one atom", kSwMax);
        default: return fail(h, FIRE_ERR_CUDA, "unknown device status %d", st);
    }
}

void fill_result(const fire_handle* h, fire_result_t* out) {
    const DevState& s = *h->h_state;
    out->energy = s.energy;
    out->iterations = s.fs.iter;
    out->force_evals = s.fs.evals;
    out->nbr_builds = s.nbr_builds;
    out->stop = s.fs.stop;
    out->reserved = 0;
    out->fmax_atom = std::sqrt(s.fmax2);
    out->f2norm = std::sqrt(s.F2);
    out->finf = s.finf;
    out->dt_final = s.fs.dt;
    out->alpha_final = s.fs.alpha;
}

fire_status check_params(fire_handle* h, const fire_params_t& p) {
    if (!(p.dt_start > 0.0) || !std::isfinite(p.dt_start)) return fail(h, FIRE_ERR_ARG, "dt_start must be > 0");
    if (!(p.tmax > 0.0) || !(p.tmin >= 0.0)) return fail(h, FIRE_ERR_ARG, "tmax must be > 0, tmin >= 0");
    if (!(p.dtgrow >= 1.0) || !(p.dtshrink > 0.0 && p.dtshrink <= 1.0))
        return fail(h, FIRE_ERR_ARG, "need dtgrow >= 1 and 0 < dtshrink <= 1");
    if (!(p.alpha0 >= 0.0 && p.alpha0 <= 1.0) || !(p.alphashrink > 0.0 && p.alphashrink <= 1.0))
        return fail(h, FIRE_ERR_ARG, "need 0 <= alpha0 <= 1 and 0 < alphashrink <= 1");
    if (p.delaystep < 0 || p.vdfmax < 0) return fail(h, FIRE_ERR_ARG, "delaystep and vdfmax must be >= 0");
    if (p.integrator < FIRE_INT_EULER_IMPLICIT || p.integrator > FIRE_INT_LEAPFROG)
        return fail(h, FIRE_ERR_ARG, "unknown integrator %d", p.integrator);
    if (p.variant != FIRE_VARIANT_FIRE2 && p.variant != FIRE_VARIANT_FIRE1)
        return fail(h, FIRE_ERR_ARG, "unknown variant %d", p.variant);
    if (p.norm < 0 || p.norm > 2) return fail(h, FIRE_ERR_ARG, "unknown norm %d", p.norm);
    if (p.confirm64 < FIRE_FP64_CHECK_OFF || p.confirm64 > FIRE_FP64_CHECK_FINISH)
        return fail(h, FIRE_ERR_ARG, "unknown confirm64 setting %d", p.confirm64);
    if (!(p.dmax >= 0.0) || !std::isfinite(p.dmax))
        return fail(h, FIRE_ERR_ARG, "dmax must be finite and >= 0");
    return FIRE_OK;
}

fire_status prepare_call(fire_handle* h, const double box[3], GeoC* g, bool neb_call = false) {
    if (h->batch) return fail(h, FIRE_ERR_STATE, "batched handle: use fire_minimize_batch");
    if (h->neb && !neb_call) return fail(h, FIRE_ERR_STATE, "NEB handle: use fire_neb_minimize");
    fire_status st = check_box(h, box);
    if (st != FIRE_OK) return st;
    CK(h, cudaSetDevice(h->device));
    *g = make_geo(h, box);
    const int cap = std::max(estimate_cap(h, *g), h->cap);
    return ensure_buffers(h, *g, cap);
}

}  // namespace

// Lets the allocation-free entry point (its own translation unit) report a
// message through fire_last_error(NULL).  Not exported from the library.
__attribute__((visibility("hidden"))) void fire2_set_global_error(const char* msg) {
    g_init_err = msg ? msg : "unknown error";
}

// Accessors for the batched form (fire2_batch.cu).  Not exported.
#define FIRE2_HIDDEN __attribute__((visibility("hidden")))
FIRE2_HIDDEN fire_status fire2_batch_fail(fire_handle_t* h, fire_status code, const char* msg) {
    return fail(h, code, "%s", msg);
}
FIRE2_HIDDEN fire_batch_state* fire2_batch_of(fire_handle_t* h) { return h->batch; }
FIRE2_HIDDEN const PotC& fire2_potc(fire_handle_t* h) { return h->potc; }
FIRE2_HIDDEN const fire_potential_t& fire2_pot(fire_handle_t* h) { return h->pot; }
FIRE2_HIDDEN const fire_params_t& fire2_params(fire_handle_t* h) { return h->par; }
FIRE2_HIDDEN const fire_system_t& fire2_sys(fire_handle_t* h) { return h->sys; }
FIRE2_HIDDEN double fire2_budget(fire_handle_t* h) { return h->budget_s; }
FIRE2_HIDDEN const double* fire2_exp_table(fire_handle_t* h) { return h->b.exp_table; }
FIRE2_HIDDEN const float* fire2_exp32_table(fire_handle_t* h) { return h->b.exp32_table; }
FIRE2_HIDDEN double fire2_qscale(fire_handle_t* h) { return h->b.qscale; }
FIRE2_HIDDEN const float* fire2_tab_ffd(fire_handle_t* h) { return h->tab_ffd; }
FIRE2_HIDDEN const float* fire2_tab_fff(fire_handle_t* h) { return h->tab_fff; }
FIRE2_HIDDEN cudaStream_t fire2_stream(fire_handle_t* h) { return h->stream; }

extern "C" {

int32_t fire_abi_version(void) { return FIRE2_ABI_VERSION; }

fire_status fire_default_params(fire_params_t* out, double dt_start) {
    if (!out || !(dt_start > 0.0)) return FIRE_ERR_ARG;
    out->dt_start = dt_start;
    out->tmax = 10.0;
    out->tmin = 0.02;
    out->dtgrow = 1.1;
    out->dtshrink = 0.5;
    out->alpha0 = 0.25;
    out->alphashrink = 0.99;
    out->delaystep = 20;
    out->vdfmax = 2000;
    out->halfstepback = 1;
    out->initialdelay = 1;
    out->integrator = FIRE_INT_EULER_IMPLICIT;
    out->norm = FIRE_NORM_MAX_ATOM;
    out->variant = FIRE_VARIANT_FIRE2;
    out->confirm64 = FIRE_FP64_CHECK_FINISH;
    out->dmax = 0.0;
    return FIRE_OK;
}

// Potential constants for the kernels from h->pot (and the fixed-point scale
// of the FP32-pair form).  Returns false if the exponent range is exceeded.
static bool fill_potc(fire_handle* h) {
    const fire_potential_t* pot = &h->pot;
    PotC& c = h->potc;
    c.kind = pot->kind;
    if (pot->kind == FIRE_POT_SW) {
        c.eps = pot->eps;
        c.sw_sigma = pot->sigma;
        c.sw_rc = pot->sw_a * pot->sigma;
        c.rc2 = c.sw_rc * c.sw_rc;
        c.sw_A = pot->sw_A;
        c.sw_B = pot->sw_B;
        c.sw_p = pot->sw_p;
        c.sw_q = pot->sw_q;
        c.sw_lambda = pot->sw_lambda;
        c.sw_gamma = pot->sw_gamma;
        // integer exponents (p = 4, q = 0 in the original set) are evaluated
        // by multiplication instead of pow()
        auto small_int = [](double e) {
            return (e >= 0.0 && e <= 32.0 && e == std::floor(e)) ? (int)e : -1;
        };
        c.sw_pi = small_int(pot->sw_p);
        c.sw_qi = small_int(pot->sw_q);
        return true;
    }
    if (pot->kind == FIRE_POT_LJ) {
        c.rc2 = pot->rc_lj * pot->rc_lj;
        c.eps = pot->eps;
        c.sigma2 = pot->sigma * pot->sigma;
        const double sr6 = std::pow(pot->sigma / pot->rc_lj, 6.0);
        c.lj_shift = 4.0 * pot->eps * (sr6 * sr6 - sr6);
        return true;
    }
    c.rc2 = pot->rc * pot->rc;
    c.r0sq = pot->r0 * pot->r0;
    c.r0sq_f = (float)c.r0sq;
    c.rc2_f = (float)c.rc2;
    c.A = pot->A;
    c.xi2 = pot->xi * pot->xi;
    c.xi_inv = 1.0 / pot->xi;
    c.p = pot->p;
    c.q2 = 2.0 * pot->q;
    c.r0inv = 1.0 / pot->r0;
    c.p_r0 = pot->p / pot->r0;
    c.q2_r0 = 2.0 * pot->q / pot->r0;
    c.rs = pot->rs;
    c.rc = pot->rc;
    c.winv = 1.0 / (pot->rc - pot->rs);
    // exponent arguments -p s and -2q s with s in [-1, rc/r0 - 1]
    const double smax = std::max(1.0, pot->rc / pot->r0 - 1.0);
    if (!(std::fabs(pot->p) * smax < 80.0 && std::fabs(2.0 * pot->q) * smax < 80.0)) return false;
    if (pot->precision == FIRE_PREC_FP32_PAIR) {
        // fixed-point scale: a power of two with (rc + 3 skin + 2) * qscale < 2^31,
        // so every list pair's separation and r^2 fit their integer types
        const double span = pot->rc + 3.0 * pot->skin + 2.0;
        const int k = (int)std::floor(std::log2(2147483648.0 / span));
        h->b.qscale = std::ldexp(1.0, k);
        c.A_f = (float)pot->A;
        c.xi2_f = (float)(pot->xi * pot->xi);
        c.p_f = (float)pot->p;
        c.q2_f = (float)(2.0 * pot->q);
        c.r0_f = (float)pot->r0;
        c.p_r0_f = (float)(pot->p / pot->r0);
        c.q2_r0_f = (float)(2.0 * pot->q / pot->r0);
        c.rs_f = (float)pot->rs;
        c.winv_f = (float)(1.0 / (pot->rc - pot->rs));
        const double q2 = h->b.qscale * h->b.qscale;
        c.rc2q = (long long)std::floor(pot->rc * pot->rc * q2);
        c.r0sq_q = std::llrint(pot->r0 * pot->r0 * q2);
        c.qinv = (float)(1.0 / h->b.qscale);
        c.qinv2 = (float)(1.0 / q2);
    }
    return true;
}

// Builds the pair-function tables for the current parameters and copies them
// to the device (allocating on the first call).
static fire_status upload_tables(fire_handle* h) {
    const fire_potential_t& p = h->pot;
    const RglTables T = build_rgl_tables(p.A, p.xi, p.p, p.q, p.r0, p.rs, p.rc, 0.04);
    const RglTables T32 = build_rgl_tables(p.A, p.xi, p.p, p.q, p.r0, p.rs, p.rc, 0.12);
    h->potc.tab = T.meta;
    h->potc.tab32 = T32.meta;
    std::vector<float> ffd, fff;
    build_ff_tables(T, p.r0, ffd, fff);
    const size_t nff = ffd.size();
    const size_t nd32 = T32.dens32.size(), nf32 = T32.force32.size();
    if (!h->tab_ffd) {
        CK(h, cudaMalloc(&h->tab_ffd, nff * sizeof(float)));
        CK(h, cudaMalloc(&h->tab_fff, nff * sizeof(float)));
        CK(h, cudaMalloc(&h->tab_d32, nd32 * sizeof(float)));
        CK(h, cudaMalloc(&h->tab_f32, nf32 * sizeof(float)));
    }
    CK(h, cudaMemcpy(h->tab_ffd, ffd.data(), nff * sizeof(float), cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->tab_fff, fff.data(), nff * sizeof(float), cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->tab_d32, T32.dens32.data(), nd32 * sizeof(float), cudaMemcpyHostToDevice));
    CK(h, cudaMemcpy(h->tab_f32, T32.force32.data(), nf32 * sizeof(float), cudaMemcpyHostToDevice));
    h->b.tab_ffd = h->tab_ffd;
    h->b.tab_fff = h->tab_fff;
    h->b.tab_d32 = h->tab_d32;
    h->b.tab_f32 = h->tab_f32;
    // FP32-pair tables sit in shared memory (one per kernel, grid-stride
    // launches); the FP64 form reads its rows through the L1 cache
    h->smem_d = nd32 * sizeof(float);
    h->smem_f = nf32 * sizeof(float);
    const int block = kTabBlock;
    const void* kd = (const void*)k_density32_tab;
    const void* kf = (const void*)k_force32_tab;
    CK(h, cudaFuncSetAttribute(kd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->smem_d));
    CK(h, cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->smem_f));
    int sms = 0, occ_d = 0, occ_f = 0;
    CK(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_d, kd, block, h->smem_d));
    CK(h, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, kf, block, h->smem_f));
    const int need = ceil_div(h->n, block);
    h->nb_tab_d = std::max(1, std::min(need, sms * std::max(occ_d, 1)));
    h->nb_tab_f = std::max(1, std::min(need, sms * std::max(occ_f, 1)));
    return FIRE_OK;
}

static fire_status init_handle(fire_handle_t** hp, const fire_system_t* sys,
                               const fire_potential_t* pot, const fire_params_t* params,
                               bool single) {
    if (!hp || !sys || !pot || !params) return fail(nullptr, FIRE_ERR_ARG, "NULL argument to fire_init");
    *hp = nullptr;
    if (sys->n_atoms < 1 || sys->n_atoms > (int64_t)kIdxMask)
        return fail(nullptr, FIRE_ERR_ARG, "n_atoms = %lld outside [1, %u]", (long long)sys->n_atoms, kIdxMask);
    if (!(sys->mass > 0.0) || !std::isfinite(sys->mass)) return fail(nullptr, FIRE_ERR_ARG, "mass must be > 0");
    if (pot->kind != FIRE_POT_LJ && pot->kind != FIRE_POT_RGL && pot->kind != FIRE_POT_SW)
        return fail(nullptr, FIRE_ERR_ARG, "unknown potential kind %d", pot->kind);
    if (pot->newton < FIRE_NEWTON_AUTO || pot->newton > FIRE_NEWTON_OFF)
        return fail(nullptr, FIRE_ERR_ARG, "unknown newton setting %d", pot->newton);
    if (pot->pair_eval != FIRE_PAIR_TABLE && pot->pair_eval != FIRE_PAIR_ANALYTIC)
        return fail(nullptr, FIRE_ERR_ARG, "unknown pair_eval %d", pot->pair_eval);
    if (pot->precision != FIRE_PREC_FP64 &&
        !(pot->precision == FIRE_PREC_FP32_PAIR && pot->kind == FIRE_POT_RGL))
        return fail(nullptr, FIRE_ERR_ARG,
                    "precision %d not available for this potential (FP32-pair is RGL only)",
                    pot->precision);
    if (!(pot->skin >= 0.0)) return fail(nullptr, FIRE_ERR_ARG, "skin must be >= 0");
    if (pot->kind == FIRE_POT_SW &&
        !(pot->eps > 0.0 && pot->sigma > 0.0 && pot->sw_a > 0.0 && pot->sw_gamma >= 0.0 &&
          std::isfinite(pot->sw_A + pot->sw_B + pot->sw_p + pot->sw_q + pot->sw_lambda)))
        return fail(nullptr, FIRE_ERR_ARG, "SW needs eps, sigma, sw_a > 0 and finite parameters");
    if (pot->kind == FIRE_POT_LJ && !(pot->rc_lj > 0.0 && pot->sigma > 0.0 && pot->eps > 0.0))
        return fail(nullptr, FIRE_ERR_ARG, "LJ needs eps, sigma, rc_lj > 0");
    if (pot->kind == FIRE_POT_RGL &&
        !(pot->rc > pot->rs && pot->rs > 0.0 && pot->r0 > 0.0 && pot->xi > 0.0 && pot->A >= 0.0))
        return fail(nullptr, FIRE_ERR_ARG, "RGL needs 0 < rs < rc, r0 > 0, xi > 0, A >= 0");

    fire_handle* h = new (std::nothrow) fire_handle();
    if (!h) return fail(nullptr, FIRE_ERR_NOMEM, "host allocation failed");
    h->sys = *sys;
    h->pot = *pot;
    h->par = *params;
    h->n = (int)sys->n_atoms;
    h->img_n = h->n;
    fire_status st = check_params(h, *params);
    if (st != FIRE_OK) {
        g_init_err = h->err;
        delete h;
        return st;
    }
    if (!fill_potc(h)) {
        g_init_err = "RGL exponents p, q too large for the exponential's range";
        delete h;
        return FIRE_ERR_ARG;
    }
    double exp_table_host[kExpTableSize];
    h->potc.ex = make_exp_constants(exp_table_host);
    float exp32_table_host[kExp32TableSize];
    h->potc.ex32 = make_exp32_constants(exp32_table_host);
    const bool fp32pair = pot->precision == FIRE_PREC_FP32_PAIR;

    auto bail = [&](fire_status s) {
        g_init_err = h->err;
        fire_destroy(h);
        return s;
    };
#define CKI(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return bail(fail(h, e_ == cudaErrorMemoryAllocation ? FIRE_ERR_NOMEM : FIRE_ERR_CUDA, \
                             "%s: %s", #call, cudaGetErrorString(e_)));                   \
    } while (0)
    CKI(cudaGetDevice(&h->device));
    CKI(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    CKI(cudaStreamCreateWithFlags(&h->cap0, cudaStreamNonBlocking));
    CKI(cudaStreamCreateWithFlags(&h->cap1, cudaStreamNonBlocking));
    CKI(cudaStreamCreateWithFlags(&h->cap2, cudaStreamNonBlocking));
    const size_t n = (size_t)h->n;
    Bufs& b = h->b;
    {
        double* t = nullptr;
        CKI(cudaMalloc(&t, kExpTableSize * sizeof(double)));
        b.exp_table = t;
        CKI(cudaMemcpy(t, exp_table_host, kExpTableSize * sizeof(double), cudaMemcpyHostToDevice));
    }
    if (fp32pair) {
        float* t = nullptr;
        CKI(cudaMalloc(&t, kExp32TableSize * sizeof(float)));
        b.exp32_table = t;
        CKI(cudaMemcpy(t, exp32_table_host, kExp32TableSize * sizeof(float), cudaMemcpyHostToDevice));
    }
    if (!single) {
        // the batched FP64 form, and the FP32-pair form confirming its stops,
        // read the same double-float pair tables
        if (fixed64_form(*pot) || (fp32pair && pot->kind == FIRE_POT_RGL && params->confirm64 != 0)) {
            const fire_status ts = upload_tables(h);
            if (ts != FIRE_OK) return bail(ts);
        }
        *hp = h;
        return FIRE_OK;
    }
    b.n = h->n;
    int sms = 0;
    CKI(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    // Grids.  The pair kernels run one atom per thread on ceil(n / kForceBlock)
    // blocks (the block scheduler evens out uneven neighbour counts), except
    // the table kernels, which hold their tables in shared memory and loop
    // over atoms on a device-sized grid (upload_tables); the element-wise
    // kernels use device-sized grids too, which keeps the partial sums the
    // control kernel adds up few.  nb_force + nb_embed energy partials,
    // nb_red rows of the (F, v) reductions.
    const bool fixed64 = fixed64_form(*pot);
    const bool whole = fp32pair || (fixed64 && !fixed64_half(*pot));   // no atomics
    b.accum = whole ? 0 : 1;
    // pair passes that split an atom's list: enough threads per atom to fill
    // the device on small systems (auto_tpa)
    h->sms = sms;
    b.tpa = tpa_form(*pot) ? auto_tpa(*pot, h->n, sms) : 1;
    b.nb_force = ceil_div((long long)h->n * b.tpa, kForceBlock);
    // blocks per SM of the embedding and the reductions, measured on 1M
    // atoms: embedding 16.4 / 14.3 / 18.4 / 22.1 us at 2 / 4 / 8 / 16;
    // reductions + control 53 / 51 / 57 / 70 us at 1 / 2 / 4 / 8
    b.nb_embed = (pot->kind == FIRE_POT_RGL && !whole)
                     ? std::max(1, std::min(ceil_div(h->n, kElemBlock), sms * 4)) : 0;
    b.nb_red = std::max(1, std::min(ceil_div(h->n, kElemBlock), sms * 2));
    // an FP32-pair stop on ftol is confirmed with the FP64 table passes
    h->verify = fp32pair && pot->kind == FIRE_POT_RGL && params->confirm64 != 0;
    if (pot->kind == FIRE_POT_RGL && (pot->pair_eval == FIRE_PAIR_TABLE || h->verify)) {
        fire_status ts = upload_tables(h);
        if (ts != FIRE_OK) return bail(ts);
        if (fp32pair && pot->pair_eval == FIRE_PAIR_TABLE) b.nb_force = h->nb_tab_d;
    }
    b.nb_verify = h->verify ? dens_ff_grid(h->n, b.tpa) : 0;
    b.pass_role = h->verify ? 1 : 0;
    b.ne_dens = b.nb_force;
    CKI(cudaMalloc(&b.x, n * sizeof(dvec4)));
    CKI(cudaMalloc(&b.v, n * sizeof(dvec4)));
    CKI(cudaMalloc(&b.f, 3 * n * sizeof(double)));
    CKI(cudaMalloc(&b.xf, n * sizeof(float4)));
    if (fp32pair) {
        CKI(cudaMalloc(&b.xq, n * sizeof(int4)));
        CKI(cudaMalloc(&b.fp32, n * sizeof(float)));
    }
    if (fixed64 || h->verify) {
        CKI(cudaMalloc(&b.xq64, n * sizeof(lvec4)));
    }
    CKI(cudaMalloc(&b.nnbr, n * sizeof(int)));
    CKI(cudaMalloc(&b.cell_of, n * sizeof(int)));
    CKI(cudaMalloc(&b.cell_atoms, n * sizeof(int)));
    if (pot->kind == FIRE_POT_RGL) {
        CKI(cudaMalloc(&b.rho, n * sizeof(double)));
        CKI(cudaMalloc(&b.fp, n * sizeof(double)));
    }
    // room for the energy partials at the largest threads per atom
    // (fire_set_threads_per_atom)
    const int nb_max = ceil_div((long long)h->n * kMaxTpa, kForceBlock);
    const size_t n_epart = (size_t)std::max(std::max(b.nb_force, nb_max) + b.nb_embed, nb_max);
    CKI(cudaMalloc(&b.epart, n_epart * sizeof(double)));
    // the FP32-pair table kernels write fewer energy partials than nb_force;
    // the rest stay 0
    CKI(cudaMemset(b.epart, 0, n_epart * sizeof(double)));
    CKI(cudaMalloc(&b.rpart, (size_t)kRedRows * b.nb_red * sizeof(double)));
    CKI(cudaMalloc(&b.st, sizeof(DevState)));
    CKI(cudaMalloc(&b.pos_io, 3 * n * sizeof(double)));
    CKI(cudaMallocHost(&h->h_state, sizeof(DevState)));
    CKI(cudaMallocHost(&h->h_pos, 3 * n * sizeof(double)));
#undef CKI
    *hp = h;
    return FIRE_OK;
}

fire_status fire_init(fire_handle_t** hp, const fire_system_t* sys, const fire_potential_t* pot,
                      const fire_params_t* params) {
    return init_handle(hp, sys, pot, params, true);
}

fire_status fire_batch_init(fire_handle_t** hp, int32_t n_sys, const int64_t* atom_offsets,
                            const fire_system_t* sys, const fire_potential_t* pot,
                            const fire_params_t* params) {
    if (!hp || !atom_offsets || !sys || !pot || !params)
        return fail(nullptr, FIRE_ERR_ARG, "NULL argument to fire_batch_init");
    *hp = nullptr;
    if (n_sys < 1) return fail(nullptr, FIRE_ERR_ARG, "n_sys must be >= 1");
    if (atom_offsets[0] != 0) return fail(nullptr, FIRE_ERR_ARG, "atom_offsets[0] must be 0");
    for (int32_t s = 0; s < n_sys; ++s) {
        const int64_t k = atom_offsets[s + 1] - atom_offsets[s];
        if (k < 1 || k > (int64_t)kIdxMask)
            return fail(nullptr, FIRE_ERR_ARG, "system %d has %lld atoms, outside [1, %u]", s,
                        (long long)k, kIdxMask);
    }
    if (atom_offsets[n_sys] > (int64_t)INT32_MAX)
        return fail(nullptr, FIRE_ERR_ARG, "more than 2^31 - 1 atoms in the batch");
    if (pot->kind != FIRE_POT_RGL)
        return fail(nullptr, FIRE_ERR_ARG, "the batched form supports the RGL potential only");
    fire_system_t s2 = *sys;
    s2.n_atoms = atom_offsets[n_sys];
    fire_status st = init_handle(hp, &s2, pot, params, false);
    if (st != FIRE_OK) return st;
    fire_handle* h = *hp;
    st = fire2_batch_create(h, n_sys, atom_offsets, &h->batch);
    if (st != FIRE_OK) {
        g_init_err = h->err;
        fire_destroy(h);
        *hp = nullptr;
    }
    return st;
}

void fire_destroy(fire_handle_t* h) {
    if (!h) return;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    drop_graph(h);
    Bufs& b = h->b;
    void* ptrs[] = {b.x, b.v, b.f, b.xf, b.xq, b.xq64, b.fp32, (void*)b.exp32_table,
                    (void*)b.exp_table, b.rho, b.fp, b.nbr, b.nnbr, b.crep, b.cden,
                    b.cell_of, b.cell_count, b.cell_start, b.cell_atoms, b.epart, b.rpart,
                    b.st, b.pos_io, b.nbr_loc, b.tile_key, b.tile_ns};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (h->batch) fire2_batch_free(h->batch);
    if (h->neb) neb_free(h->neb);
    for (void* p : {(void*)h->tab_ffd, (void*)h->tab_fff, (void*)h->tab_d32, (void*)h->tab_f32,
                    (void*)h->dofmask})
        if (p) cudaFree(p);
    {
        GradState& gs = h->grad;
        void* gp[] = {gs.x, gs.xf, gs.nbr, gs.nnbr, gs.rho, gs.F1, gs.F2, gs.drho,
                      gs.dq, gs.part, gs.vec, gs.pcache, gs.cs, gs.st};
        for (void* p : gp)
            if (p) cudaFree(p);
        if (gs.h_part) cudaFreeHost(gs.h_part);
        if (gs.h_cs) cudaFreeHost(gs.h_cs);
    }
    if (h->h_state) cudaFreeHost(h->h_state);
    if (h->h_pos) cudaFreeHost(h->h_pos);
    if (h->stream) cudaStreamDestroy(h->stream);
    if (h->cap0) cudaStreamDestroy(h->cap0);
    if (h->cap2) cudaStreamDestroy(h->cap2);
    if (h->cap1) cudaStreamDestroy(h->cap1);
    delete h;
}

const char* fire_last_error(const fire_handle_t* h) {
    return h ? h->err.c_str() : g_init_err.c_str();
}

fire_status fire_set_time_budget(fire_handle_t* h, double seconds) {
    if (!h) return FIRE_ERR_ARG;
    if (!(seconds >= 0.0)) return fail(h, FIRE_ERR_ARG, "time budget must be >= 0");
    h->budget_s = seconds;
    return FIRE_OK;
}

fire_status fire_set_dof_mask(fire_handle_t* h, const uint8_t* mask) {
    if (!h) return FIRE_ERR_ARG;
    if (h->batch) return fail(h, FIRE_ERR_ARG, "frozen degrees of freedom need a single-system handle");
    CK(h, cudaSetDevice(h->device));
    const bool was_on = h->b.dofmask != nullptr;
    if (mask) {
        for (int i = 0; i < h->img_n; ++i)
            if (mask[i] > 7u)
                return fail(h, FIRE_ERR_ARG, "mask[%d] = %u: only bits 0..2 (x, y, z) exist", i,
                            (unsigned)mask[i]);
        if (!h->dofmask) {
            cudaError_t e = cudaMalloc(&h->dofmask, (size_t)std::max(h->n, 1));
            if (e != cudaSuccess) {
                h->dofmask = nullptr;
                return fail(h, e == cudaErrorMemoryAllocation ? FIRE_ERR_NOMEM : FIRE_ERR_CUDA,
                            "cudaMalloc(mask): %s", cudaGetErrorString(e));
            }
        }
        CK(h, cudaStreamSynchronize(h->stream));
        // a NEB handle takes one image's mask and applies it to every image
        for (int k = 0; k < h->n / h->img_n; ++k)
            CK(h, cudaMemcpy(h->dofmask + (size_t)k * h->img_n, mask, (size_t)h->img_n,
                             cudaMemcpyHostToDevice));
        h->b.dofmask = h->dofmask;
    } else {
        h->b.dofmask = nullptr;
    }
    // the relaxation graph holds the kernels' arguments: capture again
    if (was_on != (h->b.dofmask != nullptr)) drop_graph(h);
    return FIRE_OK;
}

// One relaxation on the device: positions are already in b.pos_io.
static fire_status run_minimize(fire_handle* h, const GeoC& g, double ftol, int64_t maxiter,
                                cudaStream_t s) {
    const bool chunked = h->exec_mode == FIRE_EXEC_CHUNKED;
    const bool have = chunked ? h->exec_chunk != nullptr : h->exec != nullptr;
    if (!h->has_graph || !have || !same_geo(h->gkey, g)) {
        fire_status st = chunked ? build_chunked(h, g) : build_graph(h, g);
        if (st != FIRE_OK) return st;
    }
    init_state(h, ftol, maxiter);
    CK(h, cudaMemcpyAsync(h->b.st, h->h_state, sizeof(DevState), cudaMemcpyHostToDevice, s));
    if (!chunked) {
        CK(h, cudaGraphLaunch(h->exec, s));
    } else {
        CK(h, cudaGraphLaunch(h->exec_init, s));
        const long long max_chunks = maxiter / h->chunk + 2;
        for (long long c = 0; c < max_chunks; ++c) {
            CK(h, cudaMemcpyAsync(h->h_state, h->b.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
            CK(h, cudaStreamSynchronize(s));
            if (h->h_state->done) break;
            CK(h, cudaGraphLaunch(h->exec_chunk, s));
        }
        CK(h, cudaGraphLaunch(h->exec_final, s));
    }
    CK(h, cudaMemcpyAsync(h->h_state, h->b.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    return status_to_error(h, h->h_state->status);
}

fire_status fire_set_threads_per_atom(fire_handle_t* h, int32_t tpa, int32_t* chosen) {
    if (!h) return FIRE_ERR_ARG;
    if (h->batch) return fail(h, FIRE_ERR_ARG, "batched handle: use fire_batch_set_tuning");
    if (tpa != 0 && tpa != 1 && tpa != 2 && tpa != 4 && tpa != 8 && tpa != 16 && tpa != 32)
        return fail(h, FIRE_ERR_ARG, "threads per atom must be 0 (automatic), 1, 2, 4, 8, 16 or 32");
    const int t = !tpa_form(h->pot) ? 1 : tpa == 0 ? auto_tpa(h->pot, h->n, h->sms) : tpa;
    if (t != h->b.tpa) {
        drop_graph(h);
        h->b.tpa = t;
        if (!(h->pot.precision == FIRE_PREC_FP32_PAIR && h->pot.pair_eval == FIRE_PAIR_TABLE))
            h->b.nb_force = ceil_div((long long)h->n * t, kForceBlock);
        if (h->verify) h->b.nb_verify = dens_ff_grid(h->n, t);
    }
    if (chosen) *chosen = t;
    return FIRE_OK;
}

fire_status fire_set_pair_tiles(fire_handle_t* h, int32_t mode, int32_t stage_cap) {
    if (!h) return FIRE_ERR_ARG;
    if (h->batch) return fail(h, FIRE_ERR_ARG, "batched handle: tiles are per single system");
    if (mode != FIRE_TILES_AUTO && mode != FIRE_TILES_ON && mode != FIRE_TILES_OFF)
        return fail(h, FIRE_ERR_ARG, "unknown tile mode %d", mode);
    if (stage_cap != 0 && (stage_cap < 64 || stage_cap > kStageMax))
        return fail(h, FIRE_ERR_ARG, "stage_cap must be 0 or in [64, %d]", kStageMax);
    drop_graph(h);
    h->tile_mode = mode;
    h->stage_cap = stage_cap;
    return FIRE_OK;
}

fire_status fire_set_exec_mode(fire_handle_t* h, int32_t mode, int32_t chunk) {
    if (!h) return FIRE_ERR_ARG;
    if (mode != FIRE_EXEC_GRAPH_WHILE && mode != FIRE_EXEC_CHUNKED)
        return fail(h, FIRE_ERR_ARG, "unknown execution mode %d", mode);
    if (mode == FIRE_EXEC_CHUNKED && (chunk < 1 || chunk > 4096))
        return fail(h, FIRE_ERR_ARG, "chunk must be in [1, 4096]");
    if (mode == FIRE_EXEC_GRAPH_WHILE && (chunk < 0 || chunk > kMaxBodyIters))
        return fail(h, FIRE_ERR_ARG, "iterations per loop body must be in [0, %d]", kMaxBodyIters);
    drop_graph(h);
    h->exec_mode = mode;
    if (mode == FIRE_EXEC_CHUNKED) h->chunk = chunk;
    else h->body_iters = chunk;
    return FIRE_OK;
}

fire_status fire_minimize_dev(fire_handle_t* h, double* d_pos, const double box[3], double ftol,
                              int64_t maxiter, fire_result_t* out, void* stream) {
    if (!h) return FIRE_ERR_ARG;
    if (!d_pos || !out) return fail(h, FIRE_ERR_ARG, "NULL positions or result");
    if (!(ftol >= 0.0) || maxiter < 0) return fail(h, FIRE_ERR_ARG, "need ftol >= 0 and maxiter >= 0");
    GeoC g;
    fire_status st = prepare_call(h, box, &g);
    if (st != FIRE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)3 * h->n * sizeof(double);
    for (int attempt = 0; attempt < 4; ++attempt) {
        CK(h, cudaMemcpyAsync(h->b.pos_io, d_pos, bytes, cudaMemcpyDeviceToDevice, s));
        st = run_minimize(h, g, ftol, maxiter, s);
        if (st != FIRE_ERR_NBR_OVERFLOW || h->cap >= h->n - 1) break;
        st = ensure_buffers(h, g, std::min(2 * h->cap, std::max(h->n - 1, 1)));
        if (st != FIRE_OK) return st;
    }
    if (st != FIRE_OK) return st;
    CK(h, cudaMemcpyAsync(d_pos, h->b.pos_io, bytes, cudaMemcpyDeviceToDevice, s));
    CK(h, cudaStreamSynchronize(s));
    fill_result(h, out);
    return FIRE_OK;
}

// Device-to-host copy of a call's result into the caller's array, with the
// stream synchronised: straight into page-locked (pinned or registered)
// memory, through the handle's pinned staging buffer otherwise.
cudaError_t copy_to_host(fire_handle* h, double* dst, const double* src, size_t bytes,
                         cudaStream_t s) {
    cudaPointerAttributes a{};
    bool locked = false;
    if (cudaPointerGetAttributes(&a, dst) == cudaSuccess)
        locked = a.type == cudaMemoryTypeHost;
    else
        cudaGetLastError();   // the query's own error: take the staging copy
    cudaError_t e = cudaMemcpyAsync(locked ? dst : h->h_pos, src, bytes, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && !locked) std::memcpy(dst, h->h_pos, bytes);
    return e;
}

fire_status fire_minimize(fire_handle_t* h, double* pos, const double box[3], double ftol,
                          int64_t maxiter, fire_result_t* out) {
    if (!h) return FIRE_ERR_ARG;
    if (!pos || !out) return fail(h, FIRE_ERR_ARG, "NULL positions or result");
    if (!(ftol >= 0.0) || maxiter < 0) return fail(h, FIRE_ERR_ARG, "need ftol >= 0 and maxiter >= 0");
    GeoC g;
    fire_status st = prepare_call(h, box, &g);
    if (st != FIRE_OK) return st;
    cudaStream_t s = h->stream;
    const size_t bytes = (size_t)3 * h->n * sizeof(double);
    for (int attempt = 0; attempt < 4; ++attempt) {
        CK(h, cudaMemcpyAsync(h->b.pos_io, pos, bytes, cudaMemcpyHostToDevice, s));
        st = run_minimize(h, g, ftol, maxiter, s);
        if (st != FIRE_ERR_NBR_OVERFLOW || h->cap >= h->n - 1) break;
        st = ensure_buffers(h, g, std::min(2 * h->cap, std::max(h->n - 1, 1)));
        if (st != FIRE_OK) return st;
    }
    if (st != FIRE_OK) return st;
    CK(h, copy_to_host(h, pos, h->b.pos_io, bytes, s));
    fill_result(h, out);
    return FIRE_OK;
}

// Energy and forces at one configuration (plain stream launches); the
// frozen-DOF mask belongs to relaxations only.
static fire_status run_eval_unmasked(fire_handle* h, const GeoC& g, cudaStream_t s);
static fire_status run_eval(fire_handle* h, const GeoC& g, cudaStream_t s) {
    const uint8_t* mask = h->b.dofmask;
    h->b.dofmask = nullptr;
    const fire_status st = run_eval_unmasked(h, g, s);
    h->b.dofmask = mask;
    return st;
}

static fire_status run_eval_unmasked(fire_handle* h, const GeoC& g, cudaStream_t s) {
    init_state(h, 0.0, 0);
    CK(h, cudaMemcpyAsync(h->b.st, h->h_state, sizeof(DevState), cudaMemcpyHostToDevice, s));
    k_prepare<<<ceil_div(h->n, kElemBlock), kElemBlock, 0, s>>>(h->b);
    launch_build(h, g, 1, s);
    launch_forces(h, g, s);
    launch_reduce_control(h, g, s, CTL_EVAL, cudaGraphConditionalHandle{}, 0);
    k_export_forces<<<ceil_div(h->n, kElemBlock), kElemBlock, 0, s>>>(h->b);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(h->h_state, h->b.st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    return status_to_error(h, h->h_state->status);
}

fire_status fire_energy_forces_dev(fire_handle_t* h, const double* d_pos, const double box[3],
                                   double* d_forces, double* d_energy, void* stream) {
    if (!h) return FIRE_ERR_ARG;
    if (!d_pos) return fail(h, FIRE_ERR_ARG, "NULL positions");
    GeoC g;
    fire_status st = prepare_call(h, box, &g);
    if (st != FIRE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)3 * h->n * sizeof(double);
    for (int attempt = 0; attempt < 4; ++attempt) {
        CK(h, cudaMemcpyAsync(h->b.pos_io, d_pos, bytes, cudaMemcpyDeviceToDevice, s));
        h->b.f_out = d_forces;
        h->b.e_out = d_energy;
        st = run_eval(h, g, s);
        h->b.f_out = nullptr;
        h->b.e_out = nullptr;
        if (st != FIRE_ERR_NBR_OVERFLOW || h->cap >= h->n - 1) break;
        st = ensure_buffers(h, g, std::min(2 * h->cap, std::max(h->n - 1, 1)));
        if (st != FIRE_OK) return st;
    }
    return st;
}

fire_status fire_energy_forces(fire_handle_t* h, const double* pos, const double box[3],
                               double* forces, double* energy) {
    if (!h) return FIRE_ERR_ARG;
    if (!pos) return fail(h, FIRE_ERR_ARG, "NULL positions");
    GeoC g;
    fire_status st = prepare_call(h, box, &g);
    if (st != FIRE_OK) return st;
    cudaStream_t s = h->stream;
    const size_t bytes = (size_t)3 * h->n * sizeof(double);
    for (int attempt = 0; attempt < 4; ++attempt) {
        CK(h, cudaMemcpyAsync(h->b.pos_io, pos, bytes, cudaMemcpyHostToDevice, s));
        st = run_eval(h, g, s);
        if (st != FIRE_ERR_NBR_OVERFLOW || h->cap >= h->n - 1) break;
        st = ensure_buffers(h, g, std::min(2 * h->cap, std::max(h->n - 1, 1)));
        if (st != FIRE_OK) return st;
    }
    if (st != FIRE_OK) return st;
    if (forces) {
        // F is in the padded dvec4 layout; export it row-major through pos_io.
        h->b.f_out = h->b.pos_io;
        k_export_forces<<<ceil_div(h->n, kElemBlock), kElemBlock, 0, s>>>(h->b);
        h->b.f_out = nullptr;
        CK(h, cudaGetLastError());
        CK(h, copy_to_host(h, forces, h->b.pos_io, bytes, s));
    }
    if (energy) *energy = h->h_state->energy;
    return FIRE_OK;
}

// ---- differentiable form ----------------------------------------------------

static void apply_theta(PotC& c, const double th[4]) {
    c.A = th[0];
    c.xi2 = th[1] * th[1];
    c.xi_inv = 1.0 / th[1];
    c.p = th[2];
    c.q2 = 2.0 * th[3];
    c.p_r0 = th[2] * c.r0inv;
    c.q2_r0 = 2.0 * th[3] * c.r0inv;
}

static fire_status check_theta(fire_handle* h, const double th[4]) {
    if (!th) return fail(h, FIRE_ERR_ARG, "theta is NULL");
    if (!(th[0] >= 0.0 && th[1] > 0.0 && std::isfinite(th[2]) && std::isfinite(th[3])))
        return fail(h, FIRE_ERR_ARG, "theta needs A >= 0, xi > 0, finite p and q");
    const double smax = std::max(1.0, h->pot.rc / h->pot.r0 - 1.0);
    if (!(std::fabs(th[2]) * smax < 80.0 && std::fabs(2.0 * th[3]) * smax < 80.0))
        return fail(h, FIRE_ERR_ARG, "theta: p, q too large for the exponential's range");
    return FIRE_OK;
}

// Loads positions, (re)allocates the derivative buffers, builds the full
// list at pos and runs pass 1 (rho, F', F'', drho/dq, energy partials).
static fire_status grad_setup(fire_handle* h, const double* d_pos, const double box[3],
                              const double th[4], cudaStream_t s, GeoC* gout, PotC* pc,
                              GradBufs* gb) {
    if (h->pot.kind != FIRE_POT_RGL) return fail(h, FIRE_ERR_ARG, "derivatives need the RGL potential");
    if (!d_pos) return fail(h, FIRE_ERR_ARG, "NULL positions");
    fire_status st = check_theta(h, th);
    if (st != FIRE_OK) return st;
    GeoC g;
    st = prepare_call(h, box, &g);
    if (st != FIRE_OK) return st;
    g.full = 1;
    GradState& gs = h->grad;
    const int n = h->n;
    const int cap = std::min(std::max(n - 1, 1), 2 * estimate_cap(h, make_geo(h, box)) + 16);
    if (!gs.x) {
        gs.nb = ceil_div(n, kForceBlock);
        CK(h, cudaMalloc(&gs.x, (size_t)n * sizeof(dvec4)));
        CK(h, cudaMalloc(&gs.xf, (size_t)n * sizeof(float4)));
        CK(h, cudaMalloc(&gs.nnbr, (size_t)n * sizeof(int)));
        for (double** p : {&gs.rho, &gs.F1, &gs.F2, &gs.drho, &gs.dq})
            CK(h, cudaMalloc(p, (size_t)n * sizeof(double)));
        CK(h, cudaMalloc(&gs.part, (size_t)9 * gs.nb * sizeof(double)));
        CK(h, cudaMalloc(&gs.vec, (size_t)4 * 3 * n * sizeof(double)));
        CK(h, cudaMallocHost(&gs.h_part, (size_t)9 * gs.nb * sizeof(double)));
        CK(h, cudaMalloc(&gs.st, sizeof(DevState)));
    }
    if (cap > gs.cap) {
        cudaFree(gs.nbr);
        gs.nbr = nullptr;
        CK(h, cudaMalloc(&gs.nbr, (size_t)cap * n * sizeof(uint32_t)));
        gs.cap = cap;
    }
    // list build through the single-system kernels, on the derivative buffers
    Bufs lb = h->b;
    lb.x = gs.x;
    lb.xf = gs.xf;
    lb.xq = nullptr;
    lb.nbr = gs.nbr;
    lb.nnbr = gs.nnbr;
    lb.cap = gs.cap;
    lb.st = gs.st;
    CK(h, cudaMemsetAsync(gs.st, 0, sizeof(DevState), s));
    k_g_load<<<ceil_div(n, kElemBlock), kElemBlock, 0, s>>>(n, d_pos, gs.x, gs.xf);
    const bool brute = g.brute != 0;
    if (!brute) {
        k_cell_zero<<<ceil_div(lb.ncell, kElemBlock), kElemBlock, 0, s>>>(lb, g, 1);
        k_cell_count<<<ceil_div(n, kElemBlock), kElemBlock, 0, s>>>(lb, g, 1);
        k_cell_scan<<<1, 1024, 0, s>>>(lb, g, 1);
        k_cell_fill<<<ceil_div(n, kElemBlock), kElemBlock, 0, s>>>(lb, g, 1);
        k_cell_sort<<<ceil_div(lb.ncell, kElemBlock), kElemBlock, 0, s>>>(lb, g, 1);
    }
    k_nbr_build<<<ceil_div(n, kForceBlock), kForceBlock, 0, s>>>(lb, g, 1);
    CK(h, cudaGetLastError());
    int status = 0;
    CK(h, cudaMemcpyAsync(&status, &gs.st->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    if (status != ST_OK) return status_to_error(h, status);
    *pc = h->potc;
    apply_theta(*pc, th);
    GradBufs b{};
    b.n = n;
    b.cap = gs.cap;
    b.x = gs.x;
    b.nbr = gs.nbr;
    b.nnbr = gs.nnbr;
    b.rho = gs.rho;
    b.F1 = gs.F1;
    b.F2 = gs.F2;
    b.drho = gs.drho;
    b.dq = gs.dq;
    b.part = gs.part;
    GeoL L{{box[0], box[1], box[2]}};
    k_g_atom<<<gs.nb, kForceBlock, 0, s>>>(b, *pc, L, h->b.exp_table);
    CK(h, cudaGetLastError());
    *gout = g;
    *gb = b;
    return FIRE_OK;
}

// Fixed-order host sums of partial rows [k0, k0 + nk) of the derivative partials.
static fire_status grad_sums(fire_handle* h, int k0, int nk, double* out, cudaStream_t s) {
    GradState& gs = h->grad;
    CK(h, cudaMemcpyAsync(gs.h_part + (size_t)k0 * gs.nb, gs.part + (size_t)k0 * gs.nb,
                          (size_t)nk * gs.nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    for (int k = 0; k < nk; ++k) {
        double acc = 0.0;
        for (int b = 0; b < gs.nb; ++b) acc += gs.h_part[(size_t)(k0 + k) * gs.nb + b];
        out[k] = acc;
    }
    return FIRE_OK;
}

fire_status fire_set_rgl_params(fire_handle_t* h, const double theta[4]) {
    if (!h) return FIRE_ERR_ARG;
    if (h->pot.kind != FIRE_POT_RGL) return fail(h, FIRE_ERR_ARG, "not an RGL handle");
    fire_status st = check_theta(h, theta);
    if (st != FIRE_OK) return st;
    h->pot.A = theta[0];
    h->pot.xi = theta[1];
    h->pot.p = theta[2];
    h->pot.q = theta[3];
    fill_potc(h);
    if (h->tab_ffd) {
        st = upload_tables(h);
        if (st != FIRE_OK) return st;
    }
    drop_graph(h);   // the graphs hold the potential constants by value
    return FIRE_OK;
}

fire_status fire_rgl_energy_grad_dev(fire_handle_t* h, const double* d_pos, const double box[3],
                                     const double theta[4], double* d_forces, double* energy,
                                     double dE_dtheta[4], void* stream) {
    if (!h) return FIRE_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    GeoC g;
    PotC pc;
    GradBufs b;
    fire_status st = grad_setup(h, d_pos, box, theta, s, &g, &pc, &b);
    if (st != FIRE_OK) return st;
    if (d_forces) {
        GeoL L{{box[0], box[1], box[2]}};
        k_g_force<<<h->grad.nb, kForceBlock, 0, s>>>(b, pc, L, h->b.exp_table, d_forces, nullptr,
                                                     nullptr);
        CK(h, cudaGetLastError());
    }
    double sums[5];
    st = grad_sums(h, 0, 5, sums, s);
    if (st != FIRE_OK) return st;
    if (!std::isfinite(sums[0])) return fail(h, FIRE_ERR_NONFINITE, "non-finite energy");
    if (energy) *energy = sums[0];
    if (dE_dtheta)
        for (int k = 0; k < 4; ++k) dE_dtheta[k] = sums[1 + k];
    return FIRE_OK;
}

static void launch_hvp(fire_handle* h, const GradBufs& b, const PotC& pc, const double box[3],
                       const double* u, double* hu, cudaStream_t s) {
    GeoL L{{box[0], box[1], box[2]}};
    const int tpa = tpa_for(h->n, h->sms, 1024, kMaxHvpTpa);   // small systems: split the lists
    const int nb = ceil_div((long long)h->n * tpa, kForceBlock);
    const double* et = h->b.exp_table;
    switch (tpa) {
    case 8:
        k_g_hvp1<8><<<nb, kForceBlock, 0, s>>>(b, pc, L, et, u);
        k_g_hvp2<8><<<nb, kForceBlock, 0, s>>>(b, pc, L, et, u, hu);
        break;
    case 4:
        k_g_hvp1<4><<<nb, kForceBlock, 0, s>>>(b, pc, L, et, u);
        k_g_hvp2<4><<<nb, kForceBlock, 0, s>>>(b, pc, L, et, u, hu);
        break;
    case 2:
        k_g_hvp1<2><<<nb, kForceBlock, 0, s>>>(b, pc, L, et, u);
        k_g_hvp2<2><<<nb, kForceBlock, 0, s>>>(b, pc, L, et, u, hu);
        break;
    default:
        k_g_hvp1<1><<<nb, kForceBlock, 0, s>>>(b, pc, L, et, u);
        k_g_hvp2<1><<<nb, kForceBlock, 0, s>>>(b, pc, L, et, u, hu);
    }
}

fire_status fire_rgl_hvp_dev(fire_handle_t* h, const double* d_pos, const double box[3],
                             const double theta[4], const double* d_u, double* d_hu,
                             void* stream) {
    if (!h) return FIRE_ERR_ARG;
    if (!d_u || !d_hu) return fail(h, FIRE_ERR_ARG, "NULL u or Hu");
    cudaStream_t s = (cudaStream_t)stream;
    GeoC g;
    PotC pc;
    GradBufs b;
    fire_status st = grad_setup(h, d_pos, box, theta, s, &g, &pc, &b);
    if (st != FIRE_OK) return st;
    launch_hvp(h, b, pc, box, d_u, d_hu, s);
    CK(h, cudaGetLastError());
    CK(h, cudaStreamSynchronize(s));
    return FIRE_OK;
}

// v -= mean over atoms of each Cartesian component (translation modes).
static fire_status project_out_translations(fire_handle* h, double* v, cudaStream_t s) {
    GradState& gs = h->grad;
    const int n = h->n;
    const int nb = std::min(gs.nb, 1024);
    k_g_colsum<<<nb, kElemBlock, 0, s>>>(n, v, gs.part);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(gs.h_part, gs.part, (size_t)3 * nb * sizeof(double),
                          cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    double m[3];
    for (int k = 0; k < 3; ++k) {
        double acc = 0.0;
        for (int b = 0; b < nb; ++b) acc += gs.h_part[(size_t)k * nb + b];
        m[k] = acc / n;
    }
    k_g_sub_mean<<<nb, kElemBlock, 0, s>>>(n, v, m[0], m[1], m[2]);
    CK(h, cudaGetLastError());
    return FIRE_OK;
}

static fire_status dev_dot(fire_handle* h, const double* a, const double* b, double* out,
                           cudaStream_t s) {
    GradState& gs = h->grad;
    const int nb = std::min(gs.nb, 1024);
    k_g_dot<<<nb, kElemBlock, 0, s>>>(h->n, a, b, gs.part);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpyAsync(gs.h_part, gs.part, (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    double acc = 0.0;
    for (int k = 0; k < nb; ++k) acc += gs.h_part[k];
    *out = acc;
    return FIRE_OK;
}

fire_status fire_rgl_implicit_grad_dev(fire_handle_t* h, const double* d_pos, const double box[3],
                                       const double theta[4], const double* d_g, double tol,
                                       int64_t maxit, double dL_dtheta[4], double* d_lambda,
                                       int64_t* cg_iters, void* stream) {
    if (!h) return FIRE_ERR_ARG;
    if (!d_g || !dL_dtheta) return fail(h, FIRE_ERR_ARG, "NULL g or result");
    if (!(tol > 0.0) || maxit < 1) return fail(h, FIRE_ERR_ARG, "need tol > 0 and maxit >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    GeoC g;
    PotC pc;
    GradBufs b;
    fire_status st = grad_setup(h, d_pos, box, theta, s, &g, &pc, &b);
    if (st != FIRE_OK) return st;
    const int n = h->n, m = 3 * n;
    // the positions are fixed for the whole solve: cache the pair
    // coefficients of the HVP and the separations once (6 doubles per slot)
    {
        GradState& gs = h->grad;
        const size_t slots = (size_t)gs.cap * n;
        if (slots > gs.pcache_slots) {
            cudaFree(gs.pcache);
            gs.pcache = nullptr;
            gs.pcache_slots = 0;
            CK(h, cudaMalloc(&gs.pcache, 6 * slots * sizeof(double)));
            gs.pcache_slots = slots;
        }
        double* w1 = gs.pcache;
        double* fsc = w1 + slots;
        double* a2 = fsc + slots;
        double* dcx = a2 + slots;
        double* dcy = dcx + slots;
        double* dcz = dcy + slots;
        GeoL L{{box[0], box[1], box[2]}};
        k_g_pair_cache<<<gs.nb, kForceBlock, 0, s>>>(b, pc, L, h->b.exp_table, w1, fsc, a2,
                                                      dcx, dcy, dcz);
        CK(h, cudaGetLastError());
        b.w1 = w1;
        b.fsc = fsc;
        b.a2 = a2;
        b.dcx = dcx;
        b.dcy = dcy;
        b.dcz = dcz;
    }
    const size_t bytes = (size_t)m * sizeof(double);
    double* r = h->grad.vec;
    double* p = r + m;
    double* Ap = p + m;
    double* lam = Ap + m;
    const int nb = std::min(h->grad.nb, 1024);
    CK(h, cudaMemcpyAsync(r, d_g, bytes, cudaMemcpyDeviceToDevice, s));
    if ((st = project_out_translations(h, r, s)) != FIRE_OK) return st;
    CK(h, cudaMemsetAsync(lam, 0, bytes, s));
    CK(h, cudaMemcpyAsync(p, r, bytes, cudaMemcpyDeviceToDevice, s));
    double rr = 0.0;
    if ((st = dev_dot(h, r, r, &rr, s)) != FIRE_OK) return st;
    // the iterations run on device scalars (CgState): the host queues
    // kCgBatch of them at a time and reads the state once per batch; the
    // kernels of iterations after the stop return at once
    GradState& gs = h->grad;
    if (!gs.cs) {
        CK(h, cudaMalloc(&gs.cs, sizeof(CgState)));
        CK(h, cudaMallocHost(&gs.h_cs, sizeof(CgState)));
    }
    CgState c0{};
    c0.rr = rr;
    c0.stop2 = tol * tol * rr;
    c0.maxit = maxit;
    if (!std::isfinite(rr))
        return fail(h, FIRE_ERR_NONFINITE, "implicit gradient: dL/dx has a non-finite entry");
    c0.done = (rr > c0.stop2 && rr > 0.0) ? 0 : 1;
    c0.reason = c0.done ? CG_CONVERGED : CG_RUNNING;   // a zero right-hand side is solved
    *gs.h_cs = c0;
    CK(h, cudaMemcpyAsync(gs.cs, gs.h_cs, sizeof(CgState), cudaMemcpyHostToDevice, s));
    GeoL L{{box[0], box[1], box[2]}};
    const int* skip = &gs.cs->done;
    // the cached HVP passes are FP64 pair loops like the force passes: split
    // each atom's list over several threads on small systems
    const int tpa = tpa_for(n, h->sms, 1024, kMaxHvpTpa);
    constexpr int kCgBatch = 16;
    int done = c0.done;
    // the kCgBatch iterations between two reads of the state form one CUDA
    // graph (the pointers stay fixed for the whole solve), launched on s
    cudaGraphExec_t batch = nullptr;
    if (!done) {
        CK(h, cudaStreamSynchronize(s));   // the set-up above is complete before the graph runs
        st = capture_plain(h, &batch, [&](cudaStream_t cs) {
            for (int c = 0; c < kCgBatch; ++c) {
                hvp_cached(b, p, Ap, skip, tpa, n, cs);
                k_cg_colsum<<<nb, kElemBlock, 0, cs>>>(n, gs.cs, Ap, gs.part);
                k_cg_means<<<1, kElemBlock, 0, cs>>>(gs.cs, gs.part, nb, n);
                k_cg_project_dot<<<nb, kElemBlock, 0, cs>>>(n, gs.cs, Ap, p, gs.part);
                k_cg_alpha<<<1, kElemBlock, 0, cs>>>(gs.cs, gs.part, nb);
                k_cg_step<<<nb, kElemBlock, 0, cs>>>(m, gs.cs, p, Ap, lam, r, gs.part);
                k_cg_beta<<<1, kElemBlock, 0, cs>>>(gs.cs, gs.part, nb);
                k_cg_dir<<<nb, kElemBlock, 0, cs>>>(m, gs.cs, r, p);
            }
        });
        if (st != FIRE_OK) return st;
    }
    while (!done) {
        cudaError_t e = cudaGraphLaunch(batch, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(gs.h_cs, gs.cs, sizeof(CgState), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaGraphExecDestroy(batch);
            return fail(h, FIRE_ERR_CUDA, "conjugate-gradient batch: %s", cudaGetErrorString(e));
        }
        done = gs.h_cs->done;
    }
    if (batch) cudaGraphExecDestroy(batch);
    const int64_t it = gs.h_cs->it;
    const int reason = gs.h_cs->reason;
    const double rel_res = rr > 0.0 ? std::sqrt(gs.h_cs->rr / rr) : 0.0;
    k_g_force<<<h->grad.nb, kForceBlock, 0, s>>>(b, pc, L, h->b.exp_table, nullptr, nullptr, lam);
    CK(h, cudaGetLastError());
    double sums[4];
    if ((st = grad_sums(h, 5, 4, sums, s)) != FIRE_OK) return st;
    for (int k = 0; k < 4; ++k) dL_dtheta[k] = sums[k];
    if (d_lambda) CK(h, cudaMemcpyAsync(d_lambda, lam, bytes, cudaMemcpyDeviceToDevice, s));
    CK(h, cudaStreamSynchronize(s));
    if (cg_iters) *cg_iters = it;
    // the outputs above hold the last iterate in every case; a solve that did
    // not reach tol says so in its status
    if (reason == CG_BREAKDOWN)
        return fail(h, FIRE_ERR_NOT_CONVERGED,
                    "implicit gradient: conjugate gradient broke down after %lld iterations "
                    "(p.Hp <= 0 or not finite: the configuration is not at a minimum), "
                    "relative residual %.3e", (long long)it, rel_res);
    if (reason != CG_CONVERGED)
        return fail(h, FIRE_ERR_NOT_CONVERGED,
                    "implicit gradient: conjugate gradient reached maxit = %lld with relative "
                    "residual %.3e > tol = %.3e", (long long)maxit, rel_res, tol);
    return FIRE_OK;
}

fire_status fire_diag_rgl_table(const fire_potential_t* pot, int64_t n, const double* r,
                                double* out) {
    if (!pot || n < 0 || (n > 0 && (!r || !out)) || pot->kind != FIRE_POT_RGL ||
        !(pot->rc > pot->rs && pot->rs > 0.0 && pot->r0 > 0.0 && pot->xi > 0.0))
        return FIRE_ERR_ARG;
    const RglTables T = build_rgl_tables(pot->A, pot->xi, pot->p, pot->q, pot->r0, pot->rs,
                                         pot->rc, 0.04);
    std::vector<float> ffd, fff;
    build_ff_tables(T, pot->r0, ffd, fff);
    const float r0sq_f = (float)(pot->r0 * pot->r0), rc2_f = (float)(pot->rc * pot->rc);
    for (int64_t i = 0; i < n; ++i) {
        double* o = out + 4 * i;
        // the FP64 kernels' arithmetic from r^2 on (r^2 as a float pair)
        const ffloat r2 = f64_to_ff(r[i] * r[i]);
        const float* rd = ff_row(T.meta, ffd, r2.hi - r0sq_f);
        const float* rf = ff_row(T.meta, fff, r2.hi - r0sq_f);
        if (!(r2.hi < rc2_f)) {
            o[0] = o[1] = o[2] = o[3] = 0.0;
        } else if (rd) {
            ffloat d[2], f[2];
            ff_row_eval(rd, r2, d);
            ff_row_eval(rf, r2, f);
            o[0] = ff_to_f64(d[0]);                 // phi
            o[1] = ff_to_f64(d[1]);                 // g
            o[2] = 0.5 * r[i] * ff_to_f64(f[0]);    // phi' = r (2 phi'/r) / 2
            o[3] = r[i] * ff_to_f64(f[1]);          // g' = r (g'/r)
        } else {
            double a[8];
            rgl_analytic(pot->A, pot->xi, pot->p, pot->q, pot->r0, pot->rs, pot->rc, r[i], a);
            o[0] = a[0];
            o[1] = a[4];
            o[2] = a[1];
            o[3] = a[5];
        }
    }
    return FIRE_OK;
}

fire_status fire_profile_stages(fire_handle_t* h, const double* pos, const double box[3],
                                int32_t reps, double* stage_ms) {
    if (!h) return FIRE_ERR_ARG;
    if (!pos || !stage_ms || reps < 1) return fail(h, FIRE_ERR_ARG, "need pos, stage_ms and reps >= 1");
    GeoC g;
    fire_status st = prepare_call(h, box, &g);
    if (st != FIRE_OK) return st;
    cudaStream_t s = h->stream;
    const size_t bytes = (size_t)3 * h->n * sizeof(double);
    CK(h, cudaMemcpyAsync(h->b.pos_io, pos, bytes, cudaMemcpyHostToDevice, s));
    init_state(h, 0.0, 0);   // dt = 0 for the update stage: positions stay put
    h->h_state->fs.dt_cur = 0.0;
    h->h_state->fs.dtm = 0.0;
    CK(h, cudaMemcpyAsync(h->b.st, h->h_state, sizeof(DevState), cudaMemcpyHostToDevice, s));
    k_prepare<<<ceil_div(h->n, kElemBlock), kElemBlock, 0, s>>>(h->b);
    cudaEvent_t ev[FIRE_NSTAGES + 1];
    for (auto& e : ev) CK(h, cudaEventCreate(&e));
    double acc[FIRE_NSTAGES] = {0};
    const bool rgl = h->pot.kind == FIRE_POT_RGL;
    const bool f32 = h->pot.precision == FIRE_PREC_FP32_PAIR;
    for (int r = 0; r <= reps; ++r) {
        cudaEventRecord(ev[0], s);
        launch_build(h, g, 1, s);
        cudaEventRecord(ev[1], s);
        const bool tab = rgl && h->pot.pair_eval == FIRE_PAIR_TABLE;
        if (tab && f32) k_density32_tab<<<h->nb_tab_d, kTabBlock, h->smem_d, s>>>(h->b, h->potc, g);
        else if (tab && fixed64_half(h->pot) && g.tiled)
            k_density_tile<<<tile_grid(h, g), kTileThreads, kDensTileSmem, s>>>(h->b, h->potc, g);
        else if (tab && fixed64_half(h->pot)) density_ff<true>(h->b, h->potc, g, s);
        else if (tab) density_ff<false>(h->b, h->potc, g, s);
        else if (rgl && f32) density32(h->b, h->potc, g, s);
        else if (rgl) k_density<<<h->b.nb_force, kForceBlock, 0, s>>>(h->b, h->potc, g);
        cudaEventRecord(ev[2], s);
        if (h->b.nb_embed > 0) k_embed<<<h->b.nb_embed, kElemBlock, 0, s>>>(h->b);
        cudaEventRecord(ev[3], s);
        if (tab && f32) k_force32_tab<<<h->nb_tab_f, kTabBlock, h->smem_f, s>>>(h->b, h->potc, g);
        else if (tab && fixed64_half(h->pot) && g.tiled)
            k_force_tile<<<tile_grid(h, g), kTileThreads, kForceTileSmem, s>>>(h->b, h->potc, g);
        else if (tab && fixed64_half(h->pot)) force_ff<true>(h->b, h->potc, g, s);
        else if (tab) force_ff<false>(h->b, h->potc, g, s);
        else if (rgl && f32) force32(h->b, h->potc, g, s);
        else if (rgl) k_force_rgl<<<h->b.nb_force, kForceBlock, 0, s>>>(h->b, g);
        else if (h->pot.kind == FIRE_POT_SW) k_force_sw<<<h->b.nb_force, kForceBlock, 0, s>>>(h->b, h->potc, g);
        else force_lj(h->b, h->potc, g, s);
        cudaEventRecord(ev[4], s);
        // the control step runs in the last block of the reductions' launch
        // (k_reduce_ctl; for NEB handles, k_neb_project after k_neb_sums)
        const cudaGraphConditionalHandle none{};
        launch_reduce_control(h, g, s, CTL_EVAL, none, 0);
        cudaEventRecord(ev[5], s);
        cudaEventRecord(ev[6], s);
        launch_update(h, g, s, none, 0);
        cudaEventRecord(ev[7], s);
        cudaError_t e = cudaEventSynchronize(ev[7]);
        if (e != cudaSuccess) {
            for (auto& x : ev) cudaEventDestroy(x);
            return fail(h, FIRE_ERR_CUDA, "profile run failed: %s", cudaGetErrorString(e));
        }
        if (r == 0) continue;  // warm-up repetition
        for (int k = 0; k < FIRE_NSTAGES; ++k) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            acc[k] += ms;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    CK(h, cudaGetLastError());
    CK(h, cudaMemcpy(h->h_state, h->b.st, sizeof(DevState), cudaMemcpyDeviceToHost));
    st = status_to_error(h, h->h_state->status);
    if (st != FIRE_OK) return st;
    for (int k = 0; k < FIRE_NSTAGES; ++k) stage_ms[k] = acc[k] / reps;
    if (!rgl) stage_ms[FIRE_STAGE_DENSITY] = stage_ms[FIRE_STAGE_EMBED] = 0.0;
    return FIRE_OK;
}


// ---------------------------------------------------------------------------
// Nudged elastic band (Sec. 4, cases 7 and 8)

fire_status fire_neb_init(fire_handle_t** hp, int32_t n_img, const fire_system_t* sys,
                          const fire_potential_t* pot, const fire_params_t* params,
                          double k_spring, int32_t climb) {
    if (!hp || !sys || !pot || !params) return fail(nullptr, FIRE_ERR_ARG, "NULL argument to fire_neb_init");
    *hp = nullptr;
    if (n_img < 1) return fail(nullptr, FIRE_ERR_ARG, "n_img = %d must be >= 1", n_img);
    if (!(k_spring >= 0.0) || !std::isfinite(k_spring))
        return fail(nullptr, FIRE_ERR_ARG, "k_spring must be finite and >= 0");
    if (sys->n_atoms < 1 || (int64_t)n_img * sys->n_atoms > (int64_t)kIdxMask)
        return fail(nullptr, FIRE_ERR_ARG, "n_img x n_atoms = %lld outside [1, %u]",
                    (long long)n_img * (long long)sys->n_atoms, kIdxMask);
    fire_system_t all = *sys;
    all.n_atoms = (int64_t)n_img * sys->n_atoms;
    fire_handle_t* h = nullptr;
    fire_status st = init_handle(&h, &all, pot, params, true);
    if (st != FIRE_OK) return st;
    const int N = (int)sys->n_atoms;
    h->img_n = N;
    NebState* q = new (std::nothrow) NebState();
    if (!q) {
        fire_destroy(h);
        return fail(nullptr, FIRE_ERR_NOMEM, "host allocation failed");
    }
    h->neb = q;
    q->n_img = n_img;
    q->k = k_spring;
    q->climb = climb ? 1 : 0;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    q->nb = std::max(1, std::min(ceil_div(N, kNebBlock), std::max(1, sms * 4 / n_img)));
    q->nb_proj = std::max(1, std::min(ceil_div(h->n, kNebBlock), sms * 4));
#define CKN(call)                                                                            \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess) {                                                             \
            fail(nullptr, e_ == cudaErrorMemoryAllocation ? FIRE_ERR_NOMEM : FIRE_ERR_CUDA,  \
                 "%s: %s", #call, cudaGetErrorString(e_));                                   \
            fire_destroy(h);                                                                 \
            return e_ == cudaErrorMemoryAllocation ? FIRE_ERR_NOMEM : FIRE_ERR_CUDA;         \
        }                                                                                    \
    } while (0)
    CKN(cudaMalloc(&q->end, 2 * (size_t)N * sizeof(dvec4)));
    CKN(cudaMalloc(&q->eatom, (size_t)h->n * sizeof(double)));
    CKN(cudaMalloc(&q->part, (size_t)kNebSums * n_img * q->nb * sizeof(double)));
    CKN(cudaMalloc(&q->coef, (size_t)4 * n_img * sizeof(double)));
    CKN(cudaMalloc(&q->E, ((size_t)n_img + 2) * sizeof(double)));
    CKN(cudaMalloc(&q->climber, sizeof(int)));
    CKN(cudaMalloc(&q->d_end_energy, 2 * sizeof(double)));
    // the projection kernel writes the (F, v) reductions
    if (q->nb_proj > h->b.nb_red) {
        cudaFree(h->b.rpart);
        h->b.rpart = nullptr;
        CKN(cudaMalloc(&h->b.rpart, (size_t)kRedRows * q->nb_proj * sizeof(double)));
    }
    h->b.nb_red = q->nb_proj;
    h->b.eatom = q->eatom;
#undef CKN
    fire_system_t one = *sys;
    st = fire_init(&q->inner, &one, pot, params);
    if (st != FIRE_OK) {
        fire_destroy(h);
        return st;
    }
    *hp = h;
    return FIRE_OK;
}

// The band relaxation on device positions d_path ((n_img + 2) x N x 3).
static fire_status neb_run(fire_handle* h, double* d_path, const double box[3], double ftol,
                           int64_t maxiter, fire_result_t* out, double* energies,
                           int32_t* climber, cudaStream_t s) {
    NebState& q = *h->neb;
    const int N = h->img_n, M = q.n_img;
    GeoC g;
    fire_status st = prepare_call(h, box, &g, true);
    if (st != FIRE_OK) return st;
    const size_t img_bytes = (size_t)3 * N * sizeof(double);
    const double* p0 = d_path;
    const double* p1 = d_path + (size_t)3 * N * (M + 1);
    k_neb_load_ends<<<ceil_div(2 * N, kElemBlock), kElemBlock, 0, s>>>(p0, p1, q.end, N);
    CK(h, cudaGetLastError());
    // end-state energies with the one-image handle, written straight into E
    for (int e = 0; e < 2; ++e) {
        st = fire_energy_forces_dev(q.inner, e == 0 ? p0 : p1, box, nullptr, q.d_end_energy + e,
                                    (void*)s);
        if (st != FIRE_OK) return fail(h, st, "end state %d: %s", e, fire_last_error(q.inner));
    }
    CK(h, cudaMemcpyAsync(q.E, q.d_end_energy, sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(h, cudaMemcpyAsync(q.E + M + 1, q.d_end_energy + 1, sizeof(double),
                          cudaMemcpyDeviceToDevice, s));
    for (int attempt = 0; attempt < 4; ++attempt) {
        CK(h, cudaMemcpyAsync(h->b.pos_io, d_path + (size_t)3 * N, img_bytes * M,
                              cudaMemcpyDeviceToDevice, s));
        st = run_minimize(h, g, ftol, maxiter, s);
        if (st != FIRE_ERR_NBR_OVERFLOW || h->cap >= N - 1) break;
        st = ensure_buffers(h, g, std::min(2 * h->cap, std::max(N - 1, 1)));
        if (st != FIRE_OK) return st;
    }
    if (st != FIRE_OK) return st;
    CK(h, cudaMemcpyAsync(d_path + (size_t)3 * N, h->b.pos_io, img_bytes * M,
                          cudaMemcpyDeviceToDevice, s));
    int cl = 0;
    if (energies)
        CK(h, cudaMemcpyAsync(energies, q.E, ((size_t)M + 2) * sizeof(double),
                              cudaMemcpyDeviceToHost, s));
    CK(h, cudaMemcpyAsync(&cl, q.climber, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    if (climber) *climber = cl;
    fill_result(h, out);
    return FIRE_OK;
}

static fire_status neb_check(fire_handle_t* h, const void* path, fire_result_t* out, double ftol,
                             int64_t maxiter) {
    if (!h) return FIRE_ERR_ARG;
    if (!h->neb) return fail(h, FIRE_ERR_STATE, "not a NEB handle (use fire_neb_init)");
    if (!path || !out) return fail(h, FIRE_ERR_ARG, "NULL path or result");
    if (!(ftol >= 0.0) || maxiter < 0) return fail(h, FIRE_ERR_ARG, "need ftol >= 0 and maxiter >= 0");
    return FIRE_OK;
}

fire_status fire_neb_minimize_dev(fire_handle_t* h, double* d_path, const double box[3],
                                  double ftol, int64_t maxiter, fire_result_t* out,
                                  double* energies, int32_t* climber, void* stream) {
    fire_status st = neb_check(h, d_path, out, ftol, maxiter);
    if (st != FIRE_OK) return st;
    CK(h, cudaSetDevice(h->device));
    return neb_run(h, d_path, box, ftol, maxiter, out, energies, climber, (cudaStream_t)stream);
}

fire_status fire_neb_minimize(fire_handle_t* h, double* path, const double box[3], double ftol,
                              int64_t maxiter, fire_result_t* out, double* energies,
                              int32_t* climber) {
    fire_status st = neb_check(h, path, out, ftol, maxiter);
    if (st != FIRE_OK) return st;
    CK(h, cudaSetDevice(h->device));
    NebState& q = *h->neb;
    const size_t bytes = (size_t)3 * h->img_n * (q.n_img + 2) * sizeof(double);
    if (!q.d_path) CK(h, cudaMalloc(&q.d_path, bytes));
    cudaStream_t s = h->stream;
    CK(h, cudaMemcpyAsync(q.d_path, path, bytes, cudaMemcpyHostToDevice, s));
    st = neb_run(h, q.d_path, box, ftol, maxiter, out, energies, climber, s);
    if (st != FIRE_OK) return st;
    CK(h, cudaMemcpyAsync(path, q.d_path, bytes, cudaMemcpyDeviceToHost, s));
    CK(h, cudaStreamSynchronize(s));
    return FIRE_OK;
}

}  // extern "C"
