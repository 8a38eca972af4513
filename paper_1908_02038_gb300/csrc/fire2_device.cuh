// Device-side data structures and kernels of the FIRE 2.0 relaxation loop.
//
// One relaxation iteration (Algorithm 2 of Guenole et al. with the
// semi-implicit Euler integrator of Algorithm 4) is the kernel chain
//
//   [k_update_pre, with a maximum displacement per step] -> k_update
//     -> [k_cell_zero/count/scan/fill/sort -> k_nbr_build, only when an atom
//         moved > skin/2: a graph IF node set by k_update's last block]
//     -> FP64:  k_density_ff(1) -> k_embed -> k_force_ff (tables; k_density /
//               k_force_rgl with exponentials; k_*_tile on shared-memory tiles)
//        FP32-pair: k_density32(_tab) -> k_force32(_tab)
//        LJ:    k_force_lj
//     -> k_reduce_ctl
//
// k_reduce_ctl forms the FP64 reductions of P = F.v, |F|^2, |v|^2 and the
// stopping norms (Sec. 3.4); its last block adds them up, runs the scalar
// dt / alpha / counter logic of Algorithm 2 for the next iteration and sets
// the CUDA-graph WHILE condition, so the whole relaxation runs on the device
// without host syncs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fire2_common.cuh"
#include "fire2_table.cuh"

namespace fire2 {

// Box / neighbour geometry, passed by value.
struct GeoC {
    double L[3], Linv[3];
    int per[3];
    int nc[3];             // cells per axis (cell mode)
    double cinv[3];        // nc / L
    int brute;             // 1 = all-pairs list build (a periodic axis under 3 cells)
    double rlist2;         // (rc + skin)^2
    double half_skin2;     // (skin / 2)^2
    float rc2f;            // rc^2 in FP32: the list puts the pairs inside rc first
    // FP32 copies for the list build's candidate test
    float Lf[3], Linvf[3];
    float rlist2f;         // (rc + skin + margin)^2, margin covers FP32 rounding
    int full;              // 1 = full list (both directions), 0 = half list
    int Lq[3];             // box lengths in fixed-point units, modulo 2^32
    long long Lq64[3];     // box lengths in 2^-44 A units (FP64 form)
    // several images of one system in the same box (nudged elastic band):
    // atoms [k img_n, (k + 1) img_n) form image k and interact only among
    // themselves; one system: img_n = n
    int img_n;
    int ncell_img;         // cells per image (1 in all-pairs mode), bricks padded
    // cells are numbered brick by brick: bricks of bk[0] x bk[1] x bk[2] cells,
    // nbk[a] bricks per axis (the last ones padded with empty cells), cells
    // inside a brick in (x, y, z) order; bk = 1 gives the plain (x, y, z) order
    int bk[3], nbk[3];
    int tiled;             // 1: the FP64 half-list passes run on shared-memory tiles
    int ntile;             // tiles (bricks of one image) when tiled
    int stage_cap;         // staged atoms per tile used by the tile build (<= kStageMax)
};

// Linear index of cell (cx, cy, cz) of image img (brick-major numbering).
__host__ __device__ __forceinline__ int cell_index(const GeoC& g, int img, int cx, int cy, int cz) {
    const int bx = cx / g.bk[0], by = cy / g.bk[1], bz = cz / g.bk[2];
    const int lx = cx - bx * g.bk[0], ly = cy - by * g.bk[1], lz = cz - bz * g.bk[2];
    return img * g.ncell_img + ((bx * g.nbk[1] + by) * g.nbk[2] + bz) * (g.bk[0] * g.bk[1] * g.bk[2]) +
           (lx * g.bk[1] + ly) * g.bk[2] + lz;
}

// FIRE parameters (Table 1) and call arguments, device resident.
struct DevState {
    FireParamsD prm;       // Table 1 parameters and call arguments
    FireScal fs;           // Algorithm 2 state + update coefficients
    unsigned long long budget_ns, t_start;
    long long nbr_builds;
    int done, status;
    // reductions of the current (F, v)
    double P, F2, V2, fmax2, finf, energy;
    unsigned long long max_disp2;           // bits of max |x - x_ref|^2 (>= 0)
    unsigned int upd_blocks;                // k_update blocks finished (last-block test)
    unsigned long long vmax2;               // bits of max |v_i|^2 before the drift (dmax)
    // FP64 check of FP32-pair relaxations (fire_params_t.confirm64): vstate
    // 0 = off, 1 = FP32 phase, 2 = the current evaluation confirms an FP32
    // stop in FP64, 3 = FP64 phase to the end (mode 2, below fsw); prm.ftol is
    // the (possibly tightened) FP32 threshold, ftol_user the caller's, fn32
    // the FP32 norm at the configuration being confirmed
    int vstate, vcount, vmode;
    double ftol_user, fn32, fsw;
    unsigned int red_blocks;   // k_reduce_ctl / k_neb_project blocks finished (last-block test)
    unsigned int neb_blocks;   // k_neb_sums blocks finished (last-block test)
};

struct Bufs {
    int n, cap, ncell;
    int nb_force, nb_embed, nb_red;
    int ne_dens;           // energy partials written by the density (or only) pass
    int tpa;               // threads per atom of the RGL pair passes that split an
                           // atom's list (FP64 table form, FP32-pair analytic form)
    const uint8_t* dofmask;   // frozen components per atom (bit d = axis d), or NULL
    double* eatom;         // per-atom energy (images' energies), or NULL
    int accum;             // 1: forces and densities accumulate with atomics (cleared
                           //    by k_update); 0: force kernels write them whole
    dvec4 *x, *v;
    double* f;             // forces, component-major: F_x,i at f[i], F_y,i at f[n + i],
                           // F_z,i at f[2 n + i] (f_load / f_store / f_add below)
    float4* xf;            // FP32 copy of x at the last list build
    int4* xq;              // FP32-pair form: x in fixed point (qscale units), modulo 2^32
    float* fp32;           // FP32-pair form: F'(rho_i)
    const float* exp32_table;
    double qscale;         // fixed-point units per length unit (a power of two)
    double *rho, *fp;
    const double* exp_table;  // 2^(j/256), j = 0..255
    // tabulated RGL pair functions (fire2_table.cuh); nullptr when analytic
    const float *tab_ffd, *tab_fff;   // FP64 form: density / force rows (kFFRow floats)
    lvec4* xq64;               // FP64 form: positions in 2^-44 A units (x, y, z) and
                               //    F'(rho) as a float pair in w (fp_store / fp_load)
    int pass_role;             // 0: always run; 1: FP32-pair pass that sits out the FP64
                               //    confirmation; 2: FP64 pass that runs only for it
    int nb_verify;             // blocks of the FP64 confirming passes
    const float *tab_d32, *tab_f32;
    uint32_t *nbr;
    int *nnbr;
    // shared-memory tiles of the FP64 half-list passes (fire2_tile.cuh):
    // nbr_loc[k n + p] = stage slot of the k-th neighbour of the atom at
    // cell-sorted position p; tile_key[T kStageMax + s] = list entry (atom |
    // image code) of slot s of tile T; tile_ns[T] = slots in use
    uint16_t* nbr_loc;
    uint32_t* tile_key;
    int* tile_ns;
    double *crep, *cden;
    int *cell_of, *cell_count, *cell_start, *cell_atoms;
    double *epart, *rpart;
    DevState* st;
    double* pos_io;        // N x 3 row-major, in/out of a relaxation
    double* f_out;         // N x 3 row-major forces (evaluation only)
    double* e_out;         // energy (evaluation only)
};

// Forces are stored component-major (three arrays of n doubles): the three
// atomics of a pair term then go to three different 32-byte sectors, which
// the L2 serves in parallel.  With the three components of an atom in one
// sector its atomics queue behind each other: on the 1M-atom box the
// double-float force pass took 0.473 ms that way against 0.423 ms.
__device__ __forceinline__ dvec4 f_load(const Bufs& b, int i) {
    return make_dvec4(b.f[i], b.f[b.n + i], b.f[2 * b.n + i], 0.0);   // 3 n < 2^27
}
__device__ __forceinline__ void f_store(const Bufs& b, int i, double x, double y, double z) {
    b.f[i] = x;
    b.f[b.n + i] = y;
    b.f[2 * b.n + i] = z;
}
__device__ __forceinline__ void f_add(const Bufs& b, int i, double x, double y, double z) {
    atomicAdd(b.f + i, x);
    atomicAdd(b.f + b.n + i, y);
    atomicAdd(b.f + 2 * b.n + i, z);
}

// F'(rho_i) of the double-float form as a float pair, kept in the fourth
// word of the atom's fixed-point position record: the force pass gathers
// one 32-byte record per neighbour for both (1M-atom box: 0.414 against
// 0.423 ms with F' in an array of its own).  The update rewrites x, y, z
// only after the force pass, and the embedding rewrites w before the next.
__device__ __forceinline__ void fp_store(const Bufs& b, int i, ffloat f) {
    b.xq64[i].w = (long long)((unsigned long long)__float_as_uint(f.hi) |
                              ((unsigned long long)__float_as_uint(f.lo) << 32));
}
__device__ __forceinline__ ffloat fp_load(const lvec4& q) {
    return {__uint_as_float((unsigned)((unsigned long long)q.w & 0xffffffffull)),
            __uint_as_float((unsigned)((unsigned long long)q.w >> 32))};
}

// Whether a force pass sits this evaluation out (pass_role above; the state
// says whether the evaluation confirms an FP32-pair stop in FP64).
__device__ __forceinline__ bool pass_skipped(const Bufs& b) {
    if (b.st->done) return true;
    if (b.pass_role == 0) return false;
    const bool confirming = b.st->vstate >= 2;   // confirming, or the FP64 phase
    return b.pass_role == 1 ? confirming : !confirming;
}

// Image-shift table: code = (sx+2) + 5 (sy+2) + 25 (sz+2), shift = s * L.
__device__ __forceinline__ void fill_shift_table(double3* tbl, const GeoC& g) {
    for (int t = threadIdx.x; t < 125; t += blockDim.x) {
        const int sx = t % 5 - 2, sy = (t / 5) % 5 - 2, sz = t / 25 - 2;
        tbl[t] = make_double3(sx * g.L[0], sy * g.L[1], sz * g.L[2]);
    }
}

// Records the first error of a call; later errors do not overwrite it.
__device__ __forceinline__ void set_status(DevState* st, int code) {
    atomicCAS(&st->status, ST_OK, code);
}

// True when the rebuild chain must run this iteration.
__device__ __forceinline__ bool need_rebuild(const DevState* st, const GeoC& g, int force) {
    if (force) return true;
    if (st->done) return false;
    return __longlong_as_double((long long)st->max_disp2) > g.half_skin2;
}

// ---------------------------------------------------------------------------
// set-up / tear-down kernels

// Copies row-major positions into the padded dvec4 layout and clears v, F
// and rho; a non-finite coordinate sets the NONFINITE status (the control
// kernel then stops before the first iteration).  Thread 0 of block 0 stamps
// the start time of the call.
__global__ void k_prepare(Bufs b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) b.st->t_start = globaltimer_ns();
    if (i >= b.n) return;
    const double* p = b.pos_io + 3 * (size_t)i;
    if (!isfinite(p[0]) || !isfinite(p[1]) || !isfinite(p[2])) set_status(b.st, ST_NONFINITE);
    b.x[i] = make_dvec4(p[0], p[1], p[2], 0.0);
    b.xf[i] = make_float4((float)p[0], (float)p[1], (float)p[2], 0.f);
    if (b.xq)
        b.xq[i] = make_int4(to_fixed(p[0], b.qscale), to_fixed(p[1], b.qscale),
                            to_fixed(p[2], b.qscale), 0);
    if (b.xq64)
        b.xq64[i] = {to_fixed64(p[0], kFixedBits64), to_fixed64(p[1], kFixedBits64),
                     to_fixed64(p[2], kFixedBits64), 0ll};
    b.v[i] = make_dvec4(0.0, 0.0, 0.0, 0.0);
    f_store(b, i, 0.0, 0.0, 0.0);
    if (b.rho) b.rho[i] = 0.0;
}

__global__ void k_finalize(Bufs b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.n) return;
    const dvec4 x = b.x[i];
    double* p = b.pos_io + 3 * (size_t)i;
    p[0] = x.x;
    p[1] = x.y;
    p[2] = x.z;
}

__global__ void k_export_forces(Bufs b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0 && b.e_out) *b.e_out = b.st->energy;
    if (i >= b.n || !b.f_out) return;
    const dvec4 f = f_load(b, i);
    double* p = b.f_out + 3 * (size_t)i;
    p[0] = f.x;
    p[1] = f.y;
    p[2] = f.z;
}

// ---------------------------------------------------------------------------
// neighbour list: sort-based cell binning + half list (each pair once)

__global__ void k_cell_zero(Bufs b, GeoC g, int force) {
    if (!need_rebuild(b.st, g, force)) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < b.ncell; c += gridDim.x * blockDim.x)
        b.cell_count[c] = 0;
}

__global__ void k_cell_count(Bufs b, GeoC g, int force) {
    if (!need_rebuild(b.st, g, force)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.n) return;
    const dvec4 x = b.x[i];
    b.xf[i] = make_float4((float)x.x, (float)x.y, (float)x.z, 0.f);   // list-build copy
    const int cx = cell_coord(x.x, g.Linv[0], g.nc[0], g.per[0]);
    const int cy = cell_coord(x.y, g.Linv[1], g.nc[1], g.per[1]);
    const int cz = cell_coord(x.z, g.Linv[2], g.nc[2], g.per[2]);
    const int c = cell_index(g, i / g.img_n, cx, cy, cz);
    b.cell_of[i] = c;
    atomicAdd(&b.cell_count[c], 1);
}

// Exclusive scan of the cell counts (one block); cell_start[ncell] = N.
// cell_count is turned into a fill cursor (= cell_start) for k_cell_fill.
__global__ void k_cell_scan(Bufs b, GeoC g, int force) {
    if (!need_rebuild(b.st, g, force)) return;
    __shared__ int sh[1024];
    const int T = blockDim.x, t = threadIdx.x;
    const int per = (b.ncell + T - 1) / T;
    const int lo = min(t * per, b.ncell), hi = min(lo + per, b.ncell);
    int s = 0;
    for (int c = lo; c < hi; ++c) s += b.cell_count[c];
    sh[t] = s;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {
        int add = t >= o ? sh[t - o] : 0;
        __syncthreads();
        sh[t] += add;
        __syncthreads();
    }
    int run = sh[t] - s;
    for (int c = lo; c < hi; ++c) {
        const int k = b.cell_count[c];
        b.cell_start[c] = run;
        b.cell_count[c] = run;
        run += k;
    }
    if (t == T - 1) b.cell_start[b.ncell] = sh[t];
}

__global__ void k_cell_fill(Bufs b, GeoC g, int force) {
    if (!need_rebuild(b.st, g, force)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.n) return;
    const int slot = atomicAdd(&b.cell_count[b.cell_of[i]], 1);
    b.cell_atoms[slot] = i;
}

// The fill above places a cell's atoms in atomic order; sorting each cell by
// atom index makes the neighbour lists, and with them every sum over a list,
// the same from run to run (one thread per cell, ~13 atoms per cell).
__global__ void k_cell_sort(Bufs b, GeoC g, int force) {
    if (!need_rebuild(b.st, g, force)) return;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= b.ncell) return;
    int* a = b.cell_atoms + b.cell_start[c];
    const int m = b.cell_start[c + 1] - b.cell_start[c];
    for (int k = 1; k < m; ++k) {
        const int v = a[k];
        int j = k - 1;
        while (j >= 0 && a[j] > v) {
            a[j + 1] = a[j];
            --j;
        }
        a[j + 1] = v;
    }
}

// Candidate test in FP32 (the FP64 unit is ~58x slower on this part): the
// list radius carries a margin larger than the FP32 rounding of the
// positions, so every pair closer than rc + skin is kept; the force kernels
// test r < rc again in FP64.
__device__ __forceinline__ float4 xf_of(const Bufs& b, int j) {
    const dvec4 x = b.x[j];
    return make_float4((float)x.x, (float)x.y, (float)x.z, 0.f);
}

// List order: the pairs inside rc come first and the skin pairs (rc up to
// rc + skin, which the force kernels test and skip) after them, so that
// the lanes of a warp evaluate their in-range pairs together and skip their
// skin pairs together; a warp otherwise issues the whole pair evaluation
// whenever any of its lanes has an in-range pair at that list position.
// Skin pairs wait in a small per-thread buffer and are appended at the end
// (beyond kSkinBuf of them the rest are written in the order found).
constexpr int kSkinBuf = 24;
struct SkinBuf {
    uint32_t e[kSkinBuf];
    int n;
};

// FP32 positions come from xf (refreshed by k_cell_count) in cell mode and
// are converted from x in the all-pairs mode (small systems); the caller
// passes candidate j's position xj.
__device__ __forceinline__ void try_add_pair(const Bufs& b, const GeoC& g, int i, float4 xi,
                                             int j, float4 xj, int& cnt, SkinBuf& sk) {
    float d[3] = {xj.x - xi.x, xj.y - xi.y, xj.z - xi.z};
    int s[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (g.per[a]) {
            s[a] = __float2int_rn(d[a] * g.Linvf[a]);
            d[a] -= (float)s[a] * g.Lf[a];
        }
    }
    const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(r2 < g.rlist2f)) return;  // NaN fails too
    if (!g.full && !upper_half(d[0], d[1], d[2])) return;
    // image codes cover shifts of -2..2 box lengths; atoms further apart than
    // that in raw coordinates are a caller error (positions far outside the box)
    if (s[0] < -2 || s[0] > 2 || s[1] < -2 || s[1] > 2 || s[2] < -2 || s[2] > 2) {
        set_status(b.st, ST_RANGE);
        return;
    }
    const uint32_t code = (uint32_t)((s[0] + 2) + 5 * (s[1] + 2) + 25 * (s[2] + 2));
    const uint32_t e = (code << kIdxBits) | (uint32_t)j;
    if (!(r2 < g.rc2f) && sk.n < kSkinBuf) {
        sk.e[sk.n++] = e;
        return;
    }
    if (cnt < b.cap) b.nbr[(size_t)cnt * b.n + i] = e;
    ++cnt;
}

__global__ void k_nbr_build(Bufs b, GeoC g, int force) {
    if (!need_rebuild(b.st, g, force)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) b.st->nbr_builds += 1;
    if (i >= b.n) return;
    const dvec4 xi = b.x[i];
    const float4 xif = g.brute ? xf_of(b, i) : b.xf[i];
    int cnt = 0;
    SkinBuf sk;
    sk.n = 0;
    const int img = i / g.img_n;
    if (g.brute) {
        for (int j = img * g.img_n; j < (img + 1) * g.img_n; ++j)
            if (j != i) try_add_pair(b, g, i, xif, j, xf_of(b, j), cnt, sk);
    } else {
        const int cx = cell_coord(xi.x, g.Linv[0], g.nc[0], g.per[0]);
        const int cy = cell_coord(xi.y, g.Linv[1], g.nc[1], g.per[1]);
        const int cz = cell_coord(xi.z, g.Linv[2], g.nc[2], g.per[2]);
        for (int ox = -1; ox <= 1; ++ox) {
            const int ax = cell_step(cx, ox, g.nc[0], g.per[0]);
            if (ax < 0) continue;
            for (int oy = -1; oy <= 1; ++oy) {
                const int ay = cell_step(cy, oy, g.nc[1], g.per[1]);
                if (ay < 0) continue;
                for (int oz = -1; oz <= 1; ++oz) {
                    const int az = cell_step(cz, oz, g.nc[2], g.per[2]);
                    if (az < 0) continue;
                    const int c = cell_index(g, img, ax, ay, az);
                    const int k1 = b.cell_start[c + 1];
                    int k = b.cell_start[c];
                    // four candidates' indices and positions loaded before
                    // any is tested, so that their loads are in flight
                    // together (the same candidates in the same order)
                    for (; k + 4 <= k1; k += 4) {
                        int jj[4];
                        float4 xx[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) jj[u] = b.cell_atoms[k + u];
#pragma unroll
                        for (int u = 0; u < 4; ++u) xx[u] = b.xf[jj[u]];
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (jj[u] != i) try_add_pair(b, g, i, xif, jj[u], xx[u], cnt, sk);
                    }
                    for (; k < k1; ++k) {
                        const int j = b.cell_atoms[k];
                        if (j != i) try_add_pair(b, g, i, xif, j, b.xf[j], cnt, sk);
                    }
                }
            }
        }
    }
    for (int q = 0; q < sk.n; ++q) {   // the skin pairs after the in-range ones
        if (cnt < b.cap) b.nbr[(size_t)cnt * b.n + i] = sk.e[q];
        ++cnt;
    }
    if (cnt > b.cap) {
        set_status(b.st, ST_NBR_OVERFLOW);
        cnt = b.cap;
    }
    b.nnbr[i] = cnt;
    // the FP32 copy of x at this build, for the displacement test of k_update
    // (with cell lists k_cell_count wrote it already)
    if (g.brute) b.xf[i] = make_float4((float)xi.x, (float)xi.y, (float)xi.z, 0.f);
}

// ---------------------------------------------------------------------------
// RGL second-moment EAM (Sec. 5.2 EAM family), two passes over the half list.

// Pass 1: rho_i = sum_j xi^2 e^{-2q(r/r0-1)} S(r); repulsive energy; per-pair
// cache of (2 phi'(r)/r, g'(r)/r) for pass 2.
__global__ void __launch_bounds__(kForceBlock) k_density(Bufs b, PotC P, GeoC g) {
    __shared__ double3 tbl[125];
    __shared__ double etab[kExpTableSize];
    __shared__ double red[32];
    if (b.st->done) return;
    fill_shift_table(tbl, g);
    for (int t = threadIdx.x; t < kExpTableSize; t += blockDim.x) etab[t] = b.exp_table[t];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double erep = 0.0;
    if (i < b.n) {
        const dvec4 xi = b.x[i];
        const int m = b.nnbr[i];
        double rho_i = 0.0;
        for (int k = 0; k < m; ++k) {
            const size_t slot = (size_t)k * b.n + i;
            const uint32_t e = b.nbr[slot];
            const int j = (int)(e & kIdxMask);
            const int code = (int)(e >> kIdxBits);
            const dvec4 xj = b.x[j];
            double dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
            if (code != kCodeZero) {
                const double3 s = tbl[code];
                dx -= s.x;
                dy -= s.y;
                dz -= s.z;
            }
            const double r2 = dx * dx + dy * dy + dz * dz;
            double crep = 0.0, cden = 0.0;
            if (r2 < P.rc2) {
                const double rinv = rsqrt(r2);
                const double r = r2 * rinv;
                const double s = r * P.r0inv - 1.0;
                const double ep = P.A * exp_tang(-P.p * s, P.ex, etab);
                const double eq = P.xi2 * exp_tang(-P.q2 * s, P.ex, etab);
                double S = 1.0, dS = 0.0;
                if (r > P.rs) {
                    const double t = (r - P.rs) * P.winv;
                    const double t2 = t * t, t3 = t2 * t;
                    S = 1.0 - 10.0 * t3 + 15.0 * t3 * t - 6.0 * t3 * t2;
                    dS = (-30.0 * t2 + 60.0 * t3 - 30.0 * t3 * t) * P.winv;
                }
                const double gg = eq * S;
                rho_i += gg;
                atomicAdd(&b.rho[j], gg);
                erep += 2.0 * ep * S;
                crep = 2.0 * ep * (-P.p_r0 * S + dS) * rinv;
                cden = eq * (-P.q2_r0 * S + dS) * rinv;
            }
            b.crep[slot] = crep;
            b.cden[slot] = cden;
        }
        atomicAdd(&b.rho[i], rho_i);
        if (b.eatom) b.eatom[i] = erep;
    }
    const double s = block_sum(erep, red);
    if (threadIdx.x == 0) b.epart[blockIdx.x] = s;
}

// Embedding F(rho) = -sqrt(rho), F'(rho) = -1/(2 sqrt(rho)); an atom with
// rho = 0 has no pair inside rc, so its F' is never used (set to 0).
__global__ void k_embed(Bufs b) {
    __shared__ double red[32];
    if (b.st->done) return;
    double emb = 0.0;
    ffloat emb_ff = {0.f, 0.f};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < b.n; i += gridDim.x * blockDim.x) {
        const double rho = b.rho[i];
        if (b.xq64 && ff_range(rho)) {
            // FP64 form with double-float pair terms: the embedding in float
            // pairs too, F' as a float pair for the force pass (the only
            // reader of F' in this form) and the energy summed in float
            // pairs; the range test and the split of rho on the integer
            // pipes (FP64 instructions issue at 1/58 of the FP32 rate)
            ffloat sqf, fpf;
            rgl_embed_ff(f64_to_ff_int(rho), sqf, fpf);
            fp_store(b, i, fpf);
            emb_ff = ff_acc(emb_ff, {-sqf.hi, -sqf.lo});
            if (b.eatom) b.eatom[i] -= ff_to_f64(sqf);
            continue;
        }
        double sq, fp;
        rgl_embed(rho, sq, fp);
        if (b.xq64) {
            fp_store(b, i, f64_to_ff(fp));
        } else {
            b.fp[i] = fp;
        }
        emb -= sq;
        if (b.eatom) b.eatom[i] -= sq;
    }
    emb += ff_to_f64(emb_ff);
    const double s = block_sum(emb, red);
    if (threadIdx.x == 0) b.epart[b.ne_dens + blockIdx.x] = s;
}

// Pass 2: F_i += fs d, F_j -= fs d with fs = [2 phi' + (F'_i + F'_j) g'] / r
// and d = x_j - x_i (F = -grad E, Sec. 2.1).
__global__ void __launch_bounds__(kForceBlock) k_force_rgl(Bufs b, GeoC g) {
    __shared__ double3 tbl[125];
    if (b.st->done) return;
    fill_shift_table(tbl, g);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= b.n) return;
    const dvec4 xi = b.x[i];
    const double fpi = b.fp[i];
    const int m = b.nnbr[i];
    double fx = 0.0, fy = 0.0, fz = 0.0;
    for (int k = 0; k < m; ++k) {
        const size_t slot = (size_t)k * b.n + i;
        const double crep = b.crep[slot], cden = b.cden[slot];
        // pairs beyond rc carry an all-zero cache entry (integer test, no FP64 op)
        if ((__double_as_longlong(crep) | __double_as_longlong(cden)) == 0) continue;
        const uint32_t e = b.nbr[slot];
        const int j = (int)(e & kIdxMask);
        const int code = (int)(e >> kIdxBits);
        const dvec4 xj = b.x[j];
        double dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
        if (code != kCodeZero) {
            const double3 s = tbl[code];
            dx -= s.x;
            dy -= s.y;
            dz -= s.z;
        }
        const double fs = crep + (fpi + b.fp[j]) * cden;
        fx += fs * dx;
        fy += fs * dy;
        fz += fs * dz;
        f_add(b, j, -fs * dx, -fs * dy, -fs * dz);
    }
    f_add(b, i, fx, fy, fz);
}

// Stillinger-Weber, one pass over the full list (IEEE FP64): the pair term
// from both ends (half its energy to each atom, its force on i), then the
// three-body terms centred on i for every pair j < k of neighbours within
// a sigma, their gradients added to i here and to j and k by FP64 atomics:
//   h = lambda eps (c + 1/3)^2 e_j e_k,  e = exp(gamma sigma / (r - a sigma)),
//   dh/dx_j = dh/dr_j u_j + dh/dc (u_k - c u_j) / r_j   (u = unit vectors).
// Everything that depends on one neighbour only (u, 1/r, e, and
// gamma sigma / (r - a sigma)^2 = -d ln e / dr) is computed once per
// neighbour, so the triplet loop has no division or exponential.
constexpr int kSwMax = 32;   // neighbours within a sigma per atom (a solid has 4)

// x^e for the SW exponents: repeated squaring when e is a small non-negative
// integer (ei >= 0), pow() otherwise.
__device__ __forceinline__ double sw_pow(double x, double e, int ei) {
    if (ei < 0) return pow(x, e);
    double r = 1.0, b = x;
    for (int n = ei; n > 0; n >>= 1) {
        if (n & 1) r *= b;
        b *= b;
    }
    return r;
}

// Pair term phi2(r) and phi2'(r) from invr = 1/r and t = 1/(r - a sigma).
__device__ __forceinline__ void sw_pair(const PotC& P, double invr, double t, double& e2,
                                        double& de2) {
    const double s = P.sw_sigma;
    const double sr = s * invr;
    const double bp = P.sw_B * sw_pow(sr, P.sw_p, P.sw_pi), bq = sw_pow(sr, P.sw_q, P.sw_qi);
    const double ex = exp(s * t);
    e2 = P.sw_A * P.eps * (bp - bq) * ex;
    de2 = P.sw_A * P.eps * ex * ((-P.sw_p * bp + P.sw_q * bq) * invr - (bp - bq) * s * t * t);
}

__global__ void __launch_bounds__(kForceBlock) k_force_sw(Bufs b, PotC P, GeoC g) {
    __shared__ double3 tbl[125];
    __shared__ double red[32];
    if (b.st->done) return;
    fill_shift_table(tbl, g);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double e_i = 0.0;
    if (i < b.n) {
        const dvec4 xi = b.x[i];
        const int m = b.nnbr[i];
        // per neighbour: unit vector, 1/r, exp(gamma sigma / (r - a sigma)) and
        // gamma sigma / (r - a sigma)^2, so the triplet loop only multiplies
        int nj[kSwMax];
        double ux[kSwMax], uy[kSwMax], uz[kSwMax], ir[kSwMax], eg[kSwMax], gd[kSwMax];
        int cnt = 0;
        double fx = 0.0, fy = 0.0, fz = 0.0;
        const double gs = P.sw_gamma * P.sw_sigma, rc = P.sw_rc;
        const double le = P.sw_lambda * P.eps;
        for (int k = 0; k < m; ++k) {
            const uint32_t e = b.nbr[(size_t)k * b.n + i];
            const int j = (int)(e & kIdxMask);
            const int code = (int)(e >> kIdxBits);
            const dvec4 xj = b.x[j];
            double dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
            if (code != kCodeZero) {
                const double3 sh = tbl[code];
                dx -= sh.x;
                dy -= sh.y;
                dz -= sh.z;
            }
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 < P.rc2)) continue;
            const double invr = rsqrt_newton(r2);   // r2 > 0: list pairs are distinct atoms
            const double r = r2 * invr;
            const double t = 1.0 / (r - rc);
            double e2, de2;
            sw_pair(P, invr, t, e2, de2);
            e_i += 0.5 * e2;
            const double w = de2 * invr;   // force on i from the pair: +phi2'(r) d / r
            fx += w * dx;
            fy += w * dy;
            fz += w * dz;
            if (cnt < kSwMax) {
                nj[cnt] = j;
                ux[cnt] = dx * invr;
                uy[cnt] = dy * invr;
                uz[cnt] = dz * invr;
                ir[cnt] = invr;
                eg[cnt] = exp(gs * t);
                gd[cnt] = gs * t * t;
            }
            ++cnt;
        }
        if (cnt > kSwMax) {
            set_status(b.st, ST_CROWDED);
            cnt = kSwMax;
        }
        for (int p = 0; p < cnt; ++p)
            for (int q = p + 1; q < cnt; ++q) {
                const double ujx = ux[p], ujy = uy[p], ujz = uz[p];
                const double ukx = ux[q], uky = uy[q], ukz = uz[q];
                const double cs = ujx * ukx + ujy * uky + ujz * ukz;   // cos theta_jik
                const double wv = cs + 1.0 / 3.0;
                const double ee = eg[p] * eg[q];
                const double h = le * wv * wv * ee;
                e_i += h;
                const double dh_dc = 2.0 * le * wv * ee;
                const double dj = -h * gd[p], dk = -h * gd[q];
                const double cj = dh_dc * ir[p], ck = dh_dc * ir[q];
                const double gjx = dj * ujx + cj * (ukx - cs * ujx);
                const double gjy = dj * ujy + cj * (uky - cs * ujy);
                const double gjz = dj * ujz + cj * (ukz - cs * ujz);
                const double gkx = dk * ukx + ck * (ujx - cs * ukx);
                const double gky = dk * uky + ck * (ujy - cs * uky);
                const double gkz = dk * ukz + ck * (ujz - cs * ukz);
                fx += gjx + gkx;
                fy += gjy + gky;
                fz += gjz + gkz;
                f_add(b, nj[p], -gjx, -gjy, -gjz);
                f_add(b, nj[q], -gkx, -gky, -gkz);
            }
        f_add(b, i, fx, fy, fz);
        if (b.eatom) b.eatom[i] = e_i;
    }
    const double bs = block_sum(e_i, red);
    if (threadIdx.x == 0) b.epart[blockIdx.x] = bs;
}

// Lennard-Jones, one pass: w = 24 eps [2 (s/r)^12 - (s/r)^6] / r^2,
// F_i -= w d, F_j += w d; pair energy 4 eps [(s/r)^12 - (s/r)^6] - phi(rc).
template <int TPA = 1>
__global__ void __launch_bounds__(kForceBlock) k_force_lj(Bufs b, PotC P, GeoC g) {
    __shared__ double3 tbl[125];
    __shared__ double red[32];
    if (b.st->done) return;
    fill_shift_table(tbl, g);
    __syncthreads();
    // TPA threads share an atom (small systems): lane l takes list slots
    // l, l + TPA, ...; their sums meet in FP64 before lane 0 adds F_i
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / TPA, lane = t % TPA;
    double epair = 0.0;
    if (i < b.n) {
        const dvec4 xi = b.x[i];
        const int m = b.nnbr[i];
        double fx = 0.0, fy = 0.0, fz = 0.0;
        for (int k = lane; k < m; k += TPA) {
            const uint32_t e = b.nbr[(size_t)k * b.n + i];
            const int j = (int)(e & kIdxMask);
            const int code = (int)(e >> kIdxBits);
            const dvec4 xj = b.x[j];
            double dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
            if (code != kCodeZero) {
                const double3 s = tbl[code];
                dx -= s.x;
                dy -= s.y;
                dz -= s.z;
            }
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 < P.rc2)) continue;
            // one correctly rounded reciprocal in place of two FP64 divisions
            // (each a long FP64 sequence on a part where FP64 issues at 1/58
            // of the FP32 rate)
            const double ir2 = __drcp_rn(r2);
            const double sr2 = P.sigma2 * ir2;
            const double sr6 = sr2 * sr2 * sr2;
            epair += 4.0 * P.eps * (sr6 * sr6 - sr6) - P.lj_shift;
            const double w = 24.0 * P.eps * (2.0 * sr6 * sr6 - sr6) * ir2;
            fx -= w * dx;
            fy -= w * dy;
            fz -= w * dz;
            f_add(b, j, w * dx, w * dy, w * dz);
        }
        if (TPA == 32) {
            // a whole warp per atom: the four sums in one transposing
            // butterfly (6 FP64 additions in place of 20); lanes 0, 8 and 16
            // then hold F_x, F_y and F_z, lane 24 the energy
            const double s4 = warp_sum4(fx, fy, fz, epair);
            if (lane == 0 || lane == 8 || lane == 16) atomicAdd(b.f + (size_t)(lane >> 3) * b.n + i, s4);
            if (lane == 24 && b.eatom) b.eatom[i] = s4;
        } else {
            fx = group_sum<TPA>(fx);
            fy = group_sum<TPA>(fy);
            fz = group_sum<TPA>(fz);
            const double ep = group_sum<TPA>(epair);
            if (lane == 0) {
                f_add(b, i, fx, fy, fz);
                if (b.eatom) b.eatom[i] = ep;
            }
        }
    }
    const double s = block_sum(epair, red);
    if (threadIdx.x == 0) b.epart[blockIdx.x] = s;
}

// ---------------------------------------------------------------------------
// FP32-pair form of the RGL passes (full list, one thread per atom, no atomics).
//
// Pair separations are exact fixed-point integers (x_j - x_i - image shift,
// 32-bit wrap-around); r^2 and r^2 - r0^2 are exact in 64-bit integers and
// rounded once to float, so s = r/r0 - 1 = (r^2 - r0^2) / (r0 (r + r0)) keeps
// ~1e-7 relative accuracy even for nearest neighbours, where FP32 rounding
// of r itself would shift distances by ~1e-7 A.  The exponentials, taper,
// embedding and pair forces are FP32; per-atom sums are Kahan-compensated;
// forces, positions, energies and all reductions stay FP64.

__device__ __forceinline__ void fill_qshift_table(int3* tbl, const GeoC& g) {
    for (int t = threadIdx.x; t < 125; t += blockDim.x) {
        const int sx = t % 5 - 2, sy = (t / 5) % 5 - 2, sz = t / 25 - 2;
        tbl[t] = make_int3((int)((unsigned)sx * (unsigned)g.Lq[0]),
                           (int)((unsigned)sy * (unsigned)g.Lq[1]),
                           (int)((unsigned)sz * (unsigned)g.Lq[2]));
    }
}

// Fixed-point separation of list slot e from atom i; returns r^2 in
// (fixed-point unit)^2.
__device__ __forceinline__ long long pair_sep_q(const Bufs& b, const int3* qt, int4 qi,
                                                uint32_t e, int& dx, int& dy, int& dz, int& j) {
    j = (int)(e & kIdxMask);
    const int code = (int)(e >> kIdxBits);
    const int4 qj = b.xq[j];
    dx = wrap_sub(qj.x, qi.x);
    dy = wrap_sub(qj.y, qi.y);
    dz = wrap_sub(qj.z, qi.z);
    if (code != kCodeZero) {
        const int3 s = qt[code];
        dx = wrap_sub(dx, s.x);
        dy = wrap_sub(dy, s.y);
        dz = wrap_sub(dz, s.z);
    }
    return (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
}

// ---------------------------------------------------------------------------
// Per-atom part of the FP64 reductions of (F, v) (see k_reduce_ctl), shared
// by k_reduce_ctl and the NEB projection.

// Row of the partials that holds the k-th sum of warp_sum4 (P, |F|^2, |v|^2,
// energy); rows 3 and 4 hold the maxima of |F_i|^2 and |F_i,d|.
__device__ __forceinline__ int red_row(int k) { return k == 3 ? 5 : k; }

struct RedAcc {
    double P = 0.0, F2 = 0.0, V2 = 0.0, fa2 = 0.0, fin = 0.0;
    double E = 0.0;   // the block's slice of the energy partials (k_reduce_ctl)
};

// Zeroes the frozen components of f (if any); true when f changed.
__device__ __forceinline__ bool mask_force(const Bufs& b, int i, dvec4& f) {
    if (!b.dofmask) return false;
    const unsigned m = b.dofmask[i];
    if (m & 1u) f.x = 0.0;
    if (m & 2u) f.y = 0.0;
    if (m & 4u) f.z = 0.0;
    return m != 0u;
}

// Reductions of atom i's (F, v); f must be masked already.
__device__ __forceinline__ void red_atom(const Bufs& b, int i, const dvec4& f, dvec4 v,
                                         double vv_half, RedAcc& a) {
    if (vv_half != 0.0) {   // second half kick of velocity Verlet, with the new force
        v.x += vv_half * f.x;
        v.y += vv_half * f.y;
        v.z += vv_half * f.z;
        b.v[i] = v;
    }
    // FP64 arithmetic runs at 1/58 of the FP32 rate on this part and bounds
    // this pass: the sums P and |v|^2 chain their products into the running
    // sum (3 FMAs each), and the maxima of non-negative values compare the
    // IEEE bit patterns as integers, which order the same way
    a.P = fma(f.z, v.z, fma(f.y, v.y, fma(f.x, v.x, a.P)));
    const double q = fma(f.z, f.z, fma(f.y, f.y, f.x * f.x));
    a.F2 += q;
    a.V2 = fma(v.z, v.z, fma(v.y, v.y, fma(v.x, v.x, a.V2)));
    a.fa2 = max_nonneg(a.fa2, q);
    a.fin = max_nonneg(a.fin, max_nonneg(abs_bits(f.x), max_nonneg(abs_bits(f.y), abs_bits(f.z))));
}

// Reductions of the atoms of this thread (grid-stride), with the frozen-DOF
// mask applied; VV: velocity Verlet's second half kick first.
template <bool VV>
__device__ __forceinline__ void red_range(const Bufs& b, double vvh, RedAcc& acc) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < b.n; i += gridDim.x * blockDim.x) {
        dvec4 f = f_load(b, i);
        if (mask_force(b, i, f)) f_store(b, i, f.x, f.y, f.z);
        red_atom(b, i, f, b.v[i], VV ? vvh : 0.0, acc);
    }
}

// The block's six reductions written to the partials (kRedRows rows of
// gridDim.x): sums of P, |F|^2, |v|^2 and of the block's energy terms
// (warp_sum4), maxima of |F_i|^2 and |F_i,d| (integer maxima); per warp,
// then over the warps in warp 0, in a fixed order.  sh holds kRedRows x 32
// doubles.
// Row k goes to out[k * stride]: the global partials (red_write), or one row
// in shared memory (stride 1) when a single block reduces every atom.
__device__ __forceinline__ void red_write_to(const RedAcc& a, double* sh, double* out, int stride) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double s = warp_sum4(a.P, a.F2, a.V2, a.E);
    double m0 = warp_max_nonneg(a.fa2), m1 = warp_max_nonneg(a.fin);
    __syncthreads();   // sh may hold an earlier use
    if ((lane & 7) == 0) sh[red_row(lane >> 3) * 32 + w] = s;   // lanes 0, 8, 16, 24
    if (lane == 0) {
        sh[3 * 32 + w] = m0;
        sh[4 * 32 + w] = m1;
    }
    __syncthreads();
    if (w == 0) {
        const bool in = lane < (int)(blockDim.x >> 5);
        s = warp_sum4(in ? sh[lane] : 0.0, in ? sh[32 + lane] : 0.0, in ? sh[2 * 32 + lane] : 0.0,
                      in ? sh[5 * 32 + lane] : 0.0);
        m0 = warp_max_nonneg(in ? sh[3 * 32 + lane] : 0.0);
        m1 = warp_max_nonneg(in ? sh[4 * 32 + lane] : 0.0);
        if ((lane & 7) == 0) out[red_row(lane >> 3) * stride] = s;
        if (lane == 0) {
            out[3 * stride] = m0;
            out[4 * stride] = m1;
        }
    }
}
__device__ __forceinline__ void red_write(const RedAcc& a, double* sh, double* rpart) {
    red_write_to(a, sh, rpart + blockIdx.x, gridDim.x);
}

__device__ __forceinline__ double vv_half_of(const DevState* st) {
    return st->fs.vv ? st->fs.vv_half : 0.0;
}

// Pass 1 (FP32-pair): rho_i, F'(rho_i) = -1/(2 sqrt(rho_i)) and the atom's
// energy sum_j phi - sqrt(rho_i); the full list makes rho_i complete in one
// group of TPA threads (lane sums added in FP64), so the embedding step is
// fused here.
template <int TPA = 1>
__global__ void __launch_bounds__(kForceBlock) k_density32(Bufs b, PotC P, GeoC g) {
    __shared__ int3 qt[125];
    __shared__ float et[kExp32TableSize];
    __shared__ double red[32];
    if (pass_skipped(b)) return;
    fill_qshift_table(qt, g);
    for (int t = threadIdx.x; t < kExp32TableSize; t += blockDim.x) et[t] = b.exp32_table[t];
    __syncthreads();
    double e_atom = 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t / TPA < b.n;
         t += gridDim.x * blockDim.x) {
        const int i = t / TPA, lane = t % TPA;
        const int4 qi = b.xq[i];
        const int m = b.nnbr[i];
        Kahan32 rho, erep;
        for (int k = lane; k < m; k += TPA) {
            int dx, dy, dz, j;
            const long long r2q = pair_sep_q(b, qt, qi, b.nbr[(size_t)k * b.n + i], dx, dy, dz, j);
            if (r2q >= P.rc2q) continue;
            float rinv, phi, dphi, gg, dg;
            rgl_pair32(P, r2q, et, rinv, phi, dphi, gg, dg);
            rho.add(gg);
            erep.add(phi);
        }
        const double rho_d = group_sum<TPA>(rho.value());
        const double erep_d = group_sum<TPA>(erep.value());
        if (lane != 0) continue;
        const float rf = (float)rho_d;
        const float sq = sqrtf(rf);
        b.fp32[i] = rf > 0.f ? -0.5f / sq : 0.f;
        b.rho[i] = rho_d;
        const double ei = erep_d - (double)sq;
        if (b.eatom) b.eatom[i] = ei;
        e_atom += ei;
    }
    const double bs = block_sum(e_atom, red);
    if (threadIdx.x == 0) b.epart[blockIdx.x] = bs;
}

// Pass 2 (FP32-pair): F_i = sum_j [2 phi' + (F'_i + F'_j) g'] (x_j - x_i) / r,
// Kahan-compensated per component, written as FP64 (no atomics); TPA
// threads per atom as in k_density32.
template <int TPA, int BLK>
__global__ void __launch_bounds__(BLK) k_force32(Bufs b, PotC P, GeoC g) {
    __shared__ int3 qt[125];
    __shared__ float et[kExp32TableSize];
    if (pass_skipped(b)) return;
    fill_qshift_table(qt, g);
    for (int t = threadIdx.x; t < kExp32TableSize; t += blockDim.x) et[t] = b.exp32_table[t];
    __syncthreads();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t / TPA < b.n;
         t += gridDim.x * blockDim.x) {
        const int i = t / TPA, lane = t % TPA;
        const int4 qi = b.xq[i];
        const float fpi = b.fp32[i];
        const int m = b.nnbr[i];
        Kahan32 fx, fy, fz;
        for (int k = lane; k < m; k += TPA) {
            int dx, dy, dz, j;
            const long long r2q = pair_sep_q(b, qt, qi, b.nbr[(size_t)k * b.n + i], dx, dy, dz, j);
            if (r2q >= P.rc2q) continue;
            float rinv, phi, dphi, gg, dg;
            rgl_pair32(P, r2q, et, rinv, phi, dphi, gg, dg);
            const float fs = (2.f * dphi + (fpi + b.fp32[j]) * dg) * rinv * P.qinv;
            fx.add(fs * (float)dx);
            fy.add(fs * (float)dy);
            fz.add(fs * (float)dz);
        }
        const double sx = group_sum<TPA>(fx.value());
        const double sy = group_sum<TPA>(fy.value());
        const double sz = group_sum<TPA>(fz.value());
        if (lane != 0) continue;
        dvec4 f = make_dvec4(sx, sy, sz, 0.0);
        mask_force(b, i, f);
        f_store(b, i, f.x, f.y, f.z);
    }
}

// ---------------------------------------------------------------------------
// Tabulated RGL passes (quintic Hermite tables in u = r^2 - r0^2, held in
// shared memory; persistent grids stride over the atoms so each block loads
// the table once).  Pairs closer than r0/2 fall back to the analytic terms.

template <typename T>
__device__ __forceinline__ void load_table(T* dst, const T* src, int count) {
    for (int t = threadIdx.x; t < count; t += blockDim.x) dst[t] = src[t];
}

// ---------------------------------------------------------------------------
// FP64 form, tabulated RGL on the full list with no FP64 instruction per
// pair (fire2_table.cuh): exact fixed-point separations, double-float r^2,
// interval offsets, quintics and per-atom sums.  One atom per thread, no
// atomics: every atom's sums are complete in its own thread.

__device__ __forceinline__ void fill_qshift64_table(long long* qt, const GeoC& g) {
    for (int t = threadIdx.x; t < 125; t += blockDim.x) {
        const int sx = t % 5 - 2, sy = (t / 5) % 5 - 2, sz = t / 25 - 2;
        qt[3 * t] = sx * g.Lq64[0];
        qt[3 * t + 1] = sy * g.Lq64[1];
        qt[3 * t + 2] = sz * g.Lq64[2];
    }
}

// Separation x_j - x_i - shift of list slot e (atom j at fixed-point position
// qj) as float pairs (exact), and r^2.
__device__ __forceinline__ ffloat pair_sep_ff_q(const long long* qt, const lvec4& qi,
                                                const lvec4& qj, uint32_t e, ffloat& dx,
                                                ffloat& dy, ffloat& dz, int& j) {
    j = (int)(e & kIdxMask);
    const int code = (int)(e >> kIdxBits);
    long long ix = qj.x - qi.x, iy = qj.y - qi.y, iz = qj.z - qi.z;
    if (code != kCodeZero) {
        ix -= qt[3 * code];
        iy -= qt[3 * code + 1];
        iz -= qt[3 * code + 2];
    }
    dx = fixed_to_ff(ix);
    dy = fixed_to_ff(iy);
    dz = fixed_to_ff(iz);
    return ff_norm2(dx, dy, dz);
}

// The same, loading atom j's position.
__device__ __forceinline__ ffloat pair_sep_ff(const Bufs& b, const long long* qt, const lvec4& qi,
                                              uint32_t e, ffloat& dx, ffloat& dy, ffloat& dz,
                                              int& j) {
    return pair_sep_ff_q(qt, qi, b.xq64[e & kIdxMask], e, dx, dy, dz, j);
}

// Pass 1.  Full list (HALF = false): rho_i, F'(rho_i) (FP64 per atom) and the
// atom's energy sum_j phi - sqrt(rho_i), all in the atom's thread.  Half
// list (HALF = true): rho_i and rho_j (FP64 atomics), 2 phi per pair credited
// to i; k_embed then forms F'(rho) and the embedding energy.  Pairs
// compressed below r0/2 fall back to the FP64 exponentials.  TPA threads
// share an atom: lane l takes list slots l, l + TPA, ..., and the lanes'
// sums are added in FP64 (group_sum) before lane 0 finishes the atom.
template <bool HALF, int TPA>
__device__ __forceinline__ void density_ff_body(const Bufs& b, const PotC& P, const GeoC& g) {
    __shared__ long long qt[375];
    __shared__ double red[32];
    // the exponentials' table is read through L1: only pairs compressed below
    // r0/2 use it, and a shared copy per block costs more than it saves
    const double* etab = b.exp_table;
    if (pass_skipped(b)) return;
    fill_qshift64_table(qt, g);
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / TPA, lane = t % TPA;
    double e_atom = 0.0;
    if (i < b.n) {
        const lvec4 qi = b.xq64[i];
        const int m = b.nnbr[i];
        ffloat rho = {0.f, 0.f}, erep = {0.f, 0.f};
        for (int k = lane; k < m; k += TPA) {
            ffloat dx, dy, dz;
            int j;
            const ffloat r2 = pair_sep_ff(b, qt, qi, b.nbr[(size_t)k * b.n + i], dx, dy, dz, j);
            if (!(r2.hi < P.rc2_f)) continue;
            const float uf = r2.hi - P.r0sq_f;
            if (uf >= P.tab.u_lo_f) {
                float row[kFFRow];
                load_row(b.tab_ffd, ff_index(P.tab, uf), row);
                ffloat v[2];
                ff_row_eval(row, r2, v);
                erep = ff_acc(erep, v[0]);   // doubled at the end on the half list
                rho = ff_acc(rho, v[1]);
                if (HALF) atomicAdd(&b.rho[j], ff_to_f64(v[1]));
            } else {
                double rinv, phi, dphi, gg, dg;
                rgl_pair64(P, ff_to_f64(r2), etab, rinv, phi, dphi, gg, dg);
                erep = ff_acc(erep, f64_to_ff(phi));
                rho = ff_acc(rho, f64_to_ff(gg));
                if (HALF) atomicAdd(&b.rho[j], gg);
            }
        }
        const double rho_d = group_sum<TPA>(ff_to_f64(rho));
        const double erep_d = group_sum<TPA>(ff_to_f64(erep));
        if (lane == 0 && HALF) {
            atomicAdd(&b.rho[i], rho_d);
            e_atom = 2.0 * erep_d;   // each pair's 2 phi credited to i
            if (b.eatom) b.eatom[i] = e_atom;
        } else if (lane == 0) {
            double sq, fp;
            ffloat fpf;
            rgl_embed_dd(rho_d, sq, fp, fpf);
            b.rho[i] = rho_d;
            b.fp[i] = fp;
            fp_store(b, i, fpf);
            e_atom = erep_d - sq;
            if (b.eatom) b.eatom[i] = e_atom;
        }
    }
    const double s = block_sum(e_atom, red);
    if (threadIdx.x == 0) b.epart[blockIdx.x] = s;
}

template <bool HALF, int TPA = 1>
__global__ void __launch_bounds__(kForceBlock) k_density_ff(Bufs b, PotC P, GeoC g) {
    density_ff_body<HALF, TPA>(b, P, g);
}

// The same pass with one thread per atom (large systems) on blocks of 512,
// 3 per SM (40 registers; with the compiler's 44 it fits fewer threads and
// ran 4 % slower).  (The force pass keeps the compiler's 64: capped at 56 or
// 48 it spills and takes 0.51 and 0.69 against 0.48 ms.)
template <bool HALF>
__global__ void __launch_bounds__(kDensFF1Block, 3) k_density_ff1(Bufs b, PotC P, GeoC g) {
    density_ff_body<HALF, 1>(b, P, g);
}

// Pass 2: F_i = sum_j [2 phi'/r + (F'_i + F'_j) g'/r] (x_j - x_i) (F = -grad E,
// Sec. 2.1); full list: written whole; half list: F_i and F_j by FP64 atomics.
// TPA threads per atom as in k_density_ff; blocks of BLK threads (the pass
// writes no per-block partials, so its grid is free: force_ff picks it).
template <bool HALF, int TPA, int BLK>
__global__ void __launch_bounds__(BLK) k_force_ff(Bufs b, PotC P, GeoC g) {
    __shared__ long long qt[375];
    const double* etab = b.exp_table;   // through L1, as in the density pass
    if (pass_skipped(b)) return;
    fill_qshift64_table(qt, g);
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / TPA, lane = t % TPA;
    if (i >= b.n) return;   // the whole group leaves
    const lvec4 qi = b.xq64[i];
    const ffloat fpi = fp_load(qi);
    const int m = b.nnbr[i];
    ffloat fx = {0.f, 0.f}, fy = {0.f, 0.f}, fz = {0.f, 0.f};
    // software pipeline: the next list entry and its atom's record (position
    // and F') load while this pair is evaluated
    uint32_t e_nx = lane < m ? b.nbr[(size_t)lane * b.n + i] : 0u;
    lvec4 q_nx = b.xq64[lane < m ? (int)(e_nx & kIdxMask) : i];
    for (int k = lane; k < m; k += TPA) {
        const uint32_t e = e_nx;
        const lvec4 qj = q_nx;
        if (k + TPA < m) {
            e_nx = b.nbr[(size_t)(k + TPA) * b.n + i];
            q_nx = b.xq64[e_nx & kIdxMask];
        }
        ffloat dx, dy, dz;
        int j;
        const ffloat r2 = pair_sep_ff_q(qt, qi, qj, e, dx, dy, dz, j);
        if (!(r2.hi < P.rc2_f)) continue;
        const float uf = r2.hi - P.r0sq_f;
        ffloat c[2];
        if (uf >= P.tab.u_lo_f) {
            float row[kFFRow];
            load_row(b.tab_fff, ff_index(P.tab, uf), row);
            ff_row_eval(row, r2, c);
        } else {
            double rinv, phi, dphi, gg, dg;
            rgl_pair64(P, ff_to_f64(r2), etab, rinv, phi, dphi, gg, dg);
            c[0] = f64_to_ff(2.0 * dphi * rinv);
            c[1] = f64_to_ff(dg * rinv);
        }
        const ffloat fs = ff_madd(ff_add(fpi, fp_load(qj)), c[1], c[0]);
        // unnormalised products: ff_acc and ff_to_f64 take any pair
        const ffloat tx = ff_mul_nn(fs, dx), ty = ff_mul_nn(fs, dy), tz = ff_mul_nn(fs, dz);
        fx = ff_acc(fx, tx);
        fy = ff_acc(fy, ty);
        fz = ff_acc(fz, tz);
        if (HALF) {
            f_add(b, j, -ff_to_f64(tx), -ff_to_f64(ty), -ff_to_f64(tz));
        }
    }
    const double sx = group_sum<TPA>(ff_to_f64(fx));
    const double sy = group_sum<TPA>(ff_to_f64(fy));
    const double sz = group_sum<TPA>(ff_to_f64(fz));
    if (lane != 0) return;
    if (HALF) {   // k_reduce_ctl applies the frozen-DOF mask
        f_add(b, i, sx, sy, sz);
    } else {
        dvec4 f = make_dvec4(sx, sy, sz, 0.0);
        mask_force(b, i, f);
        f_store(b, i, f.x, f.y, f.z);
    }
}

// FP32-pair pass 1 (full list, tables): u = r^2 - r0^2 exact in fixed point,
// rounded once to float.
__global__ void __launch_bounds__(kTabBlock) k_density32_tab(Bufs b, PotC P, GeoC g) {
    extern __shared__ float tabd32[];
    __shared__ int3 qt[125];
    __shared__ float et[kExp32TableSize];
    __shared__ double red[32];
    if (pass_skipped(b)) return;
    fill_qshift_table(qt, g);
    load_table(tabd32, b.tab_d32, (P.tab32.nA + P.tab32.nB) * kTabDens);
    load_table(et, b.exp32_table, kExp32TableSize);
    __syncthreads();
    double e_sum = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < b.n; i += gridDim.x * blockDim.x) {
        const int4 qi = b.xq[i];
        const int m = b.nnbr[i];
        Kahan32 rho, erep;
        for (int k = 0; k < m; ++k) {
            int dx, dy, dz, j;
            const long long r2q = pair_sep_q(b, qt, qi, b.nbr[(size_t)k * b.n + i], dx, dy, dz, j);
            if (r2q >= P.rc2q) continue;
            int ki;
            float t, phi, gg;
            if (tab_locate_f(P.tab32, ll_to_float(r2q - P.r0sq_q) * P.qinv2, ki, t)) {
                const float* c = tabd32 + ki * kTabDens;
                phi = poly5(c, t);
                gg = poly5(c + 6, t);
            } else {
                float rinv, dphi, dg;
                rgl_pair32(P, r2q, et, rinv, phi, dphi, gg, dg);
            }
            rho.add(gg);
            erep.add(phi);
        }
        const double rho_d = rho.value();
        const float rf = (float)rho_d;
        const float sq = sqrtf(rf);
        b.fp32[i] = rf > 0.f ? -0.5f / sq : 0.f;
        b.rho[i] = rho_d;
        const double ei = erep.value() - (double)sq;
        if (b.eatom) b.eatom[i] = ei;
        e_sum += ei;
    }
    const double bs = block_sum(e_sum, red);
    if (threadIdx.x == 0) b.epart[blockIdx.x] = bs;
}

// FP32-pair pass 2 (full list, tables): F_i = sum_j fs d, Kahan per component.
__global__ void __launch_bounds__(kTabBlock) k_force32_tab(Bufs b, PotC P, GeoC g) {
    extern __shared__ float tabf32[];
    __shared__ int3 qt[125];
    __shared__ float et[kExp32TableSize];
    if (pass_skipped(b)) return;
    fill_qshift_table(qt, g);
    load_table(tabf32, b.tab_f32, (P.tab32.nA + P.tab32.nB) * kTabForce);
    load_table(et, b.exp32_table, kExp32TableSize);
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < b.n; i += gridDim.x * blockDim.x) {
        const int4 qi = b.xq[i];
        const float fpi = b.fp32[i];
        const int m = b.nnbr[i];
        Kahan32 fx, fy, fz;
        for (int k = 0; k < m; ++k) {
            int dx, dy, dz, j;
            const long long r2q = pair_sep_q(b, qt, qi, b.nbr[(size_t)k * b.n + i], dx, dy, dz, j);
            if (r2q >= P.rc2q) continue;
            int ki;
            float t, phiu, gu;
            if (tab_locate_f(P.tab32, ll_to_float(r2q - P.r0sq_q) * P.qinv2, ki, t)) {
                const float* c = tabf32 + ki * kTabForce;
                phiu = poly5(c, t);
                gu = poly5(c + 6, t);
            } else {
                float rinv, phi, dphi, gg, dg;
                rgl_pair32(P, r2q, et, rinv, phi, dphi, gg, dg);
                phiu = 0.5f * dphi * rinv;
                gu = 0.5f * dg * rinv;
            }
            const float fs = 2.f * (2.f * phiu + (fpi + b.fp32[j]) * gu) * P.qinv;
            fx.add(fs * (float)dx);
            fy.add(fs * (float)dy);
            fz.add(fs * (float)dz);
        }
        dvec4 f = make_dvec4(fx.value(), fy.value(), fz.value(), 0.0);
        mask_force(b, i, f);
        f_store(b, i, f.x, f.y, f.z);
    }
}

// ---------------------------------------------------------------------------
// FP64 reductions of the current (F, v): P = F.v, |F|^2, |v|^2 (Alg. 2 and
// the mixing of Algs. 3-6) and the per-atom / per-component force maxima
// (Sec. 3.4); for velocity Verlet first the second half kick (Alg. 6).  They
// run in k_reduce_ctl (below), whose last block also runs the control step.

// Fixed-order final reductions of the partials by one block (deterministic):
// the sums of P, |F|^2, |v|^2 and E and the maxima of |F_i|^2 and |F_i,d|,
// all six in one sweep so that their loads are in flight together.  Each
// quantity is added up in the order of a block_sum / block_max of its own.
// The energy is the sum of the partials' energy row plus, when ne > 0, the
// first ne energy partials of the passes (epart; the NEB chain leaves its
// energy there, k_reduce_ctl has already folded it into the rows).
struct CtlSums {
    double P, F2, V2, fa2, fin, E;
};
__device__ __forceinline__ CtlSums ctl_reduce(const Bufs& b, int ne, double* sh /* 6 x 32 */) {
    double a[kRedRows] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const int nr = b.nb_red;
    // unrolled so that a thread's loads are in flight together
#pragma unroll 4
    for (int k = threadIdx.x; k < nr; k += blockDim.x) {
        a[0] += b.rpart[k];
        a[1] += b.rpart[nr + k];
        a[2] += b.rpart[2 * nr + k];
        a[3] = max_nonneg(a[3], b.rpart[3 * nr + k]);
        a[4] = max_nonneg(a[4], b.rpart[4 * nr + k]);
        a[5] += b.rpart[5 * nr + k];
    }
    if (ne > 0) {   // four independent sums per thread, so that its loads overlap
        const int bd = blockDim.x;
        double e0 = 0.0, e1 = 0.0, e2 = 0.0, e3 = 0.0;
        int k = threadIdx.x;
        for (; k + 3 * bd < ne; k += 4 * bd) {
            e0 += b.epart[k];
            e1 += b.epart[k + bd];
            e2 += b.epart[k + 2 * bd];
            e3 += b.epart[k + 3 * bd];
        }
        for (; k < ne; k += bd) e0 += b.epart[k];
        a[5] += (e0 + e1) + (e2 + e3);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double t = warp_sum4(a[0], a[1], a[2], a[5]);
    double m0 = warp_max_nonneg(a[3]), m1 = warp_max_nonneg(a[4]);
    if ((lane & 7) == 0) sh[red_row(lane >> 3) * 32 + w] = t;
    if (lane == 0) {
        sh[3 * 32 + w] = m0;
        sh[4 * 32 + w] = m1;
    }
    __syncthreads();
    if (w == 0) {
        const bool in = lane < (int)(blockDim.x >> 5);
        t = warp_sum4(in ? sh[lane] : 0.0, in ? sh[32 + lane] : 0.0, in ? sh[2 * 32 + lane] : 0.0,
                      in ? sh[5 * 32 + lane] : 0.0);
        m0 = warp_max_nonneg(in ? sh[3 * 32 + lane] : 0.0);
        m1 = warp_max_nonneg(in ? sh[4 * 32 + lane] : 0.0);
        // the four sums sit in lanes 0, 8, 16, 24: gather them in lane 0
        a[0] = t;
        a[1] = __shfl_sync(0xffffffffu, t, 8);
        a[2] = __shfl_sync(0xffffffffu, t, 16);
        a[5] = __shfl_sync(0xffffffffu, t, 24);
        a[3] = m0;
        a[4] = m1;
    }
    return {a[0], a[1], a[2], a[3], a[4], a[5]};   // valid in thread 0
}

// The number of energy partials the passes of this evaluation wrote: the
// FP64 confirming passes' while an FP32-pair stop is confirmed, else the
// density (or only) pass's and the embedding's.
__device__ __forceinline__ int energy_partials(const Bufs& b) {
    return b.st->vstate >= 2 ? b.nb_verify : b.ne_dens + b.nb_embed;
}

// Scalar FIRE 2.0 control (Algorithm 2, fire_control_step) on the final
// sums r, by one thread: the error checks, then the convergence test and the
// preparation of the next iteration; sets the WHILE condition.
__device__ void control_apply(const Bufs& b, int mode, cudaGraphConditionalHandle h,
                              int has_handle, const CtlSums& r) {
    const double P = r.P, F2 = r.F2, V2 = r.V2, fa2 = r.fa2, fin = r.fin, E = r.E;
    DevState& s = *b.st;
    s.P = P;
    s.F2 = F2;
    s.V2 = V2;
    s.fmax2 = fa2;
    s.finf = fin;
    s.energy = E;
    s.max_disp2 = 0ull;
    s.vmax2 = 0ull;
    if (mode == CTL_EVAL) {
        if ((!isfinite(E) || !isfinite(F2)) && s.status == ST_OK) s.status = ST_NONFINITE;
        return;
    }
    bool stop = false;
    if (s.status != ST_OK) {
        s.fs.evals += 1;
        stop = true;
    } else if (!isfinite(E) || !isfinite(F2) || !isfinite(V2)) {
        s.fs.evals += 1;
        s.status = ST_NONFINITE;
        stop = true;
    } else if (s.budget_ns && globaltimer_ns() - s.t_start > s.budget_ns) {
        s.fs.evals += 1;
        s.status = ST_TIMEOUT;
        stop = true;
    } else if (s.vstate == 2) {
        // this evaluation used FP64 forces at the configuration where the
        // FP32-pair forces met the threshold
        const double fn = force_norm(s.prm.norm, F2, fa2, fin);
        if (fn < s.ftol_user) {
            s.fs.evals += 1;
            s.fs.stop = STOP_FTOL;
            stop = true;
        } else if (s.vmode == 2) {   // finish in FP64 from here
            s.prm.ftol = s.ftol_user;
            s.vstate = 3;
            stop = fire_control_step(s.prm, s.fs, P, F2, V2, fa2, fin);
        } else {
            // not converged in FP64: tighten the FP32 threshold by the FP32 to
            // FP64 difference seen here and take the step with these forces
            s.prm.ftol = fmax(s.prm.ftol - 1.5 * (fn - s.fn32), 0.4 * s.ftol_user);
            s.vstate = 1;
            stop = fire_control_step(s.prm, s.fs, P, F2, V2, fa2, fin);
        }
    } else {
        stop = fire_control_step(s.prm, s.fs, P, F2, V2, fa2, fin);
        if (stop && s.vstate == 1 && s.fs.stop == STOP_FTOL && s.status == ST_OK) {
            s.fn32 = force_norm(s.prm.norm, F2, fa2, fin);
            s.vstate = 2;
            s.vcount += 1;
            stop = false;
        } else if (!stop && s.vstate == 1 && s.vmode == 2 &&
                   force_norm(s.prm.norm, F2, fa2, fin) < s.fsw) {
            s.vstate = 3;   // the FP32-pair forces have done their part: FP64 from the next
        }
    }
    s.done = stop ? 1 : 0;
    if (has_handle) cudaGraphSetConditional(h, stop ? 0u : 1u);
}

// The control step of one block: every thread enters (the fixed-order final
// reductions of the partials), thread 0 runs the scalar part.
__device__ void control_body(const Bufs& b, int mode, cudaGraphConditionalHandle h,
                             int has_handle, double* sh, int ne) {
    const CtlSums r = ctl_reduce(b, ne, sh);
    if (threadIdx.x == 0) control_apply(b, mode, h, has_handle, r);
}

// The reductions of (F, v) and the control step in one launch (nb_red
// blocks): every block writes its partials, and the last
// block to finish (a ticket counter, reset by that block) runs the control
// step on all of them.  No block waits for another.
__global__ void k_reduce_ctl(Bufs b, int mode, cudaGraphConditionalHandle h, int has_handle) {
    __shared__ double sh[kRedRows * 32];
    __shared__ int last;
    if (b.st->done) {   // chunked loop bodies past the stop
        if (mode == CTL_LOOP && has_handle && blockIdx.x == 0 && threadIdx.x == 0)
            cudaGraphSetConditional(h, 0u);
        return;
    }
    const double vvh = vv_half_of(b.st);
    RedAcc acc;
    {   // this block's slice of the passes' energy partials, in a fixed order
        const int ne = energy_partials(b), per = (ne + gridDim.x - 1) / gridDim.x;
        const int e1 = min(ne, (int)(blockIdx.x + 1) * per);
        for (int k = blockIdx.x * per + threadIdx.x; k < e1; k += blockDim.x) acc.E += b.epart[k];
    }
    // the velocity-Verlet test outside the loop: an FP64 comparison per atom
    // costs as much as a multiply-add on the FP64 pipe, which bounds this pass
    if (vvh != 0.0)
        red_range<true>(b, vvh, acc);
    else
        red_range<false>(b, 0.0, acc);
    if (gridDim.x == 1) {
        // one block (a few hundred atoms): its sums are the final ones, and
        // the round trip of the partials, the ticket and the second tree of
        // ctl_reduce (several microseconds of latency) are left out
        __shared__ double row[kRedRows];
        red_write_to(acc, sh, row, 1);
        __syncthreads();
        if (threadIdx.x == 0)
            control_apply(b, mode, h, has_handle, {row[0], row[1], row[2], row[3], row[4], row[5]});
        return;
    }
    red_write(acc, sh, b.rpart);
    if (threadIdx.x == 0) {
        __threadfence();   // this block's partials before its ticket
        last = atomicAdd(&b.st->red_blocks, 1u) == gridDim.x - 1 ? 1 : 0;
    }
    __syncthreads();
    if (!last) return;
    if (threadIdx.x == 0) b.st->red_blocks = 0u;
    __threadfence();       // every other block's partials are visible from here
    control_body(b, mode, h, has_handle, sh, 0);
}

// The element-wise step over this thread's atoms (grid-stride); returns the
// largest squared displacement since the last list build, in FP32: x
// truncated against the copy rounded at the build, off by < 2 FP32 ulps of
// the coordinate, far inside the list radius's margin (1e-3 rc + 8 FP32 ulps
// of the box).  KICK: explicit Euler's kick after the drift.
template <bool KICK>
__device__ __forceinline__ float update_range(const Bufs& b, const FireScal& s, double dt,
                                              int after_pre) {
    float d2max = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < b.n; i += gridDim.x * blockDim.x) {
        dvec4 x = b.x[i], v = b.v[i];
        const dvec4 f = f_load(b, i);
        const float4 r = b.xf[i];    // x at the last build; loaded before the stores
        if (!after_pre) fire_update_pre(s, x, v, f);
        fire_update_drift_k<KICK>(s, dt, x, v, f);
        b.x[i] = x;
        if (b.xq)
            b.xq[i] = make_int4(to_fixed(x.x, b.qscale), to_fixed(x.y, b.qscale),
                                to_fixed(x.z, b.qscale), 0);
        if (b.xq64)
            b.xq64[i] = {to_fixed64(x.x, kFixedBits64), to_fixed64(x.y, kFixedBits64),
                         to_fixed64(x.z, kFixedBits64), 0ll};
        b.v[i] = v;
        if (b.accum) {
            f_store(b, i, 0.0, 0.0, 0.0);
            if (b.rho) b.rho[i] = 0.0;
        }
        const float ddx = f64_to_f32_trunc(x.x) - r.x;
        const float ddy = f64_to_f32_trunc(x.y) - r.y;
        const float ddz = f64_to_f32_trunc(x.z) - r.z;
        d2max = fmaxf(d2max, ddx * ddx + ddy * ddy + ddz * ddz);
    }
    return d2max;
}

// Element-wise part of one iteration: optional half step back and v = 0
// (P <= 0, Alg. 2), then Algorithm 4: v += dt F / m, mixing
// v = (1 - alpha) v + alpha |v| F / |F| (P > 0), x += dt v.  Clears F and rho
// for the next force evaluation (accumulating paths) and tracks
// max |x - x_ref|^2.  With has_if, the last block to finish sets the graph's
// IF condition to "the neighbour list must be rebuilt" (see need_rebuild).
// The element-wise step of k_update, given the state the control
// step left (s, done, vstate) and the drift dt.
__device__ void update_body(const Bufs& b, const GeoC& g, const FireScal& s, int done, int vstate,
                            double dt, int after_pre, cudaGraphConditionalHandle hif, int has_if,
                            cudaGraphConditionalHandle hconf, int has_conf, double* red) {
    // graph loop: the IF node of the FP64 confirming passes runs this pass
    // only when an FP32-pair stop is being confirmed
    if (has_conf && blockIdx.x == 0 && threadIdx.x == 0)
        cudaGraphSetConditional(hconf, vstate >= 2 ? 1u : 0u);
    // no step when stopped, nor while an FP32-pair stop is confirmed in FP64
    // (the next evaluation is at the same positions)
    if (done || vstate == 2) {
        if (has_if && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(hif, 0u);
        return;
    }
    // the explicit-Euler test once per pass (an FP64 comparison per atom would
    // cost the FP64 pipe as much as a multiply-add)
    const float d2max = s.kick_after != 0.0 ? update_range<true>(b, s, dt, after_pre)
                                            : update_range<false>(b, s, dt, after_pre);
    const double bm = block_max_nonneg(f32_to_f64(d2max), red);
    if (threadIdx.x == 0) {
        atomicMax(&b.st->max_disp2, (unsigned long long)__double_as_longlong(bm));
        if (has_if) {
            __threadfence();
            if (atomicAdd(&b.st->upd_blocks, 1u) == gridDim.x - 1) {
                b.st->upd_blocks = 0u;
                const unsigned long long d = atomicAdd(&b.st->max_disp2, 0ull);
                const bool rebuild = __longlong_as_double((long long)d) > g.half_skin2;
                cudaGraphSetConditional(hif, rebuild ? 1u : 0u);
            }
        }
    }
}

__global__ void k_update(Bufs b, GeoC g, cudaGraphConditionalHandle hif, int has_if,
                         int after_pre, cudaGraphConditionalHandle hconf, int has_conf) {
    __shared__ double red[32];
    const FireScal s = b.st->fs;
    // after k_update_pre: only the drift is left, with the capped dt
    const double dt = after_pre ? fire_capped_dt(s.dt_cur, b.st->prm.dmax,
                                                 __longlong_as_double((long long)b.st->vmax2))
                                : s.dt_cur;
    update_body(b, g, s, b.st->done, b.st->vstate, dt, after_pre, hif, has_if, hconf, has_conf,
                red);
}

// With a maximum displacement per step (dmax > 0) the element-wise step runs
// in two passes: this one applies everything before the drift and takes
// max_i |v_i|^2 of the drift velocity; k_update(after_pre = 1) then drifts
// with fire_capped_dt.
__global__ void k_update_pre(Bufs b) {
    __shared__ double red[32];
    if (b.st->done || b.st->vstate == 2) return;   // no step while confirming
    const FireScal s = b.st->fs;
    double vm = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < b.n; i += gridDim.x * blockDim.x) {
        dvec4 x = b.x[i], v = b.v[i];
        fire_update_pre(s, x, v, f_load(b, i));
        if (s.zero_v) b.x[i] = x;      // the half step back moved x
        b.v[i] = v;
        vm = fmax(vm, v.x * v.x + v.y * v.y + v.z * v.z);
    }
    const double bm = block_max_nonneg(vm, red);
    if (threadIdx.x == 0) atomicMax(&b.st->vmax2, (unsigned long long)__double_as_longlong(bm));
}

}  // namespace fire2
