// Allocation-free energy/force evaluation (fire_energy_forces_noalloc).
//
// Some callers cannot call cudaMalloc at the point where they need forces:
// plug-ins of host programs whose memory pool owns all device memory and
// forbids stray allocations, and latency-critical loops where an allocation
// could synchronise the device or fail under memory pressure.  This entry
// point serves them: the caller passes device buffers for the
// positions and the results, and the only scratch the kernels need (per-atom
// densities, embedding derivatives and per-block energy partials) lives in the
// file-scope device array `g_scratch` below, sized for at most
// kNoAllocMaxAtoms atoms.  Every GPU that loads the library holds that array
// (about 0.5 MiB) until the process exits.
//
// The evaluation is all-pairs (minimum image), each atom summing over every
// other atom, so no neighbour list is needed and nothing accumulates across
// blocks: every scratch value read in a call is written earlier in the same
// call.  Calls that overlap on the GPU (two streams, or two host threads) race
// on g_scratch and must be serialised by the caller.
#include <cuda.h>   // CUcontext and the driver function types (entry points, no link)
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "fire2.h"

void fire2_set_global_error(const char* msg);  // defined in fire2_api.cu (hidden)

namespace {

constexpr int kNoAllocMaxAtoms = 32768;
constexpr int kBlock = 128;
constexpr int kMaxBlocks = (kNoAllocMaxAtoms + kBlock - 1) / kBlock;
constexpr int kScratchDoubles = 2 * kNoAllocMaxAtoms + kMaxBlocks;

// [0, N): rho_i; [N, 2N): F'(rho_i); [2N, 2N + blocks): energy partials.
static __device__ __align__(256) double g_scratch[kScratchDoubles];

struct NaPot {
    int kind;
    double rc2;
    double eps, sigma2, lj_shift;
    double A, xi2, p, q2, r0inv, p_r0, q2_r0, rs, winv;
    double L[3], Linv[3];
    int per[3];
};

__device__ __forceinline__ void na_min_image(double& d, double L, double Linv, int per) {
    if (per) d -= L * rint(d * Linv);
}

__device__ double na_block_sum(double v) {
    __shared__ double sh[32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (w == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    return r;
}

// RGL pair terms: phi = A e^{-p s} S, g = xi^2 e^{-2q s} S, s = r/r0 - 1, with
// the quintic taper S on [rs, rc); returns the derivatives too.
__device__ __forceinline__ void na_rgl_pair(const NaPot& P, double r, double& phi, double& dphi,
                                            double& g, double& dg) {
    const double s = r * P.r0inv - 1.0;
    const double ep = P.A * exp(-P.p * s);
    const double eq = P.xi2 * exp(-P.q2 * s);
    double S = 1.0, dS = 0.0;
    if (r > P.rs) {
        const double t = (r - P.rs) * P.winv;
        const double t2 = t * t, t3 = t2 * t;
        S = 1.0 - 10.0 * t3 + 15.0 * t3 * t - 6.0 * t3 * t2;
        dS = (-30.0 * t2 + 60.0 * t3 - 30.0 * t3 * t) * P.winv;
    }
    phi = ep * S;
    dphi = ep * (-P.p_r0 * S + dS);
    g = eq * S;
    dg = eq * (-P.q2_r0 * S + dS);
}

// Pass 1 (RGL): rho_i, F'(rho_i) and the per-atom energy, all-pairs.
// LJ: the whole evaluation (forces and energy) in this one pass.
__global__ void __launch_bounds__(kBlock) k_na_pass1(const double* __restrict__ pos, int n,
                                                     NaPot P, double* scratch,
                                                     double* __restrict__ forces) {
    __shared__ double3 tile[kBlock];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double xi = 0.0, yi = 0.0, zi = 0.0;
    if (i < n) {
        xi = pos[3 * i];
        yi = pos[3 * i + 1];
        zi = pos[3 * i + 2];
    }
    double rho = 0.0, e = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
    for (int base = 0; base < n; base += kBlock) {
        const int j0 = base + threadIdx.x;
        __syncthreads();
        if (j0 < n) tile[threadIdx.x] = make_double3(pos[3 * j0], pos[3 * j0 + 1], pos[3 * j0 + 2]);
        __syncthreads();
        const int m = min(kBlock, n - base);
        if (i >= n) continue;
        for (int k = 0; k < m; ++k) {
            const int j = base + k;
            if (j == i) continue;
            double dx = tile[k].x - xi, dy = tile[k].y - yi, dz = tile[k].z - zi;
            na_min_image(dx, P.L[0], P.Linv[0], P.per[0]);
            na_min_image(dy, P.L[1], P.Linv[1], P.per[1]);
            na_min_image(dz, P.L[2], P.Linv[2], P.per[2]);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 < P.rc2)) continue;
            if (P.kind == FIRE_POT_RGL) {
                double phi, dphi, g, dg;
                na_rgl_pair(P, sqrt(r2), phi, dphi, g, dg);
                rho += g;
                e += phi;
            } else {
                const double sr2 = P.sigma2 / r2;
                const double sr6 = sr2 * sr2 * sr2;
                e += 0.5 * (4.0 * P.eps * (sr6 * sr6 - sr6) - P.lj_shift);
                const double w = 24.0 * P.eps * (2.0 * sr6 * sr6 - sr6) / r2;
                fx -= w * dx;
                fy -= w * dy;
                fz -= w * dz;
            }
        }
    }
    if (i < n) {
        if (P.kind == FIRE_POT_RGL) {
            const double sq = sqrt(rho);
            scratch[i] = rho;
            scratch[kNoAllocMaxAtoms + i] = rho > 0.0 ? -0.5 / sq : 0.0;
            e -= sq;
        } else if (forces) {
            forces[3 * i] = fx;
            forces[3 * i + 1] = fy;
            forces[3 * i + 2] = fz;
        }
    }
    const double bs = na_block_sum(e);
    if (threadIdx.x == 0) scratch[2 * kNoAllocMaxAtoms + blockIdx.x] = bs;
}

// Pass 2 (RGL): F_i = sum_j [2 phi'(r) + (F'_i + F'_j) g'(r)] (x_j - x_i) / r.
__global__ void __launch_bounds__(kBlock) k_na_pass2(const double* __restrict__ pos, int n,
                                                     NaPot P, const double* scratch,
                                                     double* __restrict__ forces) {
    __shared__ double4_32a tile[kBlock];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const double* fp = scratch + kNoAllocMaxAtoms;
    double xi = 0.0, yi = 0.0, zi = 0.0, fpi = 0.0;
    if (i < n) {
        xi = pos[3 * i];
        yi = pos[3 * i + 1];
        zi = pos[3 * i + 2];
        fpi = fp[i];
    }
    double fx = 0.0, fy = 0.0, fz = 0.0;
    for (int base = 0; base < n; base += kBlock) {
        const int j0 = base + threadIdx.x;
        __syncthreads();
        if (j0 < n)
            tile[threadIdx.x] =
                make_double4_32a(pos[3 * j0], pos[3 * j0 + 1], pos[3 * j0 + 2], fp[j0]);
        __syncthreads();
        const int m = min(kBlock, n - base);
        if (i >= n) continue;
        for (int k = 0; k < m; ++k) {
            const int j = base + k;
            if (j == i) continue;
            double dx = tile[k].x - xi, dy = tile[k].y - yi, dz = tile[k].z - zi;
            na_min_image(dx, P.L[0], P.Linv[0], P.per[0]);
            na_min_image(dy, P.L[1], P.Linv[1], P.per[1]);
            na_min_image(dz, P.L[2], P.Linv[2], P.per[2]);
            const double r2 = dx * dx + dy * dy + dz * dz;
            if (!(r2 < P.rc2)) continue;
            const double r = sqrt(r2);
            double phi, dphi, g, dg;
            na_rgl_pair(P, r, phi, dphi, g, dg);
            const double fs = (2.0 * dphi + (fpi + tile[k].w) * dg) / r;
            fx += fs * dx;
            fy += fs * dy;
            fz += fs * dz;
        }
    }
    if (i < n && forces) {
        forces[3 * i] = fx;
        forces[3 * i + 1] = fy;
        forces[3 * i + 2] = fz;
    }
}

// Fixed-order sum of the per-block energy partials into *energy.
__global__ void k_na_energy(const double* scratch, int nblocks, double* energy) {
    double s = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += blockDim.x) s += scratch[2 * kNoAllocMaxAtoms + k];
    s = na_block_sum(s);
    if (threadIdx.x == 0 && energy) *energy = s;
}

std::mutex g_mu;

// The scratch array's device address is looked up once per device context:
// cudaDeviceReset (or a reset of the primary context) gives the device a new
// context and reloads the module, so the cache is keyed on the context's
// unique id (cuCtxGetId, through the runtime's driver entry points).
struct ScratchAddr {
    unsigned long long ctx_id = 0;   // 0 = none cached
    double* ptr = nullptr;
};
ScratchAddr g_addr[128];

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

// Unique id of the current context, or 0 when it cannot be had (then the
// address is looked up on every call).
unsigned long long current_context_id() {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool resolved = false;
    if (!resolved) {   // under g_mu
        cudaDriverEntryPointQueryResult q1, q2;
        void* f1 = nullptr;
        void* f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault,
                                             &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault,
                                             &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
            get_id = reinterpret_cast<CtxGetIdFn>(f2);
        }
        resolved = true;
    }
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of g_scratch in the current device's context.
cudaError_t scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    const unsigned long long id = current_context_id();
    ScratchAddr& a = g_addr[dev];
    if (id == 0 || a.ctx_id != id || !a.ptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_scratch);   // also makes the context current
        if (e != cudaSuccess) return e;
        a.ptr = static_cast<double*>(p);
        a.ctx_id = current_context_id();
    }
    *out = a.ptr;
    return cudaSuccess;
}

fire_status na_fail(fire_status code, const char* msg) {
    fire2_set_global_error(msg);
    return code;
}

}  // namespace

extern "C" fire_status fire_energy_forces_noalloc(const fire_potential_t* pot, int64_t n_atoms,
                                                  const int32_t periodic[3], const double* d_pos,
                                                  const double box[3], double* d_forces,
                                                  double* d_energy, void* stream) {
    if (!pot || !periodic || !d_pos || !box)
        return na_fail(FIRE_ERR_ARG, "fire_energy_forces_noalloc: NULL argument");
    if (n_atoms < 1 || n_atoms > kNoAllocMaxAtoms) {
        char buf[160];
        snprintf(buf, sizeof buf,
                 "fire_energy_forces_noalloc: n_atoms = %lld outside [1, %d] (size of the "
                 "static scratch array)", (long long)n_atoms, kNoAllocMaxAtoms);
        return na_fail(FIRE_ERR_ARG, buf);
    }
    if (pot->precision != FIRE_PREC_FP64)
        return na_fail(FIRE_ERR_ARG, "fire_energy_forces_noalloc: only FIRE_PREC_FP64");
    NaPot P{};
    P.kind = pot->kind;
    double rc = 0.0;
    if (pot->kind == FIRE_POT_LJ) {
        if (!(pot->rc_lj > 0.0 && pot->sigma > 0.0 && pot->eps > 0.0))
            return na_fail(FIRE_ERR_ARG, "fire_energy_forces_noalloc: LJ needs eps, sigma, rc_lj > 0");
        rc = pot->rc_lj;
        P.eps = pot->eps;
        P.sigma2 = pot->sigma * pot->sigma;
        const double sr6 = std::pow(pot->sigma / pot->rc_lj, 6.0);
        P.lj_shift = 4.0 * pot->eps * (sr6 * sr6 - sr6);
    } else if (pot->kind == FIRE_POT_RGL) {
        if (!(pot->rc > pot->rs && pot->rs > 0.0 && pot->r0 > 0.0 && pot->xi > 0.0 && pot->A >= 0.0))
            return na_fail(FIRE_ERR_ARG, "fire_energy_forces_noalloc: bad RGL parameters");
        rc = pot->rc;
        P.A = pot->A;
        P.xi2 = pot->xi * pot->xi;
        P.p = pot->p;
        P.q2 = 2.0 * pot->q;
        P.r0inv = 1.0 / pot->r0;
        P.p_r0 = pot->p / pot->r0;
        P.q2_r0 = 2.0 * pot->q / pot->r0;
        P.rs = pot->rs;
        P.winv = 1.0 / (pot->rc - pot->rs);
    } else {
        return na_fail(FIRE_ERR_ARG, "fire_energy_forces_noalloc: unknown potential kind");
    }
    P.rc2 = rc * rc;
    for (int a = 0; a < 3; ++a) {
        if (!(box[a] > 0.0) || !std::isfinite(box[a]))
            return na_fail(FIRE_ERR_ARG, "fire_energy_forces_noalloc: box lengths must be > 0");
        if (periodic[a] && box[a] < 2.0 * rc)
            return na_fail(FIRE_ERR_ARG,
                           "fire_energy_forces_noalloc: periodic box shorter than twice the cut-off");
        P.L[a] = box[a];
        P.Linv[a] = 1.0 / box[a];
        P.per[a] = periodic[a] ? 1 : 0;
    }
    double* scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess) return na_fail(FIRE_ERR_CUDA, cudaGetErrorString(e));
    int n = (int)n_atoms;
    int blocks = (n + kBlock - 1) / kBlock;
    cudaStream_t s = (cudaStream_t)stream;
    // cudaLaunchKernel returns the status of its own launch, so an error left
    // pending by the caller's earlier work is neither reported as this call's
    // nor cleared
    const double* pos = d_pos;
    double* fout = d_forces;
    double* eout = d_energy;
    void* args12[] = {(void*)&pos, (void*)&n, (void*)&P, (void*)&scratch, (void*)&fout};
    e = cudaLaunchKernel((const void*)k_na_pass1, dim3(blocks), dim3(kBlock), args12, 0, s);
    if (e == cudaSuccess && P.kind == FIRE_POT_RGL)
        e = cudaLaunchKernel((const void*)k_na_pass2, dim3(blocks), dim3(kBlock), args12, 0, s);
    void* args3[] = {(void*)&scratch, (void*)&blocks, (void*)&eout};
    if (e == cudaSuccess)
        e = cudaLaunchKernel((const void*)k_na_energy, dim3(1), dim3(256), args3, 0, s);
    if (e != cudaSuccess) return na_fail(FIRE_ERR_CUDA, cudaGetErrorString(e));
    return FIRE_OK;
}
