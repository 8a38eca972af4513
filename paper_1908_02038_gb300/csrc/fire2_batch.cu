// Batched FIRE 2.0: hundreds of independent relaxations of uneven size in one
// persistent launch.
//
// Each CTA takes the next system from a device work queue (systems sorted
// largest first, so the long relaxations start early), relaxes it completely
// -- list build, RGL density and force passes, FP64 block reductions,
// Algorithm 2 control, Algorithm 4 update -- with __syncthreads() as the only
// synchronisation, and then takes the next one.  Every system keeps its own
// FIRE state (dt, alpha, counters), list and stop reason.  No CTA ever waits
// on another, so there is no grid barrier and nothing to time out; each
// relaxation is bounded by maxiter and by the wall-clock budget.
//
// The launch shape (threads per CTA, CTAs per SM) is chosen by the autotuner
// in fire_batch_autotune: it times every candidate shape on the caller's
// batch for a fixed number of iterations and keeps the fastest.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "fire2.h"
#include "fire2_common.cuh"
#include "fire2_table.cuh"

using namespace fire2;

namespace fire2 {

// Per-system description (device array).
struct BInst {
    long long off;          // first atom in the packed arrays
    long long list_off;     // first list slot: nbr[list_off + k * n + i]
    int n, cap;             // atoms, list capacity per atom
    int nc[3];              // cells per axis; nc[0] == 0 -> all-pairs build
    int per[3];
    int Lq[3];              // box in fixed-point units (FP32-pair form)
    long long Lq64[3];      // box in 2^-44 A units (FP64 table form)
    double L[3], Linv[3];
    float Lf[3], Linvf[3];
    float rlist2f;
    double half_skin2;
};

// Per-system result (device array).
struct BRes {
    double energy, fmax2, F2, finf, dt, alpha;
    long long iter, evals, builds;
    int stop, status;
};

struct BArgs {
    int n_sys;
    const int* order;       // systems, largest first
    int* queue;             // next index into `order`
    const BInst* inst;
    BRes* res;
    dvec4 *x, *v, *f, *xref;
    int4* xq;
    float4* xf;
    lvec4* xq64;            // FP64 table form: positions in 2^-44 A units
    float2* fpff;           // FP64 table form: F'(rho) as a float pair
    const float *tab_ffd, *tab_fff;   // FP64 table form: density / force rows
    int ff;                 // 1: FP64 table passes available (FP64 table form, or the
                            //    FP32-pair form confirming its stops)
    int confirm;            // FP32-pair form: FP64 check of its stops (confirm64 != 0)
    int vmode;              // fire_fp64_check: 1 confirm, 2 finish in FP64 below 3 ftol
    double* fp64;           // F'(rho) (FP64 form)
    float* fp32;            // F'(rho) (FP32-pair form)
    uint32_t* nbr;
    int* nnbr;
    double* pos_io;         // packed N x 3, in/out
    double* f_out;          // packed N x 3 final forces, optional
    FireParamsD prm;
    unsigned long long budget_ns;
    PotC P;
    const double* exp_table;
    const float* exp32_table;
    double qscale;
    int max_cells;          // capacity of the shared cell arrays
    int max_atoms_smem;     // capacity of the shared cell-sorted atom array
};

struct BShared {            // per-CTA scalars
    FireScal fs;
    int sys, done, status, rebuild;
    long long builds;
    double P, F2, V2, fa2, fin, E, dmax;
    // FP64 check of FP32-pair stops (as fire2_device.cuh's DevState): vstate
    // 0 off, 1 FP32 phase, 2 the next evaluation confirms in FP64, 3 FP64
    // passes to the end (vmode 2)
    int vstate;
    double ftol_work, fn32;
};

// Block reductions into shared scalars (all threads must call).
__device__ __forceinline__ double bsum(double v, double* red) {
    const double r = block_sum(v, red);
    __shared__ double out;
    if (threadIdx.x == 0) out = r;
    __syncthreads();
    return out;
}
__device__ __forceinline__ double bmax(double v, double* red) {
    const double r = block_max(v, red);
    __shared__ double out;
    if (threadIdx.x == 0) out = r;
    __syncthreads();
    return out;
}

// Adds pair (i, j) to i's full list when the FP32 candidate test passes.
__device__ __forceinline__ void b_try_pair(const BArgs& a, const BInst& I, int i, float4 xi, int j,
                                           int& cnt, int& bad) {
    const float4 xj = a.xf[I.off + j];
    float d[3] = {xj.x - xi.x, xj.y - xi.y, xj.z - xi.z};
    int s[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (I.per[k]) {
            s[k] = __float2int_rn(d[k] * I.Linvf[k]);
            d[k] -= (float)s[k] * I.Lf[k];
        }
    }
    const float r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (!(r2 < I.rlist2f)) return;
    if (s[0] < -2 || s[0] > 2 || s[1] < -2 || s[1] > 2 || s[2] < -2 || s[2] > 2) {
        bad = ST_RANGE;
        return;
    }
    if (cnt < I.cap) {
        const uint32_t code = (uint32_t)((s[0] + 2) + 5 * (s[1] + 2) + 25 * (s[2] + 2));
        a.nbr[I.list_off + (long long)cnt * I.n + i] = (code << kIdxBits) | (uint32_t)j;
    }
    ++cnt;
}

// Full neighbour list of atoms [lo, hi) of one system; cell-sorted atoms of
// the whole system in shared memory when every periodic axis holds at least
// 3 cells (open axes any number), all pairs otherwise.  Returns the CTA's error status (0, ST_RANGE or
// ST_NBR_OVERFLOW), the same in every thread.
__device__ __forceinline__ int b_build(const BArgs& a, const BInst& I, int lo, int hi, int* s_count,
                                       int* s_start, int* s_atoms, double* red) {
    const int T = blockDim.x, t = threadIdx.x;
    const bool cells = I.nc[0] > 0;
    const int ncell = cells ? I.nc[0] * I.nc[1] * I.nc[2] : 0;
    if (cells) {
        for (int c = t; c < ncell; c += T) s_count[c] = 0;
        __syncthreads();
        for (int i = t; i < I.n; i += T) {
            const dvec4 x = a.x[I.off + i];
            const int c = (cell_coord(x.x, I.Linv[0], I.nc[0], I.per[0]) * I.nc[1] +
                           cell_coord(x.y, I.Linv[1], I.nc[1], I.per[1])) * I.nc[2] +
                          cell_coord(x.z, I.Linv[2], I.nc[2], I.per[2]);
            atomicAdd(&s_count[c], 1);
        }
        __syncthreads();
        if (t == 0) {
            int run = 0;
            for (int c = 0; c < ncell; ++c) {
                s_start[c] = run;
                run += s_count[c];
                s_count[c] = s_start[c];
            }
            s_start[ncell] = run;
        }
        __syncthreads();
        for (int i = t; i < I.n; i += T) {
            const dvec4 x = a.x[I.off + i];
            const int c = (cell_coord(x.x, I.Linv[0], I.nc[0], I.per[0]) * I.nc[1] +
                           cell_coord(x.y, I.Linv[1], I.nc[1], I.per[1])) * I.nc[2] +
                          cell_coord(x.z, I.Linv[2], I.nc[2], I.per[2]);
            s_atoms[atomicAdd(&s_count[c], 1)] = i;
        }
        __syncthreads();
    }
    int bad = ST_OK, over = 0;
    for (int i = lo + t; i < hi; i += T) {
        const float4 xi = a.xf[I.off + i];
        int cnt = 0;
        if (!cells) {
            for (int j = 0; j < I.n; ++j)
                if (j != i) b_try_pair(a, I, i, xi, j, cnt, bad);
        } else {
            const dvec4 x = a.x[I.off + i];
            const int cx = cell_coord(x.x, I.Linv[0], I.nc[0], I.per[0]);
            const int cy = cell_coord(x.y, I.Linv[1], I.nc[1], I.per[1]);
            const int cz = cell_coord(x.z, I.Linv[2], I.nc[2], I.per[2]);
            for (int ox = -1; ox <= 1; ++ox) {
                const int ax = cell_step(cx, ox, I.nc[0], I.per[0]);
                if (ax < 0) continue;
                for (int oy = -1; oy <= 1; ++oy) {
                    const int ay = cell_step(cy, oy, I.nc[1], I.per[1]);
                    if (ay < 0) continue;
                    for (int oz = -1; oz <= 1; ++oz) {
                        const int az = cell_step(cz, oz, I.nc[2], I.per[2]);
                        if (az < 0) continue;
                        const int c = (ax * I.nc[1] + ay) * I.nc[2] + az;
                        for (int k = s_start[c]; k < s_start[c + 1]; ++k) {
                            const int j = s_atoms[k];
                            if (j != i) b_try_pair(a, I, i, xi, j, cnt, bad);
                        }
                    }
                }
            }
        }
        if (cnt > I.cap) {
            over = 1;
            cnt = I.cap;
        }
        a.nnbr[I.off + i] = cnt;
        a.xref[I.off + i] = a.x[I.off + i];
    }
    return (int)bmax((double)(bad != ST_OK ? bad : (over ? ST_NBR_OVERFLOW : 0)), red);
}

// Separation x_j - x_i - shift of list entry e in the FP64 table form: exact
// in 2^-44 A fixed point, split into float pairs; returns r^2.
__device__ __forceinline__ ffloat b_sep_ff(const BArgs& a, const BInst& I, const lvec4& qi,
                                           uint32_t e, ffloat& dx, ffloat& dy, ffloat& dz) {
    const int j = (int)(e & kIdxMask), code = (int)(e >> kIdxBits);
    const lvec4 qj = a.xq64[I.off + j];
    long long ix = qj.x - qi.x, iy = qj.y - qi.y, iz = qj.z - qi.z;
    if (code != kCodeZero) {
        ix -= (long long)(code % 5 - 2) * I.Lq64[0];
        iy -= (long long)((code / 5) % 5 - 2) * I.Lq64[1];
        iz -= (long long)(code / 25 - 2) * I.Lq64[2];
    }
    dx = fixed_to_ff(ix);
    dy = fixed_to_ff(iy);
    dz = fixed_to_ff(iz);
    return ff_norm2(dx, dy, dz);
}

// Energy and forces of atoms [lo, hi) of one system (full list, no
// atomics); returns their energy.  With CL, the CTAs of a thread-block
// cluster share the system: the cluster barrier between the passes makes
// every CTA's F'(rho) visible to the others.
template <bool F32, bool CL>
__device__ __forceinline__ double b_forces(const BArgs& a, const BInst& I, int lo, int hi,
                                           const double* etab, const float* et32, double* red) {
    const PotC& P = a.P;
    const int T = blockDim.x, t = threadIdx.x;
    double e_sum = 0.0;
    // pass 1: densities, embedding derivative, atom energies
    for (int i = lo + t; i < hi; i += T) {
        const long long gi = I.off + i;
        const int m = a.nnbr[gi];
        if (F32) {
            const int4 qi = a.xq[gi];
            Kahan32 rho, erep;
            for (int k = 0; k < m; ++k) {
                const uint32_t e = a.nbr[I.list_off + (long long)k * I.n + i];
                const int j = (int)(e & kIdxMask), code = (int)(e >> kIdxBits);
                const int4 qj = a.xq[I.off + j];
                int dx = wrap_sub(qj.x, qi.x), dy = wrap_sub(qj.y, qi.y), dz = wrap_sub(qj.z, qi.z);
                if (code != kCodeZero) {
                    dx = wrap_sub(dx, (int)((unsigned)(code % 5 - 2) * (unsigned)I.Lq[0]));
                    dy = wrap_sub(dy, (int)((unsigned)((code / 5) % 5 - 2) * (unsigned)I.Lq[1]));
                    dz = wrap_sub(dz, (int)((unsigned)(code / 25 - 2) * (unsigned)I.Lq[2]));
                }
                const long long r2q = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
                if (r2q >= P.rc2q) continue;
                float rinv, phi, dphi, g, dg;
                rgl_pair32(P, r2q, et32, rinv, phi, dphi, g, dg);
                rho.add(g);
                erep.add(phi);
            }
            const float rf = (float)rho.value();
            const float sq = sqrtf(rf);
            a.fp32[gi] = rf > 0.f ? -0.5f / sq : 0.f;
            e_sum += erep.value() - (double)sq;
        } else if (a.ff) {   // FP64 table form: double-float pair terms, FP64 embedding
            const lvec4 qi = a.xq64[gi];
            ffloat rho = {0.f, 0.f}, erep = {0.f, 0.f};
            for (int k = 0; k < m; ++k) {
                ffloat dx, dy, dz;
                const ffloat r2 =
                    b_sep_ff(a, I, qi, a.nbr[I.list_off + (long long)k * I.n + i], dx, dy, dz);
                if (!(r2.hi < P.rc2_f)) continue;
                const float uf = r2.hi - P.r0sq_f;
                if (uf >= P.tab.u_lo_f) {
                    float row[kFFRow];
                    load_row(a.tab_ffd, ff_index(P.tab, uf), row);
                    ffloat v[2];
                    ff_row_eval(row, r2, v);
                    erep = ff_acc(erep, v[0]);
                    rho = ff_acc(rho, v[1]);
                } else {   // compressed below the table: FP64 exponentials
                    double rinv, phi, dphi, g, dg;
                    rgl_pair64(P, ff_to_f64(r2), etab, rinv, phi, dphi, g, dg);
                    erep = ff_acc(erep, f64_to_ff(phi));
                    rho = ff_acc(rho, f64_to_ff(g));
                }
            }
            double sq, fp;
            ffloat fpf;
            rgl_embed_dd(ff_to_f64(rho), sq, fp, fpf);
            a.fp64[gi] = fp;
            a.fpff[gi] = make_float2(fpf.hi, fpf.lo);
            e_sum += ff_to_f64(erep) - sq;
        } else {
            const dvec4 xi = a.x[gi];
            double rho = 0.0, erep = 0.0;
            for (int k = 0; k < m; ++k) {
                const uint32_t e = a.nbr[I.list_off + (long long)k * I.n + i];
                const int j = (int)(e & kIdxMask), code = (int)(e >> kIdxBits);
                const dvec4 xj = a.x[I.off + j];
                double dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
                if (code != kCodeZero) {
                    dx -= (code % 5 - 2) * I.L[0];
                    dy -= ((code / 5) % 5 - 2) * I.L[1];
                    dz -= (code / 25 - 2) * I.L[2];
                }
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 < P.rc2)) continue;
                double rinv, phi, dphi, g, dg;
                rgl_pair64(P, r2, etab, rinv, phi, dphi, g, dg);
                rho += g;
                erep += phi;
            }
            double sq, fp;
            rgl_embed(rho, sq, fp);
            a.fp64[gi] = fp;
            e_sum += erep - sq;
        }
    }
    const double E = bsum(e_sum, red);  // also orders pass 1 before pass 2 in the CTA
    if (CL) cooperative_groups::this_cluster().sync();   // ... and across the cluster
    // pass 2: forces
    for (int i = lo + t; i < hi; i += T) {
        const long long gi = I.off + i;
        const int m = a.nnbr[gi];
        if (F32) {
            const int4 qi = a.xq[gi];
            const float fpi = a.fp32[gi];
            Kahan32 fx, fy, fz;
            for (int k = 0; k < m; ++k) {
                const uint32_t e = a.nbr[I.list_off + (long long)k * I.n + i];
                const int j = (int)(e & kIdxMask), code = (int)(e >> kIdxBits);
                const int4 qj = a.xq[I.off + j];
                int dx = wrap_sub(qj.x, qi.x), dy = wrap_sub(qj.y, qi.y), dz = wrap_sub(qj.z, qi.z);
                if (code != kCodeZero) {
                    dx = wrap_sub(dx, (int)((unsigned)(code % 5 - 2) * (unsigned)I.Lq[0]));
                    dy = wrap_sub(dy, (int)((unsigned)((code / 5) % 5 - 2) * (unsigned)I.Lq[1]));
                    dz = wrap_sub(dz, (int)((unsigned)(code / 25 - 2) * (unsigned)I.Lq[2]));
                }
                const long long r2q = (long long)dx * dx + (long long)dy * dy + (long long)dz * dz;
                if (r2q >= P.rc2q) continue;
                float rinv, phi, dphi, g, dg;
                rgl_pair32(P, r2q, et32, rinv, phi, dphi, g, dg);
                const float fs = (2.f * dphi + (fpi + a.fp32[I.off + j]) * dg) * rinv * P.qinv;
                fx.add(fs * (float)dx);
                fy.add(fs * (float)dy);
                fz.add(fs * (float)dz);
            }
            a.f[gi] = make_dvec4(fx.value(), fy.value(), fz.value(), 0.0);
        } else if (a.ff) {
            const lvec4 qi = a.xq64[gi];
            const float2 fpi2 = a.fpff[gi];
            const ffloat fpi = {fpi2.x, fpi2.y};
            ffloat fx = {0.f, 0.f}, fy = {0.f, 0.f}, fz = {0.f, 0.f};
            for (int k = 0; k < m; ++k) {
                const uint32_t e = a.nbr[I.list_off + (long long)k * I.n + i];
                ffloat dx, dy, dz;
                const ffloat r2 = b_sep_ff(a, I, qi, e, dx, dy, dz);
                if (!(r2.hi < P.rc2_f)) continue;
                const float uf = r2.hi - P.r0sq_f;
                ffloat c[2];
                if (uf >= P.tab.u_lo_f) {
                    float row[kFFRow];
                    load_row(a.tab_fff, ff_index(P.tab, uf), row);
                    ff_row_eval(row, r2, c);
                } else {
                    double rinv, phi, dphi, g, dg;
                    rgl_pair64(P, ff_to_f64(r2), etab, rinv, phi, dphi, g, dg);
                    c[0] = f64_to_ff(2.0 * dphi * rinv);
                    c[1] = f64_to_ff(dg * rinv);
                }
                const float2 fpj2 = a.fpff[I.off + (int)(e & kIdxMask)];
                const ffloat fs = ff_madd(ff_add(fpi, {fpj2.x, fpj2.y}), c[1], c[0]);
                fx = ff_acc(fx, ff_mul_nn(fs, dx));
                fy = ff_acc(fy, ff_mul_nn(fs, dy));
                fz = ff_acc(fz, ff_mul_nn(fs, dz));
            }
            a.f[gi] = make_dvec4(ff_to_f64(fx), ff_to_f64(fy), ff_to_f64(fz), 0.0);
        } else {
            const dvec4 xi = a.x[gi];
            const double fpi = a.fp64[gi];
            double fx = 0.0, fy = 0.0, fz = 0.0;
            for (int k = 0; k < m; ++k) {
                const uint32_t e = a.nbr[I.list_off + (long long)k * I.n + i];
                const int j = (int)(e & kIdxMask), code = (int)(e >> kIdxBits);
                const dvec4 xj = a.x[I.off + j];
                double dx = xj.x - xi.x, dy = xj.y - xi.y, dz = xj.z - xi.z;
                if (code != kCodeZero) {
                    dx -= (code % 5 - 2) * I.L[0];
                    dy -= ((code / 5) % 5 - 2) * I.L[1];
                    dz -= (code / 25 - 2) * I.L[2];
                }
                const double r2 = dx * dx + dy * dy + dz * dz;
                if (!(r2 < P.rc2)) continue;
                double rinv, phi, dphi, g, dg;
                rgl_pair64(P, r2, etab, rinv, phi, dphi, g, dg);
                const double fs = (2.0 * dphi + (fpi + a.fp64[I.off + j]) * dg) * rinv;
                fx += fs * dx;
                fy += fs * dy;
                fz += fs * dz;
            }
            a.f[gi] = make_dvec4(fx, fy, fz, 0.0);
        }
    }
    return E;
}

// Exchange of per-CTA scalars inside a thread-block cluster (distributed
// shared memory): thread 0 of every CTA stores its values, one cluster
// barrier, then thread 0 of every CTA reads all ranks' values in rank order
// and combines them -- sums for the first nsum entries, maxima for the rest
// -- so every CTA holds bit-identical results without a second barrier.  Two
// buffers alternate: the barrier of the next exchange orders the reads of
// this one before any later overwrite.  Without a cluster the values pass
// through unchanged.
struct ClX {
    double buf[2][8];
    double res[8];
    int parity;
};

template <bool CL>
__device__ __forceinline__ void cl_combine(ClX& x, const double* v, int nsum, int nval) {
    if (!CL) {
        if (threadIdx.x == 0)
            for (int k = 0; k < nval; ++k) x.res[k] = v[k];
        __syncthreads();
        return;
    }
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int par = x.parity;
    if (threadIdx.x == 0)
        for (int k = 0; k < nval; ++k) x.buf[par][k] = v[k];
    cl.sync();
    if (threadIdx.x == 0) {
        double acc[8];
        for (int r = 0; r < (int)cl.num_blocks(); ++r) {
            const double* rv = cl.map_shared_rank(&x.buf[par][0], r);
            for (int k = 0; k < nval; ++k)
                acc[k] = r == 0 ? rv[k] : (k < nsum ? acc[k] + rv[k] : fmax(acc[k], rv[k]));
        }
        for (int k = 0; k < nval; ++k) x.res[k] = acc[k];
        x.parity = par ^ 1;
    }
    __syncthreads();
}

// The element-wise step of atoms [lo, hi) of one system (Algorithm 2's half
// step back and Algorithm 4: fire_update_pre, fire_update_drift_k); returns the largest squared
// displacement since the last list build.  The tests that hold for the whole
// pass (explicit Euler's kick, the displacement cap) are taken once, and the
// FP32 copy of x and the displacement are formed on the integer and FP32
// pipes: FP64 instructions issue at 1/58 of the FP32 rate on this part.  The
// copies are truncated (off by < 1 FP32 ulp of the coordinate, the
// displacement by < 2), far inside the list radius's margin of 1e-3 rc + 8
// FP32 ulps of the box.
template <bool F32, bool KICK>
__device__ __forceinline__ float b_update(const BArgs& a, const BInst& I, int lo, int hi,
                                          const FireScal& fs, double dt_drift, bool capped,
                                          bool fp64_phase) {
    float dmax = 0.f;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const long long gi = I.off + i;
        dvec4 x = a.x[gi], v = a.v[gi];
        const dvec4 f = a.f[gi];
        const dvec4 r = a.xref[gi];
        if (!capped) fire_update_pre(fs, x, v, f);   // capped: done by the first pass
        fire_update_drift_k<KICK>(fs, dt_drift, x, v, f);
        a.x[gi] = x;
        a.v[gi] = v;
        const float fx = f64_to_f32_trunc(x.x), fy = f64_to_f32_trunc(x.y),
                    fz = f64_to_f32_trunc(x.z);
        a.xf[gi] = make_float4(fx, fy, fz, 0.f);
        if (F32)
            a.xq[gi] = make_int4(to_fixed(x.x, a.qscale), to_fixed(x.y, a.qscale),
                                 to_fixed(x.z, a.qscale), 0);
        if (a.ff && (!F32 || fp64_phase))
            a.xq64[gi] = {to_fixed64(x.x, kFixedBits64), to_fixed64(x.y, kFixedBits64),
                          to_fixed64(x.z, kFixedBits64), 0ll};
        const float ddx = fx - f64_to_f32_trunc(r.x), ddy = fy - f64_to_f32_trunc(r.y),
                    ddz = fz - f64_to_f32_trunc(r.z);
        dmax = fmaxf(dmax, ddx * ddx + ddy * ddy + ddz * ddz);
    }
    return dmax;
}

// FP64 reductions of (F, v) of atoms [lo, hi) (combined over the cluster),
// then Algorithm 2 in thread 0 of every CTA on identical inputs.  Kept out of
// line: inlined, its FP64 scalar state raised the kernel's register peak and
// made the 64-register budget spill (228 bytes) in the force loops; called,
// nothing spills and the 1024-thread shape runs 3 % faster.
template <bool CL>
__device__ __noinline__ void b_reduce_control(const BArgs& a, const BInst& I, int lo, int hi,
                                                 BShared& sh, ClX& X, double E, double* red,
                                                 unsigned long long t0) {
    double P = 0.0, F2 = 0.0, V2 = 0.0, fa2 = 0.0, fin = 0.0;
    const FireScal fs = sh.fs;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const dvec4 f = a.f[I.off + i];
        dvec4 v = a.v[I.off + i];
        if (fs.vv) {   // second half kick of velocity Verlet (Alg. 6)
            fire_vv_kick(fs, v, f);
            a.v[I.off + i] = v;
        }
        // products chained into the sums; maxima of non-negative values on
        // the integer pipes (as in the single-system reductions)
        P = fma(f.z, v.z, fma(f.y, v.y, fma(f.x, v.x, P)));
        const double q = fma(f.z, f.z, fma(f.y, f.y, f.x * f.x));
        F2 += q;
        V2 = fma(v.z, v.z, fma(v.y, v.y, fma(v.x, v.x, V2)));
        fa2 = max_nonneg(fa2, q);
        fin = max_nonneg(fin, max_nonneg(abs_bits(f.x), max_nonneg(abs_bits(f.y), abs_bits(f.z))));
    }
    double v[8];
    v[0] = bsum(P, red);
    v[1] = bsum(F2, red);
    v[2] = bsum(V2, red);
    v[3] = E;
    v[4] = bmax(fa2, red);
    v[5] = bmax(fin, red);
    v[6] = (double)sh.status;
    v[7] = (double)(globaltimer_ns() - t0);   // the cluster takes the largest
    cl_combine<CL>(X, v, 4, 8);
    if (threadIdx.x == 0) {
        const double* r = X.res;
        sh.P = r[0];
        sh.F2 = r[1];
        sh.V2 = r[2];
        sh.E = r[3];
        sh.fa2 = r[4];
        sh.fin = r[5];
        sh.status = (int)r[6];
        bool stop;
        if (sh.status != ST_OK) {
            sh.fs.evals += 1;
            stop = true;
        } else if (!isfinite(sh.E) || !isfinite(sh.F2) || !isfinite(sh.V2)) {
            sh.fs.evals += 1;
            sh.status = ST_NONFINITE;
            stop = true;
        } else if (a.budget_ns && r[7] > (double)a.budget_ns) {
            sh.fs.evals += 1;
            sh.status = ST_TIMEOUT;
            stop = true;
        } else {
            FireParamsD p = a.prm;
            p.ftol = sh.ftol_work;
            if (sh.vstate == 2) {   // these forces confirm an FP32-pair stop in FP64
                const double fn = force_norm(p.norm, sh.F2, sh.fa2, sh.fin);
                if (fn < a.prm.ftol) {
                    sh.fs.evals += 1;
                    sh.fs.stop = STOP_FTOL;
                    stop = true;
                } else if (a.vmode == 2) {   // finish in FP64 from here
                    sh.vstate = 3;
                    stop = fire_control_step(p, sh.fs, sh.P, sh.F2, sh.V2, sh.fa2, sh.fin);
                } else {   // tighten the FP32 threshold, step with these forces
                    sh.ftol_work = fmax(sh.ftol_work - 1.5 * (fn - sh.fn32), 0.4 * a.prm.ftol);
                    p.ftol = sh.ftol_work;
                    sh.vstate = 1;
                    stop = fire_control_step(p, sh.fs, sh.P, sh.F2, sh.V2, sh.fa2, sh.fin);
                }
            } else {
                stop = fire_control_step(p, sh.fs, sh.P, sh.F2, sh.V2, sh.fa2, sh.fin);
                if (stop && sh.vstate == 1 && sh.fs.stop == STOP_FTOL) {
                    sh.fn32 = force_norm(p.norm, sh.F2, sh.fa2, sh.fin);
                    sh.vstate = 2;
                    stop = false;
                } else if (!stop && sh.vstate == 1 && a.vmode == 2 &&
                           force_norm(p.norm, sh.F2, sh.fa2, sh.fin) < 3.0 * a.prm.ftol) {
                    sh.vstate = 3;   // FP64 passes from the next evaluation on
                }
            }
        }
        sh.done = stop ? 1 : 0;
    }
    __syncthreads();
}

// The FP64 table passes of one system, out of line so that the FP32-pair
// kernel that calls them to confirm a stop keeps its own register budget.
template <bool CL>
__device__ __noinline__ double b_forces_confirm(const BArgs& a, const BInst& I, int lo, int hi,
                                                const double* etab, const float* et32,
                                                double* red) {
    return b_forces<false, CL>(a, I, lo, hi, etab, et32, red);
}

// The batched relaxation.  CL = false: one CTA per system.  CL = true: the
// CTAs of a thread-block cluster share each system -- rank r owns atoms
// [r n / C, (r + 1) n / C) -- with cluster barriers where one CTA reads what
// another wrote (positions before a list build or force pass, F'(rho)
// between the passes) and the cluster exchange for every reduction; every
// decision (stop, rebuild, drift cap) is taken on bit-identical values in
// all CTAs, so they run through the same barriers.
// Register budgets: MAXT = 512 allows up to 128 registers per thread, so one
// 512-thread CTA (16 warps) per SM; MAXT = 768 holds the kernel to 80
// registers (a few spilled bytes) so 768 threads (24 warps) fit on an SM;
// MAXT = 1024 to 64 (more spills), 32 warps.  More warps keep more of the
// neighbour gathers in flight; the autotuner measures which budget wins.
template <bool F32, bool CL, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) k_batch_relax(BArgs a) {
    namespace cg = cooperative_groups;
    extern __shared__ int smem[];
    __shared__ double etab[kExpTableSize];
    __shared__ float et32[kExp32TableSize];
    __shared__ double red[32];
    __shared__ BShared sh;
    __shared__ ClX X;
    int* s_count = smem;
    int* s_start = smem + a.max_cells;
    int* s_atoms = smem + 2 * a.max_cells + 1;
    int rank = 0, C = 1;
    if (CL) {
        rank = (int)cg::this_cluster().block_rank();
        C = (int)cg::this_cluster().num_blocks();
    }
    for (int t = threadIdx.x; t < kExpTableSize; t += blockDim.x) etab[t] = a.exp_table[t];
    for (int t = threadIdx.x; t < kExp32TableSize; t += blockDim.x) et32[t] = a.exp32_table[t];
    if (threadIdx.x == 0) X.parity = 0;
    // every CTA of the cluster must be running before any distributed
    // shared memory access
    if (CL) cg::this_cluster().sync();
    for (;;) {
        // the next system: rank 0 takes it from the queue and hands it to the cluster
        if (rank == 0 && threadIdx.x == 0) {
            const int k = atomicAdd(a.queue, 1);
            const int next = k < a.n_sys ? a.order[k] : -1;
            if (CL) {
                cg::cluster_group cl = cg::this_cluster();
                for (int r = 0; r < C; ++r) cl.map_shared_rank(&sh, r)->sys = next;
            } else {
                sh.sys = next;
            }
        }
        if (CL) cg::this_cluster().sync();
        else __syncthreads();
        const int sys = sh.sys;
        if (sys < 0) return;
        const BInst I = a.inst[sys];
        const int lo = (int)((long long)I.n * rank / C), hi = (int)((long long)I.n * (rank + 1) / C);
        const unsigned long long t0 = globaltimer_ns();
        // set-up: positions in, v = 0, FIRE state (Algorithm 2 initialisation)
        int bad = 0;
        for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const long long gi = I.off + i;
            const double* p = a.pos_io + 3 * gi;
            if (!isfinite(p[0]) || !isfinite(p[1]) || !isfinite(p[2])) bad = 1;
            a.x[gi] = make_dvec4(p[0], p[1], p[2], 0.0);
            a.xf[gi] = make_float4((float)p[0], (float)p[1], (float)p[2], 0.f);
            if (F32)
                a.xq[gi] = make_int4(to_fixed(p[0], a.qscale), to_fixed(p[1], a.qscale),
                                     to_fixed(p[2], a.qscale), 0);
            else if (a.ff)
                a.xq64[gi] = {to_fixed64(p[0], kFixedBits64), to_fixed64(p[1], kFixedBits64),
                              to_fixed64(p[2], kFixedBits64), 0ll};
            a.v[gi] = make_dvec4(0.0, 0.0, 0.0, 0.0);
        }
        const double anybad = bmax((double)bad, red);
        if (threadIdx.x == 0) {
            fire_scal_init(a.prm, sh.fs);
            sh.vstate = (F32 && a.confirm) ? 1 : 0;
            sh.ftol_work = a.prm.ftol;
            sh.status = anybad > 0.0 ? ST_NONFINITE : ST_OK;
            sh.builds = 0;
            sh.done = 0;
        }
        if (CL) cg::this_cluster().sync();   // every CTA's positions before the list build
        else __syncthreads();
        int bst = b_build(a, I, lo, hi, s_count, s_start, s_atoms, red);
        if (threadIdx.x == 0) {
            if (bst != ST_OK && sh.status == ST_OK) sh.status = bst;
            sh.builds += 1;
        }
        double E = b_forces<F32, CL>(a, I, lo, hi, etab, et32, red);
        b_reduce_control<CL>(a, I, lo, hi, sh, X, E, red, t0);
        while (!sh.done) {
            if (F32 && sh.vstate == 2) {
                // confirm the FP32-pair stop: FP64 forces at the same positions
                for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
                    const dvec4 x = a.x[I.off + i];
                    a.xq64[I.off + i] = {to_fixed64(x.x, kFixedBits64),
                                         to_fixed64(x.y, kFixedBits64),
                                         to_fixed64(x.z, kFixedBits64), 0ll};
                }
                if (CL) cg::this_cluster().sync();
                else __syncthreads();
                E = b_forces_confirm<CL>(a, I, lo, hi, etab, et32, red);
                b_reduce_control<CL>(a, I, lo, hi, sh, X, E, red, t0);
                continue;
            }
            const FireScal fs = sh.fs;
            const bool fp64_phase = F32 && sh.vstate == 3;   // finishing in FP64
            // maximum displacement per step: the drift waits for max_i |v_i|
            double dt_drift = fs.dt_cur;
            if (a.prm.dmax > 0.0) {
                double vm = 0.0;
                for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
                    const long long gi = I.off + i;
                    dvec4 x = a.x[gi], v = a.v[gi];
                    fire_update_pre(fs, x, v, a.f[gi]);
                    if (fs.zero_v) a.x[gi] = x;
                    a.v[gi] = v;
                    vm = fmax(vm, v.x * v.x + v.y * v.y + v.z * v.z);
                }
                const double vb = bmax(vm, red);
                cl_combine<CL>(X, &vb, 0, 1);
                dt_drift = fire_capped_dt(fs.dt_cur, a.prm.dmax, X.res[0]);
            }
            const bool capped = a.prm.dmax > 0.0;
            const float dmax = fs.kick_after != 0.0
                                   ? b_update<F32, true>(a, I, lo, hi, fs, dt_drift, capped, fp64_phase)
                                   : b_update<F32, false>(a, I, lo, hi, fs, dt_drift, capped, fp64_phase);
            // the exchange's barrier also publishes every CTA's new positions
            const double db = bmax((double)dmax, red);
            cl_combine<CL>(X, &db, 0, 1);
            if (X.res[0] > I.half_skin2) {
                bst = b_build(a, I, lo, hi, s_count, s_start, s_atoms, red);
                if (threadIdx.x == 0) {
                    if (bst != ST_OK && sh.status == ST_OK) sh.status = bst;
                    sh.builds += 1;
                }
            }
            E = fp64_phase ? b_forces_confirm<CL>(a, I, lo, hi, etab, et32, red)
                           : b_forces<F32, CL>(a, I, lo, hi, etab, et32, red);
            b_reduce_control<CL>(a, I, lo, hi, sh, X, E, red, t0);
        }
        // write back
        for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
            const long long gi = I.off + i;
            const dvec4 x = a.x[gi];
            double* p = a.pos_io + 3 * gi;
            p[0] = x.x;
            p[1] = x.y;
            p[2] = x.z;
            if (a.f_out) {
                const dvec4 f = a.f[gi];
                double* q = a.f_out + 3 * gi;
                q[0] = f.x;
                q[1] = f.y;
                q[2] = f.z;
            }
        }
        if (rank == 0 && threadIdx.x == 0) {
            BRes& r = a.res[sys];
            r.energy = sh.E;
            r.fmax2 = sh.fa2;
            r.F2 = sh.F2;
            r.finf = sh.fin;
            r.dt = sh.fs.dt;
            r.alpha = sh.fs.alpha;
            r.iter = sh.fs.iter;
            r.evals = sh.fs.evals;
            r.builds = sh.builds;
            r.stop = sh.fs.stop;
            r.status = sh.status;
        }
        __syncthreads();
    }
}

}  // namespace fire2

// ---------------------------------------------------------------------------
// host side

struct fire_batch_state {
    int n_sys = 0;
    long long n_total = 0;
    std::vector<long long> off;      // n_sys + 1
    BArgs args{};
    BInst* d_inst = nullptr;
    BRes* d_res = nullptr;
    int* d_order = nullptr;
    int* d_queue = nullptr;
    std::vector<BInst> inst;
    std::vector<int> order;
    long long list_slots = 0;
    fire_batch_tuning_t tune{256, 2, 0, 0};
    int sms = 0;
    size_t smem_bytes = 0;
};

// Shared host helpers implemented in fire2_api.cu.
fire_status fire2_batch_fail(fire_handle_t* h, fire_status code, const char* msg);
fire_batch_state* fire2_batch_of(fire_handle_t* h);
const PotC& fire2_potc(fire_handle_t* h);
const fire_potential_t& fire2_pot(fire_handle_t* h);
const fire_params_t& fire2_params(fire_handle_t* h);
const fire_system_t& fire2_sys(fire_handle_t* h);
double fire2_budget(fire_handle_t* h);
const double* fire2_exp_table(fire_handle_t* h);
const float* fire2_exp32_table(fire_handle_t* h);
double fire2_qscale(fire_handle_t* h);
const float* fire2_tab_ffd(fire_handle_t* h);   // NULL unless the FP64 table form
const float* fire2_tab_fff(fire_handle_t* h);
cudaStream_t fire2_stream(fire_handle_t* h);

#define BCK(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fire2_batch_fail(h, e_ == cudaErrorMemoryAllocation ? FIRE_ERR_NOMEM    \
                                                                       : FIRE_ERR_CUDA,   \
                                    cudaGetErrorString(e_));                              \
    } while (0)

#define FIRE2_HIDDEN __attribute__((visibility("hidden")))

static void free_batch(fire_batch_state* b) {
    if (!b) return;
    BArgs& a = b->args;
    void* ptrs[] = {a.x, a.v, a.f, a.xref, a.xq, a.xf, a.xq64, a.fpff, a.fp64, a.fp32, a.nbr,
                    a.nnbr, a.pos_io,
                    b->d_inst, b->d_res, b->d_order, b->d_queue};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete b;
}

FIRE2_HIDDEN void fire2_batch_free(fire_batch_state* b) { free_batch(b); }

// Geometry of every system for the given boxes; sizes the lists.
static fire_status batch_geometry(fire_handle_t* h, fire_batch_state* b, const double* boxes) {
    const fire_potential_t& pot = fire2_pot(h);
    const fire_system_t& sys = fire2_sys(h);
    const double rc = pot.rc;
    const double qscale = fire2_qscale(h);
    long long slots = 0;
    int max_cells = 1, max_atoms = 1;
    for (int s = 0; s < b->n_sys; ++s) {
        BInst& I = b->inst[s];
        I.off = b->off[s];
        I.n = (int)(b->off[s + 1] - b->off[s]);
        double skin = pot.skin;
        for (int k = 0; k < 3; ++k) {
            const double L = boxes[3 * s + k];
            if (!(L > 0.0) || !std::isfinite(L)) return fire2_batch_fail(h, FIRE_ERR_ARG, "box lengths must be > 0");
            if (sys.periodic[k] && L < 2.0 * rc)
                return fire2_batch_fail(h, FIRE_ERR_ARG, "a periodic box is shorter than twice the cut-off");
            if (sys.periodic[k]) skin = std::min(skin, 0.5 * L * (1.0 - 1e-12) - rc);
        }
        skin = std::max(skin, 0.0);
        const double rl = rc + skin;
        bool cells = true;
        double lmax = 0.0, vol = 1.0;
        for (int k = 0; k < 3; ++k) {
            const double L = boxes[3 * s + k];
            I.L[k] = L;
            I.Linv[k] = 1.0 / L;
            I.Lf[k] = (float)L;
            I.Linvf[k] = (float)(1.0 / L);
            I.per[k] = sys.periodic[k] ? 1 : 0;
            I.Lq[k] = (int)(unsigned)(unsigned long long)std::llrint(L * qscale);
            I.Lq64[k] = std::llrint(std::ldexp(L, kFixedBits64));
            // open axes take any cell count (clamped cells), periodic ones 3 or more
            I.nc[k] = std::max((int)std::floor(L / rl), I.per[k] ? 0 : 1);
            if (I.per[k] && I.nc[k] < 3) cells = false;
            lmax = std::max(lmax, L);
            vol *= L;
        }
        if (!cells) I.nc[0] = I.nc[1] = I.nc[2] = 0;
        else {
            max_cells = std::max(max_cells, I.nc[0] * I.nc[1] * I.nc[2]);
            max_atoms = std::max(max_atoms, I.n);
        }
        const double margin = 1e-3 * rc + 8.0 * 1.2e-7 * (2.0 * lmax);
        I.rlist2f = (float)((rl + margin) * (rl + margin));
        I.half_skin2 = 0.25 * skin * skin;
        const double full = 4.0 / 3.0 * M_PI * rl * rl * rl * (I.n / vol);
        I.cap = (int)std::min<long long>(std::max(I.n - 1, 1), (long long)std::ceil(1.6 * full) + 16);
        I.list_off = slots;
        slots += (long long)I.cap * I.n;
    }
    b->args.max_cells = max_cells;
    b->args.max_atoms_smem = max_atoms;
    b->smem_bytes = (size_t)(2 * max_cells + 1 + max_atoms) * sizeof(int);
    if (slots > b->list_slots) {
        cudaFree(b->args.nbr);
        b->args.nbr = nullptr;
        BCK(cudaMalloc(&b->args.nbr, (size_t)slots * sizeof(uint32_t)));
        b->list_slots = slots;
    }
    return FIRE_OK;
}

FIRE2_HIDDEN fire_status fire2_batch_create(fire_handle_t* h, int32_t n_sys,
                                            const int64_t* offsets, fire_batch_state** out) {
    fire_batch_state* b = new (std::nothrow) fire_batch_state();
    if (!b) return fire2_batch_fail(h, FIRE_ERR_NOMEM, "host allocation failed");
    b->n_sys = n_sys;
    b->off.assign(offsets, offsets + n_sys + 1);
    b->n_total = offsets[n_sys];
    b->inst.resize(n_sys);
    b->order.resize(n_sys);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
        return (offsets[x + 1] - offsets[x]) > (offsets[y + 1] - offsets[y]);
    });
    const size_t n = (size_t)b->n_total;
    BArgs& a = b->args;
    const bool f32 = fire2_pot(h).precision == FIRE_PREC_FP32_PAIR;
    auto fail_free = [&](cudaError_t e) {
        free_batch(b);
        return fire2_batch_fail(h, e == cudaErrorMemoryAllocation ? FIRE_ERR_NOMEM : FIRE_ERR_CUDA,
                                cudaGetErrorString(e));
    };
    cudaError_t e = cudaSuccess;
#define BA(ptr, bytes) \
    if (e == cudaSuccess) e = cudaMalloc(&(ptr), (bytes))
    BA(a.x, n * sizeof(dvec4));
    BA(a.v, n * sizeof(dvec4));
    BA(a.f, n * sizeof(dvec4));
    BA(a.xref, n * sizeof(dvec4));
    BA(a.xf, n * sizeof(float4));
    if (f32) {
        BA(a.xq, n * sizeof(int4));
        BA(a.fp32, n * sizeof(float));
    } else {
        BA(a.fp64, n * sizeof(double));
    }
    a.confirm = f32 && fire2_params(h).confirm64 != 0 ? 1 : 0;
    a.vmode = a.confirm ? fire2_params(h).confirm64 : 0;
    a.ff = fire2_tab_ffd(h) != nullptr && (!f32 || a.confirm) ? 1 : 0;
    if (a.ff && f32) BA(a.fp64, n * sizeof(double));
    if (a.ff) {
        BA(a.xq64, n * sizeof(lvec4));
        BA(a.fpff, n * sizeof(float2));
        a.tab_ffd = fire2_tab_ffd(h);
        a.tab_fff = fire2_tab_fff(h);
    }
    BA(a.nnbr, n * sizeof(int));
    BA(a.pos_io, 3 * n * sizeof(double));
    BA(b->d_inst, (size_t)n_sys * sizeof(BInst));
    BA(b->d_res, (size_t)n_sys * sizeof(BRes));
    BA(b->d_order, (size_t)n_sys * sizeof(int));
    BA(b->d_queue, sizeof(int));
#undef BA
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_order, b->order.data(), (size_t)n_sys * sizeof(int), cudaMemcpyHostToDevice);
    int dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail_free(e);
    *out = b;
    return FIRE_OK;
}

// Cluster size of a tuning (0 means 1).
static int cluster_of(const fire_batch_tuning_t& t) { return t.cluster_size > 1 ? t.cluster_size : 1; }

// Register budget (MAXT) a tuning runs: without clusters the smallest of
// 512, 768 and 1024 threads per SM that holds threads_per_block x
// ctas_per_sm, else 512 (fewer CTAs are then resident than asked for);
// clusters always 512.
static int maxt_of(const fire_batch_tuning_t& t) {
    const int per_sm = t.threads_per_block * t.ctas_per_sm;
    if (cluster_of(t) != 1 || per_sm <= 512 || per_sm > 1024) return 512;
    return per_sm <= 768 ? 768 : 1024;
}

template <bool F32, int MAXT>
static fire_status launch_plain(fire_batch_state* b, int grid, int threads, cudaStream_t s) {
    if (cudaFuncSetAttribute(k_batch_relax<F32, false, MAXT>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)b->smem_bytes) != cudaSuccess)
        return FIRE_ERR_CUDA;
    k_batch_relax<F32, false, MAXT><<<grid, threads, b->smem_bytes, s>>>(b->args);
    return cudaGetLastError() == cudaSuccess ? FIRE_OK : FIRE_ERR_CUDA;
}

// Launches the batched kernel with b->tune: plain launch, or cluster launch
// with the grid a multiple of the cluster size.
template <bool F32>
static fire_status launch_shape(fire_handle_t* h, fire_batch_state* b, cudaStream_t s) {
    const int threads = b->tune.threads_per_block;
    const int C = cluster_of(b->tune);
    const BArgs& a = b->args;
    if (C == 1) {
        const int grid = std::max(1, std::min(b->n_sys, b->sms * b->tune.ctas_per_sm));
        const int mt = maxt_of(b->tune);
        const fire_status st = mt == 768    ? launch_plain<F32, 768>(b, grid, threads, s)
                               : mt == 1024 ? launch_plain<F32, 1024>(b, grid, threads, s)
                                            : launch_plain<F32, 512>(b, grid, threads, s);
        if (st != FIRE_OK) {
            const cudaError_t e = cudaGetLastError();
            return fire2_batch_fail(h, FIRE_ERR_CUDA, cudaGetErrorString(e));
        }
        return FIRE_OK;
    }
    const int clusters = std::max(1, std::min(b->n_sys, b->sms * b->tune.ctas_per_sm / C));
    BCK(cudaFuncSetAttribute(k_batch_relax<F32, true, 512>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem_bytes));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(clusters * C), 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = b->smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    BCK(cudaLaunchKernelEx(&cfg, k_batch_relax<F32, true, 512>, a));
    return FIRE_OK;
}

// Whether clusters of the tuning's size and shape can be co-scheduled.
template <bool F32>
static bool cluster_fits(const fire_batch_state* b, const fire_batch_tuning_t& t) {
    const int C = cluster_of(t);
    if (C == 1) return true;
    if (cudaFuncSetAttribute(k_batch_relax<F32, true, 512>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)b->smem_bytes) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C, 1, 1);
    cfg.blockDim = dim3((unsigned)t.threads_per_block, 1, 1);
    cfg.dynamicSmemBytes = b->smem_bytes;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_batch_relax<F32, true, 512>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n > 0;
}

// Launches one batched relaxation with the current tuning (asynchronous).
static fire_status batch_launch(fire_handle_t* h, fire_batch_state* b, double ftol,
                                int64_t maxiter, double* d_fout, cudaStream_t s) {
    BArgs& a = b->args;
    a.n_sys = b->n_sys;
    a.order = b->d_order;
    a.queue = b->d_queue;
    a.inst = b->d_inst;
    a.res = b->d_res;
    a.f_out = d_fout;
    const fire_params_t& p = fire2_params(h);
    FireParamsD& q = a.prm;
    std::memset(&q, 0, sizeof q);
    q.ftol = ftol;
    q.maxiter = maxiter;
    q.dt_start = p.dt_start;
    q.dtmax = p.tmax * p.dt_start;
    q.dtmin = p.tmin * p.dt_start;
    q.dtgrow = p.dtgrow;
    q.dtshrink = p.dtshrink;
    q.alpha0 = p.alpha0;
    q.alphashrink = p.alphashrink;
    q.mass = fire2_sys(h).mass;
    q.delaystep = p.delaystep;
    q.vdfmax = p.vdfmax;
    q.halfstepback = p.halfstepback;
    q.initialdelay = p.initialdelay;
    q.norm = p.norm;
    q.integrator = p.integrator;
    q.variant = p.variant;
    q.dmax = p.dmax;
    a.budget_ns = (unsigned long long)(fire2_budget(h) * 1e9);
    a.P = fire2_potc(h);
    a.exp_table = fire2_exp_table(h);
    a.exp32_table = fire2_exp32_table(h);
    a.qscale = fire2_qscale(h);
    const bool f32 = fire2_pot(h).precision == FIRE_PREC_FP32_PAIR;
    BCK(cudaMemcpyAsync(b->d_inst, b->inst.data(), (size_t)b->n_sys * sizeof(BInst),
                        cudaMemcpyHostToDevice, s));
    BCK(cudaMemsetAsync(b->d_queue, 0, sizeof(int), s));
    if (f32) return launch_shape<true>(h, b, s);
    return launch_shape<false>(h, b, s);
}

static fire_status batch_collect(fire_handle_t* h, fire_batch_state* b, fire_result_t* out,
                                 cudaStream_t s) {
    std::vector<BRes> res(b->n_sys);
    BCK(cudaMemcpyAsync(res.data(), b->d_res, (size_t)b->n_sys * sizeof(BRes),
                        cudaMemcpyDeviceToHost, s));
    BCK(cudaStreamSynchronize(s));
    int worst = ST_OK;
    for (int k = 0; k < b->n_sys; ++k) {
        const BRes& r = res[k];
        if (r.status != ST_OK && worst == ST_OK) worst = r.status;
        if (out) {
            fire_result_t& o = out[k];
            o.energy = r.energy;
            o.iterations = r.iter;
            o.force_evals = r.evals;
            o.nbr_builds = r.builds;
            o.stop = r.stop;
            o.reserved = r.status;
            o.fmax_atom = std::sqrt(r.fmax2);
            o.f2norm = std::sqrt(r.F2);
            o.finf = r.finf;
            o.dt_final = r.dt;
            o.alpha_final = r.alpha;
        }
    }
    switch (worst) {
        case ST_OK: return FIRE_OK;
        case ST_NONFINITE: return fire2_batch_fail(h, FIRE_ERR_NONFINITE, "non-finite force, energy or position in a system");
        case ST_NBR_OVERFLOW: return fire2_batch_fail(h, FIRE_ERR_NBR_OVERFLOW, "neighbour list overflow in a system");
        case ST_TIMEOUT: return fire2_batch_fail(h, FIRE_ERR_TIMEOUT, "a relaxation exceeded the time budget");
        case ST_RANGE: return fire2_batch_fail(h, FIRE_ERR_ARG, "positions lie more than one box length outside their box");
        default: return fire2_batch_fail(h, FIRE_ERR_CUDA, "unknown device status");
    }
}

extern "C" {

fire_status fire_minimize_batch_dev(fire_handle_t* h, double* d_pos, const double* boxes,
                                    double ftol, int64_t maxiter, fire_result_t* out,
                                    double* d_forces, void* stream) {
    fire_batch_state* b = h ? fire2_batch_of(h) : nullptr;
    if (!b) return h ? fire2_batch_fail(h, FIRE_ERR_STATE, "handle was not created by fire_batch_init")
                     : FIRE_ERR_ARG;
    if (!d_pos || !boxes || !out) return fire2_batch_fail(h, FIRE_ERR_ARG, "NULL argument");
    if (!(ftol >= 0.0) || maxiter < 0) return fire2_batch_fail(h, FIRE_ERR_ARG, "need ftol >= 0 and maxiter >= 0");
    fire_status st = batch_geometry(h, b, boxes);
    if (st != FIRE_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)3 * b->n_total * sizeof(double);
    BCK(cudaMemcpyAsync(b->args.pos_io, d_pos, bytes, cudaMemcpyDeviceToDevice, s));
    st = batch_launch(h, b, ftol, maxiter, d_forces, s);
    if (st != FIRE_OK) return st;
    st = batch_collect(h, b, out, s);
    if (st != FIRE_OK) return st;
    BCK(cudaMemcpyAsync(d_pos, b->args.pos_io, bytes, cudaMemcpyDeviceToDevice, s));
    BCK(cudaStreamSynchronize(s));
    return FIRE_OK;
}

fire_status fire_minimize_batch(fire_handle_t* h, double* pos, const double* boxes, double ftol,
                                int64_t maxiter, fire_result_t* out, double* forces) {
    fire_batch_state* b = h ? fire2_batch_of(h) : nullptr;
    if (!b) return h ? fire2_batch_fail(h, FIRE_ERR_STATE, "handle was not created by fire_batch_init")
                     : FIRE_ERR_ARG;
    if (!pos || !boxes || !out) return fire2_batch_fail(h, FIRE_ERR_ARG, "NULL argument");
    if (!(ftol >= 0.0) || maxiter < 0) return fire2_batch_fail(h, FIRE_ERR_ARG, "need ftol >= 0 and maxiter >= 0");
    fire_status st = batch_geometry(h, b, boxes);
    if (st != FIRE_OK) return st;
    cudaStream_t s = fire2_stream(h);
    const size_t bytes = (size_t)3 * b->n_total * sizeof(double);
    double* d_f = nullptr;
    if (forces) BCK(cudaMalloc(&d_f, bytes));
    BCK(cudaMemcpyAsync(b->args.pos_io, pos, bytes, cudaMemcpyHostToDevice, s));
    st = batch_launch(h, b, ftol, maxiter, d_f, s);
    if (st == FIRE_OK) st = batch_collect(h, b, out, s);
    if (st == FIRE_OK) {
        std::vector<double> tmp((size_t)3 * b->n_total);
        cudaError_t e = cudaMemcpy(tmp.data(), b->args.pos_io, bytes, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && forces) e = cudaMemcpy(forces, d_f, bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = fire2_batch_fail(h, FIRE_ERR_CUDA, cudaGetErrorString(e));
        else std::memcpy(pos, tmp.data(), bytes);
    }
    if (d_f) cudaFree(d_f);
    return st;
}

fire_status fire_batch_set_tuning(fire_handle_t* h, const fire_batch_tuning_t* t) {
    fire_batch_state* b = h ? fire2_batch_of(h) : nullptr;
    if (!b) return h ? fire2_batch_fail(h, FIRE_ERR_STATE, "handle was not created by fire_batch_init")
                     : FIRE_ERR_ARG;
    if (!t || t->threads_per_block < 32 || t->threads_per_block > 1024 ||
        t->threads_per_block % 32 != 0 || t->ctas_per_sm < 1 || t->ctas_per_sm > 32)
        return fire2_batch_fail(h, FIRE_ERR_ARG, "threads_per_block must be a multiple of 32 in "
                                                 "[32, 1024] and ctas_per_sm in [1, 32]");
    const int C = cluster_of(*t);
    if (C != 1 && C != 2 && C != 4 && C != 8)
        return fire2_batch_fail(h, FIRE_ERR_ARG, "cluster_size must be 0, 1, 2, 4 or 8");
    if (t->threads_per_block > maxt_of(*t))
        return fire2_batch_fail(h, FIRE_ERR_ARG, "more than 512 threads per CTA needs no "
                                                 "cluster and at most 1024 threads per SM "
                                                 "in all");
    const bool f32 = fire2_pot(h).precision == FIRE_PREC_FP32_PAIR;
    if (!(f32 ? cluster_fits<true>(b, *t) : cluster_fits<false>(b, *t)))
        return fire2_batch_fail(h, FIRE_ERR_ARG, "clusters of this size and shape cannot be "
                                                 "co-scheduled on this device");
    b->tune = *t;
    return FIRE_OK;
}

fire_status fire_batch_autotune(fire_handle_t* h, const double* pos, const double* boxes,
                                int32_t iters, fire_batch_tuning_t* chosen) {
    fire_batch_state* b = h ? fire2_batch_of(h) : nullptr;
    if (!b) return h ? fire2_batch_fail(h, FIRE_ERR_STATE, "handle was not created by fire_batch_init")
                     : FIRE_ERR_ARG;
    if (!pos || !boxes || iters < 1) return fire2_batch_fail(h, FIRE_ERR_ARG, "need pos, boxes, iters >= 1");
    fire_status st = batch_geometry(h, b, boxes);
    if (st != FIRE_OK) return st;
    cudaStream_t s = fire2_stream(h);
    const size_t bytes = (size_t)3 * b->n_total * sizeof(double);
    double* d_src = nullptr;
    BCK(cudaMalloc(&d_src, bytes));
    BCK(cudaMemcpy(d_src, pos, bytes, cudaMemcpyHostToDevice));
    // (threads, CTAs per SM, cluster): CTAs of 64..512 threads, 1..8 per SM
    // (each shape runs the register budget maxt_of gives it), clusters of 1,
    // 2 and 4; then 768 threads per SM in CTAs of 768, 384, 256, 192, 128,
    // and one CTA of 1024
    std::vector<fire_batch_tuning_t> cands;
    for (int th : {64, 128, 256, 512})
        for (int C : {1, 2, 4})
            for (int c : {1, 2, 4, 8})
                if (th * c <= 2048) cands.push_back({th, c, C, 0});
    for (int th : {768, 384, 256, 192, 128}) cands.push_back({th, 768 / th, 1, 0});
    cands.push_back({1024, 1, 1, 0});
    const bool f32 = fire2_pot(h).precision == FIRE_PREC_FP32_PAIR;
    const fire_batch_tuning_t saved = b->tune;
    double best = 1e300;
    fire_batch_tuning_t best_t = saved;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (const fire_batch_tuning_t& t : cands) {
        b->tune = t;
        if (!(f32 ? cluster_fits<true>(b, b->tune) : cluster_fits<false>(b, b->tune))) continue;
        cudaMemcpyAsync(b->args.pos_io, d_src, bytes, cudaMemcpyDeviceToDevice, s);
        cudaEventRecord(e0, s);
        st = batch_launch(h, b, 0.0, iters, nullptr, s);   // ftol = 0: every system runs `iters`
        cudaEventRecord(e1, s);
        if (st != FIRE_OK) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            st = fire2_batch_fail(h, FIRE_ERR_CUDA, "autotune launch failed");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_t = b->tune;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(d_src);
    if (st != FIRE_OK) {
        b->tune = saved;
        return st;
    }
    b->tune = best_t;
    if (chosen) *chosen = best_t;
    return FIRE_OK;
}

}  // extern "C"
