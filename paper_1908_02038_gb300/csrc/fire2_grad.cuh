// Differentiable form (RGL, FP64): energy gradient with respect to the
// potential parameters theta = (A, xi, p, q), theta-derivatives of the
// forces, the Hessian-vector product, and the vector kernels of the
// projected conjugate-gradient solve for the implicit gradient of a relaxed
// configuration.  All kernels walk a full neighbour list, one thread per
// atom, without atomics.
//
// Notation (per pair, d = x_j - x_i, r = |d|, s = r/r0 - 1):
//   phi = A e^{-p s} S,  g = xi^2 e^{-2q s} S,  rho_i = sum_j g,
//   F'_i = -1/(2 sqrt rho_i),  F''_i = 1/(4 rho_i^{3/2}),
//   F_i  = sum_j fs d,  fs = [2 phi'(r) + (F'_i + F'_j) g'(r)] / r.
// At a minimum x*(theta) the forces vanish, so dx*/dtheta = H^{-1} dF/dtheta
// and dL/dtheta = lambda . dF/dtheta with H lambda = dL/dx.
#pragma once

#include "fire2_common.cuh"

namespace fire2 {

struct GeoL {
    double L[3];
};

struct GradBufs {
    int n, cap;
    const dvec4* x;
    const uint32_t* nbr;
    const int* nnbr;
    double *rho, *F1, *F2, *drho, *dq;
    double* part;          // block partials
    // pair coefficients of the HVP at fixed positions (k_g_pair_cache), one
    // per list slot [k * n + i]; NULL when not computed
    const double *w1, *fsc, *a2;
    const double *dcx, *dcy, *dcz;   // cached separation x_j - x_i per list slot
};

struct Pair2 {
    double r, rinv, s, ep, eq, S, dS, d2S;
    double phi, dphi, d2phi, g, dg, d2g;
};

// Pair terms with first and second derivatives in r (FP64).
__device__ __forceinline__ void rgl_pair_d2(const PotC& P, double r2, const double* etab,
                                            Pair2& q) {
    q.rinv = rsqrt(r2);
    q.r = r2 * q.rinv;
    q.s = q.r * P.r0inv - 1.0;
    q.ep = exp_tang(-P.p * q.s, P.ex, etab);
    q.eq = exp_tang(-P.q2 * q.s, P.ex, etab);
    q.S = 1.0;
    q.dS = 0.0;
    q.d2S = 0.0;
    if (q.r > P.rs) {
        const double t = (q.r - P.rs) * P.winv;
        const double t2 = t * t, t3 = t2 * t;
        q.S = 1.0 - 10.0 * t3 + 15.0 * t3 * t - 6.0 * t3 * t2;
        q.dS = (-30.0 * t2 + 60.0 * t3 - 30.0 * t3 * t) * P.winv;
        q.d2S = (-60.0 * t + 180.0 * t2 - 120.0 * t3) * P.winv * P.winv;
    }
    const double a = P.p_r0, b = P.q2_r0;
    const double Ae = P.A * q.ep, Xe = P.xi2 * q.eq;
    q.phi = Ae * q.S;
    q.dphi = Ae * (-a * q.S + q.dS);
    q.d2phi = Ae * (a * a * q.S - 2.0 * a * q.dS + q.d2S);
    q.g = Xe * q.S;
    q.dg = Xe * (-b * q.S + q.dS);
    q.d2g = Xe * (b * b * q.S - 2.0 * b * q.dS + q.d2S);
}

// Minimum-image pair vector of list slot e (full list) from atom i.
__device__ __forceinline__ double grad_pair_vec(const GradBufs& g, const double3* tbl, dvec4 xi,
                                                uint32_t e, int& j, double& dx, double& dy,
                                                double& dz) {
    j = (int)(e & kIdxMask);
    const int code = (int)(e >> kIdxBits);
    const dvec4 xj = g.x[j];
    dx = xj.x - xi.x;
    dy = xj.y - xi.y;
    dz = xj.z - xi.z;
    if (code != kCodeZero) {
        const double3 s = tbl[code];
        dx -= s.x;
        dy -= s.y;
        dz -= s.z;
    }
    return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ void grad_tables(double3* tbl, double* etab, const double* exp_table,
                                            const double L[3]) {
    for (int t = threadIdx.x; t < 125; t += blockDim.x) {
        const int sx = t % 5 - 2, sy = (t / 5) % 5 - 2, sz = t / 25 - 2;
        tbl[t] = make_double3(sx * L[0], sy * L[1], sz * L[2]);
    }
    for (int t = threadIdx.x; t < kExpTableSize; t += blockDim.x) etab[t] = exp_table[t];
}

// Pass 1: rho_i, F'_i, F''_i, drho_i/dq; per-block partial sums of
// E, dE/dA, dE/dxi, dE/dp, dE/dq into part[k * gridDim.x + block].
__global__ void __launch_bounds__(kForceBlock) k_g_atom(GradBufs g, PotC P, GeoL L,
                                                        const double* exp_table) {
    __shared__ double3 tbl[125];
    __shared__ double etab[kExpTableSize];
    __shared__ double red[32];
    grad_tables(tbl, etab, exp_table, L.L);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double E = 0.0, eA = 0.0, eX = 0.0, eP = 0.0, eQ = 0.0;
    if (i < g.n) {
        const dvec4 xi = g.x[i];
        double rho = 0.0, dq = 0.0, erep = 0.0, sA = 0.0, sP = 0.0;
        const int m = g.nnbr[i];
        for (int k = 0; k < m; ++k) {
            int j;
            double dx, dy, dz;
            const double r2 = grad_pair_vec(g, tbl, xi, g.nbr[(size_t)k * g.n + i], j, dx, dy, dz);
            if (!(r2 < P.rc2)) continue;
            Pair2 q;
            rgl_pair_d2(P, r2, etab, q);
            rho += q.g;
            dq += -2.0 * q.s * q.g;
            erep += q.phi;
            sA += q.ep * q.S;
            sP += -q.s * q.phi;
        }
        const double sq = sqrt(rho);
        const double f1 = rho > 0.0 ? -0.5 / sq : 0.0;
        g.rho[i] = rho;
        g.F1[i] = f1;
        g.F2[i] = rho > 0.0 ? 0.25 / (rho * sq) : 0.0;
        g.dq[i] = dq;
        E = erep - sq;
        eA = sA;
        eX = f1 * 2.0 * rho * P.xi_inv;
        eP = sP;
        eQ = f1 * dq;
    }
    const int nb = gridDim.x;
    double r;
    r = block_sum(E, red);
    if (threadIdx.x == 0) g.part[0 * nb + blockIdx.x] = r;
    r = block_sum(eA, red);
    if (threadIdx.x == 0) g.part[1 * nb + blockIdx.x] = r;
    r = block_sum(eX, red);
    if (threadIdx.x == 0) g.part[2 * nb + blockIdx.x] = r;
    r = block_sum(eP, red);
    if (threadIdx.x == 0) g.part[3 * nb + blockIdx.x] = r;
    r = block_sum(eQ, red);
    if (threadIdx.x == 0) g.part[4 * nb + blockIdx.x] = r;
}

// Pass 2: F_i (f_out, row-major, optional), dF_i/dtheta_k (dF_out[k * 3N +
// 3 i + a], optional) and, with lam != NULL, per-block partials of
// sum_i lam_i . dF_i/dtheta_k into part[(5 + k) * gridDim.x + block].
__global__ void __launch_bounds__(kForceBlock) k_g_force(GradBufs g, PotC P, GeoL L,
                                                         const double* exp_table, double* f_out,
                                                         double* dF_out, const double* lam) {
    __shared__ double3 tbl[125];
    __shared__ double etab[kExpTableSize];
    __shared__ double red[32];
    grad_tables(tbl, etab, exp_table, L.L);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double dots[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < g.n) {
        const dvec4 xi = g.x[i];
        const double f1i = g.F1[i], dcq_i = g.F2[i] * g.dq[i];
        double F[3] = {0, 0, 0}, dA[3] = {0, 0, 0}, dX[3] = {0, 0, 0}, dP[3] = {0, 0, 0},
               dQ[3] = {0, 0, 0};
        const int m = g.nnbr[i];
        for (int k = 0; k < m; ++k) {
            int j;
            double d[3];
            const double r2 = grad_pair_vec(g, tbl, xi, g.nbr[(size_t)k * g.n + i], j, d[0], d[1], d[2]);
            if (!(r2 < P.rc2)) continue;
            Pair2 q;
            rgl_pair_d2(P, r2, etab, q);
            const double c = f1i + g.F1[j];
            const double fs = (2.0 * q.dphi + c * q.dg) * q.rinv;
            const double dphi_dp = -q.s * q.dphi - P.A * q.ep * q.S * P.r0inv;
            const double dg_dq = -2.0 * q.s * q.dg - 2.0 * P.xi2 * q.eq * q.S * P.r0inv;
            const double dc_dq = dcq_i + g.F2[j] * g.dq[j];
            const double wA = 2.0 * q.ep * (-P.p_r0 * q.S + q.dS) * q.rinv;   // d(2 phi')/dA / r
            const double wX = c * q.dg * P.xi_inv * q.rinv;
            const double wP = 2.0 * dphi_dp * q.rinv;
            const double wQ = (dc_dq * q.dg + c * dg_dq) * q.rinv;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                F[a] += fs * d[a];
                dA[a] += wA * d[a];
                dX[a] += wX * d[a];
                dP[a] += wP * d[a];
                dQ[a] += wQ * d[a];
            }
        }
        if (f_out)
            for (int a = 0; a < 3; ++a) f_out[3 * (size_t)i + a] = F[a];
        if (dF_out) {
            const size_t m3 = 3 * (size_t)g.n;
            for (int a = 0; a < 3; ++a) {
                dF_out[0 * m3 + 3 * (size_t)i + a] = dA[a];
                dF_out[1 * m3 + 3 * (size_t)i + a] = dX[a];
                dF_out[2 * m3 + 3 * (size_t)i + a] = dP[a];
                dF_out[3 * m3 + 3 * (size_t)i + a] = dQ[a];
            }
        }
        if (lam) {
            const double* l = lam + 3 * (size_t)i;
            dots[0] = l[0] * dA[0] + l[1] * dA[1] + l[2] * dA[2];
            dots[1] = l[0] * dX[0] + l[1] * dX[1] + l[2] * dX[2];
            dots[2] = l[0] * dP[0] + l[1] * dP[1] + l[2] * dP[2];
            dots[3] = l[0] * dQ[0] + l[1] * dQ[1] + l[2] * dQ[2];
        }
    }
    if (lam) {
        const int nb = gridDim.x;
        for (int k = 0; k < 4; ++k) {
            const double r = block_sum(dots[k], red);
            if (threadIdx.x == 0) g.part[(5 + k) * nb + blockIdx.x] = r;
        }
    }
}

// HVP pass 1: drho_i = sum_j g'(r) d.(u_j - u_i) / r; TPA threads per atom
// (group_sum), as in the cached passes.
template <int TPA>
__global__ void __launch_bounds__(kForceBlock) k_g_hvp1(GradBufs g, PotC P, GeoL L,
                                                        const double* exp_table, const double* u) {
    __shared__ double3 tbl[125];
    __shared__ double etab[kExpTableSize];
    grad_tables(tbl, etab, exp_table, L.L);
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / TPA, lane = t % TPA;
    if (i >= g.n) return;
    const dvec4 xi = g.x[i];
    const double* ui = u + 3 * (size_t)i;
    double acc = 0.0;
    const int m = g.nnbr[i];
    for (int k = lane; k < m; k += TPA) {
        int j;
        double dx, dy, dz;
        const double r2 = grad_pair_vec(g, tbl, xi, g.nbr[(size_t)k * g.n + i], j, dx, dy, dz);
        if (!(r2 < P.rc2)) continue;
        Pair2 q;
        rgl_pair_d2(P, r2, etab, q);
        const double* uj = u + 3 * (size_t)j;
        const double dr = (dx * (uj[0] - ui[0]) + dy * (uj[1] - ui[1]) + dz * (uj[2] - ui[2])) * q.rinv;
        acc += q.dg * dr;
    }
    acc = group_sum<TPA>(acc);
    if (lane == 0) g.drho[i] = acc;
}

// HVP pass 2: (H u)_i = -dF_i with
// dF_i = sum_j [dfs d + fs (u_j - u_i)],
// dfs = [(2 phi'' + c g'')/r - fs/r] dr + (F''_i drho_i + F''_j drho_j) g'/r.
template <int TPA>
__global__ void __launch_bounds__(kForceBlock) k_g_hvp2(GradBufs g, PotC P, GeoL L,
                                                        const double* exp_table, const double* u,
                                                        double* hu) {
    __shared__ double3 tbl[125];
    __shared__ double etab[kExpTableSize];
    grad_tables(tbl, etab, exp_table, L.L);
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / TPA, lane = t % TPA;
    if (i >= g.n) return;
    const dvec4 xi = g.x[i];
    const double* ui = u + 3 * (size_t)i;
    const double f1i = g.F1[i], dci = g.F2[i] * g.drho[i];
    double dF[3] = {0, 0, 0};
    const int m = g.nnbr[i];
    for (int k = lane; k < m; k += TPA) {
        int j;
        double d[3];
        const double r2 = grad_pair_vec(g, tbl, xi, g.nbr[(size_t)k * g.n + i], j, d[0], d[1], d[2]);
        if (!(r2 < P.rc2)) continue;
        Pair2 q;
        rgl_pair_d2(P, r2, etab, q);
        const double* uj = u + 3 * (size_t)j;
        const double du[3] = {uj[0] - ui[0], uj[1] - ui[1], uj[2] - ui[2]};
        const double c = f1i + g.F1[j];
        const double fs = (2.0 * q.dphi + c * q.dg) * q.rinv;
        const double dr = (d[0] * du[0] + d[1] * du[1] + d[2] * du[2]) * q.rinv;
        const double dc = dci + g.F2[j] * g.drho[j];
        const double dfs = ((2.0 * q.d2phi + c * q.d2g) * q.rinv - fs * q.rinv) * dr + dc * q.dg * q.rinv;
#pragma unroll
        for (int a = 0; a < 3; ++a) dF[a] += dfs * d[a] + fs * du[a];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) dF[a] = group_sum<TPA>(dF[a]);
    if (lane != 0) return;
    double* h = hu + 3 * (size_t)i;
    h[0] = -dF[0];
    h[1] = -dF[1];
    h[2] = -dF[2];
}

// Pair coefficients of the HVP at the current positions, for the many
// products of one conjugate-gradient solve (the positions do not change):
// per list slot w1 = g'/r, fs = [2 phi' + (F'_i + F'_j) g'] / r and
// a2 = [2 phi'' + (F'_i + F'_j) g'' - fs] / r^2, zero beyond rc.  With them
// dfs = a2 d.(u_j - u_i) + (F''_i drho_i + F''_j drho_j) w1 (HVP pass 2) and
// drho_i = sum_j w1 d.(u_j - u_i) (pass 1) need no pair function.  The
// separation d = x_j - x_i of each slot is cached too: the HVP passes then
// stream it instead of gathering x_j and redoing the minimum image (six FP64
// instructions per pair and pass at 1/58 of the FP32 rate).
__global__ void __launch_bounds__(kForceBlock) k_g_pair_cache(GradBufs g, PotC P, GeoL L,
                                                              const double* exp_table,
                                                              double* w1, double* fsc,
                                                              double* a2, double* dcx,
                                                              double* dcy, double* dcz) {
    __shared__ double3 tbl[125];
    __shared__ double etab[kExpTableSize];
    grad_tables(tbl, etab, exp_table, L.L);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const dvec4 xi = g.x[i];
    const double f1i = g.F1[i];
    const int m = g.nnbr[i];
    for (int k = 0; k < m; ++k) {
        const size_t slot = (size_t)k * g.n + i;
        int j;
        double dx, dy, dz;
        const double r2 = grad_pair_vec(g, tbl, xi, g.nbr[slot], j, dx, dy, dz);
        dcx[slot] = dx;
        dcy[slot] = dy;
        dcz[slot] = dz;
        if (!(r2 < P.rc2)) {
            w1[slot] = 0.0;
            fsc[slot] = 0.0;
            a2[slot] = 0.0;
            continue;
        }
        Pair2 q;
        rgl_pair_d2(P, r2, etab, q);
        const double c = f1i + g.F1[j];
        const double fs = (2.0 * q.dphi + c * q.dg) * q.rinv;
        w1[slot] = q.dg * q.rinv;
        fsc[slot] = fs;
        a2[slot] = (2.0 * q.d2phi + c * q.d2g - fs) * q.rinv * q.rinv;
    }
}

// HVP pass 1 from the pair cache.
template <int TPA>
__global__ void __launch_bounds__(kForceBlock) k_g_hvp1c(GradBufs g, const double* u,
                                                         const int* skip) {
    if (skip && *skip) return;   // a finished conjugate-gradient solve
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / TPA, lane = t % TPA;   // TPA threads per atom (group_sum)
    if (i >= g.n) return;
    const double* ui = u + 3 * (size_t)i;
    double acc = 0.0;
    const int m = g.nnbr[i];
    for (int k = lane; k < m; k += TPA) {
        const size_t slot = (size_t)k * g.n + i;
        const double w = g.w1[slot];
        if (w == 0.0) continue;
        const int j = (int)(g.nbr[slot] & kIdxMask);
        const double dx = g.dcx[slot], dy = g.dcy[slot], dz = g.dcz[slot];
        const double* uj = u + 3 * (size_t)j;
        acc += w * (dx * (uj[0] - ui[0]) + dy * (uj[1] - ui[1]) + dz * (uj[2] - ui[2]));
    }
    acc = group_sum<TPA>(acc);
    if (lane == 0) g.drho[i] = acc;
}

// HVP pass 2 from the pair cache: (H u)_i = -dF_i.
template <int TPA>
__global__ void __launch_bounds__(kForceBlock) k_g_hvp2c(GradBufs g, const double* u, double* hu,
                                                         const int* skip) {
    if (skip && *skip) return;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = t / TPA, lane = t % TPA;
    if (i >= g.n) return;
    const double* ui = u + 3 * (size_t)i;
    const double dci = g.F2[i] * g.drho[i];
    double dF[3] = {0, 0, 0};
    const int m = g.nnbr[i];
    for (int k = lane; k < m; k += TPA) {
        const size_t slot = (size_t)k * g.n + i;
        const double fs = g.fsc[slot];
        if (fs == 0.0 && g.w1[slot] == 0.0) continue;
        const int j = (int)(g.nbr[slot] & kIdxMask);
        const double d[3] = {g.dcx[slot], g.dcy[slot], g.dcz[slot]};
        const double* uj = u + 3 * (size_t)j;
        const double du[3] = {uj[0] - ui[0], uj[1] - ui[1], uj[2] - ui[2]};
        const double dd = d[0] * du[0] + d[1] * du[1] + d[2] * du[2];
        const double dfs = g.a2[slot] * dd + (dci + g.F2[j] * g.drho[j]) * g.w1[slot];
#pragma unroll
        for (int a = 0; a < 3; ++a) dF[a] += dfs * d[a] + fs * du[a];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) dF[a] = group_sum<TPA>(dF[a]);
    if (lane != 0) return;
    double* h = hu + 3 * (size_t)i;
    h[0] = -dF[0];
    h[1] = -dF[1];
    h[2] = -dF[2];
}

// Row-major positions into the padded layout used by the list build.
__global__ void k_g_load(int n, const double* pos, dvec4* x, float4* xf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* p = pos + 3 * (size_t)i;
    x[i] = make_dvec4(p[0], p[1], p[2], 0.0);
    xf[i] = make_float4((float)p[0], (float)p[1], (float)p[2], 0.f);
}

// ---- vector kernels of the conjugate-gradient solve (3N vectors) ----------

// Per-block partial sums of a.b and of the three Cartesian column sums of a.
__global__ void k_g_dot(int n, const double* a, const double* b, double* part) {
    __shared__ double red[32];
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < 3 * n; i += gridDim.x * blockDim.x)
        s += a[i] * b[i];
    s = block_sum(s, red);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_g_colsum(int n, const double* a, double* part) {
    __shared__ double red[32];
    double c[3] = {0.0, 0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        c[0] += a[3 * (size_t)i];
        c[1] += a[3 * (size_t)i + 1];
        c[2] += a[3 * (size_t)i + 2];
    }
    for (int k = 0; k < 3; ++k) {
        const double s = block_sum(c[k], red);
        if (threadIdx.x == 0) part[k * gridDim.x + blockIdx.x] = s;
    }
}

__global__ void k_g_sub_mean(int n, double* a, double m0, double m1, double m2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        a[3 * (size_t)i] -= m0;
        a[3 * (size_t)i + 1] -= m1;
        a[3 * (size_t)i + 2] -= m2;
    }
}

// Scalars of the conjugate-gradient solve, kept on the device so that the
// iterations run without a host round trip; every kernel of an iteration
// returns at once when the solve is done (done = 1), so the host can queue
// several iterations and look at the state once per batch.
// Why the solve stopped (CgState::reason).
enum CgReason { CG_RUNNING = 0, CG_CONVERGED = 1, CG_BREAKDOWN = 2, CG_MAXIT = 3 };

struct CgState {
    double rr, stop2, alpha, beta, m[3];
    long long it, maxit;
    int done;
    int reason;            // CgReason
};

// Fixed-order sum of cnt partials by one block (result in thread 0).
__device__ __forceinline__ double cg_sum(const double* a, int cnt, double* red) {
    double s = 0.0;
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) s += a[k];
    return block_sum(s, red);
}

// Column sums of Ap, as partials (k_g_colsum), unless the solve is done.
__global__ void k_cg_colsum(int n, const CgState* cs, const double* a, double* part) {
    __shared__ double red[32];
    if (cs->done) return;
    double c[3] = {0.0, 0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        c[0] += a[3 * (size_t)i];
        c[1] += a[3 * (size_t)i + 1];
        c[2] += a[3 * (size_t)i + 2];
    }
    for (int k = 0; k < 3; ++k) {
        const double s = block_sum(c[k], red);
        if (threadIdx.x == 0) part[k * gridDim.x + blockIdx.x] = s;
    }
}

// One block: the mean of each Cartesian column of Ap (the translations that
// are projected out, H being singular along them).
__global__ void k_cg_means(CgState* cs, const double* part, int nb, int n) {
    __shared__ double red[32];
    if (cs->done) return;
    for (int k = 0; k < 3; ++k) {
        const double s = cg_sum(part + (size_t)k * nb, nb, red);
        if (threadIdx.x == 0) cs->m[k] = s / n;
    }
}

// Ap -= its column means; partials of p.Ap.
__global__ void k_cg_project_dot(int n, const CgState* cs, double* ap, const double* p,
                                 double* part) {
    __shared__ double red[32];
    if (cs->done) return;
    const double m0 = cs->m[0], m1 = cs->m[1], m2 = cs->m[2];
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const size_t k = 3 * (size_t)i;
        const double a0 = ap[k] - m0, a1 = ap[k + 1] - m1, a2 = ap[k + 2] - m2;
        ap[k] = a0;
        ap[k + 1] = a1;
        ap[k + 2] = a2;
        acc += p[k] * a0 + p[k + 1] * a1 + p[k + 2] * a2;
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// One block: alpha = r.r / p.Ap; stops (CG_BREAKDOWN) when H is not
// positive definite along p or p.Ap is not finite.
__global__ void k_cg_alpha(CgState* cs, const double* part, int nb) {
    __shared__ double red[32];
    if (cs->done) return;
    const double pAp = cg_sum(part, nb, red);
    if (threadIdx.x == 0) {
        if (!(pAp > 0.0) || !isfinite(pAp)) {
            cs->done = 1;
            cs->reason = CG_BREAKDOWN;
        } else {
            cs->alpha = cs->rr / pAp;
        }
    }
}

// lam += alpha p; r -= alpha Ap; partials of r.r.
__global__ void k_cg_step(int m, const CgState* cs, const double* p, const double* Ap,
                          double* lam, double* r, double* part) {
    __shared__ double red[32];
    if (cs->done) return;
    const double alpha = cs->alpha;
    double acc = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        lam[i] += alpha * p[i];
        const double ri = r[i] - alpha * Ap[i];
        r[i] = ri;
        acc += ri * ri;
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// One block: the new r.r, beta, the iteration count and the stopping test.
__global__ void k_cg_beta(CgState* cs, const double* part, int nb) {
    __shared__ double red[32];
    if (cs->done) return;
    const double rr = cg_sum(part, nb, red);
    if (threadIdx.x == 0) {
        cs->beta = rr / cs->rr;
        cs->rr = rr;
        cs->it += 1;
        if (!isfinite(rr)) {
            cs->done = 1;
            cs->reason = CG_BREAKDOWN;
        } else if (!(rr > cs->stop2)) {
            cs->done = 1;
            cs->reason = CG_CONVERGED;
        } else if (cs->it >= cs->maxit) {
            cs->done = 1;
            cs->reason = CG_MAXIT;
        }
    }
}

// p = r + beta p
__global__ void k_cg_dir(int m, const CgState* cs, const double* r, double* p) {
    if (cs->done) return;
    const double beta = cs->beta;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        p[i] = r[i] + beta * p[i];
}

}  // namespace fire2
