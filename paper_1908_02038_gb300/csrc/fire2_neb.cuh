// Nudged elastic band on the device.
//
// The paper relaxes NEB ensembles with FIRE 2.0 (Sec. 4, cases 7 and 8: a
// simultaneous minimisation of images "with modified forces"); it cites
// Sheppard et al. (2008) for the method and states no formulas.  The forces
// here are the standard ones of that reference:
//   tangent of image i from t+ = R_{i+1} - R_i and t- = R_i - R_{i-1}
//   (minimum image) and the energies E_{i-1}, E_i, E_{i+1} (the improved
//   tangent of Henkelman and Jonsson, 2000): t+ when the energy rises
//   through i, t- when it falls, else the energy-weighted mix
//   dEmax t+ + dEmin t- (E_{i+1} > E_{i-1}) or dEmin t+ + dEmax t-;
//   F_i^NEB = F_i - (F_i.t) t + k (|t+| - |t-|) t, or F_i - 2 (F_i.t) t for
//   the climbing image (the movable image of highest energy, if enabled).
// All movable images are one system for FIRE (one dt, alpha and P over the
// band).  Frozen components are zeroed in the true force, the tangent and the
// NEB force; a vanishing tangent falls back to t+ + t-, and if that vanishes
// too the force is left unprojected.
//
// Layout: the n_img movable images are atoms [k N, (k + 1) N) of the handle's
// arrays (N = img_n); the two fixed end states sit in `end` (2 N).  Per
// iteration, after the force passes (which also write per-atom energies):
//   k_neb_sums    per image and block: E, |t+|^2, |t-|^2 (unmasked, for the
//                 springs), |t+m|^2, |t-m|^2, t+m.t-m, F.t+m, F.t-m (masked);
//                 its last block (ticket) then the fixed-order sums, climbing
//                 image, tangent weights and the per-image coefficients of
//                 F^NEB = F + s t (neb_scalars)
//   k_neb_project F^NEB per atom, written over F, plus the FP64 reductions of
//                 (F^NEB, v); its last block runs the control step
#pragma once

#include "fire2_device.cuh"

namespace fire2 {

constexpr int kNebSums = 8;      // partial sums per image and block
constexpr int kNebBlock = 256;

struct NebC {
    const dvec4* end;   // end states 0 and n_img + 1, img_n atoms each
    double* part;       // [img][kNebSums][nb]
    double* coef;       // [img][4]: a+, a- (tangent = a+ t+m + a- t-m), s (F += s t), 0
    double* E;          // n_img + 2 image energies; E[0], E[n_img + 1] set by the host
    int* climber;       // 1..n_img, or 0
    double k;           // spring constant
    int climb, n_img, img_n, nb;
};

__device__ __forceinline__ double neb_mi(double d, const GeoC& g, int a) {
    return g.per[a] ? d - g.L[a] * rint(d / g.L[a]) : d;
}

// Neighbour images of atom a of movable image img (0-based): R_{i-1}, R_{i+1}.
__device__ __forceinline__ void neb_neighbours(const Bufs& b, const NebC& c, int img, int a,
                                               dvec4& rm, dvec4& rp) {
    const size_t gi = (size_t)img * c.img_n + a;
    rm = img == 0 ? c.end[a] : b.x[gi - c.img_n];
    rp = img == c.n_img - 1 ? c.end[c.img_n + a] : b.x[gi + c.img_n];
}

__device__ __forceinline__ void neb_seps(const GeoC& g, const dvec4& r, const dvec4& rm,
                                         const dvec4& rp, double tp[3], double tm[3]) {
    tp[0] = neb_mi(rp.x - r.x, g, 0);
    tp[1] = neb_mi(rp.y - r.y, g, 1);
    tp[2] = neb_mi(rp.z - r.z, g, 2);
    tm[0] = neb_mi(r.x - rm.x, g, 0);
    tm[1] = neb_mi(r.y - rm.y, g, 1);
    tm[2] = neb_mi(r.z - rm.z, g, 2);
}

__device__ __forceinline__ unsigned neb_mask(const Bufs& b, size_t gi) {
    return b.dofmask ? (unsigned)b.dofmask[gi] : 0u;
}

__device__ void neb_scalars(const Bufs& b, const NebC& c, double* sums);

// grid (nb, n_img); dynamic shared memory: n_img x kNebSums doubles
__global__ void __launch_bounds__(kNebBlock) k_neb_sums(Bufs b, GeoC g, NebC c) {
    __shared__ double red[kNebSums * 32];
    __shared__ int last;
    extern __shared__ double sums[];   // n_img x kNebSums (last block)
    if (b.st->done) return;
    const int img = blockIdx.y;
    double acc[kNebSums] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < c.img_n; a += gridDim.x * blockDim.x) {
        const size_t gi = (size_t)img * c.img_n + a;
        const dvec4 r = b.x[gi];
        dvec4 rm, rp;
        neb_neighbours(b, c, img, a, rm, rp);
        double tp[3], tm[3];
        neb_seps(g, r, rm, rp, tp, tm);
        dvec4 f = f_load(b, (int)gi);
        mask_force(b, (int)gi, f);
        const double fv[3] = {f.x, f.y, f.z};
        const unsigned m = neb_mask(b, gi);
        acc[0] += b.eatom[gi];
        for (int d = 0; d < 3; ++d) {
            acc[1] += tp[d] * tp[d];
            acc[2] += tm[d] * tm[d];
            if (m & (1u << d)) continue;
            acc[3] += tp[d] * tp[d];
            acc[4] += tm[d] * tm[d];
            acc[5] += tp[d] * tm[d];
            acc[6] += fv[d] * tp[d];
            acc[7] += fv[d] * tm[d];
        }
    }
    // the eight block sums: two transposing butterflies per warp (warp_sum4),
    // then over the warps in warp 0, in a fixed order
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const double s0 = warp_sum4(acc[0], acc[1], acc[2], acc[3]);
    const double s1 = warp_sum4(acc[4], acc[5], acc[6], acc[7]);
    if ((lane & 7) == 0) {
        red[(lane >> 3) * 32 + w] = s0;
        red[(4 + (lane >> 3)) * 32 + w] = s1;
    }
    __syncthreads();
    if (w == 0) {
        const bool in = lane < (int)(blockDim.x >> 5);
        double t[kNebSums];
#pragma unroll
        for (int q = 0; q < kNebSums; ++q) t[q] = in ? red[q * 32 + lane] : 0.0;
        const double u0 = warp_sum4(t[0], t[1], t[2], t[3]);
        const double u1 = warp_sum4(t[4], t[5], t[6], t[7]);
        if ((lane & 7) == 0) {
            double* o = c.part + (size_t)img * kNebSums * c.nb + blockIdx.x;
            o[(size_t)(lane >> 3) * c.nb] = u0;
            o[(size_t)(4 + (lane >> 3)) * c.nb] = u1;
        }
    }
    // the last block of the grid runs the band's scalars on all partials
    if (threadIdx.x == 0) {
        __threadfence();   // this block's partials before its ticket
        const unsigned nblk = gridDim.x * gridDim.y;
        last = atomicAdd(&b.st->neb_blocks, 1u) == nblk - 1 ? 1 : 0;
    }
    __syncthreads();
    if (!last) return;
    if (threadIdx.x == 0) b.st->neb_blocks = 0u;
    __threadfence();       // every other block's partials are visible from here
    neb_scalars(b, c, sums);
}

// One block; warp w reduces the partials of images w, w + nw, ... in a fixed
// order, then thread 0 picks the climbing image and sets the coefficients.
__device__ void neb_scalars(const Bufs& b, const NebC& c, double* sums /* n_img x kNebSums */) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int img = warp; img < c.n_img; img += nw)
        for (int q = 0; q < kNebSums; ++q) {
            const double* p = c.part + ((size_t)img * kNebSums + q) * c.nb;
            double v = 0.0;
            for (int k = lane; k < c.nb; k += 32) v += p[k];
            v = warp_sum(v);
            if (lane == 0) sums[img * kNebSums + q] = v;
        }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int M = c.n_img;
    for (int i = 1; i <= M; ++i) c.E[i] = sums[(i - 1) * kNebSums];
    int climber = 0;
    if (c.climb) {
        climber = 1;
        for (int i = 2; i <= M; ++i)
            if (c.E[i] > c.E[climber]) climber = i;
    }
    *c.climber = climber;
    for (int i = 1; i <= M; ++i) {
        const double* S = sums + (i - 1) * kNebSums;
        const double Ep = c.E[i + 1], Ei = c.E[i], Em = c.E[i - 1];
        double wp, wm;
        if (Ep > Ei && Ei > Em) {
            wp = 1.0;
            wm = 0.0;
        } else if (Ep < Ei && Ei < Em) {
            wp = 0.0;
            wm = 1.0;
        } else {
            const double dmx = fmax(fabs(Ep - Ei), fabs(Em - Ei));
            const double dmn = fmin(fabs(Ep - Ei), fabs(Em - Ei));
            if (Ep > Em) {
                wp = dmx;
                wm = dmn;
            } else {
                wp = dmn;
                wm = dmx;
            }
        }
        double t2 = wp * wp * S[3] + 2.0 * wp * wm * S[5] + wm * wm * S[4];
        if (!(t2 > 0.0)) {
            wp = wm = 1.0;
            t2 = S[3] + 2.0 * S[5] + S[4];
        }
        double ap = 0.0, am = 0.0, sc = 0.0;
        if (t2 > 0.0) {
            const double tn = sqrt(t2);
            ap = wp / tn;
            am = wm / tn;
            const double ft = ap * S[6] + am * S[7];
            sc = i == climber ? -2.0 * ft : c.k * (sqrt(S[1]) - sqrt(S[2])) - ft;
        }
        double* o = c.coef + 4 * (i - 1);
        o[0] = ap;
        o[1] = am;
        o[2] = sc;
        o[3] = 0.0;
    }
}

// This thread's atoms of the projection (grid-stride): F^NEB written over F,
// then its reductions; VV: velocity Verlet's second half kick first.
template <bool VV>
__device__ __forceinline__ void neb_project_range(const Bufs& b, const GeoC& g, const NebC& c,
                                                  double vvh, RedAcc& acc) {
    const int total = c.n_img * c.img_n;
    for (int gi = blockIdx.x * blockDim.x + threadIdx.x; gi < total; gi += gridDim.x * blockDim.x) {
        const int img = gi / c.img_n, a = gi - img * c.img_n;
        const double* o = c.coef + 4 * img;
        const dvec4 r = b.x[gi];
        dvec4 rm, rp;
        neb_neighbours(b, c, img, a, rm, rp);
        double tp[3], tm[3];
        neb_seps(g, r, rm, rp, tp, tm);
        dvec4 f = f_load(b, gi);
        f.x += o[2] * (o[0] * tp[0] + o[1] * tm[0]);
        f.y += o[2] * (o[0] * tp[1] + o[1] * tm[1]);
        f.z += o[2] * (o[0] * tp[2] + o[1] * tm[2]);
        mask_force(b, gi, f);
        f_store(b, gi, f.x, f.y, f.z);
        red_atom(b, gi, f, b.v[gi], VV ? vvh : 0.0, acc);
    }
}

// grid-stride over all n_img x img_n atoms: F^NEB = mask(F + s t) written
// over F, then the (F^NEB, v) reductions (with the velocity-Verlet half
// kick); the last block (ticket) runs the control step on all partials, as
// k_reduce_ctl does for single systems.
__global__ void __launch_bounds__(kNebBlock) k_neb_project(Bufs b, GeoC g, NebC c, int mode,
                                                           cudaGraphConditionalHandle h,
                                                           int has_handle) {
    __shared__ double red[kRedRows * 32];
    __shared__ int last;
    if (b.st->done) {   // chunked loop bodies past the stop
        if (mode == CTL_LOOP && has_handle && blockIdx.x == 0 && threadIdx.x == 0)
            cudaGraphSetConditional(h, 0u);
        return;
    }
    const double vvh = vv_half_of(b.st);
    RedAcc acc;
    // the velocity-Verlet test once per pass, not per atom (an FP64
    // comparison costs the FP64 pipe as much as a multiply-add)
    if (vvh != 0.0)
        neb_project_range<true>(b, g, c, vvh, acc);
    else
        neb_project_range<false>(b, g, c, 0.0, acc);
    red_write(acc, red, b.rpart);
    if (threadIdx.x == 0) {
        __threadfence();   // this block's partials before its ticket
        last = atomicAdd(&b.st->red_blocks, 1u) == gridDim.x - 1 ? 1 : 0;
    }
    __syncthreads();
    if (!last) return;
    if (threadIdx.x == 0) b.st->red_blocks = 0u;
    __threadfence();       // every other block's partials are visible from here
    control_body(b, mode, h, has_handle, red, energy_partials(b));
}

}  // namespace fire2

namespace fire2 {

// End states (row-major x, y, z) into the padded layout of `end`.
__global__ void k_neb_load_ends(const double* p0, const double* p1, dvec4* end, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 2 * n) return;
    const double* p = i < n ? p0 + 3 * (size_t)i : p1 + 3 * (size_t)(i - n);
    end[i] = make_dvec4(p[0], p[1], p[2], 0.0);
}

}  // namespace fire2
