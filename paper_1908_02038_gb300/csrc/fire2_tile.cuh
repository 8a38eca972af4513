// Shared-memory tiles of the FP64 half-list RGL passes.
//
// The half list evaluates every pair once and owes half of each pair term
// to the neighbour j (F = -grad E, Sec. 2.1: F_j = -sum of the terms j
// takes part in; likewise rho_j).  Sending each j-side term to global memory
// by an FP64 atomic costs, per pair, one FP64 addition (hi + lo of the
// double-float term) per component and one L2 atomic per component; on this
// part the FP64 pipe runs at 1/58 of the FP32 rate, and those additions and
// atomics dominated the force pass.
//
// Here the atoms are processed in tiles: a tile is one brick of list cells
// (GeoC::bk), its own atoms are the brick's atoms in cell-sorted order, and
// its stage is the set of all (atom, image shift) pairs the own atoms' half
// lists name, own atoms first.  k_tile_build (after every list build) finds
// each tile's stage with a shared-memory hash table and rewrites the list as
// 16-bit stage slots (nbr_loc, indexed by cell-sorted position).  The pair
// passes then stage the positions (and F'(rho)) of a tile in shared memory,
// accumulate every j-side term exactly in two 32-bit fixed-point words per
// component with shared-memory integer atomics (order-independent), and
// flush each staged atom's sum with one FP64 atomic per component.  Pairs
// whose neighbour did not fit in the stage (more than stage_cap distinct
// neighbours) and terms outside the fixed-point range take the global FP64
// atomics of the untiled kernels instead.
#pragma once

#include "fire2_device.cuh"

namespace fire2 {

// Launch shape of the tile passes and the brick of cells a tile covers
// (compile-time; the defaults are the measured choice on GB300).
#ifndef FIRE_TILE_THREADS
#define FIRE_TILE_THREADS 512
#endif
#ifndef FIRE_TILE_STAGE
#define FIRE_TILE_STAGE 1920
#endif
#ifndef FIRE_TILE_MINB
#define FIRE_TILE_MINB 2
#endif
#ifndef FIRE_TILE_BRICK_X
#define FIRE_TILE_BRICK_X 4
#define FIRE_TILE_BRICK_Y 4
#define FIRE_TILE_BRICK_Z 2
#endif
constexpr int kTileThreads = FIRE_TILE_THREADS;
constexpr int kTileMinBlocks = FIRE_TILE_MINB;   // resident blocks per SM (registers)
constexpr int kStageMax = FIRE_TILE_STAGE;       // staged atoms per tile (force pass: 56 B each)
constexpr int kTileBrick[3] = {FIRE_TILE_BRICK_X, FIRE_TILE_BRICK_Y, FIRE_TILE_BRICK_Z};
constexpr int kTileHash = 4096;          // hash table of the stage build (power of 2)
constexpr int kTileHashBits = 12;
static_assert(kTileHash >= 2 * kStageMax, "hash table at most half full");
static_assert(kTileThreads % 32 == 0 && kTileThreads <= 1024, "tile block size");
constexpr uint16_t kSlotNone = 0xffffu;  // not staged: global path
constexpr uint16_t kSlotOwnOver = 0xfffeu;   // own atom beyond the stage (build only)
constexpr uint32_t kKeyEmpty = 0xffffffffu;  // never a list entry (image codes <= 124)
constexpr size_t kDensTileSmem = (size_t)kStageMax * (3 * 8 + 2 * 4);
constexpr size_t kForceTileSmem = (size_t)kStageMax * (3 * 8 + 8 + 6 * 4);

// ---------------------------------------------------------------------------
// Fixed-point words.  A double-float value v = hi + lo is carried as
// H 2^-18 + L 2^-40 with H = round(v 2^18) and L = round((v 2^18 - H) 2^22);
// sums of the words are exact integers, so the result does not depend on
// the order of the atomics.  One term is off by at most ~5e-13 (L's
// rounding); the tiled passes add at most a few dozen terms per atom.

constexpr float kFxH = 262144.0f;        // 2^18
constexpr float kFxL = 4194304.0f;       // 2^22
constexpr float kFxMagic = 12582912.0f;  // 1.5 2^23: x + magic rounds x for |x| < 2^22
constexpr float kFxPairMax = 15.0f;      // per-pair split: |hi| 2^18 < 2^22
constexpr float kFxAnyMax = 4096.0f;     // per-atom split: |hi| 2^18 < 2^30

// Split of one pair term (|hi| < 15): additions and multiplications only.
__device__ __forceinline__ bool fx_split_pair(float hi, float lo, int& H, int& L) {
    if (!(fabsf(hi) < kFxPairMax)) return false;
    const float hs = hi * kFxH;                                // exact
    const float a = __fadd_rn(hs, kFxMagic);                   // round(hs) + magic
    H = __float_as_int(a) - __float_as_int(kFxMagic);          // same binade: ulp 1
    const float hf = __fadd_rn(a, -kFxMagic);                  // round(hs), exact
    const float r = __fmaf_rn(lo, kFxH, __fadd_rn(hs, -hf));   // |r| <= 0.625
    const float c = __fmaf_rn(r, kFxL, kFxMagic);
    L = __float_as_int(c) - __float_as_int(kFxMagic);
    return true;
}

// Split of a per-atom sum (|hi| < 4096), with conversions.
__device__ __forceinline__ bool fx_split_any(float hi, float lo, int& H, int& L) {
    if (!(fabsf(hi) < kFxAnyMax)) return false;
    const float hs = hi * kFxH;
    H = __float2int_rn(hs);
    const float r = __fmaf_rn(lo, kFxH, __fadd_rn(hs, -(float)H));   // hs - H exact
    L = __float2int_rn(r * kFxL);
    return true;
}

// H 2^-18 + L 2^-40 as a double, exactly, with integer instructions only.
__device__ __forceinline__ double fx_to_double(int H, int L) {
    const long long t = ((long long)H << 22) + (long long)L;   // units of 2^-40
    if (t == 0) return 0.0;
    const unsigned long long sgn = t < 0 ? 0x8000000000000000ull : 0ull;
    const unsigned long long a = t < 0 ? (unsigned long long)(-t) : (unsigned long long)t;
    const int lz = __clzll((long long)a);
    // leading one to bit 52 (|t| < 2^53 for every sum these passes form)
    const unsigned long long m = lz >= 11 ? a << (lz - 11) : a >> (11 - lz);
    const unsigned long long e = (unsigned long long)(1023 + 63 - lz - 40);
    return __longlong_as_double((long long)(sgn | (e << 52) | (m & 0x000fffffffffffffull)));
}

// ---------------------------------------------------------------------------
// Stage build.

__device__ __forceinline__ unsigned tile_hash(uint32_t key) {
    return (key * 2654435761u) >> (32 - kTileHashBits);   // Knuth's multiplicative hash
}

// Inserts key (or finds it); table position, or -1 when the table is full.
__device__ __forceinline__ int tile_insert(uint32_t* keys, uint32_t key) {
    unsigned h = tile_hash(key);
    for (int probe = 0; probe < kTileHash; ++probe) {
        const uint32_t old = atomicCAS(&keys[h], kKeyEmpty, key);
        if (old == kKeyEmpty || old == key) return (int)h;
        h = (h + 1) & (kTileHash - 1);
    }
    return -1;
}

__device__ __forceinline__ int tile_find(const uint32_t* keys, uint32_t key) {
    unsigned h = tile_hash(key);
    for (int probe = 0; probe < kTileHash; ++probe) {
        const uint32_t k = keys[h];
        if (k == key) return (int)h;
        if (k == kKeyEmpty) return -1;
        h = (h + 1) & (kTileHash - 1);
    }
    return -1;
}

// Own atoms of tile T: cell-sorted positions [p0, p1).
__device__ __forceinline__ void tile_range(const Bufs& b, const GeoC& g, int T, int& p0, int& p1) {
    const int bc = g.bk[0] * g.bk[1] * g.bk[2];
    p0 = b.cell_start[T * bc];
    p1 = b.cell_start[(T + 1) * bc];
}

// Exclusive prefix sum over the block (blockDim.x = kTileThreads); *total
// receives the sum.  ws holds kTileThreads / 32 ints.
__device__ __forceinline__ int block_exscan(int v, int* ws, int* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) {
        int s = lane < (kTileThreads >> 5) ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < (kTileThreads >> 5)) ws[lane] = s;   // inclusive warp totals
    }
    __syncthreads();
    const int before = (w > 0 ? ws[w - 1] : 0) + x - v;
    *total = ws[(kTileThreads >> 5) - 1];
    __syncthreads();
    return before;
}

// One block per tile (grid-stride): the stage of the tile and the slots of
// its own atoms' list entries.  Slots: own atoms 0 .. nown - 1 (cell-sorted
// order), then the other keys in hash-table order (which depends on the
// order of the concurrent insertions; the sums do not, being exact integer
// sums); at most stage_cap of them, the rest kSlotNone.
__global__ void __launch_bounds__(kTileThreads) k_tile_build(Bufs b, GeoC g, int force) {
    __shared__ uint32_t keys[kTileHash];
    __shared__ uint16_t slot_of[kTileHash];
    __shared__ int ws[kTileThreads / 32];
    if (!need_rebuild(b.st, g, force)) return;
    const int cap = g.stage_cap;
    for (int T = blockIdx.x; T < g.ntile; T += gridDim.x) {
        int p0, p1;
        tile_range(b, g, T, p0, p1);
        const int nown = p1 - p0;
        for (int h = threadIdx.x; h < kTileHash; h += blockDim.x) {
            keys[h] = kKeyEmpty;
            slot_of[h] = kSlotNone;
        }
        __syncthreads();
        uint32_t* tkey = b.tile_key + (size_t)T * kStageMax;
        for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const uint32_t key = ((uint32_t)kCodeZero << kIdxBits) | (uint32_t)b.cell_atoms[p];
            const int h = tile_insert(keys, key);
            const int so = p - p0;
            if (so < cap) tkey[so] = key;   // own slots are positional
            // a full table (h < 0) leaves the atom out: lookups of it miss and
            // its pairs take the global path
            if (h >= 0) slot_of[h] = so < cap ? (uint16_t)so : kSlotOwnOver;
        }
        __syncthreads();
        for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const int i = b.cell_atoms[p];
            const int m = b.nnbr[i];
            for (int k = 0; k < m; ++k) tile_insert(keys, b.nbr[(size_t)k * b.n + i]);
        }
        __syncthreads();
        constexpr int kPer = (kTileHash + kTileThreads - 1) / kTileThreads;
        const int h0 = threadIdx.x * kPer;
        int cnt = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q)
            cnt += (h0 + q < kTileHash && keys[h0 + q] != kKeyEmpty &&
                    slot_of[h0 + q] == kSlotNone) ? 1 : 0;
        int nhalo = 0;
        int s = min(nown, cap) + block_exscan(cnt, ws, &nhalo);
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int h = h0 + q;
            if (h < kTileHash && keys[h] != kKeyEmpty && slot_of[h] == kSlotNone) {
                if (s < cap) {
                    slot_of[h] = (uint16_t)s;
                    tkey[s] = keys[h];
                }
                ++s;
            }
        }
        if (threadIdx.x == 0) b.tile_ns[T] = min(cap, min(nown, cap) + nhalo);
        __syncthreads();
        for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const int i = b.cell_atoms[p];
            const int m = b.nnbr[i];
            for (int k = 0; k < m; ++k) {
                const int h = tile_find(keys, b.nbr[(size_t)k * b.n + i]);
                uint16_t sl = h >= 0 ? slot_of[h] : kSlotNone;
                if (sl == kSlotOwnOver) sl = kSlotNone;
                b.nbr_loc[(size_t)k * b.n + p] = sl;
            }
        }
        __syncthreads();   // the table is reused by the next tile
    }
}

// ---------------------------------------------------------------------------
// The pair passes on tiles.

// Image shift of list code `code` in fixed-point units.
__device__ __forceinline__ void code_shift64(const GeoC& g, int code, long long& sx, long long& sy,
                                             long long& sz) {
    sx = (long long)(code % 5 - 2) * g.Lq64[0];
    sy = (long long)((code / 5) % 5 - 2) * g.Lq64[1];
    sz = (long long)(code / 25 - 2) * g.Lq64[2];
}

// Position of list entry e (atom and image shift) in fixed point: x_j - shift.
__device__ __forceinline__ lvec4 entry_pos64(const Bufs& b, const GeoC& g, uint32_t e) {
    lvec4 q = b.xq64[e & kIdxMask];
    const int code = (int)(e >> kIdxBits);
    if (code != kCodeZero) {
        long long sx, sy, sz;
        code_shift64(g, code, sx, sy, sz);
        q.x -= sx;
        q.y -= sy;
        q.z -= sz;
    }
    return q;
}

// Exact separation qj - qi as float pairs, and r^2.
__device__ __forceinline__ ffloat tile_sep(long long ix, long long iy, long long iz, ffloat& dx,
                                           ffloat& dy, ffloat& dz) {
    dx = fixed_to_ff(ix);
    dy = fixed_to_ff(iy);
    dz = fixed_to_ff(iz);
    return ff_norm2(dx, dy, dz);
}

// Pass 1 on tiles: rho_i (own atoms' sums plus the j-side terms of the
// tile, flushed per staged atom) and 2 phi per pair credited to i; k_embed
// then forms F'(rho) and the embedding energy.
__global__ void __launch_bounds__(kTileThreads, kTileMinBlocks) k_density_tile(Bufs b, PotC P, GeoC g) {
    extern __shared__ __align__(16) unsigned char smem[];
    long long* sx = reinterpret_cast<long long*>(smem);
    long long* sy = sx + kStageMax;
    long long* sz = sy + kStageMax;
    int* aH = reinterpret_cast<int*>(sz + kStageMax);
    int* aL = aH + kStageMax;
    __shared__ double red[32];
    if (pass_skipped(b)) return;
    double e_blk = 0.0;
    for (int T = blockIdx.x; T < g.ntile; T += gridDim.x) {
        int p0, p1;
        tile_range(b, g, T, p0, p1);
        const int ns = b.tile_ns[T];
        const uint32_t* tkey = b.tile_key + (size_t)T * kStageMax;
        for (int s = threadIdx.x; s < ns; s += blockDim.x) {
            const lvec4 q = entry_pos64(b, g, tkey[s]);
            sx[s] = q.x;
            sy[s] = q.y;
            sz[s] = q.z;
            aH[s] = 0;
            aL[s] = 0;
        }
        __syncthreads();
        for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const int so = p - p0;
            const int i = b.cell_atoms[p];
            long long qix, qiy, qiz;
            if (so < ns) {
                qix = sx[so];
                qiy = sy[so];
                qiz = sz[so];
            } else {
                const lvec4 q = b.xq64[i];
                qix = q.x;
                qiy = q.y;
                qiz = q.z;
            }
            const int m = b.nnbr[i];
            ffloat rho = {0.f, 0.f}, erep = {0.f, 0.f};
            uint16_t sl_nx = m > 0 ? b.nbr_loc[p] : kSlotNone;
            for (int k = 0; k < m; ++k) {
                const uint16_t sl = sl_nx;
                if (k + 1 < m) sl_nx = b.nbr_loc[(size_t)(k + 1) * b.n + p];
                long long qjx, qjy, qjz;
                uint32_t e = 0u;
                if (sl != kSlotNone) {
                    qjx = sx[sl];
                    qjy = sy[sl];
                    qjz = sz[sl];
                } else {
                    e = b.nbr[(size_t)k * b.n + i];
                    const lvec4 q = entry_pos64(b, g, e);
                    qjx = q.x;
                    qjy = q.y;
                    qjz = q.z;
                }
                ffloat dx, dy, dz;
                const ffloat r2 = tile_sep(qjx - qix, qjy - qiy, qjz - qiz, dx, dy, dz);
                if (!(r2.hi < P.rc2_f)) continue;
                const float uf = r2.hi - P.r0sq_f;
                ffloat v[2];
                if (uf >= P.tab.u_lo_f) {
                    float row[kFFRow];
                    load_row(b.tab_ffd, ff_index(P.tab, uf), row);
                    ff_row_eval(row, r2, v);
                } else {
                    double rinv, phi, dphi, gg, dg;
                    rgl_pair64(P, ff_to_f64(r2), b.exp_table, rinv, phi, dphi, gg, dg);
                    v[0] = f64_to_ff(phi);
                    v[1] = f64_to_ff(gg);
                }
                erep = ff_acc(erep, v[0]);
                rho = ff_acc(rho, v[1]);
                int H, L;
                if (sl != kSlotNone && fx_split_pair(v[1].hi, v[1].lo, H, L)) {
                    atomicAdd(&aH[sl], H);
                    atomicAdd(&aL[sl], L);
                } else {
                    const int j = (int)((sl != kSlotNone ? tkey[sl] : e) & kIdxMask);
                    atomicAdd(&b.rho[j], ff_to_f64(v[1]));
                }
            }
            const double e_atom = 2.0 * ff_to_f64(erep);   // each pair's 2 phi credited to i
            e_blk += e_atom;
            if (b.eatom) b.eatom[i] = e_atom;
            int H, L;
            if (so < ns && fx_split_any(rho.hi, rho.lo, H, L)) {
                atomicAdd(&aH[so], H);
                atomicAdd(&aL[so], L);
            } else {
                atomicAdd(&b.rho[i], ff_to_f64(rho));
            }
        }
        __syncthreads();
        for (int s = threadIdx.x; s < ns; s += blockDim.x) {
            const double v = fx_to_double(aH[s], aL[s]);
            if (v != 0.0) atomicAdd(&b.rho[tkey[s] & kIdxMask], v);
        }
        __syncthreads();   // the stage is reused by the next tile
    }
    const double s = block_sum(e_blk, red);
    if (threadIdx.x == 0) b.epart[blockIdx.x] = s;
}

// Pass 2 on tiles: F_i = sum_j [2 phi'/r + (F'_i + F'_j) g'/r] (x_j - x_i),
// the j-side terms accumulated per staged atom and flushed (F = -grad E,
// Sec. 2.1).  k_reduce_ctl applies the frozen-DOF mask afterwards.
__global__ void __launch_bounds__(kTileThreads, kTileMinBlocks) k_force_tile(Bufs b, PotC P, GeoC g) {
    extern __shared__ __align__(16) unsigned char smem[];
    long long* sx = reinterpret_cast<long long*>(smem);
    long long* sy = sx + kStageMax;
    long long* sz = sy + kStageMax;
    float2* sfp = reinterpret_cast<float2*>(sz + kStageMax);
    int* aH = reinterpret_cast<int*>(sfp + kStageMax);   // 3 x kStageMax: x, y, z
    int* aL = aH + 3 * kStageMax;
    if (pass_skipped(b)) return;
    for (int T = blockIdx.x; T < g.ntile; T += gridDim.x) {
        int p0, p1;
        tile_range(b, g, T, p0, p1);
        const int ns = b.tile_ns[T];
        const uint32_t* tkey = b.tile_key + (size_t)T * kStageMax;
        for (int s = threadIdx.x; s < ns; s += blockDim.x) {
            const uint32_t e = tkey[s];
            const lvec4 q = entry_pos64(b, g, e);
            sx[s] = q.x;
            sy[s] = q.y;
            sz[s] = q.z;
            const ffloat fq = fp_load(q);
            sfp[s] = make_float2(fq.hi, fq.lo);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                aH[c * kStageMax + s] = 0;
                aL[c * kStageMax + s] = 0;
            }
        }
        __syncthreads();
        for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const int so = p - p0;
            const int i = b.cell_atoms[p];
            long long qix, qiy, qiz;
            float2 fpi2;
            if (so < ns) {
                qix = sx[so];
                qiy = sy[so];
                qiz = sz[so];
                fpi2 = sfp[so];
            } else {
                const lvec4 q = b.xq64[i];
                qix = q.x;
                qiy = q.y;
                qiz = q.z;
                const ffloat fq = fp_load(q);
                fpi2 = make_float2(fq.hi, fq.lo);
            }
            const ffloat fpi = {fpi2.x, fpi2.y};
            const int m = b.nnbr[i];
            ffloat fx = {0.f, 0.f}, fy = {0.f, 0.f}, fz = {0.f, 0.f};
            uint16_t sl_nx = m > 0 ? b.nbr_loc[p] : kSlotNone;
            for (int k = 0; k < m; ++k) {
                const uint16_t sl = sl_nx;
                if (k + 1 < m) sl_nx = b.nbr_loc[(size_t)(k + 1) * b.n + p];
                long long qjx, qjy, qjz;
                float2 fpj2;
                uint32_t e = 0u;
                if (sl != kSlotNone) {
                    qjx = sx[sl];
                    qjy = sy[sl];
                    qjz = sz[sl];
                    fpj2 = sfp[sl];
                } else {
                    e = b.nbr[(size_t)k * b.n + i];
                    const lvec4 q = entry_pos64(b, g, e);
                    qjx = q.x;
                    qjy = q.y;
                    qjz = q.z;
                    const ffloat fq = fp_load(q);
                    fpj2 = make_float2(fq.hi, fq.lo);
                }
                ffloat dx, dy, dz;
                const ffloat r2 = tile_sep(qjx - qix, qjy - qiy, qjz - qiz, dx, dy, dz);
                if (!(r2.hi < P.rc2_f)) continue;
                const float uf = r2.hi - P.r0sq_f;
                ffloat c[2];
                if (uf >= P.tab.u_lo_f) {
                    float row[kFFRow];
                    load_row(b.tab_fff, ff_index(P.tab, uf), row);
                    ff_row_eval(row, r2, c);
                } else {
                    double rinv, phi, dphi, gg, dg;
                    rgl_pair64(P, ff_to_f64(r2), b.exp_table, rinv, phi, dphi, gg, dg);
                    c[0] = f64_to_ff(2.0 * dphi * rinv);
                    c[1] = f64_to_ff(dg * rinv);
                }
                const ffloat fs = ff_madd(ff_add(fpi, {fpj2.x, fpj2.y}), c[1], c[0]);
                // normalised products, as fx_split_pair assumes
                const ffloat t[3] = {ff_mul(fs, dx), ff_mul(fs, dy), ff_mul(fs, dz)};
                fx = ff_acc(fx, t[0]);
                fy = ff_acc(fy, t[1]);
                fz = ff_acc(fz, t[2]);
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    int H, L;
                    if (sl != kSlotNone && fx_split_pair(-t[cc].hi, -t[cc].lo, H, L)) {
                        atomicAdd(&aH[cc * kStageMax + sl], H);
                        atomicAdd(&aL[cc * kStageMax + sl], L);
                    } else {
                        const int j = (int)((sl != kSlotNone ? tkey[sl] : e) & kIdxMask);
                        double* fj = b.f + cc * (size_t)b.n + j;
                        atomicAdd(fj, -ff_to_f64(t[cc]));
                    }
                }
            }
            const ffloat fi[3] = {fx, fy, fz};
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                int H, L;
                if (so < ns && fx_split_any(fi[cc].hi, fi[cc].lo, H, L)) {
                    atomicAdd(&aH[cc * kStageMax + so], H);
                    atomicAdd(&aL[cc * kStageMax + so], L);
                } else {
                    double* f = b.f + cc * (size_t)b.n + i;
                    atomicAdd(f, ff_to_f64(fi[cc]));
                }
            }
        }
        __syncthreads();
        for (int s = threadIdx.x; s < ns; s += blockDim.x) {
            const int j = (int)(tkey[s] & kIdxMask);
            const double vx = fx_to_double(aH[s], aL[s]);
            const double vy = fx_to_double(aH[kStageMax + s], aL[kStageMax + s]);
            const double vz = fx_to_double(aH[2 * kStageMax + s], aL[2 * kStageMax + s]);
            if (vx != 0.0) atomicAdd(b.f + j, vx);
            if (vy != 0.0) atomicAdd(b.f + b.n + j, vy);
            if (vz != 0.0) atomicAdd(b.f + 2 * (size_t)b.n + j, vz);
        }
        __syncthreads();   // the stage is reused by the next tile
    }
}

}  // namespace fire2
