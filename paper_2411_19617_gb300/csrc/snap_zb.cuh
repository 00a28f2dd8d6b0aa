// snap_zb.cuh -- device side of compute_zi + compute_bi (see snap_zb.cu).
// Included by the FP32 and FP64 translation units, each of which owns its
// own copy of the constant-memory tables.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "mala_internal.h"
#include "snap_common.cuh"
#include "snap_pairs.cuh"

namespace mala {

constexpr int kZbWarps = 8;
constexpr int kZbMaxList = 32;
constexpr int kCgSize = cg_table_size();

// Clebsch-Gordan table as (c, c) pairs: one operand of a packed FP32x2 FMA
static __constant__ float2 c_cg2[kCgSize];

// per supported twojmax (index tj/2): [warp][slot] = global triple id | (local index << 8), -1 = end
static __constant__ int c_zb_list[kTJMax / 2 + 1][kZbWarps][kZbMaxList];

// per supported twojmax (index tj/2): J + 1 of every output column, for the
// closed form of points without neighbours
static __constant__ float c_zb_jp1[kTJMax / 2 + 1][n_triples(kTJMax)];

namespace {

template <class T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };

template <class T> __device__ __forceinline__ T cg_at(const T* gtab, int idx);
template <> __device__ __forceinline__ float cg_at<float>(const float*, int idx) { return c_cg2[idx].x; }
template <> __device__ __forceinline__ double cg_at<double>(const double* gtab, int idx) { return __ldg(gtab + idx); }

// Row `row` of u^JJ from the half set, scaled by `scale`.
template <class T, int JJ>
__device__ __forceinline__ void load_row(typename C2<T>::type (&x)[JJ + 1], const typename C2<T>::type* __restrict__ su,
                                         int row, T scale) {
    using V = typename C2<T>::type;
    if (2 * row < JJ) {
        const V* b = su + (size_t)(hoff(JJ) + row * (JJ + 1)) * 32;
#pragma unroll
        for (int mb = 0; mb <= JJ; ++mb) {
            const V v = b[mb * 32];
            x[mb].x = scale * v.x;
            x[mb].y = scale * v.y;
        }
    } else if (2 * row == JJ) {
        const V* b = su + (size_t)(hoff(JJ) + row * (JJ + 1)) * 32;
#pragma unroll
        for (int mb = 0; mb <= JJ; ++mb) {
            if (2 * mb <= JJ) {
                const V v = b[mb * 32];
                x[mb].x = scale * v.x;
                x[mb].y = scale * v.y;
            } else {
                // (JJ/2, mb) = (-1)^(mb - JJ/2) conj((JJ/2, JJ - mb))
                const V v = b[(JJ - mb) * 32];
                const T sg = (((mb - JJ / 2) & 1) ? T(-1) : T(1)) * scale;
                x[mb].x = sg * v.x;
                x[mb].y = -sg * v.y;
            }
        }
    } else {
        // (row, mb) = (-1)^(mb - row) conj((JJ - row, JJ - mb)); the row parity goes into the scale
        const int r2 = JJ - row;
        const V* b = su + (size_t)(hoff(JJ) + r2 * (JJ + 1)) * 32;
        const T s0 = (row & 1) ? -scale : scale;
#pragma unroll
        for (int mb = 0; mb <= JJ; ++mb) {
            const V v = b[(JJ - mb) * 32];
            const T sg = (mb & 1) ? -s0 : s0;
            x[mb].x = sg * v.x;
            x[mb].y = -sg * v.y;
        }
    }
}

// One row ma of Z^{J1J2J} (columns 0..NCOL-1) dotted with conj(u^J[ma]).
// MID: the middle row of even J, whose column J/2 counts once.
template <class T, int J1, int J2, int J, int NCOL, bool MID>
__device__ __forceinline__ T zb_row(const typename C2<T>::type* __restrict__ su, const T* __restrict__ gcg, int ma) {
    using V = typename C2<T>::type;
    constexpr int d = (J1 + J2 - J) / 2;
    constexpr int OFF = cg_offset(J1, J2, J);
    T zr[NCOL], zi[NCOL];
#pragma unroll
    for (int mb = 0; mb < NCOL; ++mb) zr[mb] = zi[mb] = T(0);
    const int m1lo = max(0, ma + d - J2), m1hi = min(J1, ma + d);
    for (int m1a = m1lo; m1a <= m1hi; ++m1a) {
        const int m2a = ma - m1a + d;
        const T c1 = cg_at<T>(gcg, OFF + ma * (J1 + 1) + m1a);
        V x[J1 + 1], y[J2 + 1];
        load_row<T, J1>(x, su, m1a, c1);
        load_row<T, J2>(y, su, m2a, T(1));
#pragma unroll
        for (int mb = 0; mb < NCOL; ++mb) {
#pragma unroll
            for (int m1b = 0; m1b <= J1; ++m1b) {
                const int m2b = mb - m1b + d;
                if (m2b >= 0 && m2b <= J2) {
                    const T c2 = cg_at<T>(gcg, OFF + mb * (J1 + 1) + m1b);
                    const T tr = x[m1b].x * y[m2b].x - x[m1b].y * y[m2b].y;
                    const T ti = x[m1b].x * y[m2b].y + x[m1b].y * y[m2b].x;
                    zr[mb] += c2 * tr;
                    zi[mb] += c2 * ti;
                }
            }
        }
    }
    const V* w = su + (size_t)(hoff(J) + ma * (J + 1)) * 32;
    T r = T(0);
#pragma unroll
    for (int mb = 0; mb < NCOL; ++mb) {
        const V v = w[mb * 32];
        const T t = v.x * zr[mb] + v.y * zi[mb];
        if (MID && 2 * mb == J)
            r += t;
        else
            r += T(2) * t;
    }
    return r;
}

template <class T, int J1, int J2, int J>
__device__ __forceinline__ T zb_triple(const typename C2<T>::type* __restrict__ su, const T* __restrict__ gcg) {
    T b = T(0);
    for (int ma = 0; 2 * ma < J; ++ma) b += zb_row<T, J1, J2, J, J + 1, false>(su, gcg, ma);
    if constexpr ((J & 1) == 0) b += zb_row<T, J1, J2, J, J / 2 + 1, true>(su, gcg, J / 2);
    return b;
}

// I-th triple of the kTJMax index set
__host__ __device__ constexpr int triple_field(int I, int f) {
    int n = 0;
    for (int j1 = 0; j1 <= kTJMax; ++j1)
        for (int j2 = 0; j2 <= j1; ++j2)
            for (int j = 0; j <= kTJMax; ++j) {
                if (!triple_ok(j1, j2, j, kTJMax)) continue;
                if (n == I) return f == 0 ? j1 : (f == 1 ? j2 : j);
                ++n;
            }
    return -1;
}

template <class T, int LO, int HI>
__device__ __forceinline__ T zb_dispatch(int id, const typename C2<T>::type* su, const T* gcg) {
    if constexpr (HI - LO == 1) {
        return zb_triple<T, triple_field(LO, 0), triple_field(LO, 1), triple_field(LO, 2)>(su, gcg);
    } else {
        constexpr int MID = (LO + HI) / 2;
        if (id < MID) return zb_dispatch<T, LO, MID>(id, su, gcg);
        return zb_dispatch<T, MID, HI>(id, su, gcg);
    }
}

template <class T>
__global__ void __launch_bounds__(kZbWarps * 32)
    k_zb(int tj, const typename C2<T>::type* __restrict__ u, const BatchSnap* __restrict__ batch, int nsnap,
         int64_t tile0, int64_t ntiles, const T* __restrict__ gcg, T* __restrict__ B) {
    using V = typename C2<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nh = n_half(tj);
    const int nB = n_triples(tj);
    V* su_all = reinterpret_cast<V*>(smem_raw);
    T* sB = reinterpret_cast<T*>(smem_raw + sizeof(V) * (size_t)nh * 32);
    const int64_t tl = blockIdx.x;
    if (tl >= ntiles) return;
    // stage the tile's u half set
    {
        const float4* src = reinterpret_cast<const float4*>(u + (size_t)tl * nh * 32);
        float4* dst = reinterpret_cast<float4*>(su_all);
        const int n16 = (int)(sizeof(V) * (size_t)nh * 32 / 16);
        for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = __ldg(src + i);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const V* su = su_all + lane;
    const int* list = c_zb_list[tj / 2][warp];
    for (int s = 0; s < kZbMaxList; ++s) {
        const int e = list[s];
        if (e < 0) break;
        const int id = e & 0xff, loc = e >> 8;
        const T b = zb_dispatch<T, 0, n_triples(kTJMax)>(id, su, gcg);
        sB[loc * 32 + lane] = b;
    }
    __syncthreads();
    const int si = batch_find(batch, nsnap, tile0 + tl);
    const SnapGeom& g = batch[si].sd.g;
    const int64_t row0 = batch[si].row_off;
    const int64_t tile = tile0 + tl - batch[si].tile_off;
    const int tx = (int)(tile % g.tiles[0]);
    const int ty = (int)((tile / g.tiles[0]) % g.tiles[1]);
    const int tz = (int)(tile / ((int64_t)g.tiles[0] * g.tiles[1]));
    for (int idx = threadIdx.x; idx < 32 * nB; idx += blockDim.x) {
        const int l = idx / nB, t = idx % nB;
        const int ix = tx * kTileX + (l % kTileX);
        const int iy = ty * kTileY + ((l / kTileX) % kTileY);
        const int iz = tz * kTileZ + l / (kTileX * kTileY);
        if (ix >= g.grid[0] || iy >= g.grid[1] || iz >= g.grid[2]) continue;
        const int64_t p = row0 + ix + (int64_t)g.grid[0] * (iy + (int64_t)g.grid[1] * iz);
        B[(size_t)p * nB + t] = sB[t * 32 + l];
    }
}


// ---- FP32 kernel: two grid points per lane, packed FP32x2 arithmetic --------
//
// B is linear in each (row ma, u^J1 row m1a) contribution:
//   B = sum_{ma, m1a} c1(ma, m1a) * sum_mb w(ma, mb) Re(conj(u^J[ma][mb]) conv_{ma,m1a}[mb]),
// conv[mb] = sum_m1b c2(mb, m1b) x[m1b] y[mb - m1b + d],  x = u^J1[m1a], y = u^J2[ma - m1a + d],
// so a "unit" (triple, ma, m1a) yields a scalar per point.
//
// One CTA handles 64 grid points (two tiles); lane l holds point l of both
// tiles, and every value is a pair (point A, point B), so each packed FP32x2
// instruction (FMUL2 / FFMA2) does the same scalar step for two points and the
// operands need no shuffling.  The u half set of the 64 points sits in shared
// memory as float4 (A.re, B.re, A.im, B.im) per element and lane (128 KB at
// twojmax = 10); rows above the middle are read through the mirror
// u[J-ma][J-mb] = (-1)^(ma-mb) conj(u[ma][mb]) with compile-time column signs,
// the run-time row parities folding into the unit's scalar.  The units of all
// triples are dealt round-robin to the warps, which therefore execute the same
// triple's code at nearly the same time (instruction-cache locality).  The
// units of a triple form 16 fixed groups; each group's FP32 sum meets its
// column's total in 64-bit fixed point (2^-32) through a shared-memory atomic:
// integer addition is associative, so B depends neither on the warp order nor
// on the number of warps.

constexpr int kZbUWarps = 16;                // default warps per CTA (the tuner may pick another variant)
// |value| bound per group sum: a column's total in 2^-32 fixed point must stay
// below 2^31 = 2.1e9 to fit int64, and a column takes at most 16 group sums
constexpr float kFixLimit = 1.0e8f;

template <int N, int I = 0>
__device__ __forceinline__ void negate_pairs(const float2 (&a)[N], float2 (&b)[N]) {
    if constexpr (I < N) {
        b[I] = make_float2(-a[I].x, -a[I].y);
        negate_pairs<N, I + 1>(a, b);
    }
}

// terms of column MB: zr += c2 (xr yr - xi yi), zi += c2 (xr yi + xi yr)
template <int J1, int J2, int OFF, int D, int MB, int M1B>
__device__ __forceinline__ void col_terms(const float2 (&xr)[J1 + 1], const float2 (&xi)[J1 + 1],
                                          const float2 (&yr)[J2 + 1], const float2 (&yi)[J2 + 1],
                                          const float2 (&yn)[J2 + 1], float2& zr, float2& zi) {
    if constexpr (M1B <= J1) {
        constexpr int M2B = MB - M1B + D;
        if constexpr (M2B >= 0 && M2B <= J2) {
            const float2 c = c_cg2[OFF + MB * (J1 + 1) + M1B];
            float2 tr = __fmul2_rn(xr[M1B], yr[M2B]);
            tr = __ffma2_rn(xi[M1B], yn[M2B], tr);
            float2 ti = __fmul2_rn(xr[M1B], yi[M2B]);
            ti = __ffma2_rn(xi[M1B], yr[M2B], ti);
            zr = __ffma2_rn(c, tr, zr);
            zi = __ffma2_rn(c, ti, zi);
        }
        col_terms<J1, J2, OFF, D, MB, M1B + 1>(xr, xi, yr, yi, yn, zr, zi);
    }
}

template <int J1, int J2, int J, int NCOL, bool MID, int OFF, int MB>
__device__ __forceinline__ void cols(uint32_t wa, const float2 (&xr)[J1 + 1], const float2 (&xi)[J1 + 1],
                                     const float2 (&yr)[J2 + 1], const float2 (&yi)[J2 + 1],
                                     const float2 (&yn)[J2 + 1], float2& acc, float2& accm) {
    if constexpr (MB < NCOL) {
        constexpr int D = (J1 + J2 - J) / 2;
        float2 zr = make_float2(0.f, 0.f), zi = make_float2(0.f, 0.f);
        col_terms<J1, J2, OFF, D, MB, 0>(xr, xi, yr, yi, yn, zr, zi);
        const float4 w = lds4i<MB * 512>(wa);
        if constexpr (MID && 2 * MB == J) {
            accm = __ffma2_rn(make_float2(w.x, w.y), zr, accm);
            accm = __ffma2_rn(make_float2(w.z, w.w), zi, accm);
        } else {
            acc = __ffma2_rn(make_float2(w.x, w.y), zr, acc);
            acc = __ffma2_rn(make_float2(w.z, w.w), zi, acc);
        }
        cols<J1, J2, J, NCOL, MID, OFF, MB + 1>(wa, xr, xi, yr, yi, yn, acc, accm);
    }
}

template <int J1, int J2, int J>
__device__ __forceinline__ float2 unit_pairs(uint32_t sbase, int ma, int m1a, float mult) {
    constexpr int d = (J1 + J2 - J) / 2;
    constexpr int OFF = cg_offset(J1, J2, J);
    const int m2a = ma - m1a + d;
    float2 xr[J1 + 1], xi[J1 + 1], yr[J2 + 1], yi[J2 + 1], yn[J2 + 1];
    const float sx = load_row_any<J1>(sbase, m1a, xr, xi);
    const float sy = load_row_any<J2>(sbase, m2a, yr, yi);
    negate_pairs<J2 + 1>(yi, yn);
    const uint32_t wa = sbase + ((uint32_t)hoff(J) + (uint32_t)ma * (J + 1)) * kElemBytes;
    float2 acc = make_float2(0.f, 0.f), accm = make_float2(0.f, 0.f);
    if constexpr ((J & 1) == 0) {
        if (2 * ma == J) {
            cols<J1, J2, J, J / 2 + 1, true, OFF, 0>(wa, xr, xi, yr, yi, yn, acc, accm);
        } else {
            cols<J1, J2, J, J + 1, false, OFF, 0>(wa, xr, xi, yr, yi, yn, acc, accm);
        }
    } else {
        cols<J1, J2, J, J + 1, false, OFF, 0>(wa, xr, xi, yr, yi, yn, acc, accm);
    }
    const float s = c_cg2[OFF + ma * (J1 + 1) + m1a].x * sx * sy * mult;
    return make_float2(s * (2.f * acc.x + accm.x), s * (2.f * acc.y + accm.y));
}

// Float -> 64-bit fixed point (2^-32 units), rounded to nearest with ties away
// from zero, by integer operations on the float's fields (no FP64); requires
// |v| < kFixLimit (v * 2^32 < 2^62).
__device__ __forceinline__ long long to_fixed(float v) {
    const uint32_t b = __float_as_uint(v);
    const int e = (int)((b >> 23) & 0xffu);
    if (e == 0) return 0;  // zero, or below 2^-126
    const unsigned long long m = (b & 0x7fffffu) | 0x800000u;
    const int sh = e - 118;  // v * 2^32 = m * 2^(e - 150 + 32)
    unsigned long long q;
    if (sh >= 0) q = m << sh;
    else if (sh > -25) q = (m + (1ull << (-sh - 1))) >> (-sh);
    else q = 0;
    return (b >> 31) ? -(long long)q : (long long)q;
}

// A triple's units (ma | m1a << 4 | twice << 8) fall into kZbGroups fixed groups
// (unit i in group i mod kZbGroups); a group's values are summed in FP32 in unit
// order and the sum meets its column's total in fixed point.  A warp takes the
// groups first, first + W, ... of a triple.  The groups do not depend on W,
// so every warp count gives the same bits (with W = kZbGroups a warp holds
// exactly one group per triple).
constexpr int kZbGroups = 16;

// the FP32 sum of one group g of a triple's units: units g, g + kZbGroups, ...
template <int J1, int J2, int J>
__device__ __forceinline__ float2 group_sum(uint32_t su, const unsigned short* __restrict__ ul, int n, int g) {
    float2 s = make_float2(0.f, 0.f);
    for (int i = g; i < n; i += kZbGroups) {
        const int e = ul[i];
        const float2 r = unit_pairs<J1, J2, J>(su, e & 0xf, (e >> 4) & 0xf, (e & 0x100) ? 2.f : 1.f);
        s.x += r.x;
        s.y += r.y;
    }
    return s;
}

template <int LO, int HI>
__device__ __forceinline__ float2 group_dispatch(int id, uint32_t su, const unsigned short* ul, int n, int g) {
    if constexpr (HI - LO == 1) {
        return group_sum<triple_field(LO, 0), triple_field(LO, 1), triple_field(LO, 2)>(su, ul, n, g);
    } else {
        constexpr int MIDI = (LO + HI) / 2;
        if (id < MIDI) return group_dispatch<LO, MIDI>(id, su, ul, n, g);
        return group_dispatch<MIDI, HI>(id, su, ul, n, g);
    }
}

// 64-bit fixed point (2^-32 units) -> float: the two words converted apart
__device__ __forceinline__ float from_fixed(long long q) {
    return (float)(int)(q >> 32) + (float)(unsigned)(q & 0xffffffffull) * 2.3283064365386963e-10f;  // 2^-32
}

__device__ __forceinline__ bool zb_wait(uint32_t bar, uint32_t phase) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(bar), "r"(phase)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > 2000000000LL) return false;  // about a second
    }
}

// one tile pair's u block (global) -> shared memory, completing on `bar`
__device__ __forceinline__ void zb_fetch(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Persistent: CTA b takes tile pairs b, b + gridDim.x, ...  A pair's u block
// (128 KB at twojmax 10) comes in by one bulk copy; the next pair's block is
// meanwhile pulled into L2, so the copy reads L2 rather than HBM.
// tri: per triple of this twojmax, int4 (global id, first unit, unit count, output column)
// W: warps per CTA (<= kZbGroups); the fixed groups of units make every W give the same bits
template <int W>
__global__ void __launch_bounds__(W * 32, 1)
    k_zb_units(int tj, const float4* __restrict__ u, const BatchSnap* __restrict__ batch, int nsnap, int64_t tile0,
               int64_t ntiles,
               const int4* __restrict__ tri, int ntri, const unsigned short* __restrict__ units,
               const int* __restrict__ nbr_cnt, float wself3, float* __restrict__ B, int* __restrict__ err) {
    static_assert(W <= kZbGroups, "a warp count above the group count would leave warps idle");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nh = n_half(tj);
    const int nB = n_triples(tj);
    const uint32_t ubytes = (uint32_t)nh * 32u * 16u;
    const uint32_t sbuf0 = (uint32_t)__cvta_generic_to_shared(smem_raw);
    unsigned long long* sacc = reinterpret_cast<unsigned long long*>(smem_raw + (size_t)ubytes);  // [nB][64]
    uint64_t* bars = reinterpret_cast<uint64_t*>(sacc + (size_t)nB * 64);
    long long* spix = reinterpret_cast<long long*>(bars + 2);  // [64] grid point of each (tile, lane), -1 if none
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t npairs = (ntiles + 1) / 2;
    const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&bars[0]);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = threadIdx.x; i < nB * 64; i += blockDim.x) sacc[i] = 0ull;
    __syncthreads();
    uint32_t ph = 0;
    bool bad = false, stalled = false, inflight = false;
    for (int64_t pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
        const bool hasB = 2 * pr + 1 < ntiles;
        // a pair whose 64 points have no neighbour has u^J = w_self I for every
        // J, hence Z = w_self^2 I (orthonormal coupling coefficients) and
        // B = w_self^3 (J + 1): no copy, no contraction
        const int my_cnt = (threadIdx.x < 32 || (threadIdx.x < 64 && hasB)) ? __ldg(nbr_cnt + 64 * pr + threadIdx.x) : 0;
        const bool vacuum = !__syncthreads_or(threadIdx.x < 64 && my_cnt > 0);
        if (threadIdx.x == 0) {
            if (!vacuum) {
                zb_fetch(sbuf0, u + (size_t)pr * nh * 32, ubytes, bar0);
                inflight = true;
            }
            const int64_t nxt = pr + gridDim.x;
            if (nxt < npairs)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(u + (size_t)nxt * nh * 32), "r"(ubytes)
                             : "memory");
        }
        if (!vacuum) {
            const bool got = zb_wait(bar0, ph);
            ph ^= 1u;
            inflight = false;
            if (!__syncthreads_and(got)) {
                stalled = true;
                if (threadIdx.x == 0) inflight = !got;
                break;
            }
        }
        const uint32_t su = sbuf0 + (uint32_t)lane * 16u;
        for (int t = 0; t < ntri && !vacuum; ++t) {
            const int4 d = __ldg(tri + t);  // (gid, start, count, column)
            // this warp's groups: first, first + W, ... (rotated per triple for balance)
            for (int g = ((warp - d.y) % W + W) % W; g < kZbGroups && g < d.z; g += W) {
                const float2 gs = group_dispatch<0, n_triples(kTJMax)>(d.x, su, units + d.y, d.z, g);
                const bool ok = fabsf(gs.x) < kFixLimit && fabsf(gs.y) < kFixLimit;
                bad |= !ok;
                atomicAdd(&sacc[d.w * 64 + lane], (unsigned long long)(ok ? to_fixed(gs.x) : 0ll));       // first tile
                atomicAdd(&sacc[d.w * 64 + 32 + lane], (unsigned long long)(ok ? to_fixed(gs.y) : 0ll));  // second tile
            }
        }
        __syncthreads();
        // grid points of the pair's 64 (tile, lane) slots
        if (threadIdx.x < 64) {
            const int pl = threadIdx.x, l = pl & 31;
            long long q = -1;
            if (!(pl >> 5) || hasB) {
                const int64_t gt = tile0 + 2 * pr + (pl >> 5);
                const int si = batch_find(batch, nsnap, gt);
                const SnapGeom& g = batch[si].sd.g;
                const int64_t tile = gt - batch[si].tile_off;
                const int tx = (int)(tile % g.tiles[0]);
                const int ty = (int)((tile / g.tiles[0]) % g.tiles[1]);
                const int tz = (int)(tile / ((int64_t)g.tiles[0] * g.tiles[1]));
                const int ix = tx * kTileX + (l % kTileX);
                const int iy = ty * kTileY + ((l / kTileX) % kTileY);
                const int iz = tz * kTileZ + l / (kTileX * kTileY);
                if (ix < g.grid[0] && iy < g.grid[1] && iz < g.grid[2])
                    q = batch[si].row_off + ix + (int64_t)g.grid[0] * (iy + (int64_t)g.grid[1] * iz);
            }
            spix[pl] = q;
        }
        // fixed point -> float into the (consumed) u buffer as [slot][nB | 1], accumulators reset
        const int ldo = nB | 1;
        float* out = reinterpret_cast<float*>(smem_raw);
        if (vacuum) {
            for (int i = threadIdx.x; i < nB * 64; i += blockDim.x) {
                const int t = i >> 6, pl = i & 63;
                out[pl * ldo + t] = wself3 * c_zb_jp1[tj / 2][t];
            }
        } else {
            for (int i = threadIdx.x; i < nB * 64; i += blockDim.x) {
                const int t = i >> 6, pl = i & 63;
                out[pl * ldo + t] = from_fixed((long long)sacc[i]);
                sacc[i] = 0ull;
            }
        }
        __syncthreads();
        for (int pl = warp; pl < 64; pl += W) {
            const long long q = spix[pl];
            if (q < 0) continue;
            for (int t = lane; t < nB; t += 32) B[(size_t)q * nB + t] = out[pl * ldo + t];
        }
        __syncthreads();
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicExch(err, 1);
    if (threadIdx.x == 0) {
        if (stalled) atomicExch(err, 2);
        // after a stalled wait: let the copy still in flight land before the CTA exits
        if (inflight) zb_wait(bar0, ph ^ 1u);
    }
}

}  // namespace


// the FP32 units kernel with W warps per CTA, persistent over tile pairs (one CTA per SM)
template <int W>
inline void zb_units_launch(Ctx* c, int twojmax, const float* u_half, const BatchSnap* bs, int nsnap, int64_t tile0,
                            int64_t ntiles, const int* nbr_cnt, double wself, float* B, cudaStream_t st) {
    if (ntiles <= 0) return;
    const size_t smem = sizeof(float4) * (size_t)n_half(twojmax) * 32 +
                        sizeof(long long) * (size_t)n_triples(twojmax) * 64 + 2 * sizeof(uint64_t) + 64 * sizeof(long long);
    cudaFuncSetAttribute(k_zb_units<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int k = twojmax / 2;
    const int64_t npairs = (ntiles + 1) / 2;
    const int grid = (int)std::min<int64_t>(npairs, std::max(1, c->num_sms));
    k_zb_units<W><<<(unsigned)grid, W * 32, smem, st>>>(
        twojmax, reinterpret_cast<const float4*>(u_half), bs, nsnap, tile0, ntiles, c->tables.tri_d + c->tables.tri_off[k],
        c->tables.tri_n[k], c->tables.units_d + c->tables.unit_off[k], nbr_cnt, (float)(wself * wself * wself), B,
        c->tables.err_d);
}

template <class T>
inline void zb_launch_impl(const void*, int twojmax, const T* u_half, const BatchSnap* bs, int nsnap,
                           int64_t tile0, int64_t ntiles, const T* gcg, T* B, cudaStream_t st) {
    using V = typename C2<T>::type;
    const size_t smem = sizeof(V) * (size_t)n_half(twojmax) * 32 + sizeof(T) * (size_t)n_triples(twojmax) * 32;
    k_zb<T><<<(unsigned)ntiles, kZbWarps * 32, smem, st>>>(twojmax, reinterpret_cast<const V*>(u_half), bs, nsnap,
                                                            tile0, ntiles, gcg, B);
}

}  // namespace mala
