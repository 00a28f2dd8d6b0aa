// snap_zb.cuh -- device side of compute_zi + compute_bi (see snap_zb.cu).
// Included by the FP32 and FP64 translation units, each of which owns its
// own copy of the constant-memory tables.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "mala_internal.h"
#include "snap_common.cuh"

namespace mala {

constexpr int kZbWarps = 8;
constexpr int kZbMaxList = 32;
constexpr int kCgSize = cg_table_size();

// Clebsch-Gordan table as (c, c) pairs: one operand of a packed FP32x2 FMA
static __constant__ float2 c_cg2[kCgSize];
// full (J+1)^2 element -> half-set element: index | mirrored << 16 | negate << 17
constexpr int kNFull = n_full(kTJMax);
static __constant__ int c_fullmap[kNFull];
// per supported twojmax (index tj/2): [warp][slot] = global triple id | (local index << 8), -1 = end
static __constant__ int c_zb_list[kTJMax / 2 + 1][kZbWarps][kZbMaxList];

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
    k_zb(int tj, const typename C2<T>::type* __restrict__ u, SnapGeom g, int64_t tile0, int64_t ntiles,
         const T* __restrict__ gcg, T* __restrict__ B) {
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
    const int64_t tile = tile0 + tl;
    const int tx = (int)(tile % g.tiles[0]);
    const int ty = (int)((tile / g.tiles[0]) % g.tiles[1]);
    const int tz = (int)(tile / ((int64_t)g.tiles[0] * g.tiles[1]));
    for (int idx = threadIdx.x; idx < 32 * nB; idx += blockDim.x) {
        const int l = idx / nB, t = idx % nB;
        const int ix = tx * kTileX + (l % kTileX);
        const int iy = ty * kTileY + ((l / kTileX) % kTileY);
        const int iz = tz * kTileZ + l / (kTileX * kTileY);
        if (ix >= g.grid[0] || iy >= g.grid[1] || iz >= g.grid[2]) continue;
        const int64_t p = ix + (int64_t)g.grid[0] * (iy + (int64_t)g.grid[1] * iz);
        B[(size_t)p * nB + t] = sB[t * 32 + l];
    }
}


// ---- FP32 kernel: all warps of an SM sweep the same triple -------------------
//
// B is linear in each (row ma, u^J1 row m1a) contribution:
//   B = sum_{ma, m1a} c1(ma, m1a) * sum_mb w(ma, mb) Re(conj(u^J[ma][mb]) conv_{ma,m1a}[mb]),
// so a "unit" (triple, ma, m1a) yields a scalar per point.  One CTA of 16
// warps owns an SM (the full u of its tile, 130 KB at twojmax = 10, fills the
// shared memory); the warps walk the triples in the same order and deal each
// triple's units round-robin, so the whole SM executes one triple's unrolled
// code at a time and the instruction cache holds it.  The u half set is
// expanded to full (J+1)^2 blocks while staging, so rows load without any
// mirror arithmetic.  Per-warp partial sums are added in 64-bit fixed point
// (2^-32 resolution) with shared-memory atomics: integer addition is
// associative, so B does not depend on the order of the warps.

constexpr int kZbUWarps = 16;
constexpr double kFixScale = 4294967296.0;  // 2^32
constexpr float kFixLimit = 1.0e9f;          // |partial| bound that keeps 16 partials inside int64

template <int IMM>
__device__ __forceinline__ float2 lds2(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2+%3];" : "=f"(v.x), "=f"(v.y) : "r"(addr), "n"(IMM));
    return v;
}

template <int N, int I = 0>
__device__ __forceinline__ void lds_row(float2 (&v)[N], uint32_t addr) {
    if constexpr (I < N) {
        v[I] = lds2<I * 256>(addr);
        lds_row<N, I + 1>(v, addr);
    }
}

// The contraction of one unit, fully expanded at compile time (template
// recursion: no index of a register array is ever a run-time value), in
// outer-product order: for each x element, the terms of all columns follow
// one another, so consecutive instructions update independent accumulators.
//   ACC = 0: z = (c2, c2) * t + z as one packed FMA (pair table in constant memory)
//   ACC = 1: z.re += c2 t.re, z.im += c2 t.im as scalar FMAs with a constant operand
#ifndef MALA_ZB_ACC
#define MALA_ZB_ACC 0
#endif

template <int J1, int J2, int OFF, int D, int NCOL, int M1B, int MB>
__device__ __forceinline__ void conv_row(const float2 (&xx)[J1 + 1], const float2 (&xs)[J1 + 1],
                                         const float2 (&y)[J2 + 1], const float2 (&ys)[J2 + 1], float2 (&z)[NCOL]) {
    if constexpr (MB < NCOL) {
        constexpr int M2B = MB - M1B + D;
        if constexpr (M2B >= 0 && M2B <= J2) {
            float2 t = __fmul2_rn(xx[M1B], y[M2B]);
            t = __ffma2_rn(xs[M1B], ys[M2B], t);
#if MALA_ZB_ACC == 0
            z[MB] = __ffma2_rn(c_cg2[OFF + MB * (J1 + 1) + M1B], t, z[MB]);
#else
            const float c = c_cg2[OFF + MB * (J1 + 1) + M1B].x;
            z[MB].x = fmaf(c, t.x, z[MB].x);
            z[MB].y = fmaf(c, t.y, z[MB].y);
#endif
        }
        conv_row<J1, J2, OFF, D, NCOL, M1B, MB + 1>(xx, xs, y, ys, z);
    }
}

template <int J1, int J2, int OFF, int D, int NCOL, int M1B>
__device__ __forceinline__ void conv_all(const float2 (&xx)[J1 + 1], const float2 (&xs)[J1 + 1],
                                         const float2 (&y)[J2 + 1], const float2 (&ys)[J2 + 1], float2 (&z)[NCOL]) {
    if constexpr (M1B <= J1) {
        conv_row<J1, J2, OFF, D, NCOL, M1B, 0>(xx, xs, y, ys, z);
        conv_all<J1, J2, OFF, D, NCOL, M1B + 1>(xx, xs, y, ys, z);
    }
}

template <int J, int NCOL, bool MID, int MB>
__device__ __forceinline__ void dot_cols(const float2 (&wv)[NCOL], const float2 (&z)[NCOL], float2& acc,
                                         float2& accm) {
    if constexpr (MB < NCOL) {
        if constexpr (MID && 2 * MB == J)
            accm = __ffma2_rn(wv[MB], z[MB], accm);
        else
            acc = __ffma2_rn(wv[MB], z[MB], acc);
        dot_cols<J, NCOL, MID, MB + 1>(wv, z, acc, accm);
    }
}

template <int N, int I = 0>
__device__ __forceinline__ void zero2(float2 (&z)[N]) {
    if constexpr (I < N) {
        z[I] = make_float2(0.f, 0.f);
        zero2<N, I + 1>(z);
    }
}

template <int N, int I = 0>
__device__ __forceinline__ void prep_x(const float2 (&v)[N], float2 (&xx)[N], float2 (&xs)[N]) {
    if constexpr (I < N) {
        xx[I] = make_float2(v[I].x, v[I].x);
        xs[I] = make_float2(-v[I].y, v[I].y);
        prep_x<N, I + 1>(v, xx, xs);
    }
}

template <int N, int I = 0>
__device__ __forceinline__ void prep_y(const float2 (&v)[N], float2 (&ys)[N]) {
    if constexpr (I < N) {
        ys[I] = make_float2(v[I].y, v[I].x);
        prep_y<N, I + 1>(v, ys);
    }
}

// One unit: conv[mb] = sum_m1b c2(mb, m1b) x[m1b] y[mb - m1b + d] (complex),
// returned as c1 * sum_mb weight(mb) Re(conj(w[mb]) conv[mb]).  The complex
// products run on packed FP32x2 instructions: with xx = (x.re, x.re),
// xs = (-x.im, x.im) and ys = (y.im, y.re),
//   t = xx * y;  t = xs * ys + t  (= x y);  z = (c2, c2) * t + z.
// Shared-memory addresses are 32-bit; each row is one base plus immediates.
template <int J1, int J2, int J, int NCOL, bool MID>
__device__ __forceinline__ float unit_full(uint32_t sbase, int ma, int m1a) {
    constexpr int d = (J1 + J2 - J) / 2;
    constexpr int OFF = cg_offset(J1, J2, J);
    const int m2a = ma - m1a + d;
    constexpr uint32_t F1 = full_off(J1) * 256u, F2 = full_off(J2) * 256u, FJ = full_off(J) * 256u;
    const uint32_t xa = sbase + F1 + (uint32_t)m1a * ((J1 + 1) * 256u);
    const uint32_t ya = sbase + F2 + (uint32_t)m2a * ((J2 + 1) * 256u);
    const uint32_t wa = sbase + FJ + (uint32_t)ma * ((J + 1) * 256u);
    float2 xv[J1 + 1], xx[J1 + 1], xs[J1 + 1], y[J2 + 1], ys[J2 + 1], wv[NCOL];
    lds_row<J1 + 1>(xv, xa);
    lds_row<J2 + 1>(y, ya);
    lds_row<NCOL>(wv, wa);
    prep_x<J1 + 1>(xv, xx, xs);
    prep_y<J2 + 1>(y, ys);
    float2 z[NCOL];
    zero2<NCOL>(z);
    conv_all<J1, J2, OFF, d, NCOL, 0>(xx, xs, y, ys, z);
    float2 acc = make_float2(0.f, 0.f), accm = make_float2(0.f, 0.f);
    dot_cols<J, NCOL, MID, 0>(wv, z, acc, accm);
    const float r = 2.f * (acc.x + acc.y) + (accm.x + accm.y);
    return c_cg2[OFF + ma * (J1 + 1) + m1a].x * r;
}

// this warp's units (ma | m1a << 4) of one triple, starting at `first`
template <int J1, int J2, int J>
__device__ __forceinline__ float triple_units(uint32_t su, const unsigned short* __restrict__ ul, int n, int first) {
    float acc = 0.f;
    for (int i = first; i < n; i += kZbUWarps) {
        const int e = ul[i];
        const int ma = e & 0xf, m1a = e >> 4;
        if constexpr ((J & 1) == 0) {
            if (2 * ma == J) {
                acc += unit_full<J1, J2, J, J / 2 + 1, true>(su, ma, m1a);
                continue;
            }
        }
        acc += unit_full<J1, J2, J, J + 1, false>(su, ma, m1a);
    }
    return acc;
}

template <int LO, int HI>
__device__ __forceinline__ float triple_dispatch(int id, uint32_t su, const unsigned short* ul, int n, int first) {
    if constexpr (HI - LO == 1) {
        return triple_units<triple_field(LO, 0), triple_field(LO, 1), triple_field(LO, 2)>(su, ul, n, first);
    } else {
        constexpr int MIDI = (LO + HI) / 2;
        if (id < MIDI) return triple_dispatch<LO, MIDI>(id, su, ul, n, first);
        return triple_dispatch<MIDI, HI>(id, su, ul, n, first);
    }
}

// tri: per triple of this twojmax, int4 (global id, first unit, unit count, output column)
__global__ void __launch_bounds__(kZbUWarps * 32, 1)
    k_zb_units(int tj, const float2* __restrict__ u, SnapGeom g, int64_t tile0, int64_t ntiles,
               const int4* __restrict__ tri, int ntri, const unsigned short* __restrict__ units,
               float* __restrict__ B, int* __restrict__ err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nh = n_half(tj), nf = n_full(tj);
    const int nB = n_triples(tj);
    float2* su_all = reinterpret_cast<float2*>(smem_raw);
    unsigned long long* sacc = reinterpret_cast<unsigned long long*>(smem_raw + sizeof(float2) * (size_t)nf * 32);
    const int64_t tl = blockIdx.x;
    if (tl >= ntiles) return;
    // stage: expand the half set into full (J+1)^2 blocks
    {
        const float2* src = u + (size_t)tl * nh * 32;
        for (int idx = threadIdx.x; idx < nf * 32; idx += blockDim.x) {
            const int e = idx >> 5, l = idx & 31;
            const int m = c_fullmap[e];
            float2 v = src[(size_t)(m & 0xffff) * 32 + l];
            if (m & 0x10000) {  // mirrored element: (-1)^(ma-mb) conj
                const float sg = (m & 0x20000) ? -1.f : 1.f;
                v.x = sg * v.x;
                v.y = -sg * v.y;
            }
            su_all[idx] = v;
        }
        for (int i = threadIdx.x; i < nB * 32; i += blockDim.x) sacc[i] = 0ull;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t su = (uint32_t)__cvta_generic_to_shared(su_all) + (uint32_t)lane * 8u;
    bool bad = false;
    for (int t = 0; t < ntri; ++t) {
        const int4 d = __ldg(tri + t);  // (gid, start, count, column)
        const int first = ((warp - d.y) % kZbUWarps + kZbUWarps) % kZbUWarps;
        if (first >= d.z) continue;
        const float acc = triple_dispatch<0, n_triples(kTJMax)>(d.x, su, units + d.y, d.z, first);
        bad |= !(fabsf(acc) < kFixLimit);
        atomicAdd(&sacc[d.w * 32 + lane], (unsigned long long)__double2ll_rn((double)acc * kFixScale));
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicExch(err, 1);
    __syncthreads();
    const int64_t tile = tile0 + tl;
    const int tx = (int)(tile % g.tiles[0]);
    const int ty = (int)((tile / g.tiles[0]) % g.tiles[1]);
    const int tz = (int)(tile / ((int64_t)g.tiles[0] * g.tiles[1]));
    for (int idx = threadIdx.x; idx < 32 * nB; idx += blockDim.x) {
        const int l = idx / nB, t = idx % nB;
        const int ix = tx * kTileX + (l % kTileX);
        const int iy = ty * kTileY + ((l / kTileX) % kTileY);
        const int iz = tz * kTileZ + l / (kTileX * kTileY);
        if (ix >= g.grid[0] || iy >= g.grid[1] || iz >= g.grid[2]) continue;
        const int64_t p = ix + (int64_t)g.grid[0] * (iy + (int64_t)g.grid[1] * iz);
        B[(size_t)p * nB + t] = (float)((double)(long long)sacc[t * 32 + l] * (1.0 / kFixScale));
    }
}

}  // namespace


template <class T>
inline void zb_launch_impl(const void*, int twojmax, const T* u_half, const SnapGeom& g,
                           int64_t tile0, int64_t ntiles, const T* gcg, T* B, cudaStream_t st) {
    using V = typename C2<T>::type;
    const size_t smem = sizeof(V) * (size_t)n_half(twojmax) * 32 + sizeof(T) * (size_t)n_triples(twojmax) * 32;
    k_zb<T><<<(unsigned)ntiles, kZbWarps * 32, smem, st>>>(twojmax, reinterpret_cast<const V*>(u_half), g, tile0,
                                                            ntiles, gcg, B);
}

}  // namespace mala
