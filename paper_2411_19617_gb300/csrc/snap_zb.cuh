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

static __constant__ float c_cg[kCgSize];
// per supported twojmax (index tj/2): [warp][slot] = global triple id | (local index << 8), -1 = end
static __constant__ int c_zb_list[kTJMax / 2 + 1][kZbWarps][kZbMaxList];

namespace {

template <class T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };

template <class T> __device__ __forceinline__ T cg_at(const T* gtab, int idx);
template <> __device__ __forceinline__ float cg_at<float>(const float*, int idx) { return c_cg[idx]; }
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

template <int J1, int J2, int J, int NCOL, bool MID>
__device__ __forceinline__ float unit_full(const float2* __restrict__ su, int ma, int m1a) {
    constexpr int d = (J1 + J2 - J) / 2;
    constexpr int OFF = cg_offset(J1, J2, J);
    const int m2a = ma - m1a + d;
    const float2* xr = su + (size_t)(full_off(J1) + m1a * (J1 + 1)) * 32;
    const float2* yr = su + (size_t)(full_off(J2) + m2a * (J2 + 1)) * 32;
    float2 x[J1 + 1], y[J2 + 1];
#pragma unroll
    for (int k = 0; k <= J1; ++k) x[k] = xr[k * 32];
#pragma unroll
    for (int k = 0; k <= J2; ++k) y[k] = yr[k * 32];
    float zr[NCOL], zi[NCOL];
#pragma unroll
    for (int mb = 0; mb < NCOL; ++mb) {
        zr[mb] = 0.f;
        zi[mb] = 0.f;
#pragma unroll
        for (int m1b = 0; m1b <= J1; ++m1b) {
            const int m2b = mb - m1b + d;
            if (m2b >= 0 && m2b <= J2) {
                const float c2 = c_cg[OFF + mb * (J1 + 1) + m1b];
                const float tr = x[m1b].x * y[m2b].x - x[m1b].y * y[m2b].y;
                const float ti = x[m1b].x * y[m2b].y + x[m1b].y * y[m2b].x;
                zr[mb] += c2 * tr;
                zi[mb] += c2 * ti;
            }
        }
    }
    const float2* w = su + (size_t)(full_off(J) + ma * (J + 1)) * 32;
    float r = 0.f;
#pragma unroll
    for (int mb = 0; mb < NCOL; ++mb) {
        const float2 v = w[mb * 32];
        const float t = v.x * zr[mb] + v.y * zi[mb];
        r += (MID && 2 * mb == J) ? t : 2.f * t;
    }
    return c_cg[OFF + ma * (J1 + 1) + m1a] * r;
}

// this warp's units (ma | m1a << 4) of one triple, starting at `first`
template <int J1, int J2, int J>
__device__ __forceinline__ float triple_units(const float2* __restrict__ su, const unsigned short* __restrict__ ul,
                                              int n, int first) {
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
__device__ __forceinline__ float triple_dispatch(int id, const float2* su, const unsigned short* ul, int n, int first) {
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
            int J = 0;
            while (full_off(J + 1) <= e) ++J;
            const int r = e - full_off(J);
            const int ma = r / (J + 1), mb = r % (J + 1);
            const bool direct = (2 * ma < J) || (2 * ma == J && 2 * mb <= J);
            const int sma = direct ? ma : J - ma, smb = direct ? mb : J - mb;
            float2 v = src[(size_t)(hoff(J) + sma * (J + 1) + smb) * 32 + l];
            if (!direct) {
                const float sg = ((sma - smb) & 1) ? -1.f : 1.f;
                v.x = sg * v.x;
                v.y = -sg * v.y;
            }
            su_all[idx] = v;
        }
        for (int i = threadIdx.x; i < nB * 32; i += blockDim.x) sacc[i] = 0ull;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float2* su = su_all + lane;
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
