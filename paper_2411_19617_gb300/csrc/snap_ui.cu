// snap_ui.cu -- compute_ui: expansion coefficients u_j of the ionic density
// (paper Eq. ionicdensity expanded in the hyperspherical harmonics of
// Eq. SNAPExpansion):
//     u^J = wself I + sum_k c_k U^J(a_k, b_k),   c_k = w_eta f_c(r_k).
//
// U^J of the SU(2) element [[conj a, -conj b], [b, a]] has columns
//     U^J[.][mb] = N(J, ., mb) * coeffs of (conj(a) xi - conj(b) eta)^(J-mb) (b xi + a eta)^mb
// (coefficient of xi^(J-ma) eta^ma in row ma, N the normalisation
// sqrt((J-ma)! ma! / ((J-mb)! mb!))).  A column therefore grows level by level
// by multiplying a coefficient vector with one linear form:
//     column mb of level J   = (conj a xi - conj b eta) * column mb of level J-1,
//     column mb of level 2mb = (b xi + a eta)(conj a xi - conj b eta) * column mb-1 of level 2mb-2.
// Only columns mb <= J/2 are generated; the others follow from
// U[J-ma][J-mb] = (-1)^(ma-mb) conj(U[ma][mb]).
//
// Mapping: one warp per tile of 32 grid points, lane = point.  The elements
// are split into "segments" (one column chain over a range of levels) small
// enough that their sums and Kahan compensations stay in registers; each
// segment loops over the lane's neighbours, rebuilding its column from the
// seed, and accumulates c_k * coefficient with compensated (Kahan) summation;
// the chain starts from c_k instead of 1 (the recursion is linear), so every
// coefficient arrives already weighted.
// FP32 takes the neighbours two at a time: both column chains run packed in
// FP32x2 pairs (one FFMA2 does a step of both), and the two weighted terms of
// an element are added in one rounding before the compensated add, which
// halves the compensation work per neighbour.
// The normalisation N and the self term are applied once at the end.  Output:
// the half set of u (rows ma < J/2, plus the middle row's columns <= J/2 for
// even J).  FP64: [tile][element][lane] (re, im).  FP32: tiles in pairs,
// [pair][element][lane] (re A, re B, im A, im B) with A the even tile of the
// pair and B the odd one, the layout compute_zi/bi works in.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "mala_internal.h"
#include "snap_common.cuh"

namespace mala {

namespace {

// normalisation sqrt((J-ma)! ma! / ((J-mb)! mb!)) of U^J, [J][ma][mb], filled by the host
__constant__ double c_unorm_d[(kTJMax + 1) * (kTJMax + 1) * (kTJMax + 1)];
__constant__ float c_unorm_f[(kTJMax + 1) * (kTJMax + 1) * (kTJMax + 1)];

template <class T> __device__ __forceinline__ T unorm_at(int idx);
template <> __device__ __forceinline__ float unorm_at<float>(int idx) { return c_unorm_f[idx]; }
template <> __device__ __forceinline__ double unorm_at<double>(int idx) { return c_unorm_d[idx]; }

// FP32 variants (segment elements, warps per CTA): sums + compensations of up to SEG complex
// numbers per segment live in registers, so longer segments (fewer chain re-walks) need fewer
// warps per CTA (255 registers a thread at 8 warps, 168 at 12; the register file is split over
// the four schedulers, so 10 warps get no more than 12).  Which one is fastest depends
// on the neighbour count; the tuner times them on the data.  Every variant adds every element's
// terms in the same order, so all give the same bits.
struct UiVariant {
    int seg, warps;
};
constexpr UiVariant kUiVariantsF32[] = {{36, 8}, {30, 8}, {20, 12}};
constexpr int kNumUiVariantsF32 = 3;
constexpr int kSegElemsF64 = 10;
constexpr int kUiWarpsF64 = 6;

struct Seg {
    int mb, l0, l1;
};
struct SegPlan {
    Seg s[64];
    int n;
};

__host__ __device__ constexpr int seg_level_elems(int mb, int J) { return (2 * mb == J) ? mb + 1 : J + 1; }
__host__ __device__ constexpr int seg_offset(int mb, int l0, int J) {
    int o = 0;
    for (int k = l0; k < J; ++k) o += seg_level_elems(mb, k);
    return o;
}

__host__ __device__ constexpr SegPlan make_plan(int tj, int emax) {
    SegPlan p{};
    p.n = 0;
    for (int mb = 0; 2 * mb <= tj; ++mb) {
        int l0 = 2 * mb, acc = 0;
        for (int J = 2 * mb; J <= tj; ++J) {
            const int e = seg_level_elems(mb, J);
            if (acc > 0 && acc + e > emax) {
                p.s[p.n] = Seg{mb, l0, J - 1};
                ++p.n;
                l0 = J;
                acc = 0;
            }
            acc += e;
        }
        p.s[p.n] = Seg{mb, l0, tj};
        ++p.n;
    }
    return p;
}

template <int TJ, int SEG> struct Plan {
    static constexpr SegPlan value = make_plan(TJ, SEG);
};

template <class T> struct C2;
template <> struct C2<float> { using type = float2; };
template <> struct C2<double> { using type = double2; };
template <class T> struct AB4;
template <> struct AB4<float> { using type = float4; };
template <> struct AB4<double> { using type = double4; };

// v <- (alpha xi + beta eta) v for a coefficient vector of length n
// (-> n + 1); alpha = (alr, ali), beta = (ber, bei).  n must be a
// compile-time constant after unrolling so that v stays in registers.
template <class T>
__device__ __forceinline__ void mul_linear(T (&vr)[kTJMax + 1], T (&vi)[kTJMax + 1], int n, T alr, T ali,
                                           T ber, T bei) {
#pragma unroll
    for (int i = kTJMax; i >= 0; --i) {
        if (i <= n) {
            T nr = T(0), ni = T(0);
            if (i < n) {
                nr = alr * vr[i] - ali * vi[i];
                ni = alr * vi[i] + ali * vr[i];
            }
            if (i > 0) {
                nr += ber * vr[i - 1] - bei * vi[i - 1];
                ni += ber * vi[i - 1] + bei * vr[i - 1];
            }
            vr[i] = nr;
            vi[i] = ni;
        }
    }
}

// the same for a pair of coefficient vectors (two neighbours) in FP32x2:
// v <- (alpha xi + beta eta) v per neighbour, nali = -ali and nbei = -bei
__device__ __forceinline__ void mul_linear2(float2 (&vr)[kTJMax + 1], float2 (&vi)[kTJMax + 1], int n, float2 alr,
                                            float2 ali, float2 nali, float2 ber, float2 bei, float2 nbei) {
#pragma unroll
    for (int i = kTJMax; i >= 0; --i) {
        if (i <= n) {
            float2 nr, ni;
            if (i < n) {
                nr = __ffma2_rn(nali, vi[i], __fmul2_rn(alr, vr[i]));
                ni = __ffma2_rn(ali, vr[i], __fmul2_rn(alr, vi[i]));
                if (i > 0) {
                    nr = __ffma2_rn(nbei, vi[i - 1], __ffma2_rn(ber, vr[i - 1], nr));
                    ni = __ffma2_rn(bei, vr[i - 1], __ffma2_rn(ber, vi[i - 1], ni));
                }
            } else {
                nr = __ffma2_rn(nbei, vi[i - 1], __fmul2_rn(ber, vr[i - 1]));
                ni = __ffma2_rn(bei, vr[i - 1], __fmul2_rn(ber, vi[i - 1]));
            }
            vr[i] = nr;
            vi[i] = ni;
        }
    }
}

template <class T>
__device__ __forceinline__ void kahan_add(T& s, T& c, T x) {
    const T y = x - c;
    const T t = s + y;
    c = (t - s) - y;
    s = t;
}

template <class T>
__device__ __forceinline__ void load_nbr(const typename AB4<T>::type* __restrict__ ab_t, const T* __restrict__ cw_t,
                                         int k, int cnt, int lane, typename AB4<T>::type& ab, T& c) {
    if (k < cnt) {
        ab = ab_t[(size_t)k * 32 + lane];
        c = cw_t[(size_t)k * 32 + lane];
    } else {
        ab.x = T(1);
        ab.y = ab.z = ab.w = T(0);
        c = T(0);
    }
}

// element `slot` of the lane's point; uo is the tile's (FP64) or the tile
// pair's (FP32) block, h the tile's half of the pair
template <class T>
__device__ __forceinline__ void store_u(typename C2<T>::type* __restrict__ uo, int h, int slot, int lane,
                                        typename C2<T>::type o) {
    if constexpr (sizeof(T) == 8) {
        uo[(size_t)slot * 32 + lane] = o;
    } else {
        float* q = reinterpret_cast<float*>(uo) + ((size_t)slot * 32 + lane) * 4 + h;
        q[0] = o.x;
        q[2] = o.y;
    }
}

template <class T, int TJ, int MB, int L0, int L1>
__device__ __forceinline__ void ui_segment(const typename AB4<T>::type* __restrict__ ab_t,
                                           const T* __restrict__ cw_t, int cnt, int kwarp, int lane, T wself,
                                           bool store, typename C2<T>::type* __restrict__ uo, int h) {
    constexpr int NE = seg_offset(MB, L0, L1 + 1);
    T sr[NE], si[NE], cr[NE], ci[NE];
#pragma unroll
    for (int e = 0; e < NE; ++e) sr[e] = si[e] = cr[e] = ci[e] = T(0);

    if constexpr (sizeof(T) == 4) {
        // FP32: two neighbours per step; their column chains run packed in FP32x2
        // pairs, and the two weighted terms of an element are added (one rounding)
        // before the compensated add to the sum
        float4 abn0, abn1;
        float cn0, cn1;
        load_nbr<float>(ab_t, cw_t, 0, cnt, lane, abn0, cn0);
        load_nbr<float>(ab_t, cw_t, 1, cnt, lane, abn1, cn1);
        for (int k = 0; k < kwarp; k += 2) {
            const float4 a0 = abn0, a1 = abn1;
            const float2 c2 = make_float2(cn0, cn1);
            load_nbr<float>(ab_t, cw_t, k + 2, cnt, lane, abn0, cn0);  // prefetch the next pair
            load_nbr<float>(ab_t, cw_t, k + 3, cnt, lane, abn1, cn1);
            // linear forms per neighbour: L1 = conj(a) xi - conj(b) eta, L2 = b xi + a eta
            const float2 l1ar = make_float2(a0.x, a1.x), l1ai = make_float2(-a0.y, -a1.y);
            const float2 l1br = make_float2(-a0.z, -a1.z), l1bi = make_float2(a0.w, a1.w);
            const float2 l2ar = make_float2(a0.z, a1.z), l2ai = make_float2(a0.w, a1.w);
            const float2 l2br = make_float2(a0.x, a1.x), l2bi = make_float2(a0.y, a1.y);
            const float2 nl1ai = make_float2(a0.y, a1.y), nl1bi = make_float2(-a0.w, -a1.w);
            const float2 nl2ai = make_float2(-a0.w, -a1.w), nl2bi = make_float2(-a0.y, -a1.y);
            // the chain starts from the neighbour's weight: every level comes out scaled by c
            float2 vr[kTJMax + 1], vi[kTJMax + 1];
            vr[0] = c2;
            vi[0] = make_float2(0.f, 0.f);
#pragma unroll
            for (int st = 0; st < MB; ++st) {
                mul_linear2(vr, vi, 2 * st + 1, l1ar, l1ai, nl1ai, l1br, l1bi, nl1bi);
                mul_linear2(vr, vi, 2 * st + 2, l2ar, l2ai, nl2ai, l2br, l2bi, nl2bi);
            }
#pragma unroll
            for (int J = 2 * MB; J <= L1; ++J) {
                if (J > 2 * MB) mul_linear2(vr, vi, J, l1ar, l1ai, nl1ai, l1br, l1bi, nl1bi);
                if (J >= L0) {
                    const int off = seg_offset(MB, L0, J);
                    const int ne = seg_level_elems(MB, J);
#pragma unroll
                    for (int i = 0; i < kTJMax + 1; ++i) {
                        if (i < ne) {
                            kahan_add(sr[off + i], cr[off + i], vr[i].x + vr[i].y);
                            kahan_add(si[off + i], ci[off + i], vi[i].x + vi[i].y);
                        }
                    }
                }
            }
        }
    } else {
    typename AB4<T>::type abn;
    T cn;
    load_nbr<T>(ab_t, cw_t, 0, cnt, lane, abn, cn);
    for (int k = 0; k < kwarp; ++k) {
        const typename AB4<T>::type ab = abn;
        const T c = cn;
        load_nbr<T>(ab_t, cw_t, k + 1, cnt, lane, abn, cn);  // prefetch the next record
        // linear forms: L1 = conj(a) xi - conj(b) eta, L2 = b xi + a eta
        const T l1ar = ab.x, l1ai = -ab.y, l1br = -ab.z, l1bi = ab.w;
        const T l2ar = ab.z, l2ai = ab.w, l2br = ab.x, l2bi = ab.y;
        T vr[kTJMax + 1], vi[kTJMax + 1];
        vr[0] = c;  // the chain starts from the neighbour's weight: every level comes out scaled by c
        vi[0] = T(0);
        // seed: (L1 L2)^MB at level 2 MB
#pragma unroll
        for (int st = 0; st < MB; ++st) {
            mul_linear<T>(vr, vi, 2 * st + 1, l1ar, l1ai, l1br, l1bi);
            mul_linear<T>(vr, vi, 2 * st + 2, l2ar, l2ai, l2br, l2bi);
        }
#pragma unroll
        for (int J = 2 * MB; J <= L1; ++J) {
            if (J > 2 * MB) mul_linear<T>(vr, vi, J, l1ar, l1ai, l1br, l1bi);  // length J -> J+1
            if (J >= L0) {
                const int off = seg_offset(MB, L0, J);
                const int ne = seg_level_elems(MB, J);
#pragma unroll
                for (int i = 0; i < kTJMax + 1; ++i) {
                    if (i < ne) {
                        kahan_add(sr[off + i], cr[off + i], vr[i]);
                        kahan_add(si[off + i], ci[off + i], vi[i]);
                    }
                }
            }
        }
    }
    }
    if (!store) return;
    // normalise, map to the half set, add the self term, store
#pragma unroll
    for (int J = L0; J <= L1; ++J) {
        const int off = seg_offset(MB, L0, J);
        const int ne = seg_level_elems(MB, J);
#pragma unroll
        for (int i = 0; i < kTJMax + 1; ++i) {
            if (i < ne) {
                const T nrm = unorm_at<T>((J * (kTJMax + 1) + i) * (kTJMax + 1) + MB);
                T vr_ = (sr[off + i] - cr[off + i]) * nrm;
                T vi_ = (si[off + i] - ci[off + i]) * nrm;
                typename C2<T>::type o;
                int slot;
                if (2 * i <= J) {
                    slot = hoff(J) + i * (J + 1) + MB;
                    if (i == MB) vr_ += wself;
                    o.x = vr_;
                    o.y = vi_;
                } else {
                    slot = hoff(J) + (J - i) * (J + 1) + (J - MB);
                    const T sg = ((i - MB) & 1) ? T(-1) : T(1);
                    o.x = sg * vr_;
                    o.y = -sg * vi_;
                }
                store_u<T>(uo, h, slot, lane, o);
            }
        }
    }
}

// All warps of the block run the same segment between barriers, so the SM
// fetches one segment's code at a time.
template <class T, int TJ, int SEG, int I>
__device__ __forceinline__ void run_segments(const typename AB4<T>::type* ab_t, const T* cw_t, int cnt, int kwarp,
                                             int lane, T wself, bool store, typename C2<T>::type* uo, int h) {
    if constexpr (I < Plan<TJ, SEG>::value.n) {
        constexpr Seg sg = Plan<TJ, SEG>::value.s[I];
        ui_segment<T, TJ, sg.mb, sg.l0, sg.l1>(ab_t, cw_t, cnt, kwarp, lane, wself, store, uo, h);
        __syncthreads();
        run_segments<T, TJ, SEG, I + 1>(ab_t, cw_t, cnt, kwarp, lane, wself, store, uo, h);
    }
}

template <class T, int TJ, int SEG, int W>
__global__ void __launch_bounds__(W * 32, 1)
    k_ui(const typename AB4<T>::type* __restrict__ ab, const T* __restrict__ cw, const int* __restrict__ cnt,
         int kmax, T wself, int64_t ntiles, typename C2<T>::type* __restrict__ u) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t tl = (int64_t)blockIdx.x * W + warp;
    const bool live = tl < ntiles;
    const int64_t tls = live ? tl : 0;
    const int n = live ? cnt[tls * 32 + lane] : 0;
    const int kw = __reduce_max_sync(0xffffffffu, n);
    const auto* ab_t = ab + (size_t)tls * kmax * 32;
    const T* cw_t = cw + (size_t)tls * kmax * 32;
    // FP64: one block per tile; FP32: one block of two float2 per element and lane per tile pair
    auto* uo = (sizeof(T) == 8) ? u + (size_t)tls * n_half(TJ) * 32 : u + (size_t)(tls >> 1) * n_half(TJ) * 32 * 2;
    run_segments<T, TJ, SEG, 0>(ab_t, cw_t, n, kw, lane, wself, live, uo, (int)(tls & 1));
}

// half set -> full (J+1)^2 blocks per point, point-major (for tests / the ABI)
template <class T>
__global__ void k_u_expand(int tj, const typename C2<T>::type* __restrict__ uh, SnapGeom g, int64_t tile0,
                           int64_t ntiles, T* __restrict__ uf) {
    const int64_t tl = blockIdx.x;
    if (tl >= ntiles) return;
    const int64_t tile = tile0 + tl;
    const int tx = (int)(tile % g.tiles[0]);
    const int ty = (int)((tile / g.tiles[0]) % g.tiles[1]);
    const int tz = (int)(tile / ((int64_t)g.tiles[0] * g.tiles[1]));
    const int nh = n_half(tj), nf = n_full(tj);
    for (int idx = threadIdx.x; idx < 32 * nf; idx += blockDim.x) {
        const int lane = idx / nf, e = idx % nf;
        const int ix = tx * kTileX + (lane % kTileX);
        const int iy = ty * kTileY + ((lane / kTileX) % kTileY);
        const int iz = tz * kTileZ + lane / (kTileX * kTileY);
        if (ix >= g.grid[0] || iy >= g.grid[1] || iz >= g.grid[2]) continue;
        const int64_t p = ix + (int64_t)g.grid[0] * (iy + (int64_t)g.grid[1] * iz);
        int J = 0;
        while (full_off(J + 1) <= e) ++J;
        const int r = e - full_off(J);
        const int ma = r / (J + 1), mb = r % (J + 1);
        bool direct = (2 * ma < J) || (2 * ma == J && 2 * mb <= J);
        int sma = direct ? ma : J - ma, smb = direct ? mb : J - mb;
        const int slot = hoff(J) + sma * (J + 1) + smb;
        T re, im;
        if constexpr (sizeof(T) == 8) {
            const auto v = uh[((size_t)tl * nh + slot) * 32 + lane];
            re = v.x;
            im = v.y;
        } else {
            const float* q = reinterpret_cast<const float*>(uh) + (((size_t)(tl >> 1) * nh + slot) * 32 + lane) * 4 + (tl & 1);
            re = q[0];
            im = q[2];
        }
        if (!direct) {
            const T sg = ((sma - smb) & 1) ? T(-1) : T(1);
            re = sg * re;
            im = -sg * im;
        }
        uf[((size_t)p * nf + e) * 2] = re;
        uf[((size_t)p * nf + e) * 2 + 1] = im;
    }
}

template <class T, int TJ, int SEG, int W>
void launch_ui_v(const NbrOut& nb, double wself, int64_t ntiles, T* u_half, cudaStream_t st) {
    const unsigned blocks = (unsigned)((ntiles + W - 1) / W);
    k_ui<T, TJ, SEG, W><<<blocks, W * 32, 0, st>>>(reinterpret_cast<const typename AB4<T>::type*>(nb.ab),
                                                   reinterpret_cast<const T*>(nb.cw), nb.cnt, nb.kmax, (T)wself,
                                                   ntiles, reinterpret_cast<typename C2<T>::type*>(u_half));
}

template <class T, int TJ>
void launch_ui_tj(const NbrOut& nb, double wself, int64_t ntiles, T* u_half, int variant, cudaStream_t st) {
    if constexpr (sizeof(T) == 8) {
        launch_ui_v<T, TJ, kSegElemsF64, kUiWarpsF64>(nb, wself, ntiles, u_half, st);
    } else {
        constexpr UiVariant v0 = kUiVariantsF32[0], v1 = kUiVariantsF32[1], v2 = kUiVariantsF32[2];
        if (variant == 1) launch_ui_v<T, TJ, v1.seg, v1.warps>(nb, wself, ntiles, u_half, st);
        else if (variant == 2) launch_ui_v<T, TJ, v2.seg, v2.warps>(nb, wself, ntiles, u_half, st);
        else launch_ui_v<T, TJ, v0.seg, v0.warps>(nb, wself, ntiles, u_half, st);
    }
}

}  // namespace

int upload_ui_tables() {
    constexpr int n = (kTJMax + 1) * (kTJMax + 1) * (kTJMax + 1);
    double d[n];
    float f[n];
    for (int J = 0; J <= kTJMax; ++J)
        for (int a = 0; a <= kTJMax; ++a)
            for (int b = 0; b <= kTJMax; ++b) {
                double v = 0.0;
                if (a <= J && b <= J) v = std::sqrt(fact_d(J - a) * fact_d(a) / (fact_d(J - b) * fact_d(b)));
                d[(J * (kTJMax + 1) + a) * (kTJMax + 1) + b] = v;
                f[(J * (kTJMax + 1) + a) * (kTJMax + 1) + b] = (float)v;
            }
    MALA_CUDA_TRY(cudaMemcpyToSymbol(c_unorm_d, d, sizeof(d)));
    MALA_CUDA_TRY(cudaMemcpyToSymbol(c_unorm_f, f, sizeof(f)));
    return MALA_OK;
}

int ui_variant_count(bool fp32) { return fp32 ? kNumUiVariantsF32 : 1; }

void ui_variant_shape(int v, int* seg, int* warps) {
    const UiVariant u = kUiVariantsF32[(v >= 0 && v < kNumUiVariantsF32) ? v : 0];
    *seg = u.seg;
    *warps = u.warps;
}

template <class T>
void launch_ui(int twojmax, const NbrOut& nb, double wself, int64_t ntiles, T* u_half, cudaStream_t st, int variant) {
    if (ntiles <= 0) return;
    if (sizeof(T) == 4 && (ntiles & 1)) {
        // odd tile count: the B half of the last pair holds no tile; keep it finite (zero)
        const size_t pair_floats = (size_t)n_half(twojmax) * 32 * 4;
        cudaMemsetAsync(u_half + (size_t)(ntiles >> 1) * pair_floats, 0, pair_floats * sizeof(float), st);
    }
    switch (twojmax) {
        case 0: launch_ui_tj<T, 0>(nb, wself, ntiles, u_half, variant, st); break;
        case 2: launch_ui_tj<T, 2>(nb, wself, ntiles, u_half, variant, st); break;
        case 4: launch_ui_tj<T, 4>(nb, wself, ntiles, u_half, variant, st); break;
        case 6: launch_ui_tj<T, 6>(nb, wself, ntiles, u_half, variant, st); break;
        case 8: launch_ui_tj<T, 8>(nb, wself, ntiles, u_half, variant, st); break;
        case 10: launch_ui_tj<T, 10>(nb, wself, ntiles, u_half, variant, st); break;
        default: break;
    }
}

template <class T>
void launch_u_expand(int twojmax, const T* u_half, const SnapGeom& g, int64_t tile0, int64_t ntiles, T* u_full,
                     cudaStream_t st) {
    if (ntiles <= 0) return;
    k_u_expand<T><<<(unsigned)ntiles, 256, 0, st>>>(twojmax, reinterpret_cast<const typename C2<T>::type*>(u_half),
                                                    g, tile0, ntiles, u_full);
}

template void launch_ui<float>(int, const NbrOut&, double, int64_t, float*, cudaStream_t, int);
template void launch_ui<double>(int, const NbrOut&, double, int64_t, double*, cudaStream_t, int);
template void launch_u_expand<float>(int, const float*, const SnapGeom&, int64_t, int64_t, float*, cudaStream_t);
template void launch_u_expand<double>(int, const double*, const SnapGeom&, int64_t, int64_t, double*, cudaStream_t);

}  // namespace mala
