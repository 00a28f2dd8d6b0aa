// snap_yi.cuh -- device side of the FP32 Y step as units (snap_yi.h defines
// the units and the plan).  Included only by the four group translation units
// (snap_yi_g*.cu); each owns its static copy of the constant tables below.
//
// One CTA takes 64 grid points, two per lane: the u half set of both points
// sits in shared memory as float4 (A.re, B.re, A.im, B.im) per element and
// lane (snap_pairs.cuh), so every packed FP32x2 instruction does the same
// scalar step for point A and point B.  The rows (c, ma) of the launch are
// taken one after the other by all 12 warps; each warp runs its share of the
// row's units (dealt on the host longest first, so that a coupling's units go
// to different warps and the warps run the same coupling's code at about the
// same time) with the row's columns in registers, writes its partial row to
// shared memory, and after a barrier the CTA adds the 12 partials in warp
// order (a fixed order: the result does not depend on timing) and writes
// conj(Y) N for the element and its mirror.
//
// A unit's convolution keeps u^a[m1a] and u^b[m2a] in registers; for column
// mb it accumulates, for every m1b, cxr = C xr and cxi = C xi into
//     zr += cxr yr,  zn += cxi yi,  zi += cxr yi,  zj += cxi yr,
// (Re = zr - zn, Im = zi + zj): four independent chains, no negated copy of a
// row.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "mala_internal.h"
#include "snap_common.cuh"
#include "snap_pairs.cuh"
#include "snap_yi.h"

namespace mala {

// (C, C) pairs: one operand of a packed FP32x2 multiply
static __constant__ float2 c_ycg[kYcgCap];
// N(J, ma, mb) = sqrt((J-ma)! ma! / ((J-mb)! mb!)), [J][ma][mb]
static __constant__ float c_yfnorm[(kTJMax + 1) * (kTJMax + 1) * (kTJMax + 1)];

namespace {

__device__ __forceinline__ float2 lds2(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr));
    return v;
}

template <int A, int B, int C, int OFF, int MB, int M1B>
__device__ __forceinline__ void y_terms(const float2 (&xr)[A + 1], const float2 (&xi)[A + 1],
                                        const float2 (&yr)[B + 1], const float2 (&yi)[B + 1], float2& zr, float2& zn,
                                        float2& zi, float2& zj) {
    if constexpr (M1B <= A) {
        constexpr int D = (A + B - C) / 2;
        constexpr int M2B = MB - M1B + D;
        if constexpr (M2B >= 0 && M2B <= B) {
            // columns above c/2 read the mirrored table entry; the sign is applied by the caller
            constexpr bool lo = 2 * MB <= C;
            constexpr int R = lo ? MB : C - MB;
            constexpr int M1 = lo ? M1B : A - M1B;
            const float2 c = c_ycg[OFF + R * (A + 1) + M1];
            const float2 cxr = __fmul2_rn(c, xr[M1B]);
            const float2 cxi = __fmul2_rn(c, xi[M1B]);
            zr = __ffma2_rn(cxr, yr[M2B], zr);
            zn = __ffma2_rn(cxi, yi[M2B], zn);
            zi = __ffma2_rn(cxr, yi[M2B], zi);
            zj = __ffma2_rn(cxi, yr[M2B], zj);
        }
        y_terms<A, B, C, OFF, MB, M1B + 1>(xr, xi, yr, yi, zr, zn, zi, zj);
    }
}

template <int A, int B, int C, int NCOL, int OFF, int MB>
__device__ __forceinline__ void y_cols(const float2 (&xr)[A + 1], const float2 (&xi)[A + 1],
                                       const float2 (&yr)[B + 1], const float2 (&yi)[B + 1], float2 sp, float2 sn,
                                       float2 (&Yr)[NCOL], float2 (&Yi)[NCOL]) {
    if constexpr (MB < NCOL) {
        float2 zr = make_float2(0.f, 0.f), zn = zr, zi = zr, zj = zr;
        y_terms<A, B, C, OFF, MB, 0>(xr, xi, yr, yi, zr, zn, zi, zj);
        constexpr bool flip = 2 * MB > C && (((A + B - C) / 2) & 1);
        const float2 s = flip ? sn : sp, t = flip ? sp : sn;
        Yr[MB] = __ffma2_rn(s, zr, Yr[MB]);
        Yr[MB] = __ffma2_rn(t, zn, Yr[MB]);
        Yi[MB] = __ffma2_rn(s, zi, Yi[MB]);
        Yi[MB] = __ffma2_rn(s, zj, Yi[MB]);
        y_cols<A, B, C, NCOL, OFF, MB + 1>(xr, xi, yr, yi, sp, sn, Yr, Yi);
    }
}

// unit (coupling (C; A, B), row ma, m1a) scaled by be, added to columns 0..NCOL-1 of the row
template <unsigned MASK, int C, int I, int NCOL>
__device__ __forceinline__ void y_unit(uint32_t sbase, int ma, int m1a, float2 be, float2 (&Yr)[NCOL],
                                       float2 (&Yi)[NCOL]) {
    constexpr int A = coupling_field(C, I, 0), B = coupling_field(C, I, 1);
    constexpr int OFF = ycg_offset(MASK, C, I);
    constexpr int D = (A + B - C) / 2;
    const int m2a = ma - m1a + D;
    float2 xr[A + 1], xi[A + 1], yr[B + 1], yi[B + 1];
    const float sx = load_row_any<A>(sbase, m1a, xr, xi);
    const float sy = load_row_any<B>(sbase, m2a, yr, yi);
    const float c1 = c_ycg[OFF + ma * (A + 1) + m1a].x * sx * sy;
    const float2 sp = make_float2(be.x * c1, be.y * c1);
    const float2 sn = make_float2(-sp.x, -sp.y);
    y_cols<A, B, C, NCOL, OFF, 0>(xr, xi, yr, yi, sp, sn, Yr, Yi);
}

template <unsigned MASK, int C, int NCOL, int LO, int HI>
__device__ __forceinline__ void y_dispatch(int i, uint32_t sbase, int ma, int m1a, float2 be, float2 (&Yr)[NCOL],
                                           float2 (&Yi)[NCOL]) {
    if constexpr (HI - LO == 1) {
        y_unit<MASK, C, LO, NCOL>(sbase, ma, m1a, be, Yr, Yi);
    } else {
        constexpr int MID = (LO + HI) / 2;
        if (i < MID) y_dispatch<MASK, C, NCOL, LO, MID>(i, sbase, ma, m1a, be, Yr, Yi);
        else y_dispatch<MASK, C, NCOL, MID, HI>(i, sbase, ma, m1a, be, Yr, Yi);
    }
}

// this warp's units of row (C, ma) (each i | m1a << 6); the partial row goes to
// part (float4 per column and lane)
template <unsigned MASK, int C, bool MID>
__device__ __forceinline__ void y_row(int ma, const unsigned short* __restrict__ units, int n, uint32_t sbase,
                                      uint32_t bbase, const YiPlan& plan, float4* part) {
    constexpr int NCOL = MID ? C / 2 + 1 : C + 1;
    float2 Yr[NCOL], Yi[NCOL];
#pragma unroll
    for (int mb = 0; mb < NCOL; ++mb) Yr[mb] = Yi[mb] = make_float2(0.f, 0.f);
    for (int q = 0; q < n; ++q) {
        const int e = __ldg(units + q);
        const int i = e & 63, m1a = e >> 6;
        // be = f beta_t: the coupling's triple t and the sum f of the factors of the places c takes in it
        const int kg = coupling_base(C) + i;
        const float f = __ldg(plan.be_f + kg);
        const float2 bv = lds2(bbase + (uint32_t)__ldg(plan.be_t + kg) * 256u);
        const float2 be = make_float2(f * bv.x, f * bv.y);
        y_dispatch<MASK, C, NCOL, 0, n_couplings(C)>(i, sbase, ma, m1a, be, Yr, Yi);
    }
#pragma unroll
    for (int mb = 0; mb < NCOL; ++mb) part[mb * 32] = make_float4(Yr[mb].x, Yr[mb].y, Yi[mb].x, Yi[mb].y);
}

template <unsigned MASK, int C = 0>
__device__ __forceinline__ void y_row_dispatch(int c, int ma, const unsigned short* units, int n, uint32_t sbase,
                                               uint32_t bbase, const YiPlan& plan, float4* part) {
    if constexpr (C <= kTJMax) {
        if constexpr ((MASK >> C) & 1u) {
            if (c == C) {
                if constexpr ((C & 1) == 0) {
                    if (2 * ma == C) {
                        y_row<MASK, C, true>(ma, units, n, sbase, bbase, plan, part);
                        return;
                    }
                }
                y_row<MASK, C, false>(ma, units, n, sbase, bbase, plan, part);
                return;
            }
        }
        y_row_dispatch<MASK, C + 1>(c, ma, units, n, sbase, bbase, plan, part);
    }
}

template <unsigned MASK>
__global__ void __launch_bounds__(kYuWarps * 32, 1)
    k_yi_units(int tj, const float2* __restrict__ u_full, const float* __restrict__ beta, int nB, int64_t P,
               YiPlan plan, float2* __restrict__ y_out) {
    extern __shared__ __align__(16) unsigned char smem_y[];
    const int nh = n_half(tj), nf = n_full(tj);
    float4* su = reinterpret_cast<float4*>(smem_y);                                          // [nh][32]
    float2* sb = reinterpret_cast<float2*>(smem_y + (size_t)nh * 512);                        // [nB][32]
    float4* part = reinterpret_cast<float4*>(smem_y + (size_t)nh * 512 + (size_t)nB * 256);  // [warps][cols][32]
    const int64_t p0 = (int64_t)blockIdx.x * kYuPts;
    // stage the u half set and beta of points p0 + l (A) and p0 + 32 + l (B); lane fastest
    for (int idx = threadIdx.x; idx < 32 * nh; idx += blockDim.x) {
        const int l = idx & 31, e = idx >> 5;
        int J = 0;
        while (J < tj && e >= hoff(J + 1)) ++J;
        const int fe = e - hoff(J) + full_off(J);  // half rows are the leading rows of the full block
        const int64_t pa = p0 + l, pb = p0 + 32 + l;
        float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
        if (pa < P) a = __ldg(u_full + (size_t)pa * nf + fe);
        if (pb < P) b = __ldg(u_full + (size_t)pb * nf + fe);
        su[idx] = make_float4(a.x, b.x, a.y, b.y);
    }
    for (int idx = threadIdx.x; idx < 32 * nB; idx += blockDim.x) {
        const int l = idx & 31, t = idx >> 5;
        const int64_t pa = p0 + l, pb = p0 + 32 + l;
        float2 v = make_float2(0.f, 0.f);
        if (pa < P) v.x = __ldg(beta + (size_t)pa * nB + t);
        if (pb < P) v.y = __ldg(beta + (size_t)pb * nB + t);
        sb[idx] = v;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(su) + (uint32_t)lane * 16u;
    const uint32_t bbase = (uint32_t)__cvta_generic_to_shared(sb) + (uint32_t)lane * 8u;
    float4* mine = part + (size_t)warp * kYuMaxCols * 32 + lane;
    for (int r = 0; r < plan.nrows; ++r) {
        const int row = plan.row0 + r;
        const int2 cm = __ldg(plan.rows + row);
        const int c = cm.x, ma = cm.y;
        const int* off = plan.off + (size_t)row * (kYuWarps + 1);
        const int u0 = __ldg(off + warp), u1 = __ldg(off + warp + 1);
        y_row_dispatch<MASK>(c, ma, plan.units + u0, u1 - u0, sbase, bbase, plan, mine);
        __syncthreads();
        const int ncol = 2 * ma == c ? c / 2 + 1 : c + 1;
        for (int idx = threadIdx.x; idx < 32 * ncol; idx += blockDim.x) {
            const int mb = idx >> 5, l = idx & 31;
            float4 s = part[idx];
#pragma unroll
            for (int w = 1; w < kYuWarps; ++w) {
                const float4 v = part[(size_t)w * kYuMaxCols * 32 + idx];
                s.x += v.x;
                s.y += v.y;
                s.z += v.z;
                s.w += v.w;
            }
            const float nrm = c_yfnorm[(c * (kTJMax + 1) + ma) * (kTJMax + 1) + mb];  // also N at the mirror
            const int e = full_off(c) + ma * (c + 1) + mb;
            const bool self = 2 * ma == c && 2 * mb == c;
            const int em = full_off(c) + (c - ma) * (c + 1) + (c - mb);
            const float sg = ((ma - mb) & 1) ? -nrm : nrm;  // mirror: (-1)^(ma-mb) conj(Y)
            const int64_t pa = p0 + l, pb = p0 + 32 + l;
            if (pa < P) {
                float2* o = y_out + (size_t)pa * nf;
                o[e] = make_float2(s.x * nrm, -s.z * nrm);
                if (!self) o[em] = make_float2(s.x * sg, s.z * sg);
            }
            if (pb < P) {
                float2* o = y_out + (size_t)pb * nf;
                o[e] = make_float2(s.y * nrm, -s.w * nrm);
                if (!self) o[em] = make_float2(s.y * sg, s.w * sg);
            }
        }
        __syncthreads();
    }
}

template <unsigned MASK>
int yi_upload(const float* cg, int n, const float* fnorm) {
    static_assert(ycg_size(MASK) <= kYcgCap, "Clebsch-Gordan table of a group exceeds its constant array");
    if (n != ycg_size(MASK)) return fail(MALA_ERR_UNSUPPORTED, "Y table size mismatch (%d vs %d)", n, ycg_size(MASK));
    float2 pairs[kYcgCap];
    for (int i = 0; i < n; ++i) pairs[i] = make_float2(cg[i], cg[i]);
    MALA_CUDA_TRY(cudaMemcpyToSymbol(c_ycg, pairs, sizeof(float2) * (size_t)n));
    MALA_CUDA_TRY(cudaMemcpyToSymbol(c_yfnorm, fnorm, sizeof(c_yfnorm)));
    return MALA_OK;
}

template <unsigned MASK>
int yi_launch(const YiLaunch& a) {
    if (a.plan.nrows <= 0 || a.P <= 0) return MALA_OK;
    const size_t smem = yi_units_smem(a.tj, a.nB);
    MALA_CUDA_TRY(cudaFuncSetAttribute(k_yi_units<MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t grid = (a.P + kYuPts - 1) / kYuPts;
    k_yi_units<MASK><<<(unsigned)grid, kYuWarps * 32, smem, a.st>>>(
        a.tj, reinterpret_cast<const float2*>(a.u_full), a.beta, a.nB, a.P, a.plan, reinterpret_cast<float2*>(a.y));
    MALA_CUDA_TRY(cudaGetLastError());
    return MALA_OK;
}

}  // namespace

}  // namespace mala
