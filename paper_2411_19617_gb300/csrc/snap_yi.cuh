// snap_yi.cuh -- device side of the FP32 Y step as units (snap_yi.h defines
// the units and the plan).  Included only by the four group translation units
// (snap_yi_g*.cu); each owns its static copy of the constant tables below.
//
// One CTA takes 64 grid points, two per lane: the rows ma <= J/2 of every u^J
// of both points sit in shared memory as float4 (A.re, B.re, A.im, B.im) per
// element and lane, so every packed FP32x2 instruction does the same scalar
// step for point A and point B.  The rows (c, ma) of the launch are taken one
// after the other by all 12 warps; each warp runs its share of the row's units
// (dealt on the host longest first), adds them into its partial row in shared
// memory, and after a barrier the CTA adds the 12 partials in warp order (a
// fixed order: the result does not depend on timing) and writes conj(Y) N for
// the element and its mirror.
//
// A unit (coupling c <- a b, row ma, m1a) convolves the rows u^a[m1a] and
// u^b[m2a], m2a = ma - m1a + (a + b - c)/2.  Of the two rows one lies at or
// below its middle (both above would put ma above c/2); that one is read from
// shared memory element by element, the other is held in registers (through
// the mirror symmetry when it lies above its middle).  The code depends only on
// the length R + 1 of the register row: the columns of the row of Y^c run in
// pairs in a loop, and for each pair the R + 2 shared-memory elements they need
// are read once; the Clebsch-Gordan values come from the coupling's full block
// in constant memory (zero where the partner index leaves its row, so the
// shared-memory index is clamped and the term vanishes).  The few kilobytes of
// code a row length needs stay in the instruction cache; a version with every
// coupling unrolled spent a third of its cycles waiting for instructions.
//
// A term's complex product with C: cxr = C xr, cxi = C xi,
//     zr += cxr yr,  zn += cxi yi,  zi += cxr yi,  zj += cxi yr,
// Re = zr - zn, Im = zi + zj.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "mala_internal.h"
#include "snap_common.cuh"
#include "snap_pairs.cuh"
#include "snap_yi.h"

namespace mala {

// Clebsch-Gordan blocks as (C, C) pairs: one operand of a packed FP32x2 multiply
static __constant__ float2 c_ycg[kYcgCap];
// per global coupling id: a, b, offset of the (a, b) block, offset of the (b, a) block (-1: not in this group)
static __constant__ int4 c_yinfo[kNCouplings];
// N(J, ma, mb) = sqrt((J-ma)! ma! / ((J-mb)! mb!)), [J][ma][mb]
static __constant__ float c_yfnorm[(kTJMax + 1) * (kTJMax + 1) * (kTJMax + 1)];
// frow_off(J) for J = 0..kTJMax + 1; coupling_base(c) for c = 0..kTJMax
static __constant__ int c_yfrow[kTJMax + 2];
static __constant__ int c_ycbase[kTJMax + 1];

namespace {

// full_off(J) = sum_{k<J} (k+1)^2 in closed form
__device__ __forceinline__ int full_off_cf(int J) { return J * (J + 1) * (2 * J + 1) / 6; }

__device__ __forceinline__ void sts4(uint32_t addr, float4 v) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// element K of a row of u^R read directly (b: the row's address) or through the mirror
// (b: the address of row R - row; (row, K) = (-1)^(K - row) conj((R - row, R - K)), the
// (-1)^row part applied by the caller)
template <int R, bool MIRROR, int K>
__device__ __forceinline__ void row_elems(uint32_t b, float2 (&re)[R + 1], float2 (&im)[R + 1]) {
    if constexpr (K <= R) {
        if constexpr (!MIRROR) {
            const float4 v = lds4(b + (uint32_t)K * 512u);
            re[K] = make_float2(v.x, v.y);
            im[K] = make_float2(v.z, v.w);
        } else {
            const float4 v = lds4(b + (uint32_t)(R - K) * 512u);
            if constexpr (K & 1) {
                re[K] = make_float2(-v.x, -v.y);
                im[K] = make_float2(v.z, v.w);
            } else {
                re[K] = make_float2(v.x, v.y);
                im[K] = make_float2(-v.z, -v.w);
            }
        }
        row_elems<R, MIRROR, K + 1>(b, re, im);
    }
}

// Row `row` of u^R (any row) as pairs re[k], im[k]; returns the sign (-1)^row of a
// row read through the mirror (its column signs are applied here)
template <int R>
__device__ __forceinline__ float load_row_full(uint32_t sbase, int row, float2 (&re)[R + 1], float2 (&im)[R + 1]) {
    constexpr uint32_t H = (uint32_t)frow_off(R);
    if (2 * row <= R) {
        row_elems<R, false, 0>(sbase + (H + (uint32_t)row * (R + 1)) * 512u, re, im);
        return 1.f;
    }
    row_elems<R, true, 0>(sbase + (H + (uint32_t)(R - row) * (R + 1)) * 512u, re, im);
    return (row & 1) ? -1.f : 1.f;
}

// the shared-memory elements t0 - k, k = 0..R+1, clamped into the row 0..sJ
template <int R, int K>
__device__ __forceinline__ void load_window(uint32_t ybase, int t0, int sJ, float4 (&yv)[R + 2]) {
    if constexpr (K <= R + 1) {
        yv[K] = lds4(ybase + (uint32_t)min(max(t0 - K, 0), sJ) * 512u);
        load_window<R, K + 1>(ybase, t0, sJ, yv);
    }
}

// the terms of register element r for the column pair: column mb with yv[r + 1], column mb + 1 with yv[r]
struct ColAcc {
    float2 ar, an, ai, aj, br, bn, bi, bj;
};
template <int R, int r>
__device__ __forceinline__ void pair_terms(int cgi, const float2 (&xr)[R + 1], const float2 (&xi)[R + 1],
                                           const float4 (&yv)[R + 2], ColAcc& z) {
    if constexpr (r <= R) {
        const float2 ca = c_ycg[cgi + r], cb = c_ycg[cgi + R + 1 + r];
        const float2 y0r = make_float2(yv[r + 1].x, yv[r + 1].y), y0i = make_float2(yv[r + 1].z, yv[r + 1].w);
        const float2 y1r = make_float2(yv[r].x, yv[r].y), y1i = make_float2(yv[r].z, yv[r].w);
        const float2 cxr = __fmul2_rn(ca, xr[r]), cxi = __fmul2_rn(ca, xi[r]);
        z.ar = __ffma2_rn(cxr, y0r, z.ar);
        z.an = __ffma2_rn(cxi, y0i, z.an);
        z.ai = __ffma2_rn(cxr, y0i, z.ai);
        z.aj = __ffma2_rn(cxi, y0r, z.aj);
        const float2 dxr = __fmul2_rn(cb, xr[r]), dxi = __fmul2_rn(cb, xi[r]);
        z.br = __ffma2_rn(dxr, y1r, z.br);
        z.bn = __ffma2_rn(dxi, y1i, z.bn);
        z.bi = __ffma2_rn(dxr, y1i, z.bi);
        z.bj = __ffma2_rn(dxi, y1r, z.bj);
        pair_terms<R, r + 1>(cgi, xr, xi, yv, z);
    }
}

// One unit whose register row has R + 1 elements: rrow is that row's index; the
// shared-memory row is row srow of u^sJ (at or below its middle); D = (a + b - c)/2;
// tab is the offset of the block whose columns run over the register row; the
// row's ncol columns are added into this warp's partial row (column mb at
// pbase + mb * 512) scaled by be.
template <int R>
__device__ __forceinline__ void y_unit_c(uint32_t sbase, int rrow, int sJ, int srow, int D, int tab, int ma, int ncol,
                                         float2 be, uint32_t pbase) {
    float2 xr[R + 1], xi[R + 1];
    const float sx = load_row_full<R>(sbase, rrow, xr, xi);
    const uint32_t ybase = sbase + ((uint32_t)c_yfrow[sJ] + (uint32_t)srow * (sJ + 1)) * 512u;
    const float c1 = c_ycg[tab + ma * (R + 1) + rrow].x * sx;
    const float2 sp = make_float2(be.x * c1, be.y * c1);
    const float2 sn = make_float2(-sp.x, -sp.y);
    for (int mb = 0; mb < ncol; mb += 2) {
        // the shared-memory elements mb + D + 1 - k, k = 0..R+1, clamped into the row (their
        // Clebsch-Gordan values are zero where the index leaves it)
        float4 yv[R + 2];
        load_window<R, 0>(ybase, mb + D + 1, sJ, yv);
        const int cgi = tab + mb * (R + 1);  // column mb at cgi, column mb + 1 at cgi + R + 1
        ColAcc z;
        z.ar = z.an = z.ai = z.aj = z.br = z.bn = z.bi = z.bj = make_float2(0.f, 0.f);
        pair_terms<R, 0>(cgi, xr, xi, yv, z);
        const uint32_t pa = pbase + (uint32_t)mb * 512u;
        {
            const float4 p = lds4(pa);
            float2 pr = make_float2(p.x, p.y), pi = make_float2(p.z, p.w);
            pr = __ffma2_rn(sp, z.ar, pr);
            pr = __ffma2_rn(sn, z.an, pr);
            pi = __ffma2_rn(sp, z.ai, pi);
            pi = __ffma2_rn(sp, z.aj, pi);
            sts4(pa, make_float4(pr.x, pr.y, pi.x, pi.y));
        }
        if (mb + 1 < ncol) {
            const float4 p = lds4(pa + 512u);
            float2 pr = make_float2(p.x, p.y), pi = make_float2(p.z, p.w);
            pr = __ffma2_rn(sp, z.br, pr);
            pr = __ffma2_rn(sn, z.bn, pr);
            pi = __ffma2_rn(sp, z.bi, pi);
            pi = __ffma2_rn(sp, z.bj, pi);
            sts4(pa + 512u, make_float4(pr.x, pr.y, pi.x, pi.y));
        }
    }
}

// this warp's units of row (c, ma), added into its partial row (zeroed first)
// ba, bb: beta of the lane's points A and B (null past the grid's end)
__device__ __forceinline__ void y_row(int c, int ma, const unsigned short* __restrict__ units, int n, uint32_t sbase,
                                      const float* ba, const float* bb, const YiPlan& plan, uint32_t pbase) {
    const int ncol = 2 * ma == c ? c / 2 + 1 : c + 1;
    for (int mb = 0; mb < ncol; ++mb) sts4(pbase + (uint32_t)mb * 512u, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int q = 0; q < n; ++q) {
        const int e = __ldg(units + q);
        const int i = e & 63, m1a = (e >> 6) & 15, swap = e >> 10;
        const int kg = c_ycbase[c] + i;
        const int4 info = c_yinfo[kg];
        const int a = info.x, b = info.y;
        const int D = (a + b - c) / 2;
        const int m2a = ma - m1a + D;
        // be = f beta_t: the coupling's triple t and the sum f of the factors of the places c takes in it
        const float f = __ldg(plan.be_f + kg);
        const int t = __ldg(plan.be_t + kg);
        const float2 be = make_float2(f * (ba ? __ldg(ba + t) : 0.f), f * (bb ? __ldg(bb + t) : 0.f));
        const int R = swap ? b : a, rrow = swap ? m2a : m1a, sJ = swap ? a : b, srow = swap ? m1a : m2a;
        const int tab = swap ? info.w : info.z;
        switch (R) {
            case 0: y_unit_c<0>(sbase, rrow, sJ, srow, D, tab, ma, ncol, be, pbase); break;
            case 1: y_unit_c<1>(sbase, rrow, sJ, srow, D, tab, ma, ncol, be, pbase); break;
            case 2: y_unit_c<2>(sbase, rrow, sJ, srow, D, tab, ma, ncol, be, pbase); break;
            case 3: y_unit_c<3>(sbase, rrow, sJ, srow, D, tab, ma, ncol, be, pbase); break;
            case 4: y_unit_c<4>(sbase, rrow, sJ, srow, D, tab, ma, ncol, be, pbase); break;
            case 5: y_unit_c<5>(sbase, rrow, sJ, srow, D, tab, ma, ncol, be, pbase); break;
            case 6: y_unit_c<6>(sbase, rrow, sJ, srow, D, tab, ma, ncol, be, pbase); break;
            case 7: y_unit_c<7>(sbase, rrow, sJ, srow, D, tab, ma, ncol, be, pbase); break;
            case 8: y_unit_c<8>(sbase, rrow, sJ, srow, D, tab, ma, ncol, be, pbase); break;
            case 9: y_unit_c<9>(sbase, rrow, sJ, srow, D, tab, ma, ncol, be, pbase); break;
            default: y_unit_c<10>(sbase, rrow, sJ, srow, D, tab, ma, ncol, be, pbase); break;
        }
    }
}

template <unsigned MASK>
__global__ void __launch_bounds__(kYuWarps * 32, 1)
    k_yi_units(int tj, const float2* __restrict__ u_full, const float* __restrict__ beta, int nB, int64_t P,
               YiPlan plan, float2* __restrict__ y_out) {
    extern __shared__ __align__(16) unsigned char smem_y[];
    const int nr = n_frows(tj), nf = n_full(tj);
    float4* su = reinterpret_cast<float4*>(smem_y);                                           // [nr][32]
    float4* part = reinterpret_cast<float4*>(smem_y + (size_t)nr * 512);   // [warps][cols][32]
    const int64_t p0 = (int64_t)blockIdx.x * kYuPts;
    // stage the rows ma <= J/2 of points p0 + l (A) and p0 + 32 + l (B); lane fastest
    for (int idx = threadIdx.x; idx < 32 * nr; idx += blockDim.x) {
        const int l = idx & 31, e = idx >> 5;
        int J = 0;
        while (J < tj && e >= c_yfrow[J + 1]) ++J;
        const int fe = e - c_yfrow[J] + full_off_cf(J);  // these rows are the leading rows of the full block
        const int64_t pa = p0 + l, pb = p0 + 32 + l;
        float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
        if (pa < P) a = __ldg(u_full + (size_t)pa * nf + fe);
        if (pb < P) b = __ldg(u_full + (size_t)pb * nf + fe);
        su[idx] = make_float4(a.x, b.x, a.y, b.y);
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(su) + (uint32_t)lane * 16u;
    const float* ba = p0 + lane < P ? beta + (size_t)(p0 + lane) * nB : nullptr;
    const float* bb = p0 + 32 + lane < P ? beta + (size_t)(p0 + 32 + lane) * nB : nullptr;
    const uint32_t pbase = (uint32_t)__cvta_generic_to_shared(part) + (uint32_t)(warp * kYuMaxCols * 32 + lane) * 16u;
    for (int r = 0; r < plan.nrows; ++r) {
        const int row = plan.row0 + r;
        const int2 cm = __ldg(plan.rows + row);
        const int c = cm.x, ma = cm.y;
        const int* off = plan.off + (size_t)row * (kYuWarps + 1);
        const int u0 = __ldg(off + warp), u1 = __ldg(off + warp + 1);
        y_row(c, ma, plan.units + u0, u1 - u0, sbase, ba, bb, plan, pbase);
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
            const int e = full_off_cf(c) + ma * (c + 1) + mb;
            const bool self = 2 * ma == c && 2 * mb == c;
            const int em = full_off_cf(c) + (c - ma) * (c + 1) + (c - mb);
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
int yi_upload(const float* cg, int n, const int* info, const float* fnorm) {
    if (n > kYcgCap) return fail(MALA_ERR_UNSUPPORTED, "Y table of a coupling group too large (%d pairs)", n);
    static float2 pairs[kYcgCap];  // zero beyond n: a column pair may read one row past a block
    for (int i = 0; i < kYcgCap; ++i) pairs[i] = i < n ? make_float2(cg[i], cg[i]) : make_float2(0.f, 0.f);
    MALA_CUDA_TRY(cudaMemcpyToSymbol(c_ycg, pairs, sizeof(pairs)));
    MALA_CUDA_TRY(cudaMemcpyToSymbol(c_yinfo, info, sizeof(c_yinfo)));
    int fr[kTJMax + 2];
    for (int J = 0; J <= kTJMax + 1; ++J) fr[J] = frow_off(J);
    MALA_CUDA_TRY(cudaMemcpyToSymbol(c_yfrow, fr, sizeof(fr)));
    int cb[kTJMax + 1];
    for (int c = 0; c <= kTJMax; ++c) cb[c] = coupling_base(c);
    MALA_CUDA_TRY(cudaMemcpyToSymbol(c_ycbase, cb, sizeof(cb)));
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
