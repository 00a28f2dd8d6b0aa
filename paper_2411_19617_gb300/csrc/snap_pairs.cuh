// snap_pairs.cuh -- the shared-memory layout of the u half set that the FP32
// descriptor kernels work on, two grid points per lane: element e of the half
// set (snap_common.cuh) is a float4 (A.re, B.re, A.im, B.im) per lane, 512
// bytes per element, so a packed FP32x2 instruction does the same scalar step
// for point A and point B.  Rows above the middle of u^J are read through the
// mirror u[J-ma][J-mb] = (-1)^(ma-mb) conj(u[ma][mb]).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "snap_common.cuh"

namespace mala {
namespace {

__device__ __forceinline__ float4 lds4(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}

template <int IMM>
__device__ __forceinline__ float4 lds4i(uint32_t addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4+%5];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr), "n"(IMM));
    return v;
}

// element e of the half set: float4 per lane, 512 bytes per element
constexpr uint32_t kElemBytes = 512u;

enum RowCase { kDirect = 0, kMiddle = 1, kMirror = 2 };

// Row `row` of u^JJ as pairs re[k] = (A.re, B.re), im[k] = (A.im, B.im), up to
// the sign (-1)^row of mirrored rows (returned separately by the caller).
template <int JJ, int CASE, int K>
__device__ __forceinline__ void load_row_pairs(uint32_t sbase, int row, float2 (&re)[JJ + 1], float2 (&im)[JJ + 1]) {
    if constexpr (K <= JJ) {
        constexpr uint32_t H = (uint32_t)hoff(JJ);
        float4 v;
        bool mirror;
        if constexpr (CASE == kDirect) {
            v = lds4i<K * 512>(sbase + (H + (uint32_t)row * (JJ + 1)) * kElemBytes);
            mirror = false;
        } else if constexpr (CASE == kMiddle) {
            // row JJ/2: columns <= JJ/2 stored, the others mirrored within the row
            constexpr int col = (2 * K <= JJ) ? K : JJ - K;
            v = lds4i<(H + (JJ / 2) * (JJ + 1) + col) * 512>(sbase);
            mirror = 2 * K > JJ;
        } else {
            v = lds4i<(JJ - K) * 512>(sbase + (H + (uint32_t)(JJ - row) * (JJ + 1)) * kElemBytes);
            mirror = true;
        }
        if (mirror) {
            // (-1)^(K - row) conj(v); the (-1)^row part is applied by the caller
            constexpr bool neg = CASE == kMiddle ? (((K - JJ / 2) & 1) != 0) : ((K & 1) != 0);
            if (neg) {
                re[K] = make_float2(-v.x, -v.y);
                im[K] = make_float2(v.z, v.w);
            } else {
                re[K] = make_float2(v.x, v.y);
                im[K] = make_float2(-v.z, -v.w);
            }
        } else {
            re[K] = make_float2(v.x, v.y);
            im[K] = make_float2(v.z, v.w);
        }
        load_row_pairs<JJ, CASE, K + 1>(sbase, row, re, im);
    }
}

// returns (-1)^row for mirrored rows, 1 otherwise (middle rows carry their signs inside)
template <int JJ>
__device__ __forceinline__ float load_row_any(uint32_t sbase, int row, float2 (&re)[JJ + 1], float2 (&im)[JJ + 1]) {
    if (2 * row < JJ) {
        load_row_pairs<JJ, kDirect, 0>(sbase, row, re, im);
        return 1.f;
    }
    if (2 * row == JJ) {
        load_row_pairs<JJ, kMiddle, 0>(sbase, row, re, im);
        return 1.f;
    }
    load_row_pairs<JJ, kMirror, 0>(sbase, row, re, im);
    return (row & 1) ? -1.f : 1.f;
}

}  // namespace
}  // namespace mala
