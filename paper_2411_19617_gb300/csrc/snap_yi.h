// snap_yi.h -- index sets and the launch plan of the FP32 Y step of the force
// chain (the adjoint of the bispectrum descriptors, snap_force.cu states the
// formula), shared by the host planner (snap_yi.cu) and the four translation
// units that hold the kernels (snap_yi_g*.cu).
//
// Y^c = sum over couplings (c; a >= b) of be_k Z^c_{ab}.  The three momenta
// of a coupling, sorted, are one triple t of the index set, and be_k =
// f_k beta_t, f_k the sum over the places c takes in t of 1 (c the largest
// momentum j) or (j+1)/(c+1) (c one of the two others).  Z^c_{ab}[ma][mb] = sum_{m1a, m1b} C(ma; m1a) C(mb; m1b)
// u^a[m1a][m1b] u^b[m2a][m2b], m2 = m - m1 (twice-units).  A "unit" is one
// (coupling, ma, m1a): it adds C(ma; m1a) be_k times a convolution of the row
// u^a[m1a] with the row u^b[m2a] to row ma of Y^c.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "snap_common.cuh"

namespace mala {

constexpr int kYuWarps = 16;            // warps per CTA of the unit kernels
constexpr int kYuPts = 64;              // grid points per CTA: two per lane
constexpr int kYuMaxCols = kTJMax + 1;  // columns of a Y row

// coupling (c; a >= b): a triangle with even perimeter, all momenta <= kTJMax
__host__ __device__ constexpr bool coupling_ok(int c, int a, int b) {
    return b >= 0 && b <= a && a <= kTJMax && c >= 0 && c <= kTJMax && c >= a - b && c <= a + b &&
           ((a + b + c) & 1) == 0;
}
__host__ __device__ constexpr int n_couplings(int c) {
    int n = 0;
    for (int a = 0; a <= kTJMax; ++a)
        for (int b = 0; b <= a; ++b)
            if (coupling_ok(c, a, b)) ++n;
    return n;
}
// a (f = 0) or b (f = 1) of the i-th coupling of c, (a, b) in lexicographic order
__host__ __device__ constexpr int coupling_field(int c, int i, int f) {
    int n = 0;
    for (int a = 0; a <= kTJMax; ++a)
        for (int b = 0; b <= a; ++b) {
            if (!coupling_ok(c, a, b)) continue;
            if (n == i) return f == 0 ? a : b;
            ++n;
        }
    return -1;
}
// global id of the first coupling of c (couplings ordered by c, then (a, b))
__host__ __device__ constexpr int coupling_base(int c) {
    int n = 0;
    for (int k = 0; k < c; ++k) n += n_couplings(k);
    return n;
}
constexpr int kNCouplings = coupling_base(kTJMax + 1);

// Shared-memory layout of u the unit kernels read: for every J the rows
// ma <= J/2 in full (J + 1 elements each, the middle row too), row (J, ma) at
// frow_off(J) + ma (J + 1); rows above the middle follow from
// u[J-ma][J-mb] = (-1)^(ma-mb) conj(u[ma][mb]).
__host__ __device__ constexpr int frow_off(int J) {
    int o = 0;
    for (int k = 0; k < J; ++k) o += (k / 2 + 1) * (k + 1);
    return o;
}
__host__ __device__ constexpr int n_frows(int tj) { return frow_off(tj + 1); }

// The couplings are split by c over four translation units (one launch each);
// each holds, in constant memory, the full Clebsch-Gordan blocks of its
// couplings in both orientations: [m][m1] (rows m = 0..c, columns over a) and,
// for a != b, the block of (c; b, a), [m][m2] with columns over b.
constexpr int kYiGroups = 4;
__host__ __device__ constexpr unsigned yi_mask(int g) {
    return g == 0 ? ((1u << 10) | (1u << 3) | (1u << 1))
         : g == 1 ? ((1u << 8) | (1u << 5) | 1u)
         : g == 2 ? ((1u << 6) | (1u << 7))
                  : ((1u << 4) | (1u << 9) | (1u << 2));
}
constexpr int kYcgCap = 4736;  // pairs; every group's blocks fit, with room for a read one row past the last

// Work of one launch (one group), in device memory.  Row r of the launch is
// (c, ma) = rows[row0 + r]; warp w takes units off[(row0 + r) * (kYuWarps + 1) + w]
// up to the next offset; a unit is (coupling index within c) | m1a << 6 |
// s << 10, s = 1 when the u^b row is the one held in registers (the u^a row is
// then read from shared memory), s = 0 the other way round.
struct YiPlan {
    const int2* rows;
    const int* off;
    const unsigned short* units;
    const int* be_t;    // [kNCouplings] triple (numbering of this twojmax), 0 where unused
    const float* be_f;  // [kNCouplings] f_k
    int row0, nrows;
};

// dynamic shared memory of a unit kernel: u rows and the warps' partial rows
inline size_t yi_units_smem(int tj, int) {
    return (size_t)n_frows(tj) * 512 + (size_t)kYuWarps * kYuMaxCols * 512;
}

struct YiLaunch {
    int tj;
    const float* u_full;  // [P][n_full][2]
    const float* beta;    // [P][nB]
    int nB;
    int64_t P;
    YiPlan plan;
    float* y;  // [P][n_full][2]: conj(Y) N
    cudaStream_t st;
};

// per group g: the table upload (blocks, per-coupling info {a, b, offset of the
// (a, b) block, offset of the (b, a) block}, N) and the launch (snap_yi_g<g>.cu)
int yi_upload_g0(const float* cg, int n, const int* info, const float* fnorm);
int yi_upload_g1(const float* cg, int n, const int* info, const float* fnorm);
int yi_upload_g2(const float* cg, int n, const int* info, const float* fnorm);
int yi_upload_g3(const float* cg, int n, const int* info, const float* fnorm);
int yi_launch_g0(const YiLaunch& a);
int yi_launch_g1(const YiLaunch& a);
int yi_launch_g2(const YiLaunch& a);
int yi_launch_g3(const YiLaunch& a);

}  // namespace mala
