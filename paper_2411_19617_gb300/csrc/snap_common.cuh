// snap_common.cuh -- index arithmetic shared by the descriptor kernels.
//
// Notation (paper Sec. "Bispectrum descriptors"): angular momenta in
// twice-units J = 2j; matrix indices ma, mb = 0..J stand for m = ma - J/2.
//
// Half storage.  u^J obeys u^J[J-ma][J-mb] = (-1)^(ma-mb) conj(u^J[ma][mb])
// (inherited from U^J of an SU(2) element), so only rows ma < J/2 (all
// columns) and, for even J, the middle row ma = J/2 with columns mb <= J/2
// are kept.  Element (J, ma, mb) of that set lives at
// hoff(J) + ma * (J + 1) + mb.
#pragma once
#include <cstdint>

namespace mala {

constexpr int kTileX = 4, kTileY = 4, kTileZ = 2;  // 32 grid points per tile, one per lane
constexpr int kTilePts = kTileX * kTileY * kTileZ;
constexpr int kTJMax = 10;  // largest twojmax with compiled descriptor kernels

__host__ __device__ constexpr int half_count(int J) {
    return (J & 1) ? ((J + 1) / 2) * (J + 1) : (J / 2) * (J + 1) + J / 2 + 1;
}
__host__ __device__ constexpr int hoff(int J) {
    int o = 0;
    for (int k = 0; k < J; ++k) o += half_count(k);
    return o;
}
__host__ __device__ constexpr int n_half(int tj) { return hoff(tj + 1); }
__host__ __device__ constexpr int full_off(int J) {
    int o = 0;
    for (int k = 0; k < J; ++k) o += (k + 1) * (k + 1);
    return o;
}
__host__ __device__ constexpr int n_full(int tj) { return full_off(tj + 1); }

// Triples (J1, J2, J) of the index set, lexicographic; kTJMax ordering is
// the global numbering used by the Clebsch-Gordan table.
__host__ __device__ constexpr bool triple_ok(int j1, int j2, int j, int tj) {
    return j2 <= j1 && j1 <= tj && j <= tj && j >= j1 && j >= j1 - j2 && j <= j1 + j2 &&
           ((j1 + j2 + j) & 1) == 0;
}
__host__ __device__ constexpr int n_triples(int tj) {
    int n = 0;
    for (int j1 = 0; j1 <= tj; ++j1)
        for (int j2 = 0; j2 <= j1; ++j2)
            for (int j = 0; j <= tj; ++j)
                if (triple_ok(j1, j2, j, tj)) ++n;
    return n;
}
// Offset of a triple's Clebsch-Gordan block ([ma][m1a], (J+1) x (J1+1)) in
// the global table.
__host__ __device__ constexpr int cg_offset(int J1, int J2, int J) {
    int off = 0;
    for (int j1 = 0; j1 <= kTJMax; ++j1)
        for (int j2 = 0; j2 <= j1; ++j2)
            for (int j = 0; j <= kTJMax; ++j) {
                if (!triple_ok(j1, j2, j, kTJMax)) continue;
                if (j1 == J1 && j2 == J2 && j == J) return off;
                off += (j + 1) * (j1 + 1);
            }
    return -1;
}
__host__ __device__ constexpr int cg_table_size() {
    int off = 0;
    for (int j1 = 0; j1 <= kTJMax; ++j1)
        for (int j2 = 0; j2 <= j1; ++j2)
            for (int j = 0; j <= kTJMax; ++j)
                if (triple_ok(j1, j2, j, kTJMax)) off += (j + 1) * (j1 + 1);
    return off;
}
__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }
__host__ __device__ constexpr int cmin(int a, int b) { return a < b ? a : b; }

// sqrt((J-ma)! ma! / ((J-mb)! mb!)): the factor between the polynomial
// coefficients the recursion produces and the unitary U^J.
__host__ __device__ constexpr double fact_d(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}
__host__ __device__ constexpr double csqrt_newton(double x) {
    if (x <= 0.0) return 0.0;
    double g = x > 1.0 ? x : 1.0;
    for (int i = 0; i < 200; ++i) {
        double n = 0.5 * (g + x / g);
        if (n == g) break;
        g = n;
    }
    return g;
}
__host__ __device__ constexpr double unorm(int J, int ma, int mb) {
    return csqrt_newton(fact_d(J - ma) * fact_d(ma) / (fact_d(J - mb) * fact_d(mb)));
}

}  // namespace mala
