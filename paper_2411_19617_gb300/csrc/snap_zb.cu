// snap_zb.cu -- compute_zi + compute_bi: the bispectrum components
// ("scalar triple products" of the expansion coefficients, paper Sec.
// "Bispectrum descriptors", count Eq. snap_dim):
//   Z^{J1J2J}[m][m'] = sum_{m1,m1'} C^{J m}_{J1 m1, J2 m-m1} C^{J m'}_{J1 m1', J2 m'-m1'}
//                                  u^{J1}[m1][m1'] u^{J2}[m-m1][m'-m1'],
//   B_{J1J2J}        = sum_{m,m'} Re(conj(u^J[m][m']) Z^{J1J2J}[m][m']).
// Z has the same mirror symmetry as u, so only its half set is formed and the
// mirrored half of the sum is a factor two (one for the middle element).
//
// Mapping: one CTA of 8 warps per tile of 32 grid points; lane = point, so
// every lane executes the same contraction and all Clebsch-Gordan factors are
// warp-uniform (constant-memory operands).  The tile's u half set (64 KB in
// FP32 at twojmax = 10) is staged in shared memory as [element][lane]
// (conflict-free).  Each warp takes a cost-balanced subset of the (J1,J2,J)
// triples; for every row pair (m1 row of u^J1, m-m1 row of u^J2) the two rows
// are loaded into registers and the column convolution over (m', m1') is
// fully unrolled per triple.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <vector>

#include "snap_zb.cuh"

namespace mala {

// ---- host: Clebsch-Gordan table (Racah's formula) and warp assignment ------

namespace {

double lfact(int n) {
    double r = 0.0;
    for (int i = 2; i <= n; ++i) r += std::log((double)i);
    return r;
}

// <j1 m1 j2 m2 | j m> in twice-units via Racah's formula, evaluated with
// log-factorials and an alternating sum.
double cg_racah(int j1, int m1, int j2, int m2, int j, int m) {
    if (m1 + m2 != m || std::abs(m1) > j1 || std::abs(m2) > j2 || std::abs(m) > j) return 0.0;
    if (((j1 + m1) | (j2 + m2) | (j + m)) & 1) return 0.0;
    if (j < std::abs(j1 - j2) || j > j1 + j2 || ((j1 + j2 + j) & 1)) return 0.0;
    const int A = (j1 + j2 - j) / 2, Bq = (j1 - j2 + j) / 2, Cq = (-j1 + j2 + j) / 2, D = (j1 + j2 + j) / 2 + 1;
    const double lpre = 0.5 * (std::log((double)(j + 1)) + lfact(A) + lfact(Bq) + lfact(Cq) - lfact(D) +
                               lfact((j1 + m1) / 2) + lfact((j1 - m1) / 2) + lfact((j2 + m2) / 2) +
                               lfact((j2 - m2) / 2) + lfact((j + m) / 2) + lfact((j - m) / 2));
    double s = 0.0;
    const int kmin = std::max(0, std::max((j2 - j - m1) / 2, (j1 - j + m2) / 2));
    const int kmax = std::min(A, std::min((j1 - m1) / 2, (j2 + m2) / 2));
    for (int k = kmin; k <= kmax; ++k) {
        const double l = lfact(k) + lfact(A - k) + lfact((j1 - m1) / 2 - k) + lfact((j2 + m2) / 2 - k) +
                         lfact((j - j2 + m1) / 2 + k) + lfact((j - j1 - m2) / 2 + k);
        s += ((k & 1) ? -1.0 : 1.0) * std::exp(lpre - l);
    }
    return s;
}

double triple_cost(int j1, int j2, int j) {
    const int d = (j1 + j2 - j) / 2;
    double cost = 0.0;
    for (int ma = 0; 2 * ma <= j; ++ma) {
        const int ncol = (2 * ma == j) ? j / 2 + 1 : j + 1;
        int tcol = 0;
        for (int mb = 0; mb < ncol; ++mb)
            for (int m1b = 0; m1b <= j1; ++m1b) {
                const int m2b = mb - m1b + d;
                if (m2b >= 0 && m2b <= j2) ++tcol;
            }
        int nrow = 0;
        for (int m1a = 0; m1a <= j1; ++m1a) {
            const int m2a = ma - m1a + d;
            if (m2a >= 0 && m2a <= j2) ++nrow;
        }
        cost += nrow * (6.0 * tcol + 3.0 * (j1 + j2 + 2) + 8.0) + 4.0 * ncol + 10.0;
    }
    return cost;
}

}  // namespace

double clebsch_gordan(int j1, int m1, int j2, int m2, int j, int m) { return cg_racah(j1, m1, j2, m2, j, m); }

int upload_cg_tables(Ctx* c) {
    std::vector<double> tab(kCgSize, 0.0);
    std::vector<float2> tabf(kCgSize, make_float2(0.f, 0.f));
    int n = 0;
    for (int j1 = 0; j1 <= kTJMax; ++j1)
        for (int j2 = 0; j2 <= j1; ++j2)
            for (int j = 0; j <= kTJMax; ++j) {
                if (!triple_ok(j1, j2, j, kTJMax)) continue;
                const int off = cg_offset(j1, j2, j);
                for (int ma = 0; ma <= j; ++ma)
                    for (int m1a = 0; m1a <= j1; ++m1a) {
                        const int m = 2 * ma - j, m1 = 2 * m1a - j1;
                        const double v = cg_racah(j1, m1, j2, m - m1, j, m);
                        tab[off + ma * (j1 + 1) + m1a] = v;
                        tabf[off + ma * (j1 + 1) + m1a] = make_float2((float)v, (float)v);
                    }
                ++n;
            }
    c->tables.cg = tab;
    MALA_CUDA_TRY(cudaMemcpyToSymbol(c_cg2, tabf.data(), sizeof(float2) * kCgSize));
    MALA_TRY(upload_zb_alt_cg(tabf.data(), (int)(sizeof(float2) * kCgSize)));

    MALA_TRY(c->ws_misc.reserve(c, sizeof(double) * kCgSize));
    c->tables.cg_d = c->ws_misc.as<double>();
    MALA_CUDA_TRY(cudaMemcpy(c->tables.cg_d, tab.data(), sizeof(double) * kCgSize, cudaMemcpyHostToDevice));
    // longest-processing-time assignment of triples to warps, per twojmax
    static int lists[kTJMax / 2 + 1][kZbWarps][kZbMaxList];
    for (int tj = 0; tj <= kTJMax; tj += 2) {
        std::vector<std::pair<double, int>> items;  // (cost, global id)
        std::vector<int> local_of(n_triples(kTJMax), -1);
        int gid = 0, lid = 0;
        for (int j1 = 0; j1 <= kTJMax; ++j1)
            for (int j2 = 0; j2 <= j1; ++j2)
                for (int j = 0; j <= kTJMax; ++j) {
                    if (!triple_ok(j1, j2, j, kTJMax)) continue;
                    if (triple_ok(j1, j2, j, tj)) {
                        items.push_back({triple_cost(j1, j2, j), gid});
                        local_of[gid] = lid++;
                    }
                    ++gid;
                }
        std::sort(items.begin(), items.end(), [](auto& a, auto& b) { return a.first > b.first; });
        double load[kZbWarps] = {0};
        int len[kZbWarps] = {0};
        for (int w = 0; w < kZbWarps; ++w)
            for (int s = 0; s < kZbMaxList; ++s) lists[tj / 2][w][s] = -1;
        for (auto& it : items) {
            int w = (int)(std::min_element(load, load + kZbWarps) - load);
            if (len[w] >= kZbMaxList - 1) return fail(MALA_ERR_UNSUPPORTED, "zb warp list overflow");
            lists[tj / 2][w][len[w]++] = it.second | (local_of[it.second] << 8);
            load[w] += it.first;
        }
    }
    MALA_CUDA_TRY(cudaMemcpyToSymbol(c_zb_list, lists, sizeof(lists)));
    MALA_TRY(upload_zb_lists_f64(&lists[0][0][0], (int)sizeof(lists)));
    // FP32 work units: per twojmax, for every triple (in index-set order) the
    // (ma, m1a) row pairs with a non-empty coupling, packed ma | m1a << 4 | twice << 8.
    std::vector<int> tri;               // int4 records (gid, first unit, count, column)
    std::vector<unsigned short> units;  // all units
    for (int tj = 0; tj <= kTJMax; tj += 2) {
        c->tables.tri_off[tj / 2] = (int)(tri.size() / 4);
        int gid = 0, lid = 0;
        const int ubase = (int)units.size();
        for (int j1 = 0; j1 <= kTJMax; ++j1)
            for (int j2 = 0; j2 <= j1; ++j2)
                for (int j = 0; j <= kTJMax; ++j) {
                    if (!triple_ok(j1, j2, j, kTJMax)) continue;
                    if (triple_ok(j1, j2, j, tj)) {
                        const int d = (j1 + j2 - j) / 2;
                        const int first = (int)units.size() - ubase;
                        for (int ma = 0; 2 * ma <= j; ++ma)
                            for (int m1a = 0; m1a <= j1; ++m1a) {
                                const int m2a = ma - m1a + d;
                                if (m2a < 0 || m2a > j2) continue;
                                // j1 == j2: the unit (ma, m1a) equals the unit (ma, m2a), since
                                // C(j1 m1 j1 m2|j m) = (-1)^(2 j1 - j) C(j1 m2 j1 m1|j m) and both
                                // coefficients of a term flip together; keep m1a <= m2a, count
                                // m1a < m2a twice (bit 8)
                                if (j1 == j2 && m1a > m2a) continue;
                                // a unit whose row coefficient C(j1 m1a j2 m2a | j ma) vanishes adds
                                // nothing: Racah's sum has accidental zeros (e.g. <1 0 1 0 | 1 0>),
                                // ~1e-16 in floating point against >= 1.8e-2 for every true nonzero
                                // coefficient up to twojmax 10
                                if (std::fabs(tab[cg_offset(j1, j2, j) + ma * (j1 + 1) + m1a]) < 1e-10) continue;
                                const int twice = (j1 == j2 && m1a < m2a) ? 1 : 0;
                                units.push_back((unsigned short)(ma | (m1a << 4) | (twice << 8)));
                            }
                        tri.insert(tri.end(), {gid, first, (int)units.size() - ubase - first, lid});
                        ++lid;
                    }
                    ++gid;
                }
        c->tables.unit_off[tj / 2] = ubase;
        {
            // J + 1 per output column of this twojmax (index-set order)
            float jp1[n_triples(kTJMax)] = {0};
            int col = 0;
            for (int j1 = 0; j1 <= tj; ++j1)
                for (int j2 = 0; j2 <= j1; ++j2)
                    for (int j = 0; j <= tj; ++j)
                        if (triple_ok(j1, j2, j, tj)) jp1[col++] = (float)(j + 1);
            MALA_CUDA_TRY(cudaMemcpyToSymbol(c_zb_jp1, jp1, sizeof(jp1), sizeof(jp1) * (tj / 2)));
            MALA_TRY(upload_zb_alt_jp1(jp1, (int)sizeof(jp1), (int)(sizeof(jp1) * (tj / 2))));
        }
        c->tables.tri_n[tj / 2] = lid;
    }
    const size_t tri_bytes = sizeof(int) * tri.size();
    const size_t unit_bytes = sizeof(unsigned short) * units.size();
    MALA_TRY(c->ws_units.reserve(c, tri_bytes + unit_bytes + 64));
    char* base = c->ws_units.as<char>();
    c->tables.tri_d = reinterpret_cast<int4*>(base);
    c->tables.units_d = reinterpret_cast<unsigned short*>(base + tri_bytes);
    c->tables.err_d = reinterpret_cast<int*>(base + ((tri_bytes + unit_bytes + 15) & ~size_t(15)));
    MALA_CUDA_TRY(cudaMemcpy(base, tri.data(), tri_bytes, cudaMemcpyHostToDevice));
    MALA_CUDA_TRY(cudaMemcpy(base + tri_bytes, units.data(), unit_bytes, cudaMemcpyHostToDevice));
    MALA_CUDA_TRY(cudaMemset(c->tables.err_d, 0, sizeof(int) * 8));
    return MALA_OK;
}

// variants of the FP32 kernel (warps per CTA); index 0 is the default
constexpr int kZbVariantWarps[] = {kZbUWarps, kZbWarpsAlt};

int zb_variant_count() { return 2; }
int zb_variant_warps(int v) { return kZbVariantWarps[(v == 1) ? 1 : 0]; }

template <>
void launch_zb<float>(Ctx* c, int twojmax, const float* u_half, const BatchSnap* bs, int nsnap, int64_t tile0,
                      int64_t ntiles, const int* nbr_cnt, double wself, float* B, cudaStream_t st, int variant) {
    if (variant == 1) launch_zb_alt(c, twojmax, u_half, bs, nsnap, tile0, ntiles, nbr_cnt, wself, B, st);
    else zb_units_launch<kZbUWarps>(c, twojmax, u_half, bs, nsnap, tile0, ntiles, nbr_cnt, wself, B, st);
}

}  // namespace mala
