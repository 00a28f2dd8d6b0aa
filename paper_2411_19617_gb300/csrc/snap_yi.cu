// snap_yi.cu -- host side of the FP32 Y step as units (snap_yi.h): the
// Clebsch-Gordan blocks of the couplings (uploaded once per device into each
// group's constant memory), the per-twojmax plan (rows, the units of every row
// dealt to the warps, the coupling -> triple map) and the four launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "mala_internal.h"
#include "snap_yi.h"

namespace mala {

namespace {

using UploadFn = int (*)(const float*, int, const int*, const float*);
using LaunchFn = int (*)(const YiLaunch&);
constexpr UploadFn kUpload[kYiGroups] = {yi_upload_g0, yi_upload_g1, yi_upload_g2, yi_upload_g3};
constexpr LaunchFn kLaunch[kYiGroups] = {yi_launch_g0, yi_launch_g1, yi_launch_g2, yi_launch_g3};

// entry (r, m1) of coupling (c; a, b)'s block: C(a m1, b m2 | c m), m = 2r - c, m1 = 2 m1a - a
double ycg_value(int c, int a, int b, int r, int m1a) {
    const int d = (a + b - c) / 2;
    const int m2a = r - m1a + d;
    if (m2a < 0 || m2a > b) return 0.0;
    return clebsch_gordan(a, 2 * m1a - a, b, 2 * m2a - b, c, 2 * r - c);
}

std::mutex g_upload_mu;
bool g_uploaded[64] = {false};

// Per group: the full blocks of its couplings, [m][m1] over a and (a != b) [m][m2] over b
// (C(b m2, a m1 | c m) = (-1)^((a + b - c)/2) C(a m1, b m2 | c m)), and per coupling
// {a, b, offset of the (a, b) block, offset of the (b, a) block}.
int ensure_yi_tables(int device) {
    std::lock_guard<std::mutex> lk(g_upload_mu);
    if (device >= 0 && device < 64 && g_uploaded[device]) return MALA_OK;
    std::vector<float> fn((kTJMax + 1) * (kTJMax + 1) * (kTJMax + 1), 0.f);
    for (int J = 0; J <= kTJMax; ++J)
        for (int x = 0; x <= J; ++x)
            for (int y = 0; y <= J; ++y)
                fn[(J * (kTJMax + 1) + x) * (kTJMax + 1) + y] =
                    (float)std::sqrt(fact_d(J - x) * fact_d(x) / (fact_d(J - y) * fact_d(y)));
    for (int g = 0; g < kYiGroups; ++g) {
        const unsigned mask = yi_mask(g);
        std::vector<float> tab;
        std::vector<int> info(4 * (size_t)kNCouplings, -1);
        for (int c = 0; c <= kTJMax; ++c) {
            if (!((mask >> c) & 1u)) continue;
            for (int i = 0; i < n_couplings(c); ++i) {
                const int a = coupling_field(c, i, 0), b = coupling_field(c, i, 1);
                const int k = coupling_base(c) + i;
                info[4 * k] = a;
                info[4 * k + 1] = b;
                info[4 * k + 2] = (int)tab.size();
                for (int m = 0; m <= c; ++m)
                    for (int m1a = 0; m1a <= a; ++m1a) tab.push_back((float)ycg_value(c, a, b, m, m1a));
                if (a != b) {
                    const double sg = (((a + b - c) / 2) & 1) ? -1.0 : 1.0;
                    const int d = (a + b - c) / 2;
                    info[4 * k + 3] = (int)tab.size();
                    for (int m = 0; m <= c; ++m)
                        for (int m2a = 0; m2a <= b; ++m2a) {
                            const int m1a = m - m2a + d;  // the partner in u^a
                            tab.push_back(m1a < 0 || m1a > a ? 0.f : (float)(sg * ycg_value(c, a, b, m, m1a)));
                        }
                } else {
                    info[4 * k + 3] = info[4 * k + 2];
                }
            }
        }
        MALA_TRY(kUpload[g](tab.data(), (int)tab.size(), info.data(), fn.data()));
    }
    if (device >= 0 && device < 64) g_uploaded[device] = true;
    return MALA_OK;
}

struct HostPlan {
    std::vector<int2> rows;
    std::vector<int> off;
    std::vector<unsigned short> units;
    std::vector<int> be_t;
    std::vector<float> be_f;
    int row0[kYiGroups] = {0, 0, 0, 0}, nrows[kYiGroups] = {0, 0, 0, 0};
};

int coupling_id(int c, int a, int b) {
    if (a < b) std::swap(a, b);
    for (int i = 0; i < n_couplings(c); ++i)
        if (coupling_field(c, i, 0) == a && coupling_field(c, i, 1) == b) return coupling_base(c) + i;
    return -1;
}

void build_plan(int tj, HostPlan& H) {
    // coupling -> (triple, factor): the sorted momenta of a coupling are one triple
    H.be_t.assign(kNCouplings, 0);
    H.be_f.assign(kNCouplings, 0.f);
    std::vector<double> f(kNCouplings, 0.0);
    int t = 0;
    for (int j1 = 0; j1 <= tj; ++j1)
        for (int j2 = 0; j2 <= j1; ++j2)
            for (int j = 0; j <= tj; ++j) {
                if (!triple_ok(j1, j2, j, tj)) continue;
                const int k0 = coupling_id(j, j1, j2), k1 = coupling_id(j1, j, j2), k2 = coupling_id(j2, j, j1);
                H.be_t[k0] = H.be_t[k1] = H.be_t[k2] = t;
                f[k0] += 1.0;
                f[k1] += (j + 1.0) / (j1 + 1.0);
                f[k2] += (j + 1.0) / (j2 + 1.0);
                ++t;
            }
    for (int k = 0; k < kNCouplings; ++k) H.be_f[k] = (float)f[k];
    // rows of every group; each row's units dealt to the warps longest first
    for (int g = 0; g < kYiGroups; ++g) {
        H.row0[g] = (int)H.rows.size();
        for (int c = tj; c >= 0; --c) {
            if (!((yi_mask(g) >> c) & 1u)) continue;
            for (int ma = 0; 2 * ma <= c; ++ma) {
                const int ncol = 2 * ma == c ? c / 2 + 1 : c + 1;
                std::vector<unsigned short> us;
                std::vector<double> cost;
                for (int i = 0; i < n_couplings(c); ++i) {
                    const int a = coupling_field(c, i, 0), b = coupling_field(c, i, 1);
                    if (a > tj) continue;
                    const int d = (a + b - c) / 2;
                    for (int m1a = 0; m1a <= a; ++m1a) {
                        const int m2a = ma - m1a + d;
                        if (m2a < 0 || m2a > b) continue;
                        if (std::fabs(ycg_value(c, a, b, ma, m1a)) < 1e-10) continue;
                        // the shorter row in registers when the longer one lies at or below its
                        // middle (it is then read from shared memory), else the other way round
                        const int swap = (2 * m1a <= a) ? 1 : 0;
                        const int R = swap ? b : a;
                        us.push_back((unsigned short)(i | (m1a << 6) | (swap << 10)));
                        cost.push_back(12.0 * (R + 1) * ((ncol + 1) / 2) + 4.0 * (R + 2) * ((ncol + 1) / 2) +
                                       2.0 * (R + 1) + 24.0);
                    }
                }
                std::vector<int> order(us.size());
                std::iota(order.begin(), order.end(), 0);
                std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
                std::vector<std::vector<int>> lists(kYuWarps);
                std::vector<double> load(kYuWarps, 0.0);
                for (int u : order) {
                    const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
                    lists[w].push_back(u);
                    load[w] += cost[u];
                }
                H.rows.push_back(make_int2(c, ma));
                for (int w = 0; w < kYuWarps; ++w) {
                    // each warp keeps the dealing order: a coupling's units (equal cost, adjacent in the
                    // stable order) go to different warps, so the warps run the same coupling's code at
                    // about the same time
                    H.off.push_back((int)H.units.size());
                    for (int u : lists[w]) H.units.push_back(us[u]);
                }
                H.off.push_back((int)H.units.size());
            }
        }
        H.nrows[g] = (int)H.rows.size() - H.row0[g];
    }
}

int ensure_plan(Ctx* c, int tj) {
    YiPlanState& S = c->yplan;
    if (S.tj == tj && c->ws_yplan.ptr) return MALA_OK;
    HostPlan H;
    build_plan(tj, H);
    std::vector<std::pair<const void*, size_t>> parts = {
        {H.rows.data(), H.rows.size() * sizeof(int2)},
        {H.off.data(), H.off.size() * sizeof(int)},
        {H.units.data(), H.units.size() * sizeof(unsigned short)},
        {H.be_t.data(), H.be_t.size() * sizeof(int)},
        {H.be_f.data(), H.be_f.size() * sizeof(float)}};
    std::vector<size_t> off;
    size_t total = 0;
    for (auto& p : parts) {
        off.push_back(total);
        total += (p.second + 255) & ~size_t(255);
    }
    std::vector<unsigned char> blob(total, 0);
    for (size_t i = 0; i < parts.size(); ++i)
        if (parts[i].second) memcpy(blob.data() + off[i], parts[i].first, parts[i].second);
    MALA_TRY(c->ws_yplan.reserve(c, total + 256));
    MALA_CUDA_TRY(cudaMemcpy(c->ws_yplan.ptr, blob.data(), total, cudaMemcpyHostToDevice));
    for (int i = 0; i < 5; ++i) S.off[i] = off[i];
    for (int g = 0; g < kYiGroups; ++g) {
        S.row0[g] = H.row0[g];
        S.nrows[g] = H.nrows[g];
    }
    S.tj = tj;
    return MALA_OK;
}

}  // namespace

// y[p] = conj(Y) N over the full set, FP32, from the full u and beta (both point-major).
int yi_units(Ctx* c, int tj, const float* u_full, const float* beta, int nB, int64_t P, float* y, cudaStream_t st) {
    if (tj < 0 || tj > kTJMax || (tj & 1)) return fail(MALA_ERR_UNSUPPORTED, "twojmax %d has no compiled Y kernel", tj);
    if (P <= 0) return MALA_OK;
    MALA_TRY(ensure_yi_tables(c->device));
    MALA_TRY(ensure_plan(c, tj));
    const YiPlanState& S = c->yplan;
    const char* b = c->ws_yplan.as<const char>();
    YiLaunch a;
    a.tj = tj;
    a.u_full = u_full;
    a.beta = beta;
    a.nB = nB;
    a.P = P;
    a.y = y;
    a.st = st;
    a.plan.rows = reinterpret_cast<const int2*>(b + S.off[0]);
    a.plan.off = reinterpret_cast<const int*>(b + S.off[1]);
    a.plan.units = reinterpret_cast<const unsigned short*>(b + S.off[2]);
    a.plan.be_t = reinterpret_cast<const int*>(b + S.off[3]);
    a.plan.be_f = reinterpret_cast<const float*>(b + S.off[4]);
    for (int g = 0; g < kYiGroups; ++g) {
        a.plan.row0 = S.row0[g];
        a.plan.nrows = S.nrows[g];
        int rc = MALA_OK;
        if (a.plan.nrows > 0) MALA_PROF(c, "k_yi", st, rc = kLaunch[g](a));
        MALA_TRY(rc);
    }
    return MALA_OK;
}

}  // namespace mala
