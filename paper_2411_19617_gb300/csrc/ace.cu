// ace.cu -- grid-centred ACE descriptors (paper Sec. "Atomic cluster expansion
// descriptors", Eqs. unweighted_ionicdensity, gridatom_basis, grid_base,
// product_grid_basis, ace_grid) for body orders N = 1, 2, 3.
//
// Grid basis: A_{mu n l m}(r) = sum over the neighbours of r of species mu of
// R_n(|d|) Y_l^m(d/|d|), with R_n(r) = T_n(1 - 2r/r_cut) (1 + cos(pi r/r_cut))/2
// (Chebyshev of the scaled distance, vanishing smoothly at the cutoff) and
// complex orthonormal Y_l^m (Condon-Shortley).  Y_l^m = N_lm Ptilde_l^m(z) (x + i y)^m
// for the unit vector (x, y, z), where Ptilde_l^m = P_l^m / sin^m(theta) obeys
//   Ptilde_m^m = (-1)^m (2m-1)!!,  Ptilde_{m+1}^m = (2m+1) z Ptilde_m^m,
//   (l - m) Ptilde_l^m = (2l-1) z Ptilde_{l-1}^m - (l+m-1) Ptilde_{l-2}^m,
// a polynomial form that needs no angle and no division at the poles; only
// m >= 0 is summed over the neighbours (A_{l,-m} = (-1)^m conj(A_{l,m}) for a
// real density fills the rest).
// Invariants: N = 1: A_{mu n 0 0}; N = 2: sum_m <l m l -m|0 0> A_{c1 l m} A_{c2 l -m};
// N = 3: sum <l1 m1 l2 m2|l3 M><l3 M l3 -M|0 0> A_{c1 l1 m1} A_{c2 l2 m2} A_{c3 l3 -M}.
//
// Mapping: one warp per grid point (persistent).  Lanes take neighbours; each
// lane evaluates R_n and Y_l^m of its neighbour, and for every (species, n) a
// reduce-scatter over the warp (fixed order: deterministic) leaves lane l with
// the batch's sum of value l of a chunk of 16 (l, m) elements (re, im), which
// it adds into the warp's shared-memory copy of A; the m < 0 elements are then
// filled by the symmetry.  The lanes then take descriptor columns, in descending
// order of cost so that the 32 columns taken together cost about the same, and
// contract A with host-built coefficient lists (N = 2 over m >= 0 and N = 3 over
// half of the (m1, m2) plane: the other half gives the complex conjugates), each
// column written to its place in the row.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "mala_internal.h"

namespace mala {

namespace {

constexpr int kAceWarps = 4;
constexpr int kAceLMax = 8;                                   // largest l compiled
constexpr int kAceLM = (kAceLMax + 1) * (kAceLMax + 2) / 2;   // (l, m >= 0) pairs
constexpr int kAceNMax = 16;
constexpr int kAceSpecies = 8;
constexpr int kAceMaxA = 1024;                                 // complex A elements per point

template <class T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };

// descriptor column: kind 1, 2, 3; channel bases into A (mu n block * n_lmf); l values; coefficient
// list; d: its place in the output row (the kernel takes the columns in descending order of cost)
struct AceCol {
    int kind, a1, a2, a3, l1, l2, l3, c_off, c_cnt, d;
};
// one term of an N = 3 column: c A1[i1] A2[i2] A3[i3], i = lm_full(l, m) within the channel's
// block (m of either sign), packed as i1 | i2 << 10 | i3 << 20; cf = c rounded to FP32 on the host
struct AceCoef {
    double c;
    float cf;
    uint32_t idx;
};

struct AceArgs {
    int64_t P;
    int cap;
    const int* cnt;
    const int* atoms;
    const int* shifts;
    const int* species;  // [n_atoms] or NULL
    const double* wpos;  // [3][n_atoms]
    const double* gcoord;
    int n_atoms, grid[3];
    double L[3];
    double rcut;
    int lmax, nmax, n_species;
    int n_lm;   // (l, m >= 0) elements of a channel: the elements the neighbour sums produce
    int n_lmf;  // (l, m) elements of a channel, m of either sign: its block in A
    int nA, n_desc;
    const AceCol* cols;
    const AceCoef* coefs;
    int stage;            // column and coefficient tables copied into shared memory
    int n_coef;
};

__device__ __forceinline__ int lm_index(int l, int m) { return l * (l + 1) / 2 + m; }
__host__ __device__ __forceinline__ int lm_full(int l, int m) { return l * l + l + m; }  // -l <= m <= l

// (l, m) of the m >= 0 element with index h = lm_index(l, m)
__device__ __forceinline__ int2 lm_of(int h) {
    int l = 0;
    while ((l + 1) * (l + 2) / 2 <= h) ++l;
    return make_int2(l, h - l * (l + 1) / 2);
}

// N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) by (l, m >= 0) index, every compiled l
__constant__ double c_ace_ynorm[kAceLM];
__constant__ float c_ace_ynormf[kAceLM];  // the same rounded to FP32

template <class T> __device__ __forceinline__ T ace_ynorm(int i);
template <> __device__ __forceinline__ float ace_ynorm<float>(int i) { return c_ace_ynormf[i]; }
template <> __device__ __forceinline__ double ace_ynorm<double>(int i) { return c_ace_ynorm[i]; }

__host__ __device__ inline size_t ace_coef_bytes(int n_coef) { return ((size_t)n_coef * sizeof(AceCoef) + 15) & ~size_t(15); }
__host__ __device__ inline size_t ace_table_bytes(int n_desc, int n_coef) {
    return ace_coef_bytes(n_coef) + (((size_t)n_desc * sizeof(AceCol) + 15) & ~size_t(15));
}

// Reduce-scatter over the warp: each lane holds N values (N a multiple of 32);
// after log2(32) halving steps lane l holds the warp sums of values
// (N/32) l .. (N/32) l + N/32 - 1 in v[0 .. N/32 - 1].  A step exchanges half of
// the live values with the partner lane (lane ^ mask): the lane whose mask bit
// is set keeps the upper half.  The order of the additions is fixed.
template <class T, int N, int H>
__device__ __forceinline__ void reduce_scatter(T (&v)[N], int lane) {
    if constexpr (H >= N / 32) {
        constexpr int mask = 32 * H / N;
        const bool up = (lane & mask) != 0;
#pragma unroll
        for (int i = 0; i < H; ++i) {
            const T send = up ? v[i] : v[i + H];
            const T keep = up ? v[i + H] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
        }
        reduce_scatter<T, N, H / 2>(v, lane);
    }
}

// LMX: the largest l the kernel evaluates (4, 6 or 8, at least lmax); STAGE: the column and
// coefficient tables are copied into shared memory (else read from global memory)
// (FP32 up to l = 6: four CTAs per SM, 128 registers without spills, 16 warps to hide the shuffle
// and shared-load latencies; l = 8 and FP64 need more registers and keep three)
template <class T, int LMX, bool STAGE>
__global__ void __launch_bounds__(kAceWarps * 32, (sizeof(T) == 4 && LMX <= 6) ? 4 : 3)
    k_ace(AceArgs g, T* __restrict__ out) {
    constexpr int NLM = (LMX + 1) * (LMX + 2) / 2;
    using C = typename Cx<T>::type;
    extern __shared__ __align__(16) unsigned char smem_ace[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // shared memory: [coefficients][columns] (when staged) | A of each warp
    const size_t tab_bytes = STAGE ? ace_table_bytes(g.n_desc, g.n_coef) : 0;
    // the pointers are fixed per instantiation, so staged tables are read by shared-memory loads
    const AceCoef* coefs = STAGE ? reinterpret_cast<const AceCoef*>(smem_ace) : g.coefs;
    const AceCol* cols = STAGE ? reinterpret_cast<const AceCol*>(smem_ace + ace_coef_bytes(g.n_coef)) : g.cols;
    if constexpr (STAGE) {
        AceCoef* sc = reinterpret_cast<AceCoef*>(smem_ace);
        AceCol* scl = reinterpret_cast<AceCol*>(smem_ace + ace_coef_bytes(g.n_coef));
        for (int i = threadIdx.x; i < g.n_coef; i += blockDim.x) sc[i] = g.coefs[i];
        for (int i = threadIdx.x; i < g.n_desc; i += blockDim.x) scl[i] = g.cols[i];
        __syncthreads();
    }
    C* A = reinterpret_cast<C*>(smem_ace + tab_bytes) + (size_t)warp * g.nA;
    // the block index of the m >= 0 element this lane adds in each chunk of 16 (see below), and of
    // the elements h = lane, lane + 32 it mirrors to m < 0 (m = 0: nothing to mirror)
    int fchunk[(NLM + 15) / 16];
#pragma unroll
    for (int c = 0; c < (NLM + 15) / 16; ++c) {
        const int2 lm = lm_of(16 * c + (lane >> 1));
        fchunk[c] = lm_full(lm.x, lm.y);
    }
    const int2 mir0 = lm_of(lane), mir1 = lm_of(lane + 32);
    for (int64_t p = (int64_t)blockIdx.x * kAceWarps + warp; p < g.P; p += (int64_t)gridDim.x * kAceWarps) {
        for (int e = lane; e < g.nA; e += 32) {
            A[e].x = T(0);
            A[e].y = T(0);
        }
        __syncwarp();
        const int n = min(g.cnt[p], g.cap);
        // grid index in 32 bits (P < 2^32, checked on the host)
        const uint32_t pu = (uint32_t)p, gx = (uint32_t)g.grid[0], gy = (uint32_t)g.grid[1];
        const uint32_t pyz = pu / gx;
        const int ix = (int)(pu - pyz * gx);
        const int iy = (int)(pyz % gy);
        const int iz = (int)(pyz / gy);
        const double rx = g.gcoord[ix], ry = g.gcoord[g.grid[0] + iy], rz = g.gcoord[g.grid[0] + g.grid[1] + iz];
        for (int k0 = 0; k0 < n; k0 += 32) {
            const int k = k0 + lane;
            bool valid = k < n;
            int sp = -1;
            T ux = T(0), uy = T(0), uz = T(1), xs = T(0), fc = T(0);
            bool center = false;
            if (valid) {
                const size_t q = (size_t)p * g.cap + k;
                const int a = g.atoms[q];
                sp = g.species ? g.species[a] : 0;
                const double dx = (g.wpos[a] + g.shifts[3 * q] * g.L[0]) - rx;
                const double dy = (g.wpos[g.n_atoms + a] + g.shifts[3 * q + 1] * g.L[1]) - ry;
                const double dz = (g.wpos[2 * g.n_atoms + a] + g.shifts[3 * q + 2] * g.L[2]) - rz;
                const T r = (T)sqrt(dx * dx + dy * dy + dz * dz);
                center = !(r > T(0));
                if (!center) {
                    ux = (T)dx / r;
                    uy = (T)dy / r;
                    uz = (T)dz / r;
                }
                xs = T(1) - T(2) * r / (T)g.rcut;
                T cp;
                if constexpr (sizeof(T) == 4) cp = cospif(r / (float)g.rcut);
                else cp = cospi(r / g.rcut);
                fc = T(0.5) * (T(1) + cp);
            }
            // Y_l^m (m >= 0) of the lane's neighbour
            T yr[NLM], yi[NLM];
            {
                T pmm = T(1);             // Ptilde_m^m
                T er = T(1), ei = T(0);   // (x + i y)^m
#pragma unroll
                for (int m = 0; m <= LMX; ++m) {
                    if (m > 0) {
                        pmm *= -T(2 * m - 1);
                        const T nr = er * ux - ei * uy, ni = er * uy + ei * ux;
                        er = nr;
                        ei = ni;
                    }
                    T p2 = T(0), p1 = pmm;
#pragma unroll
                    for (int l = m; l <= LMX; ++l) {
                        T pl;
                        if (l == m) {
                            pl = pmm;
                        } else if (l == m + 1) {
                            pl = T(2 * m + 1) * uz * pmm;
                        } else {
                            // (l - m) P_l = (2l - 1) z P_{l-1} - (l + m - 1) P_{l-2}, the ratios as constants
                            const T ca = T((2.0 * l - 1.0) / (double)(l - m)), cb = T((l + m - 1.0) / (double)(l - m));
                            pl = ca * uz * p1 - cb * p2;
                        }
                        if (l > m) {
                            p2 = p1;
                            p1 = pl;
                        }
                        const T nrm = ace_ynorm<T>(lm_index(l, m)) * (center && l > 0 ? T(0) : T(1));
                        yr[lm_index(l, m)] = nrm * pl * er;
                        yi[lm_index(l, m)] = nrm * pl * ei;
                    }
                }
            }
            // radial functions by the Chebyshev recurrence; reduce each A element over the warp
            for (int s = 0; s < g.n_species; ++s) {
                const bool mine = valid && sp == s;
                T t0 = T(1), t1 = xs;
                for (int nn = 0; nn < g.nmax; ++nn) {
                    T tn;
                    if (nn == 0) tn = T(1);
                    else if (nn == 1) tn = xs;
                    else {
                        tn = T(2) * xs * t1 - t0;
                        t0 = t1;
                        t1 = tn;
                    }
                    const T rn = mine ? tn * fc : T(0);
                    const int base = (s * g.nmax + nn) * g.n_lmf;
                    // the (l, m) elements in chunks of 16: v holds (re, im) of chunk element e at 2e, 2e + 1;
                    // after the reduce-scatter lane l holds the warp sum of value l of the chunk
#pragma unroll
                    for (int c0 = 0; c0 < NLM; c0 += 16) {
                        if (c0 >= g.n_lm) break;
                        T v[32];
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            const int lm = c0 + e < NLM ? c0 + e : 0;
                            v[2 * e] = c0 + e < NLM ? rn * yr[lm] : T(0);
                            v[2 * e + 1] = c0 + e < NLM ? rn * yi[lm] : T(0);
                        }
                        reduce_scatter<T, 32, 16>(v, lane);
                        if (c0 + (lane >> 1) < g.n_lm) {
                            const int f = base + fchunk[c0 / 16];
                            if (lane & 1) A[f].y += v[0];
                            else A[f].x += v[0];
                        }
                    }
                }
            }
            __syncwarp();
        }
        __syncwarp();
        // A_{l,-m} = (-1)^m conj(A_{l,m}), so that the invariants index A by (l, m) of either sign
        for (int ch = 0; ch < g.n_species * g.nmax; ++ch) {
            C* Ac = A + ch * g.n_lmf;
            if (lane < g.n_lm && mir0.y > 0) {
                const C a = Ac[lm_full(mir0.x, mir0.y)];
                Ac[lm_full(mir0.x, -mir0.y)] = (mir0.y & 1) ? C{-a.x, a.y} : C{a.x, -a.y};
            }
            if (lane + 32 < g.n_lm && mir1.y > 0) {
                const C a = Ac[lm_full(mir1.x, mir1.y)];
                Ac[lm_full(mir1.x, -mir1.y)] = (mir1.y & 1) ? C{-a.x, a.y} : C{a.x, -a.y};
            }
        }
        __syncwarp();
        // invariants
        T* o = out + (size_t)p * g.n_desc;
        for (int d = lane; d < g.n_desc; d += 32) {
            const AceCol cl = cols[d];
            T v = T(0);
            if (cl.kind == 1) {
                v = A[cl.a1].x;
            } else if (cl.kind == 2) {
                // sum_m <l m l -m|0 0> Re(A1_m A2_-m) with A_-m = (-1)^m conj(A_m) and <l m l -m|0 0> =
                // (-1)^(l-m)/sqrt(2l+1): (-1)^l/sqrt(2l+1) (Re(A1_0 A2_0) + 2 sum_{m>0} Re(A1_m conj(A2_m)))
                const int l = cl.l1, b0 = lm_full(l, 0);
                const C x0 = A[cl.a1 + b0], y0 = A[cl.a2 + b0];
                T s2 = T(0);
                for (int m = 1; m <= l; ++m) {
                    const C x = A[cl.a1 + b0 + m], y = A[cl.a2 + b0 + m];
                    s2 += x.x * y.x + x.y * y.y;
                }
                const T inv = ((l & 1) ? -T(1) : T(1)) / sqrt(T(2 * l + 1));
                v = inv * ((x0.x * y0.x - x0.y * y0.y) + T(2) * s2);
            } else {
                for (int q = cl.c_off; q < cl.c_off + cl.c_cnt; ++q) {
                    const AceCoef cf = coefs[q];
                    const C x = A[cl.a1 + (cf.idx & 1023u)], y = A[cl.a2 + ((cf.idx >> 10) & 1023u)],
                            z = A[cl.a3 + (cf.idx >> 20)];
                    const T pr = x.x * y.x - x.y * y.y, pi_ = x.x * y.y + x.y * y.x;
                    T cv;
                    if constexpr (sizeof(T) == 4) cv = cf.cf;
                    else cv = cf.c;
                    v += cv * (pr * z.x - pi_ * z.y);
                }
            }
            o[cl.d] = v;
        }
        __syncwarp();
    }
}

}  // namespace

// the kernel with the table path the arguments ask for, as one wave of the CTAs the SMs hold at once
// (the warps stride over the points, so a second wave would only add a partly idle tail)
template <class T, int LMX, bool STAGE>
static void launch_ace_k(int64_t want, int sms, size_t smem, const AceArgs& g, T* out, cudaStream_t st) {
    cudaFuncSetAttribute(k_ace<T, LMX, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ace<T, LMX, STAGE>, kAceWarps * 32, smem) !=
            cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * per_sm));
    k_ace<T, LMX, STAGE><<<grid, kAceWarps * 32, smem, st>>>(g, out);
}

template <class T, int LMX>
static void launch_ace_l(int64_t want, int sms, size_t smem, const AceArgs& g, T* out, cudaStream_t st) {
    if (g.stage) launch_ace_k<T, LMX, true>(want, sms, smem, g, out, st);
    else launch_ace_k<T, LMX, false>(want, sms, smem, g, out, st);
}

// the kernel compiled for the smallest supported l range that covers lmax
template <class T>
static void launch_ace(int lmax, int64_t want, int sms, size_t smem, const AceArgs& g, T* out, cudaStream_t st) {
    if (lmax <= 4) launch_ace_l<T, 4>(want, sms, smem, g, out, st);
    else if (lmax <= 6) launch_ace_l<T, 6>(want, sms, smem, g, out, st);
    else launch_ace_l<T, kAceLMax>(want, sms, smem, g, out, st);
}

// columns in the order of the documented enumeration; returns the count
static int ace_columns(const mala_ace_params* ap, std::vector<AceCol>* cols, std::vector<AceCoef>* coefs) {
    const int ns = ap->n_species;
    const int nmax = std::max(ap->nmax1, std::max(ap->nmax2, ap->nmax3));
    const int lmax = std::max(ap->lmax2, ap->lmax3);
    const int nlmf = (lmax + 1) * (lmax + 1);
    auto base = [&](int mu, int n) { return (mu * nmax + n) * nlmf; };
    std::vector<AceCol> cl;
    std::vector<AceCoef> cf;
    for (int mu = 0; mu < ns; ++mu)
        for (int n = 0; n < ap->nmax1; ++n) cl.push_back(AceCol{1, base(mu, n), 0, 0, 0, 0, 0, 0, 0, 0});
    std::vector<std::pair<int, int>> ch2;
    for (int mu = 0; mu < ns; ++mu)
        for (int n = 0; n < ap->nmax2; ++n) ch2.push_back({mu, n});
    for (size_t i = 0; i < ch2.size(); ++i)
        for (size_t j = i; j < ch2.size(); ++j)
            for (int l = 0; l <= ap->lmax2; ++l)
                cl.push_back(AceCol{2, base(ch2[i].first, ch2[i].second), base(ch2[j].first, ch2[j].second), 0, l, l,
                                    0, 0, 0, 0});
    struct Ch3 {
        int mu, n, l;
    };
    std::vector<Ch3> ch3;
    for (int mu = 0; mu < ns; ++mu)
        for (int n = 0; n < ap->nmax3; ++n)
            for (int l = 0; l <= ap->lmax3; ++l) ch3.push_back({mu, n, l});
    std::vector<int> lists((size_t)(lmax + 1) * (lmax + 1) * (lmax + 1) * 2, -1);  // (l1,l2,l3) -> off, cnt
    auto coef_list = [&](int l1, int l2, int l3, int* off, int* cnt) {
        const size_t key = ((size_t)l1 * (lmax + 1) + l2) * (lmax + 1) + l3;
        if (lists[2 * key] < 0) {
            lists[2 * key] = (int)cf.size();
            for (int m1 = -l1; m1 <= l1; ++m1)
                for (int m2 = -l2; m2 <= l2; ++m2) {
                    const int M = m1 + m2;
                    if (M < -l3 || M > l3) continue;
                    const double c = clebsch_gordan(2 * l1, 2 * m1, 2 * l2, 2 * m2, 2 * l3, 2 * M) *
                                     clebsch_gordan(2 * l3, 2 * M, 2 * l3, -2 * M, 0, 0);
                    // (-m1, -m2, M) gives the conjugate of the (m1, m2, -M) product with the same
                    // coefficient (l1 + l2 + l3 even, A_{l,-m} = (-1)^m conj(A_{l,m}), A_{l,0} real):
                    // keep M > 0, or M = 0 and m1 > 0, at twice the weight, and the all-zero term once
                    const bool upper = M > 0 || (M == 0 && m1 > 0);
                    if (c != 0.0 && (upper || (m1 == 0 && m2 == 0))) {
                        const double cw = upper ? 2.0 * c : c;
                        const uint32_t idx = (uint32_t)lm_full(l1, m1) | (uint32_t)lm_full(l2, m2) << 10 |
                                             (uint32_t)lm_full(l3, -M) << 20;
                        cf.push_back(AceCoef{cw, (float)cw, idx});
                    }
                }
            lists[2 * key + 1] = (int)cf.size() - lists[2 * key];
        }
        *off = lists[2 * key];
        *cnt = lists[2 * key + 1];
    };
    for (size_t i = 0; i < ch3.size(); ++i)
        for (size_t j = i; j < ch3.size(); ++j)
            for (size_t k = j; k < ch3.size(); ++k) {
                const int l1 = ch3[i].l, l2 = ch3[j].l, l3 = ch3[k].l;
                if (l3 < std::abs(l1 - l2) || l3 > l1 + l2 || ((l1 + l2 + l3) & 1)) continue;
                int off = 0, cnt = 0;
                coef_list(l1, l2, l3, &off, &cnt);
                cl.push_back(AceCol{3, base(ch3[i].mu, ch3[i].n), base(ch3[j].mu, ch3[j].n), base(ch3[k].mu, ch3[k].n),
                                    l1, l2, l3, off, cnt, 0});
            }
    for (size_t i = 0; i < cl.size(); ++i) cl[i].d = (int)i;
    if (cols) *cols = cl;
    if (coefs) *coefs = cf;
    return (int)cl.size();
}

int ace_count(const mala_ace_params* ap) { return ace_columns(ap, nullptr, nullptr); }

int check_ace_params(const mala_ace_params* ap) {
    if (!ap) return fail(MALA_ERR_INVALID_ARG, "ACE parameters are NULL");
    if (!(ap->rcut > 0.0) || !std::isfinite(ap->rcut)) return fail(MALA_ERR_INVALID_ARG, "rcut must be > 0");
    if (ap->n_species < 1 || ap->n_species > kAceSpecies)
        return fail(MALA_ERR_UNSUPPORTED, "n_species must be 1..%d", kAceSpecies);
    if (ap->nmax1 < 0 || ap->nmax2 < 0 || ap->nmax3 < 0 || ap->lmax2 < 0 || ap->lmax3 < 0)
        return fail(MALA_ERR_INVALID_ARG, "negative ACE sizes");
    const int nmax = std::max(ap->nmax1, std::max(ap->nmax2, ap->nmax3));
    const int lmax = std::max(ap->lmax2, ap->lmax3);
    if (nmax < 1 || nmax > kAceNMax) return fail(MALA_ERR_UNSUPPORTED, "radial count must be 1..%d", kAceNMax);
    if (lmax > kAceLMax) return fail(MALA_ERR_UNSUPPORTED, "lmax must be <= %d", kAceLMax);
    if (ap->n_species * nmax * (lmax + 1) * (lmax + 2) / 2 > kAceMaxA)
        return fail(MALA_ERR_UNSUPPORTED, "n_species x nmax x (lmax+1)(lmax+2)/2 must be <= %d", kAceMaxA);
    return MALA_OK;
}

// ACE descriptors of one snapshot from its staged atoms and complete neighbour lists
int ace_from_lists(Ctx* c, const SnapDev& sd, const mala_snapshot* snap, const mala_ace_params* ap,
                   const NbrOut& nl, void* out, mala_precision prec, cudaStream_t st) {
    if (sd.g.P >= ((int64_t)1 << 32))  // the kernel's grid-index arithmetic is 32-bit
        return fail(MALA_ERR_UNSUPPORTED, "ACE descriptors need fewer than 2^32 grid points");
    std::vector<AceCol> cols;
    std::vector<AceCoef> coefs;
    const int nd = ace_columns(ap, &cols, &coefs);
    // a warp takes 32 columns at a time and waits for its costliest: order them by cost (terms,
    // an N = 3 term about twice an N = 2 one), so that the columns taken together cost about the same
    // (columns of equal cost by coefficient list, so that lanes taken together read the same terms)
    auto cost = [](const AceCol& x) { return x.kind == 3 ? 2 * x.c_cnt : x.kind == 2 ? x.l1 + 1 : 1; };
    std::stable_sort(cols.begin(), cols.end(), [&](const AceCol& x, const AceCol& y) {
        return cost(x) != cost(y) ? cost(x) > cost(y) : x.c_off < y.c_off;
    });
    const int nmax = std::max(ap->nmax1, std::max(ap->nmax2, ap->nmax3));
    const int lmax = std::max(ap->lmax2, ap->lmax3);
    const int nlm = (lmax + 1) * (lmax + 2) / 2;
    const int na = sd.g.n_atoms;
    // N_lm for every compiled (l, m >= 0): the kernel evaluates Y up to kAceLMax
    std::vector<double> yn(kAceLM);
    for (int l = 0; l <= kAceLMax; ++l)
        for (int m = 0; m <= l; ++m) {
            double r = 1.0;  // (l - m)! / (l + m)!
            for (int k = l - m + 1; k <= l + m; ++k) r /= (double)k;
            yn[l * (l + 1) / 2 + m] = std::sqrt((2.0 * l + 1.0) / (4.0 * 3.14159265358979323846) * r);
        }
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const size_t b_cols = al(sizeof(AceCol) * std::max<size_t>(cols.size(), 1));
    const size_t b_coef = al(sizeof(AceCoef) * std::max<size_t>(coefs.size(), 1));
    const size_t b_sp = al(sizeof(int) * std::max(na, 1));
    MALA_TRY(c->ws_ace.reserve(c, b_cols + b_coef + b_sp));
    char* base = c->ws_ace.as<char>();
    AceCol* d_cols = reinterpret_cast<AceCol*>(base);
    AceCoef* d_coef = reinterpret_cast<AceCoef*>(base + b_cols);
    int* d_sp = reinterpret_cast<int*>(base + b_cols + b_coef);
    // the tables are host vectors of this call: copy synchronously before they go out of scope
    if (!cols.empty()) MALA_CUDA_TRY(cudaMemcpyAsync(d_cols, cols.data(), sizeof(AceCol) * cols.size(), cudaMemcpyHostToDevice, st));
    if (!coefs.empty()) MALA_CUDA_TRY(cudaMemcpyAsync(d_coef, coefs.data(), sizeof(AceCoef) * coefs.size(), cudaMemcpyHostToDevice, st));
    std::vector<float> ynf(yn.begin(), yn.end());
    MALA_CUDA_TRY(cudaMemcpyToSymbolAsync(c_ace_ynorm, yn.data(), sizeof(double) * kAceLM, 0, cudaMemcpyHostToDevice, st));
    MALA_CUDA_TRY(cudaMemcpyToSymbolAsync(c_ace_ynormf, ynf.data(), sizeof(float) * kAceLM, 0, cudaMemcpyHostToDevice, st));
    if (na > 0 && snap->species)
        MALA_CUDA_TRY(cudaMemcpyAsync(d_sp, snap->species, sizeof(int) * na, cudaMemcpyHostToDevice, st));
    AceArgs g;
    g.P = sd.g.P;
    g.cap = nl.dbg_cap;
    g.cnt = nl.dbg_counts;
    g.atoms = nl.dbg_atoms;
    g.shifts = nl.dbg_shifts;
    g.species = snap->species ? d_sp : nullptr;
    g.wpos = sd.wpos;
    g.gcoord = sd.gcoord;
    g.n_atoms = na;
    for (int k = 0; k < 3; ++k) {
        g.grid[k] = sd.g.grid[k];
        g.L[k] = sd.g.L[k];
    }
    g.rcut = ap->rcut;
    g.lmax = lmax;
    g.nmax = nmax;
    g.n_species = ap->n_species;
    g.n_lm = nlm;
    g.n_lmf = (lmax + 1) * (lmax + 1);
    g.nA = ap->n_species * nmax * g.n_lmf;
    g.n_desc = nd;
    g.cols = d_cols;
    g.coefs = d_coef;
    g.n_coef = (int)coefs.size();
    g.stage = ace_table_bytes(nd, g.n_coef) <= (size_t)96 * 1024 ? 1 : 0;
    if (g.P > 0 && nd > 0) {
        const int64_t want = (g.P + kAceWarps - 1) / kAceWarps;
        const int sms = std::max(1, c->num_sms);
        const size_t tb = g.stage ? ace_table_bytes(nd, g.n_coef) : 0;
        if (prec == MALA_MIXED) {
            const size_t smem = tb + sizeof(float2) * (size_t)g.nA * kAceWarps;
            MALA_PROF(c, "k_ace", st, (launch_ace<float>(lmax, want, sms, smem, g, static_cast<float*>(out), st)));
        } else {
            const size_t smem = tb + sizeof(double2) * (size_t)g.nA * kAceWarps;
            MALA_PROF(c, "k_ace", st, (launch_ace<double>(lmax, want, sms, smem, g, static_cast<double*>(out), st)));
        }
        MALA_CUDA_TRY(cudaGetLastError());
    }
    MALA_CUDA_TRY(cudaStreamSynchronize(st));
    return MALA_OK;
}

}  // namespace mala
