// snap_force.cu -- adjoint of the bispectrum descriptors: the third factor of
// the force chain of Eq. forcesmala applied to a vector,
//     F_alpha = - sum_r sum_j beta(r, j) dB(r, j) / dR_alpha,
// with beta = dE/dB from the network's backward pass.
//
// Y step (k_yi).  B_{j1 j2 j} = sum_{m m'} Re(conj(u^j_{m m'}) Z^j_{j1 j2; m m'}) with
// Z^c_{ab} = sum C^{c m}_{a m1 b m-m1} C^{c m'}_{a m1' b m'-m1'} u^a_{m1 m1'} u^b_{m-m1, m'-m1'}.
// The Clebsch-Gordan symmetries that exchange the coupled and a coupling
// angular momentum (they move the complex conjugate from u^j to u^{j1} at the
// cost of the factor (j+1)/(j1+1)) give, for E = sum_t beta_t B_t,
//     dE = Re sum_J sum_{m m'} conj(du^J_{m m'}) Y^J_{m m'},
//     Y^J = sum_t beta_t ( [J = j] Z^j_{j1 j2} + [J = j1] (j+1)/(j1+1) Z^{j1}_{j j2}
//                         + [J = j2] (j+1)/(j2+1) Z^{j2}_{j j1} ),
// and Z^c_{ab} = Z^c_{ba}.  Y keeps u's symmetry Y[J-ma][J-mb] = (-1)^(ma-mb) conj(Y[ma][mb]),
// so the half set is contracted and the rest mirrored.  FP32: units with the
// couplings compiled in (snap_yi.cu).  FP64 (k_yi here): one CTA holds the full
// u of 16 grid points in shared memory, lane = point; a warp walks a list of Y
// elements, each a list of couplings, each a list of (C C, u^a index, u^b
// index) terms built on the host.  Output per point:
// y_{J,mb}[ma] = conj(Y^J[ma][mb]) N(J, ma, mb) over the full set, the form
// the force step contracts with.
//
// Force step (k_force).  u^J = w_self I + sum_k c_k U^J(a_k, b_k), c = w f_c(r).
// Column mb of U^J is N(J, ., mb) times the coefficients (by power of eta) of
// alpha^(J-mb) beta^mb, alpha = conj(a) xi - conj(b) eta, beta = b xi + a eta.
// Its derivative with respect to a real Cayley-Klein parameter q is
//     (J-mb) alpha^(J-mb-1) beta^mb dalpha/dq + mb alpha^(J-mb) beta^(mb-1) dbeta/dq,
// level-(J-1) columns times linear forms, so a single walk down each column
// chain yields G_0 = Re sum conj(Y) U and G_q = Re sum conj(Y) dU/dq for
// q = Re a, Im a, Re b, Im b with a few dot products per level.  The chain rule
// through a(d), b(d) and c(|d|) gives dE/dd for the offset d = R_alpha + s L - r.
// One warp per grid point, lane = neighbour; per-atom sums in 2^-40 fixed
// point (int64 atomics: independent of the order), in shared memory when the
// atoms fit, flushed once per CTA.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "mala_internal.h"
#include "snap_common.cuh"

namespace mala {

namespace {

constexpr int kYiWarps = 32;  // one CTA per SM shares the staged u; the warps hide load latency
constexpr int kForceWarps = 8;
constexpr double kFixScale = 1099511627776.0;  // 2^40
constexpr double kFixMax = 4194304.0;          // |contribution| < 2^22 eV/A

template <class T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };

template <class T> struct YTerm {
    T c;
    unsigned short ia, ib;
};

// N(J, ma, mb) = sqrt((J-ma)! ma! / ((J-mb)! mb!)), [J][ma][mb]
__constant__ double c_fnorm_d[(kTJMax + 1) * (kTJMax + 1) * (kTJMax + 1)];
__device__ __forceinline__ double fnorm(int J, int ma, int mb) {
    return c_fnorm_d[(J * (kTJMax + 1) + ma) * (kTJMax + 1) + mb];
}

struct YiTab {
    int ncoup, list_len;
    const int* cpl_off;     // [ncoup + 1] into ent
    const int* ent_t;       // triple of each (coupling, role) entry
    const double* ent_f;    // its factor
    const int* grp_off;     // [nh + 1] groups of each half element
    const int* grp_cpl;     // coupling of each group
    const int* term_off;    // [ngrp + 1]
    const YTerm<double>* terms_d;
    const int4* elem;       // half element: J, ma, mb, full index
    const short* warp_list; // [kYiWarps][list_len], -1 padded
};


template <class T> constexpr int yi_points() { return 16; }  // FP64 only

template <class T>
__global__ void __launch_bounds__(kYiWarps * 32) k_yi(int tj, const T* __restrict__ u_full, const T* __restrict__ beta,
                                                      int nB, int64_t P, YiTab tab, T* __restrict__ y_out) {
    using C = typename Cx<T>::type;
    constexpr int NP = yi_points<T>();
    extern __shared__ __align__(16) unsigned char smem_yi[];
    const int nf = n_full(tj);
    C* us = reinterpret_cast<C*>(smem_yi);            // [nf][NP]
    T* be = reinterpret_cast<T*>(us + (size_t)nf * NP);  // [ncoup][NP]
    const int64_t p0 = (int64_t)blockIdx.x * NP;
    for (int idx = threadIdx.x; idx < nf * NP; idx += blockDim.x) {
        const int pt = idx / nf, e = idx - pt * nf;
        const int64_t p = p0 + pt;
        C v;
        v.x = T(0);
        v.y = T(0);
        if (p < P) {
            v.x = u_full[((size_t)p * nf + e) * 2];
            v.y = u_full[((size_t)p * nf + e) * 2 + 1];
        }
        us[e * NP + pt] = v;
    }
    for (int idx = threadIdx.x; idx < tab.ncoup * NP; idx += blockDim.x) {
        const int k = idx / NP, pt = idx - k * NP;
        const int64_t p = p0 + pt;
        T s = T(0);
        if (p < P)
            for (int q = tab.cpl_off[k]; q < tab.cpl_off[k + 1]; ++q)
                s += (T)tab.ent_f[q] * beta[(size_t)p * nB + tab.ent_t[q]];
        be[k * NP + pt] = s;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pt = lane % NP, sub = lane / NP;
    const int64_t p = p0 + pt;
    const short* wl = tab.warp_list + (size_t)warp * tab.list_len;
    const YTerm<T>* terms = tab.terms_d;
    for (int i = sub; i < tab.list_len; i += 32 / NP) {
        const int h = wl[i];
        if (h < 0) break;
        T yr = T(0), yi = T(0);
        for (int g = tab.grp_off[h]; g < tab.grp_off[h + 1]; ++g) {
            // two independent accumulators, four terms in flight
            T zr0 = T(0), zi0 = T(0), zr1 = T(0), zi1 = T(0);
            int q = tab.term_off[g];
            const int q1 = tab.term_off[g + 1];
            for (; q + 4 <= q1; q += 4) {
                const YTerm<T> t0 = terms[q], t1 = terms[q + 1], t2 = terms[q + 2], t3 = terms[q + 3];
                const C x0 = us[t0.ia * NP + pt], y0 = us[t0.ib * NP + pt];
                const C x1 = us[t1.ia * NP + pt], y1 = us[t1.ib * NP + pt];
                const C x2 = us[t2.ia * NP + pt], y2 = us[t2.ib * NP + pt];
                const C x3 = us[t3.ia * NP + pt], y3 = us[t3.ib * NP + pt];
                zr0 += t0.c * (x0.x * y0.x - x0.y * y0.y);
                zi0 += t0.c * (x0.x * y0.y + x0.y * y0.x);
                zr1 += t1.c * (x1.x * y1.x - x1.y * y1.y);
                zi1 += t1.c * (x1.x * y1.y + x1.y * y1.x);
                zr0 += t2.c * (x2.x * y2.x - x2.y * y2.y);
                zi0 += t2.c * (x2.x * y2.y + x2.y * y2.x);
                zr1 += t3.c * (x3.x * y3.x - x3.y * y3.y);
                zi1 += t3.c * (x3.x * y3.y + x3.y * y3.x);
            }
            for (; q < q1; ++q) {
                const YTerm<T> tm = terms[q];
                const C x = us[tm.ia * NP + pt], y = us[tm.ib * NP + pt];
                zr0 += tm.c * (x.x * y.x - x.y * y.y);
                zi0 += tm.c * (x.x * y.y + x.y * y.x);
            }
            const T b = be[tab.grp_cpl[g] * NP + pt];
            yr += b * (zr0 + zr1);
            yi += b * (zi0 + zi1);
        }
        if (p < P) {
            const int4 el = tab.elem[h];
            const int J = el.x, ma = el.y, mb = el.z;
            const T nrm = fnorm(J, ma, mb);  // N is the same at the mirrored element
            T* o = y_out + (size_t)p * nf * 2;
            o[2 * el.w] = yr * nrm;  // conj(Y) N
            o[2 * el.w + 1] = -yi * nrm;
            if (2 * ma != J || 2 * mb != J) {
                const int em = full_off(J) + (J - ma) * (J + 1) + (J - mb);
                const T sg = ((ma - mb) & 1) ? T(-1) : T(1);  // Y_mirror = sg conj(Y)
                o[2 * em] = sg * yr * nrm;
                o[2 * em + 1] = sg * yi * nrm;
            }
        }
    }
}

struct ForceGeom {
    const double* wpos;    // [3][n_atoms] wrapped positions
    const double* gcoord;  // grid coordinates [g0] | [g1] | [g2]
    const double* watom;   // element weight per atom
    int n_atoms;
    int grid[3];
    double L[3];
};

__device__ __forceinline__ long long to_fix(double x, int* err) {
    if (!(fabs(x) < kFixMax)) {
        atomicExch(err, 1);
        return 0;
    }
    return llrint(x * kFixScale);
}

// v <- (l0 xi + l1 eta) v for a coefficient vector of length n (indices 0..n-1) -> n + 1
template <class T, int N>
__device__ __forceinline__ void lin_mul(T (&vr)[N], T (&vi)[N], int n, T l0r, T l0i, T l1r, T l1i) {
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        if (i <= n) {
            T nr = T(0), ni = T(0);
            if (i < n) {
                nr = l0r * vr[i] - l0i * vi[i];
                ni = l0r * vi[i] + l0i * vr[i];
            }
            if (i > 0) {
                nr += l1r * vr[i - 1] - l1i * vi[i - 1];
                ni += l1r * vi[i - 1] + l1i * vr[i - 1];
            }
            vr[i] = nr;
            vi[i] = ni;
        }
    }
}

// The chain walk of k_force, one level at a time: level J of column chain cc
// (the chain index at run time, the level's code compiled once per J), so
// the code a neighbour runs is the eleven level bodies rather than all 66
// (chain, level) pairs unrolled, and stays in the instruction cache.
template <class T> struct GSums {
    T G0, Gar, Gai, Gbr, Gbi;
};

template <class T, int TJ, int J>
__device__ __forceinline__ void force_level(const typename Cx<T>::type* __restrict__ ys, int cc, T (&pr)[TJ + 1],
                                            T (&pim)[TJ + 1], T al0r, T al0i, T al1r, T al1i, GSums<T>& gs) {
    using C = typename Cx<T>::type;
    constexpr int o = full_off(J);
    T s0 = T(0);
#pragma unroll
    for (int k2 = 0; k2 <= J; ++k2) {
        const C yv = ys[o + k2 * (J + 1) + cc];
        s0 += yv.x * pr[k2] - yv.y * pim[k2];
    }
    gs.G0 += s0;
    if constexpr (J < TJ) {
        constexpr int o1 = full_off(J + 1);
        T a0r = T(0), a0i = T(0), a1r = T(0), a1i = T(0), b0r = T(0), b0i = T(0), b1r = T(0), b1i = T(0);
#pragma unroll
        for (int k2 = 0; k2 <= J; ++k2) {
            const C ya0 = ys[o1 + k2 * (J + 2) + cc];
            const C ya1 = ys[o1 + (k2 + 1) * (J + 2) + cc];
            const C yb0 = ys[o1 + k2 * (J + 2) + cc + 1];
            const C yb1 = ys[o1 + (k2 + 1) * (J + 2) + cc + 1];
            const T xr = pr[k2], xi = pim[k2];
            a0r += ya0.x * xr - ya0.y * xi;
            a0i += ya0.x * xi + ya0.y * xr;
            a1r += ya1.x * xr - ya1.y * xi;
            a1i += ya1.x * xi + ya1.y * xr;
            b0r += yb0.x * xr - yb0.y * xi;
            b0i += yb0.x * xi + yb0.y * xr;
            b1r += yb1.x * xr - yb1.y * xi;
            b1i += yb1.x * xi + yb1.y * xr;
        }
        const T fa = T(J + 1 - cc), fb = T(cc + 1);
        gs.Gar += fa * a0r + fb * b1r;
        gs.Gai += fa * a0i - fb * b1i;
        gs.Gbr += -fa * a1r + fb * b0r;
        gs.Gbi += -fa * a1i - fb * b0i;
        lin_mul<T, TJ + 1>(pr, pim, J + 1, al0r, al0i, al1r, al1i);  // level J: J + 1 coefficients
    }
}

template <class T, int TJ, int LO, int HI>
__device__ __forceinline__ void force_level_at(int J, const typename Cx<T>::type* ys, int cc, T (&pr)[TJ + 1],
                                               T (&pim)[TJ + 1], T al0r, T al0i, T al1r, T al1i, GSums<T>& gs) {
    if constexpr (HI - LO == 1) {
        force_level<T, TJ, LO>(ys, cc, pr, pim, al0r, al0i, al1r, al1i, gs);
    } else {
        constexpr int MID = (LO + HI) / 2;
        if (J < MID) force_level_at<T, TJ, LO, MID>(J, ys, cc, pr, pim, al0r, al0i, al1r, al1i, gs);
        else force_level_at<T, TJ, MID, HI>(J, ys, cc, pr, pim, al0r, al0i, al1r, al1i, gs);
    }
}

// beta^cc from beta^(cc-1) (cc coefficients -> cc + 1), cc >= 1 at run time
template <class T, int TJ, int LO, int HI>
__device__ __forceinline__ void beta_step_at(int cc, T (&dr)[TJ + 1], T (&di)[TJ + 1], T be0r, T be0i, T be1r,
                                             T be1i) {
    if constexpr (HI - LO == 1) {
        lin_mul<T, TJ + 1>(dr, di, LO, be0r, be0i, be1r, be1i);
    } else {
        constexpr int MID = (LO + HI) / 2;
        if (cc < MID) beta_step_at<T, TJ, LO, MID>(cc, dr, di, be0r, be0i, be1r, be1i);
        else beta_step_at<T, TJ, MID, HI>(cc, dr, di, be0r, be0i, be1r, be1i);
    }
}

template <class T, int TJ>
__global__ void __launch_bounds__(kForceWarps * 32) k_force(const T* __restrict__ y_all, int64_t P, int cap,
                                                            const int* __restrict__ cnt, const int* __restrict__ atoms,
                                                            const int* __restrict__ shifts, ForceGeom g, T rcut,
                                                            T rfac0, T rmin0, int smem_atoms,
                                                            unsigned long long* __restrict__ F_fix, int* err) {
    using C = typename Cx<T>::type;
    constexpr int NF = n_full(TJ);
    extern __shared__ __align__(16) unsigned char smem_f[];
    C* ysm = reinterpret_cast<C*>(smem_f);  // [warps][NF]
    unsigned long long* sF = reinterpret_cast<unsigned long long*>(ysm + (size_t)kForceWarps * NF);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (smem_atoms) {
        for (int i = threadIdx.x; i < 3 * g.n_atoms; i += blockDim.x) sF[i] = 0ull;
        __syncthreads();
    }
    unsigned long long* acc = smem_atoms ? sF : F_fix;
    C* ys = ysm + (size_t)warp * NF;
    const T pi = T(3.14159265358979323846);
    const T K = pi / (rcut - rmin0);
    for (int64_t p = (int64_t)blockIdx.x * kForceWarps + warp; p < P; p += (int64_t)gridDim.x * kForceWarps) {
        const C* yp = reinterpret_cast<const C*>(y_all) + (size_t)p * NF;
        for (int e = lane; e < NF; e += 32) ys[e] = yp[e];
        __syncwarp();
        int n = cnt[p];
        if (n > cap) {
            if (lane == 0) atomicExch(err, 2);
            n = cap;
        }
        const int ix = (int)(p % g.grid[0]);
        const int iy = (int)((p / g.grid[0]) % g.grid[1]);
        const int iz = (int)(p / ((int64_t)g.grid[0] * g.grid[1]));
        const double rx = g.gcoord[ix], ry = g.gcoord[g.grid[0] + iy], rz = g.gcoord[g.grid[0] + g.grid[1] + iz];
        for (int k = lane; k < n; k += 32) {
            const size_t q = (size_t)p * cap + k;
            const int a = atoms[q];
            const double sx = shifts[3 * q], sy = shifts[3 * q + 1], sz = shifts[3 * q + 2];
            const T dx = (T)((g.wpos[a] + sx * g.L[0]) - rx);
            const T dy = (T)((g.wpos[g.n_atoms + a] + sy * g.L[1]) - ry);
            const T dz = (T)((g.wpos[2 * g.n_atoms + a] + sz * g.L[2]) - rz);
            const T r = sqrt(dx * dx + dy * dy + dz * dz);
            if (!(r > T(1e-6))) continue;  // an atom on the grid point: no direction
            const T w = (T)g.watom[a];
            const T t = (r - rmin0) / (rcut - rmin0);
            T sp, cp, so, co;
            if constexpr (sizeof(T) == 4) {
                sincospif((float)t, &sp, &cp);
                sincosf((float)(rfac0 * pi * t), &so, &co);
            } else {
                sincospi((double)t, &sp, &cp);
                sincos((double)(rfac0 * pi * t), &so, &co);
            }
            const T fc = T(0.5) * (cp + T(1));
            const T dfc = -T(0.5) * K * sp;  // d fc / dr
            const T c = w * fc;
            const T s = so / r;
            const T ar = co, ai = -dz * s, br = dy * s, bi = -dx * s;
            // linear forms: alpha = (ar - i ai) xi + (-br + i bi) eta, beta = (br + i bi) xi + (ar + i ai) eta
            const T al0r = ar, al0i = -ai, al1r = -br, al1i = bi;
            const T be0r = br, be0i = bi, be1r = ar, be1i = ai;
            GSums<T> gs{T(0), T(0), T(0), T(0), T(0)};
            T dr_[TJ + 1], di_[TJ + 1];
#pragma unroll
            for (int i = 0; i <= TJ; ++i) {
                dr_[i] = T(0);
                di_[i] = T(0);
            }
            dr_[0] = T(1);
            for (int cc = 0; cc <= TJ; ++cc) {
                // beta^(cc-1) has cc coefficients
                if (cc > 0) beta_step_at<T, TJ, 1, TJ + 1>(cc, dr_, di_, be0r, be0i, be1r, be1i);
                T pr[TJ + 1], pim[TJ + 1];
#pragma unroll
                for (int i = 0; i <= TJ; ++i) {
                    pr[i] = dr_[i];
                    pim[i] = di_[i];
                }
                for (int J = cc; J <= TJ; ++J)
                    force_level_at<T, TJ, 0, TJ + 1>(J, ys, cc, pr, pim, al0r, al0i, al1r, al1i, gs);
            }
            const T G0 = gs.G0, Gar = gs.Gar, Gai = gs.Gai, Gbr = gs.Gbr, Gbi = gs.Gbi;
            // chain rule to the offset d
            const T ir = T(1) / r;
            const T dsdr = (co * rfac0 * K * r - so) * ir * ir;
            const T radial = G0 * w * dfc - c * Gar * so * rfac0 * K + c * dsdr * (-Gai * dz + Gbr * dy - Gbi * dx);
            const T gx = dx * ir * radial - c * s * Gbi;
            const T gy = dy * ir * radial + c * s * Gbr;
            const T gz = dz * ir * radial - c * s * Gai;
            // F_alpha -= dE/dd
            atomicAdd(acc + 3 * a, (unsigned long long)to_fix(-(double)gx, err));
            atomicAdd(acc + 3 * a + 1, (unsigned long long)to_fix(-(double)gy, err));
            atomicAdd(acc + 3 * a + 2, (unsigned long long)to_fix(-(double)gz, err));
        }
        __syncwarp();
    }
    if (smem_atoms) {
        __syncthreads();
        for (int i = threadIdx.x; i < 3 * g.n_atoms; i += blockDim.x)
            if (sF[i]) atomicAdd(F_fix + i, sF[i]);
    }
}

__global__ void k_fix_to_double(const unsigned long long* __restrict__ F_fix, int n, double* __restrict__ F) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) F[i] = (double)(long long)F_fix[i] * (1.0 / kFixScale);
}

// ---- host: Y tables ------------------------------------------------------------

struct HostYiTab {
    std::vector<int> cpl_off, ent_t, grp_off, grp_cpl, term_off;
    std::vector<double> ent_f;
    std::vector<YTerm<double>> td;
    std::vector<int4> elem;
    std::vector<short> wl;
    int ncoup = 0, list_len = 0;
};

void build_yi_tab(int tj, HostYiTab& H) {
    // couplings (c; a >= b) with their (triple, factor) entries
    std::vector<int3> cpl;
    std::vector<std::vector<std::pair<int, double>>> ents;
    auto coupling = [&](int cc, int a, int b) {
        if (a < b) std::swap(a, b);
        for (size_t i = 0; i < cpl.size(); ++i)
            if (cpl[i].x == cc && cpl[i].y == a && cpl[i].z == b) return (int)i;
        cpl.push_back(make_int3(cc, a, b));
        ents.emplace_back();
        return (int)cpl.size() - 1;
    };
    int t = 0;
    for (int j1 = 0; j1 <= tj; ++j1)
        for (int j2 = 0; j2 <= j1; ++j2)
            for (int j = 0; j <= tj; ++j) {
                if (!triple_ok(j1, j2, j, tj)) continue;
                ents[coupling(j, j1, j2)].push_back({t, 1.0});
                ents[coupling(j1, j, j2)].push_back({t, (j + 1.0) / (j1 + 1.0)});
                ents[coupling(j2, j, j1)].push_back({t, (j + 1.0) / (j2 + 1.0)});
                ++t;
            }
    H.ncoup = (int)cpl.size();
    H.cpl_off.assign(1, 0);
    for (auto& v : ents) {
        for (auto& e : v) {
            H.ent_t.push_back(e.first);
            H.ent_f.push_back(e.second);
        }
        H.cpl_off.push_back((int)H.ent_t.size());
    }
    // half elements of Y with their coupling groups and terms
    H.grp_off.assign(1, 0);
    H.term_off.assign(1, 0);
    std::vector<double> cost;
    for (int J = 0; J <= tj; ++J)
        for (int ma = 0; 2 * ma <= J; ++ma)
            for (int mb = 0; mb <= J; ++mb) {
                if (2 * ma == J && 2 * mb > J) continue;
                const int m = 2 * ma - J, mp = 2 * mb - J;
                double cst = 0.0;
                for (int k = 0; k < H.ncoup; ++k) {
                    if (cpl[k].x != J) continue;
                    const int a = cpl[k].y, b = cpl[k].z;
                    const size_t before = H.td.size();
                    for (int m1a = 0; m1a <= a; ++m1a) {
                        const int m1 = 2 * m1a - a, m2 = m - m1;
                        if (m2 < -b || m2 > b) continue;
                        const double c1 = clebsch_gordan(a, m1, b, m2, J, m);
                        if (c1 == 0.0) continue;
                        for (int m1b = 0; m1b <= a; ++m1b) {
                            const int m1p = 2 * m1b - a, m2p = mp - m1p;
                            if (m2p < -b || m2p > b) continue;
                            const double c2 = clebsch_gordan(a, m1p, b, m2p, J, mp);
                            if (c2 == 0.0) continue;
                            const int ia = full_off(a) + m1a * (a + 1) + m1b;
                            const int ib = full_off(b) + ((m2 + b) / 2) * (b + 1) + (m2p + b) / 2;
                            H.td.push_back(YTerm<double>{c1 * c2, (unsigned short)ia, (unsigned short)ib});
                        }
                    }
                    if (H.td.size() == before) continue;
                    H.grp_cpl.push_back(k);
                    H.term_off.push_back((int)H.td.size());
                    cst += 2.0 + (double)(H.td.size() - before);
                }
                H.grp_off.push_back((int)H.grp_cpl.size());
                H.elem.push_back(make_int4(J, ma, mb, full_off(J) + ma * (J + 1) + mb));
                cost.push_back(cst + 4.0);
            }
    // longest-first assignment of elements to the warps
    const int nh = (int)H.elem.size();
    std::vector<int> order(nh);
    for (int i = 0; i < nh; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<std::vector<int>> lists(kYiWarps);
    std::vector<double> load(kYiWarps, 0.0);
    for (int h : order) {
        const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lists[w].push_back(h);
        load[w] += cost[h];
    }
    size_t len = 0;
    for (auto& l : lists) len = std::max(len, l.size());
    H.list_len = (int)len;
    H.wl.assign((size_t)kYiWarps * len, (short)-1);
    for (int w = 0; w < kYiWarps; ++w)
        for (size_t i = 0; i < lists[w].size(); ++i) H.wl[(size_t)w * len + i] = (short)lists[w][i];
}

int ensure_yi_tab(Ctx* c, int tj, YiTab* out) {
    ForceTables& F = c->ftab;
    if (F.tj != tj) {
        HostYiTab H;
        build_yi_tab(tj, H);
        // one device buffer: pieces at 256-byte aligned offsets
        std::vector<std::pair<const void*, size_t>> parts = {
            {H.cpl_off.data(), H.cpl_off.size() * sizeof(int)}, {H.ent_t.data(), H.ent_t.size() * sizeof(int)},
            {H.ent_f.data(), H.ent_f.size() * sizeof(double)},  {H.grp_off.data(), H.grp_off.size() * sizeof(int)},
            {H.grp_cpl.data(), H.grp_cpl.size() * sizeof(int)}, {H.term_off.data(), H.term_off.size() * sizeof(int)},
            {H.td.data(), H.td.size() * sizeof(YTerm<double>)}, {H.elem.data(), H.elem.size() * sizeof(int4)},
            {H.wl.data(), H.wl.size() * sizeof(short)}};
        std::vector<size_t> off;
        size_t total = 0;
        for (auto& p : parts) {
            off.push_back(total);
            total += (p.second + 255) & ~size_t(255);
        }
        std::vector<unsigned char> blob(total, 0);
        for (size_t i = 0; i < parts.size(); ++i)
            if (parts[i].second) memcpy(blob.data() + off[i], parts[i].first, parts[i].second);
        MALA_TRY(c->ws_ftab.reserve(c, total + 256));
        MALA_CUDA_TRY(cudaMemcpy(c->ws_ftab.ptr, blob.data(), total, cudaMemcpyHostToDevice));
        for (int i = 0; i < 9; ++i) F.off[i] = off[i];
        F.ncoup = H.ncoup;
        F.list_len = H.list_len;
        F.nh = (int)H.elem.size();
        F.tj = tj;
    }
    const char* b = c->ws_ftab.as<const char>();
    out->ncoup = F.ncoup;
    out->list_len = F.list_len;
    out->cpl_off = reinterpret_cast<const int*>(b + F.off[0]);
    out->ent_t = reinterpret_cast<const int*>(b + F.off[1]);
    out->ent_f = reinterpret_cast<const double*>(b + F.off[2]);
    out->grp_off = reinterpret_cast<const int*>(b + F.off[3]);
    out->grp_cpl = reinterpret_cast<const int*>(b + F.off[4]);
    out->term_off = reinterpret_cast<const int*>(b + F.off[5]);
    out->terms_d = reinterpret_cast<const YTerm<double>*>(b + F.off[6]);
    out->elem = reinterpret_cast<const int4*>(b + F.off[7]);
    out->warp_list = reinterpret_cast<const short*>(b + F.off[8]);
    return MALA_OK;
}

bool g_fnorm_ready[64] = {false};

int ensure_fnorm(int device) {
    if (device >= 0 && device < 64 && g_fnorm_ready[device]) return MALA_OK;
    constexpr int n = (kTJMax + 1) * (kTJMax + 1) * (kTJMax + 1);
    std::vector<double> d(n, 0.0);
    for (int J = 0; J <= kTJMax; ++J)
        for (int a = 0; a <= J; ++a)
            for (int b = 0; b <= J; ++b) {
                const double v = std::sqrt(fact_d(J - a) * fact_d(a) / (fact_d(J - b) * fact_d(b)));
                d[(J * (kTJMax + 1) + a) * (kTJMax + 1) + b] = v;
            }
    MALA_CUDA_TRY(cudaMemcpyToSymbol(c_fnorm_d, d.data(), sizeof(double) * n));
    if (device >= 0 && device < 64) g_fnorm_ready[device] = true;
    return MALA_OK;
}

template <class T, int TJ>
void launch_force_tj(const T* y, int64_t P, int cap, const int* cnt, const int* atoms, const int* shifts,
                     const ForceGeom& g, const mala_bispectrum_params* bp, int smem_atoms, size_t smem, int grid,
                     unsigned long long* F_fix, int* err, cudaStream_t st) {
    cudaFuncSetAttribute(k_force<T, TJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_force<T, TJ><<<grid, kForceWarps * 32, smem, st>>>(y, P, cap, cnt, atoms, shifts, g, (T)bp->rcut,
                                                          (T)bp->rfac0, (T)bp->rmin0, smem_atoms, F_fix, err);
}

}  // namespace

// F (host, [n_atoms][3]) = -sum_r sum_j beta[r][j] dB(r, j)/dR from the full u
// and the neighbour lists of one staged snapshot.  Precision: T = float or double.
template <class T>
int descriptor_adjoint(Ctx* c, const SnapDev& sd, const mala_snapshot* snap, const mala_bispectrum_params* bp,
                       const T* u_full, const T* beta, const NbrOut& nl, double* F_host, cudaStream_t st) {
    const int tj = bp->twojmax;
    const int64_t P = sd.g.P;
    const int nf = n_full(tj), nB = n_triples(tj), na = sd.g.n_atoms;
    MALA_TRY(ensure_fnorm(c->device));
    // Y, then per-atom weights, fixed-point sums, error flag
    MALA_TRY(c->ws_force_y.reserve(c, sizeof(T) * 2 * (size_t)nf * (size_t)std::max<int64_t>(P, 1)));
    const size_t aux = sizeof(double) * na + sizeof(unsigned long long) * 3 * (size_t)na + sizeof(double) * 3 * na + 512;
    MALA_TRY(c->ws_force_aux.reserve(c, aux));
    T* y = c->ws_force_y.as<T>();
    double* watom = c->ws_force_aux.as<double>();
    unsigned long long* F_fix = reinterpret_cast<unsigned long long*>(watom + na);
    double* F_dev = reinterpret_cast<double*>(F_fix + 3 * (size_t)na);
    int* err = reinterpret_cast<int*>(F_dev + 3 * (size_t)na);
    (void)snap;
    if (na > 0) MALA_CUDA_TRY(cudaMemsetAsync(F_fix, 0, sizeof(unsigned long long) * 3 * na, st));
    MALA_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
    if (P > 0) {
        if constexpr (sizeof(T) == 4) {
            // FP32: units with compiled couplings, two points per lane (snap_yi.cu)
            MALA_TRY(yi_units(c, tj, u_full, beta, nB, P, y, st));
        } else {
            YiTab tab;
            MALA_TRY(ensure_yi_tab(c, tj, &tab));
            constexpr int NP = yi_points<T>();
            const size_t smem_yi =
                sizeof(typename Cx<T>::type) * (size_t)nf * NP + sizeof(T) * (size_t)tab.ncoup * NP;
            cudaFuncSetAttribute(k_yi<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_yi);
            MALA_PROF(c, "k_yi", st,
                      (k_yi<T><<<(unsigned)((P + NP - 1) / NP), kYiWarps * 32, smem_yi, st>>>(tj, u_full, beta, nB,
                                                                                              P, tab, y)));
            MALA_CUDA_TRY(cudaGetLastError());
        }
        ForceGeom g;
        g.wpos = sd.wpos;
        g.gcoord = sd.gcoord;
        g.watom = sd.wsp;  // the element weights the descriptors used
        g.n_atoms = na;
        for (int d = 0; d < 3; ++d) {
            g.grid[d] = sd.g.grid[d];
            g.L[d] = sd.g.L[d];
        }
        const size_t ybytes = sizeof(typename Cx<T>::type) * (size_t)kForceWarps * nf;
        const size_t fbytes = sizeof(unsigned long long) * 3 * (size_t)na;
        const int smem_atoms = ybytes + fbytes <= (size_t)160 * 1024 ? 1 : 0;
        const size_t smem = ybytes + (smem_atoms ? fbytes : 0);
        const int64_t want = (P + kForceWarps - 1) / kForceWarps;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)c->num_sms * 2));
        const int* cnt = nl.dbg_counts;
        const int* at = nl.dbg_atoms;
        const int* sh = nl.dbg_shifts;
        const int cap = nl.dbg_cap;
        switch (tj) {
            case 0: MALA_PROF(c, "k_force", st, (launch_force_tj<T, 0>(y, P, cap, cnt, at, sh, g, bp, smem_atoms, smem, grid, F_fix, err, st))); break;
            case 2: MALA_PROF(c, "k_force", st, (launch_force_tj<T, 2>(y, P, cap, cnt, at, sh, g, bp, smem_atoms, smem, grid, F_fix, err, st))); break;
            case 4: MALA_PROF(c, "k_force", st, (launch_force_tj<T, 4>(y, P, cap, cnt, at, sh, g, bp, smem_atoms, smem, grid, F_fix, err, st))); break;
            case 6: MALA_PROF(c, "k_force", st, (launch_force_tj<T, 6>(y, P, cap, cnt, at, sh, g, bp, smem_atoms, smem, grid, F_fix, err, st))); break;
            case 8: MALA_PROF(c, "k_force", st, (launch_force_tj<T, 8>(y, P, cap, cnt, at, sh, g, bp, smem_atoms, smem, grid, F_fix, err, st))); break;
            case 10: MALA_PROF(c, "k_force", st, (launch_force_tj<T, 10>(y, P, cap, cnt, at, sh, g, bp, smem_atoms, smem, grid, F_fix, err, st))); break;
            default: return fail(MALA_ERR_UNSUPPORTED, "twojmax %d has no compiled force kernel", tj);
        }
        MALA_CUDA_TRY(cudaGetLastError());
    }
    if (na > 0) k_fix_to_double<<<(3 * na + 255) / 256, 256, 0, st>>>(F_fix, 3 * na, F_dev);
    MALA_CUDA_TRY(cudaGetLastError());
    MALA_CUDA_TRY(cudaMemcpyAsync(c->host_ints + 4, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (na > 0) MALA_CUDA_TRY(cudaMemcpyAsync(F_host, F_dev, sizeof(double) * 3 * na, cudaMemcpyDeviceToHost, st));
    MALA_CUDA_TRY(cudaStreamSynchronize(st));
    if (c->host_ints[4] == 2) return fail(MALA_ERR_UNSUPPORTED, "neighbour list capacity exceeded in the force step");
    if (c->host_ints[4]) return fail(MALA_ERR_UNSUPPORTED, "a force contribution exceeded the fixed-point range (4e6 eV/A)");
    return MALA_OK;
}

template int descriptor_adjoint<float>(Ctx*, const SnapDev&, const mala_snapshot*, const mala_bispectrum_params*,
                                       const float*, const float*, const NbrOut&, double*, cudaStream_t);
template int descriptor_adjoint<double>(Ctx*, const SnapDev&, const mala_snapshot*, const mala_bispectrum_params*,
                                        const double*, const double*, const NbrOut&, double*, cudaStream_t);

}  // namespace mala
