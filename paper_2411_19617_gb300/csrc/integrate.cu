// integrate.cu -- the LDOS integrals of paper Sec. "Observable calculation":
//   D(e_xi)  = dV sum_r LDOS(r, xi)                       (Eq. DOS.from.ldos)
//   N(mu)    = sum_xi w0_xi(mu) D_xi                      (Eq. NumberElectrons_from_DOS)
//   e_F      : root of N(mu) - N_e by FP64 bisection, run "wide": each round
//              evaluates, on one SM each, the 127 midpoints that the next 7
//              bisection steps could visit, then every block replays the 7
//              decisions, so the iterates are those of plain bisection
//   E_b      = sum_xi w1_xi(e_F) D_xi                      (Eq. band.energy)
//   n(r)     = sum_xi w0_xi(e_F) LDOS(r, xi)              (Eq. density.from.ldos)
//   -tau S_s = -kT sum_xi wS_xi(e_F) D_xi                  (Eqs. electronicentropyDOS, KSfreeenergy)
// with w_n,xi(mu) = int hat_xi(e) e^n f((e - mu)/kT) de the exact weights of
// the piecewise-linear interpolant between energy-grid points
// (Eqs. ldosintegralgeneral / ldosintegralsummation).
//
// Closed forms.  With f(y) = 1/(1+e^y) and, for y >= 0, L = ln(1 + e^-y),
// z = -e^-y:
//   H0(y) = -L,  H1(y) = -y L + Li2(z),  H2(y) = -y^2 L + 2 y Li2(z) + 2 Li3(z)
// are antiderivatives of f, y f, y^2 f (the polylogarithm form of f,
// Eq. fermidiracspecial).  For the entropy density s = -[f ln f + (1-f) ln(1-f)]
// = L + y f(y) (even in y):  A0(y) = 2 Li2(z) - y L and
// A1(y) = 3 y Li2(z) + 3 Li3(z) - y^2 L are antiderivatives of s and y s.  Below the Fermi level (x < 0) f(x) = 1 - f(-x) turns
// every piece into an exact polynomial integral minus an integral over y >= 0,
// so no large terms cancel.  Li2 and Li3 on z in [-1, 0) are summed from their
// Bernoulli-number expansions in u = -ln(1 - z), |u| <= ln 2:
//   Li2 = sum_k B_k u^(k+1)/(k+1)!,
//   Li3 = sum_{n,k} B_n B_k u^(n+k+1) / ((n+1)! k! (n+k+1))
// (term-by-term integrals of dLi2/du = u/(e^u - 1), dLi3/du = Li2/(e^u - 1)).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "mala_internal.h"

namespace mala {

namespace {

constexpr int kPolyTerms = 26;
__constant__ double c_li2[kPolyTerms + 1];  // coefficient of u^m, m = 0..kPolyTerms
__constant__ double c_li3[kPolyTerms + 1];

constexpr int kFermiThreads = 256;

__device__ __forceinline__ double horner(const double* c, double u) {
    double s = 0.0;
#pragma unroll
    for (int m = kPolyTerms; m >= 1; --m) s = s * u + c[m];
    return s * u;
}

// antiderivatives of y^j f(y), j = 0, 1, 2, valid for y >= 0.  Beyond y = 40
// the leading terms of L = e^-y - e^-2y/2 + ..., Li_s(-e^-y) = -e^-y + ... are
// exact to a relative e^-40 (below FP64 rounding), so the series are skipped.
__device__ __forceinline__ void hfun(double y, double& h0, double& h1, double& h2) {
    if (y > 40.0) {
        const double e = exp(-y);
        h0 = -e;
        h1 = -(y + 1.0) * e;
        h2 = -((y + 2.0) * y + 2.0) * e;
        return;
    }
    const double L = log1p(exp(-y));
    const double u = -L;
    const double li2 = horner(c_li2, u), li3 = horner(c_li3, u);
    h0 = -L;
    h1 = -y * L + li2;
    h2 = -y * y * L + 2.0 * y * li2 + 2.0 * li3;
}

// antiderivatives of s(y) and y s(y), valid for y >= 0 (leading terms beyond y = 40)
__device__ __forceinline__ void sfun(double y, double& a0, double& a1) {
    if (y > 40.0) {
        const double e = exp(-y);
        a0 = -(y + 2.0) * e;
        a1 = -((y + 3.0) * y + 3.0) * e;
        return;
    }
    const double L = log1p(exp(-y));
    const double u = -L;
    const double li2 = horner(c_li2, u), li3 = horner(c_li3, u);
    a0 = 2.0 * li2 - y * L;
    a1 = 3.0 * y * li2 + 3.0 * li3 - y * y * L;
}

// S_k = int_a^b (e - a)^k s((e - mu)/kT) de, k = 0, 1
__device__ void entropy_moments(double a, double b, double mu, double kT, double& S0, double& S1) {
    const double ikT = 1.0 / kT;
    const double xa = (a - mu) * ikT, xb = (b - mu) * ikT;
    double s0 = 0.0, s1 = 0.0;  // int (x - xa)^k s(x) dx over [xa, xb]
    const double p0 = fmax(xa, 0.0);
    if (xb > p0) {
        double a0, a1, b0, b1;
        sfun(p0, a0, a1);
        sfun(xb, b0, b1);
        s0 += b0 - a0;
        s1 += (b1 - a1) - xa * (b0 - a0);
    }
    // x < 0: s(x) = s(-x), y = -x in [-x1, -xa]; (x - xa) = -(y + xa)
    const double x1 = fmin(xb, 0.0);
    if (x1 > xa) {
        double a0, a1, b0, b1;
        sfun(-x1, a0, a1);
        sfun(-xa, b0, b1);
        s0 += b0 - a0;
        s1 -= (b1 - a1) + xa * (b0 - a0);
    }
    S0 = kT * s0;
    S1 = kT * kT * s1;
}

// M_k = int_a^b (e - a)^k f((e - mu)/kT) de, k = 0, 1, 2
__device__ void interval_moments(double a, double b, double mu, double kT, double& M0, double& M1, double& M2) {
    const double ikT = 1.0 / kT;
    const double xa = (a - mu) * ikT, xb = (b - mu) * ikT;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;  // int (x - xa)^k f(x) dx over [xa, xb]
    // part with x >= 0: direct antiderivatives, (x - xa)^k expanded in x
    const double p0 = fmax(xa, 0.0);
    if (xb > p0) {
        double a0, a1, a2, b0, b1, b2;
        hfun(p0, a0, a1, a2);
        hfun(xb, b0, b1, b2);
        const double d0 = b0 - a0, d1 = b1 - a1, d2 = b2 - a2;
        s0 += d0;
        s1 += d1 - xa * d0;
        s2 += d2 - 2.0 * xa * d1 + xa * xa * d0;
    }
    // part with x < 0: f(x) = 1 - f(-x); y = -x in [-x1, -xa]
    const double x1 = fmin(xb, 0.0);
    if (x1 > xa) {
        const double t = x1 - xa;
        s0 += t;
        s1 += t * t / 2.0;
        s2 += t * t * t * (1.0 / 3.0);
        double a0, a1, a2, b0, b1, b2;
        hfun(-x1, a0, a1, a2);
        hfun(-xa, b0, b1, b2);
        const double d0 = b0 - a0, d1 = b1 - a1, d2 = b2 - a2;
        // int (x - xa)^k f(-x) dx = int (-(y + xa))^k f(y) dy over [-x1, -xa]
        s0 -= d0;
        s1 -= -(d1 + xa * d0);
        s2 -= d2 + 2.0 * xa * d1 + xa * xa * d0;
    }
    M0 = kT * s0;
    M1 = kT * kT * s1;
    M2 = kT * kT * kT * s2;
}

__device__ double block_sum(double v, double* sred) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) sred[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sred[w];
    __syncthreads();
    if (threadIdx.x == 0) sred[32] = t;
    __syncthreads();
    return sred[32];
}

// N(mu) with D held in shared memory
__device__ double electron_count(const double* sD, int nE, double e0, double de, double mu, double kT, double* sred) {
    const double ide = 1.0 / de;
    double part = 0.0;
    for (int i = threadIdx.x; i < nE - 1; i += blockDim.x) {
        const double a = e0 + i * de, b = e0 + (i + 1) * de;
        double M0, M1, M2;
        interval_moments(a, b, mu, kT, M0, M1, M2);
        const double m1 = M1 * ide;
        part += (M0 - m1) * sD[i] + m1 * sD[i + 1];
    }
    return block_sum(part, sred);
}

// ---- e_F by wide bisection --------------------------------------------------
//
// Bisection on [lo, hi] visits, in its next 7 steps, 7 of the 127 midpoints of
// the complete binary tree of halvings below [lo, hi] (node k in heap order,
// children 2k+1 = left half, 2k+2 = right half).  A round evaluates
// N(mu) - N_e at all 127 nodes, one block each, with the same block size and
// reduction order as a single evaluation, and the next kernel replays the 7
// decisions: the brackets, midpoints and iteration count are bit for bit those
// of the one-step-at-a-time loop.  fstate holds two slots of the bracket state
// (lo, hi, f(lo), iterations, status, done, exact) and two rows of node values,
// each written by one round and read by the next.
constexpr int kWideDepth = 7;
constexpr int kWideNodes = (1 << kWideDepth) - 1;
constexpr int kFsSlot = 8;
constexpr int kFsInit = 2 * kFsSlot;        // f(lo0), f(hi0)
constexpr int kFsNodes = kFsInit + 8;       // 2 rows of 128 node values
constexpr int kFermiStateDoubles = kFsNodes + 2 * 128;

struct Bracket {
    double lo, hi, flo;
    int it, status;
    bool done, exact;
};

__device__ __forceinline__ void load_bracket(const double* p, Bracket& b) {
    b.lo = p[0];
    b.hi = p[1];
    b.flo = p[2];
    b.it = (int)p[3];
    b.status = (int)p[4];
    b.done = p[5] != 0.0;
    b.exact = p[6] != 0.0;
}

__device__ __forceinline__ void store_bracket(double* p, const Bracket& b) {
    p[0] = b.lo;
    p[1] = b.hi;
    p[2] = b.flo;
    p[3] = (double)b.it;
    p[4] = (double)b.status;
    p[5] = b.done ? 1.0 : 0.0;
    p[6] = b.exact ? 1.0 : 0.0;
}

// bracket at the start of the bisection, from f at both ends
__device__ Bracket initial_bracket(double lo, double hi, double flo, double fhi) {
    Bracket b{lo, hi, flo, 0, 0, false, false};
    if (flo == 0.0) {
        b.hi = lo;
        b.exact = b.done = true;
    } else if (fhi == 0.0) {
        b.lo = hi;
        b.exact = b.done = true;
    } else if ((flo > 0.0) == (fhi > 0.0)) {
        b.status = 1;
        b.done = true;
    }
    return b;
}

// up to kWideDepth bisection steps with the node values fm of the tree below b
__device__ void replay(Bracket& b, const double* fm, double tol, int max_iter) {
    int k = 0;
    for (int step = 0; step < kWideDepth && !b.done; ++step) {
        if (b.it >= max_iter || b.hi - b.lo < tol) {
            b.done = true;
            break;
        }
        const double mid = 0.5 * (b.lo + b.hi);
        const double f = fm[k];
        if (f == 0.0) {
            b.lo = b.hi = mid;
            b.exact = b.done = true;
            break;
        }
        if ((f > 0.0) == (b.flo > 0.0)) {
            b.lo = mid;
            b.flo = f;
            k = 2 * k + 2;
        } else {
            b.hi = mid;
            k = 2 * k + 1;
        }
        ++b.it;
    }
}

// midpoint of tree node k below [lo, hi], halving along its path from the root
__device__ double node_mid(double lo, double hi, int k) {
    int path[kWideDepth];
    int d = 0;
    while (k > 0) {
        path[d++] = k;
        k = (k - 1) / 2;
    }
    for (int i = d - 1; i >= 0; --i) {
        const double mid = 0.5 * (lo + hi);
        if ((path[i] & 1) == 0) lo = mid;  // right child
        else hi = mid;                     // left child
    }
    return 0.5 * (lo + hi);
}

__device__ __forceinline__ void stage_D(const double* __restrict__ D, int nE, double* sD) {
    for (int i = threadIdx.x; i < nE; i += blockDim.x) sD[i] = D[i];
    __syncthreads();
}

// D = dV * dos_sum; f at the initial bracket ends (block 0: lo, block 1: hi)
__global__ void __launch_bounds__(kFermiThreads) k_fermi_init(const double* __restrict__ dos_sum, int nE, double dV,
                                                              double e0, double de, double kT, double Ne,
                                                              double* __restrict__ D, double* __restrict__ fs) {
    extern __shared__ double sD[];
    __shared__ double sred[33];
    for (int i = threadIdx.x; i < nE; i += blockDim.x) {
        sD[i] = dV * dos_sum[i];
        if (blockIdx.x == 0) D[i] = sD[i];
    }
    __syncthreads();
    const double mu = blockIdx.x == 0 ? e0 - 20.0 * kT : e0 + (nE - 1) * de + 20.0 * kT;
    const double f = electron_count(sD, nE, e0, de, mu, kT, sred) - Ne;
    if (threadIdx.x == 0) fs[kFsInit + blockIdx.x] = f;
}

// bracket at the start of round r (r = 0: from the initial ends)
__device__ Bracket round_start(const double* fs, int r, double e0, double de, double kT, int nE, double tol,
                               int max_iter) {
    if (r == 0)
        return initial_bracket(e0 - 20.0 * kT, e0 + (nE - 1) * de + 20.0 * kT, fs[kFsInit], fs[kFsInit + 1]);
    Bracket b;
    load_bracket(fs + ((r - 1) & 1) * kFsSlot, b);
    replay(b, fs + kFsNodes + ((r - 1) & 1) * 128, tol, max_iter);
    return b;
}

__global__ void __launch_bounds__(kFermiThreads) k_fermi_round(const double* __restrict__ D, int nE, double e0, double de,
                                                               double kT, double Ne, double tol, int max_iter,
                                                               double* __restrict__ fs, int r) {
    extern __shared__ double sD[];
    __shared__ double sred[33];
    const Bracket b = round_start(fs, r, e0, de, kT, nE, tol, max_iter);
    if (blockIdx.x == 0 && threadIdx.x == 0) store_bracket(fs + (r & 1) * kFsSlot, b);
    if (b.done) return;
    stage_D(D, nE, sD);
    const double mu = node_mid(b.lo, b.hi, blockIdx.x);
    const double f = electron_count(sD, nE, e0, de, mu, kT, sred) - Ne;
    if (threadIdx.x == 0) fs[kFsNodes + (r & 1) * 128 + blockIdx.x] = f;
}

// Weights at e_F, one thread per energy interval [e_i, e_{i+1}], spread over
// many CTAs (the closed forms are FP64-heavy): the interval's moments give the
// right part of hat_i and the left part of hat_{i+1}; iv[i] holds
// (w0, w1, wS) of hat_i's part and (w0, w1, wS) of hat_{i+1}'s part.
constexpr int kIvPerCta = 32;

__global__ void __launch_bounds__(kIvPerCta) k_fermi_intervals(int nE, double e0, double de, double kT, double tol,
                                                              int max_iter, const double* __restrict__ fs, int rounds,
                                                              double* __restrict__ iv) {
    const Bracket b = round_start(fs, rounds, e0, de, kT, nE, tol, max_iter);
    const double eF = b.exact ? b.lo : 0.5 * (b.lo + b.hi);
    const int i = blockIdx.x * kIvPerCta + threadIdx.x;
    if (i >= nE - 1) return;
    const double a = e0 + i * de;
    double M0, M1, M2, S0, S1;
    interval_moments(a, a + de, eF, kT, M0, M1, M2);
    entropy_moments(a, a + de, eF, kT, S0, S1);
    double* o = iv + 6 * (size_t)i;
    o[0] = M0 - M1 / de;                          // hat_i: (e_{i+1} - e) / de
    o[1] = a * M0 + M1 - (a * M1 + M2) / de;
    o[2] = S0 - S1 / de;
    o[3] = M1 / de;                               // hat_{i+1}: (e - e_i) / de
    o[4] = (a * M1 + M2) / de;
    o[5] = S1 / de;
}

// scal: [0] e_F, [1] E_b, [2] status (0 ok, 1 no bracket), [3] N(e_F), [4] iterations, [5] -tau S_s
__global__ void __launch_bounds__(kFermiThreads) k_fermi_final(const double* __restrict__ Dg, int nE, double e0,
                                                               double de, double kT, double tol, int max_iter,
                                                               const double* __restrict__ fs, int rounds,
                                                               const double* __restrict__ iv,
                                                               double* __restrict__ w0d, float* __restrict__ w0f,
                                                               double* __restrict__ scal) {
    extern __shared__ double sD[];
    __shared__ double sred[33];
    const Bracket b = round_start(fs, rounds, e0, de, kT, nE, tol, max_iter);
    stage_D(Dg, nE, sD);
    const double eF = b.exact ? b.lo : 0.5 * (b.lo + b.hi);
    const int status = b.status, it = b.it;
    // node weights from the two intervals beside each node; band energy, entropy term, electron count
    double pn = 0.0, pe = 0.0, ps = 0.0;
    for (int x = threadIdx.x; x < nE; x += blockDim.x) {
        double w0 = 0.0, w1 = 0.0, ws = 0.0;
        if (x > 0) {  // right half of hat_x on [e_{x-1}, e_x]
            const double* o = iv + 6 * (size_t)(x - 1);
            w0 += o[3];
            w1 += o[4];
            ws += o[5];
        }
        if (x < nE - 1) {  // left half of hat_x on [e_x, e_{x+1}]
            const double* o = iv + 6 * (size_t)x;
            w0 += o[0];
            w1 += o[1];
            ws += o[2];
        }
        w0d[x] = w0;
        w0f[x] = (float)w0;
        pn += w0 * sD[x];
        pe += w1 * sD[x];
        ps += ws * sD[x];
    }
    const double Nf = block_sum(pn, sred);
    const double Eb = block_sum(pe, sred);
    const double Sk = block_sum(ps, sred);  // S_s / k_B
    if (threadIdx.x == 0) {
        scal[0] = eF;
        scal[1] = Eb;
        scal[2] = (double)status;
        scal[3] = Nf;
        scal[4] = (double)it;
        scal[5] = -kT * Sk;  // -tau S_s in eV
    }
}

// dE_b/dD_x at fixed N_e (the first factor of Eq. forcesmala for E = E_b).
// E_b = sum_x w1_x(mu) D_x with mu fixed by N(mu) = sum_x w0_x(mu) D_x = N_e, so
// dE_b/dD_x = w1_x - mu~ w0_x, mu~ = (d/dmu sum w1 D) / (d/dmu sum w0 D).
// For the piecewise-linear D(e), integrating -df/de by parts over each
// interval [a, b] with slope s = (D_{i+1} - D_i) / de leaves boundary terms
// (which telescope to the two ends) and moments of f:
//   d/dmu N   = D_0 f(e_0) - D_n f(e_n) + sum_i s_i M0_i,
//   d/dmu E_b = e_0 D_0 f(e_0) - e_n D_n f(e_n) + sum_i ((D_i + s_i a_i) M0_i + 2 s_i M1_i).
// One block; mom: 3 n_E doubles of scratch; out[0] = mu~ (NaN when d/dmu N = 0).
__global__ void __launch_bounds__(kFermiThreads) k_egrad(const double* __restrict__ D, int nE, double e0, double de,
                                                         double kT, const double* __restrict__ scal, double gscale,
                                                         double* __restrict__ mom, double* __restrict__ g,
                                                         double* __restrict__ out) {
    __shared__ double sred[33];
    const double mu = scal[0];
    double pn = 0.0, pe = 0.0;
    for (int i = threadIdx.x; i < nE - 1; i += blockDim.x) {
        const double a = e0 + i * de;
        double M0, M1, M2;
        interval_moments(a, a + de, mu, kT, M0, M1, M2);
        mom[3 * i] = M0;
        mom[3 * i + 1] = M1;
        mom[3 * i + 2] = M2;
        const double sl = (D[i + 1] - D[i]) / de;
        pn += sl * M0;
        pe += (D[i] + sl * a) * M0 + 2.0 * sl * M1;
    }
    double dn = block_sum(pn, sred);
    double dE = block_sum(pe, sred);
    const double en = e0 + (nE - 1) * de;
    const double xa = (e0 - mu) / kT, xb = (en - mu) / kT;
    const double fa = xa > 0.0 ? exp(-xa) / (1.0 + exp(-xa)) : 1.0 / (1.0 + exp(xa));
    const double fb = xb > 0.0 ? exp(-xb) / (1.0 + exp(-xb)) : 1.0 / (1.0 + exp(xb));
    dn += D[0] * fa - D[nE - 1] * fb;
    dE += e0 * D[0] * fa - en * D[nE - 1] * fb;
    const double mt = dn != 0.0 ? dE / dn : nan("");
    for (int x = threadIdx.x; x < nE; x += blockDim.x) {
        double w0 = 0.0, w1 = 0.0;
        if (x > 0) {  // right half of hat_x on [e_{x-1}, e_x]
            const double a = e0 + (x - 1) * de;
            const double* m = mom + 3 * (size_t)(x - 1);
            w0 += m[1] / de;
            w1 += (a * m[1] + m[2]) / de;
        }
        if (x < nE - 1) {  // left half of hat_x on [e_x, e_{x+1}]
            const double a = e0 + x * de;
            const double* m = mom + 3 * (size_t)x;
            w0 += m[0] - m[1] / de;
            w1 += a * m[0] + m[1] - (a * m[1] + m[2]) / de;
        }
        g[x] = gscale * (w1 - mt * w0);
    }
    if (threadIdx.x == 0) out[0] = mt;
}

// column sums over blocks of 128 rows (FP32 in row order, as the network
// epilogue forms them) -> FP64 partial rows
template <class TL>
__global__ void k_colsum(const TL* __restrict__ L, int64_t P, int nE, double* __restrict__ part) {
    const int64_t r0 = (int64_t)blockIdx.x * 128;
    const int64_t r1 = min(P, r0 + 128);
    for (int c = threadIdx.x; c < nE; c += blockDim.x) {
        if constexpr (sizeof(TL) == 2) {
            float s = 0.f;
            for (int64_t r = r0; r < r1; ++r) s += __bfloat162float(L[r * nE + c]);
            part[(int64_t)blockIdx.x * nE + c] = (double)s;
        } else {
            double s = 0.0;
            for (int64_t r = r0; r < r1; ++r) s += (double)L[r * nE + c];
            part[(int64_t)blockIdx.x * nE + c] = s;
        }
    }
}

// out[c] = sum_t part[t][c]: one CTA per column, threads over row strides, then a
// fixed-order tree over the threads (deterministic)
constexpr int kSumRowsThreads = 256;
__global__ void __launch_bounds__(kSumRowsThreads) k_sum_rows(const double* __restrict__ part, int64_t nt, int nE,
                                                              double* __restrict__ out) {
    __shared__ double red[kSumRowsThreads];
    const int c = blockIdx.x;
    double s = 0.0;
    for (int64_t t = threadIdx.x; t < nt; t += kSumRowsThreads) s += part[t * nE + c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = kSumRowsThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = red[0];
}

// n(r) = sum_xi w0_xi LDOS(r, xi): one streaming pass over the LDOS.
// Persistent CTAs walk tiles of whole rows; a tile's bytes, rounded out to
// 16-byte boundaries (the LDOS of a batch member may start anywhere), arrive in
// shared memory by one cp.async.bulk, kDensStages tiles in flight per CTA, so
// HBM sees large sequential reads with no per-thread loads outstanding.  In
// shared memory a group of G lanes takes a row (lanes over energies, w0 held
// in shared memory), the group's partial sums meet by shuffles.  Per-CTA FP64
// partial sums of n give the electron-count check.  Every wait is bounded;
// on expiry the CTA sets *err, lets its copies land and returns.
constexpr int kDensThreads = 256;
constexpr int kDensStages = 6;
constexpr int kDensTileBytes = 32768;                      // payload of one stage
constexpr int kDensStageBytes = kDensTileBytes + 32;       // + the 16-byte rounding at both ends
constexpr long long kDensWaitCycles = 2000000000LL;        // about one second

struct DensPlan {
    int rows;   // rows per tile
    int G;      // lanes per row (power of two <= 32)
    int wpl;    // BF16 pairs per lane in the register path (0: shared-memory weights)
};

constexpr int kDensMaxWpl = 16;  // weights held in registers: at most 16 BF16 pairs per lane

// BF16 rows of even length: a lane takes every G-th 4-byte pair of its row with
// its weights in registers; otherwise lanes take every G-th element, weights in
// shared memory.
inline DensPlan dens_plan(int nE, int elem_bytes) {
    DensPlan d;
    int G = 1;
    d.wpl = 0;
    if (elem_bytes == 2 && (nE & 1) == 0) {
        const int nw = nE / 2;
        while (G < 32 && (nw + G - 1) / G > kDensMaxWpl) G *= 2;
        if ((nw + G - 1) / G <= kDensMaxWpl) d.wpl = (nw + G - 1) / G;
    }
    if (!d.wpl) {
        G = 1;
        while (G < 32 && G * 8 < nE) G *= 2;  // about 8 or more energies per lane
    }
    const int rb = nE * elem_bytes;
    int rows = std::max(1, kDensTileBytes / rb);
    const int pass = kDensThreads / G;     // rows one pass over the CTA's threads covers
    if (rows >= pass) rows -= rows % pass;
    d.rows = rows;
    d.G = G;
    return d;
}

inline size_t dens_smem_bytes(int nE, int w_bytes) {
    return (size_t)kDensStages * kDensStageBytes + (size_t)nE * w_bytes + kDensStages * 8 + 64 * 8 + 256;
}

__device__ __forceinline__ bool dens_try(uint32_t bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool dens_wait(uint32_t bar, uint32_t phase) {
    const long long t0 = clock64();
    while (!dens_try(bar, phase))
        if (clock64() - t0 > kDensWaitCycles) return false;
    return true;
}

template <class TL> __device__ __forceinline__ float dens_val(const unsigned char* p);
template <> __device__ __forceinline__ float dens_val<__nv_bfloat16>(const unsigned char* p) {
    return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(p));
}

// tile t of rows [t R, t R + nr): its 16-byte-rounded byte range
__device__ __forceinline__ void dens_range(const unsigned char* L, int64_t P, int R, int rb, int64_t t,
                                           uintptr_t& a0, uint32_t& bytes, uint32_t& off, int& nr) {
    const int64_t r0 = t * R;
    nr = (int)min((int64_t)R, P - r0);
    const uintptr_t s = reinterpret_cast<uintptr_t>(L) + (uintptr_t)(r0 * rb);
    const uintptr_t e = s + (uintptr_t)nr * rb;
    a0 = s & ~uintptr_t(15);
    bytes = (uint32_t)(((e + 15) & ~uintptr_t(15)) - a0);
    off = (uint32_t)(s - a0);
}

// TL: LDOS element (BF16 or FP64), TW: arithmetic and output type (float or double)
template <class TL, class TW>
__global__ void __launch_bounds__(kDensThreads) k_density(const TL* __restrict__ Lg, int64_t P, int nE, int R, int G,
                                                          int wpl, const TW* __restrict__ w0, TW* __restrict__ n,
                                                          double* __restrict__ part, int* __restrict__ err) {
    extern __shared__ __align__(128) unsigned char dsm[];
    unsigned char* stage = dsm;
    TW* sw = reinterpret_cast<TW*>(dsm + (size_t)kDensStages * kDensStageBytes);
    uint64_t* bars = reinterpret_cast<uint64_t*>(
        (reinterpret_cast<uintptr_t>(sw + nE) + 7) & ~uintptr_t(7));
    double* sred = reinterpret_cast<double*>(bars + kDensStages);
    const unsigned char* L = reinterpret_cast<const unsigned char*>(Lg);
    const int rb = nE * (int)sizeof(TL);
    const int64_t ntiles = (P + R - 1) / R;
    const int tid = threadIdx.x, lane = tid & 31;
    const int g = tid & (G - 1), grp = tid / G, ngrp = kDensThreads / G;
    for (int i = tid; i < nE; i += kDensThreads) sw[i] = w0[i];
    // register path: this lane's weights, pairs g, g + G, ... of the row
    float wr[2 * kDensMaxWpl];
    const bool regs = sizeof(TL) == 2 && wpl > 0 && (reinterpret_cast<uintptr_t>(Lg) & 3) == 0;
    if (regs) {
#pragma unroll
        for (int k = 0; k < kDensMaxWpl; ++k) {
            const int q = g + k * G;
            const bool in = k < wpl && 2 * q < nE;
            wr[2 * k] = in ? (float)w0[2 * q] : 0.f;
            wr[2 * k + 1] = in ? (float)w0[2 * q + 1] : 0.f;
        }
    }
    if (tid == 0) {
        for (int s2 = 0; s2 < kDensStages; ++s2)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((uint32_t)__cvta_generic_to_shared(&bars[s2])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    auto issue = [&](int64_t t, int s2) {
        uintptr_t a0;
        uint32_t bytes, off;
        int nr;
        dens_range(L, P, R, rb, t, a0, bytes, off, nr);
        const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&bars[s2]);
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(stage + (size_t)s2 * kDensStageBytes);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                     "l"(a0), "r"(bytes), "r"(bar)
                     : "memory");
    };
    int issued = 0;  // tiles issued by this CTA (thread 0's count)
    if (tid == 0)
        for (int s2 = 0; s2 < kDensStages; ++s2) {
            const int64_t t = (int64_t)blockIdx.x + (int64_t)s2 * gridDim.x;
            if (t >= ntiles) break;
            issue(t, s2);
            ++issued;
        }
    double acc = 0.0;
    bool ok = true;
    int it = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const int s2 = it % kDensStages;
        const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&bars[s2]);
        const bool got = dens_wait(bar, (uint32_t)((it / kDensStages) & 1));
        if (!__syncthreads_and(got)) {
            ok = false;
            break;
        }
        uintptr_t a0;
        uint32_t bytes, off;
        int nr;
        dens_range(L, P, R, rb, t, a0, bytes, off, nr);
        const unsigned char* base = stage + (size_t)s2 * kDensStageBytes + off;
        // rows of this tile: groups of G lanes, each lane a strided slice of the energies
        const int npass = (nr + ngrp - 1) / ngrp;
        for (int ps = 0; ps < npass; ++ps) {
            const int r = ps * ngrp + grp;
            TW s = TW(0);
            if (r < nr) {
                const unsigned char* row = base + (size_t)r * rb;
                if (regs) {
                    // all of the lane's pairs loaded first (independent 4-byte loads), then two FMA chains
                    const uint32_t* row32 = reinterpret_cast<const uint32_t*>(row);
                    const int nw = nE >> 1;
                    uint32_t v[kDensMaxWpl];
#pragma unroll
                    for (int k = 0; k < kDensMaxWpl; ++k) {
                        const int q = g + k * G;
                        v[k] = (k < wpl && q < nw) ? row32[q] : 0u;
                    }
                    float s0 = 0.f, s1 = 0.f;
#pragma unroll
                    for (int k = 0; k < kDensMaxWpl; ++k) {
                        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v[k]));
                        s0 = fmaf(f.x, wr[2 * k], s0);
                        s1 = fmaf(f.y, wr[2 * k + 1], s1);
                    }
                    s = (TW)(s0 + s1);
                } else {
                    for (int c = g; c < nE; c += G) {
                        TW v;
                        if constexpr (sizeof(TL) == 2) v = dens_val<TL>(row + 2 * c);
                        else v = *reinterpret_cast<const double*>(row + 8 * c);
                        s = fma(v, sw[c], s);
                    }
                }
            }
            for (int o = G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (r < nr && g == 0) {
                n[t * R + r] = s;
                acc += (double)s;
            }
        }
        __syncthreads();  // the stage is free again
        if (tid == 0) {
            const int64_t tn = t + (int64_t)kDensStages * gridDim.x;
            if (tn < ntiles) {
                issue(tn, s2);
                ++issued;
            }
        }
    }
    if (!ok) {
        if (tid == 0) {
            atomicCAS(err, 0, 1);
            // let the copies still in flight land before the CTA exits
            for (int j = it; j < issued; ++j) {
                const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&bars[j % kDensStages]);
                dens_wait(bar, (uint32_t)((j / kDensStages) & 1));
            }
        }
        __syncthreads();
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sred[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
        double tsum = 0.0;
        for (int w = 0; w < kDensThreads / 32; ++w) tsum += sred[w];
        part[blockIdx.x] = tsum;
    }
}

// BF16 rows of even length: direct loads instead of staged tiles.  A group of
// G lanes takes a row; every lane issues its (up to kDensMaxWpl) 4-byte pairs of
// the row back to back (streaming loads, read once), then one FMA chain pair
// with the weights from shared memory (one broadcast 8-byte read per pair) and
// a shuffle reduction over the group.  At most 42 registers a thread let 6 CTAs
// of 256 threads share an SM, about 100 KB of loads in flight per SM.
constexpr int kDensDirectCtasPerSm = 6;

__global__ void __launch_bounds__(kDensThreads, kDensDirectCtasPerSm)
    k_density_direct(const __nv_bfloat16* __restrict__ L, int64_t P, int nE, int G, int wpl,
                     const float* __restrict__ w0, float* __restrict__ n, double* __restrict__ part) {
    extern __shared__ __align__(16) float swd[];  // [nE] weights, then the CTA's partial sums
    double* sred = reinterpret_cast<double*>(swd + ((nE + 3) & ~3));
    const int tid = threadIdx.x, lane = tid & 31;
    const int g = tid & (G - 1), grp = tid / G, ngrp = kDensThreads / G;
    const int nw = nE >> 1;
    for (int i = tid; i < nE; i += kDensThreads) swd[i] = w0[i];
    __syncthreads();
    const float2* sw2 = reinterpret_cast<const float2*>(swd);
    double acc = 0.0;
    const int64_t stride = (int64_t)gridDim.x * ngrp;
    for (int64_t rb = (int64_t)blockIdx.x * ngrp; rb < P; rb += stride) {  // uniform over the CTA
        const int64_t r = rb + grp;
        float s0 = 0.f, s1 = 0.f;
        if (r < P) {
            const uint32_t* row32 = reinterpret_cast<const uint32_t*>(L + r * nE);
            uint32_t v[kDensMaxWpl];
#pragma unroll
            for (int k = 0; k < kDensMaxWpl; ++k) {
                const int q = g + k * G;
                v[k] = (k < wpl && q < nw) ? __ldcs(row32 + q) : 0u;
            }
#pragma unroll
            for (int k = 0; k < kDensMaxWpl; ++k) {
                const int q = g + k * G;
                if (k < wpl && q < nw) {
                    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&v[k]));
                    const float2 w = sw2[q];
                    s0 = fmaf(f.x, w.x, s0);
                    s1 = fmaf(f.y, w.y, s1);
                }
            }
        }
        float s = s0 + s1;
        for (int o = G >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (r < P && g == 0) {
            n[r] = s;
            acc += (double)s;
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) sred[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < kDensThreads / 32; ++w) t += sred[w];
        part[blockIdx.x] = t;
    }
}

// Tiled BF16 density pass.  A tile is R whole rows whose bytes start on a
// 16-byte boundary (R = 8 / gcd(n_E, 8), so R n_E is a multiple of 8 and the
// tile a whole number of 16-byte chunks of 8 energies); a warp reads a tile as
// 16-byte loads, chunk j by lane j mod 32.  Every lane meets its chunks at the
// same offsets in every tile, so their weights and the row each chunk starts
// in are fixed per lane and kept in registers.  A chunk meets at most two rows
// (n_E >= 8): the energies in its first row are weighted from registers, the
// few past that row's end (three lanes per tile at n_E = 250) from the cached
// weight array, each part goes to its own row, and the per-row sums meet by
// warp shuffles.  The warp loads the next tile before it reduces the current
// one.  Rows before the first aligned tile and after the last whole tile go
// through warp 0 of CTA 0, element by element.  One CTA of 512 threads per SM.
constexpr int kDensTileThreads = 512;
constexpr int kDensTileWarps = kDensTileThreads / 32;

inline int dens_tile_rows(int nE) {
    int g = 8;
    while (nE % g) g >>= 1;  // gcd(nE, 8)
    return 8 / g;
}

template <int R, int K>
__global__ void __launch_bounds__(kDensTileThreads, 1)
    k_density_tiled(const __nv_bfloat16* __restrict__ L, int64_t P, int nE, int64_t head, int64_t ntile,
                    const float* __restrict__ w0, float* __restrict__ n, double* __restrict__ part) {
    __shared__ double sred[kDensTileWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int C = R * nE / 8;  // chunks per tile, at most 32 K
    float w[K][8];
    int ra[K], bnd[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const int j = lane + 32 * i;
        const int e0 = 8 * j;
        ra[i] = e0 / nE;
        bnd[i] = (ra[i] + 1) * nE - e0;  // energies of the chunk in row ra (>= 8: all of them)
#pragma unroll
        for (int k = 0; k < 8; ++k)  // the weights of the energies in row ra (0 past its end)
            w[i][k] = (j < C && k < bnd[i]) ? __ldg(w0 + e0 + k - nE * ra[i]) : 0.f;
    }
    const uint4* T = reinterpret_cast<const uint4*>(L + head * nE);
    const int64_t wid = (int64_t)blockIdx.x * kDensTileWarps + warp;
    const int64_t nwarp = (int64_t)gridDim.x * kDensTileWarps;
    double dacc = 0.0;
    uint4 cur[K], nxt[K];
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const int j = lane + 32 * i;
        cur[i] = (wid < ntile && j < C) ? __ldcs(T + wid * C + j) : make_uint4(0u, 0u, 0u, 0u);
    }
    for (int64_t t = wid; t < ntile; t += nwarp) {
        const int64_t tn = t + nwarp;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const int j = lane + 32 * i;
            nxt[i] = (tn < ntile && j < C) ? __ldcs(T + tn * C + j) : make_uint4(0u, 0u, 0u, 0u);
        }
        float acc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = 0.f;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const uint32_t q[4] = {cur[i].x, cur[i].y, cur[i].z, cur[i].w};
            float f[8];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 p = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&q[k]));
                f[2 * k] = p.x;
                f[2 * k + 1] = p.y;
            }
            float lo = 0.f, hi = 0.f;
#pragma unroll
            for (int k = 0; k < 8; ++k) lo = fmaf(f[k], w[i][k], lo);
            if (bnd[i] < 8) {  // the chunk runs into the next row (a few lanes per tile)
                const int c1 = 8 * (lane + 32 * i) - (ra[i] + 1) * nE;  // its column there (< 0 before it)
#pragma unroll
                for (int k = 0; k < 8; ++k)
                    if (k >= bnd[i]) hi = fmaf(f[k], __ldg(w0 + c1 + k), hi);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] += (r == ra[i] ? lo : 0.f) + (r == ra[i] + 1 ? hi : 0.f);
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[r] += __shfl_xor_sync(0xffffffffu, acc[r], o);
        float s = acc[0];
#pragma unroll
        for (int r = 1; r < R; ++r) s = lane == r ? acc[r] : s;
        if (lane < R) {
            n[head + t * R + lane] = s;
            dacc += (double)s;
        }
#pragma unroll
        for (int i = 0; i < K; ++i) cur[i] = nxt[i];
    }
    if (blockIdx.x == 0 && warp == 0) {
        // the rows outside the whole tiles
        const int64_t tail0 = head + ntile * R;
        for (int64_t r = 0; r < P; ++r) {
            if (r == head) r = tail0;
            if (r >= P) break;
            float s = 0.f;
            for (int e = lane; e < nE; e += 32) s = fmaf(__bfloat162float(L[r * nE + e]), __ldg(w0 + e), s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) {
                n[r] = s;
                dacc += (double)s;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dacc += __shfl_xor_sync(0xffffffffu, dacc, o);
    if (lane == 0) sred[warp] = dacc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tsum = 0.0;
        for (int k = 0; k < kDensTileWarps; ++k) tsum += sred[k];
        part[blockIdx.x] = tsum;
    }
}

// the tiled path applies: BF16, n_E >= 8 and a tile of at most 128 chunks (4 per lane)
inline bool density_tiled(int nE, int elem_bytes) {
    return elem_bytes == 2 && nE >= 8 && dens_tile_rows(nE) * nE <= 1024;
}

template <int R>
void launch_density_tiled_r(const __nv_bfloat16* L, int64_t P, int nE, int64_t head, int64_t ntile, const float* w0,
                            float* n, double* part, int grid, cudaStream_t st) {
    const int K = (R * nE / 8 + 31) / 32;
    if (K <= 1) k_density_tiled<R, 1><<<grid, kDensTileThreads, 0, st>>>(L, P, nE, head, ntile, w0, n, part);
    else if (K == 2) k_density_tiled<R, 2><<<grid, kDensTileThreads, 0, st>>>(L, P, nE, head, ntile, w0, n, part);
    else if (K == 3) k_density_tiled<R, 3><<<grid, kDensTileThreads, 0, st>>>(L, P, nE, head, ntile, w0, n, part);
    else k_density_tiled<R, 4><<<grid, kDensTileThreads, 0, st>>>(L, P, nE, head, ntile, w0, n, part);
}

// false when no row of L starts on a 16-byte boundary within the first tile (then the other paths run)
inline bool launch_density_tiled(const __nv_bfloat16* L, int64_t P, int nE, const float* w0, float* n, double* part,
                                 int grid, cudaStream_t st) {
    const int R = dens_tile_rows(nE);
    int64_t head = -1;
    for (int r = 0; r < R && r <= P; ++r)
        if ((reinterpret_cast<uintptr_t>(L + (int64_t)r * nE) & 15) == 0) {
            head = r;
            break;
        }
    if (head < 0) return false;
    const int64_t ntile = P > head ? (P - head) / R : 0;
    switch (R) {
        case 1: launch_density_tiled_r<1>(L, P, nE, head, ntile, w0, n, part, grid, st); break;
        case 2: launch_density_tiled_r<2>(L, P, nE, head, ntile, w0, n, part, grid, st); break;
        case 4: launch_density_tiled_r<4>(L, P, nE, head, ntile, w0, n, part, grid, st); break;
        default: launch_density_tiled_r<8>(L, P, nE, head, ntile, w0, n, part, grid, st); break;
    }
    return true;
}

// the direct path applies: BF16, an even row length whose pairs fit the registers, 4-byte aligned rows
inline bool density_direct(int nE, int elem_bytes) {
    return elem_bytes == 2 && dens_plan(nE, elem_bytes).wpl > 0;
}

template <class TL, class TW>
void launch_density(const TL* L, int64_t P, int nE, const TW* w0, TW* n, double* part, int grid, int* err,
                    cudaStream_t st) {
    const DensPlan d = dens_plan(nE, (int)sizeof(TL));
    if constexpr (sizeof(TL) == 2 && sizeof(TW) == 4) {
        if (density_tiled(nE, 2) && launch_density_tiled(L, P, nE, w0, n, part, grid, st)) return;
    }
    if constexpr (sizeof(TL) == 2) {
        if (density_direct(nE, 2) && (reinterpret_cast<uintptr_t>(L) & 3) == 0) {
            const size_t smem = sizeof(float) * (size_t)((nE + 3) & ~3) + sizeof(double) * (kDensThreads / 32);
            k_density_direct<<<grid, kDensThreads, smem, st>>>(L, P, nE, d.G, d.wpl, w0, n, part);
            return;
        }
    }
    const size_t smem = dens_smem_bytes(nE, (int)sizeof(TW));
    cudaFuncSetAttribute(k_density<TL, TW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_density<TL, TW><<<grid, kDensThreads, smem, st>>>(L, P, nE, d.rows, d.G, d.wpl, w0, n, part, err);
}

// CTAs of the density pass (the partial-sum rows it writes): the tiled path
// runs one per SM, the direct path kDensDirectCtasPerSm per SM, the staged path
// one per SM, never more than there are row groups or tiles (any count works
// for every path: the kernels stride over the CTAs)
inline int density_grid(int64_t P, int nE, int elem_bytes, int num_sms) {
    if (density_tiled(nE, elem_bytes)) {  // one CTA per SM, at most one per kDensTileWarps tiles
        const int64_t tiles = P / dens_tile_rows(nE);
        return (int)std::max<int64_t>(1, std::min<int64_t>((tiles + kDensTileWarps - 1) / kDensTileWarps,
                                                           (int64_t)std::max(1, num_sms)));
    }
    const DensPlan d = dens_plan(nE, elem_bytes);
    if (density_direct(nE, elem_bytes)) {
        const int64_t groups = (P + kDensThreads / d.G - 1) / (kDensThreads / d.G);
        return (int)std::max<int64_t>(1, std::min<int64_t>(groups, (int64_t)std::max(1, num_sms) * kDensDirectCtasPerSm));
    }
    const int64_t ntiles = (P + d.rows - 1) / d.rows;
    return (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, std::max(1, num_sms)));
}

// N(mu) for one mu (single block)
__global__ void __launch_bounds__(kFermiThreads) k_count(const double* __restrict__ D, int nE, double e0, double de,
                                                         double kT, double mu, double* __restrict__ out) {
    extern __shared__ double sD[];
    __shared__ double sred[33];
    for (int i = threadIdx.x; i < nE; i += blockDim.x) sD[i] = D[i];
    __syncthreads();
    const double n = electron_count(sD, nE, e0, de, mu, kT, sred);
    if (threadIdx.x == 0) *out = n;
}

__global__ void k_sum_vec(const double* __restrict__ part, int n, double* __restrict__ out) {
    __shared__ double s[256];
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) t += part[i];
    s[threadIdx.x] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) a += s[i];
        *out = a;
    }
}

constexpr double kFermiTol = 1e-12;
constexpr int kFermiMaxIter = 200;

// init, enough rounds of 7 steps to shrink the bracket below the tolerance, final
// fstate: kFermiStateDoubles, then 6 n_E doubles of interval weights
void launch_fermi(const double* dos_sum, int nE, double dV, const mala_energy_grid* eg, double* D, double* w0d,
                  float* w0f, double* scal, double* fstate, cudaStream_t st) {
    double* iv = fstate + kFermiStateDoubles;
    const size_t sm = sizeof(double) * nE;
    const double width = (nE - 1) * eg->de_eV + 40.0 * eg->kT_eV;
    int steps = (int)std::ceil(std::log2(std::max(width / kFermiTol, 1.0))) + 2;
    steps = std::min(steps, kFermiMaxIter);
    const int rounds = (steps + kWideDepth - 1) / kWideDepth;
    k_fermi_init<<<2, kFermiThreads, sm, st>>>(dos_sum, nE, dV, eg->e0_eV, eg->de_eV, eg->kT_eV, eg->n_electrons, D,
                                               fstate);
    for (int r = 0; r < rounds; ++r)
        k_fermi_round<<<kWideNodes, kFermiThreads, sm, st>>>(D, nE, eg->e0_eV, eg->de_eV, eg->kT_eV, eg->n_electrons,
                                                             kFermiTol, kFermiMaxIter, fstate, r);
    k_fermi_intervals<<<(nE - 1 + kIvPerCta - 1) / kIvPerCta, kIvPerCta, 0, st>>>(
        nE, eg->e0_eV, eg->de_eV, eg->kT_eV, kFermiTol, kFermiMaxIter, fstate, rounds, iv);
    k_fermi_final<<<1, kFermiThreads, sm, st>>>(D, nE, eg->e0_eV, eg->de_eV, eg->kT_eV, kFermiTol, kFermiMaxIter,
                                                fstate, rounds, iv, w0d, w0f, scal);
}

// Bernoulli numbers B_0..B_n (B_1 = -1/2) from sum_{k=0}^{m} C(m+1, k) B_k = 0
std::vector<double> bernoulli(int n) {
    std::vector<double> B(n + 1, 0.0);
    B[0] = 1.0;
    for (int m = 1; m <= n; ++m) {
        double s = 0.0, c = 1.0;  // c = C(m+1, k)
        for (int k = 0; k < m; ++k) {
            s += c * B[k];
            c = c * (double)(m + 1 - k) / (double)(k + 1);
        }
        B[m] = -s / (double)(m + 1);
        if (m >= 3 && (m & 1)) B[m] = 0.0;  // odd Bernoulli numbers beyond B_1 vanish
    }
    return B;
}

}  // namespace

int upload_polylog_tables() {
    const std::vector<double> B = bernoulli(kPolyTerms + 1);
    std::vector<double> fact(kPolyTerms + 3, 1.0);
    for (int i = 1; i < (int)fact.size(); ++i) fact[i] = fact[i - 1] * i;
    double c2[kPolyTerms + 1] = {0}, c3[kPolyTerms + 1] = {0};
    for (int m = 1; m <= kPolyTerms; ++m) {
        c2[m] = B[m - 1] / fact[m];  // u^m: k = m - 1
        double s = 0.0;
        for (int n = 0; n <= m - 1; ++n) {
            const int k = m - 1 - n;
            s += B[n] * B[k] / (fact[n + 1] * fact[k] * (double)m);
        }
        c3[m] = s;
    }
    MALA_CUDA_TRY(cudaMemcpyToSymbol(c_li2, c2, sizeof(c2)));
    MALA_CUDA_TRY(cudaMemcpyToSymbol(c_li3, c3, sizeof(c3)));
    return MALA_OK;
}

int electron_count_at(Ctx* c, const double* D_host, const mala_energy_grid* eg, double mu, double* out,
                      cudaStream_t st) {
    const int nE = eg->n_E;
    MALA_TRY(c->ws_w.reserve(c, sizeof(double) * (nE + 1)));
    double* d = c->ws_w.as<double>();
    MALA_CUDA_TRY(cudaMemcpyAsync(d, D_host, sizeof(double) * nE, cudaMemcpyHostToDevice, st));
    MALA_PROF(c, "k_count", st,
              (k_count<<<1, kFermiThreads, sizeof(double) * nE, st>>>(d, nE, eg->e0_eV, eg->de_eV, eg->kT_eV, mu, d + nE)));
    MALA_CUDA_TRY(cudaGetLastError());
    MALA_CUDA_TRY(cudaMemcpyAsync(c->host_scalars + 16, d + nE, sizeof(double), cudaMemcpyDeviceToHost, st));
    MALA_CUDA_TRY(cudaStreamSynchronize(st));
    *out = c->host_scalars[16];
    return MALA_OK;
}

int energy_gradient(Ctx* c, const double* dos_sum, double dV, const mala_energy_grid* eg, double gscale,
                    double* g_dev, double* fermi, double* mu_tilde, cudaStream_t st) {
    const int nE = eg->n_E;
    // workspace: D[nE] | w0d[nE] | w0f[nE] (float) | scal[16] | fstate (+ 6 nE interval weights) | mom[3 nE]
    const size_t doubles = 2 * (size_t)nE + (nE + 1) / 2 + 16 + kFermiStateDoubles + 6 * (size_t)nE + 3 * (size_t)nE;
    MALA_TRY(c->ws_force_g.reserve(c, sizeof(double) * doubles));
    double* D = c->ws_force_g.as<double>();
    double* w0d = D + nE;
    float* w0f = reinterpret_cast<float*>(w0d + nE);
    double* scal = w0d + nE + (nE + 1) / 2;
    double* fstate = scal + 16;
    double* mom = fstate + kFermiStateDoubles + 6 * (size_t)nE;
    MALA_PROF(c, "k_fermi", st, launch_fermi(dos_sum, nE, dV, eg, D, w0d, w0f, scal, fstate, st));
    MALA_PROF(c, "k_egrad", st,
              (k_egrad<<<1, kFermiThreads, 0, st>>>(D, nE, eg->e0_eV, eg->de_eV, eg->kT_eV, scal, gscale, mom, g_dev,
                                                    scal + 8)));
    MALA_CUDA_TRY(cudaGetLastError());
    MALA_CUDA_TRY(cudaMemcpyAsync(c->host_scalars, scal, sizeof(double) * 9, cudaMemcpyDeviceToHost, st));
    MALA_CUDA_TRY(cudaStreamSynchronize(st));
    const double* hs = c->host_scalars;
    if (fermi) *fermi = hs[0];
    if (mu_tilde) *mu_tilde = hs[8];
    if (hs[2] != 0.0)
        return fail(MALA_ERR_FERMI_BRACKET, "N(mu) - N_e has no sign change on [e0 - 20 kT, e_max + 20 kT]");
    if (!std::isfinite(hs[8]))
        return fail(MALA_ERR_UNSUPPORTED, "dN/dmu = 0 at the Fermi level: dE_b/dD is undefined");
    return MALA_OK;
}

// doubles of the workspace of integrate(): dsum | D | w0d | w0f | scal | fstate | partial rows
static size_t integrate_doubles(int64_t P, int nE, bool mixed, int num_sms) {
    const int64_t ntile = (P + 127) / 128;
    const int dens_blocks = density_grid(P, nE, mixed ? 2 : 8, num_sms);
    const size_t n_part = std::max<size_t>((size_t)ntile * nE, (size_t)dens_blocks);
    return 3 * (size_t)nE + (nE + 1) / 2 + 16 + kFermiStateDoubles + 6 * (size_t)nE + n_part;
}

void integrate_ws_needs(Ctx* c, int64_t P, int nE, mala_precision prec, WsNeeds& out) {
    out.add(c->ws_red, sizeof(double) * integrate_doubles(P, nE, prec == MALA_MIXED, c->num_sms));
}

// error flags of the network (err_d[1]) and density (err_d[2]) kernels, read
// into host_ints[8..9] by the caller's last copy; reset once reported
static int check_device_flags(Ctx* c, cudaStream_t st) {
    const int mlp = c->host_ints[8], dens = c->host_ints[9];
    if (!mlp && !dens) return MALA_OK;
    cudaMemsetAsync(c->tables.err_d + 1, 0, sizeof(int) * 2, st);
    cudaStreamSynchronize(st);
    if (mlp) return fail(MALA_ERR_TIMEOUT, "network kernel: a wait on a shared-memory barrier expired (code %d)", mlp);
    return fail(MALA_ERR_TIMEOUT, "density pass: a copy into shared memory did not complete in time");
}

int integrate(Ctx* c, const void* ldos, int64_t P, double volume, const mala_energy_grid* eg, const double* dos_sum,
              void* density, double* dos_host, double* fermi, double* eb, double* ne, double* ts, mala_precision prec,
              cudaStream_t st) {
    const int nE = eg->n_E;
    // workspace: dsum[nE] | D[nE] | w0d[nE] | w0f[nE] (float) | scal[8] | nsum[1] | partial rows
    const int64_t ntile = (P + 127) / 128;
    const bool mixed = prec == MALA_MIXED;
    const int dens_blocks = density_grid(P, nE, mixed ? 2 : 8, c->num_sms);
    MALA_TRY(c->ws_red.reserve(c, sizeof(double) * integrate_doubles(P, nE, mixed, c->num_sms)));
    double* dsum = c->ws_red.as<double>();
    double* D = dsum + nE;
    double* w0d = D + nE;
    float* w0f = reinterpret_cast<float*>(w0d + nE);
    double* scal = w0d + nE + (nE + 1) / 2;
    double* nsum = scal + 8;
    double* fstate = scal + 16;
    double* part = fstate + kFermiStateDoubles + 6 * (size_t)nE;
    if (!dos_sum) {
        if (P > 0) {
            if (mixed)
                MALA_PROF(c, "k_dos_reduce", st,
                          (k_colsum<__nv_bfloat16><<<(unsigned)ntile, 256, 0, st>>>(
                              static_cast<const __nv_bfloat16*>(ldos), P, nE, part)));
            else
                MALA_PROF(c, "k_dos_reduce", st,
                          (k_colsum<double><<<(unsigned)ntile, 256, 0, st>>>(static_cast<const double*>(ldos), P, nE,
                                                                            part)));
            MALA_PROF(c, "k_sum_rows", st, (k_sum_rows<<<nE, kSumRowsThreads, 0, st>>>(part, ntile, nE, dsum)));
        } else {
            MALA_CUDA_TRY(cudaMemsetAsync(dsum, 0, sizeof(double) * nE, st));
        }
        dos_sum = dsum;
    }
    const double dV = volume / (double)(P > 0 ? P : 1);
    MALA_PROF(c, "k_fermi", st, launch_fermi(dos_sum, nE, dV, eg, D, w0d, w0f, scal, fstate, st));
    if (P > 0 && density) {
        int* derr = c->tables.err_d + 2;
        if (mixed)
            MALA_PROF(c, "k_density", st,
                      (launch_density<__nv_bfloat16, float>(static_cast<const __nv_bfloat16*>(ldos), P, nE, w0f,
                                                            static_cast<float*>(density), part, dens_blocks, derr, st)));
        else
            MALA_PROF(c, "k_density", st,
                      (launch_density<double, double>(static_cast<const double*>(ldos), P, nE, w0d,
                                                      static_cast<double*>(density), part, dens_blocks, derr, st)));
        MALA_PROF(c, "k_sum_vec", st, (k_sum_vec<<<1, 256, 0, st>>>(part, dens_blocks, nsum)));
    } else {
        MALA_CUDA_TRY(cudaMemsetAsync(nsum, 0, sizeof(double), st));
    }
    MALA_CUDA_TRY(cudaGetLastError());
    if (c->host_dos_len < (size_t)nE) {
        if (c->host_dos) cudaFreeHost(c->host_dos);
        c->host_dos = nullptr;
        c->host_dos_len = 0;
        MALA_CUDA_TRY(cudaMallocHost(&c->host_dos, sizeof(double) * nE));
        c->host_dos_len = nE;
    }
    MALA_CUDA_TRY(cudaMemcpyAsync(c->host_scalars, scal, sizeof(double) * 9, cudaMemcpyDeviceToHost, st));
    MALA_CUDA_TRY(cudaMemcpyAsync(c->host_dos, D, sizeof(double) * nE, cudaMemcpyDeviceToHost, st));
    MALA_CUDA_TRY(cudaMemcpyAsync(c->host_ints + 8, c->tables.err_d + 1, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
    MALA_CUDA_TRY(cudaStreamSynchronize(st));
    MALA_TRY(check_device_flags(c, st));
    if (dos_host) memcpy(dos_host, c->host_dos, sizeof(double) * nE);
    const double* hs = c->host_scalars;
    if (fermi) *fermi = hs[0];
    if (eb) *eb = hs[1];
    if (ne) *ne = dV * hs[8];
    if (ts) *ts = hs[5];
    if (hs[2] != 0.0)
        return fail(MALA_ERR_FERMI_BRACKET, "N(mu) - N_e has no sign change on [e0 - 20 kT, e_max + 20 kT]");
    return MALA_OK;
}

}  // namespace mala

// ---- the integration step without allocation -------------------------------
//
// Callers that must not allocate device memory (a process whose device memory
// is owned by another framework's allocator, a hard per-process memory cap, or
// a latency-critical loop that cannot afford the device-wide synchronisation
// cudaMalloc/cudaFree may imply) run the integrals with every scratch buffer
// taken from this fixed file-scope array instead of the context's workspaces.
// Every GPU that loads the library holds the array until the process exits.

namespace mala {

namespace {

constexpr size_t kStaticScratchDoubles = size_t(1) << 20;  // 8 MiB
static __device__ __align__(256) double g_integrate_scratch[kStaticScratchDoubles];

// Device address of the array in the current device's context, looked up on
// every call: the lookup is a host-side query that allocates nothing, and a
// cached address would go stale after a device reset or in another driver
// context.  (In host code the array's name is only a host-side stand-in.)
int scratch_address(double** out) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_integrate_scratch);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return fail(MALA_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
    }
    *out = static_cast<double*>(p);
    return MALA_OK;
}

}  // namespace

int integrate_noalloc(Ctx* c, const void* ldos, int64_t P, double volume, const mala_energy_grid* eg,
                      const double* dos_sum, void* density, double* dos_host, double* fermi, double* eb, double* ne,
                      double* ts, mala_precision prec, cudaStream_t st) {
    const int nE = eg->n_E;
    double* scratch = nullptr;
    MALA_TRY(scratch_address(&scratch));
    const int64_t ntile = (P + 127) / 128;
    const bool mixed = prec == MALA_MIXED;
    const int dens_blocks = density_grid(P, nE, mixed ? 2 : 8, c->num_sms);
    const size_t n_part = std::max<size_t>(dos_sum ? 0 : (size_t)ntile * nE, (size_t)dens_blocks);
    const size_t need = 3 * (size_t)nE + (nE + 1) / 2 + 16 + kFermiStateDoubles + 6 * (size_t)nE + n_part;
    if (need > kStaticScratchDoubles)
        return fail(MALA_ERR_UNSUPPORTED,
                    "mala_integrate_noalloc: %zu scratch doubles needed, the static array holds %zu "
                    "(ceil(P/128) * n_E must stay below about %zu when dos_sum_dev is NULL)",
                    need, kStaticScratchDoubles,
                    kStaticScratchDoubles - 9 * (size_t)nE - nE / 2 - 16 - kFermiStateDoubles);
    // the same layout as the workspace path; every buffer is rewritten before it is read
    double* dsum = scratch;
    double* D = dsum + nE;
    double* w0d = D + nE;
    float* w0f = reinterpret_cast<float*>(w0d + nE);
    double* scal = w0d + nE + (nE + 1) / 2;
    double* nsum = scal + 8;
    double* fstate = scal + 16;
    double* part = fstate + kFermiStateDoubles + 6 * (size_t)nE;
    if (!dos_sum) {
        if (P > 0) {
            if (mixed)
                k_colsum<__nv_bfloat16><<<(unsigned)ntile, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(ldos), P,
                                                                          nE, part);
            else
                k_colsum<double><<<(unsigned)ntile, 256, 0, st>>>(static_cast<const double*>(ldos), P, nE, part);
            k_sum_rows<<<nE, kSumRowsThreads, 0, st>>>(part, ntile, nE, dsum);
        } else {
            MALA_CUDA_TRY(cudaMemsetAsync(dsum, 0, sizeof(double) * nE, st));
        }
        dos_sum = dsum;
    }
    const double dV = volume / (double)(P > 0 ? P : 1);
    launch_fermi(dos_sum, nE, dV, eg, D, w0d, w0f, scal, fstate, st);
    if (P > 0 && density) {
        int* derr = c->tables.err_d + 2;
        if (mixed)
            launch_density<__nv_bfloat16, float>(static_cast<const __nv_bfloat16*>(ldos), P, nE, w0f,
                                                 static_cast<float*>(density), part, dens_blocks, derr, st);
        else
            launch_density<double, double>(static_cast<const double*>(ldos), P, nE, w0d, static_cast<double*>(density),
                                           part, dens_blocks, derr, st);
        k_sum_vec<<<1, 256, 0, st>>>(part, dens_blocks, nsum);
    } else {
        MALA_CUDA_TRY(cudaMemsetAsync(nsum, 0, sizeof(double), st));
    }
    MALA_CUDA_TRY(cudaGetLastError());
    // host results: scalars through the context's pinned buffer, D straight into the caller's array
    MALA_CUDA_TRY(cudaMemcpyAsync(c->host_scalars, scal, sizeof(double) * 9, cudaMemcpyDeviceToHost, st));
    if (dos_host) MALA_CUDA_TRY(cudaMemcpyAsync(dos_host, D, sizeof(double) * nE, cudaMemcpyDeviceToHost, st));
    MALA_CUDA_TRY(cudaMemcpyAsync(c->host_ints + 8, c->tables.err_d + 1, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
    MALA_CUDA_TRY(cudaStreamSynchronize(st));
    MALA_TRY(check_device_flags(c, st));
    const double* hs = c->host_scalars;
    if (fermi) *fermi = hs[0];
    if (eb) *eb = hs[1];
    if (ne) *ne = dV * hs[8];
    if (ts) *ts = hs[5];
    if (hs[2] != 0.0)
        return fail(MALA_ERR_FERMI_BRACKET, "N(mu) - N_e has no sign change on [e0 - 20 kT, e_max + 20 kT]");
    return MALA_OK;
}

}  // namespace mala
