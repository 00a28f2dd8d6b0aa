/*
 * mala_oracle.c -- plain, slow, FP64 CPU oracle for the grid-bispectrum
 * descriptor step of the MALA inference path (arxiv 2411.19617).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA library; neither includes the other.
 *
 * What it computes, in the paper's order (Sec. "Bispectrum descriptors"):
 *   1. the real-space grid point r_ijk = (i/Nx) a1 + (j/Ny) a2 + (k/Nz) a3 of an
 *      orthorhombic cell (reading: the paper gives no grid convention);
 *   2. the atoms (with periodic images) inside the cutoff sphere of r, the
 *      strict test |R_a - r| < R_cut of Eq. (ionicdensity), brute force over
 *      every atom and every image shift;
 *   3. the expansion coefficients u_j of the ionic density of Eq. (ionicdensity)
 *      in the hyperspherical harmonics U_j of Eq. (SNAPExpansion): the delta(0)
 *      self term plus sum_a w_a f_c(|R_a - r|) U_j(R_a - r).  U_j is the
 *      spin-j representation of the SU(2) element given by the Cayley-Klein
 *      parameters of the neighbour offset, written out EXPLICITLY by binomial
 *      expansion (no recursion in j);
 *   4. the bispectrum components B_{j1 j2 j}: the "scalar triple products" of
 *      the u_j coupled with Clebsch-Gordan coefficients (Racah's closed form),
 *      over the index set whose size is Eq. (snap_dim).
 *
 * Readings where the paper is silent:
 *   - cutoff function f_c(r) = (cos(pi (r-rmin0)/(rcut-rmin0)) + 1)/2 and the
 *     angle omega = rfac0 pi (r-rmin0)/(rcut-rmin0) of the SNAP formalism the
 *     paper cites;
 *   - Cayley-Klein a = cos(omega) - i (z/r) sin(omega), b = (y - i x)/r sin(omega);
 *     a = 1, b = 0 at r = 0;
 *   - U^J[ma][mb] (ma, mb = 0..J, J = 2j) is the coefficient of
 *     xi^(J-ma) eta^ma in (conj(a) xi - conj(b) eta)^(J-mb) (b xi + a eta)^mb,
 *     times sqrt((J-ma)! ma! / ((J-mb)! mb!));
 *   - m = ma - J/2 couples the matrix index to the Clebsch-Gordan label;
 *   - Z^{j1j2j}_{m m'} = sum C^{j m}_{j1 m1 j2 m-m1} C^{j m'}_{j1 m1' j2 m'-m1'}
 *                         u^{j1}_{m1 m1'} u^{j2}_{m-m1, m'-m1'},
 *     B_{j1 j2 j} = sum_{m m'} Re(conj(u^j_{m m'}) Z^{j1j2j}_{m m'}),
 *     no normalisation, no B_0 subtraction;
 *   - index set 0 <= J2 <= J1 <= twojmax, |J1-J2| <= J <= min(twojmax, J1+J2),
 *     J1+J2+J even, J >= J1, ordered lexicographically in (J1, J2, J).
 *
 * Build with -ffp-contract=off: the neighbour test must round exactly like
 * the plain IEEE expression it is written as.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAX_TWOJ 14

/* ------------------------------------------------------------------ */
/* index set, Eq. (snap_dim)                                           */
/* ------------------------------------------------------------------ */

/* Writes the (J1, J2, J) triples (twice-units) in lexicographic order into
 * out[3*n] when out != NULL; returns their number. */
int oracle_bispectrum_triples(int twojmax, int32_t* out)
{
    int n = 0;
    for (int j1 = 0; j1 <= twojmax; ++j1)
        for (int j2 = 0; j2 <= j1; ++j2)
            for (int j = j1 - j2; j <= j1 + j2 && j <= twojmax; j += 2) {
                if (j < j1) continue;
                if (out) { out[3 * n] = j1; out[3 * n + 1] = j2; out[3 * n + 2] = j; }
                ++n;
            }
    return n;
}

/* ------------------------------------------------------------------ */
/* Clebsch-Gordan coefficients, Racah's closed form (Condon-Shortley)   */
/* ------------------------------------------------------------------ */

static long double fact_ld(int n)
{
    long double f = 1.0L;
    for (int i = 2; i <= n; ++i) f *= (long double)i;
    return f;
}

/* <j1 m1 j2 m2 | j m>, every argument in twice-units (j1 = 2*j1_phys, ...). */
double oracle_clebsch_gordan(int j1, int m1, int j2, int m2, int j, int m)
{
    if (m1 + m2 != m) return 0.0;
    if (abs(m1) > j1 || abs(m2) > j2 || abs(m) > j) return 0.0;
    if (((j1 + m1) & 1) || ((j2 + m2) & 1) || ((j + m) & 1)) return 0.0;
    if (j < abs(j1 - j2) || j > j1 + j2 || ((j1 + j2 + j) & 1)) return 0.0;
    const int a = (j1 + j2 - j) / 2, b = (j1 - j2 + j) / 2, c = (-j1 + j2 + j) / 2;
    const int d = (j1 + j2 + j) / 2 + 1;
    long double pre = (long double)(j + 1) * fact_ld(a) * fact_ld(b) * fact_ld(c) / fact_ld(d);
    pre *= fact_ld((j1 + m1) / 2) * fact_ld((j1 - m1) / 2) * fact_ld((j2 + m2) / 2) *
           fact_ld((j2 - m2) / 2) * fact_ld((j + m) / 2) * fact_ld((j - m) / 2);
    long double s = 0.0L;
    for (int k = 0; k <= a; ++k) {
        const int d1 = (j1 - m1) / 2 - k, d2 = (j2 + m2) / 2 - k;
        const int d3 = (j - j2 + m1) / 2 + k, d4 = (j - j1 - m2) / 2 + k;
        if (d1 < 0 || d2 < 0 || d3 < 0 || d4 < 0) continue;
        long double t = fact_ld(k) * fact_ld(a - k) * fact_ld(d1) * fact_ld(d2) *
                        fact_ld(d3) * fact_ld(d4);
        s += ((k & 1) ? -1.0L : 1.0L) / t;
    }
    return (double)(sqrtl(pre) * s);
}

/* ------------------------------------------------------------------ */
/* Explicit spin-J/2 representation U^J of an SU(2) element            */
/* ------------------------------------------------------------------ */

typedef struct { double re, im; } cplx;

static cplx cmul(cplx x, cplx y) { cplx r = {x.re * y.re - x.im * y.im, x.re * y.im + x.im * y.re}; return r; }
static cplx cadd(cplx x, cplx y) { cplx r = {x.re + y.re, x.im + y.im}; return r; }
static cplx cscale(cplx x, double s) { cplx r = {x.re * s, x.im * s}; return r; }

static double binom_d(int n, int k)
{
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

/* U^J of M = [[p, q], [r, s]] (the rows are the two linear forms):
 * U[ma][mb] = sqrt((J-ma)! ma! / ((J-mb)! mb!)) *
 *             [xi^(J-ma) eta^ma] (p xi + q eta)^(J-mb) (r xi + s eta)^mb.
 * out: (J+1)*(J+1) complex numbers, row-major [ma][mb], interleaved re/im. */
void oracle_su2_rep(int J, const double* pqrs /* p,q,r,s as re,im pairs */, double* out)
{
    cplx p = {pqrs[0], pqrs[1]}, q = {pqrs[2], pqrs[3]};
    cplx r = {pqrs[4], pqrs[5]}, s = {pqrs[6], pqrs[7]};
    cplx pw_p[ORACLE_MAX_TWOJ + 1], pw_q[ORACLE_MAX_TWOJ + 1];
    cplx pw_r[ORACLE_MAX_TWOJ + 1], pw_s[ORACLE_MAX_TWOJ + 1];
    cplx one = {1.0, 0.0};
    pw_p[0] = pw_q[0] = pw_r[0] = pw_s[0] = one;
    for (int k = 1; k <= J; ++k) {
        pw_p[k] = cmul(pw_p[k - 1], p); pw_q[k] = cmul(pw_q[k - 1], q);
        pw_r[k] = cmul(pw_r[k - 1], r); pw_s[k] = cmul(pw_s[k - 1], s);
    }
    for (int mb = 0; mb <= J; ++mb) {
        /* coefficients of the product polynomial, indexed by the power of eta */
        cplx poly[ORACLE_MAX_TWOJ + 1];
        for (int k = 0; k <= J; ++k) { poly[k].re = 0.0; poly[k].im = 0.0; }
        for (int k1 = 0; k1 <= J - mb; ++k1) {
            cplx c1 = cscale(cmul(pw_p[J - mb - k1], pw_q[k1]), binom_d(J - mb, k1));
            for (int k2 = 0; k2 <= mb; ++k2) {
                cplx c2 = cscale(cmul(pw_r[mb - k2], pw_s[k2]), binom_d(mb, k2));
                poly[k1 + k2] = cadd(poly[k1 + k2], cmul(c1, c2));
            }
        }
        for (int ma = 0; ma <= J; ++ma) {
            double nrm = sqrt((double)(fact_ld(J - ma) * fact_ld(ma) /
                                       (fact_ld(J - mb) * fact_ld(mb))));
            cplx v = cscale(poly[ma], nrm);
            out[2 * (ma * (J + 1) + mb)] = v.re;
            out[2 * (ma * (J + 1) + mb) + 1] = v.im;
        }
    }
}

/* U^J(a, b): the matrix M = [[conj(a), -conj(b)], [b, a]]. */
void oracle_wigner_u(int J, double ar, double ai, double br, double bi, double* out)
{
    double pqrs[8] = {ar, -ai, -br, bi, br, bi, ar, ai};
    oracle_su2_rep(J, pqrs, out);
}

/* Cayley-Klein parameters and cutoff weight of an offset (dx, dy, dz). */
void oracle_cayley_klein(double dx, double dy, double dz, double rcut, double rfac0,
                         double rmin0, double* ab /* ar, ai, br, bi */, double* fc)
{
    const double pi = 3.14159265358979323846;
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    double t = (r - rmin0) / (rcut - rmin0);
    *fc = 0.5 * (cos(pi * t) + 1.0);
    if (r == 0.0) { ab[0] = 1.0; ab[1] = 0.0; ab[2] = 0.0; ab[3] = 0.0; return; }
    double om = rfac0 * pi * t;
    double so = sin(om), co = cos(om);
    ab[0] = co;
    ab[1] = -dz / r * so;
    ab[2] = dy / r * so;
    ab[3] = -dx / r * so;
}

/* ------------------------------------------------------------------ */
/* Staging and neighbours                                              */
/* ------------------------------------------------------------------ */

/* Wrap Cartesian positions into an orthorhombic cell along periodic axes:
 * x - L floor(x / L) in plain IEEE FP64. */
void oracle_wrap_positions(int natoms, const double* pos, const double* L, const int32_t* periodic,
                           double* out)
{
    for (int a = 0; a < natoms; ++a)
        for (int d = 0; d < 3; ++d) {
            double x = pos[3 * a + d];
            if (periodic[d]) {
                double fl = floor(x / L[d]);
                double t = L[d] * fl;
                x = x - t;
            }
            out[3 * a + d] = x;
        }
}

/* Grid point of flat index p = ix + Nx (iy + Ny iz): r_d = (i_d / N_d) L_d. */
void oracle_grid_point(int64_t p, const int32_t* grid, const double* L, double* r)
{
    int64_t ix = p % grid[0];
    int64_t iy = (p / grid[0]) % grid[1];
    int64_t iz = p / ((int64_t)grid[0] * grid[1]);
    double fx = (double)ix / (double)grid[0];
    double fy = (double)iy / (double)grid[1];
    double fz = (double)iz / (double)grid[2];
    r[0] = fx * L[0];
    r[1] = fy * L[1];
    r[2] = fz * L[2];
}

/* All (atom, image) pairs with |R_a + s L - r| < rcut, brute force over every
 * atom and every shift |s_d| <= ceil(rcut / L_d) + 1 (0 along open axes), in
 * the order (atom, s_x, s_y, s_z).  `wpos` are wrapped positions.  Writes up to
 * `cap` entries (atom into atoms[], shift into shifts[3*k]) and offsets
 * (dx, dy, dz) into offs[3*k] when offs != NULL; returns the full count. */
int oracle_neighbors_at(int natoms, const double* wpos, const double* L, const int32_t* periodic,
                        double rcut, const double* r, int cap, int32_t* atoms, int32_t* shifts,
                        double* offs)
{
    int smax[3];
    for (int d = 0; d < 3; ++d) smax[d] = periodic[d] ? (int)ceil(rcut / L[d]) + 1 : 0;
    const double rc2 = rcut * rcut;
    int n = 0;
    for (int a = 0; a < natoms; ++a)
        for (int sx = -smax[0]; sx <= smax[0]; ++sx)
            for (int sy = -smax[1]; sy <= smax[1]; ++sy)
                for (int sz = -smax[2]; sz <= smax[2]; ++sz) {
                    double tx = (double)sx * L[0], ty = (double)sy * L[1], tz = (double)sz * L[2];
                    double ux = wpos[3 * a] + tx, uy = wpos[3 * a + 1] + ty, uz = wpos[3 * a + 2] + tz;
                    double dx = ux - r[0], dy = uy - r[1], dz = uz - r[2];
                    double xx = dx * dx, yy = dy * dy, zz = dz * dz;
                    double d2 = (xx + yy) + zz;
                    if (!(d2 < rc2)) continue;
                    if (n < cap) {
                        if (atoms) atoms[n] = a;
                        if (shifts) { shifts[3 * n] = sx; shifts[3 * n + 1] = sy; shifts[3 * n + 2] = sz; }
                        if (offs) { offs[3 * n] = dx; offs[3 * n + 1] = dy; offs[3 * n + 2] = dz; }
                    }
                    ++n;
                }
    return n;
}

/* ------------------------------------------------------------------ */
/* u_j, Z and B at one point                                           */
/* ------------------------------------------------------------------ */

typedef struct {
    int twojmax;
    double rcut, rfac0, rmin0, wself;
    int nspecies;
    const double* weights;
} oracle_bparams;

static int ublock_offset(int J) { int o = 0; for (int k = 0; k < J; ++k) o += (k + 1) * (k + 1); return o; }

/* u^J for J = 0..twojmax at one point from its neighbour offsets and weights;
 * u: sum_J (J+1)^2 complex numbers (interleaved), blocks in increasing J. */
void oracle_ui(const oracle_bparams* bp, int nnbr, const double* offs, const double* wts, double* u)
{
    const int tj = bp->twojmax;
    const int nu = ublock_offset(tj + 1);
    memset(u, 0, sizeof(double) * 2 * (size_t)nu);
    for (int J = 0; J <= tj; ++J) {
        double* uJ = u + 2 * ublock_offset(J);
        for (int ma = 0; ma <= J; ++ma) uJ[2 * (ma * (J + 1) + ma)] = bp->wself;
    }
    double Ub[2 * (ORACLE_MAX_TWOJ + 1) * (ORACLE_MAX_TWOJ + 1)];
    for (int k = 0; k < nnbr; ++k) {
        double ab[4], fc;
        oracle_cayley_klein(offs[3 * k], offs[3 * k + 1], offs[3 * k + 2], bp->rcut, bp->rfac0,
                            bp->rmin0, ab, &fc);
        double c = wts[k] * fc;
        for (int J = 0; J <= tj; ++J) {
            oracle_wigner_u(J, ab[0], ab[1], ab[2], ab[3], Ub);
            double* uJ = u + 2 * ublock_offset(J);
            for (int e = 0; e < (J + 1) * (J + 1); ++e) {
                uJ[2 * e] += c * Ub[2 * e];
                uJ[2 * e + 1] += c * Ub[2 * e + 1];
            }
        }
    }
}

/* Clebsch-Gordan table of one twojmax: for triple t, entry [ma][m1a] holds
 * C^{j m}_{j1 m1, j2 m-m1} with m = ma - j/2, m1 = m1a - j1/2 (0 where the
 * coupling is forbidden).  The values are the closed form above; the table
 * only avoids re-evaluating it inside the contraction. */
typedef struct { int ntr; int32_t* tr; int* off; double* c; } oracle_cgtab;

static void cgtab_build(int twojmax, oracle_cgtab* T)
{
    T->ntr = oracle_bispectrum_triples(twojmax, NULL);
    T->tr = (int32_t*)malloc(sizeof(int32_t) * 3 * (size_t)T->ntr);
    oracle_bispectrum_triples(twojmax, T->tr);
    T->off = (int*)malloc(sizeof(int) * (size_t)(T->ntr + 1));
    int n = 0;
    for (int t = 0; t < T->ntr; ++t) { T->off[t] = n; n += (T->tr[3 * t + 2] + 1) * (T->tr[3 * t] + 1); }
    T->off[T->ntr] = n;
    T->c = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int t = 0; t < T->ntr; ++t) {
        const int j1 = T->tr[3 * t], j2 = T->tr[3 * t + 1], j = T->tr[3 * t + 2];
        for (int ma = 0; ma <= j; ++ma)
            for (int m1a = 0; m1a <= j1; ++m1a) {
                const int m = 2 * ma - j, m1 = 2 * m1a - j1;
                T->c[T->off[t] + ma * (j1 + 1) + m1a] = oracle_clebsch_gordan(j1, m1, j2, m - m1, j, m);
            }
    }
}

static void cgtab_free(oracle_cgtab* T) { free(T->tr); free(T->off); free(T->c); }

/* B_{j1 j2 j} from the u blocks, for every triple of the index set:
 * Z^{j1j2j}_{m m'} = sum_{m1, m1'} C^{j m}_{j1 m1 j2 m-m1} C^{j m'}_{j1 m1' j2 m'-m1'}
 *                    u^{j1}_{m1 m1'} u^{j2}_{m-m1, m'-m1'},
 * B = sum_{m m'} Re(conj(u^j_{m m'}) Z_{m m'}). */
static void bi_from_u_tab(const oracle_cgtab* T, const double* u, double* B)
{
    double Z[2 * (ORACLE_MAX_TWOJ + 1) * (ORACLE_MAX_TWOJ + 1)];
    for (int t = 0; t < T->ntr; ++t) {
        const int j1 = T->tr[3 * t], j2 = T->tr[3 * t + 1], j = T->tr[3 * t + 2];
        const double* cg = T->c + T->off[t];
        const double* u1 = u + 2 * ublock_offset(j1);
        const double* u2 = u + 2 * ublock_offset(j2);
        const double* uj = u + 2 * ublock_offset(j);
        for (int ma = 0; ma <= j; ++ma) {
            const int m = 2 * ma - j;
            for (int mb = 0; mb <= j; ++mb) {
                const int mp = 2 * mb - j;
                double zr = 0.0, zi = 0.0;
                for (int m1a = 0; m1a <= j1; ++m1a) {
                    const int m1 = 2 * m1a - j1, m2 = m - m1;
                    if (m2 < -j2 || m2 > j2) continue;
                    const int m2a = (m2 + j2) / 2;
                    const double c1 = cg[ma * (j1 + 1) + m1a];
                    for (int m1b = 0; m1b <= j1; ++m1b) {
                        const int m1p = 2 * m1b - j1, m2p = mp - m1p;
                        if (m2p < -j2 || m2p > j2) continue;
                        const int m2b = (m2p + j2) / 2;
                        const double c2 = cg[mb * (j1 + 1) + m1b];
                        const double ar = u1[2 * (m1a * (j1 + 1) + m1b)], ai = u1[2 * (m1a * (j1 + 1) + m1b) + 1];
                        const double br = u2[2 * (m2a * (j2 + 1) + m2b)], bi = u2[2 * (m2a * (j2 + 1) + m2b) + 1];
                        const double pr = ar * br - ai * bi, pi = ar * bi + ai * br;
                        zr += c1 * c2 * pr;
                        zi += c1 * c2 * pi;
                    }
                }
                Z[2 * (ma * (j + 1) + mb)] = zr;
                Z[2 * (ma * (j + 1) + mb) + 1] = zi;
            }
        }
        double b = 0.0;
        for (int e = 0; e < (j + 1) * (j + 1); ++e)
            b += uj[2 * e] * Z[2 * e] + uj[2 * e + 1] * Z[2 * e + 1];
        B[t] = b;
    }
}

void oracle_bi_from_u(int twojmax, const double* u, double* B)
{
    oracle_cgtab T;
    cgtab_build(twojmax, &T);
    bi_from_u_tab(&T, u, B);
    cgtab_free(&T);
}

/* ------------------------------------------------------------------ */
/* Whole grid (or a list of grid points)                               */
/* ------------------------------------------------------------------ */

/* Descriptors B[np][ntriples] at the grid points `points[np]` (flat indices;
 * NULL means 0..np-1) of an orthorhombic cell with side lengths L[3].
 * species[a] selects weights[species[a]] (NULL: weight 1).  Returns 0, or -1
 * on a bad argument.  Threads: nthreads > 0 requests an OpenMP team. */
int oracle_bispectrum_grid(int natoms, const double* pos, const int32_t* species, const double* L,
                           const int32_t* periodic, const int32_t* grid, int twojmax, double rcut,
                           double rfac0, double rmin0, double wself, int nspecies,
                           const double* weights, int64_t np, const int64_t* points, double* B,
                           int nthreads)
{
    if (twojmax < 0 || twojmax > ORACLE_MAX_TWOJ || rcut <= 0.0 || natoms < 0) return -1;
    oracle_bparams bp = {twojmax, rcut, rfac0, rmin0, wself, nspecies, weights};
    const int ntr = oracle_bispectrum_triples(twojmax, NULL);
    double* wpos = (double*)malloc(sizeof(double) * 3 * (size_t)(natoms > 0 ? natoms : 1));
    oracle_wrap_positions(natoms, pos, L, periodic, wpos);
    const int nu = ublock_offset(twojmax + 1);
    oracle_cgtab T;
    cgtab_build(twojmax, &T);
    int err = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
#endif
    for (int64_t i = 0; i < np; ++i) {
        int64_t p = points ? points[i] : i;
        double r[3];
        oracle_grid_point(p, grid, L, r);
        int cnt = oracle_neighbors_at(natoms, wpos, L, periodic, rcut, r, 0, NULL, NULL, NULL);
        int cap = cnt > 0 ? cnt : 1;
        int32_t* at = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
        double* offs = (double*)malloc(sizeof(double) * 3 * (size_t)cap);
        double* wts = (double*)malloc(sizeof(double) * (size_t)cap);
        double* u = (double*)malloc(sizeof(double) * 2 * (size_t)nu);
        oracle_neighbors_at(natoms, wpos, L, periodic, rcut, r, cap, at, NULL, offs);
        for (int k = 0; k < cnt; ++k) {
            int sp = species ? species[at[k]] : 0;
            wts[k] = weights ? weights[sp] : 1.0;
            if (species && (sp < 0 || sp >= nspecies)) err = 1;
        }
        oracle_ui(&bp, cnt, offs, wts, u);
        bi_from_u_tab(&T, u, B + (size_t)i * ntr);
        free(at); free(offs); free(wts); free(u);
    }
    cgtab_free(&T);
    free(wpos);
    return err ? -1 : 0;
}

/* u^J blocks at one grid point (for the identity tests). */
int oracle_u_at_point(int natoms, const double* pos, const int32_t* species, const double* L,
                      const int32_t* periodic, const int32_t* grid, int twojmax, double rcut,
                      double rfac0, double rmin0, double wself, int nspecies, const double* weights,
                      int64_t p, double* u)
{
    oracle_bparams bp = {twojmax, rcut, rfac0, rmin0, wself, nspecies, weights};
    double* wpos = (double*)malloc(sizeof(double) * 3 * (size_t)(natoms > 0 ? natoms : 1));
    oracle_wrap_positions(natoms, pos, L, periodic, wpos);
    double r[3];
    oracle_grid_point(p, grid, L, r);
    int cnt = oracle_neighbors_at(natoms, wpos, L, periodic, rcut, r, 0, NULL, NULL, NULL);
    int cap = cnt > 0 ? cnt : 1;
    int32_t* at = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
    double* offs = (double*)malloc(sizeof(double) * 3 * (size_t)cap);
    double* wts = (double*)malloc(sizeof(double) * (size_t)cap);
    oracle_neighbors_at(natoms, wpos, L, periodic, rcut, r, cap, at, NULL, offs);
    for (int k = 0; k < cnt; ++k) wts[k] = weights ? weights[species ? species[at[k]] : 0] : 1.0;
    oracle_ui(&bp, cnt, offs, wts, u);
    free(at); free(offs); free(wts); free(wpos);
    return cnt;
}

/* Neighbour lists of a set of grid points: counts[np]; atoms/shifts filled
 * row by row (row i starts at i*cap) up to cap entries per point. */
int oracle_neighbor_lists(int natoms, const double* pos, const double* L, const int32_t* periodic,
                          const int32_t* grid, double rcut, int64_t np, const int64_t* points,
                          int cap, int32_t* counts, int32_t* atoms, int32_t* shifts)
{
    double* wpos = (double*)malloc(sizeof(double) * 3 * (size_t)(natoms > 0 ? natoms : 1));
    oracle_wrap_positions(natoms, pos, L, periodic, wpos);
    for (int64_t i = 0; i < np; ++i) {
        int64_t p = points ? points[i] : i;
        double r[3];
        oracle_grid_point(p, grid, L, r);
        counts[i] = oracle_neighbors_at(natoms, wpos, L, periodic, rcut, r, cap,
                                        atoms + (size_t)i * cap, shifts + (size_t)i * 3 * cap, NULL);
    }
    free(wpos);
    return 0;
}

/* Descriptors at arbitrary points from explicit neighbour offsets (no cell):
 * point i has counts[i] neighbours, offsets offs[3*k] and weights wts[k] for
 * k in [starts[i], starts[i]+counts[i]).  Used by the invariance tests. */
void oracle_bispectrum_offsets(int twojmax, double rcut, double rfac0, double rmin0, double wself,
                               int64_t np, const int64_t* starts, const int32_t* counts,
                               const double* offs, const double* wts, double* B)
{
    oracle_bparams bp = {twojmax, rcut, rfac0, rmin0, wself, 0, NULL};
    const int ntr = oracle_bispectrum_triples(twojmax, NULL);
    const int nu = ublock_offset(twojmax + 1);
    double* u = (double*)malloc(sizeof(double) * 2 * (size_t)nu);
    oracle_cgtab T;
    cgtab_build(twojmax, &T);
    for (int64_t i = 0; i < np; ++i) {
        oracle_ui(&bp, counts[i], offs + 3 * starts[i], wts + starts[i], u);
        bi_from_u_tab(&T, u, B + (size_t)i * ntr);
    }
    cgtab_free(&T);
    free(u);
}
