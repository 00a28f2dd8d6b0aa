"""FP64 CPU oracle for the MALA inference hot path (arxiv 2411.19617).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package.  It shares no
code with the CUDA library (``paper_2411_19617_gb300``) and imports nothing
from it; the two meet only through the seeded input generators in
``paper_2411_19617_gb300.workloads``, which hold none of the method's arithmetic.

Contents, each following the passage of the paper cited at the function:

* descriptors (C, ``mala_oracle.c``): neighbours by brute force, explicit
  SU(2) representation matrices, Racah Clebsch-Gordan coefficients, Z and B;
* ``gaussian_grid``: the Gaussian representation of the atoms on the grid
  (Sec. "Total energy calculation", Eq. structfact_function);
* ``mlp_forward``: the feed-forward network of Eq. (ffnn) in FP64;
* ``integration_weights``: w_xi = int hat_xi(e) e^n f_beta(e - mu) de for the
  piecewise-linear reading of the LDOS/DOS between energy-grid points
  (Eqs. ldosintegralgeneral / ldosintegralsummation) by adaptive Gauss-Kronrod
  quadrature (QUADPACK through scipy) -- independent of the closed forms in
  polylogarithms that the CUDA path evaluates;
* ``fermi_level``: bisection on N(mu) - N_e (Sec. "Observable calculation");
* ``observables``: D(e) of Eq. (DOS.from.ldos), n(r) of Eq. (density.from.ldos),
  the band energy of Eq. (band.energy) and the entropy contribution -tau S_s of
  Eq. (electronicentropyDOS) (``entropy_weights`` / ``entropy_term``);
* ``oracle.forces``: the band-energy forces of Eqs. (forces, forcesmala) --
  dE_b/dD at fixed N_e, the network's vector-Jacobian product and the
  descriptor adjoint, by torch autograd of a differentiable FP64 restatement;
* ``oracle.ace``: grid-centred ACE descriptors (Sec. "Atomic cluster expansion
  descriptors"): Chebyshev x spherical-harmonic grid basis and its N = 1, 2, 3
  invariants with generalized Clebsch-Gordan coefficients.

Parity pins for every function live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional, Sequence

import numpy as np

from .build import build_oracle

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build_oracle()
        L = ctypes.CDLL(path)
        i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
        f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
        i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
        vp = ctypes.c_void_p
        L.oracle_bispectrum_triples.argtypes = [ctypes.c_int, vp]
        L.oracle_bispectrum_triples.restype = ctypes.c_int
        L.oracle_clebsch_gordan.argtypes = [ctypes.c_int] * 6
        L.oracle_clebsch_gordan.restype = ctypes.c_double
        L.oracle_su2_rep.argtypes = [ctypes.c_int, f64p, f64p]
        L.oracle_wigner_u.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4 + [f64p]
        L.oracle_cayley_klein.argtypes = [ctypes.c_double] * 6 + [f64p, f64p]
        L.oracle_wrap_positions.argtypes = [ctypes.c_int, f64p, f64p, i32p, f64p]
        L.oracle_grid_point.argtypes = [ctypes.c_int64, i32p, f64p, f64p]
        L.oracle_neighbor_lists.argtypes = [ctypes.c_int, f64p, f64p, i32p, i32p, ctypes.c_double,
                                            ctypes.c_int64, vp, ctypes.c_int, i32p, i32p, i32p]
        L.oracle_bispectrum_grid.argtypes = [ctypes.c_int, f64p, vp, f64p, i32p, i32p, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_int, vp, ctypes.c_int64, vp,
                                             f64p, ctypes.c_int]
        L.oracle_bispectrum_grid.restype = ctypes.c_int
        L.oracle_u_at_point.argtypes = [ctypes.c_int, f64p, vp, f64p, i32p, i32p, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int, vp, ctypes.c_int64, f64p]
        L.oracle_u_at_point.restype = ctypes.c_int
        L.oracle_bispectrum_offsets.argtypes = [ctypes.c_int] + [ctypes.c_double] * 4 + [
            ctypes.c_int64, i64p, i32p, f64p, f64p, f64p]
        L.oracle_bi_from_u.argtypes = [ctypes.c_int, f64p, f64p]
        _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# --------------------------------------------------------------------------
# descriptors (Sec. "Bispectrum descriptors")
# --------------------------------------------------------------------------

def triples(twojmax: int) -> np.ndarray:
    """(J1, J2, J) index set in twice-units; its size is Eq. (snap_dim)."""
    n = lib().oracle_bispectrum_triples(int(twojmax), None)
    out = np.zeros((max(n, 1), 3), np.int32)
    lib().oracle_bispectrum_triples(int(twojmax), _ptr(out))
    return out[:n]


def clebsch_gordan(j1: int, m1: int, j2: int, m2: int, j: int, m: int) -> float:
    """<j1 m1 j2 m2 | j m>, twice-units, Racah's closed form."""
    return float(lib().oracle_clebsch_gordan(j1, m1, j2, m2, j, m))


def su2_rep(J: int, M: np.ndarray) -> np.ndarray:
    """Spin-J/2 representation of the 2x2 complex matrix M (explicit expansion)."""
    M = np.asarray(M, dtype=np.complex128)
    pqrs = np.array([M[0, 0].real, M[0, 0].imag, M[0, 1].real, M[0, 1].imag,
                     M[1, 0].real, M[1, 0].imag, M[1, 1].real, M[1, 1].imag], np.float64)
    out = np.zeros(2 * (J + 1) ** 2, np.float64)
    lib().oracle_su2_rep(int(J), pqrs, out)
    return (out[0::2] + 1j * out[1::2]).reshape(J + 1, J + 1)


def wigner_u(J: int, a: complex, b: complex) -> np.ndarray:
    """U^J(a, b), the representation of [[conj a, -conj b], [b, a]]."""
    out = np.zeros(2 * (J + 1) ** 2, np.float64)
    lib().oracle_wigner_u(int(J), a.real, a.imag, b.real, b.imag, out)
    return (out[0::2] + 1j * out[1::2]).reshape(J + 1, J + 1)


def cayley_klein(d: Sequence[float], rcut: float, rfac0: float, rmin0: float):
    ab = np.zeros(4)
    fc = np.zeros(1)
    lib().oracle_cayley_klein(float(d[0]), float(d[1]), float(d[2]), rcut, rfac0, rmin0, ab, fc)
    return complex(ab[0], ab[1]), complex(ab[2], ab[3]), float(fc[0])


def _cell_args(snap):
    L = np.ascontiguousarray(np.diag(snap.cell), dtype=np.float64)
    off = snap.cell - np.diag(np.diag(snap.cell))
    if np.any(off != 0.0):
        raise ValueError("the oracle handles orthorhombic cells only")
    return L, np.asarray(snap.periodic, np.int32), np.asarray(snap.grid, np.int32)


def wrap_positions(snap) -> np.ndarray:
    L, per, _ = _cell_args(snap)
    pos = np.ascontiguousarray(snap.pos, dtype=np.float64)
    out = np.zeros_like(pos)
    lib().oracle_wrap_positions(len(pos), pos, L, per, out)
    return out


def grid_point(snap, p: int) -> np.ndarray:
    L, _, grid = _cell_args(snap)
    r = np.zeros(3)
    lib().oracle_grid_point(int(p), grid, L, r)
    return r


def neighbor_lists(snap, rcut: float, points: Optional[np.ndarray] = None, cap: int = 512):
    """Brute-force neighbour lists: (counts[np], atoms[np][cap], shifts[np][cap][3])."""
    L, per, grid = _cell_args(snap)
    pos = np.ascontiguousarray(snap.pos, dtype=np.float64)
    if points is None:
        np_ = snap.n_points
        pts = None
    else:
        pts = np.ascontiguousarray(points, dtype=np.int64)
        np_ = len(pts)
    counts = np.zeros(np_, np.int32)
    atoms = np.zeros((np_, cap), np.int32)
    shifts = np.zeros((np_, cap, 3), np.int32)
    lib().oracle_neighbor_lists(len(pos), pos, L, per, grid, float(rcut), np_, _ptr(pts), cap,
                                counts, atoms, shifts)
    if np.any(counts > cap):
        raise ValueError("neighbour capacity exceeded")
    return counts, atoms, shifts


def gaussian_grid(snap, rcut: float, sigma: float, points: Optional[np.ndarray] = None) -> np.ndarray:
    """Gaussian descriptors: the Gaussian representation of the atomic positions
    sampled on the grid (Eq. structfact_function with f a Gaussian of width
    sigma): G(r) = sum over the neighbours (atom, image) of r within rcut (the
    exact membership rule of ``neighbor_lists``) of exp(-|R + sL - r|^2 / (2 sigma^2))."""
    L, _, grid = _cell_args(snap)
    pts = np.arange(snap.n_points) if points is None else np.asarray(points, np.int64)
    counts, atoms, shifts = neighbor_lists(snap, rcut, points=pts)
    wrapped = wrap_positions(snap)
    out = np.zeros(len(pts))
    for i, p in enumerate(pts):
        n = counts[i]
        if n == 0:
            continue
        r = grid_point(snap, int(p))
        d = wrapped[atoms[i, :n]] + shifts[i, :n] * np.asarray(L)[None, :] - r[None, :]
        out[i] = float(np.sum(np.exp(-np.sum(d * d, axis=1) / (2.0 * sigma * sigma))))
    return out


def bispectrum_grid(snap, bp, points: Optional[np.ndarray] = None, nthreads: int = 1) -> np.ndarray:
    """B[np][n_triples] in FP64 at the given flat grid indices (all if None)."""
    L, per, grid = _cell_args(snap)
    pos = np.ascontiguousarray(snap.pos, dtype=np.float64)
    sp = np.ascontiguousarray(snap.species, dtype=np.int32)
    w = np.ascontiguousarray(bp.weights, dtype=np.float64)
    if points is None:
        np_ = snap.n_points
        pts = None
    else:
        pts = np.ascontiguousarray(points, dtype=np.int64)
        np_ = len(pts)
    ntr = len(triples(bp.twojmax))
    B = np.zeros((max(np_, 1), ntr), np.float64)
    rc = lib().oracle_bispectrum_grid(len(pos), pos, _ptr(sp), L, per, grid, int(bp.twojmax),
                                      float(bp.rcut), float(bp.rfac0), float(bp.rmin0),
                                      float(bp.wself), len(w), _ptr(w), np_, _ptr(pts), B,
                                      int(nthreads))
    if rc != 0:
        raise ValueError("oracle_bispectrum_grid rejected its arguments")
    return B[:np_]


def u_at_point(snap, bp, p: int):
    """List of u^J matrices (J = 0..twojmax) at grid point p, and the neighbour count."""
    L, per, grid = _cell_args(snap)
    pos = np.ascontiguousarray(snap.pos, dtype=np.float64)
    sp = np.ascontiguousarray(snap.species, dtype=np.int32)
    w = np.ascontiguousarray(bp.weights, dtype=np.float64)
    tj = int(bp.twojmax)
    nu = sum((J + 1) ** 2 for J in range(tj + 1))
    u = np.zeros(2 * nu)
    cnt = lib().oracle_u_at_point(len(pos), pos, _ptr(sp), L, per, grid, tj, float(bp.rcut),
                                  float(bp.rfac0), float(bp.rmin0), float(bp.wself), len(w),
                                  _ptr(w), int(p), u)
    uc = u[0::2] + 1j * u[1::2]
    out, o = [], 0
    for J in range(tj + 1):
        out.append(uc[o:o + (J + 1) ** 2].reshape(J + 1, J + 1))
        o += (J + 1) ** 2
    return out, cnt


def bispectrum_offsets(twojmax: int, rcut: float, offsets: Sequence[np.ndarray],
                       weights: Optional[Sequence[np.ndarray]] = None, rfac0: float = 0.99363,
                       rmin0: float = 0.0, wself: float = 1.0) -> np.ndarray:
    """B for explicit neighbour-offset lists (one list per point, no cell)."""
    offs = [np.asarray(o, np.float64).reshape(-1, 3) for o in offsets]
    if weights is None:
        weights = [np.ones(len(o)) for o in offs]
    counts = np.array([len(o) for o in offs], np.int32)
    starts = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    flat = np.ascontiguousarray(np.concatenate(offs + [np.zeros((1, 3))]), np.float64)
    wts = np.ascontiguousarray(np.concatenate([np.asarray(w, np.float64) for w in weights] + [np.zeros(1)]))
    ntr = len(triples(twojmax))
    B = np.zeros((len(offs), ntr))
    lib().oracle_bispectrum_offsets(int(twojmax), float(rcut), float(rfac0), float(rmin0),
                                    float(wself), len(offs), starts, counts, flat, wts, B)
    return B


def bi_from_u(twojmax: int, u_blocks: Sequence[np.ndarray]) -> np.ndarray:
    flat = np.concatenate([np.asarray(b, np.complex128).ravel() for b in u_blocks])
    u = np.ascontiguousarray(np.stack([flat.real, flat.imag], axis=1).ravel())
    B = np.zeros(len(triples(twojmax)))
    lib().oracle_bi_from_u(int(twojmax), u, B)
    return B


# --------------------------------------------------------------------------
# network (Sec. "Machine learning with neural networks", Eq. ffnn)
# --------------------------------------------------------------------------

def mlp_forward(x: np.ndarray, W: Sequence[np.ndarray], b: Sequence[np.ndarray],
                leaky_slope: float = 0.01, in_shift: Optional[np.ndarray] = None,
                in_scale: Optional[np.ndarray] = None, activate_output: bool = False) -> np.ndarray:
    """x_{l+1} = sigma(W_l x_l + b_l) in FP64; sigma = LeakyReLU on hidden layers,
    identity on the output layer unless activate_output.  Optional input
    standardisation (x - shift) * scale before the first layer."""
    h = np.asarray(x, np.float64)
    if in_shift is not None:
        h = h - np.asarray(in_shift, np.float64)
    if in_scale is not None:
        h = h * np.asarray(in_scale, np.float64)
    n = len(W)
    for l in range(n):
        h = h @ np.asarray(W[l], np.float64).T + np.asarray(b[l], np.float64)
        if l < n - 1 or activate_output:
            h = np.where(h > 0.0, h, leaky_slope * h)
    return h


# --------------------------------------------------------------------------
# energy integrals (Sec. "Observable calculation")
# --------------------------------------------------------------------------

def fermi_dirac(e: np.ndarray, mu: float, kT: float) -> np.ndarray:
    """Eq. (fermidistribution): 1 / (1 + exp(beta (e - mu)))."""
    x = (np.asarray(e, np.float64) - mu) / kT
    return 0.5 * (1.0 - np.tanh(0.5 * x))


def integration_weights(order: int, e0: float, de: float, n_E: int, mu: float, kT: float) -> np.ndarray:
    """w_xi = int hat_xi(e) e^order f_beta(e - mu) de, xi = 0..n_E-1.

    hat_xi is the piecewise-linear interpolation basis on the uniform energy
    grid e_xi = e0 + xi de (zero outside [e_0, e_{n_E-1}]), so that
    sum_xi w_xi D_xi is the integral of Eq. (ldosintegralgeneral) of the
    interpolant.  Each (interval, hat) piece is integrated by QUADPACK's
    adaptive Gauss-Kronrod rule, split at mu when mu lies inside.
    """
    from scipy.integrate import quad

    w = np.zeros(n_E, np.float64)
    if n_E < 2:
        raise ValueError("need at least two energies")

    def f(e):
        x = (e - mu) / kT
        return 0.5 * (1.0 - math.tanh(0.5 * x))

    for i in range(n_E - 1):
        a = e0 + i * de
        bnd = e0 + (i + 1) * de
        pts = [mu] if a < mu < bnd else None
        left = lambda e, a=a, bnd=bnd: (bnd - e) / de * e ** order * f(e)
        right = lambda e, a=a, bnd=bnd: (e - a) / de * e ** order * f(e)
        for k, g in ((i, left), (i + 1, right)):
            val, _ = quad(g, a, bnd, points=pts, epsabs=1e-15, epsrel=1e-13, limit=200)
            w[k] += val
    return w


def electron_count(D: np.ndarray, mu: float, e0: float, de: float, kT: float) -> float:
    """N(mu) = sum_xi w^(0)_xi(mu) D_xi, Eq. (NumberElectrons_from_DOS)."""
    w0 = integration_weights(0, e0, de, len(D), mu, kT)
    return float(np.dot(w0, D))


class FermiBracketError(ValueError):
    pass


def fermi_level(D: np.ndarray, e0: float, de: float, kT: float, n_electrons: float,
                tol: float = 1e-12, max_iter: int = 200) -> float:
    """Root of N(mu) - N_e by bisection on [e_0 - 20 kT, e_max + 20 kT]; stops when
    the bracket is narrower than tol (eV) or after max_iter halvings and returns
    the midpoint (the paper names TOMS748 for the same root)."""
    D = np.asarray(D, np.float64)
    lo = e0 - 20.0 * kT
    hi = e0 + (len(D) - 1) * de + 20.0 * kT
    flo = electron_count(D, lo, e0, de, kT) - n_electrons
    fhi = electron_count(D, hi, e0, de, kT) - n_electrons
    if flo == 0.0:
        return lo
    if fhi == 0.0:
        return hi
    if (flo > 0) == (fhi > 0):
        raise FermiBracketError("N(mu) - N_e has no sign change on the bracket")
    for _ in range(max_iter):
        if hi - lo < tol:
            break
        mid = 0.5 * (lo + hi)
        fm = electron_count(D, mid, e0, de, kT) - n_electrons
        if fm == 0.0:
            return mid
        if (fm > 0) == (flo > 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


def entropy_weights(e0: float, de: float, n_E: int, mu: float, kT: float) -> np.ndarray:
    """w^S_xi = int hat_xi(e) s(beta (e - mu)) de with
    s = -[f ln f + (1 - f) ln(1 - f)], the integrand of Eq. (electronicentropyDOS)
    in units of k_B, for the piecewise-linear reading of D(e) between grid
    points.  s is computed from its definition with f = f_beta (terms with
    f = 0 or 1 vanish); each (interval, hat) piece by QUADPACK, split at mu."""
    from scipy.integrate import quad

    if n_E < 2:
        raise ValueError("need at least two energies")

    def s_of(e):
        x = (e - mu) / kT
        f = 0.5 * (1.0 - math.tanh(0.5 * x))
        g = 1.0 - f
        out = 0.0
        if f > 0.0:
            out -= f * math.log(f)
        if g > 0.0:
            out -= g * math.log(g)
        return out

    w = np.zeros(n_E, np.float64)
    for i in range(n_E - 1):
        a = e0 + i * de
        bnd = e0 + (i + 1) * de
        pts = [mu] if a < mu < bnd else None
        left = lambda e, bnd=bnd: (bnd - e) / de * s_of(e)
        right = lambda e, a=a: (e - a) / de * s_of(e)
        for k, g in ((i, left), (i + 1, right)):
            val, _ = quad(g, a, bnd, points=pts, epsabs=1e-15, epsrel=1e-13, limit=200)
            w[k] += val
    return w


def entropy_term(D: np.ndarray, mu: float, e0: float, de: float, kT: float) -> float:
    """The free-energy contribution -tau S_s of Eq. (KSfreeenergy) in eV, with
    S_s from Eq. (electronicentropyDOS): -kT sum_xi w^S_xi D_xi."""
    wS = entropy_weights(e0, de, len(D), mu, kT)
    return float(-kT * np.dot(wS, np.asarray(D, np.float64)))


def dos(ldos: np.ndarray, dV: float) -> np.ndarray:
    """Eq. (DOS.from.ldos) on the grid: D_xi = dV sum_r L(r, xi)."""
    return dV * np.sum(np.asarray(ldos, np.float64), axis=0)


def observables(ldos: np.ndarray, dV: float, e0: float, de: float, kT: float, n_electrons: float):
    """D(e), the Fermi level, the band energy (Eq. band.energy) and n(r)
    (Eq. density.from.ldos) from an LDOS array [P][N_E]."""
    L = np.asarray(ldos, np.float64)
    D = dos(L, dV)
    eF = fermi_level(D, e0, de, kT, n_electrons)
    w0 = integration_weights(0, e0, de, L.shape[1], eF, kT)
    w1 = integration_weights(1, e0, de, L.shape[1], eF, kT)
    n = L @ w0
    Eb = float(np.dot(w1, D))
    TS = entropy_term(D, eF, e0, de, kT)
    return {"dos": D, "fermi": eF, "band_energy": Eb, "entropy_term": TS, "density": n, "w0": w0, "w1": w1}
