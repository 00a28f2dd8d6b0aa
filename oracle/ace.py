"""FP64 CPU oracle for the grid-centred ACE descriptors (Sec. "Atomic cluster
expansion descriptors", Eqs. unweighted_ionicdensity, gridatom_basis, grid_base,
product_grid_basis, ace_grid).

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle``).

Readings (the paper fixes the structure, not the functions):
* grid basis A_{mu n l m}(r) = sum over neighbours alpha of species mu (all periodic
  images, |d| < r_cut, d = R_alpha - r; the brute-force lists of
  ``neighbor_lists``) of R_n(|d|) Y_l^m(d / |d|): the unweighted density of
  Eq. unweighted_ionicdensity has no element weights; its delta(0) term is the
  grid point itself, which belongs to no atomic species channel and adds nothing;
* radial basis R_n(r) = T_n(1 - 2 r / r_cut) f_c(r), f_c(r) = (1 + cos(pi r / r_cut)) / 2
  (Chebyshev polynomials of the first kind of the scaled distance, made to vanish
  smoothly at the cutoff);
* Y_l^m complex, orthonormal, Condon-Shortley phase; an atom on the grid point
  (|d| = 0) contributes to l = 0 only;
* invariants of body order N = 1, 2, 3 with the generalized Clebsch-Gordan
  coefficients of the couplings l1 (x) l2 -> L1, L1 (x) l3 -> 0:
    N = 1: B = A_{mu n 0 0};
    N = 2: B = sum_m <l m l -m | 0 0> A_{c1 l m} A_{c2 l -m};
    N = 3: B = sum_{m1 m2} <l1 m1 l2 m2 | l3 M> <l3 M l3 -M | 0 0> A_{c1 l1 m1} A_{c2 l2 m2} A_{c3 l3 -M};
  each real (the imaginary parts cancel for a real density when l1 + l2 + l3 is even).
* enumeration (the order of the output columns): N = 1 over channels (mu, n),
  n < nmax1; N = 2 over channel pairs c1 <= c2 of (mu, n), n < nmax2, then
  l = 0..lmax2; N = 3 over sorted triples c1 <= c2 <= c3 of channels (mu, n, l),
  n < nmax3, l <= lmax3 (lexicographic), with |l1 - l2| <= l3 <= l1 + l2 and
  l1 + l2 + l3 even.

Pins (tests/test_oracle_ace.py): spherical harmonics against scipy and the
addition theorem; single-neighbour closed forms of N = 2 and N = 3; invariance
under rotations of the neighbour offsets, permutations and lattice translations.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import clebsch_gordan, grid_point, neighbor_lists, wrap_positions


@dataclasses.dataclass
class AceParams:
    rcut: float
    n_species: int = 1
    nmax1: int = 8
    nmax2: int = 6
    lmax2: int = 6
    nmax3: int = 3
    lmax3: int = 4


def radial(n_max: int, r: np.ndarray, rcut: float) -> np.ndarray:
    """R_n(r) = T_n(1 - 2 r / rcut) (1 + cos(pi r / rcut)) / 2, n < n_max: [n_max][len(r)]."""
    r = np.asarray(r, np.float64)
    x = 1.0 - 2.0 * r / rcut
    fc = 0.5 * (1.0 + np.cos(math.pi * r / rcut))
    T = [np.ones_like(x), x.copy()]
    for n in range(2, max(n_max, 2)):
        T.append(2.0 * x * T[-1] - T[-2])
    return np.array(T[:n_max]) * fc[None, :]


def sph_harm(l: int, m: int, d: np.ndarray) -> np.ndarray:
    """Y_l^m(d / |d|) for offsets d [k][3] from the associated Legendre function
    (scipy's lpmv, Condon-Shortley phase): sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!)
    P_l^|m|(cos theta) e^{i |m| phi}, and Y_l^{-m} = (-1)^m conj(Y_l^m)."""
    from scipy.special import lpmv
    d = np.asarray(d, np.float64).reshape(-1, 3)
    r = np.sqrt(np.sum(d * d, axis=1))
    zero = r == 0.0
    rs = np.where(zero, 1.0, r)
    ct = np.where(zero, 1.0, d[:, 2] / rs)
    phi = np.arctan2(d[:, 1], d[:, 0])
    am = abs(m)
    nrm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
    y = nrm * lpmv(am, l, np.clip(ct, -1.0, 1.0)) * np.exp(1j * am * phi)
    if m < 0:
        y = (-1) ** am * np.conj(y)
    if l > 0:
        y = np.where(zero, 0.0, y)  # no direction: l = 0 only
    return y


def _lmax(ap: AceParams) -> int:
    return max(ap.lmax2, ap.lmax3)


def _nmax(ap: AceParams) -> int:
    return max(ap.nmax1, ap.nmax2, ap.nmax3)


def grid_basis(offsets: np.ndarray, species: np.ndarray, ap: AceParams) -> np.ndarray:
    """A[mu][n][l][m + l] (complex) of one point from its neighbour offsets and their species."""
    L, N = _lmax(ap), _nmax(ap)
    A = np.zeros((ap.n_species, N, L + 1, 2 * L + 1), np.complex128)
    offsets = np.asarray(offsets, np.float64).reshape(-1, 3)
    if len(offsets) == 0:
        return A
    r = np.sqrt(np.sum(offsets * offsets, axis=1))
    R = radial(N, r, ap.rcut)
    for l in range(L + 1):
        for m in range(-l, l + 1):
            y = sph_harm(l, m, offsets)
            for mu in range(ap.n_species):
                sel = np.asarray(species) == mu
                A[mu, :, l, m + l] = R[:, sel] @ y[sel]
    return A


def _cg(l1, m1, l2, m2, l, m) -> float:
    return clebsch_gordan(2 * l1, 2 * m1, 2 * l2, 2 * m2, 2 * l, 2 * m)


def descriptor_index(ap: AceParams) -> List[Tuple]:
    """The output columns in order: ("1", mu, n), ("2", (mu1, n1), (mu2, n2), l),
    ("3", (mu1, n1, l1), (mu2, n2, l2), (mu3, n3, l3))."""
    out = []
    for mu in range(ap.n_species):
        for n in range(ap.nmax1):
            out.append(("1", mu, n))
    ch2 = [(mu, n) for mu in range(ap.n_species) for n in range(ap.nmax2)]
    for i in range(len(ch2)):
        for j in range(i, len(ch2)):
            for l in range(ap.lmax2 + 1):
                out.append(("2", ch2[i], ch2[j], l))
    ch3 = [(mu, n, l) for mu in range(ap.n_species) for n in range(ap.nmax3) for l in range(ap.lmax3 + 1)]
    for i in range(len(ch3)):
        for j in range(i, len(ch3)):
            for k in range(j, len(ch3)):
                l1, l2, l3 = ch3[i][2], ch3[j][2], ch3[k][2]
                if abs(l1 - l2) <= l3 <= l1 + l2 and (l1 + l2 + l3) % 2 == 0:
                    out.append(("3", ch3[i], ch3[j], ch3[k]))
    return out


def invariants(A: np.ndarray, ap: AceParams, index: Optional[List[Tuple]] = None) -> np.ndarray:
    """B of one point from its grid basis A (Eq. ace_grid for N = 1, 2, 3)."""
    index = descriptor_index(ap) if index is None else index
    out = np.zeros(len(index))
    for k, d in enumerate(index):
        if d[0] == "1":
            out[k] = A[d[1], d[2], 0, 0].real
        elif d[0] == "2":
            (m1_, n1), (m2_, n2), l = d[1], d[2], d[3]
            s = 0.0
            for m in range(-l, l + 1):
                s += _cg(l, m, l, -m, 0, 0) * A[m1_, n1, l, m + l] * A[m2_, n2, l, -m + l]
            out[k] = s.real
        else:
            (a1, n1, l1), (a2, n2, l2), (a3, n3, l3) = d[1], d[2], d[3]
            s = 0.0
            for m1 in range(-l1, l1 + 1):
                for m2 in range(-l2, l2 + 1):
                    M = m1 + m2
                    if abs(M) > l3:
                        continue
                    c = _cg(l1, m1, l2, m2, l3, M) * _cg(l3, M, l3, -M, 0, 0)
                    if c == 0.0:
                        continue
                    s += c * A[a1, n1, l1, m1 + l1] * A[a2, n2, l2, m2 + l2] * A[a3, n3, l3, -M + l3]
            out[k] = s.real
    return out


def ace_offsets(offsets: Sequence[np.ndarray], species: Sequence[np.ndarray], ap: AceParams) -> np.ndarray:
    """B for explicit neighbour-offset lists (one per point, no cell)."""
    idx = descriptor_index(ap)
    return np.array([invariants(grid_basis(o, s, ap), ap, idx) for o, s in zip(offsets, species)])


def ace_grid(snap, ap: AceParams, points: Optional[np.ndarray] = None) -> np.ndarray:
    """B[np][n_desc] at the given flat grid indices (all if None)."""
    pts = np.arange(snap.n_points) if points is None else np.asarray(points, np.int64)
    counts, atoms, shifts = neighbor_lists(snap, ap.rcut, points=pts)
    wpos = wrap_positions(snap)
    L = np.diag(snap.cell).astype(np.float64)
    sp = np.asarray(snap.species, np.int64)
    idx = descriptor_index(ap)
    out = np.zeros((len(pts), len(idx)))
    for i, p in enumerate(pts):
        n = int(counts[i])
        r = grid_point(snap, int(p))
        d = wpos[atoms[i, :n]] + shifts[i, :n] * L[None, :] - r[None, :]
        out[i] = invariants(grid_basis(d, sp[atoms[i, :n]], ap), ap, idx)
    return out
