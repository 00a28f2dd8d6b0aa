"""Algorithmic work of the descriptor kernels (for roofline fractions).

Counts follow the definitions, not the kernels' instruction streams:
  * compute_zi on the half set of Z (rows m < j/2, plus the middle row's
    columns m' <= j/2 for even 2j), j1 = j2 row pairs counted once: every coupling term
    C C u^{j1} u^{j2} costs a complex product (6 flop), a real scale (2 flop)
    and a complex accumulate (2 flop) = 10 flop;
  * compute_bi: Re(conj(u^j) Z) per half-set element = 4 flop;
  * compute_ui: per neighbour and half-set element of u, the level recursion
    (two complex products by the Cayley-Klein forms and a sum, 14 flop) and the
    weighted accumulate (4 flop) = 18 flop.
"""
from __future__ import annotations

from fractions import Fraction
from functools import lru_cache
from math import factorial


def triples(twojmax: int):
    return [(j1, j2, j) for j1 in range(twojmax + 1) for j2 in range(j1 + 1)
            for j in range(j1 - j2, min(twojmax, j1 + j2) + 1, 2) if j >= j1]


@lru_cache(maxsize=None)
def cg_nonzero(j1: int, m1: int, j2: int, m2: int, j: int, m: int) -> bool:
    """Whether <j1 m1 j2 m2 | j m> (twice-units) is nonzero: the selection rules, then
    Racah's alternating sum evaluated exactly in rationals (the square-root prefactor
    never vanishes for an allowed coupling; the sum has accidental zeros such as
    <1 0 1 0 | 1 0>).  Used only to count the terms an algorithm needs."""
    if m1 + m2 != m or abs(m1) > j1 or abs(m2) > j2 or abs(m) > j:
        return False
    if (j1 + m1) % 2 or (j2 + m2) % 2 or (j + m) % 2 or (j1 + j2 + j) % 2 or not abs(j1 - j2) <= j <= j1 + j2:
        return False
    A = (j1 + j2 - j) // 2
    s = Fraction(0)
    for k in range(A + 1):
        d = ((j1 - m1) // 2 - k, (j2 + m2) // 2 - k, (j - j2 + m1) // 2 + k, (j - j1 - m2) // 2 + k)
        if min(d) < 0:
            continue
        den = factorial(k) * factorial(A - k)
        for x in d:
            den *= factorial(x)
        s += Fraction(-1 if k % 2 else 1, den)
    return s != 0


@lru_cache(maxsize=None)
def zi_terms_half(twojmax: int) -> int:
    """Coupling terms of the half set of Z whose two Clebsch-Gordan factors are
    nonzero (the terms the contraction needs).  For j1 == j2 the row pairs
    (m1a, m2a) and (m2a, m1a) give the same product (the two Clebsch-Gordan
    factors change sign together under the exchange), so only m1a <= m2a
    is counted."""
    total = 0
    for (j1, j2, j) in triples(twojmax):
        d = (j1 + j2 - j) // 2
        for ma in range(j + 1):
            for mb in range(j + 1):
                if not ((2 * ma < j) or (2 * ma == j and 2 * mb <= j)):
                    continue
                rows = [m1 for m1 in range(j1 + 1) if 0 <= ma - m1 + d <= j2 and (j1 != j2 or m1 <= ma - m1 + d)
                        and cg_nonzero(j1, 2 * m1 - j1, j2, 2 * (ma - m1 + d) - j2, j, 2 * ma - j)]
                cols = [m1 for m1 in range(j1 + 1) if 0 <= mb - m1 + d <= j2
                        and cg_nonzero(j1, 2 * m1 - j1, j2, 2 * (mb - m1 + d) - j2, j, 2 * mb - j)]
                total += len(rows) * len(cols)
    return total


def half_count(J: int) -> int:
    """Elements of the half set of a (J+1) x (J+1) block."""
    return ((J + 1) // 2) * (J + 1) if J % 2 else (J // 2) * (J + 1) + J // 2 + 1


@lru_cache(maxsize=None)
def z_half_elements(twojmax: int) -> int:
    return sum(half_count(j) for (_, _, j) in triples(twojmax))


def u_half_elements(twojmax: int) -> int:
    return sum(half_count(J) for J in range(twojmax + 1))


def zb_flops_per_point(twojmax: int) -> int:
    return 10 * zi_terms_half(twojmax) + 4 * z_half_elements(twojmax)


@lru_cache(maxsize=None)
def zi_terms_full(twojmax: int) -> int:
    """Coupling terms C C u^{j1} u^{j2} of the full Z (every element (ma, mb) of every
    triple, every pair (m1a, m1b) whose partners lie inside u^{j2}, no test of the
    Clebsch-Gordan values): 7,721 at twojmax 6, 121,054 at twojmax 10."""
    total = 0
    for (j1, j2, j) in triples(twojmax):
        d = (j1 + j2 - j) // 2
        rows = [sum(1 for m1 in range(j1 + 1) if 0 <= m - m1 + d <= j2) for m in range(j + 1)]
        total += sum(rows) ** 2
    return total


def zb_flops_per_point_full_count(twojmax: int) -> int:
    """The plainer count: 10 flop per term of the full Z halved by the symmetry of
    u and Z, plus 4 flop per element of the full Z for compute_bi.  At twojmax 10:
    121,054 terms -> 605,270 + 4 x 6,832 = 632,598 flop per point."""
    return 10 * zi_terms_full(twojmax) // 2 + 4 * sum((j + 1) ** 2 for (_, _, j) in triples(twojmax))


def ui_flops_per_point(twojmax: int, mean_neighbors: float) -> float:
    return 18.0 * u_half_elements(twojmax) * mean_neighbors


def zb_bytes_per_point(twojmax: int) -> int:
    """u half set read (complex FP32) + B written (FP32)."""
    return 8 * u_half_elements(twojmax) + 4 * len(triples(twojmax))


def mlp_flops_per_point(dims) -> int:
    return sum(2 * dims[l] * dims[l + 1] for l in range(len(dims) - 1))


def density_bytes(points: int, n_e: int, ldos_bytes: int = 2, out_bytes: int = 4) -> int:
    """The density pass n(r) = sum_xi w0_xi LDOS(r, xi): the LDOS read once, n written
    once, the weights read once."""
    return points * n_e * ldos_bytes + points * out_bytes + n_e * 8


def neighbor_bytes(pairs: int, points: int) -> int:
    """What the neighbour search must write: one record per (point, neighbour) pair
    (Cayley-Klein a, b as a float4 and w f_c as a float) and a count per point."""
    return 20 * pairs + 4 * points


# FP32 lanes of one Blackwell SM (4 schedulers x 32); the SM count comes from the device
FP32_LANES_PER_SM = 128


def yi_terms_half(twojmax: int):
    """(terms, groups) of the adjoint contraction Y^J over the half set: for every
    coupling c <- (a, b) that a triple (j1, j2, j) brings in its three roles
    (j <- j1 j2, j1 <- j j2, j2 <- j j1), every Y element (ma, mb) of the half set
    of c takes the Clebsch-Gordan pairs (m1a, m1b) whose partners lie inside b."""
    coup = set()
    for (j1, j2, j) in triples(twojmax):
        for (c, a, b) in ((j, j1, j2), (j1, j, j2), (j2, j, j1)):
            coup.add((c, max(a, b), min(a, b)))
    terms = groups = 0
    for (c, a, b) in coup:
        rows = []
        for ma in range(c + 1):
            m = 2 * ma - c
            rows.append(sum(1 for m1a in range(a + 1) if abs(m - (2 * m1a - a)) <= b
                            and cg_nonzero(a, 2 * m1a - a, b, m - (2 * m1a - a), c, m)))
        for ma in range(c + 1):
            for mb in range(c + 1):
                if 2 * ma > c or (2 * ma == c and 2 * mb > c):
                    continue
                n = rows[ma] * rows[mb]
                terms += n
                groups += 1 if n else 0
    return terms, groups


def yi_flops_per_point(twojmax: int) -> int:
    """10 flop per term (complex product scaled by C C, accumulated), 4 per coupling group."""
    t, g = yi_terms_half(twojmax)
    return 10 * t + 4 * g


def force_flops_per_pair(twojmax: int) -> int:
    """The column-chain walk of one (point, neighbour) pair: per chain c and level J the
    G_0 dot (4 flop per coefficient) and, below the top level, four complex dots
    (32 flop per coefficient) and the linear-form product (16 per output coefficient);
    16 per coefficient of each chain's starting power beta^c."""
    f = 0
    for c in range(twojmax + 1):
        f += 16 * (c + 1) if c > 0 else 0
        for J in range(c, twojmax + 1):
            f += 4 * (J + 1)
            if J < twojmax:
                f += 32 * (J + 1) + 16 * (J + 2)
    return f


def ace_flops(ap, pairs: int, points: int, folded: bool = False) -> int:
    """Algorithmic FLOP of the ACE descriptors: per neighbour pair the spherical
    harmonics (8 per (l, m >= 0)), the Chebyshev radial functions (3 per n) and the
    grid-basis accumulation (4 per (n, l, m >= 0): real R times complex Y, added);
    per point the invariants (N = 2: 4 per m; N = 3: 10 per (m1, m2) term with a nonzero
    Clebsch-Gordan factor).  folded: count the invariant terms a kernel evaluates after the
    conjugate symmetry A_{l,-m} = (-1)^m conj(A_{l,m}) pairs them (N = 2: m >= 0 only;
    N = 3: M > 0, or M = 0 and m1 >= 0 with m1 = 0 only for the all-zero term)."""
    nmax = max(ap.nmax1, ap.nmax2, ap.nmax3)
    lmax = max(ap.lmax2, ap.lmax3)
    nlm = (lmax + 1) * (lmax + 2) // 2
    per_pair = 8 * nlm + 3 * nmax + 4 * nmax * nlm
    ns = ap.n_species
    n2ch = ns * ap.nmax2
    per_m2 = [(l + 1) if folded else (2 * l + 1) for l in range(ap.lmax2 + 1)]
    per_point = (n2ch * (n2ch + 1) // 2) * sum(4 * k for k in per_m2)

    def kept(m1, m2):
        M = m1 + m2
        return not folded or M > 0 or (M == 0 and m1 >= 0)

    ch3 = [(mu, n, l) for mu in range(ns) for n in range(ap.nmax3) for l in range(ap.lmax3 + 1)]
    terms = {}
    for i in range(len(ch3)):
        for j in range(i, len(ch3)):
            for k in range(j, len(ch3)):
                l1, l2, l3 = ch3[i][2], ch3[j][2], ch3[k][2]
                if abs(l1 - l2) <= l3 <= l1 + l2 and (l1 + l2 + l3) % 2 == 0:
                    key = (l1, l2, l3)
                    if key not in terms:
                        terms[key] = sum(1 for m1 in range(-l1, l1 + 1) for m2 in range(-l2, l2 + 1)
                                         if abs(m1 + m2) <= l3 and kept(m1, m2)
                                         and cg_nonzero(2 * l1, 2 * m1, 2 * l2, 2 * m2, 2 * l3, 2 * (m1 + m2)))
                    per_point += 10 * terms[key]
    return per_pair * pairs + per_point * points


def fp32_peak_tflops(sm_mhz: float, n_sms: int) -> float:
    """Nominal FP32 FMA peak: SMs x 128 lanes x 2 flop x clock."""
    return n_sms * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
