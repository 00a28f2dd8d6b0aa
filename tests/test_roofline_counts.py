"""The algorithmic work counts the benchmark divides by: the exact zero test of
Clebsch-Gordan coefficients against the oracle's values, and the term counts of
the contractions against brute-force enumerations over the oracle's coefficients."""
import oracle
from paper_2411_19617_gb300 import roofline


def test_cg_nonzero_matches_the_oracle_values():
    assert not roofline.cg_nonzero(2, 0, 2, 0, 2, 0)  # <1 0 1 0 | 1 0> = 0 (an accidental zero)
    assert roofline.cg_nonzero(2, 0, 2, 0, 4, 0)
    for j1 in range(7):
        for j2 in range(7):
            for j in range(abs(j1 - j2), j1 + j2 + 1, 2):
                for m1 in range(-j1, j1 + 1, 2):
                    for m2 in range(-j2, j2 + 1, 2):
                        m = m1 + m2
                        if abs(m) > j:
                            continue
                        c = oracle.clebsch_gordan(j1, m1, j2, m2, j, m)
                        assert roofline.cg_nonzero(j1, m1, j2, m2, j, m) == (abs(c) > 1e-12), (j1, m1, j2, m2, j, m)


def test_z_term_count_by_brute_force():
    tj = 6
    n = 0
    for (j1, j2, j) in roofline.triples(tj):
        d = (j1 + j2 - j) // 2
        for ma in range(j + 1):
            for mb in range(j + 1):
                if not ((2 * ma < j) or (2 * ma == j and 2 * mb <= j)):
                    continue
                for m1a in range(j1 + 1):
                    m2a = ma - m1a + d
                    if not 0 <= m2a <= j2 or (j1 == j2 and m1a > m2a):
                        continue
                    c1 = oracle.clebsch_gordan(j1, 2 * m1a - j1, j2, 2 * m2a - j2, j, 2 * ma - j)
                    for m1b in range(j1 + 1):
                        m2b = mb - m1b + d
                        if not 0 <= m2b <= j2:
                            continue
                        c2 = oracle.clebsch_gordan(j1, 2 * m1b - j1, j2, 2 * m2b - j2, j, 2 * mb - j)
                        n += abs(c1) > 1e-12 and abs(c2) > 1e-12
    assert roofline.zi_terms_half(tj) == n


class _AceBench:
    rcut, n_species, nmax1, nmax2, lmax2, nmax3, lmax3 = 4.676, 1, 8, 6, 6, 3, 4


def _ace_c3(l1, m1, l2, m2, l3):
    """<l1 m1 l2 m2|l3 M><l3 M l3 -M|0 0> from the oracle's Clebsch-Gordan values (integer l, m)."""
    M = m1 + m2
    return (oracle.clebsch_gordan(2 * l1, 2 * m1, 2 * l2, 2 * m2, 2 * l3, 2 * M)
            * oracle.clebsch_gordan(2 * l3, 2 * M, 2 * l3, -2 * M, 0, 0))


def test_ace_invariant_counts_by_brute_force():
    """The ACE invariant FLOP per point, as defined (every m) and as executed (the conjugate
    symmetry keeps N = 2 over m >= 0 and N = 3 over M > 0 or M = 0, m1 >= 0), against an
    enumeration over the oracle's coefficients."""
    ap = _AceBench
    ch2 = ap.n_species * ap.nmax2
    pairs2 = ch2 * (ch2 + 1) // 2
    full = pairs2 * sum(4 * (2 * l + 1) for l in range(ap.lmax2 + 1))
    kept = pairs2 * sum(4 * (l + 1) for l in range(ap.lmax2 + 1))
    ch3 = [(n, l) for n in range(ap.nmax3) for l in range(ap.lmax3 + 1)]
    for i in range(len(ch3)):
        for j in range(i, len(ch3)):
            for k in range(j, len(ch3)):
                l1, l2, l3 = ch3[i][1], ch3[j][1], ch3[k][1]
                if not (abs(l1 - l2) <= l3 <= l1 + l2 and (l1 + l2 + l3) % 2 == 0):
                    continue
                for m1 in range(-l1, l1 + 1):
                    for m2 in range(-l2, l2 + 1):
                        M = m1 + m2
                        if abs(M) > l3 or abs(_ace_c3(l1, m1, l2, m2, l3)) < 1e-12:
                            continue
                        full += 10
                        kept += 10 if (M > 0 or (M == 0 and m1 >= 0)) else 0
    assert roofline.ace_flops(ap, 0, 1) == full
    assert roofline.ace_flops(ap, 0, 1, folded=True) == kept


def test_ace_conjugate_fold_reproduces_the_full_sums():
    """For A with A_{l,-m} = (-1)^m conj(A_{l,m}) (A_{l,0} real, as for any real density), the
    N = 3 sum over M > 0, or M = 0 with m1 > 0, at twice the weight plus the all-zero term once,
    and the N = 2 sum over m >= 0 (m > 0 twice), equal the full sums."""
    import numpy as np
    rng = np.random.default_rng(7)

    def amp(l):
        a = {0: complex(rng.normal(), 0.0)}
        for m in range(1, l + 1):
            a[m] = complex(rng.normal(), rng.normal())
            a[-m] = (-1) ** m * a[m].conjugate()
        return a

    for (l1, l2, l3) in [(1, 1, 2), (2, 2, 2), (3, 2, 1), (4, 4, 4), (2, 3, 3), (0, 2, 2), (4, 3, 1)]:
        x, y, z = amp(l1), amp(l2), amp(l3)
        full = half = 0.0
        for m1 in range(-l1, l1 + 1):
            for m2 in range(-l2, l2 + 1):
                M = m1 + m2
                if abs(M) > l3:
                    continue
                t = _ace_c3(l1, m1, l2, m2, l3) * (x[m1] * y[m2] * z[-M]).real
                full += t
                if M > 0 or (M == 0 and m1 > 0):
                    half += 2.0 * t
                elif M == 0 and m1 == 0:
                    half += t
        assert abs(full - half) <= 1e-12 * max(1.0, abs(full)), (l1, l2, l3, full, half)
    for l in range(7):
        x, y = amp(l), amp(l)
        c = [oracle.clebsch_gordan(2 * l, 2 * m, 2 * l, -2 * m, 0, 0) for m in range(-l, l + 1)]
        full = sum(c[m + l] * (x[m] * y[-m]).real for m in range(-l, l + 1))
        half = c[l] * (x[0] * y[0]).real + 2.0 * sum(c[m + l] * (x[m] * y[-m]).real for m in range(1, l + 1))
        assert abs(full - half) <= 1e-12 * max(1.0, abs(full)), (l, full, half)
