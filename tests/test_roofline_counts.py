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
