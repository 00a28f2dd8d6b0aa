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

from functools import lru_cache


def triples(twojmax: int):
    return [(j1, j2, j) for j1 in range(twojmax + 1) for j2 in range(j1 + 1)
            for j in range(j1 - j2, min(twojmax, j1 + j2) + 1, 2) if j >= j1]


@lru_cache(maxsize=None)
def zi_terms_half(twojmax: int) -> int:
    """Coupling terms of the half set of Z.  For j1 == j2 the row pairs
    (m1a, m2a) and (m2a, m1a) give the same product (the two Clebsch-Gordan
    factors change sign together under the exchange), so only m1a <= m2a
    is counted."""
    total = 0
    for (j1, j2, j) in triples(twojmax):
        d = (j1 + j2 - j) // 2

        def nvalid(mb, sym=False):
            return sum(1 for m1 in range(j1 + 1) if 0 <= mb - m1 + d <= j2 and (not sym or m1 <= mb - m1 + d))

        for ma in range(j + 1):
            for mb in range(j + 1):
                if (2 * ma < j) or (2 * ma == j and 2 * mb <= j):
                    total += nvalid(ma, sym=(j1 == j2)) * nvalid(mb)
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


def ui_flops_per_point(twojmax: int, mean_neighbors: float) -> float:
    return 18.0 * u_half_elements(twojmax) * mean_neighbors


def zb_bytes_per_point(twojmax: int) -> int:
    """u half set read (complex FP32) + B written (FP32)."""
    return 8 * u_half_elements(twojmax) + 4 * len(triples(twojmax))


def mlp_flops_per_point(dims) -> int:
    return sum(2 * dims[l] * dims[l + 1] for l in range(len(dims) - 1))


# FP32 CUDA-core peak of a GB300: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x SM clock
GB300_SMS = 152
FP32_LANES_PER_SM = 128


def fp32_peak_tflops(sm_mhz: float) -> float:
    return GB300_SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
