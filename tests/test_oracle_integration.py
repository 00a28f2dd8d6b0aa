"""Pins of the FP64 energy-integral oracle (Sec. "Observable calculation").

The oracle integrates hat_xi(e) e^n f_beta(e - mu) by adaptive quadrature.
These tests hold it against closed forms that do not use quadrature: the
polylogarithm antiderivatives the paper points to (Eq. fermidiracspecial,
evaluated with mpmath), the zero-temperature limit, Gaussian DOS sums with
the paper's smearing function, and the symmetry f(x) + f(-x) = 1.
"""
import math

import numpy as np
import pytest

import oracle


def _closed_form_weights(order, e0, de, n_E, mu, kT):
    """w_xi = int hat_xi e^order f de via G_n, the antiderivatives of x^n/(1+e^x):
    G0 = x - ln(1+e^x), G1 = x^2/2 - x ln(1+e^x) - Li2(-e^x),
    G2 = x^3/3 - x^2 ln(1+e^x) - 2x Li2(-e^x) + 2 Li3(-e^x)."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40

    def G(n, x):
        x = mp.mpf(x)
        l1 = mp.log1p(mp.exp(x))
        if n == 0:
            return x - l1
        li2 = mp.polylog(2, -mp.exp(x))
        if n == 1:
            return x * x / 2 - x * l1 - li2
        li3 = mp.polylog(3, -mp.exp(x))
        return x ** 3 / 3 - x * x * l1 - 2 * x * li2 + 2 * li3

    def moment(k, a, b):
        # int_a^b (e - mu)^k f de = kT^(k+1) [G_k(xb) - G_k(xa)]
        xa, xb = (mp.mpf(a) - mu) / kT, (mp.mpf(b) - mu) / kT
        return mp.mpf(kT) ** (k + 1) * (G(k, xb) - G(k, xa))

    def poly_int(coeffs, a, b):
        # int_a^b sum_k c_k (e - mu)^k f de
        return sum(c * moment(k, a, b) for k, c in enumerate(coeffs) if c != 0)

    w = [mp.mpf(0)] * n_E
    mu_ = mp.mpf(mu)
    for i in range(n_E - 1):
        a = mp.mpf(e0) + i * mp.mpf(de)
        b = a + mp.mpf(de)
        # e^order * hat in powers of t = e - mu; e = t + mu
        # left hat (b - e)/de = (b - mu - t)/de ; right hat (e - a)/de = (t + mu - a)/de
        def expand(c0, c1):
            # (c0 + c1 t) (t + mu)^order -> coefficients in t
            base = [mp.binomial(order, k) * mu_ ** (order - k) for k in range(order + 1)]
            out = [mp.mpf(0)] * (order + 2)
            for k, v in enumerate(base):
                out[k] += c0 * v
                out[k + 1] += c1 * v
            return out
        left = expand((b - mu_) / de, mp.mpf(-1) / de)
        right = expand((mu_ - a) / de, mp.mpf(1) / de)
        w[i] += poly_int(left, a, b)
        w[i + 1] += poly_int(right, a, b)
    return np.array([float(v) for v in w])


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("mu,kT", [(0.33, 0.0259), (-4.2, 0.0259), (7.77, 0.3), (2.0, 0.01)])
def test_weights_match_polylog_closed_form(order, mu, kT):
    e0, de, n_E = -5.0, 0.5, 29
    w = oracle.integration_weights(order, e0, de, n_E, mu, kT)
    ref = _closed_form_weights(order, e0, de, n_E, mu, kT)
    scale = de * max(1.0, abs(e0 + de * n_E)) ** order
    np.testing.assert_allclose(w, ref, atol=1e-12 * scale, rtol=0)


def test_weights_zero_temperature_limit():
    # kT -> 0: f is the step at mu and the hat integrals are piecewise polynomials.
    e0, de, n_E, mu = -2.0, 0.25, 17, 0.4
    w0 = oracle.integration_weights(0, e0, de, n_E, mu, 1e-7)
    w1 = oracle.integration_weights(1, e0, de, n_E, mu, 1e-7)
    ref0, ref1 = np.zeros(n_E), np.zeros(n_E)
    for i in range(n_E - 1):
        a, b = e0 + i * de, e0 + (i + 1) * de
        top = min(b, mu)
        if top <= a:
            continue
        # int_a^top (b-e)/de de, int_a^top (e-a)/de de, and with an extra factor e
        L0 = ((b - a) ** 2 - (b - top) ** 2) / (2 * de)
        R0 = (top - a) ** 2 / (2 * de)
        L1 = (b * (top ** 2 - a ** 2) / 2 - (top ** 3 - a ** 3) / 3) / de
        R1 = ((top ** 3 - a ** 3) / 3 - a * (top ** 2 - a ** 2) / 2) / de
        ref0[i] += L0; ref0[i + 1] += R0
        ref1[i] += L1; ref1[i + 1] += R1
    np.testing.assert_allclose(w0, ref0, atol=1e-7)
    np.testing.assert_allclose(w1, ref1, atol=1e-7)


def _gaussian_dos(centres, wd, e0, de, n_E):
    # the paper's smearing function delta~(x) = exp(-x^2/wd^2) / sqrt(pi wd^2)
    e = e0 + de * np.arange(n_E)
    return sum(np.exp(-((e - c) / wd) ** 2) / math.sqrt(math.pi * wd * wd) for c in centres)


def test_gaussian_dos_electron_count_low_temperature():
    # int f D de -> sum_j erfc((e_j - mu)/wd) / 2 as kT -> 0.
    e0, de, n_E, wd = -3.0, 0.005, 1201, 0.2
    centres = [-1.1, 0.05, 0.9]
    D = _gaussian_dos(centres, wd, e0, de, n_E)
    mu = 0.31
    N = oracle.electron_count(D, mu, e0, de, 1e-4)
    ref = sum(0.5 * math.erfc((c - mu) / wd) for c in centres)
    # piecewise-linear interpolation error ~ de^2/12 * |D''| integrated
    assert N == pytest.approx(ref, abs=2e-5)


def test_gaussian_dos_sommerfeld():
    # Sommerfeld: int f D = int_{-inf}^{mu} D + (pi^2/6) (kT)^2 D1(mu)
    #                      + (7 pi^4/360) (kT)^4 D3(mu) + O(kT^6), Dk = k-th derivative.
    e0, de, n_E, wd = -3.0, 0.0025, 2401, 0.4
    c = 0.0
    D = _gaussian_dos([c], wd, e0, de, n_E)
    mu, kT = 0.25, 0.02
    N = oracle.electron_count(D, mu, e0, de, kT)
    y = (mu - c) / wd
    g = math.exp(-y * y) / math.sqrt(math.pi * wd * wd)
    d1 = g * (-2 * y) / wd
    d3 = g * (-8 * y ** 3 + 12 * y) / wd ** 3
    ref = (0.5 * math.erfc((c - mu) / wd) + math.pi ** 2 / 6 * kT ** 2 * d1
           + 7 * math.pi ** 4 / 360 * kT ** 4 * d3)
    # remaining: interpolation error ~ (de^2/12) |D1(mu)| ~ 1.6e-6
    assert N == pytest.approx(ref, abs=3e-6)


def test_fermi_level_symmetric_gaussian():
    # A single Gaussian sampled symmetrically about its centre and N_e = half its
    # weight: f(x) + f(-x) = 1 puts the Fermi level exactly at the centre.
    e0, de, n_E, wd = -2.0, 0.05, 81, 0.3
    c = e0 + de * 40
    D = _gaussian_dos([c], wd, e0, de, n_E)
    kT = 0.0259
    half = 0.5 * oracle.electron_count(D, e0 + de * (n_E - 1) + 40 * kT, e0, de, kT)
    eF = oracle.fermi_level(D, e0, de, kT, half)
    assert eF == pytest.approx(c, abs=1e-10)
    assert oracle.electron_count(D, eF, e0, de, kT) == pytest.approx(half, rel=1e-12)


def test_fermi_level_bracket_error():
    D = np.ones(11)
    with pytest.raises(oracle.FermiBracketError):
        oracle.fermi_level(D, -5.0, 1.0, 0.0259, 1e6)
    with pytest.raises(oracle.FermiBracketError):
        oracle.fermi_level(D, -5.0, 1.0, 0.0259, -1.0)


def test_electron_count_invariant_and_band_energy():
    # dV sum_r n(r) = sum_xi w0_xi D_xi = N(eF) = N_e, and E_b = sum w1 D.
    rng = np.random.default_rng(3)
    P, n_E = 300, 25
    L = rng.uniform(0.0, 1.0, size=(P, n_E))
    dV = 0.01
    e0, de, kT = -3.0, 0.25, 0.0259
    D = oracle.dos(L, dV)
    Ne = 0.6 * float(np.sum(D) * de)
    obs = oracle.observables(L, dV, e0, de, kT, Ne)
    assert dV * np.sum(obs["density"]) == pytest.approx(Ne, rel=1e-10)
    w1 = oracle.integration_weights(1, e0, de, n_E, obs["fermi"], kT)
    assert obs["band_energy"] == pytest.approx(float(w1 @ D), rel=1e-14)
    np.testing.assert_allclose(obs["dos"], dV * L.sum(axis=0), rtol=1e-14)


# ---- entropy contribution (Eq. electronicentropyDOS) ------------------------

def test_entropy_of_a_flat_dos_is_pi2_over_3():
    # int s(x) dx over the real line = pi^2/3, so a constant D0 gives
    # S_s / k_B = D0 kT pi^2 / 3 (mu deep inside the grid: the tails are below 1e-15)
    kT, D0 = 0.05, 2.5
    e0, de, n_E = -3.0, 0.25, 25
    D = np.full(n_E, D0)
    TS = oracle.entropy_term(D, 0.0, e0, de, kT)
    assert TS == pytest.approx(-kT * D0 * kT * math.pi ** 2 / 3.0, rel=1e-11)


def test_entropy_sommerfeld_for_a_smooth_dos():
    # S_s / k_B = (pi^2 / 3) kT D(mu) + (7 pi^4 / 90) kT^3 D''(mu) for a quadratic DOS (fine grid)
    e0, de, n_E = -2.0, 0.002, 2001
    e = e0 + de * np.arange(n_E)
    D = 1.0 + 0.3 * e + 0.2 * e ** 2
    for kT in (0.01, 0.02):
        mu = 0.1
        TS = oracle.entropy_term(D, mu, e0, de, kT)
        Dmu = 1.0 + 0.3 * mu + 0.2 * mu ** 2
        # next term: kT^3 D''(mu) / 2 * int x^2 s(x) dx = kT^3 D''(mu) / 2 * 7 pi^4 / 45; the
        # quadratic D has no higher one
        ref = -kT * (math.pi ** 2 / 3.0 * kT * Dmu + 0.5 * 0.4 * kT ** 3 * 7 * math.pi ** 4 / 45.0)
        assert TS == pytest.approx(ref, rel=2e-5)


def test_entropy_vanishes_at_zero_temperature_and_is_symmetric():
    e0, de, n_E = -1.0, 0.1, 21
    rng = np.random.default_rng(2)
    D = rng.uniform(0.5, 1.5, n_E)
    assert abs(oracle.entropy_term(D, 0.03, e0, de, 1e-6)) < 1e-9
    # s(x) = s(-x): mirroring the DOS about mu mirrors nothing
    w = oracle.entropy_weights(e0, de, n_E, 0.0, 0.05)
    np.testing.assert_allclose(w, w[::-1], rtol=1e-10, atol=1e-15)
