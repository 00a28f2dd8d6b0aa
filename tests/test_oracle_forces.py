"""Pins of the force oracle (oracle/forces.py) against things other than itself:
the C oracle's descriptors, central finite differences of the C oracle / numpy
functions each gradient differentiates, and closed forms of the Fermi-function
derivative weights."""
import math

import numpy as np
import pytest

import oracle
from oracle import forces as of
from paper_2411_19617_gb300 import workloads as wl

torch = pytest.importorskip("torch")


def _moved(snap, a, k, h):
    p = snap.pos.copy()
    p[a, k] += h
    return wl.Snapshot(pos=p, species=snap.species, cell=snap.cell, grid=snap.grid)


@pytest.mark.parametrize("tj,weights", [(4, (1.0,)), (6, (1.0, 0.7))])
def test_restated_descriptors_equal_the_c_oracle(tj, weights):
    snap = wl.al_fcc(2, 0.15, 5, seed=4)
    if len(weights) > 1:
        snap = wl.Snapshot(pos=snap.pos, species=(np.arange(snap.n_atoms) % 2).astype(np.int32), cell=snap.cell,
                           grid=snap.grid)
    bp = wl.BispectrumParams(twojmax=tj, rcut=4.676, weights=weights, wself=1.3)
    pts = np.arange(0, snap.n_points, 3)
    Bt = of.bispectrum_torch(snap, bp, torch.tensor(snap.pos), pts).numpy()
    Bc = oracle.bispectrum_grid(snap, bp, points=pts)
    np.testing.assert_allclose(Bt, Bc, rtol=1e-12, atol=1e-12 * np.max(np.abs(Bc)))


def test_descriptor_forces_are_minus_the_gradient_of_beta_dot_b():
    snap = wl.al_fcc(2, 0.15, 6, seed=3)
    snap = wl.Snapshot(pos=snap.pos, species=(np.arange(snap.n_atoms) % 2).astype(np.int32), cell=snap.cell,
                       grid=snap.grid)
    bp = wl.BispectrumParams(twojmax=4, rcut=4.676, weights=(1.0, 0.6))
    rng = np.random.default_rng(0)
    beta = rng.normal(size=(snap.n_points, len(oracle.triples(4))))
    F = of.descriptor_forces(snap, bp, beta)
    h = 1e-5
    for a, k in ((0, 0), (5, 1), (17, 2), (31, 0)):
        e1 = np.sum(beta * oracle.bispectrum_grid(_moved(snap, a, k, h), bp))
        e2 = np.sum(beta * oracle.bispectrum_grid(_moved(snap, a, k, -h), bp))
        fd = -(e1 - e2) / (2 * h)
        assert F[a, k] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.max(np.abs(F)))


def test_ldos_backward_is_the_network_vjp():
    rng = np.random.default_rng(2)
    mlp = wl.random_mlp((9, 17, 13, 7), seed=5, out_bias=0.5)
    mlp.in_shift = rng.normal(size=9)
    mlp.in_scale = rng.uniform(0.5, 2.0, size=9)
    B = rng.normal(size=(6, 9))
    v = rng.normal(size=7)
    beta = of.ldos_backward(B, mlp, v)
    h = 1e-6
    for p in range(6):
        for j in (0, 4, 8):
            Bp, Bm = B.copy(), B.copy()
            Bp[p, j] += h
            Bm[p, j] -= h
            fp = oracle.mlp_forward(Bp, mlp.W, mlp.b, mlp.leaky_slope, mlp.in_shift, mlp.in_scale) @ v
            fm = oracle.mlp_forward(Bm, mlp.W, mlp.b, mlp.leaky_slope, mlp.in_shift, mlp.in_scale) @ v
            assert beta[p, j] == pytest.approx((fp[p] - fm[p]) / (2 * h), rel=1e-6, abs=1e-9)


def test_fermi_derivative_weights_closed_forms():
    # sum_xi w'(0)_xi = int_{e_0}^{e_max} f (1 - f)/kT de = f(e_0 - mu) - f(e_max - mu);
    # sum_xi w'(1)_xi = [-e f] + int f de, int f de = kT ln(1 + e^{-x}) antiderivative
    e0, de, n, mu, kT = -2.0, 0.25, 17, 0.37, 0.1
    f = lambda e: 1.0 / (1.0 + math.exp((e - mu) / kT))
    F = lambda e: -kT * math.log1p(math.exp(-(e - mu) / kT))  # d/de F = f
    emax = e0 + (n - 1) * de
    d0 = of.fermi_derivative_weights(0, e0, de, n, mu, kT)
    d1 = of.fermi_derivative_weights(1, e0, de, n, mu, kT)
    assert d0.sum() == pytest.approx(f(e0) - f(emax), rel=1e-11)
    assert d1.sum() == pytest.approx(e0 * f(e0) - emax * f(emax) + F(emax) - F(e0), rel=1e-10)
    # and they are the mu-derivatives of the integration weights
    h = 1e-5
    for order, d in ((0, d0), (1, d1)):
        wp = oracle.integration_weights(order, e0, de, n, mu + h, kT)
        wm = oracle.integration_weights(order, e0, de, n, mu - h, kT)
        np.testing.assert_allclose(d, (wp - wm) / (2 * h), rtol=1e-6, atol=1e-9)


def test_band_energy_gradient_at_fixed_electron_number():
    rng = np.random.default_rng(7)
    e0, de, kT, n = -3.0, 0.2, 0.05, 31
    D = rng.uniform(0.5, 2.0, size=n)
    Ne = oracle.electron_count(D, 0.1, e0, de, kT)
    g = of.band_energy_gradient(D, e0, de, kT, Ne)

    def Eb(Dx):
        mu = oracle.fermi_level(Dx, e0, de, kT, Ne)
        return float(np.dot(oracle.integration_weights(1, e0, de, n, mu, kT), Dx))

    h = 1e-5
    for k in (0, 9, 16, 17, 30):
        Dp, Dm = D.copy(), D.copy()
        Dp[k] += h
        Dm[k] -= h
        assert g["grad"][k] == pytest.approx((Eb(Dp) - Eb(Dm)) / (2 * h), rel=1e-6, abs=1e-8)
    assert g["mu_tilde"] == pytest.approx(g["fermi"], abs=5 * kT)


def test_band_forces_are_minus_the_gradient_of_the_band_energy():
    snap = wl.al_fcc(2, 0.15, 6, seed=8)
    bp = wl.BispectrumParams(twojmax=4, rcut=4.676)
    B = oracle.bispectrum_grid(snap, bp)
    mlp = wl.random_mlp((B.shape[1], 16, 16, 21), seed=9, out_bias=1.0)
    mlp = wl.with_input_scaling(mlp, B.mean(0), 1.0 / (B.std(0) + 1e-12))
    eg = wl.EnergyGrid(n_E=21, e0_eV=-4.0, de_eV=0.4, kT_eV=0.1)
    dV = float(snap.volume) / snap.n_points

    def Eb(s):
        Bs = oracle.bispectrum_grid(s, bp)
        L = oracle.mlp_forward(Bs, mlp.W, mlp.b, mlp.leaky_slope, mlp.in_shift, mlp.in_scale)
        return oracle.observables(L, dV, eg.e0_eV, eg.de_eV, eg.kT_eV, Ne)["band_energy"]

    L0 = oracle.mlp_forward(B, mlp.W, mlp.b, mlp.leaky_slope, mlp.in_shift, mlp.in_scale)
    Ne = oracle.electron_count(oracle.dos(L0, dV), 0.0, eg.e0_eV, eg.de_eV, eg.kT_eV)
    out = of.band_forces(snap, bp, mlp, eg, Ne)
    F = out["forces"]
    h = 1e-5
    for a, k in ((0, 0), (11, 2), (26, 1)):
        fd = -(Eb(_moved(snap, a, k, h)) - Eb(_moved(snap, a, k, -h))) / (2 * h)
        assert F[a, k] == pytest.approx(fd, rel=1e-5, abs=1e-6 * np.max(np.abs(F)))
