"""GPU parity of the LDOS integrals (Sec. "Observable calculation") against
the FP64 oracle, on the same LDOS values.

The oracle integrates the piecewise-linear interpolant by adaptive quadrature,
the GPU by closed forms in Li2/Li3, so the FP64 comparison checks the weights.
Bars: FP64 path 1e-10 relative; MIXED path (BF16 LDOS summed in FP32 per 128
rows, density in FP32) 2e-6 relative; electron count dV sum_r n(r) = N_e to
1e-6.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2411_19617_gb300 import workloads as wl
from tests.gpu_util import ctx, need_gpu

pytestmark = pytest.mark.gpu


def _synthetic_ldos(P, eg, seed):
    """Positive LDOS: per point a few Gaussians with the paper's smearing width
    w_d = 2 de at random energies (Sec. "Calculation of the LDOS")."""
    rng = np.random.default_rng(seed)
    e = eg.e0_eV + eg.de_eV * np.arange(eg.n_E)
    wd = 2.0 * eg.de_eV
    L = np.zeros((P, eg.n_E))
    for k in range(4):
        c = rng.uniform(e[0], e[-1], size=(P, 1))
        amp = rng.uniform(0.2, 1.0, size=(P, 1))
        L += amp * np.exp(-((e[None, :] - c) / wd) ** 2) / math.sqrt(math.pi * wd * wd)
    return L


def _bf16_round(x):
    import torch
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.bfloat16).float().numpy().astype(np.float64)


@pytest.mark.parametrize("nE,de,e0,P", [(11, 1.0, -5.0, 5832), (250, 0.1, -8.0, 3001), (2, 0.5, 0.0, 7)])
def test_fp64_integrals_match_oracle(nE, de, e0, P):
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    eg = wl.EnergyGrid(n_E=nE, e0_eV=e0, de_eV=de)
    L = _synthetic_ldos(P, eg, seed=nE)
    vol = 512.0
    dV = vol / P
    D = oracle.dos(L, dV)
    Ne = oracle.electron_count(D, e0 + 0.37 * de * (nE - 1), e0, de, eg.kT_eV)
    ref = oracle.observables(L, dV, e0, de, eg.kT_eV, Ne)
    out = ctx().integrate(torch.from_numpy(L).cuda(), vol, eg, api.FP64_PLAIN, n_electrons=Ne)
    np.testing.assert_allclose(out["dos"], ref["dos"], rtol=1e-12)
    assert out["fermi"] == pytest.approx(ref["fermi"], abs=1e-9)
    assert out["band_energy"] == pytest.approx(ref["band_energy"], rel=1e-10, abs=1e-10)
    assert out["entropy_term"] == pytest.approx(ref["entropy_term"], rel=1e-10, abs=1e-12)
    np.testing.assert_allclose(out["density"].cpu().numpy(), ref["density"], rtol=1e-10, atol=1e-12)
    assert out["electron_count"] == pytest.approx(Ne, rel=1e-9)
    # the library's own electron count at the oracle's Fermi level
    assert ctx().electron_count(out["dos"], eg, ref["fermi"]) == pytest.approx(Ne, rel=1e-10)


@pytest.mark.parametrize("kT", [0.0259, 0.3, 1e-3])
def test_weights_across_temperatures(kT):
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    eg = wl.EnergyGrid(n_E=60, e0_eV=-3.0, de_eV=0.1, kT_eV=kT)
    L = _synthetic_ldos(200, eg, seed=5)
    D = oracle.dos(L, 1.0)
    for mu in (-2.95, -1.234, 0.0, 2.5, 2.899):
        assert ctx().electron_count(D, eg, mu) == pytest.approx(oracle.electron_count(D, mu, -3.0, 0.1, kT),
                                                                  rel=1e-11, abs=1e-12)


def test_mixed_integrals_match_oracle_on_the_same_bf16_values():
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    eg = wl.EnergyGrid(n_E=250, e0_eV=-8.0, de_eV=0.1)
    P = 20000
    L = _bf16_round(_synthetic_ldos(P, eg, seed=9))
    vol = 4251.528
    dV = vol / P
    D = oracle.dos(L, dV)
    Ne = oracle.electron_count(D, 0.0, eg.e0_eV, eg.de_eV, eg.kT_eV)
    ref = oracle.observables(L, dV, eg.e0_eV, eg.de_eV, eg.kT_eV, Ne)
    Lt = torch.from_numpy(L.astype(np.float32)).to(torch.bfloat16).cuda()
    out = ctx().integrate(Lt, vol, eg, api.MIXED, n_electrons=Ne)
    np.testing.assert_allclose(out["dos"], ref["dos"], rtol=2e-6)
    assert out["fermi"] == pytest.approx(ref["fermi"], abs=1e-5)
    assert out["band_energy"] == pytest.approx(ref["band_energy"], rel=2e-6)
    assert out["entropy_term"] == pytest.approx(ref["entropy_term"], rel=2e-6)
    np.testing.assert_allclose(out["density"].double().cpu().numpy(), ref["density"], rtol=2e-6, atol=1e-7)
    assert out["electron_count"] == pytest.approx(Ne, rel=1e-6)


def test_symmetric_gaussian_puts_fermi_level_at_its_centre():
    # f(x) + f(-x) = 1: half the weight of a symmetric DOS lies below its centre
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    eg = wl.EnergyGrid(n_E=81, e0_eV=-2.0, de_eV=0.05)
    e = eg.e0_eV + eg.de_eV * np.arange(eg.n_E)
    c = e[40]
    row = np.exp(-((e - c) / 0.3) ** 2)
    L = np.tile(row, (64, 1))
    half = 0.5 * oracle.electron_count(oracle.dos(L, 1.0), e[-1] + 40 * eg.kT_eV, eg.e0_eV, eg.de_eV, eg.kT_eV)
    out = ctx().integrate(torch.from_numpy(L).cuda(), 64.0, eg, api.FP64_PLAIN, n_electrons=half)
    assert out["fermi"] == pytest.approx(c, abs=1e-10)


def test_fermi_bracket_error():
    torch = need_gpu()
    from paper_2411_19617_gb300 import api, _lib
    eg = wl.EnergyGrid(n_E=11, e0_eV=-5.0, de_eV=1.0)
    L = np.ones((32, 11))
    out = ctx().integrate(torch.from_numpy(L).cuda(), 32.0, eg, api.FP64_PLAIN, n_electrons=1e6,
                          raise_on_bracket=False)
    assert out["status"] == _lib.MALA_ERR_FERMI_BRACKET
    np.testing.assert_allclose(out["dos"], np.ones(11) * 32.0, rtol=1e-14)
    with pytest.raises(_lib.MalaError):
        ctx().integrate(torch.from_numpy(L).cuda(), 32.0, eg, api.FP64_PLAIN, n_electrons=-1.0)


@pytest.mark.parametrize("kT", [0.0259, 0.3, 1e-3])
def test_entropy_term_matches_oracle_across_temperatures(kT):
    # closed forms (Li2/Li3 antiderivatives of s and y s) against quadrature of the definition
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    eg = wl.EnergyGrid(n_E=60, e0_eV=-3.0, de_eV=0.1, kT_eV=kT)
    P = 4000
    L = _synthetic_ldos(P, eg, seed=21)
    vol = 900.0
    D = oracle.dos(L, vol / P)
    Ne = oracle.electron_count(D, 0.05, eg.e0_eV, eg.de_eV, eg.kT_eV)
    ref = oracle.observables(L, vol / P, eg.e0_eV, eg.de_eV, eg.kT_eV, Ne)
    out = ctx().integrate(torch.from_numpy(L).cuda(), vol, eg, api.FP64_PLAIN, n_electrons=Ne)
    assert out["fermi"] == pytest.approx(ref["fermi"], abs=1e-9)
    assert out["entropy_term"] == pytest.approx(ref["entropy_term"], rel=1e-9, abs=1e-13)
    assert out["entropy_term"] <= 0.0


@pytest.mark.parametrize("mixed", [True, False])
@pytest.mark.parametrize("nE,P,row0", [(250, 20011, 1), (250, 3, 3), (11, 9000, 5), (7, 1, 1), (4096, 17, 2),
                                       (250, 729, 0), (300, 5003, 2), (1000, 999, 1), (64, 4097, 3), (8, 100, 7)])
def test_density_pass_any_alignment_and_size(mixed, nE, P, row0):
    """n(r) = sum_xi w0_xi LDOS(r, xi) on row slices that start at any row of a
    larger buffer (so the LDOS start need not be 16-byte aligned), with tiny,
    ragged and wide rows: the density equals the oracle's sum with the same
    weights, element by element."""
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    eg = wl.EnergyGrid(n_E=nE, e0_eV=-5.0, de_eV=10.0 / (nE - 1))
    L = _synthetic_ldos(P + row0, eg, seed=P + nE)
    if mixed:
        L = _bf16_round(L)
        full = torch.from_numpy(L.astype(np.float32)).to(torch.bfloat16).cuda()
    else:
        full = torch.from_numpy(L).cuda()
    view = full[row0:]
    assert view.is_contiguous() and view.shape[0] == P
    vol = 100.0
    dV = vol / P
    Ls = L[row0:]
    D = oracle.dos(Ls, dV)
    Ne = oracle.electron_count(D, -5.0 + 0.45 * 10.0, -5.0, eg.de_eV, eg.kT_eV)
    out = ctx().integrate(view, vol, eg, api.MIXED if mixed else api.FP64_PLAIN, n_electrons=Ne)
    w0 = oracle.integration_weights(0, -5.0, eg.de_eV, nE, out["fermi"], eg.kT_eV)
    ref = Ls @ w0
    got = out["density"].double().cpu().numpy()
    # the oracle's weights come from adaptive quadrature with an absolute tolerance, so rows whose
    # LDOS lies wholly above the Fermi level (weights ~1e-18) are compared with an absolute floor
    scale = np.abs(Ls) @ np.abs(w0)
    if mixed:
        # FP32 weights and sums over BF16 values: relative to the row's sum of |terms|
        assert np.all(np.abs(got - ref) <= 2e-6 * scale + 1e-9 * np.max(scale))
    else:
        assert np.all(np.abs(got - ref) <= 1e-10 * scale + 1e-12 * np.max(scale))
    assert out["electron_count"] == pytest.approx(Ne, rel=2e-6 if mixed else 1e-9)
