"""The whole path through mala_predict: descriptors -> LDOS -> integrals,
against the FP64 oracle chain on the same inputs."""
import numpy as np
import pytest

import oracle
from paper_2411_19617_gb300 import workloads as wl
from tests.gpu_util import ctx, descriptor_error, need_gpu

pytestmark = pytest.mark.gpu


def _oracle_chain(snap, bp, mlp, eg, points=None):
    B = oracle.bispectrum_grid(snap, bp, points=points, nthreads=8)
    L = oracle.mlp_forward(B, mlp.W, mlp.b, mlp.leaky_slope, mlp.in_shift, mlp.in_scale)
    return B, L


def _scaled(mlp, B):
    return wl.with_input_scaling(mlp, B.mean(axis=0), 1.0 / (B.std(axis=0) + 1e-12))


def test_al_small_fp64_plain_matches_oracle():
    need_gpu()
    from paper_2411_19617_gb300 import api
    snaps, bp, mlp, eg, _ = wl.config(1)
    snap = snaps[0]
    B, _ = _oracle_chain(snap, bp, mlp, eg)
    mlp = _scaled(mlp, B)
    L = oracle.mlp_forward(B, mlp.W, mlp.b, mlp.leaky_slope, mlp.in_shift, mlp.in_scale)
    dV = snap.volume / snap.n_points
    D = oracle.dos(L, dV)
    Ne = oracle.electron_count(D, 0.0, eg.e0_eV, eg.de_eV, eg.kT_eV)
    ref = oracle.observables(L, dV, eg.e0_eV, eg.de_eV, eg.kT_eV, Ne)
    model = api.Model(ctx(), mlp)
    dens = np.zeros(snap.n_points)
    out = ctx().predict(snap, bp, model, eg, api.FP64_PLAIN, n_electrons=Ne, density_host=dens)
    assert descriptor_error(out["B"].cpu().numpy(), B, floor=1e-3) < 1e-10
    np.testing.assert_allclose(out["ldos"].cpu().numpy(), L, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(out["dos"], ref["dos"], rtol=1e-9)
    assert out["fermi"] == pytest.approx(ref["fermi"], abs=1e-8)
    assert out["band_energy"] == pytest.approx(ref["band_energy"], rel=1e-9)
    np.testing.assert_allclose(dens, ref["density"], rtol=1e-9, atol=1e-12)
    assert out["electron_count"] == pytest.approx(Ne, rel=1e-9)


def test_al_small_mixed_matches_oracle_within_bf16_tolerance():
    need_gpu()
    from paper_2411_19617_gb300 import api
    snaps, bp, mlp, eg, _ = wl.config(1)
    snap = snaps[0]
    B, _ = _oracle_chain(snap, bp, mlp, eg)
    mlp = _scaled(mlp, B)
    L = oracle.mlp_forward(B, mlp.W, mlp.b, mlp.leaky_slope, mlp.in_shift, mlp.in_scale)
    dV = snap.volume / snap.n_points
    D = oracle.dos(L, dV)
    Ne = oracle.electron_count(D, 0.0, eg.e0_eV, eg.de_eV, eg.kT_eV)
    ref = oracle.observables(L, dV, eg.e0_eV, eg.de_eV, eg.kT_eV, Ne)
    model = api.Model(ctx(), mlp)
    dens = np.zeros(snap.n_points, np.float32)
    out = ctx().predict(snap, bp, model, eg, api.MIXED, n_electrons=Ne, density_host=dens)
    assert descriptor_error(out["B"].double().cpu().numpy(), B) < 1e-5
    Lg = out["ldos"].float().cpu().numpy().astype(np.float64)
    err = np.max(np.linalg.norm(Lg - L, axis=1) / np.linalg.norm(L, axis=1))
    assert err < 2e-2
    np.testing.assert_allclose(out["dos"], ref["dos"], rtol=2e-2)
    assert out["band_energy"] == pytest.approx(ref["band_energy"], rel=2e-2)
    assert out["fermi"] == pytest.approx(ref["fermi"], abs=2e-2 * eg.de_eV * eg.n_E)
    np.testing.assert_allclose(dens, ref["density"], rtol=2e-2)
    # electron-count invariant on the GPU's own LDOS: dV sum_r n(r) = N(eF) = N_e
    assert out["electron_count"] == pytest.approx(Ne, rel=1e-6)


def test_al_liquid_full_size_sampled_points():
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    snaps, bp, mlp, eg, _ = wl.config(2)
    snap = snaps[0]
    pts = wl.sample_points(snap.n_points, 200, seed=3)
    B = oracle.bispectrum_grid(snap, bp, points=pts, nthreads=8)
    mlp = _scaled(mlp, B)
    model = api.Model(ctx(), mlp)
    out = ctx().predict(snap, bp, model, eg, api.MIXED, n_electrons=0.0, raise_on_bracket=False)
    L = oracle.mlp_forward(B, mlp.W, mlp.b, mlp.leaky_slope, mlp.in_shift, mlp.in_scale)
    Lg = out["ldos"][torch.from_numpy(pts).cuda()].float().cpu().numpy().astype(np.float64)
    assert np.max(np.linalg.norm(Lg - L, axis=1) / np.linalg.norm(L, axis=1)) < 2e-2
    # now with a reachable electron count: N at mu = 0 of the GPU's own DOS
    Ne = ctx().electron_count(out["dos"], eg, 0.0)
    dens = np.zeros(snap.n_points, np.float32)
    out2 = ctx().predict(snap, bp, model, eg, api.MIXED, n_electrons=Ne, density_host=dens)
    assert out2["fermi"] == pytest.approx(0.0, abs=1e-6)
    assert out2["electron_count"] == pytest.approx(Ne, rel=1e-6)
    assert np.all(np.isfinite(dens))
