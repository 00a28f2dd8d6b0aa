"""The grid-sharded integrals on the GPU: the library backend of
paper_2411_19617_gb300.sharded, run over row slabs of one LDOS (the exchange
done in-process), gives the single-call D(e), e_F, E_b and n(r), and matches
the FP64 oracle on the same values."""
import math

import numpy as np
import pytest

import oracle
from paper_2411_19617_gb300 import sharded
from paper_2411_19617_gb300 import workloads as wl
from tests.gpu_util import ctx, need_gpu

pytestmark = pytest.mark.gpu


def _ldos(P, eg, seed):
    rng = np.random.default_rng(seed)
    e = eg.e0_eV + eg.de_eV * np.arange(eg.n_E)
    wd = 2.0 * eg.de_eV
    L = np.zeros((P, eg.n_E))
    for _ in range(4):
        c = rng.uniform(e[0], e[-1], size=(P, 1))
        L += rng.uniform(0.2, 1.0, size=(P, 1)) * np.exp(-((e[None, :] - c) / wd) ** 2) / math.sqrt(math.pi) / wd
    return L


@pytest.mark.parametrize("world", [1, 3])
def test_slabs_reproduce_the_whole_grid_fp64(world):
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    c = ctx()
    eg = wl.EnergyGrid(n_E=40, e0_eV=-3.0, de_eV=0.15)
    P, volume = 5000, 400.0
    L = _ldos(P, eg, seed=11)
    dV = volume / P
    ne = oracle.electron_count(oracle.dos(L, dV), 0.0, eg.e0_eV, eg.de_eV, eg.kT_eV)
    ref = oracle.observables(L, dV, eg.e0_eV, eg.de_eV, eg.kT_eV, ne)
    Ld = torch.from_numpy(L).cuda()
    whole = c.integrate(Ld, volume, eg, api.FP64_PLAIN, n_electrons=ne)
    be = sharded.DeviceBackend(c, api.FP64_PLAIN)
    slabs = [sharded.row_range(P, r, world) for r in range(world)]
    sums = sum(be.column_sums(Ld[a:b]) for a, b in slabs)  # the all-reduce, in-process
    parts = [sharded.integrate_sharded(be, Ld[a:b], P, volume, eg, ne, col_sums_local=sums if world > 1 else None)
             for a, b in slabs]
    # with the global sums handed in, every slab sees the same D and e_F
    for p in parts[1:]:
        assert p["fermi"] == parts[0]["fermi"]
        np.testing.assert_array_equal(p["dos"], parts[0]["dos"])
    np.testing.assert_allclose(parts[0]["dos"], whole["dos"], rtol=1e-12)
    assert parts[0]["fermi"] == pytest.approx(whole["fermi"], abs=1e-10)
    assert parts[0]["band_energy"] == pytest.approx(whole["band_energy"], rel=1e-10)
    dens = np.concatenate([p["density"] for p in parts])
    np.testing.assert_allclose(dens, whole["density"].cpu().numpy(), rtol=1e-10, atol=1e-12)
    # and the oracle
    assert parts[0]["fermi"] == pytest.approx(ref["fermi"], abs=1e-9)
    assert parts[0]["band_energy"] == pytest.approx(ref["band_energy"], rel=1e-10)
    np.testing.assert_allclose(dens, ref["density"], rtol=1e-10, atol=1e-12)
    local = sum(dV * float(np.sum(p["density"])) for p in parts)
    assert local == pytest.approx(ne, rel=1e-6)


@pytest.mark.parametrize("world", [1, 2])
def test_sharded_forces_pieces_reproduce_band_forces_fp64(world):
    # the library backend's per-rank pieces, the two exchanges (DOS, forces) summed in-process
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    c = ctx()
    snap = wl.al_fcc(2, 0.15, 6, seed=8)
    bp = wl.BispectrumParams(twojmax=4, rcut=4.676)
    B = oracle.bispectrum_grid(snap, bp)
    mlp = wl.random_mlp((B.shape[1], 16, 16, 21), seed=9, out_bias=1.0)
    mlp = wl.with_input_scaling(mlp, B.mean(0), 1.0 / (B.std(0) + 1e-12))
    eg = wl.EnergyGrid(n_E=21, e0_eV=-4.0, de_eV=0.4, kT_eV=0.1)
    P, vol = snap.n_points, float(snap.volume)
    dV = vol / P
    L = oracle.mlp_forward(B, mlp.W, mlp.b, mlp.leaky_slope, mlp.in_shift, mlp.in_scale)
    ne = oracle.electron_count(oracle.dos(L, dV), 0.0, eg.e0_eV, eg.de_eV, eg.kT_eV)
    model = api.Model(c, mlp)
    whole = c.band_forces(snap, bp, model, eg, api.FP64_PLAIN, n_electrons=ne)
    be = sharded.DeviceBackend(c, api.FP64_PLAIN).with_model(bp, model)
    slabs = [sharded.row_range(P, r, world) for r in range(world)]
    parts = [be.forward(snap, rows) for rows in slabs]
    sums = sum(be.column_sums(Lr) for _, Lr in parts)
    g = be.energy_gradient(dV * sums, eg, ne)
    F = sum(be.descriptor_forces(snap, be.ldos_backward(Br, dV * g), rows) for (Br, _), rows in zip(parts, slabs))
    scale = np.max(np.abs(whole["forces"]))
    np.testing.assert_allclose(F, whole["forces"], rtol=1e-9, atol=1e-9 * scale)
