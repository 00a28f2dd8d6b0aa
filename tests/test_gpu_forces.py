"""Band-energy forces on the GPU (Eqs. forces / forcesmala) against the FP64
oracle: each factor of the chain through its own C-ABI entry point, then the
whole chain, at small sizes (several tiles, ragged grids, two species) and on
the 729,000-point Al workload with beta sampled on 24 points."""
import numpy as np
import pytest

import oracle
from oracle import forces as of
from paper_2411_19617_gb300 import workloads as wl
from tests.gpu_util import ctx, need_gpu

pytestmark = pytest.mark.gpu


def _two_species(snap):
    return wl.Snapshot(pos=snap.pos, species=(np.arange(snap.n_atoms) % 2).astype(np.int32), cell=snap.cell,
                       grid=snap.grid)


def test_band_energy_gradient_matches_oracle():
    need_gpu()
    c = ctx()
    rng = np.random.default_rng(3)
    eg = wl.EnergyGrid(n_E=61, e0_eV=-4.0, de_eV=0.15, kT_eV=0.05)
    D = rng.uniform(0.2, 3.0, size=eg.n_E)
    Ne = oracle.electron_count(D, 0.4, eg.e0_eV, eg.de_eV, eg.kT_eV)
    got = c.band_energy_gradient(D, eg, n_electrons=Ne)
    ref = of.band_energy_gradient(D, eg.e0_eV, eg.de_eV, eg.kT_eV, Ne)
    assert got["fermi"] == pytest.approx(ref["fermi"], abs=1e-10)
    assert got["mu_tilde"] == pytest.approx(ref["mu_tilde"], abs=1e-9)
    np.testing.assert_allclose(got["grad"], ref["grad"], rtol=1e-9, atol=1e-10 * np.max(np.abs(ref["grad"])))


@pytest.mark.parametrize("precision,activate", [("fp64", False), ("mixed", False), ("fp64", True)])
def test_ldos_backward_matches_oracle(precision, activate):
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    c = ctx()
    rng = np.random.default_rng(4)
    mlp = wl.random_mlp((30, 64, 48, 21), seed=6, out_bias=0.5)
    mlp.in_shift = rng.normal(size=30)
    mlp.in_scale = rng.uniform(0.5, 2.0, size=30)
    P = 1000
    B = rng.normal(size=(P, 30))
    v = rng.normal(size=21)
    prec = api.MIXED if precision == "mixed" else api.FP64_PLAIN
    dt = torch.float32 if precision == "mixed" else torch.float64
    Bd = torch.tensor(B, dtype=dt, device="cuda")
    if activate:
        # a network whose output layer is activated (the LeakyReLU derivative there too)
        model = _model_with_output_activation(c, mlp)
    else:
        model = api.Model(c, mlp)
    beta = c.ldos_backward(model, Bd, v, prec).double().cpu().numpy()
    ref = of.ldos_backward(Bd.double().cpu().numpy(), mlp, v, activate_output=activate)
    if precision == "fp64":
        np.testing.assert_allclose(beta, ref, rtol=1e-10, atol=1e-12 * np.max(np.abs(ref)))
    else:
        rms = np.sqrt(np.mean(ref ** 2))
        assert np.max(np.abs(beta - ref)) < 2e-5 * rms * 30


def _model_with_output_activation(c, mlp):
    import ctypes as C
    from paper_2411_19617_gb300 import _lib, api
    m = api.Model.__new__(api.Model)
    m.ctx = c
    m.dims = tuple(int(d) for d in mlp.dims)
    nl = len(m.dims) - 1
    m._dims = np.ascontiguousarray(m.dims, dtype=np.int32)
    m._W = [np.ascontiguousarray(w, dtype=np.float64) for w in mlp.W]
    m._b = [np.ascontiguousarray(b, dtype=np.float64) for b in mlp.b]
    m._shift = np.ascontiguousarray(mlp.in_shift, dtype=np.float64)
    m._scale = np.ascontiguousarray(mlp.in_scale, dtype=np.float64)
    Wp = (C.POINTER(C.c_double) * nl)(*[w.ctypes.data_as(C.POINTER(C.c_double)) for w in m._W])
    bp = (C.POINTER(C.c_double) * nl)(*[b.ctypes.data_as(C.POINTER(C.c_double)) for b in m._b])
    d = _lib.MLPDesc()
    d.n_layers = nl
    d.dims = m._dims.ctypes.data_as(C.POINTER(C.c_int32))
    d.W = C.cast(Wp, C.POINTER(C.POINTER(C.c_double)))
    d.b = C.cast(bp, C.POINTER(C.POINTER(C.c_double)))
    d.leaky_slope = float(mlp.leaky_slope)
    d.activate_output = 1
    d.in_shift = m._shift.ctypes.data_as(C.POINTER(C.c_double))
    d.in_scale = m._scale.ctypes.data_as(C.POINTER(C.c_double))
    h = C.c_void_p()
    _lib.check(_lib.lib().mala_model_create(c.h, C.byref(d), C.byref(h)), "mala_model_create")
    m.h = h
    return m


@pytest.mark.parametrize("precision,tj,grid", [("fp64", 4, 8), ("fp64", 6, (7, 5, 6)), ("mixed", 6, 8),
                                               ("mixed", 10, (9, 7, 5)), ("fp64", 10, 5), ("mixed", 0, 5),
                                               ("mixed", 2, (7, 6, 5)), ("mixed", 4, (3, 11, 4)),
                                               ("mixed", 8, (6, 5, 7))])
def test_descriptor_forces_match_oracle(precision, tj, grid):
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    c = ctx()
    base = wl.al_fcc(2, 0.2, 8, seed=11)
    g = grid if isinstance(grid, tuple) else (grid,) * 3
    snap = _two_species(wl.Snapshot(pos=base.pos, species=base.species, cell=base.cell, grid=g))
    bp = wl.BispectrumParams(twojmax=tj, rcut=4.676, weights=(1.0, 0.7), wself=1.1)
    nB = len(oracle.triples(tj))
    rng = np.random.default_rng(tj)
    beta = rng.normal(size=(snap.n_points, nB))
    prec = api.MIXED if precision == "mixed" else api.FP64_PLAIN
    dt = torch.float32 if precision == "mixed" else torch.float64
    bd = torch.tensor(beta, dtype=dt, device="cuda")
    F = c.descriptor_forces(snap, bp, bd, prec)
    ref = of.descriptor_forces(snap, bp, bd.double().cpu().numpy())
    scale = np.max(np.abs(ref))
    tol = 1e-10 if precision == "fp64" else 2e-5
    assert np.max(np.abs(F - ref)) <= tol * scale, (np.max(np.abs(F - ref)), scale)


def test_descriptor_forces_edge_cases():
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    c = ctx()
    bp = wl.BispectrumParams(twojmax=4, rcut=4.676)
    nB = len(oracle.triples(4))
    # one atom in a large cell: most points see no neighbour; a 1x1x1 grid; no atoms at all
    one = wl.Snapshot(pos=np.array([[3.3, 4.1, 2.2]]), species=np.zeros(1, np.int32), cell=np.diag([12.0] * 3),
                      grid=(6, 6, 6))
    tiny = wl.Snapshot(pos=one.pos, species=one.species, cell=np.diag([5.0] * 3), grid=(1, 1, 1))
    for s in (one, tiny):
        beta = np.random.default_rng(1).normal(size=(s.n_points, nB))
        F = c.descriptor_forces(s, bp, torch.tensor(beta, device="cuda"), api.FP64_PLAIN)
        ref = of.descriptor_forces(s, bp, beta)
        np.testing.assert_allclose(F, ref, rtol=1e-10, atol=1e-10 * max(1.0, np.max(np.abs(ref))))
    empty = wl.Snapshot(pos=np.zeros((0, 3)), species=np.zeros(0, np.int32), cell=np.diag([7.0] * 3), grid=(4, 4, 4))
    F = c.descriptor_forces(empty, bp, torch.zeros((64, nB), dtype=torch.float64, device="cuda"), api.FP64_PLAIN)
    assert F.shape == (0, 3)


def _chain_case():
    snap = wl.al_fcc(2, 0.15, 8, seed=8)
    bp = wl.BispectrumParams(twojmax=6, rcut=4.676)
    B = oracle.bispectrum_grid(snap, bp, nthreads=8)
    mlp = wl.random_mlp((B.shape[1], 48, 48, 31), seed=9, out_bias=1.0)
    mlp = wl.with_input_scaling(mlp, B.mean(0), 1.0 / (B.std(0) + 1e-12))
    eg = wl.EnergyGrid(n_E=31, e0_eV=-4.0, de_eV=0.3, kT_eV=0.1)
    dV = float(snap.volume) / snap.n_points
    L = oracle.mlp_forward(B, mlp.W, mlp.b, mlp.leaky_slope, mlp.in_shift, mlp.in_scale)
    Ne = oracle.electron_count(oracle.dos(L, dV), 0.0, eg.e0_eV, eg.de_eV, eg.kT_eV)
    return snap, bp, mlp, eg, Ne


def test_band_forces_fp64_match_oracle():
    need_gpu()
    from paper_2411_19617_gb300 import api
    c = ctx()
    snap, bp, mlp, eg, Ne = _chain_case()
    model = api.Model(c, mlp)
    got = c.band_forces(snap, bp, model, eg, api.FP64_PLAIN, n_electrons=Ne)
    ref = of.band_forces(snap, bp, mlp, eg, Ne)
    assert got["fermi"] == pytest.approx(ref["fermi"], abs=1e-9)
    assert got["band_energy"] == pytest.approx(ref["band_energy"], rel=1e-10)
    scale = np.max(np.abs(ref["forces"]))
    assert np.max(np.abs(got["forces"] - ref["forces"])) <= 1e-8 * scale


def test_band_forces_mixed_track_oracle():
    # BF16 LDOS moves D and e_F by ~1e-3 relative; forces follow to that order
    need_gpu()
    from paper_2411_19617_gb300 import api
    c = ctx()
    snap, bp, mlp, eg, Ne = _chain_case()
    model = api.Model(c, mlp)
    got = c.band_forces(snap, bp, model, eg, api.MIXED, n_electrons=Ne)
    ref = of.band_forces(snap, bp, mlp, eg, Ne)
    F, R = got["forces"], ref["forces"]
    assert np.max(np.abs(F - R)) <= 3e-2 * np.max(np.abs(R))
    assert np.corrcoef(F.ravel(), R.ravel())[0, 1] > 0.999


def test_descriptor_forces_full_al_workload_sampled():
    # the 90^3-point Al workload (256 atoms, twojmax 10): beta nonzero on 24 sampled points
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    c = ctx()
    snaps, bp, _, _, _ = wl.config(2)
    s = snaps[0]
    pts = wl.sample_points(s.n_points, 24, seed=3)
    rng = np.random.default_rng(0)
    bs = rng.normal(size=(24, 91))
    beta = torch.zeros((s.n_points, 91), dtype=torch.float32, device="cuda")
    beta[torch.tensor(pts, device="cuda")] = torch.tensor(bs, dtype=torch.float32, device="cuda")
    F = c.descriptor_forces(s, bp, beta, api.MIXED)
    ref = of.descriptor_forces(s, bp, bs.astype(np.float32).astype(np.float64), points=pts)
    assert np.max(np.abs(F - ref)) <= 2e-5 * np.max(np.abs(ref))
