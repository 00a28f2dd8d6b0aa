"""GPU parity of the descriptor step (neighbour lists, u, B) against the FP64
oracle, through the C ABI.  Bars: neighbour membership bit-exact; B within
1e-5 of the oracle in |dB| / max(|B_ref|, RMS_component) for the FP32 path
(the error of FP32-stored u bounds what any FP32 path reaches below the RMS
scale); the FP64 path within 1e-10 even with the floor at 1e-3 RMS."""
import numpy as np
import pytest

import oracle
from paper_2411_19617_gb300 import workloads as wl
from tests.gpu_util import ctx, descriptor_error, need_gpu, neighbor_sets

pytestmark = pytest.mark.gpu

RC = 4.676
TOL32 = 1e-5
TOL64 = 1e-10


def _cubic(pos, L, grid, periodic=(1, 1, 1)):
    pos = np.asarray(pos, np.float64).reshape(-1, 3)
    return wl.Snapshot(pos=pos, species=np.zeros(len(pos), np.int32), cell=np.diag([float(L)] * 3), grid=grid,
                       periodic=periodic)


def _check_neighbors(snap, rcut, points=None):
    from paper_2411_19617_gb300 import api  # noqa: F401
    c = ctx()
    cnt, at, sh, mx = c.neighbor_lists(snap, rcut, cap=256)
    cnt, at, sh = cnt.cpu().numpy(), at.cpu().numpy(), sh.cpu().numpy()
    pts = np.arange(snap.n_points) if points is None else points
    rc, ra, rs = oracle.neighbor_lists(snap, rcut, points=pts, cap=256)
    np.testing.assert_array_equal(cnt[pts], rc)
    assert neighbor_sets(cnt, at, sh, pts) == neighbor_sets(rc, ra, rs, range(len(pts)))
    assert mx == int(rc.max()) if points is None else mx >= int(rc.max())


def test_neighbors_bit_exact_al_small():
    need_gpu()
    snaps, bp, *_ = wl.config(1)
    _check_neighbors(snaps[0], bp.rcut)


def test_neighbors_box_smaller_than_cutoff_and_ragged_grid():
    need_gpu()
    rng = np.random.default_rng(3)
    snap = _cubic(rng.uniform(-1.0, 4.0, size=(5, 3)), 3.1, (5, 7, 3))
    _check_neighbors(snap, RC)


def test_neighbors_open_axes_and_atoms_outside_cell():
    need_gpu()
    rng = np.random.default_rng(4)
    snap = _cubic(rng.uniform(-3.0, 11.0, size=(40, 3)), 8.0, (9, 6, 5), periodic=(1, 0, 0))
    _check_neighbors(snap, RC)


def test_neighbors_exact_ties_on_the_sphere():
    # atoms placed exactly at distance rcut (and one ulp inside/outside) from grid points
    need_gpu()
    L, n = 8.0, 8
    rc = 2.0
    pos = [[2.0, 1.0, 1.0], [1.0, 1.0 + np.nextafter(2.0, 0.0), 1.0], [1.0, 1.0, 1.0 + np.nextafter(2.0, 3.0)]]
    snap = _cubic(pos, L, (n, n, n))
    _check_neighbors(snap, rc)


def test_neighbors_be_slab_sampled():
    need_gpu()
    snap = wl.be_slab()
    pts = wl.sample_points(snap.n_points, 400, seed=7)
    _check_neighbors(snap, 4.5, points=pts)


def test_expansion_coefficients_match_oracle():
    need_gpu()
    from paper_2411_19617_gb300 import api
    snaps, bp, *_ = wl.config(1)
    snap = snaps[0]
    u = ctx().expansion_coefficients(snap, bp, api.MIXED).double().cpu().numpy()
    for p in (0, 1, 77, 1234, snap.n_points - 1):
        ref, _ = oracle.u_at_point(snap, bp, p)
        flat = np.concatenate([b.ravel() for b in ref])
        got = u[p, :, 0] + 1j * u[p, :, 1]
        assert np.max(np.abs(got - flat)) < 2e-6 * max(1.0, np.max(np.abs(flat)))


@pytest.mark.parametrize("twojmax", [0, 2, 4, 6, 8, 10])
def test_descriptors_all_twojmax(twojmax):
    need_gpu()
    from paper_2411_19617_gb300 import api
    snap = wl.al_fcc(2, 0.2, 7, seed=5)
    bp = wl.BispectrumParams(twojmax=twojmax, rcut=RC)
    B = ctx().descriptors(snap, bp, api.MIXED).double().cpu().numpy()
    ref = oracle.bispectrum_grid(snap, bp)
    assert B.shape == ref.shape
    assert descriptor_error(B, ref) < TOL32


def test_descriptors_al_small_fp32_and_fp64():
    need_gpu()
    from paper_2411_19617_gb300 import api
    snaps, bp, *_ = wl.config(1)
    snap = snaps[0]
    ref = oracle.bispectrum_grid(snap, bp, nthreads=8)
    B32 = ctx().descriptors(snap, bp, api.MIXED).double().cpu().numpy()
    assert descriptor_error(B32, ref) < TOL32
    B64 = ctx().descriptors(snap, bp, api.FP64_PLAIN).cpu().numpy()
    assert descriptor_error(B64, ref, floor=1e-3) < TOL64


def test_descriptors_al_liquid_full_size_sampled():
    need_gpu()
    from paper_2411_19617_gb300 import api
    snaps, bp, *_ = wl.config(2)
    snap = snaps[0]
    B = ctx().descriptors(snap, bp, api.MIXED).double().cpu().numpy()
    pts = wl.sample_points(snap.n_points, 300, seed=11)
    ref = oracle.bispectrum_grid(snap, bp, points=pts, nthreads=8)
    assert descriptor_error(B[pts], ref) < TOL32
    assert np.all(np.isfinite(B))


def test_descriptors_boron_clusters_sampled():
    need_gpu()
    from paper_2411_19617_gb300 import api
    snaps, bp, *_ = wl.config(3)
    for snap in snaps[:3]:
        B = ctx().descriptors(snap, bp, api.MIXED).double().cpu().numpy()
        # points near the cluster (nonzero neighbourhoods) and in vacuum
        pts = wl.sample_points(snap.n_points, 200, seed=snap.n_atoms)
        ref = oracle.bispectrum_grid(snap, bp, points=pts, nthreads=8)
        assert descriptor_error(B[pts], ref) < TOL32


def test_descriptors_be_slab_full_size_sampled():
    # the stacking-fault slab, ~2e7 points streamed in tile chunks: bulk, fault plane and vacuum
    need_gpu()
    from paper_2411_19617_gb300 import api
    snaps, bp, *_ = wl.config(4)
    snap = snaps[0]
    B = ctx().descriptors(snap, bp, api.MIXED)
    pts = wl.sample_points(snap.n_points, 120, seed=44)
    got = B[torch_index(pts, B.device)].double().cpu().numpy()
    ref = oracle.bispectrum_grid(snap, bp, points=pts, nthreads=8)
    assert descriptor_error(got, ref) < TOL32
    del B


def torch_index(pts, device):
    import torch
    return torch.as_tensor(pts, device=device)


def test_descriptors_empty_cell_is_self_term_only():
    # no atoms: u^J = wself I, so B_{J1 J2 J} = wself^3 (J+1) (Clebsch-Gordan orthonormality)
    need_gpu()
    from paper_2411_19617_gb300 import api
    snap = wl.Snapshot(pos=np.zeros((0, 3)), species=np.zeros(0, np.int32), cell=np.diag([5.0] * 3),
                       grid=(3, 2, 5))
    bp = wl.BispectrumParams(twojmax=6, rcut=RC, wself=1.5)
    B = ctx().descriptors(snap, bp, api.MIXED).double().cpu().numpy()
    tr = oracle.triples(6)
    np.testing.assert_allclose(B, np.broadcast_to(1.5 ** 3 * (tr[:, 2] + 1), B.shape), rtol=1e-6)


def test_descriptors_species_weights():
    need_gpu()
    from paper_2411_19617_gb300 import api
    snap = wl.al_fcc(2, 0.2, 6, seed=9)
    snap.species = (np.arange(snap.n_atoms) % 2).astype(np.int32)
    bp = wl.BispectrumParams(twojmax=4, rcut=RC, weights=(1.0, 0.4))
    B = ctx().descriptors(snap, bp, api.MIXED).double().cpu().numpy()
    ref = oracle.bispectrum_grid(snap, bp)
    assert descriptor_error(B, ref) < TOL32


def test_descriptor_argument_errors():
    need_gpu()
    from paper_2411_19617_gb300 import api
    from paper_2411_19617_gb300._lib import MalaError
    snap = wl.al_fcc(1, 0.0, 4, seed=1)
    with pytest.raises(MalaError):
        ctx().descriptors(snap, wl.BispectrumParams(twojmax=5, rcut=RC), api.MIXED)
    with pytest.raises(MalaError):
        ctx().descriptors(snap, wl.BispectrumParams(twojmax=12, rcut=RC), api.MIXED)
    with pytest.raises(MalaError):
        ctx().descriptors(snap, wl.BispectrumParams(twojmax=4, rcut=-1.0), api.MIXED)
    bad = wl.Snapshot(pos=snap.pos.copy(), species=snap.species, cell=snap.cell, grid=snap.grid)
    bad.pos[0, 0] = np.nan
    with pytest.raises(MalaError):
        ctx().descriptors(bad, wl.BispectrumParams(twojmax=4, rcut=RC), api.MIXED)
    tri = wl.Snapshot(pos=snap.pos, species=snap.species, cell=np.array([[4.0, 0.5, 0], [0, 4.0, 0], [0, 0, 4.0]]),
                      grid=snap.grid)
    with pytest.raises(MalaError):
        ctx().descriptors(tri, wl.BispectrumParams(twojmax=4, rcut=RC), api.MIXED)
    sp = wl.Snapshot(pos=snap.pos, species=np.full(snap.n_atoms, 3, np.int32), cell=snap.cell, grid=snap.grid)
    with pytest.raises(MalaError):
        ctx().descriptors(sp, wl.BispectrumParams(twojmax=4, rcut=RC), api.MIXED)
