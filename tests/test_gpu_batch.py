"""Batched snapshots: descriptors of uneven snapshots in one sequence of
launches are bit for bit the per-snapshot descriptors, the batched whole path
matches per-snapshot predictions, and the boron-cluster workload (uneven
clusters in vacuum, twojmax 10) matches the FP64 oracle on sampled points."""
import numpy as np
import pytest

import oracle
from paper_2411_19617_gb300 import workloads as wl
from tests.gpu_util import ctx, descriptor_error, need_gpu

pytestmark = pytest.mark.gpu


def _mixed_batch(seed):
    """Snapshots of different atom counts, cells and grids (odd tile counts included)."""
    rng = np.random.default_rng(seed)
    snaps = [wl.boron_cluster(int(n), 12.0, g, rng) for n, g in ((9, 21), (40, 30), (77, 17))]
    snaps.append(wl.al_fcc(2, 0.1, 18, seed=seed))
    snaps.append(wl.bulk_snapshot("Be", 50, rng, spacing=0.45))
    return snaps


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_descriptors_equal_single_snapshot_descriptors(precision):
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    prec = api.MIXED if precision == "mixed" else api.FP64_PLAIN
    c = ctx()
    bp = wl.BispectrumParams(twojmax=6 if precision == "fp64" else 10, rcut=4.676)
    snaps = _mixed_batch(seed=21)
    Bb = c.descriptors_batch(snaps, bp, prec).cpu().numpy()
    row = 0
    for s in snaps:
        B1 = c.descriptors(s, bp, prec).cpu().numpy()
        np.testing.assert_array_equal(Bb[row:row + s.n_points], B1)
        row += s.n_points
    assert row == Bb.shape[0]


def test_batch_predict_matches_single_predictions():
    need_gpu()
    from paper_2411_19617_gb300 import api
    c = ctx()
    bp = wl.BispectrumParams(twojmax=10, rcut=4.676)
    snaps = _mixed_batch(seed=5)
    mlp = wl.random_mlp((91, 400, 400, 11), seed=3, out_bias=1.0)
    B = c.descriptors_batch(snaps, bp).double()
    mlp = wl.with_input_scaling(mlp, B.mean(0).cpu().numpy(), 1.0 / (B.std(0).cpu().numpy() + 1e-12))
    model = api.Model(c, mlp)
    eg = wl.EnergyGrid(n_E=11, e0_eV=-5.0, de_eV=1.0)
    nes = []
    for s in snaps:
        r = c.predict(s, bp, model, eg, api.MIXED, n_electrons=0.0, raise_on_bracket=False)
        nes.append(c.electron_count(r["dos"], eg, 0.0))
    alone = []
    for s, ne in zip(snaps, nes):
        d = np.zeros(s.n_points, np.float32)
        r = c.predict(s, bp, model, eg, api.MIXED, n_electrons=ne, density_host=d)
        alone.append((r["ldos"].float().cpu().numpy(), r["dos"], r["fermi"], r["band_energy"], d))
    dens = np.zeros(sum(s.n_points for s in snaps), np.float32)
    res = c.predict_batch(snaps, bp, model, eg, api.MIXED, n_electrons=nes, density_host=dens)
    row = 0
    for s, r, (L1, D1, eF1, Eb1, d1), ne in zip(snaps, res, alone, nes):
        assert r["n_points"] == s.n_points and r["status"] == 0
        # the network rows are the same computation: bit for bit
        np.testing.assert_array_equal(r["ldos"].float().cpu().numpy(), L1)
        # the integrals sum the same BF16 values in another blocking
        np.testing.assert_allclose(r["dos"], D1, rtol=1e-6)
        assert r["fermi"] == pytest.approx(eF1, abs=1e-6)
        assert r["band_energy"] == pytest.approx(Eb1, rel=1e-6)
        np.testing.assert_allclose(dens[row:row + s.n_points], d1, rtol=1e-5, atol=1e-6)
        assert r["electron_count"] == pytest.approx(ne, rel=1e-6)
        row += s.n_points


def test_boron_cluster_batch_matches_oracle_on_sampled_points():
    need_gpu()
    from paper_2411_19617_gb300 import api
    c = ctx()
    snaps, bp, mlp, eg, _ = wl.config(3)
    snaps = snaps[:6]  # six clusters of the 64-cluster workload (90^3 points each)
    B = c.descriptors_batch(snaps, bp, api.MIXED)
    row = 0
    for i, s in enumerate(snaps):
        pts = wl.sample_points(s.n_points, 24, seed=100 + i)
        ref = oracle.bispectrum_grid(s, bp, points=pts, nthreads=8)
        got = B[row:row + s.n_points][pts].double().cpu().numpy()
        # clusters in vacuum: many points have no neighbour, B = u_self^3 there;
        # scale errors by each component's RMS over the sample
        assert descriptor_error(got, ref) < 1e-5, f"cluster {i}"
        row += s.n_points


def test_batch_with_empty_and_single_point_snapshots():
    # a snapshot without atoms (closed form w_self^3 (J+1)), a 1x1x1 grid and a ragged one in one batch
    need_gpu()
    from paper_2411_19617_gb300 import api
    c = ctx()
    bp = wl.BispectrumParams(twojmax=8, rcut=4.676, wself=1.25)
    empty = wl.Snapshot(pos=np.zeros((0, 3)), species=np.zeros(0, np.int32), cell=np.diag([7.0] * 3),
                        grid=(5, 3, 3))
    one = wl.al_fcc(2, 0.1, 1, seed=4)
    ragged = wl.al_fcc(2, 0.1, 7, seed=5)
    snaps = [empty, one, ragged, empty]
    Bb = c.descriptors_batch(snaps, bp).double().cpu().numpy()
    tr = oracle.triples(8)
    closed = 1.25 ** 3 * (tr[:, 2] + 1)
    np.testing.assert_allclose(Bb[:empty.n_points], np.broadcast_to(closed, (empty.n_points, len(tr))), rtol=1e-6)
    np.testing.assert_allclose(Bb[-empty.n_points:], np.broadcast_to(closed, (empty.n_points, len(tr))), rtol=1e-6)
    row = empty.n_points
    for s in (one, ragged):
        ref = oracle.bispectrum_grid(s, bp, nthreads=8)
        assert descriptor_error(Bb[row:row + s.n_points], ref) < 1e-5
        row += s.n_points
