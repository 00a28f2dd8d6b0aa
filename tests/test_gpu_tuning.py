"""Tile-shape tuning: every compiled variant of compute_ui (segment length x
warps per CTA) and compute_zi/bi (warps per CTA) adds the same terms in the same
order, so each gives the default's descriptors bit for bit, and those match the
FP64 oracle; the autotuner times them on the first pass of a key, records its
choice, and later passes give the same bits."""
import numpy as np
import pytest

import oracle
from paper_2411_19617_gb300 import workloads as wl
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("twojmax,grid", [(10, 14), (6, 11)])
def test_every_variant_gives_the_same_bits_and_oracle_parity(twojmax, grid):
    need_gpu()
    from paper_2411_19617_gb300 import api
    n_ui, n_zb = api.tuning_variants()
    assert n_ui >= 2 and n_zb >= 2
    c = api.Context(0)
    snap = wl.al_fcc(2, 0.2, grid, seed=4)  # ragged tiles: 14 and 11 are not multiples of the 4x4x2 tile
    bp = wl.BispectrumParams(twojmax=twojmax, rcut=4.676)
    c.set_tuning(0)
    ref = c.descriptors(snap, bp, api.MIXED).cpu().numpy()
    pts = np.arange(0, snap.n_points, 7)
    Bo = oracle.bispectrum_grid(snap, bp, points=pts)
    rms = np.sqrt(np.mean(Bo ** 2, axis=0))
    assert np.max(np.abs(ref[pts] - Bo) / np.maximum(np.abs(Bo), rms)) < 1e-5
    for u in range(n_ui):
        for z in range(n_zb):
            c.set_tuning(2, u, z)
            B = c.descriptors(snap, bp, api.MIXED).cpu().numpy()
            assert np.array_equal(B, ref), (u, z)
    c.set_tuning(1)
    first = c.descriptors(snap, bp, api.MIXED).cpu().numpy()   # the pass that times the variants
    again = c.descriptors(snap, bp, api.MIXED).cpu().numpy()   # the pass that uses the choice
    assert np.array_equal(first, ref) and np.array_equal(again, ref)
    rep = c.tuning_report()
    assert f"twojmax={twojmax}" in rep and "compute_ui" in rep and "compute_zi/bi" in rep, rep
    with pytest.raises(Exception):
        c.set_tuning(2, n_ui, 0)
    c.close()
