"""Grid-centred ACE descriptors on the GPU against the FP64 oracle (oracle/ace.py):
small snapshots (one and two species, ragged grids, an atom on a grid point,
no atoms) on every point, and the 729,000-point Al workload on sampled points."""
import numpy as np
import pytest

from oracle import ace
from paper_2411_19617_gb300 import workloads as wl
from tests.gpu_util import ctx, descriptor_error, need_gpu

pytestmark = pytest.mark.gpu


def _two_species(snap):
    return wl.Snapshot(pos=snap.pos, species=(np.arange(snap.n_atoms) % 2).astype(np.int32), cell=snap.cell,
                       grid=snap.grid)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", ["al", "two_species", "ragged"])
def test_ace_matches_oracle(precision, case):
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    c = ctx()
    base = wl.al_fcc(2, 0.2, 6, seed=12)
    if case == "al":
        snap, ap = base, ace.AceParams(rcut=4.676, nmax1=6, nmax2=4, lmax2=6, nmax3=3, lmax3=4)
    elif case == "two_species":
        snap = _two_species(base)
        ap = ace.AceParams(rcut=5.0, n_species=2, nmax1=3, nmax2=3, lmax2=4, nmax3=2, lmax3=4)
    else:
        snap = wl.Snapshot(pos=base.pos, species=base.species, cell=base.cell, grid=(7, 5, 3))
        ap = ace.AceParams(rcut=4.676, nmax1=4, nmax2=3, lmax2=8, nmax3=2, lmax3=6)
    prec = api.MIXED if precision == "mixed" else api.FP64_PLAIN
    D = c.ace_descriptors(snap, ap, prec).double().cpu().numpy()
    ref = ace.ace_grid(snap, ap)
    err = descriptor_error(D, ref)
    assert err < (1e-10 if precision == "fp64" else 2e-5), err


def test_ace_edge_cases():
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    c = ctx()
    ap = ace.AceParams(rcut=4.0, nmax1=3, nmax2=2, lmax2=3, nmax3=2, lmax3=2)
    # an atom exactly on a grid point (no direction: l = 0 only) and one elsewhere
    on = wl.Snapshot(pos=np.array([[2.0, 2.0, 2.0], [3.1, 2.4, 1.3]]), species=np.zeros(2, np.int32),
                     cell=np.diag([8.0] * 3), grid=(4, 4, 4))
    D = c.ace_descriptors(on, ap, api.FP64_PLAIN).cpu().numpy()
    np.testing.assert_allclose(D, ace.ace_grid(on, ap), rtol=1e-10, atol=1e-12)
    empty = wl.Snapshot(pos=np.zeros((0, 3)), species=np.zeros(0, np.int32), cell=np.diag([7.0] * 3), grid=(3, 3, 3))
    D = c.ace_descriptors(empty, ap, api.FP64_PLAIN).cpu().numpy()
    assert D.shape == (27, api.ace_count(ap)) and np.all(D == 0.0)


def test_ace_full_al_workload_sampled():
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    c = ctx()
    snaps, _, _, _, _ = wl.config(2)
    s = snaps[0]
    ap = ace.AceParams(rcut=4.676)
    D = c.ace_descriptors(s, ap, api.MIXED)
    pts = wl.sample_points(s.n_points, 24, seed=9)
    got = D[torch.as_tensor(pts, device=D.device)].double().cpu().numpy()
    ref = ace.ace_grid(s, ap, points=pts)
    assert descriptor_error(got, ref) < 2e-5


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_ace_tables_in_global_memory(precision):
    """A column set whose tables exceed what the kernel stages in shared memory (96 KB): 2,501
    columns, whose column table alone takes 97.7 KB at 40 bytes a column, so the kernel reads the
    column and coefficient tables from global memory; sampled points against the oracle."""
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    c = ctx()
    snap = wl.al_fcc(2, 0.2, 6, seed=12)
    ap = ace.AceParams(rcut=4.676, nmax1=2, nmax2=2, lmax2=2, nmax3=5, lmax3=6)
    assert api.ace_count(ap) * 40 > 96 * 1024
    prec = api.MIXED if precision == "mixed" else api.FP64_PLAIN
    D = c.ace_descriptors(snap, ap, prec)
    pts = wl.sample_points(snap.n_points, 6, seed=4)
    got = D[torch.as_tensor(pts, device=D.device)].double().cpu().numpy()
    ref = ace.ace_grid(snap, ap, points=pts)
    err = descriptor_error(got, ref)
    assert err < (1e-10 if precision == "fp64" else 2e-5), err
