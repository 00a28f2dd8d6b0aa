"""The sharded band-energy forces (paper_2411_19617_gb300.sharded.forces_sharded)
with two CPU ranks over gloo: each rank holds half of the grid rows, the DOS
and then the per-atom partial forces are all-reduced, and every rank ends with
the single-rank forces.  The per-rank arithmetic is the oracle's."""
import os
import socket

import numpy as np
import pytest

from paper_2411_19617_gb300 import sharded
from paper_2411_19617_gb300 import workloads as wl

pytest.importorskip("torch")


def _case():
    import oracle
    snap = wl.al_fcc(2, 0.15, 6, seed=8)
    bp = wl.BispectrumParams(twojmax=4, rcut=4.676)
    B = oracle.bispectrum_grid(snap, bp)
    mlp = wl.random_mlp((B.shape[1], 16, 16, 21), seed=9, out_bias=1.0)
    mlp = wl.with_input_scaling(mlp, B.mean(0), 1.0 / (B.std(0) + 1e-12))
    eg = wl.EnergyGrid(n_E=21, e0_eV=-4.0, de_eV=0.4, kT_eV=0.1)
    dV = float(snap.volume) / snap.n_points
    L = oracle.mlp_forward(B, mlp.W, mlp.b, mlp.leaky_slope, mlp.in_shift, mlp.in_scale)
    ne = oracle.electron_count(oracle.dos(L, dV), 0.0, eg.e0_eV, eg.de_eV, eg.kT_eV)
    return snap, bp, mlp, eg, ne


class OracleForcesBackend:
    def __init__(self, bp, mlp):
        self.bp, self.mlp = bp, mlp

    def forward(self, snap, rows):
        import oracle
        pts = np.arange(rows[0], rows[1])
        B = oracle.bispectrum_grid(snap, self.bp, points=pts)
        m = self.mlp
        return B, oracle.mlp_forward(B, m.W, m.b, m.leaky_slope, m.in_shift, m.in_scale)

    def column_sums(self, L):
        return np.asarray(L, np.float64).sum(axis=0)

    def integrate(self, L, sums, dV, eg, n_electrons):
        import oracle
        D = dV * np.asarray(sums, np.float64)
        eF = oracle.fermi_level(D, eg.e0_eV, eg.de_eV, eg.kT_eV, n_electrons)
        w0 = oracle.integration_weights(0, eg.e0_eV, eg.de_eV, eg.n_E, eF, eg.kT_eV)
        w1 = oracle.integration_weights(1, eg.e0_eV, eg.de_eV, eg.n_E, eF, eg.kT_eV)
        return {"fermi": eF, "band_energy": float(np.dot(w1, D)), "density": np.asarray(L) @ w0}

    def energy_gradient(self, D, eg, n_electrons):
        from oracle import forces as of
        return of.band_energy_gradient(D, eg.e0_eV, eg.de_eV, eg.kT_eV, n_electrons)["grad"]

    def ldos_backward(self, B, v):
        from oracle import forces as of
        return of.ldos_backward(B, self.mlp, v)

    def descriptor_forces(self, snap, beta, rows):
        from oracle import forces as of
        return of.descriptor_forces(snap, self.bp, beta, points=np.arange(rows[0], rows[1]))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        snap, bp, mlp, eg, ne = _case()
        rows = sharded.row_range(snap.n_points, rank, world)
        res = sharded.forces_sharded(OracleForcesBackend(bp, mlp), snap, rows, float(snap.volume), eg, ne,
                                     group=dist.group.WORLD)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), forces=res["forces"], fermi=res["fermi"],
                 band_energy=res["band_energy"])
    finally:
        dist.destroy_process_group()


def test_single_rank_forces_match_the_oracle_chain():
    from oracle import forces as of
    snap, bp, mlp, eg, ne = _case()
    got = sharded.forces_sharded(OracleForcesBackend(bp, mlp), snap, (0, snap.n_points), float(snap.volume), eg, ne)
    ref = of.band_forces(snap, bp, mlp, eg, ne)
    np.testing.assert_allclose(got["forces"], ref["forces"], rtol=1e-12, atol=1e-12 * np.max(np.abs(ref["forces"])))


def test_two_gloo_ranks_reproduce_the_single_rank_forces(tmp_path):
    import multiprocessing as mp

    from oracle import forces as of
    snap, bp, mlp, eg, ne = _case()
    ref = of.band_forces(snap, bp, mlp, eg, ne)
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(2)]
    np.testing.assert_array_equal(res[0]["forces"], res[1]["forces"])  # one all-reduce result on every rank
    scale = np.max(np.abs(ref["forces"]))
    np.testing.assert_allclose(res[0]["forces"], ref["forces"], rtol=1e-10, atol=1e-10 * scale)
    assert float(res[0]["band_energy"]) == pytest.approx(ref["band_energy"], rel=1e-10)
