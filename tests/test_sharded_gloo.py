"""The exchange step of the grid-sharded path (DOS all-reduce before a
replicated Fermi-level bisection) with two CPU ranks over gloo: every rank
gets the single-rank D(e), e_F, E_b and electron count, and its own rows of
n(r).  The per-rank arithmetic is the oracle's (the orchestration under test
holds none of the method's arithmetic)."""
import os
import socket

import numpy as np
import pytest

from paper_2411_19617_gb300 import sharded
from paper_2411_19617_gb300.workloads import EnergyGrid

NE = 24
EG = EnergyGrid(n_E=NE, e0_eV=-4.0, de_eV=0.35, kT_eV=0.0259)


def synthetic_ldos(P, seed=3):
    """Positive LDOS rows: a few Gaussians per point on the energy grid."""
    rng = np.random.default_rng(seed)
    e = EG.e0_eV + EG.de_eV * np.arange(NE)
    centres = rng.uniform(e[2], e[-3], size=(P, 3))
    L = np.zeros((P, NE))
    for k in range(3):
        L += rng.uniform(0.2, 1.0, size=(P, 1)) * np.exp(-((e[None, :] - centres[:, k:k + 1]) / 0.6) ** 2)
    return L


class OracleBackend:
    def column_sums(self, L):
        return np.asarray(L, np.float64).sum(axis=0)

    def integrate(self, L, sums, dV, eg, n_electrons):
        import oracle
        D = dV * np.asarray(sums, np.float64)
        eF = oracle.fermi_level(D, eg.e0_eV, eg.de_eV, eg.kT_eV, n_electrons)
        w0 = oracle.integration_weights(0, eg.e0_eV, eg.de_eV, NE, eF, eg.kT_eV)
        w1 = oracle.integration_weights(1, eg.e0_eV, eg.de_eV, NE, eF, eg.kT_eV)
        return {"fermi": eF, "band_energy": float(np.dot(w1, D)), "density": np.asarray(L) @ w0}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, P, volume, ne, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        L = synthetic_ldos(P)
        r0, r1 = sharded.row_range(P, rank, world)
        res = sharded.integrate_sharded(OracleBackend(), L[r0:r1], P, volume, EG, ne, group=dist.group.WORLD)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), dos=res["dos"], fermi=res["fermi"],
                 band_energy=res["band_energy"], density=res["density"], electron_count=res["electron_count"],
                 r0=r0, r1=r1)
    finally:
        dist.destroy_process_group()


def test_row_range_partitions_the_rows():
    for P in (0, 1, 7, 64, 1001):
        for world in (1, 2, 3, 8):
            ranges = [sharded.row_range(P, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == P
            for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
                assert a1 == b0
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        sharded.row_range(10, 2, 2)


def test_single_rank_matches_the_oracle():
    import oracle
    P, volume = 301, 250.0
    L = synthetic_ldos(P)
    dV = volume / P
    ne = oracle.electron_count(oracle.dos(L, dV), 0.0, EG.e0_eV, EG.de_eV, EG.kT_eV)  # reachable: N(mu = 0)
    ref = oracle.observables(L, dV, EG.e0_eV, EG.de_eV, EG.kT_eV, ne)
    got = sharded.integrate_sharded(OracleBackend(), L, P, volume, EG, ne, group=None)
    np.testing.assert_allclose(got["dos"], ref["dos"], rtol=1e-14)
    assert got["fermi"] == ref["fermi"]
    assert got["band_energy"] == pytest.approx(ref["band_energy"], rel=1e-14)
    np.testing.assert_allclose(got["density"], ref["density"], rtol=1e-14)
    assert got["electron_count"] == pytest.approx(ne, rel=1e-6)


def test_two_gloo_ranks_reproduce_the_single_rank_result(tmp_path):
    import multiprocessing as mp

    import oracle
    P, volume = 301, 250.0  # odd: the slabs differ by one row
    L = synthetic_ldos(P)
    dV = volume / P
    ne = oracle.electron_count(oracle.dos(L, dV), 0.0, EG.e0_eV, EG.de_eV, EG.kT_eV)  # reachable: N(mu = 0)
    ref = oracle.observables(L, dV, EG.e0_eV, EG.de_eV, EG.kT_eV, ne)
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, P, volume, ne, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(2)]
    # every rank holds the same global quantities, bit for bit
    for k in ("dos", "fermi", "band_energy", "electron_count"):
        np.testing.assert_array_equal(res[0][k], res[1][k])
    # and they match the single-rank oracle (the sums differ only in order)
    np.testing.assert_allclose(res[0]["dos"], ref["dos"], rtol=1e-13)
    assert float(res[0]["fermi"]) == pytest.approx(ref["fermi"], abs=1e-10)
    assert float(res[0]["band_energy"]) == pytest.approx(ref["band_energy"], rel=1e-10)
    assert float(res[0]["electron_count"]) == pytest.approx(ne, rel=1e-6)
    dens = np.concatenate([res[r]["density"] for r in range(2)])
    assert int(res[0]["r1"]) == int(res[1]["r0"])
    np.testing.assert_allclose(dens, ref["density"], rtol=1e-9)
