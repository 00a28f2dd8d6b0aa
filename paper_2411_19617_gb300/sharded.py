"""Grid-sharded LDOS integrals: the one exchange step of the multi-GPU path.

Grid points are independent up to the integrals of Sec. "Observable
calculation": each rank holds a contiguous slab of LDOS rows, and the only
quantity that couples the slabs is the DOS D(e_xi) = dV sum_r L(r, xi)
(Eq. DOS.from.ldos).  A rank therefore

1. sums its own rows per energy (FP64 column sums),
2. all-reduces the N_E sums (sum, FP64) so every rank holds the global D,
3. runs the Fermi-level bisection and the band energy on that D (the same
   input on every rank, so the same e_F everywhere), and
4. evaluates n(r) = sum_xi w0_xi(e_F) L(r, xi) (Eq. density.from.ldos) on its
   own rows; the electron-count check dV sum_r n(r) is all-reduced too.

The band-energy forces (Eq. forcesmala with E = E_b) shard the same way: with
the global D every rank forms the same dE_b/dD, runs the network's backward
pass and the descriptor adjoint on its own rows, and the per-atom partial
forces are all-reduced (sum) -- the second exchange step (``forces_sharded``).

The per-rank arithmetic is delegated to a backend (``DeviceBackend`` runs it
in the CUDA library); the module itself holds only the orchestration, so the
exchange logic can be exercised with CPU ranks.
"""
from __future__ import annotations

from typing import Optional

import numpy as np


def row_range(n_rows: int, rank: int, world: int):
    """Contiguous, balanced slab [r0, r1) of n_rows for `rank` of `world`."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("rank outside 0..world-1")
    base, extra = divmod(int(n_rows), int(world))
    r0 = rank * base + min(rank, extra)
    r1 = r0 + base + (1 if rank < extra else 0)
    return r0, r1


def _allreduce_sum(x: np.ndarray, group) -> np.ndarray:
    """Element-wise FP64 sum over the ranks of `group` (None: single rank).
    Every rank ends with the same bits (one reduction result, broadcast)."""
    if group is None:
        return np.array(x, np.float64, copy=True)
    import torch
    import torch.distributed as dist

    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.as_tensor(np.ascontiguousarray(x, np.float64)).to(dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy().astype(np.float64)


def integrate_sharded(backend, ldos_local, n_points_total: int, volume: float, eg, n_electrons: float,
                      group=None, col_sums_local=None):
    """D(e), e_F, E_b (global) and n(r) (this rank's rows) from row-sharded LDOS.

    col_sums_local: this rank's FP64 column sums if already formed (the network
    kernel emits them with the LDOS), else backend.column_sums(ldos_local);
    backend.integrate(ldos_local, col_sums_global, dV, eg, n_electrons) ->
    dict(fermi, band_energy, density) for the given global column sums.
    """
    if n_points_total <= 0:
        raise ValueError("n_points_total must be positive")
    if col_sums_local is None:
        col_sums_local = backend.column_sums(ldos_local)
    part = np.asarray(col_sums_local, np.float64)
    sums = _allreduce_sum(part, group)
    dV = float(volume) / float(n_points_total)
    r = backend.integrate(ldos_local, sums, dV, eg, n_electrons)
    dens = r["density"]
    local_count = np.array([dV * float(np.sum(np.asarray(dens, np.float64)))])
    count = float(_allreduce_sum(local_count, group)[0])
    return {"dos": dV * sums, "fermi": float(r["fermi"]), "band_energy": float(r["band_energy"]),
            "density": dens, "electron_count": count}


def forces_sharded(backend, snap, rows, volume: float, eg, n_electrons: float, group=None):
    """f_alpha = -dE_b/dR_alpha with this rank holding grid rows [rows[0], rows[1]).

    backend.forward(snap, rows) -> (B_local, ldos_local); backend.column_sums and
    backend.integrate as for ``integrate_sharded``; backend.energy_gradient(D, eg,
    n_electrons) -> dE_b/dD (host [n_E]); backend.ldos_backward(B_local, v) -> beta
    rows; backend.descriptor_forces(snap, beta_local, rows) -> this rank's partial
    forces [n_atoms][3].  Returns the integrate_sharded dict plus "forces" (the
    all-reduced sum, the same bits on every rank)."""
    P = int(np.prod(snap.grid))
    r0, r1 = rows
    B_loc, L_loc = backend.forward(snap, (r0, r1))
    res = integrate_sharded(backend, L_loc, P, volume, eg, n_electrons, group=group)
    g = np.asarray(backend.energy_gradient(res["dos"], eg, n_electrons), np.float64)
    dV = float(volume) / float(P)
    beta = backend.ldos_backward(B_loc, dV * g)
    part = np.asarray(backend.descriptor_forces(snap, beta, (r0, r1)), np.float64)
    res["forces"] = _allreduce_sum(part.reshape(-1), group).reshape(part.shape)
    return res


def _any_grid_of(ldos):
    """An energy grid with the LDOS's N_E (only the column sums are used)."""
    from .workloads import EnergyGrid
    return EnergyGrid(n_E=int(ldos.shape[1]), e0_eV=0.0, de_eV=1.0)


class DeviceBackend:
    """Per-rank arithmetic in the CUDA library (one GPU per rank)."""

    def __init__(self, ctx, precision: Optional[int] = None):
        from . import api
        self.ctx = ctx
        self.precision = api.MIXED if precision is None else precision

    def column_sums(self, ldos_local) -> np.ndarray:
        """FP64 sum over this rank's rows of each energy column, by the
        library's own reduction: with volume = P_local the library's D is
        dV * sums with dV = 1 exactly."""
        r = self.ctx.integrate(ldos_local, float(ldos_local.shape[0]), _any_grid_of(ldos_local), self.precision,
                               n_electrons=0.0, density=False, raise_on_bracket=False)
        return np.asarray(r["dos"], np.float64)

    def integrate(self, ldos_local, col_sums, dV, eg, n_electrons):
        import torch
        dev = ldos_local.device
        ds = torch.as_tensor(np.ascontiguousarray(col_sums, np.float64), device=dev)
        # the library forms D = (volume / P_local) * dos_sum: pass the slab's share of the volume
        vol_local = dV * int(ldos_local.shape[0])
        r = self.ctx.integrate(ldos_local, vol_local, eg, self.precision, dos_sum=ds, n_electrons=n_electrons)
        return {"fermi": r["fermi"], "band_energy": r["band_energy"], "density": r["density"].cpu().numpy()}

    # ---- forces (needs bp and model: set by with_model) ----------------------

    def with_model(self, bp, model):
        self.bp, self.model = bp, model
        return self

    def forward(self, snap, rows):
        """Descriptors of the snapshot (computed whole: the neighbour search is per
        tile) and the LDOS of this rank's rows."""
        r0, r1 = rows
        B = self.ctx.descriptors(snap, self.bp, self.precision)[r0:r1].contiguous()
        L, _ = self.ctx.ldos_forward(self.model, B, self.precision)
        return B, L

    def energy_gradient(self, D, eg, n_electrons):
        return self.ctx.band_energy_gradient(D, eg, n_electrons=n_electrons)["grad"]

    def ldos_backward(self, B_local, v):
        return self.ctx.ldos_backward(self.model, B_local, v, self.precision)

    def descriptor_forces(self, snap, beta_local, rows):
        """The adjoint over the whole grid with beta zero outside this rank's rows
        (zero rows contribute exactly nothing)."""
        import torch
        r0, r1 = rows
        P = int(np.prod(snap.grid))
        beta = torch.zeros((P, beta_local.shape[1]), dtype=beta_local.dtype, device=beta_local.device)
        beta[r0:r1] = beta_local
        return self.ctx.descriptor_forces(snap, self.bp, beta, self.precision)
