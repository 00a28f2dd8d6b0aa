"""Seeded synthetic inputs for the grid-descriptor -> LDOS -> observables path.

This module only draws random numbers and lays out atoms, grids and network
parameters.  It holds none of the method's arithmetic (no neighbour search, no
descriptors, no network evaluation, no integration), so the CUDA library and the
FP64 oracle can both be fed from it without sharing any of the computation.

The paper's DFT snapshots and trained networks are not available; every input
here is synthetic, shaped like the paper's aluminium, boron and beryllium
workloads (Sec. "Computational workflow example", Sec. "Scaling"):

* ``al_fcc``: fcc aluminium supercell, a = 4.05 A, Gaussian positional jitter.
* ``boron_clusters``: compact random clusters grown atom by atom with bond
  lengths 1.5-2.0 A and a 1.5 A minimum distance, centred in a cubic box.
* ``be_slab``: hcp beryllium (a = 2.29 A, c = 3.58 A) in the orthohexagonal
  4-atom cell, one stacking fault (ABAB -> CACA) half way up, vacuum along z.
* ``serving_trace``: Poisson arrivals of Al/Be periodic snapshots with atom
  counts log-uniform in [32, 2048] at bulk density.
* ``random_mlp``: fully connected network parameters drawn like
  ``torch.nn.Linear``'s default initialisation, U(-1/sqrt(fan_in), +1/sqrt(fan_in)).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

# Default SNAP-style hyperparameters of the formalism the paper cites (rfac0, rmin0) and kT at room
# temperature.
RFAC0 = 0.99363
RMIN0 = 0.0
KT_ROOM_EV = 0.0259


@dataclasses.dataclass
class Snapshot:
    """One atomic configuration on an orthorhombic cell with a real-space grid."""

    pos: np.ndarray  # [n_atoms, 3] float64, Angstrom, Cartesian
    species: np.ndarray  # [n_atoms] int32
    cell: np.ndarray  # [3, 3] float64, rows are lattice vectors (diagonal here)
    grid: Tuple[int, int, int]
    periodic: Tuple[int, int, int] = (1, 1, 1)
    name: str = ""

    @property
    def n_atoms(self) -> int:
        return int(self.pos.shape[0])

    @property
    def lengths(self) -> np.ndarray:
        return np.diag(self.cell).copy()

    @property
    def n_points(self) -> int:
        return int(self.grid[0]) * int(self.grid[1]) * int(self.grid[2])

    @property
    def volume(self) -> float:
        return float(abs(np.linalg.det(self.cell)))


@dataclasses.dataclass
class BispectrumParams:
    twojmax: int
    rcut: float
    rfac0: float = RFAC0
    rmin0: float = RMIN0
    wself: float = 1.0
    weights: Tuple[float, ...] = (1.0,)


@dataclasses.dataclass
class MLP:
    dims: Tuple[int, ...]  # dims[0] = number of descriptors ... dims[-1] = N_E
    W: List[np.ndarray]  # W[l]: [dims[l+1], dims[l]] float64
    b: List[np.ndarray]  # b[l]: [dims[l+1]] float64
    leaky_slope: float = 0.01
    in_shift: Optional[np.ndarray] = None
    in_scale: Optional[np.ndarray] = None


@dataclasses.dataclass
class EnergyGrid:
    n_E: int
    e0_eV: float
    de_eV: float
    kT_eV: float = KT_ROOM_EV
    n_electrons: float = 0.0


# --------------------------------------------------------------------------
# structures
# --------------------------------------------------------------------------

def _diag_cell(lx: float, ly: float, lz: float) -> np.ndarray:
    return np.diag([float(lx), float(ly), float(lz)])


def al_fcc(reps: int, jitter: float, grid: int, seed: int, a: float = 4.05) -> Snapshot:
    """fcc Al, reps^3 conventional cells (4 atoms each), jitter N(0, jitter)."""
    rng = np.random.default_rng(seed)
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]], dtype=np.float64)
    cells = np.array([[i, j, k] for i in range(reps) for j in range(reps) for k in range(reps)],
                     dtype=np.float64)
    frac = (cells[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    pos = frac * a + rng.normal(0.0, jitter, size=frac.shape)
    L = reps * a
    return Snapshot(pos=pos, species=np.zeros(len(pos), np.int32), cell=_diag_cell(L, L, L),
                    grid=(grid, grid, grid), name=f"Al fcc {reps}x{reps}x{reps}")


def boron_cluster(n_atoms: int, box: float, grid: int, rng: np.random.Generator,
                  dmin: float = 1.5, dmax: float = 2.0) -> Snapshot:
    """Compact random cluster: each new atom sits 1.5-2.0 A from a random existing
    atom and is rejected if it comes closer than 1.5 A to any atom."""
    pts = [np.zeros(3)]
    while len(pts) < n_atoms:
        base = pts[int(rng.integers(len(pts)))]
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        cand = base + v * rng.uniform(dmin, dmax)
        arr = np.asarray(pts)
        if np.min(np.linalg.norm(arr - cand, axis=1)) < dmin:
            continue
        pts.append(cand)
    pos = np.asarray(pts, dtype=np.float64)
    pos += box / 2 - pos.mean(axis=0)
    return Snapshot(pos=pos, species=np.zeros(len(pos), np.int32), cell=_diag_cell(box, box, box),
                    grid=(grid, grid, grid), name=f"B{n_atoms} cluster")


def boron_clusters(n_snap: int, seed: int, box: float = 18.0, grid: int = 90,
                   nmin: int = 8, nmax: int = 96) -> List[Snapshot]:
    rng = np.random.default_rng(seed)
    counts = rng.integers(nmin, nmax + 1, size=n_snap)
    return [boron_cluster(int(n), box, grid, rng) for n in counts]


def be_slab(reps: Tuple[int, int, int] = (16, 16, 16), jitter: float = 0.05, vacuum: float = 10.0,
            spacing: float = 0.2, seed: int = 4, a: float = 2.29, c: float = 3.58) -> Snapshot:
    """hcp Be in the orthohexagonal cell (a, sqrt(3) a, c; 4 atoms), one stacking
    fault: every basal layer in the upper half is shifted by a/sqrt(3) along y,
    so the stacking reads ...ABAB CACA...; `vacuum` Angstrom added along z."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = reps
    b = math.sqrt(3.0) * a
    basis = [(0.0, 0.0, 0.0), (0.5, 0.5, 0.0), (0.5, 1.0 / 6.0, 0.5), (0.0, 2.0 / 3.0, 0.5)]
    out = []
    n_layers = 2 * nz
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                for (fx, fy, fz) in basis:
                    layer = 2 * k + (1 if fz > 0 else 0)
                    shift_y = (1.0 / 3.0) if layer >= n_layers // 2 else 0.0
                    out.append(((i + fx) * a, (j + fy + shift_y) * b, (k + fz) * c))
    pos = np.asarray(out, dtype=np.float64)
    pos += rng.normal(0.0, jitter, size=pos.shape)
    lx, ly, lz = nx * a, ny * b, nz * c + vacuum
    grid = (int(round(lx / spacing)), int(round(ly / spacing)), int(round(lz / spacing)))
    return Snapshot(pos=pos, species=np.zeros(len(pos), np.int32), cell=_diag_cell(lx, ly, lz),
                    grid=grid, name="Be hcp slab with stacking fault")


BULK_DENSITY = {"Al": 0.0602, "Be": 0.1230}  # atoms per cubic Angstrom


def bulk_snapshot(material: str, n_atoms: int, rng: np.random.Generator, spacing: float = 0.2,
                  jitter_frac: float = 0.1) -> Snapshot:
    """Random-jittered simple-cubic site lattice at bulk density: n_atoms sites
    drawn without replacement from an n^3 lattice filling a cube of side
    L = (n_atoms / rho)^(1/3); jitter N(0, jitter_frac * site spacing)."""
    rho = BULK_DENSITY[material]
    L = (n_atoms / rho) ** (1.0 / 3.0)
    n = int(math.ceil(n_atoms ** (1.0 / 3.0)))
    sites = np.array([[i, j, k] for i in range(n) for j in range(n) for k in range(n)], dtype=np.float64)
    pick = rng.choice(len(sites), size=n_atoms, replace=False)
    h = L / n
    pos = (sites[pick] + 0.5) * h + rng.normal(0.0, jitter_frac * h, size=(n_atoms, 3))
    g = max(1, int(round(L / spacing)))
    return Snapshot(pos=pos, species=np.zeros(n_atoms, np.int32), cell=_diag_cell(L, L, L),
                    grid=(g, g, g), name=f"{material}{n_atoms}")


@dataclasses.dataclass
class Request:
    arrival_s: float
    snapshot: Snapshot
    material: str


def serving_trace(n_req: int = 2000, rate_per_s: float = 200.0, seed: int = 5,
                  nmin: int = 32, nmax: int = 2048) -> List[Request]:
    """Poisson arrivals; material Al or Be with p = 1/2; N log-uniform in [nmin, nmax]."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_per_s, size=n_req))
    out = []
    for i in range(n_req):
        mat = "Al" if rng.random() < 0.5 else "Be"
        n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
        out.append(Request(arrival_s=float(t[i]), snapshot=bulk_snapshot(mat, n, rng), material=mat))
    return out


# --------------------------------------------------------------------------
# network parameters
# --------------------------------------------------------------------------

def random_mlp(dims: Sequence[int], seed: int, leaky_slope: float = 0.01, out_bias: float = 0.0) -> MLP:
    """Random network; `out_bias` is added to the output layer's bias so that a
    random network on standardised inputs yields a mostly positive LDOS (a
    physical LDOS is non-negative, which makes the Fermi level unique)."""
    rng = np.random.default_rng(seed)
    W, b = [], []
    for l in range(len(dims) - 1):
        bound = 1.0 / math.sqrt(dims[l])
        W.append(rng.uniform(-bound, bound, size=(dims[l + 1], dims[l])))
        b.append(rng.uniform(-bound, bound, size=(dims[l + 1],)))
    b[-1] = b[-1] + out_bias
    return MLP(dims=tuple(int(d) for d in dims), W=W, b=b, leaky_slope=leaky_slope)


def with_input_scaling(mlp: MLP, shift: np.ndarray, scale: np.ndarray) -> MLP:
    """Copy of `mlp` with the input standardisation (x - shift) * scale."""
    return MLP(dims=mlp.dims, W=mlp.W, b=mlp.b, leaky_slope=mlp.leaky_slope,
               in_shift=np.asarray(shift, np.float64), in_scale=np.asarray(scale, np.float64))


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

def config(idx: int):
    """Return (snapshots, bispectrum params, MLP, energy grid, precision) of a
    workload.  idx 1..5 follow the Al small / Al liquid-like / B clusters /
    Be slab / serving-trace shapes of the paper's workloads."""
    if idx == 1:
        snap = al_fcc(2, 0.1, 18, seed=1)
        bp = BispectrumParams(twojmax=6, rcut=4.676)
        mlp = random_mlp((30, 100, 100, 11), seed=11, out_bias=1.0)
        eg = EnergyGrid(n_E=11, e0_eV=-5.0, de_eV=1.0)
        return [snap], bp, mlp, eg, "fp64"
    if idx == 2:
        snap = al_fcc(4, 0.3, 90, seed=2)
        bp = BispectrumParams(twojmax=10, rcut=4.676)
        mlp = random_mlp((91, 400, 400, 250), seed=12, out_bias=1.0)
        eg = EnergyGrid(n_E=250, e0_eV=-8.0, de_eV=0.1)
        return [snap], bp, mlp, eg, "mixed"
    if idx == 3:
        snaps = boron_clusters(64, seed=3)
        bp = BispectrumParams(twojmax=10, rcut=4.676)
        mlp = random_mlp((91, 400, 400, 11), seed=13, out_bias=1.0)
        eg = EnergyGrid(n_E=11, e0_eV=-5.0, de_eV=1.0)
        return snaps, bp, mlp, eg, "mixed"
    if idx == 4:
        snap = be_slab()
        bp = BispectrumParams(twojmax=10, rcut=4.5)
        mlp = random_mlp((91, 400, 400, 11), seed=14, out_bias=1.0)
        eg = EnergyGrid(n_E=11, e0_eV=-5.0, de_eV=1.0)
        return [snap], bp, mlp, eg, "mixed"
    if idx == 5:
        reqs = serving_trace()
        bp = BispectrumParams(twojmax=10, rcut=4.676)
        mlp = random_mlp((91, 400, 400, 250), seed=15, out_bias=1.0)
        eg = EnergyGrid(n_E=250, e0_eV=-8.0, de_eV=0.1)
        return reqs, bp, mlp, eg, "mixed"
    raise ValueError(f"unknown workload {idx}")


def sample_points(n_points: int, n_sample: int, seed: int) -> np.ndarray:
    """Deterministic sample of flat grid-point indices (sorted, unique)."""
    rng = np.random.default_rng(seed)
    n_sample = min(n_sample, n_points)
    return np.sort(rng.choice(n_points, size=n_sample, replace=False)).astype(np.int64)
