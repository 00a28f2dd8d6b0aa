"""Thin Python binding of the C ABI (include/mala.h).

Argument marshalling only: PyTorch supplies device memory and streams, every
step of the path runs in libmala.so's CUDA kernels.  There is no CPU fallback:
if the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes as C
from typing import List, Optional, Sequence

import numpy as np

from . import _lib
from ._lib import check, lib

MIXED = _lib.MALA_MIXED
FP64_PLAIN = _lib.MALA_FP64_PLAIN


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def n_descriptors(twojmax: int) -> int:
    return (twojmax + 2) * (twojmax + 3) * (twojmax + 4) // 24


class _SnapshotArgs:
    """Keeps the numpy buffers behind a mala_snapshot alive."""

    def __init__(self, snap):
        self.pos = np.ascontiguousarray(snap.pos, dtype=np.float64)
        self.species = np.ascontiguousarray(snap.species, dtype=np.int32)
        s = _lib.Snapshot()
        s.n_atoms = int(self.pos.shape[0])
        s.pos = self.pos.ctypes.data_as(C.POINTER(C.c_double))
        s.species = self.species.ctypes.data_as(C.POINTER(C.c_int32))
        for i in range(3):
            for j in range(3):
                s.cell[i][j] = float(snap.cell[i][j])
            s.grid[i] = int(snap.grid[i])
            s.periodic[i] = int(snap.periodic[i])
        self.c = s


class _BParamsArgs:
    def __init__(self, bp):
        self.w = np.ascontiguousarray(bp.weights, dtype=np.float64)
        p = _lib.BispectrumParams()
        p.twojmax = int(bp.twojmax)
        p.rcut = float(bp.rcut)
        p.rfac0 = float(bp.rfac0)
        p.rmin0 = float(bp.rmin0)
        p.wself = float(bp.wself)
        p.n_species = int(len(self.w))
        p.weights = self.w.ctypes.data_as(C.POINTER(C.c_double))
        self.c = p


class _EnergyGridArgs:
    def __init__(self, eg, n_electrons: Optional[float] = None):
        e = _lib.EnergyGrid()
        e.n_E = int(eg.n_E)
        e.e0_eV = float(eg.e0_eV)
        e.de_eV = float(eg.de_eV)
        e.kT_eV = float(eg.kT_eV)
        e.n_electrons = float(eg.n_electrons if n_electrons is None else n_electrons)
        self.c = e


class Context:
    """A library context on one CUDA device (owns streams, tables, workspaces)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        h = C.c_void_p()
        check(lib().mala_create(C.byref(h), int(device), int(hbm_budget_bytes)), "mala_create")
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().mala_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def device_bytes(self) -> int:
        return int(lib().mala_device_bytes(self.h))

    def profile(self, enable: bool = True):
        """Start (clearing totals) or stop per-kernel CUDA-event timing."""
        check(lib().mala_profile(self.h, 1 if enable else 0), "mala_profile")

    def profile_get(self, kernel: str):
        """(total ms, launches) of a kernel since profiling was enabled."""
        ms, n = C.c_double(0.0), C.c_int64(0)
        check(lib().mala_profile_get(self.h, kernel.encode(), C.byref(ms), C.byref(n)), "mala_profile_get")
        return float(ms.value), int(n.value)

    # ---- one step at a time --------------------------------------------

    def neighbor_lists(self, snap, rcut: float, cap: int = 128, stream=None):
        """(counts[P], atoms[P][cap], shifts[P][cap][3], max_count) on the GPU."""
        torch = _torch()
        P = int(np.prod(snap.grid))
        dev = torch.device("cuda", self.device)
        counts = torch.zeros(P, dtype=torch.int32, device=dev)
        atoms = torch.full((P, cap), -1, dtype=torch.int32, device=dev)
        shifts = torch.zeros((P, cap, 3), dtype=torch.int32, device=dev)
        a = _SnapshotArgs(snap)
        mx = C.c_int32(0)
        check(lib().mala_neighbor_lists(self.h, C.byref(a.c), float(rcut), int(cap), C.c_void_p(counts.data_ptr()),
                                        C.c_void_p(atoms.data_ptr()), C.c_void_p(shifts.data_ptr()), C.byref(mx),
                                        _stream_ptr(stream)), "mala_neighbor_lists")
        return counts, atoms, shifts, int(mx.value)

    def descriptors(self, snap, bp, precision: int = MIXED, out=None, stream=None):
        """B[P][n_B] (float32 for MIXED, float64 for FP64_PLAIN) on the GPU."""
        torch = _torch()
        P = int(np.prod(snap.grid))
        nB = n_descriptors(bp.twojmax)
        dt = torch.float32 if precision == MIXED else torch.float64
        if out is None:
            out = torch.empty((P, nB), dtype=dt, device=torch.device("cuda", self.device))
        a, b = _SnapshotArgs(snap), _BParamsArgs(bp)
        check(lib().mala_descriptors(self.h, C.byref(a.c), C.byref(b.c), C.c_void_p(out.data_ptr()), int(precision),
                                     _stream_ptr(stream)), "mala_descriptors")
        return out

    def expansion_coefficients(self, snap, bp, precision: int = MIXED, stream=None):
        """u[P][sum_J (J+1)^2] complex (as [..., 2] real) on the GPU."""
        torch = _torch()
        P = int(np.prod(snap.grid))
        nf = sum((J + 1) ** 2 for J in range(bp.twojmax + 1))
        dt = torch.float32 if precision == MIXED else torch.float64
        out = torch.empty((P, nf, 2), dtype=dt, device=torch.device("cuda", self.device))
        a, b = _SnapshotArgs(snap), _BParamsArgs(bp)
        check(lib().mala_expansion_coefficients(self.h, C.byref(a.c), C.byref(b.c), C.c_void_p(out.data_ptr()),
                                                int(precision), _stream_ptr(stream)), "mala_expansion_coefficients")
        return out
