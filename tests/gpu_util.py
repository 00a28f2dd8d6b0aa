"""Helpers shared by the GPU parity tests (no arithmetic of the method here)."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


_CTX = None


def ctx():
    """One library context per test process."""
    global _CTX
    if _CTX is None:
        from paper_2411_19617_gb300 import api
        _CTX = api.Context(0)
    return _CTX


def descriptor_error(B, ref, floor=1.0):
    """max over points and components of |dB| / max(|B_ref|, floor * RMS_j),
    RMS_j the root mean square of component j over the points compared.  With
    floor = 1 this is the relative error of every value at least as large as
    its component's RMS and the error relative to that RMS for smaller ones."""
    B = np.asarray(B, np.float64)
    ref = np.asarray(ref, np.float64)
    rms = np.sqrt(np.mean(ref ** 2, axis=0))
    scale = np.maximum(np.abs(ref), floor * rms[None, :])
    scale = np.where(scale > 0, scale, 1.0)
    return float(np.max(np.abs(B - ref) / scale))


def neighbor_sets(counts, atoms, shifts, rows):
    out = []
    for i in rows:
        n = int(counts[i])
        out.append(sorted((int(atoms[i, k]), *map(int, shifts[i, k])) for k in range(n)))
    return out
