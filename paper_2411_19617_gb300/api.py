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


def tuning_variants():
    """(compute_ui variants, compute_zi/bi variants) compiled into the library."""
    a, b = C.c_int32(0), C.c_int32(0)
    check(lib().mala_tuning_variants(C.byref(a), C.byref(b)), "mala_tuning_variants")
    return int(a.value), int(b.value)


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


def _ace_args(ap) -> "_lib.AceParams":
    """Any object with rcut, n_species, nmax1, nmax2, lmax2, nmax3, lmax3."""
    p = _lib.AceParams()
    p.rcut = float(ap.rcut)
    p.n_species = int(ap.n_species)
    p.nmax1, p.nmax2, p.lmax2 = int(ap.nmax1), int(ap.nmax2), int(ap.lmax2)
    p.nmax3, p.lmax3 = int(ap.nmax3), int(ap.lmax3)
    return p


def ace_count(ap) -> int:
    """Number of ACE descriptor columns for the parameters."""
    n = C.c_int32(0)
    p = _ace_args(ap)
    check(lib().mala_ace_count(C.byref(p), C.byref(n)), "mala_ace_count")
    return int(n.value)


def _check_tensor(t, shape, precision: int, name: str):
    """A device tensor of the given shape and the precision's element type (float32
    for MIXED, float64 for FP64_PLAIN), contiguous: the library reads raw rows."""
    torch = _torch()
    want = torch.float32 if precision == MIXED else torch.float64
    if t.dtype != want:
        raise ValueError(f"{name}: dtype {t.dtype}, expected {want} for this precision")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name}: shape {tuple(t.shape)}, expected {tuple(shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor")


class _EnergyGridArgs:
    def __init__(self, eg, n_electrons: Optional[float] = None):
        e = _lib.EnergyGrid()
        e.n_E = int(eg.n_E)
        e.e0_eV = float(eg.e0_eV)
        e.de_eV = float(eg.de_eV)
        e.kT_eV = float(eg.kT_eV)
        e.n_electrons = float(eg.n_electrons if n_electrons is None else n_electrons)
        self.c = e


class _DevView:
    """Zero-copy view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(int(x) for x in shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def device_view(ptr: int, shape, dtype):
    """torch tensor aliasing device memory the library owns (no copy)."""
    torch = _torch()
    if dtype == torch.bfloat16:
        t = torch.as_tensor(_DevView(ptr, shape, "<i2"), device="cuda")
        return t.view(torch.bfloat16)
    typestr = {torch.float32: "<f4", torch.float64: "<f8", torch.int32: "<i4"}[dtype]
    return torch.as_tensor(_DevView(ptr, shape, typestr), device="cuda")


class Model:
    """A network uploaded to the library (BF16 + tensor maps, and FP64)."""

    def __init__(self, ctx: "Context", mlp):
        self.ctx = ctx  # keeps the context alive at least as long as the network
        self.dims = tuple(int(d) for d in mlp.dims)
        nl = len(self.dims) - 1
        self._dims = np.ascontiguousarray(self.dims, dtype=np.int32)
        self._W = [np.ascontiguousarray(w, dtype=np.float64) for w in mlp.W]
        self._b = [np.ascontiguousarray(b, dtype=np.float64) for b in mlp.b]
        self._shift = None if mlp.in_shift is None else np.ascontiguousarray(mlp.in_shift, dtype=np.float64)
        self._scale = None if mlp.in_scale is None else np.ascontiguousarray(mlp.in_scale, dtype=np.float64)
        Wp = (C.POINTER(C.c_double) * nl)(*[w.ctypes.data_as(C.POINTER(C.c_double)) for w in self._W])
        bp = (C.POINTER(C.c_double) * nl)(*[b.ctypes.data_as(C.POINTER(C.c_double)) for b in self._b])
        d = _lib.MLPDesc()
        d.n_layers = nl
        d.dims = self._dims.ctypes.data_as(C.POINTER(C.c_int32))
        d.W = C.cast(Wp, C.POINTER(C.POINTER(C.c_double)))
        d.b = C.cast(bp, C.POINTER(C.POINTER(C.c_double)))
        d.leaky_slope = float(mlp.leaky_slope)
        d.activate_output = 0
        d.in_shift = None if self._shift is None else self._shift.ctypes.data_as(C.POINTER(C.c_double))
        d.in_scale = None if self._scale is None else self._scale.ctypes.data_as(C.POINTER(C.c_double))
        h = C.c_void_p()
        check(lib().mala_model_create(ctx.h, C.byref(d), C.byref(h)), "mala_model_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().mala_model_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _result_dict(r: "_lib.Result", precision: int):
    torch = _torch()
    out = {"status": int(r.status), "fermi": float(r.fermi_eV), "band_energy": float(r.band_energy_eV),
           "electron_count": float(r.electron_count), "entropy_term": float(r.entropy_term_eV),
           "n_points": int(r.n_points), "n_B": int(r.n_B),
           "n_E": int(r.n_E), "latency_s": float(r.submit_to_done_s),
           "gpu_interval_ms": (float(r.gpu_start_ms), float(r.gpu_end_ms))}
    out["dos"] = np.ctypeslib.as_array(r.dos, shape=(r.n_E,)).copy() if r.dos else None
    fdt = torch.float32 if precision == MIXED else torch.float64
    ldt = torch.bfloat16 if precision == MIXED else torch.float64
    if r.B_dev:
        out["B"] = device_view(r.B_dev, (r.n_points, r.n_B), fdt)
        out["ldos"] = device_view(r.ldos_dev, (r.n_points, r.n_E), ldt)
        out["density"] = device_view(r.density_dev, (r.n_points,), fdt)
    return out


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

    def set_tuning(self, mode: int, ui_variant: int = 0, zb_variant: int = 0):
        """0: default kernel shapes, 1: autotune per key (default), 2: force the given variants."""
        check(lib().mala_set_tuning(self.h, int(mode), int(ui_variant), int(zb_variant)), "mala_set_tuning")

    def tuning_report(self) -> str:
        buf = C.create_string_buffer(8192)
        check(lib().mala_tuning_report(self.h, buf, len(buf)), "mala_tuning_report")
        return buf.value.decode()

    def measure_peaks(self):
        """(FP32 scalar, FP32 packed FP32x2, FP64) FMA throughput of the device in TFLOP/s, measured."""
        a, b, d = C.c_double(0.0), C.c_double(0.0), C.c_double(0.0)
        check(lib().mala_measure_peaks(self.h, C.byref(a), C.byref(b), C.byref(d)), "mala_measure_peaks")
        return float(a.value), float(b.value), float(d.value)

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

    def gaussian_descriptors(self, snap, rcut: float, sigma: float, precision: int = MIXED, out=None, stream=None):
        """G[P] = sum over neighbours within rcut of exp(-d^2 / (2 sigma^2)) on the GPU."""
        torch = _torch()
        P = int(np.prod(snap.grid))
        dt = torch.float32 if precision == MIXED else torch.float64
        if out is None:
            out = torch.empty(P, dtype=dt, device=torch.device("cuda", self.device))
        a = _SnapshotArgs(snap)
        check(lib().mala_gaussian_descriptors(self.h, C.byref(a.c), float(rcut), float(sigma),
                                              C.c_void_p(out.data_ptr()), int(precision), _stream_ptr(stream)),
              "mala_gaussian_descriptors")
        return out

    def ace_descriptors(self, snap, ap, precision: int = MIXED, out=None, stream=None):
        """Grid-centred ACE descriptors D[P][ace_count(ap)] on the GPU (float32 for MIXED, float64 for FP64_PLAIN)."""
        torch = _torch()
        P = int(np.prod(snap.grid))
        dt = torch.float32 if precision == MIXED else torch.float64
        if out is None:
            out = torch.empty((P, ace_count(ap)), dtype=dt, device=torch.device("cuda", self.device))
        _check_tensor(out, (P, ace_count(ap)), precision, "out")
        a, p = _SnapshotArgs(snap), _ace_args(ap)
        check(lib().mala_ace_descriptors(self.h, C.byref(a.c), C.byref(p), C.c_void_p(out.data_ptr()),
                                         int(precision), _stream_ptr(stream)), "mala_ace_descriptors")
        return out

    def descriptors_batch(self, snaps, bp, precision: int = MIXED, out=None, stream=None):
        """B of several snapshots in one pass: rows of snapshot i follow those of
        snapshot i-1 ([sum P_i][n_B] on the GPU)."""
        torch = _torch()
        args = [_SnapshotArgs(s) for s in snaps]
        arr = (_lib.Snapshot * len(args))(*[a.c for a in args])
        P = sum(int(np.prod(s.grid)) for s in snaps)
        nB = n_descriptors(bp.twojmax)
        dt = torch.float32 if precision == MIXED else torch.float64
        if out is None:
            out = torch.empty((P, nB), dtype=dt, device=torch.device("cuda", self.device))
        b = _BParamsArgs(bp)
        check(lib().mala_descriptors_batch(self.h, len(args), arr, C.byref(b.c), C.c_void_p(out.data_ptr()),
                                           int(precision), _stream_ptr(stream)), "mala_descriptors_batch")
        return out

    def predict_batch(self, snaps, bp, model: "Model", egs, precision: int = MIXED, n_electrons=None,
                      density_host=None, stream=None, raise_on_bracket: bool = True):
        """The whole path for several snapshots at once; egs is one energy grid
        or one per snapshot, n_electrons None or one per snapshot.  Returns one
        result dict per snapshot (device tensors alias the context's workspace)."""
        n = len(snaps)
        if not isinstance(egs, (list, tuple)):
            egs = [egs] * n
        nes = [None] * n if n_electrons is None else list(n_electrons)
        args = [_SnapshotArgs(s) for s in snaps]
        arr = (_lib.Snapshot * n)(*[a.c for a in args])
        eargs = [_EnergyGridArgs(eg, ne) for eg, ne in zip(egs, nes)]
        earr = (_lib.EnergyGrid * n)(*[e.c for e in eargs])
        res = (_lib.Result * n)()
        b = _BParamsArgs(bp)
        rc = lib().mala_predict_batch(self.h, n, arr, C.byref(b.c), model.h, earr, int(precision),
                                      density_host.ctypes.data_as(C.c_void_p) if density_host is not None else None,
                                      res, _stream_ptr(stream))
        if rc != _lib.MALA_ERR_FERMI_BRACKET or raise_on_bracket:
            check(rc, "mala_predict_batch")
        out = [_result_dict(res[i], precision) for i in range(n)]
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

    # ---- network and integrals --------------------------------------------

    def ldos_forward(self, model: Model, B, precision: int = MIXED, dos_sum: bool = True, stream=None):
        """(LDOS[P][N_E] bf16/f64, column sums [N_E] f64 or None) on the GPU."""
        torch = _torch()
        P = int(B.shape[0])
        nE = model.dims[-1]
        dev = torch.device("cuda", self.device)
        ldos = torch.empty((P, nE), dtype=torch.bfloat16 if precision == MIXED else torch.float64, device=dev)
        ds = torch.zeros(nE, dtype=torch.float64, device=dev) if dos_sum else None
        check(lib().mala_ldos_forward(self.h, model.h, C.c_void_p(B.data_ptr()), P, C.c_void_p(ldos.data_ptr()),
                                      C.c_void_p(ds.data_ptr()) if ds is not None else None, int(precision),
                                      _stream_ptr(stream)), "mala_ldos_forward")
        return ldos, ds

    def integrate(self, ldos, volume: float, eg, precision: int = MIXED, dos_sum=None, n_electrons=None,
                  density: bool = True, stream=None, raise_on_bracket: bool = True):
        """D(e), Fermi level, band energy, entropy term -tau S_s, electron count and n(r) of an LDOS."""
        torch = _torch()
        P = int(ldos.shape[0])
        dev = torch.device("cuda", self.device)
        dens = None
        if density:
            dens = torch.empty(P, dtype=torch.float32 if precision == MIXED else torch.float64, device=dev)
        e = _EnergyGridArgs(eg, n_electrons)
        D = np.zeros(int(eg.n_E))
        eF, Eb, Ne, TS = C.c_double(0), C.c_double(0), C.c_double(0), C.c_double(0)
        rc = lib().mala_integrate(self.h, C.c_void_p(ldos.data_ptr()), P, float(volume), C.byref(e.c),
                                  C.c_void_p(dos_sum.data_ptr()) if dos_sum is not None else None,
                                  C.c_void_p(dens.data_ptr()) if dens is not None else None,
                                  D.ctypes.data_as(C.c_void_p), C.byref(eF), C.byref(Eb), C.byref(Ne), C.byref(TS),
                                  int(precision), _stream_ptr(stream))
        if rc != _lib.MALA_ERR_FERMI_BRACKET or raise_on_bracket:
            check(rc, "mala_integrate")
        return {"status": rc, "dos": D, "fermi": eF.value, "band_energy": Eb.value, "electron_count": Ne.value,
                "entropy_term": TS.value, "density": dens}

    def electron_count(self, D, eg, mu: float) -> float:
        """N(mu) = sum_xi w0_xi(mu) D_xi on the GPU."""
        D = np.ascontiguousarray(D, dtype=np.float64)
        e = _EnergyGridArgs(eg)
        out = C.c_double(0.0)
        check(lib().mala_electron_count(self.h, D.ctypes.data_as(C.POINTER(C.c_double)), C.byref(e.c), float(mu),
                                        C.byref(out)), "mala_electron_count")
        return float(out.value)

    # ---- the whole path ------------------------------------------------------

    def predict(self, snap, bp, model: Model, eg, precision: int = MIXED, n_electrons=None, density_host=None,
                stream=None, raise_on_bracket: bool = True):
        """Descriptors -> LDOS -> integrals.  Device outputs alias the context's
        workspace (valid until the next call); density_host (numpy) receives n(r)."""
        a, b, e = _SnapshotArgs(snap), _BParamsArgs(bp), _EnergyGridArgs(eg, n_electrons)
        r = _lib.Result()
        rc = lib().mala_predict(self.h, C.byref(a.c), C.byref(b.c), model.h, C.byref(e.c), int(precision),
                                density_host.ctypes.data_as(C.c_void_p) if density_host is not None else None,
                                C.byref(r), _stream_ptr(stream))
        if rc != _lib.MALA_ERR_FERMI_BRACKET or raise_on_bracket:
            check(rc, "mala_predict")
        out = _result_dict(r, precision)
        out["status"] = rc
        return out

    # ---- band-energy forces (Eqs. forces / forcesmala) ----------------------------

    def band_energy_gradient(self, D, eg, n_electrons=None, stream=None):
        """dE_b/dD at fixed electron number: {"grad", "fermi", "mu_tilde"}."""
        D = np.ascontiguousarray(D, dtype=np.float64)
        e = _EnergyGridArgs(eg, n_electrons)
        g = np.zeros(len(D))
        eF, mt = C.c_double(0.0), C.c_double(0.0)
        dp = C.POINTER(C.c_double)
        check(lib().mala_band_energy_gradient(self.h, D.ctypes.data_as(dp), C.byref(e.c), g.ctypes.data_as(dp),
                                              C.byref(eF), C.byref(mt), _stream_ptr(stream)),
              "mala_band_energy_gradient")
        return {"grad": g, "fermi": eF.value, "mu_tilde": mt.value}

    def ldos_backward(self, model: Model, B, v, precision: int = MIXED, out=None, stream=None):
        """beta[p][j] = sum_e v[e] dLDOS[p][e]/dB[p][j] on the GPU (B: device [P][n_B])."""
        torch = _torch()
        v = np.ascontiguousarray(v, dtype=np.float64)
        _check_tensor(B, (B.shape[0], model.dims[0]), precision, "B")
        if len(v) != model.dims[-1]:
            raise ValueError(f"v has {len(v)} entries, the network outputs {model.dims[-1]}")
        if out is None:
            out = torch.empty_like(B)
        _check_tensor(out, B.shape, precision, "out")
        check(lib().mala_ldos_backward(self.h, model.h, C.c_void_p(B.data_ptr()), int(B.shape[0]),
                                       v.ctypes.data_as(C.POINTER(C.c_double)), C.c_void_p(out.data_ptr()),
                                       int(precision), _stream_ptr(stream)), "mala_ldos_backward")
        return out

    def descriptor_forces(self, snap, bp, beta, precision: int = MIXED, stream=None):
        """F[a][k] = -sum_r sum_j beta[r][j] dB(r, j)/dR_{a,k} (beta: device [P][n_B]); numpy [n_atoms][3]."""
        _check_tensor(beta, (int(np.prod(snap.grid)), n_descriptors(bp.twojmax)), precision, "beta")
        a, b = _SnapshotArgs(snap), _BParamsArgs(bp)
        F = np.zeros((len(snap.pos), 3))
        check(lib().mala_descriptor_forces(self.h, C.byref(a.c), C.byref(b.c), C.c_void_p(beta.data_ptr()),
                                           F.ctypes.data_as(C.POINTER(C.c_double)), int(precision),
                                           _stream_ptr(stream)), "mala_descriptor_forces")
        return F

    def band_forces(self, snap, bp, model: Model, eg, precision: int = MIXED, n_electrons=None, stream=None):
        """The forward path of predict() and f = -dE_b/dR: the result dict plus "forces" [n_atoms][3]."""
        a, b, e = _SnapshotArgs(snap), _BParamsArgs(bp), _EnergyGridArgs(eg, n_electrons)
        r = _lib.Result()
        F = np.zeros((len(snap.pos), 3))
        check(lib().mala_band_forces(self.h, C.byref(a.c), C.byref(b.c), model.h, C.byref(e.c), int(precision),
                                     F.ctypes.data_as(C.POINTER(C.c_double)), C.byref(r), _stream_ptr(stream)),
              "mala_band_forces")
        out = _result_dict(r, precision)
        out["forces"] = F
        return out

    # ---- serving ----------------------------------------------------------------

    def submit(self, snap, bp, model: Model, eg, precision: int = MIXED, n_electrons=None) -> int:
        a, b, e = _SnapshotArgs(snap), _BParamsArgs(bp), _EnergyGridArgs(eg, n_electrons)
        t = C.c_uint64(0)
        check(lib().mala_submit(self.h, C.byref(a.c), C.byref(b.c), model.h, C.byref(e.c), int(precision),
                                C.byref(t)), "mala_submit")
        return int(t.value)

    def poll(self, ticket: int, precision: int = MIXED):
        """None while pending, else the result dict (raises on a failed request)."""
        r = _lib.Result()
        rc = lib().mala_poll(self.h, C.c_uint64(ticket), C.byref(r))
        if rc == _lib.MALA_PENDING:
            return None
        check(rc, "mala_poll")
        return _result_dict(r, precision)

    def poll_status(self, ticket: int) -> int:
        """The request's status without raising: 1 (MALA_PENDING) while queued or running,
        0 when done, a negative error code when it failed."""
        return int(lib().mala_poll(self.h, C.c_uint64(ticket), None))

    def wait(self, ticket: int, timeout_s: float = 60.0, precision: int = MIXED):
        r = _lib.Result()
        check(lib().mala_wait(self.h, C.c_uint64(ticket), float(timeout_s), C.byref(r)), "mala_wait")
        return _result_dict(r, precision)

    def release(self, ticket: int):
        check(lib().mala_release(self.h, C.c_uint64(ticket)), "mala_release")
