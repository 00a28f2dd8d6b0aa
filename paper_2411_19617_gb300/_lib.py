"""ctypes view of include/mala.h: structure layouts and function prototypes.

Argument marshalling only; every step of the computation runs in libmala.so.
Importing this module does not load the library; ``lib()`` does, and raises
if the CUDA library has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_build", "libmala.so")

MALA_OK = 0
MALA_PENDING = 1
MALA_ERR_INVALID_ARG = -1
MALA_ERR_OOM = -2
MALA_ERR_UNSUPPORTED = -3
MALA_ERR_FERMI_BRACKET = -4
MALA_ERR_TIMEOUT = -5
MALA_ERR_CUDA = -6
MALA_ERR_NOT_FOUND = -7

MALA_FP64_PLAIN = 0
MALA_MIXED = 1


class Snapshot(C.Structure):
    _fields_ = [("n_atoms", C.c_int32), ("pos", C.POINTER(C.c_double)), ("species", C.POINTER(C.c_int32)),
                ("cell", (C.c_double * 3) * 3), ("grid", C.c_int32 * 3), ("periodic", C.c_int32 * 3)]


class BispectrumParams(C.Structure):
    _fields_ = [("twojmax", C.c_int32), ("rcut", C.c_double), ("rfac0", C.c_double), ("rmin0", C.c_double),
                ("wself", C.c_double), ("n_species", C.c_int32), ("weights", C.POINTER(C.c_double))]


class MLPDesc(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("dims", C.POINTER(C.c_int32)),
                ("W", C.POINTER(C.POINTER(C.c_double))), ("b", C.POINTER(C.POINTER(C.c_double))),
                ("leaky_slope", C.c_double), ("activate_output", C.c_int32),
                ("in_shift", C.POINTER(C.c_double)), ("in_scale", C.POINTER(C.c_double))]


class EnergyGrid(C.Structure):
    _fields_ = [("n_E", C.c_int32), ("e0_eV", C.c_double), ("de_eV", C.c_double), ("kT_eV", C.c_double),
                ("n_electrons", C.c_double)]


class AceParams(C.Structure):
    _fields_ = [("rcut", C.c_double), ("n_species", C.c_int32), ("nmax1", C.c_int32), ("nmax2", C.c_int32),
                ("lmax2", C.c_int32), ("nmax3", C.c_int32), ("lmax3", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_B", C.c_int32), ("n_E", C.c_int32), ("n_points", C.c_int64),
                ("fermi_eV", C.c_double), ("band_energy_eV", C.c_double), ("electron_count", C.c_double),
                ("dos", C.POINTER(C.c_double)), ("B_dev", C.c_void_p), ("ldos_dev", C.c_void_p),
                ("density_dev", C.c_void_p), ("submit_to_done_s", C.c_double), ("entropy_term_eV", C.c_double),
                ("gpu_start_ms", C.c_double), ("gpu_end_ms", C.c_double)]


# name -> (restype, argtypes); every function declared in include/mala.h
PROTOTYPES = {
    "mala_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_size_t]),
    "mala_destroy": (None, [C.c_void_p]),
    "mala_last_error": (C.c_char_p, []),
    "mala_version": (C.c_int, []),
    "mala_device_bytes": (C.c_size_t, [C.c_void_p]),
    "mala_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "mala_profile_get": (C.c_int, [C.c_void_p, C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "mala_measure_peaks": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                     C.POINTER(C.c_double)]),
    "mala_set_tuning": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int]),
    "mala_tuning_variants": (C.c_int, [C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
    "mala_tuning_report": (C.c_int, [C.c_void_p, C.c_char_p, C.c_size_t]),
    "mala_model_create": (C.c_int, [C.c_void_p, C.POINTER(MLPDesc), C.POINTER(C.c_void_p)]),
    "mala_model_destroy": (None, [C.c_void_p]),
    "mala_neighbor_lists": (C.c_int, [C.c_void_p, C.POINTER(Snapshot), C.c_double, C.c_int32, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.POINTER(C.c_int32), C.c_void_p]),
    "mala_descriptors": (C.c_int, [C.c_void_p, C.POINTER(Snapshot), C.POINTER(BispectrumParams), C.c_void_p,
                                   C.c_int, C.c_void_p]),
    "mala_expansion_coefficients": (C.c_int, [C.c_void_p, C.POINTER(Snapshot), C.POINTER(BispectrumParams),
                                              C.c_void_p, C.c_int, C.c_void_p]),
    "mala_ldos_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                    C.c_int, C.c_void_p]),
    "mala_integrate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.POINTER(EnergyGrid),
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int,
                                 C.c_void_p]),
    "mala_integrate_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.POINTER(EnergyGrid),
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                                         C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int,
                                         C.c_void_p]),
    "mala_electron_count": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(EnergyGrid), C.c_double,
                                      C.POINTER(C.c_double)]),
    "mala_predict": (C.c_int, [C.c_void_p, C.POINTER(Snapshot), C.POINTER(BispectrumParams), C.c_void_p,
                               C.POINTER(EnergyGrid), C.c_int, C.c_void_p, C.POINTER(Result), C.c_void_p]),
    "mala_predict_batch": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Snapshot), C.POINTER(BispectrumParams),
                                     C.c_void_p, C.POINTER(EnergyGrid), C.c_int, C.c_void_p, C.POINTER(Result),
                                     C.c_void_p]),
    "mala_gaussian_descriptors": (C.c_int, [C.c_void_p, C.POINTER(Snapshot), C.c_double, C.c_double, C.c_void_p,
                                            C.c_int, C.c_void_p]),
    "mala_descriptors_batch": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(Snapshot), C.POINTER(BispectrumParams),
                                         C.c_void_p, C.c_int, C.c_void_p]),
    "mala_band_energy_gradient": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(EnergyGrid),
                                            C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double),
                                            C.c_void_p]),
    "mala_ldos_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_double),
                                     C.c_void_p, C.c_int, C.c_void_p]),
    "mala_descriptor_forces": (C.c_int, [C.c_void_p, C.POINTER(Snapshot), C.POINTER(BispectrumParams), C.c_void_p,
                                         C.POINTER(C.c_double), C.c_int, C.c_void_p]),
    "mala_band_forces": (C.c_int, [C.c_void_p, C.POINTER(Snapshot), C.POINTER(BispectrumParams), C.c_void_p,
                                   C.POINTER(EnergyGrid), C.c_int, C.POINTER(C.c_double), C.POINTER(Result),
                                   C.c_void_p]),
    "mala_ace_count": (C.c_int, [C.POINTER(AceParams), C.POINTER(C.c_int32)]),
    "mala_ace_descriptors": (C.c_int, [C.c_void_p, C.POINTER(Snapshot), C.POINTER(AceParams), C.c_void_p, C.c_int,
                                       C.c_void_p]),
    "mala_submit": (C.c_int, [C.c_void_p, C.POINTER(Snapshot), C.POINTER(BispectrumParams), C.c_void_p,
                              C.POINTER(EnergyGrid), C.c_int, C.POINTER(C.c_uint64)]),
    "mala_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(Result)]),
    "mala_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_double, C.POINTER(Result)]),
    "mala_release": (C.c_int, [C.c_void_p, C.c_uint64]),
}

_lib = None


def lib(path: str = LIB_PATH):
    """Load libmala.so (once) and attach the prototypes."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = C.CDLL(path)
        for name, (res, args) in PROTOTYPES.items():
            f = getattr(L, name, None)
            if f is None:
                continue
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class MalaError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().mala_last_error()
        super().__init__(f"{where} failed with status {code}: {msg.decode() if msg else ''}")
        self.code = code


def check(code: int, where: str) -> int:
    if code < 0:
        raise MalaError(code, where)
    return code
