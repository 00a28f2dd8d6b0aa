"""The C ABI library builds for sm_103a, loads on a machine without a GPU and
exports every function include/mala.h declares; the ctypes prototypes cover
the same set.  No compute call is made here."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "mala.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(mala_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_hot_path_calls():
    names = _declared_functions()
    for required in ("mala_descriptors", "mala_ldos_forward", "mala_integrate", "mala_submit", "mala_poll",
                     "mala_create", "mala_destroy", "mala_last_error", "mala_predict"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2411_19617_gb300 import _lib, build
    path = build.build()
    assert os.path.exists(path)
    L = _lib.lib(path)
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    assert set(_declared_functions()) == set(_lib.PROTOTYPES), "ctypes prototypes out of sync with mala.h"
    assert L.mala_version() == 1


def test_binding_raises_without_the_library(tmp_path):
    from paper_2411_19617_gb300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(RuntimeError):
            _lib.lib(str(tmp_path / "missing.so"))
    finally:
        _lib._lib = saved


def test_ace_column_count_matches_the_oracle_enumeration():
    # mala_ace_count runs on the host: the library's enumeration against the oracle's
    from oracle import ace
    from paper_2411_19617_gb300 import api
    for ap in (ace.AceParams(rcut=4.676), ace.AceParams(rcut=5.0, n_species=2, nmax1=3, nmax2=3, lmax2=4, nmax3=2,
                                                        lmax3=4), ace.AceParams(rcut=4.0, nmax1=1, nmax2=0, lmax2=0,
                                                                                nmax3=1, lmax3=8)):
        assert api.ace_count(ap) == len(ace.descriptor_index(ap))


def test_force_bindings_check_dtype_and_shape_before_the_library():
    # a beta of the wrong element type or shape never reaches the library
    import numpy as np
    import pytest
    torch = pytest.importorskip("torch")
    from paper_2411_19617_gb300 import api
    from paper_2411_19617_gb300 import workloads as wl
    snap = wl.al_fcc(2, 0.1, 4, seed=1)
    bp = wl.BispectrumParams(twojmax=4, rcut=4.676)
    ctx = api.Context.__new__(api.Context)  # no device needed: the checks come first
    with pytest.raises(ValueError, match="dtype"):
        ctx.descriptor_forces(snap, bp, torch.zeros((64, 14), dtype=torch.float64), api.MIXED)
    with pytest.raises(ValueError, match="shape"):
        ctx.descriptor_forces(snap, bp, torch.zeros((63, 14), dtype=torch.float32), api.MIXED)
    with pytest.raises(ValueError, match="CUDA"):
        ctx.descriptor_forces(snap, bp, torch.zeros((64, 14), dtype=torch.float32), api.MIXED)


def test_tuning_variant_counts_host_only():
    from paper_2411_19617_gb300 import api, build
    build.build()
    n_ui, n_zb = api.tuning_variants()
    assert n_ui == 3 and n_zb == 2
