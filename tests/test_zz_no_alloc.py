"""mala_integrate_noalloc: the integration step for callers that cannot
allocate device memory (their device memory belongs to another allocator, a
hard memory cap, or no room for the synchronisation an allocation may imply).

It must give the results of mala_integrate, within the tolerances of the other
integration tests, on two calls in a row (the static scratch array keeps the
previous call's contents), and refuse sizes beyond its fixed array.  Runs in
its own context so that it passes alone in a fresh process and after the
other tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2411_19617_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _gaussian_ldos(P, eg, seed):
    rng = np.random.default_rng(seed)
    e = eg.e0_eV + eg.de_eV * np.arange(eg.n_E)
    wd = 2.0 * eg.de_eV
    L = np.zeros((P, eg.n_E))
    for _ in range(3):
        c = rng.uniform(e[0], e[-1], size=(P, 1))
        L += rng.uniform(0.2, 1.0, size=(P, 1)) * np.exp(-((e[None, :] - c) / wd) ** 2)
    return L


def _raw_call(fn, ctx, ldos, P, vol, eg, ne, dos_sum, dens, precision, stream):
    """One call through the C ABI; nothing else touches the device."""
    from paper_2411_19617_gb300 import _lib
    e = _lib.EnergyGrid()
    e.n_E, e.e0_eV, e.de_eV, e.kT_eV, e.n_electrons = eg.n_E, eg.e0_eV, eg.de_eV, eg.kT_eV, ne
    D = np.zeros(eg.n_E)
    eF, Eb, Ne, TS = C.c_double(0), C.c_double(0), C.c_double(0), C.c_double(0)
    rc = fn(ctx.h, C.c_void_p(ldos.data_ptr()), P, vol, C.byref(e),
            C.c_void_p(dos_sum.data_ptr()) if dos_sum is not None else None, C.c_void_p(dens.data_ptr()),
            D.ctypes.data_as(C.c_void_p), C.byref(eF), C.byref(Eb), C.byref(Ne), C.byref(TS), precision, stream)
    return rc, D, eF.value, Eb.value, Ne.value, TS.value


def _call(fn, ctx, ldos, P, vol, eg, ne, dos_sum, dens, precision, stream):
    rc, D, eF, Eb, Ne, TS = _raw_call(fn, ctx, ldos, P, vol, eg, ne, dos_sum, dens, precision, stream)
    return rc, D, eF, Eb, Ne, dens.double().cpu().numpy(), TS


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("with_dos_sum", [False, True])
def test_noalloc_matches_integrate_twice(precision, with_dos_sum):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_19617_gb300 import _lib, api
    lib = _lib.lib()
    ctx = api.Context(0)      # the workspace path (reference results)
    bare = api.Context(0)     # the no-allocation path: a context that has never reserved a workspace
    created = bare.device_bytes  # its tables only
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    mixed = precision == "mixed"
    prec = api.MIXED if mixed else api.FP64_PLAIN
    for trial, (P, nE, de, e0) in enumerate([(20000, 250, 0.1, -8.0), (5832, 11, 1.0, -5.0)]):
        eg = wl.EnergyGrid(n_E=nE, e0_eV=e0, de_eV=de)
        L = _gaussian_ldos(P, eg, seed=trial)
        Lt = torch.from_numpy(L.astype(np.float32)).to(torch.bfloat16).cuda() if mixed else torch.from_numpy(L).cuda()
        dos_sum = Lt.double().sum(dim=0).contiguous() if with_dos_sum else None
        vol = 1000.0
        # a reachable electron count from the workspace path's own DOS
        first = ctx.integrate(Lt, vol, eg, prec, n_electrons=0.0, raise_on_bracket=False, density=False)
        ne = ctx.electron_count(first["dos"], eg, 0.3 * (e0 + e0 + de * (nE - 1)))
        dens_ref = torch.empty(P, dtype=torch.float32 if mixed else torch.float64, device="cuda")
        ref = _call(lib.mala_integrate, ctx, Lt, P, vol, eg, ne, dos_sum, dens_ref, prec, stream)
        assert ref[0] == 0
        rtol = 2e-6 if mixed else 1e-10
        dens = [torch.full((P,), float("nan"), dtype=dens_ref.dtype, device="cuda") for _ in range(3)]
        # a first call (any one-time set-up), then the device memory in use is recorded
        assert _raw_call(lib.mala_integrate_noalloc, bare, Lt, P, vol, eg, ne, dos_sum, dens[0], prec, stream)[0] == 0
        torch.cuda.synchronize()
        before = (bare.device_bytes, torch.cuda.mem_get_info()[0])
        raw = []
        for k in (1, 2):  # two calls in a row share (and reuse) the static array
            dens[k].fill_(float("nan"))
            torch.cuda.synchronize()
            raw.append(_raw_call(lib.mala_integrate_noalloc, bare, Lt, P, vol, eg, ne, dos_sum, dens[k], prec, stream))
        torch.cuda.synchronize()
        # nothing was allocated: neither through the context nor anywhere on the device
        assert (bare.device_bytes, torch.cuda.mem_get_info()[0]) == before
        assert bare.device_bytes == created
        for k in (1, 2):
            rc, D, eF, Eb, Ne, TS = raw[k - 1]
            got = (rc, D, eF, Eb, Ne, dens[k].double().cpu().numpy(), TS)
            assert got[0] == 0, lib.mala_last_error()
            np.testing.assert_allclose(got[1], ref[1], rtol=rtol)
            assert got[2] == pytest.approx(ref[2], abs=1e-9)
            assert got[3] == pytest.approx(ref[3], rel=rtol)
            assert got[4] == pytest.approx(ref[4], rel=rtol)
            np.testing.assert_allclose(got[5], ref[5], rtol=rtol, atol=1e-12)
            assert got[6] == pytest.approx(ref[6], rel=rtol)
    bare.close()
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_array():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_19617_gb300 import _lib, api
    lib = _lib.lib()
    ctx = api.Context(0)
    eg = wl.EnergyGrid(n_E=250, e0_eV=-8.0, de_eV=0.1)
    P = 600000  # ceil(P/128) * 250 doubles of column-sum partials exceed the 8 MiB array
    Lt = torch.ones((P, 250), dtype=torch.bfloat16, device="cuda")
    dens = torch.empty(P, dtype=torch.float32, device="cuda")
    rc = _call(lib.mala_integrate_noalloc, ctx, Lt, P, 1.0, eg, 1.0, None, dens, api.MIXED,
               C.c_void_p(torch.cuda.current_stream().cuda_stream))[0]
    assert rc == _lib.MALA_ERR_UNSUPPORTED
    assert b"static array" in lib.mala_last_error()
    ctx.close()
