"""GPU parity of the network step (Eq. ffnn) through the C ABI.

MIXED: BF16 tcgen05 chain with FP32 accumulation against the FP64 oracle,
per point ||dL||_2 / ||L||_2 <= 2e-2 (max over points).  The fused DOS column
sums equal the column sums of the LDOS values the kernel stored.  FP64 path
against the oracle at 1e-12.
"""
import numpy as np
import pytest

import oracle
from paper_2411_19617_gb300 import workloads as wl
from tests.gpu_util import ctx, need_gpu

pytestmark = pytest.mark.gpu

LDOS_TOL = 2e-2


def _ldos_error(L, ref):
    L = np.asarray(L, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.linalg.norm(L - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-30)))


_B_CACHE = {}


def _descriptor_sample(twojmax):
    """Oracle descriptors of a small Al cell (the network's realistic inputs)."""
    if twojmax not in _B_CACHE:
        snap = wl.al_fcc(2, 0.25, 8, seed=21)
        bp = wl.BispectrumParams(twojmax=twojmax, rcut=4.676)
        _B_CACHE[twojmax] = oracle.bispectrum_grid(snap, bp, nthreads=8)
    return _B_CACHE[twojmax]


def _model(dims, seed, B):
    mlp = wl.random_mlp(dims, seed=seed, out_bias=1.0)
    return wl.with_input_scaling(mlp, B.mean(axis=0), 1.0 / (B.std(axis=0) + 1e-12))


@pytest.mark.parametrize("dims,twojmax", [((30, 100, 100, 11), 6), ((91, 400, 400, 250), 10),
                                          ((91, 400, 400, 11), 10), ((91, 64, 16), 10), ((30, 11), 6)])
@pytest.mark.parametrize("P", [512, 511, 129, 128, 1])
def test_mixed_network_matches_oracle(dims, twojmax, P):
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    B = _descriptor_sample(twojmax)[:P]
    mlp = _model(dims, 7, _descriptor_sample(twojmax))
    model = api.Model(ctx(), mlp)
    Bt = torch.from_numpy(B.astype(np.float32)).cuda()
    ldos, dsum = ctx().ldos_forward(model, Bt, api.MIXED)
    L = ldos.float().cpu().numpy()
    ref = oracle.mlp_forward(B.astype(np.float32).astype(np.float64), mlp.W, mlp.b, mlp.leaky_slope,
                             mlp.in_shift, mlp.in_scale)
    assert L.shape == ref.shape
    assert _ldos_error(L, ref) < LDOS_TOL
    # fused column sums = sums of the stored BF16 values
    np.testing.assert_allclose(dsum.cpu().numpy(), L.astype(np.float64).sum(axis=0), rtol=2e-6, atol=1e-6)


def test_mixed_network_full_tile_count_and_empty():
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    B = _descriptor_sample(10)
    mlp = _model((91, 400, 400, 250), 3, B)
    model = api.Model(ctx(), mlp)
    # many tiles: repeat the sample
    Bbig = np.tile(B, (20, 1))[:10007]
    Bt = torch.from_numpy(Bbig.astype(np.float32)).cuda()
    ldos, dsum = ctx().ldos_forward(model, Bt, api.MIXED)
    L = ldos.float().cpu().numpy()
    ref = oracle.mlp_forward(Bbig.astype(np.float32).astype(np.float64), mlp.W, mlp.b, mlp.leaky_slope,
                             mlp.in_shift, mlp.in_scale)
    assert _ldos_error(L, ref) < LDOS_TOL
    # identical rows give identical outputs (no tile-dependent state)
    np.testing.assert_array_equal(L[:512], L[512:1024])
    empty = torch.zeros((0, 91), dtype=torch.float32, device="cuda")
    l0, d0 = ctx().ldos_forward(model, empty, api.MIXED)
    assert l0.shape == (0, 250) and float(d0.abs().sum()) == 0.0


@pytest.mark.parametrize("dims,twojmax", [((30, 100, 100, 11), 6), ((91, 400, 400, 250), 10)])
def test_fp64_network_matches_oracle(dims, twojmax):
    torch = need_gpu()
    from paper_2411_19617_gb300 import api
    B = _descriptor_sample(twojmax)[:300]
    mlp = _model(dims, 5, _descriptor_sample(twojmax))
    model = api.Model(ctx(), mlp)
    ldos, dsum = ctx().ldos_forward(model, torch.from_numpy(B).cuda(), api.FP64_PLAIN)
    ref = oracle.mlp_forward(B, mlp.W, mlp.b, mlp.leaky_slope, mlp.in_shift, mlp.in_scale)
    np.testing.assert_allclose(ldos.cpu().numpy(), ref, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(dsum.cpu().numpy(), ref.sum(axis=0), rtol=1e-12)


def test_model_shape_errors():
    need_gpu()
    from paper_2411_19617_gb300 import api
    from paper_2411_19617_gb300._lib import MalaError
    big = wl.random_mlp((91, 1000, 10), seed=1)
    m = api.Model(ctx(), big)  # accepted (FP64 path), MIXED refuses
    import torch
    with pytest.raises(MalaError):
        ctx().ldos_forward(m, torch.zeros((4, 91), device="cuda"), api.MIXED)
