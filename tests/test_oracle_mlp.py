"""Pin of the FP64 network oracle (Eq. ffnn) against torch's own layers."""
import numpy as np
import pytest

import oracle
from paper_2411_19617_gb300 import workloads as wl


def test_mlp_matches_torch_layers():
    torch = pytest.importorskip("torch")
    mlp = wl.random_mlp((30, 100, 100, 11), seed=3)
    x = np.random.default_rng(0).normal(size=(64, 30))
    ref = torch.from_numpy(x)
    for l in range(3):
        ref = torch.nn.functional.linear(ref, torch.from_numpy(mlp.W[l]), torch.from_numpy(mlp.b[l]))
        if l < 2:
            ref = torch.nn.functional.leaky_relu(ref, negative_slope=0.01)
    got = oracle.mlp_forward(x, mlp.W, mlp.b)
    np.testing.assert_allclose(got, ref.numpy(), rtol=1e-13, atol=1e-13)


def test_mlp_input_scaling_and_output_activation():
    mlp = wl.random_mlp((4, 5, 3), seed=4)
    x = np.random.default_rng(1).normal(size=(7, 4))
    shift, scale = np.arange(4.0), np.array([0.5, 2.0, 1.0, 3.0])
    got = oracle.mlp_forward(x, mlp.W, mlp.b, in_shift=shift, in_scale=scale)
    xs = (x - shift) * scale
    h = xs @ mlp.W[0].T + mlp.b[0]
    h = np.maximum(h, 0) + 0.01 * np.minimum(h, 0)
    ref = h @ mlp.W[1].T + mlp.b[1]
    np.testing.assert_allclose(got, ref, rtol=1e-14)
    got2 = oracle.mlp_forward(x, mlp.W, mlp.b, in_shift=shift, in_scale=scale, activate_output=True)
    np.testing.assert_allclose(got2, np.maximum(ref, 0) + 0.01 * np.minimum(ref, 0), rtol=1e-14)


def test_random_init_bounds():
    mlp = wl.random_mlp((91, 400, 400, 250), seed=12)
    for l, W in enumerate(mlp.W):
        bound = 1.0 / np.sqrt(mlp.dims[l])
        assert W.shape == (mlp.dims[l + 1], mlp.dims[l])
        assert np.abs(W).max() <= bound and np.abs(mlp.b[l]).max() <= bound
