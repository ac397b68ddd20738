"""Pins of the CNN oracle (oracle/cnn.py) against things other than itself:
scipy's 2D correlation, hand-built delta kernels, central finite differences
of the loss, and torch's BF16 conversion for the rounding helper."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn


def test_conv3x3_equals_scipy_correlation():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 9, 11, 3))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    out = cnn.conv3x3(x, W, b)
    for bi in range(2):
        for o in range(4):
            ref = b[o] + sum(correlate2d(x[bi, :, :, c], W[o, c], mode="same", boundary="fill")
                             for c in range(3))
            np.testing.assert_allclose(out[bi, :, :, o], ref, rtol=0, atol=1e-12)


def test_conv3x3_delta_kernels():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 6, 7, 2))
    W = np.zeros((2, 2, 3, 3))
    W[0, 0, 1, 1] = W[1, 1, 1, 1] = 1.0            # centre tap: identity
    np.testing.assert_array_equal(cnn.conv3x3(x, W, np.zeros(2)), x)
    W = np.zeros((1, 2, 3, 3))
    W[0, 1, 0, 0] = 1.0                             # tap (0, 0): x[i-1, j-1, 1]
    out = cnn.conv3x3(x, W, np.zeros(1))[0, :, :, 0]
    ref = np.zeros((6, 7))
    ref[1:, 1:] = x[0, :-1, :-1, 1]
    np.testing.assert_array_equal(out, ref)


def _perturbed_loss(params, x, t, k, which, idx, h):
    p2 = [(W.copy(), b.copy()) for W, b in params]
    arr = p2[k][which]
    arr[idx] += h
    return cnn.loss_and_grads(p2, x, t)[0]


@pytest.mark.parametrize("k", [0, 1, 2])
def test_gradients_match_finite_differences(k):
    rng = np.random.default_rng(2 + k)
    params = cnn.init_params(7)
    params = [(W, rng.normal(scale=0.1, size=b.shape)) for W, b in params]
    x = rng.normal(size=(2, 8, 10, 6))
    t = rng.normal(size=(2, 8, 10, 2))
    _, grads = cnn.loss_and_grads(params, x, t)
    dW, db = grads[k]
    W = params[k][0]
    h = 1e-6
    for _ in range(12):
        idx = tuple(int(rng.integers(0, s)) for s in W.shape)
        fd = (_perturbed_loss(params, x, t, k, 0, idx, h) -
              _perturbed_loss(params, x, t, k, 0, idx, -h)) / (2 * h)
        assert abs(fd - dW[idx]) <= 1e-6 * max(1e-3, abs(fd)), (k, idx, fd, dW[idx])
    o = int(rng.integers(0, params[k][1].size))
    fd = (_perturbed_loss(params, x, t, k, 1, (o,), h) -
          _perturbed_loss(params, x, t, k, 1, (o,), -h)) / (2 * h)
    assert abs(fd - db[o]) <= 1e-6 * max(1e-3, abs(fd))


def test_input_gradient_matches_finite_differences():
    rng = np.random.default_rng(9)
    x = rng.normal(size=(1, 5, 6, 3))
    W = rng.normal(size=(2, 3, 3, 3))
    g = rng.normal(size=(1, 5, 6, 2))
    dx, _, _ = cnn.conv3x3_backward(x, W, g)
    h = 1e-6
    for _ in range(10):
        idx = tuple(int(rng.integers(0, s)) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = ((cnn.conv3x3(xp, W, np.zeros(2)) - cnn.conv3x3(xm, W, np.zeros(2))) * g).sum() / (2 * h)
        assert abs(fd - dx[idx]) <= 1e-7 * max(1.0, abs(fd))


def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    a = np.concatenate([[1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.5, 0.0, 3e-5],
                        np.random.default_rng(4).normal(scale=50, size=1000)])
    ref = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(cnn.round_bf16(a), ref)
    assert cnn.round_bf16(np.array([1 + 2 ** -8]))[0] == 1.0           # tie to even
    assert cnn.round_bf16(np.array([1 + 3 * 2 ** -8]))[0] == 1 + 2 ** -6
