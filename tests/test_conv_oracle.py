"""Pins of the CPU convolution oracle (oracle/conv_ref.py) against independent facts."""
import numpy as np
import pytest

from oracle import conv_ref as R


def rand(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def test_forward_matches_scipy_wrap_correlation():
    """Single channel pair: the forward map is scipy's circular cross-correlation."""
    ndi = pytest.importorskip("scipy.ndimage")
    x = rand((6, 5, 7, 1), 1)
    w = rand((27, 1, 1), 2)
    k = w[:, 0, 0].reshape(3, 3, 3)       # k[dz+1, dy+1, dx+1]
    want = ndi.correlate(x[..., 0], k, mode="wrap")
    np.testing.assert_allclose(R.conv_fwd(x, w)[..., 0], want, atol=1e-12)


def test_constant_field_closed_form():
    x = np.full((4, 4, 4, 3), 2.0)
    w = rand((27, 2, 3), 3)
    b = np.array([0.5, -1.0])
    y = R.conv_fwd(x, w, b)
    np.testing.assert_allclose(y, (2.0 * w.sum(axis=(0, 2)) + b) * np.ones((4, 4, 4, 2)), atol=1e-12)


def test_dgrad_is_the_adjoint():
    x = rand((5, 4, 6, 3), 4)
    dy = rand((5, 4, 6, 2), 5)
    w = rand((27, 2, 3), 6)
    lhs = np.sum(R.conv_fwd(x, w) * dy)
    rhs = np.sum(x * R.conv_dgrad(dy, w))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_wgrad_is_the_derivative_in_w():
    """<conv(x; w), dy> is linear in w, so its gradient equals any finite difference exactly."""
    x = rand((4, 5, 3, 2), 7)
    dy = rand((4, 5, 3, 3), 8)
    w = rand((27, 3, 2), 9)
    g = R.conv_wgrad(x, dy)
    rng = np.random.default_rng(10)
    for _ in range(5):
        t, co, ci = rng.integers(27), rng.integers(3), rng.integers(2)
        e = np.zeros_like(w)
        e[t, co, ci] = 1.0
        fd = np.sum(R.conv_fwd(x, w + e) * dy) - np.sum(R.conv_fwd(x, w) * dy)
        assert g[t, co, ci] == pytest.approx(fd, rel=1e-10)


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 3.14159, -2.5e-3, 0.0])
    r = R.bf16_round(vals)
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0 + 2 ** -7   # ties to even, representable
    assert abs(r[3] - 3.140625) < 1e-12 and r[5] == 0.0
