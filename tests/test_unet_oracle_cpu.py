"""Pins of the U-Net CPU oracle (oracle/unet_ref.py), on the CPU.

With its BF16 rounding switched off the oracle is a smooth (piecewise linear through the
ReLUs) FP64 function of the parameters, so its backward pass must equal central differences
of its own loss for every parameter tensor of every layer: a wrong adjoint (pooling,
upsampling, concatenation split, skip gradient, flipped taps) fails here.  Its building
blocks are pinned separately in test_conv_oracle.py.  The grid is 16^3 (the oracle has no
size rule; the GPU network needs 64^3).
"""
import numpy as np
import pytest

from oracle import unet_ref as UR

N = 16


@pytest.fixture(scope="module")
def setup():
    rng = np.random.default_rng(0)
    lay, n = UR.layout()
    flat = np.zeros(n)
    for name, cin, cout in UR.CONVS:
        o, shp, bo, nb = lay[name]
        flat[o:o + int(np.prod(shp))] = rng.standard_normal(int(np.prod(shp))) * np.sqrt(2.0 / (27 * cin))
        flat[bo:bo + nb] = 0.1 * rng.standard_normal(nb)
    o, shp, bo, nb = lay["head"]
    flat[o:o + int(np.prod(shp))] = rng.standard_normal(int(np.prod(shp))) * 0.25
    flat[bo:bo + nb] = 0.1 * rng.standard_normal(nb)
    x0 = rng.standard_normal((N, N, N, UR.CIN0))
    t = rng.standard_normal((N, N, N, UR.COUT))
    loss, g, out = UR.loss_and_grads(UR.unpack(flat), x0, t, rounding=False)
    return rng, lay, flat, x0, t, UR.pack(g)


def loss_at(flat, x0, t):
    _, out, _ = UR.forward(UR.unpack(flat), x0, rounding=False)
    return float(np.mean((out - t) ** 2))


@pytest.mark.parametrize("name", [c[0] for c in UR.CONVS] + ["head"])
def test_gradient_equals_central_differences(setup, name):
    rng, lay, flat, x0, t, grad = setup
    o, shp, bo, nb = lay[name]
    # one weight (the largest-gradient entry of a random tap) and one bias of this layer
    size = int(np.prod(shp))
    block = grad[o:o + size]
    w_idx = o + int(np.argmax(np.abs(block)))
    b_idx = bo + int(np.argmax(np.abs(grad[bo:bo + nb])))
    for idx in (w_idx, b_idx):
        assert grad[idx] != 0.0
        eps = 1e-6 * max(1.0, abs(flat[idx]))
        fp, fm = flat.copy(), flat.copy()
        fp[idx] += eps
        fm[idx] -= eps
        fd = (loss_at(fp, x0, t) - loss_at(fm, x0, t)) / (2 * eps)
        assert fd == pytest.approx(grad[idx], rel=1e-6, abs=1e-10 * np.abs(grad).max()), (name, idx)


def test_rounded_forward_stays_close_to_the_exact_one(setup):
    """The BF16 storage points change the output by about the BF16 step, not more."""
    rng, lay, flat, x0, t, grad = setup
    x0b = UR.R.bf16_round(x0)
    _, exact, _ = UR.forward(UR.unpack(flat), x0b, rounding=False)
    _, rounded, _ = UR.forward(UR.unpack(flat), x0b, rounding=True)
    rel = np.linalg.norm(rounded - exact) / np.linalg.norm(exact)
    assert 0.0 < rel < 0.05
