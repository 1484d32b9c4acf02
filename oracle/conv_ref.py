"""Plain FP64 CPU reference of the warm-start network's convolution and its gradients.

TEST INFRASTRUCTURE ONLY (tests and smoke check); shares nothing with the CUDA library.
Tensors: numpy arrays of shape (nz, ny, nx, C) (NDHWC), periodic (circular) boundaries.
Weights: w[t, co, ci] with tap t = (dz+1)*9 + (dy+1)*3 + (dx+1); the forward convolution is
    y[v, co] = b[co] + sum_t sum_ci w[t, co, ci] x[v + d_t, ci]
(cross-correlation with circular wrap), its input gradient the adjoint map, and its weight
gradient dW[t, co, ci] = sum_v dy[v, co] x[v + d_t, ci].
"""
import numpy as np


def taps():
    return [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shift(x, d):
    """x[v + d] with circular wrap (axes z, y, x)."""
    dz, dy, dx = d
    return np.roll(x, shift=(-dz, -dy, -dx), axis=(0, 1, 2))


def conv_fwd(x, w, b=None, relu=False):
    x = np.asarray(x, dtype=np.float64)
    y = np.zeros(x.shape[:3] + (w.shape[1],))
    for t, d in enumerate(taps()):
        y += shift(x, d) @ np.asarray(w[t], dtype=np.float64).T
    if b is not None:
        y += b
    return np.maximum(y, 0.0) if relu else y


def conv_dgrad(dy, w):
    """adjoint of conv_fwd (without bias / activation) applied to dy."""
    dy = np.asarray(dy, dtype=np.float64)
    dx = np.zeros(dy.shape[:3] + (w.shape[2],))
    for t, d in enumerate(taps()):
        dx += shift(dy @ np.asarray(w[t], dtype=np.float64), tuple(-q for q in d))
    return dx


def conv_wgrad(x, dy):
    x = np.asarray(x, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    cin, cout = x.shape[3], dy.shape[3]
    dw = np.zeros((27, cout, cin))
    for t, d in enumerate(taps()):
        dw[t] = dy.reshape(-1, cout).T @ shift(x, d).reshape(-1, cin)
    return dw


def bf16_round(a):
    """Round float64/float32 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
