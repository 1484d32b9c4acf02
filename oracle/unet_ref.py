"""Plain FP64 CPU reference of the warm-start U-Net: forward pass, MSE loss and every gradient.

TEST INFRASTRUCTURE ONLY (tests); shares nothing with the CUDA library.  Composed from the
convolution reference in conv_ref.py plus pooling, upsampling, ReLU, the 1x1 head and the
loss written out plainly.

The network (the learned warm start's architecture: 4 levels with 16/32/64/64 channels, two
3x3x3 circular convolutions + ReLU per level, 2x average pooling on the way down, nearest 2x
upsampling and channel concatenation [upsampled | skip] on the way up, a 1x1 head to 4
outputs) maps the 16-channel input (rho - <rho>) s_rho, S_i s_S, K s_K, zeros to
(u / s_u, W_i / s_W).

Parameters: one flat FP32 vector, per convolution in forward order (e0a, e0, e1a, e1, e2a, e2,
ba, b, d2a, d2, d1a, d1, d0a, d0) the weights [27][cout][cin] then the bias [cout], then the head
weights [4][16] and bias [4].

Precision: the tensors the GPU keeps in BF16 (inputs, activations, pooled and concatenated
features, activation gradients) are rounded to BF16 here at the same points (conv_ref.bf16_round,
round to nearest even), so that both sides take their ReLU and rounding decisions on the same
values; every sum is FP64.  Convolution weights enter as their BF16 roundings, biases and the
head in FP32 values.
"""
import numpy as np

from . import conv_ref as R

CH = (16, 32, 64, 64)
CIN0, COUT = 16, 4
CONVS = [("e0a", CIN0, CH[0]), ("e0", CH[0], CH[0]), ("e1a", CH[0], CH[1]), ("e1", CH[1], CH[1]),
         ("e2a", CH[1], CH[2]), ("e2", CH[2], CH[2]), ("ba", CH[2], CH[3]), ("b", CH[3], CH[3]),
         ("d2a", CH[3] + CH[2], CH[2]), ("d2", CH[2], CH[2]), ("d1a", CH[2] + CH[1], CH[1]),
         ("d1", CH[1], CH[1]), ("d0a", CH[1] + CH[0], CH[0]), ("d0", CH[0], CH[0])]


def _rounder(rounding):
    return R.bf16_round if rounding else (lambda a: np.asarray(a, dtype=np.float64))


def layout():
    """{name: (weight offset, (27, cout, cin), bias offset, cout)} and the total length."""
    out, off = {}, 0
    for name, cin, cout in CONVS:
        out[name] = (off, (27, cout, cin), off + 27 * cout * cin, cout)
        off += 27 * cout * cin + cout
    out["head"] = (off, (COUT, CH[0]), off + COUT * CH[0], COUT)
    off += COUT * CH[0] + COUT
    return out, off


def unpack(flat):
    lay, n = layout()
    flat = np.asarray(flat, dtype=np.float64)
    assert flat.size == n
    return {k: (flat[o:o + int(np.prod(s))].reshape(s), flat[bo:bo + nb]) for k, (o, s, bo, nb) in lay.items()}


def pack(grads):
    lay, n = layout()
    flat = np.zeros(n)
    for k, (o, s, bo, nb) in lay.items():
        flat[o:o + int(np.prod(s))] = grads[k][0].reshape(-1)
        flat[bo:bo + nb] = grads[k][1]
    return flat


def network_input(rho0, rho2, S, K, s_rho, s_S, s_K):
    """The 16-channel BF16 input of (rho0, rho2, S) arrays of shape (n, n, n) / (3, n, n, n)."""
    r = rho0 + rho2
    x = np.zeros(r.shape + (CIN0,))
    f32 = lambda v: np.asarray(v, dtype=np.float32).astype(np.float64)
    x[..., 0] = (r - r.mean()) * f32(s_rho)
    for a in range(3):
        x[..., 1 + a] = S[a] * f32(s_S)
    x[..., 4] = K * f32(s_K)
    return R.bf16_round(np.asarray(x, dtype=np.float32))


def target(u, W, s_u, s_W):
    t = np.empty(u.shape + (COUT,))
    t[..., 0] = u / s_u
    for a in range(3):
        t[..., 1 + a] = W[a] / s_W
    return np.asarray(t, dtype=np.float32).astype(np.float64)


def pool(x):
    n = x.shape[0] // 2
    return x.reshape(n, 2, n, 2, n, 2, -1).mean(axis=(1, 3, 5))


def pool_adjoint(g):
    return np.repeat(np.repeat(np.repeat(g, 2, 0), 2, 1), 2, 2) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def up_adjoint(g):
    n = g.shape[0] // 2
    return g.reshape(n, 2, n, 2, n, 2, -1).sum(axis=(1, 3, 5))


def forward(P, x0, rounding=True):
    """Activations of every layer (dict) and the FP64 head output (n, n, n, 4).  rounding=False
    keeps everything in FP64 (the smooth function whose derivatives the tests check)."""
    bf = _rounder(rounding)
    w = {k: (bf(v[0]) if k != "head" else v[0], v[1]) for k, v in P.items()}
    conv = lambda name, x: bf(R.conv_fwd(x, w[name][0], w[name][1], relu=True))
    a = {"x0": x0}
    a["e0a"] = conv("e0a", x0)
    a["e0"] = conv("e0", a["e0a"])
    a["p1"] = bf(pool(a["e0"]))
    a["e1a"] = conv("e1a", a["p1"])
    a["e1"] = conv("e1", a["e1a"])
    a["p2"] = bf(pool(a["e1"]))
    a["e2a"] = conv("e2a", a["p2"])
    a["e2"] = conv("e2", a["e2a"])
    a["p3"] = bf(pool(a["e2"]))
    a["ba"] = conv("ba", a["p3"])
    a["b"] = conv("b", a["ba"])
    a["cat2"] = np.concatenate([up(a["b"]), a["e2"]], axis=-1)
    a["d2a"] = conv("d2a", a["cat2"])
    a["d2"] = conv("d2", a["d2a"])
    a["cat1"] = np.concatenate([up(a["d2"]), a["e1"]], axis=-1)
    a["d1a"] = conv("d1a", a["cat1"])
    a["d1"] = conv("d1", a["d1a"])
    a["cat0"] = np.concatenate([up(a["d1"]), a["e0"]], axis=-1)
    a["d0a"] = conv("d0a", a["cat0"])
    a["d0"] = conv("d0", a["d0a"])
    hw, hb = P["head"]
    out = a["d0"] @ hw.T + hb
    return a, out, w


def loss_and_grads(P, x0, t, rounding=True):
    """MSE loss mean((out - t)^2) and the gradient of every parameter: {name: (dW, db)}."""
    bf = _rounder(rounding)
    a, out, w = forward(P, x0, rounding)
    cnt = out.size
    loss = float(np.mean((out - t) ** 2))
    dout = 2.0 * (out - t) / cnt
    if rounding:
        dout = np.asarray(dout, dtype=np.float32).astype(np.float64)
    g = {}
    hw, _ = P["head"]
    g["head"] = (dout.reshape(-1, COUT).T @ a["d0"].reshape(-1, CH[0]), dout.reshape(-1, COUT).sum(axis=0))
    gd0 = bf(dout @ hw)

    def conv_bwd(name, x, y, dy, need_dx=True):
        dy = np.where(y > 0, dy, 0.0)
        g[name] = (R.conv_wgrad(x, dy), dy.reshape(-1, dy.shape[-1]).sum(axis=0))
        return bf(R.conv_dgrad(dy, w[name][0])) if need_dx else None

    gd0a = conv_bwd("d0", a["d0a"], a["d0"], gd0)
    gcat0 = conv_bwd("d0a", a["cat0"], a["d0a"], gd0a)
    gd1 = bf(up_adjoint(gcat0[..., :CH[1]]))
    gd1a = conv_bwd("d1", a["d1a"], a["d1"], gd1)
    gcat1 = conv_bwd("d1a", a["cat1"], a["d1a"], gd1a)
    gd2 = bf(up_adjoint(gcat1[..., :CH[2]]))
    gd2a = conv_bwd("d2", a["d2a"], a["d2"], gd2)
    gcat2 = conv_bwd("d2a", a["cat2"], a["d2a"], gd2a)
    gb = bf(up_adjoint(gcat2[..., :CH[3]]))
    gba = conv_bwd("b", a["ba"], a["b"], gb)
    gp3 = conv_bwd("ba", a["p3"], a["ba"], gba)
    ge2 = bf(gcat2[..., CH[3]:] + pool_adjoint(gp3))        # skip gradient + pooling adjoint
    ge2a = conv_bwd("e2", a["e2a"], a["e2"], ge2)
    gp2 = conv_bwd("e2a", a["p2"], a["e2a"], ge2a)
    ge1 = bf(gcat1[..., CH[2]:] + pool_adjoint(gp2))
    ge1a = conv_bwd("e1", a["e1a"], a["e1"], ge1)
    gp1 = conv_bwd("e1a", a["p1"], a["e1a"], ge1a)
    ge0 = bf(gcat0[..., CH[1]:] + pool_adjoint(gp1))
    ge0a = conv_bwd("e0", a["e0a"], a["e0"], ge0)
    conv_bwd("e0a", a["x0"], a["e0a"], ge0a, need_dx=False)
    return loss, g, out
