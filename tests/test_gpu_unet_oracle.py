"""The warm-start network on the GPU against the FP64 CPU oracle of the whole network.

One training step of the U-Net (input packing, forward pass with the tcgen05 convolutions,
MSE loss, backward pass through every layer: input and weight gradients of all 14
convolutions, pooling and upsampling adjoints, the head) against oracle/unet_ref.py, which
composes the plain FP64 convolution reference with pooling, upsampling, ReLU and the head,
rounding to BF16 where the GPU stores BF16.  With both sides taking their ReLU and rounding
decisions on the same BF16 values, what remains is FP32 (GPU) against FP64 (oracle)
accumulation and the rare value that lands on the other side of a BF16 rounding boundary:
the bars are 1% relative max-error of the output and 2% relative L2 error of every
parameter tensor's gradient (a dropped layer, a wrong tap, a transposed weight or a missing
skip gradient gives O(1)).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import unet_ref as UR  # noqa: E402
from paper_2501_13046_gb300 import fields  # noqa: E402

N = 64
K = -6.14


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_13046_gb300 import _build
    _build.build()
    from paper_2501_13046_gb300 import unet, warmstart
    return unet, warmstart


def test_training_step_matches_the_cpu_oracle(mods):
    U, WS = mods
    P = WS.Params(seed=3)
    flat = P.state()
    sc = WS.Scales(s_rho=1e3, s_S=1e6, s_K=1 / 6.0, s_u=0.05, s_W=1e-5)
    q = fields.batch_instance(N, 5e-5, 10000)      # host arrays: the same values go to both sides
    rng = np.random.default_rng(4)
    u = 0.03 * rng.standard_normal((N,) * 3)
    W = 1e-5 * rng.standard_normal((3,) + (N,) * 3)

    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    p = dict(q, rho0=dev(q["rho0"]), rho2=dev(q["rho2"]), S=dev(q["S"]))
    net = WS.Net(P, N, train=True)
    P.g.zero_()
    WS.train_step(net, p, K, dev(u), dev(W), sc)
    torch.cuda.synchronize()
    assert int(net.err.item()) == 0
    x0_gpu = net.x0.float().cpu().numpy().astype(np.float64)
    out_gpu = net.out.cpu().numpy().astype(np.float64)
    loss_gpu = float(net.loss.item())
    g_gpu = UR.unpack(P.g.cpu().numpy())

    x0 = UR.network_input(q["rho0"], q["rho2"], q["S"], K, sc.s_rho, sc.s_S, sc.s_K)
    t = UR.target(u, W, sc.s_u, sc.s_W)
    loss, g, out = UR.loss_and_grads(UR.unpack(flat), x0, t)

    # input packing: identical BF16 values (up to a last-bit difference of the mean's summation order)
    assert np.abs(x0_gpu - x0).max() <= 2 ** -8 * np.abs(x0).max()
    assert np.mean(x0_gpu != x0) < 1e-3
    assert np.abs(out_gpu - out).max() <= 1e-2 * np.abs(out).max()
    assert loss_gpu == pytest.approx(loss, rel=1e-3)
    worst = {}
    for name in [c[0] for c in UR.CONVS] + ["head"]:
        for part, (a, b) in zip(("w", "b"), zip(g_gpu[name], g[name])):
            err = np.linalg.norm(a - b) / np.linalg.norm(b)
            worst[name + "." + part] = err
    assert max(worst.values()) <= 2e-2, sorted(worst.items(), key=lambda kv: -kv[1])[:5]
