"""The warm-start network on the GPU against the FP64 CPU oracle of the whole network.

One training step of the U-Net (input packing, forward pass with the tcgen05 convolutions,
MSE loss, backward pass through every layer: input and weight gradients of all 14
convolutions, pooling and upsampling adjoints, the head) against oracle/unet_ref.py, which
composes the plain FP64 convolution reference with pooling, upsampling, ReLU and the head,
rounding to BF16 where the GPU stores BF16.

Both sides round the same values to BF16 at the same points, so what separates them is FP32
(GPU, tensor cores) against FP64 (oracle) accumulation: a sum that lands within an FP32
rounding of a BF16 rounding boundary goes one BF16 step (2^-8 relative) the other way, and such
one-step flips then propagate through the later layers.  The checks:

* the packed input and the first convolution's output agree value for value up to one BF16
  step (a wrong tap, weight layout or bias shows up here at O(1));
* every later activation, the output and every parameter gradient agree to a relative L2
  error of a few percent, and the output's error is of the same size as the oracle's own
  rounding noise (its BF16-stored result against the same network in exact FP64): the GPU is
  as close to the oracle as the oracle is to exact arithmetic.  A dropped layer, a wrong
  adjoint or a missing skip gradient gives O(1).
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

    # input packing and the first layer: value for value, up to one BF16 step
    assert np.abs(x0_gpu - x0).max() <= 2 ** -8 * np.abs(x0).max()
    assert np.mean(x0_gpu != x0) < 1e-3
    acts, _, _ = UR.forward(UR.unpack(flat), x0)
    e0a = net.a["e0a"].float().cpu().numpy().astype(np.float64)
    step = np.abs(e0a - acts["e0a"]) <= 2 ** -8 * np.abs(acts["e0a"]) + 1e-30
    assert np.mean(step) > 0.999, np.mean(step)
    # later layers, output, loss: relative L2 errors of a few percent, the oracle's own rounding scale
    rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
    gpu_acts = {"e0a": net.a["e0a"], "p1": net.a["p1"], "e1a": net.a["e1a"], "p2": net.a["p2"],
                "e2a": net.a["e2a"], "p3": net.a["p3"], "ba": net.a["ba"], "b": net.a["b"], "d2a": net.a["d2a"],
                "d2": net.a["d2"], "d1a": net.a["d1a"], "d1": net.a["d1"], "d0a": net.a["d0a"], "d0": net.a["d0"]}
    act_err = {k: rel(v.float().cpu().numpy().astype(np.float64), acts[k]) for k, v in gpu_acts.items()}
    _, out_exact, _ = UR.forward(UR.unpack(flat), x0, rounding=False)
    noise = rel(out, out_exact)
    out_err = rel(out_gpu, out)
    grad_err = {}
    for name in [c[0] for c in UR.CONVS] + ["head"]:
        for part, (a, b) in zip(("w", "b"), zip(g_gpu[name], g[name])):
            grad_err[name + "." + part] = rel(a, b)
    report = dict(activations=act_err, output=out_err, oracle_rounding_noise=noise, loss=(loss_gpu, loss),
                  worst_gradients=sorted(grad_err.items(), key=lambda kv: -kv[1])[:6])
    print(report)
    assert max(act_err.values()) <= 0.05, report
    assert out_err <= 0.05 and out_err <= 2.0 * noise + 1e-3, report
    assert loss_gpu == pytest.approx(loss, rel=0.02), report
    assert max(grad_err.values()) <= 0.10, report
