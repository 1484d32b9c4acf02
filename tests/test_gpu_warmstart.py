"""Warm-start network: glue kernels against numpy, the full network's backward wiring against a
directional derivative of its own forward pass, and training lowering the loss."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import conv_ref as R  # noqa: E402


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_13046_gb300 import _build
    _build.build()
    from paper_2501_13046_gb300 import unet, warmstart, fields, mg
    return unet, warmstart, fields, mg


def bf16t(a):
    return torch.from_numpy(np.ascontiguousarray(R.bf16_round(a), dtype=np.float32)).to(torch.bfloat16).cuda()


def host(t):
    return t.float().cpu().numpy().astype(np.float64)


def test_pool_upsample_and_adjoints(mods):
    U = mods[0]
    rng = np.random.default_rng(1)
    x = R.bf16_round(rng.standard_normal((8, 8, 8, 16)))
    y = torch.zeros((4, 4, 4, 16), dtype=torch.bfloat16, device="cuda")
    U.avgpool2(bf16t(x), y, 16, (8, 8, 8))
    want = x.reshape(4, 2, 4, 2, 4, 2, 16).mean(axis=(1, 3, 5))
    np.testing.assert_allclose(host(y), want, rtol=2 ** -7, atol=1e-6)
    up = torch.zeros((8, 8, 8, 16), dtype=torch.bfloat16, device="cuda")
    U.upsample2(y, up, 16, (4, 4, 4))
    np.testing.assert_array_equal(host(up), np.repeat(np.repeat(np.repeat(host(y), 2, 0), 2, 1), 2, 2))
    # adjoints: <pool x, g> = <x, pool^T g>, <up c, f> = <c, up^T f>
    g = R.bf16_round(rng.standard_normal((4, 4, 4, 16)))
    dx = torch.zeros((8, 8, 8, 16), dtype=torch.bfloat16, device="cuda")
    U.avgpool2_bwd(bf16t(g), dx, 16, (8, 8, 8), False)
    assert np.sum(want * g) == pytest.approx(np.sum(x * host(dx)), rel=1e-2)
    f = R.bf16_round(rng.standard_normal((8, 8, 8, 16)))
    dc = torch.zeros((4, 4, 4, 16), dtype=torch.bfloat16, device="cuda")
    U.upsample2_bwd(bf16t(f), dc, 16, (4, 4, 4))
    np.testing.assert_allclose(host(dc), f.reshape(4, 2, 4, 2, 4, 2, 16).sum(axis=(1, 3, 5)), rtol=2 ** -7, atol=1e-5)


def test_row_parallel_glue_on_slices_non_cubes_and_fields(mods):
    """Pooling and upsampling on channel slices of non-cubic grids (8 channels per thread), and the
    FP64 restriction (8-child mean) and prolongation (cell-centred trilinear, periodic) of several
    fields, against numpy; a channel count that is not a multiple of 8 is rejected."""
    U = mods[0]
    from paper_2501_13046_gb300.unet import Slice
    rng = np.random.default_rng(7)
    nz, ny, nx = 4, 8, 16
    big = R.bf16_round(rng.standard_normal((nz, ny, nx, 48)))
    ybuf = torch.full((nz // 2, ny // 2, nx // 2, 32), 3.0, dtype=torch.bfloat16, device="cuda")
    U.avgpool2(Slice(bf16t(big), 16, 24), Slice(ybuf, 8, 24), 24, (nx, ny, nz))
    out = host(ybuf)
    want = big[..., 16:40].reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2, 24).mean(axis=(1, 3, 5))
    np.testing.assert_allclose(out[..., 8:32], want, rtol=2 ** -7, atol=1e-6)
    assert np.all(out[..., :8] == 3.0)
    ubuf = torch.full((nz, ny, nx, 40), 5.0, dtype=torch.bfloat16, device="cuda")
    U.upsample2(Slice(ybuf, 8, 24), Slice(ubuf, 16, 24), 24, (nx // 2, ny // 2, nz // 2))
    up = host(ubuf)
    np.testing.assert_array_equal(up[..., 16:40], np.repeat(np.repeat(np.repeat(out[..., 8:32], 2, 0), 2, 1), 2, 2))
    assert np.all(up[..., :16] == 5.0)
    with pytest.raises(RuntimeError):
        U.avgpool2(bf16t(big[..., :12]), ybuf[..., :12].contiguous(), 12, (nx, ny, nz))
    # FP64 fields: restriction and prolongation of 3 fields on a (16, 8, 4) grid
    f = rng.standard_normal((3, nz, ny, nx))
    fd = torch.from_numpy(f).cuda()
    c = torch.empty((3, nz // 2, ny // 2, nx // 2), dtype=torch.float64, device="cuda")
    U.restrict2_fields(fd, c, 3, (nx // 2, ny // 2, nz // 2))
    want_c = f.reshape(3, nz // 2, 2, ny // 2, 2, nx // 2, 2).mean(axis=(2, 4, 6))
    np.testing.assert_allclose(c.cpu().numpy(), want_c, rtol=1e-14, atol=1e-15)
    fine = torch.empty((3, nz, ny, nx), dtype=torch.float64, device="cuda")
    U.prolong2_fields(c, fine, 3, (nx // 2, ny // 2, nz // 2))
    cc = c.cpu().numpy()

    def lin(a, axis):   # cell-centred linear 2x along one axis, periodic: 3/4 own + 1/4 neighbour
        lo = 0.75 * a + 0.25 * np.roll(a, 1, axis)
        hi = 0.75 * a + 0.25 * np.roll(a, -1, axis)
        return np.stack([lo, hi], axis=axis + 1).reshape(a.shape[:axis] + (2 * a.shape[axis],) + a.shape[axis + 1:])

    want_f = lin(lin(lin(cc, 1), 2), 3)
    np.testing.assert_allclose(fine.cpu().numpy(), want_f, rtol=1e-13, atol=1e-14)


def test_head_mse_bias_relu_adam(mods):
    U = mods[0]
    rng = np.random.default_rng(2)
    nv = 512
    x = R.bf16_round(rng.standard_normal((nv, 16)))
    w = rng.standard_normal((4, 16)).astype(np.float32)
    b = rng.standard_normal(4).astype(np.float32)
    out = torch.zeros((nv, 4), dtype=torch.float32, device="cuda")
    xt = bf16t(x).view(8, 8, 8, 16)
    U.head_fwd(xt, 16, torch.from_numpy(w).cuda(), torch.from_numpy(b).cuda(), out, 4, nv)
    ref = x @ w.T.astype(np.float64) + b
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-5, atol=1e-5)
    t = rng.standard_normal((nv, 4)).astype(np.float32)
    dout = torch.zeros_like(out)
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    U.mse(out, torch.from_numpy(t).cuda(), dout, loss, 4, nv)
    assert loss.item() == pytest.approx(np.mean((ref - t) ** 2), rel=1e-4)
    np.testing.assert_allclose(dout.cpu().numpy(), 2 * (ref - t) / (nv * 4), rtol=1e-4, atol=1e-8)
    dx = torch.zeros((8, 8, 8, 16), dtype=torch.bfloat16, device="cuda")
    dw = torch.zeros((4, 16), dtype=torch.float32, device="cuda")
    db = torch.zeros(4, dtype=torch.float32, device="cuda")
    U.head_bwd(xt, 16, torch.from_numpy(w).cuda(), dout, 4, dx, dw, db, nv)
    d = dout.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(dw.cpu().numpy(), d.T @ x, rtol=1e-4, atol=1e-7)
    np.testing.assert_allclose(db.cpu().numpy(), d.sum(0), rtol=1e-4, atol=1e-7)
    np.testing.assert_allclose(host(dx).reshape(nv, 16), d @ w.astype(np.float64), rtol=2 ** -7, atol=1e-6)
    # bias gradient and ReLU adjoint
    g = R.bf16_round(rng.standard_normal((8, 8, 8, 32)))
    gb = torch.zeros(32, dtype=torch.float32, device="cuda")
    U.bias_grad(bf16t(g), gb, 32, nv)
    np.testing.assert_allclose(gb.cpu().numpy(), g.reshape(-1, 32).sum(0), rtol=1e-5, atol=1e-5)
    yv = R.bf16_round(rng.standard_normal((8, 8, 8, 32)))
    gt = bf16t(g)
    U.relu_bwd(gt, bf16t(yv), 32, nv)
    np.testing.assert_array_equal(host(gt), np.where(yv > 0, g, 0.0))
    # Adam: one step equals the textbook update
    p = rng.standard_normal(100).astype(np.float32)
    gr = rng.standard_normal(100).astype(np.float32)
    pt, gt2 = torch.from_numpy(p.copy()).cuda(), torch.from_numpy(gr).cuda()
    m, v = torch.zeros_like(pt), torch.zeros_like(pt)
    U.adam(pt, gt2, m, v, 1e-3, 1)
    mh, vh = (0.1 * gr) / 0.1, (0.001 * gr * gr) / 0.001
    np.testing.assert_allclose(pt.cpu().numpy(), p - 1e-3 * mh / (np.sqrt(vh) + 1e-8), rtol=1e-5, atol=1e-7)


def sample(fields, n=64, seed=10000):
    p = fields.batch_instance(n, 5e-5, seed, device="cuda")
    return p


def test_backward_matches_directional_derivative(mods):
    U, WS, fields, mg = mods
    P = WS.Params(seed=3)
    net = WS.Net(P, 64, train=True)
    p = sample(fields)
    sc = WS.Scales(s_rho=1e3, s_S=1e6, s_K=1 / 6.0, s_u=0.05, s_W=1e-5)
    rng = np.random.default_rng(4)
    u = torch.from_numpy(0.03 * rng.standard_normal((64,) * 3)).cuda()
    W = torch.from_numpy(1e-5 * rng.standard_normal((3,) + (64,) * 3)).cuda()
    P.g.zero_()
    WS.train_step(net, p, -6.14, u, W, sc)
    torch.cuda.synchronize()
    assert int(net.err.item()) == 0
    grad = P.g.clone()
    d = torch.from_numpy(rng.standard_normal(P.n).astype(np.float32)).cuda()
    d *= 2e-2 * P.p.abs().mean() / d.abs().mean()   # well above the BF16 step of the activations
    base = P.p.clone()

    def loss_at(x):
        P.p.copy_(x)
        P.pack()
        net.loss.zero_()
        WS.pack_input(net, p, -6.14, sc)
        net.forward()
        U.pack_target(u, W, sc.s_u, sc.s_W, net.target, 64 ** 3)
        U.mse(net.out, net.target, net.dout, net.loss, 4, 64 ** 3)
        return float(net.loss.item())

    lp, lm = loss_at(base + d), loss_at(base - d)
    P.p.copy_(base)
    P.pack()
    fd = (lp - lm) / 2.0
    an = float((grad * d).sum().item())
    assert np.sign(fd) == np.sign(an) and abs(fd - an) <= 0.25 * abs(an), (fd, an)


def test_training_lowers_the_loss(mods):
    U, WS, fields, mg = mods
    P = WS.Params(seed=5)
    net = WS.Net(P, 64, train=True)
    ps = [sample(fields, seed=10000 + i) for i in range(2)]
    sols = []
    for p in ps:
        cfg = mg.config_for(p, mg.MG_MIXED, tol=1e-10)
        ctx = mg.mg_create(cfg, torch.cuda.current_stream().cuda_stream)
        mg.mg_set_sources(ctx, p["rho0"], p["rho2"], p["S"][0], p["S"][1], p["S"][2])
        mg.mg_solve(ctx)
        u = torch.empty((64,) * 3, dtype=torch.float64, device="cuda")
        W = torch.empty((3,) + (64,) * 3, dtype=torch.float64, device="cuda")
        mg.mg_get_solution(ctx, u, W)
        mg.mg_destroy(ctx)
        sols.append((u, W))
    sc = WS.Scales(s_rho=1.0 / float((ps[0]["rho0"] - ps[0]["rho0"].mean()).std()), s_S=1.0 / float(ps[0]["S"].std()),
                   s_K=1 / 6.0, s_u=float(sols[0][0].std()), s_W=float(sols[0][1].std()))
    losses = []
    for it in range(40):
        P.g.zero_()
        net.loss.zero_()
        for p, (u, W) in zip(ps, sols):
            WS.train_step(net, p, -6.14, u, W, sc)
        P.g.mul_(0.5)
        P.step(5e-4 * min(1.0, (it + 1) / 10))   # linear warm-up
        losses.append(float(net.loss.item()) / 2)
    torch.cuda.synchronize()
    assert int(net.err.item()) == 0
    assert max(losses) < 3 * losses[0] and np.mean(losses[-5:]) < 0.7 * losses[0], losses


def test_captured_inference_matches_eager(mods):
    """The warm-start inference captured once as a CUDA graph (restriction 128^3 -> 64^3, network,
    prolongation; K channel derived on the device from <rho>) gives the eager result bit for bit
    on two different instances replayed one after the other, and K = None equals the explicit
    pre-solve value -sqrt(24 pi <rho>)."""
    U, WS, fields, mg = mods
    P = WS.Params(seed=7)
    sc = WS.Scales(s_rho=1e3, s_S=1e6, s_K=1 / 6.0, s_u=0.05, s_W=1e-5)
    pred = WS.Predictor(P, 128, 64, sc)
    pred.capture()
    for seed in (20000, 20001):
        p = fields.batch_instance(128, 5e-5, seed, device="cuda")
        u0, W0 = torch.empty((128,) * 3, dtype=torch.float64, device="cuda"), \
            torch.empty((3,) + (128,) * 3, dtype=torch.float64, device="cuda")
        u1, W1 = torch.empty_like(u0), torch.empty_like(W0)
        pred.predict(p, None, u0, W0)
        pred.predict_graph(p, u1, W1)
        torch.cuda.synchronize()
        assert int(pred.net.err.item()) == 0
        assert torch.equal(u0, u1) and torch.equal(W0, W1)
        assert float(u0.abs().max()) > 0
        rho_mean = float((p["rho0"] + p["rho2"]).mean())
        u2, W2 = torch.empty_like(u0), torch.empty_like(W0)
        pred.predict(p, -np.sqrt(24 * np.pi * rho_mean), u2, W2)
        torch.cuda.synchronize()
        # the explicit value goes through the same BF16 channel; equal up to its FP64 mean order
        assert float((u2 - u0).abs().max()) <= 1e-6 * float(u0.abs().max()) + 1e-300
