"""The learned warm start behind the C ABI (mg_warmstart_load / mg_warmstart_predict /
mg_batch_warmstart_load), through ctypes.

* The library's own inference schedule gives the same guess, bit for bit, as the Python layer
  schedule (warmstart.Predictor) on the same kernels, at the network's size and at twice it.
* A network trained here on solver-generated 64^3 solutions (the library's tcgen05 training
  kernels) is the starting state on held-out instances, the solve from it reaches the same root
  as the cold solve, and it beats an untrained control: a start closer to the root (relative L2
  error of (u, W), W in units of its scale) and no more outer iterations than the cold start or
  the control on average.
* A batch serves the sizes the network takes and solves the rest cold.
* Malformed files and unsupported grids return the documented status codes.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2501_13046_gb300 import fields  # noqa: E402

SC = dict(s_rho=1e3, s_S=1e6, s_K=1 / 6.0, s_u=0.05, s_W=1e-5)


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_13046_gb300 import _build
    _build.build()
    from paper_2501_13046_gb300 import mg, warmstart
    return mg, warmstart


def context(mg, p, **over):
    cfg = mg.config_for(p, mg.MG_MIXED, tol=1e-10, max_outer=60, **over)
    ctx = mg.mg_create(cfg, torch.cuda.current_stream().cuda_stream)
    mg.mg_set_sources(ctx, p["rho0"], p["rho2"], p["S"][0], p["S"][1], p["S"][2])
    return ctx


def solution(mg, ctx, n):
    u = torch.empty((n,) * 3, dtype=torch.float64, device="cuda")
    W = torch.empty((3,) + (n,) * 3, dtype=torch.float64, device="cuda")
    mg.mg_get_solution(ctx, u, W)
    return u, W


@pytest.mark.parametrize("n", [64, 128])
def test_library_inference_matches_the_python_schedule(mods, tmp_path, n):
    mg, WS = mods
    P = WS.Params(seed=7)
    sc = WS.Scales(**SC)
    path = str(tmp_path / "net.bin")
    WS.save_weights(path, P, sc, 64)
    p = fields.batch_instance(n, 5e-5, 20000 + n, device="cuda")
    ctx = context(mg, p)
    try:
        mg.mg_warmstart_load(ctx, path)
        u = torch.empty((n,) * 3, dtype=torch.float64, device="cuda")
        W = torch.empty((3,) + (n,) * 3, dtype=torch.float64, device="cuda")
        mg.mg_warmstart_predict(ctx, u, W)
        u2, W2 = torch.empty_like(u), torch.empty_like(W)
        mg.mg_warmstart_predict(ctx, u2, W2)            # the captured graph, replayed
    finally:
        mg.mg_destroy(ctx)
    pred = WS.Predictor(P, n, 64, sc)
    ur, Wr = torch.empty_like(u), torch.empty_like(W)
    pred.predict(p, None, ur, Wr)
    torch.cuda.synchronize()
    assert float(ur.abs().max()) > 0
    assert torch.equal(u, ur) and torch.equal(W, Wr)
    assert torch.equal(u2, ur) and torch.equal(W2, Wr)


def train_network(mg, WS, samples=128, epochs=10):
    data = WS.make_dataset(mg, fields, list(range(10000, 10000 + samples)), n=64)
    sc = WS.fit_scales(data)
    P = WS.Params(seed=1)
    WS.train(P, data, sc, epochs=epochs, lr=1e-3, warmup=20, minibatch=8)
    return P, sc


def test_trained_start_is_accepted_reaches_the_cold_root_and_beats_the_control(mods, tmp_path):
    mg, WS = mods
    P, sc = train_network(mg, WS)
    trained, control = str(tmp_path / "trained.bin"), str(tmp_path / "control.bin")
    WS.save_weights(trained, P, sc, 64)
    WS.save_weights(control, WS.Params(seed=1), sc, 64)
    seeds = list(range(30000, 30008))   # held out: not among the training seeds
    it = {"cold": [], "trained": [], "control": []}
    err = {"cold": [], "trained": [], "control": []}   # relative L2 error of the start against the root
    for seed in seeds:
        a0 = float(np.random.Generator(np.random.PCG64(seed)).uniform(2e-5, 8e-5))
        p = fields.batch_instance(64, a0, seed, device="cuda")
        roots, guesses = {}, {}
        for name, path in (("cold", None), ("trained", trained), ("control", control)):
            ctx = context(mg, p, nested=0, field_tol=1e-10)
            try:
                if path:
                    mg.mg_warmstart_load(ctx, path)
                    guesses[name] = solution(mg, ctx, 64)
                    mg.mg_warmstart_predict(ctx, *guesses[name])
                    mg.mg_set_initial_guess(ctx, None, None)   # solve from the network's own start
                st, info = mg.mg_solve(ctx)
                assert st == mg.MG_OK and info["converged"]
                roots[name] = solution(mg, ctx, 64)
            finally:
                mg.mg_destroy(ctx)
            it[name].append(info["outer_iters"])
            if name == "trained":
                assert info["warm_start"] == 1, info
            elif name == "control":
                assert info["warm_start"] in (1, 3), info
        for name in ("trained", "control"):   # the same root, to the per-field accuracy
            for a, b in zip(roots[name], roots["cold"]):
                assert float((a - b).abs().max()) <= 1e-9 * float(b.abs().max()), name
        ref = torch.cat([roots["cold"][0].reshape(-1), roots["cold"][1].reshape(-1) / sc.s_W * sc.s_u])
        err["cold"].append(1.0)
        for name in ("trained", "control"):
            g = torch.cat([guesses[name][0].reshape(-1), guesses[name][1].reshape(-1) / sc.s_W * sc.s_u])
            err[name].append(float((g - ref).norm() / ref.norm()))
    print("outer iterations", {k: np.mean(v) for k, v in it.items()}, "start error", {k: np.mean(v) for k, v in err.items()})
    assert np.mean(err["trained"]) < 0.7      # the cold start (psi = 1, W = 0) is 1 by definition
    assert np.mean(err["trained"]) < np.mean(err["control"])
    assert np.mean(it["trained"]) <= np.mean(it["cold"])
    assert np.mean(it["trained"]) <= np.mean(it["control"])


def test_batch_serves_the_network_sizes_and_solves_the_rest_cold(mods, tmp_path):
    mg, WS = mods
    path = str(tmp_path / "net.bin")
    WS.save_weights(path, WS.Params(seed=2), WS.Scales(**SC), 64)
    ps = [fields.batch_instance(n, 5e-5, 4000 + i, device="cuda") for i, n in enumerate((64, 48, 128, 96))]
    cfgs = [mg.config_for(p, mg.MG_MIXED, tol=1e-10, max_outer=60) for p in ps]
    sols = {}
    for warm in (False, True):
        bt = mg.mg_batch_create(cfgs, torch.cuda.current_stream().cuda_stream)
        try:
            for b, p in enumerate(ps):
                mg.mg_batch_set_sources(bt, b, p["rho0"], p["rho2"], p["S"][0], p["S"][1], p["S"][2])
            if warm:
                mg.mg_batch_warmstart_load(bt, path)
            st, infos, _ = mg.mg_batch_solve(bt, len(ps))
            assert st == mg.MG_OK and all(i["converged"] for i in infos)
            states = [i["warm_start"] for i in infos]
            out = []
            for b, p in enumerate(ps):
                n = p["n"][0]
                u = torch.empty((n,) * 3, dtype=torch.float64, device="cuda")
                W = torch.empty((3,) + (n,) * 3, dtype=torch.float64, device="cuda")
                mg.mg_batch_get_solution(bt, b, u, W)
                out.append((u, W))
            sols[warm] = (out, states)
        finally:
            mg.mg_batch_destroy(bt)
    states = sols[True][1]
    assert states[1] == 0 and states[3] == 0          # 48^3, 96^3: not n_net * 2^k
    assert states[0] in (1, 2, 3) and states[2] in (1, 2, 3)
    assert sols[False][1] == [0, 0, 0, 0]
    for (uw, Ww), (uc, Wc) in zip(sols[True][0], sols[False][0]):
        assert float((uw - uc).abs().max()) <= 1e-8
        assert float((Ww - Wc).abs().max()) <= 1e-6 * float(Wc.abs().max()) + 1e-14


def test_bad_files_and_unsupported_grids(mods, tmp_path):
    mg, WS = mods
    good = str(tmp_path / "good.bin")
    WS.save_weights(good, WS.Params(seed=3), WS.Scales(**SC), 64)
    raw = open(good, "rb").read()
    cases = {"magic": b"XXXXXXXX" + raw[8:], "truncated": raw[:-4], "trailing": raw + b"\0",
             "size": raw[:8] + np.array([60], dtype="<i4").tobytes() + raw[12:]}
    p = fields.batch_instance(64, 5e-5, 1, device="cuda")
    ctx = context(mg, p)
    try:
        for name, data in cases.items():
            path = str(tmp_path / (name + ".bin"))
            with open(path, "wb") as f:
                f.write(data)
            with pytest.raises(mg.MGError) as e:
                mg.mg_warmstart_load(ctx, path)
            assert e.value.status == mg.MG_ERR_INVALID_ARG, name
        with pytest.raises(mg.MGError) as e:
            mg.mg_warmstart_load(ctx, str(tmp_path / "missing.bin"))
        assert e.value.status == mg.MG_ERR_INVALID_ARG
        with pytest.raises(mg.MGError) as e:
            mg.mg_warmstart_predict(ctx)               # nothing loaded
        assert e.value.status == mg.MG_ERR_STATE
        mg.mg_warmstart_load(ctx, good)
        mg.mg_warmstart_load(ctx, None)                # detach: solves cold again
        st, info = mg.mg_solve(ctx)
        assert st == mg.MG_OK and info["warm_start"] == 0
    finally:
        mg.mg_destroy(ctx)
    q = fields.batch_instance(96, 5e-5, 2, device="cuda")
    ctx = context(mg, q)
    try:
        with pytest.raises(mg.MGError) as e:
            mg.mg_warmstart_load(ctx, good)
        assert e.value.status == mg.MG_ERR_UNSUPPORTED
    finally:
        mg.mg_destroy(ctx)
    assert os.path.exists(good)
