"""Batched solves of uneven grids against solo solves through the same C ABI, and against the
oracle's residual, in both pacings: device-paced (default: the whole solve one graph launch, a
WHILE node over per-instance IF nodes, converged instances dropping out on the device) and
host-paced (use_graph = 2: one graph per round, checked on the host, lock step)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2501_13046_gb300 import fields  # noqa: E402


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_13046_gb300 import _build
    _build.build()
    from paper_2501_13046_gb300 import mg as m
    return m


def problems():
    out = []
    for n, a0, seed in ((24, 3e-5, 7), (32, 6e-5, 8), (48, 4e-5, 9), (40, 8e-5, 10)):
        out.append(fields.batch_instance(n, a0, seed))
    return out


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def solo(mg, p, **over):
    ctx = mg.mg_create(mg.config_for(p, mg.MG_MIXED, **over), torch.cuda.current_stream().cuda_stream)
    try:
        mg.mg_set_sources(ctx, *[dev(a) for a in (p["rho0"], p["rho2"], *p["S"])])
        st, info = mg.mg_solve(ctx)
        u, W = np.empty(p["rho0"].shape), np.empty((3,) + p["rho0"].shape)
        mg.mg_get_solution(ctx, u, W)
    finally:
        mg.mg_destroy(ctx)
    return info, u, W


def batch(mg, ps, **over):
    cfgs = [mg.config_for(p, mg.MG_MIXED, **over) for p in ps]
    bt = mg.mg_batch_create(cfgs, torch.cuda.current_stream().cuda_stream)
    try:
        for b, p in enumerate(ps):
            mg.mg_batch_set_sources(bt, b, *[dev(a) for a in (p["rho0"], p["rho2"], *p["S"])])
        st, infos, total = mg.mg_batch_solve(bt, len(ps))
        sols = []
        for b, p in enumerate(ps):
            u, W = np.empty(p["rho0"].shape), np.empty((3,) + p["rho0"].shape)
            mg.mg_batch_get_solution(bt, b, u, W)
            sols.append((u, W))
    finally:
        mg.mg_batch_destroy(bt)
    return st, infos, total, sols


PACING = {"device": 1, "host": 2}


@pytest.mark.parametrize("pacing", list(PACING))
def test_batch_equals_solo_after_the_same_rounds(mg, pacing):
    ps = problems()
    st, infos, total, sols = batch(mg, ps, tol=0.0, max_outer=4, use_graph=PACING[pacing])
    assert st == mg.MG_ERR_NOT_CONVERGED and total > 0
    for p, (u, W), inf in zip(ps, sols, infos):
        info, u1, W1 = solo(mg, p, tol=0.0, max_outer=4)
        assert np.array_equal(u, u1) and np.array_equal(W, W1)
        assert np.array_equal(inf["history"], info["history"])


@pytest.mark.parametrize("pacing", list(PACING))
def test_batch_converges_and_reports_rounds(mg, pacing):
    ps = problems()
    st, infos, total, sols = batch(mg, ps, tol=1e-10, max_outer=40, use_graph=PACING[pacing])
    assert st == mg.MG_OK
    for p, (u, W), inf in zip(ps, sols, infos):
        info, u1, W1 = solo(mg, p, tol=1e-10, max_outer=40)
        assert inf["converged"] and inf["outer_iters"] == info["outer_iters"]
        assert np.array_equal(inf["history"], info["history"])
        if pacing == "device":   # a converged instance stops where the solo solve stops
            assert np.array_equal(u, u1) and np.array_equal(W, W1)
        assert 0 < inf["device_ms"] <= total
        g = O.make_grid(p["n"], p["lo"], p["hi"], p["order"], p["bc"])
        res = O.residual(g, u, W, p["rho0"], p["rho2"], p["S"], O.K_INTEGRABILITY)
        assert res["norms"].max() <= 1e-10


def test_device_paced_batch_repeats_and_per_field_stop(mg):
    """The cached graph serves a second solve from psi = 1; field_tol works on the device too."""
    ps = problems()
    cfgs = [mg.config_for(p, mg.MG_MIXED, tol=1e-10, max_outer=40, field_tol=1e-10) for p in ps]
    bt = mg.mg_batch_create(cfgs, torch.cuda.current_stream().cuda_stream)
    try:
        for b, p in enumerate(ps):
            mg.mg_batch_set_sources(bt, b, *[dev(a) for a in (p["rho0"], p["rho2"], *p["S"])])
        runs = []
        for _ in range(2):
            for b in range(len(ps)):
                mg.mg_batch_set_initial_guess(bt, b, None, None)
            st, infos, total = mg.mg_batch_solve(bt, len(ps))
            assert st == mg.MG_OK
            runs.append([(i["outer_iters"], i["history"].copy()) for i in infos])
            for i in infos:
                assert i["converged"] and 0 < i["rel_change"].max() <= 1e-10
    finally:
        mg.mg_batch_destroy(bt)
    for (i0, h0), (i1, h1) in zip(*runs):
        assert i0 == i1 and np.array_equal(h0, h1)
    # the contraction estimate of the per-field test on the device: every instance stops no later,
    # and at the same round as its solo solve with the same settings (the host loop's test)
    cfge = [mg.config_for(p, mg.MG_MIXED, tol=1e-10, max_outer=40, field_tol=1e-10, field_est=1) for p in ps]
    bt = mg.mg_batch_create(cfge, torch.cuda.current_stream().cuda_stream)
    try:
        for b, p in enumerate(ps):
            mg.mg_batch_set_sources(bt, b, *[dev(a) for a in (p["rho0"], p["rho2"], *p["S"])])
            mg.mg_batch_set_initial_guess(bt, b, None, None)
        st, infos, total = mg.mg_batch_solve(bt, len(ps))
        assert st == mg.MG_OK
    finally:
        mg.mg_batch_destroy(bt)
    for b, (i, (i0, _)) in enumerate(zip(infos, runs[0])):
        assert i["converged"] and i["outer_iters"] <= i0
        ctx = mg.mg_create(cfge[b], torch.cuda.current_stream().cuda_stream)
        try:
            mg.mg_set_sources(ctx, *[dev(a) for a in (ps[b]["rho0"], ps[b]["rho2"], *ps[b]["S"])])
            st1, solo = mg.mg_solve(ctx)
        finally:
            mg.mg_destroy(ctx)
        assert st1 == mg.MG_OK and solo["outer_iters"] == i["outer_iters"]


def test_batch_rejects_mixed_orders(mg):
    p2 = fields.sine_periodic(n=16)
    p4 = fields.modes_periodic(n=16)
    with pytest.raises(mg.MGError) as e:
        mg.mg_batch_create([mg.config_for(p2), mg.config_for(p4)])
    assert e.value.status == mg.MG_ERR_INVALID_ARG
