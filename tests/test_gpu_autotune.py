"""The launch-parameter autotuner (mg_autotune): it picks a candidate that meets the
tolerance, the picked configuration solves the problem (checked with the oracle's own
residual), and a cached entry is returned without solving."""
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def sources(p):
    return [dev(a) for a in (p["rho0"], p["rho2"], *p["S"])]


@pytest.mark.parametrize("precision", ["MG_MIXED", "MG_FP64"])
def test_autotune_picks_a_converging_candidate(mg, tmp_path, precision):
    prec = getattr(mg, precision)
    p = fields.modes_periodic(n=48)
    base = mg.config_for(p, prec, tol=1e-10, max_outer=40)
    src = sources(p)
    sp = torch.cuda.current_stream().cuda_stream
    cache = tmp_path / "tune.txt"
    best, ms = mg.mg_autotune(base, *src, stream=sp, cache_path=str(cache))
    assert ms > 0
    assert best.inner_cycles in ((1, 2, 3) if prec == mg.MG_MIXED else (1, 2))
    assert best.nu_pre == best.nu_post and best.nu_pre in (1, 2, 3)
    assert best.omega in (1.0, 1.15, 1.3)
    # the tiled kernels' z chunking is tuned for the mixed form only (the FP64 form has no tiled level)
    assert best.tile_waves in ((1, 2, 3, 4) if prec == mg.MG_MIXED else (0,))
    assert best.tol == base.tol and list(best.n) == list(base.n)
    # the cache file holds this shape's entry
    lines = cache.read_text().split("\n")
    assert any(l.startswith("48 48 48 4 0 %d" % prec) for l in lines)

    # the picked configuration solves the problem: the oracle's residual of its solution
    ctx = mg.mg_create(best, sp)
    try:
        mg.mg_set_sources(ctx, *src)
        st, info = mg.mg_solve(ctx)
        assert st == mg.MG_OK and info["norms"].max() <= 1e-10
        u = torch.empty(p["rho0"].shape, dtype=torch.float64, device="cuda")
        W = torch.empty((3,) + p["rho0"].shape, dtype=torch.float64, device="cuda")
        mg.mg_get_solution(ctx, u, W)
    finally:
        mg.mg_destroy(ctx)
    g = O.make_grid(p["n"], p["lo"], p["hi"], p["order"], p["bc"], p["punctures"])
    res = O.residual(g, u.cpu().numpy(), W.cpu().numpy(), p["rho0"], p["rho2"], p["S"], O.K_INTEGRABILITY)
    assert res["norms"].max() <= 1.5e-10

    # a second call is a cache hit: same choice, same recorded time
    best2, ms2 = mg.mg_autotune(base, *src, stream=sp, cache_path=str(cache))
    assert (best2.inner_cycles, best2.nu_pre, best2.omega, best2.tile_waves) == \
        (best.inner_cycles, best.nu_pre, best.omega, best.tile_waves)
    assert ms2 == ms


def test_autotune_reads_cache_file(mg, tmp_path):
    """An entry in the cache file is returned as is, with no solve (its time is the file's)."""
    p = fields.modes_periodic(n=24)
    base = mg.config_for(p, mg.MG_MIXED, tol=1e-10, max_outer=40)
    cache = tmp_path / "tune.txt"
    # key (n, order, bc, precision, k_mode, nested), then inner, nu, threads, omega, tile_waves, ms
    cache.write_text("24 24 24 4 0 %d %d 0 3 1 128 1.15 3 1.5\n" % (mg.MG_MIXED, base.k_mode))
    best, ms = mg.mg_autotune(base, *sources(p), stream=torch.cuda.current_stream().cuda_stream,
                              cache_path=str(cache))
    assert (best.inner_cycles, best.nu_pre, best.nu_post, best.block_threads, best.tile_waves) == (3, 1, 1, 128, 3)
    assert best.omega == 1.15
    assert ms == 1.5


@pytest.mark.parametrize("case", ["periodic_o4_n64", "robin_o4_n48"])
def test_tile_waves_change_the_launch_shape_not_the_result(mg, case):
    """The z chunking of the tiled kernels (tile_waves) changes only which CTA computes which planes:
    every cell receives the same plane contributions in the same order, so the solve is bit for
    bit the same for any chunking."""
    p = fields.modes_periodic(n=64, a0=5e-5) if case.startswith("periodic") else fields.puncture_shell(n=48, half=24.0)
    sp = torch.cuda.current_stream().cuda_stream
    out = []
    for waves in (1, 3):
        cfg = mg.config_for(p, mg.MG_MIXED, tol=1e-10, max_outer=40, tile_waves=waves)
        ctx = mg.mg_create(cfg, sp)
        try:
            mg.mg_set_sources(ctx, *sources(p))
            st, info = mg.mg_solve(ctx)
            assert st == mg.MG_OK
            u = np.empty(p["rho0"].shape)
            W = np.empty((3,) + p["rho0"].shape)
            mg.mg_get_solution(ctx, u, W)
            out.append((u, W, np.asarray(info["history"])))
        finally:
            mg.mg_destroy(ctx)
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][2], out[1][2])
