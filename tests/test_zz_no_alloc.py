"""The allocation-free constraint-norm entry point against the context path.

mg_residual_norms_noalloc serves callers that cannot allocate device memory: its
scratch is a static device array inside the library.  Its norms and K^2 must
match mg_residual_norms (which uses a context's workspace) on the same state,
on two calls in a row (the second call reuses the array the first one left).
This file is collected last so that a failure here comes after every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2501_13046_gb300 import fields  # noqa: E402

RTOL = 1e-11   # as for the other FP64 residual comparisons


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_13046_gb300 import _build
    _build.build()
    from paper_2501_13046_gb300 import mg as m
    return m


def state(p, seed):
    rng = np.random.default_rng(seed)
    shape = p["rho0"].shape
    u = 0.01 * rng.standard_normal(shape)
    if p["bc"] == fields.PERIODIC:
        u -= u.mean()
    W = 0.01 * rng.standard_normal((3,) + shape)
    return u, W


def context_norms(mg, p, u, W):
    cfg = mg.config_for(p, mg.MG_FP64)
    ctx = mg.mg_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        mg.mg_set_sources(ctx, *[np.ascontiguousarray(a) for a in (p["rho0"], p["rho2"], *p["S"])])
        mg.mg_set_initial_guess(ctx, np.ascontiguousarray(u), np.ascontiguousarray(W))
        norms = mg.mg_residual_norms(ctx)
    finally:
        mg.mg_destroy(ctx)
    return norms


@pytest.mark.parametrize("case", ["periodic_o4_n32", "robin_puncture_o4_n24", "periodic_o2_n20_x16_x12"])
def test_noalloc_norms_match_context_path_twice(mg, case):
    if case == "periodic_o4_n32":
        p = fields.modes_periodic(n=32, a0=1e-3)
    elif case == "robin_puncture_o4_n24":
        p = fields.puncture_shell(n=24, half=16.0)
    else:
        X, Y, Z = fields.cell_centres([20, 16, 12], 0.0, [20.0, 16.0, 12.0])
        phi = 0.05 * np.sin(2 * np.pi * X / 20.0)
        dphi = [0.05 * 2 * np.pi / 20.0 * np.cos(2 * np.pi * X / 20.0), 0 * X, 0 * X]
        Pi = 0.02 * np.cos(2 * np.pi * Y / 16.0)
        rho0, rho2, S = fields.scalar_sources(phi, dphi, Pi)
        p = dict(n=[20, 16, 12], lo=0.0, hi=[20.0, 16.0, 12.0], order=2, bc=fields.PERIODIC,
                 kmode=fields.K_INTEGRABILITY, K=0.0, punctures=[], rho0=rho0, rho2=rho2, S=S)
    cfg = mg.config_for(p, mg.MG_FP64)
    stream = torch.cuda.current_stream().cuda_stream
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    rho0, rho2, S = dev(p["rho0"]), dev(p["rho2"]), dev(p["S"])
    for seed in (1, 2):   # two calls in a row, on different states
        u, W = state(p, seed)
        want = context_norms(mg, p, u, W)
        got, K2 = mg.mg_residual_norms_noalloc(cfg, dev(u), dev(W), rho0, rho2, S, stream)
        np.testing.assert_allclose(got, want, rtol=RTOL)
        assert np.isfinite(K2) and K2 >= 0.0


def test_noalloc_without_rho2_matches_a_context_with_zero_rho2(mg):
    """rho2 = NULL means rho2 = 0 (no gradient energy): compare with a context given zeros."""
    p = fields.modes_periodic(n=32, a0=1e-3)
    p["rho2"] = np.zeros_like(p["rho2"])
    cfg = mg.config_for(p, mg.MG_FP64)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    for seed in (3, 4):
        u, W = state(p, seed)
        want = context_norms(mg, p, u, W)
        got, _ = mg.mg_residual_norms_noalloc(cfg, dev(u), dev(W), dev(p["rho0"]), None, dev(p["S"]),
                                              torch.cuda.current_stream().cuda_stream)
        np.testing.assert_allclose(got, want, rtol=RTOL)


@pytest.mark.parametrize("n", [(64, 64, 65), (1 << 21, 1 << 21, 1 << 22), (1 << 30, 4, 4), (3, 3, 1 << 29)])
def test_noalloc_rejects_grids_beyond_the_static_limit(mg, n):
    """Larger grids are rejected before any work, including sizes whose cell count would wrap
    around 64 bits (2^21 x 2^21 x 2^22 = 2^64)."""
    p = fields.uniform(n=16)
    cfg = mg.config_for(p, mg.MG_FP64)
    for a in range(3):
        cfg.n[a] = n[a]
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MGError) as e:
        mg.mg_residual_norms_noalloc(cfg, z, z, z, None, z)
    assert e.value.status == mg.MG_ERR_INVALID_ARG
    assert "262144" in str(e.value)
