"""Nested start (mg_config.nested): the half-size problem is solved first and its solution,
interpolated tricubically, starts the fine outer iteration.  Only the starting state changes, so
the converged result must be the same discrete root as the cold start's:

* 48^3 periodic (nested_min = 24: one nesting level): the solution matches the FP64 oracle's root
  to the same bar as the cold-start parity tests (relative 1e-10 per field, both sides at their
  FP64 floor);
* 128^3 periodic (the default nested_min, one level; and nested_min = 24, two levels) and 64^3
  Robin with a puncture: converged to 1e-10, the oracle's own residual of the result is below
  1.5e-10 at every cell (a property that holds at any size), and the nested result agrees with the
  cold-start result;
* an explicit initial guess replaces the nested start; half sizes below nested_min have none.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2501_13046_gb300 import fields  # noqa: E402

FLOOR = 1e-12


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


def solve(mg, p, precision, guess=None, **over):
    over.setdefault("tol", FLOOR)
    over.setdefault("max_outer", 80)
    cfg = mg.config_for(p, precision, **over)
    ctx = mg.mg_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        S = p["S"]
        mg.mg_set_sources(ctx, dev(p["rho0"]), dev(p["rho2"]), dev(S[0]), dev(S[1]), dev(S[2]))
        if guess is not None:
            mg.mg_set_initial_guess(ctx, dev(guess[0]), dev(guess[1]))
        else:
            mg.mg_set_initial_guess(ctx, None, None)
        st, info = mg.mg_solve(ctx)
        shape = p["rho0"].shape
        u = torch.empty(shape, dtype=torch.float64, device="cuda")
        W = torch.empty((3,) + shape, dtype=torch.float64, device="cuda")
        mg.mg_get_solution(ctx, u, W)
    finally:
        mg.mg_destroy(ctx)
    return st, info, u.cpu().numpy(), W.cpu().numpy()


def grid(p):
    return O.make_grid(p["n"], p["lo"], p["hi"], p["order"], p["bc"], p["punctures"])


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module")
def root48():
    p = fields.modes_periodic(n=48, a0=5e-5)
    r = O.solve(grid(p), p["rho0"], p["rho2"], p["S"], p["kmode"], K2=p["K"] ** 2, tol=0.0, max_outer=80)
    assert r["status"] in ("floor", "converged") and np.abs(r["u"]).max() < 0.5
    return p, r


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_nested_start_reaches_the_oracle_root(mg, root48, precision):
    p, ref = root48
    prec = mg.MG_FP64 if precision == "fp64" else mg.MG_MIXED
    st, info, u, W = solve(mg, p, prec, nested=1, nested_min=24)
    assert st == mg.MG_OK and info["converged"] and info["norms"].max() <= FLOOR
    assert info["nested_iters"] > 0
    assert rel(1.0 + u, 1.0 + ref["u"]) < 1e-10
    assert rel(W, ref["W"]) < 1e-10
    assert info["K2"] == pytest.approx(ref["K2"], rel=1e-10)
    res = O.residual(grid(p), u, W, p["rho0"], p["rho2"], p["S"], p["kmode"])
    assert res["norms"].max() < 10 * FLOOR


def _full_size_pair(mg, p, kmode, **nest_over):
    st0, cold, u0, W0 = solve(mg, p, mg.MG_MIXED, tol=1e-10, nested=0)
    st1, nest, u1, W1 = solve(mg, p, mg.MG_MIXED, tol=1e-10, nested=1, **nest_over)
    assert st0 == mg.MG_OK and st1 == mg.MG_OK
    assert cold["nested_iters"] == 0 and nest["nested_iters"] > 0
    assert nest["norms"].max() <= 1e-10
    res = O.residual(grid(p), u1, W1, p["rho0"], p["rho2"], p["S"], kmode, K2=p["K"] ** 2)
    assert res["norms"].max() <= 1.5e-10
    # both are within tol of the same root: they differ by (inverse Jacobian) x (residuals)
    assert np.abs(u1 - u0).max() <= 1e-7 and np.abs(W1 - W0).max() <= 1e-7
    return cold, nest


@pytest.mark.parametrize("nested_min", [0, 24])
def test_nested_start_full_size_periodic(mg, nested_min):
    """The benchmarked workload (128^3 periodic, 4th order, 16 modes): 64^3 first, and with
    nested_min = 24 also 32^3 before it."""
    p = fields.modes_periodic(n=128)
    cold, nest = _full_size_pair(mg, p, O.K_INTEGRABILITY, nested_min=nested_min)
    assert nest["outer_iters"] < cold["outer_iters"]
    assert nest["K2"] == pytest.approx(cold["K2"], rel=1e-9)


def test_nested_start_robin_puncture(mg):
    """Puncture M = 1 in [-32, 32]^3 at 64^3, Robin 1/r boundaries, scalar shell, K = 0."""
    p = fields.puncture_shell(n=64, half=32.0)
    cold, nest = _full_size_pair(mg, p, O.K_FIXED, nested_min=32)
    assert nest["outer_iters"] <= cold["outer_iters"]


def test_guess_and_size_rules(mg):
    """A given initial guess replaces the nested start; a half size below nested_min has none."""
    p = fields.modes_periodic(n=48, a0=5e-5)
    st, info, u, W = solve(mg, p, mg.MG_MIXED, tol=1e-10, nested=1, nested_min=24)
    assert st == mg.MG_OK and info["nested_iters"] > 0
    st, info2, _, _ = solve(mg, p, mg.MG_MIXED, guess=(u, W), tol=1e-10, nested=1, nested_min=24)
    assert st == mg.MG_OK and info2["nested_iters"] == 0 and info2["outer_iters"] <= 1
    st, info3, _, _ = solve(mg, p, mg.MG_MIXED, tol=1e-10, nested=1)   # default nested_min 64
    assert st == mg.MG_OK and info3["nested_iters"] == 0
