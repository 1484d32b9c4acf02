"""Bowen-York punctures (two boosted, spinning black holes with a scalar shell) through the C ABI
against the FP64 oracle: the converged solution matches the oracle's root at 32^3 (both orders,
FP64 and mixed; both sides at their FP64 floor; psi to relative 1e-10 as in the other parity
tests, W, whose size is ~2e-5 here, to the absolute bound |J^-1| (r_gpu + r_oracle)), and at 128^3
the oracle's own residual of the GPU solution is below 1.5e-10 at every cell (a property that
holds at any size)."""
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


def solve(mg, p, precision, **over):
    over.setdefault("tol", FLOOR)
    over.setdefault("max_outer", 80)
    cfg = mg.config_for(p, precision, **over)
    ctx = mg.mg_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        S = p["S"]
        mg.mg_set_sources(ctx, dev(p["rho0"]), dev(p["rho2"]), dev(S[0]), dev(S[1]), dev(S[2]))
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


def psi_background(p):
    X, Y, Z = fields.cell_centres(p["n"], p["lo"], p["hi"])
    bg = np.ones_like(X)
    for pun in p["punctures"]:
        m, x = pun[0], pun[1]
        bg += m / (2 * np.sqrt((X - x[0]) ** 2 + (Y - x[1]) ** 2 + (Z - x[2]) ** 2))
    return bg


@pytest.fixture(scope="module")
def roots():
    out = {}
    for order in (2, 4):
        p = fields.bowen_york_binary(n=32, order=order)
        r = O.solve(grid(p), p["rho0"], p["rho2"], p["S"], p["kmode"], K2=0.0, tol=0.0, max_outer=80)
        assert r["status"] in ("floor", "converged") and np.abs(r["u"]).max() < 0.5
        out[order] = (p, r)
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("order", [2, 4])
def test_binary_matches_the_oracle_root(mg, roots, order, precision):
    p, ref = roots[order]
    prec = mg.MG_FP64 if precision == "fp64" else mg.MG_MIXED
    st, info, u, W = solve(mg, p, prec)
    assert st == mg.MG_OK and info["converged"] and info["norms"].max() <= FLOOR
    bg = psi_background(p)
    assert rel(bg + u, bg + ref["u"]) < 1e-10
    assert np.abs(ref["W"]).max() > 1e-8          # the shell's momentum density drives W
    # W is ~2e-5 here, so its bar is absolute: |dW| <~ |J^-1| (r_gpu + r_oracle) <= 30 x 2e-12
    assert np.abs(W - ref["W"]).max() <= 30 * 2 * FLOOR
    res = O.residual(grid(p), u, W, p["rho0"], p["rho2"], p["S"], O.K_FIXED)
    assert res["norms"].max() < 10 * FLOOR


def test_curvature_changes_the_solution(mg, roots):
    """The same binary without momenta and spins has a different root (the curvature reaches the
    solve): the bare solution's residual under the Bowen-York operator is far above the floor."""
    p, ref = roots[4]
    bare = dict(p, punctures=[(pun[0], pun[1]) for pun in p["punctures"]])
    st, info, u, W = solve(mg, bare, mg.MG_FP64)
    assert st == mg.MG_OK
    res = O.residual(grid(p), u, W, p["rho0"], p["rho2"], p["S"], O.K_FIXED)
    assert res["norms"].max() > 1e-6


def test_full_size_binary_with_nested_start(mg):
    """128^3 in [-16, 16]^3 (h = 0.25), 4th order, mixed precision, nested start: converges to
    1e-10 and the oracle's residual of the GPU solution is below 1.5e-10 at every cell."""
    p = fields.bowen_york_binary(n=128)
    st, info, u, W = solve(mg, p, mg.MG_MIXED, tol=1e-10, nested=1)
    assert st == mg.MG_OK and info["norms"].max() <= 1e-10 and info["nested_iters"] > 0
    res = O.residual(grid(p), u, W, p["rho0"], p["rho2"], p["S"], O.K_FIXED)
    assert res["norms"].max() <= 1.5e-10


def test_allocation_free_norms_reject_bowen_york(mg):
    p = fields.bowen_york_binary(n=32)
    cfg = mg.config_for(p, mg.MG_MIXED)
    z = torch.zeros(32 ** 3, dtype=torch.float64, device="cuda")
    z3 = torch.zeros(3 * 32 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(mg.MGError) as e:
        mg.mg_residual_norms_noalloc(cfg, z, z3, z, None, z3)
    assert e.value.status == mg.MG_ERR_UNSUPPORTED
