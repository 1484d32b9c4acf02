"""Reflection-symmetry planes (mg_config.reflect) through the C ABI: an octant problem (three
planes, Robin upper faces) matches the FP64 oracle's octant root, and equals the octant of the
same symmetric problem solved on the full box with Robin faces only (the discrete equations
restricted to the octant are the same), including with the nested start."""
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


def octant(a):
    n = a.shape[-1]
    return a[..., n // 2:, n // 2:, n // 2:]


@pytest.fixture(scope="module")
def roots():
    out = {}
    for order in (2, 4):
        p = fields.octant(fields.puncture_shell(n=48, half=12.0, order=order))
        g = O.make_grid(p["n"], p["lo"], p["hi"], order, O.ROBIN, p["punctures"], reflect=7)
        r = O.solve(g, p["rho0"], p["rho2"], p["S"], O.K_FIXED, tol=0.0, max_outer=80)
        assert r["status"] in ("floor", "converged") and np.abs(r["u"]).max() < 0.5
        out[order] = (p, g, r)
    return out


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("order", [2, 4])
def test_octant_matches_the_oracle_root(mg, roots, order, precision):
    p, g, ref = roots[order]
    st, info, u, W = solve(mg, p, mg.MG_FP64 if precision == "fp64" else mg.MG_MIXED)
    assert st == mg.MG_OK and info["norms"].max() <= FLOOR
    X, Y, Z = fields.cell_centres(p["n"], p["lo"], p["hi"])
    psi_bg = 1 + 0.5 / np.sqrt(X * X + Y * Y + Z * Z)     # M = 1 at the origin
    assert np.abs(u - ref["u"]).max() <= 1e-10 * np.abs(psi_bg + ref["u"]).max()
    assert np.abs(ref["W"]).max() > 1e-9
    assert np.abs(W - ref["W"]).max() <= 30 * 2 * FLOOR   # |J^-1| (r_gpu + r_oracle)
    res = O.residual(g, u, W, p["rho0"], p["rho2"], p["S"], O.K_FIXED)
    assert res["norms"].max() < 10 * FLOOR


@pytest.mark.parametrize("nested", [0, 1])
def test_octant_equals_the_full_box(mg, nested):
    """128^3 full box [-16, 16]^3 against its octant at 64^3 (TMA-tiled levels, fused bottom of
    the cycle; with the nested start the octant first solves 32^3), mixed precision, both to the
    FP64 floor."""
    full = fields.puncture_shell(n=128, half=16.0)
    st, _, uf, Wf = solve(mg, full, mg.MG_MIXED)
    assert st == mg.MG_OK
    p = fields.octant(full)
    st, info, u, W = solve(mg, p, mg.MG_MIXED, nested=nested, nested_min=16)
    assert st == mg.MG_OK and (info["nested_iters"] > 0) == bool(nested)
    uo, Wo = octant(uf), octant(Wf)
    assert np.abs(u - uo).max() <= 1e-10 * np.abs(1 + uo).max()
    assert np.abs(W - Wo).max() <= 30 * 2 * FLOOR
