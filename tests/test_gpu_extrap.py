"""Extrapolating faces of Robin boxes on the GPU against the oracle (through the C ABI).

The boundary rule (the paper's extrapolating boundaries, read as linear extrapolation along
the face normal; mg_config.extrap) enters every stencil evaluation next to such a face: the
FP64 outer residual, the FP32/FP64 inner smoothers (TMA-tiled halo and global-memory kernels),
the prolongation, the dense coarsest-level inverses and the nested start's interpolation.  The
GPU must reach the oracle's root (which is pinned against an independent dense restatement in
tests/test_oracle_extrap.py): psi to 1e-10 relative max-norm and W_i to the bound its small size
allows, in FP64 and mixed precision, with the tiled and the global-memory kernels.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import oracle as O  # noqa: E402
from paper_2501_13046_gb300 import fields  # noqa: E402

CASES = {
    "shell_x_faces_o4_n32": (lambda: fields.puncture_shell(n=32, half=16.0), 0b000011),
    "shell_upper_z_o4_n24": (lambda: fields.puncture_shell(n=24, half=16.0), 0b100000),
    "binary_y_faces_o2_n32": (lambda: fields.bowen_york_binary(n=32, half=16.0, order=2), 0b001100),
}


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_13046_gb300 import _build
    _build.build()
    from paper_2501_13046_gb300 import mg as m
    return m


@pytest.fixture(scope="module")
def oracle_roots():
    out = {}
    for name, (make, extrap) in CASES.items():
        p = make()
        g = O.make_grid(p["n"], p["lo"], p["hi"], p["order"], p["bc"], p["punctures"], extrap=extrap)
        r = O.solve(g, p["rho0"], p["rho2"], p["S"], p["kmode"], K2=p["K"] ** 2, tol=0.0, max_outer=120)
        assert r["status"] in ("floor", "converged"), r["status"]
        out[name] = (p, extrap, g, r)
    return out


def psi_background(p):
    X, Y, Z = fields.cell_centres(p["n"], p["lo"], p["hi"])
    bg = np.ones_like(X)
    for pun in p["punctures"]:
        bg += pun[0] / (2 * np.sqrt((X - pun[1][0]) ** 2 + (Y - pun[1][1]) ** 2 + (Z - pun[1][2]) ** 2))
    return bg


def gpu_solve(mg, p, extrap, precision, **over):
    cfg = mg.config_for(p, precision, tol=1e-12, max_outer=120, **over)
    cfg.extrap = extrap
    ctx = mg.mg_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
        mg.mg_set_sources(ctx, dev(p["rho0"]), dev(p["rho2"]), dev(p["S"][0]), dev(p["S"][1]), dev(p["S"][2]))
        st, info = mg.mg_solve(ctx)
        u, W = np.empty(p["rho0"].shape), np.empty((3,) + p["rho0"].shape)
        mg.mg_get_solution(ctx, u, W)
    finally:
        mg.mg_destroy(ctx)
    return st, info, u, W


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("kernels", ["tiled", "global"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", list(CASES))
def test_extrapolating_faces_reach_the_oracle_root(mg, oracle_roots, case, precision, kernels):
    p, extrap, g, ref = oracle_roots[case]
    prec = mg.MG_FP64 if precision == "fp64" else mg.MG_MIXED
    st, info, u, W = gpu_solve(mg, p, extrap, prec, smoother=0 if kernels == "tiled" else 1)
    assert st == mg.MG_OK and info["converged"], info["history"][-3:]
    bg = psi_background(p)
    assert rel(bg + u, bg + ref["u"]) <= 1e-10
    for i in range(3):
        # |dW| <~ |J^-1| max|M| with |J^-1| ~ (L/2pi)^2 ~ 26 and both sides at <= 1e-12
        assert np.abs(W[i] - ref["W"][i]).max() <= 1e-10 * np.abs(ref["W"][i]).max() + 6e-11, i
    res = O.residual(g, u, W, p["rho0"], p["rho2"], p["S"], p["kmode"], K2=p["K"] ** 2)
    assert res["norms"].max() <= 1e-11


def test_nested_start_with_extrapolating_faces(mg):
    """The nested start's interpolation uses the same rule; it changes the start, not the root."""
    p = fields.puncture_shell(n=64, half=16.0)
    st0, i0, u0, W0 = gpu_solve(mg, p, 0b000011, mg.MG_MIXED, nested=0)
    st1, i1, u1, W1 = gpu_solve(mg, p, 0b000011, mg.MG_MIXED, nested=1, nested_min=32)
    assert st0 == st1 == mg.MG_OK and i1["nested_iters"] > 0
    bg = psi_background(p)
    assert rel(bg + u1, bg + u0) <= 1e-10
    g = O.make_grid(p["n"], p["lo"], p["hi"], p["order"], p["bc"], p["punctures"], extrap=0b000011)
    res = O.residual(g, u1, W1, p["rho0"], p["rho2"], p["S"], p["kmode"])
    assert res["norms"].max() <= 1e-11
