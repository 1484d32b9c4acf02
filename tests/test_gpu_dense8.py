"""GPU against the dense brute-force root on 8^3 grids.

``oracle/dense_newton.py`` solves the discrete constraint system (eq:Ham,
eq:Mom in CTT form) by Newton's method with dense LAPACK solves: the exact root
of the discrete equations, reached without multigrid.  The CUDA library, called
through its C ABI, in FP64 and in the mixed FP32-inner / FP64-outer form, must
land on that root.  The bars follow from |error| <~ |J^-1| |residual| with
|J^-1| ~ (L/2pi)^2 (6.5 for L = 16, 26 for L = 32): the GPU is driven to
max(|H|, |M_i|) <= 1e-14, and psi must match to 1e-12 relative max-norm, K^2 to
1e-12 (periodic boxes).  Where W_i is small (3e-5 on the Robin boxes) the FP64
floor of the momentum residual binds: M_i cannot fall below ~1e-18 (rounding of
its stencil sums), which leaves |J^-1| * 1e-18 ~ 3e-17 in W_i, 1e-12 of its size;
W_i is held to 5e-12 relative.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.dense_newton import DenseSystem  # noqa: E402
from paper_2501_13046_gb300 import fields  # noqa: E402

CASES = {
    "sine_periodic_o2": lambda: fields.sine_periodic(n=8),
    "modes_periodic_o4": lambda: fields.modes_periodic(n=8, a0=5e-5),
    "puncture_shell_robin_o4": lambda: fields.puncture_shell(n=8, half=16.0),
    "bowen_york_binary_robin_o4": lambda: fields.bowen_york_binary(n=8, half=16.0),
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
def dense_roots():
    out = {}
    for name, make in CASES.items():
        p = make()
        ds = DenseSystem(p["n"], p["lo"], p["hi"], p["order"], p["bc"], p["punctures"], p["rho0"], p["rho2"],
                         p["S"], K2=p["K"] ** 2)
        out[name] = (p, ds, ds.solve())
    return out


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", list(CASES))
def test_gpu_root_is_the_dense_newton_root(mg, dense_roots, case, precision):
    p, ds, rd = dense_roots[case]
    assert rd["residual"] < 1e-13
    prec = mg.MG_FP64 if precision == "fp64" else mg.MG_MIXED
    cfg = mg.config_for(p, prec, tol=1e-14, max_outer=80)
    ctx = mg.mg_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
        mg.mg_set_sources(ctx, dev(p["rho0"]), dev(p["rho2"]), dev(p["S"][0]), dev(p["S"][1]), dev(p["S"][2]))
        st, info = mg.mg_solve(ctx)
        u = torch.empty(p["rho0"].shape, dtype=torch.float64, device="cuda")
        W = torch.empty((3,) + p["rho0"].shape, dtype=torch.float64, device="cuda")
        mg.mg_get_solution(ctx, u, W)
        u, W = u.cpu().numpy().reshape(-1), W.cpu().numpy().reshape(3, -1)
    finally:
        mg.mg_destroy(ctx)
    assert st == mg.MG_OK and info["converged"], info["history"][-3:]
    assert rel(ds.psibg + u, ds.psibg + rd["u"]) <= 1e-12
    for i in range(3):
        if np.abs(rd["W"][i]).max() > 1e-12:
            assert rel(W[i], rd["W"][i]) <= 5e-12, i
        else:
            assert np.abs(W[i]).max() <= 1e-13
    if p["bc"] == fields.PERIODIC:
        assert info["K2"] == pytest.approx(rd["K2"], rel=1e-12)
