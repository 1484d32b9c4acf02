"""k2_newton (periodic boxes, K from integrability): the psi correction's mean is removed along
z = L_psi^-1 dF_psi/dK^2 instead of the constant.  The solve must reach the same discrete root: its
fields match the FP64 oracle's stored 64^3 root to 1e-10 of their size, as the default solve does."""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2501_13046_gb300 import fields  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_13046_gb300 import _build
    _build.build()
    from paper_2501_13046_gb300 import mg as m
    return m


def field_errors(gold, u, W):
    cells = np.array(gold["cells"])
    gpu = {"psi": 1.0 + u.reshape(-1)[cells], "Wx": W[0].reshape(-1)[cells], "Wy": W[1].reshape(-1)[cells],
           "Wz": W[2].reshape(-1)[cells]}
    ref = {"psi": 1.0 + np.array(gold["u"]), "Wx": np.array(gold["Wx"]), "Wy": np.array(gold["Wy"]),
           "Wz": np.array(gold["Wz"])}
    return {f: float(np.abs(gpu[f] - ref[f]).max() / gold["max_abs"][f]) for f in gpu}


@pytest.mark.parametrize("inner", [2, 4])
def test_k2_newton_reaches_the_oracle_root(mg, inner):
    with open(os.path.join(HERE, "golden", "modes_periodic_64_oracle_root.json")) as f:
        gold = json.load(f)
    p = fields.modes_periodic(n=64)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    out = {}
    for k2 in (0, 1):
        cfg = mg.config_for(p, mg.MG_MIXED, tol=1e-10, max_outer=60, nested=1, field_tol=1e-10, k2_newton=k2,
                            inner_cycles=inner, nu_pre=1, nu_post=1, omega=1.3)
        ctx = mg.mg_create(cfg, torch.cuda.current_stream().cuda_stream)
        try:
            mg.mg_set_sources(ctx, *[dev(a) for a in (p["rho0"], p["rho2"], *p["S"])])
            st, info = mg.mg_solve(ctx)
            u = np.empty(p["rho0"].shape)
            W = np.empty((3,) + p["rho0"].shape)
            mg.mg_get_solution(ctx, u, W)
        finally:
            mg.mg_destroy(ctx)
        assert st == mg.MG_OK and info["converged"], (k2, info["history"][-3:])
        out[k2] = (info["outer_iters"], field_errors(gold, u, W), info["K2"])
    for k2 in (0, 1):
        assert max(out[k2][1].values()) <= 1e-10, out
        assert out[k2][2] == pytest.approx(gold["K2"], rel=1e-10)
    print("inner %d: outer iterations default %d, k2_newton %d" % (inner, out[0][0], out[1][0]))
