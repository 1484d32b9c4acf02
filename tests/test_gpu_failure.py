"""Failure detection without a GPU fault: every wait inside the pipelined (TMA-tiled) kernels is
bounded by mg_config.spin_limit.  With a limit of zero polls every bounded wait gives up at once,
as a wait on a flag that nothing sets would: the tiled kernel records the failure in the context's
error word, lets the loads already in flight complete (separately bounded) and returns; the solve
reports MG_ERR_TIMEOUT instead of hanging, and the device stays usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


def solve(mg, p, **over):
    cfg = mg.config_for(p, mg.MG_MIXED, tol=1e-10, max_outer=40, **over)
    ctx = mg.mg_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        mg.mg_set_sources(ctx, *[dev(a) for a in (p["rho0"], p["rho2"], *p["S"])])
        try:
            st, info = mg.mg_solve(ctx)
        except mg.MGError as e:
            st, info = e.status, None
    finally:
        mg.mg_destroy(ctx)
    return st, info


def test_exhausted_wait_limit_reports_timeout_and_device_recovers(mg):
    p = fields.modes_periodic(n=64)          # tiled levels 64^3, 32^3, 16^3
    statuses = [solve(mg, p, spin_limit=0)[0] for _ in range(2)]
    assert statuses == [mg.MG_ERR_TIMEOUT] * 2, statuses
    st, info = solve(mg, p)                  # default limit on the same device afterwards
    assert st == mg.MG_OK and info["norms"].max() <= 1e-10
