"""Checkpoint / resume through the C ABI: the file holds the documented header and the state
bit for bit, a context loaded from it resumes at the converged state (no outer iteration, no
nested start), and files of another grid, truncated files or missing files are rejected."""
import struct

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


def context(mg, p, **over):
    cfg = mg.config_for(p, mg.MG_MIXED, tol=1e-10, max_outer=60, **over)
    ctx = mg.mg_create(cfg, torch.cuda.current_stream().cuda_stream)
    S = p["S"]
    mg.mg_set_sources(ctx, p["rho0"], p["rho2"], S[0], S[1], S[2])
    return ctx


def solution(mg, ctx, shape):
    u, W = np.empty(shape), np.empty((3,) + shape)
    K = mg.mg_get_solution(ctx, u, W)
    return u, W, K


def test_save_and_resume(mg, tmp_path):
    p = fields.modes_periodic(n=48, a0=5e-5)
    shape = p["rho0"].shape
    N = int(np.prod(shape))
    path = tmp_path / "state.ckpt"
    ctx = context(mg, p, nested=1, nested_min=24)
    try:
        st, info = mg.mg_solve(ctx)
        assert st == mg.MG_OK and info["nested_iters"] > 0
        u0, W0, K0 = solution(mg, ctx, shape)
        mg.mg_checkpoint_save(ctx, str(path))
    finally:
        mg.mg_destroy(ctx)
    raw = path.read_bytes()
    assert len(raw) == 8 + 6 * 4 + 8 + 4 * N * 8
    assert raw[:8] == b"CTTMGCK1"
    n0, n1, n2, order, bc, zero = struct.unpack("<6i", raw[8:32])
    assert (n0, n1, n2, order, bc, zero) == (48, 48, 48, 4, mg.MG_BC_PERIODIC, 0)
    (K2,) = struct.unpack("<d", raw[32:40])
    assert K2 == pytest.approx(K0 * K0, rel=1e-14)
    data = np.frombuffer(raw[40:], dtype="<f8")
    assert np.array_equal(data[:N], u0.reshape(-1)) and np.array_equal(data[N:], W0.reshape(-1))
    # resume in a fresh context: the loaded state is the start, already converged
    ctx = context(mg, p, nested=1, nested_min=24)
    try:
        mg.mg_checkpoint_load(ctx, str(path))
        st, info = mg.mg_solve(ctx)
        assert st == mg.MG_OK and info["outer_iters"] == 0 and info["nested_iters"] == 0
        u1, W1, _ = solution(mg, ctx, shape)
        np.testing.assert_allclose(u1, u0, rtol=0, atol=1e-15)
        np.testing.assert_allclose(W1, W0, rtol=0, atol=1e-15)
    finally:
        mg.mg_destroy(ctx)


def test_bad_files_are_rejected(mg, tmp_path):
    p = fields.sine_periodic(n=32)
    q = fields.sine_periodic(n=16)
    good, short = tmp_path / "good.ckpt", tmp_path / "short.ckpt"
    ctx = context(mg, p)
    try:
        mg.mg_solve(ctx)
        mg.mg_checkpoint_save(ctx, str(good))
        short.write_bytes(good.read_bytes()[:-8])
        for bad in (short, tmp_path / "missing.ckpt"):
            with pytest.raises(mg.MGError) as e:
                mg.mg_checkpoint_load(ctx, str(bad))
            assert e.value.status == mg.MG_ERR_INVALID_ARG
    finally:
        mg.mg_destroy(ctx)
    other = context(mg, q)
    try:
        with pytest.raises(mg.MGError) as e:
            mg.mg_checkpoint_load(other, str(good))
        assert e.value.status == mg.MG_ERR_INVALID_ARG
    finally:
        mg.mg_destroy(other)
