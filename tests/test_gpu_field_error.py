"""Per-field error of GPU solves against the FP64 oracle's root at benchmark sizes.

The oracle's root of the 64^3 and 128^3 periodic random-mode workloads (L = 32,
4th order; 128^3 is the benchmarked solve) is stored as sampled values by
tests/golden/make_oracle_roots.py, which calls only the oracle (4096 seeded
cells plus the extreme cells of every field, and each field's max-norm over
the whole grid).  The GPU solves through the C ABI in the benchmark's launch
configuration (mixed FP32-inner / FP64-outer, nested start) and its psi and
W_i are compared with the oracle's at those cells, relative to the oracle
field's max-norm.

Two stopping rules:

* max(|H|, |M_i|) <= 1e-10 alone.  The error is then bounded only by
  |J^-1| |residual|: with |J^-1| <~ (L/2pi)^2 ~ 26 and the scalings
  F_psi = -psi^5 H / 8, F_W = psi^6 M, |du| <~ 26 * 1.5 * 1e-10 / 8 and
  |dW| <~ 26 * 1.6 * 1e-10, i.e. ~5e-10 of psi but ~2e-4 of W (max |W| ~ 1.7e-5).
  The test asserts those bounds and records the measured errors.
* the same plus field_tol = 1e-10 (every field's last outer update at most 1e-10
  of its size): the fields then match the oracle to <= 1e-10 relative each.
* field_tol = 1e-10 with field_est = 1 (each field's remaining error estimated
  from the contraction of its last two updates): the same bar, in no more outer
  iterations (one fewer when the estimate stops the solve before an update
  below 1e-10 has confirmed it).
The oracle's own root is accurate to ~1e-11 relative (its H floor 2.7e-12 at
128^3, M floor 1e-17), ten times below the bar.
"""
import json
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2501_13046_gb300 import fields  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
FIELDS = ("psi", "Wx", "Wy", "Wz")


@pytest.fixture(scope="module")
def mg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_13046_gb300 import _build
    _build.build()
    from paper_2501_13046_gb300 import mg as m
    return m


def golden(name):
    with open(os.path.join(HERE, "golden", name + "_oracle_root.json")) as f:
        return json.load(f)


def field_errors(gold, u, W, psibg=None):
    """Max over the stored cells of |gpu - oracle| / max|oracle field| for psi, W_x, W_y, W_z."""
    cells = np.array(gold["cells"])
    bg = 1.0 if psibg is None else psibg.reshape(-1)[cells]
    out = {}
    gpu = {"psi": bg + u.reshape(-1)[cells], "Wx": W[0].reshape(-1)[cells], "Wy": W[1].reshape(-1)[cells],
           "Wz": W[2].reshape(-1)[cells]}
    ref = {"psi": bg + np.array(gold["u"]), "Wx": np.array(gold["Wx"]), "Wy": np.array(gold["Wy"]),
           "Wz": np.array(gold["Wz"])}
    for f in FIELDS:
        out[f] = float(np.abs(gpu[f] - ref[f]).max() / gold["max_abs"][f])
    return out


def solve(mg, p, precision, **over):
    cfg = mg.config_for(p, precision, tol=1e-10, max_outer=60, nested=1, **over)
    ctx = mg.mg_create(cfg, torch.cuda.current_stream().cuda_stream)
    try:
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
        mg.mg_set_sources(ctx, dev(p["rho0"]), dev(p["rho2"]), dev(p["S"][0]), dev(p["S"][1]), dev(p["S"][2]))
        st, info = mg.mg_solve(ctx)
        u = torch.empty(p["rho0"].shape, dtype=torch.float64, device="cuda")
        W = torch.empty((3,) + p["rho0"].shape, dtype=torch.float64, device="cuda")
        mg.mg_get_solution(ctx, u, W)
    finally:
        mg.mg_destroy(ctx)
    assert st == mg.MG_OK and info["converged"], info["history"][-3:]
    return info, u.cpu().numpy(), W.cpu().numpy()


@pytest.mark.parametrize("n", [64, 128])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_field_errors_against_the_oracle_root(mg, n, precision):
    gold = golden("modes_periodic_%d" % n)
    p = fields.modes_periodic(n=n)
    prec = mg.MG_MIXED if precision == "mixed" else mg.MG_FP64
    # residual tolerance alone: only the a-priori bounds hold
    info, u, W = solve(mg, p, prec)
    assert info["norms"].max() <= 1e-10
    err = field_errors(gold, u, W)
    assert err["psi"] <= 5e-10, err
    for f in FIELDS[1:]:
        assert err[f] <= 26 * 1.6e-10 / gold["max_abs"][f], (f, err)
    # with the per-field test every field matches the oracle to 1e-10 of its size
    info2, u2, W2 = solve(mg, p, prec, field_tol=1e-10)
    err2 = field_errors(gold, u2, W2)
    assert max(err2.values()) <= 1e-10, (err, err2, info2["rel_change"])
    assert info2["rel_change"].max() <= 1e-10
    assert info2["K2"] == pytest.approx(gold["K2"], rel=1e-10)
    # the estimated remaining error instead of the last update: the same accuracy, no more iterations
    info3, u3, W3 = solve(mg, p, prec, field_tol=1e-10, field_est=1)
    err3 = field_errors(gold, u3, W3)
    assert max(err3.values()) <= 1e-10, (err3, info3["rel_change"])
    assert info3["outer_iters"] <= info2["outer_iters"]
    print("n=%d %s: tol only %s (%d outer); + field_tol %s (%d outer); estimated %s (%d outer)"
          % (n, precision, err, info["outer_iters"], err2, info2["outer_iters"], err3, info3["outer_iters"]))


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_shell_256_field_errors_against_the_oracle_root(mg, precision):
    """The 256^3 puncture + scalar shell (Robin, K = 0, 4th order): psi = 1 + M/2r + u compared
    through psi (its max-norm 2.2 at the puncture), W_i (max 1e-4) as is."""
    gold = golden("puncture_shell_256")
    p = fields.puncture_shell(n=256)
    X, Y, Z = fields.cell_centres(p["n"], p["lo"], p["hi"])
    bg = 1.0 + 1.0 / (2.0 * np.sqrt(X * X + Y * Y + Z * Z))
    prec = mg.MG_MIXED if precision == "mixed" else mg.MG_FP64
    # residual tolerance alone: on this machine the a-priori bound is loose (|J^-1| ~ (128/pi)^2 / 3 ~ 550
    # and psi^6 up to ~110 next to the puncture), so those errors are recorded, not bounded
    info, u, W = solve(mg, p, prec)
    err = field_errors(gold, u, W, bg)
    assert max(err.values()) < 1e-3, err
    info2, u2, W2 = solve(mg, p, prec, field_tol=1e-10)
    err2 = field_errors(gold, u2, W2, bg)
    assert max(err2.values()) <= 1e-10, (err, err2, info2["rel_change"])
    print("shell 256 %s: tol only %s (%d outer); + field_tol %s (%d outer)"
          % (precision, err, info["outer_iters"], err2, info2["outer_iters"]))
