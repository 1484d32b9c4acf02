"""Dense brute-force pin of the oracle on 8^3 grids (CPU).

``oracle/dense_newton.py`` restates the discrete constraint system (eq:Ham,
eq:Mom in CTT form) independently of ``oracle/ctt_oracle.c``: every stencil is a
dense matrix built from its weights and the boundary rule, the Jacobian is
analytic, and Newton's method with LAPACK solves reaches the exact discrete root
in a handful of quadratically converging steps.  These tests check

* that the two restatements give the same residual at arbitrary states (a
  dropped term, a wrong sign, index or weight in either one fails here);
* the analytic Jacobian against central differences of the residual;
* that the oracle's multigrid solve reaches the dense Newton root to 1e-12
  relative per field, and K^2 to 1e-12 (periodic boxes), on 2nd- and
  4th-order periodic boxes and on Robin boxes with a bare puncture and with
  two Bowen-York punctures.
"""
import numpy as np
import pytest

from oracle import oracle as O
from oracle.dense_newton import DenseSystem
from paper_2501_13046_gb300 import fields

CASES = {
    "sine_periodic_o2": lambda: fields.sine_periodic(n=8),
    "modes_periodic_o4": lambda: fields.modes_periodic(n=8, a0=5e-5),
    "puncture_shell_robin_o4": lambda: fields.puncture_shell(n=8, half=16.0),
    "bowen_york_binary_robin_o4": lambda: fields.bowen_york_binary(n=8, half=16.0),
}


def dense_system(p):
    return DenseSystem(p["n"], p["lo"], p["hi"], p["order"], p["bc"], p["punctures"], p["rho0"], p["rho2"], p["S"],
                       K2=p["K"] ** 2)


def oracle_grid(p):
    return O.make_grid(p["n"], p["lo"], p["hi"], p["order"], p["bc"], p["punctures"])


@pytest.fixture(scope="module")
def roots():
    """Dense Newton root and oracle root of every case (computed once)."""
    out = {}
    for name, make in CASES.items():
        p = make()
        ds = dense_system(p)
        rd = ds.solve()
        ro = O.solve(oracle_grid(p), p["rho0"], p["rho2"], p["S"], p["kmode"], K2=p["K"] ** 2, tol=0.0,
                     max_outer=80)
        out[name] = (p, ds, rd, ro)
    return out


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("case", list(CASES))
def test_residual_matches_oracle_at_arbitrary_state(case):
    p = CASES[case]()
    ds = dense_system(p)
    rng = np.random.Generator(np.random.PCG64(7))
    N = ds.N
    u = 0.05 * rng.standard_normal(N)
    W = 0.02 * rng.standard_normal((3, N))
    r = O.residual(oracle_grid(p), u, W, p["rho0"], p["rho2"], p["S"], p["kmode"], K2=p["K"] ** 2)
    K2 = r["K2"]
    Fp, FW = ds.residual(u, W, K2)
    # random states make every term of the same size as the stencil sums, so compare to that scale
    scale_p = np.abs(ds.Lap @ u).max()
    scale_w = np.abs(ds.Lap @ W[0]).max()
    assert np.abs(Fp - r["Fpsi"].reshape(-1)).max() <= 1e-12 * scale_p
    assert np.abs(FW - r["FW"].reshape(3, -1)).max() <= 1e-12 * scale_w
    if p["bc"] == fields.PERIODIC:
        # K^2 of the oracle is the one that makes the cell sum of F_psi vanish
        assert abs(Fp.sum()) <= 1e-12 * np.abs(Fp).sum()


@pytest.mark.parametrize("case", ["modes_periodic_o4", "bowen_york_binary_robin_o4"])
def test_jacobian_matches_central_differences(case):
    p = CASES[case]()
    ds = dense_system(p)
    rng = np.random.Generator(np.random.PCG64(11))
    N = ds.N
    u = 0.05 * rng.standard_normal(N)
    W = 0.02 * rng.standard_normal((3, N))
    K2 = 0.3
    J, dK = ds.jacobian(u, W, K2)
    x = np.concatenate([u, W.reshape(-1)])
    # columns at corners, faces and interior cells of every field
    cols = sorted(set([0, N - 1, 7, 63, 300] + [f * N + c for f in (1, 2, 3) for c in (0, 9, 200, N - 1)] +
                      list(rng.choice(4 * N, size=24, replace=False))))
    eps = 1e-6
    for c in cols:
        xp, xm = x.copy(), x.copy()
        xp[c] += eps
        xm[c] -= eps
        Fp1, FW1 = ds.residual(xp[:N], xp[N:].reshape(3, N), K2)
        Fp0, FW0 = ds.residual(xm[:N], xm[N:].reshape(3, N), K2)
        fd = (np.concatenate([Fp1, FW1.reshape(-1)]) - np.concatenate([Fp0, FW0.reshape(-1)])) / (2 * eps)
        assert np.abs(fd - J[:, c]).max() <= 1e-6 * max(1.0, np.abs(J[:, c]).max()), c
    Fa, _ = ds.residual(u, W, K2 + eps)
    Fb, _ = ds.residual(u, W, K2 - eps)
    assert np.abs((Fa - Fb) / (2 * eps) - dK).max() <= 1e-8 * np.abs(dK).max()


@pytest.mark.parametrize("case", list(CASES))
def test_oracle_root_is_the_dense_newton_root(roots, case):
    p, ds, rd, ro = roots[case]
    assert rd["residual"] < 1e-13
    assert ro["status"] in ("floor", "converged")
    # Newton converged quadratically: the last steps square the residual's size
    h = rd["history"]
    assert any(h[i + 1] < 10 * h[i] ** 1.8 or h[i + 1] < 1e-13 for i in range(len(h) - 1) if h[i] < 1e-3)
    psi_d = ds.psibg + rd["u"]
    psi_o = ds.psibg + ro["u"].reshape(-1)
    assert rel(psi_o, psi_d) <= 1e-12
    Wo = ro["W"].reshape(3, -1)
    for i in range(3):
        if np.abs(rd["W"][i]).max() > 1e-12:
            assert rel(Wo[i], rd["W"][i]) <= 1e-12, i
        else:
            assert np.abs(Wo[i]).max() <= 1e-14
    if p["bc"] == fields.PERIODIC:
        assert ro["K2"] == pytest.approx(rd["K2"], rel=1e-12)
        assert np.abs(rd["multipliers"]).max() < 1e-15   # the momentum source mean is removed exactly
