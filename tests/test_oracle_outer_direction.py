"""Evidence for what limits the outer (defect-correction) iteration on periodic boxes (CPU, oracle
only).

The library's outer step linearises the rows separately (the psi row sees no W, the W rows no psi),
takes K^2 from the integrability condition at the current state and removes the mean of the psi
correction (the periodic gauge <u> = 0).  On the dense 8^3 system (oracle/dense_newton.py) that
step contracts the residual linearly, by ~0.03 per iteration, as the GPU solve does at 128^3.
Replacing the constant direction along which the mean is removed by the direction dF_psi/dK^2 =
-psi^5/12 (K^2 as a Newton unknown of the psi row, the gauge row unchanged) makes the same decoupled
step converge quadratically; adding the psi-W couplings changes nothing.  So the lagged K^2, not
the decoupling, sets the iteration count, and a correction of the psi row along L_psi^-1 psi^5 is
the change that would remove it."""
import numpy as np

from oracle.dense_newton import PERIODIC, DenseSystem
from paper_2501_13046_gb300 import fields


def outer_history(ds, k_direction, coupled, iters=8):
    N = ds.N
    u, W = np.zeros(N), np.zeros((3, N))
    hist = []
    for _ in range(iters):
        psi, At, aa = ds.parts(u, W)
        nonlin = aa / 8.0 * psi ** -7 + 2 * np.pi * (ds.rho0 * psi ** 5 + ds.rho2 * psi)
        K2 = 12.0 * nonlin.sum() / (psi ** 5).sum()          # integrability at the current state
        Fp, FW = ds.residual(u, W, K2)
        hist.append(max(np.abs(Fp).max(), np.abs(FW).max()))
        if hist[-1] < 1e-13:
            break
        J, dK = ds.jacobian(u, W, K2)
        if not coupled:
            J[:N, N:] = 0.0
            J[N:, :N] = 0.0
        A = np.zeros((4 * N + 4, 4 * N + 4))
        rhs = np.zeros(4 * N + 4)
        A[:4 * N, :4 * N] = J
        rhs[:N], rhs[N:4 * N] = -Fp, -FW.reshape(-1)
        for f in range(4):                                     # mean-zero corrections, one multiplier each
            A[4 * N + f, f * N:(f + 1) * N] = 1.0
            A[f * N:(f + 1) * N, 4 * N + f] = 1.0
        if k_direction:
            A[:N, 4 * N] = dK                                  # the psi row's multiplier along dF/dK^2
        d = np.linalg.solve(A, rhs)
        u, W = u + d[:N], W + d[N:4 * N].reshape(3, N)
    return np.array(hist)


def test_lagged_k2_not_the_decoupling_limits_the_outer_iteration():
    p = fields.modes_periodic(n=8)
    ds = DenseSystem(8, p["lo"], p["hi"], p["order"], PERIODIC, rho0=p["rho0"], rho2=p["rho2"], S=p["S"])
    const_dec = outer_history(ds, k_direction=False, coupled=False)
    const_cpl = outer_history(ds, k_direction=False, coupled=True)
    k_dec = outer_history(ds, k_direction=True, coupled=False)
    k_cpl = outer_history(ds, k_direction=True, coupled=True)
    # constant direction: linear contraction of a few percent per step, coupled or not
    ratios = const_dec[3:6] / const_dec[2:5]
    assert np.all((ratios > 1e-2) & (ratios < 0.1)), const_dec
    assert np.allclose(const_cpl[:6], const_dec[:6], rtol=1e-3), (const_cpl, const_dec)
    # K^2 direction: superlinear (each step squares the error's scale), at the FP64 floor within
    # five residual evaluations, coupled or not; the constant direction needs eight
    assert k_dec[2] < 0.1 * const_dec[2] and k_dec[3] < 1e-3 * const_dec[3], (k_dec, const_dec)
    assert k_dec[-1] < 1e-13 and len(k_dec) <= 5 and k_cpl[-1] < 1e-13 and len(k_cpl) <= 5, (k_dec, k_cpl)
    assert len(const_dec) >= 7


def test_psi_row_has_a_near_null_mode_close_to_the_constant():
    """Why more inner cycles do not help the library's step: with K^2 from the integrability
    condition the psi row's coefficient c averages to ~0, so L_psi = Lap + diag(c) has an eigenvalue
    ~30 times below the next one, with an almost constant eigenvector.  An inner solve of L_psi e = r
    amplifies that mode, and removing the plain mean afterwards leaves its non-constant part."""
    p = fields.modes_periodic(n=8)
    ds = DenseSystem(8, p["lo"], p["hi"], p["order"], PERIODIC, rho0=p["rho0"], rho2=p["rho2"], S=p["S"])
    root = ds.solve()
    J, _ = ds.jacobian(root["u"], root["W"], root["K2"])
    L = J[:ds.N, :ds.N]
    w, V = np.linalg.eig(L)
    order = np.argsort(np.abs(w))
    v0 = np.real(V[:, order[0]])
    v0 /= np.linalg.norm(v0)
    assert np.abs(w[order[0]]) * 20 < np.abs(w[order[1]]), w[order[:3]]
    assert abs(v0.sum()) / np.sqrt(ds.N) > 0.95
    c = np.diag(L) - np.diag(ds.Lap)
    assert abs(c.mean()) < 0.02 * np.abs(c).max()
