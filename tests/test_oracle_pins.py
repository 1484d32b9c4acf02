"""Pins of the FP64 CPU oracle against facts it does not compute itself.

Each test checks the oracle (oracle/ctt_oracle.c) against a closed form, an
invariant, a textbook exact solution or the paper's own definition of the
constraints (eq:Ham, eq:Mom), chosen so that a dropped term, a wrong
coefficient or sign, a wrong index or a transposed operand fails one of them.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_13046_gb300 import fields as Fd

PI = np.pi


def centres(g):
    lo = [g.lo[a] for a in range(3)]
    hi = [g.lo[a] + g.n[a] * g.h[a] for a in range(3)]
    return Fd.cell_centres([g.n[0], g.n[1], g.n[2]], lo, hi)


# ---------------------------------------------------------------- stencils


def d1_symbol(order, th, h):
    return np.sin(th) / h if order == 2 else (8 * np.sin(th) - np.sin(2 * th)) / (6 * h)


def d2_symbol(order, th, h):
    if order == 2:
        return 4 * np.sin(th / 2) ** 2 / h ** 2
    return (30 - 32 * np.cos(th) + 2 * np.cos(2 * th)) / (12 * h ** 2)


@pytest.mark.parametrize("order", [2, 4])
def test_stencil_fourier_symbols(order):
    """D_a, D_aa, D_a D_b and Lap on a Fourier mode equal their closed-form symbols.

    Non-cubic grid with a different spacing per axis, so a swapped axis or
    spacing fails; every cell is checked, so the periodic wrap is pinned too.
    """
    n, h = (12, 10, 8), (0.5, 0.7, 0.9)
    g = O.make_grid(n, 0.0, [n[a] * h[a] for a in range(3)], order, O.PERIODIC)
    X, Y, Z = centres(g)
    m = (1, 2, 3)
    k = [2 * PI * m[a] / (n[a] * h[a]) for a in range(3)]
    ph = k[0] * X + k[1] * Y + k[2] * Z + 0.3
    f = np.sin(ph)
    th = [k[a] * h[a] for a in range(3)]
    sig = [d1_symbol(order, th[a], h[a]) for a in range(3)]
    lam = [d2_symbol(order, th[a], h[a]) for a in range(3)]
    for a in range(3):
        np.testing.assert_allclose(O.d1(g, a, f).reshape(f.shape), sig[a] * np.cos(ph), atol=1e-12)
        np.testing.assert_allclose(O.d2(g, a, f).reshape(f.shape), -lam[a] * f, atol=1e-11)
        for b in range(3):
            if a != b:
                np.testing.assert_allclose(O.dmix(g, a, b, f).reshape(f.shape), -sig[a] * sig[b] * f, atol=1e-11)
    np.testing.assert_allclose(O.lap(g, f).reshape(f.shape), -sum(lam) * f, atol=1e-11)


@pytest.mark.parametrize("order", [2, 4])
def test_derivatives_exact_on_polynomials(order):
    """Central differences are exact on quadratics (4th order: quartics) away from the boundary."""
    g = O.make_grid((10, 9, 11), (-3.0, -2.0, -4.0), (2.0, 2.5, 1.5), order, O.ROBIN)
    X, Y, Z = centres(g)
    f = 0.3 * X * X - 0.7 * X * Y + 1.1 * Z * Z + 0.2 * Y * Z - 0.5 * X + 0.9
    inner = (slice(2, -2),) * 3
    np.testing.assert_allclose(O.d1(g, 0, f).reshape(f.shape)[inner], (0.6 * X - 0.7 * Y - 0.5)[inner], atol=1e-12)
    np.testing.assert_allclose(O.d1(g, 2, f).reshape(f.shape)[inner], (2.2 * Z + 0.2 * Y)[inner], atol=1e-12)
    np.testing.assert_allclose(O.dmix(g, 0, 1, f).reshape(f.shape)[inner], -0.7, atol=1e-11)
    np.testing.assert_allclose(O.dmix(g, 2, 1, f).reshape(f.shape)[inner], 0.2, atol=1e-11)
    np.testing.assert_allclose(O.lap(g, f).reshape(f.shape)[inner], 0.6 + 2.2, atol=1e-11)


# ---------------------------------------------------------------- boundaries


def test_robin_reproduces_one_over_r():
    """The Robin 1/r ghost value of f = Q/|x| equals Q/|x_ghost|, at faces, edges and corners."""
    g = O.make_grid((8, 6, 7), (-8.0, -5.0, -6.0), (8.0, 9.0, 7.0), 4, O.ROBIN)
    X, Y, Z = centres(g)
    f = 2.5 / np.sqrt(X * X + Y * Y + Z * Z)
    rng = np.random.default_rng(0)
    checked = 0
    for _ in range(400):
        i, j, k = (int(rng.integers(-2, g.n[a] + 2)) for a in range(3))
        if 0 <= i < g.n[0] and 0 <= j < g.n[1] and 0 <= k < g.n[2]:
            continue
        x = [g.lo[a] + (c + 0.5) * g.h[a] for a, c in enumerate((i, j, k))]
        want = 2.5 / np.sqrt(sum(v * v for v in x))
        assert O.boundary_value(g, f, i, j, k) == pytest.approx(want, rel=1e-14)
        checked += 1
    assert checked > 100


def test_periodic_ghost_is_wrap():
    g = O.make_grid((5, 4, 6), 0.0, 1.0, 4, O.PERIODIC)
    f = np.arange(120, dtype=float)
    for (i, j, k) in [(-1, 0, 0), (5, 3, 2), (-2, -2, -2), (6, 5, 7), (2, -1, 6)]:
        want = f[(i % 5) + 5 * ((j % 4) + 4 * (k % 6))]
        assert O.boundary_value(g, f, i, j, k) == want


# ---------------------------------------------------------------- transfer operators


@pytest.mark.parametrize("bc", [O.PERIODIC, O.ROBIN])
def test_restriction_reproduces_linears(bc):
    fine = O.make_grid((8, 12, 6), (-1.0, 0.0, 2.0), (3.0, 6.0, 5.0), 2, bc)
    gc = O.coarse(fine)
    X, Y, Z = centres(fine)
    Xc, Yc, Zc = centres(gc)
    f = 1.5 + 0.25 * X - 0.5 * Y + 2.0 * Z
    np.testing.assert_allclose(O.restrict(gc, f), 1.5 + 0.25 * Xc - 0.5 * Yc + 2.0 * Zc, atol=1e-13)


def test_prolongation_reproduces_constants_and_linears():
    gcp = O.make_grid((4, 6, 3), 0.0, (4.0, 6.0, 3.0), 2, O.PERIODIC)
    out = O.prolong_add(gcp, np.full(72, 3.25), np.zeros(8 * 72))
    np.testing.assert_allclose(out, 3.25, atol=1e-15)
    # linear data on a Robin grid: exact for fine cells whose stencil stays inside the box
    gcr = O.make_grid((5, 6, 4), (-2.0, -3.0, 1.0), (3.0, 3.0, 5.0), 2, O.ROBIN)
    fine = O.make_grid((10, 12, 8), (-2.0, -3.0, 1.0), (3.0, 3.0, 5.0), 2, O.ROBIN)
    Xc, Yc, Zc = centres(gcr)
    X, Y, Z = centres(fine)
    lin = lambda x, y, z: 0.4 - 0.3 * x + 0.7 * y + 0.2 * z
    out = O.prolong_add(gcr, lin(Xc, Yc, Zc), np.zeros(X.size)).reshape(X.shape)
    inner = (slice(1, -1),) * 3
    np.testing.assert_allclose(out[inner], lin(X, Y, Z)[inner], atol=1e-13)


# ---------------------------------------------------------------- AtAt and the momentum operator


@pytest.mark.parametrize("order", [2, 4])
def test_atat_vanishes_on_conformal_killing_vectors(order):
    """At = LW vanishes for the conformal Killing vectors of flat space (translation,
    rotation, dilation, special conformal): catches a wrong trace factor or a missing transpose."""
    g = O.make_grid((9, 10, 8), (-2.0, -1.5, -2.5), (2.5, 3.5, 1.5), order, O.ROBIN)
    X, Y, Z = centres(g)
    x = np.stack([X, Y, Z])
    om = np.array([0.3, -0.8, 0.5])
    b = np.array([0.2, 0.1, -0.4])
    r2 = X * X + Y * Y + Z * Z
    bx = b[0] * X + b[1] * Y + b[2] * Z
    W = np.stack([
        0.7 + 1.3 * x[a] + (om[(a + 1) % 3] * x[(a + 2) % 3] - om[(a + 2) % 3] * x[(a + 1) % 3])
        + 2 * bx * x[a] - r2 * b[a] for a in range(3)])
    aa = O.atat(g, W)
    inner = (slice(2, -2),) * 3
    assert np.abs(aa[inner]).max() < 1e-20


def test_atat_simple_shear():
    """W = (s y, 0, 0): the traceless symmetric gradient has At_xy = At_yx = s, so AtAt = 2 s^2."""
    g = O.make_grid((6, 7, 5), 0.0, (3.0, 3.5, 2.5), 4, O.ROBIN)
    X, Y, Z = centres(g)
    W = np.stack([0.6 * Y, np.zeros_like(Y), np.zeros_like(Y)])
    np.testing.assert_allclose(O.atat(g, W)[2:-2, 2:-2, 2:-2], 2 * 0.36, rtol=1e-13)


def bowen_york(X, Y, Z, P):
    r = np.sqrt(X * X + Y * Y + Z * Z)
    n = [X / r, Y / r, Z / r]
    nP = n[0] * P[0] + n[1] * P[1] + n[2] * P[2]
    W = np.stack([-(7 * P[a] + n[a] * nP) / (4 * r) for a in range(3)])
    aa = 4.5 / r ** 4 * (P[0] ** 2 + P[1] ** 2 + P[2] ** 2 + 2 * nP * nP)
    return r, W, aa


@pytest.mark.parametrize("order", [2, 4])
def test_bowen_york_momentum(order):
    """The Bowen-York boost (a textbook exact solution of the vacuum momentum constraint,
    W_i = -(7 P_i + n_i n.P)/4r) has LW divergence-free and AtAt = 9/(2 r^4) (P^2 + 2 (n.P)^2).
    The discrete AtAt and momentum operator converge to these at the stencil's order."""
    P = (0.3, -0.2, 0.5)
    errs_aa, errs_mom = [], []
    rms = lambda a: np.sqrt(np.mean(a * a))
    for n in (48, 96):
        g = O.make_grid(n, -6.0, 6.0, order, O.ROBIN)
        X, Y, Z = centres(g)
        r, W, aa_exact = bowen_york(X, Y, Z, P)
        res = O.residual(g, np.zeros(X.size), W, np.zeros(X.size), np.zeros(X.size), np.zeros(3 * X.size), O.K_FIXED)
        mask = (r > 3.0) & (r < 5.0)
        errs_aa.append(rms((O.atat(g, W) - aa_exact)[mask]))
        errs_mom.append(rms(res["FW"][:, mask]))
    for e in (errs_aa, errs_mom):
        rate = np.log2(e[0] / e[1])
        assert abs(rate - order) < 0.25, (e, rate)
    assert errs_aa[1] < (1e-4 if order == 2 else 1e-6)


# ---------------------------------------------------------------- the constraints themselves


def trig_state(X, Y, Z, L, eps=0.05, dW=0.02):
    """Smooth periodic psi and W with analytic first and second derivatives."""
    k = 2 * PI / L * np.array([1.0, 2.0, -1.0])
    ph = k[0] * X + k[1] * Y + k[2] * Z + 0.4
    psi = 1 + eps * np.sin(ph)
    lap_psi = -eps * (k @ k) * np.sin(ph)
    q = 2 * PI / L * np.array([2.0, -1.0, 1.0])
    th = np.array([0.1, 1.2, 2.3])
    amp = dW * np.array([1.0, -0.6, 0.8])
    arg = [q[0] * X + q[1] * Y + q[2] * Z + th[b] for b in range(3)]
    W = np.stack([amp[b] * np.cos(arg[b]) for b in range(3)])
    G = np.empty((3, 3) + X.shape)   # G[a, b] = d_a W_b
    for a in range(3):
        for b in range(3):
            G[a, b] = -amp[b] * q[a] * np.sin(arg[b])
    # (Lap + (1/3) grad div) W for a single mode q: -|q|^2 W_i - (1/3) q_i q_j W_j
    momop = np.stack([-(q @ q) * W[i] - sum(q[i] * q[j] * W[j] for j in range(3)) / 3 for i in range(3)])
    return psi, lap_psi, W, G, momop


@pytest.mark.parametrize("order", [2, 4])
def test_H_and_M_match_the_paper_definitions(order):
    """H from eq:Ham and M_i from eq:Mom, evaluated with explicit tensors (gamma = psi^4 delta,
    K_ij = psi^-2 At_ij + gamma_ij K/3, K^ij raised with gamma^-1, R = -8 psi^-5 Lap psi,
    D^j A_ij = psi^-6 d_j At_ij), match the oracle's H and M up to the stencil's truncation order."""
    L, K = 16.0, -0.4
    errs = []
    for n in (16, 32):
        g = O.make_grid(n, 0.0, L, order, O.PERIODIC)
        X, Y, Z = centres(g)
        psi, lap_psi, W, G, momop = trig_state(X, Y, Z, L)
        rho0 = 0.01 + 0.004 * np.cos(2 * PI * X / L)
        rho2 = 0.003 + 0.001 * np.sin(2 * PI * Y / L)
        S = np.stack([0.002 * np.cos(2 * PI * Z / L), 0.001 * np.sin(2 * PI * X / L), 0.0015 * np.ones_like(X)])
        # paper definition, with explicit tensor algebra
        div = G[0, 0] + G[1, 1] + G[2, 2]
        At = np.empty((3, 3) + X.shape)
        for a in range(3):
            for b in range(3):
                At[a, b] = G[a, b] + G[b, a] - (2.0 / 3.0 * div if a == b else 0.0)
        Kdn = np.empty_like(At)
        for a in range(3):
            for b in range(3):
                Kdn[a, b] = psi ** -2 * At[a, b] + (psi ** 4 * K / 3.0 if a == b else 0.0)
        Kup = psi ** -8 * Kdn                      # gamma^ia gamma^jb K_ab with gamma^ij = psi^-4 delta
        trK = sum(psi ** -4 * Kdn[a, a] for a in range(3))
        KK = sum(Kdn[a, b] * Kup[a, b] for a in range(3) for b in range(3))
        R = -8.0 * psi ** -5 * lap_psi
        rho = rho0 + psi ** -4 * rho2
        H_paper = R + trK ** 2 - KK - 16 * PI * rho
        msrc = np.array([np.mean(8 * PI * psi ** 6 * S[i]) for i in range(3)])
        M_paper = np.stack([psi ** -6 * momop[i] - 8 * PI * S[i] + psi ** -6 * msrc[i] for i in range(3)])
        res = O.residual(g, psi - 1.0, W, rho0, rho2, S, O.K_FIXED, K2=K * K)
        errs.append((np.abs(res["H"] - H_paper).max(), np.abs(res["M"] - M_paper).max()))
        np.testing.assert_allclose(res["msrc"], msrc, rtol=1e-12, atol=1e-15)
    for c in range(2):
        rate = np.log2(errs[0][c] / errs[1][c])
        assert abs(rate - order) < 0.3, (errs, rate)


@pytest.mark.parametrize("order", [2, 4])
def test_uniform_density(order):
    """Uniform rho, no momentum: psi = 1, W = 0 and K^2 = 24 pi rho exactly (eq:Ham with K_ij = gamma_ij K/3)."""
    p = Fd.uniform(n=8, rho=2e-3, order=order)
    g = O.make_grid(p["n"], p["lo"], p["hi"], order, p["bc"])
    r = O.solve(g, p["rho0"], p["rho2"], p["S"], O.K_INTEGRABILITY, tol=1e-13, max_outer=5)
    assert r["status"] == "converged" and r["iters"] == 0
    assert r["K2"] == pytest.approx(24 * PI * 2e-3, rel=1e-14)
    assert np.abs(r["u"]).max() == 0.0 and np.abs(r["W"]).max() == 0.0
    assert r["hist"][0].max() < 1e-15


def test_bare_puncture_is_exact():
    """rho = S = K = 0 with one puncture: psi = 1 + M/2r, u = 0, W = 0; H vanishes at iteration 0
    because the Laplacian acts on the regular part u only."""
    n = 16
    g = O.make_grid(n, -8.0, 8.0, 4, O.ROBIN, punctures=[(1.0, (0.0, 0.0, 0.0))])
    z = np.zeros(n ** 3)
    res = O.residual(g, z, np.zeros(3 * n ** 3), z, z, np.zeros(3 * n ** 3), O.K_FIXED)
    assert res["norms"].max() == 0.0
    r = O.solve(g, z, z, np.zeros(3 * n ** 3), O.K_FIXED, tol=1e-12)
    assert r["status"] == "converged" and r["iters"] == 0


def test_integrability_and_momentum_means():
    """On a periodic box the integrability K^2 makes sum F_psi vanish, and the mean-projected
    momentum source makes sum F_W,i vanish, at any iterate."""
    p = Fd.sine_periodic(n=12)
    g = O.make_grid(p["n"], p["lo"], p["hi"], 2, O.PERIODIC)
    X, Y, Z = centres(g)
    psi, _, W, _, _ = trig_state(X, Y, Z, 16.0, eps=0.03, dW=0.01)
    res = O.residual(g, psi - 1 - np.mean(psi - 1), W, p["rho0"], p["rho2"], p["S"], O.K_INTEGRABILITY)
    scale = np.abs(res["Fpsi"]).max()
    assert abs(res["Fpsi"].sum()) < 1e-12 * scale * X.size
    for i in range(3):
        assert abs(res["FW"][i].sum()) < 1e-12 * np.abs(res["FW"][i]).max() * X.size


# ---------------------------------------------------------------- manufactured solutions


def manufactured_periodic(n, order, L=16.0, K2=0.3):
    g = O.make_grid(n, 0.0, L, order, O.PERIODIC)
    X, Y, Z = centres(g)
    psi, lap_psi, W, G, momop = trig_state(X, Y, Z, L, eps=0.02, dW=0.01)
    div = G[0, 0] + G[1, 1] + G[2, 2]
    aa = sum((G[a, b] + G[b, a] - (2.0 / 3.0 * div if a == b else 0.0)) ** 2 for a in range(3) for b in range(3))
    rho2 = 0.002 * (1 + np.cos(2 * PI * Y / L))
    # choose rho0 and S so that the continuum constraints hold exactly
    rho0 = (-lap_psi + K2 / 12 * psi ** 5 - aa / 8 * psi ** -7 - 2 * PI * rho2 * psi) / (2 * PI * psi ** 5)
    S = np.stack([momop[i] / (8 * PI * psi ** 6) for i in range(3)])
    return g, psi, W, rho0, rho2, S


@pytest.mark.parametrize("order", [2, 4])
def test_truncation_order_periodic(order):
    """The discrete residual of the exact continuum solution is O(h^p)."""
    errs = []
    for n in (16, 32, 64):
        g, psi, W, rho0, rho2, S = manufactured_periodic(n, order)
        res = O.residual(g, psi - 1, W, rho0, rho2, S, O.K_FIXED, K2=0.3)
        errs.append((np.abs(res["Fpsi"]).max(), np.abs(res["FW"]).max()))
    for c in range(2):
        rate = np.log2(errs[1][c] / errs[2][c])
        assert abs(rate - order) < 0.1, (errs, rate)


def manufactured_robin(n, order, half=16.0, sig=4.0, Q=0.3, B=(0.05, -0.03, 0.04)):
    """psi = 1 + 1/2r + Q erf(r/s)/r, W_i = B_i erf(r/s)/r: both fall off exactly as 1/r at the boundary."""
    from scipy.special import erf
    g = O.make_grid(n, -half, half, order, O.ROBIN, punctures=[(1.0, (0.0, 0.0, 0.0))])
    X, Y, Z = centres(g)
    x = [X, Y, Z]
    r = np.sqrt(X * X + Y * Y + Z * Z)
    e = np.exp(-r * r / sig ** 2)
    f = erf(r / sig) / r
    fp = 2 / (np.sqrt(PI) * sig) * e / r - erf(r / sig) / r ** 2
    fpp = -4 / (np.sqrt(PI) * sig ** 3) * e - 4 / (np.sqrt(PI) * sig) * e / r ** 2 + 2 * erf(r / sig) / r ** 3
    lapf = -4 / (np.sqrt(PI) * sig ** 3) * e
    u = Q * f
    psi = 1 + 0.5 / r + u
    W = np.stack([B[b] * f for b in range(3)])
    G = np.empty((3, 3) + X.shape)
    for a in range(3):
        for b in range(3):
            G[a, b] = B[b] * fp * x[a] / r
    div = G[0, 0] + G[1, 1] + G[2, 2]
    aa = sum((G[a, b] + G[b, a] - (2.0 / 3.0 * div if a == b else 0.0)) ** 2 for a in range(3) for b in range(3))
    hess = lambda a, b: fpp * x[a] * x[b] / r ** 2 + fp * ((1.0 if a == b else 0.0) / r - x[a] * x[b] / r ** 3)
    momop = np.stack([B[i] * lapf + sum(B[j] * hess(i, j) for j in range(3)) / 3 for i in range(3)])
    rho2 = 0.2 * e
    rho0 = (-Q * lapf - aa / 8 * psi ** -7 - 2 * PI * rho2 * psi) / (2 * PI * psi ** 5)
    S = np.stack([momop[i] / (8 * PI * psi ** 6) for i in range(3)])
    return g, u, W, rho0, rho2, S


@pytest.mark.parametrize("order", [2, 4])
def test_truncation_order_robin_puncture(order):
    errs = []
    for n in (32, 64):
        g, u, W, rho0, rho2, S = manufactured_robin(n, order)
        res = O.residual(g, u, W, rho0, rho2, S, O.K_FIXED)
        errs.append((np.abs(res["Fpsi"]).max(), np.abs(res["FW"]).max()))
    for c in range(2):
        rate = np.log2(errs[0][c] / errs[1][c])
        assert abs(rate - order) < 0.2, (errs, rate)


@pytest.mark.parametrize("order", [2, 4])
def test_solution_converges_at_formal_order(order):
    """Solving the discrete system (K^2 from integrability, <u> = <W> = 0) recovers the
    manufactured psi, W and K^2 with errors falling at the stencil's order."""
    errs = []
    for n in (8, 16, 32):
        g, psi, W, rho0, rho2, S = manufactured_periodic(n, order)
        r = O.solve(g, rho0, rho2, S, O.K_INTEGRABILITY, tol=1e-13, max_outer=40)
        assert r["status"] in ("converged", "floor")
        errs.append((np.abs(r["u"] - (psi - 1)).max(), np.abs(r["W"] - W).max(), abs(r["K2"] - 0.3)))
    for c in range(3):
        rate = np.log2(errs[1][c] / errs[2][c])
        assert rate > order - 0.4, (errs, rate)
