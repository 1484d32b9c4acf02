"""Pins of the oracle's Bowen-York punctures (boosted and/or spinning black holes, Key features,
"Flexibility") against facts the oracle does not compute itself: the ADM linear and angular
momentum integrals of the analytic curvature (which fix the momentum and spin conventions, the
factors 3/2 and 3 and the sign of the spin term), its trace and symmetry, the closed forms of
AtAt for a pure boost and a pure spin, the vacuum momentum constraint (divergence-free at the
stencil's order), and the boost's vector-potential form from the textbook."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_13046_gb300 import fields as Fd

PI = np.pi


def centres(g):
    lo = [g.lo[a] for a in range(3)]
    hi = [g.lo[a] + g.n[a] * g.h[a] for a in range(3)]
    return Fd.cell_centres([g.n[0], g.n[1], g.n[2]], lo, hi)


def sphere_rule(nmu=40, nphi=80):
    """Gauss-Legendre in cos(theta) x trapezoid in phi: exact for polynomials in n of degree < 2 nmu."""
    mu, wmu = np.polynomial.legendre.leggauss(nmu)
    phi = np.arange(nphi) * 2 * PI / nphi
    M, F = np.meshgrid(mu, phi, indexing="ij")
    st = np.sqrt(1 - M * M)
    n = np.stack([st * np.cos(F), st * np.sin(F), M], axis=-1).reshape(-1, 3)
    w = (wmu[:, None] * np.full(nphi, 2 * PI / nphi)[None, :]).reshape(-1)
    return n, w


def adm_integrals(g, centre, R, nmu=40, nphi=80):
    """P_i = (1/8 pi) surf A_ij n_j dS and J_i = (1/8 pi) surf eps_ijk x_j A_kl n_l dS on the sphere
    of radius R about `centre` (x measured from the origin)."""
    n, w = sphere_rule(nmu, nphi)
    P, J = np.zeros(3), np.zeros(3)
    for nv, wv in zip(n, w):
        x = np.asarray(centre) + R * nv
        A = O.by_point(g, x)
        An = A @ nv
        P += wv * R * R * An
        J += wv * R * R * np.cross(x, An)
    return P / (8 * PI), J / (8 * PI)


def test_adm_momentum_and_spin_of_one_puncture():
    P, S = np.array([0.3, -0.2, 0.5]), np.array([-0.1, 0.25, 0.15])
    g = O.make_grid(8, -4.0, 4.0, 4, O.ROBIN, [(1.0, (0.0, 0.0, 0.0), P, S)])
    for R in (0.7, 3.0):
        Pa, Ja = adm_integrals(g, (0.0, 0.0, 0.0), R)
        np.testing.assert_allclose(Pa, P, atol=1e-13)
        np.testing.assert_allclose(Ja, S, atol=1e-13)


def test_adm_momenta_of_a_displaced_binary():
    """Two punctures off the origin: the momenta add, and the angular momentum about the origin is
    S_1 + S_2 + x_1 x P_1 + x_2 x P_2 (the orbital part fixes the sign of the position term)."""
    x1, x2 = np.array([2.0, 0.5, -0.3]), np.array([-1.5, -0.4, 0.6])
    P1, P2 = np.array([0.0, 0.2, 0.05]), np.array([0.1, -0.2, 0.0])
    S1, S2 = np.array([0.0, 0.0, 0.2]), np.array([0.1, -0.05, 0.0])
    g = O.make_grid(8, -8.0, 8.0, 4, O.ROBIN, [(0.5, x1, P1, S1), (0.5, x2, P2, S2)])
    Pa, Ja = adm_integrals(g, (0.0, 0.0, 0.0), 12.0, nmu=80, nphi=160)
    np.testing.assert_allclose(Pa, P1 + P2, atol=1e-10)
    np.testing.assert_allclose(Ja, S1 + S2 + np.cross(x1, P1) + np.cross(x2, P2), atol=1e-10)


def test_curvature_is_symmetric_and_traceless():
    rng = np.random.default_rng(5)
    g = O.make_grid(8, -4.0, 4.0, 4, O.ROBIN, [(1.0, (0.3, -0.2, 0.1), (0.3, 0.1, -0.4), (0.2, -0.3, 0.1)),
                                               (0.7, (-1.0, 0.5, 0.0), (-0.2, 0.0, 0.3), (0.0, 0.1, 0.4))])
    for _ in range(20):
        A = O.by_point(g, rng.uniform(-4, 4, 3))
        scale = np.abs(A).max()
        assert np.abs(A - A.T).max() <= 1e-15 * scale
        assert abs(np.trace(A)) <= 1e-14 * scale


def test_atat_closed_forms_of_a_boost_and_a_spin():
    """W = 0: the oracle's AtAt is the Bowen-York part alone; a pure boost gives
    9/(2 r^4) (P^2 + 2 (n.P)^2) and a pure spin 18 |S x n|^2 / r^6."""
    P, S = np.array([0.3, -0.2, 0.5]), np.array([-0.1, 0.25, 0.15])
    zeros = np.zeros((3, 8, 8, 8))
    for kind in ("boost", "spin"):
        pun = (1.0, (0.0, 0.0, 0.0), P if kind == "boost" else (0, 0, 0), S if kind == "spin" else (0, 0, 0))
        g = O.make_grid(8, -4.0, 4.0, 4, O.ROBIN, [pun])
        X, Y, Z = centres(g)
        r = np.sqrt(X * X + Y * Y + Z * Z)
        n = np.stack([X / r, Y / r, Z / r])
        if kind == "boost":
            nP = np.einsum("a...,a->...", n, P)
            exact = 4.5 / r ** 4 * (P @ P + 2 * nP * nP)
        else:
            sxn = np.stack([S[1] * n[2] - S[2] * n[1], S[2] * n[0] - S[0] * n[2], S[0] * n[1] - S[1] * n[0]])
            exact = 18.0 * (sxn * sxn).sum(0) / r ** 6
        np.testing.assert_allclose(O.atat(g, zeros), exact, rtol=1e-13)


@pytest.mark.parametrize("order", [2, 4])
def test_curvature_is_divergence_free(order):
    """The momentum constraint in vacuum: sum_j D_j A_ij -> 0 at the stencil's order away from the
    punctures (boost and spin together)."""
    errs = []
    for n in (48, 96):
        g = O.make_grid(n, -6.0, 6.0, order, O.ROBIN, [(1.0, (0.0, 0.0, 0.0), (0.3, -0.2, 0.5), (-0.1, 0.25, 0.15))])
        X, Y, Z = centres(g)
        A = O.by_cells(g)
        assert np.array_equal(A[:, :, 5, 7, 9], O.by_point(g, (X[5, 7, 9], Y[5, 7, 9], Z[5, 7, 9])))
        div = np.stack([sum(O.d1(g, b, A[a, b]) for b in range(3)) for a in range(3)])
        r = np.sqrt(X * X + Y * Y + Z * Z)
        mask = (r > 3.0) & (r < 5.0)
        errs.append(np.sqrt(np.mean(div[:, mask] ** 2)))
    rate = np.log2(errs[0] / errs[1])
    assert abs(rate - order) < 0.3, (errs, rate)


@pytest.mark.parametrize("order", [2, 4])
def test_boost_matches_its_vector_potential(order):
    """The boost's textbook vector potential W_i = -(7 P_i + n_i n.P)/(4 r) has (LW)_ij equal to the
    analytic boost curvature: the oracle's AtAt from W (bare puncture) and from the analytic part
    (W = 0) agree at the stencil's order."""
    P = np.array([0.3, -0.2, 0.5])
    errs = []
    for n in (48, 96):
        bare = O.make_grid(n, -6.0, 6.0, order, O.ROBIN, [(1.0, (0.0, 0.0, 0.0))])
        boosted = O.make_grid(n, -6.0, 6.0, order, O.ROBIN, [(1.0, (0.0, 0.0, 0.0), P, (0, 0, 0))])
        X, Y, Z = centres(bare)
        r = np.sqrt(X * X + Y * Y + Z * Z)
        nv = [X / r, Y / r, Z / r]
        nP = nv[0] * P[0] + nv[1] * P[1] + nv[2] * P[2]
        W = np.stack([-(7 * P[a] + nv[a] * nP) / (4 * r) for a in range(3)])
        diff = O.atat(bare, W) - O.atat(boosted, np.zeros_like(W))
        mask = (r > 3.0) & (r < 5.0)
        errs.append(np.sqrt(np.mean(diff[mask] ** 2)))
    rate = np.log2(errs[0] / errs[1])
    assert abs(rate - order) < 0.3, (errs, rate)
