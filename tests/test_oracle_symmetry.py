"""Pins of the oracle's reflection-symmetry planes (Key features, "Boundary conditions":
reflective), against facts the oracle does not compute with the same code: the ghost values are
the mirror images with the sign of the normal component of W flipped (checked cell by cell,
including edges where a mirror meets a Robin face), and an octant problem solved with three
symmetry planes equals the corresponding octant of the same symmetric problem solved on the full
box with Robin faces only (the discrete equations restricted to the octant are the same)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2501_13046_gb300 import fields as Fd


def test_ghost_values_mirror_with_parity():
    g = O.make_grid((6, 5, 4), 0.0, (3.0, 2.5, 2.0), 4, O.ROBIN, reflect=7)
    rng = np.random.default_rng(3)
    f = rng.standard_normal(6 * 5 * 4)
    F = f.reshape(4, 5, 6)
    h = 0.5
    X = lambda i: (i + 0.5) * h
    for fi in range(4):
        sx, sy, sz = (-1 if fi == 1 else 1), (-1 if fi == 2 else 1), (-1 if fi == 3 else 1)
        assert O.boundary_value(g, f, -1, 2, 1, fi) == sx * F[1, 2, 0]
        assert O.boundary_value(g, f, -2, 2, 1, fi) == sx * F[1, 2, 1]
        assert O.boundary_value(g, f, 3, -1, 2, fi) == sy * F[2, 0, 3]
        assert O.boundary_value(g, f, 3, 2, -2, fi) == sz * F[1, 2, 3]
        assert O.boundary_value(g, f, -1, -2, 0, fi) == sx * sy * F[0, 1, 0]
        # mirror across x, Robin across the upper y face: the ratio of the in-box cell's distance
        # to the ghost's (mirroring keeps |x|)
        want = sx * F[1, 4, 0] * np.sqrt(X(0) ** 2 + X(4) ** 2 + X(1) ** 2) / np.sqrt(X(-1) ** 2 + X(5) ** 2 + X(1) ** 2)
        assert O.boundary_value(g, f, -1, 5, 1, fi) == pytest.approx(want, rel=1e-14)
    # an unmarked lower face stays Robin
    g2 = O.make_grid((6, 5, 4), 0.0, (3.0, 2.5, 2.0), 4, O.ROBIN, reflect=6)
    want = F[1, 2, 0] * np.sqrt(X(0) ** 2 + X(2) ** 2 + X(1) ** 2) / np.sqrt(X(-1) ** 2 + X(2) ** 2 + X(1) ** 2)
    assert O.boundary_value(g2, f, -1, 2, 1, 1) == pytest.approx(want, rel=1e-14)


def octant(a):
    n = a.shape[-1]
    return a[..., n // 2:, n // 2:, n // 2:]


@pytest.mark.parametrize("order", [2, 4])
def test_octant_solve_equals_the_full_box_solve(order):
    """Puncture at the origin with a scalar shell (u, rho even, S_i odd in x_i): full box
    [-8, 8]^3 at 32^3 with Robin faces, against the octant [0, 8]^3 at 16^3 with three symmetry
    planes and Robin upper faces; both to the FP64 floor."""
    full = Fd.puncture_shell(n=32, half=8.0, A=0.02, order=order)
    gf = O.make_grid(32, -8.0, 8.0, order, O.ROBIN, full["punctures"])
    rf = O.solve(gf, full["rho0"], full["rho2"], full["S"], O.K_FIXED, tol=0.0, max_outer=80)
    go = O.make_grid(16, 0.0, 8.0, order, O.ROBIN, full["punctures"], reflect=7)
    so = [np.ascontiguousarray(octant(a)) for a in (full["rho0"], full["rho2"], full["S"])]
    ro = O.solve(go, so[0], so[1], so[2], O.K_FIXED, tol=0.0, max_outer=80)
    assert rf["status"] in ("floor", "converged") and ro["status"] in ("floor", "converged")
    uf, Wf = octant(rf["u"]), octant(rf["W"])
    assert np.abs(np.abs(Wf)).max() > 1e-8
    assert np.abs(ro["u"] - uf).max() <= 1e-12 * np.abs(1 + uf).max()
    assert np.abs(ro["W"] - Wf).max() <= 1e-10 * np.abs(Wf).max() + 1e-15
