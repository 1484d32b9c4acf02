"""Extrapolating faces of Robin boxes in the oracle (CPU pins).

The paper lists extrapolating boundaries next to reflective and periodic ones (Key features,
"Boundary conditions") without a formula.  Reading: beyond an extrapolating face a cell at
distance d along the normal takes the linear extrapolation (1 + d) v(b) - d v(b') through the
boundary cell b and its inner neighbour b'; several extrapolating axes apply in turn (a tensor
product of linear maps), and the Robin 1/r rule then resolves any remaining out-of-box
coordinate.  Pins:

* ghost values of linear fields (and of products of linear factors across two extrapolating
  faces) are exact, at distances 1 and 2, on both faces of every axis;
* so the oracle's derivative stencils are exact for those fields at the boundary cells too;
* a ghost beyond an extrapolating face and a Robin face is the Robin rule at the extrapolated
  points;
* the oracle's solve reaches the root of the independent dense restatement (dense_newton.py) on
  8^3 Robin boxes with a puncture and extrapolating faces, to 1e-12.
"""
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from oracle.dense_newton import DenseSystem
from paper_2501_13046_gb300 import fields

N = (8, 7, 6)
LO, HI = (-4.0, -3.5, -3.0), (4.0, 3.5, 3.0)


def grid(extrap, order=4):
    return O.make_grid(N, LO, HI, order, O.ROBIN, extrap=extrap)


def cell_x(a, i):
    return LO[a] + (i + 0.5) * (HI[a] - LO[a]) / N[a]


def field(fun):
    X, Y, Z = fields.cell_centres(list(N), list(LO), list(HI))
    return np.ascontiguousarray(fun(X, Y, Z))


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("upper", [False, True])
def test_linear_fields_are_extrapolated_exactly(axis, upper):
    bit = 1 << (2 * axis + (1 if upper else 0))
    g = grid(bit)
    coef = (0.3, -1.7, 2.2)
    f = field(lambda X, Y, Z: 1.5 + coef[0] * X + coef[1] * Y + coef[2] * Z)
    for d in (1, 2):
        for idx in itertools.product(range(0, N[0], 3), range(0, N[1], 3), range(0, N[2], 3)):
            c = list(idx)
            c[axis] = N[axis] - 1 + d if upper else -d
            want = 1.5 + sum(coef[a] * cell_x(a, c[a]) for a in range(3))
            for fi in (0, 1, 3):
                assert O.boundary_value(g, f, c[0], c[1], c[2], fi) == pytest.approx(want, abs=1e-12)


def test_two_extrapolating_faces_reproduce_bilinear_fields_at_their_edge():
    g = grid(0b000101)   # lower x and lower y faces
    f = field(lambda X, Y, Z: (0.4 + X) * (1.3 - 0.5 * Y) + 0.2 * Z)
    for di, dj in itertools.product((1, 2), (1, 2)):
        for k in range(N[2]):
            want = (0.4 + cell_x(0, -di)) * (1.3 - 0.5 * cell_x(1, -dj)) + 0.2 * cell_x(2, k)
            assert O.boundary_value(g, f, -di, -dj, k) == pytest.approx(want, abs=1e-12)


def test_stencils_are_exact_for_linear_fields_at_extrapolating_faces():
    g = grid(0b111111 & ~0b100000)   # every face but the upper z face
    a0, b0 = 0.7, -1.1
    f = field(lambda X, Y, Z: 2.0 + a0 * X + b0 * Y)
    np.testing.assert_allclose(O.d1(g, 0, f), a0, atol=1e-12)
    np.testing.assert_allclose(O.d1(g, 1, f), b0, atol=1e-12)
    for a in (0, 1):
        np.testing.assert_allclose(O.d2(g, a, f), 0.0, atol=1e-11)
    fxy = field(lambda X, Y, Z: X * Y)
    np.testing.assert_allclose(O.dmix(g, 0, 1, fxy), 1.0, atol=1e-11)


def test_extrapolating_and_robin_corner():
    g = grid(0b000001)   # lower x face extrapolating, the y faces Robin
    f = field(lambda X, Y, Z: np.cos(X) + Y * Z)
    # beyond the lower x face (d = 1) and the upper y face (one cell): Robin at the two points
    j, k = N[1], 2
    robin = lambda i: f[k, N[1] - 1, i] * np.hypot(np.hypot(cell_x(0, i), cell_x(1, N[1] - 1)), cell_x(2, k)) \
        / np.hypot(np.hypot(cell_x(0, i), cell_x(1, j)), cell_x(2, k))
    want = 2.0 * robin(0) - robin(1)
    assert O.boundary_value(g, f, -1, j, k) == pytest.approx(want, rel=1e-13)


@pytest.mark.parametrize("extrap", [0b000011, 0b100000])
def test_oracle_root_is_the_dense_root_with_extrapolating_faces(extrap):
    p = fields.puncture_shell(n=8, half=16.0)
    ds = DenseSystem(p["n"], p["lo"], p["hi"], p["order"], p["bc"], p["punctures"], p["rho0"], p["rho2"], p["S"],
                     extrap=extrap)
    rd = ds.solve()
    assert rd["residual"] < 1e-15
    g = O.make_grid(p["n"], p["lo"], p["hi"], p["order"], p["bc"], p["punctures"], extrap=extrap)
    ro = O.solve(g, p["rho0"], p["rho2"], p["S"], p["kmode"], tol=0.0, max_outer=80)
    assert ro["status"] in ("floor", "converged")
    rel = lambda a, b: np.abs(a - b).max() / np.abs(b).max()
    assert rel(ds.psibg + ro["u"].reshape(-1), ds.psibg + rd["u"]) <= 1e-12
    for i in range(3):
        assert rel(ro["W"].reshape(3, -1)[i], rd["W"][i]) <= 5e-12
