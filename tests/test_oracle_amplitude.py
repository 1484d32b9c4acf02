"""Evidence for the amplitude reading of the benchmark workloads (CPU, oracle only).

With a constant K (the CTT family with K fixed or set by the periodic
integrability condition) the Hamiltonian constraint's linearisation is Lap + c,
c = -(5/12) K^2 psi^4 - (7/8) psi^-8 AtAt + 2 pi (5 rho0 psi^4 + rho2).  At
psi = 1, W = 0 with K^2 = 24 pi <rho> this is c = 10 pi (rho0 - <rho>) + ...,
so strong density contrasts make c exceed the smallest nonzero eigenvalue of
-Lap and the problem loses its root on the psi ~ 1 branch (the existence
problem that the paper's CTTK methods are built for).  These tests show, with
the oracle alone, that

* the literal amplitudes (random-mode prefactor 0.05 with phi0 = 1; Gaussian
  shell A = 0.05) put max c hundreds of times above that eigenvalue, and the
  oracle's solve from psi = 1 fails there;
* the amplitudes the benchmark uses (prefactor 5e-5; shell A = 0.02) keep c
  below it and solve;
* the bisection stored in tests/golden/amplitude_scan.json (written by
  make_amplitude_scan.py with the oracle) brackets the largest amplitude that
  still solves: its lower end solves and its upper end fails.
"""
import json
import os

import numpy as np

from oracle import oracle as O
from paper_2501_13046_gb300 import fields

HERE = os.path.dirname(os.path.abspath(__file__))
L = 32.0
N = 32


def lap_min_eigenvalue(order, n, L):
    """Smallest nonzero eigenvalue of -Lap on a periodic cube: the stencil's Fourier symbol at
    k = 2 pi / L along one axis (2nd order: 4 sin^2(theta/2)/h^2; 4th: (30 - 32 cos + 2 cos 2theta)/12h^2)."""
    h = L / n
    th = 2 * np.pi / n
    if order == 2:
        return 4 * np.sin(th / 2) ** 2 / h ** 2
    return (30 - 32 * np.cos(th) + 2 * np.cos(2 * th)) / (12 * h ** 2)


def grid(p):
    return O.make_grid(p["n"], p["lo"], p["hi"], p["order"], p["bc"], p["punctures"])


def c_at_start(p):
    z = np.zeros(p["rho0"].shape)
    r = O.residual(grid(p), z, np.zeros((3,) + z.shape), p["rho0"], p["rho2"], p["S"], p["kmode"], K2=p["K"] ** 2)
    return r["c"]


def solves(p):
    r = O.solve(grid(p), p["rho0"], p["rho2"], p["S"], p["kmode"], K2=p["K"] ** 2, tol=1e-10, max_outer=40)
    return r["status"] == "converged" and np.abs(r["u"]).max() < 0.5


def scan():
    with open(os.path.join(HERE, "golden", "amplitude_scan.json")) as f:
        return json.load(f)


def test_literal_mode_amplitude_is_indefinite_and_does_not_solve():
    p = fields.modes_periodic(n=N, L=L, a0=0.05)
    lam = lap_min_eigenvalue(4, N, L)
    assert c_at_start(p).max() > 100 * lam
    assert not solves(p)


def test_benchmark_mode_amplitude_is_definite_and_solves():
    p = fields.modes_periodic(n=N, L=L, a0=5e-5)
    assert c_at_start(p).max() < lap_min_eigenvalue(4, N, L)
    assert solves(p)


def test_literal_shell_amplitude_does_not_solve_and_the_benchmark_one_does():
    assert not solves(fields.puncture_shell(n=N, half=16.0, A=0.05))
    assert solves(fields.puncture_shell(n=N, half=16.0, A=0.02))


def test_stored_bisection_brackets_the_limit():
    """The random-mode family's bracket (the shell's, 0.02884..0.02886, is re-checked only by
    make_amplitude_scan.py: its solves near the fold take a minute)."""
    make = lambda a: fields.modes_periodic(n=N, L=L, a0=a)
    s = scan()["modes_periodic_32"]
    lo, hi = s["largest_converging"], s["smallest_failing"]
    assert lo < hi < 1.01 * lo
    assert solves(make(lo))
    assert not solves(make(hi))
