"""Find, with the FP64 oracle, the strongest inhomogeneity the constant-K solve still handles.

With a constant K the linearised Hamiltonian operator is Lap + c with
c = -(5/12) K^2 psi^4 - (7/8) psi^-8 AtAt + 2 pi (5 rho0 psi^4 + rho2).  Once c
exceeds the smallest nonzero eigenvalue of -Lap somewhere, the operator is
indefinite, and for stronger data the constant-K problem has no root on the
psi ~ 1 branch (the existence issue that the paper's CTTK methods address).
This script bisects, in log scale, for the largest amplitude at which the
oracle's solve from psi = 1 still reaches max(|H|, |M_i|) <= 1e-10 on the
psi ~ 1 branch (max |u| < 0.5), for

* the random-mode periodic cosmology (L = 32, 16 modes, amplitude prefactor a0,
  phi0 = 1, m = 1, 4th order) at 32^3;
* the Gaussian scalar shell around an M = 1 puncture (phi = A exp(-(r - 10)^2/4),
  Pi = 0.01 phi, K = 0, Robin, 4th order) on [-16, 16]^3 at 32^3.

It calls only ``oracle/`` and the seeded input generators, and writes
``amplitude_scan.json`` beside itself.  Usage: python tests/golden/make_amplitude_scan.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import oracle as O  # noqa: E402
from paper_2501_13046_gb300 import fields  # noqa: E402

FAMILIES = {
    "modes_periodic_32": (lambda a: fields.modes_periodic(n=32, a0=a), 5e-5, 0.05),
    "puncture_shell_32_half16": (lambda a: fields.puncture_shell(n=32, half=16.0, A=a), 0.02, 0.05),
}


def converges(p):
    g = O.make_grid(p["n"], p["lo"], p["hi"], p["order"], p["bc"], p["punctures"])
    r = O.solve(g, p["rho0"], p["rho2"], p["S"], p["kmode"], K2=p["K"] ** 2, tol=1e-10, max_outer=40)
    ok = bool(r["status"] == "converged" and np.abs(r["u"]).max() < 0.5)
    return ok, r["status"], r["iters"], float(np.abs(r["u"]).max()) if np.isfinite(r["u"]).all() else None


def scan(make, good, bad, steps=10):
    assert converges(make(good))[0], "the lower amplitude must converge"
    assert not converges(make(bad))[0], "the upper amplitude must fail"
    trail = []
    for _ in range(steps):
        mid = float(np.sqrt(good * bad))
        ok, st, it, umax = converges(make(mid))
        trail.append(dict(amplitude=mid, converged=ok, status=st, iters=it, max_u=umax))
        if ok:
            good = mid
        else:
            bad = mid
    return good, bad, trail


def main():
    out = {"source": "oracle/ctt_oracle.c solves from psi = 1 (tol 1e-10, 40 outer iterations), bisection in "
                     "log scale; written by tests/golden/make_amplitude_scan.py"}
    for name, (make, good, bad) in FAMILIES.items():
        g, b, trail = scan(make, good, bad)
        out[name] = dict(largest_converging=g, smallest_failing=b, trail=trail)
        print(name, g, b)
    with open(os.path.join(HERE, "amplitude_scan.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
