"""Write sampled values of the FP64 oracle's discrete root for the full-size workloads.

The oracle (a plain CPU FP64 Newton-multigrid, ``oracle/ctt_oracle.c``) takes
minutes to hours at these sizes, far too long for a test, so this script solves
each workload once, to the oracle's FP64 floor, and stores what a test or the
benchmark needs to state the error of a GPU solve per field:

* the max-norm of each field (psi = 1 + sum of m/2r + u, u, W_x, W_y, W_z) over the whole grid;
* its values at 4096 seeded cells plus the cells where each field is largest in
  magnitude and those where it changes most between neighbours;
* K^2 (periodic boxes), the oracle's iteration count, time and per-iteration norms.

Nothing here comes from the CUDA library: it calls only ``oracle/`` and the
seeded input generators.  Usage::

    python tests/golden/make_oracle_roots.py modes_periodic_128
    python tests/golden/make_oracle_roots.py puncture_shell_256
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_2501_13046_gb300 import fields  # noqa: E402

WORKLOADS = {
    # periodic random-mode cosmology, L = 32, 128^3, 4th order (the benchmarked solve)
    "modes_periodic_128": lambda: fields.modes_periodic(n=128),
    # M = 1 puncture with a Gaussian scalar shell, [-64, 64]^3, 256^3, Robin, 4th order
    "puncture_shell_256": lambda: fields.puncture_shell(n=256),
    # smaller members of the same families (test-sized)
    "modes_periodic_64": lambda: fields.modes_periodic(n=64),
}
SAMPLES = 4096


def sample_cells(shape, fields_, seed=12345):
    """Seeded random cells plus, per field, the cell of largest |value| and of largest jump."""
    nz, ny, nx = shape
    rng = np.random.Generator(np.random.PCG64(seed))
    flat = set(int(i) for i in rng.choice(nz * ny * nx, size=SAMPLES, replace=False))
    for f in fields_:
        flat.add(int(np.argmax(np.abs(f))))
        for ax in range(3):
            jump = np.abs(np.diff(f, axis=ax))
            idx = np.unravel_index(int(np.argmax(jump)), jump.shape)
            flat.add(int(np.ravel_multi_index(idx, shape)))
    return sorted(flat)


def main(name):
    p = WORKLOADS[name]()
    g = O.make_grid(p["n"], p["lo"], p["hi"], p["order"], p["bc"], p["punctures"])
    t0 = time.perf_counter()
    r = O.solve(g, p["rho0"], p["rho2"], p["S"], p["kmode"], K2=p["K"] ** 2, tol=0.0, max_outer=80)
    secs = time.perf_counter() - t0
    assert r["status"] in ("floor", "converged"), r["status"]
    assert np.abs(r["u"]).max() < 0.5, "oracle left the psi ~ 1 branch"
    u, W = r["u"], r["W"]
    X, Y, Z = fields.cell_centres(p["n"], p["lo"], p["hi"])
    psi = 1.0 + u
    for pun in p["punctures"]:
        m, x = pun[0], pun[1]
        psi = psi + m / (2.0 * np.sqrt((X - x[0]) ** 2 + (Y - x[1]) ** 2 + (Z - x[2]) ** 2))
    cells = sample_cells(u.shape, [u, W[0], W[1], W[2]])
    flat = lambda a: a.reshape(-1)[cells].tolist()
    out = {
        "workload": name,
        "source": "oracle/ctt_oracle.c solve to its FP64 floor (tol = 0), written by tests/golden/make_oracle_roots.py",
        "n": list(p["n"]), "lo": p["lo"], "hi": p["hi"], "order": p["order"], "bc": p["bc"],
        "K2": r["K2"], "oracle_iters": r["iters"], "oracle_status": r["status"],
        "oracle_final_norms": r["hist"][-1].tolist(), "oracle_seconds": secs,
        "oracle_history": r["hist"].tolist(),
        "max_abs": {"psi": float(np.abs(psi).max()), "u": float(np.abs(u).max()), "Wx": float(np.abs(W[0]).max()),
                    "Wy": float(np.abs(W[1]).max()), "Wz": float(np.abs(W[2]).max())},
        "cells": cells,
        "u": flat(u), "Wx": flat(W[0]), "Wy": flat(W[1]), "Wz": flat(W[2]),
    }
    with open(os.path.join(HERE, name + "_oracle_root.json"), "w") as f:
        json.dump(out, f)
    print(name, r["status"], r["iters"], "%.1f s" % secs, r["hist"][-1])


if __name__ == "__main__":
    main(sys.argv[1])
