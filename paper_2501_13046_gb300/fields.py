"""Seeded synthetic matter configurations (inputs only).

This module turns seeded scalar-field data (phi, Pi) into the matter sources the
constraint solve takes as input: rho0 = Pi^2/2 + V(phi), rho2 = |d phi|^2/2 (so
that rho = rho0 + psi^-4 rho2 with the conformally flat metric) and the
lower-index momentum density S_i = -Pi d_i phi.  Derivatives of phi are
analytic.  It holds none of the solver's arithmetic and is shared by the tests,
the benchmark and the oracle checks.  Arrays are float64 with shape
(nz, ny, nx), x fastest.

The paper's setups are periodic cosmological spacetimes and black holes with
general scalar-field matter (Key features, "Flexibility"; "Initial conditions"
for analytic matter data).  The concrete workloads below:

* ``uniform``        -- constant rho0, no momentum: psi = 1, W = 0, K^2 = 24 pi rho0.
* ``sine_periodic``  -- L = 16 periodic cube, phi = 0.1 sin(2 pi x/L), Pi = 0.05 sin(2 pi y/L),
                        V = m^2 phi^2 / 2, m = 1, 2nd order, K from integrability.
* ``modes_periodic`` -- L = 32 periodic cube, phi = phi0 + sum of 16 seeded Fourier modes with
                        |k| <= 4 (2 pi/L), amplitude a0/|k| and uniform phases; Pi likewise
                        without offset; phi0 = 1, m = 1, 4th order.  a0 defaults to 5e-5: with
                        a constant K the Hamiltonian constraint is only well posed for weak
                        inhomogeneity (the linearised operator turns indefinite once
                        10 pi max(rho0 - <rho>) exceeds (2 pi/L)^2), so the prefactor 0.05 is
                        scaled by 1e-3.
* ``puncture_shell`` -- box [-64, 64]^3, Robin 1/r boundaries, one bare puncture M = 1 at the
                        origin, phi = A exp(-(r - 10)^2/4), Pi = 0.01 phi, V = phi^2/2, K = 0,
                        4th order.  A defaults to 0.02: for A >= 0.03 the constant-K Hamiltonian
                        constraint has no solution on the psi >= 1 branch.
* ``batch_sizes``    -- seeded grid sizes and amplitudes for the batched periodic workload.
"""
import numpy as np

PERIODIC, ROBIN = 0, 1
K_FIXED, K_INTEGRABILITY = 0, 1


def _rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def cell_centres(n, lo, hi):
    """Cell-centre coordinate arrays X, Y, Z of shape (nz, ny, nx)."""
    n = [n] * 3 if np.isscalar(n) else list(n)
    lo = [lo] * 3 if np.isscalar(lo) else list(lo)
    hi = [hi] * 3 if np.isscalar(hi) else list(hi)
    ax = [lo[a] + (np.arange(n[a]) + 0.5) * (hi[a] - lo[a]) / n[a] for a in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return X, Y, Z


def _problem(name, n, lo, hi, order, bc, kmode, K, punctures, rho0, rho2, S, **meta):
    arr = (lambda a: a) if hasattr(rho0, "is_cuda") else np.ascontiguousarray
    return dict(name=name, n=[n] * 3 if np.isscalar(n) else list(n), lo=lo, hi=hi, order=order, bc=bc,
                kmode=kmode, K=K, punctures=list(punctures), rho0=arr(rho0), rho2=arr(rho2), S=arr(S), meta=meta)


def scalar_sources(phi, dphi, Pi, m=1.0):
    """rho0, rho2, S for a scalar field with V = m^2 phi^2 / 2."""
    rho0 = 0.5 * Pi * Pi + 0.5 * m * m * phi * phi
    rho2 = 0.5 * (dphi[0] ** 2 + dphi[1] ** 2 + dphi[2] ** 2)
    S = np.stack([-Pi * dphi[a] for a in range(3)])
    return rho0, rho2, S


def uniform(n=16, L=16.0, rho=1e-3, order=2):
    X, _, _ = cell_centres(n, 0.0, L)
    rho0 = np.full(X.shape, rho)
    z = np.zeros(X.shape)
    return _problem("uniform", n, 0.0, L, order, PERIODIC, K_INTEGRABILITY, 0.0, (), rho0, z, np.stack([z, z, z]))


def sine_periodic(n=32, L=16.0, order=2):
    X, Y, _ = cell_centres(n, 0.0, L)
    k = 2.0 * np.pi / L
    phi = 0.1 * np.sin(k * X)
    Pi = 0.05 * np.sin(k * Y)
    dphi = [0.1 * k * np.cos(k * X), np.zeros_like(X), np.zeros_like(X)]
    rho0, rho2, S = scalar_sources(phi, dphi, Pi)
    return _problem("sine_periodic", n, 0.0, L, order, PERIODIC, K_INTEGRABILITY, 0.0, (), rho0, rho2, S)


def mode_vectors(numax=4):
    """Integer vectors 0 < |nu| <= numax, one of each +-pair (first nonzero component > 0)."""
    out = []
    for a in range(-numax, numax + 1):
        for b in range(-numax, numax + 1):
            for c in range(-numax, numax + 1):
                if (a, b, c) == (0, 0, 0) or a * a + b * b + c * c > numax * numax:
                    continue
                first = next(v for v in (a, b, c) if v != 0)
                if first > 0:
                    out.append((a, b, c))
    return np.array(out, dtype=np.float64)


def draw_modes(seed, L, a0, count=16, numax=4):
    """[(k vector, amplitude, phase)] for `count` distinct modes drawn with `seed`."""
    rng = _rng(seed)
    cand = mode_vectors(numax)
    pick = rng.choice(len(cand), size=count, replace=False)
    phase = rng.uniform(0.0, 2.0 * np.pi, size=count)
    modes = []
    for i, th in zip(pick, phase):
        kv = 2.0 * np.pi * cand[i] / L
        modes.append((kv, a0 / np.linalg.norm(kv), th))
    return modes


def modes_periodic(n=128, L=32.0, seed_phi=2, seed_pi=3, a0=5e-5, phi0=1.0, order=4, m=1.0):
    X, Y, Z = cell_centres(n, 0.0, L)
    phi = np.full(X.shape, phi0)
    dphi = [np.zeros_like(X) for _ in range(3)]
    for kv, A, th in draw_modes(seed_phi, L, a0):
        arg = kv[0] * X + kv[1] * Y + kv[2] * Z + th
        phi += A * np.cos(arg)
        s = np.sin(arg)
        for a in range(3):
            dphi[a] -= A * kv[a] * s
    Pi = np.zeros_like(X)
    for kv, A, th in draw_modes(seed_pi, L, a0):
        Pi += A * np.cos(kv[0] * X + kv[1] * Y + kv[2] * Z + th)
    rho0, rho2, S = scalar_sources(phi, dphi, Pi, m)
    return _problem("modes_periodic", n, 0.0, L, order, PERIODIC, K_INTEGRABILITY, 0.0, (), rho0, rho2, S,
                    seed_phi=seed_phi, seed_pi=seed_pi, a0=a0, phi0=phi0)


def puncture_shell(n=256, half=64.0, A=0.02, mass=1.0, order=4):
    X, Y, Z = cell_centres(n, -half, half)
    r = np.sqrt(X * X + Y * Y + Z * Z)
    phi = A * np.exp(-((r - 10.0) ** 2) / 4.0)
    dphidr = -phi * (r - 10.0) / 2.0
    dphi = [dphidr * X / r, dphidr * Y / r, dphidr * Z / r]
    Pi = 0.01 * phi
    rho0, rho2, S = scalar_sources(phi, dphi, Pi)
    return _problem("puncture_shell", n, -half, half, order, ROBIN, K_FIXED, 0.0, [(mass, (0.0, 0.0, 0.0))],
                    rho0, rho2, S, A=A)


def bowen_york_binary(n=128, half=16.0, d=3.0, mass=0.5, P=0.2, S=0.1, A=0.01, order=4):
    """Two Bowen-York punctures (Key features, "Flexibility": boosted and/or spinning black holes)
    of bare mass `mass` at (+-d, 0, 0) with momenta (0, +-P, 0) (an orbiting pair) and equal spins
    (0, 0, S), in [-half, half]^3 with Robin boundaries and K = 0, plus a scalar shell
    phi = A exp(-(r - 8)^2 / 4), Pi = 0.01 phi around the origin so that the momentum sources are
    not zero.  The punctures sit on cell faces when d / h is an integer (never on a cell centre)."""
    X, Y, Z = cell_centres(n, -half, half)
    r = np.sqrt(X * X + Y * Y + Z * Z)
    phi = A * np.exp(-((r - 8.0) ** 2) / 4.0)
    dphidr = -phi * (r - 8.0) / 2.0
    dphi = [dphidr * X / r, dphidr * Y / r, dphidr * Z / r]
    Pi = 0.01 * phi
    rho0, rho2, Ssrc = scalar_sources(phi, dphi, Pi)
    punct = [(mass, (d, 0.0, 0.0), (0.0, P, 0.0), (0.0, 0.0, S)),
             (mass, (-d, 0.0, 0.0), (0.0, -P, 0.0), (0.0, 0.0, S))]
    return _problem("bowen_york_binary", n, -half, half, order, ROBIN, K_FIXED, 0.0, punct, rho0, rho2, Ssrc, A=A)


def octant(problem):
    """The upper octant x, y, z > 0 of a problem on a box [-L, L]^3 (n even) that is symmetric
    under the three reflections (u, rho even; S_i odd in x_i): the same sources on [0, L]^3 at n/2
    cells per axis, with the three lower faces marked as symmetry planes (reflect = 7)."""
    n = problem["n"]
    assert all(m % 2 == 0 for m in n) and problem["bc"] == ROBIN
    hi = problem["hi"]
    cut = lambda a: np.ascontiguousarray(a[..., n[2] // 2:, n[1] // 2:, n[0] // 2:])
    out = _problem(problem["name"] + "_octant", [m // 2 for m in n], 0.0, hi, problem["order"], ROBIN,
                   problem["kmode"], problem["K"], problem["punctures"], cut(problem["rho0"]), cut(problem["rho2"]),
                   cut(problem["S"]), **problem["meta"])
    out["reflect"] = 7
    return out


def batch_sizes(count=64, sizes=(48, 64, 96, 128, 160), base_seed=4000, a_lo=2e-5, a_hi=8e-5):
    """[(n_b, a0_b, seed_b)]: n_b uniform over `sizes`, a0_b uniform in [a_lo, a_hi]."""
    out = []
    for b in range(count):
        rng = _rng(base_seed + b)
        n = int(sizes[rng.integers(len(sizes))])
        a0 = float(rng.uniform(a_lo, a_hi))
        out.append((n, a0, base_seed + b))
    return out


def batch_instance(n, a0, seed, L=32.0, order=4, device=None):
    """One instance of the batched workload: modes_periodic with its own seeds and amplitude
    (evaluated on `device` with torch when given)."""
    if device is not None:
        return modes_periodic_device(n=n, L=L, seed_phi=2 * seed, seed_pi=2 * seed + 1, a0=a0, order=order,
                                     device=device)
    return modes_periodic(n=n, L=L, seed_phi=2 * seed, seed_pi=2 * seed + 1, a0=a0, order=order)


def modes_periodic_device(n=128, L=32.0, seed_phi=2, seed_pi=3, a0=5e-5, phi0=1.0, order=4, m=1.0, device="cuda"):
    """modes_periodic evaluated with torch float64 on a device (same seeded modes and formulas);
    for large batches, where host evaluation would dominate.  Returns the same dict with torch
    tensors for rho0, rho2 and S."""
    import torch
    ax = (torch.arange(n, dtype=torch.float64, device=device) + 0.5) * (L / n)
    Z, Y, X = torch.meshgrid(ax, ax, ax, indexing="ij")
    phi = torch.full_like(X, phi0)
    dphi = [torch.zeros_like(X) for _ in range(3)]
    for kv, A, th in draw_modes(seed_phi, L, a0):
        arg = kv[0] * X + kv[1] * Y + kv[2] * Z + th
        phi += A * torch.cos(arg)
        s = torch.sin(arg)
        for a in range(3):
            dphi[a] -= A * kv[a] * s
    Pi = torch.zeros_like(X)
    for kv, A, th in draw_modes(seed_pi, L, a0):
        Pi += A * torch.cos(kv[0] * X + kv[1] * Y + kv[2] * Z + th)
    rho0 = 0.5 * Pi * Pi + 0.5 * m * m * phi * phi
    rho2 = 0.5 * (dphi[0] ** 2 + dphi[1] ** 2 + dphi[2] ** 2)
    S = torch.stack([-Pi * dphi[a] for a in range(3)]).contiguous()
    return _problem("modes_periodic", n, 0.0, L, order, PERIODIC, K_INTEGRABILITY, 0.0, (), rho0.contiguous(),
                    rho2.contiguous(), S, seed_phi=seed_phi, seed_pi=seed_pi, a0=a0, phi0=phi0)
