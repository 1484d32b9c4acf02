"""ctypes wrapper around the plain FP64 CPU oracle (ctt_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
CPU-baseline leg of the benchmark, never by the product package.  The C file is
compiled here with gcc (``build()``); it shares no code with the CUDA library.

Every function takes and returns numpy float64 arrays in the library's layout:
one array per field, x fastest, shape (nz, ny, nx) when viewed as 3-D.
The equations are those of the Hamiltonian and momentum constraints
(eq:Ham, eq:Mom) in the CTT form spelled out in ctt_oracle.c.
"""
import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "ctt_oracle.c")
LIB = os.path.join(HERE, "libctt_oracle.so")

PERIODIC, ROBIN = 0, 1
K_FIXED, K_INTEGRABILITY = 0, 1
STATUS = {0: "converged", 1: "floor", 2: "max_outer", 3: "non_finite", -1: "bad_args"}


class Grid(C.Structure):
    _fields_ = [
        ("n", C.c_int * 3),
        ("lo", C.c_double * 3),
        ("h", C.c_double * 3),
        ("order", C.c_int),
        ("bc", C.c_int),
        ("npunct", C.c_int),
        ("pm", C.c_double * 2),
        ("px", (C.c_double * 3) * 2),
        ("pP", (C.c_double * 3) * 2),
        ("pS", (C.c_double * 3) * 2),
        ("reflect", C.c_int),
        ("extrap", C.c_int),
    ]


def build(force=False):
    """Compile the oracle into a shared library next to its source."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", "-o", tmp, SRC, "-lm"])
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        dp = C.POINTER(C.c_double)
        gp = C.POINTER(Grid)
        L.ora_d1.argtypes = [gp, C.c_int, dp, dp]
        L.ora_d2.argtypes = [gp, C.c_int, dp, dp]
        L.ora_dmix.argtypes = [gp, C.c_int, C.c_int, dp, dp]
        L.ora_lap.argtypes = [gp, dp, dp]
        L.ora_atat.argtypes = [gp, dp, dp]
        L.ora_boundary_value.argtypes = [gp, C.c_int, dp, C.c_int, C.c_int, C.c_int]
        L.ora_boundary_value.restype = C.c_double
        L.ora_by_point.argtypes = [gp, dp, dp]
        L.ora_by_cells.argtypes = [gp, dp]
        L.ora_restrict.argtypes = [gp, dp, dp]
        L.ora_prolong_add.argtypes = [gp, C.c_int, dp, dp]
        L.ora_residual.argtypes = [gp, dp, dp, dp, dp, dp, C.c_int, dp, dp, dp, dp, dp, dp, dp, dp]
        L.ora_residual.restype = C.c_int
        L.ora_auto_levels.argtypes = [C.POINTER(C.c_int)]
        L.ora_auto_levels.restype = C.c_int
        L.ora_solve.argtypes = [gp, dp, dp, dp, C.c_int, dp, C.c_double, C.c_int, C.c_int, C.c_int, C.c_int,
                                C.c_int, dp, dp, dp, C.POINTER(C.c_int)]
        L.ora_solve.restype = C.c_int
        L.ora_set_threads.argtypes = [C.c_int]
        L.ora_set_threads.restype = C.c_int
        _lib = L
    return _lib


def make_grid(n, lo, hi, order, bc, punctures=(), reflect=0, extrap=0):
    """n: int or 3 ints; lo/hi: float or 3 floats; punctures: [(mass, (x, y, z)), ...] or, with
    Bowen-York momentum and spin, [(mass, (x, y, z), (Px, Py, Pz), (Sx, Sy, Sz)), ...];
    reflect (Robin boxes): bit a makes the lower face x_a = 0 a reflection-symmetry plane;
    extrap (Robin boxes): bit 2a (lower) or 2a + 1 (upper) makes that face of axis a extrapolating."""
    n = [n] * 3 if np.isscalar(n) else list(n)
    lo = [lo] * 3 if np.isscalar(lo) else list(lo)
    hi = [hi] * 3 if np.isscalar(hi) else list(hi)
    g = Grid()
    for a in range(3):
        g.n[a] = int(n[a])
        g.lo[a] = float(lo[a])
        g.h[a] = (float(hi[a]) - float(lo[a])) / int(n[a])
    g.order, g.bc, g.npunct, g.reflect, g.extrap = int(order), int(bc), len(punctures), int(reflect), int(extrap)
    for p, pun in enumerate(punctures):
        m, x = pun[0], pun[1]
        P = pun[2] if len(pun) > 2 else (0.0, 0.0, 0.0)
        S = pun[3] if len(pun) > 3 else (0.0, 0.0, 0.0)
        g.pm[p] = float(m)
        for a in range(3):
            g.px[p][a] = float(x[a])
            g.pP[p][a] = float(P[a])
            g.pS[p][a] = float(S[a])
    return g


def set_threads(n=0):
    """Threads of the oracle's OpenMP loops (n <= 0 leaves the count); returns the count in effect."""
    return lib().ora_set_threads(int(n))


def by_point(g, x):
    """3x3 Bowen-York conformal extrinsic curvature of g's punctures at the point x."""
    out = np.empty(9)
    xs = np.ascontiguousarray(x, dtype=np.float64)
    lib().ora_by_point(C.byref(g), _p(xs), _p(out))
    return out.reshape(3, 3)


def by_cells(g):
    """Bowen-York curvature at every cell centre, shape (3, 3, nz, ny, nx)."""
    out = np.empty(9 * ncells(g))
    lib().ora_by_cells(C.byref(g), _p(out))
    return out.reshape((3, 3) + shape3(g))


def coarse(g, level=1):
    c = Grid()
    C.pointer(c)[0] = g
    for a in range(3):
        c.n[a] = g.n[a] >> level
        c.h[a] = g.h[a] * (1 << level)
    return c


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _arr(x, count):
    x = np.ascontiguousarray(x, dtype=np.float64)
    assert x.size == count, (x.size, count)
    return x


def ncells(g):
    return g.n[0] * g.n[1] * g.n[2]


def shape3(g):
    return (g.n[2], g.n[1], g.n[0])


def d1(g, axis, f):
    f = _arr(f, ncells(g)); out = np.empty_like(f)
    lib().ora_d1(C.byref(g), axis, _p(f), _p(out))
    return out


def d2(g, axis, f):
    f = _arr(f, ncells(g)); out = np.empty_like(f)
    lib().ora_d2(C.byref(g), axis, _p(f), _p(out))
    return out


def dmix(g, a, b, f):
    f = _arr(f, ncells(g)); out = np.empty_like(f)
    lib().ora_dmix(C.byref(g), a, b, _p(f), _p(out))
    return out


def lap(g, f):
    f = _arr(f, ncells(g)); out = np.empty_like(f)
    lib().ora_lap(C.byref(g), _p(f), _p(out))
    return out


def atat(g, W):
    W = _arr(W, 3 * ncells(g)); out = np.empty(ncells(g))
    lib().ora_atat(C.byref(g), _p(W), _p(out))
    return out.reshape(shape3(g))


def boundary_value(g, f, i, j, k, fi=0):
    """Value of field f (fi: 0 = u, 1..3 = W_x..W_z) at the cell (i, j, k), which may lie outside the box."""
    f = _arr(f, ncells(g))
    return lib().ora_boundary_value(C.byref(g), fi, _p(f), i, j, k)


def restrict(gc, fine):
    fine = _arr(fine, 8 * ncells(gc)); out = np.empty(ncells(gc))
    lib().ora_restrict(C.byref(gc), _p(fine), _p(out))
    return out.reshape(shape3(gc))


def prolong_add(gc, coarse_f, fine, fi=0):
    """fine + trilinear interpolation of coarse field fi (0 = u, 1..3 = W_x..W_z)."""
    coarse_f = _arr(coarse_f, ncells(gc))
    fine = np.array(fine, dtype=np.float64, copy=True).reshape(-1)
    assert fine.size == 8 * ncells(gc)
    lib().ora_prolong_add(C.byref(gc), fi, _p(coarse_f), _p(fine))
    return fine


def residual(g, u, W, rho0, rho2, S, kmode, K2=0.0):
    """Returns dict(Fpsi, FW, H, M, c, norms, K2, msrc); arrays shaped (nz, ny, nx) / (3, nz, ny, nx)."""
    N = ncells(g)
    u = _arr(u, N); W = _arr(W, 3 * N); rho0 = _arr(rho0, N); rho2 = _arr(rho2, N); S = _arr(S, 3 * N)
    Fp, H, c = np.empty(N), np.empty(N), np.empty(N)
    FW, M = np.empty(3 * N), np.empty(3 * N)
    norms, msrc = np.empty(4), np.empty(3)
    k2 = np.array([K2], dtype=np.float64)
    rc = lib().ora_residual(C.byref(g), _p(u), _p(W), _p(rho0), _p(rho2), _p(S), kmode, _p(k2), _p(Fp), _p(FW),
                            _p(H), _p(M), _p(c), _p(norms), _p(msrc))
    if rc != 0:
        raise MemoryError("oracle residual failed")
    s3 = shape3(g)
    return dict(Fpsi=Fp.reshape(s3), FW=FW.reshape((3,) + s3), H=H.reshape(s3), M=M.reshape((3,) + s3),
                c=c.reshape(s3), norms=norms, K2=float(k2[0]), msrc=msrc)


def auto_levels(n):
    arr = (C.c_int * 3)(*n)
    return lib().ora_auto_levels(arr)


def solve(g, rho0, rho2, S, kmode, K2=0.0, tol=0.0, max_outer=60, levels=0, nu1=2, nu2=2, csweeps=60,
          u0=None, W0=None):
    """Solve the discrete constraint system.  tol <= 0 iterates to the FP64 floor.

    Returns dict(u, W, K2, status, iters, hist) with hist[i] = (|H|, |Mx|, |My|, |Mz|) maxima.
    """
    N = ncells(g)
    rho0 = _arr(rho0, N); rho2 = _arr(rho2, N); S = _arr(S, 3 * N)
    u = np.zeros(N) if u0 is None else np.array(u0, dtype=np.float64).reshape(-1).copy()
    W = np.zeros(3 * N) if W0 is None else np.array(W0, dtype=np.float64).reshape(-1).copy()
    hist = np.zeros((max_outer + 1) * 4)
    k2 = np.array([K2], dtype=np.float64)
    it = C.c_int(0)
    st = lib().ora_solve(C.byref(g), _p(rho0), _p(rho2), _p(S), kmode, _p(k2), float(tol), int(max_outer),
                         int(levels), int(nu1), int(nu2), int(csweeps), _p(u), _p(W), _p(hist), C.byref(it))
    s3 = shape3(g)
    n_it = it.value
    return dict(u=u.reshape(s3), W=W.reshape((3,) + s3), K2=float(k2[0]), status=STATUS.get(st, st), iters=n_it,
                hist=hist.reshape(-1, 4)[: min(n_it, max_outer) + 1])
