"""Brute-force solve of the discrete CTT constraint system on tiny grids (dense Newton).

TEST INFRASTRUCTURE ONLY: used by the tests to pin the oracle's multigrid solve
(and, through the GPU tests, the CUDA library) to the exact root of the discrete
system.  It is an independent numpy restatement of the discrete equations: it
shares no code with ``ctt_oracle.c`` or with the CUDA library.

The system (Hamiltonian and momentum constraints, eq:Ham and eq:Mom, in the
conformal transverse-traceless form with gamma_ij = psi^4 delta_ij,
K_ij = psi^-2 At_ij + gamma_ij K/3, At_ij = D_i W_j + D_j W_i - (2/3) delta_ij D_k W_k):

    F_psi   = Lap u - (K^2/12) psi^5 + (1/8) psi^-7 AtAt + 2 pi (rho0 psi^5 + rho2 psi)
    F_W,i   = Lap W_i + (1/3) D_ii W_i + (1/3) sum_{j != i} D_i D_j W_j - (8 pi psi^6 S_i - m_i)
    psi     = 1 + sum_p m_p / (2 |x - x_p|) + u,   m_i = <8 pi psi^6 S_i> (periodic), 0 otherwise

on a cell-centred grid (x_i = lo + (i + 1/2) h) with the centred stencils of
order 2 or 4 (first derivative D_a, compact second derivative D_aa, mixed
D_a D_b as the tensor product of two first-derivative stencils), values outside
the box by periodic wrap or by the Robin 1/r rule v(g) = v(clamp(g)) |x_clamp| / |x_g|
(beyond an extrapolating face of a Robin box: first the linear extrapolation
(1 + d) v(boundary cell) - d v(its inner neighbour) along that face's normal, d the
distance), and, with punctures, the Bowen-York curvature added to At_ij before AtAt.

Every operator is assembled as a dense matrix (one row per cell, entries from
the stencil weights and the boundary rule), the Jacobian is formed
analytically, and Newton's method is run with LAPACK solves until the residual
stops decreasing.  Periodic boxes: K^2 is an unknown and the gauge <u> = 0,
<W_i> = 0 borders the system (with one multiplier per momentum component, which
vanishes at the root because the momentum source's mean is removed).  Intended
for grids of at most ~10^3 cells.
"""
import numpy as np

PERIODIC, ROBIN = 0, 1

_D1 = {2: {-1: -0.5, 1: 0.5}, 4: {-2: 1.0 / 12, -1: -8.0 / 12, 1: 8.0 / 12, 2: -1.0 / 12}}
_D2 = {2: {-1: 1.0, 0: -2.0, 1: 1.0}, 4: {-2: -1.0 / 12, -1: 16.0 / 12, 0: -30.0 / 12, 1: 16.0 / 12, 2: -1.0 / 12}}


class DenseSystem:
    """The discrete constraint system of one problem on a small grid, with dense operators."""

    def __init__(self, n, lo, hi, order, bc, punctures=(), rho0=None, rho2=None, S=None, K2=0.0,
                 k_from_integrability=True, extrap=0):
        self.n = [n] * 3 if np.isscalar(n) else list(n)
        lo = [lo] * 3 if np.isscalar(lo) else list(lo)
        hi = [hi] * 3 if np.isscalar(hi) else list(hi)
        self.lo = np.array(lo, dtype=float)
        self.h = np.array([(hi[a] - lo[a]) / self.n[a] for a in range(3)])
        self.order, self.bc = order, bc
        self.extrap = int(extrap)   # bit 2a (lower) / 2a + 1 (upper): extrapolating face of axis a
        self.periodic = bc == PERIODIC
        self.kint = self.periodic and k_from_integrability
        assert self.kint or not self.periodic, "periodic boxes take K^2 from the integrability condition"
        self.K2 = float(K2)
        self.N = N = self.n[0] * self.n[1] * self.n[2]
        nx, ny, nz = self.n
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        self.idx = np.stack([i.reshape(-1), j.reshape(-1), k.reshape(-1)])   # (3, N) cell indices
        self.x = self.lo[:, None] + (self.idx + 0.5) * self.h[:, None]       # (3, N) cell centres
        self.punct = [tuple(p) for p in punctures]
        psibg = np.ones(N)
        for p in self.punct:
            psibg += p[0] / (2.0 * np.linalg.norm(self.x - np.array(p[1], dtype=float)[:, None], axis=0))
        self.psibg = psibg
        self.B = self._bowen_york()
        self.rho0 = np.asarray(rho0, dtype=float).reshape(-1)
        self.rho2 = np.asarray(rho2, dtype=float).reshape(-1)
        self.S = np.asarray(S, dtype=float).reshape(3, N)
        # operators
        self.D1 = [self._stencil(_D1[order], a) for a in range(3)]
        self.D2 = [self._stencil(_D2[order], a, second=True) for a in range(3)]
        self.Lap = self.D2[0] + self.D2[1] + self.D2[2]
        self.Dmix = [[None] * 3 for _ in range(3)]
        for a in range(3):
            for b in range(3):
                if a != b:
                    self.Dmix[a][b] = self._mixed(a, b)

    # ------------------------------------------------------------ boundary rule and stencils
    def _sources(self, p):
        """[(cell index, factor)]: the value at the integer cells p (3, M) is the sum over the list
        of factor times the value at that cell (one term inside the box or under the Robin rule; the
        linear extrapolation through extrapolating faces splits a point in two per such axis)."""
        sets = [(p.copy(), np.ones(p.shape[1]))]
        if not self.periodic and self.extrap:
            for a in range(3):
                n, new = self.n[a], []
                for q, w in sets:
                    lo = (q[a] < 0) & bool((self.extrap >> (2 * a)) & 1)
                    hi = (q[a] >= n) & bool((self.extrap >> (2 * a + 1)) & 1)
                    d = np.where(lo, -q[a], np.where(hi, q[a] - (n - 1), 0))
                    q0, q1 = q.copy(), q.copy()
                    q0[a] = np.where(lo, 0, np.where(hi, n - 1, q[a]))
                    q1[a] = np.where(lo, 1, np.where(hi, n - 2, q[a]))
                    new += [(q0, w * (1.0 + d)), (q1, w * -d)]
                sets = new
        return [(lin, w * fac) for q, w in sets for lin, fac in [self._source(q)]]

    def _source(self, p):
        """(cell index, factor) whose value, times factor, is the value at integer cell p (3, M)."""
        n = np.array(self.n)[:, None]
        if self.periodic:
            b = np.mod(p, n)
            fac = np.ones(p.shape[1])
        else:
            b = np.clip(p, 0, n - 1)
            xb = self.lo[:, None] + (b + 0.5) * self.h[:, None]
            xg = self.lo[:, None] + (p + 0.5) * self.h[:, None]
            fac = np.where((b != p).any(axis=0),
                           np.linalg.norm(xb, axis=0) / np.linalg.norm(xg, axis=0), 1.0)
        lin = b[0] + self.n[0] * (b[1] + self.n[1] * b[2])
        return lin, fac

    def _add(self, M, offset, weight):
        p = self.idx + np.array(offset)[:, None]
        for lin, fac in self._sources(p):
            np.add.at(M, (np.arange(self.N), lin), weight * fac)

    def _stencil(self, weights, a, second=False):
        M = np.zeros((self.N, self.N))
        scale = 1.0 / (self.h[a] ** 2 if second else self.h[a])
        for s, w in weights.items():
            off = [0, 0, 0]
            off[a] = s
            self._add(M, off, w * scale)
        return M

    def _mixed(self, a, b):
        M = np.zeros((self.N, self.N))
        w1 = _D1[self.order]
        for s, ws in w1.items():
            for t, wt in w1.items():
                off = [0, 0, 0]
                off[a] += s
                off[b] += t
                self._add(M, off, ws * wt / (self.h[a] * self.h[b]))
        return M

    def _bowen_york(self):
        """Bowen-York curvature of the punctures at every cell centre, (3, 3, N)."""
        B = np.zeros((3, 3, self.N))
        for p in self.punct:
            P = np.array(p[2] if len(p) > 2 else (0, 0, 0), dtype=float)
            Sp = np.array(p[3] if len(p) > 3 else (0, 0, 0), dtype=float)
            d = self.x - np.array(p[1], dtype=float)[:, None]
            r = np.linalg.norm(d, axis=0)
            nv = d / r
            Pn = P @ nv
            Sxn = np.cross(Sp[:, None], nv, axis=0)
            for a in range(3):
                for b in range(3):
                    B[a, b] += 1.5 / r ** 2 * (P[a] * nv[b] + P[b] * nv[a] - ((a == b) - nv[a] * nv[b]) * Pn) \
                        + 3.0 / r ** 3 * (Sxn[a] * nv[b] + Sxn[b] * nv[a])
        return B

    # ------------------------------------------------------------ residual and Jacobian
    def parts(self, u, W):
        psi = self.psibg + u
        G = np.array([[self.D1[a] @ W[b] for b in range(3)] for a in range(3)])   # G[a, b] = D_a W_b
        div = G[0, 0] + G[1, 1] + G[2, 2]
        At = G + G.transpose(1, 0, 2) - (2.0 / 3.0) * np.eye(3)[:, :, None] * div + self.B
        return psi, At, (At * At).sum(axis=(0, 1))

    def residual(self, u, W, K2):
        psi, At, aa = self.parts(u, W)
        Fp = self.Lap @ u - K2 / 12.0 * psi ** 5 + aa / 8.0 * psi ** -7 + 2 * np.pi * (self.rho0 * psi ** 5 + self.rho2 * psi)
        src = 8 * np.pi * psi ** 6 * self.S
        m = src.mean(axis=1) if self.periodic else np.zeros(3)
        FW = np.empty((3, self.N))
        for i in range(3):
            v = self.Lap @ W[i] + self.D2[i] @ W[i] / 3.0
            for j in range(3):
                if j != i:
                    v = v + self.Dmix[i][j] @ W[j] / 3.0
            FW[i] = v - (src[i] - m[i])
        return Fp, FW

    def jacobian(self, u, W, K2):
        """d(F_psi, F_W) / d(u, W) (4N x 4N) and d F_psi / d K^2 (N)."""
        N = self.N
        psi, At, aa = self.parts(u, W)
        J = np.zeros((4 * N, 4 * N))
        c = -5.0 / 12.0 * K2 * psi ** 4 - 7.0 / 8.0 * psi ** -8 * aa + 2 * np.pi * (5 * self.rho0 * psi ** 4 + self.rho2)
        J[:N, :N] = self.Lap + np.diag(c)
        tr = At[0, 0] + At[1, 1] + At[2, 2]
        for j in range(3):
            daa = sum(4.0 * At[a, j][:, None] * self.D1[a] for a in range(3)) - (4.0 / 3.0) * tr[:, None] * self.D1[j]
            J[:N, N * (1 + j):N * (2 + j)] = (psi ** -7 / 8.0)[:, None] * daa
        for i in range(3):
            dsrc = 8 * np.pi * 6 * psi ** 5 * self.S[i]
            blk = -np.diag(dsrc)
            if self.periodic:
                blk = blk + np.ones((N, 1)) * (dsrc / N)[None, :]
            J[N * (1 + i):N * (2 + i), :N] = blk
            for j in range(3):
                blk = self.Lap + self.D2[i] / 3.0 if i == j else self.Dmix[i][j] / 3.0
                J[N * (1 + i):N * (2 + i), N * (1 + j):N * (2 + j)] = blk
        return J, -psi ** 5 / 12.0

    # ------------------------------------------------------------ Newton
    def solve(self, max_iter=40, u0=None, W0=None):
        """Newton's method to the FP64 floor.  Returns dict(u, W, K2, norms, iters, history)."""
        N = self.N
        u = np.zeros(N) if u0 is None else np.array(u0, dtype=float).reshape(-1)
        W = np.zeros((3, N)) if W0 is None else np.array(W0, dtype=float).reshape(3, N)
        K2 = 24 * np.pi * float(np.mean(self.rho0 + self.rho2)) if self.kint else self.K2
        mu = np.zeros(3)
        hist = []
        best = None
        for it in range(max_iter):
            Fp, FW = self.residual(u, W, K2)
            res = max(np.abs(Fp).max(), np.abs(FW + mu[:, None]).max())
            hist.append(res)
            if best is None or res < best[0]:
                best = (res, u.copy(), W.copy(), K2, it)
            if it >= 3 and res >= 0.5 * hist[-2] and res < 1e-11:
                break
            J, dK = self.jacobian(u, W, K2)
            if self.periodic:
                m = 4 * N + 4
                A = np.zeros((m, m))
                A[:4 * N, :4 * N] = J
                rhs = np.zeros(m)
                rhs[:N] = -Fp
                rhs[N:4 * N] = -(FW + mu[:, None]).reshape(-1)
                A[:N, 4 * N] = dK                      # column 4N: the unknown K^2
                # gauge rows: sum u = 0 (row 4N), sum W_i = 0 (rows 4N+1..4N+3)
                A[4 * N, :N] = 1.0
                rhs[4 * N] = -u.sum()
                for i in range(3):
                    A[4 * N + 1 + i, N * (1 + i):N * (2 + i)] = 1.0
                    A[N * (1 + i):N * (2 + i), 4 * N + 1 + i] = 1.0
                    rhs[4 * N + 1 + i] = -W[i].sum()
                d = np.linalg.solve(A, rhs)
                u = u + d[:N]
                W = W + d[N:4 * N].reshape(3, N)
                K2 = K2 + d[4 * N]
                mu = mu + d[4 * N + 1:]
            else:
                d = np.linalg.solve(J, -np.concatenate([Fp, FW.reshape(-1)]))
                u = u + d[:N]
                W = W + d[N:].reshape(3, N)
        res, u, W, K2, it = best
        return dict(u=u, W=W, K2=K2, residual=res, iters=it, history=hist, multipliers=mu)
