/*
 * ctt_oracle.c -- plain, slow FP64 CPU oracle for the CTT constraint solve.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * What it computes (GRTresna, arXiv:2501.13046):
 *   - the Hamiltonian constraint H = R + K^2 - K_ij K^ij - 16 pi rho (eq:Ham)
 *   - the momentum constraint  M_i = D^j(K_ij - gamma_ij K) - 8 pi S_i (eq:Mom)
 *   with the matter projections rho, S_i as inputs (Summary, after eq:Mom),
 *   in the conformal transverse-traceless (CTT) family that the paper's CTTK
 *   methods belong to (Summary; Key features, "Methods"):
 *     gamma_ij = psi^4 delta_ij,  K_ij = psi^-2 At_ij + gamma_ij K / 3,
 *     At_ij = d_i W_j + d_j W_i - (2/3) delta_ij d_k W_k,  K constant.
 *   Then eq:Ham times (-psi^5/8) is
 *     F_psi = Lap psi - (K^2/12) psi^5 + (1/8) psi^-7 AtAt + 2 pi (rho0 psi^5 + rho2 psi)
 *   (rho = rho0 + psi^-4 rho2 splits off the gradient energy of a scalar field),
 *   H = -8 psi^-5 F_psi, and eq:Mom is
 *     F_W,i = Lap W_i + (1/3) d_i d_j W_j - 8 pi (psi^6 S_i - m_i),  M_i = psi^-6 F_W,i
 *   with m_i = <8 pi psi^6 S_i> on periodic boxes (0 otherwise).
 *   psi = 1 + sum_p m_p / (2 |x - x_p|) + u; the Laplacian acts on u only.
 *   Punctures may carry Bowen-York momentum P and spin S (Key features, "Flexibility": boosted
 *   and/or spinning black holes): their analytic conformal extrinsic curvature
 *     Ab_ij = 3/(2 r^2) [P_i n_j + P_j n_i - (delta_ij - n_i n_j) P.n] + 3/r^3 [(S x n)_i n_j + (S x n)_j n_i]
 *   (n the unit vector from the puncture, r the distance; a vacuum solution of the momentum
 *   constraint, traceless and divergence-free away from the puncture, whose ADM momentum is P and
 *   ADM angular momentum S) is added to At_ij before AtAt is formed; F_W is unchanged.
 *   On periodic boxes K^2 is set by the exact discrete integrability
 *   sum_cells F_psi = 0, and the gauge is <u> = 0, <W_i> = 0.
 *
 * Discretisation (2nd or 4th order, cell-centred, x_i = lo + (i+1/2) h):
 *   D_a   : (f+1 - f-1)/2h            | (-f+2 + 8f+1 - 8f-1 + f-2)/12h
 *   D_aa  : (f+1 - 2f + f-1)/h^2      | (-f+2 + 16f+1 - 30f + 16f-1 - f-2)/12h^2
 *   D_ab  : D_a applied to D_b (a != b);  Lap = sum_a D_aa
 *   Boundary values outside the box: periodic wrap, or Robin 1/r falloff
 *   v(g) = v(b) |x_b| / |x_g| with b the cell obtained by clamping g into the box.  On a Robin box
 *   a lower face x_a = 0 may instead be a reflection-symmetry plane (Key features, "Boundary
 *   conditions": reflective): below it g_a -> -1 - g_a (the mirror cell), with the sign of W_a,
 *   the component normal to the plane, flipped and every other field kept.  A face of a Robin box
 *   may instead be extrapolating (same passage: extrapolating): a cell beyond it at distance
 *   d (1 or 2) along the face normal takes the linear extrapolation through the two nearest cells
 *   of its line, v = (1 + d) v(b) - d v(b'), b the boundary cell and b' its inner neighbour;
 *   extrapolating axes are resolved first (the rule is linear, so their order does not matter), then
 *   the remaining coordinates by the rules above.
 *
 * Solver (any convergent method reaches the same discrete solution): an outer
 * defect-correction loop in FP64 (residual, integrability K^2, norms), with an
 * inner linear multigrid V-cycle on the block-diagonal linearisation
 *   (Lap + c) e = -F_psi,  (Lap + (1/3) grad div) e_W = -F_W,
 *   c = dF_psi/du = -(5/12) K^2 psi^4 - (7/8) psi^-8 AtAt + 2 pi (5 rho0 psi^4 + rho2),
 * with the psi row scaled by psi^-5 (so that the K^2 direction is a constant), smoothed by
 * sequential lexicographic Gauss-Seidel, with an exact bordered solve of the psi row on the
 * coarsest level; restriction is the mean of the 8 children, prolongation is cell-centred
 * trilinear (3/4, 1/4 per axis).
 * This is the multigrid family the paper names (Key features, "Fast").
 *
 * Arrays are x-fastest, index i + nx (j + ny k), no ghost cells.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_PI 3.14159265358979323846

typedef struct {
    int n[3];
    double lo[3];
    double h[3];
    int order;       /* 2 or 4 */
    int bc;          /* 0 = periodic, 1 = Robin 1/r */
    int npunct;      /* 0, 1 or 2 punctures (Robin boxes only) */
    double pm[2];
    double px[2][3];
    double pP[2][3]; /* Bowen-York linear momentum of each puncture (0: bare) */
    double pS[2][3]; /* Bowen-York spin of each puncture (0: bare) */
    int reflect;     /* Robin boxes: bit a = the lower face of axis a (x_a = 0) is a symmetry plane */
    int extrap;      /* Robin boxes: bit 2a (lower) / 2a + 1 (upper) = that face of axis a is extrapolating */
} ora_grid;

static long ncells(const ora_grid *g) { return (long)g->n[0] * g->n[1] * g->n[2]; }

static long lin(const ora_grid *g, int i, int j, int k)
{
    return i + (long)g->n[0] * (j + (long)g->n[1] * k);
}

static double cellx(const ora_grid *g, int a, int i) { return g->lo[a] + (i + 0.5) * g->h[a]; }

/* Value of field f (fi: 0 = u, 1..3 = W_x..W_z) at integer cell (i,j,k), which may lie outside
 * the box. */
static double at(const ora_grid *g, int fi, const double *f, int i, int j, int k)
{
    int p[3] = {i, j, k};
    if (g->bc != 0 && g->extrap) {
        /* linear extrapolation through an extrapolating face, one axis at a time */
        for (int a = 0; a < 3; ++a) {
            int n = g->n[a], d = 0, b0 = 0, b1 = 0;
            if (p[a] < 0 && ((g->extrap >> (2 * a)) & 1)) {
                d = -p[a]; b0 = 0; b1 = 1;
            } else if (p[a] >= n && ((g->extrap >> (2 * a + 1)) & 1)) {
                d = p[a] - (n - 1); b0 = n - 1; b1 = n - 2;
            }
            if (d == 0) continue;
            int q0[3] = {p[0], p[1], p[2]}, q1[3] = {p[0], p[1], p[2]};
            q0[a] = b0;
            q1[a] = b1;
            return (1.0 + d) * at(g, fi, f, q0[0], q0[1], q0[2]) - d * at(g, fi, f, q1[0], q1[1], q1[2]);
        }
    }
    int b[3];
    int outside = 0;
    double sign = 1.0;
    for (int a = 0; a < 3; ++a) {
        int n = g->n[a];
        if (g->bc == 0) {
            b[a] = ((p[a] % n) + n) % n;
        } else if (p[a] < 0 && ((g->reflect >> a) & 1)) {
            b[a] = -1 - p[a];              /* mirror image across the plane x_a = 0 */
            if (fi == 1 + a) sign = -sign; /* the normal component of W is odd */
        } else {
            b[a] = p[a] < 0 ? 0 : (p[a] >= n ? n - 1 : p[a]);
            if (b[a] != p[a]) outside = 1;
        }
    }
    double v = sign * f[lin(g, b[0], b[1], b[2])];
    if (!outside) return v;
    double rb2 = 0.0, rg2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double xb = cellx(g, a, b[a]), xg = cellx(g, a, p[a]);
        rb2 += xb * xb;
        rg2 += xg * xg;
    }
    return v * sqrt(rb2) / sqrt(rg2);
}

/* f at (i,j,k) shifted by s along axis a and t along axis b */
static double at2(const ora_grid *g, int fi, const double *f, int i, int j, int k, int a, int s, int b, int t)
{
    int o[3] = {0, 0, 0};
    o[a] += s;
    o[b] += t;
    return at(g, fi, f, i + o[0], j + o[1], k + o[2]);
}

/* first-derivative weights w[s] for offsets s = -2..2 (index s+2), times 1/h */
static void d1_weights(int order, double w[5])
{
    if (order == 2) {
        double c[5] = {0.0, -0.5, 0.0, 0.5, 0.0};
        memcpy(w, c, sizeof c);
    } else {
        double c[5] = {1.0 / 12.0, -8.0 / 12.0, 0.0, 8.0 / 12.0, -1.0 / 12.0};
        memcpy(w, c, sizeof c);
    }
}

/* second-derivative weights, times 1/h^2 */
static void d2_weights(int order, double w[5])
{
    if (order == 2) {
        double c[5] = {0.0, 1.0, -2.0, 1.0, 0.0};
        memcpy(w, c, sizeof c);
    } else {
        double c[5] = {-1.0 / 12.0, 16.0 / 12.0, -30.0 / 12.0, 16.0 / 12.0, -1.0 / 12.0};
        memcpy(w, c, sizeof c);
    }
}

static double d1_at(const ora_grid *g, int fi, const double *f, int a, int i, int j, int k)
{
    double w[5], s = 0.0;
    d1_weights(g->order, w);
    for (int t = -2; t <= 2; ++t)
        if (w[t + 2] != 0.0) s += w[t + 2] * at2(g, fi, f, i, j, k, a, t, a, 0);
    return s / g->h[a];
}

static double d2_at(const ora_grid *g, int fi, const double *f, int a, int i, int j, int k)
{
    double w[5], s = 0.0;
    d2_weights(g->order, w);
    for (int t = -2; t <= 2; ++t)
        if (w[t + 2] != 0.0) s += w[t + 2] * at2(g, fi, f, i, j, k, a, t, a, 0);
    return s / (g->h[a] * g->h[a]);
}

/* D_a D_b f for a != b: tensor product of the two first-derivative stencils */
static double dmix_at(const ora_grid *g, int fi, const double *f, int a, int b, int i, int j, int k)
{
    double w[5], s = 0.0;
    d1_weights(g->order, w);
    for (int p = -2; p <= 2; ++p) {
        if (w[p + 2] == 0.0) continue;
        double inner = 0.0;
        for (int q = -2; q <= 2; ++q)
            if (w[q + 2] != 0.0) inner += w[q + 2] * at2(g, fi, f, i, j, k, a, p, b, q);
        s += w[p + 2] * inner;
    }
    return s / (g->h[a] * g->h[b]);
}

static double lap_at(const ora_grid *g, int fi, const double *f, int i, int j, int k)
{
    return d2_at(g, fi, f, 0, i, j, k) + d2_at(g, fi, f, 1, i, j, k) + d2_at(g, fi, f, 2, i, j, k);
}

/* (Lap + (1/3) d_i d_j) W at a cell, component i; W holds 3 contiguous fields */
static double momop_at(const ora_grid *g, const double *W, int comp, int i, int j, int k)
{
    long N = ncells(g);
    double v = lap_at(g, 1 + comp, W + comp * N, i, j, k) + d2_at(g, 1 + comp, W + comp * N, comp, i, j, k) / 3.0;
    for (int b = 0; b < 3; ++b)
        if (b != comp) v += dmix_at(g, 1 + b, W + b * N, comp, b, i, j, k) / 3.0;
    return v;
}

/* Bowen-York conformal extrinsic curvature of all punctures at the point x (the formula in the
 * header, summed over punctures) */
static void by_point(const ora_grid *g, const double x[3], double A[3][3])
{
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) A[a][b] = 0.0;
    for (int p = 0; p < g->npunct; ++p) {
        const double *P = g->pP[p], *S = g->pS[p];
        double d[3], r2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            d[a] = x[a] - g->px[p][a];
            r2 += d[a] * d[a];
        }
        double r = sqrt(r2), n[3] = {d[0] / r, d[1] / r, d[2] / r};
        double Pn = P[0] * n[0] + P[1] * n[1] + P[2] * n[2];
        double Sxn[3] = {S[1] * n[2] - S[2] * n[1], S[2] * n[0] - S[0] * n[2], S[0] * n[1] - S[1] * n[0]};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double delta = a == b ? 1.0 : 0.0;
                A[a][b] += 3.0 / (2.0 * r2) * (P[a] * n[b] + P[b] * n[a] - (delta - n[a] * n[b]) * Pn) +
                           3.0 / (r2 * r) * (Sxn[a] * n[b] + Sxn[b] * n[a]);
            }
    }
}

/* AtAt = sum_ij At_ij^2 with At built from first derivatives of W, plus the Bowen-York part */
static double atat_at(const ora_grid *g, const double *W, int i, int j, int k)
{
    long N = ncells(g);
    double G[3][3]; /* G[a][b] = D_a W_b */
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) G[a][b] = d1_at(g, 1 + b, W + b * N, a, i, j, k);
    double x[3] = {cellx(g, 0, i), cellx(g, 1, j), cellx(g, 2, k)}, B[3][3];
    by_point(g, x, B);
    double div = G[0][0] + G[1][1] + G[2][2];
    double s = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double A = G[a][b] + G[b][a] - (a == b ? 2.0 / 3.0 * div : 0.0) + B[a][b];
            s += A * A;
        }
    return s;
}

static double psibg_at(const ora_grid *g, int i, int j, int k)
{
    double v = 1.0;
    int c[3] = {i, j, k};
    for (int p = 0; p < g->npunct; ++p) {
        double r2 = 0.0;
        for (int a = 0; a < 3; ++a) {
            double d = cellx(g, a, c[a]) - g->px[p][a];
            r2 += d * d;
        }
        v += g->pm[p] / (2.0 * sqrt(r2));
    }
    return v;
}

/* Threads of the OpenMP loops (the pointwise residual and operator loops; the Gauss-Seidel
 * sweeps are sequential).  Returns the count now in effect (1 without OpenMP). */
int ora_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ---------------- exported operator entry points (used by the pins) ---------------- */

void ora_d1(const ora_grid *g, int a, const double *f, double *out)
{
#pragma omp parallel for
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) out[lin(g, i, j, k)] = d1_at(g, 0, f, a, i, j, k);
}

void ora_d2(const ora_grid *g, int a, const double *f, double *out)
{
#pragma omp parallel for
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) out[lin(g, i, j, k)] = d2_at(g, 0, f, a, i, j, k);
}

void ora_dmix(const ora_grid *g, int a, int b, const double *f, double *out)
{
#pragma omp parallel for
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) out[lin(g, i, j, k)] = dmix_at(g, 0, f, a, b, i, j, k);
}

void ora_lap(const ora_grid *g, const double *f, double *out)
{
#pragma omp parallel for
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) out[lin(g, i, j, k)] = lap_at(g, 0, f, i, j, k);
}

void ora_atat(const ora_grid *g, const double *W, double *out)
{
#pragma omp parallel for
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) out[lin(g, i, j, k)] = atat_at(g, W, i, j, k);
}

/* The 9 components (row-major) of the Bowen-York curvature at the point x */
void ora_by_point(const ora_grid *g, const double *x, double *out)
{
    double A[3][3];
    by_point(g, x, A);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) out[3 * a + b] = A[a][b];
}

/* The Bowen-York curvature at every cell centre: 9 fields of N (component 3a + b) */
void ora_by_cells(const ora_grid *g, double *out)
{
    long N = ncells(g);
#pragma omp parallel for
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                double x[3] = {cellx(g, 0, i), cellx(g, 1, j), cellx(g, 2, k)}, A[3][3];
                by_point(g, x, A);
                for (int c = 0; c < 9; ++c) out[c * N + lin(g, i, j, k)] = A[c / 3][c % 3];
            }
}

/* value of field f (fi: 0 = u, 1..3 = W_x..W_z) at the out-of-box cell (i,j,k) under the
 * boundary condition */
double ora_boundary_value(const ora_grid *g, int fi, const double *f, int i, int j, int k)
{
    return at(g, fi, f, i, j, k);
}

/* mean of the 8 children; gc is the coarse grid */
void ora_restrict(const ora_grid *gc, const double *fine, double *coarse)
{
    int nf0 = 2 * gc->n[0], nf1 = 2 * gc->n[1];
    for (int k = 0; k < gc->n[2]; ++k)
        for (int j = 0; j < gc->n[1]; ++j)
            for (int i = 0; i < gc->n[0]; ++i) {
                double s = 0.0;
                for (int dk = 0; dk < 2; ++dk)
                    for (int dj = 0; dj < 2; ++dj)
                        for (int di = 0; di < 2; ++di)
                            s += fine[(2 * i + di) + (long)nf0 * ((2 * j + dj) + (long)nf1 * (2 * k + dk))];
                coarse[lin(gc, i, j, k)] = s / 8.0;
            }
}

/* fine += trilinear interpolation of coarse field fi; gc is the coarse grid */
void ora_prolong_add(const ora_grid *gc, int fi, const double *coarse, double *fine)
{
    int nf0 = 2 * gc->n[0], nf1 = 2 * gc->n[1];
    for (int K = 0; K < gc->n[2]; ++K)
        for (int J = 0; J < gc->n[1]; ++J)
            for (int I = 0; I < gc->n[0]; ++I)
                for (int dk = 0; dk < 2; ++dk)
                    for (int dj = 0; dj < 2; ++dj)
                        for (int di = 0; di < 2; ++di) {
                            int sx = di ? 1 : -1, sy = dj ? 1 : -1, sz = dk ? 1 : -1;
                            double v = 0.0;
                            for (int a = 0; a < 2; ++a)
                                for (int b = 0; b < 2; ++b)
                                    for (int c = 0; c < 2; ++c) {
                                        double w = (a ? 0.25 : 0.75) * (b ? 0.25 : 0.75) * (c ? 0.25 : 0.75);
                                        v += w * at(gc, fi, coarse, I + a * sx, J + b * sy, K + c * sz);
                                    }
                            fine[(2 * I + di) + (long)nf0 * ((2 * J + dj) + (long)nf1 * (2 * K + dk))] += v;
                        }
}

/* ---------------- residual, integrability, norms ---------------- */

/*
 * Full nonlinear residual.  kmode: 0 = K fixed (K2 given in *K2), 1 = K^2 from
 * the discrete integrability condition (periodic only), written to *K2.
 * Outputs (each may be NULL): Fpsi[N], FW[3N], H[N], M[3N], c[N] (dF_psi/du),
 * norms[4] = max |H|, max |M_x|, max |M_y|, max |M_z|; msrc[3] = m_i.
 */
int ora_residual(const ora_grid *g, const double *u, const double *W, const double *rho0,
                 const double *rho2, const double *S, int kmode, double *K2, double *Fpsi, double *FW,
                 double *H, double *M, double *c, double *norms, double *msrc)
{
    long N = ncells(g);
    double *psi = malloc(N * sizeof(double));
    double *aa = malloc(N * sizeof(double));
    double *lu = malloc(N * sizeof(double));
    if (!psi || !aa || !lu) {
        free(psi); free(aa); free(lu);
        return -1;
    }
#pragma omp parallel for
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                long p = lin(g, i, j, k);
                psi[p] = psibg_at(g, i, j, k) + u[p];
                aa[p] = atat_at(g, W, i, j, k);
                lu[p] = lap_at(g, 0, u, i, j, k);
            }
    double k2 = *K2;
    if (kmode == 1) {
        /* sum_cells Lap u = 0 on a periodic grid, so sum F_psi = 0 fixes K^2 */
        double num = 0.0, den = 0.0;
        for (long p = 0; p < N; ++p) {
            double p5 = pow(psi[p], 5.0);
            num += aa[p] / 8.0 * pow(psi[p], -7.0) + 2.0 * ORA_PI * (rho0[p] * p5 + rho2[p] * psi[p]);
            den += p5;
        }
        k2 = 12.0 * num / den;
        *K2 = k2;
    }
    double m[3] = {0.0, 0.0, 0.0};
    if (g->bc == 0) {
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (long p = 0; p < N; ++p) s += 8.0 * ORA_PI * pow(psi[p], 6.0) * S[a * N + p];
            m[a] = s / (double)N;
        }
    }
    if (msrc) for (int a = 0; a < 3; ++a) msrc[a] = m[a];
    double nh = 0.0, nm[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                long p = lin(g, i, j, k);
                double ps = psi[p];
                double fp = lu[p] - k2 / 12.0 * pow(ps, 5.0) + aa[p] / 8.0 * pow(ps, -7.0) +
                            2.0 * ORA_PI * (rho0[p] * pow(ps, 5.0) + rho2[p] * ps);
                double hv = -8.0 * pow(ps, -5.0) * fp;
                if (Fpsi) Fpsi[p] = fp;
                if (H) H[p] = hv;
                if (fabs(hv) > nh || hv != hv) nh = (hv != hv) ? NAN : fabs(hv);
                if (c)
                    c[p] = -5.0 / 12.0 * k2 * pow(ps, 4.0) - 7.0 / 8.0 * pow(ps, -8.0) * aa[p] +
                           2.0 * ORA_PI * (5.0 * rho0[p] * pow(ps, 4.0) + rho2[p]);
                for (int a = 0; a < 3; ++a) {
                    double fw = momop_at(g, W, a, i, j, k) - (8.0 * ORA_PI * pow(ps, 6.0) * S[a * N + p] - m[a]);
                    double mv = pow(ps, -6.0) * fw;
                    if (FW) FW[a * N + p] = fw;
                    if (M) M[a * N + p] = mv;
                    if (fabs(mv) > nm[a] || mv != mv) nm[a] = (mv != mv) ? NAN : fabs(mv);
                }
            }
    if (norms) {
        norms[0] = nh;
        for (int a = 0; a < 3; ++a) norms[1 + a] = nm[a];
    }
    free(psi); free(aa); free(lu);
    return 0;
}

/* ---------------- inner linear multigrid ---------------- */

typedef struct {
    ora_grid g;
    long N;
    double *a;   /* psi-row coefficient of Lap (psi^-5 on the finest level) */
    double *c;   /* psi-row diagonal coefficient (psi^-5 dF_psi/du on the finest level) */
    double *f;   /* 4N right-hand side: psi row then 3 W rows */
    double *e;   /* 4N correction */
    double *r;   /* 4N scratch residual */
} ora_level;

static double diag_lap(const ora_grid *g)
{
    double w = (g->order == 2) ? -2.0 : -30.0 / 12.0;
    return w / (g->h[0] * g->h[0]) + w / (g->h[1] * g->h[1]) + w / (g->h[2] * g->h[2]);
}

static double diag_d2(const ora_grid *g, int a)
{
    double w = (g->order == 2) ? -2.0 : -30.0 / 12.0;
    return w / (g->h[a] * g->h[a]);
}

/* lexicographic Gauss-Seidel sweeps on (a Lap + c) e = f and the momentum operator */
static void gs_sweeps(ora_level *L, int sweeps)
{
    const ora_grid *g = &L->g;
    long N = L->N;
    double dl = diag_lap(g);
    for (int s = 0; s < sweeps; ++s)
        for (int k = 0; k < g->n[2]; ++k)
            for (int j = 0; j < g->n[1]; ++j)
                for (int i = 0; i < g->n[0]; ++i) {
                    long p = lin(g, i, j, k);
                    double rp = L->f[p] - (L->a[p] * lap_at(g, 0, L->e, i, j, k) + L->c[p] * L->e[p]);
                    L->e[p] += rp / (L->a[p] * dl + L->c[p]);
                    for (int a = 0; a < 3; ++a) {
                        double ra = L->f[(1 + a) * N + p] - momop_at(g, L->e + N, a, i, j, k);
                        L->e[(1 + a) * N + p] += ra / (dl + diag_d2(g, a) / 3.0);
                    }
                }
}

static void linear_residual(ora_level *L)
{
    const ora_grid *g = &L->g;
    long N = L->N;
    for (int k = 0; k < g->n[2]; ++k)
        for (int j = 0; j < g->n[1]; ++j)
            for (int i = 0; i < g->n[0]; ++i) {
                long p = lin(g, i, j, k);
                L->r[p] = L->f[p] - (L->a[p] * lap_at(g, 0, L->e, i, j, k) + L->c[p] * L->e[p]);
                for (int a = 0; a < 3; ++a)
                    L->r[(1 + a) * N + p] = L->f[(1 + a) * N + p] - momop_at(g, L->e + N, a, i, j, k);
            }
}

static void remove_means(const ora_grid *g, double *e4, long N)
{
    if (g->bc != 0) return;
    for (int a = 0; a < 4; ++a) {
        double s = 0.0;
        for (long p = 0; p < N; ++p) s += e4[a * N + p];
        s /= (double)N;
        for (long p = 0; p < N; ++p) e4[a * N + p] -= s;
    }
}

/*
 * Exact solve of the psi row on the coarsest level: (a Lap + c) e = f, bordered on periodic
 * boxes by a constant Lagrange multiplier and the constraint sum e = 0.  The matrix is built by
 * applying the operator to unit vectors and solved by Gaussian elimination with partial
 * pivoting.  Overwrites the psi part of L->e.  Returns 0, or -1 if allocation fails.
 */
static int coarse_psi_direct(ora_level *L)
{
    const ora_grid *g = &L->g;
    long N = L->N;
    int per = g->bc == 0;
    long m = N + per;
    double *A = calloc((size_t)(m * m), sizeof(double));
    double *x = calloc((size_t)m, sizeof(double));
    double *unit = calloc((size_t)N, sizeof(double));
    if (!A || !x || !unit) { free(A); free(x); free(unit); return -1; }
    for (long q = 0; q < N; ++q) {
        unit[q] = 1.0;
        for (int k = 0; k < g->n[2]; ++k)
            for (int j = 0; j < g->n[1]; ++j)
                for (int i = 0; i < g->n[0]; ++i) {
                    long p = lin(g, i, j, k);
                    A[p * m + q] = L->a[p] * lap_at(g, 0, unit, i, j, k) + L->c[p] * unit[p];
                }
        unit[q] = 0.0;
    }
    if (per) {
        for (long p = 0; p < N; ++p) {
            A[p * m + N] = 1.0;
            A[N * m + p] = 1.0;
        }
    }
    for (long p = 0; p < N; ++p) x[p] = L->f[p];
    for (long k = 0; k < m; ++k) {
        long piv = k;
        for (long i = k + 1; i < m; ++i)
            if (fabs(A[i * m + k]) > fabs(A[piv * m + k])) piv = i;
        if (piv != k) {
            for (long j = 0; j < m; ++j) {
                double t = A[k * m + j]; A[k * m + j] = A[piv * m + j]; A[piv * m + j] = t;
            }
            double t = x[k]; x[k] = x[piv]; x[piv] = t;
        }
        for (long i = k + 1; i < m; ++i) {
            double l = A[i * m + k] / A[k * m + k];
            for (long j = k; j < m; ++j) A[i * m + j] -= l * A[k * m + j];
            x[i] -= l * x[k];
        }
    }
    for (long k = m - 1; k >= 0; --k) {
        double s = x[k];
        for (long j = k + 1; j < m; ++j) s -= A[k * m + j] * x[j];
        x[k] = s / A[k * m + k];
    }
    for (long p = 0; p < N; ++p) L->e[p] = x[p];
    free(A); free(x); free(unit);
    return 0;
}

static void vcycle(ora_level *lv, int l, int nlev, int nu1, int nu2, int csweeps)
{
    ora_level *L = &lv[l];
    long N = L->N;
    memset(L->e, 0, 4 * N * sizeof(double));
    if (l == nlev - 1) {
        gs_sweeps(L, csweeps);
        remove_means(&L->g, L->e, N);
        if (L->N <= 1000) coarse_psi_direct(L);
        return;
    }
    gs_sweeps(L, nu1);
    linear_residual(L);
    ora_level *C = &lv[l + 1];
    for (int a = 0; a < 4; ++a) ora_restrict(&C->g, L->r + a * N, C->f + a * C->N);
    vcycle(lv, l + 1, nlev, nu1, nu2, csweeps);
    for (int a = 0; a < 4; ++a) ora_prolong_add(&C->g, a, C->e + a * C->N, L->e + a * N);
    gs_sweeps(L, nu2);
}

/* number of levels: coarsen while every side is even and halves to >= 3 */
int ora_auto_levels(const int n[3])
{
    int m[3] = {n[0], n[1], n[2]}, lev = 1;
    for (;;) {
        int ok = 1;
        for (int a = 0; a < 3; ++a)
            if (m[a] % 2 != 0 || m[a] / 2 < 3) ok = 0;
        if (!ok) break;
        for (int a = 0; a < 3; ++a) m[a] /= 2;
        ++lev;
    }
    return lev;
}

/* subtract the cell mean of one field (periodic gauge) */
static void remove_mean1(double *f, long N)
{
    double s = 0.0;
    for (long p = 0; p < N; ++p) s += f[p];
    s /= (double)N;
    for (long p = 0; p < N; ++p) f[p] -= s;
}

/*
 * Solve for u (N) and W (3N), in place (they hold the initial guess).
 * tol > 0: stop when max(|H|, |M_i|) <= tol.  tol <= 0: iterate to the FP64
 * floor (stop once the max norm fails to drop below 0.9x its value three
 * outer iterations earlier).
 * hist (may be NULL) receives 4 norms per residual evaluation (max_outer+1 rows).
 * Returns 0 converged, 1 floor reached, 2 out of iterations, 3 non-finite, -1 bad args.
 */
int ora_solve(const ora_grid *g0, const double *rho0, const double *rho2, const double *S, int kmode,
              double *K2, double tol, int max_outer, int levels, int nu1, int nu2, int csweeps, double *u,
              double *W, double *hist, int *iters)
{
    if (levels <= 0) levels = ora_auto_levels(g0->n);
    if (max_outer < 0) return -1;
    long N = ncells(g0);
    ora_level *lv = calloc(levels, sizeof(ora_level));
    double *F = malloc(4 * N * sizeof(double));
    double *mx_hist = malloc((max_outer + 1) * sizeof(double));
    if (!lv || !F || !mx_hist) { free(lv); free(F); free(mx_hist); return -1; }
    int status = 2, it, ok = 1;
    for (int l = 0; l < levels; ++l) {
        ora_grid g = *g0;
        for (int a = 0; a < 3; ++a) {
            g.n[a] = g0->n[a] >> l;
            g.h[a] = g0->h[a] * (double)(1 << l);
            if ((g.n[a] << l) != g0->n[a] || g.n[a] < 2) ok = 0;
        }
        lv[l].g = g;
        lv[l].N = ncells(&g);
        lv[l].a = calloc(lv[l].N, sizeof(double));
        lv[l].c = calloc(lv[l].N, sizeof(double));
        lv[l].f = calloc(4 * lv[l].N, sizeof(double));
        lv[l].e = calloc(4 * lv[l].N, sizeof(double));
        lv[l].r = calloc(4 * lv[l].N, sizeof(double));
        if (!lv[l].a || !lv[l].c || !lv[l].f || !lv[l].e || !lv[l].r) ok = 0;
    }
    if (!ok) { status = -1; it = 0; goto done; }
    for (it = 0; it <= max_outer; ++it) {
        double norms[4];
        ora_residual(g0, u, W, rho0, rho2, S, kmode, K2, F, F + N, NULL, NULL, lv[0].c, norms, NULL);
        double mx = 0.0;
        int finite = 1;
        for (int a = 0; a < 4; ++a) {
            if (!isfinite(norms[a])) finite = 0;
            if (norms[a] > mx) mx = norms[a];
        }
        mx_hist[it] = mx;
        if (hist) for (int a = 0; a < 4; ++a) hist[4 * it + a] = norms[a];
        if (!finite) { status = 3; break; }
        if (tol > 0.0 && mx <= tol) { status = 0; break; }
        if (tol <= 0.0 && (mx == 0.0 || (it >= 3 && mx > 0.9 * mx_hist[it - 3]))) { status = 1; break; }
        if (it == max_outer) break;
        /* The psi row is scaled by psi^-5: then the change of K^2, whose direction in F_psi is
         * psi^5, is a constant, which the zero-mean projection of the correction absorbs. */
        for (long p = 0; p < N; ++p) {
            double ps5 = pow(psibg_at(g0, (int)(p % g0->n[0]), (int)((p / g0->n[0]) % g0->n[1]),
                                      (int)(p / ((long)g0->n[0] * g0->n[1]))) + u[p], -5.0);
            lv[0].a[p] = ps5;
            lv[0].c[p] *= ps5;
            lv[0].f[p] = -ps5 * F[p];
        }
        for (long p = N; p < 4 * N; ++p) lv[0].f[p] = -F[p];
        for (int l = 1; l < levels; ++l) {
            ora_restrict(&lv[l].g, lv[l - 1].a, lv[l].a);
            ora_restrict(&lv[l].g, lv[l - 1].c, lv[l].c);
        }
        vcycle(lv, 0, levels, nu1, nu2, csweeps);
        for (long p = 0; p < N; ++p) u[p] += lv[0].e[p];
        for (long p = 0; p < 3 * N; ++p) W[p] += lv[0].e[N + p];
        if (g0->bc == 0) {
            remove_mean1(u, N);
            for (int a = 0; a < 3; ++a) remove_mean1(W + a * N, N);
        }
    }
done:
    if (iters) *iters = it;
    for (int l = 0; l < levels; ++l) {
        free(lv[l].a); free(lv[l].c); free(lv[l].f); free(lv[l].e); free(lv[l].r);
    }
    free(lv); free(F); free(mx_hist);
    return status;
}
