// mg_outer.cuh -- FP64 outer residual of the CTT constraints in two passes.
//
// On GB300 an FP64 instruction issues at 2 lanes per clock per SM, so this residual is bound by
// its FP64 instruction count, not by memory.  The mixed term (1/3) d_i d_j W_j of F_W,i costs
// most: written as the tensor product of first-derivative stencils it takes 16 points and ~20
// FP64 instructions per (i, j) pair.  Since D_i D_j = D_i o D_j, the same sum is
//   sum_{j != i} D_i D_j W_j = D_i q_i,   q_i = sum_{j != i} D_j W_j = div W - D_i W_i,
// so pass A stores q_0, q_1, q_2 and div W at every cell (FP64, from the same boundary values the
// tensor product uses) and pass B applies one first derivative per row.  Pass B also folds the
// 1/h factors into the stencil weights.  Pass B takes this path on the interior box (cells
// whose whole stencil lies inside the box, so the q reads need no ghost value of q); cells of
// the shell keep the direct tensor-product form.  Both give the discrete operator of the
// constraints (eq:Ham, eq:Mom in CTT form), differing only in FP64 rounding order.
#pragma once
#include "mg_kernels.cuh"

namespace ctt {

// Stencil weights with the grid spacing folded in.
struct OuterCoef {
    double c1[3], c2[3];            // D_a f = c1 (f+1 - f-1) - c2 (f+2 - f-2)
    double k1[3], nk2[3], k0;       // Lap f = k0 f + sum_a k1 (f+1 + f-1) + nk2 (f+2 + f-2)
    double m1[3][3], nm2[3][3], m0[3];   // row A: Lap W_A + (1/3) D_AA W_A, same form
    double q1[3], q2[3];            // (1/3) D_A along A
};

// t-th cell (all colours) of the interior box [G, n-G)^3, x fastest; false past the end.
__device__ __forceinline__ bool interior_cell_all(const Geo &g, int G, unsigned t, int &i, int &j, int &k)
{
    const unsigned ix = g.n[0] - 2 * G, iy = g.n[1] - 2 * G, iz = g.n[2] - 2 * G;
    if ((int)ix <= 0 || (int)iy <= 0 || (int)iz <= 0) return false;
    const unsigned row = t / ix;
    if (row >= iy * iz) return false;
    i = G + (int)(t - row * ix);
    const unsigned jj = row % iy;
    j = G + (int)jj;
    k = G + (int)((row - jj) / iy);
    return true;
}

template <int ORDER, int A, class F>
__device__ __forceinline__ double d1w(const F &f, double c1, double c2)
{
    double d = c1 * (ax<A>(f, 1) - ax<A>(f, -1));
    if constexpr (ORDER == 4) d = fma(-c2, ax<A>(f, 2) - ax<A>(f, -2), d);
    return d;
}

template <int ORDER, class F>
__device__ __forceinline__ double lapw(const F &f, const double k1[3], const double nk2[3], double k0)
{
    double s = k0 * f(0, 0, 0);
    s = fma(k1[0], f(1, 0, 0) + f(-1, 0, 0), s);
    s = fma(k1[1], f(0, 1, 0) + f(0, -1, 0), s);
    s = fma(k1[2], f(0, 0, 1) + f(0, 0, -1), s);
    if constexpr (ORDER == 4) {
        s = fma(nk2[0], f(2, 0, 0) + f(-2, 0, 0), s);
        s = fma(nk2[1], f(0, 2, 0) + f(0, -2, 0), s);
        s = fma(nk2[2], f(0, 0, 2) + f(0, 0, -2), s);
    }
    return s;
}

// Pass A: q_a = div W - D_a W_a (a = 0, 1, 2) and div W, at every cell.
template <int ORDER, int BC>
__global__ void __launch_bounds__(256) k_outer_div(Geo g, OuterCoef oc, const double *__restrict__ x,
                                                   double *__restrict__ D)
{
    const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
    const int sy = g.n[0], sz = g.n[0] * g.n[1];
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(p % g.n[0]);
        const size_t rest = p / g.n[0];
        const int j = (int)(rest % g.n[1]);
        const int k = (int)(rest / g.n[1]);
        double h0, h1, h2;
        if (is_interior(g, i, j, k, halo<ORDER>())) {
            AccI<double> a1{x + N + p, sy, sz}, a2{x + 2 * N + p, sy, sz}, a3{x + 3 * N + p, sy, sz};
            h0 = d1w<ORDER, 0>(a1, oc.c1[0], oc.c2[0]);
            h1 = d1w<ORDER, 1>(a2, oc.c1[1], oc.c2[1]);
            h2 = d1w<ORDER, 2>(a3, oc.c1[2], oc.c2[2]);
        } else {
            AccB<double, BC> a1{x + N, 1, &g, i, j, k}, a2{x + 2 * N, 2, &g, i, j, k}, a3{x + 3 * N, 3, &g, i, j, k};
            h0 = d1w<ORDER, 0>(a1, oc.c1[0], oc.c2[0]);
            h1 = d1w<ORDER, 1>(a2, oc.c1[1], oc.c2[1]);
            h2 = d1w<ORDER, 2>(a3, oc.c1[2], oc.c2[2]);
        }
        const double dv = h0 + h1 + h2;
        D[p] = dv - h0;
        D[N + p] = dv - h1;
        D[2 * N + p] = dv - h2;
        D[3 * N + p] = dv;
    }
}

// Lap u, AtAt and the momentum operator at a cell from pass A's q, div W (accessors: interior
// box, or wrapping on periodic boxes, where q and div W are exact at the wrapped cells).
template <int ORDER, class F>
__device__ __forceinline__ void outer_cell_qa(const F &u, const F &w0, const F &w1, const F &w2, const F &q0,
                                              const F &q1, const F &q2, double dv, const OuterCoef &oc, double &lu,
                                              double &aa, double mom[3], const double *by = nullptr, size_t N = 0)
{
    lu = lapw<ORDER>(u, oc.k1, oc.nk2, oc.k0);
    mom[0] = lapw<ORDER>(w0, oc.m1[0], oc.nm2[0], oc.m0[0]) + d1w<ORDER, 0>(q0, oc.q1[0], oc.q2[0]);
    mom[1] = lapw<ORDER>(w1, oc.m1[1], oc.nm2[1], oc.m0[1]) + d1w<ORDER, 1>(q1, oc.q1[1], oc.q2[1]);
    mom[2] = lapw<ORDER>(w2, oc.m1[2], oc.nm2[2], oc.m0[2]) + d1w<ORDER, 2>(q2, oc.q1[2], oc.q2[2]);
    // At_ab = G_ab + G_ba - (2/3) delta_ab div, G_ab = D_a W_b; the diagonal from pass A
    const double g00 = dv - q0(0, 0, 0), g11 = dv - q1(0, 0, 0), g22 = dv - q2(0, 0, 0);
    const double s01 = d1w<ORDER, 0>(w1, oc.c1[0], oc.c2[0]) + d1w<ORDER, 1>(w0, oc.c1[1], oc.c2[1]);
    const double s02 = d1w<ORDER, 0>(w2, oc.c1[0], oc.c2[0]) + d1w<ORDER, 2>(w0, oc.c1[2], oc.c2[2]);
    const double s12 = d1w<ORDER, 1>(w2, oc.c1[1], oc.c2[1]) + d1w<ORDER, 2>(w1, oc.c1[2], oc.c2[2]);
    const double t = (-2.0 / 3.0) * dv;
    double a00 = fma(2.0, g00, t), a11 = fma(2.0, g11, t), a22 = fma(2.0, g22, t);
    double b01 = s01, b02 = s02, b12 = s12;
    if (by) {   // Bowen-York part (by: the cell's first component, stride N)
        a00 += by[0];
        a11 += by[N];
        a22 += by[2 * N];
        b01 += by[3 * N];
        b02 += by[4 * N];
        b12 += by[5 * N];
    }
    const double off = fma(b01, b01, fma(b02, b02, b12 * b12));
    aa = fma(2.0, off, fma(a00, a00, fma(a11, a11, a22 * a22)));
}

template <int ORDER>
__device__ __forceinline__ void outer_cell_q(const double *x, const double *D, size_t N, size_t p, int sy, int sz,
                                             const OuterCoef &oc, double &lu, double &aa, double mom[3],
                                             const double *by)
{
    AccI<double> u{x + p, sy, sz}, w0{x + N + p, sy, sz}, w1{x + 2 * N + p, sy, sz}, w2{x + 3 * N + p, sy, sz};
    AccI<double> q0{D + p, sy, sz}, q1{D + N + p, sy, sz}, q2{D + 2 * N + p, sy, sz};
    outer_cell_qa<ORDER>(u, w0, w1, w2, q0, q1, q2, D[3 * N + p], oc, lu, aa, mom, by ? by + p : nullptr, N);
}

// Nonlinear terms and outputs at cell p (shared by the interior and shell paths):
//   R0 = Lap u + (1/8) psi^-7 AtAt + 2 pi (rho0 psi^5 + rho2 psi)
//   R1..3 = mom_i - 8 pi psi^6 S_i,   R4 = AtAt (pass 2 forms the linearisation coefficient from it,
//   in the inner solve's precision)
__device__ __forceinline__ void outer_tail(const Geo &g, int i, int j, int k, size_t p, size_t N, double lu, double aa,
                                           const double mom[3], const double *x, const double *src, double *R,
                                           double acc[5])
{
    const double psi = psi_bg(g, i, j, k, p) + x[p];
    const double rho0 = src[p], rho2 = src[N + p];
    const double ip = 1.0 / psi;
    const double p2 = psi * psi, p4 = p2 * p2, p5 = p4 * psi, p6 = p5 * psi;
    const double ip2 = ip * ip, ip4 = ip2 * ip2, ip7 = ip4 * ip2 * ip;
    const double nonlin = fma(0.125 * aa, ip7, (2.0 * kPi) * fma(rho0, p5, rho2 * psi));
    R[p] = lu + nonlin;
    R[4 * N + p] = aa;
    acc[0] += nonlin;
    acc[1] += p5;
    const double s8 = (8.0 * kPi) * p6;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double s = s8 * src[(2 + a) * N + p];
        R[(1 + a) * N + p] = mom[a] - s;
        acc[2 + a] += s;
    }
}

// Shell cells, out of line so that the interior path keeps its registers.  Periodic boxes: the
// q form with wrapping accessors; Robin boxes: the direct tensor-product form with boundary
// values (a ghost value of q is not the Robin value of q).  out = (Lap u, AtAt, mom_0..2).
template <int ORDER, int BC>
__device__ __noinline__ void outer_shell_cell(const Geo &g, const Coef<double> &cf, const OuterCoef &oc,
                                              const double *x, const double *D, int i, int j, int k, double *out)
{
    const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
    AccB<double, BC> a0{x, 0, &g, i, j, k}, a1{x + N, 1, &g, i, j, k}, a2{x + 2 * N, 2, &g, i, j, k},
        a3{x + 3 * N, 3, &g, i, j, k};
    double lu, aa, mom[3];
    if constexpr (BC == BC_PERIODIC) {
        AccB<double, BC> q0{D, 0, &g, i, j, k}, q1{D + N, 0, &g, i, j, k}, q2{D + 2 * N, 0, &g, i, j, k};   // periodic
        const size_t p = (size_t)i + (size_t)g.n[0] * ((size_t)j + (size_t)g.n[1] * k);
        outer_cell_qa<ORDER>(a0, a1, a2, a3, q0, q1, q2, D[3 * N + p], oc, lu, aa, mom);
    } else {
        const size_t p = (size_t)i + (size_t)g.n[0] * ((size_t)j + (size_t)g.n[1] * k);
        outer_cell<ORDER>(a0, a1, a2, a3, cf, lu, aa, mom, g.by ? g.by + p : nullptr, N);
    }
    out[0] = lu;
    out[1] = aa;
    out[2] = mom[0];
    out[3] = mom[1];
    out[4] = mom[2];
}

// Pass B: residual parts R (5 fields) and block partial sums, as k_outer_pass1.  Blocks
// [0, rg.nblk_sh) take the shell (tensor-product form), the others the interior box.
template <int ORDER, int BC>
__global__ void __launch_bounds__(256, 2) k_outer_pass1q(Geo g, Coef<double> cf, OuterCoef oc,
                                                      const double *__restrict__ x, const double *__restrict__ D,
                                                      const double *__restrict__ src, double *__restrict__ R,
                                                      double *__restrict__ partial, Regions rg, OuterFin fin)
{
    const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
    const int sy = g.n[0], sz = g.n[0] * g.n[1];
    double acc[5] = {0, 0, 0, 0, 0};
    int i, j, k;
    if ((int)blockIdx.x >= rg.nblk_sh) {
        const unsigned stride = (unsigned)(gridDim.x - rg.nblk_sh) * blockDim.x;
        for (unsigned t = (blockIdx.x - rg.nblk_sh) * blockDim.x + threadIdx.x; interior_cell_all(g, rg.G, t, i, j, k);
             t += stride) {
            const size_t p = (size_t)i + (size_t)sy * j + (size_t)sz * k;
            double lu, aa, mom[3];
            outer_cell_q<ORDER>(x, D, N, p, sy, sz, oc, lu, aa, mom, g.by);
            outer_tail(g, i, j, k, p, N, lu, aa, mom, x, src, R, acc);
        }
    } else {
        const unsigned stride = (unsigned)rg.nblk_sh * blockDim.x;
        for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; shell_cell(g, rg.G, t, i, j, k); t += stride) {
            const size_t p = (size_t)i + (size_t)sy * j + (size_t)sz * k;
            double o[5];
            outer_shell_cell<ORDER, BC>(g, cf, oc, x, D, i, j, k, o);
            const double mom[3] = {o[2], o[3], o[4]};
            outer_tail(g, i, j, k, p, N, o[0], o[1], mom, x, src, R, acc);
        }
    }
    double r[5];
    block_sum<5>(acc, r);
    if (threadIdx.x == 0)
        for (int a = 0; a < 5; ++a) partial[blockIdx.x * 5 + a] = r[a];
    if (fin.s && finalize_last<5, false>(partial, gridDim.x, fin.s->sums, &fin.s->ticket[0]) && threadIdx.x == 0)
        outer_scalars(fin.s, N, fin.kmode_integrability, fin.K2_fixed, fin.periodic);
}

}  // namespace ctt
