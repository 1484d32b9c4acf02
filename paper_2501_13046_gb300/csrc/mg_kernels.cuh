// mg_kernels.cuh -- sm_103a kernels of the CTT constraint multigrid.
//
// Discrete system (GRTresna, arXiv:2501.13046: eq:Ham, eq:Mom in CTT form with a
// conformally flat metric and constant K; multigrid per "Key features: Fast"):
//   F_psi = Lap u - (K^2/12) psi^5 + (1/8) psi^-7 AtAt + 2 pi (rho0 psi^5 + rho2 psi)
//   F_W,i = Lap W_i + (1/3) d_i d_j W_j - 8 pi (psi^6 S_i - m_i)
// Centred cell stencils of order 2 or 4; boundary values are produced on the fly by
// every kernel (periodic wrap, or Robin 1/r: v(g) = v(clamp(g)) |x_clamp| / |x_g|, or, below a
// symmetry plane x_a = 0 of a Robin box, the mirror image with W_a negated; see bc_cell), so
// arrays carry no ghost cells and no fill pass exists.
//
// Inner problem (defect correction): the block-diagonal linearisation
//   (Lap + c) e_psi = f_psi,   (Lap + (1/3) grad div) e_W = f_W,
// smoothed red-black.  Each colour pass reads buffer A and writes buffer B in full
// (the updated colour plus a copy of the other), so couplings between cells of one
// colour (4th-order +-2 reach, mixed-derivative corners) are Jacobi and every
// result is deterministic.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace ctt {

constexpr double kPi = 3.14159265358979323846;
// Kernel boundary variants: periodic; Robin on every face; Robin with symmetry planes (g.reflect)
enum { BC_PERIODIC = 0, BC_ROBIN = 1, BC_SYM = 2 };

struct Geo {
    int n[3];
    double lo[3];
    double h[3];
    float lof[3], hf[3];   // lo and h rounded to FP32 (FP32 Robin ratios; set with lo and h)
    int reflect;           // Robin boxes: bit a set = the lower face of axis a (at x_a = 0) is a
                           // reflection-symmetry plane instead of a Robin face
    int extrap;            // Robin boxes: bit 2a (lower) / 2a + 1 (upper) = that face of axis a is
                           // extrapolating (linear extrapolation along its normal; see extrap_split)
    int robin;             // 1 on Robin boxes (faces with boundary rules), 0 on periodic boxes
    int npunct;
    double pm[2];
    double px[2][3];
    const double *psibg;   // finest level with punctures: psi_background per cell (N doubles), else null
    const double *rtab;    // finest level of a Robin box: the FP64 ratio |x_b| / |x_g| on the box padded by
                           // 2 cells per side (1 inside), (n0+4)(n1+4)(n2+4) doubles, else null
    const double *by;      // finest level with Bowen-York punctures: their curvature per cell, 6 fields of N
                           // (A_00, A_11, A_22, A_01, A_02, A_12), else null
};

// Bowen-York punctures (boosted and/or spinning black holes): positions, momenta and spins.
struct ByPunct {
    int n;
    double x[2][3], P[2][3], S[2][3];
};

// by = sum over punctures of the analytic conformal extrinsic curvature
//   A_ij = 3/(2 r^2) [P_i n_j + P_j n_i - (delta_ij - n_i n_j) P.n] + 3/r^3 [(S x n)_i n_j + (S x n)_j n_i]
// (n the unit vector from the puncture to the cell centre, r the distance), once per context.
static __global__ void __launch_bounds__(256) k_fill_by(Geo g, ByPunct bp, double *__restrict__ by)
{
    const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
        const int c[3] = {(int)(p % g.n[0]), (int)((p / g.n[0]) % g.n[1]), (int)(p / ((size_t)g.n[0] * g.n[1]))};
        double A[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        for (int q = 0; q < bp.n; ++q) {
            double d[3], r2 = 0.0;
            for (int a = 0; a < 3; ++a) {
                d[a] = g.lo[a] + (c[a] + 0.5) * g.h[a] - bp.x[q][a];
                r2 += d[a] * d[a];
            }
            const double r = sqrt(r2), n[3] = {d[0] / r, d[1] / r, d[2] / r};
            const double *P = bp.P[q], *S = bp.S[q];
            const double Pn = P[0] * n[0] + P[1] * n[1] + P[2] * n[2];
            const double Sxn[3] = {S[1] * n[2] - S[2] * n[1], S[2] * n[0] - S[0] * n[2], S[0] * n[1] - S[1] * n[0]};
            const double cp = 1.5 / r2, cs = 3.0 / (r2 * r);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    A[a][b] += cp * (P[a] * n[b] + P[b] * n[a] - ((a == b ? 1.0 : 0.0) - n[a] * n[b]) * Pn) +
                               cs * (Sxn[a] * n[b] + Sxn[b] * n[a]);
        }
        by[p] = A[0][0];
        by[N + p] = A[1][1];
        by[2 * N + p] = A[2][2];
        by[3 * N + p] = A[0][1];
        by[4 * N + p] = A[0][2];
        by[5 * N + p] = A[1][2];
    }
}

// Diagonal shifts of the inner operator's rows next to the faces of a Robin box.  A colour pass
// divides a row's residual by the row's diagonal; next to a face some stencil taps lie beyond the
// box and their boundary value depends on the cell itself (the clamped cell of the 1/r rule, a
// mirror image, a weight of an extrapolation), so the row's true diagonal is the interior one plus
// each such tap's weight times that dependence.  The taps of the diagonal run along the axes, so
// the shift is a sum over axes of a term that depends only on the cell's distance to that axis's
// faces: s[axis][lower/upper face][face cell / next cell][field u, W_x, W_y, W_z], with the 1/r
// ratio of the Robin rule taken as 1 (the smoother only preconditions; the residual keeps the
// exact rule).  Zero on periodic boxes.
template <typename T>
struct FaceDiag {
    T s[3][2][2][4];
};

template <typename T>
struct Coef {
    T ih[3];    // 1/h
    T ih2[3];   // 1/h^2
    T dl;       // diagonal of the discrete Laplacian
    T idW[3];   // omega / diagonal of the momentum operator row i (relaxation weight folded in)
    T iom;      // 1 / omega: the psi-row update divides by (diagonal * iom)
    FaceDiag<T> fd;   // diagonal shifts next to the faces (Robin boxes)
};

// Host: the face table of a level (Geo g with its reflect / extrap masks), order 2 or 4.
template <typename T>
inline void face_diag(const Geo &g, int order, FaceDiag<T> &fd)
{
    for (int a = 0; a < 3; ++a)
        for (int sd = 0; sd < 2; ++sd)
            for (int o = 0; o < 2; ++o)
                for (int f = 0; f < 4; ++f) fd.s[a][sd][o][f] = 0;
    if (!g.robin) return;
    const double k1 = order == 2 ? 1.0 : 16.0 / 12.0, k2 = order == 2 ? 0.0 : -1.0 / 12.0;
    for (int a = 0; a < 3; ++a) {
        const int n = g.n[a];
        const double ih2 = 1.0 / (g.h[a] * g.h[a]);
        for (int sd = 0; sd < 2; ++sd)
            for (int o = 0; o < 2; ++o) {
                const int i = sd == 0 ? o : n - 1 - o;   // the cell's index along a
                double acc[4] = {0, 0, 0, 0};
                for (int st = 1; st <= (order == 2 ? 1 : 2); ++st) {
                    const int c = sd == 0 ? i - st : i + st;   // the tap toward this side's face
                    if (c >= 0 && c < n) continue;
                    double kap[4] = {0, 0, 0, 0};
                    if (sd == 0 && ((g.reflect >> a) & 1)) {         // mirror image across x_a = 0
                        if (-1 - c == i)
                            for (int f = 0; f < 4; ++f) kap[f] = f == 1 + a ? -1.0 : 1.0;
                    } else if ((g.extrap >> (2 * a + sd)) & 1) {     // linear extrapolation
                        const int d = sd == 0 ? -c : c - (n - 1), b0 = sd == 0 ? 0 : n - 1, b1 = sd == 0 ? 1 : n - 2;
                        const double kk = (i == b0 ? 1.0 + d : 0.0) + (i == b1 ? -(double)d : 0.0);
                        for (int f = 0; f < 4; ++f) kap[f] = kk;
                    } else if (i == (sd == 0 ? 0 : n - 1)) {         // the clamped cell of the 1/r rule
                        for (int f = 0; f < 4; ++f) kap[f] = 1.0;
                    }
                    const double w = (st == 1 ? k1 : k2) * ih2;
                    acc[0] += w * kap[0];
                    for (int A = 0; A < 3; ++A) acc[1 + A] += (a == A ? 4.0 / 3.0 : 1.0) * w * kap[1 + A];
                }
                for (int f = 0; f < 4; ++f) fd.s[a][sd][o][f] = (T)acc[f];
            }
    }
}

// Device: the shift of field f's row (0: the Laplacian of the psi row, 1 + A: row A) at cell p.
template <int F, typename T>
__device__ __forceinline__ T face_shift(const FaceDiag<T> &fd, const Geo &g, int i, int j, int k)
{
    const int p[3] = {i, j, k};
    T d = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int n = g.n[a];
        d += p[a] == 0 ? fd.s[a][0][0][F] : (p[a] == 1 ? fd.s[a][0][1][F] : (T)0);
        d += p[a] == n - 1 ? fd.s[a][1][0][F] : (p[a] == n - 2 ? fd.s[a][1][1][F] : (T)0);
    }
    return d;
}

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

__device__ __forceinline__ double cellx(const Geo &g, int a, int i) { return g.lo[a] + (i + 0.5) * g.h[a]; }

// Robin 1/r boundary: a cell g outside the box takes the value of its clamped cell b times |x_b| / |x_g|.
// The ratio is formed in the level's precision T: FP32 levels (the inner solve's preconditioner)
// take A rsqrt(A B) = sqrt(A / B) with the hardware reciprocal square root and no FP64 arithmetic,
// whose rate is 1/64 of FP32 here; FP64 takes one division and one square root.
template <typename T>
__device__ __forceinline__ T robin_ratio(const Geo &g, int bi, int bj, int bk, int gi, int gj, int gk)
{
    auto c = [&](int a, int i) {
        if constexpr (std::is_same<T, float>::value) return g.lof[a] + ((float)i + 0.5f) * g.hf[a];
        else return g.lo[a] + (i + 0.5) * g.h[a];
    };
    const T xb = c(0, bi), yb = c(1, bj), zb = c(2, bk), xg = c(0, gi), yg = c(1, gj), zg = c(2, gk);
    const T A = xb * xb + yb * yb + zb * zb, B = xg * xg + yg * yg + zg * zg;
    if constexpr (std::is_same<T, float>::value) return A * rsqrtf(A * B);
    else return sqrt(A / B);
}

// The in-box cell b that supplies the value at a cell p at most 2 cells outside the box.
// Periodic boxes wrap.  Robin boxes mirror p_a -> -1 - p_a below a lower face marked in g.reflect
// (a symmetry plane; bit a of `mirror` is set) and clamp every other out-of-box coordinate; the
// return value says whether a coordinate was clamped, in which case the value is scaled by the
// 1/r ratio |x_b| / |x_p| (mirroring keeps |x|, the planes passing through the origin).
template <int BC>
__device__ __forceinline__ bool bc_cell(const Geo &g, const int p[3], int b[3], int &mirror)
{
    mirror = 0;
    bool clamped = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int n = g.n[a];
        if constexpr (BC == BC_PERIODIC) {
            b[a] = p[a] + (p[a] < 0 ? n : 0) - (p[a] >= n ? n : 0);
        } else if constexpr (BC == BC_ROBIN) {
            b[a] = min(max(p[a], 0), n - 1);
            clamped |= b[a] != p[a];
        } else {
            if (p[a] < 0 && ((g.reflect >> a) & 1)) {
                b[a] = -1 - p[a];
                mirror |= 1 << a;
            } else {
                b[a] = min(max(p[a], 0), n - 1);
                clamped |= b[a] != p[a];
            }
        }
    }
    return clamped;
}

// Extrapolating faces (Robin boxes with symmetry planes and/or extrapolating faces: the BC_SYM
// variant).  A cell beyond such a face at distance d along its normal takes the linear
// extrapolation (1 + d) v(b) - d v(b') through the boundary cell b of its line and the next cell
// b' in; beyond several such faces the rule applies axis by axis (linear maps commute), and
// bc_cell then resolves any remaining out-of-box coordinate.  Splits p into ns <= 8 cells, inside
// the box along every extrapolating axis, with integer weights w (sum of w_s v(q_s)); returns 0
// when p lies beyond no extrapolating face.
__device__ __forceinline__ int extrap_split(const Geo &g, const int p[3], int q[8][3], int w[8])
{
    int ns = 1;
    q[0][0] = p[0];
    q[0][1] = p[1];
    q[0][2] = p[2];
    w[0] = 1;
    bool any = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int d = 0, b0 = 0, b1 = 0;
        if (p[a] < 0 && ((g.extrap >> (2 * a)) & 1)) {
            d = -p[a];
            b1 = 1;
        } else if (p[a] >= g.n[a] && ((g.extrap >> (2 * a + 1)) & 1)) {
            d = p[a] - (g.n[a] - 1);
            b0 = g.n[a] - 1;
            b1 = g.n[a] - 2;
        }
        if (d == 0) continue;
        any = true;
        for (int s = 0; s < ns; ++s) {
            q[ns + s][0] = q[s][0];
            q[ns + s][1] = q[s][1];
            q[ns + s][2] = q[s][2];
            q[ns + s][a] = b1;
            w[ns + s] = -d * w[s];
            q[s][a] = b0;
            w[s] *= 1 + d;
        }
        ns *= 2;
    }
    return any ? ns : 0;
}

// Whether p lies beyond an extrapolating face (the cheap test kept inline; the weighted sums over
// extrap_split's cells are out-of-line functions: that branch is rare, and inlining it into every
// stencil tap multiplies the code, and the compile time, of the boundary variant).
__device__ __forceinline__ bool beyond_extrap(const Geo &g, const int p[3])
{
    bool b = false;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        b |= (p[a] < 0 && ((g.extrap >> (2 * a)) & 1)) || (p[a] >= g.n[a] && ((g.extrap >> (2 * a + 1)) & 1));
    return b;
}

// Sign of field fi (0 = u, 1..3 = W_x..W_z) at a cell mirrored across the planes in `mirror`:
// the component of W normal to a symmetry plane is odd across it, everything else even.
__device__ __forceinline__ int bc_sign(int mirror, int fi) { return (fi >= 1 && ((mirror >> (fi - 1)) & 1)) ? -1 : 1; }

// v, negated when field fi changes sign across the planes in `mirror` (symmetry-plane variant only)
template <int BC, typename T>
__device__ __forceinline__ T bc_signed(T v, int mirror, int fi)
{
    if constexpr (BC == BC_SYM) return bc_sign(mirror, fi) < 0 ? -v : v;
    else return v;
}

// FP64 Robin ratio of the ghost cell (i, j, k) (at most 2 cells outside) onto its clamped cell b:
// the stored table when there is one (the division and square root run at the FP64 rate).
__device__ __forceinline__ double robin_ratio_f64(const Geo &g, int bi, int bj, int bk, int i, int j, int k)
{
    if (g.rtab)
        return g.rtab[(size_t)(i + 2) + (size_t)(g.n[0] + 4) * ((size_t)(j + 2) + (size_t)(g.n[1] + 4) * (k + 2))];
    return robin_ratio<double>(g, bi, bj, bk, i, j, k);
}

// rt[(i+2) + (n0+4)((j+2) + (n1+4)(k+2))] = |x_b| / |x_(i,j,k)| with b = bc_cell (1 when no
// coordinate is clamped: inside the box, or only mirrored), -2 <= i < n0 + 2, ...
template <int BC>
__global__ void __launch_bounds__(256) k_fill_robin_table(Geo g, double *__restrict__ rt)
{
    const int m0 = g.n[0] + 4, m1 = g.n[1] + 4;
    const size_t M = (size_t)m0 * m1 * (g.n[2] + 4);
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < M; p += (size_t)gridDim.x * blockDim.x) {
        const int c[3] = {(int)(p % m0) - 2, (int)((p / m0) % m1) - 2, (int)(p / ((size_t)m0 * m1)) - 2};
        int b[3], mirror;
        const bool clamped = bc_cell<BC>(g, c, b, mirror);
        rt[p] = clamped ? robin_ratio<double>(g, b[0], b[1], b[2], c[0], c[1], c[2]) : 1.0;
    }
}

__device__ __forceinline__ double psi_background(const Geo &g, int i, int j, int k)
{
    double v = 1.0;
    for (int p = 0; p < g.npunct; ++p) {
        double dx = cellx(g, 0, i) - g.px[p][0];
        double dy = cellx(g, 1, j) - g.px[p][1];
        double dz = cellx(g, 2, k) - g.px[p][2];
        v += g.pm[p] / (2.0 * sqrt(dx * dx + dy * dy + dz * dz));
    }
    return v;
}

// psi_background at cell p = (i, j, k): the stored table when there is one (a FP64 square root and
// division per puncture and cell cost more than the 8-byte read), else formed in place.
__device__ __forceinline__ double psi_bg(const Geo &g, int i, int j, int k, size_t p)
{
    return g.psibg ? g.psibg[p] : psi_background(g, i, j, k);
}

static __global__ void __launch_bounds__(256) k_fill_psibg(Geo g, double *__restrict__ pb)
{
    const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(p % g.n[0]), j = (int)((p / g.n[0]) % g.n[1]), k = (int)(p / ((size_t)g.n[0] * g.n[1]));
        pb[p] = psi_background(g, i, j, k);
    }
}

// value of field f (index fi, see bc_sign) at a cell that may lie outside the box (offsets are at
// most +-2 per axis)
// fetch_bc at an unwrapped cell p that lies beyond no extrapolating face.
template <typename T, int BC>
__device__ __forceinline__ T fetch_bc_one(const T *f, int fi, const Geo &g, const int p[3])
{
    int b[3], mirror;
    const bool clamped = bc_cell<BC>(g, p, b, mirror);
    const T v = bc_signed<BC>(f[b[0] + g.n[0] * (b[1] + g.n[1] * b[2])], mirror, fi);
    if (!clamped) return v;
    if constexpr (std::is_same<T, double>::value) return v * robin_ratio_f64(g, b[0], b[1], b[2], p[0], p[1], p[2]);
    else return v * robin_ratio<T>(g, b[0], b[1], b[2], p[0], p[1], p[2]);
}

// fetch_bc beyond an extrapolating face: the weighted cells of extrap_split (out of line).
template <typename T, int BC>
__device__ __noinline__ T fetch_bc_extrap(const T *f, int fi, const Geo *g, int i, int j, int k)
{
    const int p[3] = {i, j, k};
    int q[8][3], w[8];
    const int ns = extrap_split(*g, p, q, w);
    T s = 0;
    for (int t = 0; t < ns; ++t) s += (T)w[t] * fetch_bc_one<T, BC>(f, fi, *g, q[t]);
    return s;
}

template <typename T, int BC>
__device__ __forceinline__ T fetch_bc(const T *f, int fi, const Geo &g, int i, int j, int k)
{
    if constexpr (BC == BC_PERIODIC) {
        i += (i < 0) ? g.n[0] : 0; i -= (i >= g.n[0]) ? g.n[0] : 0;
        j += (j < 0) ? g.n[1] : 0; j -= (j >= g.n[1]) ? g.n[1] : 0;
        k += (k < 0) ? g.n[2] : 0; k -= (k >= g.n[2]) ? g.n[2] : 0;
        return f[i + g.n[0] * (j + g.n[1] * k)];
    } else {
        const int p[3] = {i, j, k};
        if constexpr (BC == BC_SYM)
            if (g.extrap && beyond_extrap(g, p)) return fetch_bc_extrap<T, BC>(f, fi, &g, i, j, k);
        return fetch_bc_one<T, BC>(f, fi, g, p);
    }
}

// Whether a cell is within 2 cells of a face (where the face shifts may be nonzero).
__device__ __forceinline__ bool near_face(const Geo &g, int i, int j, int k)
{
    return i < 2 || j < 2 || k < 2 || i >= g.n[0] - 2 || j >= g.n[1] - 2 || k >= g.n[2] - 2;
}

// The four rows' shifts at a cell (psi row's Laplacian, rows W_x, W_y, W_z).
template <typename T>
__device__ __forceinline__ void face_shifts(const FaceDiag<T> &fd, const Geo &g, int i, int j, int k, T &dpsi, T dW[3])
{
    dpsi = face_shift<0>(fd, g, i, j, k);
    dW[0] = face_shift<1>(fd, g, i, j, k);
    dW[1] = face_shift<2>(fd, g, i, j, k);
    dW[2] = face_shift<3>(fd, g, i, j, k);
}

// A row's relaxation factor omega / (m0 + d) from omega / m0 (idW) and 1 / omega (iom).
template <typename T>
__device__ __forceinline__ T shifted_idW(T idW, T iom, T d) { return idW / ((T)1 + d * idW * iom); }

// Relaxation factors of a cell: the psi row's Laplacian diagonal dl and the W rows' omega /
// diagonal kW.  The interior values, except on boxes with faces for a cell within 2 cells of one
// (may_be_near: the caller cannot rule that out), where the face shifts are added; periodic
// levels and interior cells do no extra arithmetic.
template <int BC, typename T>
__device__ __forceinline__ void relax_factors(const FaceDiag<T> &fd, const Geo &g, int i, int j, int k,
                                              bool may_be_near, T dl0, const T idW[3], T iom, T &dl, T kW[3])
{
    dl = dl0;
    kW[0] = idW[0];
    kW[1] = idW[1];
    kW[2] = idW[2];
    if constexpr (BC != BC_PERIODIC) {
        if (may_be_near && near_face(g, i, j, k)) {
            T dpsi, dW[3];
            face_shifts(fd, g, i, j, k, dpsi, dW);
            dl = dl0 + dpsi;
#pragma unroll
            for (int a = 0; a < 3; ++a) kW[a] = shifted_idW(idW[a], iom, dW[a]);
        }
    }
}

// Accessors: value at cell p + (dx, dy, dz) of one field.
template <typename T>
struct AccI {   // every offset of the stencil stays inside the box
    const T *p;
    int sy, sz;
    __device__ __forceinline__ T operator()(int dx, int dy, int dz) const { return p[dx + dy * sy + dz * sz]; }
};

template <typename T, int BC>
struct AccB {   // near the boundary; fi: the field (0 = u, 1..3 = W_x..W_z), for symmetry planes
    const T *f;
    int fi;
    const Geo *g;
    int i, j, k;
    __device__ __forceinline__ T operator()(int dx, int dy, int dz) const
    {
        return fetch_bc<T, BC>(f, fi, *g, i + dx, j + dy, k + dz);
    }
};

template <int A, class F>
__device__ __forceinline__ auto ax(const F &f, int s) { return f(A == 0 ? s : 0, A == 1 ? s : 0, A == 2 ? s : 0); }

template <int A, int B, class F>
__device__ __forceinline__ auto ax2(const F &f, int s, int t)
{
    return f((A == 0 ? s : 0) + (B == 0 ? t : 0), (A == 1 ? s : 0) + (B == 1 ? t : 0),
             (A == 2 ? s : 0) + (B == 2 ? t : 0));
}

// first derivative along A, times h
template <int ORDER, int A, typename T, class F>
__device__ __forceinline__ T d1(const F &f)
{
    if constexpr (ORDER == 2) {
        return (T)0.5 * (ax<A>(f, 1) - ax<A>(f, -1));
    } else {
        return (T)(8.0 / 12.0) * (ax<A>(f, 1) - ax<A>(f, -1)) + (T)(1.0 / 12.0) * (ax<A>(f, -2) - ax<A>(f, 2));
    }
}

// compact second derivative along A, times h^2 (centre value passed in)
template <int ORDER, int A, typename T, class F>
__device__ __forceinline__ T d2(const F &f, T c)
{
    if constexpr (ORDER == 2) {
        return (ax<A>(f, 1) + ax<A>(f, -1)) - (T)2 * c;
    } else {
        return (T)(16.0 / 12.0) * (ax<A>(f, 1) + ax<A>(f, -1)) - (T)(1.0 / 12.0) * (ax<A>(f, 2) + ax<A>(f, -2)) -
               (T)(30.0 / 12.0) * c;
    }
}

// D_A D_B f (A != B), times h_A h_B: tensor product of the first-derivative stencils
template <int ORDER, int A, int B, typename T, class F>
__device__ __forceinline__ T dmix(const F &f)
{
    if constexpr (ORDER == 2) {
        return (T)0.25 * ((ax2<A, B>(f, 1, 1) - ax2<A, B>(f, 1, -1)) - (ax2<A, B>(f, -1, 1) - ax2<A, B>(f, -1, -1)));
    } else {
        auto inner = [&](int s) {
            return (T)(8.0 / 12.0) * (ax2<A, B>(f, s, 1) - ax2<A, B>(f, s, -1)) +
                   (T)(1.0 / 12.0) * (ax2<A, B>(f, s, -2) - ax2<A, B>(f, s, 2));
        };
        return (T)(8.0 / 12.0) * (inner(1) - inner(-1)) + (T)(1.0 / 12.0) * (inner(-2) - inner(2));
    }
}

template <int ORDER>
__host__ __device__ constexpr int halo() { return ORDER / 2; }

__device__ __forceinline__ bool is_interior(const Geo &g, int i, int j, int k, int G)
{
    return i >= G && i < g.n[0] - G && j >= G && j < g.n[1] - G && k >= G && k < g.n[2] - G;
}

// ---------------------------------------------------------------------------------------
// Linear operator of the inner problem at one cell, all 4 rows: out = J e.
// e0..e3 accessors of the 4 correction fields.  The psi row is a Lap e0 + b e0: on the finest
// level a = psi^-5 and b = psi^-5 c (the row scaled by psi^-5, which makes the direction of the
// K^2 change, psi^5, a constant), on coarser levels a and b are their 8-child means.
template <int ORDER, typename T, class F>
__device__ __forceinline__ void apply_J(const F &e0, const F &e1, const F &e2, const F &e3, T ca, T cb,
                                        const Coef<T> &cf, T out[4], T centre[4])
{
    centre[0] = e0(0, 0, 0);
    centre[1] = e1(0, 0, 0);
    centre[2] = e2(0, 0, 0);
    centre[3] = e3(0, 0, 0);
    // psi row
    T lp = d2<ORDER, 0, T>(e0, centre[0]) * cf.ih2[0] + d2<ORDER, 1, T>(e0, centre[0]) * cf.ih2[1] +
           d2<ORDER, 2, T>(e0, centre[0]) * cf.ih2[2];
    out[0] = ca * lp + cb * centre[0];
    // momentum rows: Lap W_i + (1/3)(D_ii W_i + sum_{j != i} D_i D_j W_j)
    T dxx = d2<ORDER, 0, T>(e1, centre[1]) * cf.ih2[0];
    T lx = dxx + d2<ORDER, 1, T>(e1, centre[1]) * cf.ih2[1] + d2<ORDER, 2, T>(e1, centre[1]) * cf.ih2[2];
    T mx = dmix<ORDER, 0, 1, T>(e2) * (cf.ih[0] * cf.ih[1]) + dmix<ORDER, 0, 2, T>(e3) * (cf.ih[0] * cf.ih[2]);
    out[1] = lx + (dxx + mx) * (T)(1.0 / 3.0);
    T dyy = d2<ORDER, 1, T>(e2, centre[2]) * cf.ih2[1];
    T ly = d2<ORDER, 0, T>(e2, centre[2]) * cf.ih2[0] + dyy + d2<ORDER, 2, T>(e2, centre[2]) * cf.ih2[2];
    T my = dmix<ORDER, 1, 0, T>(e1) * (cf.ih[1] * cf.ih[0]) + dmix<ORDER, 1, 2, T>(e3) * (cf.ih[1] * cf.ih[2]);
    out[2] = ly + (dyy + my) * (T)(1.0 / 3.0);
    T dzz = d2<ORDER, 2, T>(e3, centre[3]) * cf.ih2[2];
    T lz = d2<ORDER, 0, T>(e3, centre[3]) * cf.ih2[0] + d2<ORDER, 1, T>(e3, centre[3]) * cf.ih2[1] + dzz;
    T mz = dmix<ORDER, 2, 0, T>(e1) * (cf.ih[2] * cf.ih[0]) + dmix<ORDER, 2, 1, T>(e2) * (cf.ih[2] * cf.ih[1]);
    out[3] = lz + (dzz + mz) * (T)(1.0 / 3.0);
}

// ---------------------------------------------------------------------------------------
// Storage of a level's fields.  Every level above the coarsest is colour-split: a field of N
// cells is [colour 0 half | colour 1 half], cell (i,j,k) with colour c = (i+j+k) & 1 and
// linear index lin = i + nx (j + ny k) sits at c N/2 + lin/2 (nx even, so the two cells of an
// x-pair have different colours and share lin/2).  A colour pass then reads and writes only
// the halves it needs, and every neighbour load of a warp is contiguous.  The coarsest level
// (possibly odd-sized, handled by one CTA) is plain: cell at lin.
__device__ __forceinline__ size_t sidx(const Geo &g, int i, int j, int k, size_t N, int split)
{
    size_t lin = (size_t)i + (size_t)g.n[0] * ((size_t)j + (size_t)g.n[1] * k);
    return split ? (((i + j + k) & 1) ? N / 2 : 0) + (lin >> 1) : lin;
}

// Interior accessor of a colour-split field around a cell with pair index m = lin/2 and
// sel = lin & 1.  A neighbour (dx,dy,dz) lies in the half of the other colour when dx+dy+dz is
// odd, and at pair index m + floor((sel + dx)/2) + dy nx/2 + dz nx ny/2, i.e. m + dx/2 for even
// dx and m + sel + (dx-1)/2 for odd dx.  The four base pointers absorb m and sel, so every
// offset below is a compile-time combination of dy, dz with 32-bit strides.
template <typename T>
struct AccS {
    const T *se, *so, *oe, *oo;   // same-colour half + m, + m + sel; other-colour half + m, + m + sel
    int nxh, plane;
    __device__ __forceinline__ T operator()(int dx, int dy, int dz) const
    {
        const bool other = (dx + dy + dz) & 1;
        const bool odd = dx & 1;
        const T *b = other ? (odd ? oo : oe) : (odd ? so : se);
        const int xo = odd ? ((dx - 1) >> 1) : (dx >> 1);
        return b[xo + dy * nxh + dz * plane];
    }
};

// Value of field fi at the unwrapped cell p (beyond no extrapolating face) of a colour-split level:
// `same` holds the cells of colour c, `other` the rest (both are full field bases).
template <typename T, int BC>
__device__ __forceinline__ T split_one(const T *same, const T *other, int fi, const Geo &g, size_t N, int c,
                                       const int p[3])
{
    int q[3], mirror;
    const bool outside = bc_cell<BC>(g, p, q, mirror);
    int c2 = (q[0] + q[1] + q[2]) & 1;
    size_t lin = (size_t)q[0] + (size_t)g.n[0] * ((size_t)q[1] + (size_t)g.n[1] * q[2]);
    T v = (c2 == c ? same : other)[(c2 ? N / 2 : 0) + (lin >> 1)];
    v = bc_signed<BC>(v, mirror, fi);
    if (BC != BC_PERIODIC && outside) {
        if constexpr (std::is_same<T, double>::value)
            return v * robin_ratio_f64(g, q[0], q[1], q[2], p[0], p[1], p[2]);
        else
            return v * robin_ratio<T>(g, q[0], q[1], q[2], p[0], p[1], p[2]);
    }
    return v;
}

// split_one beyond an extrapolating face: the weighted cells of extrap_split (out of line).
template <typename T, int BC>
__device__ __noinline__ T split_extrap(const T *same, const T *other, int fi, const Geo *g, size_t N, int c, int i,
                                       int j, int k)
{
    const int p[3] = {i, j, k};
    int q[8][3], w[8];
    const int ns = extrap_split(*g, p, q, w);
    T s = 0;
    for (int t = 0; t < ns; ++t) s += (T)w[t] * split_one<T, BC>(same, other, fi, *g, N, c, q[t]);
    return s;
}

// Boundary accessor of a colour-split field: cells of the centre's colour c are read from
// `same`, cells of the other colour from `other` (both are full field bases).
template <typename T, int BC>
struct AccB2 {
    const T *same, *other;
    int fi;   // the field (0 = u, 1..3 = W_x..W_z), for symmetry planes
    const Geo *g;
    size_t N;
    int i, j, k, c;
    __device__ __forceinline__ T operator()(int dx, int dy, int dz) const
    {
        const int p[3] = {i + dx, j + dy, k + dz};
        if constexpr (BC == BC_SYM)
            if (g->extrap && beyond_extrap(*g, p)) return split_extrap<T, BC>(same, other, fi, g, N, c, p[0], p[1], p[2]);
        return split_one<T, BC>(same, other, fi, *g, N, c, p);
    }
};

// J e at cell (i,j,k) of a colour-split level; X holds the cell's colour, O the other colour.
// INTERIOR: every stencil point lies inside the box (fast accessor), else the boundary accessor.
template <typename T, int ORDER, int BC, bool INTERIOR>
__device__ __forceinline__ void apply_J_split(const T *X, const T *O, size_t N, const Geo &g, int i, int j, int k,
                                              T ca, T cb, const Coef<T> &cf, T out[4], T centre[4])
{
    const int c = (i + j + k) & 1;
    if constexpr (INTERIOR) {
        const size_t Nh = N / 2;
        const unsigned lin = (unsigned)i + (unsigned)g.n[0] * ((unsigned)j + (unsigned)g.n[1] * (unsigned)k);
        const unsigned m = lin >> 1;
        const int sel = (int)(lin & 1), nxh = g.n[0] >> 1, plane = nxh * g.n[1];
        const T *Xs = X + (c ? Nh : 0) + m, *Oo = O + (c ? 0 : Nh) + m;
        AccS<T> a0{Xs, Xs + sel, Oo, Oo + sel, nxh, plane};
        AccS<T> a1{Xs + N, Xs + N + sel, Oo + N, Oo + N + sel, nxh, plane};
        AccS<T> a2{Xs + 2 * N, Xs + 2 * N + sel, Oo + 2 * N, Oo + 2 * N + sel, nxh, plane};
        AccS<T> a3{Xs + 3 * N, Xs + 3 * N + sel, Oo + 3 * N, Oo + 3 * N + sel, nxh, plane};
        apply_J<ORDER, T>(a0, a1, a2, a3, ca, cb, cf, out, centre);
    } else {
        AccB2<T, BC> a0{X, O, 0, &g, N, i, j, k, c}, a1{X + N, O + N, 1, &g, N, i, j, k, c},
            a2{X + 2 * N, O + 2 * N, 2, &g, N, i, j, k, c}, a3{X + 3 * N, O + 3 * N, 3, &g, N, i, j, k, c};
        apply_J<ORDER, T>(a0, a1, a2, a3, ca, cb, cf, out, centre);
    }
}

// Cells of a box split into two block-uniform regions so that no warp mixes the fast interior
// stencil with the boundary one: the interior box [G, n-G)^3 and the shell around it.
struct Regions {
    int G;               // halo width (cells within G of a face form the shell)
    int nblk_sh;         // blocks [0, nblk_sh) take the shell (scheduled first: the shell is the
                         // slower path, so it overlaps the interior instead of trailing it)
};

// t-th cell of the interior box [G, n-G)^3 of colour `colour` (x fastest); returns false past
// the end.  32-bit index arithmetic (grids hold at most 2^31 cells).
__device__ __forceinline__ bool interior_cell(const Geo &g, int G, int colour, unsigned t, int &i, int &j, int &k)
{
    const unsigned ix = g.n[0] - 2 * G, iy = g.n[1] - 2 * G, iz = g.n[2] - 2 * G;
    if ((int)ix <= 0 || (int)iy <= 0 || (int)iz <= 0) return false;
    const unsigned per_row = ix >> 1;   // ix is even
    const unsigned row = t / per_row;
    if (row >= iy * iz) return false;
    const unsigned q = t - row * per_row;
    const unsigned jj = row % iy;
    j = G + (int)jj;
    k = G + (int)((row - jj) / iy);
    i = G + ((colour + j + k + G) & 1) + 2 * (int)q;
    return true;
}

// t-th cell of the shell (cells within G of a face), all colours; returns false past the end.
__device__ __forceinline__ bool shell_cell(const Geo &g, int G, unsigned t, int &i, int &j, int &k)
{
    const unsigned nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int iz = g.n[2] - 2 * G, iy = g.n[1] - 2 * G;
    const unsigned G2 = 2 * G;
    if (iz <= 0 || iy <= 0) {   // the whole box is shell
        if (t >= nx * ny * nz) return false;
        i = (int)(t % nx); j = (int)((t / nx) % ny); k = (int)(t / (nx * ny));
        return true;
    }
    const unsigned A = G2 * nx * ny;                   // z-faces: k < G or k >= nz - G
    if (t < A) {
        i = (int)(t % nx); j = (int)((t / nx) % ny);
        int kk = (int)(t / (nx * ny));
        k = kk < G ? kk : (int)nz - 2 * G + kk;
        return true;
    }
    t -= A;
    const unsigned B = (unsigned)iz * G2 * nx;          // y-faces of the remaining planes
    if (t < B) {
        i = (int)(t % nx);
        int jj = (int)((t / nx) % G2);
        k = G + (int)(t / (nx * G2));
        j = jj < G ? jj : (int)ny - 2 * G + jj;
        return true;
    }
    t -= B;
    const unsigned C = (unsigned)iz * (unsigned)iy * G2;  // x-faces of the remaining rows
    if (t >= C) return false;
    int ii = (int)(t % G2);
    unsigned row = t / G2;
    j = G + (int)(row % (unsigned)iy);
    k = G + (int)(row / (unsigned)iy);
    i = ii < G ? ii : g.n[0] - 2 * G + ii;
    return true;
}

__host__ __device__ inline size_t shell_count(const int n[3], int G)
{
    size_t N = (size_t)n[0] * n[1] * n[2];
    long long ix = n[0] - 2 * G, iy = n[1] - 2 * G, iz = n[2] - 2 * G;
    if (ix <= 0 || iy <= 0 || iz <= 0) return N;
    return N - (size_t)ix * iy * iz;
}

// ---------------------------------------------------------------------------------------
// Red-black colour pass on a colour-split level.  Blocks [0, nblk_sh) update the active-colour
// cells of the shell, the other blocks those of the interior box.  Old values of the active
// colour come from X, current values of the other colour from O (X on the first pass of a
// sweep, Y on the second); the new active-colour values go to Y, so couplings inside a colour
// are Jacobi and the result is deterministic.
template <typename T, int ORDER, int BC>
__device__ __forceinline__ void smooth_cell(const Geo &g, const Coef<T> &cf, const T *X, const T *O, T *Y, const T *f,
                                            const T *ab, size_t N, int i, int j, int k, bool interior)
{
    const unsigned lin = (unsigned)i + (unsigned)g.n[0] * ((unsigned)j + (unsigned)g.n[1] * (unsigned)k);
    const size_t q = (((i + j + k) & 1) ? N / 2 : 0) + (lin >> 1);
    T ca = ab[q], cb = ab[N + q];
    T Je[4], ctr[4];
    if (interior) apply_J_split<T, ORDER, BC, true>(X, O, N, g, i, j, k, ca, cb, cf, Je, ctr);
    else apply_J_split<T, ORDER, BC, false>(X, O, N, g, i, j, k, ca, cb, cf, Je, ctr);
    T dl, kW[3];
    relax_factors<BC>(cf.fd, g, i, j, k, !interior, cf.dl, cf.idW, cf.iom, dl, kW);
    Y[q] = ctr[0] + (f[q] - Je[0]) / ((ca * dl + cb) * cf.iom);
#pragma unroll
    for (int a = 0; a < 3; ++a) Y[(1 + a) * N + q] = ctr[1 + a] + (f[(1 + a) * N + q] - Je[1 + a]) * kW[a];
}

// The shell path is a call: only shell blocks execute it, and it leaves the interior path its registers.
template <typename T, int ORDER, int BC>
__device__ __noinline__ void smooth_cell_shell(const Geo &g, const Coef<T> &cf, const T *X, const T *O, T *Y,
                                               const T *f, const T *ab, size_t N, int i, int j, int k)
{
    smooth_cell<T, ORDER, BC>(g, cf, X, O, Y, f, ab, N, i, j, k, false);
}

template <typename T, int ORDER, int BC>
__global__ void __launch_bounds__(256, 2) k_smooth_colour(Geo g, Coef<T> cf, const T *__restrict__ X,
                                                          const T *__restrict__ O, T *__restrict__ Y,
                                                          const T *__restrict__ f, const T *__restrict__ ab,
                                                          int colour, Regions rg)
{
    const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
    int i, j, k;
    if ((int)blockIdx.x >= rg.nblk_sh) {
        const unsigned stride = (unsigned)(gridDim.x - rg.nblk_sh) * blockDim.x;
        for (unsigned t = (blockIdx.x - rg.nblk_sh) * blockDim.x + threadIdx.x;
             interior_cell(g, rg.G, colour, t, i, j, k); t += stride)
            smooth_cell<T, ORDER, BC>(g, cf, X, O, Y, f, ab, N, i, j, k, true);
    } else {
        const unsigned stride = (unsigned)rg.nblk_sh * blockDim.x;
        for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; shell_cell(g, rg.G, t, i, j, k); t += stride)
            if (((i + j + k) & 1) == colour) smooth_cell_shell<T, ORDER, BC>(g, cf, X, O, Y, f, ab, N, i, j, k);
    }
}

// Residual r = f - J e on a colour-split fine level, averaged over the 8 children into the
// coarse rhs (stored colour-split, or plain when the coarse level is the coarsest).  Blocks
// [0, nblk_sh) take the coarse shell, the others the coarse cells whose children's stencils stay
// inside the fine box (the coarse interior box [1, nc-1)^3).
template <typename T, int ORDER, int BC, bool INTERIOR>
__device__ __forceinline__ void restrict_cell(const Geo &g, const Coef<T> &cf, const Geo &gc, const T *e, const T *f,
                                              const T *ab, T *fc, size_t N, size_t Nc, int csplit, int I, int J, int K)
{
    T acc[4] = {0, 0, 0, 0};
#pragma unroll 1
    for (int d = 0; d < 8; ++d) {
        int i = 2 * I + (d & 1), j = 2 * J + ((d >> 1) & 1), k = 2 * K + (d >> 2);
        size_t p = sidx(g, i, j, k, N, 1);
        T Je[4], ctr[4];
        apply_J_split<T, ORDER, BC, INTERIOR>(e, e, N, g, i, j, k, ab[p], ab[N + p], cf, Je, ctr);
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a] += f[a * N + p] - Je[a];
    }
    size_t pc = sidx(gc, I, J, K, Nc, csplit);
#pragma unroll
    for (int a = 0; a < 4; ++a) fc[a * Nc + pc] = acc[a] * (T)0.125;
}

template <typename T, int ORDER, int BC>
__device__ __noinline__ void restrict_cell_shell(const Geo &g, const Coef<T> &cf, const Geo &gc, const T *e,
                                                 const T *f, const T *ab, T *fc, size_t N, size_t Nc, int csplit,
                                                 int I, int J, int K)
{
    restrict_cell<T, ORDER, BC, false>(g, cf, gc, e, f, ab, fc, N, Nc, csplit, I, J, K);
}

template <typename T, int ORDER, int BC>
__global__ void __launch_bounds__(256, 2) k_residual_restrict(Geo g, Coef<T> cf, Geo gc, const T *__restrict__ e,
                                                              const T *__restrict__ f, const T *__restrict__ ab,
                                                              T *__restrict__ fc, int csplit, Regions rg)
{
    const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
    const size_t Nc = (size_t)gc.n[0] * gc.n[1] * gc.n[2];
    int I, J, K;
    if ((int)blockIdx.x >= rg.nblk_sh) {
        // coarse interior box [1, nc-1)^3, x fastest
        const int ix = gc.n[0] - 2, iy = gc.n[1] - 2, iz = gc.n[2] - 2;
        const unsigned total = (ix > 0 && iy > 0 && iz > 0) ? (unsigned)ix * iy * iz : 0;
        const unsigned stride = (unsigned)(gridDim.x - rg.nblk_sh) * blockDim.x;
        for (unsigned t = (blockIdx.x - rg.nblk_sh) * blockDim.x + threadIdx.x; t < total; t += stride) {
            const unsigned r = t / (unsigned)ix;
            I = 1 + (int)(t - r * (unsigned)ix);
            J = 1 + (int)(r % (unsigned)iy);
            K = 1 + (int)(r / (unsigned)iy);
            restrict_cell<T, ORDER, BC, true>(g, cf, gc, e, f, ab, fc, N, Nc, csplit, I, J, K);
        }
    } else {
        const unsigned stride = (unsigned)rg.nblk_sh * blockDim.x;
        for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; shell_cell(gc, 1, t, I, J, K); t += stride)
            restrict_cell_shell<T, ORDER, BC>(g, cf, gc, e, f, ab, fc, N, Nc, csplit, I, J, K);
    }
}

// Mean of the 8 children for nf fields (the psi-row coefficients a and b): fine colour-split,
// coarse colour-split or plain.
template <typename T>
__global__ void __launch_bounds__(256) k_restrict_mean(Geo g, Geo gc, const T *__restrict__ fine,
                                                       T *__restrict__ coarse, int nf, int csplit)
{
    const size_t Nc = (size_t)gc.n[0] * gc.n[1] * gc.n[2];
    const size_t Nf = 8 * Nc;
    for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < Nc; q += (size_t)gridDim.x * blockDim.x) {
        int I = (int)(q % gc.n[0]);
        size_t rest = q / gc.n[0];
        int J = (int)(rest % gc.n[1]);
        int K = (int)(rest / gc.n[1]);
        size_t pc = sidx(gc, I, J, K, Nc, csplit);
        for (int a = 0; a < nf; ++a) {
            T s = 0;
#pragma unroll
            for (int d = 0; d < 8; ++d)
                s += fine[a * Nf + sidx(g, 2 * I + (d & 1), 2 * J + ((d >> 1) & 1), 2 * K + (d >> 2), Nf, 1)];
            coarse[a * Nc + pc] = s * (T)0.125;
        }
    }
}

// Prolongation + add: e_fine += P e_coarse, trilinear in cell-centred coordinates (weights 3/4 for
// the parent and 1/4 for its neighbour towards the child, per axis).  One thread per fine cell
// (fine level colour-split, threads in storage order so that the read-modify-write of e_fine is
// coalesced): the 8 coarse cells and weights are set up once and serve all 4 fields.  Coarse
// neighbours outside the box take the level's boundary value (periodic wrap, the mirror image
// across a symmetry plane with W's normal component negated, or the Robin ratio |x_clamp| / |x_g|
// folded into the weight).  Coarse level colour-split or plain (csplit).
template <typename T, int BC>
__global__ void __launch_bounds__(256) k_prolong_add(Geo g, Geo gc, const T *__restrict__ ec, T *__restrict__ ef,
                                                     int csplit)
{
    const unsigned nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx >> 1;
    const unsigned N = nx * ny * nz, Nh = N >> 1;
    const int ncx = gc.n[0], ncy = gc.n[1];
    const unsigned Nc = (unsigned)ncx * ncy * gc.n[2];
    for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < N; q += gridDim.x * blockDim.x) {
        const unsigned c = q >= Nh, m = q - (c ? Nh : 0u);
        const unsigned row = m / nxh, xi = m - row * nxh;
        const int j = (int)(row % ny), k = (int)(row / ny);
        const int i = 2 * (int)xi + (int)((c + j + k) & 1);
        const int I = i >> 1, J = j >> 1, K = k >> 1;
        const int sx = (i & 1) ? 1 : -1, sy = (j & 1) ? 1 : -1, sz = (k & 1) ? 1 : -1;
        unsigned idx[8];
        T w[8];
        int mir[8];   // symmetry planes crossed to reach parent d (signs per field: bc_sign)
        // per axis the near parent (weight 3/4) and the far one (1/4); a far parent beyond an
        // extrapolating face is 2 v(near) - v(next in), which moves its weight onto those two
        int ia[3][2] = {{I, I + sx}, {J, J + sy}, {K, K + sz}};
        T wa[3][2] = {{(T)0.75, (T)0.25}, {(T)0.75, (T)0.25}, {(T)0.75, (T)0.25}};
        if constexpr (BC == BC_SYM) {
            if (gc.extrap) {
                const int st[3] = {sx, sy, sz};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const int far = ia[a][1];
                    if ((far < 0 && ((gc.extrap >> (2 * a)) & 1)) || (far >= gc.n[a] && ((gc.extrap >> (2 * a + 1)) & 1))) {
                        wa[a][0] += 2 * wa[a][1];
                        wa[a][1] = -wa[a][1];
                        ia[a][1] = ia[a][0] - st[a];
                    }
                }
            }
        }
#pragma unroll
        for (int d = 0; d < 8; ++d) {
            const int dx = d & 1, dy = (d >> 1) & 1, dz = d >> 2;
            const int c[3] = {ia[0][dx], ia[1][dy], ia[2][dz]};
            T wd = wa[0][dx] * wa[1][dy] * wa[2][dz];
            int b[3];
            if (bc_cell<BC>(gc, c, b, mir[d])) wd *= robin_ratio<T>(gc, b[0], b[1], b[2], c[0], c[1], c[2]);
            const unsigned lin = (unsigned)b[0] + (unsigned)ncx * ((unsigned)b[1] + (unsigned)ncy * (unsigned)b[2]);
            idx[d] = csplit ? (((b[0] + b[1] + b[2]) & 1) ? Nc / 2 : 0u) + (lin >> 1) : lin;
            w[d] = wd;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const T *e = ec + (size_t)a * Nc;
            T s = 0;
#pragma unroll
            for (int d = 0; d < 8; ++d) s = fma(bc_signed<BC>(w[d], mir[d], a), e[idx[d]], s);
            ef[(size_t)a * N + q] += s;
        }
    }
}

// ---------------------------------------------------------------------------------------
// Block reductions (warp shuffles + shared memory), deterministic order.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *out /* per block */)
{
    __shared__ double sh[32][NV];
#pragma unroll
    for (int a = 0; a < NV; ++a)
        for (int o = 16; o > 0; o >>= 1) v[a] += __shfl_down_sync(0xffffffffu, v[a], o);
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
        for (int a = 0; a < NV; ++a) sh[w][a] = v[a];
    __syncthreads();
    if (w == 0) {
        int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int a = 0; a < NV; ++a) {
            double s = l < nw ? sh[l][a] : 0.0;
            for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
            if (l == 0) out[a] = s;
        }
    }
    __syncthreads();
}

template <int NV>
__device__ __forceinline__ void block_max(double (&v)[NV], double *out)
{
    __shared__ double sh[32][NV];
#pragma unroll
    for (int a = 0; a < NV; ++a)
        for (int o = 16; o > 0; o >>= 1) v[a] = fmax(v[a], __shfl_down_sync(0xffffffffu, v[a], o));
    int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0)
        for (int a = 0; a < NV; ++a) sh[w][a] = v[a];
    __syncthreads();
    if (w == 0) {
        int nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int a = 0; a < NV; ++a) {
            double s = l < nw ? sh[l][a] : 0.0;
            for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
            if (l == 0) out[a] = s;
        }
    }
    __syncthreads();
}

// Last-block finalisation of a grid reduction: every block has stored its row of NV partials; the
// block whose ticket comes last reduces all rows in the order and tree of k_finalize_sum /
// k_finalize_max (blockDim.x = 256 there and here, so the result is the same) into out, and
// returns true in all its threads.  atomicInc wraps the ticket back to 0 for the next launch.
template <int NV, bool MAX>
__device__ __forceinline__ bool finalize_last(const double *partial, int nblocks, double *out, unsigned int *ticket)
{
    __shared__ unsigned int last;
    __threadfence();   // this block's row is visible before its ticket is
    __syncthreads();
    if (threadIdx.x == 0) last = atomicInc(ticket, gridDim.x - 1) == gridDim.x - 1;
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double v[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int a = 0; a < NV; ++a) {
            const double p = __ldcg(partial + b * NV + a);
            v[a] = MAX ? fmax(v[a], p) : v[a] + p;
        }
    double r[NV];
    if constexpr (MAX) block_max<NV>(v, r);
    else block_sum<NV>(v, r);
    if (threadIdx.x == 0)
        for (int a = 0; a < NV; ++a) out[a] = r[a];
    return true;
}

// |x| with NaN mapped to +inf, so that a max-reduction cannot hide it
__device__ __forceinline__ double absnan(double x) { return (x == x) ? fabs(x) : __longlong_as_double(0x7ff0000000000000ULL); }

// Scalars shared by the outer iteration (device memory).
struct Scalars {
    double K2;
    double msrc[3];
    double norms[4];
    double emean[4];
    double sums[8];
    unsigned int err;         // nonzero: a bounded wait of a pipelined kernel gave up (MG_ERR_TIMEOUT)
    unsigned int nonfinite;   // nonzero: a source value is NaN or infinite (set by k_flag_nonfinite)
    double change[8];         // last update: max |e_a - <e_a>| (a = 0..3), then max |psi|, |W_x|, |W_y|, |W_z| after it
    unsigned int ticket[4];   // last-block counters: pass-B sums, pass-2 norms, means of e, update maxima
    double zmean[4];          // k2_newton: means of the z solve's result (component 0: z of the psi row)
};

// Per-field part of the stopping test (mg_config.field_tol, field_est), shared by the host loops
// and the device-paced batch.  rel_a = max |e_a| / max |field_a| of the last outer update.  Plain
// test: every rel_a <= ftol.  With est, field a's remaining error is estimated from the contraction
// rho_a = rel_a / prev_a of the last two updates as rel_a rho_a / (1 - rho_a) (the tail of a
// geometric series of updates) when rho_a < 1/2, and that estimate is compared with ftol; else the
// plain test applies.  prev[4] carries rel_a from one call to the next (zero before the first
// update); call it once per outer iteration, with the number of updates made so far.
__host__ __device__ inline bool field_test(double ftol, int est, const double change[8], double prev[4], int updates)
{
    if (ftol <= 0.0) return true;
    if (updates < 1) return false;
    bool ok = true;
    for (int a = 0; a < 4; ++a) {
        const double size = change[4 + a];
        const double rel = size > 0.0 ? change[a] / size : (change[a] > 0.0 ? HUGE_VAL : 0.0);
        double bound = rel;
        if (est && updates >= 2 && prev[a] > 0.0) {
            const double rho = rel / prev[a];
            if (rho < 0.5) bound = rel * rho / (1.0 - rho);
        }
        ok = ok && bound <= ftol;
        prev[a] = rel;
    }
    return ok;
}

// K^2 (integrability or fixed) and the momentum-source means from the pass-1 sums.
__device__ __forceinline__ void outer_scalars(Scalars *s, size_t N, int kmode_integrability, double K2_fixed,
                                              int periodic)
{
    s->K2 = kmode_integrability ? 12.0 * s->sums[0] / s->sums[1] : K2_fixed;
    for (int a = 0; a < 3; ++a) s->msrc[a] = periodic ? s->sums[2 + a] / (double)N : 0.0;
}

// What the last block of pass B finishes when s is set: the sums, then K^2 and m_i.
struct OuterFin {
    Scalars *s;
    int kmode_integrability, periodic;
    double K2_fixed;
};

// Flags any NaN or infinity among n doubles (exponent field all ones; integer test, no FP64 op).
static __global__ void __launch_bounds__(256) k_flag_nonfinite(const double *__restrict__ a, size_t n,
                                                               unsigned int *__restrict__ flag)
{
    bool bad = false;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        bad |= ((__double_as_longlong(a[i]) >> 52) & 0x7ff) == 0x7ff;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(flag, 1u);
}

// Final single-block reduction of per-block partial sums: partial[b * NV + a].
template <int NV>
__global__ void k_finalize_sum(const double *__restrict__ partial, int nblocks, double *__restrict__ out)
{
    double v[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int a = 0; a < NV; ++a) v[a] += partial[b * NV + a];
    double r[NV];
    block_sum<NV>(v, r);
    if (threadIdx.x == 0)
        for (int a = 0; a < NV; ++a) out[a] = r[a];
}

template <int NV>
__global__ void k_finalize_max(const double *__restrict__ partial, int nblocks, double *__restrict__ out)
{
    double v[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int a = 0; a < NV; ++a) v[a] = fmax(v[a], partial[b * NV + a]);
    double r[NV];
    block_max<NV>(v, r);
    if (threadIdx.x == 0)
        for (int a = 0; a < NV; ++a) out[a] = r[a];
}

// Sums of 4 contiguous fields (block partials); with means != nullptr the last block also forms
// means[a] = sum_a / N (ticket: its finalize_last counter).
template <typename T>
__global__ void __launch_bounds__(256) k_sum4(const T *__restrict__ x, size_t N, double *__restrict__ partial,
                                              double *__restrict__ means, unsigned int *ticket)
{
    double v[4] = {0, 0, 0, 0};
    if constexpr (sizeof(T) == 4) {
        // each thread's sum as an unevaluated pair hi + lo of floats, kept exact by Knuth's
        // two-sum (the rounding error of every addition is carried in lo), then one FP64 sum
        float hi[4] = {0, 0, 0, 0}, lo[4] = {0, 0, 0, 0};
        for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x)
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float b = (float)x[a * N + p];
                const float s = __fadd_rn(hi[a], b);
                const float bv = __fsub_rn(s, hi[a]);
                const float err = __fadd_rn(__fsub_rn(hi[a], __fsub_rn(s, bv)), __fsub_rn(b, bv));
                hi[a] = s;
                lo[a] = __fadd_rn(lo[a], err);
            }
#pragma unroll
        for (int a = 0; a < 4; ++a) v[a] = (double)hi[a] + (double)lo[a];
    } else {
        for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x)
#pragma unroll
            for (int a = 0; a < 4; ++a) v[a] += (double)x[a * N + p];
    }
    double r[4];
    block_sum<4>(v, r);
    if (threadIdx.x == 0)
        for (int a = 0; a < 4; ++a) partial[blockIdx.x * 4 + a] = r[a];
    if (means && finalize_last<4, false>(partial, gridDim.x, means, ticket) && threadIdx.x == 0)
        for (int a = 0; a < 4; ++a) means[a] = means[a] / (double)N;
}

// x_a -= means_a for 4 contiguous fields (periodic gauge)
template <typename T>
__global__ void __launch_bounds__(256) k_sub_mean4(T *__restrict__ x, size_t N, const double *__restrict__ means)
{
    double m[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) m[a] = means[a];
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x)
#pragma unroll
        for (int a = 0; a < 4; ++a) x[a * N + p] -= (T)m[a];
}

// State update u += e - <e>, W_i += e_i - <e_i> (means only on periodic boxes); e is stored in
// the finest level's layout (colour-split when split != 0).  With s set, the last block also
// leaves the size of the update in s->change: per field the largest applied correction and the
// largest |psi|, |W_i| after it (psi = background + u), for the per-field stopping test.
// Launched on at most kRedBlocks blocks (partial holds 8 values per block).
template <typename T>
__global__ void __launch_bounds__(256) k_update(Geo g, double *__restrict__ x, const T *__restrict__ e, size_t N,
                                                const double *__restrict__ means, int split,
                                                double *__restrict__ partial, Scalars *s, const T *__restrict__ z,
                                                const double *__restrict__ zmean)
{
    // z (k2_newton): the psi correction's mean is removed along z, scaled so that the mean goes
    const double zr = z ? means[0] / zmean[0] : 0.0;
    double m[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) m[a] = means ? means[a] : 0.0;
    double mx[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const unsigned nx = (unsigned)g.n[0], ny = (unsigned)g.n[1];   // grids hold < 2^31 cells
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
        const unsigned pu = (unsigned)p, rest = pu / nx;
        const unsigned i = pu - rest * nx, j = rest % ny, k = rest / ny;
        const size_t q = split ? (((i + j + k) & 1) ? N / 2 : 0) + (p >> 1) : p;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const double d = (z && a == 0) ? (double)e[q] - zr * (double)z[q] : (double)e[a * N + q] - m[a];
            const double v = x[a * N + p] + d;
            x[a * N + p] = v;
            if (s) {
                mx[a] = fmax(mx[a], absnan(d));
                mx[4 + a] = fmax(mx[4 + a], absnan(a == 0 ? psi_bg(g, (int)i, (int)j, (int)k, p) + v : v));
            }
        }
    }
    if (!s) return;
    double r[8];
    block_max<8>(mx, r);
    if (threadIdx.x == 0)
        for (int a = 0; a < 8; ++a) partial[blockIdx.x * 8 + a] = r[a];
    finalize_last<8, true>(partial, gridDim.x, s->change, &s->ticket[3]);
}

// ---------------------------------------------------------------------------------------
// Outer FP64 residual, pass 1.  Per cell:
//   R0 = Lap u + (1/8) psi^-7 AtAt + 2 pi (rho0 psi^5 + rho2 psi)       (F_psi before the K^2 term)
//   R1..3 = Lap W_i + (1/3) d_i d_j W_j - 8 pi psi^6 S_i                   (F_W before adding m_i)
//   R4 = AtAt (the linearisation coefficient c is formed from it in pass 2)
// and block partial sums of (1/8) psi^-7 AtAt + 2 pi (rho0 psi^5 + rho2 psi), psi^5, 8 pi psi^6 S_i.
template <int ORDER, class F>
__device__ __forceinline__ void outer_cell(const F &u, const F &w0, const F &w1, const F &w2, const Coef<double> &cf,
                                           double &lu, double &aa, double mom[3], const double *by = nullptr,
                                           size_t N = 0)
{
    double G[3][3];   // G[a][b] = D_a W_b
    G[0][0] = d1<ORDER, 0, double>(w0) * cf.ih[0];
    G[1][0] = d1<ORDER, 1, double>(w0) * cf.ih[1];
    G[2][0] = d1<ORDER, 2, double>(w0) * cf.ih[2];
    G[0][1] = d1<ORDER, 0, double>(w1) * cf.ih[0];
    G[1][1] = d1<ORDER, 1, double>(w1) * cf.ih[1];
    G[2][1] = d1<ORDER, 2, double>(w1) * cf.ih[2];
    G[0][2] = d1<ORDER, 0, double>(w2) * cf.ih[0];
    G[1][2] = d1<ORDER, 1, double>(w2) * cf.ih[1];
    G[2][2] = d1<ORDER, 2, double>(w2) * cf.ih[2];
    double div = G[0][0] + G[1][1] + G[2][2];
    double B[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};   // Bowen-York part (by: the cell's first component)
    if (by) {
        B[0][0] = by[0];
        B[1][1] = by[N];
        B[2][2] = by[2 * N];
        B[0][1] = B[1][0] = by[3 * N];
        B[0][2] = B[2][0] = by[4 * N];
        B[1][2] = B[2][1] = by[5 * N];
    }
    aa = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            double A = G[a][b] + G[b][a] - (a == b ? (2.0 / 3.0) * div : 0.0) + B[a][b];
            aa += A * A;
        }
    double Je[4], ctr[4];
    apply_J<ORDER, double>(u, w0, w1, w2, 1.0, 0.0, cf, Je, ctr);   // row 0 with a = 1, b = 0 is Lap u
    lu = Je[0];
    mom[0] = Je[1];
    mom[1] = Je[2];
    mom[2] = Je[3];
}

// K^2 (integrability or fixed) and the momentum-source means from the pass-1 sums.
static __global__ void k_outer_scalars(Scalars *s, size_t N, int kmode_integrability, double K2_fixed, int periodic)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    outer_scalars(s, N, kmode_integrability, K2_fixed, periodic);
}

// Pass 2: final residuals, norm partials, inner right-hand side and coefficients in T:
//   f = (-psi^-5 F_psi, -F_W,i),  a = psi^-5,  b = psi^-5 c,  c = dF_psi/du.
// F_psi = R0 - (K^2/12) psi^5 and F_W,i = R_i + m_i are always formed in FP64: these are the
// differences of nearly equal terms.  With an FP32 inner solve (T = float) and no field output,
// the later products (the psi^-5, psi^-6 scalings of H and M, the inner data) are formed in FP32:
// each is a product of already-accurate factors, so the norms keep 7 significant digits and the
// FP64 ALU, at 2 lanes per clock per SM on this GPU, is spared the division and powers.
// Optionally (HM != nullptr) writes H and M (4 FP64 fields, FP64 throughout) instead.
__device__ __forceinline__ float absnanf(float x) { return (x == x) ? fabsf(x) : __int_as_float(0x7f800000); }

template <typename T>
__global__ void __launch_bounds__(256) k_outer_pass2(Geo g, const double *__restrict__ x, const double *__restrict__ R,
                                                     const double *__restrict__ src, Scalars *s,
                                                     T *__restrict__ f, T *__restrict__ ab, double *__restrict__ HM,
                                                     double *__restrict__ partial, int split, int fuse)
{
    const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
    const double K2 = s->K2;
    const double m0 = s->msrc[0], m1 = s->msrc[1], m2 = s->msrc[2];
    double mx[4] = {0, 0, 0, 0};
    float mxf[4] = {0, 0, 0, 0};
    const bool fast = sizeof(T) == 4 && HM == nullptr;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
        const unsigned pu = (unsigned)p, nx = (unsigned)g.n[0], ny = (unsigned)g.n[1];
        const int i = (int)(pu % nx);
        const unsigned rest = pu / nx;
        const int j = (int)(rest % ny);
        const int k = (int)(rest / ny);
        const double psi = psi_bg(g, i, j, k, p) + x[p];
        const double p2 = psi * psi, p4 = p2 * p2, p5 = p4 * psi;
        const double Fp = fma(-K2 / 12.0, p5, R[p]);
        const double Fw0 = R[N + p] + m0, Fw1 = R[2 * N + p] + m1, Fw2 = R[3 * N + p] + m2;
        if (fast) {
            const float ps = (float)psi, ip = 1.0f / ps, ip2 = ip * ip, ip5 = ip2 * ip2 * ip, ip6 = ip5 * ip;
            const float fp = (float)Fp, w0 = (float)Fw0, w1 = (float)Fw1, w2 = (float)Fw2;
            mxf[0] = fmaxf(mxf[0], absnanf(-8.0f * ip5 * fp));
            mxf[1] = fmaxf(mxf[1], absnanf(ip6 * w0));
            mxf[2] = fmaxf(mxf[2], absnanf(ip6 * w1));
            mxf[3] = fmaxf(mxf[3], absnanf(ip6 * w2));
            const size_t q = split ? (((i + j + k) & 1) ? N / 2 : 0) + (p >> 1) : p;
            // c = dF_psi/du = -(7/8) psi^-8 AtAt + 2 pi (5 rho0 psi^4 + rho2) - (5/12) K^2 psi^4
            const float ps2 = ps * ps, ps4 = ps2 * ps2, ip4 = ip2 * ip2;
            const float c = -0.875f * (ip4 * ip4) * (float)R[4 * N + p] +
                            (float)(2.0 * kPi) * (5.0f * (float)src[p] * ps4 + (float)src[N + p]) -
                            (float)(5.0 / 12.0 * K2) * ps4;
            f[q] = (T)(-ip5 * fp);
            f[N + q] = (T)(-w0);
            f[2 * N + q] = (T)(-w1);
            f[3 * N + q] = (T)(-w2);
            ab[q] = (T)ip5;
            ab[N + q] = (T)(ip5 * c);
            continue;
        }
        const double ip = 1.0 / psi, ip2 = ip * ip, ip5 = ip2 * ip2 * ip, ip6 = ip5 * ip;
        const double H = -8.0 * ip5 * Fp;
        const double M0 = ip6 * Fw0, M1 = ip6 * Fw1, M2 = ip6 * Fw2;
        mx[0] = fmax(mx[0], absnan(H));
        mx[1] = fmax(mx[1], absnan(M0));
        mx[2] = fmax(mx[2], absnan(M1));
        mx[3] = fmax(mx[3], absnan(M2));
        if (HM) {
            HM[p] = H;
            HM[N + p] = M0;
            HM[2 * N + p] = M1;
            HM[3 * N + p] = M2;
        } else {
            const size_t q = split ? (((i + j + k) & 1) ? N / 2 : 0) + (p >> 1) : p;
            f[q] = (T)(-ip5 * Fp);
            f[N + q] = (T)(-Fw0);
            f[2 * N + q] = (T)(-Fw1);
            f[3 * N + q] = (T)(-Fw2);
            const double ip4 = ip2 * ip2;
            const double c = -0.875 * (ip4 * ip4) * R[4 * N + p] + 2.0 * kPi * (5.0 * src[p] * p4 + src[N + p]) -
                             (5.0 / 12.0) * K2 * p4;
            ab[q] = (T)ip5;
            ab[N + q] = (T)(ip5 * c);
        }
    }
    if (fast)
        for (int a = 0; a < 4; ++a) mx[a] = (double)mxf[a];
    double r[4];
    block_max<4>(mx, r);
    if (threadIdx.x == 0)
        for (int a = 0; a < 4; ++a) partial[blockIdx.x * 4 + a] = r[a];
    if (fuse) finalize_last<4, true>(partial, gridDim.x, s->norms, &s->ticket[1]);
}

// ---------------------------------------------------------------------------------------
// Coarsest level: one CTA runs all sweeps in shared memory (same colour passes and ping-pong
// as the global smoother), then removes the means on periodic boxes and writes e.
template <typename T, int ORDER, int BC>
__global__ void __launch_bounds__(512) k_coarse_solve(Geo g, Coef<T> cf, const T *__restrict__ f,
                                                      const T *__restrict__ ab, T *__restrict__ e, int sweeps,
                                                      int periodic)
{
    extern __shared__ unsigned char smem_raw[];
    const int N = g.n[0] * g.n[1] * g.n[2];
    T *eA = reinterpret_cast<T *>(smem_raw);
    T *eB = eA + 4 * N;
    T *fs = eB + 4 * N;
    T *cs = fs + 4 * N;
    for (int q = threadIdx.x; q < N; q += blockDim.x) {
        for (int a = 0; a < 4; ++a) {
            eA[a * N + q] = 0;
            fs[a * N + q] = f[a * N + q];
        }
        cs[q] = ab[q];
        cs[N + q] = ab[N + q];
    }
    __syncthreads();
    for (int s = 0; s < sweeps; ++s)
        for (int colour = 0; colour < 2; ++colour) {
            for (int q = threadIdx.x; q < N; q += blockDim.x) {
                int i = q % g.n[0], j = (q / g.n[0]) % g.n[1], k = q / (g.n[0] * g.n[1]);
                if (((i + j + k) & 1) == colour) {
                    T Je[4], ctr[4];
                    AccB<T, BC> a0{eA, 0, &g, i, j, k}, a1{eA + N, 1, &g, i, j, k}, a2{eA + 2 * N, 2, &g, i, j, k},
                        a3{eA + 3 * N, 3, &g, i, j, k};
                    apply_J<ORDER, T>(a0, a1, a2, a3, cs[q], cs[N + q], cf, Je, ctr);
                    T dl, kW[3];
                    relax_factors<BC>(cf.fd, g, i, j, k, true, cf.dl, cf.idW, cf.iom, dl, kW);
                    eB[q] = ctr[0] + (fs[q] - Je[0]) / ((cs[q] * dl + cs[N + q]) * cf.iom);
                    for (int a = 0; a < 3; ++a)
                        eB[(1 + a) * N + q] = ctr[1 + a] + (fs[(1 + a) * N + q] - Je[1 + a]) * kW[a];
                } else {
                    for (int a = 0; a < 4; ++a) eB[a * N + q] = eA[a * N + q];
                }
            }
            __syncthreads();
            T *t = eA; eA = eB; eB = t;
        }
    if (periodic) {
        double v[4] = {0, 0, 0, 0};
        for (int q = threadIdx.x; q < N; q += blockDim.x)
            for (int a = 0; a < 4; ++a) v[a] += (double)eA[a * N + q];
        double r[4];
        block_sum<4>(v, r);
        __shared__ double mean[4];
        if (threadIdx.x == 0)
            for (int a = 0; a < 4; ++a) mean[a] = r[a] / N;
        __syncthreads();
        for (int q = threadIdx.x; q < N; q += blockDim.x)
            for (int a = 0; a < 4; ++a) e[a * N + q] = eA[a * N + q] - (T)mean[a];
    } else {
        for (int q = threadIdx.x; q < N; q += blockDim.x)
            for (int a = 0; a < 4; ++a) e[a * N + q] = eA[a * N + q];
    }
}

// Coarsest level, psi row only: assemble the dense matrix of a Lap + b (boundary values folded
// into the columns: periodic wrap, the mirror cell across a symmetry plane, or the Robin ratio
// |x_b|/|x_g| onto the clamped cell),
// bordered on periodic boxes by a constant Lagrange multiplier with the constraint <e> = 0,
// and solve it by Gaussian elimination with partial pivoting in shared memory.  The exact
// solve keeps the V-cycle contracting when the psi operator is indefinite on its lowest
// modes (c comparable to the smallest Laplacian eigenvalue), where Gauss-Seidel diverges.
// Overwrites e[0 .. N).  Shared memory: (m^2 + m) T, m = N + periodic.
template <typename T, int ORDER, int BC>
__global__ void __launch_bounds__(512) k_coarse_psi_direct(Geo g, Coef<T> cf, const T *__restrict__ f,
                                                           const T *__restrict__ ab, T *__restrict__ e,
                                                           int periodic)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ int piv;
    const int N = g.n[0] * g.n[1] * g.n[2];
    const int m = N + (periodic ? 1 : 0);
    const int tid = threadIdx.x, bs = blockDim.x;
    T *A = reinterpret_cast<T *>(smem_raw);
    T *rhs = A + (size_t)m * m;
    for (int t = tid; t < m * m; t += bs) A[t] = 0;
    __syncthreads();
    const T w1 = ORDER == 2 ? (T)1 : (T)(16.0 / 12.0);
    const T w2 = ORDER == 2 ? (T)0 : (T)(-1.0 / 12.0);
    for (int p = tid; p < N; p += bs) {
        int i = p % g.n[0], j = (p / g.n[0]) % g.n[1], k = p / (g.n[0] * g.n[1]);
        T a = ab[p], b = ab[N + p];
        T *row = A + (size_t)p * m;
        row[p] += a * cf.dl + b;
        for (int ax = 0; ax < 3; ++ax)
            for (int s = -2; s <= 2; ++s) {
                if (s == 0 || (ORDER == 2 && (s == 2 || s == -2))) continue;
                T w = a * ((s == 1 || s == -1) ? w1 : w2) * cf.ih2[ax];
                int c[3] = {i, j, k};
                c[ax] += s;
                if (BC == BC_PERIODIC) {
                    c[ax] += c[ax] < 0 ? g.n[ax] : 0;
                    c[ax] -= c[ax] >= g.n[ax] ? g.n[ax] : 0;
                    row[c[0] + g.n[0] * (c[1] + g.n[1] * c[2])] += w;
                } else {   // psi is even across symmetry planes: mirror, or clamp with the 1/r ratio
                    int bc[3], mirror;
                    double ratio = 1.0;
                    if (bc_cell<BC>(g, c, bc, mirror)) ratio = robin_ratio<double>(g, bc[0], bc[1], bc[2], c[0], c[1], c[2]);
                    row[bc[0] + g.n[0] * (bc[1] + g.n[1] * bc[2])] += (T)((double)w * ratio);
                }
            }
        if (periodic) {
            row[N] = 1;
            A[(size_t)N * m + p] = 1;
        }
        rhs[p] = f[p];
    }
    if (periodic && tid == 0) rhs[N] = 0;
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        if (tid < 32) {   // pivot: largest |A[i][k]|, i >= k (ties: smallest i)
            T best = (T)-1;
            int bi = m;
            for (int i = k + tid; i < m; i += 32) {
                T v = fabs(A[(size_t)i * m + k]);
                if (v > best) { best = v; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                T ov = __shfl_down_sync(0xffffffffu, best, o);
                int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (tid == 0) piv = bi;
        }
        __syncthreads();
        const int pr = piv;
        if (pr != k) {
            for (int jj = k + tid; jj <= m; jj += bs) {
                T *x = jj < m ? &A[(size_t)k * m + jj] : &rhs[k];
                T *y = jj < m ? &A[(size_t)pr * m + jj] : &rhs[pr];
                T t = *x; *x = *y; *y = t;
            }
            __syncthreads();
        }
        const T pv = A[(size_t)k * m + k];
        for (int i = k + 1 + tid; i < m; i += bs) A[(size_t)i * m + k] /= pv;
        __syncthreads();
        const int rows = m - k - 1, cols = m - k;   // cols: A[i][k+1 .. m-1] and rhs[i]
        for (int t = tid; t < rows * cols; t += bs) {
            int i = k + 1 + t / cols, jj = t % cols;
            T l = A[(size_t)i * m + k];
            if (jj < cols - 1) A[(size_t)i * m + k + 1 + jj] -= l * A[(size_t)k * m + k + 1 + jj];
            else rhs[i] -= l * rhs[k];
        }
        __syncthreads();
    }
    for (int k = m - 1; k >= 0; --k) {
        if (tid == 0) rhs[k] /= A[(size_t)k * m + k];
        __syncthreads();
        for (int i = tid; i < k; i += bs) rhs[i] -= A[(size_t)i * m + k] * rhs[k];
        __syncthreads();
    }
    for (int p = tid; p < N; p += bs) e[p] = rhs[p];
}

}  // namespace ctt
