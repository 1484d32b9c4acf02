// mg_coarse.cuh -- coarsest-level solve by precomputed dense inverses.
//
// The coarsest grid of the hierarchy has at most a few hundred cells, so its two linear blocks
// are solved exactly by multiplying with explicit inverses:
//   psi row: a Lap + b (a, b: the restricted psi-row coefficients of the current outer iteration),
//            re-inverted once per outer iteration;
//   W rows:  Lap W_i + (1/3) (D_ii W_i + sum_{j != i} D_i D_j W_j), which does not depend on the
//            state, inverted once when the context is created.
// On periodic boxes both operators annihilate constants; each is bordered by one Lagrange
// multiplier per field with the constraint <e> = 0, so the inverse maps any right-hand side to
// the zero-mean solution of the projected problem.  The matrices are assembled from the same
// stencil code as the smoother (boundary values folded into the columns) and inverted in one
// CTA; a V-cycle then spends one small matrix-vector kernel on its coarsest level.
#pragma once
#include "mg_kernels.cuh"
#include "mg_tile.cuh"

namespace ctt {

constexpr int kDenseMaxW = 400;   // largest bordered W system (3 N + 3) solved densely

__host__ __device__ inline int dense_m_psi(int N, int periodic) { return N + (periodic ? 1 : 0); }
__host__ __device__ inline int dense_m_w(int N, int periodic) { return 3 * N + (periodic ? 3 : 0); }

// [A | I] of the psi row, row stride 2m (global scratch, zeroed here).
template <typename T, typename C, int ORDER, int BC>
__global__ void __launch_bounds__(512) k_dense_psi_assemble(Geo g, Coef<T> cf, const T *__restrict__ ab,
                                                            C *__restrict__ aug, int periodic)
{
    const int N = g.n[0] * g.n[1] * g.n[2];
    const int m = dense_m_psi(N, periodic), w2 = 2 * m;
    for (int t = threadIdx.x; t < m * w2; t += blockDim.x) aug[t] = 0;
    __syncthreads();
    const double w1 = ORDER == 2 ? 1.0 : 16.0 / 12.0;
    const double wb = ORDER == 2 ? 0.0 : -1.0 / 12.0;
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
        const int i = p % g.n[0], j = (p / g.n[0]) % g.n[1], k = p / (g.n[0] * g.n[1]);
        const double a = (double)ab[p], b = (double)ab[N + p];
        C *row = aug + (size_t)p * w2;
        row[p] += (C)(a * (double)cf.dl + b);
        for (int ax = 0; ax < 3; ++ax)
            for (int s = -2; s <= 2; ++s) {
                if (s == 0 || (ORDER == 2 && (s == 2 || s == -2))) continue;
                const double w = a * ((s == 1 || s == -1) ? w1 : wb) * (double)cf.ih2[ax];
                int c[3] = {i, j, k};
                c[ax] += s;
                if (BC == BC_PERIODIC) {
                    c[ax] += c[ax] < 0 ? g.n[ax] : 0;
                    c[ax] -= c[ax] >= g.n[ax] ? g.n[ax] : 0;
                    row[c[0] + g.n[0] * (c[1] + g.n[1] * c[2])] += (C)w;
                } else {   // psi is even across symmetry planes: mirror, or clamp with the 1/r ratio
                    auto add = [&](const int q[3], double wq) {
                        int bc[3], mirror;
                        double ratio = 1.0;
                        if (bc_cell<BC>(g, q, bc, mirror)) ratio = robin_ratio<double>(g, bc[0], bc[1], bc[2], q[0], q[1], q[2]);
                        row[bc[0] + g.n[0] * (bc[1] + g.n[1] * bc[2])] += (C)(wq * ratio);
                    };
                    int q[8][3], wx[8], ns = 0;
                    if constexpr (BC == BC_SYM) ns = g.extrap ? extrap_split(g, c, q, wx) : 0;
                    if (ns)   // beyond an extrapolating face: the weighted in-box cells
                        for (int t = 0; t < ns; ++t) add(q[t], w * wx[t]);
                    else
                        add(c, w);
                }
            }
        if (periodic) {
            row[N] = 1;
            aug[(size_t)N * w2 + p] = 1;
        }
    }
    for (int r = threadIdx.x; r < m; r += blockDim.x) aug[(size_t)r * w2 + m + r] = 1;
}

// [A | I] of the W rows: one CTA per column (field B, cell q) applies the operator to the unit
// vector e_(B,q) held in shared memory (4 N T) and writes the column; one more CTA (index 3N)
// writes the multiplier columns and the identity entries of the constraint rows.  aug must be
// zero beforehand.
template <typename T, typename C, int ORDER, int BC>
__global__ void __launch_bounds__(256) k_dense_w_assemble(Geo g, Coef<T> cf, C *__restrict__ aug, int periodic)
{
    extern __shared__ unsigned char smem_raw[];
    T *e = reinterpret_cast<T *>(smem_raw);
    const int N = g.n[0] * g.n[1] * g.n[2];
    const int m = dense_m_w(N, periodic), w2 = 2 * m;
    const int col = blockIdx.x;
    if (col >= 3 * N) {   // multiplier columns and their identity entries
        if (periodic && threadIdx.x < 3) {
            const int B = threadIdx.x;
            aug[(size_t)(3 * N + B) * w2 + m + 3 * N + B] = 1;
        }
        return;
    }
    const int B = col / N, q = col % N;
    for (int t = threadIdx.x; t < 4 * N; t += blockDim.x) e[t] = 0;
    __syncthreads();
    if (threadIdx.x == 0) e[(1 + B) * N + q] = 1;
    __syncthreads();
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
        const int i = p % g.n[0], j = (p / g.n[0]) % g.n[1], k = p / (g.n[0] * g.n[1]);
        AccB<T, BC> a0{e, 0, &g, i, j, k}, a1{e + N, 1, &g, i, j, k}, a2{e + 2 * N, 2, &g, i, j, k},
            a3{e + 3 * N, 3, &g, i, j, k};
        T Je[4], ctr[4];
        apply_J<ORDER, T>(a0, a1, a2, a3, (T)1, (T)0, cf, Je, ctr);
        for (int A = 0; A < 3; ++A) aug[(size_t)(A * N + p) * w2 + col] = (C)Je[1 + A];
    }
    if (threadIdx.x == 0) {
        if (periodic) {
            aug[(size_t)(3 * N + B) * w2 + col] = 1;   // constraint row of field B: sum of its cells
            aug[(size_t)col * w2 + 3 * N + B] = 1;     // multiplier column of field B
        }
        aug[(size_t)col * w2 + m + col] = 1;           // identity block
    }
}

// Gauss-Jordan elimination with partial pivoting of the m x 2m augmented matrix [A | I] (row
// stride 2m) into [I | A^-1]; writes A^-1 (row-major, m x m) as T.  One CTA.  Scratch after the
// matrix: pivot row (2m), old row k (2m), column factors (m), gj_scratch_elems(m) in all; with
// smem_ok it is all copied into dynamic shared memory first.  Per column: pivot search (one
// warp), staging of the scaled pivot row, the old row k and the factors, then one elimination
// pass (one warp per row) in which row k takes the pivot row and the pivot row's slot takes
// the old row k (the swap).  A zero pivot yields non-finite entries, which the outer iteration reports as
// divergence.
__host__ __device__ inline size_t gj_scratch_elems(int m) { return (size_t)2 * m * m + 5 * (size_t)m; }

template <typename C, typename T>
__global__ void __launch_bounds__(1024) k_gauss_jordan(C *__restrict__ gaug, int m, int smem_ok, T *__restrict__ inv)
{
    extern __shared__ unsigned char smem_raw[];
    const int w2 = 2 * m, tid = threadIdx.x, bs = blockDim.x;
    C *A = smem_ok ? reinterpret_cast<C *>(smem_raw) : gaug;
    C *prow = A + (size_t)m * w2, *krow = prow + w2, *fct = krow + w2;
    __shared__ int piv;
    if (smem_ok)
        for (int t = tid; t < m * w2; t += bs) A[t] = gaug[t];
    __syncthreads();
    for (int k = 0; k < m; ++k) {
        if (tid < 32) {
            C best = -1;
            int bi = m;
            for (int i = k + tid; i < m; i += 32) {
                const C v = fabs(A[(size_t)i * w2 + k]);
                if (v > best) { best = v; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const C ov = __shfl_down_sync(0xffffffffu, best, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
            }
            if (tid == 0) piv = bi;
        }
        __syncthreads();
        const int pr = piv < m ? piv : k;   // an all-NaN column leaves the rows in place
        const C ip = (C)1 / A[(size_t)pr * w2 + k];
        // columns left of k are already reduced (zero in rows k and pr), so only j >= k change
        for (int j = k + tid; j < w2; j += bs) {
            prow[j] = A[(size_t)pr * w2 + j] * ip;
            krow[j] = A[(size_t)k * w2 + j];
        }
        for (int i = tid; i < m; i += bs) fct[i] = A[(size_t)(i == pr ? k : i) * w2 + k];
        __syncthreads();
        for (int i = tid >> 5; i < m; i += bs >> 5) {   // one warp per row, lanes along the row
            C *row = A + (size_t)i * w2;
            const C fi = fct[i];
            if (i == k)
                for (int j = k + (tid & 31); j < w2; j += 32) row[j] = prow[j];
            else if (i == pr)
                for (int j = k + (tid & 31); j < w2; j += 32) row[j] = krow[j] - fi * prow[j];
            else
                for (int j = k + (tid & 31); j < w2; j += 32) row[j] -= fi * prow[j];
        }
        __syncthreads();
    }
    for (int t = tid; t < m * m; t += bs) {
        const int i = t / m, j = t - i * m;
        inv[t] = (T)A[(size_t)i * w2 + m + j];
    }
}

// Coarsest-level correction: e_psi = Gpsi[0:N, 0:N] f_psi, e_W = GW[0:3N, 0:3N] f_W (the
// bordered rows and columns belong to the multipliers; their right-hand side is zero).  One
// warp per output row; FP32 rows accumulate in FP32, FP64 rows in FP64.
template <typename T>
__global__ void __launch_bounds__(256) k_dense_apply(const T *__restrict__ Gpsi, int mpsi, const T *__restrict__ GW,
                                                     int mw, const T *__restrict__ f, T *__restrict__ e, int N)
{
    const int row = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (row >= 4 * N) return;
    T acc = 0;
    if (row < N) {
        const T *g = Gpsi + (size_t)row * mpsi;
        for (int j = lane; j < N; j += 32) acc = fma(g[j], f[j], acc);
    } else {
        const T *g = GW + (size_t)(row - N) * mw;
        for (int j = lane; j < 3 * N; j += 32) acc = fma(g[j], f[N + j], acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) e[row] = acc;
}

// ---------------------------------------------------------------------------------------
// The bottom of a cycle in one CTA: when the next-to-coarsest level (l = Lc - 1) is small, its
// pre-smoothing, the residual's 8-child restriction, the coarsest solve by the dense inverses,
// the trilinear prolongation and the post-smoothing run in shared memory in one launch (the same
// operator, colour passes and Jacobi-within-colour reads as the per-kernel path).  Level l is
// colour-split in global memory and plain in shared memory; the coarsest level is plain.
constexpr int kFusedMaxCells = 1728;   // next-to-coarsest level up to 12^3 cells
// threads of k_coarse_cycle: 128 registers per thread for FP32 (255 for FP64), which the 4th-order
// stencil with Robin ratios needs without spilling
template <typename T> constexpr int fused_threads() { return sizeof(T) == 8 ? 256 : 512; }

// Shared memory of k_coarse_cycle: the level's state, ping-pong copy, rhs and coefficients, the
// coarsest level's rhs and solution, and on Robin boxes the level's ghost ratios (rt_cells =
// (n0+4)(n1+4)(n2+4), else 0).
__host__ __device__ inline size_t fused_smem_bytes(int N1, int Nc, size_t tb, size_t rt_cells)
{
    return (14 * (size_t)N1 + 8 * (size_t)Nc + rt_cells) * tb;
}

inline size_t fused_ratio_cells(const Geo &g, int robin)
{
    return robin ? (size_t)(g.n[0] + 4) * (g.n[1] + 4) * (g.n[2] + 4) : 0;
}

// Robin accessor of the fused cycle: the value of the cell bc_cell maps to, times the level's
// ghost ratio read from the table rt over the box padded by 2 (1 inside or only mirrored), so no
// square root per access; fi is the field (0 = u, 1..3 = W_x..W_z) for the sign across symmetry
// planes.
template <typename T, int BC>
struct AccRT {
    const T *f;
    int fi;
    const T *rt;
    const Geo *g;
    int i, j, k;
    __device__ __forceinline__ T operator()(int dx, int dy, int dz) const
    {
        const int p[3] = {i + dx, j + dy, k + dz};
        int b[3], mirror;
        bc_cell<BC>(*g, p, b, mirror);
        const T v = f[b[0] + g->n[0] * (b[1] + g->n[1] * b[2])] *
                    rt[(p[0] + 2) + (g->n[0] + 4) * ((p[1] + 2) + (g->n[1] + 4) * (p[2] + 2))];
        return bc_signed<BC>(v, mirror, fi);
    }
};

// gsm = 1: the shared memory also holds the coarsest level's dense inverses (Gpsi's Nc x Nc block,
// then GW's 3Nc x 3Nc block); their per-thread cp.async copies are issued first and land while the
// level is smoothed, so the coarsest solve reads shared memory instead of waiting on global loads.
template <typename T, int ORDER, int BC>
__global__ void __launch_bounds__(fused_threads<T>()) k_coarse_cycle(Geo g, Coef<T> cf, Geo gc, const T *__restrict__ f,
                                                       const T *__restrict__ ab, const T *__restrict__ e_in,
                                                       T *__restrict__ e_out, int zero, int nu_pre, int nu_post,
                                                       const T *__restrict__ Gpsi, int mpsi,
                                                       const T *__restrict__ GW, int mw, int gsm)
{
    extern __shared__ unsigned char smem_raw[];
    const int N = g.n[0] * g.n[1] * g.n[2], Nc = gc.n[0] * gc.n[1] * gc.n[2];
    const int tid = threadIdx.x, bs = blockDim.x;
    T *cur = reinterpret_cast<T *>(smem_raw);
    T *alt = cur + 4 * N;
    T *fs = alt + 4 * N;
    T *cs = fs + 4 * N;
    T *fc = cs + 2 * N;
    T *ec = fc + 4 * Nc;
    T *rt = ec + 4 * Nc;   // Robin: ghost ratios of the level over its box padded by 2
    T *sG = rt + (BC != BC_PERIODIC ? (g.n[0] + 4) * (g.n[1] + 4) * (g.n[2] + 4) : 0);   // staged inverses
    const int M3 = 3 * Nc;
    if (gsm) {
        for (int e = threadIdx.x; e < Nc * Nc; e += blockDim.x) {
            const int r = e / Nc;
            tile_copy_async(sG + e, Gpsi + (size_t)r * mpsi + (e - r * Nc));
        }
        for (int e = threadIdx.x; e < M3 * M3; e += blockDim.x) {
            const int r = e / M3;
            tile_copy_async(sG + Nc * Nc + e, GW + (size_t)r * mw + (e - r * M3));
        }
        tile_copy_commit();
    }
    auto ijk = [&](int q, int &i, int &j, int &k) {
        i = q % g.n[0];
        j = (q / g.n[0]) % g.n[1];
        k = q / (g.n[0] * g.n[1]);
    };
    auto split_idx = [&](int q) {
        int i, j, k;
        ijk(q, i, j, k);
        return (((i + j + k) & 1) ? N / 2 : 0) + (q >> 1);
    };
    for (int q = tid; q < N; q += bs) {
        const int sq = split_idx(q);
        for (int a = 0; a < 4; ++a) {
            fs[a * N + q] = f[a * N + sq];
            cur[a * N + q] = zero ? (T)0 : e_in[a * N + sq];
        }
        cs[q] = ab[sq];
        cs[N + q] = ab[N + sq];
    }
    if constexpr (BC != BC_PERIODIC) {
        const int m0 = g.n[0] + 4, m1 = g.n[1] + 4, M = m0 * m1 * (g.n[2] + 4);
        for (int e = tid; e < M; e += bs) {
            const int c[3] = {e % m0 - 2, (e / m0) % m1 - 2, e / (m0 * m1) - 2};
            int b[3], mirror;
            rt[e] = bc_cell<BC>(g, c, b, mirror) ? robin_ratio<T>(g, b[0], b[1], b[2], c[0], c[1], c[2]) : (T)1;
        }
    }
    __syncthreads();
    // J e at cell (i, j, k) of the level held in e
    auto apply = [&](const T *e, int i, int j, int k, T a, T b, T Je[4], T ctr[4]) {
        if constexpr (BC != BC_PERIODIC) {
            AccRT<T, BC> a0{e, 0, rt, &g, i, j, k}, a1{e + N, 1, rt, &g, i, j, k}, a2{e + 2 * N, 2, rt, &g, i, j, k},
                a3{e + 3 * N, 3, rt, &g, i, j, k};
            apply_J<ORDER, T>(a0, a1, a2, a3, a, b, cf, Je, ctr);
        } else {
            AccB<T, BC> a0{e, 0, &g, i, j, k}, a1{e + N, 1, &g, i, j, k}, a2{e + 2 * N, 2, &g, i, j, k},
                a3{e + 3 * N, 3, &g, i, j, k};
            apply_J<ORDER, T>(a0, a1, a2, a3, a, b, cf, Je, ctr);
        }
    };
    // one colour pass, ping-pong: thread t takes pair t % (nx/2) of row t / (nx/2) (nx is even on
    // every level above the coarsest); the pair's cell of the colour gets its new value in alt
    // (Jacobi within the colour: all reads see cur), the other cell is copied; then swap
    const int nxh = g.n[0] >> 1, Nh = N >> 1;
    auto sweeps = [&](int n) {
        for (int s = 0; s < n; ++s)
            for (int colour = 0; colour < 2; ++colour) {
                for (int t = tid; t < Nh; t += bs) {
                    const int row = t / nxh, j = row % g.n[1], k = row / g.n[1];
                    const int par = (colour + j + k) & 1;
                    const int i = 2 * (t - row * nxh) + par;
                    const int q = i + g.n[0] * row, qo = q + 1 - 2 * par;   // the pair's other cell
                    T Je[4], ctr[4];
                    apply(cur, i, j, k, cs[q], cs[N + q], Je, ctr);
                    T dl, kW[3];
                    relax_factors<BC>(cf.fd, g, i, j, k, true, cf.dl, cf.idW, cf.iom, dl, kW);
                    alt[q] = ctr[0] + (fs[q] - Je[0]) / ((cs[q] * dl + cs[N + q]) * cf.iom);
                    for (int a = 0; a < 3; ++a)
                        alt[(1 + a) * N + q] = ctr[1 + a] + (fs[(1 + a) * N + q] - Je[1 + a]) * kW[a];
                    for (int a = 0; a < 4; ++a) alt[a * N + qo] = cur[a * N + qo];
                }
                __syncthreads();
                T *tmp = cur;
                cur = alt;
                alt = tmp;
            }
    };
    sweeps(nu_pre);
    // residual r = f - J e at every cell (into alt), then the 8-child means
    for (int q = tid; q < N; q += bs) {
        int i, j, k;
        ijk(q, i, j, k);
        T Je[4], ctr[4];
        apply(cur, i, j, k, cs[q], cs[N + q], Je, ctr);
        for (int a = 0; a < 4; ++a) alt[a * N + q] = fs[a * N + q] - Je[a];
    }
    __syncthreads();
    for (int t = tid; t < 4 * Nc; t += bs) {
        const int a = t / Nc, c = t - a * Nc;
        const int I = c % gc.n[0], J = (c / gc.n[0]) % gc.n[1], K = c / (gc.n[0] * gc.n[1]);
        T sum = 0;
        for (int d = 0; d < 8; ++d) {
            const int i = 2 * I + (d & 1), j = 2 * J + ((d >> 1) & 1), k = 2 * K + (d >> 2);
            sum += alt[a * N + i + g.n[0] * (j + g.n[1] * k)];
        }
        fc[t] = sum * (T)0.125;
    }
    if (gsm) tile_copy_wait_all();
    __syncthreads();
    // coarsest level: e_c = G f_c (psi rows: Gpsi, W rows: GW), one warp per row
    for (int r = tid >> 5; r < 4 * Nc; r += bs >> 5) {
        T acc = 0;
        if (r < Nc) {
            const T *gr = gsm ? sG + r * Nc : Gpsi + (size_t)r * mpsi;
            for (int j = tid & 31; j < Nc; j += 32) acc = fma(gr[j], fc[j], acc);
        } else {
            const T *gr = gsm ? sG + Nc * Nc + (r - Nc) * M3 : GW + (size_t)(r - Nc) * mw;
            for (int j = tid & 31; j < 3 * Nc; j += 32) acc = fma(gr[j], fc[Nc + j], acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if ((tid & 31) == 0) ec[r] = acc;
    }
    __syncthreads();
    // trilinear prolongation (3/4, 1/4 per axis; coarse boundary values from the BC) into e
    const int ncx = gc.n[0], ncy = gc.n[1];
    for (int q = tid; q < N; q += bs) {
        int i, j, k;
        ijk(q, i, j, k);
        const int I = i >> 1, J = j >> 1, K = k >> 1;
        const int sx = (i & 1) ? 1 : -1, sy = (j & 1) ? 1 : -1, sz = (k & 1) ? 1 : -1;
        T s4[4] = {0, 0, 0, 0};
        for (int d = 0; d < 8; ++d) {
            const int dx = d & 1, dy = (d >> 1) & 1, dz = d >> 2;
            const int cc[3] = {I + dx * sx, J + dy * sy, K + dz * sz};
            T w = (T)((dx ? 0.25 : 0.75) * (dy ? 0.25 : 0.75) * (dz ? 0.25 : 0.75));
            int b[3], mirror;
            if (bc_cell<BC>(gc, cc, b, mirror)) w *= robin_ratio<T>(gc, b[0], b[1], b[2], cc[0], cc[1], cc[2]);
            const int c = b[0] + ncx * (b[1] + ncy * b[2]);
            for (int a = 0; a < 4; ++a) s4[a] = fma(bc_signed<BC>(w, mirror, a), ec[a * Nc + c], s4[a]);
        }
        for (int a = 0; a < 4; ++a) cur[a * N + q] += s4[a];
    }
    __syncthreads();
    sweeps(nu_post);
    for (int q = tid; q < N; q += bs) {
        const int sq = split_idx(q);
        for (int a = 0; a < 4; ++a) e_out[a * N + sq] = cur[a * N + q];
    }
}

}  // namespace ctt
