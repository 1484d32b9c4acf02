// mg_common.cuh -- context, status helpers and workspace layout shared by the host TUs.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/ctt_mg.h"
#include "mg_kernels.cuh"
#include "mg_tile.cuh"
#include "mg_outer.cuh"
#include "mg_coarse.cuh"

namespace ctt {

mg_status fail(mg_status s, const std::string &msg);

#define CK(...)                                                                                        \
    do {                                                                                               \
        cudaError_t e_ = (__VA_ARGS__);                                                                     \
        if (e_ != cudaSuccess)                                                                         \
            return ::ctt::fail(e_ == cudaErrorMemoryAllocation ? MG_ERR_OOM : MG_ERR_CUDA,              \
                               std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_));                    \
    } while (0)

#define CKS(...)                                                                                       \
    do {                                                                                               \
        mg_status s_ = (__VA_ARGS__);                                                                       \
        if (s_ != MG_OK) return s_;                                                                    \
    } while (0)

constexpr int kThreads = 256;
constexpr int kRedBlocks = 152 * 8;   // reduction partials per pass (grid-stride beyond this)

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

inline int grid_for(size_t work, int maxb = 152 * 16, int threads = kThreads)
{
    size_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)std::min<size_t>(b, (size_t)maxb);
}

inline int auto_levels(const int n[3])
{
    int m[3] = {n[0], n[1], n[2]}, lev = 1;
    for (;;) {
        bool ok = true;
        for (int a = 0; a < 3; ++a)
            if (m[a] % 2 != 0 || m[a] / 2 < 3) ok = false;
        if (!ok) break;
        for (int a = 0; a < 3; ++a) m[a] /= 2;
        ++lev;
    }
    return lev;
}

struct LevelBufs {
    Geo geo;
    size_t N;
    void *eA, *eB, *f, *c;   // T arrays: 4N, 4N, 4N, 2N (c holds the psi-row coefficients a, b)
    int split;               // 1: colour-split storage (every level above the coarsest), 0: plain
    int curB;                // enqueue-time bookkeeping: 1 when eB holds the current correction
    int tiled;               // 1: colour passes and the restriction run the TMA-tiled kernels
    TileGrid tg, tgr;        // launch shapes of the colour pass and of the residual + restriction
    CUtensorMap tmA, tmB;    // 5-D maps of eA, eB: (pair, row, plane, field, colour half)
    void *cur() const { return curB ? eB : eA; }
    void *alt() const { return curB ? eA : eB; }
    const CUtensorMap &tm_cur() const { return curB ? tmB : tmA; }
    const CUtensorMap &tm_alt() const { return curB ? tmA : tmB; }
};

// Level eligibility and launch shape of the tiled colour pass; `sms` = multiprocessors.
inline bool tile_eligible(const Geo &g, int split)
{
    return split && g.n[0] % 8 == 0 && g.n[1] % 8 == 0 && g.n[0] >= 16 && g.n[1] >= 16 && g.n[2] >= 8;
}

// even: chunks of an even number of planes starting at even z (the restriction pairs planes)
inline TileGrid tile_grid(const Geo &g, int sms, int ctas_per_sm, bool even = false)
{
    TileGrid t;
    t.ntx = (g.n[0] / 2 + kTileP - 1) / kTileP;
    t.nty = g.n[1] / kTileY;
    int chunks = std::max(1, sms * ctas_per_sm / (t.ntx * t.nty));
    // a colour pass may take single planes (small levels: fewer serial plane steps per CTA); the
    // restriction pairs planes
    t.zc = std::max(even ? 2 : 1, (g.n[2] + chunks - 1) / chunks);
    if (even) t.zc += t.zc & 1;
    return t;
}

// Folded inner-operator weights of a level (the discrete operator of apply_J).
template <typename T>
TileCoef<T> make_tile_coef(const Geo &g, int order, double omega = 1.0)
{
    TileCoef<T> t;
    const double c1 = order == 2 ? 0.5 : 8.0 / 12.0, c2 = order == 2 ? 0.0 : 1.0 / 12.0;
    const double k1 = order == 2 ? 1.0 : 16.0 / 12.0, k2 = order == 2 ? 0.0 : -1.0 / 12.0;
    const double k0 = order == 2 ? -2.0 : -30.0 / 12.0;
    double lk0 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double ih2 = 1.0 / (g.h[a] * g.h[a]);
        t.lk1[a] = (T)(k1 * ih2);
        t.lnk2[a] = (T)(k2 * ih2);
        lk0 += k0 * ih2;
    }
    t.lk0 = (T)lk0;
    t.dl = (T)lk0;
    for (int A = 0; A < 3; ++A) {
        const double ihA2 = 1.0 / (g.h[A] * g.h[A]);
        const double m0 = lk0 + k0 * ihA2 / 3.0;
        t.mk0[A] = (T)m0;
        for (int a = 0; a < 3; ++a) {
            const double ih2 = 1.0 / (g.h[a] * g.h[a]), s = a == A ? 4.0 / 3.0 : 1.0;
            t.mk1[A][a] = (T)(s * k1 * ih2);
            t.mnk2[A][a] = (T)(s * k2 * ih2);
        }
        t.d1[A] = (T)(c1 / g.h[A]);
        t.d2[A] = (T)(c2 / g.h[A]);
        t.t1[A] = (T)(c1 / (3.0 * g.h[A]));
        t.t2[A] = (T)(c2 / (3.0 * g.h[A]));
        t.idW[A] = (T)(omega / m0);
    }
    t.iom = (T)(1.0 / omega);
    face_diag<T>(g, order, t.fd);
    return t;
}

inline int tile_ctas(const Geo &g, const TileGrid &t) { return t.ntx * t.nty * ((g.n[2] + t.zc - 1) / t.zc); }

// omega: red-black relaxation weight (1 = plain Gauss-Seidel within the colour pass).
template <typename T>
Coef<T> make_coef(const Geo &g, int order, double omega = 1.0)
{
    Coef<T> cf;
    double w0 = order == 2 ? -2.0 : -30.0 / 12.0;
    double dl = 0.0;
    for (int a = 0; a < 3; ++a) {
        cf.ih[a] = (T)(1.0 / g.h[a]);
        cf.ih2[a] = (T)(1.0 / (g.h[a] * g.h[a]));
        dl += w0 / (g.h[a] * g.h[a]);
    }
    cf.dl = (T)dl;
    for (int a = 0; a < 3; ++a) cf.idW[a] = (T)(omega / (dl + w0 / (g.h[a] * g.h[a]) / 3.0));
    cf.iom = (T)(1.0 / omega);
    face_diag<T>(g, order, cf.fd);
    return cf;
}

inline OuterCoef make_outer_coef(const Geo &g, int order)
{
    OuterCoef o;
    const double w0 = order == 2 ? -2.0 : -30.0 / 12.0;
    o.k0 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double h = g.h[a], h2 = h * h;
        o.c1[a] = (order == 2 ? 0.5 : 8.0 / 12.0) / h;
        o.c2[a] = order == 2 ? 0.0 : (1.0 / 12.0) / h;
        o.k1[a] = (order == 2 ? 1.0 : 16.0 / 12.0) / h2;
        o.nk2[a] = order == 2 ? 0.0 : -(1.0 / 12.0) / h2;
        o.k0 += w0 / h2;
        o.q1[a] = o.c1[a] / 3.0;
        o.q2[a] = o.c2[a] / 3.0;
    }
    for (int A = 0; A < 3; ++A) {
        for (int a = 0; a < 3; ++a) {
            const double s = a == A ? 4.0 / 3.0 : 1.0;
            o.m1[A][a] = s * o.k1[a];
            o.nm2[A][a] = s * o.nk2[a];
        }
        o.m0[A] = o.k0 + w0 / (3.0 * g.h[A] * g.h[A]);
    }
    return o;
}

// Block split of the FP64 residual pass B: shell blocks first, then interior-box blocks; at most
// kRedBlocks blocks in all (one reduction partial each).  A periodic shell cell costs about an
// interior cell (q form, wrapped); a Robin shell cell takes the tensor-product form with boundary
// values, several times the arithmetic, so Robin boxes give the shell up to half the blocks.
inline Regions outer_regions(const Geo &g, int order, int robin, int *grid)
{
    Regions r;
    r.G = order / 2;
    long long ix = g.n[0] - 2 * r.G, iy = g.n[1] - 2 * r.G, iz = g.n[2] - 2 * r.G;
    size_t nint = (ix > 0 && iy > 0 && iz > 0) ? (size_t)ix * iy * iz : 0;
    size_t nsh = shell_count(g.n, r.G);
    int bs = nsh ? grid_for(nsh, robin ? kRedBlocks / 2 : 152, kThreads) : 0;
    int bi = nint ? grid_for(nint, kRedBlocks - bs, kThreads) : 0;
    r.nblk_sh = bs;
    *grid = std::max(1, bi + bs);
    return r;
}

// Dense coarsest-level solve: available when the bordered W system has at most kDenseMaxW rows.
inline bool dense_eligible(const int nc[3], int periodic)
{
    return dense_m_w(nc[0] * nc[1] * nc[2], periodic) <= kDenseMaxW;
}

inline size_t coarse_smem_bytes(size_t Nc, size_t tb) { return 14 * Nc * tb; }
constexpr size_t kMaxCoarseSmem = 200 * 1024;
inline size_t direct_smem_bytes(size_t Nc, int periodic, size_t tb)
{
    size_t m = Nc + (periodic ? 1 : 0);
    return (m * m + m) * tb;
}

}  // namespace ctt

struct mg_ctx;
namespace ctt {
// The learned warm start (mg_warmstart.cu).
struct WarmNet;
mg_status warm_load(const char *path, cudaStream_t st, WarmNet **out);
void warm_free(WarmNet *w);
bool warm_supported(const WarmNet *w, const mg_ctx *x);
mg_status warm_enqueue(WarmNet *w, mg_ctx *x, cudaStream_t st);
bool warm_timed_out(WarmNet *w, cudaStream_t st);
}  // namespace ctt

struct mg_ctx {
    mg_config cfg;
    cudaStream_t user_stream = nullptr;   // the caller's stream (may be the legacy default stream)
    cudaStream_t stream = nullptr;        // private non-blocking stream: all library work and captures
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaStream_t side = nullptr;           // parallel branch: the per-iteration psi inverse
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool join_pending = false;             // enqueue-time: the next coarse solve waits for ev_join
    int nlev = 0;
    size_t N = 0;
    size_t tbytes = 8;   // sizeof(T) of the inner solve
    int threads = 256;   // threads per block of the smoother, residual+restriction and prolongation
    int sms = 152;       // multiprocessors of the device
    double omega = 1.0;  // red-black relaxation weight
    int gamma = 1;       // coarse-level visits per cycle (1 = V, 2 = W)
    std::vector<ctt::LevelBufs> lev;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false;
    double *X = nullptr;     // 4N: u, Wx, Wy, Wz
    double *SRC = nullptr;   // 5N: rho0, rho2, Sx, Sy, Sz
    double *R = nullptr;     // 5N: outer pass-1 output
    double *D = nullptr;     // 4N: q_0, q_1, q_2, div W of the FP64 residual's pass A
    int dense = 0;           // 1: the coarsest level is solved with the dense inverses below
    int fused = 0;           // 1: the next-to-coarsest level's cycle runs in one CTA (k_coarse_cycle)
    int mpsi = 0, mw = 0;    // orders of the (bordered) psi and W systems
    void *Gpsi = nullptr;    // mpsi^2 T: inverse of the psi row (per outer iteration)
    void *GW = nullptr;      // mw^2 T: inverse of the W rows (once, at creation)
    void *gj = nullptr;      // Gauss-Jordan scratch, gj_scratch_elems(mw) doubles
    double *partial = nullptr;
    ctt::Scalars *scal = nullptr;
    ctt::Scalars *host_scal = nullptr;   // pinned
    bool have_sources = false;
    cudaGraphExec_t graph_exec = nullptr;   // one captured outer iteration
    cudaGraphExec_t graph_start = nullptr;  // gauge projection + first residual
    long long launches_iter = 0, launches_start = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<double> history;
    mg_ctx *child = nullptr;   // half-size problem of the nested start (its workspace is carved from ws)
    bool guess_set = false;    // the caller gave an initial guess since the previous solve
    ctt::WarmNet *warm = nullptr;           // learned warm start (mg_warmstart_load); a batch's is shared
    bool warm_owned = false;                // this context frees it
    cudaGraphExec_t warm_graph = nullptr;   // the inference, captured for this context's buffers
    long long launches_warm = 0;
    bool device_paced = false;              // enqueue-time: a batch controller kernel reads the scalars on the device
    void *zbuf = nullptr;                   // k2_newton: the z solve's result, 4N T in the finest layout (psi: z)
    void *zrhs = nullptr;                   // k2_newton: its right-hand side, 4N T (psi row -1/12, W rows 0)
    bool zsolve = false;                    // enqueue-time: the next inner solve is the z solve
    cudaGraphExec_t graph_z = nullptr;      // the z solve, captured
    long long launches_z = 0;
};

namespace ctt {
// Per-(precision, order, boundary variant) engine entry points, instantiated in mg_engine_*.cu.
template <typename T, int ORDER, int BC> mg_status engine_iteration(mg_ctx *x);
template <typename T, int ORDER, int BC> mg_status engine_residual(mg_ctx *x, double *HM);
template <typename T, int ORDER, int BC> mg_status engine_time_kernel(mg_ctx *x, int which, int reps, float *ms);
template <typename T, int ORDER, int BC> mg_status engine_prepare(mg_ctx *x);
template <typename T, int ORDER, int BC> mg_status engine_dense_setup(mg_ctx *x);
}  // namespace ctt
