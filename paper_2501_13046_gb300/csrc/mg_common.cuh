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
    void *cur() const { return curB ? eB : eA; }
    void *alt() const { return curB ? eA : eB; }
};

template <typename T>
Coef<T> make_coef(const Geo &g, int order)
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
    for (int a = 0; a < 3; ++a) cf.idW[a] = (T)(1.0 / (dl + w0 / (g.h[a] * g.h[a]) / 3.0));
    return cf;
}

inline size_t coarse_smem_bytes(size_t Nc, size_t tb) { return 14 * Nc * tb; }
constexpr size_t kMaxCoarseSmem = 200 * 1024;
inline size_t direct_smem_bytes(size_t Nc, int periodic, size_t tb)
{
    size_t m = Nc + (periodic ? 1 : 0);
    return (m * m + m) * tb;
}

}  // namespace ctt

struct mg_ctx {
    mg_config cfg;
    cudaStream_t user_stream = nullptr;   // the caller's stream (may be the legacy default stream)
    cudaStream_t stream = nullptr;        // private non-blocking stream: all library work and captures
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int nlev = 0;
    size_t N = 0;
    size_t tbytes = 8;   // sizeof(T) of the inner solve
    int threads = 256;   // threads per block of the smoother, residual+restriction and prolongation
    std::vector<ctt::LevelBufs> lev;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false;
    double *X = nullptr;     // 4N: u, Wx, Wy, Wz
    double *SRC = nullptr;   // 5N: rho0, rho2, Sx, Sy, Sz
    double *R = nullptr;     // 5N: outer pass-1 output
    double *partial = nullptr;
    ctt::Scalars *scal = nullptr;
    ctt::Scalars *host_scal = nullptr;   // pinned
    bool have_sources = false;
    cudaGraphExec_t graph_exec = nullptr;   // one captured outer iteration
    cudaGraphExec_t graph_start = nullptr;  // gauge projection + first residual
    long long launches_iter = 0, launches_start = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<double> history;
};

namespace ctt {
// Per-(precision, order) engine entry points, instantiated in mg_engine_*.cu.
template <typename T, int ORDER> mg_status engine_iteration(mg_ctx *x);
template <typename T, int ORDER> mg_status engine_residual(mg_ctx *x, double *HM);
template <typename T, int ORDER> mg_status engine_time_kernel(mg_ctx *x, int which, int reps, float *ms);
template <typename T, int ORDER> mg_status engine_prepare(mg_ctx *x);
mg_status engine_project_gauge(mg_ctx *x);
}  // namespace ctt
