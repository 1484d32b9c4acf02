// ctt_mg.cu -- C ABI of the CTT constraint multigrid (see include/ctt_mg.h).
//
// Solve (GRTresna, arXiv:2501.13046, eq:Ham/eq:Mom; multigrid, "Key features: Fast"):
//   outer loop in FP64 -- residual, K^2 from the discrete integrability sum on periodic
//   boxes, constraint norms (Key features, "Diagnostics"), convergence test;
//   inner solve -- one linear V-cycle on the block-diagonal linearisation, in FP64
//   (MG_FP64) or FP32 (MG_MIXED: FP32 smoothing/residual/transfer under FP64 defect
//   correction); update u += e, W += e_W in FP64 (zero-mean corrections on periodic boxes).
// Each outer iteration after the first is one replay of a captured CUDA graph; the only
// host synchronisation per iteration is the read of K^2 and the four norms.
#include "mg_common.cuh"
#include "mg_nested.cuh"
#include "mg_batch.cuh"

#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

namespace ctt {

thread_local std::string g_last_error;

mg_status fail(mg_status s, const std::string &msg)
{
    g_last_error = msg;
    return s;
}

// NVTX range for the duration of a scope (host-side phases of a solve; free when no tool listens)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

}  // namespace ctt

using namespace ctt;

namespace {
mg_status validate(const mg_config *c)
{
    if (!c) return fail(MG_ERR_INVALID_ARG, "null config");
    for (int a = 0; a < 3; ++a) {
        if (c->n[a] < 3) return fail(MG_ERR_INVALID_ARG, "n[a] must be >= 3");
        if (!(c->hi[a] > c->lo[a])) return fail(MG_ERR_INVALID_ARG, "hi must exceed lo");
    }
    if ((long long)c->n[0] * c->n[1] * c->n[2] > (1LL << 31)) return fail(MG_ERR_INVALID_ARG, "grid too large");
    if (c->order != 2 && c->order != 4) return fail(MG_ERR_INVALID_ARG, "order must be 2 or 4");
    if (c->bc != MG_BC_PERIODIC && c->bc != MG_BC_ROBIN) return fail(MG_ERR_INVALID_ARG, "bad bc");
    if (c->precision != MG_FP64 && c->precision != MG_MIXED) return fail(MG_ERR_INVALID_ARG, "bad precision");
    if (c->k_mode != MG_K_FIXED && c->k_mode != MG_K_INTEGRABILITY) return fail(MG_ERR_INVALID_ARG, "bad k_mode");
    if (c->k_mode == MG_K_INTEGRABILITY && c->bc != MG_BC_PERIODIC)
        return fail(MG_ERR_INVALID_ARG, "integrability K needs a periodic box");
    if (c->npunct < 0 || c->npunct > 2) return fail(MG_ERR_INVALID_ARG, "npunct must be 0..2");
    if (c->npunct > 0 && c->bc == MG_BC_PERIODIC)
        return fail(MG_ERR_UNSUPPORTED, "punctures need Robin boundaries");
    if (!(c->tol >= 0.0) || c->max_outer < 0 || c->nu_pre < 0 || c->nu_post < 0 || c->coarse_sweeps < 1)
        return fail(MG_ERR_INVALID_ARG, "bad iteration parameters");
    if (!std::isfinite(c->K)) return fail(MG_ERR_INVALID_ARG, "K not finite");
    if (c->inner_cycles < 0 || c->inner_cycles > 8) return fail(MG_ERR_INVALID_ARG, "inner_cycles must be 0..8");
    if (c->block_threads != 0 && c->block_threads != 64 && c->block_threads != 128 && c->block_threads != 256)
        return fail(MG_ERR_INVALID_ARG, "block_threads must be 0, 64, 128 or 256");
    if (c->smoother != 0 && c->smoother != 1) return fail(MG_ERR_INVALID_ARG, "smoother must be 0 or 1");
    if (c->cycle < 0 || c->cycle > 2) return fail(MG_ERR_INVALID_ARG, "cycle must be 0, 1 (V) or 2 (W)");
    if (!(c->omega == 0.0 || (c->omega > 0.0 && c->omega < 2.0)))
        return fail(MG_ERR_INVALID_ARG, "omega must be 0 (default 1) or in (0, 2)");
    for (int p = 0; p < 2; ++p)
        for (int a = 0; a < 3; ++a)
            if (!std::isfinite(c->punct_P[p][a]) || !std::isfinite(c->punct_S[p][a]))
                return fail(MG_ERR_INVALID_ARG, "puncture momentum or spin not finite");
    if (c->reflect < 0 || c->reflect > 7) return fail(MG_ERR_INVALID_ARG, "reflect must be a mask of 3 bits");
    if (c->reflect != 0 && c->bc != MG_BC_ROBIN) return fail(MG_ERR_INVALID_ARG, "symmetry planes need a Robin box");
    if (c->tile_waves < 0 || c->tile_waves > 8) return fail(MG_ERR_INVALID_ARG, "tile_waves must be 0..8");
    if (c->field_est != 0 && c->field_est != 1) return fail(MG_ERR_INVALID_ARG, "field_est must be 0 or 1");
    if (c->k2_newton != 0 && c->k2_newton != 1) return fail(MG_ERR_INVALID_ARG, "k2_newton must be 0 or 1");
    if (c->extrap < 0 || c->extrap > 63) return fail(MG_ERR_INVALID_ARG, "extrap must be a mask of 6 bits");
    if (c->extrap != 0 && c->bc != MG_BC_ROBIN) return fail(MG_ERR_INVALID_ARG, "extrapolating faces need a Robin box");
    for (int a = 0; a < 3; ++a)
        if (((c->reflect >> a) & 1) && ((c->extrap >> (2 * a)) & 1))
            return fail(MG_ERR_INVALID_ARG, "a lower face cannot be both a symmetry plane and extrapolating");
    if (c->bc == MG_BC_ROBIN) {
        int special = c->extrap;
        for (int a = 0; a < 3; ++a) special |= ((c->reflect >> a) & 1) << (2 * a);
        if (special == 63) return fail(MG_ERR_UNSUPPORTED, "a Robin box needs at least one Robin face");
    }
    for (int a = 0; a < 3; ++a)
        if (((c->reflect >> a) & 1) && c->lo[a] != 0.0)
            return fail(MG_ERR_INVALID_ARG, "a symmetry plane must be the face x_a = 0 (lo[a] = 0)");
    if (c->nested != 0 && c->nested != 1) return fail(MG_ERR_INVALID_ARG, "nested must be 0 or 1");
    if (c->nested_min != 0 && c->nested_min < 3) return fail(MG_ERR_INVALID_ARG, "nested_min must be 0 or >= 3");
    if (!(c->nested_tol >= 0.0) || !std::isfinite(c->nested_tol)) return fail(MG_ERR_INVALID_ARG, "bad nested_tol");
    if (!(c->field_tol >= 0.0) || !std::isfinite(c->field_tol)) return fail(MG_ERR_INVALID_ARG, "bad field_tol");
    if (c->use_graph < 0 || c->use_graph > 2) return fail(MG_ERR_INVALID_ARG, "use_graph must be 0, 1 or 2");
    int lv = c->levels > 0 ? c->levels : auto_levels(c->n);
    for (int l = 0; l + 1 < lv; ++l)
        for (int a = 0; a < 3; ++a) {
            int m = c->n[a] >> l;
            if ((m << l) != c->n[a] || m % 2 != 0 || m / 2 < 3)
                return fail(MG_ERR_INVALID_ARG, "levels: every level above the coarsest needs even sizes >= 6");
        }
    return MG_OK;
}

// Punctures with a Bowen-York momentum or spin (only the first npunct count).
bool has_bowen_york(const mg_config *c)
{
    for (int p = 0; p < c->npunct; ++p)
        for (int a = 0; a < 3; ++a)
            if (c->punct_P[p][a] != 0.0 || c->punct_S[p][a] != 0.0) return true;
    return false;
}

// Nested start defaults.  Half sizes below kNestedMinN are not worth solving first: their outer
// iterations cost launch latency, not bandwidth, and save little fine work.  The fine residual of
// the interpolated start is set by the half-size root's own discretisation error (about 1.5e-4 at
// 128^3 from 64^3) once the half-size solve is below it, so kNestedTol stops it near that level
// (measured: 128^3 periodic and 256^3 Robin shell both fastest at 1e-4..3e-4; 1e-3 costs a fine
// iteration on the shell).
constexpr int kNestedMinN = 64;
constexpr double kNestedTol = 3e-4;

// Configuration of the half-size problem of c's nested start; false when c has none.  A valid c gives a
// valid child: its level l is c's level l + 1.
bool nested_child_config(const mg_config *c, mg_config *cc)
{
    if (c->nested != 1) return false;
    const int nmin = c->nested_min > 0 ? c->nested_min : kNestedMinN;
    for (int a = 0; a < 3; ++a)
        if (c->n[a] % 2 != 0 || c->n[a] / 2 < nmin) return false;
    *cc = *c;
    for (int a = 0; a < 3; ++a) cc->n[a] = c->n[a] / 2;
    cc->levels = c->levels > 1 ? c->levels - 1 : 0;
    cc->tol = std::max(c->tol, c->nested_tol > 0.0 ? c->nested_tol : kNestedTol);
    cc->field_tol = 0.0;   // the half-size solve only supplies a starting state
    cc->k2_newton = 0;
    return true;
}

// The per-field part of the stopping test (field_test; always true when field_tol is off, false
// before the first update); prev carries the last relative updates between calls.
bool fields_settled(const mg_config &c, const Scalars &s, int updates, double prev[4])
{
    return field_test(c.field_tol, c.field_est, s.change, prev, updates);
}

void fill_rel_change(const mg_config &c, const Scalars &s, int updates, double out[4])
{
    const bool on = c.field_tol > 0.0 && updates > 0;
    for (int a = 0; a < 4; ++a) out[a] = (on && s.change[4 + a] > 0.0) ? s.change[a] / s.change[4 + a] : 0.0;
}

// k2_newton applies to periodic boxes whose K comes from the integrability condition.
bool k2_newton_on(const mg_config *c)
{
    return c->k2_newton == 1 && c->bc == MG_BC_PERIODIC && c->k_mode == MG_K_INTEGRABILITY;
}

struct Layout {
    size_t X, SRC, R, D, PB, RT, BY, partial, scal, Z, ZR, Gpsi, GW, gj, own, child, total;
    int dense, mpsi, mw, has_child;
    std::vector<size_t> eA, eB, f, c;
};

Layout layout_for(const mg_config *c)
{
    Layout L{};
    int lv = c->levels > 0 ? c->levels : auto_levels(c->n);
    size_t N = (size_t)c->n[0] * c->n[1] * c->n[2];
    size_t tb = c->precision == MG_FP64 ? 8 : 4;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
    L.X = take(4 * N * 8);
    L.SRC = take(5 * N * 8);
    L.R = take(5 * N * 8);
    L.D = take(4 * N * 8);
    if (c->npunct > 0) L.PB = take(N * 8);
    if (c->bc == MG_BC_ROBIN) L.RT = take((size_t)(c->n[0] + 4) * (c->n[1] + 4) * (c->n[2] + 4) * 8);
    if (has_bowen_york(c)) L.BY = take(6 * N * 8);
    for (int l = 0; l < lv; ++l) {
        size_t Nl = ((size_t)(c->n[0] >> l)) * (c->n[1] >> l) * (c->n[2] >> l);
        L.eA.push_back(take(4 * Nl * tb));
        L.eB.push_back(take(4 * Nl * tb));
        L.f.push_back(take(4 * Nl * tb));
        L.c.push_back(take(2 * Nl * tb));
    }
    L.partial = take((size_t)kRedBlocks * 8 * 8);
    L.scal = take(sizeof(Scalars));
    if (k2_newton_on(c)) {
        L.Z = take(4 * N * tb);
        L.ZR = take(4 * N * tb);
    }
    {
        const int periodic = c->bc == MG_BC_PERIODIC;
        int nc[3];
        for (int a = 0; a < 3; ++a) nc[a] = c->n[a] >> (lv - 1);
        const int Nc = nc[0] * nc[1] * nc[2];
        L.dense = lv > 1 && dense_eligible(nc, periodic);
        L.mpsi = dense_m_psi(Nc, periodic);
        L.mw = dense_m_w(Nc, periodic);
        if (L.dense) {
            L.Gpsi = take((size_t)L.mpsi * L.mpsi * tb);
            L.GW = take((size_t)L.mw * L.mw * tb);
            L.gj = take(gj_scratch_elems(L.mw) * 8);
        }
    }
    L.own = off;
    mg_config cc;
    L.has_child = nested_child_config(c, &cc) ? 1 : 0;
    if (L.has_child) L.child = take(layout_for(&cc).total);
    L.total = off;
    return L;
}


// Driver entry point of the tensor-map encoder (resolved once; no link against libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 5-D map of a colour-split level buffer (4 fields x 2 colour halves): dims (pair, row, plane,
// field, half), box (kTileW pairs, tile rows, 1 plane, 4 fields, 1 half).
bool encode_level_map(CUtensorMap *m, void *base, const Geo &g, size_t N, size_t tb, int order)
{
    auto enc = tensor_map_encoder();
    if (!enc) return false;
    const cuuint64_t nxh = (cuuint64_t)(g.n[0] / 2);
    cuuint64_t dims[5] = {nxh, (cuuint64_t)g.n[1], (cuuint64_t)g.n[2], 4, 2};
    cuuint64_t strides[4] = {nxh * tb, nxh * g.n[1] * tb, N * tb, N / 2 * tb};
    cuuint32_t box[5] = {(cuuint32_t)kTileW, (cuuint32_t)(kTileY + order), 1, 4, 1};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(m, tb == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 5, base, dims,
                     strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Calls fn(T{}, ORDER tag, BC tag) for the context's inner precision, stencil order and boundary
// variant (periodic; Robin; Robin with symmetry planes), the engine instantiation to use.
template <class Fn>
mg_status with_engine(const mg_ctx *x, Fn &&fn)
{
    auto by_bc = [&](auto t, auto o) -> mg_status {
        if (x->cfg.bc == MG_BC_PERIODIC) return fn(t, o, std::integral_constant<int, BC_PERIODIC>());
        if (x->cfg.reflect == 0 && x->cfg.extrap == 0) return fn(t, o, std::integral_constant<int, BC_ROBIN>());
        return fn(t, o, std::integral_constant<int, BC_SYM>());
    };
    using O2 = std::integral_constant<int, 2>;
    using O4 = std::integral_constant<int, 4>;
    if (x->tbytes == 8) return x->cfg.order == 2 ? by_bc(double{}, O2{}) : by_bc(double{}, O4{});
    return x->cfg.order == 2 ? by_bc(float{}, O2{}) : by_bc(float{}, O4{});
}

#define ENGINE_CALL(name, ...)                                                                          \
    with_engine(x, [&](auto t, auto o, auto b) {                                                      \
        return name<decltype(t), decltype(o)::value, decltype(b)::value>(__VA_ARGS__);                \
    })

mg_status residual_any(mg_ctx *x, double *HM) { return ENGINE_CALL(engine_residual, x, HM); }

mg_status iteration_any(mg_ctx *x) { return ENGINE_CALL(engine_iteration, x); }

// k2_newton: the z solve (the inner cycles on zrhs, at the current linearisation), then its means.
mg_status zsolve_any(mg_ctx *x)
{
    x->zsolve = true;
    mg_status st = ENGINE_CALL(engine_iteration, x);
    x->zsolve = false;
    return st;
}

__global__ void k_fill_value(void *p, size_t n, int tb, double v)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        if (tb == 4) ((float *)p)[i] = (float)v;
        else ((double *)p)[i] = v;
    }
}

// Periodic gauge <u> = <W_i> = 0: the means (one grid reduction, finished in its last block) removed.
mg_status project_gauge(mg_ctx *x)
{
    if (x->cfg.bc != MG_BC_PERIODIC) return MG_OK;
    int g = grid_for(x->N, kRedBlocks);
    k_sum4<double><<<g, kThreads, 0, x->stream>>>(x->X, x->N, x->partial, x->scal->emean, &x->scal->ticket[2]);
    k_sub_mean4<double><<<grid_for(x->N), kThreads, 0, x->stream>>>(x->X, x->N, x->scal->emean);
    CK(cudaGetLastError());
    return MG_OK;
}

mg_status start_any(mg_ctx *x)
{
    CKS(project_gauge(x));
    return residual_any(x, nullptr);
}

// Capture fn's launches on the context stream into an executable graph; count its kernel nodes.
template <class Fn>
mg_status capture(mg_ctx *x, Fn &&fn, cudaGraphExec_t *exec, long long *kernels)
{
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(x->stream, cudaStreamCaptureModeThreadLocal));
    mg_status st = fn(x);
    cudaError_t e = cudaStreamEndCapture(x->stream, &graph);
    CKS(st);
    if (e != cudaSuccess) return fail(MG_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
    size_t n = 0;
    cudaGraphGetNodes(graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    cudaGraphGetNodes(graph, nodes.data(), &n);
    long long k = 0;
    for (auto &nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    *kernels = k;
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        *exec = nullptr;
        return fail(MG_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
    }
    return MG_OK;
}

// Gauge projection + residual of the current state (captured graph or direct launches), then wait
// for its scalars.
mg_status run_start(mg_ctx *x, long long *launches)
{
    if (x->cfg.use_graph) {
        if (!x->graph_start) CKS(capture(x, start_any, &x->graph_start, &x->launches_start));
        CK(cudaGraphLaunch(x->graph_start, x->stream));
        *launches += x->launches_start;
    } else {
        CKS(start_any(x));
    }
    CK(cudaStreamSynchronize(x->stream));
    return MG_OK;
}

double max_norm(const Scalars &s)
{
    double m = 0.0;
    for (int a = 0; a < 4; ++a) m = std::isfinite(s.norms[a]) ? std::max(m, s.norms[a]) : INFINITY;
    return m;
}

// The network's guess for the current sources into X (captured once per context).
mg_status warm_infer(mg_ctx *x, long long *launches)
{
    if (x->cfg.use_graph) {
        if (!x->warm_graph) {
            // one direct run first: it allocates the network's level buffers for this grid size,
            // which a capture must not do
            CKS(warm_enqueue(x->warm, x, x->stream));
            CK(cudaStreamSynchronize(x->stream));
            CKS(capture(x, [](mg_ctx *c) { return warm_enqueue(c->warm, c, c->stream); }, &x->warm_graph,
                        &x->launches_warm));
        }
        CK(cudaGraphLaunch(x->warm_graph, x->stream));
        *launches += x->launches_warm;
    } else {
        CKS(warm_enqueue(x->warm, x, x->stream));
    }
    if (warm_timed_out(x->warm, x->stream))
        return fail(MG_ERR_TIMEOUT, "a bounded wait of the warm start's tensor-core kernels gave up");
    return MG_OK;
}

// The learned start.  The multigrid judges it: the guess is the starting state whenever its
// residual is finite (state 1: X holds it, its residual evaluated), else X = 0 (state 2); a solve
// that then fails is repeated from the cold start by the caller.  A max-norm residual test against
// psi = 1 would be the wrong filter: the guess's small-scale error dominates its max |H| (the
// Laplacian weighs a mode by k^2) although the first smoothing sweeps remove it.
mg_status warm_start(mg_ctx *x, int *state, long long *launches)
{
    CKS(warm_infer(x, launches));
    CKS(run_start(x, launches));
    if (std::isfinite(max_norm(*x->host_scal))) {
        *state = 1;
        x->guess_set = true;
        return MG_OK;
    }
    *state = 2;
    CK(cudaMemsetAsync(x->X, 0, 4 * x->N * sizeof(double), x->stream));
    return MG_OK;
}

void warm_drop(mg_ctx *x)
{
    if (x->warm_graph) cudaGraphExecDestroy(x->warm_graph);
    x->warm_graph = nullptr;
    x->launches_warm = 0;
    if (x->warm && x->warm_owned) {
        cudaStreamSynchronize(x->stream);
        warm_free(x->warm);
    }
    x->warm = nullptr;
    x->warm_owned = false;
}

mg_status copy_in(double *dst, const double *src, size_t n, int on_device, cudaStream_t st)
{
    if (!src) {
        CK(cudaMemsetAsync(dst, 0, n * 8, st));
        return MG_OK;
    }
    CK(cudaMemcpyAsync(dst, src, n * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    return MG_OK;
}

mg_status copy_out(double *dst, const double *src, size_t n, int on_device, cudaStream_t st)
{
    if (!dst) return MG_OK;
    CK(cudaMemcpyAsync(dst, src, n * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    return MG_OK;
}

// Order the library's private stream after the caller's stream (entry) and the caller's
// stream after the library's work (exit), so every call behaves as if issued on the caller's stream.
mg_status enter(mg_ctx *x)
{
    CK(cudaEventRecord(x->ev_in, x->user_stream));
    CK(cudaStreamWaitEvent(x->stream, x->ev_in, 0));
    return MG_OK;
}

mg_status leave(mg_ctx *x, mg_status st)
{
    cudaError_t e1 = cudaEventRecord(x->ev_out, x->stream);
    cudaError_t e2 = cudaStreamWaitEvent(x->user_stream, x->ev_out, 0);
    if (st == MG_OK && (e1 != cudaSuccess || e2 != cudaSuccess))
        return fail(MG_ERR_CUDA, "stream ordering event failed");
    return st;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

mg_status mg_config_default(mg_config *c)
{
    if (!c) return fail(MG_ERR_INVALID_ARG, "null config");
    std::memset(c, 0, sizeof(*c));
    for (int a = 0; a < 3; ++a) {
        c->n[a] = 32;
        c->lo[a] = 0.0;
        c->hi[a] = 16.0;
    }
    c->order = 2;
    c->bc = MG_BC_PERIODIC;
    c->levels = 0;
    c->precision = MG_MIXED;
    c->k_mode = MG_K_INTEGRABILITY;
    c->K = 0.0;
    c->tol = 1e-10;
    c->max_outer = 60;
    c->nu_pre = 2;
    c->nu_post = 2;
    c->coarse_sweeps = 60;
    c->use_graph = 1;
    c->spin_limit = 1LL << 24;
    c->inner_cycles = 0;
    c->block_threads = 0;
    return MG_OK;
}

mg_status mg_workspace_size(const mg_config *cfg, size_t *bytes)
{
    CKS(validate(cfg));
    if (!bytes) return fail(MG_ERR_INVALID_ARG, "null bytes");
    *bytes = layout_for(cfg).total;
    return MG_OK;
}

mg_status mg_create(const mg_config *cfg, void *cuda_stream, void *workspace, size_t workspace_bytes, mg_ctx **out)
{
    if (!out) return fail(MG_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    CKS(validate(cfg));
    Layout lay = layout_for(cfg);
    if (workspace && ((uintptr_t)workspace % 256 != 0 || workspace_bytes < lay.total))
        return fail(MG_ERR_INVALID_ARG, "workspace misaligned or smaller than mg_workspace_size()");
    mg_ctx *x = new (std::nothrow) mg_ctx();
    if (!x) return fail(MG_ERR_OOM, "host allocation");
    x->cfg = *cfg;
    if (x->cfg.inner_cycles == 0) x->cfg.inner_cycles = cfg->precision == MG_FP64 ? 1 : 2;
    x->threads = cfg->block_threads > 0 ? cfg->block_threads : 256;
    x->omega = cfg->omega > 0.0 ? cfg->omega : 1.0;
    x->gamma = cfg->cycle == 2 ? 2 : 1;
    x->user_stream = (cudaStream_t)cuda_stream;
    x->nlev = cfg->levels > 0 ? cfg->levels : auto_levels(cfg->n);
    x->N = (size_t)cfg->n[0] * cfg->n[1] * cfg->n[2];
    x->tbytes = cfg->precision == MG_FP64 ? 8 : 4;
    mg_status st = MG_OK;
    do {
        if (workspace) {
            x->ws = workspace;
        } else {
            cudaError_t e = cudaMalloc(&x->ws, lay.total);
            if (e != cudaSuccess) { st = fail(MG_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e)); break; }
            x->own_ws = true;
        }
        x->ws_bytes = lay.total;
        char *b = (char *)x->ws;
        x->X = (double *)(b + lay.X);
        x->SRC = (double *)(b + lay.SRC);
        x->R = (double *)(b + lay.R);
        x->D = (double *)(b + lay.D);
        x->dense = lay.dense;
        x->mpsi = lay.mpsi;
        x->mw = lay.mw;
        if (lay.dense) {
            x->Gpsi = b + lay.Gpsi;
            x->GW = b + lay.GW;
            x->gj = b + lay.gj;
        }
        x->partial = (double *)(b + lay.partial);
        x->scal = (Scalars *)(b + lay.scal);
        if (k2_newton_on(cfg)) {
            x->zbuf = b + lay.Z;
            x->zrhs = b + lay.ZR;
        }
        for (int l = 0; l < x->nlev; ++l) {
            LevelBufs L;
            Geo &g = L.geo;
            std::memset(&g, 0, sizeof(g));
            for (int a = 0; a < 3; ++a) {
                g.n[a] = cfg->n[a] >> l;
                g.lo[a] = cfg->lo[a];
                g.h[a] = (cfg->hi[a] - cfg->lo[a]) / cfg->n[a] * (double)(1 << l);
                g.lof[a] = (float)g.lo[a];
                g.hf[a] = (float)g.h[a];
            }
            g.reflect = cfg->bc == MG_BC_ROBIN ? cfg->reflect : 0;
            g.extrap = cfg->bc == MG_BC_ROBIN ? cfg->extrap : 0;
            g.robin = cfg->bc == MG_BC_ROBIN ? 1 : 0;
            g.npunct = cfg->npunct;
            for (int p = 0; p < cfg->npunct; ++p) {
                g.pm[p] = cfg->punct_m[p];
                for (int a = 0; a < 3; ++a) g.px[p][a] = cfg->punct_x[p][a];
            }
            L.N = (size_t)g.n[0] * g.n[1] * g.n[2];
            L.eA = b + lay.eA[l];
            L.eB = b + lay.eB[l];
            L.f = b + lay.f[l];
            L.c = b + lay.c[l];
            L.split = l + 1 < x->nlev ? 1 : 0;
            L.curB = 0;
            L.tiled = 0;
            x->lev.push_back(L);
        }
        {
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&x->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
                st = fail(MG_ERR_CUDA, "device query");
                break;
            }
            for (auto &L : x->lev) {
                // FP32 levels only: the FP64 tile needs twice the shared memory, leaving one CTA per SM
                if (cfg->smoother != 0 || x->tbytes != 4 || !tile_eligible(L.geo, L.split)) continue;
                if (!encode_level_map(&L.tmA, L.eA, L.geo, L.N, x->tbytes, cfg->order) ||
                    !encode_level_map(&L.tmB, L.eB, L.geo, L.N, x->tbytes, cfg->order)) {
                    st = fail(MG_ERR_CUDA, "cuTensorMapEncodeTiled failed for a level buffer");
                    break;
                }
                const int waves = cfg->tile_waves ? cfg->tile_waves : 2;
                L.tg = tile_grid(L.geo, x->sms, waves);
                L.tgr = tile_grid(L.geo, x->sms, waves, true);
                L.tiled = 1;
            }
            if (st != MG_OK) break;
        }
        if (cudaStreamCreateWithFlags(&x->stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&x->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&x->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&x->ev_join, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&x->ev_in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&x->ev_out, cudaEventDisableTiming) != cudaSuccess) {
            st = fail(MG_ERR_CUDA, "stream/event creation");
            break;
        }
        cudaError_t e = cudaMallocHost(&x->host_scal, sizeof(Scalars));
        if (e != cudaSuccess) { st = fail(MG_ERR_OOM, "cudaMallocHost"); break; }
        if (cudaEventCreate(&x->ev0) != cudaSuccess || cudaEventCreate(&x->ev1) != cudaSuccess) {
            st = fail(MG_ERR_CUDA, "cudaEventCreate");
            break;
        }
        if ((st = ENGINE_CALL(engine_prepare, x)) != MG_OK) break;
        if ((st = enter(x)) != MG_OK) break;
        e = cudaMemsetAsync(x->ws, 0, lay.own, x->stream);
        if (e != cudaSuccess) { st = fail(MG_ERR_CUDA, std::string("memset: ") + cudaGetErrorString(e)); break; }
        if (cfg->npunct > 0) {
            double *pb = (double *)(b + lay.PB);
            k_fill_psibg<<<grid_for(x->N), kThreads, 0, x->stream>>>(x->lev[0].geo, pb);
            if ((e = cudaGetLastError()) != cudaSuccess) { st = fail(MG_ERR_CUDA, cudaGetErrorString(e)); break; }
            x->lev[0].geo.psibg = pb;
        }
        if (cfg->bc == MG_BC_ROBIN) {
            double *rt = (double *)(b + lay.RT);
            const size_t M = (size_t)(cfg->n[0] + 4) * (cfg->n[1] + 4) * (cfg->n[2] + 4);
            if (cfg->reflect || cfg->extrap)
                k_fill_robin_table<BC_SYM><<<grid_for(M), kThreads, 0, x->stream>>>(x->lev[0].geo, rt);
            else
                k_fill_robin_table<BC_ROBIN><<<grid_for(M), kThreads, 0, x->stream>>>(x->lev[0].geo, rt);
            if ((e = cudaGetLastError()) != cudaSuccess) { st = fail(MG_ERR_CUDA, cudaGetErrorString(e)); break; }
            x->lev[0].geo.rtab = rt;
        }
        if (has_bowen_york(cfg)) {
            ByPunct bp;
            std::memset(&bp, 0, sizeof(bp));
            bp.n = cfg->npunct;
            for (int p = 0; p < cfg->npunct; ++p)
                for (int a = 0; a < 3; ++a) {
                    bp.x[p][a] = cfg->punct_x[p][a];
                    bp.P[p][a] = cfg->punct_P[p][a];
                    bp.S[p][a] = cfg->punct_S[p][a];
                }
            double *by = (double *)(b + lay.BY);
            k_fill_by<<<grid_for(x->N), kThreads, 0, x->stream>>>(x->lev[0].geo, bp, by);
            if ((e = cudaGetLastError()) != cudaSuccess) { st = fail(MG_ERR_CUDA, cudaGetErrorString(e)); break; }
            x->lev[0].geo.by = by;
        }
        if (x->dense && x->nlev >= 2) {
            const LevelBufs &L1 = x->lev[x->nlev - 2], &Lc = x->lev[x->nlev - 1];
            // extrapolating faces take the unfused path (the fused cycle's ghost table holds one
            // scaled cell per ghost; an extrapolated ghost needs two)
            x->fused = cfg->smoother == 0 && cfg->extrap == 0 && L1.N <= (size_t)kFusedMaxCells &&
                       fused_smem_bytes((int)L1.N, (int)Lc.N, x->tbytes,
                                        fused_ratio_cells(L1.geo, cfg->bc == MG_BC_ROBIN)) <= kMaxCoarseSmem;
        }
        if (x->dense && (st = ENGINE_CALL(engine_dense_setup, x)) != MG_OK) break;
        if (x->zrhs) {   // the z solve's right-hand side: dF_psi/dK^2 = -psi^5/12 in the psi row's inner form
            cudaError_t e = cudaMemsetAsync(x->zrhs, 0, 4 * x->N * x->tbytes, x->stream);
            if (e == cudaSuccess) {
                k_fill_value<<<grid_for(x->N), kThreads, 0, x->stream>>>(x->zrhs, x->N, (int)x->tbytes, -1.0 / 12.0);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaStreamSynchronize(x->stream);
            if (e != cudaSuccess) { st = fail(MG_ERR_CUDA, cudaGetErrorString(e)); break; }
        }
        if ((st = leave(x, MG_OK)) != MG_OK) break;
        if (lay.has_child) {
            mg_config cc;
            nested_child_config(cfg, &cc);
            if ((st = mg_create(&cc, x->stream, b + lay.child, lay.total - lay.child, &x->child)) != MG_OK) break;
        }
    } while (0);
    if (st != MG_OK) {
        mg_destroy(x);
        return st;
    }
    *out = x;
    return MG_OK;
}

static mg_status mg_set_conformal_metric_impl(mg_ctx *x, const double *gt, int on_device)
{
    if (!gt) return MG_OK;
    std::vector<double> h(6 * x->N);
    if (on_device) {
        CK(cudaMemcpyAsync(h.data(), gt, 6 * x->N * 8, cudaMemcpyDeviceToHost, x->stream));
        CK(cudaStreamSynchronize(x->stream));
    } else {
        std::memcpy(h.data(), gt, 6 * x->N * 8);
    }
    const double want[6] = {1, 0, 0, 1, 0, 1};
    for (int c = 0; c < 6; ++c)
        for (size_t p = 0; p < x->N; ++p)
            if (h[c * x->N + p] != want[c])
                return fail(MG_ERR_UNSUPPORTED, "only the conformally flat metric gt_ij = delta_ij is supported");
    return MG_OK;
}

static mg_status mg_set_sources_impl(mg_ctx *x, const double *rho0, const double *rho2, const double *Sx, const double *Sy,
                         const double *Sz, int on_device)
{
    if (!x) return fail(MG_ERR_INVALID_ARG, "null ctx");
    if (!rho0 || !Sx || !Sy || !Sz) return fail(MG_ERR_INVALID_ARG, "rho0 and S must be given");
    for (mg_ctx *p = x; p; p = p->child) p->have_sources = false;
    CKS(copy_in(x->SRC, rho0, x->N, on_device, x->stream));
    CKS(copy_in(x->SRC + x->N, rho2, x->N, on_device, x->stream));
    CKS(copy_in(x->SRC + 2 * x->N, Sx, x->N, on_device, x->stream));
    CKS(copy_in(x->SRC + 3 * x->N, Sy, x->N, on_device, x->stream));
    CKS(copy_in(x->SRC + 4 * x->N, Sz, x->N, on_device, x->stream));
    // finiteness of the copied sources, checked on the device (host and device inputs alike)
    CK(cudaMemsetAsync(&x->scal->nonfinite, 0, sizeof(unsigned int), x->stream));
    k_flag_nonfinite<<<grid_for(5 * x->N, kRedBlocks), kThreads, 0, x->stream>>>(x->SRC, 5 * x->N, &x->scal->nonfinite);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&x->host_scal->nonfinite, &x->scal->nonfinite, sizeof(unsigned int), cudaMemcpyDeviceToHost,
                       x->stream));
    CK(cudaStreamSynchronize(x->stream));
    if (x->host_scal->nonfinite) return fail(MG_ERR_INVALID_ARG, "non-finite source value");
    // the nested start's sources, level by level: means over the 2^3 cells of each half-size cell
    for (mg_ctx *p = x; p->child; p = p->child) {
        mg_ctx *c = p->child;
        k_restrict_fields_f64<<<grid_for(5 * c->N), kThreads, 0, x->stream>>>(p->lev[0].geo, c->lev[0].geo, p->SRC,
                                                                             c->SRC, 5);
        CK(cudaGetLastError());
        c->have_sources = true;
    }
    x->have_sources = true;
    return MG_OK;
}

static mg_status mg_set_initial_guess_impl(mg_ctx *x, const double *u, const double *W, int on_device)
{
    if (!x) return fail(MG_ERR_INVALID_ARG, "null ctx");
    CKS(copy_in(x->X, u, x->N, on_device, x->stream));
    CKS(copy_in(x->X + x->N, W, 3 * x->N, on_device, x->stream));
    x->guess_set = u != nullptr || W != nullptr;
    return MG_OK;
}

static mg_status mg_solve_impl(mg_ctx *x, mg_solve_info *info)
{
    if (!x) return fail(MG_ERR_INVALID_ARG, "null ctx");
    if (!x->have_sources) return fail(MG_ERR_STATE, "mg_set_sources must come before mg_solve");
    NvtxRange solve_range(x->child ? "mg_solve (nested)" : "mg_solve");
    x->history.clear();
    long long launches = 0;
    int nested_iters = 0, warm_state = 0;
    CK(cudaEventRecord(x->ev0, x->stream));
    if (x->warm && !x->guess_set && warm_supported(x->warm, x)) {
        NvtxRange warm_range("learned warm start");
        CKS(warm_start(x, &warm_state, &launches));
    }
    if (x->child && !x->guess_set) {
        NvtxRange nested_range("nested start: half-size solve + tricubic interpolation");
        // nested start: solve the half-size problem from zero (nesting in turn), interpolate its solution
        mg_ctx *c = x->child;
        mg_solve_info ci{};
        CKS(mg_set_initial_guess(c, nullptr, nullptr, 1));
        mg_status cs = mg_solve(c, &ci);
        if (cs != MG_OK && cs != MG_ERR_NOT_CONVERGED && cs != MG_ERR_DIVERGED) return cs;
        if (cs == MG_ERR_DIVERGED) {
            CK(cudaMemsetAsync(x->X, 0, 4 * x->N * 8, x->stream));   // no usable start: the zero state
        } else {
            const dim3 nb = prolong_cubic_grid(c->lev[0].geo);
            if (x->cfg.bc == MG_BC_PERIODIC)
                k_prolong_cubic<BC_PERIODIC><<<nb, 256, 0, x->stream>>>(c->lev[0].geo, x->lev[0].geo, c->X, x->X);
            else if (x->cfg.reflect || x->cfg.extrap)
                k_prolong_cubic<BC_SYM><<<nb, 256, 0, x->stream>>>(c->lev[0].geo, x->lev[0].geo, c->X, x->X);
            else
                k_prolong_cubic<BC_ROBIN><<<nb, 256, 0, x->stream>>>(c->lev[0].geo, x->lev[0].geo, c->X, x->X);
            CK(cudaGetLastError());
            launches += ci.kernel_launches + 1;
        }
        nested_iters = ci.outer_iters;
    }
    x->guess_set = false;
    if (warm_state != 1) CKS(run_start(x, &launches));   // an accepted warm start has evaluated it
    if (x->zbuf) {   // k2_newton: z at the starting state's linearisation, kept for the whole solve
        if (x->cfg.use_graph) {
            if (!x->graph_z) CKS(capture(x, zsolve_any, &x->graph_z, &x->launches_z));
            CK(cudaGraphLaunch(x->graph_z, x->stream));
            launches += x->launches_z;
        } else {
            CKS(zsolve_any(x));
        }
    }
    mg_status result = MG_ERR_NOT_CONVERGED;
    int it = 0, grow = 0;
    double prev = INFINITY, prev_rel[4] = {0, 0, 0, 0};
    for (;;) {
        const Scalars &s = *x->host_scal;
        double mx = 0.0;
        bool finite = true;
        for (int a = 0; a < 4; ++a) {
            x->history.push_back(s.norms[a]);
            if (!std::isfinite(s.norms[a])) finite = false;
            mx = std::max(mx, s.norms[a]);
        }
        if (s.err) { result = fail(MG_ERR_TIMEOUT, "a bounded device wait gave up (spin_limit)"); break; }
        if (!finite || !std::isfinite(s.K2)) { result = fail(MG_ERR_DIVERGED, "constraint norm is not finite"); break; }
        const bool settled = fields_settled(x->cfg, s, it, prev_rel);
        if (mx <= x->cfg.tol && settled) { result = MG_OK; break; }
        // growth counts only above tol: below it (the per-field test still waiting) the norm sits
        // at its rounding floor and may wobble
        grow = (mx > prev && mx > x->cfg.tol) ? grow + 1 : 0;
        if (grow >= 3) { result = fail(MG_ERR_DIVERGED, "constraint norm grew for 3 outer iterations"); break; }
        prev = mx;
        if (it >= x->cfg.max_outer) { result = fail(MG_ERR_NOT_CONVERGED, "max_outer reached"); break; }
        NvtxRange iter_range("outer iteration");
        if (x->cfg.use_graph) {
            if (!x->graph_exec) CKS(capture(x, iteration_any, &x->graph_exec, &x->launches_iter));
            CK(cudaGraphLaunch(x->graph_exec, x->stream));
            launches += x->launches_iter;
        } else {
            CKS(iteration_any(x));
        }
        CK(cudaStreamSynchronize(x->stream));
        ++it;
    }
    CK(cudaEventRecord(x->ev1, x->stream));
    CK(cudaEventSynchronize(x->ev1));
    if (warm_state == 1 && (result == MG_ERR_NOT_CONVERGED || result == MG_ERR_DIVERGED)) {
        // the multigrid judges the learned start: it failed, so solve again from psi = 1
        float first = 0.f;
        cudaEventElapsedTime(&first, x->ev0, x->ev1);
        ctt::WarmNet *w = x->warm;
        x->warm = nullptr;
        CK(cudaMemsetAsync(x->X, 0, 4 * x->N * sizeof(double), x->stream));
        x->guess_set = false;   // the context's own cold start (psi = 1, or its nested start)
        mg_status again = mg_solve_impl(x, info);
        x->warm = w;
        if (info) {
            info->warm_start = 3;
            info->device_ms += first;
            if (info->kernel_launches) info->kernel_launches += launches;
        }
        return again;
    }
    if (info) {
        const Scalars &s = *x->host_scal;
        info->warm_start = warm_state;
        info->outer_iters = it;
        info->converged = result == MG_OK;
        info->K2 = s.K2;
        info->K = -std::sqrt(std::max(0.0, s.K2));
        for (int a = 0; a < 4; ++a) info->norms[a] = s.norms[a];
        for (int a = 0; a < 3; ++a) info->mom_mean[a] = s.msrc[a];
        info->history = x->history.data();
        info->history_len = (int)(x->history.size() / 4);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, x->ev0, x->ev1);
        info->device_ms = ms;
        info->kernel_launches = x->cfg.use_graph ? launches : 0;
        info->nested_iters = nested_iters;
        fill_rel_change(x->cfg, s, it, info->rel_change);
    }
    return result;
}

static mg_status mg_get_solution_impl(mg_ctx *x, double *u, double *W, double *K, int on_device)
{
    if (!x) return fail(MG_ERR_INVALID_ARG, "null ctx");
    CKS(copy_out(u, x->X, x->N, on_device, x->stream));
    CKS(copy_out(W, x->X + x->N, 3 * x->N, on_device, x->stream));
    CK(cudaStreamSynchronize(x->stream));
    if (K) *K = -std::sqrt(std::max(0.0, x->host_scal->K2));
    return MG_OK;
}

// ---- checkpoint / resume
static const char kCkptMagic[8] = {'C', 'T', 'T', 'M', 'G', 'C', 'K', '1'};

static bool host_little_endian()
{
    const uint32_t one = 1;
    unsigned char b;
    std::memcpy(&b, &one, 1);
    return b == 1;
}

static mg_status mg_checkpoint_save_impl(mg_ctx *x, const char *path)
{
    if (!x || !path) return fail(MG_ERR_INVALID_ARG, "null argument");
    if (!host_little_endian()) return fail(MG_ERR_UNSUPPORTED, "checkpoint files are little-endian");
    std::vector<double> h(4 * x->N);
    CK(cudaMemcpyAsync(h.data(), x->X, 4 * x->N * 8, cudaMemcpyDeviceToHost, x->stream));
    CK(cudaStreamSynchronize(x->stream));
    const int32_t hdr[6] = {x->cfg.n[0], x->cfg.n[1], x->cfg.n[2], x->cfg.order, x->cfg.bc, 0};
    const double K2 = x->host_scal->K2;
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(MG_ERR_INVALID_ARG, std::string("cannot open for writing: ") + path);
    bool ok = std::fwrite(kCkptMagic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(int32_t), 6, f) == 6 &&
              std::fwrite(&K2, sizeof(double), 1, f) == 1 && std::fwrite(h.data(), 8, h.size(), f) == h.size();
    ok = (std::fclose(f) == 0) && ok;
    return ok ? MG_OK : fail(MG_ERR_INVALID_ARG, std::string("write failed: ") + path);
}

static mg_status mg_checkpoint_load_impl(mg_ctx *x, const char *path)
{
    if (!x || !path) return fail(MG_ERR_INVALID_ARG, "null argument");
    if (!host_little_endian()) return fail(MG_ERR_UNSUPPORTED, "checkpoint files are little-endian");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(MG_ERR_INVALID_ARG, std::string("cannot open: ") + path);
    char magic[8];
    int32_t hdr[6];
    double K2 = 0.0;
    std::vector<double> h(4 * x->N);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kCkptMagic, 8) == 0 &&
              std::fread(hdr, sizeof(int32_t), 6, f) == 6;
    ok = ok && hdr[0] == x->cfg.n[0] && hdr[1] == x->cfg.n[1] && hdr[2] == x->cfg.n[2] && hdr[3] == x->cfg.order &&
         hdr[4] == x->cfg.bc;
    ok = ok && std::fread(&K2, sizeof(double), 1, f) == 1 && std::fread(h.data(), 8, h.size(), f) == h.size();
    char extra;
    ok = ok && std::fread(&extra, 1, 1, f) == 0;   // nothing after the state
    std::fclose(f);
    if (!ok) return fail(MG_ERR_INVALID_ARG, std::string("not a checkpoint of this grid: ") + path);
    CK(cudaMemcpyAsync(x->X, h.data(), 4 * x->N * 8, cudaMemcpyHostToDevice, x->stream));
    CK(cudaStreamSynchronize(x->stream));
    x->guess_set = true;
    return MG_OK;
}

static mg_status mg_residual_norms_impl(mg_ctx *x, double out[4])
{
    if (!x || !out) return fail(MG_ERR_INVALID_ARG, "null argument");
    if (!x->have_sources) return fail(MG_ERR_STATE, "mg_set_sources must come first");
    CKS(residual_any(x, nullptr));
    CK(cudaStreamSynchronize(x->stream));
    for (int a = 0; a < 4; ++a) out[a] = x->host_scal->norms[a];
    return MG_OK;
}

static mg_status mg_constraint_fields_impl(mg_ctx *x, double *H, double *M, int on_device)
{
    if (!x) return fail(MG_ERR_INVALID_ARG, "null ctx");
    if (!x->have_sources) return fail(MG_ERR_STATE, "mg_set_sources must come first");
    // H and M overwrite the pass-1 buffer R (4 of its 5 fields); it is rebuilt on the next residual.
    CKS(residual_any(x, x->R));
    CKS(copy_out(H, x->R, x->N, on_device, x->stream));
    CKS(copy_out(M, x->R + x->N, 3 * x->N, on_device, x->stream));
    CK(cudaStreamSynchronize(x->stream));
    return MG_OK;
}

static mg_status mg_time_kernel_impl(mg_ctx *x, int which, int reps, double *ms_per_launch, double *bytes_per_launch)
{
    if (!x || reps < 1 || which < 0 || which > 3) return fail(MG_ERR_INVALID_ARG, "bad argument");
    float ms = 0.f;
    CKS(ENGINE_CALL(engine_time_kernel, x, which, reps, &ms));
    double N = (double)x->N, s = (double)x->tbytes, b = 0.0;
    if (which == 0) b = 0.5 * 14.0 * s * N;               // half of a two-colour sweep: (2 F + 6) s per cell (algorithmic)
    else if (which == 1) b = (10.0 * s + 4.0 * s / 8.0) * N; // read e, f, a, b; write the coarse rhs
    else if (which == 2) b = (3.0 + 4.0 + 4.0 + 4.0 + 5.0 + 5.0) * 8.0 * N; // A: W -> q/div; B: u, W, q/div, 5 sources -> 5
    else b = (4.0 + 4.0 + 5.0 + 5.0) * 8.0 * N;                   // B: read u, W, q/div, 5 sources; write 5
    if (ms_per_launch) *ms_per_launch = ms / reps;
    if (bytes_per_launch) *bytes_per_launch = b;
    return MG_OK;
}

// FP64 FMA probe: 8 independent FMA chains per thread, folded into one value that is compared
// with a constant it never equals, so that no chain is optimised away.
__global__ void __launch_bounds__(256) k_fp64_probe(int iters, double seed, double *sink)
{
    double a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = seed * (double)(threadIdx.x + k + 1);
    const double b = 0.999999999, c = 1e-12;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 42.0) sink[0] = s;
}

static mg_status mg_fp64_fma_rate_impl(mg_ctx *x, int reps, double *tflops)
{
    if (reps < 1 || !tflops) return fail(MG_ERR_INVALID_ARG, "bad argument");
    const int blocks = x->sms * 8, iters = 2048;
    k_fp64_probe<<<blocks, 256, 0, x->stream>>>(iters, 1e-3, x->partial);
    CK(cudaGetLastError());
    CK(cudaEventRecord(x->ev0, x->stream));
    for (int r = 0; r < reps; ++r) k_fp64_probe<<<blocks, 256, 0, x->stream>>>(iters, 1e-3, x->partial);
    CK(cudaGetLastError());
    CK(cudaEventRecord(x->ev1, x->stream));
    CK(cudaEventSynchronize(x->ev1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, x->ev0, x->ev1));
    const double flops = 2.0 * 8.0 * iters * (double)blocks * 256.0 * reps;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return MG_OK;
}

// ---- public entry points: argument check, stream ordering, then the implementation
#define MG_WRAP(call)                                                                                  \
    do {                                                                                               \
        if (!x) return fail(MG_ERR_INVALID_ARG, "null ctx");                                           \
        mg_status s0 = enter(x);                                                                       \
        if (s0 != MG_OK) return s0;                                                                    \
        return leave(x, call);                                                                         \
    } while (0)

mg_status mg_set_sources(mg_ctx *x, const double *rho0, const double *rho2, const double *Sx, const double *Sy,
                         const double *Sz, int on_device)
{
    MG_WRAP(mg_set_sources_impl(x, rho0, rho2, Sx, Sy, Sz, on_device));
}
mg_status mg_set_initial_guess(mg_ctx *x, const double *u, const double *W, int on_device)
{
    MG_WRAP(mg_set_initial_guess_impl(x, u, W, on_device));
}
mg_status mg_solve(mg_ctx *x, mg_solve_info *info) { MG_WRAP(mg_solve_impl(x, info)); }
mg_status mg_set_conformal_metric(mg_ctx *x, const double *gt, int on_device)
{
    MG_WRAP(mg_set_conformal_metric_impl(x, gt, on_device));
}
mg_status mg_get_solution(mg_ctx *x, double *u, double *W, double *K, int on_device)
{
    MG_WRAP(mg_get_solution_impl(x, u, W, K, on_device));
}
mg_status mg_residual_norms(mg_ctx *x, double out[4]) { MG_WRAP(mg_residual_norms_impl(x, out)); }
static mg_status mg_warmstart_load_impl(mg_ctx *x, const char *path)
{
    warm_drop(x);
    if (!path) return MG_OK;
    ctt::WarmNet *w = nullptr;
    CKS(warm_load(path, x->stream, &w));
    if (!warm_supported(w, x)) {
        warm_free(w);
        return fail(MG_ERR_UNSUPPORTED, "the learned warm start serves periodic cubes whose side is the network's "
                                        "size times a power of two");
    }
    x->warm = w;
    x->warm_owned = true;
    return MG_OK;
}

static mg_status mg_warmstart_predict_impl(mg_ctx *x, double *u, double *W, int on_device)
{
    if (!x->warm) return fail(MG_ERR_STATE, "no warm start loaded (mg_warmstart_load)");
    if (!x->have_sources) return fail(MG_ERR_STATE, "mg_set_sources must come before mg_warmstart_predict");
    long long launches = 0;
    CKS(warm_infer(x, &launches));
    x->guess_set = true;
    CKS(copy_out(u, x->X, x->N, on_device, x->stream));
    CKS(copy_out(W, x->X + x->N, 3 * x->N, on_device, x->stream));
    CK(cudaStreamSynchronize(x->stream));
    return MG_OK;
}

mg_status mg_warmstart_load(mg_ctx *x, const char *path) { MG_WRAP(mg_warmstart_load_impl(x, path)); }
mg_status mg_warmstart_predict(mg_ctx *x, double *u, double *W, int on_device)
{
    MG_WRAP(mg_warmstart_predict_impl(x, u, W, on_device));
}
mg_status mg_checkpoint_save(mg_ctx *x, const char *path) { MG_WRAP(mg_checkpoint_save_impl(x, path)); }
mg_status mg_checkpoint_load(mg_ctx *x, const char *path) { MG_WRAP(mg_checkpoint_load_impl(x, path)); }
mg_status mg_constraint_fields(mg_ctx *x, double *H, double *M, int on_device)
{
    MG_WRAP(mg_constraint_fields_impl(x, H, M, on_device));
}
mg_status mg_time_kernel(mg_ctx *x, int which, int reps, double *ms_per_launch, double *bytes_per_launch)
{
    MG_WRAP(mg_time_kernel_impl(x, which, reps, ms_per_launch, bytes_per_launch));
}
mg_status mg_fp64_fma_rate(mg_ctx *x, int reps, double *tflops) { MG_WRAP(mg_fp64_fma_rate_impl(x, reps, tflops)); }

void mg_destroy(mg_ctx *x)
{
    if (!x) return;
    if (x->child) mg_destroy(x->child);
    warm_drop(x);
    if (x->graph_exec) cudaGraphExecDestroy(x->graph_exec);
    if (x->graph_start) cudaGraphExecDestroy(x->graph_start);
    if (x->graph_z) cudaGraphExecDestroy(x->graph_z);
    if (x->ev0) cudaEventDestroy(x->ev0);
    if (x->ev1) cudaEventDestroy(x->ev1);
    if (x->stream) {
        cudaStreamSynchronize(x->stream);
        cudaStreamDestroy(x->stream);
    }
    if (x->side) {
        cudaStreamSynchronize(x->side);
        cudaStreamDestroy(x->side);
    }
    if (x->ev_fork) cudaEventDestroy(x->ev_fork);
    if (x->ev_join) cudaEventDestroy(x->ev_join);
    if (x->ev_in) cudaEventDestroy(x->ev_in);
    if (x->ev_out) cudaEventDestroy(x->ev_out);
    if (x->host_scal) cudaFreeHost(x->host_scal);
    if (x->own_ws && x->ws) cudaFree(x->ws);
    delete x;
}

const char *mg_status_string(mg_status s)
{
    switch (s) {
    case MG_OK: return "MG_OK";
    case MG_ERR_INVALID_ARG: return "MG_ERR_INVALID_ARG";
    case MG_ERR_UNSUPPORTED: return "MG_ERR_UNSUPPORTED";
    case MG_ERR_CUDA: return "MG_ERR_CUDA";
    case MG_ERR_OOM: return "MG_ERR_OOM";
    case MG_ERR_STATE: return "MG_ERR_STATE";
    case MG_ERR_NOT_CONVERGED: return "MG_ERR_NOT_CONVERGED";
    case MG_ERR_DIVERGED: return "MG_ERR_DIVERGED";
    case MG_ERR_TIMEOUT: return "MG_ERR_TIMEOUT";
    }
    return "MG_ERR_UNKNOWN";
}

const char *mg_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"

// ====================================================================== batched solves
struct mg_batch {
    std::vector<mg_ctx *> ctx;
    cudaStream_t user_stream = nullptr;
    cudaStream_t stream = nullptr;   // master stream: graph launches, fork/join of the branches
    cudaEvent_t ev_fork = nullptr, ev_in = nullptr, ev_out = nullptr;
    std::vector<cudaEvent_t> ev_join, ev_round;
    cudaGraphExec_t graph_start = nullptr, graph_iter = nullptr;
    long long launches_start = 0, launches_iter = 0;
    ctt::WarmNet *warm = nullptr;   // learned warm start shared by the instances it serves
    // device-paced rounds: the whole solve as one graph (mg_batch.cuh)
    cudaGraphExec_t graph_all = nullptr;
    void *ctl_mem = nullptr;
    ctt::BatchCtlArgs ctl{};
    int ctl_maxr = -1;
    std::vector<long long> kernels_iter;
    long long kernels_start = 0;
};

namespace {

// Capture `fn(ctx)` of every instance as parallel branches of one graph on the master stream.
template <class Fn>
mg_status capture_batch(mg_batch *bt, Fn &&fn, cudaGraphExec_t *exec, long long *kernels)
{
    cudaGraph_t graph;
    CK(cudaStreamBeginCapture(bt->stream, cudaStreamCaptureModeThreadLocal));
    mg_status st = MG_OK;
    cudaError_t e = cudaEventRecord(bt->ev_fork, bt->stream);
    for (size_t b = 0; b < bt->ctx.size() && st == MG_OK && e == cudaSuccess; ++b) {
        mg_ctx *x = bt->ctx[b];
        e = cudaStreamWaitEvent(x->stream, bt->ev_fork, 0);
        if (e == cudaSuccess) st = fn(x);
        if (st == MG_OK && e == cudaSuccess) e = cudaEventRecord(bt->ev_join[b], x->stream);
        if (st == MG_OK && e == cudaSuccess) e = cudaStreamWaitEvent(bt->stream, bt->ev_join[b], 0);
    }
    cudaError_t e2 = cudaStreamEndCapture(bt->stream, &graph);
    CKS(st);
    if (e != cudaSuccess || e2 != cudaSuccess)
        return fail(MG_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    size_t n = 0;
    cudaGraphGetNodes(graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    cudaGraphGetNodes(graph, nodes.data(), &n);
    long long k = 0;
    for (auto &nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    *kernels = k;
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        *exec = nullptr;
        return fail(MG_ERR_CUDA, std::string("batch instantiate: ") + cudaGetErrorString(e));
    }
    return MG_OK;
}

mg_status batch_enter(mg_batch *bt)
{
    CK(cudaEventRecord(bt->ev_in, bt->user_stream));
    CK(cudaStreamWaitEvent(bt->stream, bt->ev_in, 0));
    for (mg_ctx *x : bt->ctx) CK(cudaStreamWaitEvent(x->stream, bt->ev_in, 0));
    return MG_OK;
}

mg_status batch_leave(mg_batch *bt, mg_status st)
{
    for (mg_ctx *x : bt->ctx) {
        if (cudaEventRecord(x->ev_out, x->stream) != cudaSuccess ||
            cudaStreamWaitEvent(bt->stream, x->ev_out, 0) != cudaSuccess)
            return st == MG_OK ? fail(MG_ERR_CUDA, "batch ordering event failed") : st;
    }
    if (cudaEventRecord(bt->ev_out, bt->stream) != cudaSuccess ||
        cudaStreamWaitEvent(bt->user_stream, bt->ev_out, 0) != cudaSuccess)
        return st == MG_OK ? fail(MG_ERR_CUDA, "batch ordering event failed") : st;
    return st;
}

}  // namespace

extern "C" {

void mg_batch_destroy(mg_batch *bt)
{
    if (!bt) return;
    if (bt->stream) cudaStreamSynchronize(bt->stream);
    if (bt->graph_start) cudaGraphExecDestroy(bt->graph_start);
    if (bt->graph_iter) cudaGraphExecDestroy(bt->graph_iter);
    if (bt->graph_all) cudaGraphExecDestroy(bt->graph_all);
    if (bt->ctl_mem) cudaFree(bt->ctl_mem);
    for (mg_ctx *x : bt->ctx) mg_destroy(x);
    warm_free(bt->warm);
    for (auto e : bt->ev_join) cudaEventDestroy(e);
    for (auto e : bt->ev_round) cudaEventDestroy(e);
    if (bt->ev_fork) cudaEventDestroy(bt->ev_fork);
    if (bt->ev_in) cudaEventDestroy(bt->ev_in);
    if (bt->ev_out) cudaEventDestroy(bt->ev_out);
    if (bt->stream) cudaStreamDestroy(bt->stream);
    delete bt;
}

mg_status mg_batch_create(int count, const mg_config *cfgs, void *cuda_stream, mg_batch **out)
{
    if (!out || !cfgs || count < 1 || count > 4096) return fail(MG_ERR_INVALID_ARG, "bad batch arguments");
    *out = nullptr;
    for (int b = 1; b < count; ++b)
        if (cfgs[b].order != cfgs[0].order || cfgs[b].bc != cfgs[0].bc || cfgs[b].precision != cfgs[0].precision ||
            cfgs[b].k_mode != cfgs[0].k_mode)
            return fail(MG_ERR_INVALID_ARG, "batch instances must share order, bc, precision and k_mode");
    mg_batch *bt = new (std::nothrow) mg_batch();
    if (!bt) return fail(MG_ERR_OOM, "host allocation");
    bt->user_stream = (cudaStream_t)cuda_stream;
    mg_status st = MG_OK;
    if (cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&bt->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&bt->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&bt->ev_out, cudaEventDisableTiming) != cudaSuccess)
        st = fail(MG_ERR_CUDA, "stream/event creation");
    for (int b = 0; b < count && st == MG_OK; ++b) {
        mg_ctx *x = nullptr;
        mg_config cb = cfgs[b];
        cb.nested = 0;   // the batch replays one graph per round: no per-instance nested start
        cb.k2_newton = 0;   // nor a per-instance z solve
        st = mg_create(&cb, cuda_stream, nullptr, 0, &x);
        if (st == MG_OK) bt->ctx.push_back(x);
        cudaEvent_t e;
        if (st == MG_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess) bt->ev_join.push_back(e);
        else if (st == MG_OK) st = fail(MG_ERR_CUDA, "event creation");
    }
    if (st != MG_OK) {
        mg_batch_destroy(bt);
        return st;
    }
    *out = bt;
    return MG_OK;
}

mg_status mg_batch_set_sources(mg_batch *bt, int b, const double *rho0, const double *rho2, const double *Sx,
                               const double *Sy, const double *Sz, int on_device)
{
    if (!bt || b < 0 || b >= (int)bt->ctx.size()) return fail(MG_ERR_INVALID_ARG, "bad instance");
    return mg_set_sources(bt->ctx[b], rho0, rho2, Sx, Sy, Sz, on_device);
}

mg_status mg_batch_set_initial_guess(mg_batch *bt, int b, const double *u, const double *W, int on_device)
{
    if (!bt || b < 0 || b >= (int)bt->ctx.size()) return fail(MG_ERR_INVALID_ARG, "bad instance");
    return mg_set_initial_guess(bt->ctx[b], u, W, on_device);
}

mg_status mg_batch_get_solution(mg_batch *bt, int b, double *u, double *W, double *K, int on_device)
{
    if (!bt || b < 0 || b >= (int)bt->ctx.size()) return fail(MG_ERR_INVALID_ARG, "bad instance");
    return mg_get_solution(bt->ctx[b], u, W, K, on_device);
}

mg_status mg_batch_warmstart_load(mg_batch *bt, const char *path)
{
    if (!bt) return fail(MG_ERR_INVALID_ARG, "null batch");
    CKS(batch_enter(bt));
    mg_status st = MG_OK;
    for (mg_ctx *x : bt->ctx) warm_drop(x);
    cudaStreamSynchronize(bt->stream);
    warm_free(bt->warm);
    bt->warm = nullptr;
    if (path) {
        st = warm_load(path, bt->stream, &bt->warm);
        if (st == MG_OK)
            for (mg_ctx *x : bt->ctx)
                if (warm_supported(bt->warm, x)) x->warm = bt->warm;   // shared, not owned
    }
    return batch_leave(bt, st);
}

}  // extern "C"

namespace {

// What the rounds of a batched solve leave behind, per instance.
struct BatchOutcome {
    std::vector<int> conv;        // round at which the instance met its tolerance, -1 if it did not
    std::vector<int> rounds;      // outer iterations it made
    std::vector<char> bad;        // a norm became non-finite
    std::vector<float> conv_ms;   // time from the start of the solve to its convergence
    std::vector<std::vector<double>> hist;   // 4 norms per recorded round
    std::vector<long long> launches;
    float total_ms = 0.f;
    bool timeout = false;
};

// Host-paced rounds (use_graph == 2): one graph per round for all instances, read back and
// checked on the host after every round; converged instances keep iterating in lock step.
mg_status batch_rounds_host(mg_batch *bt, int max_outer, BatchOutcome &o)
{
    const int nb = (int)bt->ctx.size();
    while ((int)bt->ev_round.size() < max_outer + 1) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return fail(MG_ERR_CUDA, "event creation");
        bt->ev_round.push_back(e);
    }
    if (!bt->graph_start) CKS(capture_batch(bt, start_any, &bt->graph_start, &bt->launches_start));
    if (!bt->graph_iter) CKS(capture_batch(bt, iteration_any, &bt->graph_iter, &bt->launches_iter));
    cudaEvent_t t0 = bt->ev_round[0];
    if (cudaEventRecord(t0, bt->stream) != cudaSuccess || cudaGraphLaunch(bt->graph_start, bt->stream) != cudaSuccess ||
        cudaStreamSynchronize(bt->stream) != cudaSuccess)
        return fail(MG_ERR_CUDA, "batch start");
    int round = 0, done = 0;
    std::vector<double> prev_rel(4 * (size_t)nb, 0.0);
    for (;;) {
        float ms = 0.f;
        if (round > 0) cudaEventElapsedTime(&ms, t0, bt->ev_round[round]);
        for (int b = 0; b < nb; ++b) {
            mg_ctx *x = bt->ctx[b];
            const Scalars &s = *x->host_scal;
            double mx = 0.0;
            bool finite = std::isfinite(s.K2);
            const bool live = o.conv[b] < 0 && !o.bad[b];   // still iterating: its row is recorded
            for (int a = 0; a < 4; ++a) {
                if (live) o.hist[b].push_back(s.norms[a]);
                finite = finite && std::isfinite(s.norms[a]);
                mx = std::max(mx, s.norms[a]);
            }
            if (o.conv[b] < 0 && !o.bad[b] && !finite) {
                o.bad[b] = 1;
                o.rounds[b] = round;
                ++done;
            }
            const bool settled = o.conv[b] < 0 && !o.bad[b] && fields_settled(x->cfg, s, round, &prev_rel[4 * b]);
            if (o.conv[b] < 0 && !o.bad[b] && mx <= x->cfg.tol && settled) {
                o.conv[b] = round;
                o.conv_ms[b] = ms;
                o.rounds[b] = round;
                ++done;
            }
        }
        for (int b = 0; b < nb; ++b) o.timeout = o.timeout || bt->ctx[b]->host_scal->err != 0;
        if (o.timeout || done == nb || round >= max_outer) break;
        if (cudaGraphLaunch(bt->graph_iter, bt->stream) != cudaSuccess ||
            cudaEventRecord(bt->ev_round[round + 1], bt->stream) != cudaSuccess ||
            cudaStreamSynchronize(bt->stream) != cudaSuccess)
            return fail(MG_ERR_CUDA, "batch iteration");
        ++round;
    }
    cudaEventElapsedTime(&o.total_ms, t0, bt->ev_round[round]);
    for (int b = 0; b < nb; ++b) {
        if (o.conv[b] < 0 && !o.bad[b]) o.rounds[b] = round;
        o.launches[b] = (bt->launches_start + (long long)round * bt->launches_iter) / nb;
    }
    return MG_OK;
}

long long count_kernels(cudaGraph_t g)
{
    size_t n = 0;
    cudaGraphGetNodes(g, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    cudaGraphGetNodes(g, nodes.data(), &n);
    long long k = 0;
    for (auto &nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
    }
    return k;
}

// The device-paced graph of the batch (built once per batch and round limit; see mg_batch.cuh).
mg_status build_device_graph(mg_batch *bt, int maxr)
{
    const int nb = (int)bt->ctx.size();
    if (bt->graph_all) {
        cudaGraphExecDestroy(bt->graph_all);
        bt->graph_all = nullptr;
    }
    if (bt->ctl_mem) {
        cudaFree(bt->ctl_mem);
        bt->ctl_mem = nullptr;
    }
    // control block: BatchCtl, scal pointers, tol, ftol, maxo, conv, bad, tconv, handles, history,
    // field_est, the last relative updates
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align256(off + bytes); return o; };
    const size_t oc = take(sizeof(BatchCtl)), os = take(nb * sizeof(Scalars *)), ot = take(nb * 8),
                 of = take(nb * 8), om = take(nb * 4), ov = take(nb * 4), ob = take(nb * 4), oT = take(nb * 8),
                 oh = take(nb * sizeof(cudaGraphConditionalHandle)), oH = take((size_t)(maxr + 1) * nb * 4 * 8),
                 oe = take(nb * 4), op = take(nb * 4 * 8);
    CK(cudaMalloc(&bt->ctl_mem, off));
    char *m = (char *)bt->ctl_mem;
    BatchCtlArgs &a = bt->ctl;
    a.c = (BatchCtl *)(m + oc);
    a.scal = (Scalars *const *)(m + os);
    a.tol = (const double *)(m + ot);
    a.ftol = (const double *)(m + of);
    a.maxo = (const int *)(m + om);
    a.conv = (int *)(m + ov);
    a.bad = (int *)(m + ob);
    a.tconv = (unsigned long long *)(m + oT);
    a.h = (const cudaGraphConditionalHandle *)(m + oh);
    a.hist = (double *)(m + oH);
    a.fest = (const int *)(m + oe);
    a.prev = (double *)(m + op);
    a.nb = nb;
    a.maxr = maxr;
    bt->ctl_maxr = maxr;
    std::vector<Scalars *> sp(nb);
    std::vector<double> tl(nb), ft(nb);
    std::vector<int> mo(nb), fe(nb);
    for (int b = 0; b < nb; ++b) {
        sp[b] = bt->ctx[b]->scal;
        tl[b] = bt->ctx[b]->cfg.tol;
        ft[b] = bt->ctx[b]->cfg.field_tol;
        mo[b] = bt->ctx[b]->cfg.max_outer;
        fe[b] = bt->ctx[b]->cfg.field_est;
    }
    cudaGraph_t G = nullptr;
    CK(cudaGraphCreate(&G, 0));
    std::vector<cudaGraphConditionalHandle> h(nb);
    cudaError_t e = cudaGraphConditionalHandleCreate(&a.hw, G, 0, 0);
    for (int b = 0; b < nb && e == cudaSuccess; ++b) e = cudaGraphConditionalHandleCreate(&h[b], G, 0, 0);
    if (e == cudaSuccess) e = cudaMemcpy(m + os, sp.data(), nb * sizeof(Scalars *), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m + ot, tl.data(), nb * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m + of, ft.data(), nb * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m + oe, fe.data(), nb * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m + om, mo.data(), nb * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m + oh, h.data(), nb * sizeof(cudaGraphConditionalHandle), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGraphDestroy(G);
        return fail(MG_ERR_CUDA, std::string("batch control set-up: ") + cudaGetErrorString(e));
    }
    mg_status st = MG_OK;
    cudaGraph_t cap = nullptr;
    for (mg_ctx *x : bt->ctx) x->device_paced = true;
    // the starts of all instances and the first control step, then the WHILE node after them
    e = cudaStreamBeginCaptureToGraph(bt->stream, G, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        k_batch_begin<<<1, 256, 0, bt->stream>>>(a);
        e = cudaEventRecord(bt->ev_fork, bt->stream);
        for (int b = 0; b < nb && st == MG_OK && e == cudaSuccess; ++b) {
            mg_ctx *x = bt->ctx[b];
            e = cudaStreamWaitEvent(x->stream, bt->ev_fork, 0);
            if (e == cudaSuccess) st = start_any(x);
            if (st == MG_OK && e == cudaSuccess) e = cudaEventRecord(bt->ev_join[b], x->stream);
            if (st == MG_OK && e == cudaSuccess) e = cudaStreamWaitEvent(bt->stream, bt->ev_join[b], 0);
        }
        if (st == MG_OK && e == cudaSuccess) {
            k_batch_control<<<1, 256, 0, bt->stream>>>(a);
            e = cudaGetLastError();
        }
        cudaGraphNode_t wnode = nullptr;
        cudaGraph_t body = nullptr;
        if (st == MG_OK && e == cudaSuccess) {
            cudaStreamCaptureStatus cs;
            const cudaGraphNode_t *deps = nullptr;
            size_t ndeps = 0;
            e = cudaStreamGetCaptureInfo(bt->stream, &cs, nullptr, nullptr, &deps, nullptr, &ndeps);
            cudaGraphNodeParams wp = {};
            wp.type = cudaGraphNodeTypeConditional;
            wp.conditional.handle = a.hw;
            wp.conditional.type = cudaGraphCondTypeWhile;
            wp.conditional.size = 1;
            if (e == cudaSuccess) e = cudaGraphAddNode(&wnode, G, deps, nullptr, ndeps, &wp);
            if (e == cudaSuccess) {
                body = wp.conditional.phGraph_out[0];
                e = cudaStreamUpdateCaptureDependencies(bt->stream, &wnode, nullptr, 1, cudaStreamSetCaptureDependencies);
            }
        }
        cudaError_t e2 = cudaStreamEndCapture(bt->stream, &cap);
        if (e == cudaSuccess) e = e2;
        // the loop body: one IF node per instance (its outer iteration), then the control step
        std::vector<cudaGraphNode_t> ifs(nb);
        bt->kernels_iter.assign(nb, 0);
        for (int b = 0; b < nb && st == MG_OK && e == cudaSuccess; ++b) {
            mg_ctx *x = bt->ctx[b];
            cudaGraphNodeParams ip = {};
            ip.type = cudaGraphNodeTypeConditional;
            ip.conditional.handle = h[b];
            ip.conditional.type = cudaGraphCondTypeIf;
            ip.conditional.size = 1;
            e = cudaGraphAddNode(&ifs[b], body, nullptr, nullptr, 0, &ip);
            if (e != cudaSuccess) break;
            cudaGraph_t ib = ip.conditional.phGraph_out[0];
            e = cudaStreamBeginCaptureToGraph(x->stream, ib, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) break;
            st = iteration_any(x);
            cudaGraph_t tmp = nullptr;
            e2 = cudaStreamEndCapture(x->stream, &tmp);
            if (e == cudaSuccess) e = e2;
            bt->kernels_iter[b] = count_kernels(ib);
        }
        if (st == MG_OK && e == cudaSuccess) {
            e = cudaStreamBeginCaptureToGraph(bt->stream, body, ifs.data(), nullptr, nb, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                k_batch_control<<<1, 256, 0, bt->stream>>>(a);
                cudaGraph_t tmp = nullptr;
                e2 = cudaStreamEndCapture(bt->stream, &tmp);
                e = cudaGetLastError() != cudaSuccess ? cudaErrorLaunchFailure : e2;
            }
        }
        if (st == MG_OK && e == cudaSuccess) bt->kernels_start = count_kernels(G) - 1;   // less the first control step
    }
    for (mg_ctx *x : bt->ctx) x->device_paced = false;
    if (st == MG_OK && e == cudaSuccess) e = cudaGraphInstantiate(&bt->graph_all, G, 0);
    cudaGraphDestroy(G);
    if (st != MG_OK) return st;
    if (e != cudaSuccess) {
        bt->graph_all = nullptr;
        return fail(MG_ERR_CUDA, std::string("device-paced batch graph: ") + cudaGetErrorString(e));
    }
    return MG_OK;
}

// Device-paced rounds (default): the whole solve is one graph launch and one synchronisation.
mg_status batch_rounds_device(mg_batch *bt, int max_outer, BatchOutcome &o)
{
    const int nb = (int)bt->ctx.size();
    if (!bt->graph_all || bt->ctl_maxr != max_outer) CKS(build_device_graph(bt, max_outer));
    if (bt->ev_round.empty()) {
        cudaEvent_t e0, e1;
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
            return fail(MG_ERR_CUDA, "event creation");
        bt->ev_round.push_back(e0);
        bt->ev_round.push_back(e1);
    }
    CK(cudaEventRecord(bt->ev_round[0], bt->stream));
    CK(cudaGraphLaunch(bt->graph_all, bt->stream));
    CK(cudaEventRecord(bt->ev_round[1], bt->stream));
    CK(cudaStreamSynchronize(bt->stream));
    CK(cudaEventElapsedTime(&o.total_ms, bt->ev_round[0], bt->ev_round[1]));
    BatchCtl c;
    std::vector<int> conv(nb), bad(nb);
    std::vector<unsigned long long> tconv(nb);
    CK(cudaMemcpy(&c, bt->ctl.c, sizeof(c), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(conv.data(), bt->ctl.conv, nb * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(bad.data(), bt->ctl.bad, nb * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(tconv.data(), bt->ctl.tconv, nb * 8, cudaMemcpyDeviceToHost));
    const int recorded = std::min(c.round, max_outer + 1);   // rounds 0 .. recorded - 1
    std::vector<double> hist((size_t)recorded * nb * 4);
    CK(cudaMemcpy(hist.data(), bt->ctl.hist, hist.size() * 8, cudaMemcpyDeviceToHost));
    o.timeout = c.timeout != 0;
    for (int b = 0; b < nb; ++b) {
        mg_ctx *x = bt->ctx[b];
        CK(cudaMemcpy(x->host_scal, x->scal, sizeof(Scalars), cudaMemcpyDeviceToHost));
        o.conv[b] = conv[b];
        o.bad[b] = (char)bad[b];
        // the last round in which the instance was still iterating (or the one it stopped at)
        int last = recorded - 1;
        if (conv[b] >= 0) last = conv[b];
        else last = std::min(last, x->cfg.max_outer);
        if (bad[b]) {   // the first round recorded with a non-finite norm
            for (int r = 0; r < recorded; ++r) {
                bool fin = true;
                for (int k = 0; k < 4; ++k) fin = fin && std::isfinite(hist[((size_t)r * nb + b) * 4 + k]);
                if (!fin) { last = r; break; }
            }
        }
        o.rounds[b] = last;
        for (int r = 0; r <= last && r < recorded; ++r)
            for (int k = 0; k < 4; ++k) o.hist[b].push_back(hist[((size_t)r * nb + b) * 4 + k]);
        o.conv_ms[b] = conv[b] >= 0 ? (float)((double)(tconv[b] - c.t0) * 1e-6) : o.total_ms;
        o.launches[b] = (bt->kernels_start / nb) + (long long)last * (bt->kernels_iter[b] + 1);
    }
    return MG_OK;
}

}  // namespace

extern "C" {

mg_status mg_batch_solve(mg_batch *bt, mg_solve_info *infos, double *total_ms)
{
    if (!bt) return fail(MG_ERR_INVALID_ARG, "null batch");
    NvtxRange range("mg_batch_solve");
    const int nb = (int)bt->ctx.size();
    for (mg_ctx *x : bt->ctx)
        if (!x->have_sources) return fail(MG_ERR_STATE, "every instance needs mg_batch_set_sources first");
    CKS(batch_enter(bt));
    mg_status result = MG_OK;
    std::vector<int> warm_state(nb, 0);
    for (int b = 0; b < nb && result == MG_OK; ++b) {   // learned starts, each judged by its residual
        mg_ctx *x = bt->ctx[b];
        long long dummy = 0;
        if (x->warm && !x->guess_set) {
            NvtxRange warm_range("learned warm start");
            result = warm_start(x, &warm_state[b], &dummy);
        }
    }
    BatchOutcome o;
    o.conv.assign(nb, -1);
    o.rounds.assign(nb, 0);
    o.bad.assign(nb, 0);
    o.conv_ms.assign(nb, 0.f);
    o.hist.assign(nb, {});
    o.launches.assign(nb, 0);
    int max_outer = 0;
    for (mg_ctx *x : bt->ctx) max_outer = std::max(max_outer, x->cfg.max_outer);
    if (result == MG_OK)
        result = bt->ctx[0]->cfg.use_graph == 2 ? batch_rounds_host(bt, max_outer, o) : batch_rounds_device(bt, max_outer, o);
    if (result == MG_OK) {
        int nconv = 0, nbad = 0;
        for (int b = 0; b < nb; ++b) {
            nconv += o.conv[b] >= 0;
            nbad += o.bad[b] != 0;
        }
        if (o.timeout) result = fail(MG_ERR_TIMEOUT, "a bounded device wait gave up (spin_limit)");
        else if (nbad) result = fail(MG_ERR_DIVERGED, "a batch instance's norm is not finite");
        else if (nconv < nb) result = fail(MG_ERR_NOT_CONVERGED, "max_outer reached in the batch");
        if (total_ms) *total_ms = o.total_ms;
        for (int b = 0; b < nb; ++b) {
            mg_ctx *x = bt->ctx[b];
            x->history = o.hist[b];
            x->guess_set = false;
            if (!infos) continue;
            const Scalars &s = *x->host_scal;
            mg_solve_info &in = infos[b];
            in.outer_iters = o.rounds[b];
            in.converged = o.conv[b] >= 0;
            in.K2 = s.K2;
            in.K = -std::sqrt(std::max(0.0, s.K2));
            for (int a = 0; a < 4; ++a) in.norms[a] = s.norms[a];
            for (int a = 0; a < 3; ++a) in.mom_mean[a] = s.msrc[a];
            in.history = x->history.data();
            in.history_len = (int)(x->history.size() / 4);
            in.device_ms = o.conv[b] >= 0 ? o.conv_ms[b] : o.total_ms;
            in.kernel_launches = o.launches[b];
            in.nested_iters = 0;
            in.warm_start = warm_state[b];
            fill_rel_change(x->cfg, s, o.rounds[b], in.rel_change);
        }
        // the multigrid judges the learned starts: an instance that failed from its warm start is
        // solved again, alone, from its cold start
        for (int b = 0; b < nb && (result == MG_ERR_NOT_CONVERGED || result == MG_ERR_DIVERGED); ++b) {
            if (warm_state[b] != 1 || o.conv[b] >= 0) continue;
            mg_ctx *x = bt->ctx[b];
            mg_solve_info again{};
            ctt::WarmNet *w = x->warm;
            x->warm = nullptr;
            mg_status sb = mg_set_initial_guess(x, nullptr, nullptr, 1);
            if (sb == MG_OK) sb = mg_solve_impl(x, &again);
            x->warm = w;
            if (sb != MG_OK && sb != MG_ERR_NOT_CONVERGED && sb != MG_ERR_DIVERGED) {
                result = sb;
                break;
            }
            if (infos) {
                again.warm_start = 3;
                again.device_ms += o.total_ms;
                infos[b] = again;
            }
            if (total_ms) *total_ms += again.device_ms - o.total_ms;
            o.conv[b] = sb == MG_OK ? again.outer_iters : -1;
            o.bad[b] = sb == MG_ERR_DIVERGED;
        }
        if (result == MG_ERR_NOT_CONVERGED || result == MG_ERR_DIVERGED) {
            bool all = true;
            for (int b = 0; b < nb; ++b) all = all && o.conv[b] >= 0;
            if (all) result = MG_OK;
        }
    }
    return batch_leave(bt, result);
}

}  // extern "C"

// ====================================================================== autotuner
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>

namespace {

struct TuneResult {
    int inner, nu, threads;
    double omega;
    int waves;   // tile_waves
    double ms;
};

std::mutex g_tune_mu;
std::map<std::string, TuneResult> g_tune_cache;

std::string tune_key(const mg_config *c)
{
    std::ostringstream k;
    k << c->n[0] << ' ' << c->n[1] << ' ' << c->n[2] << ' ' << c->order << ' ' << c->bc << ' ' << c->precision << ' '
      << c->k_mode << ' ' << c->nested;
    return k.str();
}

void tune_load(const char *path)
{
    if (!path) return;
    std::ifstream f(path);
    std::string line;
    while (std::getline(f, line)) {
        std::istringstream in(line);
        int n0, n1, n2, order, bc, prec, km, nested;
        TuneResult r;
        std::string extra;
        if (in >> n0 >> n1 >> n2 >> order >> bc >> prec >> km >> nested >> r.inner >> r.nu >> r.threads >> r.omega >>
                r.waves >> r.ms &&
            !(in >> extra)) {
            std::ostringstream k;
            k << n0 << ' ' << n1 << ' ' << n2 << ' ' << order << ' ' << bc << ' ' << prec << ' ' << km << ' ' << nested;
            g_tune_cache.emplace(k.str(), r);
        }
    }
}

void tune_save(const char *path)
{
    if (!path) return;
    std::ofstream f(path, std::ios::trunc);
    for (auto &kv : g_tune_cache)
        f << kv.first << ' ' << kv.second.inner << ' ' << kv.second.nu << ' ' << kv.second.threads << ' '
          << kv.second.omega << ' ' << kv.second.waves << ' ' << kv.second.ms << '\n';
}

}  // namespace

extern "C" mg_status mg_autotune(const mg_config *base, const double *rho0, const double *rho2, const double *Sx,
                                 const double *Sy, const double *Sz, int on_device, void *cuda_stream,
                                 const char *cache_path, mg_config *best, double *best_ms)
{
    CKS(validate(base));
    if (!best) return fail(MG_ERR_INVALID_ARG, "null best");
    NvtxRange range("mg_autotune");
    std::lock_guard<std::mutex> lock(g_tune_mu);
    tune_load(cache_path);
    const std::string key = tune_key(base);
    auto hit = g_tune_cache.find(key);
    TuneResult win{0, 0, 0, 1.0, 0, INFINITY};
    if (hit != g_tune_cache.end()) {
        win = hit->second;
    } else {
        const int inners_mixed[] = {1, 2, 3}, inners_fp64[] = {1, 2};
        const int nus[] = {1, 2, 3};
        const double omegas[] = {1.0, 1.15, 1.3};
        const int *inners = base->precision == MG_FP64 ? inners_fp64 : inners_mixed;
        const int ninner = base->precision == MG_FP64 ? 2 : 3;
        const int th = base->block_threads;
        // one timed solve (after an untimed one that captures the graphs) of a candidate setting
        auto trial = [&](int inner, int nu, double om, int waves, double *ms) -> mg_status {
            mg_config c = *base;
            c.inner_cycles = inner;
            c.nu_pre = c.nu_post = nu;
            c.omega = om;
            c.tile_waves = waves;
            c.use_graph = 1;
            mg_ctx *x = nullptr;
            CKS(mg_create(&c, cuda_stream, nullptr, 0, &x));
            mg_status st = mg_set_sources(x, rho0, rho2, Sx, Sy, Sz, on_device);
            mg_solve_info info;
            if (st == MG_OK) st = mg_solve(x, &info);
            if (st == MG_OK) st = mg_set_initial_guess(x, nullptr, nullptr, 1);
            if (st == MG_OK) st = mg_solve(x, &info);
            mg_destroy(x);
            *ms = st == MG_OK ? info.device_ms : INFINITY;
            return st == MG_ERR_NOT_CONVERGED || st == MG_ERR_DIVERGED ? MG_OK : st;
        };
        // solver settings first, at the base launch shape
        for (int ii = 0; ii < ninner; ++ii)
            for (int nu : nus)
                for (double om : omegas) {
                    double ms;
                    CKS(trial(inners[ii], nu, om, base->tile_waves, &ms));
                    if (ms < win.ms) win = TuneResult{inners[ii], nu, th, om, base->tile_waves, ms};
                }
        if (!std::isfinite(win.ms)) return fail(MG_ERR_NOT_CONVERGED, "no autotuner candidate met the tolerance");
        // then the z chunking of the tiled kernels (CTAs per SM the grid aims at), for the winner
        if (base->precision == MG_MIXED && base->smoother == 0)
            for (int waves : {1, 2, 3, 4}) {
                if (waves == (win.waves ? win.waves : 2)) continue;
                double ms;
                CKS(trial(win.inner, win.nu, win.omega, waves, &ms));
                if (ms < win.ms) {
                    win.waves = waves;
                    win.ms = ms;
                }
            }
        g_tune_cache[key] = win;
        tune_save(cache_path);
    }
    *best = *base;
    best->inner_cycles = win.inner;
    best->nu_pre = best->nu_post = win.nu;
    best->block_threads = win.threads;
    best->omega = win.omega;
    best->tile_waves = win.waves;
    if (best_ms) *best_ms = win.ms;
    return MG_OK;
}
