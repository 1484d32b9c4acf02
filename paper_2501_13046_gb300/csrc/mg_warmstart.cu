// mg_warmstart.cu -- the learned warm start inside the library: a trained 3-D U-Net (BF16
// tcgen05 convolutions with FP32 accumulation, the kernels of ctt_unet.h) maps a context's
// sources (rho, S_i, and the pre-solve K) to an initial guess (u, W_i) before the multigrid
// solve.  Not in the paper: the learned start is an addition to its multigrid solver.  Plain
// multigrid from psi = 1 remains the fallback, and the multigrid solve decides every result.
//
// Network (4 levels, 16/32/64/64 channels): two 3x3x3 circular convolutions + ReLU per level,
// 2x average pooling down, nearest 2x upsampling and concatenation [upsampled | skip] up, a 1x1
// head to (u / s_u, W_i / s_W).  It runs at its training size n_net; a finer periodic cube of
// side n_net 2^k is restricted (8-child means) to n_net first and the output prolongated back
// (cell-centred trilinear), both preserving the periodic means.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../include/ctt_unet.h"
#include "mg_common.cuh"

namespace ctt {

namespace {

struct ConvSpec {
    int cin, cout;
};
// forward order: e0a e0 e1a e1 e2a e2 ba b d2a d2 d1a d1 d0a d0
constexpr ConvSpec kConvs[14] = {{16, 16}, {16, 16}, {16, 32}, {32, 32}, {32, 64}, {64, 64}, {64, 64},
                                 {64, 64}, {128, 64}, {64, 64}, {96, 32}, {32, 32}, {48, 16}, {16, 16}};
enum { E0A, E0, E1A, E1, E2A, E2, BA, B, D2A, D2, D1A, D1, D0A, D0 };
constexpr int kHeadIn = 16, kHeadOut = 4;
constexpr char kMagic[8] = {'C', 'T', 'T', 'U', 'N', 'E', 'T', '1'};
constexpr long long kWarmSpin = 1LL << 22;   // bounded waits of the tensor-core kernels

size_t param_count()
{
    size_t n = 0;
    for (const ConvSpec &c : kConvs) n += 27 * (size_t)c.cin * c.cout + c.cout;
    return n + (size_t)kHeadIn * kHeadOut + kHeadOut;
}

bool host_little_endian()
{
    const uint32_t one = 1;
    unsigned char b;
    std::memcpy(&b, &one, 1);
    return b == 1;
}

}  // namespace

struct WarmNet {
    int n_net = 0;
    float s_rho = 1, s_S = 1, s_K = 1, s_u = 1, s_W = 1;
    float *params = nullptr;                  // FP32, the file's flat layout
    __nv_bfloat16 *wf[14] = {};               // packed forward operands
    size_t woff[14] = {}, boff[14] = {}, hw = 0, hb = 0;
    void *x0 = nullptr, *e0a = nullptr, *cat0 = nullptr, *p1 = nullptr, *e1a = nullptr, *cat1 = nullptr,
         *p2 = nullptr, *e2a = nullptr, *cat2 = nullptr, *p3 = nullptr, *ba = nullptr, *b = nullptr,
         *d2a = nullptr, *d2 = nullptr, *d1a = nullptr, *d1 = nullptr, *d0a = nullptr, *d0 = nullptr;
    float *out = nullptr;
    float *ws = nullptr;                      // split-K partial sums of the small-grid convolutions
    size_t ws_bytes = 0;
    int *err = nullptr;
    double *mean = nullptr;                   // means and the partials of their reductions (264)
    std::vector<void *> allocs;
    // FP64 restriction / prolongation buffers per cube side above n_net (5 source, 4 solution fields)
    std::vector<int> side;
    std::vector<double *> src, sol;
};

namespace {

mg_status dev_alloc(WarmNet *w, size_t bytes, void **out)
{
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return fail(MG_ERR_OOM, std::string("warm start cudaMalloc: ") + cudaGetErrorString(e));
    w->allocs.push_back(p);
    *out = p;
    return MG_OK;
}

template <class P>
mg_status dev_alloc_t(WarmNet *w, size_t bytes, P **out)
{
    void *p = nullptr;
    CKS(dev_alloc(w, bytes, &p));
    *out = static_cast<P *>(p);
    return MG_OK;
}

mg_status unet_rc(int rc, const char *what)
{
    if (rc == 0) return MG_OK;
    return fail(rc == 1 ? MG_ERR_INVALID_ARG : MG_ERR_CUDA, std::string("warm start: ") + what + " failed");
}

}  // namespace

void warm_free(WarmNet *w)
{
    if (!w) return;
    for (void *p : w->allocs) cudaFree(p);
    delete w;
}

mg_status warm_load(const char *path, cudaStream_t st, WarmNet **out)
{
    *out = nullptr;
    if (!host_little_endian()) return fail(MG_ERR_UNSUPPORTED, "warm start files are little-endian");
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(MG_ERR_INVALID_ARG, std::string("cannot open warm start weights: ") + path);
    char magic[8];
    int32_t hdr[2];
    float sc[5];
    const size_t count = param_count();
    std::vector<float> host(count);
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              std::fread(hdr, sizeof(int32_t), 2, f) == 2 && std::fread(sc, sizeof(float), 5, f) == 5;
    ok = ok && hdr[1] == (int32_t)count && std::fread(host.data(), sizeof(float), count, f) == count;
    char extra;
    ok = ok && std::fread(&extra, 1, 1, f) == 0;   // nothing after the parameters
    std::fclose(f);
    if (!ok) return fail(MG_ERR_INVALID_ARG, "warm start weights: bad magic, parameter count or length");
    const int n = hdr[0];
    if (n < 64 || n % 8 != 0 || (long long)(n / 8) * (n / 8) * (n / 8) % 128 != 0)
        return fail(MG_ERR_INVALID_ARG, "warm start weights: the network size must be a multiple of 8, >= 64, with "
                                        "(n/8)^3 a multiple of 128");
    for (float v : sc)
        if (!std::isfinite(v) || v == 0.f) return fail(MG_ERR_INVALID_ARG, "warm start weights: bad scale");
    for (float v : host)
        if (!std::isfinite(v)) return fail(MG_ERR_INVALID_ARG, "warm start weights: non-finite parameter");
    WarmNet *w = new (std::nothrow) WarmNet();
    if (!w) return fail(MG_ERR_OOM, "host allocation");
    w->n_net = n;
    w->s_rho = sc[0];
    w->s_S = sc[1];
    w->s_K = sc[2];
    w->s_u = sc[3];
    w->s_W = sc[4];
    mg_status s = MG_OK;
    do {
        size_t off = 0;
        for (int l = 0; l < 14; ++l) {
            w->woff[l] = off;
            off += 27 * (size_t)kConvs[l].cin * kConvs[l].cout;
            w->boff[l] = off;
            off += kConvs[l].cout;
        }
        w->hw = off;
        w->hb = off + (size_t)kHeadIn * kHeadOut;
        if ((s = dev_alloc_t(w, count * sizeof(float), &w->params)) != MG_OK) break;
        cudaError_t e = cudaMemcpyAsync(w->params, host.data(), count * sizeof(float), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { s = fail(MG_ERR_CUDA, "warm start weight upload"); break; }
        for (int l = 0; l < 14 && s == MG_OK; ++l) {
            const size_t nw = 27 * (size_t)kConvs[l].cin * kConvs[l].cout;
            if ((s = dev_alloc_t(w, nw * sizeof(__nv_bfloat16), &w->wf[l])) != MG_OK) break;
            s = unet_rc(unet_pack_weights(w->params + w->woff[l], kConvs[l].cin, kConvs[l].cout, 0, w->wf[l], st),
                        "weight packing");
        }
        if (s != MG_OK) break;
        const size_t v0 = (size_t)n * n * n, v1 = v0 / 8, v2 = v1 / 8, v3 = v2 / 8, bf = sizeof(__nv_bfloat16);
        struct Buf {
            void **p;
            size_t bytes;
        } bufs[] = {{&w->x0, v0 * 16 * bf},  {&w->e0a, v0 * 16 * bf}, {&w->cat0, v0 * 48 * bf},
                    {&w->p1, v1 * 16 * bf},  {&w->e1a, v1 * 32 * bf}, {&w->cat1, v1 * 96 * bf},
                    {&w->p2, v2 * 32 * bf},  {&w->e2a, v2 * 64 * bf}, {&w->cat2, v2 * 128 * bf},
                    {&w->p3, v3 * 64 * bf},  {&w->ba, v3 * 64 * bf},  {&w->b, v3 * 64 * bf},
                    {&w->d2a, v2 * 64 * bf}, {&w->d2, v2 * 64 * bf},  {&w->d1a, v1 * 32 * bf},
                    {&w->d1, v1 * 32 * bf},  {&w->d0a, v0 * 16 * bf}, {&w->d0, v0 * 16 * bf}};
        for (Buf &bb : bufs)
            if ((s = dev_alloc(w, bb.bytes, bb.p)) != MG_OK) break;
        if (s != MG_OK) break;
        if ((s = dev_alloc_t(w, v0 * kHeadOut * sizeof(float), &w->out)) != MG_OK) break;
        for (int l = 0; l < 14; ++l)
            for (int m = n; m >= n / 8; m /= 2)
                w->ws_bytes = std::max(w->ws_bytes, unet_conv3d_fwd_workspace(m, m, m, kConvs[l].cout));
        if (w->ws_bytes && (s = dev_alloc_t(w, w->ws_bytes, &w->ws)) != MG_OK) break;
        if ((s = dev_alloc_t(w, sizeof(int), &w->err)) != MG_OK) break;
        if ((s = dev_alloc_t(w, 264 * sizeof(double), &w->mean)) != MG_OK) break;
        if (cudaMemsetAsync(w->err, 0, sizeof(int), st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            s = fail(MG_ERR_CUDA, "warm start set-up");
            break;
        }
    } while (0);
    if (s != MG_OK) {
        cudaStreamSynchronize(st);
        warm_free(w);
        return s;
    }
    *out = w;
    return MG_OK;
}

// A context the network serves: a periodic cube of side n_net 2^k.
bool warm_supported(const WarmNet *w, const mg_ctx *x)
{
    if (!w || x->cfg.bc != MG_BC_PERIODIC || x->cfg.n[0] != x->cfg.n[1] || x->cfg.n[0] != x->cfg.n[2]) return false;
    int m = x->cfg.n[0];
    while (m > w->n_net && m % 2 == 0) m /= 2;
    return m == w->n_net;
}

namespace {

// FP64 buffers for the sides between n and n_net (allocated once per side, kept).
mg_status warm_levels(WarmNet *w, int n, std::vector<int> *sides, std::vector<double *> *src,
                      std::vector<double *> *sol)
{
    sides->clear();
    src->clear();
    sol->clear();
    for (int m = n / 2; m >= w->n_net; m /= 2) {
        size_t i = 0;
        while (i < w->side.size() && w->side[i] != m) ++i;
        if (i == w->side.size()) {
            const size_t v = (size_t)m * m * m;
            double *a = nullptr, *b = nullptr;
            CKS(dev_alloc_t(w, 5 * v * sizeof(double), &a));
            CKS(dev_alloc_t(w, 4 * v * sizeof(double), &b));
            w->side.push_back(m);
            w->src.push_back(a);
            w->sol.push_back(b);
        }
        sides->push_back(m);
        src->push_back(w->src[i]);
        sol->push_back(w->sol[i]);
    }
    return MG_OK;
}

mg_status warm_forward(WarmNet *w, cudaStream_t st)
{
    const int s0 = w->n_net, s1 = s0 / 2, s2 = s1 / 2, s3 = s2 / 2;
    auto conv = [&](int l, const void *x, int xcs, int xc0, void *y, int ycs, int yc0, int n) {
        return unet_rc(unet_conv3d_fwd(x, xcs, xc0, w->wf[l], w->params + w->boff[l], y, ycs, yc0, n, n, n,
                                       kConvs[l].cin, kConvs[l].cout, 1, w->ws, w->ws_bytes, kWarmSpin, w->err, st),
                       "convolution");
    };
    auto pool = [&](const void *x, int xcs, int xc0, void *y, int c, int n) {
        return unet_rc(unet_avgpool2(x, xcs, xc0, y, c, 0, c, n, n, n, st), "pooling");
    };
    auto up = [&](const void *x, int c, void *y, int ycs, int n) {
        return unet_rc(unet_upsample2(x, c, 0, y, ycs, 0, c, n, n, n, st), "upsampling");
    };
    CKS(conv(E0A, w->x0, 16, 0, w->e0a, 16, 0, s0));
    CKS(conv(E0, w->e0a, 16, 0, w->cat0, 48, 32, s0));   // skip features in channels [32, 48)
    CKS(pool(w->cat0, 48, 32, w->p1, 16, s0));
    CKS(conv(E1A, w->p1, 16, 0, w->e1a, 32, 0, s1));
    CKS(conv(E1, w->e1a, 32, 0, w->cat1, 96, 64, s1));
    CKS(pool(w->cat1, 96, 64, w->p2, 32, s1));
    CKS(conv(E2A, w->p2, 32, 0, w->e2a, 64, 0, s2));
    CKS(conv(E2, w->e2a, 64, 0, w->cat2, 128, 64, s2));
    CKS(pool(w->cat2, 128, 64, w->p3, 64, s2));
    CKS(conv(BA, w->p3, 64, 0, w->ba, 64, 0, s3));
    CKS(conv(B, w->ba, 64, 0, w->b, 64, 0, s3));
    CKS(up(w->b, 64, w->cat2, 128, s3));                  // upsampled features in channels [0, 64)
    CKS(conv(D2A, w->cat2, 128, 0, w->d2a, 64, 0, s2));
    CKS(conv(D2, w->d2a, 64, 0, w->d2, 64, 0, s2));
    CKS(up(w->d2, 64, w->cat1, 96, s2));
    CKS(conv(D1A, w->cat1, 96, 0, w->d1a, 32, 0, s1));
    CKS(conv(D1, w->d1a, 32, 0, w->d1, 32, 0, s1));
    CKS(up(w->d1, 32, w->cat0, 48, s1));
    CKS(conv(D0A, w->cat0, 48, 0, w->d0a, 16, 0, s0));
    CKS(conv(D0, w->d0a, 16, 0, w->d0, 16, 0, s0));
    return unet_rc(unet_head_fwd(w->d0, 16, 0, kHeadIn, w->params + w->hw, w->params + w->hb, w->out, kHeadOut,
                                 (long long)s0 * s0 * s0, st),
                   "head");
}

}  // namespace

// Enqueue the inference for context x on stream st: the guess lands in x->X (u, then W_i).
mg_status warm_enqueue(WarmNet *w, mg_ctx *x, cudaStream_t st)
{
    std::vector<int> sides;
    std::vector<double *> src, sol;
    CKS(warm_levels(w, x->cfg.n[0], &sides, &src, &sol));
    const long long nv = (long long)w->n_net * w->n_net * w->n_net;
    const double *rho0 = x->SRC, *rho2 = x->SRC + x->N, *S = x->SRC + 2 * x->N;
    for (size_t l = 0; l < sides.size(); ++l) {
        const int m = sides[l];
        CKS(unet_rc(unet_restrict2_fields(l == 0 ? x->SRC : src[l - 1], src[l], 5, m, m, m, st), "restriction"));
    }
    if (!sides.empty()) {
        const size_t v = (size_t)nv;
        rho0 = src.back();
        rho2 = src.back() + v;
        S = src.back() + 2 * v;
    }
    // K channel: NaN asks for the value known before the solve, K = -sqrt(24 pi <rho>)
    CKS(unet_rc(unet_pack_input(rho0, rho2, S, NAN, w->s_rho, w->s_S, w->s_K, w->x0, nv, w->mean, st), "input"));
    CKS(warm_forward(w, st));
    double *u = sides.empty() ? x->X : sol.back();
    CKS(unet_rc(unet_unpack_output(w->out, w->s_u, w->s_W, u, u + nv, nv, w->mean, st), "output"));
    for (size_t l = sides.size(); l-- > 0;) {
        const int m = sides[l];
        CKS(unet_rc(unet_prolong2_fields(sol[l], l == 0 ? x->X : sol[l - 1], 4, m, m, m, st), "prolongation"));
    }
    CK(cudaGetLastError());
    return MG_OK;
}

bool warm_timed_out(WarmNet *w, cudaStream_t st)
{
    int h = 0;
    if (cudaMemcpyAsync(&h, w->err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return true;
    return h != 0;
}

}  // namespace ctt
