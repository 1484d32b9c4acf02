// mg_noalloc.cu -- constraint norms of a caller-held state without any device allocation.
//
// For callers that must not allocate device memory: the scratch of this entry point (the
// four FP64 pass-1 fields, the per-block reduction partials and the reduced scalars) lives in
// one file-scope device array, sized for grids of at most kNoallocMaxCells cells, that every
// GPU loading the library holds until the process exits.  The arithmetic is that of the
// context path (mg_residual_norms): the same per-cell residual, integrability K^2 and
// momentum-source means, and max-norms of H and M.
#include <mutex>

#include "mg_common.cuh"

namespace ctt {
namespace {

constexpr size_t kNoallocMaxCells = 64 * 64 * 64;                 // 262,144 cells
constexpr size_t kNoallocR = 4 * kNoallocMaxCells;                // pass-1 output, 4 FP64 fields
constexpr size_t kNoallocPartials = (size_t)kRedBlocks * 8;       // block partials
constexpr size_t kNoallocScalars = 64;                            // >= sizeof(Scalars) / 8
constexpr size_t kNoallocDoubles = kNoallocR + kNoallocPartials + kNoallocScalars;   // 8.47 MB
static_assert(sizeof(Scalars) <= kNoallocScalars * sizeof(double), "scalar slot too small");

static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

// Host code cannot use g_noalloc_scratch as a device address; each device's address is
// looked up once, with that device current, and cached here.
constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
double *g_addr[kMaxDevices] = {};

mg_status scratch_address(double **out)
{
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(MG_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_addr_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return MG_OK;
}

// Pass 1 of the outer residual with the state and sources in separate caller arrays.
template <int ORDER, int BC>
__global__ void __launch_bounds__(256) k_noalloc_pass1(Geo g, Coef<double> cf, const double *__restrict__ u,
                                                       const double *__restrict__ W, const double *__restrict__ rho0,
                                                       const double *__restrict__ rho2, const double *__restrict__ S,
                                                       double *__restrict__ R, double *__restrict__ partial)
{
    const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
    const int sy = g.n[0], sz = g.n[0] * g.n[1];
    double acc[5] = {0, 0, 0, 0, 0};
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(p % g.n[0]);
        size_t rest = p / g.n[0];
        int j = (int)(rest % g.n[1]);
        int k = (int)(rest / g.n[1]);
        double lu, aa, mom[3];
        if (is_interior(g, i, j, k, halo<ORDER>())) {
            AccI<double> a0{u + p, sy, sz}, a1{W + p, sy, sz}, a2{W + N + p, sy, sz}, a3{W + 2 * N + p, sy, sz};
            outer_cell<ORDER>(a0, a1, a2, a3, cf, lu, aa, mom);
        } else {
            AccB<double, BC> a0{u, 0, &g, i, j, k}, a1{W, 1, &g, i, j, k}, a2{W + N, 2, &g, i, j, k},
                a3{W + 2 * N, 3, &g, i, j, k};
            outer_cell<ORDER>(a0, a1, a2, a3, cf, lu, aa, mom);
        }
        double psi = psi_background(g, i, j, k) + u[p];
        double r0 = rho0[p], r2 = rho2 ? rho2[p] : 0.0;
        double ip = 1.0 / psi;
        double p2 = psi * psi, p5 = p2 * p2 * psi, p6 = p5 * psi;
        double ip2 = ip * ip, ip4 = ip2 * ip2, ip7 = ip4 * ip2 * ip;
        double nonlin = 0.125 * aa * ip7 + 2.0 * kPi * (r0 * p5 + r2 * psi);
        R[p] = lu + nonlin;
        acc[0] += nonlin;
        acc[1] += p5;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double s = 8.0 * kPi * p6 * S[a * N + p];
            R[(1 + a) * N + p] = mom[a] - s;
            acc[2 + a] += s;
        }
    }
    double r[5];
    block_sum<5>(acc, r);
    if (threadIdx.x == 0)
        for (int a = 0; a < 5; ++a) partial[blockIdx.x * 5 + a] = r[a];
}

// Block partial maxima of |H| and |M_i| (nothing else is written).
__global__ void __launch_bounds__(256) k_noalloc_norms(Geo g, const double *__restrict__ u,
                                                       const double *__restrict__ R, const Scalars *__restrict__ s,
                                                       double *__restrict__ partial)
{
    const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
    const double K2 = s->K2;
    double mx[4] = {0, 0, 0, 0};
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < N; p += (size_t)gridDim.x * blockDim.x) {
        int i = (int)(p % g.n[0]);
        size_t rest = p / g.n[0];
        int j = (int)(rest % g.n[1]);
        int k = (int)(rest / g.n[1]);
        double psi = psi_background(g, i, j, k) + u[p];
        double p2 = psi * psi, p4 = p2 * p2, p5 = p4 * psi;
        double ip = 1.0 / psi, ip2 = ip * ip, ip5 = ip2 * ip2 * ip, ip6 = ip5 * ip;
        mx[0] = fmax(mx[0], absnan(-8.0 * ip5 * (R[p] - (K2 / 12.0) * p5)));
#pragma unroll
        for (int a = 0; a < 3; ++a) mx[1 + a] = fmax(mx[1 + a], absnan(ip6 * (R[(1 + a) * N + p] + s->msrc[a])));
    }
    double r[4];
    block_max<4>(mx, r);
    if (threadIdx.x == 0)
        for (int a = 0; a < 4; ++a) partial[blockIdx.x * 4 + a] = r[a];
}

mg_status check_config(const mg_config *c)
{
    if (!c) return fail(MG_ERR_INVALID_ARG, "null config");
    for (int a = 0; a < 3; ++a)
        if (c->n[a] < 3 || !(c->hi[a] > c->lo[a])) return fail(MG_ERR_INVALID_ARG, "bad grid size or box");
    if (c->order != 2 && c->order != 4) return fail(MG_ERR_INVALID_ARG, "order must be 2 or 4");
    if (c->bc != MG_BC_PERIODIC && c->bc != MG_BC_ROBIN) return fail(MG_ERR_INVALID_ARG, "bad bc");
    if (c->k_mode != MG_K_FIXED && c->k_mode != MG_K_INTEGRABILITY) return fail(MG_ERR_INVALID_ARG, "bad k_mode");
    if (c->k_mode == MG_K_INTEGRABILITY && c->bc != MG_BC_PERIODIC)
        return fail(MG_ERR_INVALID_ARG, "integrability K needs a periodic box");
    if (c->npunct < 0 || c->npunct > 2) return fail(MG_ERR_INVALID_ARG, "npunct must be 0..2");
    if (c->npunct > 0 && c->bc == MG_BC_PERIODIC) return fail(MG_ERR_UNSUPPORTED, "punctures need Robin boundaries");
    for (int p = 0; p < c->npunct; ++p)
        for (int a = 0; a < 3; ++a)
            if (c->punct_P[p][a] != 0.0 || c->punct_S[p][a] != 0.0)
                return fail(MG_ERR_UNSUPPORTED, "Bowen-York punctures are not supported by the allocation-free norms");
    if (c->reflect != 0) return fail(MG_ERR_UNSUPPORTED, "symmetry planes are not supported by the allocation-free norms");
    if (c->extrap != 0)
        return fail(MG_ERR_UNSUPPORTED, "extrapolating faces are not supported by the allocation-free norms");
    if (!std::isfinite(c->K)) return fail(MG_ERR_INVALID_ARG, "K not finite");
    // each product is checked before the next one is formed, so no cell count wraps around
    const char *msg = "mg_residual_norms_noalloc: the grid exceeds the static scratch limit of 262144 cells (64^3)";
    for (int a = 0; a < 3; ++a)
        if ((size_t)c->n[a] > kNoallocMaxCells) return fail(MG_ERR_INVALID_ARG, msg);
    const size_t n01 = (size_t)c->n[0] * c->n[1];
    if (n01 > kNoallocMaxCells || n01 * c->n[2] > kNoallocMaxCells) return fail(MG_ERR_INVALID_ARG, msg);
    return MG_OK;
}

}  // namespace
}  // namespace ctt

using namespace ctt;

extern "C" mg_status mg_residual_norms_noalloc(const mg_config *cfg, const double *u, const double *W,
                                               const double *rho0, const double *rho2, const double *S,
                                               double out[4], double *K2, void *cuda_stream)
{
    CKS(check_config(cfg));
    if (!u || !W || !rho0 || !S || !out) return fail(MG_ERR_INVALID_ARG, "null pointer");
    double *scratch = nullptr;
    CKS(scratch_address(&scratch));
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Geo g;
    std::memset(&g, 0, sizeof(g));
    for (int a = 0; a < 3; ++a) {
        g.n[a] = cfg->n[a];
        g.lo[a] = cfg->lo[a];
        g.h[a] = (cfg->hi[a] - cfg->lo[a]) / cfg->n[a];
        g.lof[a] = (float)g.lo[a];
        g.hf[a] = (float)g.h[a];
    }
    g.npunct = cfg->npunct;
    for (int p = 0; p < cfg->npunct; ++p) {
        g.pm[p] = cfg->punct_m[p];
        for (int a = 0; a < 3; ++a) g.px[p][a] = cfg->punct_x[p][a];
    }
    const size_t N = (size_t)g.n[0] * g.n[1] * g.n[2];
    double *R = scratch;
    double *partial = scratch + kNoallocR;
    Scalars *sc = reinterpret_cast<Scalars *>(scratch + kNoallocR + kNoallocPartials);
    // the scalars are read back below: start them at zero on every call
    CK(cudaMemsetAsync(sc, 0, sizeof(Scalars), st));
    Coef<double> cf = make_coef<double>(g, cfg->order);
    const int g1 = grid_for(N, kRedBlocks);
    auto launch1 = [&](auto O, auto B) {
        k_noalloc_pass1<decltype(O)::value, decltype(B)::value><<<g1, kThreads, 0, st>>>(g, cf, u, W, rho0, rho2, S, R,
                                                                                         partial);
    };
    using I2 = std::integral_constant<int, 2>;
    using I4 = std::integral_constant<int, 4>;
    using P = std::integral_constant<int, BC_PERIODIC>;
    using Rb = std::integral_constant<int, BC_ROBIN>;
    if (cfg->order == 2) {
        if (cfg->bc == MG_BC_PERIODIC) launch1(I2(), P()); else launch1(I2(), Rb());
    } else {
        if (cfg->bc == MG_BC_PERIODIC) launch1(I4(), P()); else launch1(I4(), Rb());
    }
    k_finalize_sum<5><<<1, 256, 0, st>>>(partial, g1, sc->sums);
    k_outer_scalars<<<1, 1, 0, st>>>(sc, N, cfg->k_mode == MG_K_INTEGRABILITY, cfg->K * cfg->K,
                                     cfg->bc == MG_BC_PERIODIC);
    k_noalloc_norms<<<g1, kThreads, 0, st>>>(g, u, R, sc, partial);
    k_finalize_max<4><<<1, 256, 0, st>>>(partial, g1, sc->norms);
    CK(cudaGetLastError());
    Scalars h;
    CK(cudaMemcpyAsync(&h, sc, sizeof(Scalars), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int a = 0; a < 4; ++a) out[a] = h.norms[a];
    if (K2) *K2 = h.K2;
    return MG_OK;
}
