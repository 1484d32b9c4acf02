// unet_glue.cu -- the non-convolution kernels of the warm-start network and its training:
// weight packing, pooling / upsampling and their adjoints, ReLU adjoint, bias gradients, the
// 1x1 head, MSE loss, Adam, and the conversion between solver fields and network tensors.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/ctt_unet.h"

namespace {

constexpr int kT = 256;

inline int blocks(long long n) { return (int)std::min<long long>((n + kT - 1) / kT, 152LL * 32); }

__global__ void k_pack_weights(const float *w, int cin, int cout, int mode, __nv_bfloat16 *out)
{
    const long long n = 27LL * cin * cout;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        if (mode == 0) {
            out[q] = __float2bfloat16_rn(w[q]);
        } else {   // out[t][ci][co] = w[26 - t][co][ci]
            int co = (int)(q % cout);
            int ci = (int)((q / cout) % cin);
            int t = (int)(q / ((long long)cout * cin));
            out[q] = __float2bfloat16_rn(w[((long long)(26 - t) * cout + co) * cin + ci]);
        }
    }
}

__device__ __forceinline__ long long vox(int i, int j, int k, int n0, int n1) { return i + (long long)n0 * (j + (long long)n1 * k); }

// Row-parallel launches (the inference path): blockIdx.x = one output row (j + n1 * k [+ field]),
// blockIdx.y * blockDim.x + threadIdx.x = the position along it (voxel x, times 8-channel chunks
// for the BF16 tensors), so the per-thread index arithmetic is one 32-bit division.
struct RowLaunch {
    dim3 grid, block;
};

inline RowLaunch row_launch(long long rows, int per_row)
{
    const int t = std::min(256, std::max(32, (per_row + 31) / 32 * 32));
    return {dim3((unsigned)rows, (unsigned)((per_row + t - 1) / t)), dim3(t)};
}

// 2x2x2 average pooling, n = fine size; 8 channels (16 bytes) per thread.
__global__ void k_avgpool2(const __nv_bfloat16 *x, int xcs, int xc0, __nv_bfloat16 *y, int ycs, int yc0, int c,
                           int n0, int n1, int n2)
{
    const int m0 = n0 / 2, m1 = n1 / 2, cc = c / 8;
    const int J = blockIdx.x % m1, K = blockIdx.x / m1;
    const int piece = blockIdx.y * blockDim.x + threadIdx.x;
    if (piece >= m0 * cc) return;
    const int I = piece / cc, ch = (piece - I * cc) * 8;
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int d = 0; d < 8; ++d) {
        const uint4 v = *reinterpret_cast<const uint4 *>(
            x + vox(2 * I + (d & 1), 2 * J + ((d >> 1) & 1), 2 * K + (d >> 2), n0, n1) * xcs + xc0 + ch);
        const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&v);
#pragma unroll
        for (int q = 0; q < 8; ++q) s[q] += __bfloat162float(e[q]);
    }
    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) o[q] = __float2bfloat16_rn(0.125f * s[q]);
    *reinterpret_cast<uint4 *>(y + vox(I, J, K, m0, m1) * ycs + yc0 + ch) = *reinterpret_cast<const uint4 *>(o);
}

__global__ void k_avgpool2_bwd(const __nv_bfloat16 *dy, int dcs, int dc0, __nv_bfloat16 *dx, int xcs, int xc0,
                               int c, int n0, int n1, int n2, int acc)
{
    const long long n = (long long)n0 * n1 * n2 * c;
    const int m0 = n0 / 2, m1 = n1 / 2;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        int ch = (int)(q % c);
        long long v = q / c;
        int i = (int)(v % n0), j = (int)((v / n0) % n1), k = (int)(v / ((long long)n0 * n1));
        float g = 0.125f * __bfloat162float(dy[vox(i / 2, j / 2, k / 2, m0, m1) * dcs + dc0 + ch]);
        __nv_bfloat16 *d = dx + v * xcs + xc0 + ch;
        *d = __float2bfloat16_rn(acc ? __bfloat162float(*d) + g : g);
    }
}

// nearest 2x upsampling, n = coarse size; 8 channels (16 bytes) per thread.
__global__ void k_upsample2(const __nv_bfloat16 *x, int xcs, int xc0, __nv_bfloat16 *y, int ycs, int yc0, int c,
                            int n0, int n1, int n2)
{
    const int f0 = 2 * n0, f1 = 2 * n1, cc = c / 8;
    const int j = blockIdx.x % f1, k = blockIdx.x / f1;
    const int piece = blockIdx.y * blockDim.x + threadIdx.x;
    if (piece >= f0 * cc) return;
    const int i = piece / cc, ch = (piece - i * cc) * 8;
    *reinterpret_cast<uint4 *>(y + vox(i, j, k, f0, f1) * ycs + yc0 + ch) =
        *reinterpret_cast<const uint4 *>(x + vox(i / 2, j / 2, k / 2, n0, n1) * xcs + xc0 + ch);
}

__global__ void k_upsample2_bwd(const __nv_bfloat16 *dy, int dcs, int dc0, __nv_bfloat16 *dx, int xcs, int xc0,
                                int c, int n0, int n1, int n2)
{
    const int f0 = 2 * n0, f1 = 2 * n1;
    const long long n = (long long)n0 * n1 * n2 * c;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        int ch = (int)(q % c);
        long long V = q / c;
        int I = (int)(V % n0), J = (int)((V / n0) % n1), K = (int)(V / ((long long)n0 * n1));
        float s = 0.f;
        for (int d = 0; d < 8; ++d)
            s += __bfloat162float(dy[vox(2 * I + (d & 1), 2 * J + ((d >> 1) & 1), 2 * K + (d >> 2), f0, f1) * dcs + dc0 + ch]);
        dx[V * xcs + xc0 + ch] = __float2bfloat16_rn(s);
    }
}

__global__ void k_relu_bwd(__nv_bfloat16 *dy, int dcs, int dc0, const __nv_bfloat16 *y, int ycs, int yc0, int c,
                           long long nvox)
{
    const long long n = nvox * c;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        int ch = (int)(q % c);
        long long v = q / c;
        if (!(__bfloat162float(y[v * ycs + yc0 + ch]) > 0.f)) dy[v * dcs + dc0 + ch] = __float2bfloat16_rn(0.f);
    }
}

// one block per channel slice of up to 32 channels: partial sums over voxels, then atomics
__global__ void k_bias_grad(const __nv_bfloat16 *dy, int dcs, int dc0, float *db, int c, long long nvox)
{
    __shared__ float sh[8][32];
    const int ch = threadIdx.x & 31, lane_row = threadIdx.x >> 5;
    const int cbase = blockIdx.y * 32;
    float s = 0.f;
    if (cbase + ch < c)
        for (long long v = blockIdx.x * 8LL + lane_row; v < nvox; v += (long long)gridDim.x * 8)
            s += __bfloat162float(dy[v * dcs + dc0 + cbase + ch]);
    sh[lane_row][ch] = s;
    __syncthreads();
    if (lane_row == 0 && cbase + ch < c) {
        float t = 0.f;
        for (int r = 0; r < 8; ++r) t += sh[r][ch];
        atomicAdd(db + cbase + ch, t);
    }
}

__global__ void k_head_fwd(const __nv_bfloat16 *x, int xcs, int xc0, int cin, const float *w, const float *b,
                           float *out, int cout, long long nvox)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        float acc[8];
        for (int o = 0; o < cout; ++o) acc[o] = b[o];
        for (int c = 0; c < cin; ++c) {
            float xv = __bfloat162float(x[v * xcs + xc0 + c]);
            for (int o = 0; o < cout; ++o) acc[o] += w[o * cin + c] * xv;
        }
        for (int o = 0; o < cout; ++o) out[v * cout + o] = acc[o];
    }
}

// dx = w^T dout (BF16); dw, db accumulated per block in shared memory, then atomics
__global__ void k_head_bwd(const __nv_bfloat16 *x, int xcs, int xc0, int cin, const float *w, const float *dout,
                           int cout, __nv_bfloat16 *dx, int dxcs, int dxc0, float *dw, float *db, long long nvox)
{
    __shared__ float sdw[8 * 64], sdb[8];
    for (int q = threadIdx.x; q < cout * cin; q += blockDim.x) sdw[q] = 0.f;
    if (threadIdx.x < 8) sdb[threadIdx.x] = 0.f;
    __syncthreads();
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        float g[8];
        for (int o = 0; o < cout; ++o) {
            g[o] = dout[v * cout + o];
            atomicAdd(&sdb[o], g[o]);
        }
        for (int c = 0; c < cin; ++c) {
            float xv = __bfloat162float(x[v * xcs + xc0 + c]);
            float s = 0.f;
            for (int o = 0; o < cout; ++o) {
                s += w[o * cin + c] * g[o];
                atomicAdd(&sdw[o * cin + c], g[o] * xv);
            }
            dx[v * dxcs + dxc0 + c] = __float2bfloat16_rn(s);
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < cout * cin; q += blockDim.x) atomicAdd(dw + q, sdw[q]);
    if (threadIdx.x < cout) atomicAdd(db + threadIdx.x, sdb[threadIdx.x]);
}

__global__ void k_mse(const float *out, const float *t, float *dout, float *loss, long long n)
{
    __shared__ float sh[kT];
    float s = 0.f;
    const float inv = 1.0f / (float)n;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        float d = out[q] - t[q];
        s += d * d;
        dout[q] = 2.f * d * inv;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, sh[0] * inv);
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2,
                       float eps, float c1, float c2)
{
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        float gq = g[q];
        float mq = b1 * m[q] + (1.f - b1) * gq;
        float vq = b2 * v[q] + (1.f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        p[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
    }
}

// Mean of one FP64 field (a + b when b is given), deterministic: kMeanBlocks blocks each sum a
// fixed grid-stride subset into partial[block], then one block adds the partials in order.
constexpr int kMeanBlocks = 256;

__device__ __forceinline__ double block_reduce_sum(double s)
{
    __shared__ double sh[kT];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    return sh[0];
}

__global__ void k_mean_partial(const double *a, const double *b, long long n, double *partial)
{
    double s = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        s += a[q] + (b ? b[q] : 0.0);
    const double t = block_reduce_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void k_mean_finish(const double *partial, int np, long long n, double *mean)
{
    double s = 0.0;
    for (int q = threadIdx.x; q < np; q += blockDim.x) s += partial[q];
    const double t = block_reduce_sum(s);
    if (threadIdx.x == 0) *mean = t / (double)n;
}

// scratch: means in [0, 8), block partials in [8, 8 + kMeanBlocks)
void launch_mean(const double *a, const double *b, long long n, double *scratch, int slot, cudaStream_t st)
{
    k_mean_partial<<<kMeanBlocks, kT, 0, st>>>(a, b, n, scratch + 8);
    k_mean_finish<<<1, kT, 0, st>>>(scratch + 8, kMeanBlocks, n, scratch + slot);
}

__global__ void k_pack_input(const double *rho0, const double *rho2, const double *S, double K, float s_rho,
                             float s_S, float s_K, __nv_bfloat16 *x16, long long nvox, const double *mean)
{
    const double mu = *mean;
    // K given, or (NaN) its value at psi = 1 from the discrete integrability condition, K^2 = 24 pi <rho>
    const double Kv = (K == K) ? K : -sqrt(24.0 * 3.14159265358979323846 * fmax(mu, 0.0));
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        __align__(16) __nv_bfloat16 o[16];
        double r = rho0[v] + (rho2 ? rho2[v] : 0.0);
        o[0] = __float2bfloat16_rn((float)((r - mu) * s_rho));
        for (int a = 0; a < 3; ++a) o[1 + a] = __float2bfloat16_rn((float)(S[a * nvox + v] * s_S));
        o[4] = __float2bfloat16_rn((float)(Kv * s_K));
        for (int c = 5; c < 16; ++c) o[c] = __float2bfloat16_rn(0.f);
        uint4 *d = reinterpret_cast<uint4 *>(x16 + v * 16);
        d[0] = reinterpret_cast<uint4 *>(o)[0];
        d[1] = reinterpret_cast<uint4 *>(o)[1];
    }
}

__global__ void k_unpack_output(const float *out4, float s_u, float s_W, double *u, double *W, long long nvox)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        u[v] = (double)out4[v * 4] * s_u;
        for (int a = 0; a < 3; ++a) W[a * nvox + v] = (double)out4[v * 4 + 1 + a] * s_W;
    }
}

__global__ void k_sub_mean(double *a, long long n, const double *mean)
{
    const double mu = *mean;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        a[q] -= mu;
}

__global__ void k_pack_target(const double *u, const double *W, float s_u, float s_W, float *t4, long long nvox)
{
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nvox; v += (long long)gridDim.x * blockDim.x) {
        t4[v * 4] = (float)(u[v] / s_u);
        for (int a = 0; a < 3; ++a) t4[v * 4 + 1 + a] = (float)(W[a * nvox + v] / s_W);
    }
}

// mean of the 8 children of FP64 fields: nf fields of the fine grid (2 m)^3 -> m^3
__global__ void k_restrict2_f64(const double *fine, double *coarse, int nf, int m0, int m1, int m2)
{
    const long long nc = (long long)m0 * m1 * m2, nfv = 8 * nc;
    const int row = blockIdx.x, J = row % m1, K = (row / m1) % m2, f = row / (m1 * m2);
    const int I = blockIdx.y * blockDim.x + threadIdx.x;
    if (I >= m0) return;
    const double *src = fine + f * nfv;
    double s = 0.0;
#pragma unroll
    for (int d = 0; d < 8; ++d) s += src[vox(2 * I + (d & 1), 2 * J + ((d >> 1) & 1), 2 * K + (d >> 2), 2 * m0, 2 * m1)];
    coarse[f * nc + vox(I, J, K, m0, m1)] = 0.125 * s;
}

// cell-centred trilinear interpolation (weights 3/4, 1/4 per axis, periodic) of nf FP64 fields
// from m^3 to (2 m)^3
__global__ void k_prolong2_f64(const double *coarse, double *fine, int nf, int m0, int m1, int m2)
{
    const long long nc = (long long)m0 * m1 * m2, nfv = 8 * nc;
    const int f0 = 2 * m0, f1 = 2 * m1, f2 = 2 * m2;
    const int row = blockIdx.x, j = row % f1, k = (row / f1) % f2, f = row / (f1 * f2);
    const int i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= f0) return;
    const int I = i >> 1, J = j >> 1, K = k >> 1;
    const int sx = (i & 1) ? 1 : -1, sy = (j & 1) ? 1 : -1, sz = (k & 1) ? 1 : -1;
    const double *src = coarse + f * nc;
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int a = c & 1, b = (c >> 1) & 1, e = c >> 2;
        const double w = (a ? 0.25 : 0.75) * (b ? 0.25 : 0.75) * (e ? 0.25 : 0.75);
        int ii = I + a * sx, jj = J + b * sy, kk = K + e * sz;
        ii += ii < 0 ? m0 : (ii >= m0 ? -m0 : 0);
        jj += jj < 0 ? m1 : (jj >= m1 ? -m1 : 0);
        kk += kk < 0 ? m2 : (kk >= m2 ? -m2 : 0);
        s += w * src[vox(ii, jj, kk, m0, m1)];
    }
    fine[f * nfv + vox(i, j, k, f0, f1)] = s;
}

inline int ok() { return cudaGetLastError() == cudaSuccess ? 0 : 3; }

}  // namespace

extern "C" {

int unet_pack_weights(const float *w, int cin, int cout, int mode, void *out, void *stream)
{
    if (!w || !out || cin <= 0 || cout <= 0 || (mode != 0 && mode != 1)) return 1;
    k_pack_weights<<<blocks(27LL * cin * cout), kT, 0, (cudaStream_t)stream>>>(w, cin, cout, mode, (__nv_bfloat16 *)out);
    return ok();
}

int unet_avgpool2(const void *x, int xcs, int xc0, void *y, int ycs, int yc0, int c, int n0, int n1, int n2, void *stream)
{
    if (!x || !y || (n0 | n1 | n2) & 1 || n0 <= 0 || n1 <= 0 || n2 <= 0 || c <= 0 || (c | xcs | xc0 | ycs | yc0) & 7)
        return 1;
    const RowLaunch L = row_launch((long long)(n1 / 2) * (n2 / 2), n0 / 2 * (c / 8));
    k_avgpool2<<<L.grid, L.block, 0, (cudaStream_t)stream>>>((const __nv_bfloat16 *)x, xcs, xc0, (__nv_bfloat16 *)y,
                                                             ycs, yc0, c, n0, n1, n2);
    return ok();
}

int unet_avgpool2_bwd(const void *dy, int dcs, int dc0, void *dx, int xcs, int xc0, int c, int n0, int n1, int n2,
                      int accumulate, void *stream)
{
    if (!dy || !dx || (n0 | n1 | n2) & 1) return 1;
    k_avgpool2_bwd<<<blocks((long long)n0 * n1 * n2 * c), kT, 0, (cudaStream_t)stream>>>(
        (const __nv_bfloat16 *)dy, dcs, dc0, (__nv_bfloat16 *)dx, xcs, xc0, c, n0, n1, n2, accumulate);
    return ok();
}

int unet_upsample2(const void *x, int xcs, int xc0, void *y, int ycs, int yc0, int c, int n0, int n1, int n2, void *stream)
{
    if (!x || !y || n0 <= 0 || n1 <= 0 || n2 <= 0 || c <= 0 || (c | xcs | xc0 | ycs | yc0) & 7) return 1;
    const RowLaunch L = row_launch(4LL * n1 * n2, 2 * n0 * (c / 8));
    k_upsample2<<<L.grid, L.block, 0, (cudaStream_t)stream>>>((const __nv_bfloat16 *)x, xcs, xc0, (__nv_bfloat16 *)y,
                                                              ycs, yc0, c, n0, n1, n2);
    return ok();
}

int unet_upsample2_bwd(const void *dy, int dcs, int dc0, void *dx, int xcs, int xc0, int c, int n0, int n1, int n2,
                       void *stream)
{
    if (!dy || !dx) return 1;
    k_upsample2_bwd<<<blocks((long long)n0 * n1 * n2 * c), kT, 0, (cudaStream_t)stream>>>(
        (const __nv_bfloat16 *)dy, dcs, dc0, (__nv_bfloat16 *)dx, xcs, xc0, c, n0, n1, n2);
    return ok();
}

int unet_relu_bwd(void *dy, int dcs, int dc0, const void *y, int ycs, int yc0, int c, long long nvox, void *stream)
{
    if (!dy || !y) return 1;
    k_relu_bwd<<<blocks(nvox * c), kT, 0, (cudaStream_t)stream>>>((__nv_bfloat16 *)dy, dcs, dc0,
                                                                   (const __nv_bfloat16 *)y, ycs, yc0, c, nvox);
    return ok();
}

int unet_bias_grad(const void *dy, int dcs, int dc0, float *db, int c, long long nvox, void *stream)
{
    if (!dy || !db) return 1;
    dim3 grid((unsigned)std::min<long long>((nvox + 7) / 8, 1024), (c + 31) / 32);
    k_bias_grad<<<grid, 256, 0, (cudaStream_t)stream>>>((const __nv_bfloat16 *)dy, dcs, dc0, db, c, nvox);
    return ok();
}

int unet_head_fwd(const void *x, int xcs, int xc0, int cin, const float *w, const float *b, float *out, int cout,
                  long long nvox, void *stream)
{
    if (!x || !w || !b || !out || cout > 8 || cin > 64) return 1;
    k_head_fwd<<<blocks(nvox), kT, 0, (cudaStream_t)stream>>>((const __nv_bfloat16 *)x, xcs, xc0, cin, w, b, out,
                                                               cout, nvox);
    return ok();
}

int unet_head_bwd(const void *x, int xcs, int xc0, int cin, const float *w, const float *dout, int cout, void *dx,
                  int dxcs, int dxc0, float *dw, float *db, long long nvox, void *stream)
{
    if (!x || !w || !dout || !dx || !dw || !db || cout > 8 || cin > 64) return 1;
    k_head_bwd<<<(int)std::min<long long>((nvox + kT - 1) / kT, 152LL * 4), kT, 0, (cudaStream_t)stream>>>(
        (const __nv_bfloat16 *)x, xcs, xc0, cin, w, dout, cout, (__nv_bfloat16 *)dx, dxcs, dxc0, dw, db, nvox);
    return ok();
}

int unet_mse(const float *out, const float *target, float *dout, float *loss, int c, long long nvox, void *stream)
{
    if (!out || !target || !dout || !loss) return 1;
    k_mse<<<(int)std::min<long long>((nvox * c + kT - 1) / kT, 152LL * 8), kT, 0, (cudaStream_t)stream>>>(
        out, target, dout, loss, nvox * c);
    return ok();
}

int unet_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2, float eps, int t,
              void *stream)
{
    if (!p || !g || !m || !v || t < 1) return 1;
    float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam<<<blocks(n), kT, 0, (cudaStream_t)stream>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return ok();
}

int unet_pack_input(const double *rho0, const double *rho2, const double *S, double K, float s_rho, float s_S,
                    float s_K, void *x16, long long nvox, double *scratch_mean, void *stream)
{
    if (!rho0 || !S || !x16 || !scratch_mean) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    launch_mean(rho0, rho2, nvox, scratch_mean, 0, st);
    k_pack_input<<<blocks(nvox), kT, 0, st>>>(rho0, rho2, S, K, s_rho, s_S, s_K, (__nv_bfloat16 *)x16, nvox,
                                               scratch_mean);
    return ok();
}

int unet_unpack_output(const float *out4, float s_u, float s_W, double *u, double *W, long long nvox,
                       double *scratch_mean, void *stream)
{
    if (!out4 || !u || !W || !scratch_mean) return 1;
    cudaStream_t st = (cudaStream_t)stream;
    k_unpack_output<<<blocks(nvox), kT, 0, st>>>(out4, s_u, s_W, u, W, nvox);
    for (int a = 0; a < 4; ++a) {
        double *f = a == 0 ? u : W + (a - 1) * nvox;
        launch_mean(f, nullptr, nvox, scratch_mean, a, st);
        k_sub_mean<<<blocks(nvox), kT, 0, st>>>(f, nvox, scratch_mean + a);
    }
    return ok();
}

int unet_restrict2_fields(const double *fine, double *coarse, int nfields, int m0, int m1, int m2, void *stream)
{
    if (!fine || !coarse || nfields < 1 || m0 <= 0 || m1 <= 0 || m2 <= 0) return 1;
    const RowLaunch L = row_launch((long long)m1 * m2 * nfields, m0);
    k_restrict2_f64<<<L.grid, L.block, 0, (cudaStream_t)stream>>>(fine, coarse, nfields, m0, m1, m2);
    return ok();
}

int unet_prolong2_fields(const double *coarse, double *fine, int nfields, int m0, int m1, int m2, void *stream)
{
    if (!fine || !coarse || nfields < 1 || m0 <= 0 || m1 <= 0 || m2 <= 0) return 1;
    const RowLaunch L = row_launch(4LL * m1 * m2 * nfields, 2 * m0);
    k_prolong2_f64<<<L.grid, L.block, 0, (cudaStream_t)stream>>>(coarse, fine, nfields, m0, m1, m2);
    return ok();
}

int unet_pack_target(const double *u, const double *W, float s_u, float s_W, float *t4, long long nvox, void *stream)
{
    if (!u || !W || !t4) return 1;
    k_pack_target<<<blocks(nvox), kT, 0, (cudaStream_t)stream>>>(u, W, s_u, s_W, t4, nvox);
    return ok();
}

}  // extern "C"
