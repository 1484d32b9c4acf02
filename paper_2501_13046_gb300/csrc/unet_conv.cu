// unet_conv.cu -- implicit-GEMM 3x3x3 convolutions with circular padding on tcgen05.
//
// Tensors are NDHWC BF16 (a voxel's channels contiguous); a tensor may be a channel slice
// [c0, c0 + C) of a buffer with cs channels per voxel, which makes channel concatenation free.
// Weights: FP32 master [27 taps][Cout][Cin] (tap = (dz+1)*9 + (dy+1)*3 + (dx+1)), packed to
// BF16 in the same order for the forward pass.
//
// Forward / input gradient (k_conv3d_tc): one CTA = 128 consecutive output voxels x all Cout.
// For each of the 27 taps the CTA gathers the shifted input rows (128 x Cin, wrapped) and the
// tap's weights (Cout x Cin) into shared memory in the canonical K-major core-matrix layout and
// thread 0 issues Cin/16 MMAs (M = 128, N = Cout, K = 16) accumulating in TMEM; buffers are
// double-buffered and recycled when the tap's commit arrives.  Epilogue: TMEM -> registers,
// + bias, ReLU, BF16, store.  The input gradient of a convolution is the convolution of the
// output gradient with the tap-flipped, transposed weights, so it reuses this kernel.
//
// Weight gradient (k_conv3d_wgrad_tc): dW[t][co][ci] = sum_v dY[v][co] X[v + t][ci] as a GEMM
// with M = 128 rows of (tap, ci), N = Cout, K = voxels; each CTA reduces one chunk of voxels in
// TMEM and adds its partial into FP32 dW with atomics (split-K).
#include <algorithm>

#include "unet_tc.cuh"

namespace unet {

constexpr int kTile = 128;

struct ConvArgs {
    const __nv_bfloat16 *x;
    int xcs, xc0;             // input channel stride and offset
    const __nv_bfloat16 *w;   // [27][Cout][Cin] BF16
    const float *bias;        // Cout (may be null)
    __nv_bfloat16 *y;
    int ycs, yc0;
    int n0, n1, n2;
    int relu;
    long long spin_limit;
    int *err;                 // set to 1 when a bounded wait gave up
};

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <int CIN, int COUT>
__global__ void __launch_bounds__(128) k_conv3d_tc(ConvArgs a)
{
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= 128, "channel counts");
    constexpr int NCOLS = COUT <= 32 ? 32 : (COUT <= 64 ? 64 : 128);
    constexpr uint32_t A_BYTES = kTile * CIN * 2, B_BYTES = COUT * CIN * 2;
    constexpr uint32_t SBO_A = (CIN / 8) * 128, SBO_B = (CIN / 8) * 128;
    constexpr uint32_t IDESC = idesc_bf16(kTile, COUT);
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Abuf = smem;                       // 2 x A_BYTES
    unsigned char *Bbuf = smem + 2 * A_BYTES;         // 2 x B_BYTES
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nx = a.n0, ny = a.n1, nz = a.n2;
    const int v0 = blockIdx.x * kTile;
    if (warp == 0) tmem_alloc(&tmem_slot, NCOLS);
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;

    for (int tap = 0; tap < 27; ++tap) {
        const int buf = tap & 1;
        if (tap >= 2) {   // the MMAs of tap - 2 have finished reading this buffer
            if (tid == 0 && !failed && !mbar_wait_bounded(&mbar[buf], ((tap - 2) >> 1) & 1, a.spin_limit)) failed = 1;
            __syncthreads();
            if (failed) break;
        }
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        unsigned char *A = Abuf + buf * A_BYTES;
        unsigned char *B = Bbuf + buf * B_BYTES;
        constexpr int CH = CIN / 8;   // 16-byte chunks per row
        for (int idx = tid; idx < kTile * CH; idx += 128) {
            int r = idx / CH, c = idx - r * CH;
            int v = v0 + r;
            int i = v % nx, j = (v / nx) % ny, k = v / (nx * ny);
            int nb = wrapi(i + dx, nx) + nx * (wrapi(j + dy, ny) + ny * wrapi(k + dz, nz));
            uint4 val = *reinterpret_cast<const uint4 *>(a.x + (size_t)nb * a.xcs + a.xc0 + c * 8);
            *reinterpret_cast<uint4 *>(A + (r >> 3) * SBO_A + c * 128 + (r & 7) * 16) = val;
        }
        const __nv_bfloat16 *wt = a.w + (size_t)tap * COUT * CIN;
        for (int idx = tid; idx < COUT * CH; idx += 128) {
            int r = idx / CH, c = idx - r * CH;
            uint4 val = *reinterpret_cast<const uint4 *>(wt + r * CIN + c * 8);
            *reinterpret_cast<uint4 *>(B + (r >> 3) * SBO_B + c * 128 + (r & 7) * 16) = val;
        }
        fence_proxy_async();
        fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            fence_after_sync();
            const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
#pragma unroll
            for (int kk = 0; kk < CIN / 16; ++kk)
                mma_bf16(tmem, smem_desc(a0 + kk * 256, 128, SBO_A), smem_desc(b0 + kk * 256, 128, SBO_B), IDESC,
                         (tap > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&mbar[buf]);
        }
    }
    // wait for the last tap (tap 26 on buffer 0, its 14th use: parity 1); the MMAs complete in order
    if (tid == 0) {
        bool ok = !failed && mbar_wait_bounded(&mbar[0], 1, a.spin_limit);
        if (!ok) {
            failed = 1;
            // give any MMA still in flight a second bounded wait before the buffers go away
            mbar_wait_bounded(&mbar[0], 1, a.spin_limit);
            mbar_wait_bounded(&mbar[1], 0, a.spin_limit);
        }
    }
    __syncthreads();
    fence_after_sync();
    if (!failed) {
        const int row = warp * 32 + lane;
        const size_t v = (size_t)v0 + row;
#pragma unroll
        for (int cc = 0; cc < COUT / 16; ++cc) {
            float acc[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + cc * 16, acc);
            __align__(16) __nv_bfloat16 o[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                float t = acc[q] + (a.bias ? a.bias[cc * 16 + q] : 0.f);
                if (a.relu) t = fmaxf(t, 0.f);
                o[q] = __float2bfloat16_rn(t);
            }
            uint4 *dst = reinterpret_cast<uint4 *>(a.y + v * a.ycs + a.yc0 + cc * 16);
            dst[0] = reinterpret_cast<uint4 *>(o)[0];
            dst[1] = reinterpret_cast<uint4 *>(o)[1];
        }
    } else if (tid == 0) {
        atomicExch(a.err, 1);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

struct WgradArgs {
    const __nv_bfloat16 *x;
    int xcs, xc0;
    const __nv_bfloat16 *dy;
    int dcs, dc0;
    float *dw;                // [27][Cout][Cin] FP32, accumulated
    int n0, n1, n2;
    int chunks_per_cta;       // voxel chunks of 128 reduced by one CTA
    long long spin_limit;
    int *err;
};

// grid: x = tap groups (TPG taps of CIN rows each, TPG * CIN <= 128), y = voxel splits.
template <int CIN, int COUT>
__global__ void __launch_bounds__(128) k_conv3d_wgrad_tc(WgradArgs a)
{
    static_assert(CIN % 8 == 0 && COUT % 16 == 0 && COUT <= 128, "channel counts");
    constexpr int TPG = CIN <= 128 ? 128 / CIN : 1;       // taps per group
    constexpr int NCOLS = COUT <= 32 ? 32 : (COUT <= 64 ? 64 : 128);
    constexpr int KV = 128;                                // voxels per stage
    constexpr uint32_t A_BYTES = 128 * KV * 2, B_BYTES = COUT * KV * 2;
    constexpr uint32_t SBO = (KV / 8) * 128;
    constexpr uint32_t IDESC = idesc_bf16(128, COUT);
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Abuf = smem;
    unsigned char *Bbuf = smem + 2 * A_BYTES;
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nx = a.n0, ny = a.n1, nz = a.n2;
    const int nvox = nx * ny * nz;
    const int tap0 = blockIdx.x * TPG;
    const int ntap = min(TPG, 27 - tap0);
    if (warp == 0) tmem_alloc(&tmem_slot, NCOLS);
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;
    const int chunk0 = blockIdx.y * a.chunks_per_cta;
    const int nchunks = min(a.chunks_per_cta, nvox / KV - chunk0);
    int issued = 0;
    for (int s = 0; s < nchunks; ++s) {
        const int buf = s & 1;
        if (s >= 2) {
            if (tid == 0 && !failed && !mbar_wait_bounded(&mbar[buf], ((s - 2) >> 1) & 1, a.spin_limit)) failed = 1;
            __syncthreads();
            if (failed) break;
        }
        unsigned char *A = Abuf + buf * A_BYTES;
        unsigned char *B = Bbuf + buf * B_BYTES;
        const int vbase = (chunk0 + s) * KV;
        // A rows r = tl * CIN + ci (tap tl of the group, input channel ci), K = voxel kv
        for (int idx = tid; idx < 128 * (KV / 8); idx += 128) {   // zero unused rows first
            int r = idx / (KV / 8), kc = idx % (KV / 8);
            if (r >= ntap * CIN) *reinterpret_cast<uint4 *>(A + (r >> 3) * SBO + kc * 128 + (r & 7) * 16) = make_uint4(0, 0, 0, 0);
        }
        for (int idx = tid; idx < ntap * KV * (CIN / 8); idx += 128) {
            int c = idx % (CIN / 8);
            int kv = (idx / (CIN / 8)) % KV;
            int tl = idx / ((CIN / 8) * KV);
            int tap = tap0 + tl;
            int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
            int v = vbase + kv;
            int i = v % nx, j = (v / nx) % ny, k = v / (nx * ny);
            int nb = wrapi(i + dx, nx) + nx * (wrapi(j + dy, ny) + ny * wrapi(k + dz, nz));
            uint4 val = *reinterpret_cast<const uint4 *>(a.x + (size_t)nb * a.xcs + a.xc0 + c * 8);
            const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&val);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                int r = tl * CIN + c * 8 + q;
                *reinterpret_cast<__nv_bfloat16 *>(A + (r >> 3) * SBO + (kv >> 3) * 128 + (r & 7) * 16 + (kv & 7) * 2) = e[q];
            }
        }
        for (int idx = tid; idx < KV * (COUT / 8); idx += 128) {
            int c = idx % (COUT / 8), kv = idx / (COUT / 8);
            uint4 val = *reinterpret_cast<const uint4 *>(a.dy + (size_t)(vbase + kv) * a.dcs + a.dc0 + c * 8);
            const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&val);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                int r = c * 8 + q;
                *reinterpret_cast<__nv_bfloat16 *>(B + (r >> 3) * SBO + (kv >> 3) * 128 + (r & 7) * 16 + (kv & 7) * 2) = e[q];
            }
        }
        fence_proxy_async();
        fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            fence_after_sync();
            const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
#pragma unroll
            for (int kk = 0; kk < KV / 16; ++kk)
                mma_bf16(tmem, smem_desc(a0 + kk * 256, 128, SBO), smem_desc(b0 + kk * 256, 128, SBO), IDESC,
                         (s > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&mbar[buf]);
        }
        ++issued;
    }
    if (tid == 0 && issued > 0) {
        const int last = issued - 1;
        bool ok = !failed && mbar_wait_bounded(&mbar[last & 1], (last >> 1) & 1, a.spin_limit);
        if (!ok) {
            failed = 1;
            mbar_wait_bounded(&mbar[last & 1], (last >> 1) & 1, a.spin_limit);
        }
    }
    __syncthreads();
    fence_after_sync();
    if (!failed && issued > 0) {
        const int row = warp * 32 + lane;   // (tap tl, ci)
        const int tl = row / CIN, ci = row % CIN;
#pragma unroll
        for (int cc = 0; cc < COUT / 16; ++cc) {
            float acc[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + cc * 16, acc);
            if (tl < ntap) {
                float *d = a.dw + ((size_t)(tap0 + tl) * COUT + cc * 16) * CIN + ci;
#pragma unroll
                for (int q = 0; q < 16; ++q) atomicAdd(d + (size_t)q * CIN, acc[q]);
            }
        }
    } else if (failed && tid == 0) {
        atomicExch(a.err, 1);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

}  // namespace unet

// ====================================================================== host side
#include "../../include/ctt_unet.h"

namespace unet {
namespace {

template <int CIN, int COUT>
int launch_fwd(const ConvArgs &a, int nvox, cudaStream_t st)
{
    constexpr size_t smem = 2 * (kTile * CIN * 2) + 2 * (COUT * CIN * 2);
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_conv3d_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return 3;
        attr = true;
    }
    k_conv3d_tc<CIN, COUT><<<nvox / kTile, 128, smem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

template <int CIN, int COUT>
int launch_wgrad(const WgradArgs &a0, int nvox, cudaStream_t st)
{
    constexpr int TPG = 128 / CIN > 0 ? 128 / CIN : 1;
    constexpr size_t smem = 2 * (128 * 128 * 2) + 2 * (COUT * 128 * 2);
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_conv3d_wgrad_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return 3;
        attr = true;
    }
    WgradArgs a = a0;
    const int chunks = nvox / 128;
    const int groups = (27 + TPG - 1) / TPG;
    // enough CTAs to fill the GPU a few times over: split the voxel chunks
    int splits = std::max(1, std::min(chunks, (152 * 4 + groups - 1) / groups));
    a.chunks_per_cta = (chunks + splits - 1) / splits;
    splits = (chunks + a.chunks_per_cta - 1) / a.chunks_per_cta;
    k_conv3d_wgrad_tc<CIN, COUT><<<dim3(groups, splits), 128, smem, st>>>(a);
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

#define PAIR(ci, co) (((ci) << 8) | (co))

}  // namespace
}  // namespace unet

using namespace unet;

extern "C" int unet_conv3d_fwd(const void *x, int xcs, int xc0, const void *w_bf16, const float *bias, void *y,
                               int ycs, int yc0, int n0, int n1, int n2, int cin, int cout, int relu,
                               long long spin_limit, int *err, void *stream)
{
    long long nvox = (long long)n0 * n1 * n2;
    if (!x || !w_bf16 || !y || !err || nvox <= 0 || nvox % kTile || (xcs | xc0 | ycs | yc0) % 8 ||
        xc0 + cin > xcs || yc0 + cout > ycs)
        return 1;
    ConvArgs a{(const __nv_bfloat16 *)x, xcs, xc0, (const __nv_bfloat16 *)w_bf16, bias, (__nv_bfloat16 *)y,
               ycs, yc0, n0, n1, n2, relu, spin_limit, err};
    cudaStream_t st = (cudaStream_t)stream;
    switch (PAIR(cin, cout)) {
    case PAIR(16, 16): return launch_fwd<16, 16>(a, (int)nvox, st);
    case PAIR(16, 32): return launch_fwd<16, 32>(a, (int)nvox, st);
    case PAIR(16, 48): return launch_fwd<16, 48>(a, (int)nvox, st);
    case PAIR(32, 16): return launch_fwd<32, 16>(a, (int)nvox, st);
    case PAIR(32, 32): return launch_fwd<32, 32>(a, (int)nvox, st);
    case PAIR(32, 64): return launch_fwd<32, 64>(a, (int)nvox, st);
    case PAIR(32, 96): return launch_fwd<32, 96>(a, (int)nvox, st);
    case PAIR(48, 16): return launch_fwd<48, 16>(a, (int)nvox, st);
    case PAIR(64, 32): return launch_fwd<64, 32>(a, (int)nvox, st);
    case PAIR(64, 64): return launch_fwd<64, 64>(a, (int)nvox, st);
    case PAIR(64, 128): return launch_fwd<64, 128>(a, (int)nvox, st);
    case PAIR(96, 32): return launch_fwd<96, 32>(a, (int)nvox, st);
    case PAIR(128, 64): return launch_fwd<128, 64>(a, (int)nvox, st);
    default: return 1;
    }
}

extern "C" int unet_conv3d_wgrad(const void *x, int xcs, int xc0, const void *dy, int dcs, int dc0, float *dw,
                                 int n0, int n1, int n2, int cin, int cout, long long spin_limit, int *err,
                                 void *stream)
{
    long long nvox = (long long)n0 * n1 * n2;
    if (!x || !dy || !dw || !err || nvox <= 0 || nvox % 128 || (xcs | xc0 | dcs | dc0) % 8 || xc0 + cin > xcs ||
        dc0 + cout > dcs)
        return 1;
    WgradArgs a{(const __nv_bfloat16 *)x, xcs, xc0, (const __nv_bfloat16 *)dy, dcs, dc0, dw, n0, n1, n2, 1,
                spin_limit, err};
    cudaStream_t st = (cudaStream_t)stream;
    switch (PAIR(cin, cout)) {
    case PAIR(16, 16): return launch_wgrad<16, 16>(a, (int)nvox, st);
    case PAIR(16, 32): return launch_wgrad<16, 32>(a, (int)nvox, st);
    case PAIR(32, 32): return launch_wgrad<32, 32>(a, (int)nvox, st);
    case PAIR(32, 64): return launch_wgrad<32, 64>(a, (int)nvox, st);
    case PAIR(48, 16): return launch_wgrad<48, 16>(a, (int)nvox, st);
    case PAIR(64, 64): return launch_wgrad<64, 64>(a, (int)nvox, st);
    case PAIR(96, 32): return launch_wgrad<96, 32>(a, (int)nvox, st);
    case PAIR(128, 64): return launch_wgrad<128, 64>(a, (int)nvox, st);
    default: return 1;
    }
}
