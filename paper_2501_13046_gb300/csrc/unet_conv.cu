// unet_conv.cu -- implicit-GEMM 3x3x3 convolutions with circular padding on tcgen05.
//
// Tensors are NDHWC BF16 (a voxel's channels contiguous); a tensor may be a channel slice
// [c0, c0 + C) of a buffer with cs channels per voxel, which makes channel concatenation free.
// Weights: FP32 master [27 taps][Cout][Cin] (tap = (dz+1)*9 + (dy+1)*3 + (dx+1)), packed to
// BF16 in the same order for the forward pass.
//
// Forward / input gradient: volumes that tile by 8 x 16 x 2 voxels (with the input block and all
// weights in shared memory) take the block-tile kernel k_conv3d_blk (below); the others take the
// per-tap kernel k_conv3d_taps: one CTA = 128 consecutive output voxels x all Cout; for each of
// the 27 taps the shifted input rows (128 x Cin, wrapped) and the tap's weights (Cout x Cin) are
// staged in shared memory in the canonical K-major core-matrix layout and thread 0 issues Cin/16
// MMAs (M = 128, N = Cout, K = 16) accumulating in TMEM; buffers are double-buffered and recycled
// when the tap's commit arrives.  Epilogue: TMEM -> registers, + bias, ReLU, BF16, store.  Grids
// with few tiles split the taps over groups of CTAs that write FP32 partials, added in order by
// k_conv3d_finish.  The input gradient of a convolution is the convolution of the output gradient
// with the tap-flipped, transposed weights, so it reuses these kernels.
//
// Weight gradient (k_conv3d_wgrad_tc): dW[t][co][ci] = sum_v dY[v][co] X[v + t][ci] as a GEMM
// with M = 128 rows of (tap, ci), N = Cout, K = voxels; each CTA reduces one chunk of voxels in
// TMEM and adds its partial into FP32 dW with atomics (split-K).
#include <algorithm>

#include "unet_tc.cuh"

namespace unet {

constexpr int kTile = 128;
constexpr long long kDrain = 1LL << 26;   // polls allowed for MMAs in flight after a failed wait

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

// Piece idx of a (rows x CH chunks) operand: groups of 8 consecutive pieces are 8 consecutive rows
// of one 16-byte chunk, so the 8 lanes of a quarter warp store to 8 different 16-byte slots of one
// 128-byte core-matrix row (no bank conflict in the non-swizzled K-major layout, where the chunks
// of a row lie 128 bytes apart), and a warp reads 64 contiguous bytes of each of 8 rows.
template <int CH>
__device__ __forceinline__ void piece_rc(int idx, int &r, int &c)
{
    r = (idx & 7) + ((idx / (8 * CH)) << 3);
    c = (idx >> 3) % CH;
}

// The operands one thread stages for every tap of its 128-voxel M-tile at v0: A rows (the input
// shifted by the tap, wrapped) and the tap's weights, pieces mapped by piece_rc.  The rows' voxel
// coordinates are computed once (a tap only shifts and wraps them; packed 10 bits per axis, so
// every side is below 1024).  load() puts all of a tap's pieces in flight at once (registers),
// store() writes them into shared memory in the canonical K-major core-matrix layout; the kernel
// issues the next tap's load() right after the current tap's MMAs, before it waits for a buffer.
template <int CIN, int COUT>
struct TapStage {
    static constexpr int CH = CIN / 8, AIT = kTile * CH / 128, BIT = (COUT * CH + 127) / 128;
    static constexpr uint32_t SBO = (CIN / 8) * 128;
    int cijk[AIT];
    uint4 av[AIT], bv[BIT];

    __device__ __forceinline__ void init(const ConvArgs &a, int v0, int tid)
    {
        const int nx = a.n0, ny = a.n1;
#pragma unroll
        for (int it = 0; it < AIT; ++it) {
            int r, c;
            piece_rc<CH>(tid + it * 128, r, c);
            const int v = v0 + r;
            cijk[it] = (v % nx) | (((v / nx) % ny) << 10) | ((v / (nx * ny)) << 20);
        }
    }

    __device__ __forceinline__ void load(const ConvArgs &a, int tap, int tid)
    {
        const int nx = a.n0, ny = a.n1, nz = a.n2;
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
#pragma unroll
        for (int it = 0; it < AIT; ++it) {
            int r, c;
            piece_rc<CH>(tid + it * 128, r, c);
            int i = (cijk[it] & 1023) + dx, j = ((cijk[it] >> 10) & 1023) + dy, k = (cijk[it] >> 20) + dz;
            i += i < 0 ? nx : (i >= nx ? -nx : 0);
            j += j < 0 ? ny : (j >= ny ? -ny : 0);
            k += k < 0 ? nz : (k >= nz ? -nz : 0);
            const size_t nb = (size_t)i + (size_t)nx * (j + (size_t)ny * k);
            av[it] = *reinterpret_cast<const uint4 *>(a.x + nb * a.xcs + a.xc0 + c * 8);
        }
        const __nv_bfloat16 *wt = a.w + (size_t)tap * COUT * CIN;
#pragma unroll
        for (int it = 0; it < BIT; ++it) {
            const int idx = tid + it * 128;
            int r, c;
            piece_rc<CH>(idx, r, c);
            if (idx < COUT * CH) bv[it] = *reinterpret_cast<const uint4 *>(wt + r * CIN + c * 8);
        }
    }

    __device__ __forceinline__ void store(unsigned char *A, unsigned char *B, int tid) const
    {
#pragma unroll
        for (int it = 0; it < AIT; ++it) {
            int r, c;
            piece_rc<CH>(tid + it * 128, r, c);
            *reinterpret_cast<uint4 *>(A + (r >> 3) * SBO + c * 128 + (r & 7) * 16) = av[it];
        }
#pragma unroll
        for (int it = 0; it < BIT; ++it) {
            const int idx = tid + it * 128;
            int r, c;
            piece_rc<CH>(idx, r, c);
            if (idx < COUT * CH) *reinterpret_cast<uint4 *>(B + (r >> 3) * SBO + c * 128 + (r & 7) * 16) = bv[it];
        }
    }
};

template <int CIN, int COUT>
__host__ __device__ constexpr size_t taps_smem_bytes() { return 2 * (size_t)(kTile + COUT) * CIN * 2; }

// Per-tap kernel (k_conv3d_taps): one CTA = 128 consecutive output voxels x all Cout over the taps
// [t0, t1) of its group (blockIdx.y; one group of all 27 taps when unsplit).  Two shared-memory
// buffers; thread 0 issues Cin/16 MMAs per tap (M = 128, N = Cout, K = 16, FP32 accumulation in
// TMEM) and a buffer is refilled once the commit of its previous tap has arrived.  Epilogue:
// part == NULL: + bias, ReLU, BF16 store into the output slice; else the group's FP32 partial
// sums to part[group][voxel][Cout] (k_conv3d_finish adds the groups).
template <int CIN, int COUT>
__global__ void __launch_bounds__(128) k_conv3d_taps(ConvArgs a, int taps_per_group, float *__restrict__ part)
{
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && COUT <= 128, "channel counts");
    constexpr int NCOLS = COUT <= 32 ? 32 : (COUT <= 64 ? 64 : 128);
    constexpr uint32_t A_BYTES = kTile * CIN * 2, B_BYTES = COUT * CIN * 2;
    constexpr uint32_t SBO = (CIN / 8) * 128;
    constexpr uint32_t IDESC = idesc_bf16(kTile, COUT);
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Abuf = smem;
    unsigned char *Bbuf = smem + 2 * A_BYTES;
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int v0 = blockIdx.x * kTile;
    const int t0 = blockIdx.y * taps_per_group, t1 = min(27, t0 + taps_per_group), nt = t1 - t0;
    if (warp == 0) tmem_alloc(&tmem_slot, NCOLS);
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
    }
    TapStage<CIN, COUT> stage;
    stage.init(a, v0, tid);
    stage.load(a, t0, tid);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;
    int issued = 0;
    for (int s = 0; s < nt; ++s) {
        const int buf = s & 1;
        if (s >= 2) {   // the MMAs of tap s - 2 have finished reading this buffer
            if (tid == 0 && !failed && !mbar_wait_bounded(&mbar[buf], ((s - 2) >> 1) & 1, a.spin_limit)) failed = 1;
            __syncthreads();
            if (failed) break;
        }
        unsigned char *A = Abuf + buf * A_BYTES;
        unsigned char *B = Bbuf + buf * B_BYTES;
        stage.store(A, B, tid);
        fence_proxy_async();
        fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            fence_after_sync();
            const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
#pragma unroll
            for (int kk = 0; kk < CIN / 16; ++kk)
                mma_bf16(tmem, smem_desc(a0 + kk * 256, 128, SBO), smem_desc(b0 + kk * 256, 128, SBO), IDESC,
                         (s > 0 || kk > 0) ? 1u : 0u);
            mma_commit(&mbar[buf]);
        }
        ++issued;
        if (s + 1 < nt) stage.load(a, t0 + s + 1, tid);   // in flight during the next buffer wait
    }
    // the last issued tap's commit; the MMAs complete in order.  After a failed wait the drain gets
    // a floor (kDrain polls) so that no MMA still reads shared memory when the CTA exits.
    if (tid == 0 && issued > 0) {
        const int last = issued - 1;
        bool ok = !failed && mbar_wait_bounded(&mbar[last & 1], (last >> 1) & 1, a.spin_limit);
        if (!ok) {
            failed = 1;
            mbar_wait_bounded(&mbar[last & 1], (last >> 1) & 1, a.spin_limit > kDrain ? a.spin_limit : kDrain);
        }
    }
    __syncthreads();
    fence_after_sync();
    if (!failed && issued > 0) {
        const int row = warp * 32 + lane;
        const size_t v = (size_t)v0 + row;
#pragma unroll
        for (int cc = 0; cc < COUT / 16; ++cc) {
            float acc[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + cc * 16, acc);
            if (part) {
                float *dst = part + ((size_t)blockIdx.y * a.n0 * a.n1 * a.n2 + v) * COUT + cc * 16;
#pragma unroll
                for (int q = 0; q < 16; q += 4)
                    *reinterpret_cast<float4 *>(dst + q) = make_float4(acc[q], acc[q + 1], acc[q + 2], acc[q + 3]);
            } else {
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
        }
    } else if (failed && tid == 0) {
        atomicExch(a.err, 1);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

// Forward / input gradient on a block tile (k_conv3d_blk): one CTA = 8 (x) x 16 (y) x ZT (z)
// output voxels, i.e. ZT M-tiles of 128 rows (row r: x = x0 + (r & 7), y = y0 + (r >> 3)).  The
// CTA loads its input block with a one-voxel halo (wrapped) into shared memory once, in three
// copies shifted by dx = -1, 0, +1: copy s holds, for every 8-channel chunk, z and y of the
// halo'd block, the 8 voxels x0 + s - 1 .. x0 + s + 6 as one 128-byte row (a core matrix of the
// K-major layout: 8 rows of 16 bytes).  For a tap (dx, dy, dz) the A operand of an M-tile is copy
// dx + 1 seen through a descriptor that starts dy + 1 rows and zt + dz + 1 planes in: the next y
// is the next 128-byte row (stride between 8-row groups), the next channel chunk is one chunk
// plane further (stride between K-adjacent core matrices).  Every core matrix stays 128-byte
// aligned and no data moves per tap: thread 0 issues all 27 x CIN/16 MMAs of every M-tile back
// to back into TMEM, with all 27 taps' weights resident, and one commit ends the CTA's work.
constexpr int kBlkX = 8, kBlkY = 16;
constexpr int kBlkThreads = 256;   // 8 warps: staging in parallel, the epilogue's M-tiles split by warp quad

template <int CIN, int COUT, int ZT>
__host__ __device__ constexpr size_t blk_in_bytes() { return (size_t)3 * (CIN / 8) * (kBlkY + 2) * (ZT + 2) * 128; }
template <int CIN, int COUT, int ZT>
__host__ __device__ constexpr size_t blk_smem_bytes() { return blk_in_bytes<CIN, COUT, ZT>() + (size_t)27 * COUT * CIN * 2; }

template <int CIN, int COUT, int ZT>
__global__ void __launch_bounds__(kBlkThreads) k_conv3d_blk(ConvArgs a)
{
    static_assert(CIN % 16 == 0 && COUT % 16 == 0 && ZT * COUT <= 256, "channel counts");
    constexpr int CH = CIN / 8;
    constexpr int BX = kBlkX + 2, BY = kBlkY + 2, BZ = ZT + 2;
    constexpr uint32_t PLANE = BY * 128;             // one z plane of one chunk of one copy
    constexpr uint32_t CHUNK = BZ * PLANE;           // one chunk of one copy (K-adjacent core matrices)
    constexpr uint32_t COPY = CH * CHUNK;            // one shifted copy
    constexpr uint32_t W_TAP = COUT * CIN * 2;       // bytes of one tap's weights
    constexpr uint32_t SBO_B = (CIN / 8) * 128;
    constexpr int NCOLS = ZT * COUT <= 32 ? 32 : (ZT * COUT <= 64 ? 64 : (ZT * COUT <= 128 ? 128 : 256));
    constexpr uint32_t IDESC = idesc_bf16(kTile, COUT);
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *In = smem;
    unsigned char *Wt = smem + blk_in_bytes<CIN, COUT, ZT>();
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    __shared__ int failed;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nx = a.n0, ny = a.n1, nz = a.n2;
    const int ntx = nx / kBlkX, nty = ny / kBlkY;
    int b = blockIdx.x;
    const int x0 = (b % ntx) * kBlkX;
    b /= ntx;
    const int y0 = (b % nty) * kBlkY;
    const int z0 = (b / nty) * ZT;
    if (warp == 0) tmem_alloc(&tmem_slot, NCOLS);
    if (tid == 0) {
        mbar_init(&mbar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        failed = 0;
    }
    // halo'd input block: one global load per (voxel, chunk), chunks fastest (coalesced), stored
    // into every shifted copy that contains the voxel (block x = bx is row position bx - s of copy s)
    // (batches of kBatch pieces per thread: all loads of a batch in flight before its stores)
    constexpr int kBatch = 8;
    constexpr int IN_TOT = BX * BY * BZ * CH, IN_IT = (IN_TOT + kBlkThreads - 1) / kBlkThreads;
    for (int i0 = 0; i0 < IN_IT; i0 += kBatch) {
        uint4 val[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int idx = tid + (i0 + u) * kBlkThreads;
            if (i0 + u < IN_IT && idx < IN_TOT) {
                const int bx = idx % BX, rest = idx / BX, c = rest % CH, row = rest / CH, by = row % BY, bz = row / BY;
                const int nb = wrapi(x0 - 1 + bx, nx) + nx * (wrapi(y0 - 1 + by, ny) + ny * wrapi(z0 - 1 + bz, nz));
                val[u] = *reinterpret_cast<const uint4 *>(a.x + (size_t)nb * a.xcs + a.xc0 + c * 8);
            }
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int idx = tid + (i0 + u) * kBlkThreads;
            if (i0 + u < IN_IT && idx < IN_TOT) {
                const int bx = idx % BX, rest = idx / BX, c = rest % CH, row = rest / CH, by = row % BY, bz = row / BY;
#pragma unroll
                for (int sft = 0; sft < 3; ++sft) {
                    const int xr = bx - sft;
                    if (xr >= 0 && xr < kBlkX)
                        *reinterpret_cast<uint4 *>(In + sft * COPY + c * CHUNK + bz * PLANE + by * 128 + xr * 16) = val[u];
                }
            }
        }
    }
    // weights of the 27 taps, each in the K-major core-matrix layout of the B operand
    constexpr int W_TOT = 27 * COUT * CH, W_IT = (W_TOT + kBlkThreads - 1) / kBlkThreads;
    for (int i0 = 0; i0 < W_IT; i0 += kBatch) {
        uint4 val[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int idx = tid + (i0 + u) * kBlkThreads;
            if (i0 + u < W_IT && idx < W_TOT) {
                const int t = idx / (COUT * CH);
                int r, c;
                piece_rc<CH>(idx - t * (COUT * CH), r, c);
                val[u] = *reinterpret_cast<const uint4 *>(a.w + ((size_t)t * COUT + r) * CIN + c * 8);
            }
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int idx = tid + (i0 + u) * kBlkThreads;
            if (i0 + u < W_IT && idx < W_TOT) {
                const int t = idx / (COUT * CH);
                int r, c;
                piece_rc<CH>(idx - t * (COUT * CH), r, c);
                *reinterpret_cast<uint4 *>(Wt + t * W_TAP + (r >> 3) * SBO_B + c * 128 + (r & 7) * 16) = val[u];
            }
        }
    }
    fence_proxy_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;
    if (tid == 0) {
        // every MMA's descriptors are the block's base descriptors plus a compile-time offset (in
        // 16-byte units of the start-address field; the block lies below 256 KB, so no carry)
        const uint64_t da = smem_desc(smem_u32(In), CHUNK, 128), db = smem_desc(smem_u32(Wt), 128, SBO_B);
#pragma unroll
        for (int zt = 0; zt < ZT; ++zt)
#pragma unroll
            for (int tap = 0; tap < 27; ++tap) {
                const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                const uint32_t ab = (uint32_t)(dx + 1) * COPY + (uint32_t)(zt + dz + 1) * PLANE + (uint32_t)(dy + 1) * 128;
#pragma unroll
                for (int kk = 0; kk < CIN / 16; ++kk)
                    mma_bf16(tmem + zt * COUT, da + ((ab + kk * 2 * CHUNK) >> 4), db + ((tap * W_TAP + kk * 256) >> 4),
                             IDESC, (tap > 0 || kk > 0) ? 1u : 0u);
            }
        mma_commit(&mbar);
        if (!mbar_wait_bounded(&mbar, 0, a.spin_limit)) {
            failed = 1;
            mbar_wait_bounded(&mbar, 0, a.spin_limit > kDrain ? a.spin_limit : kDrain);   // before smem goes away
        }
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (!failed) {   // warp w reads TMEM lanes 32 (w % 4) ..: M-tile zt = w / 4, w / 4 + 2, ...
        const int row = (warp & 3) * 32 + lane;
        for (int zt = warp >> 2; zt < ZT; zt += kBlkThreads / 128) {
            const size_t v = (size_t)(x0 + (row & 7)) + (size_t)nx * ((y0 + (row >> 3)) + (size_t)ny * (z0 + zt));
#pragma unroll
            for (int cc = 0; cc < COUT / 16; ++cc) {
                float acc[16];
                tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + zt * COUT + cc * 16, acc);
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
        }
    } else if (tid == 0) {
        atomicExch(a.err, 1);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, NCOLS);
}

// y = act(sum over groups of part + bias), BF16, 8 output channels per thread.
template <int COUT>
__global__ void __launch_bounds__(256) k_conv3d_finish(ConvArgs a, int groups, const float *__restrict__ part)
{
    const long long nvox = (long long)a.n0 * a.n1 * a.n2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nvox * (COUT / 8);
         e += (long long)gridDim.x * blockDim.x) {
        const long long v = e / (COUT / 8);
        const int c0 = (int)(e - v * (COUT / 8)) * 8;
        float t[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) t[q] = a.bias ? a.bias[c0 + q] : 0.f;
        for (int g = 0; g < groups; ++g) {
            const float *pp = part + ((size_t)g * nvox + v) * COUT + c0;
            const float4 lo = *reinterpret_cast<const float4 *>(pp), hi = *reinterpret_cast<const float4 *>(pp + 4);
            t[0] += lo.x; t[1] += lo.y; t[2] += lo.z; t[3] += lo.w;
            t[4] += hi.x; t[5] += hi.y; t[6] += hi.z; t[7] += hi.w;
        }
        __align__(16) __nv_bfloat16 o[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) o[q] = __float2bfloat16_rn(a.relu ? fmaxf(t[q], 0.f) : t[q]);
        *reinterpret_cast<uint4 *>(a.y + v * a.ycs + a.yc0 + c0) = *reinterpret_cast<uint4 *>(o);
    }
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
        // (batches of 8 pieces per thread: all loads of a batch in flight before its stores)
        constexpr int A_IT = TPG * KV * (CIN / 8) / 128;
        const int a_tot = ntap * KV * (CIN / 8);
        for (int i0 = 0; i0 < A_IT; i0 += 8) {
            uint4 val[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = tid + (i0 + u) * 128;
                if (i0 + u < A_IT && idx < a_tot) {
                    const int c = idx % (CIN / 8), kv = (idx / (CIN / 8)) % KV, tl = idx / ((CIN / 8) * KV);
                    const int tap = tap0 + tl;
                    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                    const int v = vbase + kv;
                    const int i = v % nx, j = (v / nx) % ny, k = v / (nx * ny);
                    const int nb = wrapi(i + dx, nx) + nx * (wrapi(j + dy, ny) + ny * wrapi(k + dz, nz));
                    val[u] = *reinterpret_cast<const uint4 *>(a.x + (size_t)nb * a.xcs + a.xc0 + c * 8);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = tid + (i0 + u) * 128;
                if (i0 + u < A_IT && idx < a_tot) {
                    const int c = idx % (CIN / 8), kv = (idx / (CIN / 8)) % KV, tl = idx / ((CIN / 8) * KV);
                    const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&val[u]);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int r = tl * CIN + c * 8 + q;
                        *reinterpret_cast<__nv_bfloat16 *>(A + (r >> 3) * SBO + (kv >> 3) * 128 + (r & 7) * 16 +
                                                           (kv & 7) * 2) = e[q];
                    }
                }
            }
        }
        constexpr int B_IT = (KV * (COUT / 8) + 127) / 128;
        for (int i0 = 0; i0 < B_IT; i0 += 8) {
            uint4 val[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = tid + (i0 + u) * 128;
                if (i0 + u < B_IT && idx < KV * (COUT / 8)) {
                    const int c = idx % (COUT / 8), kv = idx / (COUT / 8);
                    val[u] = *reinterpret_cast<const uint4 *>(a.dy + (size_t)(vbase + kv) * a.dcs + a.dc0 + c * 8);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = tid + (i0 + u) * 128;
                if (i0 + u < B_IT && idx < KV * (COUT / 8)) {
                    const int c = idx % (COUT / 8), kv = idx / (COUT / 8);
                    const __nv_bfloat16 *e = reinterpret_cast<const __nv_bfloat16 *>(&val[u]);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int r = c * 8 + q;
                        *reinterpret_cast<__nv_bfloat16 *>(B + (r >> 3) * SBO + (kv >> 3) * 128 + (r & 7) * 16 +
                                                           (kv & 7) * 2) = e[q];
                    }
                }
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
        if (!ok) {   // the drain gets a floor (kDrain polls): no MMA may still read shared memory at exit
            failed = 1;
            mbar_wait_bounded(&mbar[last & 1], (last >> 1) & 1, a.spin_limit > kDrain ? a.spin_limit : kDrain);
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

constexpr int kSms = 152;

// Split-K plan of a per-tap forward convolution: taps per group and number of groups (1: no
// split).  The taps are split where the grid has fewer than four 128-voxel tiles per SM, into
// enough groups for about four CTAs per SM in all.
struct SplitPlan {
    int tpg, groups;
};

SplitPlan split_plan(long long nvox)
{
    const long long tiles = nvox / kTile;
    if (tiles <= 0 || tiles >= 4 * kSms) return {27, 1};
    const int want = (int)std::min<long long>(27, (4 * kSms + tiles - 1) / tiles);
    const int tpg = (27 + want - 1) / want;
    return {tpg, (27 + tpg - 1) / tpg};
}

template <int CIN, int COUT>
int launch_fwd(const ConvArgs &a, int nvox, float *ws, cudaStream_t st)
{
    // block-tile kernel where the grid tiles evenly and the block and all weights fit in shared
    // memory: it reads each input voxel about 3 times (halo), the per-tap kernel 27 times (L2)
    constexpr int ZT = 2;
    constexpr size_t bsm = blk_smem_bytes<CIN, COUT, ZT>();
    if constexpr (bsm <= 220 * 1024) {
        if (a.n0 % kBlkX == 0 && a.n1 % kBlkY == 0 && a.n2 % ZT == 0) {
            static bool attr_blk = false;
            if (!attr_blk) {
                if (cudaFuncSetAttribute(k_conv3d_blk<CIN, COUT, ZT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bsm) != cudaSuccess)
                    return 3;
                attr_blk = true;
            }
            const int grid = (a.n0 / kBlkX) * (a.n1 / kBlkY) * (a.n2 / ZT);
            k_conv3d_blk<CIN, COUT, ZT><<<grid, kBlkThreads, bsm, st>>>(a);
            return cudaGetLastError() == cudaSuccess ? 0 : 3;
        }
    }
    constexpr size_t smem = taps_smem_bytes<CIN, COUT>();
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_conv3d_taps<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return 3;
        attr = true;
    }
    const int tiles = nvox / kTile;
    const SplitPlan sp = split_plan(nvox);
    if (ws && sp.groups > 1) {   // few tiles: the taps in groups, FP32 partials added in order
        k_conv3d_taps<CIN, COUT><<<dim3(tiles, sp.groups), 128, smem, st>>>(a, sp.tpg, ws);
        const long long work = (long long)nvox * (COUT / 8);
        k_conv3d_finish<COUT><<<(int)std::min<long long>((work + 255) / 256, 152LL * 16), 256, 0, st>>>(a, sp.groups, ws);
        return cudaGetLastError() == cudaSuccess ? 0 : 3;
    }
    k_conv3d_taps<CIN, COUT><<<tiles, 128, smem, st>>>(a, 27, nullptr);
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

extern "C" size_t unet_conv3d_fwd_workspace(int n0, int n1, int n2, int cout)
{
    const long long nvox = (long long)n0 * n1 * n2;
    if (n0 <= 0 || n1 <= 0 || n2 <= 0 || cout <= 0 || nvox % kTile) return 0;
    const SplitPlan sp = split_plan(nvox);
    return sp.groups > 1 ? (size_t)sp.groups * (size_t)nvox * (size_t)cout * sizeof(float) : 0;
}

extern "C" int unet_conv3d_fwd(const void *x, int xcs, int xc0, const void *w_bf16, const float *bias, void *y,
                               int ycs, int yc0, int n0, int n1, int n2, int cin, int cout, int relu, float *ws,
                               size_t ws_bytes, long long spin_limit, int *err, void *stream)
{
    long long nvox = (long long)n0 * n1 * n2;
    if (!x || !w_bf16 || !y || !err || nvox <= 0 || nvox % kTile || (xcs | xc0 | ycs | yc0) % 8 ||
        xc0 + cin > xcs || yc0 + cout > ycs || n0 >= 1024 || n1 >= 1024 || n2 >= 1024)
        return 1;
    if (ws && (ws_bytes < unet_conv3d_fwd_workspace(n0, n1, n2, cout) || (reinterpret_cast<size_t>(ws) & 15)))
        return 1;
    ConvArgs a{(const __nv_bfloat16 *)x, xcs, xc0, (const __nv_bfloat16 *)w_bf16, bias, (__nv_bfloat16 *)y,
               ycs, yc0, n0, n1, n2, relu, spin_limit, err};
    cudaStream_t st = (cudaStream_t)stream;
    switch (PAIR(cin, cout)) {
    case PAIR(16, 16): return launch_fwd<16, 16>(a, (int)nvox, ws, st);
    case PAIR(16, 32): return launch_fwd<16, 32>(a, (int)nvox, ws, st);
    case PAIR(16, 48): return launch_fwd<16, 48>(a, (int)nvox, ws, st);
    case PAIR(32, 16): return launch_fwd<32, 16>(a, (int)nvox, ws, st);
    case PAIR(32, 32): return launch_fwd<32, 32>(a, (int)nvox, ws, st);
    case PAIR(32, 64): return launch_fwd<32, 64>(a, (int)nvox, ws, st);
    case PAIR(32, 96): return launch_fwd<32, 96>(a, (int)nvox, ws, st);
    case PAIR(48, 16): return launch_fwd<48, 16>(a, (int)nvox, ws, st);
    case PAIR(64, 32): return launch_fwd<64, 32>(a, (int)nvox, ws, st);
    case PAIR(64, 64): return launch_fwd<64, 64>(a, (int)nvox, ws, st);
    case PAIR(64, 128): return launch_fwd<64, 128>(a, (int)nvox, ws, st);
    case PAIR(96, 32): return launch_fwd<96, 32>(a, (int)nvox, ws, st);
    case PAIR(128, 64): return launch_fwd<128, 64>(a, (int)nvox, ws, st);
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
