// mg_tile.cuh -- shared-memory tiled red-black colour pass for colour-split levels.
//
// A CTA owns a tile of 32 colour pairs (64 cells) in x by 8 rows in y and marches through a
// chunk of z planes.  Each plane of the 4 correction fields (both colour halves, the tile plus
// its stencil halo) is brought into a ring of shared-memory slots by two TMA tensor loads
// (cp.async.bulk.tensor, one per colour half) completing on an mbarrier; the stencil of
// apply_J then reads only shared memory.  Halo cells outside the box (periodic wrap, or the
// Robin 1/r ghost value v(clamp(g)) |x_clamp| / |x_g|) are not addressable by the tensor
// load, which fills them with zeros: the CTA fetches them with plain loads one plane ahead and
// writes them over the zero fill once the plane's TMA has completed.  The arithmetic per cell
// is that of k_smooth_colour (same operator, same update, same Jacobi-within-colour reads), so
// both kernels compute the same iterate up to FP rounding order.
//
// Requirements (checked on the host): colour-split level, nx and ny multiples of 8 and >= 16,
// nz >= 8, so every TMA x coordinate and stride is 16-byte aligned and no tile row is both
// the first and the last of the box.
#pragma once
#include <cuda.h>

#include "mg_kernels.cuh"

namespace ctt {

constexpr int kTileP = 32;                      // colour pairs per tile row (64 cells)
constexpr int kTileY = 8;                       // rows per tile, one warp each
constexpr int kTilePad = 4;                     // pairs loaded left of the tile: 16-byte aligned x
constexpr int kTileW = kTileP + 2 * kTilePad;   // pairs per loaded row (40)
constexpr int kTileThreads = kTileP * kTileY;   // 256
constexpr int kTileFix = 3;                     // halo fix-up elements per thread and plane
constexpr long long kTileDrain = 1LL << 26;     // polls allowed for in-flight loads after a failed wait

template <int ORDER> __host__ __device__ constexpr int tile_rows() { return kTileY + ORDER; }   // 8 + 2 halo
template <int ORDER> __host__ __device__ constexpr int tile_slots() { return ORDER + 2; }      // 2H+1 + 1
template <int ORDER> __host__ __device__ constexpr int tile_field_elems() { return tile_rows<ORDER>() * kTileW; }
template <int ORDER> __host__ __device__ constexpr int tile_half_elems() { return 4 * tile_field_elems<ORDER>(); }
template <int ORDER> __host__ __device__ constexpr int tile_slot_elems() { return 2 * tile_half_elems<ORDER>(); }
template <typename T, int ORDER> __host__ __device__ constexpr size_t tile_smem_bytes()
{
    return (size_t)tile_slots<ORDER>() * tile_slot_elems<ORDER>() * sizeof(T) + 8 * tile_slots<ORDER>();
}

struct TileGrid {
    int ntx, nty;   // tiles along x (pairs) and y (rows)
    int zc;         // planes per CTA
};

// ---------------------------------------------------------------- TMA / mbarrier (inline PTX)
__device__ __forceinline__ uint32_t sm_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tile_mbar_init(uint64_t *mb, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(sm_addr(mb)), "r"(count) : "memory");
}

__device__ __forceinline__ void tile_mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tile_mbar_arrive(uint64_t *mb)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(sm_addr(mb)) : "memory");
}

__device__ __forceinline__ void tile_mbar_expect_tx(uint64_t *mb, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sm_addr(mb)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool tile_mbar_try_wait(uint64_t *mb, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(sm_addr(mb)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool tile_mbar_wait(uint64_t *mb, uint32_t parity, long long limit)
{
    for (long long i = 0; i < limit; ++i)
        if (tile_mbar_try_wait(mb, parity)) return true;
    return false;
}

// generic-proxy accesses of shared memory are ordered before later async-proxy (TMA) writes
__device__ __forceinline__ void tile_fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 5-D tiled tensor load into shared memory, completing `bytes` on the mbarrier.
__device__ __forceinline__ void tile_tma_load(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                              int c4, uint64_t *mb)
{
    asm volatile(
        "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
        "%6}], [%7];" ::"r"(sm_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(sm_addr(mb))
        : "memory");
}

// ---------------------------------------------------------------- halo values
// Value of field f at the cell of colour h in pair P of row (y, z), coordinates unwrapped
// (at most one period outside the box).  Same colour as the pass: old value from X; other
// colour: current value from O.
template <typename T, int BC>
__device__ __forceinline__ T tile_fetch(const Geo &g, const T *X, const T *O, int colour, int P, int y, int z, int h,
                                        int f)
{
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int x = 2 * P + ((h + y + z) & 1);
    int xb = x, yb = y, zb = z;
    if (BC == BC_PERIODIC) {
        xb += xb < 0 ? nx : 0; xb -= xb >= nx ? nx : 0;
        yb += yb < 0 ? ny : 0; yb -= yb >= ny ? ny : 0;
        zb += zb < 0 ? nz : 0; zb -= zb >= nz ? nz : 0;
    } else {
        xb = min(max(xb, 0), nx - 1);
        yb = min(max(yb, 0), ny - 1);
        zb = min(max(zb, 0), nz - 1);
    }
    const int hb = (xb + yb + zb) & 1;
    const size_t N = (size_t)nx * ny * nz;
    const size_t idx = (size_t)f * N + (hb ? N / 2 : 0) + (size_t)(xb >> 1) + (size_t)(nx >> 1) * (yb + (size_t)ny * zb);
    T v = (hb == colour ? X : O)[idx];
    if (BC == BC_ROBIN && (xb != x || yb != y || zb != z)) {
        double ax = cellx(g, 0, xb), ay = cellx(g, 1, yb), az = cellx(g, 2, zb);
        double gx = cellx(g, 0, x), gy = cellx(g, 1, y), gz = cellx(g, 2, z);
        v = (T)((double)v * sqrt(ax * ax + ay * ay + az * az) / sqrt(gx * gx + gy * gy + gz * gz));
    }
    return v;
}

// Shared-memory accessor of one field around the active cell: ob[dz + H] is the cell's offset in
// the same-colour half of plane z + dz; oh moves to the other colour half; pa is the x parity
// of the active cells of this row (a neighbour at odd dx sits in pair m + pa + (dx-1)/2).
template <typename T, int ORDER>
struct AccT {
    const T *sm;
    const int *ob;
    int oh, pa;
    int fo;   // field offset, F * tile_field_elems
    __device__ __forceinline__ T operator()(int dx, int dy, int dz) const
    {
        int o = ob[dz + ORDER / 2] + fo + dy * kTileW;
        if ((dx + dy + dz) & 1) o += oh;
        o += (dx & 1) ? pa + ((dx - 1) >> 1) : (dx >> 1);
        return sm[o];
    }
};

template <typename T, int ORDER, int BC>
__global__ void __launch_bounds__(kTileThreads, sizeof(T) == 4 ? 2 : 1)
    k_smooth_tile(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmO, Geo g,
                  Coef<T> cf, const T *__restrict__ X, const T *__restrict__ O, T *__restrict__ Y,
                  const T *__restrict__ f, const T *__restrict__ ab, int colour, TileGrid tg,
                  unsigned int *__restrict__ err, long long spin)
{
    constexpr int H = ORDER / 2, RY = tile_rows<ORDER>(), S = tile_slots<ORDER>();
    constexpr int FE = tile_field_elems<ORDER>(), HE = tile_half_elems<ORDER>(), SE = tile_slot_elems<ORDER>();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + (size_t)S * SE * sizeof(T));

    const int nx = g.n[0], ny = g.n[1], nz = g.n[2], nxh = nx >> 1;
    const unsigned N = (unsigned)nx * ny * nz, Nh = N >> 1;
    int b = blockIdx.x;
    const int tx = b % tg.ntx;
    b /= tg.ntx;
    const int ty = b % tg.nty;
    const int tz = b / tg.nty;
    const int P0 = tx * kTileP, y0 = ty * kTileY, z0 = tz * tg.zc;
    const int z1 = min(z0 + tg.zc, nz);
    if (z0 >= z1) return;
    const int tpt = min(kTileP, nxh - P0);   // pairs in this tile
    const int zs = z0 - H;                   // first loaded plane; plane p (relative) is zs + p
    const int NP = (z1 - z0) + 2 * H;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;

    auto ghost_plane = [&](int p) { return BC == BC_ROBIN && (zs + p < 0 || zs + p >= nz); };
    auto issue = [&](int p) {   // one thread: start the loads of relative plane p
        uint64_t *mb = bar + p % S;
        if (ghost_plane(p)) { tile_mbar_arrive(mb); return; }   // filled by plain loads instead
        int z = zs + p;
        if (BC == BC_PERIODIC) { z += z < 0 ? nz : 0; z -= z >= nz ? nz : 0; }
        T *dst = sm + (p % S) * SE;
        tile_mbar_expect_tx(mb, (uint32_t)(2 * HE * sizeof(T)));
        tile_tma_load(dst + colour * HE, &tmX, P0 - kTilePad, y0 - H, z, 0, colour, mb);
        tile_tma_load(dst + (1 - colour) * HE, &tmO, P0 - kTilePad, y0 - H, z, 0, 1 - colour, mb);
    };

    // Halo elements the tensor load leaves zero: rows outside [0, ny) and pairs outside
    // [0, nxh), restricted to what the stencil reads (pairs P0-1 .. P0+tpt).
    const int npos = tpt + 2;
    const int top = y0 == 0 ? H : 0, bot = (y0 + kTileY >= ny) ? H : 0;
    const int ngr = top + bot;
    const int lcol = P0 == 0 ? 1 : 0, rcol = (P0 + tpt >= nxh) ? 1 : 0, ngc = lcol + rcol;
    const int nfix = (ngr * npos + (RY - ngr) * ngc) * 8;
    int fo[kTileFix], fP[kTileFix], fy[kTileFix], fh[kTileFix], ff[kTileFix];
#pragma unroll
    for (int i = 0; i < kTileFix; ++i) {
        int e = tid + i * kTileThreads;
        fo[i] = -1;
        if (e < nfix) {
            const int hf = e & 7, h = hf >> 2, fld = hf & 3;
            int rest = e >> 3, r, pos;
            if (rest < ngr * npos) {
                const int gr = rest / npos;
                pos = kTilePad - 1 + rest % npos;
                r = gr < top ? gr : RY - bot + (gr - top);
            } else {
                rest -= ngr * npos;
                const int c = rest % ngc;
                r = top + rest / ngc;
                pos = (c == 0 && lcol) ? kTilePad - 1 : kTilePad + tpt;
            }
            fo[i] = h * HE + fld * FE + r * kTileW + pos;
            fP[i] = P0 - kTilePad + pos;
            fy[i] = y0 - H + r;
            fh[i] = h;
            ff[i] = fld;
        }
    }
    // every element of a Robin ghost plane (no tensor load for it)
    auto fill_plane = [&](int p) {
        T *dst = sm + (p % S) * SE;
        const int tot = 8 * RY * npos;
        for (int e = tid; e < tot; e += kTileThreads) {
            const int hf = e & 7, h = hf >> 2, fld = hf & 3;
            const int rest = e >> 3, r = rest / npos, pos = kTilePad - 1 + rest % npos;
            dst[h * HE + fld * FE + r * kTileW + pos] =
                tile_fetch<T, BC>(g, X, O, colour, P0 - kTilePad + pos, y0 - H + r, zs + p, h, fld);
        }
    };
    auto load_fix = [&](int p, T (&v)[kTileFix]) {
#pragma unroll
        for (int i = 0; i < kTileFix; ++i)
            if (fo[i] >= 0) v[i] = tile_fetch<T, BC>(g, X, O, colour, fP[i], fy[i], zs + p, fh[i], ff[i]);
    };
    auto store_fix = [&](int p, const T (&v)[kTileFix]) {
        T *dst = sm + (p % S) * SE;
#pragma unroll
        for (int i = 0; i < kTileFix; ++i)
            if (fo[i] >= 0) dst[fo[i]] = v[i];
    };
    auto wait_plane = [&](int p) { return tile_mbar_wait(bar + p % S, (uint32_t)((p / S) & 1), spin); };

    if (tid < S) tile_mbar_init(bar + tid, 1);
    tile_mbar_init_fence();
    __syncthreads();
    const int pre = min(2 * H + 1, NP);
    if (tid == 0)
        for (int p = 0; p < pre; ++p) issue(p);
    // prologue: planes 0 .. 2H-1 completed here, plane 2H staged (its halo stored after its wait)
    bool ok = true;
    for (int p = 0; p < 2 * H && ok; ++p) {
        if (ghost_plane(p)) { fill_plane(p); continue; }
        ok = wait_plane(p);
        T v[kTileFix];
        load_fix(p, v);
        store_fix(p, v);
    }
    T cur[kTileFix], nxt[kTileFix];
    if (ghost_plane(2 * H)) fill_plane(2 * H);
    else load_fix(2 * H, cur);
    int done = -1;             // planes 0 .. done completed for the whole CTA
    int issued = pre - 1;      // planes 0 .. issued have loads in flight or completed
    bool failed = false;       // uniform across the CTA

    for (int z = z0; z < z1; ++z) {
        const int p = z - zs;   // relative index of the computed plane
        if (__syncthreads_or(!ok)) { failed = true; break; }   // (A) slot of plane p - H - 1 is free again
        done = p + H - 1;
        const int pn = p + H + 1;
        if (pn < NP) {
            if (tid == 0) {
                tile_fence_proxy_async();
                issue(pn);
            }
            issued = pn;
            if (ghost_plane(pn)) fill_plane(pn);
            else load_fix(pn, nxt);
        }
        const int y = y0 + w;
        const bool act = lane < tpt;
        const unsigned q = (colour ? Nh : 0u) + (unsigned)(P0 + lane) + (unsigned)nxh * ((unsigned)y + (unsigned)ny * z);
        T ca = 0, cb = 0, fq[4] = {0, 0, 0, 0};
        if (act) {
            ca = ab[q];
            cb = ab[N + q];
#pragma unroll
            for (int a = 0; a < 4; ++a) fq[a] = f[a * N + q];
        }
        ok = wait_plane(p + H);
        if (!ghost_plane(p + H)) store_fix(p + H, cur);
#pragma unroll
        for (int i = 0; i < kTileFix; ++i) cur[i] = nxt[i];
        if (__syncthreads_or(!ok)) { failed = true; break; }   // (B) plane p + H and its halo are in place
        if (act) {
            const int pa = (colour + y + z) & 1;
            int ob[2 * H + 1];
#pragma unroll
            for (int d = -H; d <= H; ++d)
                ob[d + H] = ((p + d) % S) * SE + colour * HE + (w + H) * kTileW + kTilePad + lane;
            const int oh = (1 - 2 * colour) * HE;
            AccT<T, ORDER> a0{sm, ob, oh, pa, 0}, a1{sm, ob, oh, pa, FE}, a2{sm, ob, oh, pa, 2 * FE},
                a3{sm, ob, oh, pa, 3 * FE};
            T Je[4], ctr[4];
            apply_J<ORDER, T>(a0, a1, a2, a3, ca, cb, cf, Je, ctr);
            Y[q] = ctr[0] + (fq[0] - Je[0]) / ((ca * cf.dl + cb) * cf.iom);
#pragma unroll
            for (int a = 0; a < 3; ++a) Y[(1 + a) * N + q] = ctr[1 + a] + (fq[1 + a] - Je[1 + a]) * cf.idW[a];
        }
    }
    if (failed) {
        if (tid == 0) atomicOr(err, 1u);
        // let the loads still in flight land before the CTA's shared memory is released (a
        // tensor load of an in-bounds box always completes; the bound only guards the poll)
        for (int p = done + 1; p <= issued; ++p)
            tile_mbar_wait(bar + p % S, (uint32_t)((p / S) & 1), spin > kTileDrain ? spin : kTileDrain);
    }
}

}  // namespace ctt
