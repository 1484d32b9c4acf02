// mg_tile.cuh -- shared-memory tiled kernels of the colour-split levels: the red-black colour
// pass of the smoother and the fused residual + restriction.
//
// A CTA owns a tile of 32 colour pairs (64 cells) in x by 8 rows in y and marches through a
// chunk of z planes.  Each plane of the 4 correction fields (both colour halves, the tile plus
// its stencil halo) is brought into a ring of shared-memory slots by two TMA tensor loads
// (cp.async.bulk.tensor, one per colour half) completing on an mbarrier; the stencils then read
// only shared memory.  Halo cells outside the box (periodic wrap, the Robin 1/r ghost value
// v(clamp(g)) |x_clamp| / |x_g|, or a mirror image across a symmetry plane with W's normal component
// negated) are not addressable by the tensor load, which fills them with
// zeros: the CTA fetches them with plain loads one plane ahead and writes them over the zero
// fill once the plane's TMA has completed.  One barrier per plane orders everything: before it
// the plane about to enter the stencil window is completed (TMA wait + halo), after it the slot
// of the plane that left the window is refilled while the current plane is computed.
//
// The operator is that of apply_J (same discrete stencils and reads) with the grid spacing,
// the 1/3 of the grad-div term and the tensor-product weights folded into per-level constants.
//
// Requirements (checked on the host): colour-split level, nx and ny multiples of 8 and >= 16,
// nz >= 8 (and even chunks for the restriction), so every TMA x coordinate and stride is
// 16-byte aligned and no tile row is both the first and the last of the box.
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
// restriction: plus the staging of the odd rows' partial sums (4 warps x 32 lanes x 4 fields)
template <typename T, int ORDER> __host__ __device__ constexpr size_t tile_restrict_smem_bytes()
{
    return tile_smem_bytes<T, ORDER>() + 16 + (size_t)(kTileY / 2) * 32 * 4 * sizeof(T);
}

struct TileGrid {
    int ntx, nty;   // tiles along x (pairs) and y (rows)
    int zc;         // planes per CTA
};

// Folded stencil weights of the inner operator on one level.
template <typename T>
struct TileCoef {
    T lk0, lk1[3], lnk2[3];              // Lap f = lk0 f + sum_a lk1 (f+a + f-a) + lnk2 (f+2a + f-2a)
    T mk0[3], mk1[3][3], mnk2[3][3];     // row A: Lap W_A + (1/3) D_AA W_A, same form
    T x11[3][3], x12[3][3], x22[3][3];   // (1/3) D_A D_B f = x11 g11 + x12 (g12 + g21) + x22 g22
    T dl;                                // diagonal of Lap (psi-row update)
    T idW[3];                            // omega / diagonal of row A
    T iom;                               // 1 / omega
    FaceDiag<T> fd;                      // diagonal shifts next to the faces (Robin boxes)
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

// 5-D tiled tensor load into shared memory, completing its bytes on the mbarrier.
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
// tile_fetch's value at the unwrapped cell c (beyond no extrapolating face); f is the field.
template <typename T, int BC>
__device__ __forceinline__ T tile_one(const Geo &g, const T *X, const T *O, int colour, int f, const int c[3])
{
    const int nx = g.n[0], ny = g.n[1];
    const size_t N = (size_t)nx * ny * g.n[2];
    int b[3], mirror;
    const bool clamped = bc_cell<BC>(g, c, b, mirror);   // wrap; or mirror / clamp (field f's sign)
    const int hb = (b[0] + b[1] + b[2]) & 1;
    const size_t idx =
        (size_t)f * N + (hb ? N / 2 : 0) + (size_t)(b[0] >> 1) + (size_t)(nx >> 1) * (b[1] + (size_t)ny * b[2]);
    T v = (hb == colour ? X : O)[idx];
    v = bc_signed<BC>(v, mirror, f);
    if (BC != BC_PERIODIC && clamped) v *= robin_ratio<T>(g, b[0], b[1], b[2], c[0], c[1], c[2]);
    return v;
}

// Beyond an extrapolating face: the weighted in-box cells of extrap_split (out of line).
template <typename T, int BC>
__device__ __noinline__ T tile_extrap(const Geo *g, const T *X, const T *O, int colour, int f, int i, int j, int k)
{
    const int p[3] = {i, j, k};
    int q[8][3], w[8];
    const int ns = extrap_split(*g, p, q, w);
    T s = 0;
    for (int t = 0; t < ns; ++t) s += (T)w[t] * tile_one<T, BC>(*g, X, O, colour, f, q[t]);
    return s;
}

template <typename T, int BC>
__device__ __forceinline__ T tile_fetch(const Geo &g, const T *X, const T *O, int colour, int P, int y, int z, int h,
                                        int f)
{
    const int p[3] = {2 * P + ((h + y + z) & 1), y, z};
    if constexpr (BC == BC_SYM)
        if (g.extrap && beyond_extrap(g, p)) return tile_extrap<T, BC>(&g, X, O, colour, f, p[0], p[1], p[2]);
    return tile_one<T, BC>(g, X, O, colour, f, p);
}

// ---------------------------------------------------------------- the plane ring
// Loading side of a tiled kernel: geometry of the CTA's tile, the TMA ring and the halo fix-ups.
// Usage: prologue(); then for every plane z of the chunk: advance(z) (false: stop, the CTA
// failed a bounded wait) followed by the plane's computation; finally finish(failed).
template <typename T, int ORDER, int BC>
struct TileRing {
    static constexpr int H = ORDER / 2, RY = tile_rows<ORDER>(), S = tile_slots<ORDER>();
    static constexpr int FE = tile_field_elems<ORDER>(), HE = tile_half_elems<ORDER>(), SE = tile_slot_elems<ORDER>();

    T *sm;
    uint64_t *bar;
    const Geo *g;
    const T *X, *O;
    const CUtensorMap *tmX, *tmO;
    int colour;   // the half loaded from X (tmX); the other half comes from O (tmO)
    long long spin;
    int P0, y0, z0, z1, tpt, zs, NP, tid;
    int npos, done, issued;
    int fo[kTileFix], fP[kTileFix], fy[kTileFix], fh[kTileFix], ff[kTileFix];
    T fv[kTileFix];   // halo values of the plane issued last, stored after its TMA completes

    __device__ __forceinline__ void setup(unsigned char *smem_raw, const Geo &geo, const T *X_, const T *O_,
                                          const CUtensorMap *mX, const CUtensorMap *mO, int col, const TileGrid &tg,
                                          long long spin_)
    {
        sm = reinterpret_cast<T *>(smem_raw);
        bar = reinterpret_cast<uint64_t *>(smem_raw + (size_t)S * SE * sizeof(T));
        g = &geo;
        X = X_;
        O = O_;
        tmX = mX;
        tmO = mO;
        colour = col;
        spin = spin_;
        const int nxh = geo.n[0] >> 1, ny = geo.n[1], nz = geo.n[2];
        int b = blockIdx.x;
        const int tx = b % tg.ntx;
        b /= tg.ntx;
        const int ty = b % tg.nty;
        const int tz = b / tg.nty;
        P0 = tx * kTileP;
        y0 = ty * kTileY;
        z0 = tz * tg.zc;
        z1 = min(z0 + tg.zc, nz);
        tpt = min(kTileP, nxh - P0);
        zs = z0 - H;
        NP = (z1 - z0) + 2 * H;
        tid = threadIdx.x;
        done = -1;
        issued = -1;
        // halo elements the tensor load leaves zero: rows outside [0, ny) and pairs outside
        // [0, nxh), restricted to what the stencil reads (pairs P0-1 .. P0+tpt)
        npos = tpt + 2;
        const int top = y0 == 0 ? H : 0, bot = (y0 + kTileY >= ny) ? H : 0;
        const int ngr = top + bot;
        const int lcol = P0 == 0 ? 1 : 0, rcol = (P0 + tpt >= nxh) ? 1 : 0, ngc = lcol + rcol;
        const int nfix = (ngr * npos + (RY - ngr) * ngc) * 8;
#pragma unroll
        for (int i = 0; i < kTileFix; ++i) {
            const int e = tid + i * kTileThreads;
            fo[i] = -1;
            fP[i] = fy[i] = fh[i] = ff[i] = 0;
            fv[i] = 0;
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
    }

    __device__ __forceinline__ bool ghost(int p) const { return BC != BC_PERIODIC && (zs + p < 0 || zs + p >= g->n[2]); }

    __device__ __forceinline__ void issue(int p)   // one thread: start the loads of relative plane p
    {
        uint64_t *mb = bar + p % S;
        if (ghost(p)) { tile_mbar_arrive(mb); return; }   // filled by plain loads instead
        int z = zs + p;
        const int nz = g->n[2];
        if (BC == BC_PERIODIC) { z += z < 0 ? nz : 0; z -= z >= nz ? nz : 0; }
        T *dst = sm + (p % S) * SE;
        tile_mbar_expect_tx(mb, (uint32_t)(2 * HE * sizeof(T)));
        tile_tma_load(dst + colour * HE, tmX, P0 - kTilePad, y0 - H, z, 0, colour, mb);
        tile_tma_load(dst + (1 - colour) * HE, tmO, P0 - kTilePad, y0 - H, z, 0, 1 - colour, mb);
    }

    __device__ __forceinline__ void fill_plane(int p)   // every element of a Robin ghost plane
    {
        T *dst = sm + (p % S) * SE;
        const int tot = 8 * RY * npos;
        for (int e = tid; e < tot; e += kTileThreads) {
            const int hf = e & 7, h = hf >> 2, fld = hf & 3;
            const int rest = e >> 3, r = rest / npos, pos = kTilePad - 1 + rest % npos;
            dst[h * HE + fld * FE + r * kTileW + pos] =
                tile_fetch<T, BC>(*g, X, O, colour, P0 - kTilePad + pos, y0 - H + r, zs + p, h, fld);
        }
    }

    __device__ __forceinline__ void load_fix(int p)
    {
#pragma unroll
        for (int i = 0; i < kTileFix; ++i)
            if (fo[i] >= 0) fv[i] = tile_fetch<T, BC>(*g, X, O, colour, fP[i], fy[i], zs + p, fh[i], ff[i]);
    }

    __device__ __forceinline__ void store_fix(int p)
    {
        T *dst = sm + (p % S) * SE;
#pragma unroll
        for (int i = 0; i < kTileFix; ++i)
            if (fo[i] >= 0) dst[fo[i]] = fv[i];
    }

    __device__ __forceinline__ bool wait(int p, long long limit)
    {
        return tile_mbar_wait(bar + p % S, (uint32_t)((p / S) & 1), limit);
    }

    // planes 0 .. 2H: issue all, complete 0 .. 2H-1 here, stage the halo of 2H
    __device__ __forceinline__ bool prologue()
    {
        if (tid < S) tile_mbar_init(bar + tid, 1);
        tile_mbar_init_fence();
        __syncthreads();
        if (tid == 0)
            for (int p = 0; p <= 2 * H; ++p) issue(p);
        issued = 2 * H;
        bool ok = true;
        for (int p = 0; p < 2 * H; ++p) {
            if (ghost(p)) { fill_plane(p); continue; }
            ok = ok && wait(p, spin);
            load_fix(p);
            store_fix(p);
        }
        if (ghost(2 * H)) fill_plane(2 * H);
        else load_fix(2 * H);
        return ok;
    }

    // Before computing plane z: complete plane z + H, then (after the barrier) refill the slot of
    // plane z - H - 1 with plane z + H + 1.  Returns false, for every thread, if a wait gave up.
    __device__ __forceinline__ bool advance(int z, bool ok)
    {
        const int p = z - zs;
        ok = ok && wait(p + H, spin);
        if (!ghost(p + H)) store_fix(p + H);
        if (__syncthreads_or(!ok)) return false;
        done = p + H;
        const int pn = p + H + 1;
        if (pn < NP) {
            if (tid == 0) {
                tile_fence_proxy_async();
                issue(pn);
            }
            issued = pn;
            if (ghost(pn)) fill_plane(pn);
            else load_fix(pn);
        }
        return true;
    }

    __device__ __forceinline__ void finish(bool failed, unsigned int *err)
    {
        if (!failed) return;
        if (tid == 0) atomicOr(err, 1u);
        // let the loads still in flight land before the CTA's shared memory is released (a
        // tensor load of an in-bounds box always completes; the bound only guards the poll)
        for (int p = done + 1; p <= issued; ++p) wait(p, spin > kTileDrain ? spin : kTileDrain);
    }

    // offset of the cell (lane, warp row w, plane z) in the colour half `half` of each window plane
    __device__ __forceinline__ void bases(int z, int w, int lane, int half, int (&ob)[2 * H + 1]) const
    {
        const int p = z - zs;
#pragma unroll
        for (int d = -H; d <= H; ++d) ob[d + H] = ((p + d) % S) * SE + half * HE + (w + H) * kTileW + kTilePad + lane;
    }
};

// Shared-memory accessor of one field around a cell: ob[dz + H] is the cell's offset in its
// colour half of plane z + dz, OH moves to the other colour half, PA is the cell's x parity (a
// neighbour at odd dx sits in pair m + PA + (dx-1)/2); fo is the field offset.
template <typename T, int ORDER, int OH, int PA>
struct AccT {
    const T *sm;
    const int *ob;
    int fo;
    __device__ __forceinline__ T operator()(int dx, int dy, int dz) const
    {
        int o = ob[dz + ORDER / 2] + fo + dy * kTileW;
        if ((dx + dy + dz) & 1) o += OH;
        o += (dx & 1) ? PA + ((dx - 1) >> 1) : (dx >> 1);
        return sm[o];
    }
};

// ---------------------------------------------------------------- folded operator
template <int ORDER, typename T, class F>
__device__ __forceinline__ T lap_fold(const F &f, T c, T k0, const T *k1, const T *nk2)
{
    T s = k0 * c;
    s = fma(k1[0], f(1, 0, 0) + f(-1, 0, 0), s);
    s = fma(k1[1], f(0, 1, 0) + f(0, -1, 0), s);
    s = fma(k1[2], f(0, 0, 1) + f(0, 0, -1), s);
    if constexpr (ORDER == 4) {
        s = fma(nk2[0], f(2, 0, 0) + f(-2, 0, 0), s);
        s = fma(nk2[1], f(0, 2, 0) + f(0, -2, 0), s);
        s = fma(nk2[2], f(0, 0, 2) + f(0, 0, -2), s);
    }
    return s;
}

// (1/3) D_A D_B f from the antisymmetric corner sums g(a, b) = f(a,b) + f(-a,-b) - f(a,-b) - f(-a,b)
template <int ORDER, int A, int B, typename T, class F>
__device__ __forceinline__ T dmix_fold(const F &f, T x11, T x12, T x22)
{
    auto gq = [&](int a, int b) {
        return (ax2<A, B>(f, a, b) + ax2<A, B>(f, -a, -b)) - (ax2<A, B>(f, a, -b) + ax2<A, B>(f, -a, b));
    };
    T r = x11 * gq(1, 1);
    if constexpr (ORDER == 4) {
        r = fma(x12, gq(1, 2) + gq(2, 1), r);
        r = fma(x22, gq(2, 2), r);
    }
    return r;
}

// out = J e at one cell (the operator of apply_J), centre values in ctr.
template <int ORDER, typename T, class F>
__device__ __forceinline__ void apply_J_fold(const F &e0, const F &e1, const F &e2, const F &e3, T ca, T cb,
                                             const TileCoef<T> &tc, T out[4], T ctr[4])
{
    ctr[0] = e0(0, 0, 0);
    ctr[1] = e1(0, 0, 0);
    ctr[2] = e2(0, 0, 0);
    ctr[3] = e3(0, 0, 0);
    out[0] = fma(ca, lap_fold<ORDER>(e0, ctr[0], tc.lk0, tc.lk1, tc.lnk2), cb * ctr[0]);
    out[1] = lap_fold<ORDER>(e1, ctr[1], tc.mk0[0], tc.mk1[0], tc.mnk2[0]) +
             (dmix_fold<ORDER, 0, 1>(e2, tc.x11[0][1], tc.x12[0][1], tc.x22[0][1]) +
              dmix_fold<ORDER, 0, 2>(e3, tc.x11[0][2], tc.x12[0][2], tc.x22[0][2]));
    out[2] = lap_fold<ORDER>(e2, ctr[2], tc.mk0[1], tc.mk1[1], tc.mnk2[1]) +
             (dmix_fold<ORDER, 1, 0>(e1, tc.x11[1][0], tc.x12[1][0], tc.x22[1][0]) +
              dmix_fold<ORDER, 1, 2>(e3, tc.x11[1][2], tc.x12[1][2], tc.x22[1][2]));
    out[3] = lap_fold<ORDER>(e3, ctr[3], tc.mk0[2], tc.mk1[2], tc.mnk2[2]) +
             (dmix_fold<ORDER, 2, 0>(e1, tc.x11[2][0], tc.x12[2][0], tc.x22[2][0]) +
              dmix_fold<ORDER, 2, 1>(e2, tc.x11[2][1], tc.x12[2][1], tc.x22[2][1]));
}

// J e of the cell with x parity PA in colour half HALF (both compile-time) from the window.
template <typename T, int ORDER, int HALF, int PA>
__device__ __forceinline__ void tile_apply(const T *sm, const int *ob, T ca, T cb, const TileCoef<T> &tc, T Je[4],
                                           T ctr[4])
{
    constexpr int FE = tile_field_elems<ORDER>(), OH = (1 - 2 * HALF) * tile_half_elems<ORDER>();
    AccT<T, ORDER, OH, PA> a0{sm, ob, 0}, a1{sm, ob, FE}, a2{sm, ob, 2 * FE}, a3{sm, ob, 3 * FE};
    apply_J_fold<ORDER, T>(a0, a1, a2, a3, ca, cb, tc, Je, ctr);
}

// ---------------------------------------------------------------- colour pass
template <typename T, int ORDER, int BC, int COLOUR>
__global__ void __launch_bounds__(kTileThreads, sizeof(T) == 4 ? 2 : 1)
    k_smooth_tile(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmO, Geo g,
                  TileCoef<T> tc, const T *__restrict__ X, const T *__restrict__ O, T *__restrict__ Y,
                  const T *__restrict__ f, const T *__restrict__ ab, TileGrid tg, unsigned int *__restrict__ err,
                  long long spin)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int H = ORDER / 2;
    TileRing<T, ORDER, BC> ring;
    ring.setup(smem_raw, g, X, O, &tmX, &tmO, COLOUR, tg, spin);
    if (ring.z0 >= ring.z1) return;
    const int nxh = g.n[0] >> 1, ny = g.n[1];
    const unsigned N = (unsigned)g.n[0] * ny * g.n[2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool act = lane < ring.tpt;
    bool ok = ring.prologue(), failed = false;
    for (int z = ring.z0; z < ring.z1; ++z) {
        const int y = ring.y0 + w;
        const unsigned q = (COLOUR ? N / 2 : 0u) + (unsigned)(ring.P0 + lane) + (unsigned)nxh * ((unsigned)y + (unsigned)ny * z);
        T ca = 0, cb = 0, fq[4] = {0, 0, 0, 0};
        if (act) {   // in flight during the wait and the barrier
            ca = ab[q];
            cb = ab[N + q];
#pragma unroll
            for (int a = 0; a < 4; ++a) fq[a] = f[a * N + q];
        }
        if (!ring.advance(z, ok)) { failed = true; break; }
        if (act) {
            int ob[2 * H + 1];
            ring.bases(z, w, lane, COLOUR, ob);
            T Je[4], ctr[4];
            if ((COLOUR + y + z) & 1) tile_apply<T, ORDER, COLOUR, 1>(ring.sm, ob, ca, cb, tc, Je, ctr);
            else tile_apply<T, ORDER, COLOUR, 0>(ring.sm, ob, ca, cb, tc, Je, ctr);
            T dl, kW[3];   // the true diagonal next to a face (boxes with faces only)
            relax_factors<BC>(tc.fd, g, 2 * (ring.P0 + lane) + ((COLOUR + y + z) & 1), y, z, true, tc.dl, tc.idW, tc.iom,
                              dl, kW);
            Y[q] = ctr[0] + (fq[0] - Je[0]) / ((ca * dl + cb) * tc.iom);
#pragma unroll
            for (int a = 0; a < 3; ++a) Y[(1 + a) * N + q] = ctr[1 + a] + (fq[1 + a] - Je[1 + a]) * kW[a];
        }
    }
    ring.finish(failed, err);
}

// ---------------------------------------------------------------- residual + restriction
// r = f - J e at both cells of each thread's pair on every plane, summed over the pair (x), the
// two planes of a coarse plane (z, in registers) and the two rows of a coarse row (y, odd warps
// hand their sums to the even ones through shared memory); the 8-child mean goes to the coarse
// right-hand side fc (colour-split, or plain when the coarse level is the coarsest).
template <typename T, int ORDER, int BC>
__global__ void __launch_bounds__(kTileThreads, sizeof(T) == 4 ? 2 : 1)
    k_restrict_tile(const __grid_constant__ CUtensorMap tm, Geo g, TileCoef<T> tc, Geo gc, const T *__restrict__ e,
                    const T *__restrict__ f, const T *__restrict__ ab, T *__restrict__ fc, int csplit, TileGrid tg,
                    unsigned int *__restrict__ err, long long spin)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int H = ORDER / 2;
    TileRing<T, ORDER, BC> ring;
    ring.setup(smem_raw, g, e, e, &tm, &tm, 0, tg, spin);
    if (ring.z0 >= ring.z1) return;
    T *stage = reinterpret_cast<T *>(smem_raw + tile_smem_bytes<T, ORDER>() + 16);   // [4 rows][32 lanes][4]
    const int nxh = g.n[0] >> 1, ny = g.n[1];
    const unsigned N = (unsigned)g.n[0] * ny * g.n[2];
    const unsigned Nc = (unsigned)gc.n[0] * gc.n[1] * gc.n[2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const bool act = lane < ring.tpt;
    T acc[4] = {0, 0, 0, 0};
    auto flush = [&](int K) {   // even warps: add the odd row's sums and write coarse plane K's cell
        if ((w & 1) == 0 && act) {
            const int I = ring.P0 + lane, J = (ring.y0 + w) >> 1;
            const unsigned linc = (unsigned)I + (unsigned)gc.n[0] * ((unsigned)J + (unsigned)gc.n[1] * (unsigned)K);
            const unsigned pc = csplit ? (((I + J + K) & 1) ? Nc / 2 : 0u) + (linc >> 1) : linc;
            const T *st = stage + ((w >> 1) * 32 + lane) * 4;
#pragma unroll
            for (int a = 0; a < 4; ++a) fc[a * Nc + pc] = (acc[a] + st[a]) * (T)0.125;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[a] = 0;
    };
    bool ok = ring.prologue(), failed = false;
    for (int z = ring.z0; z < ring.z1; ++z) {
        const int y = ring.y0 + w;
        const unsigned m = (unsigned)(ring.P0 + lane) + (unsigned)nxh * ((unsigned)y + (unsigned)ny * z);
        const int c0 = (y + z) & 1;   // colour of the pair's even-x cell
        const unsigned q0 = (c0 ? N / 2 : 0u) + m, q1 = (c0 ? 0u : N / 2) + m;
        T a0 = 0, b0 = 0, a1 = 0, b1 = 0, f0[4] = {0, 0, 0, 0}, f1[4] = {0, 0, 0, 0};
        if (act) {
            a0 = ab[q0];
            b0 = ab[N + q0];
            a1 = ab[q1];
            b1 = ab[N + q1];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                f0[a] = f[a * N + q0];
                f1[a] = f[a * N + q1];
            }
        }
        if (!ring.advance(z, ok)) { failed = true; break; }
        if ((z & 1) == 0 && z > ring.z0) flush((z >> 1) - 1);   // the previous coarse plane
        if (act) {
            int obA[2 * H + 1], obB[2 * H + 1];
            ring.bases(z, w, lane, c0, obA);       // even-x cell, colour c0
            ring.bases(z, w, lane, 1 - c0, obB);   // odd-x cell, the other colour
            T Je[4], ctr[4];
            if (c0 == 0) tile_apply<T, ORDER, 0, 0>(ring.sm, obA, a0, b0, tc, Je, ctr);
            else tile_apply<T, ORDER, 1, 0>(ring.sm, obA, a0, b0, tc, Je, ctr);
#pragma unroll
            for (int a = 0; a < 4; ++a) acc[a] += f0[a] - Je[a];
            if (c0 == 0) tile_apply<T, ORDER, 1, 1>(ring.sm, obB, a1, b1, tc, Je, ctr);
            else tile_apply<T, ORDER, 0, 1>(ring.sm, obB, a1, b1, tc, Je, ctr);
#pragma unroll
            for (int a = 0; a < 4; ++a) acc[a] += f1[a] - Je[a];
        }
        if ((z & 1) && (w & 1)) {   // odd row of a coarse row: hand the sums to the even warp
            T *st = stage + ((w >> 1) * 32 + lane) * 4;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                st[a] = acc[a];
                acc[a] = 0;
            }
        }
    }
    if (!failed) {
        __syncthreads();
        flush((ring.z1 >> 1) - 1);
    }
    ring.finish(failed, err);
}

}  // namespace ctt
