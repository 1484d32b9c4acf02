// mg_tile.cuh -- shared-memory tiled kernels of the colour-split levels: the red-black colour
// pass of the smoother and the fused residual + restriction.
//
// A CTA owns a tile of 32 colour pairs (64 cells) in x by 8 rows in y and marches through a
// chunk of z planes; thread (lane, warp) keeps the pair `lane` of row `warp` for the whole march.
// Each plane of the 4 correction fields (both colour halves, the tile plus its stencil halo in x
// and y) is brought into a ring of shared-memory slots by two TMA tensor loads
// (cp.async.bulk.tensor, one per colour half) completing on an mbarrier.  Halo cells outside the
// box (periodic wrap, the Robin 1/r ghost value v(clamp(g)) |x_clamp| / |x_g|, a mirror image
// across a symmetry plane with W's normal component negated, or an extrapolated value) are not
// addressable by the tensor load, which fills them with zeros: the CTA fetches them with plain
// loads while the plane is in flight and writes them over the zero fill once its TMA has completed.
//
// Only the plane being computed is read from shared memory.  Its contribution to every stencil
// that reaches it along z is pushed into per-thread pending sums of the planes z - H .. z + H
// (registers), and a cell is finished H planes later, once its last z tap has arrived:
//  * the z taps of the four Laplacians take the pair's own two cells;
//  * the mixed terms that involve z are applied as a z derivative of an in-plane first
//    derivative, D_A D_z f = D_z (D_A f) (A = x, y), so D_x W_x, D_y W_y, D_x W_z and D_y W_z are
//    formed once per plane at both cells of the pair;
//  * the in-plane parts (x and y taps, D_x D_y) are summed from the plane directly.
// That is 74 shared-memory reads per updated cell in the colour pass (the direct form of the
// whole stencil takes 148) and 44 per cell in the residual.  The ring holds the plane being
// computed plus four (colour pass) or three (residual) in flight; one barrier per plane orders
// everything.  The 2H halo planes of a chunk only push their z taps (no in-plane part).  The
// per-cell inputs of a finished cell (psi-row coefficients a, b and the right-hand side f) arrive
// by per-thread cp.async copies into a shared staging ring a few planes ahead, so their DRAM
// latency is hidden behind the stencil work of the planes in between.
//
// The operator is that of apply_J (the same discrete stencils on the same values) with the grid
// spacing, the 1/3 of the grad-div term and the tensor-product weights folded into per-level
// constants; only the FP rounding order differs.
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
constexpr int kColourSlots = 5;                 // colour pass ring: the plane being computed + 4 in flight
constexpr int kRestrictSlots = 4;               // residual ring: + 3 in flight
constexpr int kColourAhead = 3;                 // planes ahead at which a cell's right-hand side is fetched
constexpr int kRestrictAhead = 2;
constexpr int kColourVals = 6;                  // fetched per thread and plane: a, b, f_0..3 of one cell
constexpr int kRestrictVals = 12;               // ... of both cells of the pair
constexpr long long kTileDrain = 1LL << 26;     // polls allowed for in-flight loads after a failed wait

template <int ORDER> __host__ __device__ constexpr int tile_rows() { return kTileY + ORDER; }   // 8 + 2 halo
template <int ORDER> __host__ __device__ constexpr int tile_field_elems() { return tile_rows<ORDER>() * kTileW; }
template <int ORDER> __host__ __device__ constexpr int tile_half_elems() { return 4 * tile_field_elems<ORDER>(); }
template <int ORDER> __host__ __device__ constexpr int tile_slot_elems() { return 2 * tile_half_elems<ORDER>(); }
// shared memory: the ring's slots, its mbarriers (16-byte padded), then the per-thread staging of
// the fetched right-hand sides ([plane slot][value][thread]); the restriction adds the hand-over of
// the odd rows' partial sums (4 warps x 32 lanes x 4 fields)
template <typename T, int ORDER, int S> __host__ __device__ constexpr size_t tile_ring_bytes()
{
    return (size_t)S * tile_slot_elems<ORDER>() * sizeof(T) + 16 * ((8 * S + 15) / 16);
}
template <typename T, int ORDER> __host__ __device__ constexpr size_t tile_smem_bytes()
{
    return tile_ring_bytes<T, ORDER, kColourSlots>() + (size_t)(kColourAhead + 1) * kColourVals * kTileThreads * sizeof(T);
}
template <typename T, int ORDER> __host__ __device__ constexpr size_t tile_restrict_smem_bytes()
{
    return tile_ring_bytes<T, ORDER, kRestrictSlots>() +
           (size_t)(kRestrictAhead + 1) * kRestrictVals * kTileThreads * sizeof(T) + (size_t)(kTileY / 2) * 32 * 4 * sizeof(T);
}
static_assert(tile_smem_bytes<double, 4>() <= 227 * 1024 && tile_restrict_smem_bytes<double, 4>() <= 227 * 1024,
              "tiles fit the shared memory of one CTA");
static_assert(2 * tile_smem_bytes<float, 4>() <= 227 * 1024 && 2 * tile_restrict_smem_bytes<float, 4>() <= 227 * 1024,
              "two FP32 CTAs fit one SM");

struct TileGrid {
    int ntx, nty;   // tiles along x (pairs) and y (rows)
    int zc;         // planes per CTA
};

// Folded stencil weights of the inner operator on one level.
template <typename T>
struct TileCoef {
    T lk0, lk1[3], lnk2[3];              // Lap f = lk0 f + sum_a lk1 (f+a + f-a) + lnk2 (f+2a + f-2a)
    T mk0[3], mk1[3][3], mnk2[3][3];     // row A: Lap W_A + (1/3) D_AA W_A, same form
    T d1[3], d2[3];                      // D_a f = d1 (f+a - f-a) - d2 (f+2a - f-2a)
    T t1[3], t2[3];                      // the same with the 1/3 of the grad-div term: (1/3) D_a
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

// Per-thread asynchronous copy of one element from global into shared memory; it completes with the
// thread's cp.async groups (commit / wait), so only the issuing thread reads it back.
template <typename T>
__device__ __forceinline__ void tile_copy_async(T *dst, const T *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sm_addr(dst)), "l"(__cvta_generic_to_global(src)),
                 "n"((int)sizeof(T))
                 : "memory");
}
__device__ __forceinline__ void tile_copy_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void tile_copy_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void tile_copy_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

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
// Relative plane p = 0 .. NP-1 is plane zs + p (zs = z0 - H: the chunk plus H halo planes on each
// side) and lives in slot p % S; its tensor loads are issued DEP = S - 1 planes ahead, its halo
// values fetched one plane ahead (while the previous plane is computed).  Usage: prologue(); then
// for every p: advance(p) (false: stop, the CTA failed a bounded wait) followed by the plane's
// computation from slot(p); finally finish(failed).
template <typename T, int ORDER, int BC, int S>
struct TileRing {
    static constexpr int H = ORDER / 2, RY = tile_rows<ORDER>(), DEP = S - 1;
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
    T fv[kTileFix];   // halo values of the next plane, stored once its tensor loads have landed

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

    __device__ __forceinline__ T *slot(int p) const { return sm + (p % S) * SE; }

    __device__ __forceinline__ void issue(int p)   // one thread: start the loads of relative plane p
    {
        uint64_t *mb = bar + p % S;
        if (ghost(p)) { tile_mbar_arrive(mb); return; }   // filled by plain loads instead
        int z = zs + p;
        const int nz = g->n[2];
        if (BC == BC_PERIODIC) { z += z < 0 ? nz : 0; z -= z >= nz ? nz : 0; }
        T *dst = slot(p);
        tile_mbar_expect_tx(mb, (uint32_t)(2 * HE * sizeof(T)));
        tile_tma_load(dst + colour * HE, tmX, P0 - kTilePad, y0 - H, z, 0, colour, mb);
        tile_tma_load(dst + (1 - colour) * HE, tmO, P0 - kTilePad, y0 - H, z, 0, 1 - colour, mb);
    }

    __device__ __forceinline__ void fill_plane(int p)   // every element of a Robin ghost plane
    {
        T *dst = slot(p);
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
        T *dst = slot(p);
#pragma unroll
        for (int i = 0; i < kTileFix; ++i)
            if (fo[i] >= 0) dst[fo[i]] = fv[i];
    }

    // one plane ahead: fill plane p (ghost plane; its slot receives no tensor load) or fetch its
    // halo values (stored once its tensor loads have landed)
    __device__ __forceinline__ void stage(int p)
    {
        if (ghost(p)) fill_plane(p);
        else load_fix(p);
    }

    __device__ __forceinline__ bool wait(int p, long long limit)
    {
        return tile_mbar_wait(bar + p % S, (uint32_t)((p / S) & 1), limit);
    }

    // issue planes 0 .. DEP-1, stage plane 0
    __device__ __forceinline__ bool prologue()
    {
        if (tid < S) tile_mbar_init(bar + tid, 1);
        tile_mbar_init_fence();
        __syncthreads();
        const int np = min(DEP, NP);
        if (tid == 0)
            for (int p = 0; p < np; ++p) issue(p);
        issued = np - 1;
        stage(0);
        return true;
    }

    // Before computing plane p: complete it, then (after the barrier) reuse the slot of plane p - 1
    // for plane p + DEP and stage plane p + 1.  Returns false, for every thread, if a wait gave up.
    __device__ __forceinline__ bool advance(int p, bool ok)
    {
        ok = ok && wait(p, spin);
        if (!ghost(p)) store_fix(p);
        if (__syncthreads_or(!ok)) return false;
        done = p;
        const int pn = p + DEP;
        if (pn < NP) {
            if (tid == 0) {
                tile_fence_proxy_async();
                issue(pn);
            }
            issued = pn;
        }
        if (p + 1 < NP) stage(p + 1);
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
};

// ---------------------------------------------------------------- one plane of the tile
// Field F at the cell of x-bit `bit` in pair P + dp, row y + dy of a plane (HB: the colour of the
// pair's even-x cell in row y; s: pair P, row y, field 0 of colour half 0 of the plane's slot).
template <typename T, int ORDER, int HB>
struct PlaneView {
    const T *s;
    __device__ __forceinline__ T operator()(int F, int bit, int dp, int dy) const
    {
        return s[((bit + HB + dy) & 1) * tile_half_elems<ORDER>() + F * tile_field_elems<ORDER>() + dy * kTileW + dp];
    }
};

// column tap j of c[bit][j] is row offset col_dy(j): -H .. -1, 1 .. H
__host__ __device__ constexpr int col_dy(int j, int H) { return j < H ? j - H : j - H + 1; }

// row y of field F: r[k] is the cell x = 2P - 2 + k (k = 0 .. 5; ORDER 2 reads 1 .. 4)
template <int ORDER, typename T, class V>
__device__ __forceinline__ void tile_row(const V &v, int F, T (&r)[6])
{
#pragma unroll
    for (int k = 0; k < 6; ++k) r[k] = (ORDER == 4 || (k >= 1 && k <= 4)) ? v(F, k & 1, (k >> 1) - 1, 0) : (T)0;
}

// columns of the pair's two cells: c[bit][j] at row y + col_dy(j)
template <int ORDER, typename T, class V>
__device__ __forceinline__ void tile_cols(const V &v, int F, T (&c)[2][ORDER])
{
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int j = 0; j < ORDER; ++j) c[b][j] = v(F, b, 0, col_dy(j, ORDER / 2));
}

// first derivative along x at the pair's cell of bit b, from its row
template <int ORDER, typename T>
__device__ __forceinline__ T dx_row(const T (&r)[6], int b, T d1, T d2)
{
    T s = d1 * (r[3 + b] - r[1 + b]);
    if constexpr (ORDER == 4) s = fma(-d2, r[4 + b] - r[b], s);
    return s;
}

// first derivative along a column (taps col_dy(j))
template <int ORDER, typename T>
__device__ __forceinline__ T d_col(const T (&c)[ORDER], T d1, T d2)
{
    constexpr int H = ORDER / 2;
    T s = d1 * (c[H] - c[H - 1]);
    if constexpr (ORDER == 4) s = fma(-d2, c[3] - c[0], s);
    return s;
}

// in-plane part (centre, x and y taps) of a Laplacian-form stencil at the pair's cell of bit b
template <int ORDER, typename T>
__device__ __forceinline__ T lap_xy(const T (&r)[6], const T (&c)[ORDER], int b, T k0, const T *k1, const T *nk2)
{
    constexpr int H = ORDER / 2;
    T s = k0 * r[2 + b];
    s = fma(k1[0], r[1 + b] + r[3 + b], s);
    s = fma(k1[1], c[H - 1] + c[H], s);
    if constexpr (ORDER == 4) {
        s = fma(nk2[0], r[b] + r[4 + b], s);
        s = fma(nk2[1], c[0] + c[3], s);
    }
    return s;
}

// (1/3) D_x D_y f at the pair's cell of bit b: D_x along the rows y + dy, then (1/3) D_y of those.
// own: the pair's columns of f (tile_cols); the neighbouring pairs' columns are read here.
template <int ORDER, typename T, class V>
__device__ __forceinline__ T mix_xy(const V &v, int F, const T (&own)[2][ORDER], int b, const TileCoef<T> &tc)
{
    T u[ORDER];
#pragma unroll
    for (int j = 0; j < ORDER; ++j) {
        const int dy = col_dy(j, ORDER / 2);
        auto col = [&](int k) -> T { return (k == 2 || k == 3) ? own[k - 2][j] : v(F, k & 1, (k >> 1) - 1, dy); };
        T s = tc.d1[0] * (col(3 + b) - col(1 + b));
        if constexpr (ORDER == 4) s = fma(-tc.d2[0], col(4 + b) - col(b), s);
        u[j] = s;
    }
    return d_col<ORDER>(u, tc.t1[1], tc.t2[1]);
}

// Pushes of one plane's value into the pending sums acc(k) of planes zq - H + k: a symmetric z tap
// (Laplacian weights w1 at distance 1, w2 at 2; vq: the value seen at distance 1, vp at distance 2)
template <int ORDER, typename T, class A>
__device__ __forceinline__ void push_lap(A &&acc, T vq, T vp, T w1, T w2)
{
    constexpr int H = ORDER / 2;
    acc(H - 1) = fma(w1, vq, acc(H - 1));
    acc(H + 1) = fma(w1, vq, acc(H + 1));
    if constexpr (ORDER == 4) {
        acc(0) = fma(w2, vp, acc(0));
        acc(4) = fma(w2, vp, acc(4));
    }
}

// ... and an antisymmetric one: the z derivative t1 (g(z+1) - g(z-1)) - t2 (g(z+2) - g(z-2))
template <int ORDER, typename T, class A>
__device__ __forceinline__ void push_dz(A &&acc, T gq, T gp, T t1, T t2)
{
    constexpr int H = ORDER / 2;
    acc(H - 1) = fma(t1, gq, acc(H - 1));    // this plane is the +1 tap of plane zq - 1
    acc(H + 1) = fma(-t1, gq, acc(H + 1));   // and the -1 tap of plane zq + 1
    if constexpr (ORDER == 4) {
        acc(0) = fma(-t2, gp, acc(0));
        acc(4) = fma(t2, gp, acc(4));
    }
}

// Colour pass: contributions of the current plane to the pending sums acc[k][row] (planes
// zq - H + k, each at its cell of the pass's colour), with the cell of this plane at x-bit PQ.
// The cell of plane zq +- 1 sits at the other bit, that of zq +- 2 at PQ.  FULL = false: a halo
// plane of the chunk, whose own cell is not updated (z taps only).
template <typename T, int ORDER, int HB, int PQ, bool FULL>
__device__ __forceinline__ void colour_plane(const T *s, const TileCoef<T> &tc, T (&acc)[ORDER + 1][4], T (&ctr)[4])
{
    constexpr int H = ORDER / 2, Q = 1 - PQ;
    const PlaneView<T, ORDER, HB> v{s};
    T r[6], c[2][ORDER];
    auto row = [&](int a) { return [&acc, a](int k) -> T & { return acc[k][a]; }; };
    // psi row: Laplacian
    tile_row<ORDER>(v, 0, r);
    tile_cols<ORDER>(v, 0, c);
    if constexpr (FULL) {
        ctr[0] = r[2 + PQ];
        acc[H][0] += lap_xy<ORDER>(r, c[PQ], PQ, tc.lk0, tc.lk1, tc.lnk2);
    }
    push_lap<ORDER>(row(0), r[2 + Q], r[2 + PQ], tc.lk1[2], tc.lnk2[2]);
    // W_x: its row's Laplacian, (1/3) D_z D_x W_x of the z row, (1/3) D_y D_x W_x of the y row
    tile_row<ORDER>(v, 1, r);
    tile_cols<ORDER>(v, 1, c);
    if constexpr (FULL) {
        ctr[1] = r[2 + PQ];
        acc[H][1] += lap_xy<ORDER>(r, c[PQ], PQ, tc.mk0[0], tc.mk1[0], tc.mnk2[0]);
        acc[H][2] += mix_xy<ORDER>(v, 1, c, PQ, tc);
    }
    push_lap<ORDER>(row(1), r[2 + Q], r[2 + PQ], tc.mk1[0][2], tc.mnk2[0][2]);
    push_dz<ORDER>(row(3), dx_row<ORDER>(r, Q, tc.d1[0], tc.d2[0]), dx_row<ORDER>(r, PQ, tc.d1[0], tc.d2[0]),
                   tc.t1[2], tc.t2[2]);
    // W_y: its row's Laplacian, (1/3) D_z D_y W_y of the z row, (1/3) D_x D_y W_y of the x row
    tile_row<ORDER>(v, 2, r);
    tile_cols<ORDER>(v, 2, c);
    if constexpr (FULL) {
        ctr[2] = r[2 + PQ];
        acc[H][2] += lap_xy<ORDER>(r, c[PQ], PQ, tc.mk0[1], tc.mk1[1], tc.mnk2[1]);
        acc[H][1] += mix_xy<ORDER>(v, 2, c, PQ, tc);
    }
    push_lap<ORDER>(row(2), r[2 + Q], r[2 + PQ], tc.mk1[1][2], tc.mnk2[1][2]);
    push_dz<ORDER>(row(3), d_col<ORDER>(c[Q], tc.d1[1], tc.d2[1]), d_col<ORDER>(c[PQ], tc.d1[1], tc.d2[1]), tc.t1[2],
                   tc.t2[2]);
    // W_z: its row's Laplacian, (1/3) D_z D_x W_z of the x row, (1/3) D_z D_y W_z of the y row
    tile_row<ORDER>(v, 3, r);
    tile_cols<ORDER>(v, 3, c);
    if constexpr (FULL) {
        ctr[3] = r[2 + PQ];
        acc[H][3] += lap_xy<ORDER>(r, c[PQ], PQ, tc.mk0[2], tc.mk1[2], tc.mnk2[2]);
    }
    push_lap<ORDER>(row(3), r[2 + Q], r[2 + PQ], tc.mk1[2][2], tc.mnk2[2][2]);
    push_dz<ORDER>(row(1), dx_row<ORDER>(r, Q, tc.d1[0], tc.d2[0]), dx_row<ORDER>(r, PQ, tc.d1[0], tc.d2[0]),
                   tc.t1[2], tc.t2[2]);
    push_dz<ORDER>(row(2), d_col<ORDER>(c[Q], tc.d1[1], tc.d2[1]), d_col<ORDER>(c[PQ], tc.d1[1], tc.d2[1]), tc.t1[2],
                   tc.t2[2]);
}

// Residual: contributions of the current plane at both cells of the pair (acc[k][bit][row]; every
// z tap of a cell comes from the same bit of the other planes); cp: the psi values (the psi row's
// b coefficient multiplies its centre value when the cell is finished).  FULL = false: a halo plane.
template <typename T, int ORDER, int HB, bool FULL>
__device__ __forceinline__ void residual_plane(const T *s, const TileCoef<T> &tc, T (&acc)[ORDER + 1][2][4],
                                               T (&cp)[2])
{
    constexpr int H = ORDER / 2;
    const PlaneView<T, ORDER, HB> v{s};
    T r[6], c[2][ORDER];
    auto row = [&](int b, int a) { return [&acc, b, a](int k) -> T & { return acc[k][b][a]; }; };
    tile_row<ORDER>(v, 0, r);
    tile_cols<ORDER>(v, 0, c);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        if constexpr (FULL) {
            cp[b] = r[2 + b];
            acc[H][b][0] += lap_xy<ORDER>(r, c[b], b, tc.lk0, tc.lk1, tc.lnk2);
        }
        push_lap<ORDER>(row(b, 0), r[2 + b], r[2 + b], tc.lk1[2], tc.lnk2[2]);
    }
    tile_row<ORDER>(v, 1, r);
    tile_cols<ORDER>(v, 1, c);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        if constexpr (FULL) {
            acc[H][b][1] += lap_xy<ORDER>(r, c[b], b, tc.mk0[0], tc.mk1[0], tc.mnk2[0]);
            acc[H][b][2] += mix_xy<ORDER>(v, 1, c, b, tc);
        }
        push_lap<ORDER>(row(b, 1), r[2 + b], r[2 + b], tc.mk1[0][2], tc.mnk2[0][2]);
        const T gx = dx_row<ORDER>(r, b, tc.d1[0], tc.d2[0]);
        push_dz<ORDER>(row(b, 3), gx, gx, tc.t1[2], tc.t2[2]);
    }
    tile_row<ORDER>(v, 2, r);
    tile_cols<ORDER>(v, 2, c);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        if constexpr (FULL) {
            acc[H][b][2] += lap_xy<ORDER>(r, c[b], b, tc.mk0[1], tc.mk1[1], tc.mnk2[1]);
            acc[H][b][1] += mix_xy<ORDER>(v, 2, c, b, tc);
        }
        push_lap<ORDER>(row(b, 2), r[2 + b], r[2 + b], tc.mk1[1][2], tc.mnk2[1][2]);
        const T gy = d_col<ORDER>(c[b], tc.d1[1], tc.d2[1]);
        push_dz<ORDER>(row(b, 3), gy, gy, tc.t1[2], tc.t2[2]);
    }
    tile_row<ORDER>(v, 3, r);
    tile_cols<ORDER>(v, 3, c);
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        if constexpr (FULL) acc[H][b][3] += lap_xy<ORDER>(r, c[b], b, tc.mk0[2], tc.mk1[2], tc.mnk2[2]);
        push_lap<ORDER>(row(b, 3), r[2 + b], r[2 + b], tc.mk1[2][2], tc.mnk2[2][2]);
        const T gx = dx_row<ORDER>(r, b, tc.d1[0], tc.d2[0]), gy = d_col<ORDER>(c[b], tc.d1[1], tc.d2[1]);
        push_dz<ORDER>(row(b, 1), gx, gx, tc.t1[2], tc.t2[2]);
        push_dz<ORDER>(row(b, 2), gy, gy, tc.t1[2], tc.t2[2]);
    }
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
    TileRing<T, ORDER, BC, kColourSlots> ring;
    ring.setup(smem_raw, g, X, O, &tmX, &tmO, COLOUR, tg, spin);
    if (ring.z0 >= ring.z1) return;
    const int nxh = g.n[0] >> 1, ny = g.n[1];
    const unsigned N = (unsigned)g.n[0] * ny * g.n[2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, y = ring.y0 + w;
    const bool act = lane < ring.tpt;
    T acc[2 * H + 1][4], ctr[H + 1][4];   // pending sums of planes zq - H .. zq + H; centre values
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int k = 0; k <= 2 * H; ++k) acc[k][a] = 0;
#pragma unroll
        for (int k = 0; k <= H; ++k) ctr[k][a] = 0;
    }
    // the psi-row coefficients and right-hand side of the cell finished at iteration p, copied into
    // this thread's staging kColourAhead iterations ahead: [slot][value][thread]
    T *fst = reinterpret_cast<T *>(smem_raw + tile_ring_bytes<T, ORDER, kColourSlots>()) + threadIdx.x;
    auto cell = [&](int zu) {
        return (COLOUR ? N / 2 : 0u) + (unsigned)(ring.P0 + lane) + (unsigned)nxh * ((unsigned)y + (unsigned)ny * zu);
    };
    auto fetch = [&](int p) {
        const int zu = ring.zs + p - H;
        if (act && p < ring.NP && zu >= ring.z0) {
            const unsigned q = cell(zu);
            T *d = fst + (p % (kColourAhead + 1)) * kColourVals * kTileThreads;
            tile_copy_async(d, ab + q);
            tile_copy_async(d + kTileThreads, ab + N + q);
#pragma unroll
            for (int a = 0; a < 4; ++a) tile_copy_async(d + (2 + a) * kTileThreads, f + a * N + q);
        }
        tile_copy_commit();
    };
    for (int p = 0; p < kColourAhead; ++p) fetch(p);
    bool ok = ring.prologue(), failed = false;
    for (int p = 0; p < ring.NP; ++p) {
        const int zq = ring.zs + p, zu = zq - H;   // zu: the plane finished after this one
        const bool fin = act && zu >= ring.z0;
        fetch(p + kColourAhead);
        if (!ring.advance(p, ok)) { failed = true; break; }
        if (act) {
            const T *s = ring.slot(p) + (w + H) * kTileW + kTilePad + lane;
            const bool own = zq >= ring.z0 && zq < ring.z1;   // a plane of the chunk, not a halo plane
            if ((y + zq) & 1) {
                if (own) colour_plane<T, ORDER, 1, (COLOUR + 1) & 1, true>(s, tc, acc, ctr[H]);
                else colour_plane<T, ORDER, 1, (COLOUR + 1) & 1, false>(s, tc, acc, ctr[H]);
            } else {
                if (own) colour_plane<T, ORDER, 0, COLOUR, true>(s, tc, acc, ctr[H]);
                else colour_plane<T, ORDER, 0, COLOUR, false>(s, tc, acc, ctr[H]);
            }
        }
        if (fin) {
            tile_copy_wait<kColourAhead>();
            const T *d = fst + (p % (kColourAhead + 1)) * kColourVals * kTileThreads;
            const T ca = d[0], cb = d[kTileThreads];
            T fq[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) fq[a] = d[(2 + a) * kTileThreads];
            const unsigned q = cell(zu);
            const T Je0 = fma(ca, acc[0][0], cb * ctr[0][0]);
            T dl, kW[3];   // the true diagonal next to a face (boxes with faces only)
            relax_factors<BC>(tc.fd, g, 2 * (ring.P0 + lane) + ((COLOUR + y + zu) & 1), y, zu, true, tc.dl, tc.idW,
                              tc.iom, dl, kW);
            Y[q] = ctr[0][0] + (fq[0] - Je0) / ((ca * dl + cb) * tc.iom);
#pragma unroll
            for (int a = 0; a < 3; ++a) Y[(1 + a) * N + q] = ctr[0][1 + a] + (fq[1 + a] - acc[0][1 + a]) * kW[a];
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) {
#pragma unroll
            for (int k = 0; k < 2 * H; ++k) acc[k][a] = acc[k + 1][a];
            acc[2 * H][a] = 0;
#pragma unroll
            for (int k = 0; k < H; ++k) ctr[k][a] = ctr[k + 1][a];
        }
    }
    tile_copy_wait_all();   // no copy may land after the CTA has left (a failed wait breaks out early)
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
    TileRing<T, ORDER, BC, kRestrictSlots> ring;
    ring.setup(smem_raw, g, e, e, &tm, &tm, 0, tg, spin);
    if (ring.z0 >= ring.z1) return;
    // staging of the fetched a, b, f of both cells ([slot][value][thread]), then the odd rows' sums
    T *fst = reinterpret_cast<T *>(smem_raw + tile_ring_bytes<T, ORDER, kRestrictSlots>()) + threadIdx.x;
    T *stage = reinterpret_cast<T *>(smem_raw + tile_ring_bytes<T, ORDER, kRestrictSlots>()) +
               (kRestrictAhead + 1) * kRestrictVals * kTileThreads;   // [4 rows][32 lanes][4]
    const int nxh = g.n[0] >> 1, ny = g.n[1];
    const unsigned N = (unsigned)g.n[0] * ny * g.n[2];
    const unsigned Nc = (unsigned)gc.n[0] * gc.n[1] * gc.n[2];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, y = ring.y0 + w;
    const bool act = lane < ring.tpt;
    T acc[2 * H + 1][2][4], cp[H + 1][2], racc[4] = {0, 0, 0, 0};
#pragma unroll
    for (int b = 0; b < 2; ++b) {
#pragma unroll
        for (int k = 0; k <= 2 * H; ++k)
#pragma unroll
            for (int a = 0; a < 4; ++a) acc[k][b][a] = 0;
#pragma unroll
        for (int k = 0; k <= H; ++k) cp[k][b] = 0;
    }
    auto flush = [&](int K) {   // even warps: add the odd row's sums and write coarse plane K's cell
        if ((w & 1) == 0 && act) {
            const int I = ring.P0 + lane, J = y >> 1;
            const unsigned linc = (unsigned)I + (unsigned)gc.n[0] * ((unsigned)J + (unsigned)gc.n[1] * (unsigned)K);
            const unsigned pc = csplit ? (((I + J + K) & 1) ? Nc / 2 : 0u) + (linc >> 1) : linc;
            const T *st = stage + ((w >> 1) * 32 + lane) * 4;
#pragma unroll
            for (int a = 0; a < 4; ++a) fc[a * Nc + pc] = (racc[a] + st[a]) * (T)0.125;
        }
#pragma unroll
        for (int a = 0; a < 4; ++a) racc[a] = 0;
    };
    // the pair's two cells in plane zu: colour of the even-x cell, pair index, and their offsets
    auto cells = [&](int zu, unsigned &q0, unsigned &q1) {
        const unsigned m = (unsigned)(ring.P0 + lane) + (unsigned)nxh * ((unsigned)y + (unsigned)ny * zu);
        const int c0 = (y + zu) & 1;
        q0 = (c0 ? N / 2 : 0u) + m;
        q1 = (c0 ? 0u : N / 2) + m;
    };
    auto fetch = [&](int p) {   // a, b, f of both cells finished at iteration p, kRestrictAhead ahead
        const int zu = ring.zs + p - H;
        if (act && p < ring.NP && zu >= ring.z0) {
            unsigned q0, q1;
            cells(zu, q0, q1);
            T *d = fst + (p % (kRestrictAhead + 1)) * kRestrictVals * kTileThreads;
            tile_copy_async(d, ab + q0);
            tile_copy_async(d + kTileThreads, ab + N + q0);
            tile_copy_async(d + 2 * kTileThreads, ab + q1);
            tile_copy_async(d + 3 * kTileThreads, ab + N + q1);
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                tile_copy_async(d + (4 + a) * kTileThreads, f + a * N + q0);
                tile_copy_async(d + (8 + a) * kTileThreads, f + a * N + q1);
            }
        }
        tile_copy_commit();
    };
    for (int p = 0; p < kRestrictAhead; ++p) fetch(p);
    bool ok = ring.prologue(), failed = false;
    for (int p = 0; p < ring.NP; ++p) {
        const int zq = ring.zs + p, zu = zq - H;   // zu: the plane finished after this one
        const bool fin = zu >= ring.z0;
        fetch(p + kRestrictAhead);
        if (!ring.advance(p, ok)) { failed = true; break; }
        if (fin && (zu & 1) == 0 && zu > ring.z0) flush((zu >> 1) - 1);   // the previous coarse plane
        if (act) {
            const T *s = ring.slot(p) + (w + H) * kTileW + kTilePad + lane;
            const bool own = zq >= ring.z0 && zq < ring.z1;   // a plane of the chunk, not a halo plane
            if ((y + zq) & 1) {
                if (own) residual_plane<T, ORDER, 1, true>(s, tc, acc, cp[H]);
                else residual_plane<T, ORDER, 1, false>(s, tc, acc, cp[H]);
            } else {
                if (own) residual_plane<T, ORDER, 0, true>(s, tc, acc, cp[H]);
                else residual_plane<T, ORDER, 0, false>(s, tc, acc, cp[H]);
            }
        }
        if (act && fin) {
            tile_copy_wait<kRestrictAhead>();
            const T *d = fst + (p % (kRestrictAhead + 1)) * kRestrictVals * kTileThreads;
            const T a0 = d[0], b0 = d[kTileThreads], a1 = d[2 * kTileThreads], b1 = d[3 * kTileThreads];
            racc[0] += (d[4 * kTileThreads] - fma(a0, acc[0][0][0], b0 * cp[0][0])) +
                       (d[8 * kTileThreads] - fma(a1, acc[0][1][0], b1 * cp[0][1]));
#pragma unroll
            for (int a = 1; a < 4; ++a)
                racc[a] += (d[(4 + a) * kTileThreads] - acc[0][0][a]) + (d[(8 + a) * kTileThreads] - acc[0][1][a]);
        }
        if (fin && (zu & 1) && (w & 1)) {   // odd row of a coarse row: hand the sums to the even warp
            T *st = stage + ((w >> 1) * 32 + lane) * 4;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                st[a] = racc[a];
                racc[a] = 0;
            }
        }
#pragma unroll
        for (int b = 0; b < 2; ++b) {
#pragma unroll
            for (int a = 0; a < 4; ++a) {
#pragma unroll
                for (int k = 0; k < 2 * H; ++k) acc[k][b][a] = acc[k + 1][b][a];
                acc[2 * H][b][a] = 0;
            }
#pragma unroll
            for (int k = 0; k < H; ++k) cp[k][b] = cp[k + 1][b];
        }
    }
    if (!failed) {
        __syncthreads();
        flush((ring.z1 >> 1) - 1);
    }
    tile_copy_wait_all();   // no copy may land after the CTA has left (a failed wait breaks out early)
    ring.finish(failed, err);
}

}  // namespace ctt
