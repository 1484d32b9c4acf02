// mg_engine.cuh -- enqueue logic of one outer iteration (V-cycle, update, FP64 residual),
// templated on the inner precision T and the stencil order; included by mg_engine_*.cu.
#pragma once
#include "mg_common.cuh"

namespace ctt {

// Block split of a colour pass: shell blocks first, then interior-box blocks.
inline Regions smooth_regions(const Geo &g, int order, int *grid, int threads)
{
    Regions r;
    r.G = order / 2;
    long long ix = g.n[0] - 2 * r.G, iy = g.n[1] - 2 * r.G, iz = g.n[2] - 2 * r.G;
    size_t nint = (ix > 0 && iy > 0 && iz > 0) ? (size_t)ix * iy * iz / 2 : 0;
    size_t nsh = shell_count(g.n, r.G);
    // one thread per cell: blocks then sweep the box in z order, so neighbouring planes are
    // reused from L2 while they are still resident
    int bi = nint ? grid_for(nint, 1 << 24, threads) : 0;
    int bs = nsh ? grid_for(nsh, 152 * 4, threads) : 0;
    r.nblk_sh = bs;
    *grid = std::max(1, bi + bs);
    return r;
}

// Block split of residual+restriction over the coarse cells: coarse interior box [1, nc-1)^3, shell.
inline Regions restrict_regions(const Geo &gc, int *grid, int threads)
{
    Regions r;
    r.G = 1;
    long long ix = gc.n[0] - 2, iy = gc.n[1] - 2, iz = gc.n[2] - 2;
    size_t nint = (ix > 0 && iy > 0 && iz > 0) ? (size_t)ix * iy * iz : 0;
    size_t nsh = shell_count(gc.n, 1);
    int bi = nint ? grid_for(nint, 1 << 24, threads) : 0;
    int bs = nsh ? grid_for(nsh, 152 * 4, threads) : 0;
    r.nblk_sh = bs;
    *grid = std::max(1, bi + bs);
    return r;
}

// The engine is instantiated per boundary variant BC (periodic, Robin, Robin with symmetry planes;
// one translation unit each, so they compile in parallel); kernels take it as a type tag.
template <int BC, class Fn>
void with_bc(Fn &&fn)
{
    fn(std::integral_constant<int, BC>());
}

// One colour pass of the TMA-tiled kernel (X: old values, O: other colour, Y: output).
template <typename T, int ORDER, int BC>
mg_status launch_tile(mg_ctx *x, const LevelBufs &L, const TileCoef<T> &tc, const CUtensorMap &mX,
                      const CUtensorMap &mO, const T *X, const T *O, T *Y, int colour)
{
    const int grid = tile_ctas(L.geo, L.tg);
    const size_t smem = tile_smem_bytes<T, ORDER>();
    with_bc<BC>([&](auto B) {
        auto k = colour ? k_smooth_tile<T, ORDER, BC, 1> : k_smooth_tile<T, ORDER, BC, 0>;
        k<<<grid, kTileThreads, smem, x->stream>>>(mX, mO, L.geo, tc, X, O, Y, (const T *)L.f, (const T *)L.c, L.tg,
                                                   &x->scal->err, (long long)x->cfg.spin_limit);
    });
    CK(cudaGetLastError());
    return MG_OK;
}

// Residual of level l's current correction, restricted to the right-hand side of level l + 1.
template <typename T, int ORDER, int BC>
mg_status enqueue_restrict(mg_ctx *x, int l)
{
    LevelBufs &L = x->lev[l];
    LevelBufs &C = x->lev[l + 1];
    if (L.tiled) {
        const TileCoef<T> tc = make_tile_coef<T>(L.geo, x->cfg.order);
        const int grid = tile_ctas(L.geo, L.tgr);
        const size_t smem = tile_restrict_smem_bytes<T, ORDER>();
        with_bc<BC>([&](auto B) {
            k_restrict_tile<T, ORDER, decltype(B)::value><<<grid, kTileThreads, smem, x->stream>>>(
                L.tm_cur(), L.geo, tc, C.geo, (const T *)L.cur(), (const T *)L.f, (const T *)L.c, (T *)C.f, C.split,
                L.tgr, &x->scal->err, (long long)x->cfg.spin_limit);
        });
    } else {
        Coef<T> cf = make_coef<T>(L.geo, x->cfg.order);
        int rgrid = 0;
        Regions rr = restrict_regions(C.geo, &rgrid, x->threads);
        with_bc<BC>([&](auto B) {
            k_residual_restrict<T, ORDER, decltype(B)::value><<<rgrid, x->threads, 0, x->stream>>>(
                L.geo, cf, C.geo, (const T *)L.cur(), (const T *)L.f, (const T *)L.c, (T *)C.f, C.split, rr);
        });
    }
    CK(cudaGetLastError());
    return MG_OK;
}

// `sweeps` red-black sweeps on a colour-split level.  Each sweep reads the current buffer and
// writes the alternate one (red half, then black half), then the two swap roles.
template <typename T, int ORDER, int BC>
mg_status enqueue_sweeps(mg_ctx *x, int l, int sweeps)
{
    LevelBufs &L = x->lev[l];
    Coef<T> cf = make_coef<T>(L.geo, x->cfg.order, x->omega);
    const TileCoef<T> tc = make_tile_coef<T>(L.geo, x->cfg.order, x->omega);
    int grid = 0;
    Regions rg = smooth_regions(L.geo, ORDER, &grid, x->threads);
    for (int s = 0; s < sweeps; ++s) {
        const T *X = (const T *)L.cur();
        T *Y = (T *)L.alt();
        for (int colour = 0; colour < 2; ++colour) {
            const T *O = colour == 0 ? X : Y;
            if (L.tiled) {
                const CUtensorMap &mO = colour == 0 ? L.tm_cur() : L.tm_alt();
                CKS(launch_tile<T, ORDER, BC>(x, L, tc, L.tm_cur(), mO, X, O, Y, colour));
            } else {
                with_bc<BC>([&](auto B) {
                    k_smooth_colour<T, ORDER, decltype(B)::value><<<grid, x->threads, 0, x->stream>>>(
                        L.geo, cf, X, O, Y, (const T *)L.f, (const T *)L.c, colour, rg);
                });
            }
        }
        L.curB ^= 1;
    }
    CK(cudaGetLastError());
    return MG_OK;
}

template <typename T, int ORDER, int BC>
mg_status enqueue_coarse(mg_ctx *x, int l)
{
    LevelBufs &L = x->lev[l];
    const size_t tb = sizeof(T);
    const int periodic = x->cfg.bc == MG_BC_PERIODIC;
    if (x->dense) {   // exact coarse correction by the precomputed inverses
        if (x->join_pending) {
            CK(cudaStreamWaitEvent(x->stream, x->ev_join, 0));
            x->join_pending = false;
        }
        const int N = (int)L.N;
        k_dense_apply<T><<<(4 * N * 32 + 255) / 256, 256, 0, x->stream>>>(
            (const T *)x->Gpsi, x->mpsi, (const T *)x->GW, x->mw, (const T *)L.f, (T *)L.eA, N);
        CK(cudaGetLastError());
        return MG_OK;
    }
    Coef<T> cf = make_coef<T>(L.geo, x->cfg.order, x->omega);
    const size_t smem = coarse_smem_bytes(L.N, tb);
    if (smem <= kMaxCoarseSmem) {
        with_bc<BC>([&](auto B) {
            k_coarse_solve<T, ORDER, decltype(B)::value><<<1, 512, smem, x->stream>>>(
                L.geo, cf, (const T *)L.f, (const T *)L.c, (T *)L.eA, x->cfg.coarse_sweeps, periodic);
        });
        CK(cudaGetLastError());
        const size_t dsm = direct_smem_bytes(L.N, periodic, tb);
        if (dsm <= kMaxCoarseSmem) {
            with_bc<BC>([&](auto B) {
                k_coarse_psi_direct<T, ORDER, decltype(B)::value><<<1, 512, dsm, x->stream>>>(
                    L.geo, cf, (const T *)L.f, (const T *)L.c, (T *)L.eA, periodic);
            });
            CK(cudaGetLastError());
        }
        return MG_OK;
    }
    return fail(MG_ERR_UNSUPPORTED, "coarsest level too large for the one-CTA coarse solve; use more levels");
}

// One multigrid cycle on J e = f at level l (the coarsest level is solved directly).  zero: the
// level's correction starts at zero, else the cycle continues from it.  After pre-smoothing
// the residual is restricted once; the coarser level is then cycled gamma times on that right-
// hand side (1: V-cycle, 2: W-cycle), the later visits continuing from its correction, and the
// result is prolongated and post-smoothed.  The coarsest level is visited once (exact solve).
template <typename T, int ORDER, int BC>
mg_status enqueue_cycle(mg_ctx *x, int l, bool zero)
{
    const int Lc = x->nlev - 1;
    LevelBufs &L = x->lev[l];
    if (l == Lc) {   // the coarse solve writes the whole correction
        L.curB = 0;
        return enqueue_coarse<T, ORDER, BC>(x, Lc);
    }
    if (x->fused && l == Lc - 1) {   // this level and the coarsest in one CTA
        LevelBufs &C = x->lev[Lc];
        if (x->join_pending) {
            CK(cudaStreamWaitEvent(x->stream, x->ev_join, 0));
            x->join_pending = false;
        }
        const T *ein = zero ? (const T *)L.eA : (const T *)L.cur();
        size_t smem =
            fused_smem_bytes((int)L.N, (int)C.N, sizeof(T), fused_ratio_cells(L.geo, x->cfg.bc == MG_BC_ROBIN));
        const size_t gbytes = (size_t)10 * C.N * C.N * sizeof(T);   // Nc^2 + (3 Nc)^2 dense entries
        const int gsm = smem + gbytes <= kMaxCoarseSmem ? 1 : 0;
        if (gsm) smem += gbytes;
        with_bc<BC>([&](auto B) {
            k_coarse_cycle<T, ORDER, decltype(B)::value><<<1, fused_threads<T>(), smem, x->stream>>>(
                L.geo, make_coef<T>(L.geo, x->cfg.order, x->omega), C.geo, (const T *)L.f, (const T *)L.c, ein,
                (T *)L.eA, zero ? 1 : 0, x->cfg.nu_pre, x->cfg.nu_post, (const T *)x->Gpsi, x->mpsi,
                (const T *)x->GW, x->mw, gsm);
        });
        CK(cudaGetLastError());
        L.curB = 0;
        return MG_OK;
    }
    if (zero) {
        L.curB = 0;
        CK(cudaMemsetAsync(L.eA, 0, 4 * L.N * sizeof(T), x->stream));
    }
    CKS(enqueue_sweeps<T, ORDER, BC>(x, l, x->cfg.nu_pre));
    LevelBufs &C = x->lev[l + 1];
    CKS(enqueue_restrict<T, ORDER, BC>(x, l));
    const int visits = l + 1 == Lc ? 1 : x->gamma;
    for (int v = 0; v < visits; ++v) CKS(enqueue_cycle<T, ORDER, BC>(x, l + 1, v == 0));
    with_bc<BC>([&](auto B) {
        k_prolong_add<T, decltype(B)::value><<<grid_for(L.N, 1 << 24, x->threads), x->threads, 0, x->stream>>>(
            L.geo, C.geo, (const T *)C.cur(), (T *)L.cur(), C.split);
    });
    CK(cudaGetLastError());
    return enqueue_sweeps<T, ORDER, BC>(x, l, x->cfg.nu_post);
}

template <typename T, int ORDER, int BC>
mg_status enqueue_vcycle(mg_ctx *x, bool first) { return enqueue_cycle<T, ORDER, BC>(x, 0, first); }

// FP64 residual pass 1 (pass A: q, div W; pass B: R and the integrability sums), then the
// final reduction of the sums.
// Pass B finishes the outer scalars in its last block (sums, K^2, m_i).
inline OuterFin outer_fin(mg_ctx *x)
{
    return OuterFin{x->scal, x->cfg.k_mode == MG_K_INTEGRABILITY, x->cfg.bc == MG_BC_PERIODIC, x->cfg.K * x->cfg.K};
}

template <int ORDER, int BC>
mg_status enqueue_outer_pass1(mg_ctx *x)
{
    LevelBufs &L0 = x->lev[0];
    Coef<double> cf = make_coef<double>(L0.geo, x->cfg.order);
    OuterCoef oc = make_outer_coef(L0.geo, x->cfg.order);
    int gb = 0;
    Regions rg = outer_regions(L0.geo, ORDER, x->cfg.bc == MG_BC_ROBIN, &gb);
    with_bc<BC>([&](auto B) {
        k_outer_div<ORDER, decltype(B)::value><<<grid_for(x->N, 1 << 24), kThreads, 0, x->stream>>>(L0.geo, oc, x->X,
                                                                                                      x->D);
        k_outer_pass1q<ORDER, decltype(B)::value><<<gb, kThreads, 0, x->stream>>>(L0.geo, cf, oc, x->X, x->D, x->SRC,
                                                                                  x->R, x->partial, rg, outer_fin(x));
    });
    CK(cudaGetLastError());
    return MG_OK;
}

// Outer residual.  HM != nullptr: write H, M instead of the inner rhs/coefficient.
template <typename T, int ORDER, int BC>
mg_status enqueue_residual(mg_ctx *x, double *HM)
{
    LevelBufs &L0 = x->lev[0];
    CKS(enqueue_outer_pass1<ORDER, BC>(x));
    int g1 = grid_for(x->N, kRedBlocks);
    k_outer_pass2<T><<<g1, kThreads, 0, x->stream>>>(L0.geo, x->X, x->R, x->SRC, x->scal, (T *)L0.f, (T *)L0.c, HM,
                                                     x->partial, L0.split, 1);
    CK(cudaGetLastError());
    // the scalars go to the host, unless a device-side controller reads them (device-paced batch)
    if (!x->device_paced) CK(cudaMemcpyAsync(x->host_scal, x->scal, sizeof(Scalars), cudaMemcpyDeviceToHost, x->stream));
    return MG_OK;
}

// Shared memory of a one-CTA Gauss-Jordan inversion of order m in type C (0: the matrix stays in
// global memory, which the kernel then uses in place).
template <typename C>
inline size_t gj_smem(int m)
{
    const size_t b = gj_scratch_elems(m) * sizeof(C);
    return b <= kMaxCoarseSmem ? b : 0;
}

// Inverse of the coarsest psi row for this outer iteration (its coefficients were just restricted),
// on a parallel branch: the one-CTA elimination overlaps the first cycle's descent, and the first
// coarse solve of the iteration waits for it (enqueue_coarse).
template <typename T, int ORDER, int BC>
mg_status enqueue_dense_psi_inverse(mg_ctx *x)
{
    LevelBufs &C = x->lev[x->nlev - 1];
    const int periodic = x->cfg.bc == MG_BC_PERIODIC;
    Coef<T> cf = make_coef<T>(C.geo, x->cfg.order);
    const size_t sm = gj_smem<T>(x->mpsi);
    CK(cudaEventRecord(x->ev_fork, x->stream));
    CK(cudaStreamWaitEvent(x->side, x->ev_fork, 0));
    with_bc<BC>([&](auto B) {
        k_dense_psi_assemble<T, T, ORDER, decltype(B)::value><<<1, 512, 0, x->side>>>(C.geo, cf, (const T *)C.c,
                                                                                    (T *)x->gj, periodic);
    });
    k_gauss_jordan<T, T><<<1, 1024, sm, x->side>>>((T *)x->gj, x->mpsi, sm > 0, (T *)x->Gpsi);
    CK(cudaGetLastError());
    CK(cudaEventRecord(x->ev_join, x->side));
    x->join_pending = true;
    return MG_OK;
}

// Inverse of the coarsest W rows, once per context (FP64 elimination, stored as T).
template <typename T, int ORDER, int BC>
mg_status engine_dense_setup(mg_ctx *x)
{
    LevelBufs &C = x->lev[x->nlev - 1];
    const int periodic = x->cfg.bc == MG_BC_PERIODIC;
    const int N = (int)C.N;
    Coef<double> cf = make_coef<double>(C.geo, x->cfg.order);
    CK(cudaMemsetAsync(x->gj, 0, gj_scratch_elems(x->mw) * sizeof(double), x->stream));
    with_bc<BC>([&](auto B) {
        k_dense_w_assemble<double, double, ORDER, decltype(B)::value><<<3 * N + 1, 256, 4 * N * sizeof(double),
                                                                        x->stream>>>(C.geo, cf, (double *)x->gj,
                                                                                     periodic);
    });
    const size_t sm = gj_smem<double>(x->mw);
    k_gauss_jordan<double, T><<<1, 1024, sm, x->stream>>>((double *)x->gj, x->mw, sm > 0, (T *)x->GW);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(x->stream));
    return MG_OK;
}

template <typename T, int ORDER, int BC>
mg_status enqueue_iteration(mg_ctx *x)
{
    for (int l = 1; l < x->nlev; ++l) {
        LevelBufs &C = x->lev[l];
        k_restrict_mean<T><<<grid_for(C.N), kThreads, 0, x->stream>>>(x->lev[l - 1].geo, C.geo,
                                                                       (const T *)x->lev[l - 1].c, (T *)C.c, 2, C.split);
    }
    CK(cudaGetLastError());
    if (x->dense) CKS(enqueue_dense_psi_inverse<T, ORDER, BC>(x));
    LevelBufs &L0 = x->lev[0];
    if (x->zsolve) {   // z = L^-1 (dF/dK^2) in the inner form: the cycles on zrhs, its means
        void *f = L0.f;
        L0.f = x->zrhs;
        mg_status st = MG_OK;
        for (int cyc = 0; cyc < x->cfg.inner_cycles && st == MG_OK; ++cyc) st = enqueue_vcycle<T, ORDER, BC>(x, cyc == 0);
        L0.f = f;
        CKS(st);
        CK(cudaMemcpyAsync(x->zbuf, L0.cur(), 4 * x->N * sizeof(T), cudaMemcpyDeviceToDevice, x->stream));
        k_sum4<T><<<grid_for(x->N, kRedBlocks), kThreads, 0, x->stream>>>((const T *)x->zbuf, x->N, x->partial,
                                                                        x->scal->zmean, &x->scal->ticket[2]);
        CK(cudaGetLastError());
        return MG_OK;
    }
    for (int cyc = 0; cyc < x->cfg.inner_cycles; ++cyc) CKS(enqueue_vcycle<T, ORDER, BC>(x, cyc == 0));
    int periodic = x->cfg.bc == MG_BC_PERIODIC;
    if (periodic) {
        int g = grid_for(x->N, kRedBlocks);
        k_sum4<T><<<g, kThreads, 0, x->stream>>>((const T *)L0.cur(), x->N, x->partial, x->scal->emean,
                                                 &x->scal->ticket[2]);
    }
    // the size of the update is reduced only for the per-field stopping test (field_tol > 0)
    const bool sized = x->cfg.field_tol > 0.0;
    k_update<T><<<sized ? grid_for(x->N, kRedBlocks) : grid_for(x->N), kThreads, 0, x->stream>>>(
        L0.geo, x->X, (const T *)L0.cur(), x->N, periodic ? x->scal->emean : nullptr, L0.split, x->partial,
        sized ? x->scal : nullptr, x->zbuf && periodic ? (const T *)x->zbuf : nullptr, x->scal->zmean);
    CK(cudaGetLastError());
    return enqueue_residual<T, ORDER, BC>(x, nullptr);
}

template <typename T, int ORDER, int BC>
mg_status engine_iteration(mg_ctx *x) { return enqueue_iteration<T, ORDER, BC>(x); }

// Kernel attributes, set once at context creation (never inside a stream capture).
template <typename T, int ORDER, int BC>
mg_status engine_prepare(mg_ctx *x)
{
    mg_status st = MG_OK;
    with_bc<BC>([&](auto B) {
        if (cudaFuncSetAttribute(k_coarse_solve<T, ORDER, decltype(B)::value>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxCoarseSmem) != cudaSuccess ||
            cudaFuncSetAttribute(k_coarse_psi_direct<T, ORDER, decltype(B)::value>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxCoarseSmem) != cudaSuccess)
            st = fail(MG_ERR_CUDA, "cudaFuncSetAttribute(coarse kernels)");
        if (cudaFuncSetAttribute(k_coarse_cycle<T, ORDER, decltype(B)::value>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxCoarseSmem) != cudaSuccess)
            st = fail(MG_ERR_CUDA, "cudaFuncSetAttribute(k_coarse_cycle)");
        if (cudaFuncSetAttribute(k_gauss_jordan<T, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMaxCoarseSmem) != cudaSuccess ||
            cudaFuncSetAttribute(k_gauss_jordan<double, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kMaxCoarseSmem) != cudaSuccess)
            st = fail(MG_ERR_CUDA, "cudaFuncSetAttribute(k_gauss_jordan)");
        if (cudaFuncSetAttribute(k_smooth_tile<T, ORDER, BC, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile_smem_bytes<T, ORDER>()) != cudaSuccess ||
            cudaFuncSetAttribute(k_smooth_tile<T, ORDER, BC, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile_smem_bytes<T, ORDER>()) != cudaSuccess ||
            cudaFuncSetAttribute(k_restrict_tile<T, ORDER, BC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)tile_restrict_smem_bytes<T, ORDER>()) != cudaSuccess)
            st = fail(MG_ERR_CUDA, "cudaFuncSetAttribute(tiled kernels)");
    });
    return st;
}

// Back-to-back launches of one kernel between events (measurement aid).
template <typename T, int ORDER, int BC>
mg_status engine_time_kernel(mg_ctx *x, int which, int reps, float *ms)
{
    LevelBufs &L = x->lev[0];
    Coef<T> cf = make_coef<T>(L.geo, x->cfg.order);
    CK(cudaEventRecord(x->ev0, x->stream));
    for (int r = 0; r < reps; ++r) {
        if (which == 0) {
            if (!L.split) return fail(MG_ERR_INVALID_ARG, "one-level hierarchy has no global smoother");
            if (L.tiled) {
                const TileCoef<T> tc = make_tile_coef<T>(L.geo, x->cfg.order, x->omega);
                CKS(launch_tile<T, ORDER, BC>(x, L, tc, L.tmA, L.tmA, (const T *)L.eA, (const T *)L.eA, (T *)L.eB, r & 1));
                continue;
            }
            int grid = 0;
            Regions rg = smooth_regions(L.geo, ORDER, &grid, x->threads);
            with_bc<BC>([&](auto B) {
                k_smooth_colour<T, ORDER, decltype(B)::value><<<grid, x->threads, 0, x->stream>>>(
                    L.geo, cf, (const T *)L.eA, (const T *)L.eA, (T *)L.eB, (const T *)L.f, (const T *)L.c, r & 1, rg);
            });
        } else if (which == 1) {
            if (x->nlev < 2) return fail(MG_ERR_INVALID_ARG, "one-level hierarchy has no restriction");
            const int keep = L.curB;
            L.curB = 0;   // residual of eA
            CKS(enqueue_restrict<T, ORDER, BC>(x, 0));
            L.curB = keep;
        } else if (which == 2) {
            CKS(enqueue_outer_pass1<ORDER, BC>(x));
        } else {   // pass B alone (reads pass A's q, div W from the last residual evaluation)
            Coef<double> cd = make_coef<double>(L.geo, x->cfg.order);
            OuterCoef oc = make_outer_coef(L.geo, x->cfg.order);
            int gb = 0;
            Regions rg = outer_regions(L.geo, ORDER, x->cfg.bc == MG_BC_ROBIN, &gb);
            with_bc<BC>([&](auto B) {
                k_outer_pass1q<ORDER, decltype(B)::value><<<gb, kThreads, 0, x->stream>>>(
                    L.geo, cd, oc, x->X, x->D, x->SRC, x->R, x->partial, rg, OuterFin{nullptr, 0, 0, 0.0});
            });
        }
    }
    CK(cudaGetLastError());
    CK(cudaEventRecord(x->ev1, x->stream));
    CK(cudaEventSynchronize(x->ev1));
    CK(cudaEventElapsedTime(ms, x->ev0, x->ev1));
    return MG_OK;
}

template <typename T, int ORDER, int BC>
mg_status engine_residual(mg_ctx *x, double *HM) { return enqueue_residual<T, ORDER, BC>(x, HM); }

}  // namespace ctt
