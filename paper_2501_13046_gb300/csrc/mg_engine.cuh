// mg_engine.cuh -- enqueue logic of one outer iteration (V-cycle, update, FP64 residual),
// templated on the inner precision T and the stencil order; included by mg_engine_*.cu.
#pragma once
#include "mg_common.cuh"

namespace ctt {

template <class Fn>
void dispatch_bc(int bc, Fn &&fn)
{
    if (bc == MG_BC_PERIODIC) fn(std::integral_constant<int, BC_PERIODIC>());
    else fn(std::integral_constant<int, BC_ROBIN>());
}

template <typename T, int ORDER>
mg_status enqueue_sweeps(mg_ctx *x, int l, int sweeps)
{
    LevelBufs &L = x->lev[l];
    Coef<T> cf = make_coef<T>(L.geo, x->cfg.order);
    size_t pairs = L.N / 2;
    int grid = grid_for(pairs);
    for (int s = 0; s < sweeps; ++s)
        for (int colour = 0; colour < 2; ++colour) {
            const T *ein = (const T *)(colour == 0 ? L.eA : L.eB);
            T *eout = (T *)(colour == 0 ? L.eB : L.eA);
            dispatch_bc(x->cfg.bc, [&](auto B) {
                k_smooth_colour<T, ORDER, decltype(B)::value><<<grid, kThreads, 0, x->stream>>>(
                    L.geo, cf, ein, eout, (const T *)L.f, (const T *)L.c, colour);
            });
        }
    CK(cudaGetLastError());
    return MG_OK;
}

template <typename T, int ORDER>
mg_status enqueue_coarse(mg_ctx *x, int l)
{
    LevelBufs &L = x->lev[l];
    const size_t tb = sizeof(T);
    const int periodic = x->cfg.bc == MG_BC_PERIODIC;
    Coef<T> cf = make_coef<T>(L.geo, x->cfg.order);
    const size_t smem = coarse_smem_bytes(L.N, tb);
    if (smem <= kMaxCoarseSmem) {
        dispatch_bc(x->cfg.bc, [&](auto B) {
            k_coarse_solve<T, ORDER, decltype(B)::value><<<1, 512, smem, x->stream>>>(
                L.geo, cf, (const T *)L.f, (const T *)L.c, (T *)L.eA, x->cfg.coarse_sweeps, periodic);
        });
        CK(cudaGetLastError());
        const size_t dsm = direct_smem_bytes(L.N, periodic, tb);
        if (dsm <= kMaxCoarseSmem) {
            dispatch_bc(x->cfg.bc, [&](auto B) {
                k_coarse_psi_direct<T, ORDER, decltype(B)::value><<<1, 512, dsm, x->stream>>>(
                    L.geo, cf, (const T *)L.f, (const T *)L.c, (T *)L.eA, periodic);
            });
            CK(cudaGetLastError());
        }
        return MG_OK;
    }
    // coarsest level too large for one CTA: global colour passes, then the periodic mean projection
    if (L.geo.n[0] % 2 != 0) return fail(MG_ERR_UNSUPPORTED, "coarsest level too large for one CTA and odd in x");
    CK(cudaMemsetAsync(L.eA, 0, 4 * L.N * tb, x->stream));
    CKS(enqueue_sweeps<T, ORDER>(x, l, x->cfg.coarse_sweeps));
    if (periodic) {
        int g = grid_for(L.N, kRedBlocks);
        k_sum4<T><<<g, kThreads, 0, x->stream>>>((const T *)L.eA, L.N, x->partial);
        k_finalize_sum<4><<<1, 256, 0, x->stream>>>(x->partial, g, x->scal->emean);
        k_sub_mean4<T><<<grid_for(L.N), kThreads, 0, x->stream>>>((T *)L.eA, L.N, x->scal->emean);
        CK(cudaGetLastError());
    }
    return MG_OK;
}

template <typename T, int ORDER>
mg_status enqueue_vcycle(mg_ctx *x)
{
    const int Lc = x->nlev - 1;
    size_t tb = sizeof(T);
    for (int l = 0; l < Lc; ++l) {
        LevelBufs &L = x->lev[l];
        CK(cudaMemsetAsync(L.eA, 0, 4 * L.N * tb, x->stream));
        CKS(enqueue_sweeps<T, ORDER>(x, l, x->cfg.nu_pre));
        LevelBufs &C = x->lev[l + 1];
        Coef<T> cf = make_coef<T>(L.geo, x->cfg.order);
        dispatch_bc(x->cfg.bc, [&](auto B) {
            k_residual_restrict<T, ORDER, decltype(B)::value><<<grid_for(C.N), kThreads, 0, x->stream>>>(
                L.geo, cf, C.geo, (const T *)L.eA, (const T *)L.f, (const T *)L.c, (T *)C.f);
        });
        CK(cudaGetLastError());
    }
    CKS(enqueue_coarse<T, ORDER>(x, Lc));
    for (int l = Lc - 1; l >= 0; --l) {
        LevelBufs &L = x->lev[l];
        LevelBufs &C = x->lev[l + 1];
        if (x->cfg.bc == MG_BC_PERIODIC)
            k_prolong_add<T, BC_PERIODIC><<<grid_for(C.N), kThreads, 0, x->stream>>>(C.geo, (const T *)C.eA, (T *)L.eA);
        else
            k_prolong_add<T, BC_ROBIN><<<grid_for(C.N), kThreads, 0, x->stream>>>(C.geo, (const T *)C.eA, (T *)L.eA);
        CK(cudaGetLastError());
        CKS(enqueue_sweeps<T, ORDER>(x, l, x->cfg.nu_post));
    }
    return MG_OK;
}

// Outer residual.  HM != nullptr: write H, M instead of the inner rhs/coefficient.
template <typename T, int ORDER>
mg_status enqueue_residual(mg_ctx *x, double *HM)
{
    LevelBufs &L0 = x->lev[0];
    Coef<double> cf = make_coef<double>(L0.geo, x->cfg.order);
    int g1 = grid_for(x->N, kRedBlocks);
    dispatch_bc(x->cfg.bc, [&](auto B) {
        k_outer_pass1<ORDER, decltype(B)::value><<<g1, kThreads, 0, x->stream>>>(L0.geo, cf, x->X, x->SRC,
                                                                                              x->R, x->partial);
    });
    k_finalize_sum<5><<<1, 256, 0, x->stream>>>(x->partial, g1, x->scal->sums);
    double K2f = x->cfg.K * x->cfg.K;
    k_outer_scalars<<<1, 1, 0, x->stream>>>(x->scal, x->N, x->cfg.k_mode == MG_K_INTEGRABILITY, K2f,
                                           x->cfg.bc == MG_BC_PERIODIC);
    k_outer_pass2<T><<<g1, kThreads, 0, x->stream>>>(L0.geo, x->X, x->R, x->scal, (T *)L0.f, (T *)L0.c, HM,
                                                     x->partial);
    k_finalize_max<4><<<1, 256, 0, x->stream>>>(x->partial, g1, x->scal->norms);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(x->host_scal, x->scal, sizeof(Scalars), cudaMemcpyDeviceToHost, x->stream));
    return MG_OK;
}

template <typename T, int ORDER>
mg_status enqueue_iteration(mg_ctx *x)
{
    for (int l = 1; l < x->nlev; ++l) {
        LevelBufs &C = x->lev[l];
        k_restrict_mean<T><<<grid_for(C.N), kThreads, 0, x->stream>>>(C.geo, (const T *)x->lev[l - 1].c, (T *)C.c, 2);
    }
    CK(cudaGetLastError());
    CKS(enqueue_vcycle<T, ORDER>(x));
    int periodic = x->cfg.bc == MG_BC_PERIODIC;
    LevelBufs &L0 = x->lev[0];
    if (periodic) {
        int g = grid_for(x->N, kRedBlocks);
        k_sum4<T><<<g, kThreads, 0, x->stream>>>((const T *)L0.eA, x->N, x->partial);
        k_finalize_sum<4><<<1, 256, 0, x->stream>>>(x->partial, g, x->scal->emean);
    }
    k_update<T><<<grid_for(x->N), kThreads, 0, x->stream>>>(x->X, (const T *)L0.eA, x->N, x->scal->emean, periodic);
    CK(cudaGetLastError());
    return enqueue_residual<T, ORDER>(x, nullptr);
}

template <typename T, int ORDER>
mg_status engine_iteration(mg_ctx *x) { return enqueue_iteration<T, ORDER>(x); }

// Kernel attributes, set once at context creation (never inside a stream capture).
template <typename T, int ORDER>
mg_status engine_prepare(mg_ctx *x)
{
    mg_status st = MG_OK;
    dispatch_bc(x->cfg.bc, [&](auto B) {
        if (cudaFuncSetAttribute(k_coarse_solve<T, ORDER, decltype(B)::value>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxCoarseSmem) != cudaSuccess ||
            cudaFuncSetAttribute(k_coarse_psi_direct<T, ORDER, decltype(B)::value>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxCoarseSmem) != cudaSuccess)
            st = fail(MG_ERR_CUDA, "cudaFuncSetAttribute(coarse kernels)");
    });
    return st;
}

// Back-to-back launches of one kernel between events (measurement aid).
template <typename T, int ORDER>
mg_status engine_time_kernel(mg_ctx *x, int which, int reps, float *ms)
{
    LevelBufs &L = x->lev[0];
    Coef<T> cf = make_coef<T>(L.geo, x->cfg.order);
    CK(cudaEventRecord(x->ev0, x->stream));
    for (int r = 0; r < reps; ++r) {
        if (which == 0) {
            int grid = grid_for(L.N / 2);
            dispatch_bc(x->cfg.bc, [&](auto B) {
                k_smooth_colour<T, ORDER, decltype(B)::value><<<grid, kThreads, 0, x->stream>>>(
                    L.geo, cf, (const T *)L.eA, (T *)L.eB, (const T *)L.f, (const T *)L.c, r & 1);
            });
        } else if (which == 1) {
            if (x->nlev < 2) return fail(MG_ERR_INVALID_ARG, "one-level hierarchy has no restriction");
            LevelBufs &Cl = x->lev[1];
            dispatch_bc(x->cfg.bc, [&](auto B) {
                k_residual_restrict<T, ORDER, decltype(B)::value><<<grid_for(Cl.N), kThreads, 0, x->stream>>>(
                    L.geo, cf, Cl.geo, (const T *)L.eA, (const T *)L.f, (const T *)L.c, (T *)Cl.f);
            });
        } else {
            Coef<double> cd = make_coef<double>(L.geo, x->cfg.order);
            int g1 = grid_for(x->N, kRedBlocks);
            dispatch_bc(x->cfg.bc, [&](auto B) {
                k_outer_pass1<ORDER, decltype(B)::value><<<g1, kThreads, 0, x->stream>>>(L.geo, cd, x->X, x->SRC, x->R,
                                                                                         x->partial);
            });
        }
    }
    CK(cudaGetLastError());
    CK(cudaEventRecord(x->ev1, x->stream));
    CK(cudaEventSynchronize(x->ev1));
    CK(cudaEventElapsedTime(ms, x->ev0, x->ev1));
    return MG_OK;
}

template <typename T, int ORDER>
mg_status engine_residual(mg_ctx *x, double *HM) { return enqueue_residual<T, ORDER>(x, HM); }

}  // namespace ctt
