// Instantiation of the multigrid engine for inner precision double, stencil order 2.
#include "mg_engine.cuh"

namespace ctt {
template mg_status engine_iteration<double, 2>(mg_ctx *);
template mg_status engine_residual<double, 2>(mg_ctx *, double *);
template mg_status engine_time_kernel<double, 2>(mg_ctx *, int, int, float *);
template mg_status engine_prepare<double, 2>(mg_ctx *);
template mg_status engine_dense_setup<double, 2>(mg_ctx *);

mg_status engine_project_gauge(mg_ctx *x)
{
    if (x->cfg.bc != MG_BC_PERIODIC) return MG_OK;
    int g = grid_for(x->N, kRedBlocks);
    k_sum4<double><<<g, kThreads, 0, x->stream>>>(x->X, x->N, x->partial, x->scal->emean, &x->scal->ticket[2]);
    k_sub_mean4<double><<<grid_for(x->N), kThreads, 0, x->stream>>>(x->X, x->N, x->scal->emean);
    CK(cudaGetLastError());
    return MG_OK;
}
}  // namespace ctt
