// Instantiation of the multigrid engine for inner precision float, stencil order 2, Robin boxes.
#include "mg_engine.cuh"

namespace ctt {
template mg_status engine_iteration<float, 2, BC_ROBIN>(mg_ctx *);
template mg_status engine_residual<float, 2, BC_ROBIN>(mg_ctx *, double *);
template mg_status engine_time_kernel<float, 2, BC_ROBIN>(mg_ctx *, int, int, float *);
template mg_status engine_prepare<float, 2, BC_ROBIN>(mg_ctx *);
template mg_status engine_dense_setup<float, 2, BC_ROBIN>(mg_ctx *);
}  // namespace ctt
