// Instantiation of the multigrid engine for inner precision float, stencil order 4, Robin boxes with symmetry planes.
#include "mg_engine.cuh"

namespace ctt {
template mg_status engine_iteration<float, 4, BC_SYM>(mg_ctx *);
template mg_status engine_residual<float, 4, BC_SYM>(mg_ctx *, double *);
template mg_status engine_time_kernel<float, 4, BC_SYM>(mg_ctx *, int, int, float *);
template mg_status engine_prepare<float, 4, BC_SYM>(mg_ctx *);
template mg_status engine_dense_setup<float, 4, BC_SYM>(mg_ctx *);
}  // namespace ctt
