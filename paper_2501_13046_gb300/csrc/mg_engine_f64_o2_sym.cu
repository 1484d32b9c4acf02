// Instantiation of the multigrid engine for inner precision double, stencil order 2, Robin boxes with symmetry planes.
#include "mg_engine.cuh"

namespace ctt {
template mg_status engine_iteration<double, 2, BC_SYM>(mg_ctx *);
template mg_status engine_residual<double, 2, BC_SYM>(mg_ctx *, double *);
template mg_status engine_time_kernel<double, 2, BC_SYM>(mg_ctx *, int, int, float *);
template mg_status engine_prepare<double, 2, BC_SYM>(mg_ctx *);
template mg_status engine_dense_setup<double, 2, BC_SYM>(mg_ctx *);
}  // namespace ctt
