// mg_batch.cuh -- device-side control of a batched solve: one CUDA graph runs every instance's
// start, then a WHILE conditional node whose body is one IF conditional node per instance (that
// instance's outer iteration) followed by k_batch_control.  The controller reads each instance's
// scalars on the device, records its norms, its convergence round and the time it converged,
// and sets the conditions: an instance that has met its tolerance (or whose norm became non-
// finite, or that used its max_outer) drops out of the next round, and the loop ends when no
// instance is left or a bounded wait gave up.  The host launches the graph once and synchronises
// once.
#pragma once
#include <cuda_runtime.h>

#include "mg_kernels.cuh"

namespace ctt {

struct BatchCtl {
    int round;                // next round to record (round 0: the starting state)
    int timeout;              // an instance's bounded device wait gave up
    unsigned long long t0;    // %globaltimer at the start of the solve (ns)
    unsigned long long tend;  // %globaltimer at the last control step
};

struct BatchCtlArgs {
    BatchCtl *c;
    Scalars *const *scal;                    // per instance: its device scalars
    const double *tol, *ftol;                // per instance: tol, field_tol
    const int *maxo;                         // per instance: max_outer
    int *conv;                               // per instance: round it converged, -1 not yet
    int *bad;                                // per instance: 1 once a norm (or K^2) was not finite
    unsigned long long *tconv;               // per instance: %globaltimer when it converged
    const cudaGraphConditionalHandle *h;     // per instance: its IF node
    cudaGraphConditionalHandle hw;           // the WHILE node
    double *hist;                            // [maxr + 1][nb][4] norms per round
    const int *fest;                         // per instance: field_est
    double *prev;                            // per instance: [4] last relative updates (field_test)
    int nb, maxr;
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Start of a solve: clear the per-instance records and take the start time.
__global__ void k_batch_begin(BatchCtlArgs a)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.c->round = 0;
        a.c->timeout = 0;
        a.c->t0 = global_ns();
    }
    for (int b = threadIdx.x; b < a.nb; b += blockDim.x) {
        a.conv[b] = -1;
        a.bad[b] = 0;
        a.tconv[b] = 0;
        for (int k = 0; k < 4; ++k) a.prev[4 * b + k] = 0.0;
    }
}

// One control step (one CTA): record round r of every instance and set the conditions of round r + 1.
__global__ void k_batch_control(BatchCtlArgs a)
{
    __shared__ int any, late;
    const int r = a.c->round;
    if (threadIdx.x == 0) {
        any = 0;
        late = 0;
    }
    __syncthreads();
    const unsigned long long now = global_ns();
    for (int b = threadIdx.x; b < a.nb; b += blockDim.x) {
        const Scalars *s = a.scal[b];
        bool finite = isfinite(s->K2);
        double mx = 0.0;
        for (int k = 0; k < 4; ++k) {
            const double v = s->norms[k];
            if (r <= a.maxr) a.hist[((size_t)r * a.nb + b) * 4 + k] = v;
            finite = finite && isfinite(v);
            mx = fmax(mx, v);
        }
        if (s->err) late = 1;
        if (a.conv[b] < 0 && !a.bad[b]) {
            // the per-field part of the stopping test (see mg_config.field_tol, field_est)
            double change[8];
            for (int k = 0; k < 8; ++k) change[k] = s->change[k];
            const bool settled = field_test(a.ftol[b], a.fest[b], change, a.prev + 4 * b, r);
            if (!finite) {
                a.bad[b] = 1;
            } else if (mx <= a.tol[b] && settled) {
                a.conv[b] = r;
                a.tconv[b] = now;
            }
        }
        const int active = a.conv[b] < 0 && !a.bad[b] && r < a.maxo[b];
        cudaGraphSetConditional(a.h[b], active ? 1u : 0u);
        if (active) any = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (late) a.c->timeout = 1;
        cudaGraphSetConditional(a.hw, (any && !late && r < a.maxr) ? 1u : 0u);
        a.c->round = r + 1;
        a.c->tend = now;
    }
}

}  // namespace ctt
