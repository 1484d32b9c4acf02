// mg_nested.cuh -- nested start of a solve: the same problem on the grid of half the size is solved
// first (recursively), and its solution, interpolated to the fine grid, is the fine iteration's
// starting state.  Only the starting state changes: the fine outer iteration, its FP64 residual
// and its tolerance are the same, so the converged result is the same discrete root.
//
// The interpolation is tricubic in cell-centred coordinates: along each axis a fine cell lies a
// quarter of a coarse cell from its parent, and takes the cubic Lagrange weights of the coarse
// cells at offsets (-1, 0, 1, 2) from the parent toward the fine cell, (-7, 105, 35, -5)/128
// (O(h^4), against O(h^2) for trilinear weights, whose interpolation error the fine Laplacian
// amplifies into a large starting residual).  Coarse cells outside the box take the level's
// boundary values (periodic wrap, the mirror image across a symmetry plane, or the Robin 1/r
// value).  The arithmetic is FP32: the result
// is only a starting state.  The weights factor per axis, so the interpolation runs as three
// one-dimensional passes over a shared-memory tile.
#pragma once
#include "mg_kernels.cuh"

namespace ctt {

// coarse = mean of the 8 children, nf plain FP64 fields (the matter sources)
static __global__ void __launch_bounds__(256) k_restrict_fields_f64(Geo g, Geo gc, const double *__restrict__ fine,
                                                             double *__restrict__ coarse, int nf)
{
    const unsigned nc0 = gc.n[0], nc1 = gc.n[1], nc2 = gc.n[2], Nc = nc0 * nc1 * nc2;
    const unsigned nf0 = g.n[0], nf1 = g.n[1], N = nf0 * nf1 * g.n[2];
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < Nc * (unsigned)nf; t += gridDim.x * blockDim.x) {
        const unsigned f = t / Nc, c = t - f * Nc;
        const unsigned I = c % nc0, J = (c / nc0) % nc1, K = c / (nc0 * nc1);
        double s = 0.0;
        for (int d = 0; d < 8; ++d) {
            const unsigned i = 2 * I + (d & 1), j = 2 * J + ((d >> 1) & 1), k = 2 * K + (d >> 2);
            s += fine[(size_t)f * N + i + nf0 * (j + nf1 * k)];
        }
        coarse[(size_t)f * Nc + c] = 0.125 * s;
    }
}

// fine X (4 plain FP64 fields) = tricubic interpolation of coarse X.  One CTA per tile of
// kPcX x kPcY x kPcZ coarse cells (2x that in fine cells), one field at a time: the tile and a halo of
// two coarse cells go to shared memory with the boundary rule applied, then three separable passes
// (x, y, z) each take the four cubic weights along one axis; the z pass writes the fine cells.
constexpr int kPcX = 8, kPcY = 8, kPcZ = 4;
constexpr int kPhX = kPcX + 4, kPhY = kPcY + 4, kPhZ = kPcZ + 4;   // with the halo of 2 on each side

__device__ __forceinline__ float cubic_tap(int c) { return c == 0 ? -7.f / 128.f : c == 1 ? 105.f / 128.f : c == 2 ? 35.f / 128.f : -5.f / 128.f; }

template <int BC>
__global__ void __launch_bounds__(256) k_prolong_cubic(Geo gc, Geo g, const double *__restrict__ xc,
                                                       double *__restrict__ xf)
{
    __shared__ float tin[kPhZ][kPhY][kPhX];
    __shared__ float tx[kPhZ][kPhY][2 * kPcX];
    __shared__ float ty[kPhZ][2 * kPcY][2 * kPcX];
    const int nc0 = gc.n[0], nc1 = gc.n[1], nc2 = gc.n[2];
    const size_t Nc = (size_t)nc0 * nc1 * nc2, N = (size_t)g.n[0] * g.n[1] * g.n[2];
    const int I0 = blockIdx.x * kPcX, J0 = blockIdx.y * kPcY, K0 = blockIdx.z * kPcZ;
    const int t = threadIdx.x;
    for (int f = 0; f < 4; ++f) {
        const double *src = xc + (size_t)f * Nc;
        for (int e = t; e < kPhX * kPhY * kPhZ; e += blockDim.x) {
            const int lx = e % kPhX, ly = (e / kPhX) % kPhY, lz = e / (kPhX * kPhY);
            const int p[3] = {I0 - 2 + lx, J0 - 2 + ly, K0 - 2 + lz};
            auto one = [&](const int c[3]) {
                int b[3];
                bool outside = false;
                int mirror = 0;
                if (BC == BC_PERIODIC) {
                    for (int a = 0; a < 3; ++a) b[a] = ((c[a] % gc.n[a]) + gc.n[a]) % gc.n[a];
                } else {   // the halo reaches at most 2 cells below the box, where the mirror applies
                    outside = bc_cell<BC>(gc, c, b, mirror);
                }
                double v = src[(size_t)b[0] + (size_t)nc0 * ((size_t)b[1] + (size_t)nc1 * b[2])];
                v = bc_signed<BC>(v, mirror, f);
                if (BC != BC_PERIODIC && outside) v *= (double)robin_ratio<float>(gc, b[0], b[1], b[2], c[0], c[1], c[2]);
                return v;
            };
            double v = 0.0;
            int q[8][3], w[8], ns = 0;
            if constexpr (BC == BC_SYM) ns = gc.extrap ? extrap_split(gc, p, q, w) : 0;
            if (ns)
                for (int s = 0; s < ns; ++s) v += w[s] * one(q[s]);
            else
                v = one(p);
            tin[lz][ly][lx] = (float)v;
        }
        __syncthreads();
        // x: fine column fx of the tile lies a quarter coarse cell from parent (fx >> 1), on side sg
        for (int e = t; e < kPhZ * kPhY * 2 * kPcX; e += blockDim.x) {
            const int fx = e % (2 * kPcX), ly = (e / (2 * kPcX)) % kPhY, lz = e / (2 * kPcX * kPhY);
            const int c0 = (fx >> 1) + 2, sg = (fx & 1) ? 1 : -1;
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < 4; ++c) s = fmaf(cubic_tap(c), tin[lz][ly][c0 + sg * (c - 1)], s);
            tx[lz][ly][fx] = s;
        }
        __syncthreads();
        for (int e = t; e < kPhZ * 2 * kPcY * 2 * kPcX; e += blockDim.x) {
            const int fx = e % (2 * kPcX), fy = (e / (2 * kPcX)) % (2 * kPcY), lz = e / (4 * kPcX * kPcY);
            const int c0 = (fy >> 1) + 2, sg = (fy & 1) ? 1 : -1;
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < 4; ++c) s = fmaf(cubic_tap(c), tx[lz][c0 + sg * (c - 1)][fx], s);
            ty[lz][fy][fx] = s;
        }
        __syncthreads();
        double *dst = xf + (size_t)f * N;
        for (int e = t; e < 2 * kPcZ * 2 * kPcY * 2 * kPcX; e += blockDim.x) {
            const int fx = e % (2 * kPcX), fy = (e / (2 * kPcX)) % (2 * kPcY), fz = e / (4 * kPcX * kPcY);
            const int i = 2 * I0 + fx, j = 2 * J0 + fy, k = 2 * K0 + fz;
            if (i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) continue;
            const int c0 = (fz >> 1) + 2, sg = (fz & 1) ? 1 : -1;
            float s = 0.f;
#pragma unroll
            for (int c = 0; c < 4; ++c) s = fmaf(cubic_tap(c), ty[c0 + sg * (c - 1)][fy][fx], s);
            dst[(size_t)i + (size_t)g.n[0] * ((size_t)j + (size_t)g.n[1] * k)] = (double)s;
        }
        __syncthreads();   // the tile buffers are refilled for the next field
    }
}

inline dim3 prolong_cubic_grid(const Geo &gc)
{
    return dim3((gc.n[0] + kPcX - 1) / kPcX, (gc.n[1] + kPcY - 1) / kPcY, (gc.n[2] + kPcZ - 1) / kPcZ);
}

}  // namespace ctt
