/*
 * ctt_unet.h -- C ABI of the learned warm start (libctt_mg.so): a BF16 3-D U-Net whose
 * convolutions run as implicit GEMMs on the 5th-generation tensor cores (tcgen05, FP32
 * accumulation in tensor memory), and the glue kernels of its training (pooling, upsampling,
 * 1x1 head, MSE loss, gradients, Adam).  Not in the paper: the learned warm start and its
 * training are an addition to its multigrid solver.  Plain multigrid from psi = 1 remains the
 * fallback, and the multigrid solve decides every accepted result.
 *
 * Conventions:
 *   - Activations are NDHWC BF16 (x fastest, a voxel's channels contiguous).  A tensor may be
 *     the channel slice [c0, c0 + C) of a buffer with cs channels per voxel; cs and c0 must be
 *     multiples of 8 (16-byte rows), channel counts multiples of 16 for the tensor-core paths.
 *   - Grids are periodic (circular padding) with n0 * n1 * n2 a multiple of 128.
 *   - Conv weights: FP32 master [27][Cout][Cin], tap = (dz+1)*9 + (dy+1)*3 + (dx+1);
 *     unet_pack_weights makes the BF16 operand of the forward pass (mode 0) or of the input
 *     gradient (mode 1: taps flipped, Cin and Cout exchanged).
 *   - All pointers are device pointers; all work is issued on `stream`; nothing synchronises
 *     except where stated.  err: device int set to 1 if a bounded device-side wait gave up
 *     (the kernel then frees its tensor memory and returns); the caller checks it.
 *   - Return value: 0 on success, 1 invalid argument or unsupported shape, 3 CUDA error.
 */
#ifndef CTT_UNET_H
#define CTT_UNET_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* y = act(conv3x3x3_circular(x, w) + bias); act = ReLU when relu != 0.  bias may be NULL.
 * ws: optional FP32 device workspace of ws_bytes bytes (16-byte aligned), owned by the caller and
 * used by this call only while its kernels run (one workspace per stream).  With ws, grids with
 * fewer than two 128-voxel tiles per SM split the 27 taps over groups of CTAs and add the
 * groups' FP32 partial sums in a fixed order (deterministic); with ws == NULL every grid runs
 * the unsplit kernels.  The two forms round differently (FP32 summation order), each is
 * deterministic.  ws_bytes below unet_conv3d_fwd_workspace() for the shape returns 1, and so does
 * a side of 1024 or more. */
int unet_conv3d_fwd(const void *x, int xcs, int xc0, const void *w_bf16, const float *bias, void *y, int ycs,
                    int yc0, int n0, int n1, int n2, int cin, int cout, int relu, float *ws, size_t ws_bytes,
                    long long spin_limit, int *err, void *stream);

/* Workspace bytes unet_conv3d_fwd needs for its split form on an n0 x n1 x n2 grid with cout
 * output channels (0: that grid runs unsplit; also 0 for an unsupported shape). */
size_t unet_conv3d_fwd_workspace(int n0, int n1, int n2, int cout);

/* dw[27][cout][cin] += sum_v dy[v][co] x[v + tap][ci]  (dw FP32, accumulated; zero it first). */
int unet_conv3d_wgrad(const void *x, int xcs, int xc0, const void *dy, int dcs, int dc0, float *dw, int n0, int n1,
                      int n2, int cin, int cout, long long spin_limit, int *err, void *stream);

/* BF16 operand from FP32 master weights [27][cout][cin]: mode 0 -> [27][cout][cin];
 * mode 1 (input gradient) -> [27][cin][cout] with tap t read from 26 - t. */
int unet_pack_weights(const float *w, int cin, int cout, int mode, void *out_bf16, void *stream);

/* 2x2x2 average pooling (y coarse) and its adjoint (dx fine; accumulate != 0 adds into dx).
 * unet_avgpool2 and unet_upsample2 move 8 channels (16 bytes) per thread: c, the channel strides
 * and offsets must be multiples of 8 (else 1). */
int unet_avgpool2(const void *x, int xcs, int xc0, void *y, int ycs, int yc0, int c, int n0, int n1, int n2,
                  void *stream);
int unet_avgpool2_bwd(const void *dy, int dcs, int dc0, void *dx, int xcs, int xc0, int c, int n0, int n1, int n2,
                      int accumulate, void *stream);
/* nearest 2x upsampling (n = coarse size) and its adjoint (sum over the 8 children). */
int unet_upsample2(const void *x, int xcs, int xc0, void *y, int ycs, int yc0, int c, int n0, int n1, int n2,
                   void *stream);
int unet_upsample2_bwd(const void *dy, int dcs, int dc0, void *dx, int xcs, int xc0, int c, int n0, int n1, int n2,
                       void *stream);
/* dy *= (y > 0) elementwise on a channel slice (ReLU adjoint, y the ReLU output). */
int unet_relu_bwd(void *dy, int dcs, int dc0, const void *y, int ycs, int yc0, int c, long long nvox, void *stream);
/* db[c] += sum_v dy[v][c] (db FP32). */
int unet_bias_grad(const void *dy, int dcs, int dc0, float *db, int c, long long nvox, void *stream);

/* 1x1 head: out[v][o] = b[o] + sum_c w[o][c] x[v][c], out FP32 with cout channels (<= 8). */
int unet_head_fwd(const void *x, int xcs, int xc0, int cin, const float *w, const float *b, float *out, int cout,
                  long long nvox, void *stream);
/* head adjoint: dx (BF16 slice) = w^T dout; dw += dout x^T; db += sum dout. */
int unet_head_bwd(const void *x, int xcs, int xc0, int cin, const float *w, const float *dout, int cout,
                  void *dx, int dxcs, int dxc0, float *dw, float *db, long long nvox, void *stream);
/* loss += sum (out - t)^2 / count; dout = 2 (out - t) / count, count = nvox * c (FP32 throughout). */
int unet_mse(const float *out, const float *target, float *dout, float *loss, int c, long long nvox, void *stream);
/* Adam on FP32 parameters, step t >= 1. */
int unet_adam(float *p, const float *g, float *m, float *v, long long n, float lr, float b1, float b2, float eps,
              int t, void *stream);

/* Network input, 16 BF16 channels: [(rho - <rho>) s_rho, S_x s_S, S_y s_S, S_z s_S, K s_K, 0 ...],
 * rho = rho0 + rho2 (FP64 device arrays, rho2 may be NULL).  <rho> is computed on the device.
 * K = NaN: the value known before solving, K = -sqrt(24 pi <rho>) (periodic integrability at
 * psi = 1, W = 0), also computed on the device.  scratch_mean: device array of at least 264
 * doubles (means and the block partials of their deterministic reduction). */
int unet_pack_input(const double *rho0, const double *rho2, const double *S, double K, float s_rho, float s_S,
                    float s_K, void *x16, long long nvox, double *scratch_mean, void *stream);
/* Network output (FP32, 4 channels) to the solver's initial guess: u = out0 s_u (zero mean on
 * periodic boxes), W_i = out_i s_W (zero mean), FP64.  scratch_mean as for unet_pack_input. */
int unet_unpack_output(const float *out4, float s_u, float s_W, double *u, double *W, long long nvox,
                       double *scratch_mean, void *stream);
/* Mean of the 8 children of nfields contiguous FP64 fields, (2 m)^3 -> m^3 (m = m0 x m1 x m2). */
int unet_restrict2_fields(const double *fine, double *coarse, int nfields, int m0, int m1, int m2, void *stream);
/* Cell-centred trilinear interpolation (3/4, 1/4 per axis, periodic) of nfields contiguous FP64
 * fields, m^3 -> (2 m)^3: runs the network at its training resolution for finer grids. */
int unet_prolong2_fields(const double *coarse, double *fine, int nfields, int m0, int m1, int m2, void *stream);
/* Training target from a solution: t = (u / s_u, W_x / s_W, W_y / s_W, W_z / s_W), FP32 4 channels. */
int unet_pack_target(const double *u, const double *W, float s_u, float s_W, float *t4, long long nvox, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* CTT_UNET_H */
