/*
 * ctt_mg.h -- C ABI of the GB300 CTT constraint multigrid library (libctt_mg.so).
 *
 * The library solves the Hamiltonian and momentum constraints of numerical
 * relativity initial data (GRTresna, arXiv:2501.13046, Summary, eq:Ham and
 * eq:Mom), given the matter projections rho and S_i, in the conformal
 * transverse-traceless form with a conformally flat metric and constant K:
 *
 *   F_psi  = Lap u - (K^2/12) psi^5 + (1/8) psi^-7 AtAt + 2 pi (rho0 psi^5 + rho2 psi)
 *   F_W,i  = Lap W_i + (1/3) d_i d_j W_j - 8 pi (psi^6 S_i - m_i)
 *   H = -8 psi^-5 F_psi,  M_i = psi^-6 F_W,i,
 *   psi = 1 + sum_p m_p / (2 |x - x_p|) + u,   At_ij = d_i W_j + d_j W_i - (2/3) delta_ij d_k W_k
 *           (+ the analytic Bowen-York curvature of punctures that carry momentum or spin),
 *
 * with rho = rho0 + psi^-4 rho2 (rho2 = gradient energy of a scalar field), on a
 * cell-centred uniform grid (x_i = lo + (i + 1/2) h) with 2nd- or 4th-order
 * centred stencils, periodic or Robin 1/r boundaries, optionally with reflection-symmetry
 * planes (Key features, "Boundary conditions"), by multigrid (Key features, "Fast").  On periodic boxes K^2 is
 * set every outer iteration by the discrete integrability condition
 * sum_cells F_psi = 0, the gauge is <u> = <W_i> = 0, and m_i = <8 pi psi^6 S_i>;
 * elsewhere K is the configured constant and m_i = 0.  The constraint norms
 * are evaluated every outer iteration (Key features, "Diagnostics").
 *
 * Conventions for every call:
 *   - Field arrays hold N = n[0]*n[1]*n[2] doubles, x fastest: index i + n0 (j + n1 k),
 *     no ghost cells.  W and S are 3 such arrays back to back (x, y, z components).
 *   - on_device = 1: the pointer is CUDA device memory on the library's current device
 *     (for instance a torch tensor's data_ptr()); on_device = 0: host memory.
 *   - The caller owns every buffer it passes; the library copies inputs on the call and
 *     never keeps caller pointers (except the optional workspace, see mg_create).
 *   - Every call returns a status; nothing aborts, throws or traps.  mg_last_error()
 *     gives a one-line description of the last failure on the calling thread.
 *   - A context is not thread safe; calls on one context must be serialised.
 *   - All device work of a context is issued on the CUDA stream given to mg_create.
 */
#ifndef CTT_MG_H
#define CTT_MG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    MG_OK = 0,
    MG_ERR_INVALID_ARG = 1,   /* bad size, pointer, order, level count, NaN/inf input  */
    MG_ERR_UNSUPPORTED = 2,   /* a feature outside this library (e.g. non-flat metric) */
    MG_ERR_CUDA = 3,          /* a CUDA runtime call failed                            */
    MG_ERR_OOM = 4,           /* device or host allocation failed / workspace too small */
    MG_ERR_STATE = 5,         /* call out of order (e.g. solve before set_sources)     */
    MG_ERR_NOT_CONVERGED = 6, /* max_outer iterations used without reaching tol        */
    MG_ERR_DIVERGED = 7,      /* a norm became NaN/inf or grew for 3 outer iterations  */
    MG_ERR_TIMEOUT = 8        /* a bounded device-side wait ran out                     */
} mg_status;

enum { MG_BC_PERIODIC = 0, MG_BC_ROBIN = 1 };
enum { MG_FP64 = 0, MG_MIXED = 1 };            /* inner V-cycle in FP64, or FP32 under FP64 defect correction */
enum { MG_K_FIXED = 0, MG_K_INTEGRABILITY = 1 };

typedef struct {
    int n[3];             /* cells per axis; every level above the coarsest must have even sizes */
    double lo[3], hi[3];  /* box; h[a] = (hi[a] - lo[a]) / n[a]                                   */
    int order;            /* 2 or 4                                                               */
    int bc;               /* MG_BC_PERIODIC or MG_BC_ROBIN (1/r falloff about the origin)         */
    int levels;           /* multigrid levels, 0 = coarsen while all sizes are even and halve to >= 3 */
    int precision;        /* MG_FP64 or MG_MIXED                                                  */
    int k_mode;           /* MG_K_INTEGRABILITY (periodic only) or MG_K_FIXED                     */
    double K;             /* used when k_mode == MG_K_FIXED                                       */
    int npunct;           /* 0..2 bare punctures (Robin boxes only)                               */
    double punct_m[2];
    double punct_x[2][3];
    double tol;           /* stop when max(|H|, |M_i|) <= tol (default 1e-10)                     */
    int max_outer;        /* outer (defect-correction) iterations (default 60)                    */
    int nu_pre, nu_post;  /* red-black sweeps before / after the coarse correction (default 2, 2) */
    int coarse_sweeps;    /* red-black sweeps on the coarsest level (default 60)                  */
    int use_graph;        /* 1 = replay each outer iteration as a captured CUDA graph (default 1); 0 = direct
                             launches; 2 = as 1, and a batch (mg_batch_solve) is paced from the host     */
    long long spin_limit; /* bound on any device-side wait, in polls (default 1<<24; 0: every wait
                             gives up at once and the solve returns MG_ERR_TIMEOUT)                 */
    int inner_cycles;     /* V-cycles per outer iteration, 0 = auto (1 for MG_FP64, 2 for MG_MIXED) */
    int block_threads;    /* threads per block of the global-memory stencil kernels: 0 = 256, else 64, 128 or 256 */
    int smoother;         /* 0 = auto: the TMA-tiled colour pass and restriction on FP32 levels with nx, ny
                             multiples of 8, >= 16 and nz >= 8, the next-to-coarsest level and the coarsest in one
                             CTA when small, global-memory kernels elsewhere; 1 = one global-memory kernel per
                             step on every level */
    int cycle;            /* coarse-level visits per cycle: 0 or 1 = V-cycle (default), 2 = W-cycle           */
    double omega;         /* red-black relaxation weight in (0, 2); 0 = 1.0 (plain Gauss-Seidel per colour)   */
    int nested;           /* 1 = nested start: when every size is even and its half at least nested_min, a solve
                             that was given no initial guess (mg_set_initial_guess with a non-NULL u or W) since
                             the previous solve first solves the same problem on the grid of half the size
                             (sources: means over 2^3 cells; tolerance max(tol, nested_tol); nested in turn while
                             it stays eligible) and starts the outer iteration from its solution, interpolated
                             tricubically.  Only the starting state changes: the stopping test and the discrete
                             root are the same.  The half-size context lives in this context's workspace.
                             Ignored by mg_batch_*.  0 = off (default).                                         */
    int nested_min;       /* smallest half size per axis that is solved first; 0 = 64, else >= 3             */
    double nested_tol;    /* tolerance of the half-size solve (raised to tol); 0 = 3e-4                      */
    double punct_P[2][3]; /* Bowen-York linear momentum of puncture p (0 = bare).  With P or S set, the
                             analytic curvature 3/(2r^2)[P_i n_j + P_j n_i - (delta_ij - n_i n_j) P.n]
                             + 3/r^3 [(S x n)_i n_j + (S x n)_j n_i] (n, r from the puncture; ADM momentum P,
                             ADM angular momentum S) is added to At_ij before AtAt; F_W is unchanged     */
    double punct_S[2][3]; /* Bowen-York spin of puncture p (0 = bare)                                    */
    int reflect;          /* Robin boxes: bit a (a = 0, 1, 2) makes the lower face of axis a a reflection-
                             symmetry plane (lo[a] must be 0): a cell below it takes the value of its mirror
                             image, with the sign flipped for W_a (the component normal to the plane) and kept
                             for u and the other components.  7 = octant symmetry.  0 = all faces Robin.    */
    double field_tol;     /* > 0: a solve stops only when, besides max(|H|, |M_i|) <= tol, the last outer update
                             changed every field by at most field_tol times its size (max |e_u| <= field_tol
                             max |psi|, max |e_W_i| <= field_tol max |W_i|); with the outer iteration's
                             contraction rho, the remaining error per field is then about rho / (1 - rho) of
                             that.  A residual bound alone fixes each field only to |J^-1| tol in absolute
                             terms, which for a small W_i can be far from tol relative to W_i.  Needs at least
                             one outer update.  The half-size solve of a nested start ignores it.  0 = off.  */
    int extrap;           /* Robin boxes: bit 2a (lower) / 2a + 1 (upper) makes that face of axis a extrapolating
                             (the paper lists extrapolating, reflective and periodic boundaries, Key features,
                             "Boundary conditions"): a cell beyond it at distance d along its normal takes the
                             linear extrapolation (1 + d) v(b) - d v(b') through the boundary cell b of its line
                             and the next one in, for u and every W_i; beyond several such faces the rule applies
                             axis by axis, and the Robin or mirror rule then handles the remaining coordinates.
                             Linear fields are reproduced exactly.  Such a face leaves the field's normal
                             behaviour free, so whether the problem stays well posed depends on the faces
                             chosen: at least one face must stay Robin (MG_ERR_UNSUPPORTED otherwise), and some
                             sets (e.g. the three lower faces) give a nearly singular system that does not
                             converge.  A lower face cannot be both extrapolating and a symmetry plane.  0 = none. */
    int tile_waves;       /* launch shape of the TMA-tiled colour pass and restriction: each tile column is cut
                             into z chunks so that the grid holds about tile_waves CTAs per SM (1..8; chunks of
                             at least 2 planes).  0 = 2, the CTAs one SM holds at once (mg_autotune picks it). */
    int field_est;        /* with field_tol > 0: 1 = compare each field's estimated remaining error, not its last
                             update, with field_tol.  The estimate is rel rho / (1 - rho), where rel is the last
                             update relative to the field's size and rho = rel / (the previous update's rel) is the
                             observed contraction (used when rho < 1/2; otherwise the update itself is compared).
                             It saves the outer iteration that only confirms a small update.  0 = off.       */
    int k2_newton;        /* periodic boxes with K from integrability: 1 = remove the mean of each outer psi
                             correction along z = L_psi^-1 dF_psi/dK^2 (K^2 as a Newton unknown of the psi row)
                             instead of along the constant vector; z comes from one extra inner solve at the
                             start of each solve.  With K from integrability the psi row has a near-null mode
                             close to the constant, which the plain mean removal leaves partly in place.
                             Ignored elsewhere, by mg_batch_* and by the nested start's half-size solve.
                             0 = off (default).                                                         */
} mg_config;

typedef struct {
    int outer_iters;      /* residual evaluations made minus one                                  */
    int converged;        /* 1 when max(|H|, |M_i|) <= tol                                        */
    double K;             /* final K (negative root on periodic boxes: expanding slice)          */
    double K2;            /* final K^2                                                            */
    double norms[4];      /* final max |H|, max |M_x|, max |M_y|, max |M_z|                       */
    double mom_mean[3];   /* m_i removed from the momentum source (periodic), else 0              */
    const double *history;/* 4 norms per outer iteration, owned by the context, valid until the next solve */
    int history_len;      /* rows in history                                                     */
    double device_ms;     /* device time of the solve, nested start included (CUDA events)        */
    long long kernel_launches; /* library kernels launched by this solve (0 if use_graph == 0)    */
    int nested_iters;     /* outer iterations of the nested start's half-size solve, 0 without one    */
    double rel_change[4]; /* with field_tol > 0, the last outer update per field: max |e_u| / max |psi|,
                             max |e_W_i| / max |W_i| (0 before the first update, where the field is
                             zero, or with field_tol = 0)                                          */
    int warm_start;       /* learned warm start: 0 not used, 1 its guess was the starting state, 2 its guess
                             was rejected (non-finite residual), 3 the solve from its guess
                             failed and was repeated from the cold start (this info describes the repeat,
                             device_ms and kernel_launches include both)                            */
} mg_solve_info;

/* Fill *cfg with defaults: order 2, periodic, integrability K, MG_MIXED, tol 1e-10, ... */
mg_status mg_config_default(mg_config *cfg);

/* Device bytes the context needs for cfg (states, sources, all levels, reduction scratch, and the
 * half-size contexts of a nested start, recursively). */
mg_status mg_workspace_size(const mg_config *cfg, size_t *bytes);

/*
 * Create a context for one problem.  cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * workspace: NULL lets the library allocate its device memory itself; otherwise a device
 * buffer of at least mg_workspace_size() bytes, 256-byte aligned, owned by the caller and
 * kept alive until mg_destroy (for instance a torch uint8 tensor).
 */
mg_status mg_create(const mg_config *cfg, void *cuda_stream, void *workspace, size_t workspace_bytes,
                    struct mg_ctx **out);

/* Conformal metric gt_ij (6 arrays xx, xy, xz, yy, yz, zz) or NULL.  Only the flat metric
 * (NULL, or exactly delta_ij everywhere) is supported; anything else returns MG_ERR_UNSUPPORTED
 * (non-conformally-flat data is listed as forthcoming in the paper's feature list). */
mg_status mg_set_conformal_metric(struct mg_ctx *ctx, const double *gt, int on_device);

/* Matter sources (the matter projections rho and S_i of the paper's Summary, after eq:Mom, given by a
 * scalar field: Key features, "Flexibility"): rho = rho0 + psi^-4 rho2; S_i lower-index momentum density.
 * rho2 may be NULL (0).
 * Returns MG_ERR_INVALID_ARG (and leaves the context without sources) if any value is NaN or
 * infinite; the check runs on the device after the copy, and the call returns once it is done. */
mg_status mg_set_sources(struct mg_ctx *ctx, const double *rho0, const double *rho2, const double *Sx,
                         const double *Sy, const double *Sz, int on_device);

/* Initial guess for u (N) and W (3N) of the CTT unknowns (psi = background + u, W_i of At_ij; Summary,
 * "Methods"); either may be NULL (zero).  Default: u = 0, W = 0.
 * On periodic boxes the means are projected out at the start of mg_solve.  With cfg.nested, a
 * non-NULL u or W replaces the next solve's nested start; (NULL, NULL) keeps it (a half-size solve
 * that diverges leaves the zero state as the start). */
mg_status mg_set_initial_guess(struct mg_ctx *ctx, const double *u, const double *W, int on_device);

/* Solve the constraints eq:Ham and eq:Mom (Summary) by multigrid (Key features, "Fast"): iterate until
 * max(|H|, |M_i|) <= tol (and, with field_tol, the per-field test of field_tol / field_est), recording
 * the norms of every outer iteration (Key features, "Diagnostics").  info may be NULL. */
mg_status mg_solve(struct mg_ctx *ctx, mg_solve_info *info);

/* Copy out the solution of the constraint problem (Summary: psi through u, W_i, and K, the mean
 * curvature of the constant-K slice): u (N doubles), W (3N doubles) and K; any pointer may be NULL. */
mg_status mg_get_solution(struct mg_ctx *ctx, double *u, double *W, double *K, int on_device);

/*
 * Checkpoint / resume (the paper writes checkpoints to restart from: Key features, "Output"; this
 * library writes a raw file instead of HDF5).  mg_checkpoint_save writes the context's state to `path` as a raw
 * little-endian file: the 8 bytes "CTTMGCK1", int32 n[3], order, bc, 0, the last K^2 (double),
 * then u (N doubles) and W (3N doubles), x fastest, no ghost cells.  mg_checkpoint_load reads such
 * a file written for the same n, order and bc and makes its (u, W) the next solve's initial guess
 * (as mg_set_initial_guess with non-NULL u and W: a nested start is skipped).  Both return
 * MG_ERR_INVALID_ARG for a file that cannot be opened, read or written, a bad header or another
 * grid, and MG_ERR_UNSUPPORTED on a big-endian host; both synchronise the context's stream.
 */
mg_status mg_checkpoint_save(struct mg_ctx *ctx, const char *path);
mg_status mg_checkpoint_load(struct mg_ctx *ctx, const char *path);

/*
 * Learned warm start (not in the paper: a learned initial guess added to its multigrid solver; plain
 * multigrid stays the fallback, and the multigrid solve decides every result).  mg_warmstart_load reads a trained 3-D U-Net from
 * `weights_path` (NULL: switch the warm start off) into device memory it allocates (about 70 MB
 * for a 64^3 network) and attaches it to the context.  From then on, a solve that was given no
 * initial guess first runs the network (BF16 tcgen05 convolutions, FP32 accumulation; captured
 * once as a CUDA graph) on the sources: inputs (rho0 + rho2 - <rho>, S_i, and the pre-solve
 * K = -sqrt(24 pi <rho>)) at the network's size, output (u, W_i) with zero means; a grid finer
 * than the network's is restricted (8-child means) before and the guess prolongated (cell-centred
 * trilinear) after.  The multigrid judges the guess: it is the starting state whenever its
 * residual is finite (otherwise the solve starts as without it: psi = 1, or the nested start), and
 * if the solve from it does not converge or diverges, the problem is solved again from the cold
 * start; mg_solve_info.warm_start reports which happened.  (A test of the guess's max(|H|, |M_i|)
 * against that of psi = 1 would reject useful guesses: the Laplacian weighs a mode of the guess's
 * error by k^2, so its small-scale error, which the first smoothing sweeps remove, dominates.)
 *
 * Serves periodic cubes whose side is the network's size n_net times a power of two; other grids
 * return MG_ERR_UNSUPPORTED.  The file (little-endian) is: the 8 bytes "CTTUNET1"; int32 n_net
 * (a multiple of 8, >= 64, (n_net/8)^3 a multiple of 128); int32 count; float32 s_rho, s_S, s_K,
 * s_u, s_W (input scales of rho - <rho>, S_i, K and output scales of u, W_i, all nonzero); then
 * count float32 parameters: for each 3x3x3 convolution in the order e0a, e0, e1a, e1, e2a, e2, ba,
 * b, d2a, d2, d1a, d1, d0a, d0 (channels in -> out: 16->16, 16->16, 16->32, 32->32, 32->64,
 * 64->64, 64->64, 64->64, 128->64, 64->64, 96->32, 32->32, 48->16, 16->16) its weights
 * [27][cout][cin] (tap (dz+1)*9 + (dy+1)*3 + (dx+1)) and bias [cout], then the 1x1 head's weights
 * [4][16] and bias [4]; nothing after them.  A malformed file returns MG_ERR_INVALID_ARG.
 *
 * mg_warmstart_predict runs only the network on the current sources: the guess becomes the
 * context's state (as if given to mg_set_initial_guess) and is copied to u (N doubles) and W (3N
 * doubles) when they are not NULL (on_device as for mg_get_solution).
 */
mg_status mg_warmstart_load(struct mg_ctx *ctx, const char *weights_path);
mg_status mg_warmstart_predict(struct mg_ctx *ctx, double *u, double *W, int on_device);

/* Evaluate the constraints at the current state (H of eq:Ham, M_i of eq:Mom, the maximum over the grid
 * of the errors the paper's solver reports every iteration: Key features, "Diagnostics"):
 * out = max |H|, max |M_x|, |M_y|, |M_z|. */
mg_status mg_residual_norms(struct mg_ctx *ctx, double out[4]);

/* Write the constraint fields H (N, eq:Ham) and M (3N, eq:Mom) at the current state (either may be
 * NULL). */
mg_status mg_constraint_fields(struct mg_ctx *ctx, double *H, double *M, int on_device);

/*
 * Measurement aid: launch one kernel of the solve `reps` times back to back on the context's
 * stream, bracketed by CUDA events, at the current state (call after mg_solve or
 * mg_residual_norms).  which: 0 = one red-black colour pass of the finest-level smoother,
 * 1 = residual + restriction of the finest level, 2 = outer FP64 residual pass 1 (its two
 * kernels, q/div W then the residual parts, and the reduction of the integrability sums),
 * 3 = the second of those kernels alone (the residual parts; FP64-ALU bound).
 * Returns the mean device time per launch and the algorithmic DRAM bytes one launch must
 * move (every array it reads once, every array it writes once).  The solver state is not
 * changed except for scratch buffers.
 */
mg_status mg_time_kernel(struct mg_ctx *ctx, int which, int reps, double *ms_per_launch, double *bytes_per_launch);

/*
 * Measurement aid: the FP64 FMA rate of the GPU the context runs on, in TFLOP/s (an FMA counts as
 * two flops).  A probe kernel runs 8 independent FMA chains per thread on every SM (enough to keep
 * the FP64 pipe busy) on the context's stream, once untimed and `reps` times between CUDA events.
 * bench.py reports it beside the unit-count FP64 peak.  The solver state is not changed.
 */
mg_status mg_fp64_fma_rate(struct mg_ctx *ctx, int reps, double *tflops);

/*
 * mg_residual_norms_noalloc -- the constraint norms of mg_residual_norms for a state held by the
 * caller, computed without allocating anything.  The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc or any other allocator, for example a host
 * process whose device memory belongs to a fixed arena or another framework's allocator, or a
 * loop that must not allocate after start-up.  It takes no context.
 *
 *   cfg         grid, order, bc, k_mode, K and bare punctures (the iteration fields are ignored);
 *               at most 262144 cells (64^3), larger grids return MG_ERR_INVALID_ARG; punctures with a
 *               Bowen-York momentum or spin return MG_ERR_UNSUPPORTED.
 *   u, W        device arrays, N and 3N doubles (layout as above); psi = 1 + punctures + u.
 *   rho0, S     device arrays, N and 3N doubles; rho2 device array or NULL (zero).
 *   out         host array of 4 doubles: max |H|, max |M_x|, max |M_y|, max |M_z|.
 *   K2          host pointer or NULL: the K^2 used (integrability value on periodic boxes).
 *   cuda_stream stream for all work (NULL = legacy default stream); the call synchronises it.
 *
 * Scratch: one file-scope device array of 8.47 MB, which every GPU that loads the library
 * holds until the process exits.  The first call on a device looks up that device's address of
 * the array (with the device current) and caches it: that first call on each device should come
 * before any stream capture begins.  All calls share the array and it keeps the last call's contents;
 * two calls whose work overlaps on the GPU (different streams, or different threads) race on
 * it and give undefined results, so serialise them.  The call allocates no device or host memory.
 */
mg_status mg_residual_norms_noalloc(const mg_config *cfg, const double *u, const double *W, const double *rho0,
                                    const double *rho2, const double *S, double out[4], double *K2,
                                    void *cuda_stream);

/*
 * Autotuner: times candidate settings of (inner_cycles in {1, 2, 3} ({1, 2} for MG_FP64),
 * nu_pre = nu_post in {1, 2, 3}, omega in {1, 1.15, 1.3}; V-cycles) on the
 * given problem (sources as for mg_set_sources; each candidate runs one untimed and one timed solve
 * from psi = 1 on a private context), then, for MG_MIXED with the tiled kernels, the launch shape
 * of those kernels (tile_waves in {1, 2, 3, 4}) at the winning setting, and writes the fastest
 * setting that meets base->tol into *best (the other fields copied from *base), with its solve
 * time in *best_ms.  Results are cached
 * per (grid size, order, bc, precision, k_mode, nested) for the process, and, when cache_path is not NULL,
 * in that text file (one line per key; read before tuning, rewritten after).  A cache hit runs no
 * solve.  Returns MG_ERR_NOT_CONVERGED if no candidate met the tolerance.
 */
mg_status mg_autotune(const mg_config *base, const double *rho0, const double *rho2, const double *Sx,
                      const double *Sy, const double *Sz, int on_device, void *cuda_stream, const char *cache_path,
                      mg_config *best, double *best_ms);

void mg_destroy(struct mg_ctx *ctx);

/*
 * Batched solves: many independent problems of uneven grid sizes in one call (not in the paper,
 * which solves one problem per run).  All instances must
 * share order, bc, precision and k_mode; sizes, boxes and sources differ.  Each instance owns its
 * workspace and a private stream.
 *
 * Device-paced (default, use_graph != 2): mg_batch_solve is one CUDA graph launch and one host
 * synchronisation.  The graph holds every instance's start, then a conditional WHILE node whose
 * body is one conditional IF node per instance (that instance's captured outer iteration) and a
 * one-block control kernel; the control kernel reads each instance's scalars on the device,
 * records its norms, the round it met its tolerance and the time it did (%globaltimer), and sets
 * the conditions, so an instance drops out of the rounds once it has converged (or its norm became
 * non-finite, or it used its max_outer) and the loop ends when none is left.  A converged
 * instance's state is exactly that of a solo mg_solve.  The graph is built on the first call and
 * reused (rebuilt when the largest max_outer changes).
 * Host-paced (cfgs[0].use_graph == 2): one graph per round for all instances, checked on the
 * host after every round; converged instances keep iterating in lock step until the last one
 * converges (their residual only decreases further).
 *   infos: count entries (may be NULL); infos[b].outer_iters is the round at which instance b
 *   met its tolerance; infos[b].device_ms the time from the start of the solve to that round
 *   (device timestamps, or events when host-paced); infos[b].history its norms up to that round;
 *   infos[b].converged = 0 for an instance that did not.  An instance whose norm becomes
 *   non-finite is abandoned (the others continue) and the call returns MG_ERR_DIVERGED.
 */
typedef struct mg_batch mg_batch;
mg_status mg_batch_create(int count, const mg_config *cfgs, void *cuda_stream, mg_batch **out);
mg_status mg_batch_set_sources(mg_batch *bt, int b, const double *rho0, const double *rho2, const double *Sx,
                               const double *Sy, const double *Sz, int on_device);
mg_status mg_batch_set_initial_guess(mg_batch *bt, int b, const double *u, const double *W, int on_device);
mg_status mg_batch_solve(mg_batch *bt, mg_solve_info *infos, double *total_ms);
/* The learned warm start (see mg_warmstart_load) for every instance it serves, the network shared
 * by them (instances of other sizes start cold).  Before the batch's rounds each such instance
 * without an initial guess gets the network's guess (kept where its residual is finite); an
 * instance that does not converge from its guess is solved again alone from its
 * cold start after the rounds (infos[b].warm_start = 3, its time added to infos[b].device_ms and to
 * *total_ms).  NULL switches it off. */
mg_status mg_batch_warmstart_load(mg_batch *bt, const char *weights_path);
mg_status mg_batch_get_solution(mg_batch *bt, int b, double *u, double *W, double *K, int on_device);
void mg_batch_destroy(mg_batch *bt);

const char *mg_status_string(mg_status s);
const char *mg_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CTT_MG_H */
