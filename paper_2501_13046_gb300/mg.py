"""Thin Python binding of the C ABI in include/ctt_mg.h (libctt_mg.so).

Argument marshalling only: every step of the solve runs in the CUDA library.
The functions carry the C names.  Device buffers may be torch tensors (their
data_ptr() is passed with on_device=1) and host buffers numpy float64 arrays.
torch supplies device memory (the workspace) and the CUDA stream.

There is no fallback: if the shared library is missing or fails to load, the
import raises.
"""
import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libctt_mg.so")

MG_OK, MG_ERR_INVALID_ARG, MG_ERR_UNSUPPORTED, MG_ERR_CUDA, MG_ERR_OOM, MG_ERR_STATE, \
    MG_ERR_NOT_CONVERGED, MG_ERR_DIVERGED, MG_ERR_TIMEOUT = range(9)
MG_BC_PERIODIC, MG_BC_ROBIN = 0, 1
MG_FP64, MG_MIXED = 0, 1
MG_K_FIXED, MG_K_INTEGRABILITY = 0, 1

EXPORTS = ("mg_config_default", "mg_workspace_size", "mg_create", "mg_set_conformal_metric", "mg_set_sources",
           "mg_set_initial_guess", "mg_solve", "mg_get_solution", "mg_residual_norms", "mg_constraint_fields",
           "mg_time_kernel", "mg_fp64_fma_rate", "mg_residual_norms_noalloc", "mg_destroy", "mg_status_string", "mg_last_error",
           "mg_batch_create", "mg_batch_set_sources", "mg_batch_set_initial_guess", "mg_batch_solve",
           "mg_batch_get_solution", "mg_batch_destroy", "mg_autotune", "mg_checkpoint_save", "mg_checkpoint_load",
           "mg_warmstart_load", "mg_warmstart_predict", "mg_batch_warmstart_load")


class mg_config(C.Structure):
    _fields_ = [
        ("n", C.c_int * 3), ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("order", C.c_int), ("bc", C.c_int),
        ("levels", C.c_int), ("precision", C.c_int), ("k_mode", C.c_int), ("K", C.c_double), ("npunct", C.c_int),
        ("punct_m", C.c_double * 2), ("punct_x", (C.c_double * 3) * 2), ("tol", C.c_double), ("max_outer", C.c_int),
        ("nu_pre", C.c_int), ("nu_post", C.c_int), ("coarse_sweeps", C.c_int), ("use_graph", C.c_int),
        ("spin_limit", C.c_longlong), ("inner_cycles", C.c_int), ("block_threads", C.c_int),
        ("smoother", C.c_int), ("cycle", C.c_int), ("omega", C.c_double), ("nested", C.c_int),
        ("nested_min", C.c_int), ("nested_tol", C.c_double),
        ("punct_P", (C.c_double * 3) * 2), ("punct_S", (C.c_double * 3) * 2), ("reflect", C.c_int),
        ("field_tol", C.c_double), ("extrap", C.c_int), ("tile_waves", C.c_int), ("field_est", C.c_int), ("k2_newton", C.c_int),
    ]


class mg_solve_info(C.Structure):
    _fields_ = [
        ("outer_iters", C.c_int), ("converged", C.c_int), ("K", C.c_double), ("K2", C.c_double),
        ("norms", C.c_double * 4), ("mom_mean", C.c_double * 3), ("history", C.POINTER(C.c_double)),
        ("history_len", C.c_int), ("device_ms", C.c_double), ("kernel_launches", C.c_longlong),
        ("nested_iters", C.c_int), ("rel_change", C.c_double * 4), ("warm_start", C.c_int),
    ]


class MGError(RuntimeError):
    def __init__(self, status, where, detail):
        self.status = status
        super().__init__("%s: %s (%s)" % (where, _lib.mg_status_string(status).decode(), detail))


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libctt_mg.so is not built; run __graft_entry__.build() (no CPU fallback exists)")
    L = C.CDLL(LIB_PATH)
    vp, dp = C.c_void_p, C.POINTER(C.c_double)
    L.mg_config_default.argtypes = [C.POINTER(mg_config)]
    L.mg_workspace_size.argtypes = [C.POINTER(mg_config), C.POINTER(C.c_size_t)]
    L.mg_create.argtypes = [C.POINTER(mg_config), vp, vp, C.c_size_t, C.POINTER(vp)]
    L.mg_set_conformal_metric.argtypes = [vp, vp, C.c_int]
    L.mg_set_sources.argtypes = [vp, vp, vp, vp, vp, vp, C.c_int]
    L.mg_set_initial_guess.argtypes = [vp, vp, vp, C.c_int]
    L.mg_solve.argtypes = [vp, C.POINTER(mg_solve_info)]
    L.mg_get_solution.argtypes = [vp, vp, vp, dp, C.c_int]
    L.mg_residual_norms.argtypes = [vp, dp]
    L.mg_constraint_fields.argtypes = [vp, vp, vp, C.c_int]
    L.mg_time_kernel.argtypes = [vp, C.c_int, C.c_int, dp, dp]
    L.mg_fp64_fma_rate.argtypes = [vp, C.c_int, dp]
    L.mg_residual_norms_noalloc.argtypes = [C.POINTER(mg_config), vp, vp, vp, vp, vp, dp, dp, vp]
    L.mg_destroy.argtypes = [vp]
    L.mg_checkpoint_save.argtypes = [vp, C.c_char_p]
    L.mg_checkpoint_load.argtypes = [vp, C.c_char_p]
    L.mg_warmstart_load.argtypes = [vp, C.c_char_p]
    L.mg_warmstart_predict.argtypes = [vp, vp, vp, C.c_int]
    L.mg_batch_warmstart_load.argtypes = [vp, C.c_char_p]
    L.mg_destroy.restype = None
    L.mg_batch_create.argtypes = [C.c_int, C.POINTER(mg_config), vp, C.POINTER(vp)]
    L.mg_batch_set_sources.argtypes = [vp, C.c_int, vp, vp, vp, vp, vp, C.c_int]
    L.mg_batch_set_initial_guess.argtypes = [vp, C.c_int, vp, vp, C.c_int]
    L.mg_batch_solve.argtypes = [vp, C.POINTER(mg_solve_info), dp]
    L.mg_batch_get_solution.argtypes = [vp, C.c_int, vp, vp, dp, C.c_int]
    L.mg_autotune.argtypes = [C.POINTER(mg_config), vp, vp, vp, vp, vp, C.c_int, vp, C.c_char_p,
                              C.POINTER(mg_config), dp]
    L.mg_batch_destroy.argtypes = [vp]
    L.mg_batch_destroy.restype = None
    L.mg_status_string.argtypes = [C.c_int]
    L.mg_status_string.restype = C.c_char_p
    L.mg_last_error.argtypes = []
    L.mg_last_error.restype = C.c_char_p
    for name in EXPORTS:
        if name not in ("mg_destroy", "mg_status_string", "mg_last_error", "mg_batch_destroy"):
            getattr(L, name).restype = C.c_int
    return L


_lib = _load()


def lib():
    return _lib


def _check(st, where, allow=()):
    if st != MG_OK and st not in allow:
        raise MGError(st, where, _lib.mg_last_error().decode())
    return st


def _ptr(x):
    """(pointer, on_device) for a torch tensor, numpy array or None."""
    if x is None:
        return None, 0
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous(), "tensor must be contiguous"
        return x.data_ptr(), int(x.is_cuda)
    assert isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous
    return x.ctypes.data, 0


def mg_config_default():
    cfg = mg_config()
    _check(_lib.mg_config_default(C.byref(cfg)), "mg_config_default")
    return cfg


def mg_workspace_size(cfg):
    n = C.c_size_t(0)
    _check(_lib.mg_workspace_size(C.byref(cfg), C.byref(n)), "mg_workspace_size")
    return n.value


def mg_create(cfg, stream=0, workspace=None):
    """stream: a cudaStream_t as int (e.g. torch.cuda.current_stream().cuda_stream);
    workspace: optional device tensor of at least mg_workspace_size(cfg) bytes."""
    out = C.c_void_p()
    wp, nb = (None, 0) if workspace is None else (workspace.data_ptr(), workspace.numel() * workspace.element_size())
    _check(_lib.mg_create(C.byref(cfg), C.c_void_p(stream or None), C.c_void_p(wp), nb, C.byref(out)), "mg_create")
    return out


def mg_set_conformal_metric(ctx, gt):
    p, dev = _ptr(gt)
    return _check(_lib.mg_set_conformal_metric(ctx, p, dev), "mg_set_conformal_metric")


def mg_set_sources(ctx, rho0, rho2, Sx, Sy, Sz):
    ps = [_ptr(a) for a in (rho0, rho2, Sx, Sy, Sz)]
    dev = max(d for _, d in ps)
    return _check(_lib.mg_set_sources(ctx, *[p for p, _ in ps], dev), "mg_set_sources")


def mg_set_initial_guess(ctx, u, W):
    (pu, du), (pw, dw) = _ptr(u), _ptr(W)
    return _check(_lib.mg_set_initial_guess(ctx, pu, pw, max(du, dw)), "mg_set_initial_guess")


def mg_solve(ctx, allow=(MG_ERR_NOT_CONVERGED,)):
    """Returns (status, info dict)."""
    info = mg_solve_info()
    st = _check(_lib.mg_solve(ctx, C.byref(info)), "mg_solve", allow)
    hist = np.ctypeslib.as_array(info.history, shape=(info.history_len * 4,)).reshape(-1, 4).copy() \
        if info.history_len > 0 else np.zeros((0, 4))
    return st, dict(outer_iters=info.outer_iters, converged=bool(info.converged), K=info.K, K2=info.K2,
                    norms=np.array(info.norms[:]), mom_mean=np.array(info.mom_mean[:]), history=hist,
                    device_ms=info.device_ms, kernel_launches=info.kernel_launches,
                    nested_iters=info.nested_iters, rel_change=np.array(info.rel_change[:]),
                    warm_start=info.warm_start)


def mg_get_solution(ctx, u=None, W=None):
    (pu, du), (pw, dw) = _ptr(u), _ptr(W)
    K = C.c_double(0.0)
    _check(_lib.mg_get_solution(ctx, pu, pw, C.byref(K), max(du, dw)), "mg_get_solution")
    return K.value


def mg_residual_norms(ctx):
    out = (C.c_double * 4)()
    _check(_lib.mg_residual_norms(ctx, out), "mg_residual_norms")
    return np.array(out[:])


def mg_constraint_fields(ctx, H=None, M=None):
    (ph, dh), (pm, dm) = _ptr(H), _ptr(M)
    return _check(_lib.mg_constraint_fields(ctx, ph, pm, max(dh, dm)), "mg_constraint_fields")


def mg_time_kernel(ctx, which, reps):
    """(ms per launch, algorithmic bytes per launch) of one solver kernel; see the header."""
    ms, b = C.c_double(0.0), C.c_double(0.0)
    _check(_lib.mg_time_kernel(ctx, which, reps, C.byref(ms), C.byref(b)), "mg_time_kernel")
    return ms.value, b.value


def mg_fp64_fma_rate(ctx, reps=3):
    """FP64 FMA rate of the context's GPU in TFLOP/s (probe kernel on the context's stream)."""
    r = C.c_double(0.0)
    _check(_lib.mg_fp64_fma_rate(ctx, reps, C.byref(r)), "mg_fp64_fma_rate")
    return r.value


def mg_residual_norms_noalloc(cfg, u, W, rho0, rho2, S, stream=0):
    """Constraint norms (and K^2) of a caller-held device state, with no allocation in the library.
    u, W, rho0, rho2 (or None), S: contiguous float64 CUDA tensors.  Returns (norms[4], K2)."""
    out = (C.c_double * 4)()
    k2 = C.c_double(0.0)
    ptr = lambda t: None if t is None else t.data_ptr()
    _check(_lib.mg_residual_norms_noalloc(C.byref(cfg), ptr(u), ptr(W), ptr(rho0), ptr(rho2), ptr(S), out,
                                          C.byref(k2), C.c_void_p(stream or None)), "mg_residual_norms_noalloc")
    return np.array(out[:]), k2.value


def mg_warmstart_load(ctx, path):
    """Attach the learned warm start stored at `path` (None: detach)."""
    _check(_lib.mg_warmstart_load(ctx, None if path is None else os.fsencode(path)), "mg_warmstart_load")


def mg_warmstart_predict(ctx, u=None, W=None):
    (pu, du), (pw, dw) = _ptr(u), _ptr(W)
    _check(_lib.mg_warmstart_predict(ctx, pu, pw, max(du, dw)), "mg_warmstart_predict")


def mg_batch_warmstart_load(bt, path):
    _check(_lib.mg_batch_warmstart_load(bt, None if path is None else os.fsencode(path)), "mg_batch_warmstart_load")


def mg_checkpoint_save(ctx, path):
    _check(_lib.mg_checkpoint_save(ctx, os.fsencode(path)), "mg_checkpoint_save")


def mg_checkpoint_load(ctx, path):
    _check(_lib.mg_checkpoint_load(ctx, os.fsencode(path)), "mg_checkpoint_load")


def mg_destroy(ctx):
    _lib.mg_destroy(ctx)


def mg_batch_create(cfgs, stream=0):
    arr = (mg_config * len(cfgs))(*cfgs)
    out = C.c_void_p()
    _check(_lib.mg_batch_create(len(cfgs), arr, C.c_void_p(stream or None), C.byref(out)), "mg_batch_create")
    return out


def mg_batch_set_sources(bt, b, rho0, rho2, Sx, Sy, Sz):
    ps = [_ptr(a) for a in (rho0, rho2, Sx, Sy, Sz)]
    dev = max(d for _, d in ps)
    return _check(_lib.mg_batch_set_sources(bt, b, *[p for p, _ in ps], dev), "mg_batch_set_sources")


def mg_batch_set_initial_guess(bt, b, u, W):
    (pu, du), (pw, dw) = _ptr(u), _ptr(W)
    return _check(_lib.mg_batch_set_initial_guess(bt, b, pu, pw, max(du, dw)), "mg_batch_set_initial_guess")


def mg_batch_solve(bt, count, allow=(MG_ERR_NOT_CONVERGED,)):
    """Returns (status, [info dict per instance], total_ms)."""
    infos = (mg_solve_info * count)()
    tot = C.c_double(0.0)
    st = _check(_lib.mg_batch_solve(bt, infos, C.byref(tot)), "mg_batch_solve", allow)
    out = []
    for inf in infos:
        hist = np.ctypeslib.as_array(inf.history, shape=(inf.history_len * 4,)).reshape(-1, 4).copy() \
            if inf.history_len > 0 else np.zeros((0, 4))
        out.append(dict(outer_iters=inf.outer_iters, converged=bool(inf.converged), K=inf.K, K2=inf.K2,
                        norms=np.array(inf.norms[:]), history=hist, device_ms=inf.device_ms,
                        kernel_launches=inf.kernel_launches, rel_change=np.array(inf.rel_change[:]),
                        warm_start=inf.warm_start))
    return st, out, tot.value


def mg_batch_get_solution(bt, b, u=None, W=None):
    (pu, du), (pw, dw) = _ptr(u), _ptr(W)
    K = C.c_double(0.0)
    _check(_lib.mg_batch_get_solution(bt, b, pu, pw, C.byref(K), max(du, dw)), "mg_batch_get_solution")
    return K.value


def mg_autotune(cfg, rho0, rho2, Sx, Sy, Sz, stream=0, cache_path=None):
    """(best mg_config, its solve ms) for this problem; see the header for the candidates and cache."""
    ps = [_ptr(a) for a in (rho0, rho2, Sx, Sy, Sz)]
    dev = max(d for _, d in ps)
    best = mg_config()
    ms = C.c_double(0.0)
    _check(_lib.mg_autotune(C.byref(cfg), *[p for p, _ in ps], dev, C.c_void_p(stream or None),
                            None if cache_path is None else cache_path.encode(), C.byref(best), C.byref(ms)),
           "mg_autotune")
    return best, ms.value


def mg_batch_destroy(bt):
    _lib.mg_batch_destroy(bt)


def config_for(problem, precision=MG_MIXED, **overrides):
    """mg_config for a problem dict of paper_2501_13046_gb300.fields (marshalling only)."""
    cfg = mg_config_default()
    n = problem["n"]
    lo, hi = problem["lo"], problem["hi"]
    for a in range(3):
        cfg.n[a] = n[a]
        cfg.lo[a] = lo if np.isscalar(lo) else lo[a]
        cfg.hi[a] = hi if np.isscalar(hi) else hi[a]
    cfg.order = problem["order"]
    cfg.bc = problem["bc"]
    cfg.k_mode = problem["kmode"]
    cfg.K = problem["K"]
    cfg.precision = precision
    cfg.npunct = len(problem["punctures"])
    cfg.reflect = problem.get("reflect", 0)
    cfg.extrap = problem.get("extrap", 0)
    for p, pun in enumerate(problem["punctures"]):
        m, x = pun[0], pun[1]
        cfg.punct_m[p] = m
        for a in range(3):
            cfg.punct_x[p][a] = x[a]
            if len(pun) > 2:
                cfg.punct_P[p][a] = pun[2][a]
            if len(pun) > 3:
                cfg.punct_S[p][a] = pun[3][a]
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg
