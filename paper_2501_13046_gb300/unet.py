"""Thin ctypes binding of include/ctt_unet.h (the warm-start network's kernels in libctt_mg.so).

Argument marshalling only: tensors are torch CUDA tensors (device memory from torch), every
computation runs in the library's kernels, and each call raises if the library reports an error.
"""
import ctypes as C

from . import mg as _mg

_lib = _mg.lib()
vp, i32, i64, f32, f64 = C.c_void_p, C.c_int, C.c_longlong, C.c_float, C.c_double

_SIGS = {
    "unet_conv3d_fwd": [vp, i32, i32, vp, vp, vp, i32, i32, i32, i32, i32, i32, i32, i32, vp, C.c_size_t, i64, vp,
                        vp],
    "unet_conv3d_wgrad": [vp, i32, i32, vp, i32, i32, vp, i32, i32, i32, i32, i32, i64, vp, vp],
    "unet_pack_weights": [vp, i32, i32, i32, vp, vp],
    "unet_avgpool2": [vp, i32, i32, vp, i32, i32, i32, i32, i32, i32, vp],
    "unet_avgpool2_bwd": [vp, i32, i32, vp, i32, i32, i32, i32, i32, i32, i32, vp],
    "unet_upsample2": [vp, i32, i32, vp, i32, i32, i32, i32, i32, i32, vp],
    "unet_upsample2_bwd": [vp, i32, i32, vp, i32, i32, i32, i32, i32, i32, vp],
    "unet_relu_bwd": [vp, i32, i32, vp, i32, i32, i32, i64, vp],
    "unet_bias_grad": [vp, i32, i32, vp, i32, i64, vp],
    "unet_head_fwd": [vp, i32, i32, i32, vp, vp, vp, i32, i64, vp],
    "unet_head_bwd": [vp, i32, i32, i32, vp, vp, i32, vp, i32, i32, vp, vp, i64, vp],
    "unet_mse": [vp, vp, vp, vp, i32, i64, vp],
    "unet_adam": [vp, vp, vp, vp, i64, f32, f32, f32, f32, i32, vp],
    "unet_pack_input": [vp, vp, vp, f64, f32, f32, f32, vp, i64, vp, vp],
    "unet_unpack_output": [vp, f32, f32, vp, vp, i64, vp, vp],
    "unet_pack_target": [vp, vp, f32, f32, vp, i64, vp],
    "unet_restrict2_fields": [vp, vp, i32, i32, i32, i32, vp],
    "unet_prolong2_fields": [vp, vp, i32, i32, i32, i32, vp],
}
for _n, _a in _SIGS.items():
    getattr(_lib, _n).argtypes = _a
    getattr(_lib, _n).restype = C.c_int
_lib.unet_conv3d_fwd_workspace.argtypes = [i32, i32, i32, i32]
_lib.unet_conv3d_fwd_workspace.restype = C.c_size_t

SPIN = 1 << 22


def _p(t):
    return None if t is None else t.data_ptr()


def _call(name, *args):
    rc = getattr(_lib, name)(*args)
    if rc != 0:
        raise RuntimeError("%s failed with code %d" % (name, rc))


class Slice:
    """Channel slice [c0, c0 + c) of an NDHWC buffer `buf` with buf.shape[-1] channels per voxel."""

    def __init__(self, buf, c0=0, c=None):
        self.buf, self.c0 = buf, c0
        self.cs = buf.shape[-1]
        self.c = self.cs - c0 if c is None else c


def as_slice(t):
    return t if isinstance(t, Slice) else Slice(t)


def conv3d_workspace(n, cout):
    """Bytes of FP32 workspace conv3d_fwd's split form needs on grid n with cout channels (0: none)."""
    return int(_lib.unet_conv3d_fwd_workspace(n[0], n[1], n[2], cout))


def conv3d_fwd(x, w_bf16, bias, y, n, cin, cout, relu, err, stream=0, ws=None):
    """ws: optional FP32 device tensor (the split-K workspace); None runs the unsplit kernels."""
    x, y = as_slice(x), as_slice(y)
    wsb = 0 if ws is None else ws.numel() * ws.element_size()
    _call("unet_conv3d_fwd", _p(x.buf), x.cs, x.c0, _p(w_bf16), _p(bias), _p(y.buf), y.cs, y.c0, n[0], n[1], n[2],
          cin, cout, int(relu), _p(ws), wsb, SPIN, _p(err), stream)


def conv3d_wgrad(x, dy, dw, n, cin, cout, err, stream=0):
    x, dy = as_slice(x), as_slice(dy)
    _call("unet_conv3d_wgrad", _p(x.buf), x.cs, x.c0, _p(dy.buf), dy.cs, dy.c0, _p(dw), n[0], n[1], n[2], cin, cout,
          SPIN, _p(err), stream)


def pack_weights(w, cin, cout, mode, out, stream=0):
    _call("unet_pack_weights", _p(w), cin, cout, mode, _p(out), stream)


def avgpool2(x, y, c, n, stream=0):
    x, y = as_slice(x), as_slice(y)
    _call("unet_avgpool2", _p(x.buf), x.cs, x.c0, _p(y.buf), y.cs, y.c0, c, n[0], n[1], n[2], stream)


def avgpool2_bwd(dy, dx, c, n, accumulate, stream=0):
    dy, dx = as_slice(dy), as_slice(dx)
    _call("unet_avgpool2_bwd", _p(dy.buf), dy.cs, dy.c0, _p(dx.buf), dx.cs, dx.c0, c, n[0], n[1], n[2],
          int(accumulate), stream)


def upsample2(x, y, c, n, stream=0):
    x, y = as_slice(x), as_slice(y)
    _call("unet_upsample2", _p(x.buf), x.cs, x.c0, _p(y.buf), y.cs, y.c0, c, n[0], n[1], n[2], stream)


def upsample2_bwd(dy, dx, c, n, stream=0):
    dy, dx = as_slice(dy), as_slice(dx)
    _call("unet_upsample2_bwd", _p(dy.buf), dy.cs, dy.c0, _p(dx.buf), dx.cs, dx.c0, c, n[0], n[1], n[2], stream)


def relu_bwd(dy, y, c, nvox, stream=0):
    dy, y = as_slice(dy), as_slice(y)
    _call("unet_relu_bwd", _p(dy.buf), dy.cs, dy.c0, _p(y.buf), y.cs, y.c0, c, nvox, stream)


def bias_grad(dy, db, c, nvox, stream=0):
    dy = as_slice(dy)
    _call("unet_bias_grad", _p(dy.buf), dy.cs, dy.c0, _p(db), c, nvox, stream)


def head_fwd(x, cin, w, b, out, cout, nvox, stream=0):
    x = as_slice(x)
    _call("unet_head_fwd", _p(x.buf), x.cs, x.c0, cin, _p(w), _p(b), _p(out), cout, nvox, stream)


def head_bwd(x, cin, w, dout, cout, dx, dw, db, nvox, stream=0):
    x, dx = as_slice(x), as_slice(dx)
    _call("unet_head_bwd", _p(x.buf), x.cs, x.c0, cin, _p(w), _p(dout), cout, _p(dx.buf), dx.cs, dx.c0, _p(dw),
          _p(db), nvox, stream)


def mse(out, target, dout, loss, c, nvox, stream=0):
    _call("unet_mse", _p(out), _p(target), _p(dout), _p(loss), c, nvox, stream)


def adam(p, g, m, v, lr, t, b1=0.9, b2=0.999, eps=1e-8, stream=0):
    _call("unet_adam", _p(p), _p(g), _p(m), _p(v), p.numel(), lr, b1, b2, eps, t, stream)


def pack_input(rho0, rho2, S, K, s_rho, s_S, s_K, x16, nvox, scratch, stream=0):
    _call("unet_pack_input", _p(rho0), _p(rho2), _p(S), K, s_rho, s_S, s_K, _p(x16), nvox, _p(scratch), stream)


def unpack_output(out4, s_u, s_W, u, W, nvox, scratch, stream=0):
    _call("unet_unpack_output", _p(out4), s_u, s_W, _p(u), _p(W), nvox, _p(scratch), stream)


def pack_target(u, W, s_u, s_W, t4, nvox, stream=0):
    _call("unet_pack_target", _p(u), _p(W), s_u, s_W, _p(t4), nvox, stream)


def restrict2_fields(fine, coarse, nfields, m, stream=0):
    _call("unet_restrict2_fields", _p(fine), _p(coarse), nfields, m[0], m[1], m[2], stream)


def prolong2_fields(coarse, fine, nfields, m, stream=0):
    _call("unet_prolong2_fields", _p(coarse), _p(fine), nfields, m[0], m[1], m[2], stream)
