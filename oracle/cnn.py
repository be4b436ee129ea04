"""numpy wrappers of the FP64 CNN oracle (cnn_oracle.c); test infrastructure.

Arrays are float64, C order: inputs [N, 2, H, W], outputs/targets/loss
weights [N, H, W], parameters flat (see cnn_oracle.c for the layout).
"""
from __future__ import annotations

import ctypes

import numpy as np

LAYERS = [(2, 32, 1), (32, 32, 2), (32, 32, 4), (32, 1, 8)]   # (Cin, Cout, dilation)


def _register(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    i = ctypes.c_int
    lib.oracle_cnn_param_count.restype = i
    lib.oracle_bf16.argtypes = [ctypes.c_double]
    lib.oracle_bf16.restype = ctypes.c_double
    lib.oracle_conv3x3_fwd.argtypes = [i, i, i, i, i, i, dp, dp, dp, dp]
    lib.oracle_conv3x3_bwd.argtypes = [i, i, i, i, i, i, dp, dp, dp, dp, dp, dp]
    lib.oracle_cnn_forward.argtypes = [i, i, i, dp, dp, dp, dp, i]
    lib.oracle_cnn_forward.restype = i
    lib.oracle_cnn_loss_grad.argtypes = [i, i, i, dp, dp, dp, dp, dp, dp, i]
    lib.oracle_cnn_loss_grad.restype = ctypes.c_double
    lib.oracle_adam.argtypes = [i, dp, dp, dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, i]


def _lib():
    from . import _load
    return _load()


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def param_count() -> int:
    return int(_lib().oracle_cnn_param_count())


def layer_slices():
    """[(w_slice, b_slice, Cin, Cout, dil)] into the flat parameter vector."""
    out, o = [], 0
    for cin, cout, d in LAYERS:
        nw = cout * cin * 9
        out.append((slice(o, o + nw), slice(o + nw, o + nw + cout), cin, cout, d))
        o += nw + cout
    return out


def bf16(x):
    f = np.vectorize(lambda v: _lib().oracle_bf16(float(v)))
    return f(np.asarray(x, dtype=np.float64))


def conv3x3(x, w, b, dil):
    x, w = _c(x), _c(w)
    N, Cin, H, W = x.shape
    Cout = w.shape[0]
    y = np.zeros((N, Cout, H, W))
    _lib().oracle_conv3x3_fwd(N, H, W, Cin, Cout, dil, _p(x), _p(w), _p(_c(b)) if b is not None else None, _p(y))
    return y


def conv3x3_bwd(x, w, dy, dil):
    x, w, dy = _c(x), _c(w), _c(dy)
    N, Cin, H, W = x.shape
    Cout = w.shape[0]
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    db = np.zeros(Cout)
    _lib().oracle_conv3x3_bwd(N, H, W, Cin, Cout, dil, _p(x), _p(w), _p(dy), _p(dx), _p(dw), _p(db))
    return dx, dw, db


def forward(params, x, round_bf16=True, return_acts=False):
    params, x = _c(params), _c(x)
    N, _, H, W = x.shape
    out = np.zeros((N, H, W))
    acts = np.zeros(N * H * W * (32 * 3 + 1)) if return_acts else None
    rc = _lib().oracle_cnn_forward(N, H, W, _p(params), _p(x), _p(out), _p(acts), int(round_bf16))
    if rc != 0:
        raise MemoryError("oracle_cnn_forward")
    return (out, acts) if return_acts else out


def loss_grad(params, x, target, lam=None, round_bf16=True, want_grad_x=False):
    params, x, target = _c(params), _c(x), _c(target)
    N, _, H, W = x.shape
    g = np.zeros_like(params)
    gx = np.zeros_like(x) if want_grad_x else None
    lam = _c(lam) if lam is not None else None
    loss = _lib().oracle_cnn_loss_grad(N, H, W, _p(params), _p(x), _p(target), _p(lam), _p(g), _p(gx),
                                       int(round_bf16))
    return (loss, g, gx) if want_grad_x else (loss, g)


def adam(p, m, v, g, lr, t, b1=0.9, b2=0.999, eps=1e-8):
    p, m, v, g = _c(p).copy(), _c(m).copy(), _c(v).copy(), _c(g)
    _lib().oracle_adam(p.size, _p(p), _p(m), _p(v), _p(g), lr, b1, b2, eps, t)
    return p, m, v
