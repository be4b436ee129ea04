"""FP64 CPU oracle for complex-valued Frequency Selective Extrapolation.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports this package, and this package never imports the product.

The numerical kernels live in plain C (``fse_oracle.c``, ``cnn_oracle.c``,
``fse3_oracle.c`` for video volumes), compiled with gcc into
``liboracle.so`` beside them; this module wraps them with numpy arrays.
``image`` holds the image-level driver (gather of the extrapolation area,
Eq. (3) weighting, fill of the loss area; warm start, video volumes and
ordered concealment), ``cnn`` the learned-initialisation network.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["fse_oracle.c", "cnn_oracle.c", "fse3_oracle.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (portable flags only) into liboracle.so."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    stale = force or not os.path.exists(_LIB_PATH) or any(
        os.path.getmtime(s) > os.path.getmtime(_LIB_PATH) for s in srcs)
    if stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
               "-std=c11", "-o", tmp] + srcs + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int32)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            lib.oracle_fft2.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int]
            lib.oracle_dft2_direct.argtypes = [ctypes.c_int, dp, dp, dp, dp, ctypes.c_int]
            lib.oracle_weight.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, u8p, dp]
            lib.oracle_cfse.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_double, ctypes.c_int,
                                        ip, ip, dp, dp, dp, dp, dp, dp, dp]
            lib.oracle_cfse_fixw.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_int, ip, ip, dp, dp, dp, dp, dp, dp, dp]
            lib.oracle_fix_code.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.oracle_fix_code.restype = ctypes.c_int
            lib.oracle_cfse_spatial.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_double,
                                                ctypes.c_int, ip, dp, dp, dp]
            lib.oracle_fft3.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int]
            lib.oracle_weight3.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, u8p, dp]
            lib.oracle_cfse3.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_double, ctypes.c_int,
                                         ip, ip, dp, dp, dp, dp]
            lib.oracle_cfse3_spatial.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_double,
                                                 ctypes.c_int, ip, dp, dp]
            for name in ("oracle_fft2", "oracle_cfse", "oracle_cfse_fixw", "oracle_cfse_spatial", "oracle_fft3", "oracle_cfse3",
                         "oracle_cfse3_spatial"):
                getattr(lib, name).restype = ctypes.c_int
            if hasattr(lib, "oracle_conv3x3_fwd"):
                from . import cnn as _cnn  # noqa: F401  (registers CNN prototypes)
                _cnn._register(lib)
            _lib = lib
    return _lib


def _ptr(a, ctype=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _split(s):
    """(real part, imaginary part or None) as contiguous float64 arrays."""
    s = np.asarray(s)
    if np.iscomplexobj(s):
        return (np.ascontiguousarray(s.real, dtype=np.float64),
                np.ascontiguousarray(s.imag, dtype=np.float64))
    return np.ascontiguousarray(s, dtype=np.float64), None


def fft2(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Unnormalised 2-D DFT (forward sign e^{-j}) of a square power-of-two array."""
    x = np.asarray(x, dtype=np.complex128)
    F = x.shape[0]
    assert x.shape == (F, F)
    re = np.ascontiguousarray(x.real).copy()
    im = np.ascontiguousarray(x.imag).copy()
    if _load().oracle_fft2(F, _ptr(re), _ptr(im), 1 if inverse else -1) != 0:
        raise ValueError("F must be a power of two")
    return re + 1j * im


def dft2_direct(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Eq. (7) evaluated literally, O(F^4)."""
    x = np.asarray(x, dtype=np.complex128)
    F = x.shape[0]
    re = np.ascontiguousarray(x.real).copy()
    im = np.ascontiguousarray(x.imag).copy()
    ore = np.zeros((F, F))
    oim = np.zeros((F, F))
    _load().oracle_dft2_direct(F, _ptr(re), _ptr(im), _ptr(ore), _ptr(oim), 1 if inverse else -1)
    return ore + 1j * oim


def weight(M: int, N: int, rho: float, support: np.ndarray) -> np.ndarray:
    """Eq. (3) weighting function on an M x N area (support != 0 marks A)."""
    sup = np.ascontiguousarray(support, dtype=np.uint8)
    assert sup.shape == (M, N)
    w = np.zeros((M, N))
    _load().oracle_weight(M, N, float(rho), _ptr(sup, ctypes.c_uint8), _ptr(w))
    return w


class CfseResult:
    """Outputs of one run of Algorithm 1 (see ``cfse``)."""

    def __init__(self, sel, coef, e_sel, e_max, e_second, g, R, W):
        self.sel = sel            # int32[I] linear index k*F+l
        self.coef = coef          # complex[I]
        self.e_sel = e_sel        # float[I] |R_w[u,v]|^2 before the update
        self.e_max = e_max        # float[I] max |R_w|^2 before the update
        self.e_second = e_second  # float[I] runner-up energy
        self.g = g                # complex[F,F] model IFFT{G}
        self.R = R                # complex[F,F] residual spectrum after I iterations
        self.W = W                # complex[F,F] spectrum of w


def fix_code(x: float, W00: float) -> int:
    """16-bit fixed-point code of a spectrum value x of W: x / W[0,0] in units
    of 1/32767, rounded to nearest (ties to even, decided in FP32), held to
    [-32767, 32767].  The code stands for code * W00 / 32767."""
    return int(_load().oracle_fix_code(float(x), float(W00)))


def cfse(s: np.ndarray, w: np.ndarray, gamma: float, iters: int,
         forced: np.ndarray | None = None, wfix_from: int | None = None) -> CfseResult:
    """Algorithm 1 on an F x F grid (w real, 0 off the support area; s real or
    complex).

    ``forced`` replaces each iteration's argmax by the given linear index
    (guided replay); the recorded energies still describe the oracle's own
    residual at that point, so callers can check that each forced pick is an
    epsilon-argmax.

    ``wfix_from`` = K makes the residual updates of iterations K, K+1, ...
    (0-based) read W in 16-bit fixed point (``fix_code``; reduced-precision
    residual storage); None keeps every update in FP64.
    """
    s_re, s_im = _split(s)
    w = np.ascontiguousarray(w, dtype=np.float64)
    F = s_re.shape[0]
    assert s_re.shape == (F, F) and w.shape == (F, F)
    I = int(iters)
    sel = np.zeros(max(I, 1), np.int32)
    coef = np.zeros(2 * max(I, 1))
    e_sel = np.zeros(max(I, 1))
    e_max = np.zeros(max(I, 1))
    e_sec = np.zeros(max(I, 1))
    g = np.zeros(2 * F * F)
    R = np.zeros(2 * F * F)
    W = np.zeros(2 * F * F)
    fp = None
    if forced is not None:
        fp = np.ascontiguousarray(forced, dtype=np.int32)
        assert fp.shape[0] >= I
    if wfix_from is None:
        rc = _load().oracle_cfse(F, _ptr(s_re), _ptr(s_im), _ptr(w), float(gamma), I,
                                 _ptr(fp, ctypes.c_int32),
                                 _ptr(sel, ctypes.c_int32), _ptr(coef), _ptr(e_sel), _ptr(e_max),
                                 _ptr(e_sec), _ptr(g), _ptr(R), _ptr(W))
    else:
        rc = _load().oracle_cfse_fixw(F, _ptr(s_re), _ptr(s_im), _ptr(w), float(gamma), I,
                                      max(0, int(wfix_from)), _ptr(fp, ctypes.c_int32),
                                      _ptr(sel, ctypes.c_int32), _ptr(coef), _ptr(e_sel),
                                      _ptr(e_max), _ptr(e_sec), _ptr(g), _ptr(R), _ptr(W))
    if rc != 0:
        raise ValueError("oracle_cfse: bad argument")
    cplx = lambda a: (a[0::2] + 1j * a[1::2]).reshape(F, F)  # noqa: E731
    return CfseResult(sel[:I].copy(), (coef[0::2] + 1j * coef[1::2])[:I].copy(), e_sel[:I].copy(),
                      e_max[:I].copy(), e_sec[:I].copy(), cplx(g), cplx(R), cplx(W))


def cfse_spatial(s: np.ndarray, w: np.ndarray, gamma: float, iters: int):
    """Brute-force spatial-domain cFSE; returns (sel, coef, crit, g)."""
    s_re, s_im = _split(s)
    w = np.ascontiguousarray(w, dtype=np.float64)
    F = s_re.shape[0]
    I = int(iters)
    sel = np.zeros(max(I, 1), np.int32)
    coef = np.zeros(2 * max(I, 1))
    crit = np.zeros(max(I, 1))
    g = np.zeros(2 * F * F)
    rc = _load().oracle_cfse_spatial(F, _ptr(s_re), _ptr(s_im), _ptr(w), float(gamma), I,
                                     _ptr(sel, ctypes.c_int32), _ptr(coef), _ptr(crit), _ptr(g))
    if rc != 0:
        raise ValueError("oracle_cfse_spatial: bad argument")
    return (sel[:I].copy(), (coef[0::2] + 1j * coef[1::2])[:I].copy(), crit[:I].copy(),
            (g[0::2] + 1j * g[1::2]).reshape(F, F))


# ----------------------------------------------------------------- 3-D (video)
def fft3(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Unnormalised 3-D DFT (forward sign e^{-j}) of an Ft x F x F array."""
    x = np.asarray(x, dtype=np.complex128)
    Ft, F = x.shape[0], x.shape[1]
    assert x.shape == (Ft, F, F)
    re = np.ascontiguousarray(x.real)
    im = np.ascontiguousarray(x.imag)
    if _load().oracle_fft3(Ft, F, _ptr(re), _ptr(im), 1 if inverse else -1) != 0:
        raise ValueError("oracle_fft3: sizes must be powers of two")
    return re + 1j * im


def weight3(T: int, M: int, rho: float, support: np.ndarray) -> np.ndarray:
    """Weighting function on a T x M x M volume (support != 0 marks A)."""
    sup = np.ascontiguousarray(support, dtype=np.uint8)
    assert sup.shape == (T, M, M)
    w = np.zeros((T, M, M))
    _load().oracle_weight3(T, M, float(rho), _ptr(sup, ctypes.c_uint8), _ptr(w))
    return w


def cfse3(s: np.ndarray, w: np.ndarray, gamma: float, iters: int,
          forced: np.ndarray | None = None) -> CfseResult:
    """Algorithm 1 on an Ft x F x F grid; bins indexed (t F + k) F + l.
    Returns a CfseResult with g of shape (Ft, F, F); e_second, R and W are not
    computed (None)."""
    s_re, s_im = _split(s)
    w = np.ascontiguousarray(w, dtype=np.float64)
    Ft, F = s_re.shape[0], s_re.shape[1]
    assert s_re.shape == (Ft, F, F) and w.shape == (Ft, F, F)
    I = int(iters)
    sel = np.zeros(max(I, 1), np.int32)
    coef = np.zeros(2 * max(I, 1))
    e_sel = np.zeros(max(I, 1))
    e_max = np.zeros(max(I, 1))
    g = np.zeros(2 * Ft * F * F)
    fp = None
    if forced is not None:
        fp = np.ascontiguousarray(forced, dtype=np.int32)
        assert fp.shape[0] >= I
    rc = _load().oracle_cfse3(Ft, F, _ptr(s_re), _ptr(s_im), _ptr(w), float(gamma), I, _ptr(fp, ctypes.c_int32),
                              _ptr(sel, ctypes.c_int32), _ptr(coef), _ptr(e_sel), _ptr(e_max), _ptr(g))
    if rc != 0:
        raise ValueError("oracle_cfse3: bad argument")
    return CfseResult(sel[:I].copy(), (coef[0::2] + 1j * coef[1::2])[:I].copy(), e_sel[:I].copy(),
                      e_max[:I].copy(), None, (g[0::2] + 1j * g[1::2]).reshape(Ft, F, F), None, None)


def cfse3_spatial(s: np.ndarray, w: np.ndarray, gamma: float, iters: int):
    """Brute-force spatial-domain cFSE on an Ft x F x F grid; returns
    (sel, coef, g)."""
    s_re, s_im = _split(s)
    w = np.ascontiguousarray(w, dtype=np.float64)
    Ft, F = s_re.shape[0], s_re.shape[1]
    I = int(iters)
    sel = np.zeros(max(I, 1), np.int32)
    coef = np.zeros(2 * max(I, 1))
    g = np.zeros(2 * Ft * F * F)
    rc = _load().oracle_cfse3_spatial(Ft, F, _ptr(s_re), _ptr(s_im), _ptr(w), float(gamma), I,
                                      _ptr(sel, ctypes.c_int32), _ptr(coef), _ptr(g))
    if rc != 0:
        raise ValueError("oracle_cfse3_spatial: bad argument")
    return sel[:I].copy(), (coef[0::2] + 1j * coef[1::2])[:I].copy(), (g[0::2] + 1j * g[1::2]).reshape(Ft, F, F)
