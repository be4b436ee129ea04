"""GB300 (sm_103a) complex-valued Frequency Selective Extrapolation.

Thin Python binding of the C ABI declared in ``include/fse.h``: the functions
below carry the C names and only marshal arguments; every step of the
computation runs in the CUDA kernels of ``libfse.so``.  PyTorch is used for
device memory and streams only.  There is no CPU fallback: if the library
cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = ["fse_class", "fse_config", "fse_block", "FseError", "fse_create", "fse_extrapolate_batch",
           "fse_extrapolate_batch_host", "fse_extrapolate_batch_noalloc", "fse_get_trace", "fse_last_error", "fse_destroy", "Engine",
           "fse_measure_smem_bandwidth",
           "library_path", "FSE_DTYPE_U8", "FSE_DTYPE_F32", "FSE_FLAG_TRACE", "FSE_FLAG_FIXED_W",
           "FSE_FIXED_W_FROM", "FSE_INIT_ZERO", "FSE_INIT_LEARNED"]

FSE_MAX_CLASSES = 4
FSE_DTYPE_U8, FSE_DTYPE_F32 = 0, 1
FSE_INIT_ZERO, FSE_INIT_LEARNED = 0, 1
FSE_FLAG_TRACE = 1
FSE_FLAG_ORDERED = 2
FSE_FLAG_CLAMP_U8 = 4
FSE_FLAG_FIXED_W = 8
FSE_FIXED_W_FROM = 20     # FP32 residual updates before the switch to 16-bit W
STATUS = {0: "FSE_OK", 1: "FSE_ERR_INVALID_ARG", 2: "FSE_ERR_UNSUPPORTED", 3: "FSE_ERR_CUDA",
          4: "FSE_ERR_OOM", 5: "FSE_ERR_TIMEOUT", 6: "FSE_ERR_NOT_TRAINED"}


class fse_class(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("border", ctypes.c_int), ("fft", ctypes.c_int),
                ("rho", ctypes.c_float), ("gamma", ctypes.c_float), ("iters", ctypes.c_int),
                ("frames", ctypes.c_int)]


class fse_config(ctypes.Structure):
    _fields_ = [("n_classes", ctypes.c_int), ("cls", fse_class * FSE_MAX_CLASSES),
                ("init", ctypes.c_int), ("init_iters", ctypes.c_int), ("device", ctypes.c_int),
                ("flags", ctypes.c_uint), ("reuse_weight", ctypes.c_float)]


class fse_block(ctypes.Structure):
    _fields_ = [("image", ctypes.c_int32), ("x", ctypes.c_int32), ("y", ctypes.c_int32),
                ("cls", ctypes.c_int32)]


class FseError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    """The library this process loads: libfse.so, or the bounds-checked
    libfse_checked.so when the environment sets FSE_BOUNDS_CHECK=1."""
    return _build.LIB_CHECKED if os.environ.get("FSE_BOUNDS_CHECK") == "1" else _build.LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if _build.needs_build():
                _build.build_library()
            lib = ctypes.CDLL(library_path())
            vp, c_int, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
            lib.fse_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(fse_config)]
            lib.fse_extrapolate_batch.argtypes = [vp, vp, c_int, c_int, c_int, c_int, sz, vp, vp, c_int,
                                                  vp, vp, vp]
            lib.fse_extrapolate_batch_host.argtypes = [vp, vp, c_int, c_int, c_int, c_int, sz, vp, vp,
                                                       c_int, vp, vp]
            lib.fse_extrapolate_batch_init.argtypes = [vp, vp, c_int, c_int, c_int, c_int, sz, vp, vp, c_int,
                                                       vp, sz, vp, vp, vp]
            lib.fse_load_init_weights.argtypes = [vp, vp, sz]
            lib.fse_get_area_model.argtypes = [vp, vp, sz, vp]
            lib.fse_sync.argtypes = [vp]
            lib.fse_set_wait_limit.argtypes = [vp, ctypes.c_ulonglong]
            lib.fse_set_tuning.argtypes = [vp, c_int]
            lib.fse_get_tuning.argtypes = [vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]
            lib.fse_test_clear_tuning_cache.argtypes = []
            lib.fse_test_clear_tuning_cache.restype = None
            lib.fse_extrapolate_batch_noalloc.argtypes = [ctypes.POINTER(fse_class), c_int, vp, c_int, c_int,
                                                          c_int, c_int, sz, vp, vp, c_int, vp, vp]
            lib.fse_get_trace.argtypes = [vp, vp, vp, vp, sz, ctypes.POINTER(c_int)]
            lib.fse_get_trace_gap.argtypes = [vp, vp, sz]
            lib.fse_test_fail_allocation.argtypes = [c_int]
            lib.fse_test_fail_allocation.restype = None
            lib.fse_test_live_allocations.argtypes = []
            lib.fse_test_live_allocations.restype = ctypes.c_longlong
            lib.fse_measure_smem_bandwidth.argtypes = [c_int, ctypes.POINTER(ctypes.c_double)]
            lib.fse_measure_smem_bandwidth.restype = c_int
            lib.fse_last_error.argtypes = [vp]
            lib.fse_last_error.restype = ctypes.c_char_p
            lib.fse_destroy.argtypes = [vp]
            lib.fse_destroy.restype = None
            for n in ("fse_create", "fse_extrapolate_batch", "fse_extrapolate_batch_host",
                      "fse_extrapolate_batch_noalloc", "fse_get_trace", "fse_extrapolate_batch_init",
                      "fse_load_init_weights", "fse_get_area_model", "fse_sync", "fse_set_wait_limit",
                      "fse_get_trace_gap", "fse_set_tuning", "fse_get_tuning"):
                getattr(lib, n).restype = c_int
            fp = ctypes.POINTER(ctypes.c_float)
            lib.fse_cnn_param_count.restype = sz
            lib.fse_cnn_create.argtypes = [ctypes.POINTER(vp), c_int, c_int, c_int, c_int]
            lib.fse_cnn_set_params.argtypes = [vp, vp, sz]
            lib.fse_cnn_get_params.argtypes = [vp, vp, sz]
            lib.fse_cnn_forward.argtypes = [vp, vp, c_int, vp, vp]
            lib.fse_cnn_get_state.argtypes = [vp, vp, vp, vp, ctypes.POINTER(ctypes.c_longlong)]
            lib.fse_cnn_set_state.argtypes = [vp, vp, vp, vp, ctypes.c_longlong]
            lib.fse_cnn_loss_grad.argtypes = [vp, vp, vp, vp, c_int, vp, fp, vp]
            lib.fse_cnn_train_step.argtypes = [vp, vp, vp, vp, c_int, ctypes.c_float, fp, vp]
            lib.fse_cnn_last_error.argtypes = [vp]
            lib.fse_cnn_last_error.restype = ctypes.c_char_p
            lib.fse_cnn_destroy.argtypes = [vp]
            lib.fse_cnn_destroy.restype = None
            for n in ("fse_cnn_create", "fse_cnn_set_params", "fse_cnn_get_params", "fse_cnn_forward",
                      "fse_cnn_loss_grad", "fse_cnn_train_step", "fse_cnn_get_state", "fse_cnn_set_state"):
                getattr(lib, n).restype = c_int
            _lib = lib
    return _lib


def _check(status: int, h):
    if status != 0:
        raise FseError(status, fse_last_error(h))


# ------------------------------------------------------------ C-ABI mirror
def fse_last_error(h) -> str:
    return _load().fse_last_error(h).decode()


def fse_create(cfg: fse_config):
    """fse_create(): returns an opaque handle (c_void_p)."""
    h = ctypes.c_void_p()
    st = _load().fse_create(ctypes.byref(h), ctypes.byref(cfg))
    _check(st, None)
    return h


def fse_extrapolate_batch(h, images: int, dtype: int, n_images: int, height: int, width: int,
                          pitch_bytes: int, loss_mask: int, blocks: np.ndarray, n_blocks: int,
                          out: int | None, patches: int | None, stream: int | None) -> None:
    """Device-pointer entry point; ``blocks`` is a host int32 [n, 4] array or
    the address (int) of such an array in device memory."""
    if isinstance(blocks, int):
        bptr = blocks if n_blocks else None
    else:
        blocks = np.ascontiguousarray(blocks, dtype=np.int32).reshape(-1, 4)
        bptr = blocks.ctypes.data if n_blocks else None
    st = _load().fse_extrapolate_batch(h, images, dtype, n_images, height, width, pitch_bytes,
                                       loss_mask, bptr, n_blocks, out, patches, stream)
    _check(st, h)


def fse_extrapolate_batch_init(h, images: int, dtype: int, n_images: int, height: int, width: int,
                               pitch_bytes: int, loss_mask: int, blocks: np.ndarray, n_blocks: int,
                               init_estimate: int, est_stride: int, out: int | None, patches: int | None,
                               stream: int | None) -> None:
    """Warm start from caller estimates (device pointer, block i at i * est_stride)."""
    blocks = np.ascontiguousarray(blocks, dtype=np.int32).reshape(-1, 4)
    st = _load().fse_extrapolate_batch_init(h, images, dtype, n_images, height, width, pitch_bytes, loss_mask,
                                            blocks.ctypes.data if n_blocks else None, n_blocks, init_estimate,
                                            est_stride, out, patches, stream)
    _check(st, h)


def fse_load_init_weights(h, params: np.ndarray) -> None:
    params = np.ascontiguousarray(params, dtype=np.float32)
    _check(_load().fse_load_init_weights(h, params.ctypes.data, params.size), h)


def fse_extrapolate_batch_host(h, images: np.ndarray, dtype: int, n_images: int, height: int,
                               width: int, pitch_bytes: int, loss_mask: np.ndarray,
                               blocks: np.ndarray, n_blocks: int, patches: np.ndarray,
                               stream: int | None) -> None:
    """Host-buffer entry point (numpy arrays, C-contiguous)."""
    blocks = np.ascontiguousarray(blocks, dtype=np.int32).reshape(-1, 4)
    st = _load().fse_extrapolate_batch_host(h, images.ctypes.data, dtype, n_images, height, width,
                                            pitch_bytes, loss_mask.ctypes.data,
                                            blocks.ctypes.data if n_blocks else None, n_blocks,
                                            patches.ctypes.data, stream)
    _check(st, h)


def fse_extrapolate_batch_noalloc(classes, images: int, dtype: int, n_images: int, height: int,
                                  width: int, pitch_bytes: int, loss_mask: int, blocks: np.ndarray,
                                  n_blocks: int, out: int, stream: int | None) -> None:
    """Handle-free entry point that allocates no device memory (its scratch is
    a fixed array inside the library); ``classes`` is a list of class dicts,
    ``blocks`` a host int32 [n, 4] array, the other buffers device pointers."""
    arr = (fse_class * len(classes))(*[
        fse_class(int(c["block"]), int(c["border"]), int(c["fft"]), float(c["rho"]), float(c["gamma"]),
                  int(c["iters"]), int(c.get("frames", 0))) for c in classes])
    blocks = np.ascontiguousarray(blocks, dtype=np.int32).reshape(-1, 4)
    st = _load().fse_extrapolate_batch_noalloc(arr, len(classes), images, dtype, n_images, height, width,
                                               pitch_bytes, loss_mask,
                                               blocks.ctypes.data if n_blocks else None, n_blocks, out,
                                               stream)
    _check(st, None)


def fse_get_trace(h, n_blocks: int):
    """Returns (sel int32 [n, stride], energy float32 [n, stride], coef complex64 [n, stride])."""
    stride = ctypes.c_int(0)
    lib = _load()
    _check(lib.fse_get_trace(h, None, None, None, 0, ctypes.byref(stride)), h)
    n = n_blocks * stride.value
    sel = np.zeros(max(n, 1), np.int32)
    en = np.zeros(max(n, 1), np.float32)
    co = np.zeros(2 * max(n, 1), np.float32)
    _check(lib.fse_get_trace(h, sel.ctypes.data, en.ctypes.data, co.ctypes.data, max(n, 1),
                             ctypes.byref(stride)), h)
    s = stride.value
    return (sel[:n].reshape(n_blocks, s), en[:n].reshape(n_blocks, s),
            (co[0:2 * n:2] + 1j * co[1:2 * n:2]).astype(np.complex64).reshape(n_blocks, s))


def fse_get_trace_gap(h, n_blocks: int) -> np.ndarray:
    """Top-two gap (e1 - e2) / e1 of every selection, float32 [n, stride]."""
    stride = ctypes.c_int(0)
    lib = _load()
    _check(lib.fse_get_trace(h, None, None, None, 0, ctypes.byref(stride)), h)
    n = n_blocks * stride.value
    gap = np.zeros(max(n, 1), np.float32)
    _check(lib.fse_get_trace_gap(h, gap.ctypes.data, max(n, 1)), h)
    return gap[:n].reshape(n_blocks, stride.value)


def fse_get_area_model(h, model: int, model_stride: int, stream: int | None) -> None:
    _check(_load().fse_get_area_model(h, model, model_stride, stream), h)


def fse_sync(h) -> None:
    _check(_load().fse_sync(h), h)


def fse_set_wait_limit(h, ns: int) -> None:
    _check(_load().fse_set_wait_limit(h, int(ns)), h)


FSE_TUNE_SYNC, FSE_TUNE_ASYNC, FSE_TUNE_OFF = 0, 1, 2
TUNE_MODES = {"sync": FSE_TUNE_SYNC, "async": FSE_TUNE_ASYNC, "off": FSE_TUNE_OFF}


def fse_set_tuning(h, mode: int) -> None:
    _check(_load().fse_set_tuning(h, int(mode)), h)


def fse_get_tuning(h):
    """(mode, class mixes still being timed asynchronously)."""
    m, p = ctypes.c_int(0), ctypes.c_int(0)
    _check(_load().fse_get_tuning(h, ctypes.byref(m), ctypes.byref(p)), h)
    return m.value, p.value


def fse_test_clear_tuning_cache() -> None:
    _load().fse_test_clear_tuning_cache()


def fse_measure_smem_bandwidth(device: int = 0) -> float:
    """Measured shared-memory load bandwidth of the device in GB/s."""
    out = ctypes.c_double(0.0)
    _check(_load().fse_measure_smem_bandwidth(device, ctypes.byref(out)), None)
    return float(out.value)


def fse_destroy(h) -> None:
    if h is not None:
        _load().fse_destroy(h)


# ------------------------------------------------ learned-init network ABI
FSE_CNN_PARAMS = 19393


def _cnn_check(status: int, c):
    if status != 0:
        raise FseError(status, _load().fse_cnn_last_error(c).decode())


def fse_cnn_create(device: int, height: int, width: int, max_batch: int):
    c = ctypes.c_void_p()
    _cnn_check(_load().fse_cnn_create(ctypes.byref(c), device, height, width, max_batch), None)
    return c


def fse_cnn_set_params(c, params: np.ndarray) -> None:
    params = np.ascontiguousarray(params, dtype=np.float32)
    _cnn_check(_load().fse_cnn_set_params(c, params.ctypes.data, params.size), c)


def fse_cnn_get_params(c) -> np.ndarray:
    out = np.zeros(FSE_CNN_PARAMS, np.float32)
    _cnn_check(_load().fse_cnn_get_params(c, out.ctypes.data, out.size), c)
    return out


def fse_cnn_get_state(c):
    """(params, m, v, step): the network's full training state."""
    p, m, v = (np.zeros(FSE_CNN_PARAMS, np.float32) for _ in range(3))
    step = ctypes.c_longlong(0)
    _cnn_check(_load().fse_cnn_get_state(c, p.ctypes.data, m.ctypes.data, v.ctypes.data, ctypes.byref(step)), c)
    return p, m, v, int(step.value)


def fse_cnn_set_state(c, params, m, v, step: int) -> None:
    p, m, v = (np.ascontiguousarray(a, dtype=np.float32) for a in (params, m, v))
    _cnn_check(_load().fse_cnn_set_state(c, p.ctypes.data, m.ctypes.data, v.ctypes.data, int(step)), c)


def fse_cnn_forward(c, x: int, n: int, y: int, stream: int | None) -> None:
    _cnn_check(_load().fse_cnn_forward(c, x, n, y, stream), c)


def fse_cnn_loss_grad(c, x: int, target: int, lam: int | None, n: int, stream: int | None):
    g = np.zeros(FSE_CNN_PARAMS, np.float32)
    loss = ctypes.c_float(0.0)
    _cnn_check(_load().fse_cnn_loss_grad(c, x, target, lam, n, g.ctypes.data, ctypes.byref(loss), stream), c)
    return float(loss.value), g


def fse_cnn_train_step(c, x: int, target: int, lam: int | None, n: int, lr: float, stream: int | None,
                       want_loss: bool = True):
    loss = ctypes.c_float(0.0)
    _cnn_check(_load().fse_cnn_train_step(c, x, target, lam, n, lr, ctypes.byref(loss) if want_loss else None,
                                          stream), c)
    return float(loss.value) if want_loss else None


def fse_cnn_destroy(c) -> None:
    if c is not None:
        _load().fse_cnn_destroy(c)


class Cnn:
    """The learned-initialisation network on one device (torch tensors in,
    torch tensors out; every computation runs in libfse.so)."""

    def __init__(self, height: int = 48, width: int = 48, max_batch: int = 256, device: int = 0):
        self.H, self.W, self.max_batch, self.device = height, width, max_batch, device
        self.c = fse_cnn_create(device, height, width, max_batch)

    def set_params(self, p):
        fse_cnn_set_params(self.c, p)

    def get_params(self):
        return fse_cnn_get_params(self.c)

    def get_state(self):
        """(params, m, v, step): parameters, Adam moments and step count."""
        return fse_cnn_get_state(self.c)

    def set_state(self, params, m, v, step):
        fse_cnn_set_state(self.c, params, m, v, step)

    def _stream(self):
        import torch
        return torch.cuda.current_stream(self.device).cuda_stream

    def forward(self, x):
        import torch
        assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous() and x.shape[1:] == (2, self.H, self.W)
        y = torch.empty((x.shape[0], self.H, self.W), dtype=torch.float32, device=x.device)
        fse_cnn_forward(self.c, x.data_ptr(), x.shape[0], y.data_ptr(), self._stream())
        return y

    def loss_grad(self, x, target, lam=None):
        return fse_cnn_loss_grad(self.c, x.data_ptr(), target.data_ptr(),
                                 lam.data_ptr() if lam is not None else None, x.shape[0], self._stream())

    def train_step(self, x, target, lam=None, lr=1e-3, want_loss=True):
        return fse_cnn_train_step(self.c, x.data_ptr(), target.data_ptr(),
                                  lam.data_ptr() if lam is not None else None, x.shape[0], lr, self._stream(),
                                  want_loss)

    def close(self):
        if self.c is not None:
            fse_cnn_destroy(self.c)
            self.c = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def he_init(seed: int) -> np.ndarray:
    """Seeded He-normal initial parameters (biases zero) in the flat layout."""
    rng = np.random.default_rng(seed)
    out = []
    for cin, cout in ((2, 32), (32, 32), (32, 32), (32, 1)):
        out.append(rng.normal(0.0, np.sqrt(2.0 / (9 * cin)), size=cout * cin * 9))
        out.append(np.zeros(cout))
    return np.concatenate(out).astype(np.float32)


# --------------------------------------------------------- convenience API
def make_config(classes, device: int = 0, trace: bool = False, init: str = "zero",
                init_iters: int = 0, ordered: bool = False, reuse_weight: float = 0.5,
                clamp_u8: bool = False, fixed_w: bool = False) -> fse_config:
    cfg = fse_config()
    cfg.n_classes = len(classes)
    for i, c in enumerate(classes):
        cfg.cls[i] = fse_class(int(c["block"]), int(c["border"]), int(c["fft"]), float(c["rho"]),
                               float(c["gamma"]), int(c["iters"]), int(c.get("frames", 0)))
    cfg.init = FSE_INIT_LEARNED if init == "learned" else FSE_INIT_ZERO
    cfg.init_iters = int(init_iters)
    cfg.device = device
    cfg.flags = ((FSE_FLAG_TRACE if trace else 0) | (FSE_FLAG_ORDERED if ordered else 0)
                 | (FSE_FLAG_CLAMP_U8 if clamp_u8 else 0) | (FSE_FLAG_FIXED_W if fixed_w else 0))
    cfg.reuse_weight = float(reuse_weight)
    return cfg


class Engine:
    """A handle plus torch-tensor marshalling.

    classes: list of dicts with keys block, border, fft, rho, gamma, iters.
    fixed_w: reduced-precision residual storage (FSE_FLAG_FIXED_W: 16-bit
    fixed-point W after the first FSE_FIXED_W_FROM updates; fft 64 classes).
    """

    def __init__(self, classes, device: int = 0, trace: bool = False, init: str = "zero", init_iters: int = 0,
                 weights=None, ordered: bool = False, reuse_weight: float = 0.5, clamp_u8: bool = False,
                 fixed_w: bool = False):
        self.classes = [dict(c) for c in classes]
        self.h = fse_create(make_config(classes, device, trace, init, init_iters, ordered, reuse_weight,
                                        clamp_u8, fixed_w))
        self.last_n = 0
        if weights is not None:
            fse_load_init_weights(self.h, weights)

    def load_init_weights(self, weights):
        fse_load_init_weights(self.h, weights)

    def patch_total(self, blocks) -> int:
        b = np.array([self.classes[int(c)]["block"] for c in np.asarray(blocks).reshape(-1, 4)[:, 3]])
        return int(np.sum(b * b)) if b.size else 0

    def run(self, images, mask, blocks, out=None, patches=None, stream=None) -> None:
        """images: cuda uint8/float32 [N, H, W] (row pitch may exceed W);
        mask: cuda uint8 [N, H, W] contiguous; blocks: int32 [n, 4]."""
        import torch
        assert images.is_cuda and mask.is_cuda and mask.dtype == torch.uint8 and mask.is_contiguous()
        N, H, W = images.shape
        dtype = FSE_DTYPE_U8 if images.dtype == torch.uint8 else FSE_DTYPE_F32
        if dtype == FSE_DTYPE_F32:
            assert images.dtype == torch.float32
        assert images.stride(2) == 1 and (N == 1 or images.stride(0) == H * images.stride(1)), \
            "images must be [N, H, W] with unit column stride and image stride H * row stride"
        pitch = images.stride(1) * images.element_size()
        blocks = np.ascontiguousarray(blocks, dtype=np.int32).reshape(-1, 4)
        if stream is None:
            stream = torch.cuda.current_stream(images.device).cuda_stream
        for t in (out, patches):
            if t is not None:
                assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
        fse_extrapolate_batch(self.h, images.data_ptr(), dtype, N, H, W, pitch, mask.data_ptr(), blocks,
                              len(blocks), out.data_ptr() if out is not None else None,
                              patches.data_ptr() if patches is not None else None, stream)
        self.last_n = len(blocks)

    def run_init(self, images, mask, blocks, est, out=None, patches=None, stream=None) -> None:
        """Warm start: est is a cuda float32 [n_blocks, M*M] (or wider) tensor of
        per-block area estimates in sample units."""
        import torch
        N, H, W = images.shape
        dtype = FSE_DTYPE_U8 if images.dtype == torch.uint8 else FSE_DTYPE_F32
        pitch = images.stride(1) * images.element_size()
        blocks = np.ascontiguousarray(blocks, dtype=np.int32).reshape(-1, 4)
        assert est.is_cuda and est.dtype == torch.float32 and est.is_contiguous() and est.shape[0] == len(blocks)
        if stream is None:
            stream = torch.cuda.current_stream(images.device).cuda_stream
        fse_extrapolate_batch_init(self.h, images.data_ptr(), dtype, N, H, W, pitch, mask.data_ptr(), blocks,
                                   len(blocks), est.data_ptr(), est.stride(0),
                                   out.data_ptr() if out is not None else None,
                                   patches.data_ptr() if patches is not None else None, stream)
        self.last_n = len(blocks)

    def run_host(self, images: np.ndarray, mask: np.ndarray, blocks, patches: np.ndarray = None):
        images = np.ascontiguousarray(images)
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        N, H, W = images.shape
        dtype = FSE_DTYPE_U8 if images.dtype == np.uint8 else FSE_DTYPE_F32
        if dtype == FSE_DTYPE_F32:
            images = np.ascontiguousarray(images, dtype=np.float32)
        blocks = np.ascontiguousarray(blocks, dtype=np.int32).reshape(-1, 4)
        if patches is None:
            patches = np.zeros(max(self.patch_total(blocks), 1), np.float32)
        fse_extrapolate_batch_host(self.h, images, dtype, N, H, W, W * images.itemsize, mask, blocks,
                                   len(blocks), patches, None)
        self.last_n = len(blocks)
        return patches

    def trace(self):
        return fse_get_trace(self.h, self.last_n)

    def trace_gap(self):
        """Top-two gap of every selection of the last batch (trace handles)."""
        return fse_get_trace_gap(self.h, self.last_n)

    def sync(self):
        """Wait for the last launch; raises FseError(FSE_ERR_TIMEOUT) when a
        bounded device-side wait expired, FseError(FSE_ERR_INVALID_ARG) when a
        block's loss area was not marked lost in the mask."""
        fse_sync(self.h)

    def set_wait_limit(self, ns: int):
        """Limit of the bounded device waits in nanoseconds (default 1 s)."""
        fse_set_wait_limit(self.h, ns)

    def set_tuning(self, mode: str):
        """How new class mixes choose their launch shape: "sync" (default:
        the first call times the candidates and waits), "async" (no call
        waits; candidates are timed on the real launches) or "off"."""
        fse_set_tuning(self.h, TUNE_MODES[mode])

    def tuning(self):
        """(mode name, class mixes still being timed asynchronously)."""
        m, p = fse_get_tuning(self.h)
        return {v: k for k, v in TUNE_MODES.items()}[m], p

    def area_model(self, stream=None):
        """Re{g} over every block's M x M area of the last batch (trace
        handles only): cuda float32 [n_blocks, max M*M]."""
        import torch
        mm = max((c["block"] + 2 * c["border"]) ** 2 for c in self.classes)
        out = torch.zeros((self.last_n, mm), dtype=torch.float32, device="cuda")
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        fse_get_area_model(self.h, out.data_ptr() if self.last_n else None, mm, stream)
        return out

    def close(self):
        if self.h is not None:
            fse_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
