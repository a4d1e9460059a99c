"""Thin ctypes binding of the C ABI declared in include/cat.h.

Every function keeps the C name and only marshals arguments; all work runs in
libcat.so.  Loading fails loudly when the library is missing (build it with
``paper_2406_17284_gb300.build.build()``): there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

CAT_OK = 0
CAT_ERR_INVALID_ARG = -1
CAT_ERR_UNSUPPORTED = -2
CAT_ERR_OOM = -3
CAT_ERR_CUDA = -4
CAT_ERR_TIMEOUT = -5
CAT_ERR_STATE = -6

BOUNDARY_ZERO = 0
BOUNDARY_PERIODIC = 1

DTYPE_AUTO, DTYPE_FP16, DTYPE_FP8_E4M3, DTYPE_INT8, DTYPE_FP4_E2M1 = 0, 1, 2, 3, 4
STORE_U8, STORE_BIT1, STORE_NIB4 = 0, 1, 2
KERNEL_AUTO, KERNEL_TCGEN05, KERNEL_MMA_SYNC, KERNEL_STENCIL, KERNEL_BITSLICE, KERNEL_RUNSUM = 0, 1, 2, 3, 4, 5

DTYPES = {"auto": DTYPE_AUTO, "fp16": DTYPE_FP16, "fp8": DTYPE_FP8_E4M3, "int8": DTYPE_INT8,
          "fp4": DTYPE_FP4_E2M1}
KERNELS = {"auto": KERNEL_AUTO, "tcgen05": KERNEL_TCGEN05, "mma_sync": KERNEL_MMA_SYNC,
           "stencil": KERNEL_STENCIL, "bitslice": KERNEL_BITSLICE, "runsum": KERNEL_RUNSUM}

EXPORTED = ["cat_create", "cat_create_ex", "cat_bind", "cat_set_options", "cat_set_tile", "cat_set_state", "cat_get_state", "cat_state_ptr",
            "cat_step", "cat_batch_step", "cat_box_sums", "cat_status", "cat_debug_control",
            "cat_destroy", "cat_last_error", "cat_version", "cat_batch_step_static",
            "cat_tensor_probe", "cat_get_options", "cat_autotune", "cat_autotune_batch"]

CAT_TUNE_REMEASURE = 1
CAT_TUNE_NO_WRITE = 2

CAT_STATIC_MAX_GRIDS = 256
CAT_STATIC_MAX_TILES = 65536


class cat_rule_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("r", "C", "M", "s1", "s2", "b1", "b2", "nbhd")]


class cat_grid_desc_t(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("out", ctypes.c_void_p), ("H", ctypes.c_int64),
                ("W", ctypes.c_int64), ("pitch", ctypes.c_int64), ("rule", cat_rule_t)]


class CatError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (code {code})")
        self.code = code


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libcat.so (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        so = path or _build.LIB
        try:  # share torch's CUDA runtime when it is installed
            import torch  # noqa: F401
        except Exception:
            pass
        if not os.path.exists(so):
            raise ImportError(f"{so} is missing: build it with paper_2406_17284_gb300.build.build()")
        lib = ctypes.CDLL(so)
        h, i32, i64, p = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        sig = {
            "cat_create": [i64, i64, ctypes.POINTER(cat_rule_t), i32, ctypes.POINTER(ctypes.c_void_p)],
            "cat_create_ex": [i64, i64, ctypes.POINTER(cat_rule_t), i32, i32, ctypes.POINTER(ctypes.c_void_p)],
            "cat_set_options": [h, i32, i32, i32, i32],
            "cat_set_tile": [h, i32, i32, i32],
            "cat_set_state": [h, p, i64, i32, p],
            "cat_get_state": [h, p, i64, i32, p],
            "cat_state_ptr": [h, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int64)],
            "cat_bind": [h, p, p, i64],
            "cat_step": [h, i64, p],
            "cat_batch_step": [ctypes.POINTER(ctypes.c_void_p), i32, i64, p],
            "cat_box_sums": [h, p, i64, p],
            "cat_status": [h, p],
            "cat_debug_control": [h, i32, i64],
            "cat_destroy": [h],
            "cat_last_error": [],
            "cat_version": [],
            "cat_batch_step_static": [ctypes.POINTER(cat_grid_desc_t), i32, i32, p, p],
            "cat_tensor_probe": [i32, i64, p, p],
            "cat_get_options": [h] + [ctypes.POINTER(ctypes.c_int32)] * 6,
            "cat_autotune": [h, i32, ctypes.c_char_p, i32, p],
            "cat_autotune_batch": [ctypes.POINTER(ctypes.c_void_p), i32, i32, ctypes.POINTER(ctypes.c_int32), p],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_char_p if name in ("cat_last_error", "cat_version") else ctypes.c_int
        _lib = lib
        return lib


def _check(rc: int):
    if rc != CAT_OK:
        raise CatError(rc, load().cat_last_error().decode())


def _stream_ptr(stream) -> int | None:
    if stream is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_rule(r: int, C: int, M: int, s1: int, s2: int, b1: int, b2: int, nbhd: str = "M") -> cat_rule_t:
    return cat_rule_t(r, C, M, s1, s2, b1, b2, ord(nbhd))


# ------------------------------------------------------------- C-named calls
def cat_create(H: int, W: int, rule: cat_rule_t, boundary: int = BOUNDARY_ZERO) -> int:
    out = ctypes.c_void_p()
    _check(load().cat_create(H, W, ctypes.byref(rule), boundary, ctypes.byref(out)))
    return out.value


def cat_create_ex(H: int, W: int, rule: cat_rule_t, boundary: int = BOUNDARY_ZERO, storage: int = STORE_U8) -> int:
    out = ctypes.c_void_p()
    _check(load().cat_create_ex(H, W, ctypes.byref(rule), boundary, storage, ctypes.byref(out)))
    return out.value


def cat_set_options(h: int, kernel: int = KERNEL_AUTO, dtype: int = DTYPE_AUTO, storage: int = STORE_U8,
                    steps_per_launch: int = 1):
    _check(load().cat_set_options(h, kernel, dtype, storage, steps_per_launch))


def cat_set_tile(h: int, ty: int = 0, tx: int = 0, window_rows: int = 0):
    _check(load().cat_set_tile(h, ty, tx, window_rows))


def cat_set_state(h: int, src_ptr: int, pitch: int, on_device: bool, stream=None):
    _check(load().cat_set_state(h, src_ptr, pitch, int(on_device), _stream_ptr(stream)))


def cat_get_state(h: int, dst_ptr: int, pitch: int, on_device: bool, stream=None):
    _check(load().cat_get_state(h, dst_ptr, pitch, int(on_device), _stream_ptr(stream)))


def cat_state_ptr(h: int) -> tuple[int, int]:
    p, pitch = ctypes.c_void_p(), ctypes.c_int64()
    _check(load().cat_state_ptr(h, ctypes.byref(p), ctypes.byref(pitch)))
    return p.value, pitch.value


def cat_bind(h: int, a_ptr: int, b_ptr: int, pitch: int):
    _check(load().cat_bind(h, a_ptr, b_ptr, pitch))


def cat_step(h: int, n_steps: int = 1, stream=None):
    _check(load().cat_step(h, n_steps, _stream_ptr(stream)))


def cat_batch_step(handles: list[int], n_steps: int = 1, stream=None):
    arr = (ctypes.c_void_p * len(handles))(*handles)
    _check(load().cat_batch_step(arr, len(handles), n_steps, _stream_ptr(stream)))


def cat_box_sums(h: int, dst_ptr: int, ld: int, stream=None):
    _check(load().cat_box_sums(h, dst_ptr, ld, _stream_ptr(stream)))


def cat_status(h: int, stream=None) -> int:
    return load().cat_status(h, _stream_ptr(stream))


def cat_debug_control(h: int, what: int, value: int):
    _check(load().cat_debug_control(h, what, value))


def cat_destroy(h: int):
    _check(load().cat_destroy(h))


def cat_batch_step_static(descs: list, dtype: int = DTYPE_FP8_E4M3, status_ptr: int | None = None,
                          stream=None) -> int:
    """One step of every grid in `descs` (cat_grid_desc_t) without device allocation."""
    arr = (cat_grid_desc_t * len(descs))(*descs)
    return load().cat_batch_step_static(arr, len(descs), dtype, status_ptr, _stream_ptr(stream))


def cat_tensor_probe(dtype: int, mmas_per_sm: int, status_ptr: int, stream=None):
    """Launches the dense tcgen05 MMA rate probe (flops per launch: SMs x
    mmas_per_sm x 2 x 128 x 256 x K, K = 32 for FP8 e4m3, 16 for FP16)."""
    _check(load().cat_tensor_probe(dtype, mmas_per_sm, status_ptr, _stream_ptr(stream)))


def cat_get_options(h: int) -> dict:
    v = [ctypes.c_int32() for _ in range(6)]
    _check(load().cat_get_options(h, *[ctypes.byref(x) for x in v]))
    return dict(zip(("kernel", "dtype", "storage", "steps_per_launch", "tile", "window"), (x.value for x in v)))


def cat_autotune(h: int, n_steps: int = 8, cache_path: str | None = None, flags: int = 0, stream=None):
    _check(load().cat_autotune(h, n_steps, cache_path.encode() if cache_path else None, flags,
                               _stream_ptr(stream)))


def cat_autotune_batch(handles: list[int], n_steps: int = 4, stream=None) -> int:
    arr = (ctypes.c_void_p * len(handles))(*handles)
    d = ctypes.c_int32()
    _check(load().cat_autotune_batch(arr, len(handles), n_steps, ctypes.byref(d), _stream_ptr(stream)))
    return d.value


def cat_version() -> str:
    return load().cat_version().decode()


# ----------------------------------------------------------- convenience API
class Grid:
    """One LTL instance: owns a cat handle; state in/out as numpy or torch tensors."""

    def __init__(self, H: int, W: int, rule: dict, kernel: str = "tcgen05", dtype: str = "fp8",
                 boundary: int = BOUNDARY_ZERO, storage: int = STORE_U8, steps_per_launch: int = 1,
                 tile: int = 0, window: int = 0):
        self.H, self.W = int(H), int(W)
        self.rule = dict(rule)
        self.storage = int(storage)
        self.handle = cat_create_ex(self.H, self.W, make_rule(**{k: rule[k] for k in
                                                                 ("r", "C", "M", "s1", "s2", "b1", "b2")},
                                                              nbhd=rule.get("nbhd", "M")),
                                    boundary, self.storage)
        try:
            cat_set_options(self.handle, KERNELS[kernel], DTYPES[dtype], self.storage, steps_per_launch)
            if tile or window:
                cat_set_tile(self.handle, tile, tile, window)
        except Exception:
            cat_destroy(self.handle)
            self.handle = None   # __del__ must not free it again
            raise

    def close(self):
        if self.handle:
            cat_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, grid, stream=None):
        import torch
        if isinstance(grid, np.ndarray):
            g = np.ascontiguousarray(grid, dtype=np.uint8)
            assert g.shape == (self.H, self.W)
            cat_set_state(self.handle, g.ctypes.data, self.W, False, stream)
            if stream is None:
                torch.cuda.current_stream().synchronize()
        else:
            assert grid.dtype == torch.uint8 and tuple(grid.shape) == (self.H, self.W)
            g = grid.contiguous()
            cat_set_state(self.handle, g.data_ptr(), g.stride(0), g.is_cuda, stream)

    def get_state(self, stream=None) -> np.ndarray:
        import torch
        out = np.empty((self.H, self.W), dtype=np.uint8)
        cat_get_state(self.handle, out.ctypes.data, self.W, False, stream)
        (torch.cuda.current_stream() if stream is None else stream).synchronize()
        return out

    def state_tensor(self):
        """Zero-copy torch view of the current device buffer (H x pitch, uint8):
        H x W cells, or H x ceil(W / 8) / ceil(W / 2) packed bytes with one- /
        four-bit storage."""
        import torch
        ptr, pitch = cat_state_ptr(self.handle)

        class _Arr:
            __cuda_array_interface__ = {"shape": (self.H, pitch), "typestr": "|u1",
                                        "data": (ptr, False), "version": 3}
        cols = {STORE_BIT1: (self.W + 7) // 8, STORE_NIB4: (self.W + 1) // 2}.get(self.storage, self.W)
        return torch.as_tensor(_Arr(), device="cuda")[:, :cols]

    def step(self, n_steps: int = 1, stream=None):
        cat_step(self.handle, n_steps, stream)

    def box_sums(self, stream=None) -> np.ndarray:
        import torch
        S = torch.empty((self.H, self.W), dtype=torch.int32, device="cuda")
        cat_box_sums(self.handle, S.data_ptr(), self.W, stream)
        return S.cpu().numpy()

    def status(self, stream=None) -> int:
        return cat_status(self.handle, stream)
