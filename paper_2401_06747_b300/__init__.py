"""B300-native homogeneous diffusion inpainting and data optimisation.

Thin Python binding over libhdi.so (include/hdi.h). Every step of the solvers
runs in the library's CUDA kernels; this module only marshals arguments.
PyTorch tensors (CUDA or CPU) and NumPy arrays are accepted: CUDA tensors
are passed as device pointers, CPU tensors / arrays as host buffers, which
the library stages through its own workspace. There is no CPU fallback:
loading fails loudly if the library is missing.
"""

from __future__ import annotations

import ctypes
import json
import os

import numpy as np

from .build import LIB

HDI_OK = 0
ERRORS = {
    -1: "INVALID_ARG", -2: "EMPTY_MASK", -3: "NOT_CONVERGED", -4: "OUT_OF_MEMORY",
    -5: "CUDA", -6: "NONFINITE", -7: "TIMEOUT", -8: "UNSUPPORTED",
}
F32, F64 = 0, 1
DEVICE, HOST = 0, 1


class HdiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"hdi error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class Image(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("height", ctypes.c_int32), ("width", ctypes.c_int32),
                ("channels", ctypes.c_int32), ("dtype", ctypes.c_int32), ("row_stride", ctypes.c_int64),
                ("channel_stride", ctypes.c_int64), ("location", ctypes.c_int32)]


class Mask(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("height", ctypes.c_int32), ("width", ctypes.c_int32),
                ("row_stride", ctypes.c_int64), ("location", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iterations", ctypes.c_int32), ("vcycles", ctypes.c_int32),
                ("init_steps", ctypes.c_int32), ("local_iters", ctypes.c_int64), ("rel_res", ctypes.c_double),
                ("mse", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


SYMBOLS = ["hdi_create", "hdi_destroy", "hdi_set_param", "hdi_get_param", "hdi_inpaint",
           "hdi_tonal_opt", "hdi_densify_step", "hdi_densify", "hdi_last_error", "hdi_version", "hdi_launch_count",
           "hdi_timing", "hdi_timing_bytes", "hdi_timing_name", "hdi_inpaint_noalloc", "hdi_inpaint_batch",
           "hdi_engine_create", "hdi_engine_destroy", "hdi_engine_submit", "hdi_engine_step", "hdi_engine_status",
           "hdi_engine_request_bytes", "hdi_engine_launch_count", "hdi_engine_last_error", "hdi_workspace_bytes"]
TIMING_CLASSES = 9

_lib = None


def load(path: str | None = None):
    """Load libhdi.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("HDI_LIBRARY") or LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libhdi.so not found at {path}; run paper_2401_06747_b300/build.py")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    lib.hdi_create.argtypes = [P(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p, ctypes.c_char_p]
    lib.hdi_destroy.argtypes = [ctypes.c_void_p]
    lib.hdi_set_param.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_double]
    lib.hdi_get_param.argtypes = [ctypes.c_void_p, ctypes.c_char_p, P(ctypes.c_double)]
    lib.hdi_inpaint.argtypes = [ctypes.c_void_p, P(Image), P(Mask), P(Image), P(Image), ctypes.c_double, P(Stats)]
    lib.hdi_tonal_opt.argtypes = [ctypes.c_void_p, P(Image), P(Mask), P(Image), P(Image), ctypes.c_double, P(Stats)]
    lib.hdi_densify_step.argtypes = [ctypes.c_void_p, P(Image), P(Mask), P(Image), ctypes.c_int64,
                                     ctypes.c_uint64, P(ctypes.c_int64)]
    lib.hdi_densify.argtypes = [ctypes.c_void_p, P(Image), P(Mask), P(Image), ctypes.c_int32, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64, P(ctypes.c_int64)]
    lib.hdi_last_error.argtypes = [ctypes.c_void_p]
    lib.hdi_last_error.restype = ctypes.c_char_p
    lib.hdi_version.restype = ctypes.c_char_p
    lib.hdi_launch_count.argtypes = [ctypes.c_void_p]
    lib.hdi_launch_count.restype = ctypes.c_int64
    lib.hdi_workspace_bytes.argtypes = [ctypes.c_void_p]
    lib.hdi_workspace_bytes.restype = ctypes.c_int64
    lib.hdi_timing.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, P(ctypes.c_double), P(ctypes.c_int64)]
    lib.hdi_timing_bytes.argtypes = [ctypes.c_void_p, P(ctypes.c_double)]
    lib.hdi_timing_name.restype = ctypes.c_char_p
    lib.hdi_inpaint_batch.argtypes = [ctypes.c_void_p, ctypes.c_int, P(Image), P(Mask), P(Image), ctypes.c_double,
                                      P(Stats)]
    lib.hdi_inpaint_noalloc.argtypes = [ctypes.c_int, ctypes.c_void_p, P(Image), P(Mask), P(Image),
                                        ctypes.c_double, P(Stats)]
    lib.hdi_engine_create.argtypes = [P(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p, ctypes.c_char_p,
                                      ctypes.c_double]
    lib.hdi_engine_destroy.argtypes = [ctypes.c_void_p]
    lib.hdi_engine_submit.argtypes = [ctypes.c_void_p, P(Image), P(Mask), P(Image), ctypes.c_double, ctypes.c_int64]
    lib.hdi_engine_step.argtypes = [ctypes.c_void_p, P(ctypes.c_int64), P(Stats), ctypes.c_int, P(ctypes.c_int)]
    lib.hdi_engine_status.argtypes = [ctypes.c_void_p, P(ctypes.c_int64), P(ctypes.c_int64), P(ctypes.c_int64)]
    lib.hdi_engine_request_bytes.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
    lib.hdi_engine_request_bytes.restype = ctypes.c_int64
    lib.hdi_engine_launch_count.argtypes = [ctypes.c_void_p]
    lib.hdi_engine_launch_count.restype = ctypes.c_int64
    lib.hdi_engine_last_error.argtypes = [ctypes.c_void_p]
    lib.hdi_engine_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def image_of(x) -> Image:
    """Describe a (H, W) or (C, H, W) float32/float64 tensor or array."""
    if _is_torch(x):
        import torch
        if x.dim() == 2:
            x = x.unsqueeze(0)
        dt = {torch.float32: F32, torch.float64: F64}.get(x.dtype)
        if dt is None:
            raise TypeError("image must be float32 or float64")
        if x.stride(2) != 1:
            raise ValueError("image rows must be contiguous")
        loc = DEVICE if x.is_cuda else HOST
        return Image(x.data_ptr(), x.shape[1], x.shape[2], x.shape[0], dt, x.stride(1), x.stride(0), loc)
    a = x if x.ndim == 3 else x[None]
    if a.dtype not in (np.float32, np.float64):
        raise TypeError("image must be float32 or float64")
    es = a.itemsize
    if a.strides[2] != es:
        raise ValueError("image rows must be contiguous")
    return Image(a.ctypes.data, a.shape[1], a.shape[2], a.shape[0], F64 if a.dtype == np.float64 else F32,
                 a.strides[1] // es, a.strides[0] // es, HOST)


def mask_of(m) -> Mask:
    if _is_torch(m):
        import torch
        if m.dtype != torch.uint8 or m.dim() != 2 or m.stride(1) != 1:
            raise TypeError("mask must be a 2-D uint8 tensor with contiguous rows")
        return Mask(m.data_ptr(), m.shape[0], m.shape[1], m.stride(0), DEVICE if m.is_cuda else HOST)
    if m.dtype != np.uint8 or m.ndim != 2 or m.strides[1] != 1:
        raise TypeError("mask must be a 2-D uint8 array with contiguous rows")
    return Mask(m.ctypes.data, m.shape[0], m.shape[1], m.strides[0], HOST)


class Context:
    """One libhdi context (device, stream, workspace)."""

    def __init__(self, device: int = 0, stream=None, **params):
        self.lib = load()
        self.h = ctypes.c_void_p()
        s = 0
        if stream is not None:
            s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        cfg = json.dumps({k: float(v) for k, v in params.items()}).encode() if params else None
        rc = self.lib.hdi_create(ctypes.byref(self.h), device, ctypes.c_void_p(s), cfg)
        if rc != HDI_OK:
            raise HdiError(rc, "hdi_create failed" + (f" (config {cfg.decode()})" if cfg else ""))

    def close(self):
        if self.h:
            self.lib.hdi_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow_not_converged=False):
        if rc == HDI_OK or (allow_not_converged and rc == -3):
            return rc
        raise HdiError(rc, self.lib.hdi_last_error(self.h).decode())

    def set_param(self, name: str, value: float):
        self._check(self.lib.hdi_set_param(self.h, name.encode(), float(value)))

    def get_param(self, name: str) -> float:
        v = ctypes.c_double()
        self._check(self.lib.hdi_get_param(self.h, name.encode(), ctypes.byref(v)))
        return v.value

    def inpaint(self, f, mask, out, u0=None, tol: float = 1e-6, allow_not_converged=False) -> dict:
        """Solve (C + (I-C)L) u = C f into `out` (same shape/dtype as f)."""
        fi, mi, oi = image_of(f), mask_of(mask), image_of(out)
        ui = image_of(u0) if u0 is not None else None
        st = Stats()
        rc = self.lib.hdi_inpaint(self.h, ctypes.byref(fi), ctypes.byref(mi),
                                  ctypes.byref(ui) if ui is not None else None, ctypes.byref(oi),
                                  float(tol), ctypes.byref(st))
        self._check(rc, allow_not_converged)
        return st.as_dict()

    def inpaint_batch(self, fs, masks, outs, tol: float = 1e-6, allow_not_converged=False) -> list:
        """Batched inpainting of independent images of any sizes (lists of
        tensors/arrays): one launch per solver phase over all of them."""
        n = len(fs)
        FI = (Image * n)(*[image_of(x) for x in fs])
        MI = (Mask * n)(*[mask_of(x) for x in masks])
        OI = (Image * n)(*[image_of(x) for x in outs])
        ST = (Stats * n)()
        rc = self.lib.hdi_inpaint_batch(self.h, n, FI, MI, OI, float(tol), ST)
        self._check(rc, allow_not_converged)
        return [s.as_dict() for s in ST]

    def tonal_opt(self, f, mask, out, g0=None, tol: float = 1e-6, allow_not_converged=False) -> dict:
        """Optimised tonal values g (zero off the mask) into `out`."""
        fi, mi, oi = image_of(f), mask_of(mask), image_of(out)
        gi = image_of(g0) if g0 is not None else None
        st = Stats()
        rc = self.lib.hdi_tonal_opt(self.h, ctypes.byref(fi), ctypes.byref(mi),
                                    ctypes.byref(gi) if gi is not None else None, ctypes.byref(oi),
                                    float(tol), ctypes.byref(st))
        self._check(rc, allow_not_converged)
        return st.as_dict()

    def densify_step(self, f, mask, u, k: int, seed: int = 0) -> int:
        """Add up to k mask pixels in place; returns the number added."""
        fi, mi = image_of(f), mask_of(mask)
        ui = image_of(u) if u is not None else None
        added = ctypes.c_int64()
        rc = self.lib.hdi_densify_step(self.h, ctypes.byref(fi), ctypes.byref(mi),
                                       ctypes.byref(ui) if ui is not None else None, int(k),
                                       ctypes.c_uint64(seed), ctypes.byref(added))
        self._check(rc)
        return added.value

    def densify(self, f, mask, u, n: int = 20, t: float = 1.0, density: float = 0.05, seed: int = 0) -> list:
        """Densification loop into `mask` (in/out) and its inpainting into `u`;
        returns the mask size after every iteration."""
        fi, mi, ui = image_of(f), mask_of(mask), image_of(u)
        sizes = (ctypes.c_int64 * n)()
        rc = self.lib.hdi_densify(self.h, ctypes.byref(fi), ctypes.byref(mi), ctypes.byref(ui), int(n), float(t),
                                  float(density), ctypes.c_uint64(seed), sizes)
        self._check(rc)
        return list(sizes)


    def launch_count(self) -> int:
        return self.lib.hdi_launch_count(self.h)

    def workspace_bytes(self) -> int:
        """Device bytes the context's workspaces hold now (they grow to the
        largest call served and stay until the context is closed)."""
        return self.lib.hdi_workspace_bytes(self.h)

    def timing(self, enable: bool = True, reset: bool = False) -> dict:
        """Per-class device time {name: (ms, launches)} since the last reset."""
        ms = (ctypes.c_double * TIMING_CLASSES)()
        n = (ctypes.c_int64 * TIMING_CLASSES)()
        self._check(self.lib.hdi_timing(self.h, int(enable), int(reset), ms, n))
        return {self.lib.hdi_timing_name(i).decode(): (ms[i], n[i]) for i in range(TIMING_CLASSES)}

    def timing_bytes(self) -> dict:
        """Algorithmic HBM bytes of the timed launches per class {name: bytes}
        since the last timing reset (0 for the classes that do not count them)."""
        b = (ctypes.c_double * TIMING_CLASSES)()
        self._check(self.lib.hdi_timing_bytes(self.h, b))
        return {self.lib.hdi_timing_name(i).decode(): b[i] for i in range(TIMING_CLASSES)}


class Engine:
    """Batched inpainting engine (hdi_engine_*): requests of any size are
    submitted while their workspaces fit the budget, every step advances all
    requests in flight by one V-cycle (new ones by full multigrid) with one
    launch per solver phase, and finished requests are returned by step()."""

    def __init__(self, device: int = 0, stream=None, budget_gb: float = 120.0, **params):
        self.lib = load()
        self.h = ctypes.c_void_p()
        s = 0
        if stream is not None:
            s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        cfg = json.dumps({k: float(v) for k, v in params.items()}).encode() if params else None
        rc = self.lib.hdi_engine_create(ctypes.byref(self.h), device, ctypes.c_void_p(s), cfg, float(budget_gb))
        if rc != HDI_OK:
            raise HdiError(rc, "hdi_engine_create failed")
        self._held = {}   # tag -> buffers that must outlive the request

    def close(self):
        if self.h:
            self.lib.hdi_engine_destroy(self.h)
            self.h = ctypes.c_void_p()
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, f, mask, out, tol: float = 1e-6, tag: int = 0) -> bool:
        """Admit one request; False (nothing changed) if its workspace does not
        fit the budget now."""
        fi, mi, oi = image_of(f), mask_of(mask), image_of(out)
        rc = self.lib.hdi_engine_submit(self.h, ctypes.byref(fi), ctypes.byref(mi), ctypes.byref(oi), float(tol),
                                        int(tag))
        if rc == -4:
            return False
        if rc != HDI_OK:
            raise HdiError(rc, self.lib.hdi_engine_last_error(self.h).decode())
        self._held[int(tag)] = (f, mask, out)
        return True

    def step(self, capacity: int = 1024) -> list:
        """One step; returns [(tag, stats dict)] of the requests that finished."""
        tags = (ctypes.c_int64 * capacity)()
        sts = (Stats * capacity)()
        nd = ctypes.c_int()
        rc = self.lib.hdi_engine_step(self.h, tags, sts, capacity, ctypes.byref(nd))
        if rc != HDI_OK:
            raise HdiError(rc, self.lib.hdi_engine_last_error(self.h).decode())
        out = []
        for i in range(nd.value):
            self._held.pop(int(tags[i]), None)
            out.append((int(tags[i]), sts[i].as_dict()))
        return out

    def status(self) -> dict:
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self.lib.hdi_engine_status(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        return {"in_flight": a.value, "bytes_in_use": b.value, "budget_bytes": c.value}

    def launch_count(self) -> int:
        return self.lib.hdi_engine_launch_count(self.h)

    @staticmethod
    def request_bytes(height: int, width: int, channels: int) -> int:
        """Workspace bytes the engine reserves for one request of this shape."""
        return load().hdi_engine_request_bytes(int(height), int(width), int(channels))


def inpaint_noalloc(f, mask, out, tol: float = 1e-6, device: int = 0, stream=None) -> dict:
    """hdi_inpaint_noalloc: inpainting for callers that must not allocate
    device memory while they run. f, mask and out must be CUDA tensors; the
    workspace is the library's static 24 MiB device array, so images beyond
    about 500,000 pixel x channel values are refused and calls on one device
    that overlap race with each other."""
    lib = load()
    s = 0
    if stream is not None:
        s = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    st = Stats()
    rc = lib.hdi_inpaint_noalloc(device, ctypes.c_void_p(s), ctypes.byref(image_of(f)), ctypes.byref(mask_of(mask)),
                                 ctypes.byref(image_of(out)), float(tol), ctypes.byref(st))
    if rc != HDI_OK and rc != -3:
        raise HdiError(rc, "hdi_inpaint_noalloc failed")
    return st.as_dict()


def version() -> str:
    return load().hdi_version().decode()
