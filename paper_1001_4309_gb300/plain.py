"""ctypes wrapper of the cuFFT comparison library (the paper's steps 2-10 per view).

Used by the benchmark and its parity test only; the product path never
calls it.
"""

from __future__ import annotations

import ctypes
import os

from . import build as _build
from .binding import sf_view, make_view

_lib = None


def load():
    global _lib
    if _lib is None:
        path = _build.plain_library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing; call paper_1001_4309_gb300.build.build_plain() first")
        lib = ctypes.CDLL(path)
        vp, pp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)
        lib.sf_plain_create.argtypes = [pp, ctypes.POINTER(sf_view), ctypes.c_int, ctypes.c_int]
        lib.sf_plain_execute.argtypes = [vp, vp, pp, pp, vp]
        lib.sf_plain_destroy.argtypes = [vp]
        for f in ("sf_plain_create", "sf_plain_execute", "sf_plain_destroy"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


class PlainPath:
    """Plan of the cuFFT procedure for a set of views of one hologram."""

    def __init__(self, views, device=0):
        import torch
        self.torch = torch
        self.views = [dict(v) for v in views]
        self.device = torch.device("cuda", device)
        arr = (sf_view * len(views))(*[make_view(v) for v in views])
        h = ctypes.c_void_p()
        rc = load().sf_plain_create(ctypes.byref(h), arr, len(views), device)
        if rc != 0:
            raise RuntimeError(f"sf_plain_create failed ({rc})")
        self.handle = h

    def execute(self, holo, fields, intensities=None, stream=None):
        t = self.torch
        arr = lambda xs: (ctypes.c_void_p * len(xs))(*[x.data_ptr() if x is not None else None for x in xs])  # noqa
        s = stream if stream is not None else t.cuda.current_stream(self.device).cuda_stream
        rc = load().sf_plain_execute(self.handle, holo.data_ptr(), arr(fields),
                                     arr(intensities) if intensities is not None else None,
                                     ctypes.c_void_p(s) if s else None)
        if rc != 0:
            raise RuntimeError(f"sf_plain_execute failed ({rc})")

    def close(self):
        if getattr(self, "handle", None):
            load().sf_plain_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
