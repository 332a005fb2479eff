"""Python driver for the FP64 C oracle (test infrastructure only).

Builds ``sf_oracle.c`` with gcc (OpenMP, -O2, no fast-math) into
``oracle/_build/`` and calls it through ctypes.  Complex data cross as
interleaved float64 (complex128 numpy arrays).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sf_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD_DIR, "libsf_oracle.so")
_lock = threading.Lock()


class _View(ctypes.Structure):
    _fields_ = [
        ("wavelength", ctypes.c_double), ("z", ctypes.c_double),
        ("px0", ctypes.c_double), ("py0", ctypes.c_double),
        ("px1", ctypes.c_double), ("py1", ctypes.c_double),
        ("ox0", ctypes.c_double), ("oy0", ctypes.c_double),
        ("ox1", ctypes.c_double), ("oy1", ctypes.c_double),
        ("nx0", ctypes.c_int), ("ny0", ctypes.c_int),
        ("nx1", ctypes.c_int), ("ny1", ctypes.c_int),
        ("no_prefactor", ctypes.c_int),
    ]


NO_PREFACTOR_FLAG = 1 << 2  # same bit the views use for "drop exp(ikz)/(i lambda z)"


def compile_oracle(src=_SRC, out=_LIB, extra=()):
    """Compile an oracle source file into a shared library; returns its path."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", "-std=c11", "-O2", "-fopenmp", "-fPIC", "-shared", *extra, src, "-o", out, "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return out


def build(force=False):
    """Build the oracle library if it is missing or older than its source."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            compile_oracle()
    return _LIB


class OracleLib:
    """ctypes handle on one compiled oracle library."""

    def __init__(self, path=None):
        self.path = path or build()
        lib = ctypes.CDLL(self.path)
        dp = ctypes.POINTER(ctypes.c_double)
        vp = ctypes.POINTER(_View)
        lib.sfo_forward.argtypes = [vp, dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int]
        lib.sfo_adjoint.argtypes = [vp, dp, dp, ctypes.c_int]
        lib.sfo_forward_dz.argtypes = [vp, dp, dp, ctypes.c_int]
        for f in (lib.sfo_forward, lib.sfo_adjoint, lib.sfo_forward_dz):
            f.restype = ctypes.c_int
        lib.sfo_max_threads.restype = ctypes.c_int
        self.lib = lib

    @staticmethod
    def _view(v):
        return _View(v["wavelength"], v["z"], v["px0"], v["py0"], v["px1"], v["py1"],
                     v["ox0"], v["oy0"], v["ox1"], v["oy1"],
                     v["nx0"], v["ny0"], v["nx1"], v["ny1"],
                     1 if (v.get("flags", 0) & NO_PREFACTOR_FLAG) else 0)

    @staticmethod
    def _c128(a, shape):
        a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
        if a.shape != shape:
            raise ValueError(f"expected shape {shape}, got {a.shape}")
        return a

    def forward(self, u0, v, cols=None, threads=0):
        """u1[:, cols] (complex128 [ny1, len(cols)]) for a contiguous column range."""
        c0, c1 = (0, v["nx1"]) if cols is None else cols
        u0 = self._c128(u0, (v["ny0"], v["nx0"]))
        out = np.empty((v["ny1"], c1 - c0), dtype=np.complex128)
        dp = ctypes.POINTER(ctypes.c_double)
        rc = self.lib.sfo_forward(ctypes.byref(self._view(v)), u0.ctypes.data_as(dp), c0, c1,
                                  out.ctypes.data_as(dp), threads)
        if rc != 0:
            raise ValueError(f"oracle forward failed ({rc})")
        return out

    def adjoint(self, g, v, threads=0):
        g = self._c128(g, (v["ny1"], v["nx1"]))
        out = np.empty((v["ny0"], v["nx0"]), dtype=np.complex128)
        dp = ctypes.POINTER(ctypes.c_double)
        rc = self.lib.sfo_adjoint(ctypes.byref(self._view(v)), g.ctypes.data_as(dp),
                                  out.ctypes.data_as(dp), threads)
        if rc != 0:
            raise ValueError(f"oracle adjoint failed ({rc})")
        return out

    def forward_dz(self, u0, v, threads=0):
        u0 = self._c128(u0, (v["ny0"], v["nx0"]))
        out = np.empty((v["ny1"], v["nx1"]), dtype=np.complex128)
        dp = ctypes.POINTER(ctypes.c_double)
        rc = self.lib.sfo_forward_dz(ctypes.byref(self._view(v)), u0.ctypes.data_as(dp),
                                     out.ctypes.data_as(dp), threads)
        if rc != 0:
            raise ValueError(f"oracle forward_dz failed ({rc})")
        return out

    def max_threads(self):
        return int(self.lib.sfo_max_threads())


_default = None


def _lib():
    global _default
    if _default is None:
        _default = OracleLib()
    return _default


def forward(u0, v, cols=None, threads=0):
    """Eqs. 1-4: complex view u1 (complex128 [ny1, nx1] or the given column range)."""
    return _lib().forward(u0, v, cols, threads)


def adjoint(g, v, threads=0):
    """Conjugate transpose of ``forward``: complex128 [ny0, nx0]."""
    return _lib().adjoint(g, v, threads)


def forward_dz(u0, v, threads=0):
    """Derivative of ``forward`` with respect to z: complex128 [ny1, nx1]."""
    return _lib().forward_dz(u0, v, threads)


def intensity(u1):
    """Eq. 5: I = |u1|^2."""
    return np.abs(u1) ** 2


def phase(u1):
    """Phase image in (-pi, pi]; 0 where u1 = 0."""
    p = np.arctan2(u1.imag, u1.real)
    return np.where(p <= -np.pi, np.pi, p)


def max_threads():
    return _lib().max_threads()
