"""Thin ctypes binding of the C ABI in include/shifted_fresnel.h.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Functions keep the C names; ``ShiftedFresnel`` is a convenience
wrapper that allocates torch tensors for the outputs and passes their device
pointers and the current torch stream.

Loading fails loudly (``RuntimeError``) when the compiled library is missing;
there is no fallback implementation.
"""

from __future__ import annotations

import ctypes
import os

from . import build as _build

SF_OK = 0
SF_ERR_INVALID_ARG = -1
SF_ERR_UNSUPPORTED_SIZE = -2
SF_ERR_CUDA = -3
SF_ERR_OOM = -4
SF_ERR_TIMEOUT = -5
SF_ERR_DEVICE_MISMATCH = -6

SF_OUT_INTENSITY = 1
SF_OUT_PHASE = 2
SF_NO_PREFACTOR = 4
SF_IN_COMPLEX = 8

SF_PREC_FP32 = 0
SF_PREC_FP16TC = 1
SF_PREC_BF16TC = 2
SF_PREC_FP16X3TC = 3
SF_PREC_BF16X3TC = 4
SF_MAX_CONV_LENGTH = 8192


class SFError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {shifted_fresnel_strerror(code)} ({code})")


class sf_view(ctypes.Structure):
    _fields_ = [
        ("wavelength", ctypes.c_double), ("z", ctypes.c_double),
        ("px0", ctypes.c_double), ("py0", ctypes.c_double),
        ("px1", ctypes.c_double), ("py1", ctypes.c_double),
        ("ox0", ctypes.c_double), ("oy0", ctypes.c_double),
        ("ox1", ctypes.c_double), ("oy1", ctypes.c_double),
        ("nx0", ctypes.c_int32), ("ny0", ctypes.c_int32),
        ("nx1", ctypes.c_int32), ("ny1", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
    ]


_lib = None


def library_path():
    return _build.library_path()


def load():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; call paper_1001_4309_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    vp, pp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)
    lib.shifted_fresnel_plan.argtypes = [pp, ctypes.POINTER(sf_view), ctypes.c_int, ctypes.c_int, ctypes.c_int, vp]
    lib.shifted_fresnel_execute.argtypes = [vp, vp, pp, pp, pp, vp]
    lib.shifted_fresnel_destroy.argtypes = [vp]
    lib.shifted_fresnel_plan_update.argtypes = [vp, ctypes.POINTER(sf_view), ctypes.c_int, vp]
    lib.shifted_fresnel_intensity_loss.argtypes = [vp, pp, pp, pp, vp, vp]
    lib.shifted_fresnel_intensity_loss.restype = ctypes.c_int
    lib.shifted_fresnel_plan_update.restype = ctypes.c_int
    lib.shifted_fresnel_strerror.argtypes = [ctypes.c_int]
    lib.shifted_fresnel_strerror.restype = ctypes.c_char_p
    lib.shifted_fresnel_plan_query.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int32),
                                               ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_size_t)]
    lib.shifted_fresnel_kernel_launches.restype = ctypes.c_uint64
    lib.shifted_fresnel_execute_static.argtypes = [ctypes.POINTER(sf_view), vp, vp, vp, vp, vp]
    lib.shifted_fresnel_execute_static.restype = ctypes.c_int
    lib.shifted_fresnel_execute_batch.argtypes = [vp, pp, ctypes.c_int, pp, pp, pp, vp]
    lib.shifted_fresnel_execute_batch.restype = ctypes.c_int
    lib.shifted_fresnel_batch_status.argtypes = [vp, vp]
    lib.shifted_fresnel_batch_status.restype = ctypes.c_int
    lib.shifted_fresnel_adjoint.argtypes = [vp, vp, pp, vp, vp, vp]
    lib.shifted_fresnel_adjoint.restype = ctypes.c_int
    lib.shifted_fresnel_set_profile_events.argtypes = [vp, pp, ctypes.c_int]
    lib.shifted_fresnel_set_profile_events.restype = ctypes.c_int
    lib.shifted_fresnel_fft_length.argtypes = [ctypes.c_int32, ctypes.c_int32]
    lib.shifted_fresnel_fft_length.restype = ctypes.c_int32
    for f in ("shifted_fresnel_plan", "shifted_fresnel_execute", "shifted_fresnel_destroy",
              "shifted_fresnel_plan_query"):
        getattr(lib, f).restype = ctypes.c_int
    _lib = lib
    return lib


def make_view(v):
    """sf_view from a dict with the keys of synth.view (or an sf_view)."""
    if isinstance(v, sf_view):
        return v
    return sf_view(v["wavelength"], v["z"], v["px0"], v["py0"], v["px1"], v["py1"],
                   v["ox0"], v["oy0"], v["ox1"], v["oy1"],
                   v["nx0"], v["ny0"], v["nx1"], v["ny1"], v.get("flags", 0))


def _ptr_array(ptrs):
    if ptrs is None:
        return None
    arr = (ctypes.c_void_p * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = p if p else None
    return arr


def shifted_fresnel_strerror(code):
    return load().shifted_fresnel_strerror(int(code)).decode()


def shifted_fresnel_plan(views, precision=SF_PREC_FP32, device=0, stream=0, check=True):
    """Create a plan; returns (status, handle) with check=False, else the handle."""
    arr = (sf_view * len(views))(*[make_view(v) for v in views])
    h = ctypes.c_void_p()
    rc = load().shifted_fresnel_plan(ctypes.byref(h), arr, len(views), precision, device,
                                     ctypes.c_void_p(stream) if stream else None)
    if not check:
        return rc, h
    if rc != SF_OK:
        raise SFError(rc, "shifted_fresnel_plan")
    return h


def shifted_fresnel_execute(plan, holo_ptr, view_out=None, intensity=None, phase=None, stream=0, check=True):
    """Run every view of the plan; pointers are ints (device or host addresses) or None."""
    rc = load().shifted_fresnel_execute(plan, ctypes.c_void_p(holo_ptr) if holo_ptr else None,
                                        _ptr_array(view_out), _ptr_array(intensity), _ptr_array(phase),
                                        ctypes.c_void_p(stream) if stream else None)
    if check and rc != SF_OK:
        raise SFError(rc, "shifted_fresnel_execute")
    return rc


def shifted_fresnel_execute_static(view, holo_ptr, view_out=None, intensity=None, phase=None, stream=0,
                                   check=True):
    """One view without a plan and without allocating (device pointers as ints, or None).

    For callers that cannot allocate device memory while running; the
    library's fixed scratch array is shared by all calls on a device.
    """
    v = make_view(view)
    p = lambda x: ctypes.c_void_p(x) if x else None  # noqa: E731
    rc = load().shifted_fresnel_execute_static(ctypes.byref(v), p(holo_ptr), p(view_out), p(intensity), p(phase),
                                               ctypes.c_void_p(stream) if stream else None)
    if check and rc != SF_OK:
        raise SFError(rc, "shifted_fresnel_execute_static")
    return rc


def shifted_fresnel_execute_batch(plan, holo_ptrs, view_out=None, intensity=None, phase=None, stream=0,
                                  check=True):
    """All views for each hologram in one persistent graph launch; outputs indexed h * n_views + v."""
    rc = load().shifted_fresnel_execute_batch(plan, _ptr_array(list(holo_ptrs)), len(holo_ptrs),
                                              _ptr_array(view_out), _ptr_array(intensity), _ptr_array(phase),
                                              ctypes.c_void_p(stream) if stream else None)
    if check and rc != SF_OK:
        raise SFError(rc, "shifted_fresnel_execute_batch")
    return rc


def shifted_fresnel_intensity_loss(plan, fields, measured, grads, loss_ptr, stream=0, check=True):
    """loss (device double) = sum_v ||(|u_v|^2 - I_v)||^2; grads[v] = 4 (|u_v|^2 - I_v) u_v (or grads None)."""
    rc = load().shifted_fresnel_intensity_loss(plan, _ptr_array(fields), _ptr_array(measured), _ptr_array(grads),
                                               ctypes.c_void_p(loss_ptr) if loss_ptr else None,
                                               ctypes.c_void_p(stream) if stream else None)
    if check and rc != SF_OK:
        raise SFError(rc, "shifted_fresnel_intensity_loss")
    return rc


def shifted_fresnel_batch_status(plan, stream=0):
    return load().shifted_fresnel_batch_status(plan, ctypes.c_void_p(stream) if stream else None)


def shifted_fresnel_adjoint(plan, holo_ptr, grad_view, grad_holo=None, grad_z=None, stream=0, check=True):
    """grad_holo = sum_v A_v^H g_v and grad_z[v] = Re sum conj(g_v) du1_v/dz (pointers as ints or None)."""
    p = lambda x: ctypes.c_void_p(x) if x else None  # noqa: E731
    rc = load().shifted_fresnel_adjoint(plan, p(holo_ptr), _ptr_array(list(grad_view)), p(grad_holo), p(grad_z),
                                        ctypes.c_void_p(stream) if stream else None)
    if check and rc != SF_OK:
        raise SFError(rc, "shifted_fresnel_adjoint")
    return rc


def shifted_fresnel_destroy(plan, check=True):
    rc = load().shifted_fresnel_destroy(plan)
    if check and rc != SF_OK:
        raise SFError(rc, "shifted_fresnel_destroy")
    return rc


def shifted_fresnel_plan_update(plan, views, stream=0, check=True):
    """New depths / pitches / offsets / wavelength for the plan's views (same sizes), in place."""
    arr = (sf_view * len(views))(*[make_view(v) for v in views])
    rc = load().shifted_fresnel_plan_update(plan, arr, len(views), ctypes.c_void_p(stream) if stream else None)
    if check and rc != SF_OK:
        raise SFError(rc, "shifted_fresnel_plan_update")
    return rc


def shifted_fresnel_plan_query(plan, view):
    lx, ly, ws = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_size_t()
    rc = load().shifted_fresnel_plan_query(plan, view, ctypes.byref(lx), ctypes.byref(ly), ctypes.byref(ws))
    if rc != SF_OK:
        raise SFError(rc, "shifted_fresnel_plan_query")
    return lx.value, ly.value, ws.value


def shifted_fresnel_set_profile_events(plan, events):
    """Attach three cudaEvent_t handles (ints, e.g. torch.cuda.Event().cuda_event) or detach with None."""
    if not events:
        rc = load().shifted_fresnel_set_profile_events(plan, None, 0)
    else:
        rc = load().shifted_fresnel_set_profile_events(plan, _ptr_array(list(events)), len(events))
    if rc != SF_OK:
        raise SFError(rc, "shifted_fresnel_set_profile_events")
    return rc


def shifted_fresnel_kernel_launches():
    return int(load().shifted_fresnel_kernel_launches())


def shifted_fresnel_fft_length(need, allow_mixed=True):
    """FFT length an untuned plan uses for an axis with n0 + n1 - 1 = need (negative status on error)."""
    return int(load().shifted_fresnel_fft_length(int(need), 1 if allow_mixed else 0))


class ShiftedFresnel:
    """Plan + execute over torch tensors (the views of one hologram).

    ``views`` are dicts as made by ``synth.view``.  ``reconstruct`` takes a
    hologram tensor (float32, or complex64 with SF_IN_COMPLEX) on the plan's
    device and returns per-view complex64 fields and optional float32
    intensity / phase images.
    """

    def __init__(self, views, device=None, precision=SF_PREC_FP32):
        import torch
        self.torch = torch
        self.views = [dict(v) for v in views]
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream(self.device).cuda_stream
            self.handle = shifted_fresnel_plan(self.views, precision=precision, device=self.device.index,
                                               stream=stream)

    def sizes(self, i):
        return shifted_fresnel_plan_query(self.handle, i)

    def update(self, views, stream=None):
        """Re-target the plan's views (same sizes) in place, ordered on the current stream."""
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device).cuda_stream
        shifted_fresnel_plan_update(self.handle, views, stream=s)
        self.views = [dict(v) for v in views]

    def alloc_outputs(self, field=True, intensity=False, phase=False):
        t = self.torch
        outs = {"field": [], "intensity": [], "phase": []}
        for v in self.views:
            shp = (v["ny1"], v["nx1"])
            outs["field"].append(t.empty(shp, dtype=t.complex64, device=self.device) if field else None)
            outs["intensity"].append(t.empty(shp, dtype=t.float32, device=self.device) if intensity else None)
            outs["phase"].append(t.empty(shp, dtype=t.float32, device=self.device) if phase else None)
        return outs

    def execute(self, holo, outs, stream=None):
        ptr = lambda x: x.data_ptr() if x is not None else None  # noqa: E731
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device).cuda_stream
        shifted_fresnel_execute(self.handle, holo.data_ptr(),
                                [ptr(x) for x in outs["field"]],
                                [ptr(x) for x in outs["intensity"]],
                                [ptr(x) for x in outs["phase"]], stream=s)
        return outs

    def reconstruct(self, holo, field=True, intensity=False, phase=False):
        outs = self.alloc_outputs(field, intensity, phase)
        return self.execute(holo, outs)

    def execute_batch(self, holos, outs, stream=None):
        """outs: dict of lists indexed [h][v] (from alloc_batch_outputs)."""
        ptr = lambda x: x.data_ptr() if x is not None else None  # noqa: E731
        flat = lambda key: ([ptr(o) for row in outs[key] for o in row]  # noqa: E731
                            if outs.get(key) and any(o is not None for row in outs[key] for o in row) else None)
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device).cuda_stream
        shifted_fresnel_execute_batch(self.handle, [h.data_ptr() for h in holos], flat("field"),
                                      flat("intensity"), flat("phase"), stream=s)
        return outs

    def alloc_batch_outputs(self, n_holos, field=True, intensity=False, phase=False):
        per = [self.alloc_outputs(field, intensity, phase) for _ in range(n_holos)]
        return {k: [o[k] for o in per] for k in ("field", "intensity", "phase")}

    def adjoint(self, grad_views, holo=None, grad_holo=None, grad_z=None, stream=None):
        """grad_holo (complex64 [ny0][nx0]) and grad_z (float64 [n_views]) from per-view gradients."""
        t = self.torch
        v0 = self.views[0]
        if grad_holo is None:
            grad_holo = t.empty((v0["ny0"], v0["nx0"]), dtype=t.complex64, device=self.device)
        s = stream if stream is not None else t.cuda.current_stream(self.device).cuda_stream
        shifted_fresnel_adjoint(self.handle, holo.data_ptr() if holo is not None else None,
                                [g.data_ptr() if g is not None else None for g in grad_views],
                                grad_holo.data_ptr() if grad_holo is not False else None,
                                grad_z.data_ptr() if grad_z is not None else None, stream=s)
        return grad_holo, grad_z

    def close(self):
        if getattr(self, "handle", None):
            shifted_fresnel_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
