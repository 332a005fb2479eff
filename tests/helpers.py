"""Shared helpers for the parity tests (no method arithmetic here)."""

import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def max_abs(a, b):
    return float(np.max(np.abs(np.asarray(a, dtype=np.complex128) - np.asarray(b, dtype=np.complex128))))


def wrapped_phase_err(ph, ref_field, rel_floor=1e-3):
    """Max |wrap(ph - angle(ref))| over pixels where |ref| > rel_floor * max|ref|."""
    mag = np.abs(ref_field)
    mask = mag > rel_floor * mag.max()
    d = np.angle(np.exp(1j * (ph[mask] - np.angle(ref_field[mask]))))
    return float(np.max(np.abs(d))) if d.size else 0.0


def header_functions(path):
    """Names of the extern "C" functions declared in a header."""
    import re
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(shifted_fresnel_\w+)\s*\(", src, flags=re.M)))


def aligned_rel_l2(u, ref):
    """Relative L2 error of u against ref after the best global complex scale
    (least squares: alpha = <u, ref> / <u, u>), i.e. up to global phase and amplitude."""
    u = np.asarray(u, dtype=np.complex128).ravel()
    ref = np.asarray(ref, dtype=np.complex128).ravel()
    alpha = np.vdot(u, ref) / np.vdot(u, u)
    return float(np.linalg.norm(alpha * u - ref) / np.linalg.norm(ref))
