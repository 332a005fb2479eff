"""Seeded in-line (Gabor) holograms and view sets shaped like the paper's workloads.

Physical constants follow the paper's set-up (Section 2): a He-Ne reference
at 632.8 nm and a CCD with a 4.65 um pixel pitch, holograms resized to
1024 x 1024 grids.  The paper's real holograms (USAF target, mosquito head,
fly) are not available, so seeded synthetic objects stand in for them:

* ``bars_disks_object``: random opaque bars and disks (transmittance 0/1) on
  a unit background.
* ``target_blobs_object``: a resolution-target-like set of bar triplets of
  halving width plus smooth random-phase Gaussian blobs.

Recording: the object transmittance ``t`` is lit by a unit plane wave and
propagated over ``z_rec`` with the band-limited angular-spectrum method in
float64 (``asm_propagate``), the intensity ``|U|^2`` is optionally given
Poisson photon noise and then quantised to 8 bits and stored as float32.
The angular-spectrum transfer function is a different diffraction model from
the Fresnel/Shifted-Fresnel sums under test, so the recording shares no
arithmetic with either side of a parity check.

Seeds: ``seed = config_index * 1000 + hologram_index``.
"""

from __future__ import annotations

import math

import numpy as np

WAVELENGTH = 632.8e-9  # He-Ne reference light, metres (Section 2)
PITCH = 4.65e-6  # CCD pixel pitch, metres (Section 2)


def view(wavelength, z, p0, p1, o0=(0.0, 0.0), o1=(0.0, 0.0), n0=(1024, 1024),
         n1=(1024, 1024), flags=0):
    """One view's parameters as a plain dict (lengths in metres, sizes as (nx, ny)).

    ``p0``/``p1`` are the hologram and view pitches (scalar or (px, py));
    ``o0``/``o1`` are the physical offsets of the two planes.
    """
    px0, py0 = (p0, p0) if np.isscalar(p0) else p0
    px1, py1 = (p1, p1) if np.isscalar(p1) else p1
    return dict(wavelength=float(wavelength), z=float(z),
                px0=float(px0), py0=float(py0), px1=float(px1), py1=float(py1),
                ox0=float(o0[0]), oy0=float(o0[1]), ox1=float(o1[0]), oy1=float(o1[1]),
                nx0=int(n0[0]), ny0=int(n0[1]), nx1=int(n1[0]), ny1=int(n1[1]),
                flags=int(flags))


def asm_propagate(field, pitch, wavelength, z, pad=2):
    """Band-limited angular-spectrum propagation of a complex field (float64).

    The field is zero-padded ``pad`` times per axis to avoid wrap-around, the
    transfer function exp(i 2 pi z sqrt(1/lambda^2 - fx^2 - fy^2)) is applied
    with its global phase exp(i k z) removed, and frequencies beyond the
    band limit 1/(lambda sqrt((2 df z)^2 + 1)) (df = 1/(pad n pitch)) or in
    the evanescent region are dropped.
    """
    ny, nx = field.shape
    Py, Px = pad * ny, pad * nx
    buf = np.zeros((Py, Px), dtype=np.complex128)
    y0, x0 = (Py - ny) // 2, (Px - nx) // 2
    buf[y0:y0 + ny, x0:x0 + nx] = field
    fy = np.fft.fftfreq(Py, d=pitch)[:, None]
    fx = np.fft.fftfreq(Px, d=pitch)[None, :]
    arg = 1.0 / wavelength ** 2 - fx ** 2 - fy ** 2
    prop = arg > 0
    kz = np.sqrt(np.where(prop, arg, 0.0))
    H = np.exp(1j * 2 * np.pi * z * (kz - 1.0 / wavelength))
    lim_x = 1.0 / (wavelength * math.sqrt((2.0 * z / (Px * pitch)) ** 2 + 1.0))
    lim_y = 1.0 / (wavelength * math.sqrt((2.0 * z / (Py * pitch)) ** 2 + 1.0))
    H = np.where(prop & (np.abs(fx) <= lim_x) & (np.abs(fy) <= lim_y), H, 0.0)
    out = np.fft.ifft2(np.fft.fft2(buf) * H)
    return out[y0:y0 + ny, x0:x0 + nx]


def bars_disks_object(n, rng, n_bars=10, n_disks=8):
    """Opaque (t = 0) random bars and disks on a unit background, float64 [n, n]."""
    t = np.ones((n, n), dtype=np.complex128)
    yy, xx = np.mgrid[0:n, 0:n]
    lo, hi = int(0.2 * n), int(0.8 * n)
    for _ in range(n_bars):
        cx, cy = rng.integers(lo, hi, size=2)
        length = max(2, int(rng.uniform(0.05, 0.25) * n))
        width = max(1, int(rng.uniform(0.006, 0.03) * n))
        if rng.random() < 0.5:
            t[max(cy - width // 2, 0):cy + (width + 1) // 2, max(cx - length // 2, 0):cx + length // 2] = 0
        else:
            t[max(cy - length // 2, 0):cy + length // 2, max(cx - width // 2, 0):cx + (width + 1) // 2] = 0
    for _ in range(n_disks):
        cx, cy = rng.integers(lo, hi, size=2)
        r = rng.uniform(0.008, 0.05) * n
        t[(xx - cx) ** 2 + (yy - cy) ** 2 <= r * r] = 0
    return t


def target_blobs_object(n, rng, n_blobs=6):
    """Bar triplets of halving width (resolution-target-like) plus random-phase blobs.

    Each element is three horizontal and three vertical opaque bars of width
    w and length 5w separated by w; widths run 32, 16, ..., 1 pixels scaled by
    n/1024.  Smooth Gaussian phase blobs (peak phase within +-pi/2, radius
    2-8 % of n) multiply the transmittance by exp(i phi).
    """
    t = np.ones((n, n), dtype=np.complex128)
    scale = n / 1024.0
    widths = [max(1, int(round(w * scale))) for w in (32, 16, 8, 4, 2, 1)]
    cx, cy = int(0.25 * n), int(0.3 * n)
    for w in widths:
        L = 5 * w
        for k in range(3):  # horizontal triplet
            y = cy + 2 * k * w
            t[y:y + w, cx:cx + L] = 0
        x0 = cx + L + 2 * w
        for k in range(3):  # vertical triplet
            x = x0 + 2 * k * w
            t[cy:cy + L, x:x + w] = 0
        cx = x0 + 6 * w + 2 * max(w, 2)
        if cx + 12 * w > 0.8 * n:
            cx, cy = int(0.25 * n), cy + 7 * w + 4
    yy, xx = np.mgrid[0:n, 0:n].astype(np.float64)
    phi = np.zeros((n, n))
    for _ in range(n_blobs):
        bx, by = rng.uniform(0.2 * n, 0.8 * n, size=2)
        r = rng.uniform(0.02, 0.08) * n
        amp = rng.uniform(-0.5 * np.pi, 0.5 * np.pi)
        phi += amp * np.exp(-((xx - bx) ** 2 + (yy - by) ** 2) / (r * r))
    return t * np.exp(1j * phi)


def gabor_hologram(n, seed, kind="bars_disks", z_rec=0.05, pitch=PITCH,
                   wavelength=WAVELENGTH, photons=None):
    """8-bit in-line hologram I = |1 + O|^2 as float32 [n, n] (values 0..255).

    ``kind`` selects the object ("bars_disks" or "target_blobs"); ``photons``
    adds Poisson noise at that mean photon count per pixel before
    quantisation q = clip(round(127.5 I), 0, 255).
    """
    rng = np.random.default_rng(seed)
    if kind == "bars_disks":
        t = bars_disks_object(n, rng)
    elif kind == "target_blobs":
        t = target_blobs_object(n, rng)
    else:
        raise ValueError(f"unknown object kind {kind!r}")
    U = 1.0 + asm_propagate(t - 1.0, pitch, wavelength, z_rec)
    I = np.abs(U) ** 2
    if photons is not None:
        I = rng.poisson(photons * I) / float(photons)
    q = np.clip(np.round(127.5 * I), 0, 255)
    return q.astype(np.float32)


def random_field(ny, nx, seed, complex_=True, dtype=None):
    """Standard-normal test field (complex128 by default), seeded."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((ny, nx))
    if complex_:
        a = a + 1j * rng.standard_normal((ny, nx))
    return a if dtype is None else a.astype(dtype)


# --------------------------------------------------------------------------
# Workload configurations (hologram recipe + view sets)
# --------------------------------------------------------------------------

def config_c1():
    """Single view: 256^2 hologram -> one 256^2 view at z=-5 cm, 2.325 um, offset (+100, -50) um."""
    holo = gabor_hologram(256, seed=0 * 1000 + 0, kind="bars_disks")
    v = view(WAVELENGTH, -0.05, PITCH, 2.325e-6, o1=(100e-6, -50e-6), n0=(256, 256), n1=(256, 256))
    return holo, [v]


def config_c2(with_hologram=True):
    """Paper scale: 1024^2 hologram -> four 1024^2 views (z = 3, 5, 7, 10 cm; p1 = 4.65, 2, 1, 0.5 um).

    Offsets are uniform within +-1 mm, seeded; the hologram carries Poisson
    noise at a 2000-photon mean.
    """
    seed = 1 * 1000 + 0
    holo = (gabor_hologram(1024, seed=seed, kind="target_blobs", photons=2000)
            if with_hologram else None)
    rng = np.random.default_rng(seed + 500)
    views = []
    for z, p1 in zip((0.03, 0.05, 0.07, 0.10), (4.65e-6, 2.0e-6, 1.0e-6, 0.5e-6)):
        o1 = tuple(rng.uniform(-1e-3, 1e-3, size=2))
        views.append(view(WAVELENGTH, z, PITCH, p1, o1=o1, n0=(1024, 1024), n1=(1024, 1024)))
    return holo, views


def config_c3(n_holos=16, n_views=64, with_holograms=True, n=2048):
    """Ragged batch: 2048^2 holograms, 64 views each with N1 in {256, 512, 1024, 2048}.

    z ~ U[2, 12] cm, log p1 ~ U[ln 0.25, ln 9.3] um, offsets ~ U[-2, 2] mm.
    Returns (list of holograms or None, list of per-hologram view lists).
    """
    holos, all_views = [], []
    for h in range(n_holos):
        seed = 2 * 1000 + h
        holos.append(gabor_hologram(n, seed=seed, kind="target_blobs", photons=2000)
                     if with_holograms else None)
        rng = np.random.default_rng(seed + 500)
        vs = []
        for _ in range(n_views):
            n1 = int(rng.choice([256, 512, 1024, 2048]))
            z = rng.uniform(0.02, 0.12)
            p1 = math.exp(rng.uniform(math.log(0.25e-6), math.log(9.3e-6)))
            o1 = tuple(rng.uniform(-2e-3, 2e-3, size=2))
            vs.append(view(WAVELENGTH, z, PITCH, p1, o1=o1, n0=(n, n), n1=(n1, n1)))
        all_views.append(vs)
    return holos, all_views


def config_c4():
    """Mixed precision set: the c1 view plus single 1024^2 and 2048^2 views."""
    out = [config_c1()]
    for n, s in ((1024, 3 * 1000 + 1), (2048, 3 * 1000 + 2)):
        holo = gabor_hologram(n, seed=s, kind="bars_disks")
        v = view(WAVELENGTH, -0.05, PITCH, 2.325e-6, o1=(100e-6, -50e-6), n0=(n, n), n1=(n, n))
        out.append((holo, [v]))
    return out


def config_c5(n=1024):
    """Adjoint workload: a complex n^2 object, four depths (3, 5, 7, 10 cm), output pitch 1 um.

    Returns (object field complex128, views); the measured intensities are
    made by the caller from a known random object.
    """
    seed = 4 * 1000 + 0
    rng = np.random.default_rng(seed)
    t = bars_disks_object(n, rng) * np.exp(1j * 0.5 * rng.standard_normal() )
    views = [view(WAVELENGTH, z, PITCH, 1.0e-6, n0=(n, n), n1=(n, n)) for z in (0.03, 0.05, 0.07, 0.10)]
    return t, views


def retrieval_object(n, seed):
    """Mixed amplitude and phase object for multi-depth retrieval, complex128 [n, n].

    Amplitude 1 on the background and 0.3 inside random bars and disks
    (``bars_disks_object``); phase from the smooth random-phase blobs of
    ``target_blobs_object`` (peak phase within +-pi/2).
    """
    rng = np.random.default_rng(seed)
    t = bars_disks_object(n, rng)
    phase = np.angle(target_blobs_object(n, rng))
    return np.where(np.abs(t) > 0, 1.0, 0.3) * np.exp(1j * phase)


def poisson_intensity(I, photons, seed):
    """Photon noise at a mean count of ``photons`` per pixel: Poisson(photons I / mean I) mean I / photons."""
    rng = np.random.default_rng(seed)
    s = float(np.mean(I))
    return rng.poisson(photons * I / s) * (s / photons)


def config_c5_inline(n=1024):
    """Multi-depth in-line (Gabor) retrieval set: the object of ``retrieval_object``
    and four views at z = 3, 5, 7, 10 cm with the hologram's own pitch and no
    offset (the in-line recording geometry; every view covers the whole object).

    Returns (object complex128, views).  Callers add the measured intensities
    (with ``poisson_intensity`` at 2000 photons) from a model of their choice.
    """
    obj = retrieval_object(n, seed=4 * 1000 + 1)
    views = [view(WAVELENGTH, z, PITCH, PITCH, n0=(n, n), n1=(n, n)) for z in (0.03, 0.05, 0.07, 0.10)]
    return obj, views
