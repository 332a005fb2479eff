"""Pins for the FP64 oracle against things other than itself (CPU only).

Each test fixes the oracle to something the paper or the mathematics gives:
brute-force quadruple sums, the paper's Eqs. 1-4 written out literally, the
ordinary Fresnel convolution, the single-FFT special case, the Gaussian-beam
and point-source closed forms, invariants and the paper's view-area figure.
"""

import json
import math
import os

import numpy as np
import pytest

import oracle
from synth import view, random_field, WAVELENGTH, PITCH

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


def coords(n, p, o):
    """Centred sample coordinates o + (m - floor(n/2)) p."""
    return o + (np.arange(n) - n // 2) * p


def prefactor(v):
    k = 2 * np.pi / v["wavelength"]
    return np.exp(1j * k * v["z"]) / (1j * v["wavelength"] * v["z"])


def brute_force(u0, v):
    """O(N^4) non-separable sum over every (input, output) pixel pair."""
    beta = 1.0 / (v["wavelength"] * v["z"])
    x0 = coords(v["nx0"], v["px0"], v["ox0"])[None, :]
    y0 = coords(v["ny0"], v["py0"], v["oy0"])[:, None]
    x1 = coords(v["nx1"], v["px1"], v["ox1"])
    y1 = coords(v["ny1"], v["py1"], v["oy1"])
    out = np.empty((v["ny1"], v["nx1"]), dtype=np.complex128)
    for j in range(v["ny1"]):
        for i in range(v["nx1"]):
            r2 = (x1[i] - x0) ** 2 + (y1[j] - y0) ** 2
            out[j, i] = np.sum(u0 * np.exp(1j * np.pi * beta * r2))
    return prefactor(v) * out


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


TINY_CASES = [
    # (nx0, ny0, nx1, ny1, z, p0, p1, o0, o1)
    (8, 8, 8, 8, 0.05, PITCH, 2.325e-6, (0, 0), (100e-6, -50e-6)),
    (7, 5, 9, 6, -0.03, (PITCH, 3.1e-6), (1.7e-6, 2.9e-6), (20e-6, -35e-6), (-60e-6, 75e-6)),
    (16, 12, 11, 13, 0.1, 5.0e-6, 0.5e-6, (-10e-6, 0), (1e-3, -0.8e-3)),
    (1, 3, 4, 1, 0.02, PITCH, PITCH, (0, 0), (0, 0)),
    (32, 2, 17, 3, -0.07, (2.0e-6, 6.0e-6), (9.3e-6, 0.25e-6), (0, 5e-6), (2e-3, -2e-3)),
]


@pytest.mark.parametrize("case", TINY_CASES)
def test_p1_brute_force(case):
    nx0, ny0, nx1, ny1, z, p0, p1, o0, o1 = case
    v = view(WAVELENGTH, z, p0, p1, o0, o1, (nx0, ny0), (nx1, ny1))
    u0 = random_field(ny0, nx0, seed=11 + nx0)
    ref = brute_force(u0, v)
    got = oracle.forward(u0, v)
    assert rel_l2(got, ref) < 1e-12


def test_p1_column_range_matches_full():
    v = view(WAVELENGTH, 0.05, PITCH, 2.0e-6, (0, 0), (3e-4, 1e-4), (24, 20), (19, 22))
    u0 = random_field(20, 24, seed=3)
    full = oracle.forward(u0, v)
    part = oracle.forward(u0, v, cols=(5, 13))
    assert np.array_equal(part, full[:, 5:13])


def paper_equations_1_to_4(u0, v):
    """Eqs. 1-4 written out as printed, with the index origin at -N/2.

    Offsets O are in pixels of their own plane (O = o / p) and
    x0 = (m0 - N0/2 + O_x0) p_x0, x1 = (m1 - N1/2 + O_x1) p_x1; the
    convolution of Eq. 1 is a direct linear sum (no FFT).
    """
    lam, z = v["wavelength"], v["z"]
    out_axes = []
    for ax in ("x", "y"):
        n0, n1 = v[f"n{ax}0"], v[f"n{ax}1"]
        p0, p1 = v[f"p{ax}0"], v[f"p{ax}1"]
        O0, O1 = v[f"o{ax}0"] / p0, v[f"o{ax}1"] / p1
        S = p0 * p1 / (lam * z)
        m0, m1 = np.arange(n0), np.arange(n1)
        x0 = (m0 - n0 // 2 + O0) * p0
        x1 = (m1 - n1 // 2 + O1) * p1
        # Eq. 3, one axis: exp(i pi x0^2/(lz)) exp(-i 2 pi m0 S(-N/2 + O1)) exp(-i pi S m0^2)
        chirp_in = (np.exp(1j * np.pi * x0 ** 2 / (lam * z))
                    * np.exp(-1j * 2 * np.pi * m0 * S * (-(n1 // 2) + O1))
                    * np.exp(-1j * np.pi * S * m0 ** 2))
        # Eq. 2 without exp(ikz)/(i l z): exp(i pi x1^2/(lz)) exp(-i 2pi/(lz) (-N/2+O0) p0 x1) exp(-i pi S m1^2)
        chirp_out = (np.exp(1j * np.pi * x1 ** 2 / (lam * z))
                     * np.exp(-1j * 2 * np.pi / (lam * z) * (-(n0 // 2) + O0) * p0 * x1)
                     * np.exp(-1j * np.pi * S * m1 ** 2))
        # Eq. 4: h[m1 - m0] = exp(i pi S (m1 - m0)^2)
        h = np.exp(1j * np.pi * S * (m1[:, None] - m0[None, :]) ** 2)
        out_axes.append(chirp_out[:, None] * h * chirp_in[None, :])  # [n1, n0]
    Kx, Ky = out_axes
    C = np.exp(1j * 2 * np.pi * z / lam) / (1j * lam * z)
    return C * (Ky @ u0 @ Kx.T)


@pytest.mark.parametrize("case", TINY_CASES[:3] + [
    (48, 40, 48, 40, -0.05, PITCH, 2.325e-6, (0, 0), (100e-6, -50e-6)),
])
def test_paper_equations_1_to_4(case):
    nx0, ny0, nx1, ny1, z, p0, p1, o0, o1 = case
    v = view(WAVELENGTH, z, p0, p1, o0, o1, (nx0, ny0), (nx1, ny1))
    u0 = random_field(ny0, nx0, seed=5)
    assert rel_l2(oracle.forward(u0, v), paper_equations_1_to_4(u0, v)) < 1e-11


def test_p2_equal_pitch_is_fresnel_convolution():
    """p1 = p0, zero offsets: the sum is a linear convolution with the Fresnel response."""
    from scipy.signal import fftconvolve
    n = 40
    for z in (0.05, -0.02):
        v = view(WAVELENGTH, z, PITCH, PITCH, n0=(n, n), n1=(n, n))
        u0 = random_field(n, n, seed=21)
        d = np.arange(-(n - 1), n) * PITCH
        g = np.exp(1j * np.pi * (d[:, None] ** 2 + d[None, :] ** 2) / (WAVELENGTH * z))
        full = fftconvolve(u0, g)  # index (n1 + n - 1) <-> displacement n1 - n0
        ref = prefactor(v) * full[n - 1:2 * n - 1, n - 1:2 * n - 1]
        assert rel_l2(oracle.forward(u0, v), ref) < 1e-11


def test_p3_single_fft_special_case():
    """p1 = lambda z / (N0 p0) makes the cross term an exact length-N0 DFT."""
    nx, ny = 30, 24
    z = 0.04
    p0x, p0y = PITCH, 3.0e-6
    p1x, p1y = WAVELENGTH * z / (nx * p0x), WAVELENGTH * z / (ny * p0y)
    o0, o1 = (15e-6, -7e-6), (2e-4, -1.5e-4)
    v = view(WAVELENGTH, z, (p0x, p0y), (p1x, p1y), o0, o1, (nx, ny), (nx, ny))
    u0 = random_field(ny, nx, seed=8)
    beta = 1 / (WAVELENGTH * z)
    pre, post = [], []
    for n, p0, p1, oo0, oo1 in ((nx, p0x, p1x, o0[0], o1[0]), (ny, p0y, p1y, o0[1], o1[1])):
        a0 = oo0 - (n // 2) * p0
        a1 = oo1 - (n // 2) * p1
        m = np.arange(n)
        x0, x1 = a0 + m * p0, a1 + m * p1
        pre.append(np.exp(1j * np.pi * beta * (x0 ** 2 - 2 * a1 * p0 * m)))
        post.append(np.exp(1j * np.pi * beta * (x1 ** 2 - 2 * a0 * a1 - 2 * a0 * p1 * m)))
    F = np.fft.fft2(u0 * pre[1][:, None] * pre[0][None, :])
    ref = prefactor(v) * F * post[1][:, None] * post[0][None, :]
    assert rel_l2(oracle.forward(u0, v), ref) < 1e-11


def gaussian_axis(x1, w, beta, p0):
    """(1/p0) * integral exp(-x^2/w^2) exp(i pi beta (x1 - x)^2) dx in closed form."""
    a = 1.0 / w ** 2 - 1j * np.pi * beta
    return (np.sqrt(np.pi / a) * np.exp(-(np.pi * beta * x1) ** 2 / a)
            * np.exp(1j * np.pi * beta * x1 ** 2)) / p0


@pytest.mark.parametrize("z", [0.05, -0.05])
def test_p4_gaussian_beam_closed_form(z):
    n, w = 256, 100e-6
    v = view(WAVELENGTH, z, PITCH, 2.325e-6, (10e-6, -20e-6), (100e-6, -50e-6), (n, n), (n, n))
    x0 = coords(n, PITCH, 10e-6)
    y0 = coords(n, PITCH, -20e-6)
    u0 = np.exp(-(x0[None, :] ** 2 + y0[:, None] ** 2) / w ** 2)
    beta = 1 / (WAVELENGTH * z)
    gx = gaussian_axis(coords(n, 2.325e-6, 100e-6), w, beta, PITCH)
    gy = gaussian_axis(coords(n, 2.325e-6, -50e-6), w, beta, PITCH)
    ref = prefactor(v) * gy[:, None] * gx[None, :]
    assert rel_l2(oracle.forward(u0, v), ref) < 1e-12


def point_source_axis(x1, a0, p0, n0, xs, beta):
    """sum_m exp(i pi beta ((x1 - x0)^2 - (x0 - xs)^2)), x0 = a0 + m p0, as a geometric series."""
    d = x1 - xs
    q = np.exp(-2j * np.pi * beta * p0 * d)
    with np.errstate(invalid="ignore", divide="ignore"):
        geo = np.where(np.abs(1 - q) < 1e-300, n0, (1 - q ** n0) / (1 - q))
    return np.exp(1j * np.pi * beta * (x1 ** 2 - xs ** 2)) * np.exp(-2j * np.pi * beta * a0 * d) * geo


def test_p5_point_source_lands_at_shifted_scaled_position():
    nx0, ny0, nx1, ny1 = 64, 48, 40, 36
    p0, p1 = PITCH, 1.0e-6
    o0, o1 = (0.0, 0.0), (150e-6, -80e-6)
    z = 0.03
    v = view(WAVELENGTH, z, p0, p1, o0, o1, (nx0, ny0), (nx1, ny1))
    beta = 1 / (WAVELENGTH * z)
    # the source sits on view pixel (mx, my) = (27, 9)
    mx, my = 27, 9
    xs = o1[0] + (mx - nx1 // 2) * p1
    ys = o1[1] + (my - ny1 // 2) * p1
    x0, y0 = coords(nx0, p0, o0[0]), coords(ny0, p0, o0[1])
    u0 = np.exp(-1j * np.pi * beta * ((x0[None, :] - xs) ** 2 + (y0[:, None] - ys) ** 2))
    got = oracle.forward(u0, v)
    fx = point_source_axis(coords(nx1, p1, o1[0]), o0[0] - (nx0 // 2) * p0, p0, nx0, xs, beta)
    fy = point_source_axis(coords(ny1, p1, o1[1]), o0[1] - (ny0 // 2) * p0, p0, ny0, ys, beta)
    ref = prefactor(v) * fy[:, None] * fx[None, :]
    assert rel_l2(got, ref) < 1e-11
    peak = np.unravel_index(np.argmax(np.abs(got)), got.shape)
    assert peak == (my, mx)
    assert abs(abs(got[my, mx]) - abs(prefactor(v)) * nx0 * ny0) < 1e-9 * abs(prefactor(v)) * nx0 * ny0


def test_p6_linearity_and_rank_one():
    v = view(WAVELENGTH, -0.06, (PITCH, 3.5e-6), (1.5e-6, 2.5e-6), (5e-6, -5e-6), (-2e-4, 3e-4), (20, 14), (18, 16))
    u = random_field(14, 20, seed=1)
    w = random_field(14, 20, seed=2)
    a, b = 0.7 - 0.2j, -1.3 + 0.5j
    lhs = oracle.forward(a * u + b * w, v)
    rhs = a * oracle.forward(u, v) + b * oracle.forward(w, v)
    assert rel_l2(lhs, rhs) < 1e-13
    # rank one in, rank one out (separability of the kernel)
    col = random_field(14, 1, seed=3)[:, 0]
    row = random_field(1, 20, seed=4)[0]
    out = oracle.forward(np.outer(col, row), v)
    s = np.linalg.svd(out, compute_uv=False)
    assert s[1] / s[0] < 1e-12


def test_p6_adjoint_dot_product_and_brute_force():
    v = view(WAVELENGTH, 0.04, (PITCH, 3.0e-6), (2.0e-6, 1.2e-6), (0, 1e-5), (1e-4, -2e-4), (13, 9), (11, 10))
    u = random_field(9, 13, seed=31)
    g = random_field(10, 11, seed=32)
    lhs = np.vdot(g, oracle.forward(u, v))  # <A u, g>
    rhs = np.vdot(oracle.adjoint(g, v), u)  # <u, A^H g>
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    # brute-force conjugate transpose of the explicit matrix
    n_in = 9 * 13
    A = np.empty((10 * 11, n_in), dtype=np.complex128)
    for k in range(n_in):
        e = np.zeros(n_in, dtype=np.complex128)
        e[k] = 1
        A[:, k] = brute_force(e.reshape(9, 13), v).ravel()
    ref = (A.conj().T @ g.ravel()).reshape(9, 13)
    assert rel_l2(oracle.adjoint(g, v), ref) < 1e-12


@pytest.mark.parametrize("flags", [0, 4])
def test_forward_dz_matches_central_differences(flags):
    v = view(WAVELENGTH, 0.05, PITCH, 1.5e-6, (0, 0), (1e-4, 2e-4), (12, 10), (9, 11), flags=flags)
    u = random_field(10, 12, seed=41)
    h = 1e-9 * v["z"]  # k h stays ~5e-4 rad so the exp(ikz) factor is resolved
    vp, vm = dict(v, z=v["z"] + h), dict(v, z=v["z"] - h)
    fd = (oracle.forward(u, vp) - oracle.forward(u, vm)) / (2 * h)
    assert rel_l2(oracle.forward_dz(u, v), fd) < 1e-6


def test_no_prefactor_flag_drops_only_the_constant():
    v = view(WAVELENGTH, 0.05, PITCH, 2e-6, (0, 0), (1e-4, 0), (10, 8), (9, 7))
    u = random_field(8, 10, seed=9)
    full = oracle.forward(u, v)
    bare = oracle.forward(u, dict(v, flags=4))
    assert rel_l2(full, prefactor(v) * bare) < 1e-14


def test_intensity_and_phase():
    u = np.array([[1 + 1j, -1 + 0j, 0j, -1 - 1e-300j]])
    assert np.allclose(oracle.intensity(u), [[2, 1, 0, 1]])
    ph = oracle.phase(u)
    assert np.allclose(ph[0, :3], [np.pi / 4, np.pi, 0.0])
    assert -np.pi < ph[0, 3] <= np.pi


def test_p7_paper_view_area():
    """Section 3: a view at p1 = 4.65 um on a 1024 grid covers about 4.8 mm.

    Point sources at the first and last view pixels land on those pixels, so
    the reconstructed field spans N p1 of the object plane.
    """
    with open(GOLDEN) as f:
        g = json.load(f)
    n = g["grid"]["value"]
    p = g["ccd_pitch_m"]["value"]
    lam = g["wavelength_m"]["value"]
    area = g["wide_view_area_m"]
    assert abs(n * p - area["value"]) / area["value"] < area["rel_tol"]
    z = 0.05
    v = view(lam, z, p, p, n0=(n, 1), n1=(n, 1))
    beta = 1 / (lam * z)
    x0 = coords(n, p, 0.0)
    x1 = coords(n, p, 0.0)
    for m in (0, n - 1):
        u0 = np.exp(-1j * np.pi * beta * (x0 - x1[m]) ** 2)[None, :]
        out = oracle.forward(u0, v)
        assert int(np.argmax(np.abs(out[0]))) == m
    assert abs((x1[-1] - x1[0] + p) - n * p) < 1e-12


def test_paper_padding_is_enough_for_linear_convolution():
    """Section 2.2 step 2 / Section 3: 2N >= N0 + N1 - 1 for the 1024 -> 1024 views."""
    with open(GOLDEN) as f:
        g = json.load(f)
    n, L = g["grid"]["value"], g["padded_grid"]["value"]
    assert L >= 2 * n - 1
