"""FFT lengths with a factor 3 (radix-24 first stage) and the plan-time autotuner.

Every supported length computes the same zero-padded circular convolution
(Section 2.2, steps 2-9), so a view must match the FP64 oracle within the
FP32 tolerance whichever length the plan picks: the smallest one
(1536 / 2304 / 3072 / 4608 / 6144 here), a power of two
(SF_FFT_LENGTHS=pow2) or the autotuner's measured choice (SF_AUTOTUNE=1).
"""

import os

import numpy as np
import pytest

import oracle
import synth
from synth import view, random_field, WAVELENGTH, PITCH
from helpers import rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1001_4309_gb300 import build as b
    b.build()
    import paper_1001_4309_gb300 as P
    return P


def reconstruct(P, views, holo):
    import torch
    cplx = bool(views[0].get("flags", 0) & P.SF_IN_COMPLEX)
    h = torch.from_numpy(np.ascontiguousarray(holo.astype(np.complex64 if cplx else np.float32))).cuda()
    sf = P.ShiftedFresnel(views)
    try:
        lens = [sf.sizes(i)[:2] for i in range(len(views))]
        out = sf.reconstruct(h, field=True)["field"]
        torch.cuda.synchronize()
        return lens, [o.cpu().numpy() for o in out]
    finally:
        sf.close()


def cols_of(n, w=8):
    return [(0, w), (n // 2 - w // 2, n // 2 + w // 2), (n - w, n)]


MIXED = [(1024, 512, 1536), (2048, 256, 2304), (2048, 1024, 3072), (4096, 512, 4608), (4096, 2048, 6144)]


@pytest.mark.parametrize("n0,n1,L", MIXED, ids=lambda x: str(x))
def test_mixed_length_x_axis_sampled(P, n0, n1, L):
    ny = 8
    v = view(WAVELENGTH, 0.05, PITCH, 1.7e-6, o1=(2e-4, -3e-5), n0=(n0, ny), n1=(n1, ny))
    holo = random_field(ny, n0, seed=n0 + 3 * n1).real
    lens, out = reconstruct(P, [v], holo)
    assert lens[0] == (L, 64)
    for c in cols_of(n1):
        err = rel_l2(out[0][:, c[0]:c[1]], oracle.forward(holo, v, cols=c))
        assert err <= TOL, (c, err)


@pytest.mark.parametrize("n0,n1,L", MIXED, ids=lambda x: str(x))
def test_mixed_length_y_axis_full(P, n0, n1, L):
    """The transposed geometry puts the mixed length on the y pass (complex rows, view epilogue)."""
    nx = 8
    v = view(WAVELENGTH, -0.04, PITCH, 2.9e-6, o1=(-1e-5, 4e-4), n0=(nx, n0), n1=(nx, n1))
    holo = random_field(n0, nx, seed=n0 + 5 * n1).real
    lens, out = reconstruct(P, [v], holo)
    assert lens[0] == (64, L)
    assert rel_l2(out[0], oracle.forward(holo, v)) <= TOL


def test_mixed_lengths_complex_input_both_axes(P):
    """Complex hologram (SF_IN_COMPLEX): the complex x pass at 1536 and a 2304 y pass."""
    v = view(WAVELENGTH, 0.03, PITCH, 3.1e-6, o1=(1e-4, 1e-4), n0=(1024, 1500), n1=(400, 700),
             flags=8)  # SF_IN_COMPLEX
    holo = random_field(1500, 1024, seed=21, complex_=True)
    lens, out = reconstruct(P, [v], holo)
    assert lens[0] == (1536, 2304)
    for c in cols_of(400):
        assert rel_l2(out[0][:, c[0]:c[1]], oracle.forward(holo, v, cols=c)) <= TOL


def test_power_of_two_lengths_on_request(P, monkeypatch):
    """SF_FFT_LENGTHS=pow2: same views through 4096-point transforms, equal within rounding."""
    ny = 8
    v = view(WAVELENGTH, 0.07, PITCH, 1.1e-6, o1=(3e-4, 0.0), n0=(2048, ny), n1=(1024, ny))
    holo = random_field(ny, 2048, seed=5).real
    lens_m, out_m = reconstruct(P, [v], holo)
    monkeypatch.setenv("SF_FFT_LENGTHS", "pow2")
    lens_p, out_p = reconstruct(P, [v], holo)
    assert lens_m[0][0] == 3072 and lens_p[0][0] == 4096
    assert rel_l2(out_m[0], out_p[0]) <= 2 * TOL
    for c in cols_of(1024):
        assert rel_l2(out_p[0][:, c[0]:c[1]], oracle.forward(holo, v, cols=c)) <= TOL


def test_autotuner_choices_cache_and_parity(P, monkeypatch, tmp_path):
    """SF_AUTOTUNE=1 picks, per axis, a length that holds the convolution; measurements land in the cache file."""
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("SF_AUTOTUNE", "1")
    monkeypatch.setenv("SF_AUTOTUNE_CACHE", str(cache))
    n0 = (2048, 300)
    sizes = [(256, 300), (512, 64), (1024, 200), (2048, 40)]
    rng = np.random.default_rng(3)
    views = [view(WAVELENGTH, float(rng.uniform(0.02, 0.12)), PITCH,
                  float(np.exp(rng.uniform(np.log(0.25e-6), np.log(9.3e-6)))),
                  o1=tuple(rng.uniform(-2e-3, 2e-3, size=2)), n0=n0, n1=n1) for n1 in sizes]
    holo = random_field(n0[1], n0[0], seed=9).real
    lens, out = reconstruct(P, views, holo)
    lines = cache.read_text().split()
    assert len(lines) > 0 and len(lines) % 6 == 0  # device, L, kind, kernel, prunable, ns per row
    for (lx, ly), v in zip(lens, views):
        for L, need in ((lx, v["nx0"] + v["nx1"] - 1), (ly, v["ny0"] + v["ny1"] - 1)):
            assert L in (P.shifted_fresnel_fft_length(need, True), P.shifted_fresnel_fft_length(need, False))
    for i, v in enumerate(views):
        c = cols_of(v["nx1"], 4)[1]
        assert rel_l2(out[i][:, c[0]:c[1]], oracle.forward(holo, v, cols=c)) <= TOL
    # a second plan with the same lengths reads the measurements back instead of timing again
    n_before = len(lines)
    reconstruct(P, views, holo)
    assert len(cache.read_text().split()) == n_before


def test_batch_with_mixed_lengths_matches_execute(P):
    """The persistent batch kernel runs mixed-length tiles (with spare threads) like execute does."""
    import torch
    n0 = (1024, 1200)
    sizes = [(512, 337), (1024, 1105), (2048, 20), (50, 2000)]
    rng = np.random.default_rng(8)
    views = [view(WAVELENGTH, float(rng.uniform(0.02, 0.12)), PITCH,
                  float(np.exp(rng.uniform(np.log(0.5e-6), np.log(6e-6)))),
                  o1=tuple(rng.uniform(-1e-3, 1e-3, size=2)), n0=n0, n1=n1) for n1 in sizes]
    holos_np = [random_field(n0[1], n0[0], seed=40 + h).real.astype(np.float32) for h in range(3)]
    holos = [torch.from_numpy(h).cuda() for h in holos_np]
    sf = P.ShiftedFresnel(views)
    try:
        lens = [sf.sizes(i)[:2] for i in range(len(views))]
        assert lens == [(1536, 1536), (2048, 2304), (3072, 1536), (1536, 4096)]
        ref = []
        for h in holos:
            ref.append([f.clone() for f in sf.reconstruct(h, field=True)["field"]])
        outs = sf.alloc_batch_outputs(len(holos), field=True)
        sf.execute_batch(holos, outs)
        torch.cuda.synchronize()
        assert P.shifted_fresnel_batch_status(sf.handle) == P.SF_OK
        for h in range(len(holos)):
            for v in range(len(views)):
                a, b = outs["field"][h][v].cpu().numpy(), ref[h][v].cpu().numpy()
                assert rel_l2(a, b) <= 1e-6, (h, v)
        for v in range(len(views)):
            c = cols_of(views[v]["nx1"], 4)[1]
            got = outs["field"][1][v].cpu().numpy()[:, c[0]:c[1]]
            assert rel_l2(got, oracle.forward(holos_np[1].astype(np.float64), views[v], cols=c)) <= TOL
    finally:
        sf.close()
