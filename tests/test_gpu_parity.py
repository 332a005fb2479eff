"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerance: relative L2 error <= 1e-5 per view for the FP32 path, measured
against the oracle's complex field; intensities and phases are checked from
the same outputs.  Every case up to the paper-scale four-view workload
compares every pixel; the longest FFT lengths (4096, 8192) on thin
holograms compare sampled output columns along x, which the oracle computes
on their own, and every pixel along y.
"""

import numpy as np
import pytest

import oracle
import synth
from synth import view, random_field, WAVELENGTH, PITCH
from helpers import rel_l2, wrapped_phase_err

pytestmark = pytest.mark.gpu

TOL = 1e-5  # relative L2, FP32 path


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1001_4309_gb300 import build as b
    b.build()
    import paper_1001_4309_gb300 as P
    return P


def run(P, views, holo, field=True, intensity=True, phase=True):
    """Execute a plan on a device copy of the numpy hologram; returns numpy outputs."""
    import torch
    complex_in = bool(views[0].get("flags", 0) & P.SF_IN_COMPLEX)
    h = torch.from_numpy(np.ascontiguousarray(holo.astype(np.complex64 if complex_in else np.float32))).cuda()
    sf = P.ShiftedFresnel(views)
    try:
        outs = sf.reconstruct(h, field=field, intensity=intensity, phase=phase)
        torch.cuda.synchronize()
        res = {k: [None if t is None else t.cpu().numpy() for t in v] for k, v in outs.items()}
    finally:
        sf.close()
    return res


def check_view(res, i, ref, tol=TOL):
    f = res["field"][i]
    err = rel_l2(f, ref)
    assert err <= tol, f"view {i}: field rel-L2 {err:.3e} > {tol}"
    if res["intensity"][i] is not None:
        I = res["intensity"][i]
        ierr = rel_l2(I, np.abs(ref) ** 2)
        assert ierr <= 3 * tol, f"view {i}: intensity rel-L2 {ierr:.3e}"
        # the intensity is |u|^2 of the same float32 field
        assert np.allclose(I, np.abs(f.astype(np.complex128)) ** 2, rtol=1e-5, atol=1e-30 + 1e-6 * I.max())
    if res["phase"][i] is not None:
        ph = res["phase"][i]
        assert np.all(ph > -np.pi) and np.all(ph <= np.pi + 1e-6)
        weighted = rel_l2(np.abs(ref) * np.exp(1j * ph), ref)
        assert weighted <= 3 * tol, f"view {i}: phase-weighted error {weighted:.3e}"
        assert wrapped_phase_err(ph, ref, rel_floor=0.1) < 1e-3
    return err


def test_config_c1_single_view_full_parity(P):
    holo, views = synth.config_c1()
    res = run(P, views, holo)
    ref = oracle.forward(holo, views[0])
    check_view(res, 0, ref)


SMALL = [
    # (nx0, ny0, nx1, ny1, z, p0, p1, o0, o1, flags)
    (1, 1, 1, 1, 0.05, PITCH, PITCH, (0, 0), (0, 0), 0),
    (2, 3, 3, 2, -0.02, PITCH, 2e-6, (1e-5, 0), (-3e-5, 2e-5), 0),
    (17, 33, 33, 17, 0.03, (PITCH, 3.3e-6), (1.1e-6, 5e-6), (0, 4e-5), (2e-4, -1e-4), 0),
    (100, 64, 37, 100, -0.07, PITCH, 0.9e-6, (-2e-5, 1e-5), (5e-4, 3e-4), 8),
    (33, 17, 100, 3, 0.1, 2e-6, 9.3e-6, (0, 0), (-2e-3, 2e-3), 8 | 4),
    (64, 65, 65, 64, 0.04, PITCH, 2.325e-6, (0, 0), (1e-4, -5e-5), 4),
    (255, 129, 258, 127, 0.05, PITCH, 1.0e-6, (3e-5, -3e-5), (-4e-4, 6e-4), 0),
    # exactly L / 2 in and out on both axes (L = 64 and 512): the pruned network at its limit
    (32, 256, 32, 256, 0.045, PITCH, 3.3e-6, (1e-5, 2e-5), (1e-4, -1e-4), 8),
]


@pytest.mark.parametrize("case", SMALL, ids=lambda c: f"{c[0]}x{c[1]}-{c[2]}x{c[3]}-f{c[9]}")
def test_small_and_ragged_sizes(P, case):
    nx0, ny0, nx1, ny1, z, p0, p1, o0, o1, flags = case
    v = view(WAVELENGTH, z, p0, p1, o0, o1, (nx0, ny0), (nx1, ny1), flags=flags)
    holo = random_field(ny0, nx0, seed=nx0 * 7 + ny1, complex_=bool(flags & 8))
    if not flags & 8:
        holo = holo.real
    res = run(P, [v], holo)
    check_view(res, 0, oracle.forward(holo, v))


def test_multi_view_plan_with_mixed_fft_lengths(P):
    """One plan, views whose axes need different FFT lengths (several launches per pass)."""
    n0 = (96, 80)
    sizes = [(96, 80), (17, 200), (300, 5), (64, 64), (1, 1), (160, 33)]
    views = []
    rng = np.random.default_rng(5)
    for k, (nx1, ny1) in enumerate(sizes):
        views.append(view(WAVELENGTH, float(rng.uniform(0.02, 0.12)) * (-1) ** k, PITCH,
                          float(np.exp(rng.uniform(np.log(0.25e-6), np.log(9.3e-6)))),
                          o1=tuple(rng.uniform(-2e-4, 2e-4, size=2)), n0=n0, n1=(nx1, ny1)))
    holo = synth.gabor_hologram(96, seed=77)[:80, :96]
    res = run(P, views, holo)
    for i, v in enumerate(views):
        check_view(res, i, oracle.forward(holo, v))


def test_plan_query_reports_lengths(P):
    import paper_1001_4309_gb300 as PP
    v = view(WAVELENGTH, 0.05, PITCH, 2e-6, n0=(1024, 1024), n1=(1024, 1024))
    sf = PP.ShiftedFresnel([v])
    try:
        lx, ly, ws = sf.sizes(0)
    finally:
        sf.close()
    assert (lx, ly) == (2048, 2048)  # the paper's 2N padding (Section 2.2 step 2)
    assert ws == 8 * 1024 * 1024


def test_config_c2_paper_scale_full(P):
    """All four paper-scale 1024^2 views (FFT length 2048 on both axes, the
    launch shape the benchmark times): every output pixel of the field, the
    intensity and the phase against the FP64 oracle."""
    holo, views = synth.config_c2()
    res = run(P, views, holo)
    for i, v in enumerate(views):
        check_view(res, i, oracle.forward(holo, v))


@pytest.mark.parametrize("n0,n1", [(2048, 2048), (4096, 4097), (2048, 256)])
def test_large_fft_lengths(P, n0, n1):
    """Longest supported convolutions (L = 4096 and 8192) on thin holograms, every pixel."""
    ny = 8
    v = view(WAVELENGTH, 0.06, PITCH, 1.3e-6, o1=(3e-4, -1e-5), n0=(n0, ny), n1=(n1, ny))
    holo = random_field(ny, n0, seed=n0 + n1).real
    res = run(P, [v], holo, phase=False)
    check_view(res, 0, oracle.forward(holo, v))
    # the transposed direction exercises the y pass at the same lengths
    vt = view(WAVELENGTH, 0.06, PITCH, 1.3e-6, o1=(3e-4, -1e-5), n0=(ny, n0), n1=(ny, n1))
    res = run(P, [vt], holo.T.copy(), phase=False)
    check_view(res, 0, oracle.forward(holo.T.copy(), vt))


def test_host_buffers_match_device_buffers(P):
    import torch
    holo, views = synth.config_c1()
    dev = run(P, views, holo)
    v = views[0]
    sf = P.ShiftedFresnel(views)
    try:
        for pinned in (False, True):
            h = torch.from_numpy(holo.copy())
            f = torch.empty((v["ny1"], v["nx1"]), dtype=torch.complex64)
            I = torch.empty((v["ny1"], v["nx1"]), dtype=torch.float32)
            if pinned:
                h, f, I = h.pin_memory(), f.pin_memory(), I.pin_memory()
            P.shifted_fresnel_execute(sf.handle, h.data_ptr(), [f.data_ptr()], [I.data_ptr()], None,
                                      stream=torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            assert np.array_equal(f.numpy(), dev["field"][0])
            assert np.array_equal(I.numpy(), dev["intensity"][0])
    finally:
        sf.close()


@pytest.mark.parametrize("single_stream", [False, True])
def test_host_pipeline_matches_device_buffers(P, single_stream, monkeypatch):
    """Host hologram >= 1 MiB and host outputs: the pipelined schedule (x passes
    on one stream, y passes on another, the first x pass split at the
    hologram's halves, one on the persistent 4096-point kernel, the first and
    last views' y passes in column halves with 2-D copies) and the
    single-stream schedule give the device-buffer results bit for bit, over
    repeated calls with different holograms and a mix of host (pinned and
    pageable) and device outputs."""
    import torch
    if single_stream:
        monkeypatch.setenv("SF_EXECUTE_SINGLE_STREAM", "1")
    ny0, nx0 = 512, 2000
    views = [view(WAVELENGTH, 0.05, PITCH, 2e-6, o1=(1e-4, -2e-4), n0=(nx0, ny0), n1=(2000, 64)),  # x: L 4096
             view(WAVELENGTH, 0.08, PITCH, 7e-6, o1=(-3e-4, 0.0), n0=(nx0, ny0), n1=(33, 17)),
             view(WAVELENGTH, -0.04, PITCH, PITCH, n0=(nx0, ny0), n1=(300, 500))]
    holos = [random_field(ny0, nx0, seed=40 + k).real.astype(np.float32) for k in range(2)]
    refs = [run(P, views, h, phase=False) for h in holos]
    sf = P.ShiftedFresnel(views)
    try:
        assert sf.sizes(0)[0] == 4096
        s = torch.cuda.current_stream().cuda_stream
        for k in (0, 1, 0):
            h = torch.from_numpy(holos[k].copy()).pin_memory()
            f = [torch.empty((v["ny1"], v["nx1"]), dtype=torch.complex64).pin_memory() for v in views]
            f[2] = f[2].cuda()  # one view's field stays on the device
            I = [torch.empty((v["ny1"], v["nx1"]), dtype=torch.float32) for v in views]  # pageable
            P.shifted_fresnel_execute(sf.handle, h.data_ptr(), [x.data_ptr() for x in f], [x.data_ptr() for x in I],
                                      None, stream=s)
            torch.cuda.synchronize()
            for i in range(len(views)):
                assert np.array_equal(f[i].cpu().numpy(), refs[k]["field"][i]), (k, i)
                assert np.array_equal(I[i].numpy(), refs[k]["intensity"][i]), (k, i)
    finally:
        sf.close()


@pytest.mark.parametrize("pinned", [True, False])
def test_host_pipeline_single_complex_view(P, pinned):
    """One view (first and last at once: both y-pass column halves) from a complex host
    hologram split in halves, pinned or pageable: equal to the device-buffer result."""
    import torch
    ny0, nx0 = 384, 400
    v = view(WAVELENGTH, 0.04, PITCH, 3e-6, o1=(2e-4, -1e-4), n0=(nx0, ny0), n1=(512, 300), flags=P.SF_IN_COMPLEX)
    holo = random_field(ny0, nx0, seed=77).astype(np.complex64)
    ref = run(P, [v], holo, phase=True)
    sf = P.ShiftedFresnel([v])
    try:
        h = torch.from_numpy(holo.copy())
        f = torch.empty((v["ny1"], v["nx1"]), dtype=torch.complex64)
        I = torch.empty((v["ny1"], v["nx1"]), dtype=torch.float32)
        ph = torch.empty((v["ny1"], v["nx1"]), dtype=torch.float32)
        if pinned:
            h, f, I, ph = h.pin_memory(), f.pin_memory(), I.pin_memory(), ph.pin_memory()
        for _ in range(2):
            P.shifted_fresnel_execute(sf.handle, h.data_ptr(), [f.data_ptr()], [I.data_ptr()], [ph.data_ptr()],
                                      stream=torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            assert np.array_equal(f.numpy(), ref["field"][0])
            assert np.array_equal(I.numpy(), ref["intensity"][0])
            assert np.array_equal(ph.numpy(), ref["phase"][0])
    finally:
        sf.close()


def test_repeat_execute_is_deterministic(P):
    import torch
    holo, views = synth.config_c1()
    sf = P.ShiftedFresnel(views)
    try:
        h = torch.from_numpy(holo).cuda()
        a = sf.reconstruct(h)["field"][0].clone()
        b = sf.reconstruct(h)["field"][0].clone()
        torch.cuda.synchronize()
        assert torch.equal(a, b)
    finally:
        sf.close()


def test_execute_rejects_views_without_outputs(P):
    import torch
    holo, views = synth.config_c1()
    sf = P.ShiftedFresnel(views)
    try:
        h = torch.from_numpy(holo).cuda()
        rc = P.shifted_fresnel_execute(sf.handle, h.data_ptr(), [None], None, None, check=False)
        assert rc == P.SF_ERR_INVALID_ARG
    finally:
        sf.close()


def test_kernel_launch_counter_counts_two_passes(P):
    import torch
    holo, views = synth.config_c1()
    sf = P.ShiftedFresnel(views)
    try:
        h = torch.from_numpy(holo).cuda()
        before = P.shifted_fresnel_kernel_launches()
        sf.reconstruct(h)
        assert P.shifted_fresnel_kernel_launches() - before == 2
    finally:
        sf.close()


def test_plain_cufft_comparison_path_matches_oracle(P):
    """The benchmark's comparison path (the paper's steps 2-10 with cuFFT) is itself correct."""
    import torch
    from paper_1001_4309_gb300 import build as b
    from paper_1001_4309_gb300.plain import PlainPath
    b.build_plain()
    holo, views = synth.config_c1()
    views = views + [view(WAVELENGTH, 0.07, (PITCH, 3.1e-6), (1.0e-6, 2.2e-6), o1=(-3e-4, 2e-4),
                          n0=(256, 256), n1=(200, 120))]
    pp = PlainPath(views)
    try:
        h = torch.from_numpy(holo).cuda()
        outs = [torch.empty((v["ny1"], v["nx1"]), dtype=torch.complex64, device="cuda") for v in views]
        pp.execute(h, outs)
        torch.cuda.synchronize()
        for o, v in zip(outs, views):
            assert rel_l2(o.cpu().numpy(), oracle.forward(holo, v)) <= TOL
    finally:
        pp.close()


@pytest.mark.parametrize("n0,n1", [(1024, 1024), (2048, 2048), (1500, 1200)])
def test_row_pass_kernels_agree(P, n0, n1, monkeypatch):
    """The one-tile-per-CTA row pass (default, half and twice the rows per CTA, where those exist) and
    the persistent (bulk-copy prefetch) row pass give identical views."""
    ny0, ny1 = 24, 20
    v = view(WAVELENGTH, 0.045, PITCH, 1.9e-6, o1=(1e-4, 2e-5), n0=(n0, ny0), n1=(n1, ny1))
    holo = random_field(ny0, n0, seed=n0 + 11).real
    res = {}
    for impl in ("grid", "tma", "half", "double"):
        monkeypatch.setenv("SF_PASS_IMPL", impl)
        res[impl] = run(P, [v], holo, intensity=False, phase=False)["field"][0]
    for impl in ("tma", "half", "double"):
        assert np.array_equal(res["grid"], res[impl]), impl
    check_view({"field": [res["tma"]], "intensity": [None], "phase": [None]}, 0, oracle.forward(holo, v))


def test_many_views_one_plan(P):
    """40 ragged views of one hologram: several launches per FFT length (16 passes each), both halves of
    the two-stream split, every length family; every pixel of every view against the oracle."""
    rng = np.random.default_rng(21)
    n0 = (300, 260)
    sizes = [(int(a), int(b)) for a, b in rng.integers(1, 1300, size=(40, 2))]
    views = [view(WAVELENGTH, float(rng.uniform(0.02, 0.12)) * (-1) ** k, PITCH,
                  float(np.exp(rng.uniform(np.log(0.25e-6), np.log(9.3e-6)))),
                  o1=tuple(rng.uniform(-1e-3, 1e-3, size=2)), n0=n0, n1=n1) for k, n1 in enumerate(sizes)]
    holo = random_field(n0[1], n0[0], seed=99).real
    res = run(P, views, holo, intensity=False, phase=False)
    for i, v in enumerate(views):
        check_view(res, i, oracle.forward(holo, v))
