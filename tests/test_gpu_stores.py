"""Output paths that must not change a single bit of the result.

* Row-pass output tiles leave either through 2D tensor stores (TMA: complex
  outputs in plain device memory, 16-byte aligned rows) or through the plain
  store loop (intensity / phase outputs, accumulation, unaligned rows).  Both
  write the values the tile computed, so the complex field of a view is
  bit-identical whichever way it left.
* FP16 / BF16 plans whose axes all run the tcgen05 pass execute both passes
  in one fused launch; with SF_EXECUTE_SINGLE_STREAM=1 (or profiling events)
  they run one launch per pass.  The tile arithmetic is the same, so the
  results are bit-identical.
"""

import os

import numpy as np
import pytest

import oracle
import synth
from synth import view, random_field, WAVELENGTH, PITCH
from helpers import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1001_4309_gb300 import build as b
    b.build()
    import paper_1001_4309_gb300 as P
    return P


def execute(P, handle, views, holo, intensity=False, phase=False, complex_out=True):
    import torch
    s = torch.cuda.current_stream().cuda_stream
    shape = [(v["ny1"], v["nx1"]) for v in views]
    outs = [torch.empty(sh, dtype=torch.complex64, device="cuda") for sh in shape] if complex_out else None
    ints = [torch.empty(sh, dtype=torch.float32, device="cuda") for sh in shape] if intensity else None
    phs = [torch.empty(sh, dtype=torch.float32, device="cuda") for sh in shape] if phase else None
    ptr = lambda ts: [t.data_ptr() for t in ts] if ts else None
    P.shifted_fresnel_execute(handle, holo.data_ptr(), ptr(outs), ptr(ints), ptr(phs), stream=s)
    torch.cuda.synchronize()
    assert P.binding.shifted_fresnel_batch_status(handle, stream=s) == 0
    cpu = lambda ts: [t.cpu().numpy() for t in ts] if ts else None
    return cpu(outs), cpu(ints), cpu(phs)


def plan(P, views, precision):
    import torch
    return P.shifted_fresnel_plan(views, precision=precision, stream=torch.cuda.current_stream().cuda_stream)


@pytest.fixture(scope="module")
def c2():
    import torch
    holo, views = synth.config_c2()
    return torch.from_numpy(holo).cuda(), views, holo


@pytest.mark.parametrize("precision", [0, 1, 3])
def test_tensor_stores_match_plain_stores(P, c2, precision):
    """Complex output alone (tensor stores on the y pass) against complex +
    intensity + phase (plain stores): the same bits; intensity and phase agree
    with the field."""
    h, views, _ = c2
    handle = plan(P, views, precision)
    try:
        a, _, _ = execute(P, handle, views, h)
        b, ints, phs = execute(P, handle, views, h, intensity=True, phase=True)
    finally:
        P.shifted_fresnel_destroy(handle)
    for fa, fb, i, ph in zip(a, b, ints, phs):
        assert np.array_equal(fa.view(np.uint64), fb.view(np.uint64))
        f = fb.astype(np.complex128)
        assert np.allclose(i, np.abs(f) ** 2, rtol=1e-5, atol=1e-6 * float(i.max()))
        d = np.angle(np.exp(1j * (ph - np.angle(f))))
        big = np.abs(f) > 1e-3 * np.abs(f).max()
        assert np.abs(d[big]).max() < 1e-4


@pytest.mark.parametrize("precision", [1, 2])
def test_fused_launch_matches_per_pass_launches(P, c2, precision):
    """FP16 / BF16: the fused launch (both passes, tiles claimed from a counter)
    against one launch per pass, complex outputs and intensity-only outputs."""
    h, views, _ = c2
    handle = plan(P, views, precision)
    try:
        n0 = P.shifted_fresnel_kernel_launches()
        fused, _, _ = execute(P, handle, views, h)
        assert P.shifted_fresnel_kernel_launches() - n0 == 1  # both passes of the four views in one launch
        _, fused_int, _ = execute(P, handle, views, h, intensity=True, complex_out=False)
        os.environ["SF_EXECUTE_SINGLE_STREAM"] = "1"
        try:
            n0 = P.shifted_fresnel_kernel_launches()
            single, _, _ = execute(P, handle, views, h)
            assert P.shifted_fresnel_kernel_launches() - n0 == 2  # one launch per pass
            _, single_int, _ = execute(P, handle, views, h, intensity=True, complex_out=False)
        finally:
            del os.environ["SF_EXECUTE_SINGLE_STREAM"]
    finally:
        P.shifted_fresnel_destroy(handle)
    for a, b in zip(fused, single):
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    for a, b in zip(fused_int, single_int):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))


def test_fused_launch_eight_views_and_repeat(P):
    """The largest fused launch (eight views, 4096 tiles) against the oracle on
    two of its views, and a second execute of the same plan (the tile counter
    is reset per launch) giving the same bits."""
    import torch
    holo = synth.gabor_hologram(1024, seed=4401)
    views = [view(WAVELENGTH, z, PITCH, p1, o1=(dx, -dx)) for z, p1, dx in
             ((0.02, 0.6e-6, 1e-4), (0.03, 1.0e-6, -2e-4), (0.045, 1.5e-6, 3e-4), (0.06, 2.0e-6, 0.0),
              (0.075, 2.5e-6, -1e-4), (0.09, 3.0e-6, 2e-4), (0.11, 3.5e-6, -3e-4), (0.13, 4.65e-6, 5e-5))]
    h = torch.from_numpy(holo.astype(np.float32)).cuda()
    handle = plan(P, views, 1)
    try:
        n0 = P.shifted_fresnel_kernel_launches()
        first, _, _ = execute(P, handle, views, h)
        assert P.shifted_fresnel_kernel_launches() - n0 == 1
        again, _, _ = execute(P, handle, views, h)
    finally:
        P.shifted_fresnel_destroy(handle)
    for a, b in zip(first, again):
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
    for i in (0, 7):
        err = rel_l2(first[i], oracle.forward(holo, views[i]))
        print(f"view {i}: rel-L2 {err:.3e}")
        assert err <= 2e-3


@pytest.mark.parametrize("impl", ["half", "double"])
def test_rows_per_cta_variants_paper_scale(P, c2, impl, monkeypatch):
    """The FP32 row pass with half (one row, plain stores) and twice (four rows, tensor stores) the
    default rows per CTA on the paper-scale step: the same bits as the default plan."""
    h, views, _ = c2
    handle = plan(P, views, 0)
    try:
        ref, _, _ = execute(P, handle, views, h)
    finally:
        P.shifted_fresnel_destroy(handle)
    monkeypatch.setenv("SF_PASS_IMPL", impl)
    handle = plan(P, views, 0)
    try:
        got, _, _ = execute(P, handle, views, h)
    finally:
        P.shifted_fresnel_destroy(handle)
    for a, b in zip(got, ref):
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))



def test_fused_launch_poisoned_dependency_times_out(P, c2, monkeypatch):
    """A y-tile dependency that the host makes unsatisfiable (view 1) ends the fused launch through its
    bounded waits: the plan reports SF_ERR_TIMEOUT once, and the next execute gives the same bits again."""
    import torch
    h, views, _ = c2
    handle = plan(P, views, 1)
    try:
        ref, _, _ = execute(P, handle, views, h)
        monkeypatch.setenv("SF_T5_POISON_VIEW", "1")
        monkeypatch.setenv("SF_T5_SPIN_LIMIT", "2000")
        s = torch.cuda.current_stream().cuda_stream
        outs = [torch.empty((v["ny1"], v["nx1"]), dtype=torch.complex64, device="cuda") for v in views]
        n0 = P.shifted_fresnel_kernel_launches()
        P.shifted_fresnel_execute(handle, h.data_ptr(), [o.data_ptr() for o in outs], stream=s)
        assert P.shifted_fresnel_kernel_launches() - n0 == 1
        assert P.binding.shifted_fresnel_batch_status(handle, stream=s) == P.SF_ERR_TIMEOUT
        assert P.binding.shifted_fresnel_batch_status(handle, stream=s) == 0  # cleared
        monkeypatch.delenv("SF_T5_POISON_VIEW")
        monkeypatch.delenv("SF_T5_SPIN_LIMIT")
        again, _, _ = execute(P, handle, views, h)
    finally:
        P.shifted_fresnel_destroy(handle)
    for a, b in zip(again, ref):
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))
