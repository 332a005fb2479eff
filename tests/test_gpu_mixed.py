"""Mixed-precision (tensor-core) row passes against the FP64 oracle.

SF_PREC_FP16TC runs the radix-16/8 DFT stages of axes with FFT length 2048
or 4096 as FP16 tensor-core products with FP32 accumulation; the
reduced-precision tolerance is relative L2 <= 2e-3 per view.  SF_PREC_BF16TC
is measured and bounded more loosely (its 8-bit mantissa is expected to miss
2e-3).  Axes of other lengths run in FP32 and keep the 1e-5 bar.
"""

import numpy as np
import pytest

import oracle
import synth
from synth import view, random_field, WAVELENGTH, PITCH
from helpers import rel_l2

pytestmark = pytest.mark.gpu

FP16 = 1
BF16 = 2
TOL_FP16 = 2e-3
TOL_BF16 = 2e-2


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1001_4309_gb300 import build as b
    b.build()
    import paper_1001_4309_gb300 as P
    return P


def run(P, views, holo, precision):
    import torch
    complex_in = bool(views[0].get("flags", 0) & 8)
    h = torch.from_numpy(np.ascontiguousarray(holo.astype(np.complex64 if complex_in else np.float32))).cuda()
    handle = P.shifted_fresnel_plan(views, precision=precision, stream=torch.cuda.current_stream().cuda_stream)
    try:
        outs = [torch.empty((v["ny1"], v["nx1"]), dtype=torch.complex64, device="cuda") for v in views]
        P.shifted_fresnel_execute(handle, h.data_ptr(), [o.data_ptr() for o in outs],
                                  stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        return [o.cpu().numpy() for o in outs]
    finally:
        P.shifted_fresnel_destroy(handle)


@pytest.mark.parametrize("prec,tol", [(FP16, TOL_FP16), (BF16, TOL_BF16)])
def test_tensor_core_x_pass_full_parity(P, prec, tol):
    """FFT length 2048 along x (tensor cores), a thin y axis (FP32): every output pixel."""
    v = view(WAVELENGTH, -0.05, PITCH, 2.325e-6, o1=(100e-6, -50e-6), n0=(1024, 16), n1=(1024, 12))
    holo = synth.gabor_hologram(1024, seed=3001)[:16]
    got = run(P, [v], holo, prec)[0]
    err = rel_l2(got, oracle.forward(holo, v))
    print(f"precision {prec}: rel-L2 {err:.3e}")
    assert err <= tol


@pytest.mark.parametrize("prec,tol", [(FP16, TOL_FP16), (BF16, TOL_BF16)])
def test_tensor_core_both_axes_sampled(P, prec, tol):
    """The 1024^2 and 2048^2 single views (FFT lengths 2048 and 4096 on both axes)."""
    for holo, views in synth.config_c4()[1:]:
        got = run(P, views, holo, prec)[0]
        v = views[0]
        n = v["nx1"]
        for cols in ((0, 4), (n // 2 - 2, n // 2 + 2), (n - 4, n)):
            err = rel_l2(got[:, cols[0]:cols[1]], oracle.forward(holo, v, cols=cols))
            print(f"precision {prec} n {n} cols {cols}: rel-L2 {err:.3e}")
            assert err <= tol


def test_tensor_core_paper_scale_four_views(P):
    holo, views = synth.config_c2()
    got = run(P, views, holo, FP16)
    for i, v in enumerate(views):
        cols = (500, 508)
        err = rel_l2(got[i][:, cols[0]:cols[1]], oracle.forward(holo, v, cols=cols))
        assert err <= TOL_FP16, (i, err)


def test_tensor_core_complex_input_and_fallback_lengths(P):
    """Complex object, and axes whose lengths are not tensor-core lengths fall back to FP32."""
    v = view(WAVELENGTH, 0.04, PITCH, 1.5e-6, o1=(2e-4, -1e-4), n0=(1024, 100), n1=(1000, 90), flags=8)
    holo = random_field(100, 1024, seed=7)
    got = run(P, [v], holo, FP16)[0]
    assert rel_l2(got, oracle.forward(holo, v)) <= TOL_FP16
    small = view(WAVELENGTH, 0.05, PITCH, 2e-6, n0=(200, 150), n1=(180, 160))
    h2 = random_field(150, 200, seed=8).real
    got = run(P, [small], h2, FP16)[0]
    assert rel_l2(got, oracle.forward(h2, small)) <= 1e-5
