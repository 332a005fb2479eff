"""Mixed-precision (tensor-core) row passes against the FP64 oracle.

Axes of FFT length 2048, 1024 or 512 with input and output lengths of at most
half of it run the four-step tcgen05 pass; other axes of length 2048 or 4096 run
the mma.sync radix-16/8 stages (FP16TC / BF16TC only); every other axis runs
in FP32.  Bars, relative L2 per view against the oracle over every pixel:

* FP16TC and BF16X3TC: 2e-3, the reduced-precision tolerance.
* FP16X3TC: 1e-5 (on the tcgen05 axes; its other axes run in FP32).
* BF16TC is out of the 2e-3 tolerance by construction (an 8-bit mantissa
  rounded at every stage): its tests check that the error stays inside the
  band the documentation reports (2e-3 .. 1.5e-2), not parity.
"""

import numpy as np
import pytest

import oracle
import synth
from synth import view, random_field, WAVELENGTH, PITCH
from helpers import rel_l2

pytestmark = pytest.mark.gpu

FP16, BF16, FP16X3, BF16X3 = 1, 2, 3, 4
TOL_FP16 = 2e-3
BF16_BAND = (2e-3, 1.5e-2)


def check(prec, err, split_bar=1e-5):
    if prec == BF16:
        assert BF16_BAND[0] < err < BF16_BAND[1], f"bf16 error {err:.3e} outside its documented band"
    elif prec == FP16X3:
        assert err <= split_bar, err
    else:
        assert err <= TOL_FP16, err


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


@pytest.mark.parametrize("prec", [FP16, BF16, FP16X3, BF16X3])
def test_tensor_core_x_pass_full_parity(P, prec):
    """FFT length 2048 along x (tcgen05 pass), a thin y axis (FP32): every output pixel."""
    v = view(WAVELENGTH, -0.05, PITCH, 2.325e-6, o1=(100e-6, -50e-6), n0=(1024, 16), n1=(1024, 12))
    holo = synth.gabor_hologram(1024, seed=3001)[:16]
    got = run(P, [v], holo, prec)[0]
    err = rel_l2(got, oracle.forward(holo, v))
    print(f"precision {prec}: rel-L2 {err:.3e}")
    check(prec, err)


_C4 = {}


@pytest.mark.parametrize("prec", [FP16, BF16, FP16X3, BF16X3])
def test_tensor_core_single_views_every_pixel(P, prec):
    """The 1024^2 and 2048^2 single views (FFT lengths 2048 and 4096 on both axes): every pixel.
    At 4096 the FP16 / BF16 plans run the mma.sync stages and the x3 plans FP32."""
    for holo, views in synth.config_c4()[1:]:
        v = views[0]
        key = v["nx1"]
        if key not in _C4:
            _C4[key] = oracle.forward(holo, v)
        got = run(P, views, holo, prec)[0]
        err = rel_l2(got, _C4[key])
        print(f"precision {prec} n {key}: rel-L2 {err:.3e}")
        check(prec, err)


def test_tensor_core_complex_input_and_fallback_lengths(P):
    """Complex object, and axes whose lengths are not tensor-core lengths fall back to FP32."""
    v = view(WAVELENGTH, 0.04, PITCH, 1.5e-6, o1=(2e-4, -1e-4), n0=(1024, 100), n1=(1000, 90), flags=8)
    holo = random_field(100, 1024, seed=7)
    got = run(P, [v], holo, FP16)[0]
    assert rel_l2(got, oracle.forward(holo, v)) <= TOL_FP16
    # lengths beyond half the FFT length (no 2N padding) take no tensor-core pass: FP32 (FFT length 512)
    small = view(WAVELENGTH, 0.05, PITCH, 2e-6, n0=(300, 270), n1=(180, 200))
    h2 = random_field(270, 300, seed=8).real
    got = run(P, [small], h2, FP16)[0]
    assert rel_l2(got, oracle.forward(h2, small)) <= 1e-5
