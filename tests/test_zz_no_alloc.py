"""The allocation-free entry point gives the same views as the plan path.

shifted_fresnel_execute_static is for callers that cannot allocate device
memory while they run (for example a plugin whose host application owns
all device allocations, or an acquisition loop with a memory budget fixed
before the first frame): they cannot create a plan, which calls cudaMalloc.
It keeps everything in one fixed device array shared by all calls, so the
check below runs two different views back to back on one stream (the second
call reuses the array the first left behind) and compares both with a
one-view plan's shifted_fresnel_execute, then repeats the first view.

This file is named so that pytest collects it last.
"""

import numpy as np
import pytest

from synth import view, random_field, WAVELENGTH, PITCH
from helpers import rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5  # relative L2, the FP32 tolerance of the parity tests


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1001_4309_gb300 import build as b
    b.build()
    import paper_1001_4309_gb300 as P
    return P


VIEW_A = view(WAVELENGTH, -0.05, PITCH, 2.325e-6, o1=(100e-6, -50e-6), n0=(256, 256), n1=(256, 256))
VIEW_B = view(WAVELENGTH, 0.07, (PITCH, 3.1e-6), (1.0e-6, 2.2e-6), o0=(1e-5, 0), o1=(-3e-4, 2e-4),
              n0=(300, 200), n1=(500, 120), flags=8)
VIEW_C = view(WAVELENGTH, 0.035, PITCH, 2.9e-6, o1=(1e-4, -2e-4), n0=(1024, 64), n1=(400, 64))  # FFT length 1536


def inputs(v, seed):
    import torch
    h = random_field(v["ny0"], v["nx0"], seed=seed, complex_=bool(v["flags"] & 8))
    h = h.astype(np.complex64) if v["flags"] & 8 else h.real.astype(np.float32)
    return torch.from_numpy(h).cuda()


def plan_path(P, v, holo):
    sf = P.ShiftedFresnel([v])
    try:
        out = sf.reconstruct(holo, field=True, intensity=True, phase=True)
        return {k: x[0].clone() for k, x in out.items()}
    finally:
        sf.close()


def static_path(P, v, holo):
    import torch
    shp = (v["ny1"], v["nx1"])
    f = torch.empty(shp, dtype=torch.complex64, device="cuda")
    I = torch.empty(shp, dtype=torch.float32, device="cuda")
    ph = torch.empty(shp, dtype=torch.float32, device="cuda")
    P.shifted_fresnel_execute_static(v, holo.data_ptr(), f.data_ptr(), I.data_ptr(), ph.data_ptr(),
                                     stream=torch.cuda.current_stream().cuda_stream)
    return {"field": f, "intensity": I, "phase": ph}


def compare(got, ref):
    import torch
    torch.cuda.synchronize()
    f, fr = got["field"].cpu().numpy(), ref["field"].cpu().numpy()
    assert rel_l2(f, fr) <= TOL
    assert rel_l2(got["intensity"].cpu().numpy(), ref["intensity"].cpu().numpy()) <= 3 * TOL
    w = np.abs(fr) * np.exp(1j * got["phase"].cpu().numpy())
    assert rel_l2(w, fr) <= 3 * TOL


def test_static_entry_matches_plan_on_consecutive_calls(P):
    ha, hb = inputs(VIEW_A, 1), inputs(VIEW_B, 2)
    ref_a, ref_b = plan_path(P, VIEW_A, ha), plan_path(P, VIEW_B, hb)
    first = static_path(P, VIEW_A, ha)
    second = static_path(P, VIEW_B, hb)
    compare(first, ref_a)
    compare(second, ref_b)
    third = static_path(P, VIEW_A, ha)  # after a larger view left its data in the array
    compare(third, ref_a)
    hc = inputs(VIEW_C, 3)
    compare(static_path(P, VIEW_C, hc), plan_path(P, VIEW_C, hc))  # a length with a factor 3


def test_static_entry_rejects_sizes_beyond_its_scratch(P):
    import torch
    holo = torch.zeros((1, 1), dtype=torch.float32, device="cuda")
    out = torch.empty((1, 1), dtype=torch.complex64, device="cuda")
    too_long = view(WAVELENGTH, 0.05, PITCH, PITCH, n0=(1500, 1), n1=(600, 1))  # needs FFT length 2304
    assert P.shifted_fresnel_execute_static(too_long, holo.data_ptr(), out.data_ptr(), check=False) \
        == P.SF_ERR_UNSUPPORTED_SIZE
    too_big = view(WAVELENGTH, 0.05, PITCH, PITCH, n0=(8, 1100), n1=(1000, 8))  # nx1 * ny0 > 2^20
    assert P.shifted_fresnel_execute_static(too_big, holo.data_ptr(), out.data_ptr(), check=False) \
        == P.SF_ERR_UNSUPPORTED_SIZE


VIEW_D = view(WAVELENGTH, 0.05, PITCH, 2.0e-6, o1=(2e-4, -1e-4), n0=(1024, 1024), n1=(1024, 1024))  # L 2048, 2^20


def test_static_entry_allocates_nothing_at_its_largest_view(P):
    """The largest supported view (FFT length 2048 on both axes, nx1 * ny0 = 2^20), with every output
    combination, including an intensity image alone: same results as the plan path, and the device's
    free memory does not change across the calls (after a first call, which may load the module)."""
    import torch
    hd = inputs(VIEW_D, 4)
    ref = plan_path(P, VIEW_D, hd)
    shp = (VIEW_D["ny1"], VIEW_D["nx1"])
    f = torch.empty(shp, dtype=torch.complex64, device="cuda")
    I = torch.empty(shp, dtype=torch.float32, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    P.shifted_fresnel_execute_static(VIEW_D, hd.data_ptr(), f.data_ptr(), None, None, stream=s)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    I.zero_()
    P.shifted_fresnel_execute_static(VIEW_D, hd.data_ptr(), None, I.data_ptr(), None, stream=s)  # intensity only
    torch.cuda.synchronize()
    intensity_only = I.cpu().numpy()
    P.shifted_fresnel_execute_static(VIEW_D, hd.data_ptr(), f.data_ptr(), I.data_ptr(), None, stream=s)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert rel_l2(f.cpu().numpy(), ref["field"].cpu().numpy()) <= TOL
    assert rel_l2(intensity_only, ref["intensity"].cpu().numpy()) <= 3 * TOL
    assert np.array_equal(intensity_only, I.cpu().numpy())
