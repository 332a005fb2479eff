"""C-ABI checks that need no GPU: the library loads, exports every declared
symbol, and rejects bad arguments before touching the device."""

import ctypes
import glob
import math
import os

import pytest

from helpers import header_functions

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1001_4309_gb300 import build as b
    b.build()
    import paper_1001_4309_gb300 as P
    return P


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(lib.binding.library_path())
    headers = glob.glob(os.path.join(ROOT, "include", "*.h"))
    assert headers
    names = []
    for h in headers:
        names += header_functions(h)
    assert "shifted_fresnel_plan" in names and "shifted_fresnel_execute" in names
    for n in names:
        assert hasattr(raw, n), f"{n} declared but not exported"


def test_library_is_in_tree_and_built_for_sm103a(lib):
    path = lib.binding.library_path()
    assert path.startswith(ROOT)
    assert os.path.getsize(path) > 0


def base_view(**kw):
    from synth import view
    v = view(632.8e-9, 0.05, 4.65e-6, 2.0e-6, n0=(16, 16), n1=(16, 16))
    v.update(kw)
    return v


@pytest.mark.parametrize("bad", [
    dict(z=0.0), dict(z=float("nan")), dict(z=float("inf")), dict(wavelength=0.0), dict(wavelength=-1e-6),
    dict(px0=0.0), dict(py1=-1e-6), dict(px1=float("nan")), dict(ox1=float("inf")),
    dict(nx0=0), dict(ny1=-3), dict(flags=1 << 10),
])
def test_plan_rejects_invalid_view(lib, bad):
    rc, h = lib.shifted_fresnel_plan([base_view(**bad)], check=False)
    assert rc == lib.SF_ERR_INVALID_ARG
    assert not h.value


def test_plan_rejects_oversize(lib):
    rc, _ = lib.shifted_fresnel_plan([base_view(nx0=4097, nx1=4097)], check=False)
    assert rc == lib.SF_ERR_UNSUPPORTED_SIZE
    rc, _ = lib.shifted_fresnel_plan([base_view(ny0=8000, ny1=200)], check=False)
    assert rc == lib.SF_ERR_UNSUPPORTED_SIZE


def test_plan_rejects_inconsistent_views(lib):
    rc, _ = lib.shifted_fresnel_plan([base_view(), base_view(nx0=17)], check=False)
    assert rc == lib.SF_ERR_INVALID_ARG
    rc, _ = lib.shifted_fresnel_plan([base_view(), base_view(flags=lib.SF_IN_COMPLEX)], check=False)
    assert rc == lib.SF_ERR_INVALID_ARG


def test_plan_rejects_bad_counts_and_precision(lib):
    L = lib.load()
    from paper_1001_4309_gb300.binding import sf_view
    h = ctypes.c_void_p()
    arr = (sf_view * 1)(lib.make_view(base_view()))
    assert L.shifted_fresnel_plan(ctypes.byref(h), arr, 0, 0, 0, None) == lib.SF_ERR_INVALID_ARG
    assert L.shifted_fresnel_plan(ctypes.byref(h), None, 1, 0, 0, None) == lib.SF_ERR_INVALID_ARG
    assert L.shifted_fresnel_plan(None, arr, 1, 0, 0, None) == lib.SF_ERR_INVALID_ARG
    assert L.shifted_fresnel_plan(ctypes.byref(h), arr, 1, 99, 0, None) == lib.SF_ERR_INVALID_ARG


def test_null_plan_calls(lib):
    L = lib.load()
    assert L.shifted_fresnel_execute(None, None, None, None, None, None) == lib.SF_ERR_INVALID_ARG
    assert L.shifted_fresnel_destroy(None) == lib.SF_ERR_INVALID_ARG
    assert L.shifted_fresnel_plan_query(None, 0, None, None, None) == lib.SF_ERR_INVALID_ARG


def test_strerror_covers_every_code(lib):
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert lib.shifted_fresnel_strerror(code) != "unknown status"
    assert lib.shifted_fresnel_strerror(-99) == "unknown status"


def test_valid_plan_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, h = lib.shifted_fresnel_plan([base_view()], check=False)
    assert rc == lib.SF_ERR_CUDA
    assert not h.value


def test_fft_length_choice_without_gpu():
    """Smallest supported length >= n0 + n1 - 1 (Section 2.2, step 2's zero padding), host only."""
    from paper_1001_4309_gb300 import shifted_fresnel_fft_length as fl, SF_ERR_INVALID_ARG, SF_ERR_UNSUPPORTED_SIZE
    # the paper's 1024 -> 1024 views pad to 2N = 2048
    assert fl(1024 + 1024 - 1) == 2048
    cases = {1: 64, 64: 64, 65: 128, 1025: 1536, 1535: 1536, 1536: 1536, 1537: 2048, 2048: 2048,
             2049: 2304, 2303: 2304, 2305: 3072, 3071: 3072, 3073: 4096, 4095: 4096, 4097: 4608,
             4608: 4608, 4609: 6144, 6143: 6144, 6145: 8192, 8192: 8192}
    for need, L in cases.items():
        assert fl(need) == L, need
        p2 = fl(need, allow_mixed=False)
        assert p2 >= need and p2 & (p2 - 1) == 0 and p2 // 2 < max(need, 64)
    assert fl(0) == SF_ERR_INVALID_ARG
    assert fl(8193) == SF_ERR_UNSUPPORTED_SIZE


def test_missing_library_fails_loudly(lib, monkeypatch, tmp_path):
    """No CPU fallback: without the compiled library every entry point raises."""
    from paper_1001_4309_gb300 import binding
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "library_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        binding.load()
    with pytest.raises(RuntimeError, match="missing"):
        binding.shifted_fresnel_plan([base_view()])
    with pytest.raises(RuntimeError, match="missing"):
        binding.shifted_fresnel_fft_length(2047)


def test_plan_update_rejects_null_arguments(lib):
    """shifted_fresnel_plan_update checks its arguments before touching a device."""
    assert lib.shifted_fresnel_plan_update(None, [base_view()], check=False) == lib.SF_ERR_INVALID_ARG
    raw = lib.load().shifted_fresnel_plan_update
    assert raw(None, None, 1, None) == lib.SF_ERR_INVALID_ARG


def test_intensity_loss_rejects_null_arguments(lib):
    raw = lib.load().shifted_fresnel_intensity_loss
    assert raw(None, None, None, None, None, None) == lib.SF_ERR_INVALID_ARG
