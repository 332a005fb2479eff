"""Batched execution of ragged views over a stream of holograms.

shifted_fresnel_execute_batch runs every (hologram, view) of a call either
as one graph launch of the persistent kernel or as the per-length row-pass
kernels on two streams; with either implementation its outputs must equal,
bit for bit, shifted_fresnel_execute on each hologram (same arithmetic),
across power-of-two and mixed (factor 3) FFT lengths in one call, more
holograms than intermediate slots, changing hologram counts and repeated
calls.  A host-poisoned work queue must end the persistent launch through
its bounded waits and be reported as SF_ERR_TIMEOUT.
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


N0 = (300, 280)


def ragged_views():
    rng = np.random.default_rng(11)
    sizes = [(300, 280), (64, 512), (1000, 30), (7, 3), (2000, 16), (33, 65), (200, 200)]
    out = []
    for k, n1 in enumerate(sizes):
        out.append(view(WAVELENGTH, float(rng.uniform(0.02, 0.12)), PITCH,
                        float(np.exp(rng.uniform(np.log(0.25e-6), np.log(9.3e-6)))),
                        o1=tuple(rng.uniform(-2e-3, 2e-3, size=2)), n0=N0, n1=n1))
    return out


def holograms(n, shape=N0, seed=0):
    import torch
    return [torch.from_numpy(random_field(shape[1], shape[0], seed=seed + h).real.astype(np.float32)).cuda()
            for h in range(n)]


def per_hologram(sf, holos):
    import torch
    res = []
    for h in holos:
        o = sf.reconstruct(h, field=True, intensity=True)
        res.append(([f.clone() for f in o["field"]], [i.clone() for i in o["intensity"]]))
    torch.cuda.synchronize()
    return res


def check_equal(outs, ref):
    for h, (f_ref, i_ref) in enumerate(ref):
        for v in range(len(f_ref)):
            assert np.array_equal(outs["field"][h][v].cpu().numpy(), f_ref[v].cpu().numpy()), (h, v)
            assert np.array_equal(outs["intensity"][h][v].cpu().numpy(), i_ref[v].cpu().numpy()), (h, v)


IMPLS = ["persistent", "streams"]


@pytest.mark.parametrize("impl", IMPLS)
def test_batch_equals_per_hologram_execute(P, impl, monkeypatch):
    import torch
    monkeypatch.setenv("SF_BATCH_IMPL", impl)
    vs = ragged_views()
    sf = P.ShiftedFresnel(vs)
    try:
        lengths = {sf.sizes(i)[0] for i in range(len(vs))} | {sf.sizes(i)[1] for i in range(len(vs))}
        assert min(lengths) <= 512 and max(lengths) >= 2304 and any(L & (L - 1) for L in lengths)
        holos = holograms(5)
        ref = per_hologram(sf, holos)
        outs = sf.alloc_batch_outputs(5, field=True, intensity=True)
        sf.execute_batch(holos, outs)
        assert P.shifted_fresnel_batch_status(sf.handle, torch.cuda.current_stream().cuda_stream) == P.SF_OK
        check_equal(outs, ref)
        # a different hologram count rebuilds the graph; the original count again reuses a new one
        outs2 = sf.alloc_batch_outputs(2, field=True, intensity=True)
        sf.execute_batch(holos[3:], outs2)
        torch.cuda.synchronize()
        check_equal(outs2, ref[3:])
        for _ in range(3):  # repeated calls alternate the pinned descriptor tables
            sf.execute_batch(holos, outs)
        torch.cuda.synchronize()
        check_equal(outs, ref)
        # and the batch agrees with the oracle on a sampled view
        h_np = holos[4].cpu().numpy()
        v = vs[0]
        cols = (140, 148)
        got = outs["field"][4][0].cpu().numpy()[:, cols[0]:cols[1]]
        assert rel_l2(got, oracle.forward(h_np, v, cols=cols)) <= 1e-5
    finally:
        sf.close()


_RAGGED_REF = {}  # oracle views of the ragged-set test, shared by both implementations


@pytest.mark.parametrize("impl", IMPLS)
def test_batch_paper_sized_ragged_views(P, impl, monkeypatch):
    """2048^2 holograms with views of 256^2 .. 2048^2 (FFT lengths 2304, 3072 and 4096)."""
    import torch
    monkeypatch.setenv("SF_BATCH_IMPL", impl)
    _, all_views = synth.config_c3(n_holos=1, n_views=64, with_holograms=False)
    picked = {}
    for v in all_views[0]:
        picked.setdefault(v["nx1"], v)
    vs = [picked[k] for k in sorted(picked)]
    holos = [torch.from_numpy(synth.gabor_hologram(2048, seed=2000 + h, kind="target_blobs", photons=2000)).cuda()
             for h in range(3)]
    sf = P.ShiftedFresnel(vs)
    try:
        ref = per_hologram(sf, holos)
        outs = sf.alloc_batch_outputs(3, field=True, intensity=True)
        sf.execute_batch(holos, outs)
        torch.cuda.synchronize()
        check_equal(outs, ref)
        # full-size parity against the oracle: every pixel of one view of each size class
        h_np = holos[2].cpu().numpy()
        for v_i, v in enumerate(vs):
            got = outs["field"][2][v_i].cpu().numpy()
            key = (v["nx1"], v["z"], v["px1"])
            if key not in _RAGGED_REF:
                _RAGGED_REF[key] = oracle.forward(h_np, v)
            err = rel_l2(got, _RAGGED_REF[key])
            assert err <= 1e-5, (v["nx1"], err)
    finally:
        sf.close()


@pytest.mark.parametrize("general,cplx", [(False, False), (True, False), (False, True)])
def test_batch_one_length_kernel(P, general, cplx, monkeypatch):
    """Every pass at one power-of-two length with n0, n1 <= L / 2: the persistent
    batch runs the kernel specialised to that length (pruned network), bit for
    bit equal to per-hologram execute, for real and complex holograms;
    SF_BATCH_GENERAL=1 keeps the general kernel (unpruned network: equal up to
    rounding)."""
    import torch
    monkeypatch.setenv("SF_BATCH_IMPL", "persistent")
    if general:
        monkeypatch.setenv("SF_BATCH_GENERAL", "1")
    n = 512
    rng = np.random.default_rng(5)
    flags = P.SF_IN_COMPLEX if cplx else 0
    vs = [view(WAVELENGTH, z, PITCH, p1, o1=tuple(rng.uniform(-5e-4, 5e-4, size=2)), n0=(n, n), n1=(n1x, n1y),
               flags=flags)
          for z, p1, n1x, n1y in ((0.03, 4.65e-6, 512, 512), (0.05, 2e-6, 512, 400), (0.07, 1e-6, 300, 512),
                                  (0.1, 0.5e-6, 512, 512))]
    sf = P.ShiftedFresnel(vs)
    try:
        assert all(sf.sizes(i)[:2] == (1024, 1024) for i in range(len(vs)))
        if cplx:
            holos = [torch.from_numpy(random_field(n, n, seed=60 + h).astype(np.complex64)).cuda() for h in range(5)]
        else:
            holos = holograms(5, shape=(n, n), seed=60)
        ref = per_hologram(sf, holos)
        outs = sf.alloc_batch_outputs(5, field=True, intensity=True)
        for _ in range(2):
            sf.execute_batch(holos, outs)
            assert P.shifted_fresnel_batch_status(sf.handle, torch.cuda.current_stream().cuda_stream) == P.SF_OK
            if general:
                for h, (f_ref, _) in enumerate(ref):
                    for v in range(len(vs)):
                        assert rel_l2(outs["field"][h][v].cpu().numpy(), f_ref[v].cpu().numpy()) <= 1e-6
            else:
                check_equal(outs, ref)
    finally:
        sf.close()


@pytest.mark.parametrize("n_holos", [1, 20, 37])
def test_batch_streams_many_small_holograms(P, n_holos, monkeypatch):
    """Small views: the two-stream batch puts up to 16 holograms in each row-pass
    launch (each with its own intermediate slot; chunks alternate streams).
    Equal to per-hologram execute for a partial last chunk and over replays."""
    import torch
    monkeypatch.setenv("SF_BATCH_IMPL", "streams")
    n = 256
    vs = [view(WAVELENGTH, -0.05, PITCH, 2.325e-6, o1=(1e-4, -5e-5), n0=(n, n), n1=(n, n))]
    sf = P.ShiftedFresnel(vs)
    try:
        holos = holograms(n_holos, shape=(n, n), seed=90)
        ref = per_hologram(sf, holos)
        outs = sf.alloc_batch_outputs(n_holos, field=True, intensity=True)
        for _ in range(3):  # capture, then replays
            sf.execute_batch(holos, outs)
            torch.cuda.synchronize()
            check_equal(outs, ref)
    finally:
        sf.close()


def test_batch_tensor_core_plan(P, monkeypatch):
    """A tensor-core plan batches through the streams implementation (bit-identical
    to its per-hologram execute); the persistent kernel, FP32 only, refuses it."""
    import torch
    n = 1024
    vs = [view(WAVELENGTH, z, PITCH, p1, n0=(n, n), n1=(n, n)) for z, p1 in ((0.03, 4.65e-6), (0.07, 1e-6))]
    sf = P.ShiftedFresnel(vs, precision=P.SF_PREC_FP16TC)
    try:
        holos = holograms(3, shape=(n, n), seed=30)
        ref = per_hologram(sf, holos)
        outs = sf.alloc_batch_outputs(3, field=True, intensity=True)
        sf.execute_batch(holos, outs)
        torch.cuda.synchronize()
        check_equal(outs, ref)
        monkeypatch.setenv("SF_BATCH_IMPL", "persistent")
        rc = P.shifted_fresnel_execute_batch(sf.handle, [h.data_ptr() for h in holos],
                                             [o.data_ptr() for row in outs["field"] for o in row], check=False)
        assert rc == P.SF_ERR_UNSUPPORTED_SIZE
    finally:
        sf.close()


def test_batch_rejects_bad_arguments(P):
    import torch
    vs = ragged_views()[:2]
    sf = P.ShiftedFresnel(vs)
    try:
        h = holograms(1)
        f = [torch.empty((v["ny1"], v["nx1"]), dtype=torch.complex64, device="cuda") for v in vs]
        rc = P.shifted_fresnel_execute_batch(sf.handle, [h[0].data_ptr()], [f[0].data_ptr(), None], check=False)
        assert rc == P.SF_ERR_INVALID_ARG  # a (hologram, view) without outputs
        host = torch.empty_like(f[0], device="cpu")
        rc = P.shifted_fresnel_execute_batch(sf.handle, [h[0].data_ptr()], [host.data_ptr(), f[1].data_ptr()],
                                             check=False)
        assert rc == P.SF_ERR_INVALID_ARG  # host memory is not staged by the batch path
        assert P.shifted_fresnel_execute_batch(sf.handle, [], None, check=False) == P.SF_ERR_INVALID_ARG
    finally:
        sf.close()
    big = view(WAVELENGTH, 0.05, PITCH, PITCH, n0=(6000, 4), n1=(200, 4))  # FFT length 8192
    sfb = P.ShiftedFresnel([big])
    try:
        hb = torch.from_numpy(random_field(4, 6000, seed=1).real.astype(np.float32)).cuda()
        fb = torch.empty((4, 200), dtype=torch.complex64, device="cuda")
        os.environ["SF_BATCH_IMPL"] = "persistent"  # beyond the persistent kernel's lengths
        try:
            rc = P.shifted_fresnel_execute_batch(sfb.handle, [hb.data_ptr()], [fb.data_ptr()], check=False)
        finally:
            del os.environ["SF_BATCH_IMPL"]
        assert rc == P.SF_ERR_UNSUPPORTED_SIZE
        # the default falls back to the per-length kernels, which take any length
        rc = P.shifted_fresnel_execute_batch(sfb.handle, [hb.data_ptr()], [fb.data_ptr()], check=False)
        assert rc == P.SF_OK
        ref = sfb.reconstruct(hb, field=True)["field"][0]
        torch.cuda.synchronize()
        assert torch.equal(fb, ref)
    finally:
        sfb.close()


def test_poisoned_queue_times_out_and_is_reported(P):
    """A dependency the host makes unsatisfiable ends the launch through the bounded waits."""
    import torch
    vs = ragged_views()[:3]
    os.environ["SF_BATCH_POISON_GROUP"] = str(len(vs))  # the first y-pass group never sees its x tiles
    os.environ["SF_BATCH_SPIN_LIMIT"] = "2000"
    os.environ["SF_BATCH_IMPL"] = "persistent"
    try:
        sf = P.ShiftedFresnel(vs)
        outs = sf.alloc_batch_outputs(2, field=True)
        sf.execute_batch(holograms(2), outs)
        s = torch.cuda.current_stream().cuda_stream
        assert P.shifted_fresnel_batch_status(sf.handle, s) == P.SF_ERR_TIMEOUT
        assert P.shifted_fresnel_batch_status(sf.handle, s) == P.SF_OK  # cleared
        sf.close()
    finally:
        del os.environ["SF_BATCH_POISON_GROUP"]
        del os.environ["SF_BATCH_SPIN_LIMIT"]
        del os.environ["SF_BATCH_IMPL"]
    # the context is still usable
    sf = P.ShiftedFresnel(vs)
    try:
        holos = holograms(2)
        ref = per_hologram(sf, holos)
        outs = sf.alloc_batch_outputs(2, field=True, intensity=True)
        sf.execute_batch(holos, outs)
        torch.cuda.synchronize()
        check_equal(outs, ref)
    finally:
        sf.close()


def test_batch_autotuned_implementation(P, monkeypatch):
    """SF_AUTOTUNE=1: the first call per hologram count times both implementations; outputs stay exact."""
    import torch
    monkeypatch.setenv("SF_AUTOTUNE", "1")
    vs = ragged_views()[:4]
    sf = P.ShiftedFresnel(vs)
    try:
        holos = holograms(3, seed=7)
        ref = per_hologram(sf, holos)
        for _ in range(2):  # the first call measures, the second uses the choice
            outs = sf.alloc_batch_outputs(3, field=True, intensity=True)
            sf.execute_batch(holos, outs)
            torch.cuda.synchronize()
            check_equal(outs, ref)
    finally:
        sf.close()


@pytest.mark.parametrize("fused", ["default", "per-pass"])
def test_tensor_core_batch_equals_per_hologram(P, fused, monkeypatch):
    """FP16 plan of two 1024^2 views (both axes on the tcgen05 pass): the streams batch with one fused
    launch per hologram on alternating streams (default) or one launch per pass gives the bits of
    per-hologram execute, field and intensity."""
    import torch
    if fused == "per-pass":
        monkeypatch.setenv("SF_T5_FUSED", "0")
    n = 1024
    vs = [view(WAVELENGTH, 0.04, PITCH, 2e-6, n0=(n, n), n1=(n, n)),
          view(WAVELENGTH, 0.07, PITCH, 1e-6, o1=(1e-4, 0.0), n0=(n, n), n1=(n, n))]
    sf = P.ShiftedFresnel(vs, precision=P.SF_PREC_FP16TC)
    try:
        holos = holograms(3, shape=(n, n), seed=40)
        ref = per_hologram(sf, holos)
        outs = sf.alloc_batch_outputs(3, field=True, intensity=True)
        sf.execute_batch(holos, outs)
        torch.cuda.synchronize()
        assert P.shifted_fresnel_batch_status(sf.handle, torch.cuda.current_stream().cuda_stream) == P.SF_OK
        check_equal(outs, ref)
    finally:
        sf.close()
