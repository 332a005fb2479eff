"""shifted_fresnel_plan_update: a plan re-targeted to new depths, pitches,
offsets, wavelength or prefactor flag (same sizes) computes exactly what a new
plan with those views computes -- forward, adjoint, tensor-core plans and the
batch -- and rejects views of other sizes without touching the plan.
"""

import numpy as np
import pytest

import oracle
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


N0 = (600, 512)


def views_a(flags=0):
    return [view(WAVELENGTH, 0.05, PITCH, 2e-6, o1=(1e-4, -2e-4), n0=N0, n1=(512, 512), flags=flags),
            view(WAVELENGTH, 0.08, PITCH, PITCH, n0=N0, n1=(900, 300), flags=flags),
            view(WAVELENGTH, -0.03, PITCH, 7e-6, o1=(-3e-4, 0.0), n0=N0, n1=(33, 17), flags=flags)]


def views_b(P, flags=0):
    return [view(532e-9, 0.11, PITCH, 1e-6, o1=(-5e-4, 3e-4), n0=N0, n1=(512, 512), flags=flags),
            view(532e-9, -0.06, PITCH, 3e-6, o1=(2e-4, 1e-4), n0=N0, n1=(900, 300),
                 flags=flags | P.SF_NO_PREFACTOR),
            view(532e-9, 0.02, PITCH, 0.5e-6, o1=(0.0, -1e-4), n0=N0, n1=(33, 17), flags=flags)]


def run_all(sf, h):
    import torch
    o = sf.reconstruct(h, field=True, intensity=True, phase=True)
    torch.cuda.synchronize()
    return [[t.cpu().numpy() for t in o[k]] for k in ("field", "intensity", "phase")]


def same(a, b):
    for x, y in zip(a, b):
        for u, v in zip(x, y):
            assert np.array_equal(u, v)


def test_update_equals_new_plan_and_back(P):
    import torch
    h = torch.from_numpy(random_field(N0[1], N0[0], seed=3).real.astype(np.float32)).cuda()
    va, vb = views_a(), views_b(P)
    fresh_a, fresh_b = P.ShiftedFresnel(va), P.ShiftedFresnel(vb)
    sf = P.ShiftedFresnel(va)
    try:
        ref_a, ref_b = run_all(fresh_a, h), run_all(fresh_b, h)
        assert [sf.sizes(i)[:2] for i in range(3)] == [fresh_b.sizes(i)[:2] for i in range(3)]
        sf.update(vb)
        got = run_all(sf, h)
        same(got, ref_b)
        # and against the oracle on a sampled block of each view
        h_np = h.cpu().numpy()
        for i, v in enumerate(vb):
            cols = (0, min(4, v["nx1"]))
            assert rel_l2(got[0][i][:, cols[0]:cols[1]], oracle.forward(h_np, v, cols=cols)) <= 1e-5
        sf.update(va)
        same(run_all(sf, h), ref_a)
    finally:
        for x in (fresh_a, fresh_b, sf):
            x.close()


def test_update_rejects_other_sizes(P):
    import torch
    h = torch.from_numpy(random_field(N0[1], N0[0], seed=4).real.astype(np.float32)).cuda()
    va = views_a()
    sf = P.ShiftedFresnel(va)
    try:
        ref = run_all(sf, h)
        bad_size = [dict(v) for v in va]
        bad_size[1]["nx1"] = 901
        bad_cplx = views_a(flags=P.SF_IN_COMPLEX)
        for bad in (bad_size, bad_cplx, va[:2]):
            assert P.shifted_fresnel_plan_update(sf.handle, bad, check=False) == P.SF_ERR_INVALID_ARG
        bad_z = [dict(v) for v in va]
        bad_z[0]["z"] = 0.0
        assert P.shifted_fresnel_plan_update(sf.handle, bad_z, check=False) == P.SF_ERR_INVALID_ARG
        same(run_all(sf, h), ref)  # the plan is untouched
    finally:
        sf.close()


def test_update_adjoint_and_z_gradient(P):
    import torch
    u = torch.from_numpy(random_field(N0[1], N0[0], seed=5).astype(np.complex64)).cuda()
    vb = views_b(P, flags=P.SF_IN_COMPLEX)
    fresh = P.ShiftedFresnel(vb)
    sf = P.ShiftedFresnel(views_a(flags=P.SF_IN_COMPLEX))
    try:
        sf.update(vb)
        g = [torch.from_numpy(random_field(v["ny1"], v["nx1"], seed=10 + i).astype(np.complex64)).cuda()
             for i, v in enumerate(vb)]
        res = []
        for p in (fresh, sf):
            gh = torch.empty_like(u)
            gz = torch.zeros(len(vb), dtype=torch.float64, device="cuda")
            p.adjoint(g, holo=u, grad_holo=gh, grad_z=gz)
            torch.cuda.synchronize()
            res.append((gh.cpu().numpy(), gz.cpu().numpy()))
        assert np.array_equal(res[0][0], res[1][0])
        assert np.array_equal(res[0][1], res[1][1])
    finally:
        fresh.close()
        sf.close()


@pytest.mark.parametrize("impl", ["persistent", "streams"])
def test_update_then_batch(P, impl, monkeypatch):
    import torch
    monkeypatch.setenv("SF_BATCH_IMPL", impl)
    va, vb = views_a(), views_b(P)
    holos = [torch.from_numpy(random_field(N0[1], N0[0], seed=20 + k).real.astype(np.float32)).cuda()
             for k in range(3)]
    fresh = P.ShiftedFresnel(vb)
    sf = P.ShiftedFresnel(va)
    try:
        outs = sf.alloc_batch_outputs(3, field=True)
        sf.execute_batch(holos, outs)  # builds the batch state (and graph) for the old views
        sf.update(vb)
        sf.execute_batch(holos, outs)  # same buffers: the streams graph is replayed
        torch.cuda.synchronize()
        for k, h in enumerate(holos):
            ref = fresh.reconstruct(h, field=True)["field"]
            torch.cuda.synchronize()
            for i in range(len(vb)):
                assert torch.equal(outs["field"][k][i], ref[i]), (k, i)
    finally:
        fresh.close()
        sf.close()


@pytest.mark.parametrize("n,prec", [(1024, 1), (512, 1), (1024, 3)], ids=["2048-fp16", "1024-fp16", "2048-fp16x3"])
def test_update_tensor_core_plan(P, n, prec):
    """Tensor-core plans at both tcgen05 lengths (fused launch for FP16, one launch per pass for FP16X3):
    the natural-order kernel spectra are rebuilt with the new views."""
    import torch
    mk = lambda z, p1, o: view(WAVELENGTH, z, PITCH, p1, o1=o, n0=(n, n), n1=(n, n))  # noqa: E731
    va = [mk(0.03, 4.65e-6, (0.0, 0.0)), mk(0.05, 2e-6, (1e-4, 0.0))]
    vb = [mk(0.07, 1e-6, (-2e-4, 1e-4)), mk(0.1, 0.5e-6, (3e-4, -3e-4))]
    h = torch.from_numpy(random_field(n, n, seed=6).real.astype(np.float32)).cuda()
    fresh = P.ShiftedFresnel(vb, precision=prec)
    sf = P.ShiftedFresnel(va, precision=prec)
    try:
        sf.update(vb)
        a = fresh.reconstruct(h, field=True)["field"]
        b = sf.reconstruct(h, field=True)["field"]
        torch.cuda.synchronize()
        for x, y in zip(a, b):
            assert torch.equal(x, y)
    finally:
        fresh.close()
        sf.close()
