"""Adjoint, z-gradient and autograd of the CUDA path against the FP64 oracle.

* A^H g through shifted_fresnel_adjoint vs the oracle's conjugate transpose
  (relative L2 <= 1e-5), single and multi-view (sum over views), odd sizes,
  z < 0, with and without the prefactor.
* The dot-product identity <A u, g> = <u, A^H g> with both sides on the GPU.
* dL/dz vs Re sum conj(g) du1/dz from the oracle's derivative (1e-3), and
  vs central finite differences of the loss in z (relative step 1e-3 per
  side, plans rebuilt at z +- h).
* torch.autograd gradient of the intensity loss vs finite differences.
* The same object gradient and dL/dz at the full 1024^2, four-depth size
  against the oracle, and its autograd gradients against finite differences.
* 200 iterations of multi-depth phase retrieval on the 1024^2 object, and
  the twin-image test: multi-depth retrieval against single-hologram
  back-propagation on in-line holograms made by the oracle.
"""

import numpy as np
import pytest

import oracle
import synth
from synth import view, random_field, WAVELENGTH, PITCH
from helpers import rel_l2, aligned_rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-5
CPLX = 8
NOPRE = 4


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1001_4309_gb300 import build as b
    b.build()
    import paper_1001_4309_gb300 as P
    return P


def to_dev(a, complex_=True):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.complex64 if complex_ else np.float32))).cuda()


def gpu_adjoint(P, views, gs, holo=None, want_z=False):
    import torch
    sf = P.ShiftedFresnel(views)
    try:
        gz = torch.zeros(len(views), dtype=torch.float64, device="cuda") if want_z else None
        gh, _ = sf.adjoint([to_dev(g) for g in gs], holo=holo, grad_z=gz)
        torch.cuda.synchronize()
        return gh.cpu().numpy(), (gz.cpu().numpy() if want_z else None)
    finally:
        sf.close()


CASES = [
    # (nx0, ny0, nx1, ny1, z, p0, p1, o0, o1, flags)
    (17, 33, 33, 17, 0.03, (PITCH, 3.3e-6), (1.1e-6, 5e-6), (0, 4e-5), (2e-4, -1e-4), CPLX),
    (100, 64, 37, 100, -0.07, PITCH, 0.9e-6, (-2e-5, 1e-5), (5e-4, 3e-4), CPLX | NOPRE),
    (64, 65, 65, 64, 0.04, PITCH, 2.325e-6, (0, 0), (1e-4, -5e-5), 0),
    (256, 256, 256, 256, -0.05, PITCH, 2.325e-6, (0, 0), (100e-6, -50e-6), CPLX),
    # FFT lengths with a factor 3: 1536 along x (1024 -> 400), 2304 along y (1500 -> 700)
    (1024, 24, 400, 20, 0.03, PITCH, 3.1e-6, (0, 0), (1e-4, 1e-4), CPLX),
    (16, 1500, 12, 700, -0.045, PITCH, 2.2e-6, (2e-5, 0), (-1e-4, 3e-4), CPLX | NOPRE),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}-{c[2]}x{c[3]}-f{c[9]}")
def test_adjoint_matches_oracle(P, case):
    nx0, ny0, nx1, ny1, z, p0, p1, o0, o1, flags = case
    v = view(WAVELENGTH, z, p0, p1, o0, o1, (nx0, ny0), (nx1, ny1), flags=flags)
    g = random_field(ny1, nx1, seed=nx1 + 3 * ny1)
    got, _ = gpu_adjoint(P, [v], [g])
    assert rel_l2(got, oracle.adjoint(g, v)) <= TOL


def test_adjoint_sums_over_views(P):
    n0 = (48, 40)
    vs = [view(WAVELENGTH, 0.03, PITCH, 1.5e-6, o1=(1e-4, 0), n0=n0, n1=(30, 50), flags=CPLX),
          view(WAVELENGTH, -0.06, PITCH, 4.65e-6, o1=(-2e-4, 1e-4), n0=n0, n1=(64, 64), flags=CPLX | NOPRE),
          view(WAVELENGTH, 0.10, PITCH, 0.5e-6, n0=n0, n1=(17, 9), flags=CPLX)]
    gs = [random_field(v["ny1"], v["nx1"], seed=10 + i) for i, v in enumerate(vs)]
    got, _ = gpu_adjoint(P, vs, gs)
    ref = sum(oracle.adjoint(g, v) for g, v in zip(gs, vs))
    assert rel_l2(got, ref) <= TOL


def test_dot_product_identity_on_gpu(P):
    import torch
    v = view(WAVELENGTH, 0.05, PITCH, 2.0e-6, o1=(3e-4, -2e-4), n0=(300, 200), n1=(250, 220), flags=CPLX)
    u = random_field(200, 300, seed=1)
    g = random_field(220, 250, seed=2)
    sf = P.ShiftedFresnel([v])
    try:
        Au = sf.reconstruct(to_dev(u))["field"][0].cpu().numpy().astype(np.complex128)
        AHg, _ = sf.adjoint([to_dev(g)])
        AHg = AHg.cpu().numpy().astype(np.complex128)
    finally:
        sf.close()
    lhs, rhs = np.vdot(g, Au), np.vdot(AHg, u)
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def oracle_dldz(u0, g, v):
    return float(np.real(np.vdot(g, oracle.forward_dz(u0, v))))


@pytest.mark.parametrize("flags", [CPLX, CPLX | NOPRE])
def test_grad_z_matches_oracle_derivative(P, flags):
    import torch
    vs = [view(WAVELENGTH, 0.04, PITCH, 1.7e-6, o0=(1e-5, -2e-5), o1=(1e-4, -5e-5), n0=(72, 60), n1=(64, 48),
               flags=flags),
          view(WAVELENGTH, -0.03, PITCH, 3.0e-6, o1=(-3e-4, 2e-4), n0=(72, 60), n1=(40, 70), flags=flags)]
    u0 = random_field(60, 72, seed=5)
    gs = []
    for i, v in enumerate(vs):
        if flags & NOPRE:
            # loss = sum_v || |u1|^2 - I_v ||^2 with arbitrary I: g = 4 (|u1|^2 - I) u1
            u1 = oracle.forward(u0, v)
            I = np.abs(u1) ** 2 * (1 + 0.3 * np.random.default_rng(i).standard_normal(u1.shape))
            g = 4 * (np.abs(u1) ** 2 - I) * u1
        else:
            # with the physical prefactor |C| = 1/(lambda z) the intensity loss leaves float32 range;
            # use a bounded view gradient (a linear loss) instead
            g = random_field(v["ny1"], v["nx1"], seed=20 + i)
        gs.append(g)
    _, gz = gpu_adjoint(P, vs, gs, holo=to_dev(u0), want_z=True)
    for i, v in enumerate(vs):
        ref = oracle_dldz(u0, gs[i], v)
        assert abs(gz[i] - ref) <= 1e-3 * abs(ref), (i, gz[i], ref)


def test_autograd_matches_finite_differences(P):
    import torch
    from paper_1001_4309_gb300.autograd import intensity_loss
    n = 64
    zs = (0.03, 0.05)
    vs = [view(WAVELENGTH, z, PITCH, 1.0e-6 * (1 + i), o1=(2e-5, -1e-5), n0=(n, n), n1=(n, n), flags=CPLX | NOPRE)
          for i, z in enumerate(zs)]
    rng = np.random.default_rng(3)
    u0 = to_dev(np.exp(1j * rng.uniform(-1, 1, (n, n))) * (1 + 0.2 * rng.standard_normal((n, n))))
    sf = P.ShiftedFresnel(vs)
    truth = [o.abs() ** 2 for o in sf.reconstruct(u0 * 0.9 + 0.1)["field"]]
    z = torch.tensor(zs, dtype=torch.float64, device="cuda", requires_grad=True)
    u = u0.clone().requires_grad_(True)
    loss = intensity_loss(u, sf, truth, z)
    loss.backward()
    # direction derivative in u: Re <grad, d>
    d = to_dev(random_field(n, n, seed=9)) * 1e-3
    with torch.no_grad():
        lp = intensity_loss(u0 + d, sf, truth).double()
        lm = intensity_loss(u0 - d, sf, truth).double()
    fd = float((lp - lm) / 2)
    an = float(torch.real(torch.vdot(u.grad.flatten(), d.flatten())))
    assert abs(fd - an) <= 2e-2 * abs(an), (fd, an)
    # z: rebuild plans at z +- h, relative step 1e-3
    for i, z0 in enumerate(zs):
        h = 1e-3 * z0
        vals = []
        for sgn in (1, -1):
            vv = [dict(v) for v in vs]
            vv[i]["z"] = z0 + sgn * h
            sfz = P.ShiftedFresnel(vv)
            with torch.no_grad():
                vals.append(float(intensity_loss(u0, sfz, truth).double()))
            sfz.close()
        fdz = (vals[0] - vals[1]) / (2 * h)
        assert abs(fdz - float(z.grad[i])) <= 2e-2 * abs(fdz), (i, fdz, float(z.grad[i]))
    sf.close()


@pytest.fixture(scope="module")
def c5():
    """The 1024^2 four-depth workload (3, 5, 7, 10 cm at 1 um view pitch): its
    views, intensities of the known object from the FP64 oracle, a trial
    object u (the known one perturbed, rounded to complex64) and the view
    gradients g_v = 4 (|A_v u|^2 - I_v) A_v u of the intensity loss at u,
    also from the oracle."""
    t, vs = synth.config_c5()
    vs = [dict(v, flags=CPLX | NOPRE) for v in vs]
    meas = [np.abs(oracle.forward(t, v)) ** 2 for v in vs]
    rng = np.random.default_rng(55)
    u = (t * (1 + 0.1 * rng.standard_normal(t.shape)) + 0.05 * random_field(*t.shape, seed=56)).astype(np.complex64)
    gs = []
    for v, I in zip(vs, meas):
        u1 = oracle.forward(u, v)
        gs.append(4 * (np.abs(u1) ** 2 - I) * u1)
    return t, vs, meas, u, gs


def test_adjoint_and_grad_z_paper_scale(P, c5):
    """Object gradient sum_v A_v^H g_v and dL/dz of all four depths at the full
    1024^2 size against the FP64 oracle's adjoint and z-derivative."""
    _, vs, _, u, gs = c5
    got, gz = gpu_adjoint(P, vs, gs, holo=to_dev(u), want_z=True)
    ref = sum(oracle.adjoint(g.astype(np.complex64), v) for g, v in zip(gs, vs))
    err = rel_l2(got, ref)
    print(f"object gradient rel-L2 {err:.3e}")
    assert err <= TOL
    for i, v in enumerate(vs):
        r = oracle_dldz(u, gs[i].astype(np.complex64), v)
        print(f"z = {v['z']}: dL/dz {gz[i]:.6e} oracle {r:.6e} rel {abs(gz[i] - r) / abs(r):.2e}")
        assert abs(gz[i] - r) <= 1e-3 * abs(r), (i, gz[i], r)


def test_autograd_paper_scale_vs_finite_differences(P, c5):
    """torch.autograd gradients of the intensity loss at 1024^2 and four depths
    against central finite differences of the GPU loss: a random direction in
    u (step 1e-3 of the object's RMS) and each z (relative steps 1e-3, 5e-4
    and 2.5e-4, Richardson-extrapolated)."""
    import torch
    from paper_1001_4309_gb300.autograd import intensity_loss
    _, vs, meas, u_np, _ = c5
    I = [to_dev(m, complex_=False) for m in meas]
    sf = P.ShiftedFresnel(vs)
    try:
        zs = [v["z"] for v in vs]
        z = torch.tensor(zs, dtype=torch.float64, device="cuda", requires_grad=True)
        u = to_dev(u_np).requires_grad_(True)
        intensity_loss(u, sf, I, z).backward()
        u0 = u.detach()
        d = to_dev(random_field(*u_np.shape, seed=57)) * (1e-3 * float(np.sqrt(np.mean(np.abs(u_np) ** 2))))
        with torch.no_grad():
            lp = float(intensity_loss(u0 + d, sf, I))
            lm = float(intensity_loss(u0 - d, sf, I))
        fd = (lp - lm) / 2
        an = float(torch.real(torch.vdot(u.grad.flatten(), d.flatten())))
        print(f"direction: fd {fd:.6e} autograd {an:.6e}")
        assert abs(fd - an) <= 1e-2 * abs(an), (fd, an)
        # z: at this size a relative step of 1e-3 moves the outermost Fresnel phases by about 1.4 rad, so
        # the plain central difference carries an h^2 truncation error of 10-50 % (FP64 oracle at z = 3 cm:
        # 10.9 %, 2.8 %, 0.7 % at 1e-3, 5e-4, 2.5e-4); two Richardson levels over the three steps cancel
        # the h^2 and h^4 terms
        for i, z0 in enumerate(zs):
            fds = []
            for rel in (1e-3, 5e-4, 2.5e-4):
                h = rel * z0
                vals = []
                for sgn in (1, -1):
                    zz = torch.tensor(zs, dtype=torch.float64)
                    zz[i] = z0 + sgn * h
                    with torch.no_grad():
                        vals.append(float(intensity_loss(u0, sf, I, zz)))
                fds.append((vals[0] - vals[1]) / (2 * h))
            r1 = [(4 * fds[k + 1] - fds[k]) / 3 for k in range(2)]
            fdz = (16 * r1[1] - r1[0]) / 15
            print(f"z = {z0}: fd {fds[0]:.6e} / {fds[1]:.6e} / {fds[2]:.6e} -> {fdz:.6e}, "
                  f"autograd {float(z.grad[i]):.6e}")
            assert abs(fdz - float(z.grad[i])) <= 5e-3 * abs(fdz), (i, fdz, float(z.grad[i]))
    finally:
        sf.close()


def test_phase_retrieval_200_iterations_paper_scale(P):
    """Config-5 geometry: the 1024^2 object seen at four depths (3, 5, 7, 10 cm)
    at 1 um view pitch, intensities of the known object from the FP64 oracle;
    200 Adam iterations from a flat start lower the loss tenfold."""
    import torch
    from paper_1001_4309_gb300.autograd import phase_retrieval
    t, vs = synth.config_c5()
    vs = [dict(v, flags=CPLX | NOPRE) for v in vs]
    meas = [np.abs(oracle.forward(t, v)) ** 2 for v in vs]
    scale = float(np.mean([m.mean() for m in meas]))
    I = [to_dev(m / scale, complex_=False) for m in meas]
    sf = P.ShiftedFresnel(vs)
    try:
        u_init = torch.ones((t.shape[0], t.shape[1]), dtype=torch.complex64, device="cuda") / scale ** 0.5
        u, losses = phase_retrieval(sf, I, n_iter=200, u_init=u_init, lr=0.05 / scale ** 0.5)
        torch.cuda.synchronize()
    finally:
        sf.close()
    assert np.all(np.isfinite(losses))
    assert losses[-1] < 0.1 * losses[0], (losses[0], losses[-1])


def inline_measurements(P):
    """The multi-depth in-line set at 1024^2: views at the hologram pitch, and
    intensities of the known object from the FP64 oracle with photon noise at
    a mean of 2000 photons per pixel, scaled to unit mean."""
    obj, vs = synth.config_c5_inline(1024)
    vs = [dict(v, flags=CPLX | NOPRE) for v in vs]
    meas = [synth.poisson_intensity(np.abs(oracle.forward(obj, v)) ** 2, 2000, seed=40 + k)
            for k, v in enumerate(vs)]
    scale = float(np.mean([m.mean() for m in meas]))
    return obj, vs, [m / scale for m in meas], scale


def test_multi_depth_retrieval_suppresses_twin_image(P):
    """In-line holograms of a known amplitude-and-phase object at 3, 5, 7 and
    10 cm (FP64 oracle, 2000-photon noise).  Back-propagating the 5 cm hologram
    alone (its amplitude, by z = -5 cm) leaves the twin image in the object;
    200 iterations of the multi-depth intensity retrieval from a flat start
    must reach at most half of that object error (both measured after the
    best global complex scale)."""
    import torch
    from paper_1001_4309_gb300.autograd import phase_retrieval
    obj, vs, meas, scale = inline_measurements(P)
    n = obj.shape[0]
    bp_view = dict(vs[1], z=-vs[1]["z"])
    bp_sf = P.ShiftedFresnel([bp_view])
    try:
        bp = bp_sf.reconstruct(to_dev(np.sqrt(meas[1]).astype(np.complex64)))["field"][0].cpu().numpy()
    finally:
        bp_sf.close()
    e_bp = aligned_rel_l2(bp, obj)
    sf = P.ShiftedFresnel(vs)
    try:
        I = [to_dev(m, complex_=False) for m in meas]
        # intensities are scaled to unit mean: start and step at the matching object scale
        u_init = torch.ones((n, n), dtype=torch.complex64, device="cuda") / scale ** 0.5
        u, losses = phase_retrieval(sf, I, n_iter=200, u_init=u_init, lr=0.1 / scale ** 0.5)
        torch.cuda.synchronize()
    finally:
        sf.close()
    e_pr = aligned_rel_l2(u.cpu().numpy(), obj)
    print(f"object error: back-propagation {e_bp:.4f}, retrieval {e_pr:.4f}; loss {losses[0]:.4e} -> {losses[-1]:.4e}")
    assert np.all(np.isfinite(losses))
    assert e_pr <= 0.5 * e_bp, (e_pr, e_bp)


def test_phase_retrieval_recompute_matches_stored_views(P):
    """recompute=True (no view-sized buffers kept between forward and backward)
    follows the same trajectory as keeping the view gradients."""
    import torch
    from paper_1001_4309_gb300.autograd import phase_retrieval
    obj, vs = synth.config_c5_inline(256)
    vs = [dict(v, flags=CPLX | NOPRE) for v in vs]
    meas = [np.abs(oracle.forward(obj, v)) ** 2 for v in vs]
    scale = float(np.mean([m.mean() for m in meas]))
    I = [to_dev(m / scale, complex_=False) for m in meas]
    sf = P.ShiftedFresnel(vs)
    try:
        runs = []
        for recompute in (False, True):
            u_init = torch.ones((256, 256), dtype=torch.complex64, device="cuda") / scale ** 0.5
            u, losses = phase_retrieval(sf, I, n_iter=20, u_init=u_init, lr=0.1 / scale ** 0.5, recompute=recompute)
            runs.append((u.cpu().numpy(), losses))
    finally:
        sf.close()
    (u0, l0), (u1, l1) = runs
    assert np.allclose(l0, l1, rtol=1e-9, atol=0), (l0[-1], l1[-1])
    assert rel_l2(u1, u0) <= 1e-6


def test_backward_uses_the_forward_depths(P):
    """Two losses at different depths through one plan, one backward: each
    gradient is taken at its own forward pass's z (the plan is re-targeted
    back), and a host z tensor receives its gradient on the host."""
    import torch
    from paper_1001_4309_gb300.autograd import intensity_loss
    n = 64
    vs = [view(WAVELENGTH, 0.04, PITCH, 2e-6, n0=(n, n), n1=(n, n), flags=CPLX | NOPRE)]
    u0 = to_dev(random_field(n, n, seed=31))
    sf = P.ShiftedFresnel(vs)
    try:
        meas = [o.abs() ** 2 * 1.1 for o in sf.reconstruct(u0 * 0.8)["field"]]
        za = torch.tensor([0.04], dtype=torch.float64, requires_grad=True)  # host tensors
        zb = torch.tensor([0.05], dtype=torch.float64, requires_grad=True)
        u = u0.clone().requires_grad_(True)
        (intensity_loss(u, sf, meas, za) + intensity_loss(u, sf, meas, zb)).backward()
        assert za.grad.device.type == "cpu" and zb.grad.device.type == "cpu"
        both = (u.grad.clone(), float(za.grad), float(zb.grad))
        ref = []
        for z in (0.04, 0.05):
            zz = torch.tensor([z], dtype=torch.float64, device="cuda", requires_grad=True)
            uu = u0.clone().requires_grad_(True)
            intensity_loss(uu, sf, meas, zz).backward()
            ref.append((uu.grad.clone(), float(zz.grad)))
    finally:
        sf.close()
    assert rel_l2(both[0].cpu().numpy(), (ref[0][0] + ref[1][0]).cpu().numpy()) <= 1e-6
    assert abs(both[1] - ref[0][1]) <= 1e-9 * abs(ref[0][1])
    assert abs(both[2] - ref[1][1]) <= 1e-9 * abs(ref[1][1])


def test_fit_depths_recovers_z(P):
    """z as a trained parameter: the plan follows it (plan update) and Adam on the
    adjoint's dL/dz recovers both views' depths from a 3 % start."""
    import torch
    from paper_1001_4309_gb300.autograd import fit_depths
    n = 128
    rng = np.random.default_rng(1)
    u_np = (synth.gabor.bars_disks_object(n, rng) * np.exp(1j * 0.3)).astype(np.complex64)
    u = to_dev(u_np)
    z_true, pitches = (0.03, 0.045), (PITCH, 2e-6)
    mk = lambda z, p1: view(WAVELENGTH, z, PITCH, p1, n0=(n, n), n1=(n, n), flags=CPLX | NOPRE)  # noqa: E731
    # measured intensities from the FP64 oracle at the true depths
    I = [torch.from_numpy((np.abs(oracle.forward(u_np, mk(z, p))) ** 2).astype(np.float32)).cuda()
         for z, p in zip(z_true, pitches)]
    sf = P.ShiftedFresnel([mk(1.03 * z, p) for z, p in zip(z_true, pitches)])
    try:
        z, losses = fit_depths(sf, u, I, n_iter=100, lr=5e-5)
        assert np.all(np.abs(z.cpu().numpy() - np.array(z_true)) < 3e-5), z
        assert losses[-1] < 1e-3 * losses[0], (losses[0], losses[-1])
        assert [v["z"] for v in sf.views] == [float(a) for a in z.cpu()]  # the plan holds the fitted depths
    finally:
        sf.close()


def test_fused_intensity_loss_matches_composed(P):
    """shifted_fresnel_intensity_loss (one kernel per view) against the same loss
    composed from torch operations on the differentiable views: loss, object
    gradient and dL/dz agree to rounding."""
    import torch
    from paper_1001_4309_gb300.autograd import intensity_loss, views
    n = 96
    vs = [view(WAVELENGTH, z, PITCH, p1, o1=(3e-5, -2e-5), n0=(n, n), n1=(n, 80), flags=CPLX | NOPRE)
          for z, p1 in ((0.02, PITCH), (0.04, 2e-6), (-0.03, 3e-6))]
    rng = np.random.default_rng(8)
    u0 = to_dev(np.exp(1j * rng.uniform(-1, 1, (n, n))) * (1 + 0.2 * rng.standard_normal((n, n))))
    sf = P.ShiftedFresnel(vs)
    try:
        meas = [o.abs() ** 2 * 0.9 for o in sf.reconstruct(u0 * 1.1)["field"]]
        zs = [v["z"] for v in vs]
        res = []
        for fused in (True, False):
            u = u0.clone().requires_grad_(True)
            z = torch.tensor(zs, dtype=torch.float64, device="cuda", requires_grad=True)
            if fused:
                loss = intensity_loss(u, sf, meas, z)
            else:
                loss = sum(((o.real ** 2 + o.imag ** 2 - I).double() ** 2).sum()
                           for o, I in zip(views(u, sf, z), meas))
            (2.0 * loss).backward()  # a non-unit incoming gradient
            res.append((float(loss.detach()), u.grad.cpu().numpy(), z.grad.cpu().numpy()))
        (lf, gf, zf), (lc, gc, zc) = res
        assert abs(lf - lc) <= 1e-5 * abs(lc), (lf, lc)
        assert rel_l2(gf, gc) <= 1e-5
        assert np.allclose(zf, zc, rtol=1e-4, atol=0), (zf, zc)
        # the loss alone (no gradients requested)
        with torch.no_grad():
            assert abs(float(intensity_loss(u0, sf, meas)) - lc) <= 1e-5 * abs(lc)
    finally:
        sf.close()
