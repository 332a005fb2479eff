"""Differentiable Shifted-Fresnel views and gradient-descent phase retrieval.

``ShiftedFresnelFunction`` wraps a plan as a ``torch.autograd.Function``:
the forward pass is ``shifted_fresnel_execute`` and the backward pass is
``shifted_fresnel_adjoint``, which returns the gradient with respect to the
complex object field (sum over views of A_v^H g_v) and, when asked, with
respect to each view's z.  The z values are part of the plan (the chirps and
kernel spectra depend on them): a ``z`` tensor that differs from the plan's
depths re-targets the plan first (``shifted_fresnel_plan_update``), so z can
be a trained parameter.

``phase_retrieval`` fits a complex object to measured view intensities
(twin-image-free in-line holography from several depths) by minimising
sum_v || |A_v u|^2 - I_v ||^2 with Adam; ``fit_depths`` fits the views' z to
measured intensities of a known object with the same loss.
"""

from __future__ import annotations

import torch

from .binding import ShiftedFresnel, shifted_fresnel_adjoint, shifted_fresnel_intensity_loss, SF_IN_COMPLEX


def _follow_z(sf, z):
    """Re-target the plan when the z tensor differs from its depths."""
    if z is None:
        return
    zv = [float(a) for a in z.detach().cpu()]
    if len(zv) != len(sf.views):
        raise ValueError("z must hold one distance per view")
    if any(a != v["z"] for a, v in zip(zv, sf.views)):
        sf.update([dict(v, z=a) for v, a in zip(sf.views, zv)])


def _save_plan_state(ctx, sf, z):
    """Record the views the forward pass ran with, and z's device and dtype."""
    ctx.sf = sf
    ctx.views = [dict(v) for v in sf.views]
    ctx.z_meta = (z.device, z.dtype) if isinstance(z, torch.Tensor) else None


def _restore_plan_state(ctx):
    """Put the plan back on the forward pass's views when another forward
    re-targeted it in between (two losses at different z before one backward):
    the adjoint and dL/dz must use the depths the views were computed at."""
    sf = ctx.sf
    if sf.views != ctx.views:
        sf.update([dict(v) for v in ctx.views])
    return sf


def _grad_z_out(ctx, grad_z):
    """dL/dz on z's own device and dtype (z may live on the host)."""
    if grad_z is None or ctx.z_meta is None:
        return grad_z
    device, dtype = ctx.z_meta
    return grad_z.to(device=device, dtype=dtype)


class ShiftedFresnelFunction(torch.autograd.Function):
    """views = ShiftedFresnelFunction.apply(u0, z, sf) -> tuple of complex64 view fields."""

    @staticmethod
    def forward(ctx, u0, z, sf):
        if not (sf.views[0].get("flags", 0) & SF_IN_COMPLEX):
            raise ValueError("the plan must take a complex object (SF_IN_COMPLEX)")
        _follow_z(sf, z)
        u0c = u0.contiguous()
        outs = sf.reconstruct(u0c, field=True)
        _save_plan_state(ctx, sf, z)
        ctx.save_for_backward(u0c)
        return tuple(outs["field"])

    @staticmethod
    def backward(ctx, *grads):
        (u0,) = ctx.saved_tensors
        need_u, need_z = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_u or need_z):
            return None, None, None
        sf = _restore_plan_state(ctx)
        gs = [g.contiguous() if g is not None else None for g in grads]
        grad_u = torch.empty_like(u0) if need_u else None
        grad_z = torch.zeros(len(sf.views), dtype=torch.float64, device=u0.device) if need_z else None
        shifted_fresnel_adjoint(sf.handle, u0.data_ptr() if need_z else None,
                                [g.data_ptr() if g is not None else None for g in gs],
                                grad_u.data_ptr() if need_u else None,
                                grad_z.data_ptr() if need_z else None,
                                stream=torch.cuda.current_stream(u0.device).cuda_stream)
        return grad_u, _grad_z_out(ctx, grad_z), None


def views(u0, sf, z=None):
    """Differentiable views of a complex object field through plan ``sf``."""
    return ShiftedFresnelFunction.apply(u0, z, sf)


class IntensityLossFunction(torch.autograd.Function):
    """loss = IntensityLossFunction.apply(u0, z, sf, intensities, recompute): the fused multi-depth intensity loss.

    Forward: execute, then shifted_fresnel_intensity_loss (loss in double
    precision and the view gradients 4 (|u|^2 - I) u in one kernel per view).
    Backward: shifted_fresnel_adjoint of those view gradients (and dL/dz when
    z requires it), scaled by the incoming gradient.  With ``recompute`` the
    forward pass keeps nothing of view size (it computes the loss alone) and
    the backward pass recomputes the view fields and their gradients first:
    one more execute per step for V fewer view-sized buffers held between the
    passes.
    """

    @staticmethod
    def forward(ctx, u0, z, sf, intensities, recompute=False):
        if not (sf.views[0].get("flags", 0) & SF_IN_COMPLEX):
            raise ValueError("the plan must take a complex object (SF_IN_COMPLEX)")
        _follow_z(sf, z)
        u0c = u0.contiguous()
        meas = [I.contiguous() for I in intensities]
        need = (ctx.needs_input_grad[0] or ctx.needs_input_grad[1]) and not recompute
        grads, loss = _loss_and_view_grads(sf, u0c, meas, need)
        _save_plan_state(ctx, sf, z)
        ctx.grads = grads
        ctx.meas = meas if recompute else None
        ctx.save_for_backward(u0c)
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        (u0,) = ctx.saved_tensors
        need_u, need_z = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        if not (need_u or need_z):
            return None, None, None, None, None
        sf = _restore_plan_state(ctx)
        grads = ctx.grads
        if grads is None:  # recompute: the views and their gradients at the forward pass's depths
            grads, _ = _loss_and_view_grads(sf, u0, ctx.meas, True)
        grad_u = torch.empty_like(u0) if need_u else None
        grad_z = torch.zeros(len(sf.views), dtype=torch.float64, device=u0.device) if need_z else None
        shifted_fresnel_adjoint(sf.handle, u0.data_ptr() if need_z else None, [g.data_ptr() for g in grads],
                                grad_u.data_ptr() if need_u else None, grad_z.data_ptr() if need_z else None,
                                stream=torch.cuda.current_stream(u0.device).cuda_stream)
        ctx.grads = None
        if need_u:
            grad_u.mul_(grad_loss.to(grad_u.real.dtype))
        if need_z:
            grad_z.mul_(grad_loss.to(grad_z.device))
        return grad_u, _grad_z_out(ctx, grad_z), None, None, None


def _loss_and_view_grads(sf, u0, meas, want_grads):
    """Execute the plan on u0, then the fused loss kernel: (view gradients or None, float64 loss)."""
    fields = sf.reconstruct(u0, field=True)["field"]
    grads = [torch.empty_like(f) for f in fields] if want_grads else None
    loss = torch.empty((), dtype=torch.float64, device=u0.device)
    shifted_fresnel_intensity_loss(sf.handle, [f.data_ptr() for f in fields], [I.data_ptr() for I in meas],
                                   [g.data_ptr() for g in grads] if grads else None, loss.data_ptr(),
                                   stream=torch.cuda.current_stream(u0.device).cuda_stream)
    return grads, loss


def intensity_loss(u0, sf, intensities, z=None, recompute=False):
    """sum_v || |A_v u0|^2 - I_v ||^2 (the loss of the multi-depth phase retrieval), float64 scalar.

    ``recompute=True`` holds no view-sized buffer between forward and backward
    (the backward pass recomputes the views)."""
    return IntensityLossFunction.apply(u0, z, sf, intensities, recompute)


def phase_retrieval(sf, intensities, n_iter=200, u_init=None, lr=0.05, recompute=False, callback=None):
    """Fit a complex object to measured view intensities by gradient descent (Adam).

    ``recompute=True`` keeps no view fields or view gradients between
    forward and backward (the backward pass recomputes them: one more execute
    per iteration), for view sets whose buffers do not fit beside the object.
    Returns (u, losses).
    """
    v0 = sf.views[0]
    if u_init is None:
        u_init = torch.ones((v0["ny0"], v0["nx0"]), dtype=torch.complex64, device=sf.device)
    u = u_init.detach().clone().requires_grad_(True)
    opt = torch.optim.Adam([u], lr=lr)
    losses = []
    for it in range(n_iter):
        opt.zero_grad(set_to_none=True)
        loss = intensity_loss(u, sf, intensities, recompute=recompute)
        loss.backward()
        opt.step()
        losses.append(loss.detach())
        if callback is not None:
            callback(it, u, loss)
    return u.detach(), [float(x) for x in torch.stack(losses).cpu()]


def fit_depths(sf, u0, intensities, n_iter=100, lr=5e-5):
    """Fit each view's z to measured intensities of a known object u0 (Adam on dL/dz).

    The plan follows z through every step and holds the fitted depths on
    return.  Returns (z, losses).
    """
    z = torch.tensor([v["z"] for v in sf.views], dtype=torch.float64, device=u0.device, requires_grad=True)
    opt = torch.optim.Adam([z], lr=lr)
    u = u0.detach()
    losses = []
    for _ in range(n_iter):
        opt.zero_grad(set_to_none=True)
        loss = intensity_loss(u, sf, intensities, z=z)
        loss.backward()
        opt.step()
        losses.append(loss.detach())
    sf.update([dict(v, z=float(a)) for v, a in zip(sf.views, z.detach().cpu())])
    return z.detach(), [float(x) for x in torch.stack(losses).cpu()]


__all__ = ["ShiftedFresnelFunction", "IntensityLossFunction", "views", "intensity_loss", "phase_retrieval",
           "fit_depths", "ShiftedFresnel"]
