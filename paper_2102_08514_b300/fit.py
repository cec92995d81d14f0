"""Fit lattice coefficients to samples of a signal by gradient descent through the adjoint.

loss(c) = mean_q (f_c(x_q) - y_q)^2 with f_c(x) = sum_n c_n phi(x - n); the forward pass is
interp_eval and the gradient dloss/dc is the hand-written adjoint interp_backward (through the
``lattice_interp`` autograd function).  The loss is reduced in FP64; the optimiser is Adam.  Not
in the paper (which prefilters instead, Sec. 2); it exercises the adjoint end to end.
"""
from __future__ import annotations

from .binding import Interpolator, lattice_interp


def mse_loss(f, y):
    """Mean squared error reduced in FP64."""
    d = f.double() - y.double()
    return (d * d).mean()


def fit(interp: Interpolator, pts, targets, steps: int = 200, lr: float = 0.05, betas=(0.9, 0.999),
        eps: float = 1e-8, coeffs=None, record_every: int = 1, sort: bool = True):
    """Adam on the coefficients (start: zeros, or `coeffs`).  Returns (coefficients, losses).

    With sort=True the samples are reordered once by interp_sort_points (the loss does not
    depend on their order); every evaluation and adjoint then runs on spatially sorted queries."""
    import torch
    if sort:
        perm, pts = interp.sort_points(pts)
        targets = targets[perm.long()]
    c = (torch.zeros(interp.shape, device=pts.device, dtype=torch.float32) if coeffs is None
         else coeffs.detach().clone().float()).requires_grad_(True)
    opt = torch.optim.Adam([c], lr=lr, betas=betas, eps=eps)
    losses = []
    for it in range(steps):
        opt.zero_grad(set_to_none=False)
        loss = mse_loss(lattice_interp(pts, c, interp), targets)
        loss.backward()
        opt.step()
        if record_every and it % record_every == 0:
            losses.append(float(loss.detach()))
    return c.detach(), losses
