"""The Landau-Brazovskii energy as a differentiable torch function.

E(phi, tau, gamma, box) is the energy of the paper's §2 (eq. interaction_bulk_energy) on a
zero-mean field given by its grid values; its derivatives come from one call of the C
entry point lb_energy_derivs:
  dE/dphi   = g / N  (g the gradient in the <.,.>_N metric; the derivative with respect to
              the grid values, restricted to zero-mean fields),
  dE/dtau   = <phi^2 / 2>_N,   dE/dgamma = -<phi^3 / 6>_N,
  dE/dL_a   = sum_k 1/2 |phi_hat_k|^2 4 xi^2 (1 - |Bk|^2) (Bk)_a^2 / L_a  at fixed grid values.
The box is given per array axis (the order of phi.shape).  Contexts are cached per
(shape, box, precision, xi); every call with a new box creates one.
"""
from __future__ import annotations

from collections import OrderedDict

import torch

from . import lbtr

_CACHE: "OrderedDict[tuple, lbtr.Context]" = OrderedDict()
_CACHE_SIZE = 4


def _context(shape, box, precision, xi, tau, gamma) -> lbtr.Context:
    key = (tuple(shape), tuple(box), precision, xi)
    c = _CACHE.pop(key, None)
    if c is None:
        c = lbtr.lb_create_from_array_box(shape, box, xi, tau, gamma, precision)
    _CACHE[key] = c
    while len(_CACHE) > _CACHE_SIZE:
        _CACHE.popitem(last=False)
    lbtr.lb_set_params(c, xi, tau, gamma)
    return c


class LBEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, tau, gamma, box, xi, precision):
        boxl = [float(b) for b in box.detach().cpu().tolist()]
        c = _context(tuple(phi.shape), boxl, precision, float(xi), float(tau), float(gamma))
        field = phi.detach().to(c.dtype).contiguous()
        grad = torch.empty_like(field)
        d = lbtr.lb_energy_derivs(c, field, grad)
        ctx.save_for_backward(grad)
        ctx.n = field.numel()
        ctx.dtau, ctx.dgamma = d["dtau"], d["dgamma"]
        ctx.dbox = list(reversed(d["dL_xyz"]))          # array-axis order
        ctx.phi_dtype = phi.dtype
        return torch.tensor(d["energy"], dtype=torch.float64, device=phi.device)

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        g = float(gout)
        dphi = (grad * (g / ctx.n)).to(ctx.phi_dtype)
        dev = grad.device
        dtau = torch.tensor(g * ctx.dtau, dtype=torch.float64, device=dev)
        dgamma = torch.tensor(g * ctx.dgamma, dtype=torch.float64, device=dev)
        dbox = torch.tensor([g * x for x in ctx.dbox], dtype=torch.float64, device=dev)
        return dphi, dtau, dgamma, dbox, None, None


def lb_energy(phi, tau, gamma, box, xi: float = 1.0, precision: int = lbtr.LB_FP64):
    """E(phi, tau, gamma, box) as a 0-d float64 tensor, differentiable in all four.

    phi: zero-mean device field (float64 for LB_FP64, float32 for LB_MIXED), shape
    [y][x] or [z][y][x] with equal sides; tau, gamma: floats or 0-d tensors; box: box
    lengths per array axis (sequence or 1-d tensor).
    """
    dev = phi.device
    as_t = lambda v: v if torch.is_tensor(v) else torch.tensor(float(v), dtype=torch.float64, device=dev)
    box_t = box if torch.is_tensor(box) else torch.tensor([float(b) for b in box], dtype=torch.float64, device=dev)
    return LBEnergy.apply(phi, as_t(tau), as_t(gamma), box_t, xi, precision)
