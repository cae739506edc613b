"""torch.autograd face of the library's discrete adjoint (kbc_adjoint).

``kbc_objective(u0, beta, ...)`` returns J (a 0-d float64 tensor) of the
field obtained by initialising at f^eq(rho0, u0) and advancing ``steps``
stream-collide steps; its backward hands PyTorch dJ/du0 and dJ/dbeta, which
the CUDA adjoint computed in the same call (one forward sweep with
checkpoints every ``ckpt_every`` steps, one reverse sweep with recompute).
"""
from __future__ import annotations

import torch

from . import DTYPES, VARIANTS, Lattice, capi

OBJECTIVES = {"ke": 0, "kinetic_energy": 0, "misfit": 1, "l2": 1}


class KBCObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, beta, rho0, variant, dtype, steps, ckpt_every, objective, u_target,
                gamma_fixed):
        ny, nx = u0.shape[-2:]
        lat = Lattice(nx, ny, variant=variant, beta=float(beta), dtype=dtype)
        if gamma_fixed is not None:
            lat.set_gamma(gamma_fixed)
        u = u0.detach().to(torch.float64).contiguous()
        r = rho0.detach().to(torch.float64).contiguous()
        tgt = None if u_target is None else u_target.detach().to(torch.float64).contiguous()
        grad = torch.empty_like(u)
        J, gb = capi.kbc_adjoint(lat.h, r, u, steps, ckpt_every, objective, tgt, grad)
        lat.close()
        ctx.save_for_backward(grad.to(u0.dtype), torch.tensor(gb, dtype=torch.float64))
        ctx.beta_like = beta
        return torch.tensor(J, dtype=torch.float64, device=u0.device)

    @staticmethod
    def backward(ctx, gJ):
        grad, gb = ctx.saved_tensors
        gbeta = None
        if torch.is_tensor(ctx.beta_like):
            gbeta = (gJ.to(gb.device) * gb).to(ctx.beta_like.dtype).to(ctx.beta_like.device)
        return gJ * grad, gbeta, None, None, None, None, None, None, None, None


def kbc_objective(u0, beta, rho0=None, variant="B", dtype="f64", steps=100, ckpt_every=100,
                  objective="ke", u_target=None, gamma_fixed=None):
    """J(u0, beta) with gradients through the hand-written CUDA adjoint.

    u0: [2][ny][nx] CUDA tensor (u_x, u_y); beta: float or 0-d tensor
    (requires_grad for dJ/dbeta); rho0 defaults to 1 everywhere; objective
    "ke" (sum rho |u|^2 / 2) or "misfit" (sum |u - u_target|^2 / 2).
    """
    if rho0 is None:
        rho0 = torch.ones(u0.shape[-2:], dtype=torch.float64, device=u0.device)
    obj = OBJECTIVES[objective] if isinstance(objective, str) else int(objective)
    if obj == 1 and u_target is None:
        raise ValueError("the misfit objective needs u_target")
    v = VARIANTS[variant] if isinstance(variant, str) else int(variant)
    d = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    return KBCObjective.apply(u0, beta, rho0, v, d, int(steps), int(ckpt_every), obj, u_target,
                              gamma_fixed)
