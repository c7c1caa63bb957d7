"""ERIs as a differentiable function of shell centres and primitive exponents.

``eri(centers, exps, basis, quartets)`` returns the FP64 ERIs of the quartets (layout of
``eri_compute``: class-sorted, row major per quartet) through ``EriFunction``, whose backward
calls the adjoint kernel ``eri_backward`` -- the Rys recurrences are recomputed in the
backward pass, nothing but the plan is kept from the forward pass.  Marshalling only.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api
from .workloads import ShellSet


class EriFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, centers, exps, basis: ShellSet, quartets):
        shells = ShellSet(centers.detach().cpu().numpy().astype(np.float64), basis.L, basis.nprim,
                          basis.pofs, exps.detach().cpu().numpy().astype(np.float64), basis.coefs)
        plan = api.eri_plan_create(shells, quartets, precision="fp64", device=torch.cuda.current_device())
        nbytes, _ = api.eri_output_bytes(plan, 0)
        out = torch.empty(nbytes // 8, dtype=torch.float64, device="cuda")
        api.eri_compute(plan, out, torch.cuda.current_stream())
        ctx.plan = plan
        ctx.n_shells = len(basis.L)
        ctx.n_prims = len(basis.exps)
        ctx.devices = (centers.device, exps.device)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        dR = torch.empty((ctx.n_shells, 3), dtype=torch.float64, device="cuda")
        da = torch.empty(ctx.n_prims, dtype=torch.float64, device="cuda")
        api.eri_backward(ctx.plan, grad_out.contiguous().to(torch.float64), dR, da,
                         torch.cuda.current_stream())
        return dR.to(ctx.devices[0]), da.to(ctx.devices[1]), None, None


def eri(centers: torch.Tensor, exps: torch.Tensor, basis: ShellSet, quartets) -> torch.Tensor:
    """Differentiable ERIs; centers [n_shells, 3] and exps [n_prims] are float64 tensors."""
    return EriFunction.apply(centers, exps, basis, quartets)


def quartet_order(basis: ShellSet, quartets) -> np.ndarray:
    """Caller's index of each quartet in the output order (stable sort by class id)."""
    L = np.asarray(basis.L)
    q = np.asarray(quartets)
    cls = ((L[q[:, 0]] * 4 + L[q[:, 1]]) * 4 + L[q[:, 2]]) * 4 + L[q[:, 3]]
    return np.argsort(cls, kind="stable")
