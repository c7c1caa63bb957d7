"""ERIs as a differentiable function of shell centres and primitive exponents.

``EriGeometry(basis, quartets)`` builds one plan for a fixed basis layout (L and primitive count
of every shell) and quartet list; each call ``g(centers, exps)`` moves the plan's shells to the
given geometry (``eri_plan_update_shells``: host-to-device copies of the shell data and, where
the plan has one, a rebuild of the primitive-pair table -- no new plan, sort or allocation) and
returns the FP64 ERIs through ``EriFunction``, whose backward calls the adjoint kernel
``eri_backward``.  The Rys recurrences are recomputed in the backward pass; nothing but the
geometry of the forward pass is kept.  Outputs are in the plan's order (``eri_compute``:
class-sorted, row major per quartet); ``order()`` gives the caller's index of every quartet.
``eri(centers, exps, basis, quartets)`` is the one-shot form (a plan per call).  Marshalling
only.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api
from .workloads import ShellSet


class EriGeometry:
    """One plan re-used across geometries (a molecular-dynamics or optimisation loop)."""

    def __init__(self, basis: ShellSet, quartets, precision: str = "fp64", device: int | None = None):
        self.basis = basis
        self.device = torch.cuda.current_device() if device is None else device
        self.plan = api.eri_plan_create(basis, quartets, precision=precision, device=self.device)
        nbytes, _ = api.eri_output_bytes(self.plan, 0)
        self.n_out = nbytes // 8
        self._geometry = None  # (centres, exponents) the plan's shells hold now

    def shells(self, centers: np.ndarray, exps: np.ndarray) -> ShellSet:
        b = self.basis
        return ShellSet(centers, b.L, b.nprim, b.pofs, exps, b.coefs)

    def move_to(self, centers: np.ndarray, exps: np.ndarray, stream=None) -> None:
        """Puts the plan's shells at this geometry (skipped when they are there already)."""
        g = self._geometry
        if g is not None and np.array_equal(g[0], centers) and np.array_equal(g[1], exps):
            return
        api.eri_plan_update_shells(self.plan, self.shells(centers, exps), stream)
        self._geometry = (centers.copy(), exps.copy())

    def order(self) -> np.ndarray:
        """Caller's index of each quartet in the output order."""
        return api.eri_plan_quartet_order(self.plan)

    def __call__(self, centers: torch.Tensor, exps: torch.Tensor) -> torch.Tensor:
        return EriFunction.apply(centers, exps, self)

    def destroy(self) -> None:
        if self.plan is not None:
            self.plan.destroy()
            self.plan = None


class EriFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, centers, exps, geo: EriGeometry):
        c = centers.detach().cpu().numpy().astype(np.float64)
        e = exps.detach().cpu().numpy().astype(np.float64)
        stream = torch.cuda.current_stream()
        geo.move_to(c, e, stream)
        out = torch.empty(geo.n_out, dtype=torch.float64, device=torch.device("cuda", geo.device))
        api.eri_compute(geo.plan, out, stream)
        ctx.geo = geo
        ctx.geometry = (c, e)
        ctx.devices = (centers.device, exps.device)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        geo = ctx.geo
        stream = torch.cuda.current_stream()
        # another forward call may have moved the shared plan since: put back this call's geometry
        geo.move_to(*ctx.geometry, stream)
        dev = torch.device("cuda", geo.device)
        dR = torch.empty((len(geo.basis.L), 3), dtype=torch.float64, device=dev)
        da = torch.empty(len(geo.basis.exps), dtype=torch.float64, device=dev)
        api.eri_backward(geo.plan, grad_out.contiguous().to(torch.float64), dR, da, stream)
        return dR.to(ctx.devices[0]), da.to(ctx.devices[1]), None


def eri(centers: torch.Tensor, exps: torch.Tensor, basis: ShellSet, quartets) -> torch.Tensor:
    """Differentiable ERIs; centers [n_shells, 3] and exps [n_prims] are float64 tensors.  Builds
    a plan per call (use EriGeometry to keep one across geometries)."""
    return EriGeometry(basis, quartets)(centers, exps)


def quartet_order(basis: ShellSet, quartets) -> np.ndarray:
    """Caller's index of each quartet in the output order (stable sort by class id; classes with
    a g shell have ids 256 + base-5 index, after the 256 classes of s..f shells)."""
    L = np.asarray(basis.L)
    q = np.asarray(quartets)
    La, Lb, Lc, Ld = (L[q[:, k]] for k in range(4))
    g = np.maximum(np.maximum(La, Lb), np.maximum(Lc, Ld)) > 3
    cls = np.where(g, 256 + ((La * 5 + Lb) * 5 + Lc) * 5 + Ld, ((La * 4 + Lb) * 4 + Lc) * 4 + Ld)
    return np.argsort(cls, kind="stable")
