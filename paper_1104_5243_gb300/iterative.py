"""Iterative reconstruction with the two kernels of the library.

The paper notes (Sect. 1.1) that iterative methods for sparse or irregular
data repeat the backprojection many times; here the voxel-driven operators of
the library form the pair such a method needs:

* forward model  P f = c * B^T f   (bp_adjoint: every voxel spread onto the
  detector with the bilinear weights and 1/w^2; with c = R^3 / tau^2 it
  approximates the line integrals, R the voxel size and tau the detector
  pitch at the isocenter: a voxel of volume R^3 covers about tau^2 w^2 of a
  pixel's beam at relative depth w);
* its transpose  P^T q = c * B q   (bp_add_projections).

``cgls`` runs conjugate gradients on the normal equations P^T P f = P^T p
(CGLS), whose iterates from f = 0 converge to the minimum-norm least-squares
solution.  Vector updates (axpy) and the recurrence's scalars (squared
2-norms, from torch's float32 norm reduction: about 1e-7 relative, and a
tenth of the time of a float64 copy-and-sum on these sizes) are torch
operations on the GPU; every application of P and P^T runs in the
library's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import api


def model_scale(vol_R: float, tau: float) -> float:
    """c = R^3 / tau^2 (see the module docstring)."""
    return vol_R ** 3 / tau ** 2


class Operators:
    """P and P^T for one geometry, on one library context."""

    def __init__(self, bp: api.Backprojector, A, scale: float = 1.0):
        self.bp, self.A, self.scale = bp, np.ascontiguousarray(A, dtype=np.float64), float(scale)

    def forward(self, f: torch.Tensor) -> torch.Tensor:
        return self.bp.adjoint(f, self.A).mul_(self.scale)

    def transpose(self, q: torch.Tensor) -> torch.Tensor:
        self.bp.reset()
        self.bp.add_projections(q.contiguous(), self.A)
        return self.bp.finalize().mul_(self.scale)


def _sq_norm(x: torch.Tensor) -> float:
    """||x||_2^2 from the float32 norm reduction, squared in float64."""
    return float(torch.linalg.vector_norm(x)) ** 2


@torch.no_grad()
def cgls(ops: Operators, p: torch.Tensor, iters: int, f0: torch.Tensor | None = None, callback=None):
    """CGLS for min ||P f - p||_2.  Returns (f, residual norms per iteration)."""
    f = torch.zeros((ops.bp.L,) * 3, dtype=torch.float32, device=p.device) if f0 is None else f0.clone()
    r = p - ops.forward(f) if f0 is not None else p.clone()
    s = ops.transpose(r)
    d = s.clone()
    gamma = _sq_norm(s)
    norms = [float(torch.linalg.vector_norm(r))]
    for k in range(iters):
        q = ops.forward(d)
        qq = _sq_norm(q)
        if qq == 0.0 or gamma == 0.0:
            break
        alpha = gamma / qq
        f.add_(d, alpha=alpha)
        r.sub_(q, alpha=alpha)
        s = ops.transpose(r)
        gamma_new = _sq_norm(s)
        d.mul_(gamma_new / gamma).add_(s)
        gamma = gamma_new
        norms.append(float(torch.linalg.vector_norm(r)))
        if callback is not None:
            callback(k, f, norms[-1])
    return f, norms
