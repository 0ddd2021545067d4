"""The level M2L translation as a differentiable PyTorch operation.

Forward: locals = M2L(multipoles) for one octree level (Eq. (7), through
m2l_plan_apply).  Backward: the adjoint translation, grad_multipoles =
M2L^T(grad_locals), which the library runs as the forward translation on the
transposed interaction list (K_{-t} = K_t^T, Sec. 3.1).  Both directions use
plans built once per level, so repeated steps skip the classification.

The map is linear in the multipoles; the operators (kernel, order, level
geometry) are constants, so only the multipoles receive a gradient.
"""
from __future__ import annotations

import torch

from . import m2l


class M2LLevelOperator:
    """One level's M2L translation with cached forward and adjoint plans."""

    def __init__(self, ops: m2l.Ops, level: m2l.Level, precision: str = "fp32"):
        self.ops, self.level, self.precision = ops, level, precision
        self.fwd = m2l.m2l_plan_create(ops, level, adjoint=False)
        self.adj = m2l.m2l_plan_create(ops, level, adjoint=True)
        self.n_src = level.struct.ncells_src
        self.n_tgt = level.struct.ncells_tgt

    @property
    def dtype(self):
        return torch.float64 if self.precision == "fp64" else torch.float32

    def apply_forward(self, multipoles: torch.Tensor) -> torch.Tensor:
        out = torch.zeros(self.n_tgt, self.ops.n3, dtype=self.dtype, device=multipoles.device)
        m2l.m2l_plan_apply(self.fwd, multipoles.contiguous(), out, self.precision)
        return out

    def apply_adjoint(self, grad_locals: torch.Tensor) -> torch.Tensor:
        out = torch.zeros(self.n_src, self.ops.n3, dtype=self.dtype, device=grad_locals.device)
        m2l.m2l_plan_apply(self.adj, grad_locals.contiguous(), out, self.precision)
        return out

    def __call__(self, multipoles: torch.Tensor) -> torch.Tensor:
        return M2LFunction.apply(multipoles, self)


class M2LFunction(torch.autograd.Function):
    """locals = M2L(multipoles); d loss / d multipoles = M2L^T(d loss / d locals)."""

    @staticmethod
    def forward(ctx, multipoles: torch.Tensor, op: M2LLevelOperator) -> torch.Tensor:
        if multipoles.dtype != op.dtype:
            raise TypeError("multipoles must be %s for precision %s" % (op.dtype, op.precision))
        ctx.op = op
        return op.apply_forward(multipoles)

    @staticmethod
    def backward(ctx, grad_locals: torch.Tensor):
        op = ctx.op
        return op.apply_adjoint(grad_locals.to(op.dtype)), None
