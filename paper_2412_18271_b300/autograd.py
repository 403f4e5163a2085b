"""torch.autograd.Function wrappers over the library's learned path.

LearnedEnergy:      E(positions) with backward dE/dx = -F, the forces of the
                    hand-written feature adjoint (no autograd graph through
                    the model).
ForceMatchingLoss:  L(params) for a batch of frames; the forward pass runs the
                    device trainer, which evaluates the loss and its gradient
                    (the force term by reverse mode over the MLP's tangent
                    pass along U = J dL/dF) in one sweep; backward returns that
                    gradient scaled by the incoming one.
CosineAdamW:        AdamW (decoupled weight decay) with lr_t = lr (1 + cos(pi t/T))/2,
                    one device kernel per step.
Every tensor is a CUDA tensor on the current device; the kernels are enqueued
on torch's current stream.
"""
from __future__ import annotations

import math

import torch

from . import mdpf


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


class LearnedEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pos: torch.Tensor, context: "mdpf.Context"):
        if not (pos.is_cuda and pos.dtype == torch.float64 and pos.is_contiguous()):
            raise ValueError("positions must be a contiguous CUDA float64 tensor [N, 3]")
        E = torch.empty(1, dtype=torch.float64, device=pos.device)
        F = torch.empty(pos.shape, dtype=torch.float32, device=pos.device)
        context.compute_device(pos.data_ptr(), E.data_ptr(), F.data_ptr(), _stream())
        ctx.save_for_backward(F)
        return E[0]

    @staticmethod
    def backward(ctx, grad_E):
        (F,) = ctx.saved_tensors
        return -(grad_E * F.to(torch.float64)), None


class ForceMatchingLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, trainer: "mdpf.Trainer", pos: torch.Tensor, element: torch.Tensor,
                E_ref: torch.Tensor, F_ref: torch.Tensor):
        for t, dt in ((params, torch.float32), (pos, torch.float64), (element, torch.int32),
                      (E_ref, torch.float64), (F_ref, torch.float32)):
            if not (t.is_cuda and t.dtype == dt and t.is_contiguous()):
                raise ValueError("ForceMatchingLoss: expected contiguous CUDA tensors of the documented dtypes")
        n_frames = E_ref.shape[0]
        grad = torch.empty_like(params)
        loss3 = torch.empty(3, dtype=torch.float64, device=params.device)
        trainer.loss_grad(params.data_ptr(), grad.data_ptr(), n_frames, pos.data_ptr(), element.data_ptr(),
                          E_ref.data_ptr(), F_ref.data_ptr(), loss3.data_ptr(), _stream())
        ctx.save_for_backward(grad)
        ctx.mark_non_differentiable(loss3)
        return loss3[0].clone(), loss3

    @staticmethod
    def backward(ctx, grad_L, _grad_parts):
        (grad,) = ctx.saved_tensors
        return grad * grad_L.to(grad.dtype), None, None, None, None, None


class CosineAdamW(torch.optim.Optimizer):
    def __init__(self, params, lr: float = 1e-3, total_steps: int = 20000, betas=(0.9, 0.999), eps: float = 1e-8,
                 weight_decay: float = 0.01):
        super().__init__(params, dict(lr=lr, total_steps=total_steps, betas=betas, eps=eps,
                                      weight_decay=weight_decay))

    def lr_at(self, t: int, group) -> float:
        T = group["total_steps"]
        return 0.0 if t >= T else group["lr"] * 0.5 * (1.0 + math.cos(math.pi * t / T))

    @torch.no_grad()
    def step(self, closure=None):
        loss = closure() if closure is not None else None
        for group in self.param_groups:
            for p in group["params"]:
                if p.grad is None:
                    continue
                if not (p.is_cuda and p.dtype == torch.float32 and p.is_contiguous()):
                    raise ValueError("CosineAdamW: parameters must be contiguous CUDA float32 tensors")
                st = self.state[p]
                if not st:
                    st["t"] = 0
                    st["m"] = torch.zeros_like(p)
                    st["v"] = torch.zeros_like(p)
                lr = self.lr_at(st["t"], group)
                st["t"] += 1
                g = p.grad.contiguous()
                b1, b2 = group["betas"]
                mdpf.adamw_step(p.data_ptr(), g.data_ptr(), st["m"].data_ptr(), st["v"].data_ptr(), p.numel(),
                                st["t"], lr, b1, b2, group["eps"], group["weight_decay"], _stream())
        return loss
