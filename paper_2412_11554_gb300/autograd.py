"""torch.autograd binding of the ACCORD smooth loss.

SmoothLoss.apply(Omega, X) = -sum_i log omega_ii + 1/2 tr(Omega^T Omega S),
S = X^T X / n: the pseudolikelihood part of Eq. 3.2 (no penalty).  Forward and
backward both run in libaccord: the forward through accord_loss, the backward
through accord_grad (dL/dOmega = -diag(1/omega_ii) + Omega S) and
accord_grad_x (dL/dX = (1/n) X Omega^T Omega).  Omega float64 selects the FP64
kernels, float32 the mixed BF16x3 ones; X is float32 data.
"""
import torch

from .accord import accord_grad, accord_grad_x, accord_loss


class SmoothLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Omega: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
        prec = "fp64" if Omega.dtype == torch.float64 else "mixed"
        f, _ = accord_loss(X, Omega, 0.0, precision=prec, penalize_diag=False)
        ctx.save_for_backward(Omega, X)
        return torch.tensor(f, dtype=Omega.dtype, device=Omega.device)

    @staticmethod
    def backward(ctx, gout: torch.Tensor):
        Omega, X = ctx.saved_tensors
        gO = gX = None
        # the incoming gradient stays on the device: scaling by it always,
        # rather than testing it for 1 on the host, keeps backward free of a
        # stream synchronisation
        if ctx.needs_input_grad[0]:
            gO = accord_grad(X, Omega, smooth=True) * gout.to(Omega.dtype)
        if ctx.needs_input_grad[1]:
            gX = accord_grad_x(X, Omega).to(X.dtype) * gout.to(X.dtype)
        return gO, gX


def smooth_loss(Omega: torch.Tensor, X: torch.Tensor) -> torch.Tensor:
    """Differentiable smooth ACCORD loss (see SmoothLoss)."""
    return SmoothLoss.apply(Omega, X)
