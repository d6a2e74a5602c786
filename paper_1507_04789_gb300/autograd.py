"""PyTorch autograd bridge and maximum-likelihood fitting for the M-RA.

``loglik(handle, theta)`` returns the M-RA log-likelihood (Sec. 3.3) as a
differentiable scalar of ``theta = (sigma2, range, tau2)`` (a float64 CPU
tensor): the forward pass calls ``mra_loglik_grad`` once, which runs the FP64
evaluation and its hand-written reverse-mode adjoint on the GPU, and the
backward pass scales that stored gradient by the incoming gradient.

``fit_mle`` maximises the log-likelihood numerically over the three parameters
(the fit of Sec. 4.3; the paper does not name an optimiser): Adam on the
log-parameters, so every iterate stays positive.
"""
from __future__ import annotations

import numpy as np
import torch

from .mra import Handle


class MRALogLik(torch.autograd.Function):
    """loglik(theta) with the gradient from the library's adjoint."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, handle: Handle):
        th = theta.detach().to("cpu", torch.float64).numpy()
        ll, g = handle.loglik_grad(th)
        ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
        return torch.as_tensor(ll, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None


def loglik(handle: Handle, theta: torch.Tensor) -> torch.Tensor:
    return MRALogLik.apply(theta, handle)


def fit_mle(handle: Handle, theta0, steps: int = 20, lr: float = 0.1, fixed=()):
    """Adam ascent on log(theta); returns (theta, history of (theta, loglik))."""
    log_t = torch.tensor(np.log(np.asarray(theta0, dtype=np.float64)), requires_grad=True)
    mask = torch.ones(3, dtype=torch.float64)
    for k in fixed:
        mask[k] = 0.0
    opt = torch.optim.Adam([log_t], lr=lr)
    hist = []
    for _ in range(steps):
        opt.zero_grad()
        theta = torch.exp(log_t)
        ll = loglik(handle, theta)
        (-ll).backward()
        log_t.grad *= mask
        hist.append((theta.detach().numpy().copy(), float(ll.detach())))
        opt.step()
    theta = torch.exp(log_t).detach().numpy()
    hist.append((theta.copy(), handle.loglik(theta)))
    return theta, hist
