"""The learned unrolled DCF network as a torch.autograd.Function.

The network (K exact-consensus iterations with learned per-step
``lambda_k = lambda e^{a_k}``, ``rho_k = rho e^{b_k}`` and relaxation ``c_k``)
and its reverse pass both run in libdcf.so (``dcf_unrolled_forward`` /
``dcf_unrolled_backward``); this module only carries the three length-K
parameter vectors through autograd and provides a small training loop over
a list of problems.
"""
from __future__ import annotations

import numpy as np
import torch

from . import dcf

__all__ = ["UnrolledLoss", "UnrolledDCF", "train"]


class UnrolledLoss(torch.autograd.Function):
    """loss = sum_k w_k ||U_k V_k^T - A B^T||^2 / ||A B^T||^2 of one problem.

    Inputs a, b, c: float64 CPU tensors of length K; ``solver`` is a
    :class:`dcf.Solver` holding M, the truth factors (``set_truth``) and the
    start point.  After the call the solver holds U_K, V_K.
    """

    @staticmethod
    def forward(ctx, a, b, c, solver, weights=None):
        tot, _ = solver.unrolled_forward(a.detach().cpu().numpy(), b.detach().cpu().numpy(),
                                         c.detach().cpu().numpy(), weights)
        ctx.solver = solver
        ctx.K = int(a.numel())
        return torch.tensor(tot, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        ga, gb, gc = ctx.solver.unrolled_backward(ctx.K)
        g = float(grad_out)
        as_t = lambda x: torch.from_numpy(np.asarray(x) * g)
        return as_t(ga), as_t(gb), as_t(gc), None, None


class UnrolledDCF(torch.nn.Module):
    """Parameters of a K-step network; zero a, b and unit c give K plain steps."""

    def __init__(self, K):
        super().__init__()
        self.K = int(K)
        self.a = torch.nn.Parameter(torch.zeros(self.K, dtype=torch.float64))
        self.b = torch.nn.Parameter(torch.zeros(self.K, dtype=torch.float64))
        self.c = torch.nn.Parameter(torch.ones(self.K, dtype=torch.float64))

    def forward(self, solver, start=None, weights=None):
        """Loss of one problem; ``start=(U0, V0)`` reloads the start point first."""
        if start is not None:
            solver.load_init(*start)
        return UnrolledLoss.apply(self.a, self.b, self.c, solver, weights)

    def theta(self):
        return tuple(p.detach().cpu().numpy().copy() for p in (self.a, self.b, self.c))


def train(net, problems, steps, lr=0.05, log=None):
    """Adam on the mean loss over ``problems`` = [(solver, (U0, V0)), ...].

    Returns the list of mean losses, one per step (before that step's update).
    """
    opt = torch.optim.Adam(net.parameters(), lr=lr)
    hist = []
    for it in range(int(steps)):
        opt.zero_grad()
        total = 0.0
        for solver, start in problems:
            loss = net(solver, start) / len(problems)
            loss.backward()
            total += float(loss.detach())
        hist.append(total)
        if log is not None:
            log(it, total)
        opt.step()
    return hist


# ---------------------------------------------------------------------------
# Helpers of the learned workload: the plain method's fixed point is the
# target the network is trained toward and the reference its output is measured against.
# ---------------------------------------------------------------------------
def fixed_point(solver, U0, iters):
    """Plain iterations from (U0, V0 = S = 0 sweep); returns the factors
    reached after ``iters`` steps (the method's fixed point to rounding)."""
    solver.load_init(U0)
    solver.step(iters)
    return solver.factors()


def steps_to_tolerance(solver, U0, tol, max_steps, theta=None):
    """Plain steps needed (after the network ``theta``, if given) until
    ||U V^T - L_target|| / ||L_target|| <= tol, where L_target is the solver's
    registered truth.  Returns max_steps + 1 when the tolerance is not met."""
    solver.load_init(U0)
    if theta is not None:
        solver.unrolled_forward(*theta, want_loss=False)
        if solver.rel_err() <= tol:
            return 0
    for t in range(1, max_steps + 1):
        solver.step(1)
        if solver.rel_err() <= tol:
            return t
    return max_steps + 1
