"""torch.autograd wrappers: the degridding operator and the chi-square loss.

Degrid.forward  = muser_degrid(FORWARD):  sky image x [N, N] -> predicted visibilities A x.
Degrid.backward = muser_degrid(ADJOINT):  grad_x = Re A^H grad_v.  For a real loss, torch
passes grad_v = dL/dRe v + i dL/dIm v, and dL/dx = Re(A^H grad_v) because A is linear.
Chi2.forward    = muser_chi2: sum_k w_k |v_k - obs_k|^2 / sigma^2; its backward returns the
kernel's residual seed 2 w (v - obs) / sigma^2 times the incoming gradient (muser_axpy).

Every step of the arithmetic is a library call; this module only allocates tensors and passes
them on (and, across ranks, sums tensors with torch.distributed).
"""
from __future__ import annotations

import torch

from . import api
from . import dist as _dist
from ._lib import ADJOINT, FORWARD


class Degrid(torch.autograd.Function):
    """vis = A img with a DegridPlan; backward applies the plan's adjoint."""

    @staticmethod
    def forward(ctx, img, plan):
        ctx.plan = plan
        return plan.forward(img.detach())

    @staticmethod
    def backward(ctx, grad_vis):
        return ctx.plan.adjoint(grad_vis.contiguous()), None


class Chi2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pred, obs, plan, inv_sigma2):
        loss, resid = plan.chi2(pred.detach(), obs, inv_sigma2)
        ctx.save_for_backward(resid)
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        (resid,) = ctx.saved_tensors
        out = torch.zeros_like(resid)
        api.axpy(out, resid, 1.0, grad_loss.detach().reshape(1).float().contiguous())
        return out, None, None, None


def chi2_loss(img, plan, obs, inv_sigma2):
    """chi2(img) through both autograd functions (plan: api.DegridPlan of the records).  Chi2 weighs
    the visibilities by the records' own weights, so a plan with uniform weighting (weight_mode 1,
    whose weights only the library's fused calls apply) is refused here."""
    if plan.cfg.weight_mode != 0:
        raise ValueError("chi2_loss uses the records' own weights: with weight_mode 1 use "
                         "GradientImaging.step (muser_grad_step), which applies the uniform weights")
    return Chi2.apply(Degrid.apply(img, plan), obs, plan, inv_sigma2)


class GradientImaging:
    """Gradient-descent imaging of one sky image from visibilities (chi-square data term).

    Each step evaluates chi2 and its gradient through Degrid/Chi2 (forward operator,
    chi-square seed and adjoint are library kernels) and applies x <- x - eta * grad.
    `capture()` records one step (or several chained steps) in a CUDA graph so that `replay()`
    runs them without host work; the image, loss and gradient live in fixed device tensors.

    Under torch.distributed each rank passes the records and visibilities of its own block of
    channels (`dist.block`); the loss and the gradient are summed over ranks every step, so
    every rank applies the same update to its copy of the image.
    """

    def __init__(self, rec, obs, sigma, cfg, x0=None, eta=None):
        import torch
        self.rec, self.cfg = rec, cfg
        self.plan = api.DegridPlan(rec, cfg)
        self.obs = obs.to(torch.complex64).contiguous()
        self.inv_s2 = 1.0 / float(sigma) ** 2
        self.x = (torch.zeros((cfg.N, cfg.N), dtype=torch.float32, device="cuda") if x0 is None
                  else x0.detach().clone().float()).requires_grad_(True)
        self.eta = eta
        self.loss = None
        self.graph = None

    def lipschitz(self, iters=20, seed=0):
        """Largest eigenvalue of the chi2 Hessian 2 Re(A^H W A)/sigma^2 by power iteration from a
        seeded random start direction (muser_lipschitz; across ranks the Hessian products are summed
        before each normalisation).  Returns L as a Python float."""
        import torch
        g = torch.Generator(device="cuda").manual_seed(seed)
        v = torch.randn((self.cfg.N, self.cfg.N), generator=g, device="cuda")
        if _dist.rank_world()[1] == 1:
            L = self.plan.lipschitz(v, self.inv_s2, iters)
        else:
            L = torch.empty(1, dtype=torch.float32, device="cuda")
            api.normalize(v, v, L)
            u = torch.empty_like(v)
            for _ in range(iters):
                self.plan.normal_apply(v, self.inv_s2, out=u)
                _dist.all_sum_(u)
                api.normalize(u, v, L)
        return float(L[0])

    def reset_chain(self):
        """Forget the forward pass the last chained step left in the workspace (call it after
        writing self.x outside step())."""
        self.plan.rows_ready = None

    def _buffers(self):
        import torch
        if not hasattr(self, "_loss_buf"):
            self._loss_buf = torch.zeros(1, dtype=torch.float32, device="cuda")
            self._grad_buf = torch.zeros((self.cfg.N, self.cfg.N), dtype=torch.float32, device="cuda")

    def step(self):
        """One step.  In a single process one library call does it all (muser_grad_step: forward,
        chi-square, adjoint and update).  Across ranks each rank's call returns its loss and gradient
        (eta = 0 leaves the image), both are summed over ranks, and muser_axpy applies the update."""
        import torch
        self._buffers()
        single = _dist.rank_world()[1] == 1
        with torch.no_grad():
            if single:                  # chained: each step leaves the next one's first pass done
                self.plan.grad_step(self.x, self.obs, self.inv_s2, self.eta, self._loss_buf, chain=True)
            else:
                self.plan.grad_step(self.x, self.obs, self.inv_s2, 0.0, self._loss_buf, self._grad_buf)
                _dist.all_sum_(self._grad_buf)
                _dist.all_sum_(self._loss_buf)
                api.axpy(self.x.data, self._grad_buf, -self.eta)
        self.loss = self._loss_buf[0]
        return self.loss

    def step_autograd(self):
        """The same step through Degrid/Chi2 and loss.backward(), the update by muser_axpy."""
        import torch
        self.x.grad = None
        loss = chi2_loss(self.x, self.plan, self.obs, self.inv_s2)
        loss.backward()
        with torch.no_grad():
            loss = loss.detach()
            if _dist.rank_world()[1] > 1:
                _dist.all_sum_(self.x.grad)
                loss = _dist.all_sum_(loss.clone())
            api.axpy(self.x.data, self.x.grad.contiguous(), -self.eta)
        self.loss = loss
        return self.loss

    def capture(self, warmup=3, steps=1):
        """Record `steps` consecutive steps in one CUDA graph (after `warmup` eager steps on a side
        stream): a descent loop of many steps replays it and pays one graph launch per `steps`."""
        import torch
        if self.eta is None:
            self.eta = 1.0 / self.lipschitz()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self.step()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            for _ in range(steps):
                self.static_loss = self.step()
        self.graph_steps = steps
        return self

    def replay(self, n=1):
        """Replay the captured graph n times (n * `steps` steps); returns the last step's loss."""
        for _ in range(n):
            self.graph.replay()
        return self.static_loss
