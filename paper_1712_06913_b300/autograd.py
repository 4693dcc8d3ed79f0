"""torch.autograd wrappers: the degridding operator and the chi-square loss.

Degrid.forward  = muser_degrid(FORWARD):  sky image x [N, N] -> predicted visibilities A x.
Degrid.backward = muser_degrid(ADJOINT):  grad_x = Re A^H grad_v.  For a real loss, torch
passes grad_v = dL/dRe v + i dL/dIm v, and dL/dx = Re(A^H grad_v) because A is linear.
Chi2.forward    = muser_chi2: sum_k w_k |v_k - obs_k|^2 / sigma^2; its backward returns the
kernel's residual seed 2 w (v - obs) / sigma^2 times the incoming gradient.
"""
from __future__ import annotations

import torch

from . import api
from ._lib import ADJOINT, FORWARD


class Degrid(torch.autograd.Function):
    @staticmethod
    def forward(ctx, img, rec, cfg):
        ctx.save_for_backward(rec)
        ctx.cfg = cfg
        return api.degrid(FORWARD, rec, cfg, img=img.detach())

    @staticmethod
    def backward(ctx, grad_vis):
        (rec,) = ctx.saved_tensors
        g = api.degrid(ADJOINT, rec, ctx.cfg, vis=grad_vis.contiguous())
        return g, None, None


class Chi2(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pred, obs, rec, inv_sigma2):
        loss, resid = api.chi2(pred.detach(), obs, rec, inv_sigma2, want_resid=True)
        ctx.save_for_backward(resid)
        return loss

    @staticmethod
    def backward(ctx, grad_loss):
        (resid,) = ctx.saved_tensors
        return resid * grad_loss, None, None, None


def chi2_loss(img, rec, obs, inv_sigma2, cfg):
    """chi2(img) through both autograd functions."""
    return Chi2.apply(Degrid.apply(img, rec, cfg), obs, rec, inv_sigma2)
