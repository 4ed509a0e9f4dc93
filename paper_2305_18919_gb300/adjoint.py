"""Gradients of observables of an IB-LB run with respect to the interface parameters, through
torch.autograd.

`run(theta, workload, nsteps, every, precision)` is a torch.autograd.Function: its forward builds
a fresh FP64 (or FP32) context from the workload with theta = (alpha1, alpha2, alpha3, eps) (Eq. 2, Eq. 19),
advances it nsteps steps while recording the trajectory (iblb_adjoint_record), and returns the
final vertex positions; its backward maps dJ/dq to dJ/dtheta with the discrete adjoint on the
GPU (iblb_adjoint_gradient). Any observable written in torch on the returned positions can then
be differentiated, e.g. the apparent contact angle and the wetted radius below.
"""
from __future__ import annotations

import copy

import torch

from . import binding
# the observables live in their own module; re-exported here, where they were first written
from .observables import contact_angle, contact_angle_selection, wetted_radius  # noqa: F401


class IBLBRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, workload, nsteps, every, precision="fp64"):
        wl = copy.deepcopy(workload)
        th = [float(t) for t in theta.detach().cpu().reshape(4)]
        wl.alpha, wl.eps = tuple(th[:3]), th[3]
        lat = binding.Lattice.from_workload(wl, precision=precision)
        lat.adjoint_record(int(nsteps), int(every))
        ctx.lat = lat
        return torch.tensor(lat.vertices(), dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_q):
        lat = ctx.lat
        g = lat.adjoint_gradient(grad_q.detach().cpu().numpy())
        lat.close()
        ctx.lat = None
        return torch.tensor(g, dtype=torch.float64), None, None, None, None


def run(theta, workload, nsteps, every=100, precision="fp64"):
    """Final vertex positions [nv][3] of `workload` run nsteps steps with parameters theta
    (a float64 tensor (alpha1, alpha2, alpha3, eps)), differentiable in theta. precision: the
    forward run's storage, "fp64" or "fp32" (the reverse pass is in double either way)."""
    return IBLBRun.apply(theta, workload, nsteps, every, precision)
