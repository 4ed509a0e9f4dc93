"""Gradients of observables of an IB-LB run with respect to the interface parameters, through
torch.autograd.

`run(theta, workload, nsteps, every)` is a torch.autograd.Function: its forward builds a fresh
FP64 context from the workload with theta = (alpha1, alpha2, alpha3, eps) (Eq. 2, Eq. 19),
advances it nsteps steps while recording the trajectory (iblb_adjoint_record), and returns the
final vertex positions; its backward maps dJ/dq to dJ/dtheta with the discrete adjoint on the
GPU (iblb_adjoint_gradient). Any observable written in torch on the returned positions can then
be differentiated, e.g. the apparent contact angle and the wetted radius below.
"""
from __future__ import annotations

import copy
import math

import numpy as np
import torch

from . import binding


class IBLBRun(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, workload, nsteps, every):
        wl = copy.deepcopy(workload)
        th = [float(t) for t in theta.detach().cpu().reshape(4)]
        wl.alpha, wl.eps = tuple(th[:3]), th[3]
        lat = binding.Lattice.from_workload(wl, precision="fp64")
        lat.adjoint_record(int(nsteps), int(every))
        ctx.lat = lat
        return torch.tensor(lat.vertices(), dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_q):
        lat = ctx.lat
        g = lat.adjoint_gradient(grad_q.detach().cpu().numpy())
        lat.close()
        ctx.lat = None
        return torch.tensor(g, dtype=torch.float64), None, None, None


def run(theta, workload, nsteps, every=100):
    """Final vertex positions [nv][3] of `workload` run nsteps steps with parameters theta
    (a float64 tensor (alpha1, alpha2, alpha3, eps)), differentiable in theta."""
    return IBLBRun.apply(theta, workload, nsteps, every)


def contact_angle(q, faces, z_wall=0.5, exclude=1.0, select=None):
    """Apparent contact angle in degrees of a particle resting on the wall plane z_wall.

    The vertices of a central slab |y - y_centroid| < h (h = the mean edge length, so that the
    slab holds about one ring of vertices per height) away from the contact region
    (z - z_wall >= exclude) are fitted by a circle in the x-z plane (algebraic least squares,
    x^2 + z^2 + D x + E z + G = 0); the angle is arccos(-(z_c - z_wall) / R_c) with the circle's
    centre height z_c and radius R_c (defined once the fitted circle reaches the plane, i.e.
    once the droplet has spread; a plane higher up can serve before). The vertex selection is
    taken from the values (it is
    constant under small changes), or is the boolean mask `select` if given (e.g. the one of
    `contact_angle_selection` for a reference configuration); the fit and the angle are
    differentiable.
    """
    sel = contact_angle_selection(q, faces, z_wall, exclude) if select is None else select
    x, z = q[sel, 0], q[sel, 2]
    A = torch.stack([x, z, torch.ones_like(x)], dim=1)
    b = -(x * x + z * z)
    D, E, G = torch.linalg.solve(A.T @ A, A.T @ b)
    zc = -E / 2
    R = torch.sqrt(D * D / 4 + E * E / 4 - G)
    return torch.rad2deg(torch.arccos(-(zc - z_wall) / R))


def contact_angle_selection(q, faces, z_wall=0.5, exclude=1.0):
    """The vertices contact_angle fits: a central slab one mean edge length wide in y, away
    from the contact region."""
    f = torch.as_tensor(np.asarray(faces), dtype=torch.long)
    edges = torch.cat([q[f[:, 1]] - q[f[:, 0]], q[f[:, 2]] - q[f[:, 1]], q[f[:, 0]] - q[f[:, 2]]])
    h = float(edges.detach().norm(dim=1).mean())
    qd = q.detach()
    return ((qd[:, 1] - qd[:, 1].mean()).abs() < h) & (qd[:, 2] - z_wall >= exclude)


def wetted_radius(q, faces, z_wall=0.5, within=1.0, select=None):
    """sqrt(A_c / pi) with A_c the area of the faces whose centroid lies within `within` of the
    wall plane (the selection from the values, or the face mask `select`; the areas are
    differentiable)."""
    f = torch.as_tensor(np.asarray(faces), dtype=torch.long)
    a = q[f[:, 1]] - q[f[:, 0]]
    b = q[f[:, 2]] - q[f[:, 0]]
    area = 0.5 * torch.linalg.cross(a, b).norm(dim=1)
    if select is None:
        gz = (q[f[:, 0], 2] + q[f[:, 1], 2] + q[f[:, 2], 2]).detach() / 3
        select = gz - z_wall < within
    return torch.sqrt(area[select].sum() / math.pi)
