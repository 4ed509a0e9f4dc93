"""Observables of the particle, written in torch on the vertex positions so that they can be
differentiated (through paper_2305_18919_gb300.adjoint.run) with respect to the interface
parameters.

Shear flow (Sec. V): the deformation index D = (r1 - r3) / (r1 + r3) of Eq. taylor_deform and the
inclination angle Theta, with r1, r3 the semi-axes in the shear plane. The semi-axes are those of
the ellipsoid with the same second moments as the enclosed volume: a solid ellipsoid with
semi-axes a_k has the covariance diag(a_k^2) / 5, so a_k = (5 lambda_k)^(1/2) for the eigenvalues
lambda_k of the volume's covariance. The shear plane is the plane of the flow (x) and the
velocity gradient (z, the wall normal); Theta is the angle of the major axis from +x towards +z.

Wetting (Sec. V): the centre-of-mass height Z_CM, the apparent contact angle and the wetted
radius r = (A_c / pi)^(1/2) (A_c the area of the faces near the wall).

The volume, centroid and covariance are exact for the triangulated surface: each face and a
fixed point o span a tetrahedron of signed volume v = (x0 - o) . ((x1 - o) x (x2 - o)) / 6,
whose first and second moments about o are v s / 4 and v (sum_k p_k p_k^T + s s^T) / 20 (p_k the
corners relative to o, s their sum); the sums over the faces are those of the enclosed volume.

The theory curves the paper compares D and Theta with (small deformations) are given as plain
functions: Eq. deformation (coated droplets and particles), Eq. deformation_droplet (pure droplet),
Eq. inclination_angle, and the transient of Eq. evJK integrated numerically (bbr_evolution).
"""
from __future__ import annotations

import math

import numpy as np
import torch


def _faces(faces):
    return torch.as_tensor(np.asarray(faces), dtype=torch.long)


def volume_moments(q, faces):
    """(V, centroid [3], covariance [3][3]) of the volume enclosed by the mesh (faces oriented
    counter-clockwise seen from outside, so that V > 0)."""
    f = _faces(faces)
    o = q.detach().mean(dim=0)  # a nearby fixed point keeps the sums free of cancellation
    p0, p1, p2 = q[f[:, 0]] - o, q[f[:, 1]] - o, q[f[:, 2]] - o
    v = (p0 * torch.linalg.cross(p1, p2)).sum(dim=1) / 6.0
    s = p0 + p1 + p2
    V = v.sum()
    m1 = (v[:, None] * s).sum(dim=0) / 4.0
    outer = lambda a, b: a[:, :, None] * b[:, None, :]
    m2 = (v[:, None, None] * (outer(p0, p0) + outer(p1, p1) + outer(p2, p2) + outer(s, s))).sum(dim=0) / 20.0
    c = m1 / V
    cov = m2 / V - c[:, None] * c[None, :]
    return V, o + c, cov


def center_of_mass(q, faces):
    """Centroid of the enclosed volume (Z_CM = its z component)."""
    return volume_moments(q, faces)[1]


def shear_plane_axes(q, faces, plane=(0, 2)):
    """(r1, r3, Theta): semi-axes (r1 >= r3) of the equivalent ellipsoid in the shear plane
    (axes `plane`, default x and z) and the angle of the r1 axis from the first axis towards the
    second, in (-pi/2, pi/2]."""
    _, _, cov = volume_moments(q, faces)
    i, j = plane
    a, b, c = cov[i, i], cov[i, j], cov[j, j]
    mean = 0.5 * (a + c)
    rad = torch.sqrt(0.25 * (a - c) ** 2 + b * b)
    r1 = torch.sqrt(5.0 * (mean + rad))
    r3 = torch.sqrt(5.0 * (mean - rad))
    theta = 0.5 * torch.atan2(2.0 * b, a - c)
    return r1, r3, theta


def deformation(q, faces, plane=(0, 2)):
    """(D, Theta): the deformation index of Eq. taylor_deform and the inclination angle."""
    r1, r3, theta = shear_plane_axes(q, faces, plane)
    return (r1 - r3) / (r1 + r3), theta


def theory_deformation(alpha, Ca):
    """Steady small-deformation D of Eq. deformation for alpha = (alpha1, alpha2, alpha3) with
    alpha2, alpha3 not both zero; Ca = mu R gamma_dot / alpha1."""
    a1, a2, a3 = (float(a) for a in alpha)
    num = 5.0 * a1 * (3.0 * a2 + 4.0 * a3)
    den = 4.0 * (3.0 * a1 * a2 + 5.0 * a1 * a3 + 2.0 * a2 * a3 + 2.0 * a3 * a3)
    return num / den * Ca


def theory_deformation_droplet(Ca, lam=1.0):
    """Steady small-deformation D of a pure droplet, Eq. deformation_droplet (viscosity ratio
    lam)."""
    return (19.0 * lam + 16.0) / (16.0 * lam + 16.0) * Ca


def theory_inclination_droplet(Ca, lam=1.0):
    """Inclination angle of a pure droplet at small Ca, Eq. inclination_angle (radians)."""
    return math.pi / 4.0 - (19.0 * lam + 16.0) * (2.0 * lam + 3.0) / (80.0 * (lam + 1.0)) * Ca


def bbr_evolution(alpha, Ca, t_end, dt=0.002, lam=1.0, every=1):
    """Small-deformation shape evolution of Eq. evJK (Sec. II), integrated by classical RK4.

    Returns (t, D, Theta): the time t in units of the inverse shear rate, the deformation index
    D = (J_11^2 + J_12^2)^(1/2) of Eq. deformation_J and the inclination Theta (radians) of the
    major axis of J from the flow direction, every `every` steps of dt.

    Reading of the garbled dimensions: time runs in t_hat = gamma_dot t; E and Omega are the
    symmetric and antisymmetric parts of the velocity gradient of a unit simple shear
    u = (x_2, 0, 0) (index 1 the flow, 2 the gradient direction; here x and z); the material
    tensors L and M of Eq. L_M are formed with alpha divided by the alpha of Ca (alpha1 for
    pre-stressed particles, alpha3 otherwise) and divided by Ca, which makes J of order Ca so
    that D needs no factor Ca. The Jaumann derivative is dA/dt - (Omega A - A Omega) with
    Omega_ab = (du_a/dx_b - du_b/dx_a) / 2. J and K start at zero (a sphere at rest).
    Under this reading the steady state reproduces Eq. deformation (coated droplets and
    capsules), Eq. deformation_droplet and, for a droplet, Eq. inclination_angle.
    """
    a = np.asarray(alpha, dtype=np.float64)
    ref = a[0] if a[0] > 0 else a[2]
    a1, a2, a3 = a / ref
    E = np.zeros((3, 3))
    E[0, 2] = E[2, 0] = 0.5
    W = np.zeros((3, 3))
    W[0, 2], W[2, 0] = 0.5, -0.5
    c1 = 1.0 / (2.0 * lam + 3.0)
    c2 = (6.0 * lam + 4.0) / ((2.0 * lam + 3.0) * (19.0 * lam + 16.0))
    c3 = 2.0 / (19.0 * lam + 16.0)

    def rates(J, K):
        L = (4.0 * (a2 + a3) * J - (6.0 * a2 + 10.0 * a3) * K) / Ca
        M = (-4.0 * (a1 + 2.0 * a2 + 2.0 * a3) * J + (12.0 * a2 + 16.0 * a3) * K) / Ca
        dK = W @ K - K @ W + c1 * (5.0 * E + L) + c2 * M
        dJK = W @ (J - K) - (J - K) @ W + c3 * M
        return dK + dJK, dK

    J = np.zeros((3, 3))
    K = np.zeros((3, 3))
    n = int(round(t_end / dt))
    ts, Ds, Th = [0.0], [0.0], [math.pi / 4.0]
    for k in range(1, n + 1):
        j1, k1 = rates(J, K)
        j2, k2 = rates(J + 0.5 * dt * j1, K + 0.5 * dt * k1)
        j3, k3 = rates(J + 0.5 * dt * j2, K + 0.5 * dt * k2)
        j4, k4 = rates(J + dt * j3, K + dt * k3)
        J = J + dt / 6.0 * (j1 + 2.0 * j2 + 2.0 * j3 + j4)
        K = K + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        if k % every == 0:
            ts.append(k * dt)
            Ds.append(math.hypot(J[0, 0], J[0, 2]))
            Th.append(0.5 * math.atan2(2.0 * J[0, 2], J[0, 0] - J[2, 2]))
    return np.array(ts), np.array(Ds), np.array(Th)


def contact_angle(q, faces, z_wall=0.5, exclude=1.0, select=None):
    """Apparent contact angle in degrees of a particle resting on the wall plane z_wall.

    The vertices of a central slab |y - y_centroid| < h (h = the mean edge length, so that the
    slab holds about one ring of vertices per height) away from the contact region
    (z - z_wall >= exclude) are fitted by a circle in the x-z plane (algebraic least squares,
    x^2 + z^2 + D x + E z + G = 0); the angle is arccos(-(z_c - z_wall) / R_c) with the circle's
    centre height z_c and radius R_c (defined once the fitted circle reaches the plane, i.e.
    once the droplet has spread; a plane higher up can serve before). The vertex selection is
    taken from the values (it is constant under small changes), or is the boolean mask `select`
    if given (e.g. the one of `contact_angle_selection` for a reference configuration); the fit
    and the angle are differentiable.
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
    f = _faces(faces)
    edges = torch.cat([q[f[:, 1]] - q[f[:, 0]], q[f[:, 2]] - q[f[:, 1]], q[f[:, 0]] - q[f[:, 2]]])
    h = float(edges.detach().norm(dim=1).mean())
    qd = q.detach()
    return ((qd[:, 1] - qd[:, 1].mean()).abs() < h) & (qd[:, 2] - z_wall >= exclude)


def wetted_radius(q, faces, z_wall=0.5, within=1.0, select=None):
    """sqrt(A_c / pi) with A_c the area of the faces whose centroid lies within `within` of the
    wall plane (the selection from the values, or the face mask `select`; the areas are
    differentiable)."""
    f = _faces(faces)
    a = q[f[:, 1]] - q[f[:, 0]]
    b = q[f[:, 2]] - q[f[:, 0]]
    area = 0.5 * torch.linalg.cross(a, b).norm(dim=1)
    if select is None:
        gz = (q[f[:, 0], 2] + q[f[:, 1], 2] + q[f[:, 2], 2]).detach() / 3
        select = gz - z_wall < within
    return torch.sqrt(area[select].sum() / math.pi)
