"""Shape observables used by the physics pins (Sec. IV): Taylor deformation D (Eq. 20) and
inclination angle Theta, from the second moments of the enclosed volume.

For a solid ellipsoid with semi-axes r_k the volume second moment along a principal axis is
V r_k^2 / 5, so r_k = sqrt(5 lambda_k / V) for the eigenvalues lambda_k of the centred volume
second-moment tensor restricted to the shear (x, z) plane.
"""
import math

import numpy as np


def volume_moments(q, faces):
    """Volume V, centroid and centred second-moment tensor of a closed outward mesh."""
    x0, x1, x2 = q[faces[:, 0]], q[faces[:, 1]], q[faces[:, 2]]
    vol = np.einsum("ij,ij->i", x0, np.cross(x1, x2)) / 6.0  # tetrahedra with the origin
    V = vol.sum()
    cen = (vol[:, None] * (x0 + x1 + x2) / 4.0).sum(0) / V
    y0, y1, y2 = x0 - cen, x1 - cen, x2 - cen
    vol = np.einsum("ij,ij->i", y0, np.cross(y1, y2)) / 6.0
    s = y0 + y1 + y2
    # second moment of a tetrahedron with one vertex at the origin
    M = (np.einsum("i,ia,ib->ab", vol, y0, y0) + np.einsum("i,ia,ib->ab", vol, y1, y1)
         + np.einsum("i,ia,ib->ab", vol, y2, y2) + np.einsum("i,ia,ib->ab", vol, s, s)) / 20.0
    return V, cen, M


def taylor_deformation(q, faces):
    """(D, Theta) in the x-z shear plane; Theta is the major axis angle from +x (radians)."""
    V, _, M = volume_moments(q, faces)
    Mxz = np.array([[M[0, 0], M[0, 2]], [M[2, 0], M[2, 2]]])
    lam, vec = np.linalg.eigh(Mxz)
    r3, r1 = np.sqrt(5 * lam / V)
    major = vec[:, 1]
    theta = math.atan2(major[1], major[0])
    if theta > math.pi / 2:
        theta -= math.pi
    if theta < -math.pi / 2:
        theta += math.pi
    return (r1 - r3) / (r1 + r3), theta
