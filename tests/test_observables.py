"""Observables of the particle (paper_2305_18919_gb300.observables) against closed forms: the
volume moments of a box, whose equivalent ellipsoid has the box's aspect ratio, a box turned in
the shear plane (the inclination angle is the turn), a fine icosphere stretched into an ellipsoid
(the discretisation error), invariances, and the theory curves at values stated in the paper's
setting. The deformation index D and the inclination angle Theta follow Eq. taylor_deform and
the paper's definition of Theta (Sec. V); the semi-axes are those of the equivalent ellipsoid."""
import math

import numpy as np
import pytest
import torch

from paper_2305_18919_gb300 import inputs
from paper_2305_18919_gb300 import observables as ob


def box_mesh(A, B, C, centre=(0.0, 0.0, 0.0)):
    """A cuboid with half-extents A, B, C as 12 triangles, oriented outwards."""
    v = np.array([[sx * A, sy * B, sz * C] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)],
                 float) + np.asarray(centre, float)
    idx = lambda sx, sy, sz: 4 * (sx > 0) + 2 * (sy > 0) + (sz > 0)
    quads = []
    for axis in range(3):
        for s in (-1, 1):
            corners = []
            for a in (-1, 1):
                for b in (-1, 1):
                    c = [0, 0, 0]
                    c[axis] = s
                    o = [k for k in range(3) if k != axis]
                    c[o[0]], c[o[1]] = a, b
                    corners.append(idx(*c))
            quads.append((corners[0], corners[1], corners[3], corners[2]))
    faces = []
    ctr = v.mean(axis=0)
    for q in quads:
        for tri in ((q[0], q[1], q[2]), (q[0], q[2], q[3])):
            a, b, c = v[list(tri)]
            n = np.cross(b - a, c - a)
            faces.append(tri if np.dot(n, a - ctr) > 0 else (tri[0], tri[2], tri[1]))
    return v, np.array(faces, np.int64)


def rotate_xz(v, phi, about=(0.0, 0.0, 0.0)):
    """Turn points by phi in the x-z plane (from +x towards +z) about a point."""
    c, s = math.cos(phi), math.sin(phi)
    p = v - np.asarray(about)
    out = p.copy()
    out[:, 0] = c * p[:, 0] - s * p[:, 2]
    out[:, 2] = s * p[:, 0] + c * p[:, 2]
    return out + np.asarray(about)


def t(v):
    return torch.tensor(v, dtype=torch.float64)


def test_box_moments_exact():
    A, B, C, ctr = 3.0, 2.0, 1.25, (5.0, -1.0, 7.5)
    v, f = box_mesh(A, B, C, ctr)
    V, c, cov = ob.volume_moments(t(v), f)
    assert float(V) == pytest.approx(8 * A * B * C, rel=1e-14)
    np.testing.assert_allclose(c.numpy(), ctr, atol=1e-13)
    np.testing.assert_allclose(cov.numpy(), np.diag([A * A, B * B, C * C]) / 3.0, atol=1e-13)


@pytest.mark.parametrize("phi", [0.0, 0.3, -0.6, math.pi / 4, 1.2])
def test_box_in_shear_plane(phi):
    """The equivalent ellipsoid of a box has semi-axes sqrt(5/3) times the half-extents, so D is
    (A - C)/(A + C); the box turned by phi in the x-z plane has Theta = phi."""
    A, C = 3.0, 1.0
    v, f = box_mesh(A, 2.0, C, (1.0, 2.0, 3.0))
    v = rotate_xz(v, phi, about=(1.0, 2.0, 3.0))
    r1, r3, theta = ob.shear_plane_axes(t(v), f)
    assert float(r1) == pytest.approx(math.sqrt(5.0 / 3.0) * A, rel=1e-12)
    assert float(r3) == pytest.approx(math.sqrt(5.0 / 3.0) * C, rel=1e-12)
    D, th = ob.deformation(t(v), f)
    assert float(D) == pytest.approx((A - C) / (A + C), rel=1e-12)
    assert float(th) == pytest.approx(phi, abs=1e-12)


def test_ellipsoid_from_fine_icosphere():
    """A subdivision-5 icosphere stretched to semi-axes (a, b, c): D within the discretisation
    error of (a - c)/(a + c), Theta = 0, and the semi-axes themselves."""
    a, b, c = 12.0, 9.0, 7.0
    v, f = inputs.icosphere(5, 1.0, (0.0, 0.0, 0.0))
    v = v * np.array([a, b, c])
    r1, r3, theta = ob.shear_plane_axes(t(v), f)
    assert float(r1) == pytest.approx(a, rel=2e-3)
    assert float(r3) == pytest.approx(c, rel=2e-3)
    D, th = ob.deformation(t(v), f)
    assert float(D) == pytest.approx((a - c) / (a + c), rel=2e-3)
    assert abs(float(th)) < 1e-12
    V, cm, _ = ob.volume_moments(t(v), f)
    assert float(V) == pytest.approx(4.0 / 3.0 * math.pi * a * b * c, rel=2e-3)
    np.testing.assert_allclose(cm.numpy(), 0.0, atol=1e-12)


def test_sphere_has_no_deformation_and_translates():
    v, f = inputs.icosphere(4, 6.0, (16.0, 16.0, 15.5))
    D, _ = ob.deformation(t(v), f)
    assert abs(float(D)) < 1e-12
    np.testing.assert_allclose(ob.center_of_mass(t(v), f).numpy(), (16.0, 16.0, 15.5), atol=1e-12)
    shifted = v + np.array([3.0, -2.0, 0.25])
    np.testing.assert_allclose(ob.center_of_mass(t(shifted), f).numpy(), (19.0, 14.0, 15.75),
                               atol=1e-12)


def test_invariant_to_translation_and_vertex_order():
    v, f = inputs.icosphere(3, 5.0, (0.0, 0.0, 0.0))
    v = rotate_xz(v * np.array([1.3, 1.0, 0.8]), 0.4)
    D0, th0 = ob.deformation(t(v), f)
    D1, th1 = ob.deformation(t(v + np.array([10.0, 5.0, -3.0])), f)
    perm = np.random.default_rng(1).permutation(len(v))
    inv = np.argsort(perm)
    D2, th2 = ob.deformation(t(v[perm]), inv[f])
    for D, th in ((D1, th1), (D2, th2)):
        assert float(D) == pytest.approx(float(D0), rel=1e-12)
        assert float(th) == pytest.approx(float(th0), abs=1e-12)
    assert float(th0) == pytest.approx(0.4, abs=1e-12)


def test_deformation_gradient_matches_finite_differences():
    v, f = inputs.icosphere(2, 4.0, (0.0, 0.0, 0.0))
    v = rotate_xz(v * np.array([1.2, 1.0, 0.9]), 0.3)
    q = t(v).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x: ob.deformation(x, f)[0], (q,), eps=1e-6, atol=1e-8)
    assert torch.autograd.gradcheck(lambda x: ob.deformation(x, f)[1], (q,), eps=1e-6, atol=1e-8)
    assert torch.autograd.gradcheck(lambda x: ob.center_of_mass(x, f)[2], (q,), eps=1e-6,
                                    atol=1e-8)


def test_theory_curves():
    # a pure droplet of viscosity ratio 1: D = 35/32 Ca, Theta = pi/4 - 35/32 Ca
    assert ob.theory_deformation_droplet(0.1) == pytest.approx(0.109375, rel=1e-15)
    assert ob.theory_inclination_droplet(0.1) == pytest.approx(math.pi / 4 - 0.109375, rel=1e-15)
    # the 32^3 shear case (walls at -/+0.01, R = 6, alpha_bar = 0.01): Ca = 0.0667, D = 0.073
    Ca = (1.0 / 6.0) * 6.0 * (0.02 / 30.0) / 0.01
    assert ob.theory_deformation_droplet(Ca) == pytest.approx(0.0729, abs=1e-4)
    # Eq. deformation: alpha = (1, 1, 1) gives 35/48 Ca, (1, 0, 1) gives 5/7 Ca
    assert ob.theory_deformation((1, 1, 1), 0.048) == pytest.approx(0.035, rel=1e-14)
    assert ob.theory_deformation((1, 0, 1), 0.07) == pytest.approx(0.05, rel=1e-14)


def test_agrees_with_the_physics_pins_helper():
    """The numpy helper the oracle's physics pins use (tests/observables.py, written apart
    from this module) gives the same D, Theta and volume on deformed, turned meshes."""
    import observables as tob
    rng = np.random.default_rng(3)
    for sub, axes, phi in ((2, (1.3, 1.0, 0.8), 0.4), (3, (1.0, 1.1, 1.6), -0.9),
                           (4, (2.0, 1.0, 1.0), 0.05)):
        v, f = inputs.icosphere(sub, 5.0, (0.0, 0.0, 0.0))
        v = rotate_xz(v * np.array(axes), phi) + rng.uniform(-0.05, 0.05, v.shape)
        v = v + np.array([30.0, 20.0, 12.0])
        D_ref, th_ref = tob.taylor_deformation(v, np.asarray(f))
        D, th = ob.deformation(t(v), f)
        assert float(D) == pytest.approx(D_ref, rel=1e-10)
        assert float(th) == pytest.approx(th_ref, abs=1e-10)
        V_ref, c_ref, _ = tob.volume_moments(v, np.asarray(f))
        V, c, _ = ob.volume_moments(t(v), f)
        assert float(V) == pytest.approx(V_ref, rel=1e-12)
        np.testing.assert_allclose(c.numpy(), c_ref, atol=1e-10)
