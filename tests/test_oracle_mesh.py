"""Pins of the oracle's interface forces (Eqs. 2, 16-19) and of the mesh inputs.

- the face energy equals the strain-energy law of Eq. 2 evaluated on principal stretches
  obtained by an SVD of the in-plane deformation (a different route from the oracle's
  metric tensors);
- forces are minus the finite-difference gradient of the total energy (Eqs. 17-19);
- strain and volume forces have zero net force and torque; energies are invariant under
  rigid motions (the wall energy under x,y translation and z rotation);
- on the rest shape the volume force vanishes and the strain force is -alpha_1 times the
  area gradient (zero for the capsule classes);
- the Lennard-Jones force vanishes at d = 2^(1/6) xi and equals 24 eps / xi at d = xi;
- polyhedral volumes match closed forms (cube, icosahedron).
"""
import math

import numpy as np
import pytest

from paper_2305_18919_gb300 import inputs


def _rot(rng):
    Qm, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Qm) < 0:
        Qm[:, 0] *= -1
    return Qm


def _strain_energy_law(l1, l2, alpha):
    """Eq. 2 written on principal stretches (w_S0 dropped)."""
    I1 = l1 ** 2 + l2 ** 2 - 2
    I2 = l1 ** 2 * l2 ** 2 - 1
    a1, a2, a3 = alpha
    L = math.log(I2 + 1)
    return 0.5 * (a1 - a3) * L + 0.125 * (a1 + a2) * L * L + a3 * (0.5 * (I1 + 2) - 1)


def test_face_energy_matches_principal_stretch_law(oracle_mod):
    rng = np.random.default_rng(20)
    for trial in range(30):
        alpha = rng.uniform(0, 1, 3)
        # reference triangle in its plane, then embedded by a random rotation + shift
        P = rng.normal(size=(3, 2))
        R0, R1 = _rot(rng), _rot(rng)
        Fd = np.eye(2) + rng.uniform(-0.3, 0.3, (2, 2))
        if np.linalg.det(Fd) <= 0.2:
            continue
        X = np.column_stack([P, np.zeros(3)]) @ R0.T + rng.normal(size=3)
        x = np.column_stack([P @ Fd.T, np.zeros(3)]) @ R1.T + rng.normal(size=3)
        l1, l2 = np.linalg.svd(Fd, compute_uv=False)
        e1, e2 = P[1] - P[0], P[2] - P[0]
        A0 = 0.5 * abs(e1[0] * e2[1] - e1[1] * e2[0])
        expected = A0 * _strain_energy_law(l1, l2, alpha)
        face = np.array([[0, 1, 2]], np.int32)
        _, en, _ = oracle_mod.mesh_forces(x, face, X, [0, 0, 0], 1.0, alpha, volume_on=0)
        np.testing.assert_allclose(en[0], expected, rtol=1e-12, atol=1e-14)


def _total_energy(oracle_mod, q, faces, X, centre, V0, alpha, **kw):
    _, en, _ = oracle_mod.mesh_forces(q, faces, X, centre, V0, alpha, **kw)
    return en.sum()


@pytest.mark.parametrize("cls", list(inputs.ALPHA_CLASSES))
def test_forces_are_minus_energy_gradient(oracle_mod, cls):
    rng = np.random.default_rng(hash(cls) % 2 ** 32)
    X, faces = inputs.icosphere(1, 3.0, (5.0, 5.0, 4.2))
    q = inputs.perturb(X, 0.25, seed=21)
    alpha = np.array(inputs.ALPHA_CLASSES[cls]) * rng.uniform(0.5, 2.0)
    centre = X.mean(0)
    V0 = oracle_mod.mesh_volume(X, faces, centre)
    kw = dict(kV=1.0, eps=0.3, xi=0.5, wall_on=1, volume_on=1, has_walls=1, z_bottom=0.5, z_top=12.5)
    phi, _, _ = oracle_mod.mesh_forces(q, faces, X, centre, V0, alpha, **kw)
    h = 1e-6
    grad = np.zeros_like(q)
    for v in range(q.shape[0]):
        for k in range(3):
            qp = q.copy(); qp[v, k] += h
            qm = q.copy(); qm[v, k] -= h
            grad[v, k] = (_total_energy(oracle_mod, qp, faces, X, centre, V0, alpha, **kw)
                          - _total_energy(oracle_mod, qm, faces, X, centre, V0, alpha, **kw)) / (2 * h)
    scale = np.abs(phi).max()
    np.testing.assert_allclose(phi, -grad, atol=2e-7 * scale + 1e-12)


def test_strain_and_volume_forces_free_of_net_force_and_torque(oracle_mod):
    X, faces = inputs.icosphere(2, 4.0, (0.3, -0.2, 0.1))
    q = inputs.perturb(X, 0.3, seed=22)
    centre = X.mean(0)
    V0 = oracle_mod.mesh_volume(X, faces, centre)
    phi, _, _ = oracle_mod.mesh_forces(q, faces, X, centre, V0, [0.7, 0.4, 1.1], wall_on=0)
    s = np.abs(phi).max()
    np.testing.assert_allclose(phi.sum(0), 0, atol=1e-13 * s * len(q))
    np.testing.assert_allclose(np.cross(q, phi).sum(0), 0, atol=1e-12 * s * len(q))


def test_energies_invariant_under_rigid_motion(oracle_mod):
    rng = np.random.default_rng(23)
    X, faces = inputs.icosphere(2, 4.0, (8.0, 8.0, 6.0))
    q = inputs.perturb(X, 0.3, seed=24)
    centre = X.mean(0)
    V0 = oracle_mod.mesh_volume(X, faces, centre)
    alpha = [0.7, 0.4, 1.1]
    kw = dict(eps=0.2, wall_on=1, has_walls=1, z_bottom=0.5, z_top=20.5)
    _, e0, V = oracle_mod.mesh_forces(q, faces, X, centre, V0, alpha, **kw)
    R = _rot(rng)
    t = rng.normal(size=3)
    _, e1, V1 = oracle_mod.mesh_forces(q @ R.T + t, faces, X, centre, V0, alpha, **kw)
    np.testing.assert_allclose(e1[:2], e0[:2], rtol=1e-11)
    np.testing.assert_allclose(V1, V, rtol=1e-12)
    # wall energy: invariant under x,y shifts and rotations about z only
    c, s_ = math.cos(0.7), math.sin(0.7)
    Rz = np.array([[c, -s_, 0], [s_, c, 0], [0, 0, 1]])
    _, e2, _ = oracle_mod.mesh_forces(q @ Rz.T + [3.0, -2.0, 0.0], faces, X, centre, V0, alpha, **kw)
    np.testing.assert_allclose(e2, e0, rtol=1e-11)


def test_rest_shape_forces(oracle_mod):
    """At rest phi^V = 0 and phi^S = -alpha_1 grad(area) (alpha_2, alpha_3 do not act)."""
    X, faces = inputs.icosphere(2, 5.0, (1.0, 2.0, 3.0))
    centre = X.mean(0)
    V0 = oracle_mod.mesh_volume(X, faces, centre)

    def area(q):
        a = q[faces[:, 1]] - q[faces[:, 0]]
        b = q[faces[:, 2]] - q[faces[:, 0]]
        return 0.5 * np.linalg.norm(np.cross(a, b), axis=1).sum()

    h = 1e-6
    gA = np.zeros_like(X)
    for v in range(X.shape[0]):
        for k in range(3):
            qp = X.copy(); qp[v, k] += h
            qm = X.copy(); qm[v, k] -= h
            gA[v, k] = (area(qp) - area(qm)) / (2 * h)
    for alpha in ([0.3, 0.0, 0.0], [0.3, 0.5, 0.7], [0.0, 0.0, 1.0], [0.0, 1.0, 1.0]):
        phi, en, V = oracle_mod.mesh_forces(X, faces, X, centre, V0, alpha, volume_on=1)
        np.testing.assert_allclose(phi, -alpha[0] * gA, atol=1e-8)
        assert abs(V - V0) < 1e-12 * V0
        assert abs(en[1]) < 1e-20
    phi, _, _ = oracle_mod.mesh_forces(X, faces, X, centre, V0, [0.0, 0.0, 1.0])
    assert np.abs(phi).max() < 1e-13


def test_shear_term_force_is_linear_in_positions(oracle_mod):
    """With alpha = (a, -a, a) both log terms of Eq. 2 cancel and the energy is a A0 I1/2,
    quadratic in q, so the force is affine in q (second difference zero)."""
    X, faces = inputs.icosphere(1, 3.0)
    rng = np.random.default_rng(25)
    q0 = inputs.perturb(X, 0.2, seed=26)
    d = rng.normal(size=q0.shape) * 0.1
    f = [oracle_mod.mesh_forces(q0 + k * d, faces, X, [0, 0, 0], 1.0, [1.3, -1.3, 1.3], volume_on=0)[0]
         for k in range(3)]
    np.testing.assert_allclose(f[2] - 2 * f[1] + f[0], 0, atol=1e-13)


def test_lennard_jones_closed_form(oracle_mod):
    """One face parallel to the bottom wall at height d above the plane z = 0.5: the summed
    nodal force is 48 eps [(xi/d)^12 - (xi/d)^6/2] / d along +z (Eq. 19)."""
    eps, xi = 0.37, 0.5
    face = np.array([[0, 1, 2]], np.int32)
    for d, expected in ((2 ** (1 / 6) * xi, 0.0), (xi, 24 * eps / xi), (0.8, None), (1.7, None)):
        zc = 0.5 + d
        q = np.array([[0, 0, zc], [1, 0, zc], [0, 1, zc]], float)
        phi, en, _ = oracle_mod.mesh_forces(q, face, q, [0, 0, 0], 1.0, [0, 0, 0], eps=eps, xi=xi,
                                            wall_on=1, volume_on=0, has_walls=1, z_bottom=0.5,
                                            z_top=1e7)
        fz = 48 * eps * ((xi / d) ** 12 - 0.5 * (xi / d) ** 6) / d
        if expected is not None:
            assert abs(fz - expected) < 1e-12
        np.testing.assert_allclose(phi[:, 2], fz / 3, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(phi[:, :2], 0, atol=1e-18)
        np.testing.assert_allclose(en[2], 4 * eps * ((xi / d) ** 12 - (xi / d) ** 6), rtol=1e-12, atol=1e-18)


def test_polyhedral_volume_closed_forms(oracle_mod):
    # unit cube scaled by s, 12 outward triangles
    s = 2.5
    v = np.array([[x, y, z] for z in (0, 1) for y in (0, 1) for x in (0, 1)], float) * s
    f = np.array([[0, 2, 1], [1, 2, 3], [4, 5, 6], [5, 7, 6], [0, 1, 4], [1, 5, 4],
                  [2, 6, 3], [3, 6, 7], [0, 4, 2], [2, 4, 6], [1, 3, 5], [3, 7, 5]], np.int32)
    for c in ([0, 0, 0], [10, -3, 2], [1.2, 1.2, 1.2]):
        np.testing.assert_allclose(oracle_mod.mesh_volume(v, f, c), s ** 3, rtol=1e-13)
    # regular icosahedron of circumradius R: edge a = 4R / sqrt(10 + 2 sqrt5)
    R = 3.0
    X, faces = inputs.icosphere(0, R)
    a = 4 * R / math.sqrt(10 + 2 * math.sqrt(5))
    np.testing.assert_allclose(oracle_mod.mesh_volume(X, faces), 5 / 12 * (3 + math.sqrt(5)) * a ** 3, rtol=1e-13)
    # refined spheres approach 4/3 pi R^3 from below
    vols = [oracle_mod.mesh_volume(*inputs.icosphere(n, R)) for n in range(1, 6)]
    assert all(v1 > v0 for v0, v1 in zip(vols, vols[1:]))
    err = [1 - v / (4 / 3 * math.pi * R ** 3) for v in vols]
    assert 0 < err[-1] < 1e-3
    # inscribed polyhedra converge at second order in the edge length (halved per level)
    assert 3.8 < err[-2] / err[-1] < 4.2


def test_icosphere_counts_and_closure():
    for n, (nv, nf) in enumerate([(12, 20), (42, 80), (162, 320), (642, 1280)]):
        v, f = inputs.icosphere(n, 2.0)
        assert v.shape == (nv, 3) and f.shape == (nf, 3) and nf == 2 * nv - 4
        np.testing.assert_allclose(np.linalg.norm(v, axis=1), 2.0, rtol=1e-14)
        # every directed edge appears once and its reverse once (closed, consistently oriented)
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
        s = set(map(tuple, e.tolist()))
        assert len(s) == len(e) and all((b, a) in s for a, b in s)
