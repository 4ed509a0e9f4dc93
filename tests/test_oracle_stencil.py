"""Pins of the oracle's immersed-boundary coupling (Eqs. 11-15): Peskin's defining
conditions of the 4-point function, exactness of interpolation for constant and linear
fields, force and first-moment conservation of spreading, and the adjoint relation
between spreading (Eq. 13) and interpolation (Eq. 11)."""
import numpy as np


def test_phi4_defining_conditions(oracle_mod):
    """For every shift s: sum_j phi(s-j) = 1, sum_j (s-j) phi(s-j) = 0,
    sum_j phi(s-j)^2 = 3/8, and the even-j and odd-j sums are 1/2 each."""
    rng = np.random.default_rng(10)
    j = np.arange(-4, 5)
    for s in np.concatenate([rng.uniform(-1, 1, 200), [0.0, 0.5, 1.0, -1.0]]):
        w = oracle_mod.phi4(s - j)
        assert abs(w.sum() - 1) < 1e-14
        assert abs(((s - j) * w).sum()) < 1e-14
        assert abs((w ** 2).sum() - 3 / 8) < 1e-14
        assert abs(w[j % 2 == 0].sum() - 0.5) < 1e-14
        assert abs(w[j % 2 == 1].sum() - 0.5) < 1e-14


def test_phi4_values_and_support(oracle_mod):
    r = np.array([0.0, 1.0, 2.0, 2.5, -1.0, -2.0, 3.0])
    np.testing.assert_allclose(oracle_mod.phi4(r), [0.5, 0.25, 0.0, 0.0, 0.25, 0.0, 0.0], atol=1e-16)
    x = np.linspace(-2.5, 2.5, 2001)
    w = oracle_mod.phi4(x)
    assert (w >= 0).all()
    np.testing.assert_allclose(w, oracle_mod.phi4(-x), atol=1e-16)  # even
    # continuity and C^1 at |r| = 1 and 2
    for a in (1.0, 2.0):
        h = 1e-7
        assert abs(oracle_mod.phi4(a - h) - oracle_mod.phi4(a + h)) < 1e-6
        dl = (oracle_mod.phi4(a - h) - oracle_mod.phi4(a - 2 * h)) / h
        dr = (oracle_mod.phi4(a + 2 * h) - oracle_mod.phi4(a + h)) / h
        assert abs(dl - dr) < 1e-5


def _random_vertices(rng, n, lo, hi):
    return rng.uniform(lo, hi, (n, 3))


def test_interpolation_exact_for_linear_fields(oracle_mod):
    """Zeroth and first moment conditions make interpolation exact for u = A x + b."""
    shape = (16, 16, 16)
    rng = np.random.default_rng(11)
    A = rng.normal(size=(3, 3)) * 1e-3
    b = rng.normal(size=3) * 1e-2
    z, y, x = np.meshgrid(np.arange(16), np.arange(16), np.arange(16), indexing="ij")
    pos = np.stack([x, y, z], -1).astype(float)
    u = pos @ A.T + b
    q = _random_vertices(rng, 50, 4.0, 11.0)
    qd = oracle_mod.interpolate(shape, 0, [0, 0, 0], [0, 0, 0], u, q)
    np.testing.assert_allclose(qd, q @ A.T + b, atol=1e-15)


def test_interpolation_constant_near_walls(oracle_mod):
    """Wall-layer stencil nodes carry the wall velocity: a uniform field equal to the wall
    velocity interpolates exactly up to the wall."""
    shape = (8, 8, 10)
    U = np.array([0.01, -0.02, 0.0])
    u = np.broadcast_to(U, (10, 8, 8, 3)).copy()
    rng = np.random.default_rng(12)
    q = np.column_stack([rng.uniform(0, 8, 40), rng.uniform(0, 8, 40), rng.uniform(1.0, 8.0, 40)])
    qd = oracle_mod.interpolate(shape, 1, U, U, u, q)
    np.testing.assert_allclose(qd, np.broadcast_to(U, qd.shape), atol=1e-15)


def test_spread_conserves_force_and_moment(oracle_mod):
    shape = (20, 20, 20)
    rng = np.random.default_rng(13)
    q = _random_vertices(rng, 30, 5.0, 14.0)
    phi = rng.normal(size=(30, 3))
    F = oracle_mod.spread(shape, 0, q, phi)
    np.testing.assert_allclose(F.sum((0, 1, 2)), phi.sum(0), rtol=1e-13)
    z, y, x = np.meshgrid(np.arange(20), np.arange(20), np.arange(20), indexing="ij")
    pos = np.stack([x, y, z], -1).astype(float)
    # sum_x x_a F_b = sum_i q_ia phi_ib (first-moment condition)
    np.testing.assert_allclose(np.einsum("zyxa,zyxb->ab", pos, F), q.T @ phi, rtol=1e-12, atol=1e-12)


def test_spread_is_adjoint_of_interpolation(oracle_mod):
    """<spread(phi), u> = <phi, interpolate(u)> with periodic wrap, for random fields; with
    walls (zero wall velocity) force on wall layers is dropped and they interpolate as 0."""
    rng = np.random.default_rng(14)
    for has_walls, shape in ((0, (7, 6, 5)), (1, (6, 7, 9))):
        nx, ny, nz = shape
        q = np.column_stack([rng.uniform(-3, 10, 25), rng.uniform(-3, 10, 25),
                             rng.uniform(1.0, nz - 2.0, 25) if has_walls else rng.uniform(-3, 10, 25)])
        phi = rng.normal(size=(25, 3))
        u = rng.normal(size=(nz, ny, nx, 3))
        if has_walls:
            u[0] = 0
            u[-1] = 0
        F = oracle_mod.spread(shape, has_walls, q, phi)
        qd = oracle_mod.interpolate(shape, has_walls, [0, 0, 0], [0, 0, 0], u, q)
        np.testing.assert_allclose((F * u).sum(), (phi * qd).sum(), rtol=1e-12)
        if has_walls:
            assert np.all(F[0] == 0) and np.all(F[-1] == 0)


def test_spread_wraps_periodic_axes(oracle_mod):
    """A vertex near x=0 spreads onto x = nx-1 (periodic x, y)."""
    F = oracle_mod.spread((8, 8, 8), 0, np.array([[0.2, 4.5, 4.5]]), np.array([[1.0, 0, 0]]))
    assert F[:, :, 7, 0].sum() > 0
    np.testing.assert_allclose(F[..., 0].sum(), 1.0, rtol=1e-14)
