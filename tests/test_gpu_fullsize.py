"""Parity at the full size of the benchmark workload (256^3 lattice, 40962-vertex mesh,
FP32, the launch configuration bench.py times): nodal forces and the spread force field in
full, one complete coupled step against one oracle step and 20 more, and mass conservation
over many steps (a property that holds at any size)."""
import numpy as np
import pytest

from pairs import make_pair, rel_l2
from paper_2305_18919_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full_pair():
    wl = inputs.shear_256_fp32()
    ref, gpu = make_pair(wl, "fp32")
    q = inputs.perturb(wl.mesh()[0], 0.05, seed=17)  # a slightly deformed interface
    ref.set_vertices(q)
    gpu.set_vertices(q)
    yield wl, ref, gpu
    ref.close()
    gpu.close()


def test_full_size_forces_and_spread(full_pair):
    wl, ref, gpu = full_pair
    phi_ref, _ = ref.forces()
    assert rel_l2(gpu.forces(), phi_ref) < 2e-6
    F_ref = ref.force_field()
    F = gpu.force_field()
    support = np.abs(F_ref).sum(-1) > 0
    assert support.sum() > 50000
    assert rel_l2(F[support], F_ref[support]) < 2e-6
    assert np.abs(F[~support]).max() == 0.0


def test_full_size_one_step(full_pair):
    wl, ref, gpu = full_pair
    ref.step(1)
    gpu.step(1)
    assert rel_l2(gpu.vertex_velocities(), ref.vertex_velocities()) < 1e-5
    assert np.abs(gpu.vertices() - ref.vertices()).max() < 1e-9 * wl.radius
    r0, u0 = ref.fields()
    r1, u1 = gpu.fields()
    assert rel_l2(u1, u0) < 1e-5
    assert rel_l2(r1, r0) < 1e-6
    # populations at a random sample of nodes, including the wall-adjacent layers
    f0 = ref.populations()
    f1 = gpu.populations()
    rng = np.random.default_rng(3)
    z = np.concatenate([[1, 254], rng.integers(1, 255, 200)])
    y = rng.integers(0, 256, z.size)
    x = rng.integers(0, 256, z.size)
    np.testing.assert_allclose(f1[:, z, y, x], f0[:, z, y, x], rtol=0, atol=2e-8)


def test_full_size_twenty_more_steps(full_pair):
    """The same pair 20 steps further (21 in all), in the launch configuration the bench times
    (the interface chain on its own SMs beside the stream-collide pass): vertices, velocities
    and densities against the oracle at the FP32 bars."""
    wl, ref, gpu = full_pair
    ref.step(20)
    gpu.step(20)
    assert np.abs(gpu.vertices() - ref.vertices()).max() < 1e-6 * wl.radius
    assert rel_l2(gpu.vertex_velocities(), ref.vertex_velocities()) < 1e-5
    r0, u0 = ref.fields()
    r1, u1 = gpu.fields()
    assert rel_l2(u1, u0) < 1e-5
    assert rel_l2(r1 - 1.0, r0 - 1.0) < 2e-5  # rho - rho0 is small: as on the 32^3 run


def test_full_size_mass_conservation():
    from paper_2305_18919_gb300 import binding
    wl = inputs.shear_256_fp32()
    lat = binding.Lattice.from_workload(wl, precision="fp32")
    m0 = lat.populations()[:, 1:-1].sum()
    lat.step(50)
    m1 = lat.populations()[:, 1:-1].sum()
    assert abs(m1 - m0) / m0 < 1e-9
    V, V0 = lat.volume()
    assert abs(V / V0 - 1) < 1e-3
    lat.close()


@pytest.mark.parametrize("precision,kind", [("fp32", "direct"), ("fp16", "staged")])
def test_beyond_32_bit_element_offsets(precision, kind):
    """A 512 x 512 x 520 lattice: each population array holds 19 x 136 M = 2.6 G elements, past
    2^31, so every element offset must be formed in 64 bits. Started from a state that repeats
    in x and y with period 32, it must evolve bit for bit like the 32 x 32 x 520 lattice (whose
    parity with the oracle the smaller tests check), at both ends of the big arrays."""
    from paper_2305_18919_gb300 import binding
    nz, p, n = 520, 32, 512
    rng = np.random.default_rng(12)
    rho = 1 + rng.uniform(-0.01, 0.01, (nz, p, p))
    u = rng.uniform(-0.03, 0.03, (nz, p, p, 3))
    walls = ((-0.02, 0.01, 0), (0.03, -0.01, 0))
    small = binding.Lattice(p, p, nz, 0.8, 1.0, *walls, precision=precision)
    small.set_stream_collide(kind)
    small.init_equilibrium(rho, u)
    small.step(3)
    r_s, u_s = small.fields()
    small.close()
    big = binding.Lattice(n, n, nz, 0.8, 1.0, *walls, precision=precision)
    assert big.stream_collide_staged() == (kind == "staged")
    reps = (1, n // p, n // p)
    big.init_equilibrium(np.tile(rho, reps), np.tile(u, reps + (1,)))
    big.step(3)
    r_b, u_b = big.fields()
    big.close()
    for ys, xs in ((slice(0, p), slice(0, p)), (slice(n - p, n), slice(n - p, n)),
                   (slice(n - p, n), slice(0, p))):
        assert np.array_equal(r_b[:, ys, xs], r_s)
        assert np.array_equal(u_b[:, ys, xs], u_s)


def test_wetting_128_full_size():
    """The static-wetting workload at its full size (128 x 128 x 96, R = 20, subdivision 5,
    FP32, the first of its eight wall strengths): three coupled steps against the oracle."""
    wl = inputs.wetting_128x128x96()
    ref, gpu = make_pair(wl, "fp32")
    ref.step(3)
    gpu.step(3)
    assert np.abs(gpu.vertices() - ref.vertices()).max() <= 1e-6 * wl.radius
    _, u0 = ref.fields()
    _, u1 = gpu.fields()
    assert rel_l2(u1[1:-1], u0[1:-1]) < 1e-5
    phi0, _ = ref.forces()
    assert rel_l2(gpu.forces(), phi0) < 2e-6
    ref.close()
    gpu.close()
