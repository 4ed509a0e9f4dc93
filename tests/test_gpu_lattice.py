"""GPU parity of the lattice-Boltzmann part (stream-collide with Guo forcing and bounce-back,
Eqs. 9-10) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from pairs import rel_l2

pytestmark = pytest.mark.gpu


def _lat_pair(nx, ny, nz, tau, ub, ut, g, precision, z_periodic=False, seed=0):
    import oracle
    from paper_2305_18919_gb300 import binding
    ref = oracle.Simulation(nx, ny, nz, tau, 1.0, ub, ut, g, z_periodic)
    gpu = binding.Lattice(nx, ny, nz, tau, 1.0, ub, ut, g, precision, z_periodic)
    rng = np.random.default_rng(seed)
    rho = 1 + rng.uniform(-0.01, 0.01, (nz, ny, nx))
    u = rng.uniform(-0.03, 0.03, (nz, ny, nx, 3))
    ref.init_equilibrium(rho, u)
    gpu.init_equilibrium(rho, u)
    return ref, gpu


@pytest.mark.parametrize("shape", [(8, 8, 6), (12, 8, 9), (132, 4, 7), (48, 20, 11)])
def test_stream_collide_fp64_bitclose(shape):
    nx, ny, nz = shape
    ref, gpu = _lat_pair(nx, ny, nz, 0.8, (-0.02, 0.01, 0), (0.03, -0.01, 0), (1e-5, -2e-5, 0), "fp64")
    for steps in (1, 7):
        ref.step(steps)
        gpu.step(steps)
        np.testing.assert_allclose(gpu.populations(), ref.populations(), rtol=0, atol=1e-14)
        r0, u0 = ref.fields()
        r1, u1 = gpu.fields()
        np.testing.assert_allclose(r1, r0, rtol=1e-13)
        np.testing.assert_allclose(u1, u0, rtol=0, atol=1e-14)


def test_stream_collide_periodic_z_fp64():
    ref, gpu = _lat_pair(8, 12, 8, 1.3, (0, 0, 0), (0, 0, 0), (1e-5, 2e-5, -3e-5), "fp64", z_periodic=True)
    ref.step(5)
    gpu.step(5)
    np.testing.assert_allclose(gpu.populations(), ref.populations(), rtol=0, atol=1e-14)


def test_stream_collide_fp32_tolerance():
    ref, gpu = _lat_pair(32, 16, 18, 0.8, (-0.02, 0, 0), (0.02, 0, 0), (0, 0, 0), "fp32")
    ref.step(200)
    gpu.step(200)
    r0, u0 = ref.fields()
    r1, u1 = gpu.fields()
    assert rel_l2(u1, u0) < 1e-5
    assert rel_l2(r1, r0) < 1e-5
    assert rel_l2(r1 - 1, r0 - 1) < 1e-4


def test_couette_gpu_fp32():
    """The CUDA path also reproduces the exact Couette profile (closed form, not the oracle)."""
    from paper_2305_18919_gb300 import binding
    nz, U = 16, 0.01
    lat = binding.Lattice(4, 4, nz, 1.0, 1.0, (-U, 0, 0), (U, 0, 0), precision="fp32")
    lat.step(6000)
    _, u = lat.fields()
    z = np.arange(1, nz - 1)
    expected = np.broadcast_to((-U + 2 * U * (z - 0.5) / (nz - 2))[:, None, None], u[1:-1, :, :, 0].shape)
    np.testing.assert_allclose(u[1:-1, :, :, 0], expected, atol=2e-8)


def test_mass_conservation_gpu_fp64():
    ref, gpu = _lat_pair(16, 8, 10, 0.7, (-0.03, 0.02, 0), (0.01, -0.02, 0), (0, 0, 0), "fp64", seed=3)
    m0 = gpu.populations()[:, 1:-1].sum()
    gpu.step(100)
    m1 = gpu.populations()[:, 1:-1].sum()
    assert abs(m1 - m0) / m0 < 1e-13
