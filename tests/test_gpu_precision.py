"""16-bit population storage (FP16, BF16; collision and forcing in FP32) against the FP64
oracle, through the C ABI.

The populations are stored as scaled deviations (f_i - w_i rho0) K / w_i, so every stored
value carries the storage type's unit roundoff u_s relative to its own size (2^-11 for FP16,
2^-8 for BF16) at every step. The bars below are stated in units of u_s; they hold with a
margin of about two over the measured errors:

- velocity, relative L2 over the fluid:               <= 2 u_s
- density, largest absolute difference:               <= 0.2 u_s
- vertex positions after the run, largest difference: <= 2 u_s R
- Couette profile, largest difference from the exact linear profile: <= 10 u_s U_wall
"""
import numpy as np
import pytest

from pairs import make_pair, rel_l2
from paper_2305_18919_gb300 import inputs

pytestmark = pytest.mark.gpu

U_S = {"fp16": 2.0 ** -11, "bf16": 2.0 ** -8}


@pytest.fixture(scope="module")
def shear32_oracle():
    """The 32^3 shear workload (R = 6 droplet, walls at -/+0.01) after 1000 FP64 oracle steps."""
    import oracle
    wl = inputs.shear_32_fp64()
    sim = oracle.Simulation.from_workload(wl)
    sim.step(1000)
    rho, u = sim.fields()
    q = sim.vertices()
    sim.close()
    return wl, rho, u, q


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_shear32_1000_steps(shear32_oracle, precision):
    from paper_2305_18919_gb300 import binding
    wl, rho_o, u_o, q_o = shear32_oracle
    us = U_S[precision]
    lat = binding.Lattice.from_workload(wl, precision=precision)
    assert lat.bytes_per_cell() == 76
    lat.step(1000)
    rho, u = lat.fields()
    q = lat.vertices()
    lat.close()
    fl = slice(1, wl.nz - 1)
    assert rel_l2(u[fl], u_o[fl]) <= 2 * us
    assert np.abs(rho[fl] - rho_o[fl]).max() <= 0.2 * us
    assert np.abs(q - q_o).max() <= 2 * us * wl.radius


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_couette_closed_form(precision):
    """Steady Couette flow between walls at -/+U: linear between the bounce-back planes."""
    from paper_2305_18919_gb300 import binding
    nz, U = 16, 0.01
    lat = binding.Lattice(4, 4, nz, 1.0, 1.0, (-U, 0, 0), (U, 0, 0), precision=precision)
    lat.step(3000)
    _, u = lat.fields()
    lat.close()
    z = np.arange(1, nz - 1)
    exact = -U + 2 * U * (z - 0.5) / (nz - 2)
    assert np.abs(u[1:nz - 1, :, :, 0] - exact[:, None, None]).max() <= 10 * U_S[precision] * U


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
@pytest.mark.parametrize("shape,z_periodic", [((8, 12, 8), True), ((132, 4, 7), False),
                                              ((4, 8, 9), False)])
def test_random_state_body_force(precision, shape, z_periodic):
    """A random equilibrium state with a body force: the first (in-place) collision and the
    forced pull kernel, x-rows of one to 33 four-node groups, periodic and walled z."""
    import oracle
    from paper_2305_18919_gb300 import binding
    nx, ny, nz = shape
    args = (nx, ny, nz, 0.8, 1.0, (0, 0, 0) if z_periodic else (-0.02, 0.01, 0),
            (0, 0, 0) if z_periodic else (0.03, -0.01, 0), (1e-5, -2e-5, 3e-5 if z_periodic else 0))
    ref = oracle.Simulation(*args, z_periodic)
    gpu = binding.Lattice(*args, precision, z_periodic)
    rng = np.random.default_rng(7)
    rho = 1 + rng.uniform(-0.01, 0.01, (nz, ny, nx))
    u = rng.uniform(-0.03, 0.03, (nz, ny, nx, 3))
    ref.init_equilibrium(rho, u)
    gpu.init_equilibrium(rho, u)
    ref.step(20)
    gpu.step(20)
    r0, u0 = ref.fields()
    r1, u1 = gpu.fields()
    gpu.close()
    ref.close()
    us = U_S[precision]
    fl = slice(None) if z_periodic else slice(1, nz - 1)
    assert rel_l2(u1[fl], u0[fl]) <= 2 * us
    assert np.abs(r1[fl] - r0[fl]).max() <= 0.2 * us


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_wetting_200_steps(precision):
    wl = inputs.scaled_wetting(32, 24, 3, 6.0, alpha=(1e-3, 0, 1e-3), eps=2e-4, precision="fp64")
    ref, gpu = make_pair(wl, precision)
    ref.step(200)
    gpu.step(200)
    _, u0 = ref.fields()
    _, u1 = gpu.fields()
    q0, q1 = ref.vertices(), gpu.vertices()
    gpu.close()
    ref.close()
    us = U_S[precision]
    fl = slice(1, wl.nz - 1)
    assert rel_l2(u1[fl], u0[fl]) <= 2 * us
    assert np.abs(q1 - q0).max() <= 2 * us * wl.radius
