"""Edge cases of the CUDA path against the FP64 oracle: no steps at all, the smallest lattices
(a single fluid layer between the walls, the shortest periodic z), the coarsest mesh (the bare
icosahedron, 12 vertices), and a fluid at rest, which the collision must leave exactly at
rest (Eq. 10 at u = 0, rho = rho0 is the stored state itself). Also the default SM split of
a context for each lattice size and storage precision."""
import numpy as np
import pytest

from pairs import rel_l2
from paper_2305_18919_gb300 import inputs

pytestmark = pytest.mark.gpu


def test_zero_steps_change_nothing():
    from paper_2305_18919_gb300 import binding
    wl = inputs.scaled_shear(24, 2, 5.0, alpha=(0.01, 0.01, 0.01))
    lat = binding.Lattice.from_workload(wl, precision="fp32")
    lat.step(3)
    f0, q0 = lat.populations(), lat.vertices()
    lat.step(0)
    assert lat.steps_done == 3
    assert np.array_equal(lat.populations(), f0)
    assert np.array_equal(lat.vertices(), q0)
    lat.close()
    b = binding.Batch.from_workloads([wl, wl])
    b.step(2)
    g0 = [c.populations() for c in b.contexts]
    b.step(0)
    assert list(b.status()) == [0, 0]
    for c, g in zip(b.contexts, g0):
        assert np.array_equal(c.populations(), g)
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp16"])
@pytest.mark.parametrize("shape,z_periodic", [((4, 4, 3), False), ((4, 8, 4), True),
                                              ((8, 4, 3), False)])
def test_smallest_lattices(precision, shape, z_periodic):
    import oracle
    from paper_2305_18919_gb300 import binding
    nx, ny, nz = shape
    walls = ((0, 0, 0), (0, 0, 0)) if z_periodic else ((-0.02, 0.01, 0), (0.03, -0.01, 0))
    g = (1e-5, -2e-5, 3e-5 if z_periodic else 0)
    ref = oracle.Simulation(nx, ny, nz, 0.8, 1.0, walls[0], walls[1], g, z_periodic)
    gpu = binding.Lattice(nx, ny, nz, 0.8, 1.0, walls[0], walls[1], g, precision, z_periodic)
    rng = np.random.default_rng(9)
    rho = 1 + rng.uniform(-0.01, 0.01, (nz, ny, nx))
    u = rng.uniform(-0.03, 0.03, (nz, ny, nx, 3))
    ref.init_equilibrium(rho, u)
    gpu.init_equilibrium(rho, u)
    ref.step(25)
    gpu.step(25)
    r0, u0 = ref.fields()
    r1, u1 = gpu.fields()
    tol = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 2 * 2.0 ** -11}[precision]
    fl = slice(None) if z_periodic else slice(1, nz - 1)
    assert rel_l2(u1[fl], u0[fl]) <= tol
    gpu.close()
    ref.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_bare_icosahedron(precision):
    """The coarsest closed mesh (subdivision 0: 12 vertices, 20 faces) in a small shear box."""
    from pairs import make_pair
    wl = inputs.scaled_shear(16, 0, 3.0, alpha=(0.01, 0.01, 0.01))
    assert wl.mesh()[0].shape == (12, 3)
    ref, gpu = make_pair(wl, precision)
    ref.step(60)
    gpu.step(60)
    tol = 1e-11 if precision == "fp64" else 1e-6
    assert np.abs(gpu.vertices() - ref.vertices()).max() <= tol * wl.radius
    gpu.close()
    ref.close()


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
def test_rest_stays_exactly_at_rest(precision):
    """No walls moving, no force, no particle: f = f^eq(rho0, 0) is a fixed point, and the
    shifted populations stay exactly zero through both stream-collide kernels."""
    from paper_2305_18919_gb300 import binding
    lat = binding.Lattice(64, 32, 20, 0.8, precision=precision)
    lat.step(1)
    lat.step(9)
    f = lat.populations()
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    fl = f[:, 1:-1]
    assert np.array_equal(fl, np.broadcast_to(w[:, None, None, None], fl.shape))
    lat.close()


def test_fields_into_device_buffers():
    """iblb_read_fields_device writes the same rho and u as iblb_read_fields, into torch tensors
    on the device, ordered on the context's stream."""
    torch = pytest.importorskip("torch")
    from paper_2305_18919_gb300 import binding
    wl = inputs.scaled_shear(24, 2, 5.0, alpha=(0.01, 0.01, 0.01))
    lat = binding.Lattice.from_workload(wl, precision="fp32")
    lat.step(7)
    rho, u = lat.fields()
    rho_d, u_d = lat.fields_device()
    torch.cuda.synchronize()
    assert rho_d.is_cuda and u_d.shape == u.shape
    assert np.array_equal(rho_d.cpu().numpy(), rho)
    assert np.array_equal(u_d.cpu().numpy(), u)
    lat.close()


@pytest.mark.parametrize("shape, precision, expected", [
    ((256, 256, 256), "fp32", 24),  # 2.5 GB pass: the interface chain fits on 24 SMs
    ((256, 256, 256), "fp16", 40),  # half the pass: the chain needs more SMs
    ((256, 256, 256), "fp64", 0),   # FP64-bound pass: no partition
    ((128, 128, 96), "fp32", 64),   # a short pass leaves the chain as the critical path
    ((32, 32, 32), "fp64", 64),
])
def test_default_interface_partition(shape, precision, expected):
    """The default SM split of iblb_create follows the size of the stream-collide pass
    (2 x 19 x nodes x storage bytes, against 1 GiB) and the storage precision; an explicit
    ib_sms < 0 asks for no partition."""
    from paper_2305_18919_gb300 import binding
    nx, ny, nz = shape
    lat = binding.Lattice(nx, ny, nz, 0.8, precision=precision)
    assert lat.interface_sms() == expected
    lat.close()
    lat = binding.Lattice(nx, ny, nz, 0.8, precision=precision, ib_sms=-1)
    assert lat.interface_sms() == 0
    lat.close()
