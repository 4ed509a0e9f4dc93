"""The staged stream-collide kernel (population rows copied into shared memory by a producer
warp, Eqs. 9-10 with pull streaming) against the direct kernel: the same populations bit for bit
on every shape, storage type, buffer depth and warp count, alone and inside the coupled step.
Its agreement with the FP64 oracle is covered by the lattice, precision and interface tests,
which run it by default from the second step on."""
import numpy as np
import pytest

from pairs import rel_l2

pytestmark = pytest.mark.gpu

# (nx, ny, nz, z_periodic): rows of 1, 2 and 4 lattice rows per unit, walls and periodic z,
# units that do not divide evenly among the blocks
SHAPES = [(32, 16, 18, False), (256, 8, 5, False), (24, 20, 7, False), (64, 12, 12, True),
          (8, 12, 8, True), (4, 4, 16, False)]


def _pair(shape, precision, force, seed=11):
    from paper_2305_18919_gb300 import binding
    nx, ny, nz, zp = shape
    walls = ((0, 0, 0), (0, 0, 0)) if zp else ((-0.02, 0.01, 0), (0.03, -0.01, 0))
    g = (1e-5, -2e-5, 3e-5 if zp else 0) if force else (0, 0, 0)
    rng = np.random.default_rng(seed)
    rho = 1 + rng.uniform(-0.01, 0.01, (nz, ny, nx))
    u = rng.uniform(-0.03, 0.03, (nz, ny, nx, 3))
    lats = []
    for kind in ("direct", "staged"):
        lat = binding.Lattice(nx, ny, nz, 0.8, 1.0, walls[0], walls[1], g, precision, zp)
        lat.set_stream_collide(kind)
        lat.init_equilibrium(rho, u)
        lats.append(lat)
    return lats


@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("force", [False, True])
def test_staged_equals_direct(precision, shape, force):
    direct, staged = _pair(shape, precision, force)
    for n in (1, 1, 7):  # the first step reads in place; the staged kernel runs from the second
        direct.step(n)
        staged.step(n)
        np.testing.assert_array_equal(staged.populations(), direct.populations())
    direct.close()
    staged.close()


@pytest.mark.parametrize("stages,warps,rows,nodes", [(2, 1, 0, 0), (3, 5, 1, 0), (8, 8, 4, 4),
                                                     (2, 8, 2, 2), (5, 2, 0, 2), (4, 3, 4, 4),
                                                     (2, 16, 0, 2), (3, 12, 4, 2), (4, 16, 1, 4)])
@pytest.mark.parametrize("precision", ["fp32", "fp16", "bf16"])
def test_stage_depths_and_warps(precision, stages, warps, rows, nodes):
    """Buffer depths, warp counts, unit heights and nodes per lane, including units of one row,
    units whose rows wrap around y (rows of 4 over ny = 20) and more warps than the four-node
    form takes (it keeps 8)."""
    direct, staged = _pair((48, 20, 11, False), precision, True, seed=5)
    staged.set_stream_collide("staged", stages, warps, rows, nodes)
    direct.step(9)
    staged.step(9)
    np.testing.assert_array_equal(staged.populations(), direct.populations())


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_coupled_step_staged_equals_direct(precision):
    """Whole coupled steps (the interface chain overwrites the nodes of the active tiles
    after the full-lattice pass): both kernels give the same populations and vertices."""
    from paper_2305_18919_gb300 import binding, inputs
    wl = inputs.scaled_wetting(32, 24, 3, 6.0, alpha=(1e-3, 0, 1e-3), eps=2e-4, precision="fp64")
    lats = []
    for kind in ("direct", "staged"):
        lat = binding.Lattice.from_workload(wl, precision=precision)
        lat.set_stream_collide(kind)
        lat.step(60)
        lats.append(lat)
    np.testing.assert_array_equal(lats[1].populations(), lats[0].populations())
    np.testing.assert_array_equal(lats[1].vertices(), lats[0].vertices())


def test_staged_full_size_against_direct():
    """The 256^3 shear lattice (FP16 storage) in the launch configuration of the benchmark:
    the staged kernel on the lattice partition reproduces the direct kernel exactly."""
    from paper_2305_18919_gb300 import binding, inputs
    wl = inputs.shear_256_fp32()
    out = []
    for kind in ("direct", "staged"):
        lat = binding.Lattice.from_workload(wl, precision="fp16")
        lat.set_stream_collide(kind)
        lat.step(20)
        r, u = lat.fields()
        out.append((u[::17, ::13, ::11].copy(), lat.vertices()))
        lat.close()
    np.testing.assert_array_equal(out[1][0], out[0][0])
    np.testing.assert_array_equal(out[1][1], out[0][1])
    assert rel_l2(out[1][0], out[0][0]) == 0.0


def test_set_stream_collide_arguments():
    from paper_2305_18919_gb300 import binding
    lat = binding.Lattice(8, 8, 6, 0.8)
    for args in ((3, 0, 0, 0, 0), (-1, 0, 0, 0, 0), (1, 1, 0, 0, 0), (1, 9, 0, 0, 0),
                 (1, 0, -1, 0, 0), (1, 0, 17, 0, 0), (1, 0, 0, 3, 0), (1, 0, 0, 16, 0),
                 (1, 0, 0, -2, 0), (1, 0, 0, 0, 3), (1, 0, 0, 0, 1)):
        with pytest.raises(binding.IBLBError) as e:
            lat._check(lat._L.iblb_set_stream_collide(lat.h, *args))
        assert e.value.code == binding.IBLB_EINVAL
    lat.set_stream_collide("direct", 2, 8, 8, 2)
    lat.set_stream_collide("staged")
    lat.step(3)
    lat.close()


@pytest.mark.parametrize("precision,shape,kind,expected", [
    ("fp16", (64, 8, 6), "auto", True), ("bf16", (64, 8, 6), "auto", True),
    ("fp32", (64, 8, 6), "auto", False), ("fp64", (64, 8, 6), "auto", False),
    ("fp32", (64, 8, 6), "staged", True), ("fp64", (64, 8, 6), "staged", False),
    ("fp16", (132, 4, 7), "staged", False), ("fp16", (64, 8, 6), "direct", False),
    ("fp32", (4, 4, 6), "staged", True), ("fp16", (4, 4, 6), "staged", False)])
def test_kernel_choice(precision, shape, kind, expected):
    """AUTO takes the staged kernel for 16-bit storage; rows that are not a whole number of
    16-byte blocks (132 or 4 values of 2 bytes) and FP64 always take the direct kernel."""
    from paper_2305_18919_gb300 import binding
    lat = binding.Lattice(*shape, 0.8, precision=precision)
    lat.set_stream_collide(kind)
    assert lat.stream_collide_staged() is expected
    lat.step(2)
    lat.close()


@pytest.mark.parametrize("precision", ["fp16", "fp32"])
def test_wait_limit_runs_out_and_context_recovers(precision):
    """A wait limit of 0 (one non-blocking test) makes the staged kernel's first wait for a
    buffer run out (its copies have not landed yet): the blocks stop, iblb_step reports the
    timeout from the health word, and the same context then reproduces a fresh context's run
    exactly."""
    from paper_2305_18919_gb300 import binding
    shape = (64, 64, 34)
    rng = np.random.default_rng(3)
    rho = 1 + rng.uniform(-0.01, 0.01, shape[::-1])
    u = rng.uniform(-0.03, 0.03, shape[::-1] + (3,))
    lat = binding.Lattice(*shape, 0.8, 1.0, (-0.02, 0, 0), (0.02, 0, 0), precision=precision)
    lat.set_stream_collide("staged", 4, 8, 1)  # units of one row: many units per block
    lat.init_equilibrium(rho, u)
    lat.step(1)  # the first step reads in place with the direct kernel
    assert lat.stream_collide_staged()
    lat.set_stage_wait_limit(0)
    with pytest.raises(binding.IBLBError) as e:
        lat.step(2)
    assert e.value.code == binding.IBLB_ETIMEOUT
    assert "bounded wait" in str(e.value)
    with pytest.raises(binding.IBLBError):
        lat.set_stage_wait_limit(-1)
    lat.set_stage_wait_limit(10**9)
    lat.init_equilibrium(rho, u)
    lat.step(6)
    ref = binding.Lattice(*shape, 0.8, 1.0, (-0.02, 0, 0), (0.02, 0, 0), precision=precision)
    ref.set_stream_collide("staged", 4, 8, 1)
    ref.init_equilibrium(rho, u)
    ref.step(6)
    np.testing.assert_array_equal(lat.populations(), ref.populations())
    lat.close()
    ref.close()
