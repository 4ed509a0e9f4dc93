"""Spreading when a tile's bucket spills (Eq. 13 on a mesh much finer than the lattice).

Each 4x4x4 source tile keeps up to 64 of the vertices whose stencil base node it holds in a
bucket; which 64 depends on the order of the binning atomics. A tile with more vertices adds
all of them in increasing vertex index instead, so the force field does not depend on that
order. An icosphere of subdivision 5 at R = 6 (10242 vertices, about 23 per unit area) puts
hundreds of vertex bases into each tile the surface crosses. The tests check the spread field
and three coupled steps against the oracle, and that two runs give the same bits (the
save/load round trip, the batched ensemble and the adjoint's recomputation all rely on it).
"""
import numpy as np
import pytest

from pairs import make_pair, rel_l2
from paper_2305_18919_gb300 import inputs

pytestmark = pytest.mark.gpu

# FP64: 1e-11 rather than the 1e-12 of the coarser meshes. This mesh's field sums ~400 vertex
# forces per node (the spread is 15x ill-conditioned: sum |w phi| / |sum w phi|), and the
# oracle's volume force rests on V - V0, a difference of two sums over 20480 tetrahedra that
# keeps about 11 digits at this 1.5 % dilation; measured 1.4e-12 (field) and 2.0e-12 (u after
# 3 steps). A vertex added twice or left out would show at about 1e-4.
TOL = {"fp64": 1e-11, "fp32": 2e-6}


def _dense(precision, lift=2.0):
    a = tuple(0.01 * x for x in inputs.ALPHA_CLASSES["softly_coated"])
    return inputs.scaled_wetting(24, 20, 5, 6.0, a, 0.5 * 0.01, precision=precision, lift=lift)


def _deformed(wl, seed):
    """Random vertex noise plus a 0.5 % dilation about the centre. The noise alone leaves the
    volume within 3e-5 of V0, where the oracle's V - V0 (a difference of two sums of 20480
    tetrahedra) keeps only about 6 digits: the dilation keeps that difference well conditioned
    for the FP64 comparison."""
    v, _ = wl.mesh()
    c = v.mean(0)
    return c + 1.005 * (inputs.perturb(v, 0.05, seed=seed) - c)


def _bases_per_tile(q):
    base = np.floor(q).astype(int) - 1
    tiles = base // 4
    _, counts = np.unique(tiles, axis=0, return_counts=True)
    return counts


def test_the_workload_spills():
    wl = _dense("fp32")
    assert _bases_per_tile(wl.mesh()[0]).max() > 4 * 64


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_spilled_force_field_matches_oracle(precision):
    wl = _dense(precision)
    ref, gpu = make_pair(wl, precision)
    q = _deformed(wl, 21)
    ref.set_vertices(q)
    gpu.set_vertices(q)
    F_ref = ref.force_field()
    F = gpu.force_field()
    assert rel_l2(F, F_ref) < TOL[precision]
    phi = gpu.forces()
    scale = np.abs(phi).sum() * (1e-12 if precision == "fp64" else 2e-6)
    np.testing.assert_allclose(F.sum((0, 1, 2)), phi.sum(0), rtol=0, atol=scale)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_spilled_steps_match_oracle_and_repeat_bit_for_bit(precision):
    wl = _dense(precision)
    ref, gpu = make_pair(wl, precision)
    _, gpu2 = make_pair(wl, precision)
    q = _deformed(wl, 22)
    for s in (ref, gpu, gpu2):
        s.set_vertices(q)
    for _ in range(3):
        ref.step(1)
        gpu.step(1)
        gpu2.step(1)
        assert rel_l2(gpu.vertex_velocities(), ref.vertex_velocities()) < (
            1e-11 if precision == "fp64" else 1e-5)
        _, u0 = ref.fields()
        _, u1 = gpu.fields()
        assert rel_l2(u1, u0) < (1e-11 if precision == "fp64" else 1e-5)
    # a second context on the same inputs: identical bits (no dependence on atomic order)
    assert np.array_equal(gpu.vertices(), gpu2.vertices())
    assert np.array_equal(gpu.populations(), gpu2.populations())
    assert np.array_equal(gpu.force_field(), gpu2.force_field())
    gpu.close()
    gpu2.close()
