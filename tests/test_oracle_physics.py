"""Whole-step pins of the oracle against the paper's small-deformation shear-flow theory
(Sec. IV): steady Taylor deformation of a pure droplet (Eq. 22), of a rigidly coated
droplet (Eq. 21), linearity of D in Ca, and the Chaffey-Brenner inclination (Eq. 23).

Workload: the 32^3 shear box (walls at -/+0.01, tau = 1, R = 6, subdivision 3), started
from the linear Couette profile. At R/H = 0.2 wall confinement raises D above the
unbounded theory; the absolute bound is therefore one-sided and loose, while the ratios
(which confinement affects alike) are tight.
"""
import concurrent.futures as cf
import math

import numpy as np
import pytest

from observables import taylor_deformation
from pairs import shear_profile
from paper_2305_18919_gb300 import inputs


def _run(alpha, steps):
    import oracle
    wl = inputs.shear_32_fp64()
    wl.alpha = alpha
    s = oracle.Simulation.from_workload(wl)
    s.init_equilibrium(*shear_profile(wl))
    s.step(steps)
    v, f = wl.mesh()
    D, theta = taylor_deformation(s.vertices(), f)
    V, V0 = s.volume()
    s.close()
    return D, theta, V / V0 - 1


@pytest.fixture(scope="module")
def shear_results(oracle_mod):
    jobs = {"droplet": ((0.01, 0, 0), 1000), "droplet_stiff": ((0.02, 0, 0), 600),
            "rigid": ((0.01, 0.01, 0.01), 600)}
    with cf.ThreadPoolExecutor(3) as ex:  # ctypes calls release the GIL
        futs = {k: ex.submit(_run, *v) for k, v in jobs.items()}
        return {k: f.result() for k, f in futs.items()}


def _ca(alpha1):
    wl = inputs.shear_32_fp64()
    mu = (wl.tau - 0.5) / 3.0
    gamma = (wl.wall_u_top[0] - wl.wall_u_bottom[0]) / (wl.nz - 2)
    return mu * wl.radius * gamma / alpha1


@pytest.mark.slow
def test_droplet_deformation_and_inclination(shear_results):
    D, theta, dV = shear_results["droplet"]
    Ca = _ca(0.01)
    D_theory = (19 + 16) / (16 + 16) * Ca               # Eq. 22, lambda = 1
    theta_theory = math.pi / 4 - (35 * 5) / (80 * 2) * Ca  # Eq. 23, lambda = 1
    assert D_theory < D < 1.4 * D_theory
    assert abs(theta - theta_theory) < math.radians(1.5)
    assert abs(dV) < 5e-3


@pytest.mark.slow
def test_deformation_linear_in_capillary_number(shear_results):
    D1 = shear_results["droplet"][0]
    D2 = shear_results["droplet_stiff"][0]
    assert abs(D2 / D1 - 0.5) < 0.04


@pytest.mark.slow
def test_rigidly_coated_to_droplet_ratio(shear_results):
    """Eq. 21 with alpha = abar(1,1,1) gives D = 35/48 Ca; Eq. 22 gives 35/32 Ca: ratio 2/3."""
    a1 = a2 = a3 = 1.0
    coef = 5 * a1 * (3 * a2 + 4 * a3) / (4 * (3 * a1 * a2 + 5 * a1 * a3 + 2 * a2 * a3 + 2 * a3 ** 2))
    assert abs(coef - 35 / 48) < 1e-15
    ratio = shear_results["rigid"][0] / shear_results["droplet"][0]
    assert abs(ratio / (coef / (35 / 32)) - 1) < 0.1


def test_capsule_at_rest_stays_at_rest(oracle_mod):
    """alpha1 = 0 and the undeformed shape: every nodal force vanishes, so a quiescent
    fluid and the mesh stay exactly at rest."""
    wl = inputs.scaled_wetting(16, 16, 2, 4.0, (0.0, 0.01, 0.01), 0.0)
    wl.wall_force_on = 0
    s = oracle_mod.Simulation.from_workload(wl)
    q0 = s.vertices()
    s.step(20)
    _, u = s.fields()
    assert np.abs(u).max() < 1e-15
    np.testing.assert_allclose(s.vertices(), q0, rtol=0, atol=1e-15)


def test_periodic_box_momentum_is_conserved_with_a_particle(oracle_mod):
    """Strain and volume forces have zero sum, and spreading preserves the sum, so a fully
    periodic box with a deformed particle keeps its total momentum."""
    wl = inputs.scaled_wetting(16, 16, 2, 4.0, (0.01, 0.01, 0.01), 0.0, lift=3.0)
    wl.wall_force_on = 0
    s = oracle_mod.Simulation.from_workload(wl, z_periodic=True)
    s.set_vertices(inputs.perturb(wl.mesh()[0], 0.3, seed=3))
    c, _, _ = oracle_mod.lattice_table()
    P0 = np.einsum("izyx,ia->a", s.populations(), c)
    m0 = s.populations().sum()
    phi, _ = s.forces()
    impulse = np.abs(phi).sum() * 10  # scale of the momentum the forces move in 10 steps
    s.step(10)
    P1 = np.einsum("izyx,ia->a", s.populations(), c)
    assert np.abs(P1 - P0).max() < 1e-10 * impulse
    assert abs(s.populations().sum() - m0) < 1e-11 * m0
