"""Pins of the small-deformation shape theory (Sec. II, Eq. evJK) as integrated by
observables.bbr_evolution, against what the paper and the equations fix:

- the steady state reproduces the closed forms of Sec. IV: Eq. deformation for the coated
  droplets and the capsules (Ca on alpha1, resp. alpha3), Eq. deformation_droplet for a pure
  droplet, and Eq. inclination_angle for the droplet's angle;
- at the start the particle is deformed by the flow alone: J = K = 0 gives
  dJ/dt = 5 E / (2 lambda + 3), so D(t) = 5 t / (2 (2 lambda + 3)) + O(t^2) whatever alpha is;
- RK4 converges at fourth order in the time step.
"""
import math

import numpy as np
import pytest

from paper_2305_18919_gb300 import inputs
from paper_2305_18919_gb300 import observables as ob


def _closed_form(alpha, Ca):
    a1, a2, a3 = alpha
    if a1 > 0 and (a2 > 0 or a3 > 0):
        return ob.theory_deformation(alpha, Ca)
    if a1 > 0:
        return ob.theory_deformation_droplet(Ca)
    # capsules: Eq. deformation with Ca = mu R gamma / alpha1 rewritten on alpha3
    return 5.0 * (3 * a2 + 4 * a3) / (8.0 * a3 * (a2 + a3)) * Ca


@pytest.mark.parametrize("cls", list(inputs.ALPHA_CLASSES))
def test_steady_state_reproduces_the_closed_forms(cls):
    alpha = inputs.ALPHA_CLASSES[cls]
    Ca = 0.01  # relaxation rates scale as 1/Ca: dt = 1e-3 keeps RK4 stable for every class
    t, D, _ = ob.bbr_evolution(alpha, Ca, 6.0, dt=1e-3, every=100)
    assert abs(D[-1] - D[-10]) < 1e-9 * Ca     # steady
    # the closed forms are the O(Ca) limit: the O(Ca^2) remainder is below 1e-2 Ca here
    assert abs(D[-1] / _closed_form(alpha, Ca) - 1.0) < 5e-3


def test_droplet_inclination_matches_eq_inclination_angle():
    Ca = 0.01
    _, _, th = ob.bbr_evolution((1, 0, 0), Ca, 6.0, dt=1e-3, every=100)
    assert abs(th[-1] - ob.theory_inclination_droplet(Ca)) < 0.05 * (math.pi / 4 - th[-1])


def test_initial_growth_is_the_affine_deformation():
    for alpha in ((1, 0, 0), (1, 1, 1), (0, 0, 1)):
        # Ca = 1: the material relaxation (rates of order 1/Ca) bends D(t) by < 1e-3 here
        t, D, th = ob.bbr_evolution(alpha, 1.0, 5e-4, dt=1e-4, every=1)
        slope = D[1:6] / t[1:6]
        np.testing.assert_allclose(slope, 5.0 / (2 * (2 + 3)), rtol=2e-3)
        assert abs(th[5] - math.pi / 4) < 1e-3   # stretched along the extension axis


def test_rk4_converges_at_fourth_order():
    alpha, Ca, T = (1, 1, 1), 0.1, 1.0
    ref = ob.bbr_evolution(alpha, Ca, T, dt=1e-4)[1][-1]
    e1 = abs(ob.bbr_evolution(alpha, Ca, T, dt=0.04)[1][-1] - ref)
    e2 = abs(ob.bbr_evolution(alpha, Ca, T, dt=0.02)[1][-1] - ref)
    assert 10.0 < e1 / e2 < 24.0                 # 2^4 = 16
