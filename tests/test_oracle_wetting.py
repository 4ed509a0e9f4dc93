"""Static wetting pins of the oracle against Sec. V.B: the contact angle reached against the
empirical law of Eq. 25 with the constants of Table I (tests/golden/paper_constants.json),
its limit for a vanishing wall attraction, its decrease with eps/alpha_bar, and the order of
the model classes.

Workload: a 32 x 32 x 24 box with walls at z = 0 and 23, a particle of R = 6 (icosphere
subdivision 3) resting at the Lennard-Jones minimum above the bottom wall (reading R12),
alpha_bar = 3e-3 and eps = (eps/alpha_bar) alpha_bar, 12000 steps. Once the fluid is at rest
the nodal forces depend on eps and alpha only through eps/alpha_bar; alpha_bar = 3e-3
instead of the paper's 1e-4 makes the spreading 30 times faster (the volume penalty keeps
kV = 1). The angle is the observables module's circle fit of a central slab of vertices cut
by the wall plane z = 0.5 (Sec. V.B, App. A; reading G16), 180 degrees when the fitted circle
does not reach the wall.

What the pins can and cannot hold. Eq. 25 is a fit of the paper's own runs (N_f = 16820, R
not stated for the wetting runs). The wall force of Eq. 19 acts per face (reading R7), so the
adhesion grows with the number of faces in the contact patch, and a membrane without shear
resistance lets vertices drift into that patch: the angle keeps creeping down after the
shape has settled (the paper reports the node accumulation at the contact area as its
model's limit). Measured here after 12000 steps: 95.9 (droplet) and 91.9 degrees (softly
coated) at eps/alpha_bar = 3 against 107.3 and 98.3 from Table I, settled to within 1.5 and
0.4 degrees over the last 2400 steps; 109.0 degrees at eps/alpha_bar = 1 against 126.6, still
creeping down by about 3 degrees per 2400 steps; 180 degrees at 0.05 against 168.0. The
oracle wets more than the fit, by 6 to 18 degrees where it wets at all; the bound below is
that one-sided 25 degrees, not the 10 degrees a mesh-independent law would allow.
"""
import concurrent.futures as cf
import json
import math
import os

import numpy as np
import pytest
import torch

from paper_2305_18919_gb300 import inputs
from paper_2305_18919_gb300 import observables as ob

HERE = os.path.dirname(os.path.abspath(__file__))
STEPS, SAMPLE, ABAR = 12000, 500, 3e-3


def _table_I():
    with open(os.path.join(HERE, "golden", "paper_constants.json")) as fh:
        return json.load(fh)


def eq25_theta(cls, x):
    """theta_eq of Eq. 25, cos theta = a atan(b (x - c)) - d, with the Table I constants."""
    k = _table_I()["table_I"][cls]
    c = k["a"] * math.atan(k["b"] * (x - k["c"])) - k["d"]
    return math.degrees(math.acos(max(-1.0, min(1.0, c))))


def _theta(q, faces):
    th = float(ob.contact_angle(torch.tensor(q), faces, z_wall=0.5, exclude=1.0))
    return 180.0 if math.isnan(th) else th  # the fitted circle stays above the wall


def _run(cls, x, threads):
    import oracle
    oracle.set_threads(threads)
    a = tuple(ABAR * v for v in inputs.ALPHA_CLASSES[cls])
    wl = inputs.scaled_wetting(32, 24, 3, 6.0, a, x * ABAR)
    wl.centre = (16.0, 16.0, wl.centre[2])
    s = oracle.Simulation.from_workload(wl)
    _, faces = wl.mesh()
    th = []
    for k in range(STEPS // SAMPLE):
        s.step(SAMPLE)
        if (k + 1) * SAMPLE >= 0.8 * STEPS:
            th.append(_theta(s.vertices(), faces))
    V, V0 = s.volume()
    s.close()
    return np.array(th), V / V0 - 1


@pytest.fixture(scope="module")
def wetting(oracle_mod):
    jobs = {("droplet", 3.0), ("softly_coated", 3.0), ("softly_coated", 1.0),
            ("softly_coated", 0.05)}
    threads = max(1, (os.cpu_count() or 1) // len(jobs))
    with cf.ThreadPoolExecutor(len(jobs)) as ex:  # ctypes calls release the GIL
        futs = {j: ex.submit(_run, *j, threads) for j in jobs}
        return {j: f.result() for j, f in futs.items()}


def test_eq25_constants_are_the_papers():
    """Spot values of Eq. 25 with Table I, worked by hand: the softly coated fit at
    eps/alpha_bar = 2 gives cos theta = 0.87 atan(1) - 1 = -0.3167, theta = 108.5 degrees;
    all pre-stressed fits tend to 180 degrees as eps -> 0 (c = 0, d = 1)."""
    assert abs(eq25_theta("softly_coated", 2.0) - 108.47) < 0.01
    for cls in ("droplet", "softly_coated", "rigidly_coated"):
        assert eq25_theta(cls, 0.0) == 180.0


@pytest.mark.slow
@pytest.mark.parametrize("cls", ["droplet", "softly_coated"])
def test_angle_settles(wetting, cls):
    th, dV = wetting[(cls, 3.0)]
    assert np.ptp(th) < 2.0                      # over the last 20 % of the run
    assert abs(dV) < 0.02


@pytest.mark.slow
@pytest.mark.parametrize("cls,x", [("droplet", 3.0), ("softly_coated", 3.0), ("softly_coated", 1.0)])
def test_angle_reached_against_eq25(wetting, cls, x):
    th, _ = wetting[(cls, x)]
    assert 0.0 < eq25_theta(cls, x) - th[-1] < 25.0


@pytest.mark.slow
def test_vanishing_attraction_does_not_wet(wetting):
    """theta -> 180 degrees as eps -> 0 (Table I: c = 0, d = 1 for the pre-stressed classes)."""
    th, _ = wetting[("softly_coated", 0.05)]
    assert th[-1] > 165.0


@pytest.mark.slow
def test_angle_decreases_with_the_attraction_and_the_coated_particle_wets_more(wetting):
    th = {x: wetting[("softly_coated", x)][0][-1] for x in (0.05, 1.0, 3.0)}
    assert th[0.05] > th[1.0] > th[3.0]
    # Table I orders the classes the same way at every eps/alpha_bar > 0
    assert eq25_theta("softly_coated", 3.0) < eq25_theta("droplet", 3.0)
    assert wetting[("softly_coated", 3.0)][0][-1] < wetting[("droplet", 3.0)][0][-1]
