"""The reference gradients (oracle/adjoint.py: the oracle's step restated in float64 PyTorch
and differentiated by autograd) pinned to the C oracle: same trajectory, and gradients equal
to central finite differences of the C oracle's own runs."""
import copy

import numpy as np
import pytest

from paper_2305_18919_gb300 import inputs

torch = pytest.importorskip("torch")


def _case():
    wl = inputs.scaled_wetting(16, 14, 2, 4.0, alpha=(2e-3, 1e-3, 2e-3), eps=1e-3)
    wl.wall_u_bottom = (-0.005, 0.002, 0.0)
    wl.wall_u_top = (0.004, 0.0, 0.0)
    return wl


def objective(q):
    """A smooth observable touching every direction: height of the centroid plus second
    moments of the shape (works on numpy arrays and torch tensors)."""
    c = q.mean(0)
    return ((q[:, 2] - c[2]) ** 2).mean() + 0.3 * ((q[:, 0] - c[0]) ** 2).mean() + c[2]


def test_torch_restatement_follows_the_c_oracle(oracle_mod):
    from oracle import adjoint as oa
    wl = _case()
    sim = oracle_mod.Simulation.from_workload(wl)
    sim.step(15)
    q0, f0 = sim.vertices(), sim.populations()
    sim.close()
    ts = oa.from_workload(wl)
    f, q = ts.run(15, torch.tensor(wl.alpha, dtype=torch.float64),
                  torch.tensor(wl.eps, dtype=torch.float64))
    assert np.abs(q.detach().numpy() - q0).max() < 1e-12
    assert np.abs(f.detach().numpy() - f0).max() < 1e-13


def test_autograd_gradient_equals_oracle_finite_differences(oracle_mod):
    from oracle import adjoint as oa
    wl = _case()
    N = 30
    _, g, _ = oa.gradient(wl, N, objective)

    def J(params):
        w = copy.deepcopy(wl)
        w.alpha, w.eps = tuple(params[:3]), params[3]
        s = oracle_mod.Simulation.from_workload(w)
        s.step(N)
        q = s.vertices()
        s.close()
        return float(objective(q))

    p0 = np.array(list(wl.alpha) + [wl.eps])
    for k in range(4):
        h = 1e-3 * p0[k]  # central differences: O(h^2) truncation, far above rounding
        pp, pm = p0.copy(), p0.copy()
        pp[k] += h
        pm[k] -= h
        fd = (J(pp) - J(pm)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * abs(fd)
