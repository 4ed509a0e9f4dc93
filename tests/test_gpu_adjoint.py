"""The discrete adjoint on the GPU (iblb_adjoint_*, FP64 and FP32 forward runs) against the reference gradients of
oracle/adjoint.py (the oracle's step restated in float64 PyTorch and differentiated by
autograd, itself pinned to finite differences of the C oracle), and against central finite
differences of the GPU's own forward runs on a larger box."""
import copy

import numpy as np
import pytest

from paper_2305_18919_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def objective(q):
    c = q.mean(0)
    return ((q[:, 2] - c[2]) ** 2).mean() + 0.3 * ((q[:, 0] - c[0]) ** 2).mean() + c[2]


def objective_grad(q):
    qt = torch.tensor(q, dtype=torch.float64, requires_grad=True)
    (g,) = torch.autograd.grad(objective(qt), qt)
    return g.numpy()


def _small():
    wl = inputs.scaled_wetting(16, 14, 2, 4.0, alpha=(2e-3, 1e-3, 2e-3), eps=1e-3,
                               precision="fp64")
    wl.wall_u_bottom = (-0.005, 0.002, 0.0)
    wl.wall_u_top = (0.004, 0.0, 0.0)
    return wl


def _gpu_gradient(wl, nsteps, every):
    from paper_2305_18919_gb300 import binding
    lat = binding.Lattice.from_workload(wl, precision="fp64")
    lat.adjoint_record(nsteps, every)
    q = lat.vertices()
    g = lat.adjoint_gradient(objective_grad(q))
    q_after = lat.vertices()
    lat.close()
    return g, q, q_after


@pytest.mark.parametrize("every", [30, 7, 1])
def test_gpu_adjoint_equals_reference_gradients(every):
    from oracle import adjoint as oa
    wl = _small()
    _, g_ref, q_ref = oa.gradient(wl, 30, objective)
    g, q, q_after = _gpu_gradient(wl, 30, every)
    assert np.abs(q - q_ref).max() < 1e-11           # the same trajectory
    assert np.array_equal(q_after, q)                # the context is back at the end
    np.testing.assert_allclose(g, g_ref, rtol=1e-7, atol=1e-12 * np.abs(g_ref).max())


def test_gpu_adjoint_equals_finite_differences_of_gpu_runs():
    from paper_2305_18919_gb300 import binding
    wl = inputs.scaled_wetting(32, 24, 3, 6.0, alpha=(4e-3, 2e-3, 1e-3), eps=5e-4,
                               precision="fp64")
    N = 120
    g, _, _ = _gpu_gradient(wl, N, 40)

    def J(params):
        w = copy.deepcopy(wl)
        w.alpha, w.eps = tuple(params[:3]), params[3]
        lat = binding.Lattice.from_workload(w, precision="fp64")
        lat.step(N)
        q = lat.vertices()
        lat.close()
        return float(objective(q))

    p0 = np.array(list(wl.alpha) + [wl.eps])
    for k in range(4):
        h = 1e-3 * p0[k]
        pp, pm = p0.copy(), p0.copy()
        pp[k] += h
        pm[k] -= h
        fd = (J(pp) - J(pm)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * abs(fd)


def test_adjoint_rejects_what_it_cannot_do():
    from paper_2305_18919_gb300 import binding
    wl = _small()
    for precision in ("fp16", "bf16"):  # 16-bit storage has no adjoint
        lat = binding.Lattice.from_workload(wl, precision=precision)
        with pytest.raises(binding.IBLBError) as e:
            lat.adjoint_record(5, 5)
        assert e.value.code == binding.IBLB_EINVAL
        lat.close()
    lat = binding.Lattice.from_workload(wl, precision="fp64")
    with pytest.raises(binding.IBLBError):
        lat.adjoint_gradient(np.zeros((lat.nv, 3)))  # nothing recorded
    lat.close()


def _masked_fd(wl, N, obs, grad, select):
    """Central differences of obs(q_N) over GPU runs, with the observable's vertex or face
    selection held at the base run's."""
    from paper_2305_18919_gb300 import binding

    def J(params):
        w = copy.deepcopy(wl)
        w.alpha, w.eps = tuple(params[:3]), params[3]
        lat = binding.Lattice.from_workload(w, precision="fp64")
        lat.step(N)
        q = torch.tensor(lat.vertices())
        lat.close()
        return float(obs(q, select))

    p0 = np.array(list(wl.alpha) + [wl.eps])
    for k in range(4):
        h = 1e-3 * max(abs(p0[k]), 1e-3)  # a parameter may be 0 (alpha2 of this class)
        pp, pm = p0.copy(), p0.copy()
        pp[k] += h
        pm[k] -= h
        fd = (J(pp) - J(pm)) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-4 * abs(fd) + 1e-9 * abs(grad).max()


def test_autograd_function_contact_angle_and_wetted_radius():
    """torch.autograd through the adjoint (paper_2305_18919_gb300.adjoint.run) for the apparent
    contact angle and the wetted radius, against central differences of GPU runs."""
    from paper_2305_18919_gb300 import adjoint as ad
    wl = inputs.scaled_wetting(32, 24, 3, 6.0, alpha=(2e-3, 0.0, 2e-3), eps=2e-3,
                               precision="fp64")
    _, faces = wl.mesh()
    N = 120
    theta = torch.tensor(list(wl.alpha) + [wl.eps], dtype=torch.float64, requires_grad=True)
    q = ad.run(theta, wl, N, every=40)
    # the angle with a plane through the lower half of the particle: the droplet has not
    # spread yet after 120 steps, so the circle does not reach the wall plane itself
    z_ref = wl.centre[2] - 0.5 * wl.radius
    sel_v = ad.contact_angle_selection(q, faces, z_wall=z_ref, exclude=0.0)
    theta_deg = ad.contact_angle(q, faces, z_wall=z_ref, select=sel_v)
    assert 90 < float(theta_deg.detach()) < 180
    (g_angle,) = torch.autograd.grad(theta_deg, theta)
    q = ad.run(theta, wl, N, every=40)
    gz = (q[faces[:, 0], 2] + q[faces[:, 1], 2] + q[faces[:, 2], 2]).detach() / 3
    sel_f = torch.as_tensor(gz - 0.5 < 1.0)
    r = ad.wetted_radius(q, faces, select=sel_f)
    assert float(r.detach()) > 0
    (g_r,) = torch.autograd.grad(r, theta)
    _masked_fd(wl, N, lambda qq, s: ad.contact_angle(qq, faces, z_wall=z_ref, select=s),
               g_angle.numpy(), sel_v)
    _masked_fd(wl, N, lambda qq, s: ad.wetted_radius(qq, faces, select=s), g_r.numpy(), sel_f)


def test_adjoint_24_cubed_200_steps_vs_fp64_reference():
    """The check the 64^3 adjoint workload names: a 24^3, subdivision-2 copy of it (the same
    particle class, alpha and wall strength, R scaled by 24/64) over 200 steps, the GPU adjoint
    against the FP64 CPU reference gradient."""
    from oracle import adjoint as oa
    base = inputs.adjoint_wetting_64()
    wl = inputs.scaled_wetting(24, 24, 2, base.radius * 24 / 64, alpha=base.alpha, eps=base.eps,
                               precision="fp64")
    _, g_ref, q_ref = oa.gradient(wl, 200, objective)
    g, q, _ = _gpu_gradient(wl, 200, 100)
    assert np.abs(q - q_ref).max() < 1e-10
    np.testing.assert_allclose(g, g_ref, rtol=1e-6, atol=1e-11 * np.abs(g_ref).max())


def test_full_size_adjoint_vs_finite_differences():
    """The 64^3 adjoint workload itself (subdivision 4, 5000 steps, a state copy every 100):
    the gradient of the wetted radius through torch.autograd against central differences of
    full GPU runs, with the face selection held at the base run's."""
    from paper_2305_18919_gb300 import adjoint as ad
    wl = inputs.adjoint_wetting_64()
    _, faces = wl.mesh()
    N = 5000
    theta = torch.tensor(list(wl.alpha) + [wl.eps], dtype=torch.float64, requires_grad=True)
    q = ad.run(theta, wl, N, every=100)
    gz = (q[faces[:, 0], 2] + q[faces[:, 1], 2] + q[faces[:, 2], 2]).detach() / 3
    sel_f = torch.as_tensor(gz - 0.5 < 1.0)
    r = ad.wetted_radius(q, faces, select=sel_f)
    (g_r,) = torch.autograd.grad(r, theta)
    _masked_fd(wl, N, lambda qq, s: ad.wetted_radius(qq, faces, select=s), g_r.numpy(), sel_f)


def _gradient_with(wl, nsteps, every, precision):
    from paper_2305_18919_gb300 import binding
    lat = binding.Lattice.from_workload(wl, precision=precision)
    lat.adjoint_record(nsteps, every)
    q = lat.vertices()
    g = lat.adjoint_gradient(objective_grad(q))
    lat.close()
    return g, q


@pytest.mark.parametrize("every", [30, 7])
def test_fp32_forward_adjoint(every):
    """With FP32 storage the forward run (and its recomputation) is FP32 and the reverse pass
    linearises the double step about that trajectory: the gradient is the FP64 one to within
    what the FP32 trajectory's rounding moves it, and a second call recomputes the same
    trajectory (the reverse pass's dense spreading sums with atomics, so the two gradients agree
    to rounding, not bit for bit)."""
    from paper_2305_18919_gb300 import binding
    wl = inputs.scaled_wetting(32, 24, 3, 6.0, alpha=(4e-3, 2e-3, 1e-3), eps=5e-4,
                               precision="fp64")
    g64, q64 = _gradient_with(wl, 120, every, "fp64")
    lat = binding.Lattice.from_workload(wl, precision="fp32")
    lat.adjoint_record(120, every)
    q32 = lat.vertices()
    g32 = lat.adjoint_gradient(objective_grad(q32))
    g32b = lat.adjoint_gradient(objective_grad(q32))
    lat.close()
    np.testing.assert_allclose(g32b, g32, rtol=1e-12)
    assert np.abs(q32 - q64).max() < 1e-5 * wl.radius
    # measured on GB300: 2e-8 .. 2.5e-6 relative over these 120 steps
    np.testing.assert_allclose(g32, g64, rtol=2e-5)
