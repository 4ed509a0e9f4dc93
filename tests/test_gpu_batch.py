"""The batched ensemble (iblb_batch_*): independent contexts of different sizes and
precisions advanced together, each kernel of a step one launch over all instances. Every
instance must end bit for bit where the same context stepped alone ends, whatever the step
count (fresh first step, pairs of batched steps, odd tail), the tuned launch shape or a reconfiguration between
calls; a failing instance is reported by index."""
import numpy as np
import pytest

from paper_2305_18919_gb300 import inputs

pytestmark = pytest.mark.gpu


def _small_ensemble():
    return [inputs.scaled_wetting(32, 24, 2, 5.0, alpha=(2e-3, 0, 2e-3), eps=1e-3),
            inputs.scaled_shear(24, 3, 6.0, alpha=(0.01, 0.01, 0.01)),
            inputs.scaled_wetting(40, 28, 3, 8.0, alpha=(5e-3, 0, 0), eps=2e-3)]


def _alone(wl, precision, steps, alpha=None):
    from paper_2305_18919_gb300 import binding
    lat = binding.Lattice.from_workload(wl, precision=precision, ib_sms=-1)
    lat.step(steps[0])
    if alpha is not None:
        lat.set_interface(alpha, wl.kV, wl.eps, wl.xi, wl.wall_force_on, wl.volume_force_on)
    for k in steps[1:]:
        lat.step(k)
    out = lat.vertices(), lat.fields()
    lat.close()
    return out


def _same(lat, ref):
    q, (rho, u) = ref
    assert np.array_equal(lat.vertices(), q)
    r1, u1 = lat.fields()
    assert np.array_equal(r1, rho) and np.array_equal(u1, u)


@pytest.mark.parametrize("steps", [1, 2, 7])
def test_batch_equals_contexts_stepped_alone(steps):
    from paper_2305_18919_gb300 import binding
    wls = _small_ensemble()
    b = binding.Batch.from_workloads(wls)
    b.step(steps)
    assert list(b.status()) == [0, 0, 0]
    for lat, wl in zip(b.contexts, wls):
        assert lat.steps_done == steps
        _same(lat, _alone(wl, "fp32", [steps]))
    b.close()


def test_batch_mixed_precisions_and_repeated_calls():
    from paper_2305_18919_gb300 import binding
    wls = _small_ensemble()
    precs = ["fp16", "fp32", "fp64"]
    b = binding.Batch([binding.workload_desc(wl, p) for wl, p in zip(wls, precs)])
    for lat, wl in zip(b.contexts, wls):
        v, f = wl.mesh()
        lat.add_mesh(v, f)
        lat.set_interface(wl.alpha, wl.kV, wl.eps, wl.xi, wl.wall_force_on, wl.volume_force_on)
    for k in (5, 4, 3):  # batched pairs across calls, tails of one step
        b.step(k)
    for lat, wl, p in zip(b.contexts, wls, precs):
        _same(lat, _alone(wl, p, [12]))
    b.close()


def test_tuned_launch_shape_keeps_results():
    from paper_2305_18919_gb300 import binding
    wls = _small_ensemble()
    b = binding.Batch.from_workloads(wls)
    rows = b.tune(trials=3)
    assert all(r in (1, 2, 4) for r in rows)
    b.step(6)
    for lat, wl in zip(b.contexts, wls):
        _same(lat, _alone(wl, "fp32", [6]))
    b.close()


def test_reconfiguration_between_calls_is_recorded():
    from paper_2305_18919_gb300 import binding
    wls = _small_ensemble()
    b = binding.Batch.from_workloads(wls)
    b.step(4)
    wl1 = wls[1]
    new_alpha = (0.02, 0.0, 0.005)
    b.contexts[1].set_interface(new_alpha, wl1.kV, wl1.eps, wl1.xi, wl1.wall_force_on,
                                wl1.volume_force_on)
    b.step(4)
    _same(b.contexts[1], _alone(wl1, "fp32", [4, 4], alpha=new_alpha))
    _same(b.contexts[0], _alone(wls[0], "fp32", [8]))
    b.close()


def test_failing_instance_is_reported_by_index():
    from paper_2305_18919_gb300 import binding
    wls = _small_ensemble()
    b = binding.Batch.from_workloads(wls)
    wl = wls[2]
    v, _ = wl.mesh()
    # a strongly compressed interface drives |V/V0 - 1| past 5% in that instance only
    b.contexts[2].set_vertices(np.asarray(wl.centre) + (v - np.asarray(wl.centre)) * 0.9)
    with pytest.raises(binding.IBLBError) as e:
        b.step(3)
    assert e.value.code == binding.IBLB_EUNSTABLE
    assert list(b.status()) == [0, 0, binding.IBLB_EUNSTABLE]
    b.close()


def test_lattice_only_instances_beside_meshes():
    """Contexts without a mesh take only the stream-collide launches of the batched step;
    they and the mesh contexts beside them end as when stepped alone."""
    from paper_2305_18919_gb300 import binding
    wls = _small_ensemble()
    descs = [binding.workload_desc(wl, "fp32") for wl in wls]
    descs.insert(1, binding.lattice_desc(16, 12, 10, 0.9, 1.0, (-0.01, 0, 0), (0.02, 0, 0),
                                         (1e-5, 0, 0), "fp32", False, -1))
    b = binding.Batch(descs)
    meshed = [b.contexts[0], b.contexts[2], b.contexts[3]]
    for lat, wl in zip(meshed, wls):
        v, f = wl.mesh()
        lat.add_mesh(v, f)
        lat.set_interface(wl.alpha, wl.kV, wl.eps, wl.xi, wl.wall_force_on, wl.volume_force_on)
    b.step(6)
    assert list(b.status()) == [0, 0, 0, 0]
    for lat, wl in zip(meshed, wls):
        _same(lat, _alone(wl, "fp32", [6]))
    ref = binding.Lattice(16, 12, 10, 0.9, 1.0, (-0.01, 0, 0), (0.02, 0, 0), (1e-5, 0, 0),
                          "fp32", False, None, -1)
    ref.step(6)
    assert np.array_equal(b.contexts[1].populations(), ref.populations())
    ref.close()
    b.close()


def test_more_instances_than_one_launch_holds():
    """260 contexts of one precision: the batched launches split them into groups of at most
    256; every context still ends as when stepped alone."""
    from paper_2305_18919_gb300 import binding
    rng = np.random.default_rng(4)
    descs, ubs = [], []
    for k in range(260):
        ubs.append((float(rng.uniform(-0.02, 0.02)), 0.0, 0.0))
        descs.append(binding.lattice_desc(8, 8, 6, 0.8, 1.0, ubs[k], (0, 0, 0), (0, 0, 0), "fp32",
                                          False, -1))
    b = binding.Batch(descs)
    b.step(4)
    assert all(s == 0 for s in b.status())
    for k in (0, 255, 256, 259):
        ref = binding.Lattice(8, 8, 6, 0.8, 1.0, ubs[k], (0, 0, 0), precision="fp32",
                              ib_sms=-1)
        ref.step(4)
        assert np.array_equal(b.contexts[k].populations(), ref.populations())
        ref.close()
    b.close()


def test_full_ensemble_sampled_instances():
    """The 96-box ensemble of the benchmark (33 M nodes, edges from {48, 64, 80, 96}) in the
    launch configuration the benchmark times: after 5 steps, sampled instances equal the same
    contexts stepped alone, bit for bit."""
    from paper_2305_18919_gb300 import binding
    wls = inputs.wetting_ensemble(96, 2305)
    b = binding.Batch.from_workloads(wls)
    b.tune(trials=1)
    b.step(5)
    assert all(s == 0 for s in b.status())
    for k in (0, 31, 58, 95):
        ref = _alone(wls[k], "fp32", [5])
        _same(b.contexts[k], ref)
    b.close()


def _oracle_ensemble():
    """One instance per pre-stressed model class of Table I, uneven edges, walls on."""
    a = 0.01
    return [
        inputs.scaled_wetting(24, 20, 2, 4.5, alpha=(a, 0, 0), eps=0.5 * a),            # droplet
        inputs.scaled_shear(20, 2, 4.0, alpha=(a, 0, a)),                                # softly coated
        inputs.scaled_wetting(28, 22, 3, 5.5, alpha=(a, a, a), eps=0.8 * a),            # rigidly coated
    ]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_matches_the_oracle(precision):
    """The batched path against the FP64 oracle itself (not only against the library stepped
    one context at a time): 120 steps of three instances of different sizes and classes, at
    the FP32 bars (u and rho relative L2 <= 1e-5, vertices <= 1e-6 R; FP64 to rounding)."""
    import oracle
    from paper_2305_18919_gb300 import binding
    from pairs import rel_l2
    wls = _oracle_ensemble()
    for wl in wls:
        wl.centre = (wl.centre[0] - 0.37, wl.centre[1] + 0.21, wl.centre[2])
    b = binding.Batch.from_workloads(wls, precision=precision)
    b.step(120)
    assert list(b.status()) == [0, 0, 0]
    for lat, wl in zip(b.contexts, wls):
        ref = oracle.Simulation.from_workload(wl)
        ref.step(120)
        r0, u0 = ref.fields()
        r1, u1 = lat.fields()
        dq = np.abs(lat.vertices() - ref.vertices()).max()
        if precision == "fp32":
            assert rel_l2(u1, u0) < 1e-5 and rel_l2(r1 - 1, r0 - 1) < 1e-5
            assert dq < 1e-6 * wl.radius
        else:
            assert rel_l2(u1, u0) < 1e-11 and dq < 1e-11 * wl.radius
        ref.close()
    b.close()
