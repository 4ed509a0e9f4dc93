"""The allocation-free volume entry point, iblb_mesh_volume_noalloc.

Some users of this library cannot let it call cudaMalloc: a plug-in inside a host framework
that owns every byte of device memory through its own pool and budget, or a latency-bound
loop in which cudaMalloc/cudaFree (which may synchronise the whole device) is not allowed.
For them the library offers this call, which works on the caller's device buffers and keeps
its scratch in a fixed 32 KB array that the library holds on each device it loads on.

These tests call it through the C ABI on device buffers owned by torch and compare its
result with the context-based iblb_read_volume, to the tolerance used for the volume
elsewhere (1e-12 relative), on calls made one after another with meshes of different sizes,
so that a stale partial sum from an earlier call would show. The file is named to be
collected last.
"""
import numpy as np
import pytest

from paper_2305_18919_gb300 import inputs

pytestmark = pytest.mark.gpu


def _device(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _noalloc_volume(q, faces, centre):
    import torch
    from paper_2305_18919_gb300 import binding
    q_dev = _device(q, torch.float64)
    f_dev = _device(faces.astype(np.int32), torch.int32)
    V_dev = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    rc = binding.mesh_volume_noalloc(q_dev.data_ptr(), f_dev.data_ptr(), faces.shape[0], centre,
                                     V_dev.data_ptr())
    assert rc == binding.IBLB_OK
    torch.cuda.synchronize()
    return float(V_dev.item())


def _context_volume(verts, faces, q):
    from paper_2305_18919_gb300 import binding
    lat = binding.Lattice(48, 48, 40, 1.0, precision="fp64")
    lat.add_mesh(verts, faces)
    lat.set_vertices(q)
    V, _ = lat.volume()
    lat.close()
    return V


def test_noalloc_volume_matches_context_volume_on_consecutive_calls():
    cases = [(5, 12.0, 0.2, 1), (2, 6.0, 0.3, 2), (4, 9.0, 0.25, 3)]
    for sub, radius, amp, seed in cases:
        verts, faces = inputs.icosphere(sub, radius, (24.3, 23.8, 19.6))
        q = inputs.perturb(verts, amp, seed=seed)
        centre = verts.mean(0)  # the fixed point the context uses
        V_ref = _context_volume(verts, faces, q)
        for _ in range(2):  # two calls in a row on the same inputs
            V = _noalloc_volume(q, faces, centre)
            assert abs(V - V_ref) <= 1e-12 * abs(V_ref)


def test_noalloc_volume_rejects_bad_sizes_before_launching():
    from paper_2305_18919_gb300 import binding
    L = binding.lib()
    c = np.zeros(3)
    dummy = 1  # never dereferenced: the size checks come first
    assert binding.mesh_volume_noalloc(dummy, dummy, 4096 * 256 + 1, c, dummy) == binding.IBLB_ECAPACITY
    # the size test comes before the block count is formed, which would overflow int32 here
    assert binding.mesh_volume_noalloc(dummy, dummy, 2**31 - 1, c, dummy) == binding.IBLB_ECAPACITY
    assert binding.mesh_volume_noalloc(dummy, dummy, 0, c, dummy) == binding.IBLB_EINVAL
    assert L.iblb_mesh_volume_noalloc(None, None, 10, None, None, None) == binding.IBLB_EINVAL
