"""Host-side helpers of bench.py: the roofline traffic is taken from the committed ncu summary
only for the kernel it covers and only while the kernel sources hash as when it was captured;
the L2 note states whether the population arrays fit; the kernel named in the roofline is the
one the context will run; and the throughput arithmetic."""
import os
import re
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
from paper_2305_18919_gb300 import inputs  # noqa: E402


def test_traffic_only_for_the_summarised_kernel_and_sources():
    for name, kernel in (("stream_collide_kernel_shear256.md",
                          "stream_collide_kernel<float,float,false,false,false>"),
                         ("stream_collide_staged_kernel_shear256_fp16.md",
                          "stream_collide_staged_kernel<__half,false,4>")):
        text = open(os.path.join(ROOT, "profiles", name)).read()
        per_node = float(re.search(r"traffic per fluid node: ([0-9.]+) B", text).group(1))
        stored = re.search(r"kernel source sha256: ([0-9a-f]{64})", text).group(1)
        got = bench.k1_traffic_per_node(kernel)
        if stored == bench.k1_source_hash():
            assert got == per_node
            # the traffic of a full launch is within a few percent of the algorithmic bytes
            algorithmic = 152.0 if "float,float" in kernel else 76.0
            assert 0.9 * algorithmic < per_node <= 1.001 * algorithmic
        else:
            assert got is None
    assert bench.k1_traffic_per_node("stream_collide_kernel<double,double,false,false,false>") is None


def test_source_hash_follows_the_kernel_files(tmp_path, monkeypatch):
    h = bench.k1_source_hash()
    assert re.fullmatch(r"[0-9a-f]{64}", h)
    assert bench.k1_source_hash() == h  # stable
    fake = tmp_path / "paper_2305_18919_gb300" / "csrc"
    fake.mkdir(parents=True)
    for f in ("lattice_kernels.cu", "iblb_internal.cuh"):
        src = open(os.path.join(ROOT, "paper_2305_18919_gb300", "csrc", f), "rb").read()
        (fake / f).write_bytes(src + (b"\n" if f == "lattice_kernels.cu" else b""))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.k1_source_hash() != h  # one byte more in the kernel source


def test_l2_note():
    big = bench.config_of(inputs.shear_256_fp32())
    assert "exceed the 129 MB L2" in big["l2"]
    small = bench.config_of(inputs.shear_32_fp64())
    assert "fit in the 129 MB L2" in small["l2"]
    wl = inputs.shear_256_fp32()
    wl.precision = "fp16"
    assert "exceed" in bench.config_of(wl)["l2"]  # 2 x 0.64 GB


class _FakeLattice:
    def __init__(self, nx, staged):
        self.shape = (nx, nx, nx)
        self._staged = staged

    def stream_collide_staged(self):
        return self._staged


@pytest.mark.parametrize("precision,staged,name", [
    ("fp32", False, "stream_collide_kernel<float,float,false,false,false>"),
    ("fp64", False, "stream_collide_kernel<double,double,false,false,false>"),
    ("fp16", True, "stream_collide_staged_kernel<__half,false,4>"),
    ("bf16", True, "stream_collide_staged_kernel<__nv_bfloat16,false,4>"),
    ("fp16", False, "stream_collide_quad_kernel<__half,false,false>"),
    ("fp32", True, "stream_collide_staged_kernel<float,false,2>")])
def test_kernel_name(precision, staged, name):
    assert bench.k1_kernel_name(_FakeLattice(256, staged), precision) == name


def test_replica_mlups():
    # 2 replicas of 256^3 nodes, 100 steps in 0.5 s: 2 * 16.777216e6 * 100 / 0.5 / 1e6
    assert bench.replica_mlups(2, 256 ** 3, 100, 0.5) == pytest.approx(6710.8864)
    assert bench.max_over_ranks(0.3) == 0.3  # one process: its own value
