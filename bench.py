"""Throughput of the coupled IB-LB step (arXiv:2305.18919, Sec. III) on GB300.

Metric: MLUPS including the interface coupling = lattice nodes (wall layers counted) x steps
/ time of the whole step (face forces, spreading, stream-collide, velocity gather,
interpolation and update). Default workload: the 256^3 FP32 shear flow with a rigidly coated
particle (R = 40, icosphere subdivision 6, 40962 vertices, 81920 faces), tau = 0.8, walls
moving at -/+0.02.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]

Prints one JSON line. With --impl reference the FP64 CPU oracle runs the same workload on the
host (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2305_18919_gb300 import inputs  # noqa: E402

METRIC = "MLUPS incl. IB coupling"


def workload(name: str):
    if name == "shear256":
        return inputs.shear_256_fp32()
    if name == "wetting128":
        return inputs.wetting_128x128x96()
    if name == "box128":
        return inputs.shear_256_fp32_box(128)
    if name == "shear32":
        return inputs.shear_32_fp64()
    raise SystemExit(f"unknown workload {name}")


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model() -> str:
    """The host CPU's model name (from /proc/cpuinfo; 'unknown' where it is not given)."""
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu model", "hardware"):
                return line.split(":", 1)[1].strip()
        for line in open("/proc/cpuinfo"):  # Arm: implementer / part numbers only
            if line.lower().startswith("cpu part"):
                return "Arm CPU part " + line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _oracle_mlups(wl, seconds_target, threads):
    """The FP64 oracle, as it stands, on a bounded number of full steps of the workload with
    `threads` threads (0: all host cores); returns (MLUPS, steps, seconds, threads, set-up s)."""
    import oracle
    used = oracle.set_threads(threads if threads > 0 else (os.cpu_count() or 1))
    t0 = time.perf_counter()
    sim = oracle.Simulation.from_workload(wl)
    setup = time.perf_counter() - t0
    steps = 0
    t0 = time.perf_counter()
    while True:
        sim.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds_target or steps >= 1000:
            break
    sim.close()
    return wl.cells * steps / el / 1e6, steps, el, used, setup


def cpu_baseline(wl, seconds_target=20.0):
    """The FP64 oracle on the host cores (its per-node loops split over z-planes by OpenMP),
    with the single-thread figure beside it: bounded samples of full steps of the same
    workload."""
    v1, n1, e1, _, _ = _oracle_mlups(wl, seconds_target, 1)
    vN, nN, eN, used, setup = _oracle_mlups(wl, seconds_target, 0)
    return {"value": round(vN, 4), "unit": "MLUPS", "cores": used, "kind": "oracle",
            "sample": f"{nN} full IB-LB steps of the {wl.nx}x{wl.ny}x{wl.nz} workload (FP64 "
                      f"oracle, {used} threads, {eN:.1f} s timed, set-up {setup:.1f} s untimed)",
            "single_thread": {"value": round(v1, 4), "unit": "MLUPS", "cores": 1,
                              "sample": f"{n1} full steps, {e1:.1f} s timed"},
            "host": {"nproc": os.cpu_count(), "cpu_model": cpu_model()}}


def run_reference(args, wl, rank):
    """--impl reference: the oracle on the host, rank 0 only."""
    if rank != 0:
        return
    import oracle
    cores = oracle.set_threads(os.cpu_count() or 1)
    t0 = time.perf_counter()
    sim = oracle.Simulation.from_workload(wl)
    setup = time.perf_counter() - t0
    # each oracle step of the full lattice takes seconds; cap the run at about three minutes
    t1 = time.perf_counter()
    sim.step(1)
    one = time.perf_counter() - t1
    budget = 150.0
    warm = max(0, min(args.warmup - 1, int(budget * 0.2 / max(one, 1e-9))))
    sim.step(warm)
    k = max(1, min(args.steps, int(budget * 0.8 / max(one, 1e-9))))
    t1 = time.perf_counter()
    sim.step(k)
    el = time.perf_counter() - t1
    sim.close()
    value = wl.cells * k / el / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "MLUPS",
        "n_gpus": args.gpus, "steps": k, "warmup": warm + 1, "ms_per_step": round(el / k * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(wl),
        "cpu_baseline": {"value": round(value, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                         "sample": f"{k} full IB-LB steps of the {wl.nx}x{wl.ny}x{wl.nz} workload "
                                   f"timed of {args.steps} requested (FP64 oracle, {cores} threads; "
                                   f"set-up {setup:.1f} s untimed)",
                         "host": {"nproc": os.cpu_count(), "cpu_model": cpu_model()}},
        "e2e": {"value": round(value, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def config_of(wl):
    v, f = wl.mesh()
    pop_bytes = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2}[wl.precision]
    arr_gb = 19 * wl.cells * pop_bytes / 1e9
    l2 = (f"no flush: the two population arrays (2 x {arr_gb:.2f} GB) exceed the 129 MB L2"
          if 2 * arr_gb > 0.129 else
          f"no flush: the two population arrays (2 x {arr_gb:.3f} GB) fit in the 129 MB L2 "
          "(a small case; the benchmark workload's do not)")
    return {"workload": wl.name, "lattice": [wl.nx, wl.ny, wl.nz], "nodes": wl.cells,
            "vertices": int(v.shape[0]), "faces": int(f.shape[0]), "tau": wl.tau,
            "wall_u": [wl.wall_u_bottom[0], wl.wall_u_top[0]],
            "alpha": list(wl.alpha), "precision": wl.precision, "l2": l2}


def k1_source_hash():
    """Hash of the stream-collide kernel's sources: DRAM counters taken on another build of
    the kernel do not describe this one."""
    import hashlib
    h = hashlib.sha256()
    for f in ("lattice_kernels.cu", "iblb_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2305_18919_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


K1_PROFILES = ("stream_collide_kernel_shear256.md", "stream_collide_staged_kernel_shear256_fp16.md",
               "stream_collide_staged_kernel_shear256_bf16.md")


def k1_traffic_per_node(kernel):
    """DRAM bytes (read + write) per fluid node of one launch of `kernel` on the 256^3 lattice,
    from the committed ncu summary that covers it, if that was taken on the current kernel
    source; else None."""
    import re
    for name in K1_PROFILES:
        try:
            text = open(os.path.join(ROOT, "profiles", name)).read()
        except OSError:
            continue
        k = re.search(r"- kernel: `([^`]+)`", text)
        m = re.search(r"traffic per fluid node: ([0-9.]+) B", text)
        hsh = re.search(r"kernel source sha256: ([0-9a-f]{64})", text)
        if k and k.group(1) == kernel and m and hsh and hsh.group(1) == k1_source_hash():
            return float(m.group(1))
    return None


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest of the ranks' values (each rank's own value without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_mlups(world: int, cells: int, steps: int, seconds: float) -> float:
    """Whole-job throughput of `world` replicas that each advanced `cells` nodes `steps` times
    in at most `seconds` (the slowest rank's time)."""
    return world * cells * steps / seconds / 1e6


def k1_kernel_name(lat, precision):
    """Name of the kernel that runs the full-lattice pass of the timed steps."""
    storage = {"fp64": "double", "fp32": "float", "fp16": "__half", "bf16": "__nv_bfloat16"}
    if lat.stream_collide_staged():  # four nodes per compute lane with 16-bit storage
        nodes = 4 if precision in ("fp16", "bf16") else 2
        return f"stream_collide_staged_kernel<{storage[precision]},false,{nodes}>"
    if precision in ("fp16", "bf16"):
        return f"stream_collide_quad_kernel<{storage[precision]},false,false>"
    real = "double" if precision == "fp64" else "float"
    return f"stream_collide_kernel<{real},{storage[precision]},false,false,false>"


def time_variant(wl, precision, steps, warmup, sc=("auto", 0, 0, 0)):
    """Device-timed throughput of the same workload with another population storage type
    (inputs resident, CUDA events on the caller's stream, same step as the headline)."""
    import torch
    from paper_2305_18919_gb300 import binding
    lat = binding.Lattice.from_workload(wl, precision=precision)
    lat.set_stream_collide(*sc)
    lat.step(max(3, warmup))
    lat.set_profiling(True)
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    lat.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    k1_ms, k1_launches, _ = lat.profile()
    bpc = lat.bytes_per_cell()
    sms = lat.interface_sms()
    kernel = k1_kernel_name(lat, precision)
    per_node = k1_traffic_per_node(kernel) if wl.nx == 256 else None
    lat.close()
    fluid = wl.nx * wl.ny * (wl.nz - 2)
    peak = (measured_peaks() or {}).get("hbm_gbs", 6800.0)
    k1_avg = k1_ms / max(1, k1_launches)
    return {"value": round(replica_mlups(1, wl.cells, steps, ms * 1e-3), 1),
            "ms_per_step": round(ms / steps, 5), "steps": steps, "bytes_per_cell": bpc,
            "k1_ms_avg": round(k1_avg, 5),
            "k1_frac": round(bpc * fluid / (k1_avg * 1e-3) / 1e9 / peak, 4),
            "step_frac": round(bpc * fluid / (ms / steps * 1e-3) / 1e9 / peak, 4),
            "interface_sms": sms, "kernel": kernel,
            "traffic": int(round(per_node * fluid)) if per_node is not None else None}


def time_workloads(steps, warmup):
    """The two other single-box workloads, each in its own precision: the 32^3 shear box (FP64,
    304 B per node) and the 128 x 128 x 96 static-wetting box (FP32, 152 B per node); same
    timing as the headline, MLUPS and the roofline fractions of the stream-collide pass and of
    the whole step."""
    out = {}
    for wl in (inputs.shear_32_fp64(), inputs.wetting_128x128x96()):
        r = time_variant(wl, wl.precision, steps, warmup)
        r["config"] = config_of(wl)
        out[wl.name] = r
    return out


def time_ensemble(steps, warmup, n=96, seed=2305, ib_sms=0):
    """The batched-ensemble workload: n independent wetting boxes of uneven sizes (edges from
    {48, 64, 80, 96}), advanced together by iblb_batch_step (each kernel of a step one launch
    over all boxes) after iblb_batch_tune, against the same boxes stepped one after another."""
    import torch
    from paper_2305_18919_gb300 import binding
    wls = inputs.wetting_ensemble(n, seed)
    cells = sum(w.cells for w in wls)
    fluid = sum(w.nx * w.ny * (w.nz - 2) for w in wls)
    b = binding.Batch.from_workloads(wls, ib_sms=ib_sms)
    rows = b.tune(trials=3)
    b.step(max(4, warmup))
    stream = torch.cuda.current_stream()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    b.step(steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    # the same instances, one context after another (each iblb_step(steps) on its own stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for lat in b.contexts:
        lat.step(steps)
    torch.cuda.synchronize()
    seq_s = time.perf_counter() - t0
    b.close()
    peak = (measured_peaks() or {}).get("hbm_gbs", 6800.0)
    return {"workload": f"wetting_ensemble_{n}_seed{seed}", "instances": n, "nodes": cells,
            "value": round(replica_mlups(1, cells, steps, ms * 1e-3), 1), "unit": "MLUPS",
            "ms_per_step": round(ms / steps, 4), "steps": steps,
            "step_frac": round(152 * fluid / (ms / steps * 1e-3) / 1e9 / peak, 4),
            "sequential_value": round(replica_mlups(1, cells, steps, seq_s), 1),
            "k1_rows_chosen": {str(r): rows.count(r) for r in sorted(set(rows))},
            "eps_over_alpha_range": [0.0, 0.1],
            "eps_note": "wall strength eps/alpha_bar drawn uniformly in [0, 0.1] rather than the "
                        "workload's [0, 1]: at the upper end the finest meshes are pulled "
                        "through the wall within a few steps, in the FP64 oracle as well",
            "path": "iblb_batch_step: each kernel of a step one launch over all instances "
                    "(8 launches per step), FP32"}


def time_adjoint(steps, every, ref_steps=2):
    """Adjoint steps/s on the 64^3 wetting workload with an FP32 forward run: iblb_adjoint_record
    of `steps` steps with a state copy every `every`, then iblb_adjoint_gradient (reverse pass
    in double) of the wetted radius (torch observable); the autograd reference
    (oracle/adjoint.py, one host thread, FP64) is timed on `ref_steps` steps of the same
    workload."""
    import torch
    from paper_2305_18919_gb300 import adjoint as ad
    from paper_2305_18919_gb300 import binding
    wl = inputs.adjoint_wetting_64()
    _, faces = wl.mesh()
    lat = binding.Lattice.from_workload(wl, precision="fp32")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lat.adjoint_record(steps, every)
    t_fwd = time.perf_counter() - t0
    qt = torch.tensor(lat.vertices(), requires_grad=True)
    radius = ad.wetted_radius(qt, faces)
    (dJdq,) = torch.autograd.grad(radius, qt)
    t0 = time.perf_counter()
    g = lat.adjoint_gradient(dJdq.numpy())
    t_adj = time.perf_counter() - t0
    lat.close()
    out = {"workload": wl.name, "steps": steps, "checkpoint_every": every,
           "value": round(steps / t_adj, 1), "unit": "adjoint steps/s",
           "forward_steps_per_s": round(steps / t_fwd, 1),
           "observable": "wetted radius", "J": round(float(radius.detach()), 4),
           "dJ_dtheta": [float(x) for x in g],
           "path": "iblb_adjoint_record + iblb_adjoint_gradient (recompute per segment + reverse "
                   "step): FP32 forward, reverse in double"}
    try:
        torch.set_num_threads(1)
        from oracle import adjoint as oa
        t0 = time.perf_counter()
        oa.gradient(wl, ref_steps, lambda q: ad.wetted_radius(q, faces))
        t_ref = time.perf_counter() - t0
        out["reference"] = {"value": round(ref_steps / t_ref, 4), "unit": "adjoint steps/s",
                            "cores": 1, "kind": "oracle",
                            "sample": f"{ref_steps} steps forward and reverse with autograd "
                                      "(float64 PyTorch restatement of the oracle, one thread)"}
    except Exception as e:  # the reference needs torch with autograd on the host
        out["reference"] = {"unavailable": str(e)[:200]}
    return out


def run_gpu(args, wl, rank, world):
    import torch
    from paper_2305_18919_gb300 import binding

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    lat = binding.Lattice.from_workload(wl, precision=wl.precision, ib_sms=args.ib_sms)
    sc = (args.stream_collide, args.stages, args.stage_warps, args.stage_rows)
    lat.set_stream_collide(*sc)
    lat.step(max(3, args.warmup))
    torch.cuda.synchronize()

    # --- device-resident timed region ------------------------------------------------------
    lat.set_profiling(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        lat.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms_total = ev0.elapsed_time(ev1)
    k1_ms, k1_launches, launches = lat.profile()
    lat.set_profiling(False)
    ms_total = max_over_ranks(ms_total, dist, "cuda")
    if dist:
        dist.barrier()
    ms_step = ms_total / args.steps
    value = replica_mlups(world, wl.cells, args.steps, ms_total * 1e-3)

    # --- end to end through the C ABI with host buffers -------------------------------------
    nv = lat.nv
    q_host = torch.empty((nv, 3), dtype=torch.float64, pin_memory=True).numpy()
    lat.vertices(out=q_host)
    e2e_steps = max(1, min(args.steps, 200))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        lat.set_vertices(q_host)   # H2D: this step's vertex positions
        lat.step_async(1)          # its health check is read with the vertices
        lat.vertices(out=q_host)   # D2H: the step's result (and the step's health word)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, "cuda")
    e2e_value = replica_mlups(world, wl.cells, e2e_steps, e2e_s)

    bpc = lat.bytes_per_cell()
    fluid = wl.nx * wl.ny * (wl.nz - 2)
    k1_avg_ms = k1_ms / max(1, k1_launches)
    peaks = measured_peaks()
    if peaks and peaks.get("hbm_gbs"):
        peak, peak_note = float(peaks["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy)"
    else:
        peak, peak_note = 6800.0, "fallback"
    achieved = bpc * fluid / (k1_avg_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "kernel": k1_kernel_name(lat, wl.precision),
                "algorithmic_bytes_per_launch": bpc * fluid,
                "k1_ms_avg": round(k1_avg_ms, 5), "peak_source": peak_note,
                "step_frac": round(bpc * fluid / (ms_step * 1e-3) / 1e9 / peak, 4)}
    per_node = k1_traffic_per_node(roofline["kernel"]) if wl.nx == 256 else None
    if per_node is not None:
        # measured at full size on the 256^3 lattice (one ncu launch), per fluid node
        roofline["traffic"] = int(round(per_node * fluid))
    clocks = clk.summary()
    ib_sms = lat.interface_sms()
    lat.close()
    variants = None
    if rank == 0 and world == 1 and args.variant_steps > 0 and wl.precision == "fp32":
        variants = {p: time_variant(wl, p, args.variant_steps, args.warmup, sc)
                    for p in ("fp16", "bf16")}
        variants["note"] = ("populations stored in 16 bits as (f_i - w_i rho0) K / w_i, FP32 "
                            "collision; errors against the FP64 oracle in tests/test_gpu_precision.py")
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = cpu_baseline(wl, args.cpu_seconds) if (world == 1 and args.cpu_seconds > 0) else None
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": round(ms_step, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if wl.precision == "fp64" else "f32",
        "data": "synthetic", "config": config_of(wl),
        "interface_sms": ib_sms,  # the SM partition (a launch setting, not part of the workload)
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": round(e2e_value, 1), "unit": "MLUPS", "h2d_bytes_per_step": nv * 24,
                "d2h_bytes_per_step": nv * 24, "steps": e2e_steps,
                "path": "iblb_set_vertices + iblb_step_async(1) + iblb_read_vertices (which reads the step's health word in its synchronisation), pinned host buffers"},
        "gpu_launches": int(launches), "clocks": clocks,
    }
    if variants:
        line["precision_variants"] = variants
    if rank == 0 and world == 1 and args.workload_steps > 0 and wl.name.startswith("shear256"):
        line["workloads"] = time_workloads(args.workload_steps, args.warmup)
    if rank == 0 and world == 1 and args.ensemble_steps > 0 and wl.name.startswith("shear256"):
        line["ensemble"] = time_ensemble(args.ensemble_steps, 10)
    if rank == 0 and world == 1 and args.adjoint_steps > 0 and wl.name.startswith("shear256"):
        line["adjoint"] = time_adjoint(args.adjoint_steps, 100)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="shear256")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--adjoint-steps", type=int, default=5000,
                    help="steps of the 64^3 adjoint workload timed beside the headline (0: skip)")
    ap.add_argument("--workload-steps", type=int, default=2000,
                    help="steps timed for the 32^3 FP64 shear and 128x128x96 FP32 wetting "
                         "workloads reported beside the headline (0: skip)")
    ap.add_argument("--ensemble-steps", type=int, default=200,
                    help="steps timed for the 96-box batched ensemble reported beside the "
                         "headline (0: skip)")
    ap.add_argument("--variant-steps", type=int, default=1000,
                    help="steps timed for each 16-bit storage variant reported beside the FP32 "
                         "headline (0: skip)")
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32", "fp16", "bf16"],
                    help="population storage (default: the workload's; fp16/bf16 keep FP32 "
                         "arithmetic)")
    ap.add_argument("--ib-sms", type=int, default=0,
                    help="SMs for the interface chain (0: library default, <0: no partition)")
    ap.add_argument("--stream-collide", default="auto", choices=["auto", "staged", "direct"],
                    help="kernel of the full-lattice pass: rows staged in shared memory by bulk "
                         "copies, loaded directly by each thread, or the library's choice for "
                         "the storage type (auto)")
    ap.add_argument("--stages", type=int, default=0, help="buffers per block of the staged pass "
                                                           "(0: library default)")
    ap.add_argument("--stage-warps", type=int, default=0,
                    help="compute warps per block of the staged pass (0: library default)")
    ap.add_argument("--stage-rows", type=int, default=0,
                    help="lattice rows per unit of the staged pass (0: library default)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.warmup < 3:
        args.warmup = 3
    wl = workload(args.workload)
    if args.precision and args.impl != "reference":
        wl.precision = args.precision
        wl.name = f"{wl.name}_{args.precision}" if args.precision not in wl.name else wl.name
    if args.impl == "reference":
        run_reference(args, wl, rank)
    else:
        run_gpu(args, wl, rank, world)


if __name__ == "__main__":
    main()
