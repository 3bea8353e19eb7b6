#!/usr/bin/env python3
"""Benchmark: reconstructed voxels/s of the NEDNER forward path on GB300.

One step = one full reconstruction p0 = R g (stages a-d: NED-NUFFT, NER-NUFFT,
Jacobian, inverse 3-D FFT) of one synthetic workload, inputs resident in HBM.
Default workload: 64 x 64 centre-dense tensor-grid sensors over 20 mm,
Nt = 512 at 16.7 ns, 128 x 128 x 256 voxels, Kaiser-Bessel w = 12, sigma = 2,
20 balls + 20 dB noise (seeded).  L2 is flushed (256 MB write) between timed
steps.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config c2|c3|c1|c4|c5]
  python bench.py --impl reference ...   # the FP64 oracle on the host cores

With N > 1 (torchrun) every rank reconstructs its own workload (independent
problems, no data-path collective): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CONFIGS = {"c1": 0, "c2": 1, "c3": 2, "c4": 3, "c5": 4}
METRIC = "recon voxels/s + % HBM roofline (spread/interp) at stated rel-L2 vs FP64 oracle"


def describe(cfg) -> str:
    M = cfg["sensor_xy"].shape[0]
    return ("%s: %d sensors, Nt=%d at dt=%.3g s, %dx%dx%d voxels (dx=%.3g m, dz=%.3g m), KB w=12, sigma=2"
            % (cfg["name"], M, cfg["Nt"], cfg["dt"], cfg["nx"], cfg["ny"], cfg["nz"], cfg["dx"], cfg["dz"]))


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def algorithmic_bytes(cfg):
    """Minimum HBM bytes per launch of each forward kernel (inputs read once,
    outputs written once; complex64 intermediates on the half lattice)."""
    M, Nt, nx, ny, nz = cfg["sensor_xy"].shape[0], cfg["Nt"], cfg["nx"], cfg["ny"], cfg["nz"]
    nxh, Ly = nx // 2 + 1, 2 * ny
    g = M * Nt * 4
    R = nxh * Ly * Nt * 8
    Gh = nxh * (ny + 1) * Nt * 8
    V = nxh * ny * nz * 8
    p0 = nx * ny * nz * 4
    return {"ned_spread_xfft": g + R, "ned_yfft": R + Gh, "ner_lines": Gh + V, "img_yifft": 2 * V,
            "img_xc2r": V + p0}


def sources_sha(sources) -> str:
    """SHA-256 (16 hex digits) of the kernel's source files, in order."""
    if isinstance(sources, str):
        sources = [sources]
    h = hashlib.sha256()
    for name in sources:
        with open(os.path.join(ROOT, "paper_1510_01078_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, if it
    was taken on the current kernel sources (every file the kernel is built
    from: its .cu file and the headers holding its device code)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        ent = d.get(kernel)
        return float(ent["bytes_per_launch"]) if sources_sha(ent["source"]) == ent["source_sha"] else None
    except Exception:
        return None


def oracle_forward_seconds(cfg, steps: int = 1, want_output: bool = False):
    import numpy as np
    import oracle
    pr = oracle.Problem(sensor_xy=cfg["sensor_xy"], h=cfg["h"], Nt=cfg["Nt"], dt=cfg["dt"], c=cfg["c"],
                        nx=cfg["nx"], ny=cfg["ny"], nz=cfg["nz"], dx=cfg["dx"], dy=cfg["dy"], dz=cfg["dz"])
    times = []
    out = None
    for _ in range(steps):
        t0 = time.perf_counter()
        out = oracle.forward(pr, np.asarray(cfg["g"], dtype=np.float64))
        times.append(time.perf_counter() - t0)
    return (times, out) if want_output else times




def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over all ranks: the slowest replica sets the step time."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(voxels: int, world: int, ms_step: float) -> float:
    """Voxels/s of the whole job: every rank reconstructs its own workload of
    `voxels` voxels in at most `ms_step` milliseconds."""
    return voxels * world / (ms_step / 1e3)


def run_reference(args, cfg, voxels, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = os.cpu_count()
    for _ in range(args.warmup):
        oracle_forward_seconds(cfg, 1)
    times = oracle_forward_seconds(cfg, args.steps)
    sec = sum(times) / len(times)
    value = voxels / sec
    line = {"metric": METRIC, "value": value, "unit": "voxels/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded balls + noise)",
            "config": {"workload": describe(cfg), "l2": "n/a (host)"}, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "voxels/s", "cores": cores, "kind": "oracle",
                             "sample": "one full FP64 oracle reconstruction of the workload per step"},
            "e2e": {"value": value, "unit": "voxels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="nedner", choices=["nedner", "reference"])
    ap.add_argument("--config", default="c2", choices=sorted(CONFIGS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ned-mode", default="nufft", choices=["nufft", "tensor_bf16"],
                    help="stage (a) as NUFFT (any layout) or tensor-core GEMMs (128x128 tensor grids)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_1510_01078_gb300 import inputs
    cfg = inputs.make_config(CONFIGS[args.config])
    voxels = cfg["nx"] * cfg["ny"] * cfg["nz"]

    if args.impl == "reference":
        run_reference(args, cfg, voxels, rank, world)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_1510_01078_gb300 import build as b
    if rank == 0:
        b.build()
    if world > 1:
        dist.barrier()
    from paper_1510_01078_gb300 import nedner

    stream = torch.cuda.current_stream(dev)
    plan = nedner.plan_from_config(cfg, ned_mode=args.ned_mode)
    g = torch.as_tensor(np.asarray(cfg["g"], dtype=np.float32), device=dev).contiguous()
    p0 = torch.empty((cfg["nz"], cfg["ny"], cfg["nx"]), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        plan.forward(g, out=p0)
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    per_kernel = {k: [] for k in nedner.Plan.FORWARD_KERNELS}
    step_ms = []
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)                                     # evict L2 between steps (not timed)
        ms = plan.forward_profiled(g, p0)                    # events around each kernel, same stream
        for k, v in ms.items():
            per_kernel[k].append(v)
        step_ms.append(sum(ms.values()))
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    clk = clocks.stop()

    ms_step = max_over_ranks(sum(step_ms) / len(step_ms), world, dev)
    value = whole_job_value(voxels, world, ms_step)

    # end to end through the public API with host buffers (pinned), copies timed
    g_host = torch.as_tensor(np.asarray(cfg["g"], dtype=np.float32)).pin_memory()
    p_host = torch.empty((cfg["nz"], cfg["ny"], cfg["nx"]), dtype=torch.float32).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # nedner_forward_host: the public call with host buffers, uploads and
    # downloads overlapped with the kernels inside the timed region
    for _ in range(args.warmup):
        plan.forward_host(g_host, out=p_host, stream=stream)
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0.record(stream)
        plan.forward_host(g_host, out=p_host, stream=stream)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_step = max_over_ranks(sum(e2e_ms) / len(e2e_ms), world, dev)

    # roofline of the dominant kernel
    abytes = algorithmic_bytes(cfg)
    avg = {k: sum(v) / len(v) for k, v in per_kernel.items()}
    if args.ned_mode != "nufft":
        # stage (a) is one group of tensor-core kernels, reported under the first name
        avg = {("tp_ned_gemm" if k == "ned_spread_xfft" else k): v for k, v in avg.items() if k != "ned_yfft"}
        M, Nt = cfg["sensor_xy"].shape[0], cfg["Nt"]
        abytes = dict(abytes, tp_ned_gemm=M * Nt * 4 + (cfg["nx"] // 2 + 1) * (cfg["ny"] + 1) * Nt * 8)
    dom = max(avg, key=avg.get)
    peak, peak_kind = peaks()
    kernels = {k: {"ms": round(avg[k], 5), "share": round(avg[k] / sum(avg.values()), 4),
                   "alg_bytes": abytes[k], "gbs": round(abytes[k] / (avg[k] * 1e-3) / 1e9, 1)} for k in avg}
    achieved = abytes[dom] / (avg[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic_for(dom), "peak_source": peak_kind}
    # the spread kernel's own fraction (the metric names spread/interp)
    spread_frac = (round(abytes["ned_spread_xfft"] / (avg["ned_spread_xfft"] * 1e-3) / 1e9 / peak, 4)
                   if "ned_spread_xfft" in avg else None)

    # kernels launched per reconstruction: five for the NUFFT path; the tensor-core
    # stage a runs prep + two GEMMs per pass of 512 time samples, then the Nyquist line
    if args.ned_mode == "nufft":
        launches_per_step = len(nedner.Plan.FORWARD_KERNELS)
    else:
        launches_per_step = 3 * (cfg["Nt"] // min(512, cfg["Nt"])) + 1 + 3

    cpu = None
    accuracy = {"rel_l2_vs_oracle": None, "tolerance": 1e-5 if args.ned_mode == "nufft" else 3e-5}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            import oracle
            oracle.build()
            secs, ref = oracle_forward_seconds(cfg, 1, want_output=True)
            secs = secs[0]
            cpu = {"value": voxels / secs, "unit": "voxels/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": "one full FP64 oracle reconstruction of the workload (%.1f s)" % secs}
            # the accuracy the throughput is quoted at: the timed run's p0 against the oracle's
            got = p_host.double().numpy()                     # the result of the host-buffer call
            accuracy["rel_l2_vs_oracle"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        except Exception as ex:  # the baseline is reported, not required
            cpu = {"value": None, "unit": "voxels/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": "failed: %s" % ex}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "voxels/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded balls + 20 dB noise)",
                "config": {"workload": describe(cfg), "l2": "flushed between timed steps (256 MB write)",
                           "parallelism": "independent reconstruction per GPU", "ned_mode": args.ned_mode},
                "roofline": roofline, "spread_frac_of_peak": spread_frac, "accuracy": accuracy, "kernels": kernels,
                "cpu_baseline": cpu, "clocks": clk,
                "e2e": {"value": whole_job_value(voxels, world, e2e_step), "unit": "voxels/s",
                        "h2d_bytes_per_step": int(g_host.numel() * 4), "d2h_bytes_per_step": int(p_host.numel() * 4)},
                "gpu_launches": launches_per_step * args.steps,
                "wall_s_timed_region": round(wall, 3)}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
