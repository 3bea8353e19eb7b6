#!/usr/bin/env python3
"""Benchmark: reconstructed voxels/s of the NEDNER path on GB300.

One step = one full reconstruction p0 = R g (stages a-d: NED-NUFFT, NER-NUFFT,
Jacobian, inverse 3-D FFT) of one synthetic workload, inputs resident in HBM;
`value` is voxels/s of that reconstruction.  The same run also times the
transposed path (nedner_adjoint, R^T) and the sensor-position gradient
(nedner_grad_positions) per step, so the spread ("NED spread") and the
interpolation ("transposed gather") kernels both get a roofline figure.
L2 is flushed (a 256 MB write, outside the timed events) before every timed
call.  Prints one JSON line.

Default workload (paper scale): 16384 scattered centre-dense sensors in a 30 mm
disc, Nt = 2048 at 8.3 ns, 256 x 256 x 512 voxels, Kaiser-Bessel w = 12,
sigma = 2, 200 balls + 20 dB noise (seeded).

Accuracy is checked against the FP64 oracle on a seeded sample of the
spectrum: 1 % of the lateral lines (a product set of jx and jy values, no
Nyquist index) at every depth frequency.  The GPU's spectrum there is the DFT
of its p0 (exact: p0 is the real part of an inverse DFT of a Hermitian
spectrum).  The oracle's time for that sample, scaled to all lines, is the
cpu_baseline (its work is proportional to the number of lines).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config c3|c2|c1|c4|c5]
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
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

CONFIGS = {"c1": 0, "c2": 1, "c3": 2, "c4": 3, "c5": 4}
METRIC = "recon voxels/s + % HBM roofline (spread/interp) at stated rel-L2 vs FP64 oracle"
NED_MODES = ("nufft", "tensor_bf16", "tensor_fp16")


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
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,utilization.gpu")

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
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        # samples taken while a kernel was running (utilization above half)
        busy = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit() and r[9].isdigit() and int(r[9]) >= 50]
        return {"sm_mhz": statistics.median(busy or sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "samples_under_load": len(busy)}


# --------------------------------------------------------------------------
# algorithmic bytes per launch
# --------------------------------------------------------------------------
def algorithmic_bytes(cfg, split=True):
    """Minimum HBM bytes per reconstruction of each forward kernel (inputs read
    once, outputs written once; complex64 intermediates on the half lattice).
    Stage (a) split: the spread writes the oversampled real grid Q (2nx x 2ny
    per time sample), the x-FFT reads it and writes R; fused: one kernel reads
    g and writes R."""
    M, Nt, nx, ny, nz = cfg["sensor_xy"].shape[0], cfg["Nt"], cfg["nx"], cfg["ny"], cfg["nz"]
    nxh, Ly, Lx = nx // 2 + 1, 2 * ny, 2 * nx
    g = M * Nt * 4
    Q = Ly * Lx * Nt * 4
    R = nxh * Ly * Nt * 8
    Gh = nxh * (ny + 1) * Nt * 8
    V = nxh * ny * nz * 8
    p0 = nx * ny * nz * 4
    d = {"ned_yfft": R + Gh, "ner_lines": Gh + V, "img_yifft": 2 * V, "img_xc2r": V + p0}
    if split:
        d.update(ned_spread=g + Q, ned_xfft=Q + R)
    else:
        d.update(ned_spread=g + R, ned_xfft=0)
    return d


def algorithmic_bytes_transposed(cfg, grad: bool, split=True):
    """The same for the transposed stages (each forward stage's bytes with
    input and output swapped).  Split: the transposed x-FFT reads R and
    writes the oversampled real grid Q, the block gather reads Q; fused: the
    gather reads R and rebuilds the rows itself.  The gather writes one value
    per entry and time sample (adjoint), or reads g and writes 2 floats per
    entry and 64-sample chunk (gradient); the entry sum reads those and
    writes g (adjoint) or 2 floats per sensor (gradient)."""
    f = algorithmic_bytes(cfg, split=split)
    M, Nt, nx, ny, w = cfg["sensor_xy"].shape[0], cfg["Nt"], cfg["nx"], cfg["ny"], 12
    g = M * Nt * 4
    Q = 2 * ny * 2 * nx * Nt * 4
    R = (nx // 2 + 1) * 2 * ny * Nt * 8
    src = Q if split else R
    if grad:
        nch = Nt // 64
        gather, esum = src + g + M * w * nch * 8, M * w * nch * 8 + M * 8
    else:
        gather, esum = src + M * w * Nt * 4, M * w * Nt * 4 + g
    return {"img_xr2c_adj": f["img_xc2r"], "img_yfft_adj": f["img_yifft"], "ner_lines_adj": f["ner_lines"],
            "ned_yfft_adj": f["ned_yfft"], "ned_xfft_adj": f["ned_xfft"], "gather": gather, "entry_sum": esum}


def gather_alg_bytes(cfg):
    """Algorithmic bytes of the transposed interpolation as a whole (read the
    grid rows R once, write g once): the fused forward spread's bytes reversed."""
    return algorithmic_bytes(cfg, split=False)["ned_spread"]


# --------------------------------------------------------------------------
# ncu DRAM traffic recorded under profiles/ (per kernel and workload)
# --------------------------------------------------------------------------
def sources_sha(sources) -> str:
    """SHA-256 (16 hex digits) of the kernel's source files, in order."""
    if isinstance(sources, str):
        sources = [sources]
    h = hashlib.sha256()
    for name in sources:
        with open(os.path.join(ROOT, "paper_1510_01078_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str, workload: str):
    """Per-launch DRAM bytes of `kernel` on `workload` (a config name) from the
    committed ncu summary, if it was taken on the current kernel sources (its
    .cu file and the headers holding its device code); else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for ent in d.get("entries", []):
            if ent["kernel"] == kernel and ent["workload"] == workload:
                if sources_sha(ent["source"]) == ent["source_sha"]:
                    return float(ent["bytes_per_launch"])
        return None
    except Exception:
        return None


# --------------------------------------------------------------------------
# sampled oracle check
# --------------------------------------------------------------------------
def sample_lines(cfg, fraction: float, seed: int):
    """A seeded product set of lateral frequencies (jx, jy), about `fraction`
    of all nx ny lines, without the Nyquist indices -nx/2, -ny/2."""
    import numpy as np
    rng = np.random.default_rng(seed)
    nx, ny = cfg["nx"], cfg["ny"]
    kx = max(1, int(round((fraction * nx * ny) ** 0.5 * (nx / ny) ** 0.5)))
    ky = max(1, int(round(fraction * nx * ny / kx)))
    jx = np.sort(rng.choice(np.arange(-(nx // 2) + 1, nx // 2), size=min(kx, nx - 1), replace=False))
    jy = np.sort(rng.choice(np.arange(-(ny // 2) + 1, ny // 2), size=min(ky, ny - 1), replace=False))
    return jx, jy


def spectrum_of_volume(p0, jx, jy):
    """F[a, b, l] of the inverse DFT whose real part is p0 (nz, ny, nx), at the
    lines (jx[a], jy[b]) and every depth index l = -nz/2..nz/2-1 (index l + nz/2):
    the forward DFT of p0 on those lines (explicit sums along x and y, FFT
    along z), times the voxel-centring sign (-1)^(jx + jy).  Exact where no
    index is a Nyquist index and the spectrum is Hermitian."""
    import numpy as np
    nz, ny, nx = p0.shape
    p = np.asarray(p0, dtype=np.float64)
    ex = np.exp(-2j * np.pi * np.outer(np.arange(nx), jx) / nx)          # (nx, A)
    ey = np.exp(-2j * np.pi * np.outer(np.arange(ny), jy) / ny)          # (ny, B)
    a = p.reshape(nz * ny, nx) @ ex                                       # (nz*ny, A)
    b = np.einsum("zya,yb->zab", a.reshape(nz, ny, len(jx)), ey)         # (nz, A, B)
    c = np.fft.fft(b, axis=0)                                             # l mod nz
    c = np.fft.fftshift(c, axes=0)                                        # l + nz/2
    sign = np.where(((jx[:, None] + jy[None, :]) % 2) == 0, 1.0, -1.0)
    return np.transpose(c, (1, 2, 0)) * sign[:, :, None]                 # (A, B, nz)


def oracle_problem(cfg):
    import oracle
    return oracle.Problem(sensor_xy=cfg["sensor_xy"], h=cfg["h"], Nt=cfg["Nt"], dt=cfg["dt"], c=cfg["c"],
                          nx=cfg["nx"], ny=cfg["ny"], nz=cfg["nz"], dx=cfg["dx"], dy=cfg["dy"], dz=cfg["dz"])


def oracle_sample(cfg, fraction: float, seed: int):
    """The oracle's spectrum on a sample of lines; returns (jx, jy, F, seconds,
    scale) with scale = all lines / sampled lines."""
    import numpy as np
    import oracle
    jx, jy = sample_lines(cfg, fraction, seed)
    pr = oracle_problem(cfg)
    ls = oracle.index_set(cfg["nz"])
    t0 = time.perf_counter()
    F = oracle.spectrum_block(pr, np.asarray(cfg["g"], dtype=np.float64), jx, jy, ls)
    secs = time.perf_counter() - t0
    return jx, jy, F, secs, (cfg["nx"] * cfg["ny"]) / float(len(jx) * len(jy))


def sampled_errors(p0_gpu, jx, jy, F_orc):
    """rel-L2 and max-abs (relative to max |F|) of the GPU spectrum on the
    sampled lines, all depth frequencies but the Nyquist one."""
    import numpy as np
    got = spectrum_of_volume(p0_gpu, jx, jy)[:, :, 1:]
    want = F_orc[:, :, 1:]
    d = got - want
    return (float(np.linalg.norm(d) / np.linalg.norm(want)), float(np.abs(d).max() / np.abs(want).max()))


# --------------------------------------------------------------------------
# multi-rank bookkeeping
# --------------------------------------------------------------------------
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


# --------------------------------------------------------------------------
# the reference arm: the FP64 oracle on the host cores
# --------------------------------------------------------------------------
def run_reference(args, cfg, voxels, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = os.cpu_count()
    frac = args.reference_fraction
    for w in range(args.warmup):
        oracle_sample(cfg, frac, 9000 + w)
    secs = []
    lines = 0
    for k in range(args.steps):
        jx, jy, _, t, scale = oracle_sample(cfg, frac, 1000 + k)
        secs.append(t * scale)                 # one full reconstruction, extrapolated from the sample
        lines = len(jx) * len(jy)
    sec = sum(secs) / len(secs)
    value = voxels / sec
    sample = ("per step a seeded sample of %d of %d lateral lines (%.2f %%) at all %d depth frequencies "
              "(FP64 direct NED and NER sums, OpenMP); time scaled by lines to one full reconstruction"
              % (lines, cfg["nx"] * cfg["ny"], 100.0 * lines / (cfg["nx"] * cfg["ny"]), cfg["nz"]))
    line = {"metric": METRIC, "value": value, "unit": "voxels/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded balls + noise)",
            "config": {"workload": describe(cfg), "l2": "n/a (host)"}, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "voxels/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "voxels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------
# the GPU arm
# --------------------------------------------------------------------------
def timed_loop(fn, steps, flush):
    """Calls fn() `steps` times after an L2 flush each; fn returns a dict of
    per-kernel device times (ms).  Returns the per-kernel lists."""
    per = {}
    for _ in range(steps):
        flush.fill_(1.0)                       # evict L2 (not timed: outside fn's events)
        ms = fn()
        for k, v in ms.items():
            per.setdefault(k, []).append(v)
    return per


def cufft_comparison(cfg, dev, flush, reps, ours):
    """cuFFT (through torch.fft), timed as a reference point only, on the
    transforms our FFT stages contain: the 2-D real FFT of the oversampled
    grid per time sample (stage a2 without the crop, deconvolution and our
    layout), the zero-padded length-2Nt line FFT of the NER (without its
    interpolation and z-IFFT) and the 2-D inverse real FFT per depth plane
    (stage d).  ``ours``: our kernels' ms for the same stages."""
    import torch
    nx, ny, nz, Nt = cfg["nx"], cfg["ny"], cfg["nz"], cfg["Nt"]
    Lx, Ly = 2 * nx, 2 * ny
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def time_op(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            flush.fill_(1.0)
            ev0.record()
            fn()
            ev1.record()
            ev1.synchronize()
            ts.append(ev0.elapsed_time(ev1))
        return round(sum(ts) / len(ts), 5)

    out = {"library": "cuFFT via torch.fft %s" % torch.__version__, "note": "reference point only, not on the "
           "product path; each transform alone, inputs in HBM, L2 flushed before each call"}
    q = torch.randn((Nt, Ly, Lx), dtype=torch.float32, device=dev)
    out["ned_rfft2"] = {"shape": [Nt, Ly, Lx], "ms": time_op(lambda: torch.fft.rfft2(q)),
                        "ours_ms": ours.get("ned_xy"), "ours": "ned_xfft + ned_yfft (with crop, deconvolution)"}
    del q
    G = torch.randn(((nx // 2 + 1) * (ny + 1), Nt), dtype=torch.complex64, device=dev)
    out["ner_line_fft"] = {"shape": [G.shape[0], Nt], "n": 2 * Nt,
                           "ms": time_op(lambda: torch.fft.fft(G, n=2 * Nt, dim=-1)),
                           "ours_ms": ours.get("ner"), "ours": "ner_lines (line FFT, 12-tap interpolation, "
                                                                "Jacobian and z-IFFT)"}
    del G
    V = torch.randn((nz, ny, nx // 2 + 1), dtype=torch.complex64, device=dev)
    out["image_irfft2"] = {"shape": [nz, ny, nx // 2 + 1], "ms": time_op(lambda: torch.fft.irfft2(V, s=(ny, nx))),
                           "ours_ms": ours.get("image"), "ours": "img_yifft + img_xc2r"}
    del V
    torch.cuda.empty_cache()
    return out


def kernel_table(per, abytes):
    avg = {k: sum(v) / len(v) for k, v in per.items()}
    avg = {k: v for k, v in avg.items() if v > 0.0}              # stages this path does not launch
    tot = sum(avg.values())
    return avg, {k: {"ms": round(avg[k], 5), "share": round(avg[k] / tot, 4), "alg_bytes": abytes[k],
                     "gbs": round(abytes[k] / (avg[k] * 1e-3) / 1e9, 1)} for k in avg}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=80)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="nedner", choices=["nedner", "reference"])
    ap.add_argument("--config", default="c3", choices=sorted(CONFIGS))
    ap.add_argument("--nt", type=int, default=None,
                    help="record length override (nz scaled with it): the workload's lateral geometry and kernels "
                         "on a smaller case, for profiler captures; not a bench line")
    ap.add_argument("--lateral", type=int, default=None,
                    help="lateral grid override (the central lateral x lateral voxels at the same spacing, the "
                         "sensors inside): the workload's record and depth on fewer lines, for profiler "
                         "captures; not a bench line")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-transposed", action="store_true", help="time the forward only")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT reference timings")
    ap.add_argument("--oracle-fraction", type=float, default=0.01,
                    help="fraction of lateral lines of the accuracy check / cpu_baseline sample")
    ap.add_argument("--reference-fraction", type=float, default=0.001,
                    help="fraction of lateral lines per step of the reference arm")
    ap.add_argument("--ned-mode", default="nufft", choices=NED_MODES,
                    help="stage (a) as NUFFT (any layout) or tensor-core GEMMs (128x128 tensor grids)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_1510_01078_gb300 import inputs
    cfg = inputs.make_config(CONFIGS[args.config], Nt=args.nt, lateral=args.lateral)
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
    do_t = not args.no_transposed
    if do_t:
        rng = np.random.default_rng(cfg["seed"] + 99)
        lam = torch.as_tensor(rng.standard_normal((cfg["nz"], cfg["ny"], cfg["nx"])), dtype=torch.float32,
                              device=dev)
        g_adj = torch.empty_like(g)
        dxy = torch.empty((plan.M, 2), dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        plan.forward(g, out=p0)
        if do_t:
            plan.adjoint(lam, out=g_adj)
            plan.grad_positions(g, lam, out=dxy)
    torch.cuda.synchronize()

    clocks = ClockSampler(torch.cuda.current_device())
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def forward_timed():
        ev0.record(stream)
        plan.forward(g, out=p0, stream=stream)
        ev1.record(stream)
        ev1.synchronize()
        return {"forward": ev0.elapsed_time(ev1)}

    # the step: the plain public call; the per-kernel table: the profiled call
    per_step = timed_loop(forward_timed, args.steps, flush)
    prof_steps = min(args.steps, 20)
    per_fwd = timed_loop(lambda: plan.forward_profiled(g, p0), prof_steps, flush)
    if do_t:
        per_adj = timed_loop(lambda: plan.adjoint_profiled(lam, g_adj), args.steps, flush)
        per_grad = timed_loop(lambda: plan.grad_positions_profiled(g, lam, dxy), args.steps, flush)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    status_flags = plan.device_status()

    step_ms = per_step["forward"]
    ms_step = max_over_ranks(sum(step_ms) / len(step_ms), world, dev)
    value = whole_job_value(voxels, world, ms_step)

    # end to end through the public API with host buffers (pinned), copies timed
    g_host = torch.as_tensor(np.asarray(cfg["g"], dtype=np.float32)).pin_memory()
    p_host = torch.empty((cfg["nz"], cfg["ny"], cfg["nx"]), dtype=torch.float32).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):
        plan.forward_host(g_host, out=p_host, stream=stream)
    torch.cuda.synchronize()
    e2e_ms = []
    for _ in range(min(args.steps, 20)):
        flush.fill_(1.0)
        e0.record(stream)
        plan.forward_host(g_host, out=p_host, stream=stream)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_step = max_over_ranks(sum(e2e_ms) / len(e2e_ms), world, dev)

    # per-kernel tables and rooflines
    peak, peak_kind = peaks()
    split = bool(nedner.work_split(cfg["nx"], cfg["ny"], cfg["nz"], cfg["Nt"], 12)["split1"])
    abytes = algorithmic_bytes(cfg, split)
    if args.ned_mode != "nufft":
        # stage (a) is one group of tensor-core kernels, reported under one name
        per_fwd = {("tp_ned_gemm" if k == "ned_spread" else k): v for k, v in per_fwd.items()
                   if k not in ("ned_xfft", "ned_yfft")}
        M, Nt = cfg["sensor_xy"].shape[0], cfg["Nt"]
        abytes = dict(abytes, tp_ned_gemm=M * Nt * 4 + (cfg["nx"] // 2 + 1) * (cfg["ny"] + 1) * Nt * 8)
    avg, kernels = kernel_table(per_fwd, abytes)
    dom = max(avg, key=avg.get)
    achieved = abytes[dom] / (avg[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic_for(dom, cfg["name"]),
                "peak_source": peak_kind + " (burst copy bandwidth)"}
    spread_frac = (round(abytes["ned_spread"] / (avg["ned_spread"] * 1e-3) / 1e9 / peak, 4)
                   if "ned_spread" in avg else None)

    transposed = None
    interp_roofline = None
    info = plan.info()
    passes = cfg["Nt"] // info["tp_adj"]
    if do_t:
        aa, ak = kernel_table(per_adj, algorithmic_bytes_transposed(cfg, False, split))
        ga, gk = kernel_table(per_grad, algorithmic_bytes_transposed(cfg, True, split))
        adj_ms = max_over_ranks(sum(aa.values()), world, dev)
        grad_ms = max_over_ranks(sum(ga.values()), world, dev)
        transposed = {"adjoint": {"ms": round(adj_ms, 4), "voxels_per_s": whole_job_value(voxels, world, adj_ms),
                                  "kernels": ak},
                      "grad_positions": {"ms": round(grad_ms, 4),
                                         "voxels_per_s": whole_job_value(voxels, world, grad_ms), "kernels": gk}}
        gb = gather_alg_bytes(cfg)
        parts = [k for k in ("ned_xfft_adj", "gather", "entry_sum") if k in aa]
        gms = sum(aa[k] for k in parts)
        tr = [traffic_for(k, cfg["name"]) for k in parts]
        interp_roofline = {"bound": "hbm",
                           "kernel": "adjoint " + " + ".join(parts) + " (transposed interpolation)",
                           "achieved": round(gb / (gms * 1e-3) / 1e9, 1), "peak": peak, "unit": "GB/s",
                           "frac": round(gb / (gms * 1e-3) / 1e9 / peak, 4),
                           "traffic": None if any(t is None for t in tr) else sum(tr) * passes,
                           "traffic_note": ("DRAM bytes of one launch of each of %s, times the %d passes of one "
                                            "adjoint" % (", ".join(parts), passes)),
                           "alg_bytes": gb, "alg_note": "read the grid rows R once, write g once",
                           "peak_source": peak_kind}

    # kernels launched in the timed region: the plan's own count per call
    # (forward, adjoint, gradient; nedner_plan_info)
    fwd_launches = info["launches_forward"]
    t_launches = info["launches_adjoint"] + info["launches_grad_positions"] if do_t else 0
    launches = fwd_launches * (args.steps + prof_steps) + t_launches * args.steps

    cufft = None
    if rank == 0 and not args.no_cufft:
        try:
            ours = {"ned_xy": (round(avg["ned_xfft"] + avg["ned_yfft"], 5)
                               if "ned_xfft" in avg and "ned_yfft" in avg else None),
                    "ner": round(avg["ner_lines"], 5) if "ner_lines" in avg else None,
                    "image": round(avg.get("img_yifft", 0.0) + avg.get("img_xc2r", 0.0), 5)}
            cufft = cufft_comparison(cfg, dev, flush, min(args.steps, 10), ours)
        except Exception as ex:  # a reference point, not required
            cufft = {"failed": str(ex)}

    cpu = None
    tol = {"nufft": 1e-5, "tensor_bf16": 3e-5, "tensor_fp16": 1e-5}[args.ned_mode]
    accuracy = {"rel_l2_vs_oracle": None, "max_abs_rel_vs_oracle": None, "tolerance_rel_l2": tol,
                "check": None}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            import oracle
            oracle.build()
            got = p_host.double().numpy()                      # the result of the timed host-buffer call
            if cfg["sensor_xy"].shape[0] * cfg["nx"] * cfg["ny"] * cfg["Nt"] <= 1e11:
                # small workloads: the whole oracle reconstruction, every voxel
                pr = oracle_problem(cfg)
                t0 = time.perf_counter()
                ref = oracle.forward(pr, np.asarray(cfg["g"], dtype=np.float64))
                secs = time.perf_counter() - t0
                accuracy["rel_l2_vs_oracle"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
                accuracy["max_abs_rel_vs_oracle"] = float(np.abs(got - ref).max() / np.abs(ref).max())
                accuracy["check"] = "every voxel against one full FP64 oracle reconstruction"
                cpu = {"value": voxels / secs, "unit": "voxels/s", "cores": os.cpu_count(), "kind": "oracle",
                       "sample": "one full FP64 oracle reconstruction of the workload (%.1f s)" % secs}
            else:
                jx, jy, F, secs, scale = oracle_sample(cfg, args.oracle_fraction, cfg["seed"] + 7)
                rl2, mx = sampled_errors(got, jx, jy, F)
                accuracy["rel_l2_vs_oracle"] = rl2
                accuracy["max_abs_rel_vs_oracle"] = mx
                lines = len(jx) * len(jy)
                accuracy["check"] = ("spectrum of the timed p0 on a seeded sample of %d of %d lateral lines "
                                     "(%.2f %%, no Nyquist index) at every depth frequency, against the FP64 "
                                     "oracle's direct sums there" % (lines, cfg["nx"] * cfg["ny"],
                                                                    100.0 * lines / (cfg["nx"] * cfg["ny"])))
                cpu = {"value": voxels / (secs * scale), "unit": "voxels/s", "cores": os.cpu_count(),
                       "kind": "oracle",
                       "sample": ("FP64 oracle on %d of %d lateral lines at all %d depth frequencies: %.1f s, "
                                  "scaled by lines (x%.1f) to one full reconstruction"
                                  % (lines, cfg["nx"] * cfg["ny"], cfg["nz"], secs, scale))}
        except Exception as ex:  # the baseline is reported, not required
            cpu = {"value": None, "unit": "voxels/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": "failed: %s" % ex}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "voxels/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded balls + 20 dB noise)",
                "config": {"workload": describe(cfg), "l2": "flushed before every timed call (256 MB write)",
                           "parallelism": "independent reconstruction per GPU", "ned_mode": args.ned_mode},
                "roofline": roofline, "spread_frac_of_peak": spread_frac, "interp_roofline": interp_roofline,
                "accuracy": accuracy, "kernels": kernels,
                "kernels_note": ("per-kernel times from nedner_forward_profiled (%d steps, CUDA events between "
                                 "the launches); ms_per_step from CUDA events around nedner_forward on its stream"
                                 % prof_steps),
                "transposed": transposed,
                "cpu_baseline": cpu, "cufft_comparison": cufft, "clocks": clk, "device_status_flags": status_flags,
                "e2e": {"value": whole_job_value(voxels, world, e2e_step), "unit": "voxels/s",
                        "h2d_bytes_per_step": int(g_host.numel() * 4), "d2h_bytes_per_step": int(p_host.numel() * 4)},
                "gpu_launches": launches,
                "wall_s_timed_region": round(wall, 3)}
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
