"""Benchmark: SU(3) Landau gauge fixing on 32^4 (eps = 0.5, seed 2), FP32 bulk
sweeps (12-real links, omega = 1.7) + FP64 polish to theta < 1e-14.

One step = the whole hot path on one field: ingest (layout + precision
conversion), bulk FP32 sweeps with the accumulated transformation G, exact
theta checks, promotion (G applied to the FP64 input), FP64 polishing sweeps
to theta < 1e-14, and egress of the fixed field.  The metric is site updates
per second (sweeps x V / time).  Inputs (604 MB complex128 links; 201 MB of
FP32 working links) are larger than the 129 MB L2, so no L2 flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank fixes its own field (replicas: independent problems,
no data-path collective) and rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DIMS = (32, 32, 32, 32)
EPS, SEED, OMEGA, TOL = 0.5, 2, 1.7, 1e-14
METRIC = "site updates/s (Landau 32^4, FP32-12 bulk + FP64 polish to theta<1e-14)"
WORKLOAD = "SU(3) Landau 32^4, eps=0.5, seed 2, OR omega=1.7, FP32-12 bulk + FP64 polish to theta<1e-14"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        finally:
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        for r in rows:
            for name, val in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"],
                                 r[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def algorithmic_bytes_per_site(kind: str) -> int:
    """Bytes one site update must move: its 8 links in and out, plus G(x) in and
    out during the FP32 bulk phase (FP32-12 links 48 B, FP64 links 144 B, G 72 B)."""
    if kind == "fp32_12":
        return 16 * 48 + 2 * 72
    if kind == "fp32_18":
        return 16 * 72 + 2 * 72
    return 16 * 144


def cpu_baseline(budget_s: float = 12.0):
    """The FP64 oracle, as it stands, on this host's cores: full sweeps of the
    same 32^4 field until about budget_s of work; site updates per second."""
    import oracle as O
    from paper_1305_3440_gb300 import synth
    U = synth.field(DIMS, EPS, SEED)
    vol = int(np.prod(DIMS))
    n = 0
    t0 = time.perf_counter()
    while True:
        O.sweeps(U, 1, omega=OMEGA, sweep0=n)
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": n * vol / dt, "unit": "site updates/s", "cores": O.max_threads(), "kind": "oracle",
            "sample": f"{n} FP64 OR sweeps of the 32^4 field ({n * vol} site updates, {dt:.1f} s)"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    from paper_1305_3440_gb300 import synth
    U = synth.field(DIMS, EPS, SEED)
    vol = int(np.prod(DIMS))
    per_step = 2  # bounded sample: two full sweeps of the field per step
    for w in range(args.warmup):
        O.sweeps(U, 1, omega=OMEGA, sweep0=w)
    t0 = time.perf_counter()
    for s in range(args.steps):
        O.sweeps(U, per_step, omega=OMEGA, sweep0=args.warmup + per_step * s)
    dt = time.perf_counter() - t0
    value = args.steps * per_step * vol / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "site updates/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "l2": "inputs larger than L2"},
            "cpu_baseline": {"value": value, "unit": "site updates/s", "cores": O.max_threads(), "kind": "oracle",
                             "sample": f"{per_step} FP64 OR sweeps of the 32^4 field per step"},
            "e2e": {"value": value, "unit": "site updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1305_3440_gb300 import lgt, synth

    vol = int(np.prod(DIMS))
    U = synth.field(DIMS, EPS, SEED + rank)
    host_in = torch.from_numpy(U).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    dev_in = host_in.to(f"cuda:{local}")
    dev_out = torch.empty_like(dev_in)
    stream = torch.cuda.Stream()
    p = lgt.lgt_params_default(dims=DIMS, omega=OMEGA, bulk=lgt.LGT_FP32_12, theta_tol=TOL, max_sweeps=20000)
    ctx = lgt.lgt_create(p, dev_in, stream=stream)

    def step(src, dst):
        lgt.lgt_load(ctx, src)
        st, res = lgt.lgt_fix(ctx)
        if st != lgt.LGT_OK:
            raise RuntimeError(f"not converged: {res.as_dict()}")
        lgt.lgt_get_links(ctx, out=dst)
        return res

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        step(dev_in, dev_out)
    # ---- timed: inputs resident in HBM
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sweeps = 0
    stats_kernel = {"bulk_ms": 0.0, "bulk_launches": 0, "fp64_ms": 0.0, "fp64_launches": 0, "launches": 0}
    results = []
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            res = step(dev_in, dev_out)
            st = lgt.lgt_get_stats(ctx)
            stats_kernel["bulk_ms"] += st.sweep_ms[0]
            stats_kernel["bulk_launches"] += st.sweep_launches[0]
            stats_kernel["fp64_ms"] += st.sweep_ms[1]
            stats_kernel["fp64_launches"] += st.sweep_launches[1]
            stats_kernel["launches"] += st.launches
            sweeps += res.sweeps_bulk + res.sweeps_fp64
            results.append(res.as_dict())
        ev1.record(stream)
        torch.cuda.synchronize()
    clocks = clk.summary()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    barrier()
    t_max = elapsed
    upd = float(sweeps * vol)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([elapsed], device=f"cuda:{local}")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
        u = torch.tensor([upd], device=f"cuda:{local}", dtype=torch.float64)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        upd = float(u.item())
    value = upd / t_max

    # ---- end to end through the C ABI with host buffers (copies timed)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e_sweeps = 0
    e0.record(stream)
    for _ in range(args.steps):
        res = step(host_in.numpy(), host_out.numpy())
        e_sweeps += res.sweeps_bulk + res.sweeps_fp64
    e1.record(stream)
    torch.cuda.synchronize()
    e_elapsed = e0.elapsed_time(e1) / 1e3
    e2e = {"value": e_sweeps * vol * world / e_elapsed, "unit": "site updates/s",
           "h2d_bytes_per_step": int(host_in.numel() * 16), "d2h_bytes_per_step": int(host_out.numel() * 16)}
    assert np.array_equal(host_out.numpy(), dev_out.cpu().numpy())

    # ---- roofline of the dominant kernel (live CUDA events on the launching stream)
    peaks, src = measured_peaks()
    kinds = {"fp32_12": (stats_kernel["bulk_ms"], stats_kernel["bulk_launches"]),
             "fp64": (stats_kernel["fp64_ms"], stats_kernel["fp64_launches"])}
    dom = max(kinds, key=lambda k: kinds[k][0])
    kernels = {}
    for k, (ms, n) in kinds.items():
        if n == 0:
            continue
        avg_s = ms / 1e3 / n
        bytes_launch = algorithmic_bytes_per_site(k) * (vol // 2)
        kernels[k] = {"avg_launch_us": avg_s * 1e6, "launches": n, "total_ms": ms,
                      "achieved_gbs": bytes_launch / avg_s / 1e9, "bytes_per_launch": bytes_launch}
    d = kernels[dom]
    roofline = {"bound": "hbm", "achieved": d["achieved_gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": d["achieved_gbs"] / peaks["hbm_gbs"], "traffic": None,
                "kernel": f"half-sweep {dom}", "peak_source": src}

    # ---- all-FP64 time to theta < 1e-14 on the same field, for the ladder comparison
    ttt = {"mixed_s": elapsed / args.steps}
    if not args.no_fp64_compare and rank == 0:
        p64 = lgt.lgt_params_default(dims=DIMS, omega=OMEGA, bulk=lgt.LGT_FP64, theta_tol=TOL, max_sweeps=50000)
        c64 = lgt.lgt_create(p64, dev_in, stream=stream)
        try:
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            st64, r64 = lgt.lgt_fix(c64)
            f1.record(stream)
            torch.cuda.synchronize()
            ttt.update({"fp64_s": f0.elapsed_time(f1) / 1e3, "fp64_sweeps": r64.sweeps_fp64,
                        "fp64_F": r64.F, "fp64_theta": r64.theta})
            ttt["speedup"] = ttt["fp64_s"] / ttt["mixed_s"]
            s64 = lgt.lgt_get_stats(c64)
            if s64.sweep_launches[1]:
                avg = s64.sweep_ms[1] / 1e3 / s64.sweep_launches[1]
                kernels["fp64_only_run"] = {"avg_launch_us": avg * 1e6, "launches": s64.sweep_launches[1],
                                            "site_updates_per_s": (vol // 2) / avg}
        finally:
            lgt.lgt_destroy(c64)
    lgt.lgt_destroy(ctx)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
    if rank == 0:
        last = results[-1]
        line = {"metric": METRIC, "value": value, "unit": "site updates/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "fp32+f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "dims": list(DIMS), "bulk": "fp32_12", "omega": OMEGA,
                           "theta_tol": TOL, "l2": "inputs larger than L2 (604 MB FP64 + 201 MB FP32 links)",
                           "parallelism": f"replicas x{world}"},
                "sweeps_per_step": {"bulk": last["sweeps_bulk"], "fp64": last["sweeps_fp64"]},
                "result": {"F": last["F"], "theta": last["theta"], "plaquette": last["plaquette"]},
                "time_to_theta_1e-14": ttt, "kernels": kernels, "roofline": roofline, "e2e": e2e,
                "gpu_launches": stats_kernel["launches"], "clocks": clocks, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
