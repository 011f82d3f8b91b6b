"""Benchmark: SU(3) Landau gauge fixing on 32^4 (eps = 0.5, seed 2), FP32 bulk
sweeps (12-real links, omega = 1.7) + anchored polish to theta < 1e-14.

One step = the whole hot path on one field: ingest (layout + precision
conversion), bulk FP32 sweeps with the accumulated transformation G and the
sweeps' fused theta estimate, promotion (G applied in FP64 to the FP64 input),
anchored polishing sweeps (the promoted field fixed, only G = 1 + D relaxed,
in FP32-pair precision) to theta < 1e-14 certified by the exact FP64
measurement, and egress of the fixed field.  The metric is site updates
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
METRIC = "site updates/s (Landau 32^4 to theta<1e-14, mixed precision)"
WORKLOAD = ("SU(3) Landau 32^4, eps=0.5, seed 2, OR omega=1.7, FP32-12 bulk + anchored polish to theta<1e-14 "
            "(exact FP64 measurement certifies)")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--workload", default="landau32",
                    choices=["landau32", "coulomb", "landau64", "serve", "mag", "profile", "slab"],
                    help="landau32 (default; the headline line), or one of the other workloads, each "
                         "printing its own line; profile: a short fixed run of the sweep kernels for ncu")
    ap.add_argument("--jobs", type=int, default=256, help="serve: number of jobs in the stream")
    ap.add_argument("--serve-jobs", type=int, default=32,
                    help="landau32: jobs of the served-stream sample reported beside the headline")
    ap.add_argument("--no-serve", action="store_true", help="landau32: skip the served-stream sample")
    prof = ap.add_argument_group("profile", "the short fixed run of --workload profile")
    prof.add_argument("--dims", type=int, nargs=4, default=[32, 32, 32, 32])
    prof.add_argument("--eps", type=float, default=0.5)
    prof.add_argument("--seed", type=int, default=2)
    prof.add_argument("--gauge", default="landau", choices=["landau", "coulomb", "mag"])
    prof.add_argument("--bulk", default="fp32_12", choices=["fp32_12", "fp32_18", "fp64"])
    prof.add_argument("--omega", type=float, default=1.7)
    prof.add_argument("--bulk-sweeps", type=int, default=8)
    prof.add_argument("--polish-sweeps", type=int, default=4)
    prof.add_argument("--polish", default="anchor", choices=["anchor", "pair", "fp64"])
    prof.add_argument("--launch-config", type=int, default=-1,
                      help="force launch configuration k of the sweep kernels (-1: autotuned)")
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


# The sources of the bulk sweep kernel: a recorded ncu traffic figure is used
# only while their hash equals the one recorded with it.
KERNEL_SOURCES = ("paper_1305_3440_gb300/csrc/lgt_sweep.cuh", "paper_1305_3440_gb300/csrc/lgt_sweep_f32.cu",
                  "paper_1305_3440_gb300/csrc/lgt_device.cuh", "paper_1305_3440_gb300/csrc/lgt_anchor.cuh",
                  "paper_1305_3440_gb300/csrc/lgt_pair.cuh", "paper_1305_3440_gb300/csrc/lgt_internal.h")


def kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, launch_config: int):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) that an
    ncu capture recorded for this kernel and launch configuration at 32^4, from
    the `traffic-record:` lines of profiles/*.md; None when there is none or the
    kernel sources changed since."""
    import glob
    import re
    want = kernel_source_hash()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for line in f:
                m = re.match(r"\s*traffic-record: kernel=(\S+) config=(\d+) bytes_per_launch=(\d+) sources=(\w+)", line)
                if m and m.group(1) == kernel and int(m.group(2)) == launch_config and m.group(4) == want:
                    return int(m.group(3))
    return None


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
        watts = []
        for r in rows:
            try:
                watts.append(float(r[3]))
            except ValueError:
                pass
        reasons = set()
        for r in rows:
            for name, val in zip(["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"],
                                 r[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows), "sm_mhz_min": min(sm) if sm else None,
                "power_w_max": max(watts) if watts else None}


def algorithmic_bytes_per_site(kind: str) -> int:
    """Bytes one site update must move.  Bulk: its 8 links in and out plus G(x) in
    and out (FP32-12 links 48 B, FP32-18 72 B, G stored as 2 rows: 48 B).
    FP32-pair and FP64 polish: 8 links of 144 B in and out.  Anchored polish:
    K0(x) (144 B) and the 8 links' FP32-12 copies (384 B) in, its own D (96 B:
    rows 0, 1 as pairs) in and out, and the other parity's D high parts (48 B
    per site: each is read by 8 neighbours, compulsory once)."""
    if kind == "fp32_12":
        return 16 * 48 + 2 * 48
    if kind == "fp32_18":
        return 16 * 72 + 2 * 48
    if kind == "anchor":
        return 144 + 8 * 48 + 48 + 2 * 96
    if kind == "anchor_coulomb":  # spatial directions only
        return 144 + 6 * 48 + 48 + 2 * 96
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
    cores = O.max_threads()
    # one core, one sweep, for the per-core rate
    O.set_threads(1)
    try:
        t1 = time.perf_counter()
        O.sweeps(U, 1, omega=OMEGA, sweep0=n)
        dt1 = time.perf_counter() - t1
    finally:
        O.set_threads(cores)
    # the 8^4 latency case to convergence
    U8 = synth.field((8, 8, 8, 8), 0.3, 1)
    t2 = time.perf_counter()
    r8 = O.fix(U8, omega=OMEGA, tol=TOL, max_sweeps=1000)
    dt8 = time.perf_counter() - t2
    return {"value": n * vol / dt, "unit": "site updates/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} FP64 OR sweeps of the 32^4 field ({n * vol} site updates, {dt:.1f} s)",
            "single_core": {"value": vol / dt1, "sample": "1 sweep of the 32^4 field on 1 thread"},
            "fix_8x4": {"seconds": dt8, "sweeps": r8["sweeps"], "converged": bool(r8["converged"]),
                        "sample": "8^4, eps 0.3, seed 1, OR omega 1.7 to theta < 1e-14"}}


def aggregate_over_ranks(elapsed_s: float, units: float, device=None):
    """(max elapsed over ranks, sum of units over ranks); plain values on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return elapsed_s, units
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


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
    # the workload fixes omega = 1.7 for the FP32 sweeps; the polish uses the
    # library's default omega_polish
    p = lgt.lgt_params_default(dims=DIMS, omega=OMEGA, bulk=lgt.LGT_FP32_12, theta_tol=TOL, max_sweeps=20000)
    # The timed fixes issue their chunks from the host (LGT_FIX_GRAPHS=0), so each
    # chunk's events bracket that chunk's sweep-kernel launches and nothing else:
    # the roofline divides by the kernel's own time.  The device loop (one graph
    # launch per many chunks) runs the same kernels in the same time and is timed
    # beside it (other_runs.device_loop).
    saved = os.environ.get("LGT_FIX_GRAPHS")
    os.environ["LGT_FIX_GRAPHS"] = "0"
    try:
        ctx = lgt.lgt_create(p, dev_in, stream=stream)
    finally:
        if saved is None:
            os.environ.pop("LGT_FIX_GRAPHS", None)
        else:
            os.environ["LGT_FIX_GRAPHS"] = saved

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
        # profilers started with "collect from cudaProfilerStart" see the timed steps only
        torch.cuda.profiler.start()
        ev0.record(stream)
        step_ev = []
        for _ in range(args.steps):
            step_ev.append(torch.cuda.Event(enable_timing=True))
            step_ev[-1].record(stream)
            res = step(dev_in, dev_out)
            st = lgt.lgt_get_stats(ctx)
            stats_kernel["bulk_ms"] += st.sweep_ms[0]
            stats_kernel["bulk_launches"] += st.sweep_launches[0]
            stats_kernel["fp64_ms"] += st.sweep_ms[1]
            stats_kernel["fp64_launches"] += st.sweep_launches[1]
            stats_kernel["launches"] += st.launches
            stats_kernel["launch_config"] = list(st.launch_config)
            stats_kernel["loop_launches"] = stats_kernel.get("loop_launches", 0) + st.loop_launches
            stats_kernel["loop_chunks"] = stats_kernel.get("loop_chunks", 0) + st.loop_chunks
            sweeps += res.sweeps_bulk + res.sweeps_fp64
            results.append(res.as_dict())
        ev1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
    clocks = clk.summary()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    step_ev.append(ev1)
    step_ms = [round(step_ev[k].elapsed_time(step_ev[k + 1]), 2) for k in range(args.steps)]
    barrier()
    t_max, upd = aggregate_over_ranks(elapsed, float(sweeps * vol), device=f"cuda:{local}")
    value = upd / t_max

    # ---- end to end through the C ABI with host buffers (copies timed); one untimed
    # step first allocates the context's staging buffer for host links
    step(host_in.numpy(), host_out.numpy())
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the host link of this machine: one timed copy each way of the step's buffers
    # (outside the timed region; the same transfers lgt_load / lgt_get_links make)
    c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    c0.record(stream)
    with torch.cuda.stream(stream):
        dev_out.copy_(host_in, non_blocking=True)
        c1.record(stream)
        host_out.copy_(dev_out, non_blocking=True)
    c2.record(stream)
    torch.cuda.synchronize()
    copy_gbs = {"h2d": round(host_in.numel() * 16 / c0.elapsed_time(c1) / 1e6, 1),
                "d2h": round(host_out.numel() * 16 / c1.elapsed_time(c2) / 1e6, 1)}
    lgt.lgt_get_links(ctx, out=dev_out)
    e_sweeps = 0
    with ClockSampler(local) as e_clk:
        e0.record(stream)
        e_ev = []
        for _ in range(args.steps):
            e_ev.append(torch.cuda.Event(enable_timing=True))
            e_ev[-1].record(stream)
            res = step(host_in.numpy(), host_out.numpy())
            e_sweeps += res.sweeps_bulk + res.sweeps_fp64
        e1.record(stream)
        torch.cuda.synchronize()
    e_elapsed = e0.elapsed_time(e1) / 1e3
    e_ev.append(e1)
    e2e = {"value": e_sweeps * vol * world / e_elapsed, "unit": "site updates/s",
           "h2d_bytes_per_step": int(host_in.numel() * 16), "d2h_bytes_per_step": int(host_out.numel() * 16),
           "step_ms": [round(e_ev[k].elapsed_time(e_ev[k + 1]), 2) for k in range(args.steps)],
           "clocks": e_clk.summary(), "pinned_copy_gbs": copy_gbs}
    assert np.array_equal(host_out.numpy(), dev_out.cpu().numpy())

    # ---- roofline of the dominant kernel (live CUDA events on the launching stream)
    peaks, src = measured_peaks()
    kinds = {"fp32_12": (stats_kernel["bulk_ms"], stats_kernel["bulk_launches"]),
             "anchor": (stats_kernel["fp64_ms"], stats_kernel["fp64_launches"])}
    dom = max(kinds, key=lambda k: kinds[k][0])
    kernels = {}
    for k, (ms, n) in kinds.items():
        if n == 0:
            continue
        avg_s = ms / 1e3 / n
        bytes_launch = algorithmic_bytes_per_site(k) * (vol // 2)
        kernels[k] = {"avg_launch_us": avg_s * 1e6, "launches": n, "total_ms": ms,
                      "achieved_gbs": bytes_launch / avg_s / 1e9, "bytes_per_launch": bytes_launch,
                      "launch_config": stats_kernel["launch_config"][0 if k == "fp32_12" else 1]}
    d = kernels[dom]
    roofline = {"bound": "hbm", "achieved": d["achieved_gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": d["achieved_gbs"] / peaks["hbm_gbs"],
                "traffic": recorded_traffic("k_sweep_f32" if dom == "fp32_12" else "k_sweep_anchor",
                                            d["launch_config"]),
                "kernel": f"half-sweep {dom}", "peak_source": src,
                "bytes_per_site_update": algorithmic_bytes_per_site(dom), "units_per_launch": vol // 2}
    if roofline["traffic"]:  # the DRAM bandwidth the kernel draws (L2 serves the rest of the algorithmic bytes)
        avg_s = d["bytes_per_launch"] / (d["achieved_gbs"] * 1e9)
        roofline["dram_gbs"] = roofline["traffic"] / avg_s / 1e9
        roofline["dram_frac"] = roofline["dram_gbs"] / peaks["hbm_gbs"]

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
                kernels["fp64"] = {"avg_launch_us": avg * 1e6, "launches": s64.sweep_launches[1],
                                   "achieved_gbs": algorithmic_bytes_per_site("fp64") * (vol // 2) / avg / 1e9,
                                   "site_updates_per_s": (vol // 2) / avg, "run": "all-FP64 comparison"}
        finally:
            lgt.lgt_destroy(c64)
    # ---- the other runs of the 32^4 workload (FP32-18 bulk; SR p = 0.8 on the same
    # ladder) and the 8^4 latency case, one timed lgt_fix each, reported beside
    variants = {}
    if not args.no_fp64_compare and rank == 0:
        runs = [("device_loop", DIMS, dev_in, dict(bulk=lgt.LGT_FP32_12, omega=OMEGA)),
                ("fp32_18_bulk", DIMS, dev_in, dict(bulk=lgt.LGT_FP32_18, omega=OMEGA)),
                ("sr_p0.8", DIMS, dev_in, dict(bulk=lgt.LGT_FP32_12, algo=lgt.LGT_SR, p=0.8, seed=SEED)),
                # the same stochastic relaxation, polished by overrelaxation after promotion
                ("sr_p0.8_or_polish", DIMS, dev_in, dict(bulk=lgt.LGT_FP32_12, algo=lgt.LGT_SR, p=0.8, seed=SEED,
                                                         polish_algo=lgt.LGT_POLISH_OR)),
                # an omega schedule, not the workload's fixed omega: 1.7 until the sweeps'
                # estimate of theta drops below 1e-2, then 1.1
                ("omega_schedule_1.7_to_1.1", DIMS, dev_in,
                 dict(bulk=lgt.LGT_FP32_12, omega=OMEGA, omega_late=1.1, theta_omega=1e-2)),
                # simulated annealing first (200 heat-bath sweeps, beta 1 -> 100), then the ladder
                ("annealing_200", DIMS, dev_in,
                 dict(bulk=lgt.LGT_FP32_12, omega=OMEGA, sa_sweeps=200, sa_beta0=1.0, sa_beta1=100.0))]
        small = torch.from_numpy(synth.field((8, 8, 8, 8), 0.3, 1)).to(f"cuda:{local}")
        runs += [("8x4_fp64", (8, 8, 8, 8), small, dict(bulk=lgt.LGT_FP64, omega=OMEGA, max_sweeps=1000)),
                 ("8x4_mixed", (8, 8, 8, 8), small, dict(bulk=lgt.LGT_FP32_12, omega=OMEGA, max_sweeps=1000))]
        for name, dims, src, kw in runs:
            kw = dict(dict(theta_tol=TOL, max_sweeps=50000), **kw)
            cv = lgt.lgt_create(lgt.lgt_params_default(dims=dims, **kw), src, stream=stream)
            try:
                times = []
                for _ in range(3 if dims != DIMS else 1):
                    sec, stv, rv, sv = _timed_fix(lgt, cv, src, stream)
                    times.append(sec)
                variants[name] = {"seconds": float(np.median(times)), "status": stv, "sweeps_bulk": rv.sweeps_bulk,
                                  "sweeps_polish": rv.sweeps_fp64, "F": rv.F, "theta": rv.theta,
                                  "launch_config": list(sv.launch_config)}
                if dims == DIMS:
                    variants[name]["F_minus_headline_F"] = rv.F - results[-1]["F"]
                if name == "device_loop":
                    variants[name].update(graph_launches=sv.loop_launches, chunks=sv.loop_chunks,
                                          mixed_s_host_chunks=elapsed / args.steps)
            finally:
                lgt.lgt_destroy(cv)
    # ---- SU(3) Coulomb gauge on 48^3 x 96 (96 timeslices per launch, per-slice theta_t <
    # 1e-14, eps 0.5, seed 3; the workload fixes no omega: the measured schedule)
    if not args.no_fp64_compare and rank == 0:
        cdims = (96, 48, 48, 48)
        cdev = torch.from_numpy(synth.field(cdims, 0.5, 3)).to(f"cuda:{local}")
        pc = lgt.lgt_params_default(dims=cdims, gauge=lgt.LGT_COULOMB, bulk=lgt.LGT_FP32_12, max_sweeps=50000,
                                    **SERVE_OMEGA)
        cc = lgt.lgt_create(pc, cdev, stream=stream)
        try:
            sec, stc, rc, sc = _timed_fix(lgt, cc, cdev, stream)
            th_t = lgt.lgt_measure_slices(cc, cdims[0])[1]
            variants["coulomb_48x3x96"] = {
                "seconds": sec, "status": stc, "sweeps_bulk": rc.sweeps_bulk, "sweeps_polish": rc.sweeps_fp64,
                "F_mean": rc.F, "theta_t_max": float(th_t.max()), "slices": cdims[0],
                "site_updates_per_s": (sc.site_updates[0] + sc.site_updates[1]) / sec,
                "launch_config": list(sc.launch_config), "omega": "1.7 -> 1.1 below theta 1e-2"}
        finally:
            lgt.lgt_destroy(cc)
        del cdev
    lgt.lgt_destroy(ctx)
    # ---- a bounded sample of the served stream (p50/p99 latency beside jobs/s)
    serve = None
    if rank == 0 and world == 1 and not args.no_serve:
        specs, gaps = serve_specs(args.serve_jobs)
        serve = serve_stream(lgt, specs, gaps, cap_jobs=len(specs))
        serve["workload"] = f"the first {len(specs)} jobs of the served stream: " + SERVE_WORKLOAD

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline()
    if rank == 0:
        last = results[-1]
        line = {"metric": METRIC, "value": value, "unit": "site updates/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "fp32+f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "dims": list(DIMS), "bulk": "fp32_12", "omega": OMEGA,
                           "omega_polish": p.omega_polish,
                           "theta_tol": TOL, "l2": "inputs larger than L2 (604 MB FP64 + 201 MB FP32 links)",
                           "parallelism": f"replicas x{world}"},
                "step_ms": step_ms,
                "sweeps_per_step": {"bulk_fp32": last["sweeps_bulk"], "polish": last["sweeps_fp64"]},
                "result": {"F": last["F"], "theta": last["theta"], "plaquette": last["plaquette"]},
                "time_to_theta_1e-14": ttt, "other_runs": variants, "kernels": kernels, "roofline": roofline,
                "e2e": e2e,
                "gpu_launches": stats_kernel["launches"],
                "chunks": "issued from the host in the timed steps; the device loop is other_runs.device_loop",
                "clocks": clocks, "cpu_baseline": cpu, "serve_sample": serve}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ------------------------------------------------------------ other workloads
def _timed_fix(lgt, ctx, src, stream):
    import torch
    lgt.lgt_load(ctx, src)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st, res = lgt.lgt_fix(ctx)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3, st, res, lgt.lgt_get_stats(ctx)


def _kernel_summary(stats, bytes_bulk, bytes_polish, vol):
    """Per sweep kernel: mean launch time and achieved GB/s from the site updates it
    actually did (converged Coulomb slices are skipped)."""
    out = {}
    for idx, (name, b) in enumerate([("bulk", bytes_bulk), ("polish", bytes_polish)]):
        if stats.sweep_launches[idx]:
            secs = stats.sweep_ms[idx] / 1e3
            out[name] = {"avg_launch_us": secs / stats.sweep_launches[idx] * 1e6,
                         "launches": stats.sweep_launches[idx], "site_updates": stats.site_updates[idx],
                         "achieved_gbs": b * stats.site_updates[idx] / secs / 1e9,
                         "launch_config": stats.launch_config[idx]}
    return out


def run_coulomb(args):
    """48^3 x 96 Coulomb gauge: 96 timeslice problems in one launch per half-sweep,
    per-slice convergence theta_t < 1e-14 (converged slices masked off)."""
    import torch
    from paper_1305_3440_gb300 import lgt, synth
    dims = (96, 48, 48, 48)
    vol = int(np.prod(dims))
    U = synth.field(dims, 0.5, 3)
    dev = torch.from_numpy(U).cuda()
    del U
    stream = torch.cuda.Stream()
    p = lgt.lgt_params_default(dims=dims, gauge=lgt.LGT_COULOMB, omega=1.7, bulk=lgt.LGT_FP32_12, max_sweeps=50000)
    ctx = lgt.lgt_create(p, dev, stream=stream)
    for _ in range(args.warmup):
        _timed_fix(lgt, ctx, dev, stream)
    times, res, stats = [], None, None
    for _ in range(args.steps):
        t, st, res, stats = _timed_fix(lgt, ctx, dev, stream)
        assert st == lgt.LGT_OK, res.as_dict()
        times.append(t)
    F_t, th_t = lgt.lgt_measure_slices(ctx, dims[0])
    lgt.lgt_destroy(ctx)
    # converged slices are skipped: count the site updates actually done
    t = float(np.median(times))
    updates = stats.site_updates[0] + stats.site_updates[1]
    peaks, src = measured_peaks()
    kern = _kernel_summary(stats, 12 * 48 + 2 * 48 + 4 * 48, algorithmic_bytes_per_site("anchor_coulomb"), vol)
    line = {"workload": "coulomb", "metric": "time to max_t theta_t<1e-14 (s)", "value": t, "unit": "s",
            "higher_is_better": False, "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": "SU(3) Coulomb 48^3x96, eps=0.5, seed 3, OR omega=1.7, FP32-12 bulk + "
                                   "anchored polish, 96 slices per launch, per-slice convergence",
                       "block_sizes": "autotuned"},
            "sweeps": {"bulk_fp32": res.sweeps_bulk, "polish": res.sweeps_fp64},
            "site_updates_per_s": updates / t, "site_updates": updates,
            "result": {"F_mean": res.F, "theta_max": res.theta, "theta_t_max": float(th_t.max()),
                       "theta_t_min": float(th_t.min()), "plaquette": res.plaquette},
            "kernels": kern, "hbm_peak_gbs": peaks["hbm_gbs"], "peak_source": src}
    print(json.dumps(line), flush=True)


def run_landau64(args):
    """64^4 Landau, eps 0.7, seed 5: OR omega 1.8 vs SR p 0.9 through the ladder
    to theta < 1e-14, and the all-FP64 sweep rate (50 sweeps) for the same field."""
    import torch
    from paper_1305_3440_gb300 import lgt, synth
    dims = (64, 64, 64, 64)
    vol = int(np.prod(dims))
    U = synth.field(dims, 0.7, 5)
    dev = torch.from_numpy(U).cuda()
    stream = torch.cuda.Stream()
    out = {}
    for name, kw in [("or_1.8", dict(algo=lgt.LGT_OR, omega=1.8)), ("sr_0.9", dict(algo=lgt.LGT_SR, p=0.9, seed=5)),
                     ("sr_0.9_or_polish", dict(algo=lgt.LGT_SR, p=0.9, seed=5, polish_algo=lgt.LGT_POLISH_OR))]:
        p = lgt.lgt_params_default(dims=dims, bulk=lgt.LGT_FP32_12, max_sweeps=100000, **kw)
        ctx = lgt.lgt_create(p, dev, stream=stream)
        t, st, res, stats = _timed_fix(lgt, ctx, dev, stream)
        lgt.lgt_destroy(ctx)
        out[name] = {"status": st, "seconds": t, "sweeps_bulk": res.sweeps_bulk, "sweeps_polish": res.sweeps_fp64,
                     "F": res.F, "theta": res.theta, "site_updates_per_s": (res.sweeps_bulk + res.sweeps_fp64) * vol / t,
                     "kernels": _kernel_summary(stats, 16 * 48 + 2 * 48, algorithmic_bytes_per_site("anchor"), vol)}
    p = lgt.lgt_params_default(dims=dims, bulk=lgt.LGT_FP64, omega=1.8)
    ctx = lgt.lgt_create(p, dev, stream=stream)
    lgt.lgt_sweep(ctx, 2)
    s0 = lgt.lgt_get_stats(ctx)
    lgt.lgt_sweep(ctx, 50)
    s1 = lgt.lgt_get_stats(ctx)
    lgt.lgt_destroy(ctx)
    avg = (s1.sweep_ms[1] - s0.sweep_ms[1]) / 1e3 / (s1.sweep_launches[1] - s0.sweep_launches[1])
    out["fp64_rate"] = {"avg_launch_us": avg * 1e6, "site_updates_per_s": (vol // 2) / avg,
                        "achieved_gbs": 2304 * (vol // 2) / avg / 1e9}
    for name in ("or_1.8", "sr_0.9", "sr_0.9_or_polish"):
        n = out[name]["sweeps_bulk"] + out[name]["sweeps_polish"]
        out[name]["fp64_estimate_s"] = n * 2 * avg
    # the FP64 oracle on the host cores: one untimed sweep, then 5 timed OR sweeps
    # of the same field (ω 1.8)
    cpu = None
    if not args.no_cpu_baseline:
        import oracle as O
        O.sweeps(U, 1, omega=1.8, sweep0=0)
        t0 = time.perf_counter()
        O.sweeps(U, 5, omega=1.8, sweep0=1)
        dt = time.perf_counter() - t0
        cpu = {"value": 5 * vol / dt, "unit": "site updates/s", "cores": O.max_threads(), "kind": "oracle",
               "sample": f"5 FP64 OR sweeps of the 64^4 field ({dt:.1f} s)"}
    del U
    peaks, src = measured_peaks()
    print(json.dumps({"workload": "landau64", "config": {"workload": "SU(3) Landau 64^4, eps=0.7, seed 5"},
                      "runs": out, "hbm_peak_gbs": peaks["hbm_gbs"], "peak_source": src,
                      "cpu_baseline": cpu}), flush=True)


def run_mag(args):
    """Maximally Abelian gauge.  The bulk sweep rate on the 32^4 field of the headline
    workload (FP32-12 links, OR omega 1.7; 20 sweeps untimed, then 200 sweeps timed by
    the sweep kernels' CUDA events; algorithmic bytes per site as the Landau bulk
    kernel: the 8 links and G read and written once, 864 B) and the FP64 sweep rate
    of the same field; then a 16^4 field (eps 0.5, seed 3) fixed to theta_MAG < 1e-12
    through the ladder, and an 8^4 gauge-transformed Abelian field fixed back to
    F_MAG = 1."""
    import torch
    from paper_1305_3440_gb300 import lgt, synth
    stream = torch.cuda.Stream()
    peaks, src = measured_peaks()
    out = {}
    dims = (32, 32, 32, 32)
    vol = int(np.prod(dims))
    dev = torch.from_numpy(synth.field(dims, 0.5, 2)).cuda()
    for name, bulk, bytes_per_site in [("bulk_fp32_12", lgt.LGT_FP32_12, algorithmic_bytes_per_site("fp32_12")),
                                       ("fp64", lgt.LGT_FP64, 2304)]:
        p = lgt.lgt_params_default(dims=dims, gauge=lgt.LGT_MAG, bulk=bulk, omega=1.7)
        ctx = lgt.lgt_create(p, dev, stream=stream)
        n = 200 if bulk != lgt.LGT_FP64 else 20
        kind = 0 if bulk != lgt.LGT_FP64 else 1
        lgt.lgt_sweep(ctx, 20)
        s0 = lgt.lgt_get_stats(ctx)
        lgt.lgt_sweep(ctx, n)
        s1 = lgt.lgt_get_stats(ctx)
        F, theta, _ = lgt.lgt_measure(ctx)
        lgt.lgt_destroy(ctx)
        avg = (s1.sweep_ms[kind] - s0.sweep_ms[kind]) / 1e3 / (s1.sweep_launches[kind] - s0.sweep_launches[kind])
        gbs = bytes_per_site * (vol // 2) / avg / 1e9
        out[name] = {"sweeps": n, "avg_half_sweep_us": avg * 1e6, "site_updates_per_s": (vol // 2) / avg,
                     "achieved_gbs": gbs, "frac_of_hbm_peak": gbs / peaks["hbm_gbs"],
                     "bytes_per_site_update": bytes_per_site, "launch_config": list(s1.launch_config),
                     "F_after": F, "theta_after": theta}
    del dev
    dims = (16, 16, 16, 16)
    dev = torch.from_numpy(synth.field(dims, 0.5, 3)).cuda()
    p = lgt.lgt_params_default(dims=dims, gauge=lgt.LGT_MAG, bulk=lgt.LGT_FP32_12, omega=1.7, theta_tol=1e-12,
                               max_sweeps=30000)
    ctx = lgt.lgt_create(p, dev, stream=stream)
    t, st, res, stats = _timed_fix(lgt, ctx, dev, stream)
    lgt.lgt_destroy(ctx)
    out["fix_16x4"] = {"status": st, "seconds": t, "sweeps_bulk": res.sweeps_bulk, "sweeps_polish": res.sweeps_fp64,
                       "F": res.F, "theta": res.theta,
                       "site_updates_per_s": (res.sweeps_bulk + res.sweeps_fp64) * int(np.prod(dims)) / t}
    print(json.dumps({"workload": "mag", "metric": "site updates/s (maximally Abelian gauge sweeps, 32^4)",
                      "value": out["bulk_fp32_12"]["site_updates_per_s"], "unit": "site updates/s",
                      "config": {"workload": "SU(3) maximally Abelian gauge: 32^4 eps 0.5 seed 2 sweep rates; "
                                             "16^4 eps 0.5 seed 3 fixed to theta_MAG < 1e-12"},
                      "runs": out, "hbm_peak_gbs": peaks["hbm_gbs"], "peak_source": src}), flush=True)


def serve_specs(n_jobs: int, seed: int = 4):
    """The served stream: dims uniform over six lattices, Landau/Coulomb 50/50,
    tol 1e-12/1e-14, eps ~ U[0.3, 0.7], job seed 1000 + j."""
    rng = np.random.default_rng(seed)
    shapes = [(16, 16, 16, 16), (24, 24, 24, 24), (32, 32, 32, 32), (32, 16, 16, 16), (64, 32, 32, 32),
              (48, 48, 48, 48)]
    specs = []
    for j in range(n_jobs):
        specs.append(dict(dims=shapes[rng.integers(len(shapes))], gauge=int(rng.integers(2)),
                          tol=[1e-12, 1e-14][rng.integers(2)], eps=float(rng.uniform(0.3, 0.7)), seed=1000 + j))
    gaps = rng.exponential(1.0, size=n_jobs)  # unit-rate inter-arrival times, scaled later
    return specs, gaps


# The served jobs fix no omega, so they run the measured omega schedule: overrelaxation
# at 1.7 until the sweeps' estimate of theta drops below 1e-2, then 1.1 (on GB300 the
# best or within 1% of it for every lattice of the stream, Landau and Coulomb, eps 0.3
# to 0.7: about half the sweeps of a fixed 1.7).
SERVE_OMEGA = dict(omega=1.7, omega_late=1.1, theta_omega=1e-2)


def serve_stream(lgt, specs, gaps, cap_jobs: int, load: float = 0.8, max_outstanding: int = 12):
    """Continuous batching, measured twice on one job list.  Capacity: the first
    cap_jobs jobs in a closed loop (at most max_outstanding outstanding, so inputs
    are generated as the GPU drains them).  Then every job of the list with Poisson
    arrivals at `load` x capacity.  Latency is submit-to-completion of each job
    (lgt_result.seconds); the breakdown is per lattice size."""
    import queue
    import threading
    from paper_1305_3440_gb300 import synth

    def params(sp):
        return lgt.lgt_params_default(dims=sp["dims"], gauge=sp["gauge"], theta_tol=sp["tol"],
                                      bulk=lgt.LGT_FP32_12, max_sweeps=100000, **SERVE_OMEGA)

    # The clients' inputs.  Made before timing when they fit in a modest share of
    # host memory; otherwise a producer thread makes them during the run on all but
    # three cores, so that the server's worker thread (which issues the GPU's ticks)
    # and the polling thread are never starved by the generator.
    n_bytes = sum(int(np.prod(sp["dims"])) * 4 * 9 * 16 for sp in specs)
    try:
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    except (ValueError, OSError):
        avail = 0
    made = {}
    gen_threads = max(1, (os.cpu_count() or 4) - 3)
    if n_bytes <= min(48 << 30, avail // 3):
        for j, sp in enumerate(specs):
            made[j] = synth.field(sp["dims"], sp["eps"], sp["seed"])
        inputs = f"made before timing ({n_bytes / 2**30:.1f} GB)"
    else:
        inputs = f"made during the run by a producer thread on {gen_threads} cores"

    def producer(qu, subset):
        for j, sp in enumerate(subset):
            U = made.get(j)
            if U is None:
                U = synth.field(sp["dims"], sp["eps"], sp["seed"], threads=gen_threads)
            qu.put((sp, U))
        qu.put(None)

    def drain(srv, pending, done):
        for j in list(pending):
            st, res = lgt.lgt_poll(srv, j)
            if st != lgt.LGT_EAGAIN:
                sp = pending.pop(j)
                upd = (res.sweeps_bulk + res.sweeps_fp64) * int(np.prod(sp["dims"]))
                done.append((sp, res.seconds, st, upd))

    def run_stream(subset, rate, max_out):
        srv = lgt.lgt_server_create(150 << 30, 0)
        qu = queue.Queue(maxsize=4)
        threading.Thread(target=producer, args=(qu, subset), daemon=True).start()
        pending, done = {}, []
        t0 = time.perf_counter()
        t_next = t0
        k = 0
        while True:
            item = qu.get()
            if item is None:
                break
            sp, U = item
            if rate:
                t_next += gaps[k] / rate
                while time.perf_counter() < t_next:
                    time.sleep(0.0005)
                    drain(srv, pending, done)
            while max_out and len(pending) >= max_out:
                time.sleep(0.001)
                drain(srv, pending, done)
            jid = lgt.lgt_submit(srv, params(sp), U)
            pending[jid] = sp
            del U
            k += 1
            drain(srv, pending, done)
        while pending:
            time.sleep(0.001)
            drain(srv, pending, done)
        wall = time.perf_counter() - t0
        lgt.lgt_server_destroy(srv)
        return wall, done

    cap_list = specs[:min(cap_jobs, len(specs))]
    wall_c, done_c = run_stream(cap_list, None, max_outstanding)
    capacity = len(cap_list) / wall_c
    rate = load * capacity
    wall, done = run_stream(specs, rate, 0)
    lat = np.array([d[1] for d in done])
    per_size = {}
    for sp, sec, _, _ in done:
        key = "x".join(str(v) for v in sp["dims"][::-1]) + (" coulomb" if sp["gauge"] else " landau")
        per_size.setdefault(key, []).append(sec)
    breakdown = {k: {"jobs": len(v), "p50_s": float(np.percentile(v, 50)), "p99_s": float(np.percentile(v, 99)),
                     "max_s": float(np.max(v))} for k, v in sorted(per_size.items())}
    return {"jobs": len(specs), "capacity_jobs_per_s": capacity, "capacity_jobs": len(cap_list),
            "offered_rate_jobs_per_s": rate, "jobs_per_s": len(specs) / wall,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)), "max_s": float(lat.max()),
            "closed_loop_p50_s": float(np.percentile([d[1] for d in done_c], 50)),
            "all_converged": all(d[2] == lgt.LGT_OK for d in done + done_c), "inputs": inputs,
            # site updates the closed loop delivered per second of wall time (sweeps x volume
            # of every job), to set beside a single context's rate
            "closed_loop_site_updates_per_s": sum(d[3] for d in done_c) / wall_c,
            "per_size": breakdown}


SERVE_WORKLOAD = ("dims in {16^4, 24^4, 32^4, 16^3x32, 32^3x64, 48^4}, Landau/Coulomb 50/50, tol 1e-12/1e-14, "
                  "eps U[0.3,0.7], seeds 1000+j, 150 GB budget, FP32-12 bulk + anchored polish, omega 1.7 -> 1.1 "
                  "below theta 1e-2, Poisson arrivals at 80% of the capacity measured closed-loop (12 outstanding) "
                  "on the same list")


def run_serve(args):
    """The served stream of the full job list: capacity from the whole list in a
    closed loop, then the list again with Poisson arrivals at 80% of it."""
    from paper_1305_3440_gb300 import lgt
    specs, gaps = serve_specs(args.jobs)
    r = serve_stream(lgt, specs, gaps, cap_jobs=len(specs))
    print(json.dumps(dict({"workload": "serve", "metric": "p50/p99 job latency (s) at 80% of capacity",
                           "config": {"workload": f"{len(specs)} jobs, " + SERVE_WORKLOAD}}, **r)), flush=True)


def run_slab(args):
    """Temporal slab decomposition (Sec. 5).  One process: the 32^4 field cut into
    1, 2 and 4 slabs on this GPU (the boundary links move by device copies), FP32-12
    sweeps (omega 1.7, lean launch configuration 8, as the whole-lattice context
    forced to the same configuration), time per sweep against the whole lattice:
    the cost of the protocol's extra launches and copies.  Under torchrun (N GPUs):
    one slab of 32 slices per rank, a 32^3 x (32 N) lattice (weak scaling), the
    boundary links over NCCL; site updates per second over all ranks."""
    import torch
    from paper_1305_3440_gb300 import lgt, synth
    from paper_1305_3440_gb300.slab import DistRing, GpuSlab, LocalRing, SlabDriver
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    n_sweeps = 100
    L = 32
    dims = (L * world, 32, 32, 32)
    p = lgt.lgt_params_default(dims=dims, bulk=lgt.LGT_FP32_12, omega=1.7, launch_config=16)  # staged configuration 15
    out = {}

    def timed(fn):
        with torch.cuda.stream(stream):
            fn(3)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(n_sweeps)
            e1.record(stream)
            torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3

    if world == 1:
        U = synth.field(dims, 0.5, 2)
        ctx = lgt.lgt_create(p, U, stream=stream)
        t = timed(lambda n: lgt.lgt_sweep(ctx, n))
        lgt.lgt_destroy(ctx)
        out["whole"] = {"us_per_sweep": t / n_sweeps * 1e6}
        for n in (1, 2, 4):
            Ls = dims[0] // n
            eng = [GpuSlab(p, r * Ls, Ls, np.ascontiguousarray(U[r * Ls:(r + 1) * Ls]), stream) for r in range(n)]
            drv = SlabDriver(eng, LocalRing(n))
            ts = timed(drv.sweep)
            out[f"slabs_{n}"] = {"us_per_sweep": ts / n_sweeps * 1e6, "overhead": ts / t - 1.0,
                                 "boundary_bytes_per_transfer": eng[0].nbytes}
            for e in eng:
                e.close()
        value = n_sweeps * int(np.prod(dims)) / (out["slabs_4"]["us_per_sweep"] * n_sweeps / 1e6)
    else:
        U = synth.field((L,) + dims[1:], 0.5, 2 + rank)  # this rank's slab (weak scaling, synthetic)
        eng = GpuSlab(p, rank * L, L, U, stream)
        drv = SlabDriver([eng], DistRing())
        t = timed(drv.sweep)
        t_max, upd = aggregate_over_ranks(t, float(n_sweeps * int(np.prod(U.shape[:4]))), device=f"cuda:{local}")
        value = upd / t_max
        out[f"ranks_{world}"] = {"us_per_sweep": t_max / n_sweeps * 1e6, "boundary_bytes_per_transfer": eng.nbytes}
        eng.close()
    if rank == 0:
        print(json.dumps({"workload": "slab", "metric": "site updates/s (temporal slabs, FP32-12 sweeps)",
                          "value": value, "unit": "site updates/s", "n_gpus": world, "scaling": "weak",
                          "config": {"workload": f"SU(3) Landau {dims[1]}^3 x {dims[0]}, eps 0.5, {n_sweeps} sweeps, "
                                                 f"slabs of {dims[0] if world == 1 else L} slices"},
                          "runs": out}), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_profile(args):
    """A short, fixed run of the sweep kernels for profilers (ncu -k ... -c ...):
    one context on cuda:0, `--bulk-sweeps` sweeps in the bulk precision, promotion
    (G applied to the FP64 input, then the polish set-up), `--polish-sweeps` polish
    sweeps, one exact measurement.  Profilers serialise launches, which misleads
    the autotuner: pass `--launch-config` to profile the configuration a normal run
    picks.  At 32^4 the FP32 links (201 MB for 12 reals) are larger than the 129 MB
    L2 while the whole context stays under 2 GB of device memory (FP64: 3 GB)."""
    import torch
    from paper_1305_3440_gb300 import lgt, synth
    dims = tuple(args.dims)
    dev = torch.from_numpy(synth.field(dims, args.eps, args.seed)).cuda()
    bulk = {"fp32_12": lgt.LGT_FP32_12, "fp32_18": lgt.LGT_FP32_18, "fp64": lgt.LGT_FP64}[args.bulk]
    gauge = {"landau": lgt.LGT_LANDAU, "coulomb": lgt.LGT_COULOMB, "mag": lgt.LGT_MAG}[args.gauge]
    polish = {"anchor": lgt.LGT_POLISH_ANCHOR, "pair": lgt.LGT_POLISH_PAIR, "fp64": lgt.LGT_POLISH_FP64}[args.polish]
    p = lgt.lgt_params_default(dims=dims, gauge=gauge, omega=args.omega, bulk=bulk, polish=polish,
                               launch_config=args.launch_config + 1)
    ctx = lgt.lgt_create(p, dev)
    try:
        lgt.lgt_sweep(ctx, args.bulk_sweeps)
        lgt.lgt_promote(ctx)
        lgt.lgt_sweep(ctx, args.polish_sweeps)
        F, theta, plaq = lgt.lgt_measure(ctx)
        st = lgt.lgt_get_stats(ctx)
        print(json.dumps({"workload": "profile", "dims": list(dims), "gauge": args.gauge, "bulk": args.bulk,
                          "sweeps": [args.bulk_sweeps, args.polish_sweeps], "F": F, "theta": theta,
                          "plaquette": plaq, "launch_config": list(st.launch_config),
                          "sweep_ms": list(st.sweep_ms), "sweep_launches": list(st.sweep_launches)}), flush=True)
        if not np.isfinite(F):
            raise SystemExit("non-finite F")
    finally:
        lgt.lgt_destroy(ctx)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "coulomb":
        run_coulomb(args)
    elif args.workload == "landau64":
        run_landau64(args)
    elif args.workload == "serve":
        run_serve(args)
    elif args.workload == "mag":
        run_mag(args)
    elif args.workload == "profile":
        run_profile(args)
    elif args.workload == "slab":
        run_slab(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
