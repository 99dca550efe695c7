"""Benchmark of the leapfrog hot path (GLUPS, HBM roofline fraction).

One bench step = one pass of the whole forward hot path over the 8192^2 point-singularity
workload: mollified face depth (tsu_make_depth), Taylor start (tsu_init), 4999 leapfrog steps
with the discrete energy of every step fused in (tsu_step_n), and the final energy (tsu_observe):
5000 steps of (N-2)^2 interior lattice-point updates.  Inputs live in HBM before the timed
region; the four fields (4 x 256 MiB) exceed the 129 MB L2, so no flush is needed.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

N > 1 runs N independent replicas (one problem per rank, weak scaling; the path has no
exchange step).  ``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload instead.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-point updates/s (GLUPS) and HBM roofline %; adjoint/forward time ratio"
# DRAM bytes (read + write) per pass of the dominant kernel from ncu captures (profiles/),
# keyed by (kernel, form, n, steps per pass); only for kernels unchanged since the capture.
TRAFFIC = {
    # profiles/k_leapfrog_wtb_increment_8192.md: one launch of the timed configuration (8192^2,
    # 4 steps per pass, 117 rows per chunk, two rows per loop trip, outer strips first),
    # dram__bytes_read.sum + dram__bytes_write.sum
    ("k_leapfrog_wtb", "increment", 8192, 4): 1.665618e9,
    # profiles/k_leapfrog_wtb_flow_8192_2048.md: the persistent pass (sector-aligned reads, 96 rows
    # per tile) at the bench's launch shape, one launch of 10 passes (41 steps),
    # dram__bytes_read.sum + dram__bytes_write.sum / 10
    ("k_leapfrog_wtb_flow", "increment", 8192, 4): 1.7419624e9,
}
UNIT = "GLUPS"
ORACLE_SAMPLE_STEPS = 32  # leapfrog steps of each timed oracle sample (depth evaluation included once)
DEFAULT_KERNEL = 4  # warp-blocked pass, 4 steps per HBM pass, every pass of a call in one persistent launch


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tsu", choices=["tsu", "reference"])
    ap.add_argument("--n", type=int, default=8192, help="grid nodes per side (default: the 8192^2 workload)")
    ap.add_argument("--nsteps", type=int, default=5000, help="leapfrog steps per bench step")
    ap.add_argument("--form", default="increment", choices=["increment", "standard"])
    ap.add_argument("--rows", type=int, default=0)
    ap.add_argument("--kernel", type=int, default=0,
                    help="0 = 4; 1 one step per pass, 2 warp-blocked (tdepth 2/4), 3 CTA-blocked (tdepth 4/8), "
                         "4 warp-blocked passes in one persistent launch")
    ap.add_argument("--tdepth", type=int, default=0, help="steps per blocked pass (0: 4 for kernel 2, 8 for 3)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the adjoint, batched, 16384^2 and paper Case 1 measurements")
    ap.add_argument("--traffic", type=float, default=None, help="ncu dram bytes per launch (from profiles/)")
    ap.add_argument("--measure", choices=["adjoint", "batched", "large", "paper_case1", "implicit"], default=None,
                    help="run only this side measurement and print its result (a profiling aid)")
    ap.add_argument("--measure-n", type=int, default=0,
                    help="grid side of --measure adjoint (0: 2048) or implicit (0: every Table 1 size)")
    ap.add_argument("--measure-steps", type=int, default=4000, help="leapfrog steps of --measure adjoint/batched")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, device) -> float:
    """The slowest rank's figure (a MAX all-reduce); the value itself on one rank."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_glups(world: int, lups_per_rank: float, reps: int, ms: float) -> float:
    """Lattice updates of all ranks (each runs its own replica) over the slowest rank's time."""
    return world * lups_per_rank * reps / (ms / 1e3) / 1e9


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except Exception:
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                   "samples": len(sm)}
        os.unlink(self.path)
        return out


# -----------------------------------------------------------------------------------------------
# CPU oracle leg (the `--impl reference` arm and the cpu_baseline object)
# -----------------------------------------------------------------------------------------------
def oracle_sample(n: int, steps_sample: int, threads: int = 0, total_steps: int = 0):
    """Time the FP64 oracle, as it stands, on the workload's full grid (on every core of the
    process, or on `threads` threads): the depth evaluation once and `steps_sample` steps (start,
    leapfrog steps with the energy of every step), extrapolated to the whole workload's
    `total_steps` steps (default: the workload's 5000), so that the depth weighs what it weighs in
    the GPU bench step."""
    import oracle
    from paper_2005_11931_gb300 import inputs

    cores = len(os.sched_getaffinity(0))
    threads = oracle.set_threads(threads or cores)
    p = inputs.point_fp32(n)
    g = oracle.grid(n, n)
    u0 = p.initial()
    t0 = time.perf_counter()
    hx, hy, ext = oracle.make_depth(g, p.depth)
    t1 = time.perf_counter()
    tau = inputs.CFL * g.dx / max(ext[1], ext[3]) ** 0.5
    oracle.forward(g, tau, hx, hy, u0, None, steps_sample, want_energy=True)
    t2 = time.perf_counter()
    S = total_steps or p.steps
    est = (t1 - t0) + (t2 - t1) * S / steps_sample
    return dict(value=(n - 2) ** 2 * S / est / 1e9, unit=UNIT, cores=threads, kind="oracle",
                sample=f"FP64 oracle, {n}x{n} point workload: depth ({t1 - t0:.2f} s) + Taylor start + "
                       f"{steps_sample - 1} leapfrog steps with energy every step ({t2 - t1:.2f} s), "
                       f"extrapolated to the workload's {S} steps; {threads} OpenMP threads",
                seconds=t2 - t0)


def oracle_implicit_sample(sizes=(256, 512, 1024)):
    """The oracle's implicit comparator (FP64, Thomas elimination line by line) on the smaller
    Table 1 runs, whole (100 steps each): the CPU time beside the GPU's."""
    import oracle
    from paper_2005_11931_gb300 import inputs

    threads = oracle.set_threads(len(os.sched_getaffinity(0)))
    runs = []
    for n in sizes:
        p = inputs.paper_table1(n)
        g = oracle.grid(n, n)
        t0 = time.perf_counter()
        hx, hy, _ = oracle.make_depth(g, p.depth)
        oracle.implicit_forward(g, p.extra["tau"], 0.25, hx, hy, p.initial(), None, p.steps)
        dt = time.perf_counter() - t0
        runs.append({"n": n, "ms": dt * 1e3, "glups": (n - 2) ** 2 * p.steps / dt / 1e9})
    return {"kind": "oracle", "cores": threads, "unit": "ms for the 100-step run",
            "sample": "FP64 oracle implicit comparator, whole Table 1 runs, depth included", "runs": runs}


def workload_config(n: int, S: int, form: str, world: int) -> dict:
    """The config both arms report: the workload they measure (the reference arm times a bounded
    sample of it, described in its cpu_baseline)."""
    return {"workload": f"point_fp32_{n}: {n}x{n} grid, depth 0.5 + 0.01 phi_eps(|r-(0.5,0.5)|), eps = 4dx, "
                        f"Gaussian hump width 0.02 at (0.3,0.5), {S} steps, energy every step",
            "n": n, "leapfrog_steps": S, "form": form,
            "l2": (f"inputs larger than L2 (four {n * ((n + 31) // 32 * 32) * 4 / 2**20:.0f} MiB fields), no flush"
                   if 4 * n * n * 4 > 129e6 else "inputs smaller than L2 (129 MB)"),
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    # bounded sample: a few steps of the full grid per bench step (the same sample as the GPU
    # line's cpu_baseline)
    steps_sample = ORACLE_SAMPLE_STEPS
    for _ in range(args.warmup):
        oracle_sample(args.n, 2, total_steps=args.nsteps)
    vals, secs = [], 0.0
    for _ in range(args.steps):
        r = oracle_sample(args.n, steps_sample, total_steps=args.nsteps)
        vals.append(r["value"])
        secs += r["seconds"]
    v = statistics.mean(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.n, args.nsteps, args.form, world),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": r["cores"], "kind": "oracle", "sample": r["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# -----------------------------------------------------------------------------------------------
# GPU leg
# -----------------------------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2005_11931_gb300 import inputs, tsu

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    form = tsu.TSU_FORM_INCREMENT if args.form == "increment" else tsu.TSU_FORM_STANDARD
    p = inputs.point_fp32(args.n, args.nsteps)
    S = p.steps
    g = tsu.grid(p.n)
    code = tsu.TSU_F32

    # device-resident inputs and buffers
    hx = tsu.empty_field(g, code, dev)
    hy = tsu.empty_field(g, code, dev)
    ext_dev = torch.zeros(4, dtype=torch.float64, device=dev)
    u0 = torch.from_numpy(p.initial(g.ld, np.float32)).to(dev)
    nb = 4
    bufs = [tsu.empty_field(g, code, dev) for _ in range(nb)]
    st = tsu.State()
    ws_bytes = tsu.tsu_step_workspace(g, code)
    ws = torch.zeros(ws_bytes, dtype=torch.uint8, device=dev)
    energy = torch.zeros(S, dtype=torch.float64, device=dev)
    ext = tsu.tsu_make_depth(g, p.depth, code, hx, hy, ext_dev, sync=True)
    med = tsu.medium(hx, hy, ext)
    tau = tsu.tsu_tau_courant(g, med, inputs.CFL)
    # kernel: --kernel, else the default below; the blocked kernels' steps and the leftover single
    # steps are separate calls so that each is timed on its own
    kernel = args.kernel or DEFAULT_KERNEL
    blocked = kernel in (2, 3, 4)
    K = (args.tdepth or (8 if kernel == 3 else 4)) if blocked else 1
    n_main = ((S - 1) // K) * K if blocked else S - 1
    n_left = (S - 1) - n_main
    opts = tsu.StepOpts()
    opts.energy = energy.data_ptr()
    opts.kernel, opts.rows, opts.tdepth = kernel, args.rows, (K if blocked else 0)
    opts_left = tsu.StepOpts()
    opts_left.energy = energy.data_ptr() + 8 * n_main
    opts_left.kernel = 1
    ev_k0 = torch.cuda.Event(enable_timing=True)
    ev_k1 = torch.cuda.Event(enable_timing=True)
    kernel_ms = []

    def one_step(u0_dev, timed_kernel=False):
        for k, b in enumerate(bufs):
            st.buf[k] = b.data_ptr()
        st.nbuf = nb
        st.form = form
        tsu.tsu_make_depth(g, p.depth, code, hx, hy, ext_dev, sync=False, stream=stream)
        tsu.tsu_init(g, code, tau, med, u0_dev, None, st, stream)
        if timed_kernel:
            ev_k0.record(stream)
        tsu.tsu_step_n(g, code, tau, med, st, n_main, opts, ws, ws_bytes, stream)
        if timed_kernel:
            ev_k1.record(stream)
        if n_left:
            tsu.tsu_step_n(g, code, tau, med, st, n_left, opts_left, ws, ws_bytes, stream)
        o_e = energy[S - 1:]
        tsu.tsu_observe(g, code, tau, med, st, o_e, None, None, ws, ws_bytes, stream)

    main_launches = n_main // K if blocked else n_main  # passes (kernel 4: all in one launch)
    # depth (reset, eval, decode), init, main passes (kernel 4: its counters' reset and one
    # launch), leftover passes, observe
    launches_per_step = 3 + 1 + (2 if kernel == 4 else main_launches) + n_left + 1

    for _ in range(args.warmup):
        one_step(u0)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            one_step(u0, timed_kernel=True)
            ev_k1.synchronize()
            kernel_ms.append(ev_k0.elapsed_time(ev_k1))
        t1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(t0.elapsed_time(t1), dev)
    lups_step = (p.n - 2) ** 2 * S
    value = whole_job_glups(world, lups_step, args.steps, ms)
    tsu.tsu_sync_status(ws, ws_bytes, stream)  # raises if a bounded device wait expired
    # roofline of the dominant kernel.  Algorithmic bytes per launch: one read of the state and
    # the faces and one write of the state: 24 B per node (increment form) / 20 B (standard,
    # one step per pass); the blocked pass reads and writes two state fields: 24 B per node for
    # K steps.
    if blocked:
        bpn = 24
        kname = {2: "k_leapfrog_wtb", 3: "k_leapfrog_tb", 4: "k_leapfrog_wtb_flow"}[kernel]
    else:
        bpn = 24 if form == tsu.TSU_FORM_INCREMENT else 20
        kname = "k_leapfrog"
    # per pass (K steps); kernel 4 runs every pass of the call in one launch (its counters' reset,
    # a few microseconds, included)
    pass_ms = sum(kernel_ms) / (len(kernel_ms) * main_launches)
    passes_per_launch = main_launches if kernel == 4 else 1
    achieved = bpn * (p.n - 2) ** 2 / (pass_ms / 1e3) / 1e9
    traffic = args.traffic
    if traffic is None and args.rows == 0:  # the captured launches used the automatic rows per chunk
        traffic = TRAFFIC.get((kname, args.form, p.n, K if blocked else 1))
    peak, peak_kind = load_peaks()
    e_final = energy.cpu().numpy()
    drift = float(np.max(np.abs(e_final - e_final[0])) / e_final[0])

    # end to end through the C ABI with host buffers: H2D of u0, full run, D2H of u^S and energy
    e2e = None
    if not args.no_e2e:
        u0_host = torch.from_numpy(p.initial(g.ld, np.float32)).pin_memory()
        u_host = torch.empty_like(u0_host).pin_memory()
        e_host = torch.empty(S, dtype=torch.float64).pin_memory()
        u0_stage = torch.empty_like(u0)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        reps = max(1, min(args.steps, 3))
        a0.record(stream)
        for _ in range(reps):
            u0_stage.copy_(u0_host, non_blocking=True)
            one_step(u0_stage)
            u_host.copy_(bufs[st.cur], non_blocking=True)
            e_host.copy_(energy, non_blocking=True)
        a1.record(stream)
        torch.cuda.synchronize()
        ems = max_over_ranks(a0.elapsed_time(a1), dev)
        e2e = {"value": whole_job_glups(world, lups_step, reps, ems), "unit": UNIT,
               "h2d_bytes_per_step": int(u0_host.numel() * 4),
               "d2h_bytes_per_step": int(u_host.numel() * 4 + e_host.numel() * 8)}

    if world > 1:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return 0
    extras = {}
    if not args.no_extras and world == 1:
        extras["implicit_table1"] = compact_implicit(measure_implicit())
        extras["paper_case1"] = measure_paper_case1()
        extras["large"] = measure_large()
        extras["single_sizes"] = [measure_single(n) for n in (2048, 4096)]
        extras["batched"] = measure_batched()
        extras["adjoint"] = measure_adjoint()
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        r = oracle_sample(p.n, ORACLE_SAMPLE_STEPS, total_steps=args.nsteps)
        cpu = {k: r[k] for k in ("value", "unit", "cores", "kind", "sample")}
        r1 = oracle_sample(p.n, 8, threads=1, total_steps=args.nsteps)
        cpu["single_thread"] = {k: r1[k] for k in ("value", "unit", "cores", "sample")}
        if "implicit_table1" in extras:
            cpu["implicit_table1"] = oracle_implicit_sample()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": workload_config(p.n, S, args.form, world),
        "kernel": f"{'%d steps per blocked pass' % K if blocked else 'one step per pass'}, tau = {tau:.6g}",
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "peak_kind": peak_kind, "bytes_per_pass_per_node": bpn,
                     "steps_per_pass": K if blocked else 1, "kernel": kname, "pass_ms": pass_ms,
                     "passes_per_launch": passes_per_launch, "launch_ms": pass_ms * passes_per_launch,
                     "launches_per_step": main_launches // passes_per_launch,
                     # DRAM bytes the ncu capture counted per pass over the live pass time, and the
                     # algorithmic rate against the 8 TB/s nominal figure (context)
                     "dram_frac": (traffic / (pass_ms / 1e3) / 1e9 / peak) if traffic else None,
                     "frac_of_nominal_8tbs": achieved / 8000.0},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk.summary(),
        "gpu_launches": launches_per_step * args.steps,
        "energy_drift": drift,
        **extras,
    }
    if extras:
        # the other parts of the metric in a few numbers, last in the line
        a, b = extras["adjoint"], extras["batched"]
        line["summary"] = {
            "glups_8192_point": value, "roofline_frac": achieved / peak,
            **{f"glups_{r['n']}_point": r["glups"] for r in extras["single_sizes"]},
            "glups_16384_lines": extras["large"]["glups"], "glups_paper_case1_4097": extras["paper_case1"]["glups"],
            "batched_glups": b["batched_glups"], "batched_tuned_glups": b.get("batched_tuned_glups"),
            "batched_speedup_vs_sequential_auto": b["speedup_vs_sequential_auto"],
            "batched_speedup_vs_sequential_one_step": b["speedup_vs_sequential_one_step"],
            "adjoint_forward_ms": a["forward_ms"], "adjoint_ms": a["adjoint_ms"], "adjoint_ratio": a["ratio"]}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# -----------------------------------------------------------------------------------------------
# The other workloads of the metric, measured in the same run (device-resident inputs, CUDA events)
# -----------------------------------------------------------------------------------------------
def _events_ms(fn, reps=1):
    import torch
    s = torch.cuda.current_stream()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(s)
    for _ in range(reps):
        fn()
    b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def measure_single(n, steps=2000, warm=2):
    """The point workload's problem on an n x n grid (one wave of tiles or less at 2048^2 and
    4096^2): the bench step's calls (depth, start, steps with the energy of every step), timed
    whole."""
    import numpy as np
    import torch

    from paper_2005_11931_gb300 import inputs, tsu

    p = inputs.point_fp32(n, steps)
    sim = tsu.Simulation.create(n, p.depth, dtype="f32", form=tsu.TSU_FORM_INCREMENT)
    u0 = torch.from_numpy(p.initial(sim.g.ld, np.float32)).cuda()
    e = torch.zeros(steps, dtype=torch.float64, device="cuda")

    def run():
        sim.init(u0)
        sim.step(steps - 1, energy=e[: steps - 1])
        sim.observe(energy=e[steps - 1:])

    for _ in range(warm):
        run()
    t = _events_ms(run, 3)
    tsu.tsu_sync_status(sim.ws, sim.ws.numel())
    return {"n": n, "steps": steps, "ms": t, "glups": (n - 2) ** 2 * steps / t / 1e6}


def compact_implicit(r):
    """Table 1 runs as {dtype: {n: ms}} plus the largest run's bandwidth fraction."""
    out = {"workload": r["workload"], "ms": {}}
    for x in r["runs"]:
        out["ms"].setdefault(x["dtype"], {})[x["n"]] = round(x["ms"], 3)
    big = [x for x in r["runs"] if x["dtype"] == "f32"][-1]
    out["f32_largest_frac_of_measured_peak"] = big["frac_of_measured_peak"]
    return out


def measure_adjoint(n=2048, steps=4000, warm=1, reps=2):
    """Adjoint/forward time ratio on the receiver-misfit workload: forward with traces and
    checkpoints every 64 steps vs tsu_adjoint (segment recompute + reverse sweep)."""
    import numpy as np
    import torch

    from paper_2005_11931_gb300 import inputs, tsu

    case = inputs.adjoint_case(n, steps)
    p, every = case["problem"], case["ckpt_every"]
    S = p.steps
    sim = tsu.Simulation.create(p.n, p.depth, dtype="f32", form=tsu.TSU_FORM_INCREMENT)
    g = sim.g
    u0 = torch.from_numpy(p.initial(g.ld, np.float32)).cuda()
    rec = torch.from_numpy(inputs.flat_index(case["receivers"], g.ld)).cuda()
    nrec = rec.numel()
    traces = torch.zeros((S, nrec), dtype=torch.float32, device="cuda")
    slots = tsu.tsu_ckpt_slots(S, every)
    ck = torch.empty((slots, 2, g.ny, g.ld), dtype=torch.float32, device="cuda")
    obs = torch.zeros_like(traces)

    def forward(tr):
        sim.init(u0)
        sim.step(S - 1, rec_idx=rec, traces=tr[: S - 1], ckpt=ck, ckpt_every=every)
        sim.observe(rec_idx=rec, trace=tr[S - 1])

    # observations: the same run with eps = 0.012 (a different medium)
    osim = tsu.Simulation.create(p.n, case["depth_obs"], dtype="f32", form=tsu.TSU_FORM_INCREMENT,
                                 tau=sim.tau)
    osim.init(u0)
    osim.step(S - 1, rec_idx=rec, traces=obs[: S - 1])
    osim.observe(rec_idx=rec, trace=obs[S - 1])
    gx = torch.zeros((g.ny, g.ld), dtype=torch.float64, device="cuda")
    gy = torch.zeros_like(gx)
    gu0 = torch.zeros_like(u0)
    gu1 = torch.zeros_like(u0)
    wsb = tsu.tsu_adjoint_workspace(g, tsu.TSU_F32, tsu.TSU_FORM_INCREMENT, S, every, nrec)
    ws = torch.empty(wsb, dtype=torch.uint8, device="cuda")

    def adjoint():
        tsu.tsu_adjoint(g, tsu.TSU_F32, tsu.TSU_FORM_INCREMENT, sim.tau, sim.medium, S, every, ck, u0, rec,
                        traces - obs, gx, gy, gu0, gu1, ws, wsb)

    for _ in range(warm):
        forward(traces)
        adjoint()
    t_f = _events_ms(lambda: forward(traces), reps)
    t_a = _events_ms(adjoint, reps)
    lups = (n - 2) ** 2 * S
    J = 0.5 * float(((traces - obs).double() ** 2).sum())
    # algorithmic bytes: the forward (warp-blocked, receivers and checkpoints recorded in it) reads
    # u, v, hx, hy and writes u, v once per 4 steps (1.5 fields per step); the adjoint moves 23
    # fields per 4 reverse steps (the 4-step sweep 14: lam^{n+1}, lam^{n+2},
    # u^n..u^{n-3}, hx, hy and the two accumulators read, two multipliers and the accumulators
    # written; the 4-step recompute 9: u, v, hx, hy read, 4 states and v written)
    fb = g.ny * g.ld * 4
    peak, _ = load_peaks()
    return {"workload": f"adjoint_{n}: {n}^2 FP32 (increment form), depth 1 + 0.5 phi_eps(x-0.5), eps 0.01, "
                        f"{S} steps, {nrec} receivers on y = 0.8, checkpoints every {every}",
            "forward_ms": t_f, "adjoint_ms": t_a, "ratio": t_a / t_f, "forward_glups": lups / t_f / 1e6,
            "adjoint_glups": lups / t_a / 1e6, "J": J, "grad_norm_hx": float(gx.norm()),
            "forward_gbs_algorithmic": 1.5 * fb * S / (t_f / 1e3) / 1e9,
            "adjoint_gbs_algorithmic": 23 / 4 * fb * S / (t_a / 1e3) / 1e9,
            "adjoint_frac_of_measured_peak": 23 / 4 * fb * S / (t_a / 1e3) / 1e9 / peak}


def measure_batched(steps=2000, warm=1, rows=0):
    """The 64-problem eps-family: one batched launch per K steps vs the same problems run one
    after the other (one step per pass, and the automatic kernel choice)."""
    import numpy as np
    import torch

    from paper_2005_11931_gb300 import inputs, tsu

    probs = inputs.batched_family(steps=steps)
    sims = []
    for pr in probs:
        sim = tsu.Simulation.create(pr.n, pr.depth, dtype="f32", form=tsu.TSU_FORM_INCREMENT)
        sims.append((pr, sim, torch.from_numpy(pr.initial(sim.g.ld, np.float32)).cuda()))
    nsteps = [pr.steps - 1 for pr in probs]
    wsb = tsu.tsu_batch_workspace([s for _, s, _ in sims], nsteps, rows=rows)
    ws = torch.zeros(wsb, dtype=torch.uint8, device="cuda")

    def init_all():
        for _, sim, u0 in sims:
            sim.init(u0)

    def batched():
        init_all()
        tsu.tsu_batch_run([s for _, s, _ in sims], nsteps, ws, wsb, rows=rows)

    def sequential(kernel):
        init_all()
        for (pr, sim, _), n in zip(sims, nsteps):
            sim.step(n, kernel=kernel)

    for _ in range(warm):
        batched()
        sequential(1)
    t_init = _events_ms(init_all)
    t_b = _events_ms(batched)
    snap = [sim.u.clone() for _, sim, _ in sims]
    t_s1 = _events_ms(lambda: sequential(1))
    diff = max(float((sim.u - a).abs().max() / a.abs().max().clamp_min(1e-30)) for (_, sim, _), a in zip(sims, snap))
    t_s0 = _events_ms(lambda: sequential(0))
    tsu.tsu_sync_status(ws, wsb)
    # the autotuner's packing of the same family (tuned here, with a cache of this run only), timed
    # the same way on a side stream (a graph launch needs one)
    import tempfile

    from paper_2005_11931_gb300 import autotune

    with tempfile.TemporaryDirectory() as td:
        choice = autotune.tune_batch([s for _, s, _ in sims], cache=autotune.Cache(os.path.join(td, "tune.json")))
    topts = choice.batch_opts([s for _, s, _ in sims])
    twsb = tsu.tsu_batch_workspace([s for _, s, _ in sims], nsteps,
                                   **{k: v for k, v in topts.items() if k != "graph"})
    tws = torch.zeros(twsb, dtype=torch.uint8, device="cuda")
    side = torch.cuda.Stream()

    def tuned():
        init_all()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            tsu.tsu_batch_run([s for _, s, _ in sims], nsteps, tws, twsb, stream=side, **topts)
        torch.cuda.current_stream().wait_stream(side)

    tuned()
    t_t = _events_ms(tuned)
    lups = sum((pr.n - 2) ** 2 * pr.steps for pr in probs)
    # algorithmic bytes of the 4-step batched pass: u, v, hx, hy read and u, v written once per
    # 4 steps (1.5 fields per step) for every problem
    peak, _ = load_peaks()
    gbs = sum(1.5 * s.g.ny * s.g.ld * 4 * (pr.steps - 1) for (pr, s, _) in sims) / (t_b / 1e3) / 1e9
    return {"workload": f"eps-family: {len(probs)} problems (16 eps x line-x, line-y, point, line+point), "
                        f"N in {{512..2048}}, {steps} steps each, FP32 increment form",
            "lups": lups, "batched_ms": t_b, "sequential_one_step_ms": t_s1, "sequential_auto_ms": t_s0,
            "init_ms": t_init, "batched_glups": lups / t_b / 1e6, "batched_gbs_algorithmic": gbs,
            "batched_tuned_ms": t_t, "batched_tuned_glups": lups / t_t / 1e6,
            "tuned_choice": {k: v for k, v in topts.items() if k != "rows_per_problem"} | {
                "size_rows": choice.size_rows},
            "batched_frac_of_measured_peak": gbs / peak, "speedup_vs_sequential_one_step": t_s1 / t_b,
            "speedup_vs_sequential_auto": t_s0 / t_b, "max_rel_diff_batched_vs_sequential": diff}


def measure_large(n=16384, steps=20000, warm_steps=400):
    """16384^2 crossing lines, FP32: the whole 20000-step run timed (about 5 s on one GB300), after
    a short warm-up run of the same problem."""
    import numpy as np
    import torch

    from paper_2005_11931_gb300 import inputs, tsu

    p = inputs.crossing_lines_fp32(n, steps)
    sim = tsu.Simulation.create(n, p.depth, dtype="f32", form=tsu.TSU_FORM_INCREMENT)
    u0 = torch.from_numpy(p.initial(sim.g.ld, np.float32)).cuda()
    e = torch.zeros(steps, dtype=torch.float64, device="cuda")

    def run(k):
        sim.init(u0)
        sim.step(k - 1, energy=e[: k - 1])

    run(min(warm_steps, steps))
    t = _events_ms(lambda: run(steps))
    tsu.tsu_sync_status(sim.ws, sim.ws.numel())
    en = e[: steps - 1].cpu().numpy()
    return {"workload": f"crossing_lines_fp32_{n}: {n}^2, 1 + phi(x-0.5) + phi(y-0.5), eps 8dx, {steps} steps "
                        f"timed, energy every step", "ms": t, "glups": (n - 2) ** 2 * steps / t / 1e6,
            "energy_drift": float(np.max(np.abs(en - en[0])) / en[0])}


def measure_paper_case1(n=4097, steps=2000, warm=1):
    """The paper's own 2D workload (Sec. 3.3, rescaled to the unit box): Friedrichs-mollified
    depth step 100 -> 10 at x = 0.75, eps = 0.8/100, hump 50 exp(-r^2/8) at (0.40, 0.50); FP32,
    energy every step."""
    import numpy as np
    import torch

    from paper_2005_11931_gb300 import inputs, tsu

    p = inputs.paper_case1_2d(n=n, steps=steps)["problem"]
    sim = tsu.Simulation.create(n, p.depth, dtype="f32", form=tsu.TSU_FORM_INCREMENT)
    u0 = torch.from_numpy(p.initial(sim.g.ld, np.float32)).cuda()
    e = torch.zeros(steps, dtype=torch.float64, device="cuda")

    def run():
        sim.init(u0)
        sim.step(steps - 1, energy=e[: steps - 1])

    for _ in range(warm):
        run()
    t = _events_ms(run)
    tsu.tsu_sync_status(sim.ws, sim.ws.numel())
    en = e[: steps - 1].cpu().numpy()
    return {"workload": f"paper_case1_{n}: {n}^2, depth step 100 -> 10 at x = 0.75 (Friedrichs, eps 0.008), "
                        f"hump 50 exp(-r^2/8) at (0.40, 0.50) in paper units, {steps} steps, energy every step",
            "ms": t, "glups": (n - 2) ** 2 * steps / t / 1e6,
            "energy_drift": float(np.max(np.abs(en - en[0])) / en[0])}


# Sec. 4, Table 1: GPU time in seconds of the paper's implicit solver (cyclic reduction, Case 1, dt
# = 0.05, T = 5, 100 steps) on an RTX 2080 Ti, per grid side.  Context only: other hardware.
PAPER_TABLE1_GPU_S = {256: 0.88, 512: 2.07, 1024: 7.16, 2048: 20.30, 4096: 62.76}


def measure_implicit(sizes=(256, 512, 1024, 2048, 4096)):
    """The implicit comparator on the paper's Table 1 runs: the 2D Case 1 problem on n x n nodes,
    dt = 0.05 in paper units (Courant number 1.3 .. 20), 100 steps, sigma = 1/4, FP64 and FP32.
    Algorithmic bytes per node and step: the x pass reads u, hx, hy and the pivots and writes
    the transposed result; the y pass reads it with the y pivots and coefficients, and reads and
    writes v and u: 12 fields, 48 B in FP32, 96 B in FP64."""
    import torch

    from paper_2005_11931_gb300 import inputs, tsu

    peak, _ = load_peaks()
    out = {"workload": "paper Table 1 runs: Case 1 depth (step 100 -> 10, Friedrichs, eps 0.8), n x n nodes, "
                       "dt = 0.05 (paper units), 100 steps, factorized implicit scheme, sigma = 1/4; on a side "
                       "stream (the step call then runs as one CUDA graph)",
           "bytes_per_node_step": {"f32": 48, "f64": 96}, "runs": []}
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        _implicit_runs(out, sizes, peak)
    torch.cuda.current_stream().wait_stream(side)
    return out


def _implicit_runs(out, sizes, peak):
    import torch

    from paper_2005_11931_gb300 import inputs, tsu

    for dtype in ("f32", "f64"):
        for n in sizes:
            p = inputs.paper_table1(n)
            sim = tsu.ImplicitSimulation.create(n, p.depth, dtype=dtype, tau=p.extra["tau"])
            u0 = torch.from_numpy(p.initial(sim.g.ld)).to(tsu.DTYPES[sim.dtype]).cuda()

            def run():
                sim.init(u0)
                sim.step(p.steps - 1)

            run()
            ms = _events_ms(run)
            nodes = (n - 2) ** 2
            gbs = nodes * p.steps * (48 if dtype == "f32" else 96) / (ms / 1e3) / 1e9
            out["runs"].append({"dtype": dtype, "n": n, "ms": ms, "glups": nodes * p.steps / ms / 1e6,
                                "gbs_algorithmic": gbs, "frac_of_measured_peak": gbs / peak,
                                "paper_table1_gpu_s": PAPER_TABLE1_GPU_S.get(n)})
            del sim


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.measure:
        fn = {"adjoint": lambda: measure_adjoint(args.measure_n or 2048, args.measure_steps),
              "batched": lambda: measure_batched(args.measure_steps, rows=args.rows),
              "large": measure_large, "paper_case1": measure_paper_case1,
              "implicit": lambda: measure_implicit((args.measure_n,) if args.measure_n else (256, 512, 1024, 2048, 4096))
              }[args.measure]
        print(json.dumps(fn()))
        return 0
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
