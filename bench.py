#!/usr/bin/env python3
"""Benchmark: ridge solves/s of M-IHS (Algorithm 1) on one GB300 per rank.

Workload (the bandwidth-scale plain-FP32 problem): A = G·diag(σ)·Vᵀ/√n with
n = 262144, d = 1024, σ_i = 1/i, λ = 1e-4, b = A x0 + ω at 40 dB SNR, sketch
size m = 4·sd = 588 (sd = 146.85).  One step = one full solve (sketch + outer
iterations until ‖g‖ ≤ tol·‖Aᵀb‖) with each of the three sketch families
(Gaussian, CountSketch, SRHT).  A is 1.07 GB (> L2), so every pass streams
from HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl mihs|reference]

Prints one JSON line (rank 0).  `value` is device time with A and b resident;
`e2e` takes every step's A and b from pinned host memory and returns each x
to the host, copies inside the timed region (by default double-buffered:
problem k+1 is copied in by a copy engine while problem k solves;
`--e2e-mode serial` copies, then solves); `roofline` is the gradient A-pass kernel, timed with CUDA events on
its stream; `cpu_baseline` is the oracle on the host cores (bounded sample).
Under torchrun (N > 1) every rank solves its own replica (weak scaling; the
method needs no collective on one problem per GPU).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FAMILIES = ["gaussian", "countsketch", "srht"]

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one A-pass
# launch, taken by ncu on the 65536×1024 case of this kernel.  Traffic is one
# read of A plus O(d) vectors, so it scales with the rows processed.
APASS_NCU = {"n": 65536, "d": 1024, "bytes": 268737536 + 3024896}
METRIC = "ridge solves/s at stated rel. error"
# The oracle's sample, identical in the cpu_baseline leg and the reference
# arm: rows of each dense SA timed (scaled to m) and M-IHS iterations per
# solve (the steps at the rate √(sd/m) = 1/2 from residual 1 to 2e-8).
ORACLE_ROWS = 2
ORACLE_ITERS = 25


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["mihs", "reference"], default="mihs")
    ap.add_argument("--families", default=",".join(FAMILIES))
    ap.add_argument("--tol", type=float, default=2e-8)
    ap.add_argument("--max-outer", type=int, default=200)
    ap.add_argument("--n", "--rows", dest="n", type=int, default=262144)
    ap.add_argument("--d", "--cols", dest="d", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-mode", choices=["pipelined", "serial"], default="pipelined",
                    help="pipelined: problem k+1's inputs are copied in (two device buffers) while problem k "
                         "solves; serial: copy, then solve, one problem at a time")
    ap.add_argument("--e2e-copy", choices=["auto", "sm", "dma"], default="auto",
                    help="host-to-device copy of the e2e leg: the SMs (mihs_copy_to_device) or a copy engine "
                         "(mihs_copy_to_device_dma); auto: dma when pipelined, sm when serial")
    ap.add_argument("--h2d-blocks", type=int, default=0,
                    help="SMs the SM copy may use in the e2e leg (MIHS_H2D_BLOCKS; 0: all)")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-refined", action="store_true", help="skip the compensated-refinement leg")
    ap.add_argument("--refined-tol", type=float, default=1e-10)
    ap.add_argument("--no-backward", action="store_true", help="skip the differentiable-solve leg")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched λ-path leg")
    ap.add_argument("--no-small", action="store_true", help="skip the 4096 x 256 leg")
    ap.add_argument("--oracle-sample", default="", help=argparse.SUPPRESS)
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision leg (2^21 x 2048)")
    ap.add_argument("--no-dual", action="store_true", help="skip the Dual M-IHS leg (2048 x 2^18)")
    ap.add_argument("--mixed-tol", type=float, default=3e-14,
                    help="relative residual the mixed-precision solves refine to")
    ap.add_argument("--mixed-sample-rows", type=int, default=1 << 17,
                    help="rows of the same-conditioning sample whose error is checked against the oracle (0: off)")
    ap.add_argument("--mixed-oracle", action="store_true",
                    help="also solve the mixed-precision workload with the fp64 oracle on the host (slow)")
    ap.add_argument("--sequential", action="store_true",
                    help="run the per-family solves of a step one after another on one stream")
    ap.add_argument("--aab", default="",
                    help="form of AAb_Solver in the step's solves: auto, cluster, grid or grid:<blocks> "
                         "(default: grid:24 when the solves share the GPU on concurrent streams, else auto)")
    ap.add_argument("--aab-refined", default="auto",
                    help="form of AAb_Solver in the refined leg's solves (same values as --aab)")
    ap.add_argument("--profile-op", choices=["apass", "apass-dd", "backward", "path", "aab", "aab-late", "aab-wide",
                                            "aab-wide-bf16", "dual-grad",
                                            "gaussian", "gaussian-bf16", "gaussian-fp8", "countsketch", "srht"],
                    help="time one kernel family alone on the workload (for ncu captures)")
    return ap.parse_args()


# --------------------------------------------------------------- plumbing
def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if torch.cuda.is_available():
        torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, ws: int) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_id}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power) if power else None}


def gpu_uuid():
    import torch
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(torch.cuda.current_device())


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ------------------------------------------------------------ CPU oracle
class OracleTimer:
    """The oracle (numpy fp64, as it stands) timed on the host cores in
    pieces: the sketch of each family (a few rows of SA, scaled to m; the
    CountSketch SA in full) and one fp64 M-IHS iteration on the full problem
    (with the CountSketch SA), combined into solves/s for the iteration
    counts given.  `measure` re-times one piece, so that a caller can spread
    the pieces over steps and keep each step short."""

    def __init__(self, A_host, b_host, p, families, rows):
        from oracle import mihs_oracle as o
        self.o, self.p, self.families, self.rows = o, p, list(families), rows
        self.A, self.b = A_host.numpy(), b_host.numpy()
        self.fam_id = {"gaussian": o.GAUSSIAN, "countsketch": o.COUNTSKETCH, "srht": o.SRHT}
        self.parts = [("sketch", f) for f in self.families] + [("iter", None)]
        self.t = {}
        self.SA = None

    def measure(self, part):
        import numpy as np
        o, p = self.o, self.p
        kind, f = part
        if kind == "iter" and self.SA is None:
            self.SA = o.sketch_apply(o.COUNTSKETCH, self.A, p.m, 7)
        t0 = time.perf_counter()
        if kind == "iter":
            o.mihs(self.A, self.b, p.lam, self.SA, p.sd, 1, eps_sub=0.1)
            self.t[part] = time.perf_counter() - t0
        elif f == "countsketch":
            self.SA = o.sketch_apply(o.COUNTSKETCH, self.A, p.m, 7)
            self.t[part] = time.perf_counter() - t0
        else:
            o.sketch_rows(self.fam_id[f], np.arange(self.rows), self.A, p.m, 7)
            self.t[part] = (time.perf_counter() - t0) * p.m / self.rows

    def measure_all(self):
        for part in self.parts:
            self.measure(part)

    def value(self, iters=None):
        iters = ORACLE_ITERS if iters is None else iters
        t_it = self.t[("iter", None)]
        total = sum(self.t[("sketch", f)] + (iters + 1) * t_it for f in self.families)
        return len(self.families) / total

    def sample(self, iters=None):
        iters = ORACLE_ITERS if iters is None else iters
        return (f"oracle (numpy fp64) on the full {self.p.n}x{self.p.d} problem: {self.rows} rows of SA per "
                f"dense family scaled to m={self.p.m}, the full CountSketch SA, one M-IHS iteration "
                f"scaled to {iters} iterations + 1 gradient per family")

    def detail(self):
        return {"sketch_s": {f: round(self.t[("sketch", f)], 3) for f in self.families},
                "iter_s": round(self.t[("iter", None)], 4)}


def oracle_one_core(A_host, b_host, families):
    """The same oracle sample in a fresh interpreter whose BLAS and OpenMP
    pools have one thread, pinned to one core; A and b reach it through a
    temporary .npy file."""
    import tempfile

    import numpy as np
    tmpdir = "/dev/shm" if os.path.isdir("/dev/shm") else None
    with tempfile.TemporaryDirectory(dir=tmpdir) as td:
        np.save(os.path.join(td, "A.npy"), A_host.numpy())
        np.save(os.path.join(td, "b.npy"), b_host.numpy())
        env = dict(os.environ)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
            env[k] = "1"
        env.pop("RANK", None)
        cmd = [sys.executable, os.path.abspath(__file__), "--oracle-sample", td, "--families", ",".join(families)]
        try:
            r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=300)
            line = [ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1]
            return json.loads(line)
        except Exception as e:  # reported, not fatal: the all-core number stands
            return {"error": f"{type(e).__name__}: {str(e)[:200]}"}


def run_oracle_sample(args):
    """Child of oracle_one_core: the oracle sample on one core."""
    import numpy as np
    import torch

    from paper_1912_03514_gb300 import workloads as W
    try:
        os.sched_setaffinity(0, {sorted(os.sched_getaffinity(0))[0]})
    except (AttributeError, OSError):
        pass
    A = torch.from_numpy(np.load(os.path.join(args.oracle_sample, "A.npy")))
    b = torch.from_numpy(np.load(os.path.join(args.oracle_sample, "b.npy")))
    n, d = A.shape
    sigma = W.profile_polynomial(d, 1.0)
    lam = 1e-4
    sd = W.nominal_sd(sigma, lam)
    p = W.RidgeProblem(name=f"ridge-{n}x{d}", A=A, b=b, lam=lam, sd=sd, m=min(n, W.round_up(4 * sd, 4)),
                       x0=None, sigma=sigma, meta={})
    families = [f for f in args.families.split(",") if f]
    ot = OracleTimer(A, b, p, families, rows=ORACLE_ROWS)
    ot.measure_all()
    print(json.dumps({"value": round(ot.value(), 5), "unit": "solves/s", "cores": 1, "kind": "oracle",
                      "sample": "the same sample on one core", "detail": ot.detail()}), flush=True)


# ------------------------------------------------------------------ main
def main():
    args = parse()
    import torch
    ws, rank, local = dist_setup()
    families = [f for f in args.families.split(",") if f]

    from paper_1912_03514_gb300 import workloads as W

    if args.oracle_sample:
        return run_oracle_sample(args)
    if args.impl == "reference":
        return run_reference(args, ws, rank, families)
    if args.profile_op:
        return run_profile_op(args, local)

    from paper_1912_03514_gb300 import mihs

    dev = torch.device("cuda", local)
    p = W.problem_bandwidth(device=str(dev), seed=1001 + rank, n=args.n, d=args.d)
    A, b = p.A, p.b
    n, d, m = p.n, p.d, p.m
    seed = 0x5EED0000 + rank
    sketches = {f: mihs.Sketch(A, f, m, seed) for f in families}
    # Concurrent solves: a 24-block grid AAb starts on whichever SMs the other
    # streams' gradient passes leave free; a 16-block cluster needs one GPU
    # processing cluster with 16 free SMs and waits for it.
    aab = args.aab or ("auto" if args.sequential or len(families) == 1 else "grid:24")
    aab_form, _, aab_blocks = aab.partition(":")
    for sk in sketches.values():
        sk.set_aab(aab_form, int(aab_blocks or 0))
    xs = {f: torch.empty(d, dtype=torch.float32, device=dev) for f in families}
    kw = dict(tol=args.tol, max_outer=args.max_outer, eps_sub=0.1)

    main_stream = torch.cuda.current_stream()
    streams = {f: (main_stream if args.sequential else torch.cuda.Stream()) for f in families}

    def step(want_info=False):
        # The solves of one step (one per sketch family, same A and b) are
        # independent of one another: each runs on its
        # own stream (so one solve's latency-bound inner solver overlaps
        # another's bandwidth-bound gradient pass), joined back to the main
        # stream at the end of the step.
        infos = {}
        ev = torch.cuda.Event()
        ev.record(main_stream)
        for f in families:
            s = streams[f]
            s.wait_event(ev)
            with torch.cuda.stream(s):
                sk = sketches[f]
                sk.resketch(A, seed)
                _, infos[f] = sk.solve(A, b, p.lam, p.sd, x=xs[f], want_info=want_info, **kw)
        for f in families:
            main_stream.wait_stream(streams[f])
        return infos

    # Warm-up; the last warm-up step reports iteration counts.
    for _ in range(max(args.warmup - 1, 0)):
        step()
    infos = step(want_info=True)
    not_converged = {f: inf.status for f, inf in infos.items() if inf.status != mihs.OK}
    # Launches per step: sketch kernels (counted by the library) + ctl init +
    # 3 per outer iteration (+1 final gradient) in the device-side loop.
    c0 = mihs.launch_count()
    for f in families:
        sketches[f].resketch(A, seed)
    torch.cuda.synchronize()
    sketch_launches = mihs.launch_count() - c0
    launches_per_step = sketch_launches + sum(1 + 3 * (inf.outer_iters + 1) for inf in infos.values())

    # ---------------- timed region (device-resident inputs)
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(gpu_uuid())
    time.sleep(1.0)  # let the sampler start before the timed region
    barrier(ws)
    torch.cuda.synchronize()
    t_host0 = time.perf_counter()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    wall = time.perf_counter() - t_host0
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    ms = max_over_ranks(ms, ws)
    value = ws * len(families) / (ms / 1e3)

    # ---------------- per-family and per-kernel times (event timing, one extra step)
    mihs.timing(True)
    per_family = {}
    for f in families:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sketches[f].resketch(A, seed)
        sketches[f].solve(A, b, p.lam, p.sd, x=xs[f], want_info=True, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
        per_family[f] = round(e0.elapsed_time(e1), 4)
    apass_ms, apass_n = mihs.timing_read(mihs.TIMER_APASS)
    aab_ms, aab_n = mihs.timing_read(mihs.TIMER_AAB)
    sk_ms, sk_n = mihs.timing_read(mihs.TIMER_SKETCH)
    mihs.timing(False)
    apass_avg_s = apass_ms / 1e3 / max(apass_n, 1)
    bytes_per_pass = 4 * (n * d + n + 2 * d)          # A, b, x read; g written
    achieved = bytes_per_pass / apass_avg_s / 1e9
    peaks, peak_src = measured_peaks()
    roofline = {"bound": "hbm", "kernel": "apass_partial_kernel (gradient g = Aᵀ(b−Ax) − λx)",
                "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / peaks["hbm_gbs"], 4), "peak_source": f"{peak_src} hbm_gbs",
                "traffic": (round(APASS_NCU["bytes"] * n / APASS_NCU["n"]) if d == APASS_NCU["d"] else None),
                "traffic_source": "ncu capture at 65536 rows, scaled by rows",
                "bytes_per_launch": bytes_per_pass,
                "avg_launch_us": round(apass_avg_s * 1e6, 2), "launches_timed": apass_n}

    # ---------------- compensated refinement: the same step with fp64 iterates
    refined = None
    if not args.no_refined:
        x64 = {f: torch.empty(d, dtype=torch.float64, device=dev) for f in families}
        kw_r = dict(tol=args.refined_tol, max_outer=args.max_outer, eps_sub=0.1)
        # Measured on this step: the one-cluster inner solver is the faster
        # form here (the grid form is the faster one in the plain step).
        form_r, _, blocks_r = args.aab_refined.partition(":")
        for sk in sketches.values():
            sk.set_aab(form_r, int(blocks_r or 0))

        def step_refined(want_info=False):
            infos_r = {}
            ev = torch.cuda.Event()
            ev.record(main_stream)
            for f in families:
                s_ = streams[f]
                s_.wait_event(ev)
                with torch.cuda.stream(s_):
                    sketches[f].resketch(A, seed)
                    _, infos_r[f] = sketches[f].solve_refined(A, b, p.lam, p.sd, x=x64[f], want_info=want_info, **kw_r)
            for f in families:
                main_stream.wait_stream(streams[f])
            return infos_r

        step_refined()
        inf_r = step_refined(want_info=True)
        n_ref = max(3, args.steps // 5)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n_ref):
            step_refined()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_r = max_over_ranks(e0.elapsed_time(e1) / n_ref, ws)
        mihs.timing(True)
        sketches[families[0]].solve_refined(A, b, p.lam, p.sd, x=x64[families[0]], **kw_r)
        dd_ms, dd_n = mihs.timing_read(mihs.TIMER_APASS_DD)
        pl_ms, pl_n = mihs.timing_read(mihs.TIMER_APASS)
        co_ms, co_n = mihs.timing_read(mihs.TIMER_APASS_CORR)
        mihs.timing(False)
        dd_avg_s = dd_ms / 1e3 / max(dd_n, 1)
        refined = {"value": round(ws * len(families) / (ms_r / 1e3), 3), "unit": "solves/s",
                   "ms_per_step": round(ms_r, 4), "steps": n_ref, "tol": args.refined_tol,
                   "status": {f: inf_r[f].status for f in families},
                   "outer_iters": {f: inf_r[f].outer_iters for f in families},
                   "switch_tol": 1e-7, "plain_steps": pl_n, "compensated_steps": dd_n,
                   "correction_steps": co_n, "aab": args.aab_refined,
                   "apass_dd_avg_us": round(dd_avg_s * 1e6, 2),
                   "apass_dd_frac_of_hbm": round(bytes_per_pass / dd_avg_s / 1e9 / peaks["hbm_gbs"], 4)}
        for sk in sketches.values():
            sk.set_aab(aab_form, int(aab_blocks or 0))

    # ---------------- accuracy vs the oracle's exact solution
    accuracy = None
    A_host = b_host = None
    if rank == 0 and not args.no_accuracy:
        from oracle import mihs_oracle as o
        A_host, b_host = A.cpu(), b.cpu()
        xstar = o.exact_solve(A_host.numpy(), b_host.numpy(), p.lam)  # κ(H) ≈ 1e4: fp64 refinement suffices
        accuracy = {}
        for f in families:
            _, inf = sketches[f].solve(A, b, p.lam, p.sd, x=xs[f], want_info=True, **kw)
            trace = sketches[f].history()
            accuracy[f] = {"rel_err_vs_oracle": float(f"{o.rel_error(xs[f].cpu().double().numpy(), xstar):.3e}"),
                           "rel_resid": float(f"{inf.rel_resid:.3e}"), "outer_iters": inf.outer_iters,
                           "inner_iters": inf.inner_iters_total,
                           "resid_trace_every_4": [float(f"{t:.2e}") for t in trace[::4]]}
        if refined is not None:
            refined["rel_err_vs_oracle"] = {
                f: float(f"{o.rel_error(x64[f].cpu().numpy(), xstar):.3e}") for f in families}

    # ---------------- end to end through the one-call API with host buffers
    e2e = None
    if not args.no_e2e:
        if A_host is None:
            A_host, b_host = A.cpu(), b.cpu()
        A_pin, b_pin = A_host.pin_memory(), b_host.pin_memory()
        outs = {f: torch.empty(d, dtype=torch.float32, pin_memory=True) for f in families}
        A_devs = [torch.empty(n, d, dtype=torch.float32, device=dev) for _ in range(2)]
        b_devs = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(2)]
        h2d_env = os.environ.get("MIHS_H2D_BLOCKS")
        if args.h2d_blocks > 0:
            os.environ["MIHS_H2D_BLOCKS"] = str(args.h2d_blocks)

        def measure_e2e(mode):
            """ms per step of `mode`: 'pipelined' (two device buffers, problem
            k+1 copied in on its own stream while problem k solves) or
            'serial' (copy, then solve, one problem at a time)."""
            nbuf = 2 if mode == "pipelined" else 1
            copy_stream = torch.cuda.Stream() if nbuf > 1 else main_stream
            free_ev = [[] for _ in range(nbuf)]  # events of the solves that last read each buffer
            engine = args.e2e_copy if args.e2e_copy != "auto" else ("dma" if nbuf > 1 else "sm")

            def e2e_step(k):
                # One problem per step: its A and b go to the device (the SMs
                # read the pinned host memory, or a copy engine does the copy),
                # the three family solves run on that copy and each x comes back
                # to the host.
                q = k % nbuf
                for e in free_ev[q]:
                    copy_stream.wait_event(e)
                mihs.copy_to_device(A_devs[q], A_pin, stream=copy_stream, engine=engine)
                mihs.copy_to_device(b_devs[q], b_pin, stream=copy_stream, engine=engine)
                ready = torch.cuda.Event()
                ready.record(copy_stream)
                done = []
                for f in families:
                    streams[f].wait_event(ready)
                    with torch.cuda.stream(streams[f]):
                        xf, _ = mihs.solve(A_devs[q], b_devs[q], p.lam, f, m, p.sd, seed=seed, want_info=False,
                                           aab=aab, **kw)
                        outs[f].copy_(xf, non_blocking=True)
                        ev = torch.cuda.Event()
                        ev.record(streams[f])
                        done.append(ev)
                free_ev[q] = done

            def drain():
                for f in families:
                    main_stream.wait_stream(streams[f])
                main_stream.wait_stream(copy_stream)

            for k in range(max(args.warmup, 1)):
                e2e_step(k)
            drain()
            torch.cuda.synchronize()
            barrier(ws)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            copy_stream.wait_stream(main_stream)
            for k in range(args.steps):
                e2e_step(k)
            drain()
            e1.record(stream)
            torch.cuda.synchronize()
            barrier(ws)
            ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, ws)
            how = ("a copy engine, mihs_copy_to_device_dma" if engine == "dma" else
                   f"the SMs, mihs_copy_to_device on {args.h2d_blocks or 'all'} SMs")
            return ms, how

        ms_e2e, how = measure_e2e(args.e2e_mode)
        other = "serial" if args.e2e_mode == "pipelined" else "pipelined"
        ms_other, how_other = measure_e2e(other)
        if h2d_env is None:
            os.environ.pop("MIHS_H2D_BLOCKS", None)
        else:
            os.environ["MIHS_H2D_BLOCKS"] = h2d_env
        desc = {"pipelined": "two device buffers: problem k+1 is copied in on its own stream while problem k's "
                             "three solves run",
                "serial": "copy, then the three solves, one problem at a time"}
        e2e = {"value": round(ws * len(families) / (ms_e2e / 1e3), 3), "unit": "solves/s",
               "ms_per_step": round(ms_e2e, 4),
               "h2d_bytes_per_step": 4 * (n * d + n),
               "d2h_bytes_per_step": len(families) * 4 * d,
               "mode": args.e2e_mode,
               "copies": (f"each step copies its problem's A and b in (1.07 GB from pinned host memory, {how}) "
                          f"and each family's x out; {desc[args.e2e_mode]}"),
               other: {"value": round(ws * len(families) / (ms_other / 1e3), 3),
                       "ms_per_step": round(ms_other, 4),
                       "copies": f"{how_other}; {desc[other]}"}}

    # ---------------- the 4096 × 256 problem (L2-resident, latency-bound)
    small = None
    if not args.no_small:
        small = run_small(args, dev, ws)

    # ---------------- differentiable solve: forward + adjoint backward
    differentiable = None
    if not args.no_backward:
        differentiable = run_differentiable(args, dev, ws, peaks, peak_src)

    # ---------------- batched λ-paths: 64 matrices × 16 λ
    batched = None
    if not args.no_batched:
        batched = run_batched(args, dev, ws, peaks, peak_src)

    # ---------------- mixed precision: 2²¹ × 2048, κ(H) ≈ 1e6, refined to --mixed-tol
    mixed = None
    if not args.no_mixed:
        mixed = run_mixed(args, dev, ws)

    dual = None
    if not args.no_dual:
        dual = run_dual(args, dev, ws, peaks, peak_src)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        if A_host is None:
            A_host, b_host = A.cpu(), b.cpu()
        ot = OracleTimer(A_host, b_host, p, families, rows=ORACLE_ROWS)
        ot.measure_all()
        cpu = {"value": round(ot.value(), 5), "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": ot.sample(), "detail": ot.detail(),
               "one_core": oracle_one_core(A_host, b_host, families)}

    if rank == 0:
        out = {
            "metric": METRIC, "value": round(value, 3), "unit": "solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{p.name}, SNR 40 dB, m={m} (4·sd, sd={p.sd:.2f}), "
                                   f"one solve per family {families}",
                       "n": n, "d": d, "m": m, "lambda": p.lam, "sd": round(p.sd, 3), "tol": args.tol,
                       "stop": "‖Aᵀ(b−Ax)−λx‖ ≤ tol·‖Aᵀb‖", "eps_sub": 0.1,
                       "families": families, "l2": "inputs larger than L2 (A = %.2f GB)" % (4 * n * d / 1e9),
                       "streams": "sequential" if args.sequential else "one CUDA stream per family (independent solves run concurrently)",
                       "aab": aab,
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "gpu_launches": launches_per_step * args.steps,
            "per_family_ms": per_family,
            "kernel_ms": {"apass_avg": round(apass_avg_s * 1e3, 4), "aab_avg": round(aab_ms / max(aab_n, 1), 4),
                          "aab_launches": aab_n, "sketch_total": round(sk_ms, 4)},
            "roofline": roofline,
            "accuracy": accuracy,
            "small": small,
            "refined": refined,
            "differentiable": differentiable,
            "batched": batched,
            "mixed": mixed,
            "dual": dual,
            "not_converged": not_converged or None,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clk,
            "host_wall_s_timed": round(wall, 3),
        }
        print(json.dumps(out), flush=True)
    for sk in sketches.values():
        sk.close()


def run_small(args, dev, ws):
    """The 4096 × 256 problem (σ_i = 10^(−4(i−1)/255), λ with sd = 64, 30 dB
    SNR, Gaussian sketch m = 256, stop at relative residual 1e-6): A is 4 MB
    and stays in L2, so this measures latency, not bandwidth.  One step =
    sketch + solve on one stream; the oracle's whole CPU solve (sketch +
    Algorithm 1 in fp64) is timed beside it on the host cores."""
    import torch

    from oracle import mihs_oracle as o
    from paper_1912_03514_gb300 import mihs
    from paper_1912_03514_gb300 import workloads as W
    p = W.problem_small(device=str(dev))
    tol = 1e-6
    x = torch.empty(p.d, device=dev)
    sk = mihs.Sketch(p.A, "gaussian", p.m, seed=3)

    def step(want_info=False):
        sk.resketch(p.A, 3)
        return sk.solve(p.A, p.b, p.lam, p.sd, tol=tol, max_outer=200, x=x, want_info=want_info)[1]

    for _ in range(max(args.warmup, 3)):
        step()
    info = step(want_info=True)
    nsteps = 200
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(nsteps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / nsteps, ws)
    sk.close()
    out = {"workload": f"{p.name}: 4096×256, σ_i = 10^(−4(i−1)/255), λ = {p.lam:.6g} (sd = 64), 30 dB SNR, "
                       f"Gaussian m = {p.m}, stop at relative residual {tol:g}; A = 4 MB (L2-resident)",
           "value": round(ws / (ms / 1e3), 2), "unit": "solves/s", "ms_per_step": round(ms, 4), "steps": nsteps,
           "status": info.status, "outer_iters": info.outer_iters, "inner_iters": info.inner_iters_total,
           "rel_resid": float(f"{info.rel_resid:.3e}")}
    if int(os.environ.get("RANK", "0")) == 0:
        An, bn = p.A.cpu().numpy(), p.b.cpu().numpy()
        xs = o.exact_solve(An, bn, p.lam)
        out["rel_err_vs_oracle"] = float(f"{o.rel_error(x.cpu().double().numpy(), xs):.3e}")
        t0 = time.perf_counter()
        reps = 0
        while reps < 3 or time.perf_counter() - t0 < 3.0:
            xo, io = o.mihs_solve(An, bn, p.lam, o.GAUSSIAN, p.m, p.sd, 3, N=200, tol=tol)
            reps += 1
        t_o = (time.perf_counter() - t0) / reps
        out["oracle_cpu"] = {"value": round(1.0 / t_o, 3), "unit": "solves/s", "cores": os.cpu_count(),
                             "kind": "oracle", "sample": f"the whole solve (sketch + Algorithm 1, fp64), "
                                                         f"{reps} runs", "outer_iters": io["outer"],
                             "rel_err_vs_exact": float(f"{o.rel_error(xo, xs):.3e}")}
    return out


def run_differentiable(args, dev, ws, peaks, peak_src):
    """Forward solve plus backward (adjoint solve with the same sketch and the
    fused gradient pass) on 2²⁰ × 1024, σᵢ = i^(−1.5), λ = 1e-4, 40 dB SNR,
    CountSketch with m = 4·sd; upstream gradient ḡ a seeded N(0, 1) vector."""
    import torch

    from paper_1912_03514_gb300 import mihs
    from paper_1912_03514_gb300 import workloads as W
    p = W.problem_differentiable(device=str(dev))
    A, b = p.A, p.b
    n, d = p.n, p.d
    gbar = W.randn((d,), seed=1004).to(dev)
    sk = mihs.Sketch(A, "countsketch", p.m, seed=11)
    # κ(H) ≈ 1e4: the adjoint of a generic ḡ has an fp32 residual floor of a
    # few 1e-6, so both solves use compensated refinement to 1e-10.
    tol = 1e-10
    x = torch.empty(d, device=dev, dtype=torch.float64)
    v = torch.empty(d, device=dev, dtype=torch.float64)

    def step(want_info=False):
        sk.resketch(A, 11)
        _, ix = sk.solve_refined(A, b, p.lam, p.sd, tol=tol, x=x, want_info=want_info)
        dA, db, dl, _, iv = sk.backward_refined(A, b, p.lam, p.sd, x, gbar, tol=tol, v=v, want_info=want_info)
        return ix, iv, dA, db, dl

    for _ in range(max(args.warmup, 3)):
        step()
    ix, iv, dA, db, dl = step(want_info=True)
    del dA, db
    steps = max(3, args.steps // 10)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, ws)
    mihs.timing(True)
    x32, v32 = x.float(), v.float()
    for _ in range(3):
        mihs.backward_grads(A, b, x32, v32)
    bw_ms, bw_n = mihs.timing_read(mihs.TIMER_BACKWARD)
    mihs.timing(False)
    bw_s = bw_ms / 1e3 / max(bw_n, 1)
    by = 8 * n * d + 8 * n
    sk.close()
    return {"value": round(ws / (ms / 1e3), 3), "unit": "forward+backward solves/s", "ms_per_step": round(ms, 4),
            "steps": steps,
            "workload": f"{p.name}, SNR 40 dB, countsketch m={p.m} (4·sd, sd={p.sd:.2f}), "
                        f"refined solves to tol {tol:g} for x and the adjoint v",
            "forward": {"outer_iters": ix.outer_iters, "rel_resid": float(f"{ix.rel_resid:.3e}"), "status": ix.status},
            "adjoint": {"outer_iters": iv.outer_iters, "rel_resid": float(f"{iv.rel_resid:.3e}"), "status": iv.status},
            "dlambda": dl.item(),
            "backward_kernel": {"bound": "hbm", "bytes_per_launch": by, "avg_launch_us": round(bw_s * 1e6, 2),
                                "achieved": round(by / bw_s / 1e9, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                "frac": round(by / bw_s / 1e9 / peaks["hbm_gbs"], 4),
                                "peak_source": f"{peak_src} hbm_gbs"}}


def run_batched(args, dev, ws, peaks, peak_src):
    """64 matrices (n log-uniform in [8192, 262144], d in {64 … 1024}, σ_i =
    10^(−r(i−1)/(d−1)), r ~ U[2, 6]) × one 16-value λ path in [1e-6, 1e-1]:
    per matrix a Gaussian sketch with m = 4·sd(λ_min), then the whole path
    (mihs_solve_batched: one fused gradient pass per step for all 16 λ) to a
    relative residual of 1e-7, then compensated refinement
    (mihs_refine_batched) of the λ whose κ(AᵀA + λI) = (σ₁² + λ)/λ exceeds
    5e3 (σ₁ = 1 by construction), where no fp32 residual certifies a relative
    error of 1e-5.  One step = sketch + path solve + refinement for all 64
    matrices; value = (matrix, λ) solves per second.  The error of every
    (matrix, λ) against the oracle's x*(λ) is measured on a sample of
    matrices, for this form and for one plain solve per (matrix, λ)."""
    import numpy as np
    import torch

    from paper_1912_03514_gb300 import mihs
    from paper_1912_03514_gb300 import workloads as W
    probs, lams, sds = W.batch_lambda_path(device=str(dev), device_rng=True)
    tol, tol_ref, kappa_fp32 = 1e-7, 1e-10, 5e3
    tols = [tol_ref if (1.0 + lam) / lam > kappa_fp32 else 0.0 for lam in lams]
    handles = [mihs.Sketch(q.A, "gaussian", q.m, seed=100 + i) for i, q in enumerate(probs)]
    Xs = [torch.empty(len(lams), q.d, device=dev) for q in probs]
    entries = [(sk, q.A, q.b, X) for sk, q, X in zip(handles, probs, Xs)]

    def step(want_info=False, sub=None, marks=None):
        ent = entries if sub is None else entries[:sub]
        for i, (sk, q) in enumerate(zip(handles[:len(ent)], probs)):
            sk.resketch(q.A, 100 + i)
        sd_ = sds[:len(ent)]
        inf = mihs.solve_batched(ent, lams, sds=sd_, tol=tol, max_outer=200, want_info=want_info)
        if marks is not None:  # end of the fp32 path phase, on the caller's stream
            marks.append(torch.cuda.Event(enable_timing=True))
            marks[-1].record(torch.cuda.current_stream())
        rinf = mihs.refine_batched(ent, lams, tols, sds=sd_, max_outer=200, want_info=want_info)
        return inf, rinf

    step()
    infos, rinfos = step(want_info=True)
    steps = 2
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    marks = []
    starts = [e0]
    for k in range(steps):
        step(marks=marks)
        if k + 1 < steps:
            starts.append(torch.cuda.Event(enable_timing=True))
            starts[-1].record(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, ws)
    ends = starts[1:] + [e1]
    path_ms = sum(a.elapsed_time(b) for a, b in zip(starts, marks)) / steps
    refine_ms = sum(a.elapsed_time(b) for a, b in zip(marks, ends)) / steps
    # per-kernel split and the fused pass's arithmetic rate (host-driven, timed)
    mihs.timing(True)
    for i, (sk, q) in enumerate(zip(handles, probs)):
        sk.resketch(q.A, 100 + i)
    mihs.solve_batched(entries, lams, sds=sds, tol=tol, max_outer=200, want_info=False)
    sk_ms, _ = mihs.timing_read(mihs.TIMER_SKETCH)
    pa_ms, pa_n = mihs.timing_read(mihs.TIMER_APASS_PATH)
    aab_ms, aab_n = mihs.timing_read(mihs.TIMER_AAB)
    mihs.timing(False)
    # flops of the fused passes that ran: 64 per element of A per pass (16 λ × 2 products)
    steps_per = [max(i.outer_iters for i in row) + 1 for row in infos]
    flops = sum(64.0 * q.n * q.d * k for q, k in zip(probs, steps_per))
    nom_fp32 = 152 * 128 * 2 * 2.07e9 / 1e12  # TFLOP/s: 152 SMs × 128 FP32 lanes × FMA × 2.07 GHz
    flat = [i for row in infos for i in row]
    rflat = [i for row in rinfos for i in row if i is not None]
    out = {"value": round(ws * len(probs) * len(lams) / (ms / 1e3), 2), "unit": "(matrix, λ) solves/s",
           "ms_per_step": round(ms, 3), "steps": steps,
           "phase_ms": {"sketch_and_fp32_paths": round(path_ms, 1), "refinement": round(refine_ms, 1)},
           "workload": f"{len(probs)} matrices (n log-uniform 8192–262144, d in 64–1024, "
                       f"{sum(4 * q.n * q.d for q in probs) / 1e9:.2f} GB of A), 16 λ in [1e-6, 1e-1], "
                       f"Gaussian m = 4·sd(λ_min); fp32 path to residual {tol:g}, then the "
                       f"{sum(t > 0 for t in tols)} λ with κ(H) > {kappa_fp32:g} refined to {tol_ref:g}",
           "converged": sum(i.status == 0 for i in flat), "solves": len(flat),
           "refined_converged": sum(i.status == 0 for i in rflat), "refined_solves": len(rflat),
           "max_rel_resid_fp32": float(f"{max(i.rel_resid for i in flat):.3e}"),
           "max_rel_resid_refined": float(f"{max(i.rel_resid for i in rflat):.3e}") if rflat else None,
           "refined_outer_iters_mean": round(sum(i.outer_iters for i in rflat) / max(len(rflat), 1), 1),
           "refined_inner_passes_mean": round(sum(i.inner_iters_total for i in rflat) / max(len(rflat), 1), 1),
           "outer_iters_max": max(i.outer_iters for i in flat),
           "kernel_ms_path_solve": {"sketch": round(sk_ms, 3), "path_apass": round(pa_ms, 3),
                                    "path_apass_launches": pa_n, "aab": round(aab_ms, 3), "aab_launches": aab_n},
           "path_apass_roofline": {"bound": "alu", "achieved": round(flops / (pa_ms / 1e3) / 1e12, 2),
                                   "peak": round(nom_fp32, 1), "unit": "TFLOP/s",
                                   "frac": round(flops / (pa_ms / 1e3) / 1e12 / nom_fp32, 4),
                                   "peak_source": "derived: 152 SMs × 128 FP32 FMA/clk × 2 flops × 2.07 GHz"}}
    # the plain single-λ form on the same problems at the same accuracy: one
    # mihs_solve (residual 1e-7) or, for the refined λ, one
    # mihs_solve_refined (residual 1e-10) per (matrix, λ) on the matrix's
    # handle, over the first 8 matrices
    nsub = min(8, len(probs))
    x1 = [torch.empty(q.d, device=dev) for q in probs[:nsub]]
    x64 = [torch.empty(q.d, dtype=torch.float64, device=dev) for q in probs[:nsub]]
    Xp = [torch.empty(len(lams), q.d, device=dev) for q in probs[:nsub]]

    def plain_pass(keep=False):
        for i in range(nsub):
            q, sk = probs[i], handles[i]
            sk.resketch(q.A, 100 + i)
            for l, lam in enumerate(lams):
                if tols[l] > 0:
                    sk.solve_refined(q.A, q.b, lam, sds[i][l], tol=tol_ref, max_outer=200, x=x64[i],
                                     want_info=False)
                    if keep:
                        Xp[i][l].copy_(x64[i])
                else:
                    sk.solve(q.A, q.b, lam, sds[i][l], tol=tol, max_outer=200, x=x1[i], want_info=False)
                    if keep:
                        Xp[i][l].copy_(x1[i])

    plain_pass(keep=True)
    torch.cuda.synchronize()
    e0.record(stream)
    plain_pass()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_p = max_over_ranks(e0.elapsed_time(e1), ws)

    step(sub=nsub)
    torch.cuda.synchronize()
    e0.record(stream)
    step(sub=nsub)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_b = max_over_ranks(e0.elapsed_time(e1), ws)
    out["plain_single_lambda"] = {
        "value": round(ws * nsub * len(lams) / (ms_p / 1e3), 2), "unit": "(matrix, λ) solves/s",
        "batched_same_sample": round(ws * nsub * len(lams) / (ms_b / 1e3), 2),
        "sample": f"the first {nsub} matrices × {len(lams)} λ: one mihs_solve (residual {tol:g}) or "
                  f"mihs_solve_refined (residual {tol_ref:g}, the same λ as the batched form refines) per "
                  f"(matrix, λ) on the matrix's handle (same sketch), against mihs_solve_batched + "
                  f"mihs_refine_batched on the same {nsub} matrices"}
    # error against the oracle on the sample, both forms (rank 0)
    if int(os.environ.get("RANK", "0")) == 0:
        from oracle import mihs_oracle as o
        t0 = time.time()
        err_b, err_p, per_lam = [], [], [0.0] * len(lams)
        for i in range(nsub):
            q = probs[i]
            XS = o.ridge_path(q.A.cpu().numpy(), q.b.cpu().numpy(), lams)
            Xb, Xq = Xs[i].cpu().double().numpy(), Xp[i].cpu().double().numpy()
            for l in range(len(lams)):
                eb, ep = o.rel_error(Xb[l], XS[l]), o.rel_error(Xq[l], XS[l])
                err_b.append(eb)
                err_p.append(ep)
                per_lam[l] = max(per_lam[l], eb)
        out["accuracy_vs_oracle"] = {
            "sample": f"the first {nsub} matrices ({', '.join(q.name for q in probs[:nsub])}) × all "
                      f"{len(lams)} λ; oracle: fp64 Gram, Cholesky per λ, two fp64 refinement steps",
            "max_rel_err_batched": float(f"{max(err_b):.3e}"),
            "max_rel_err_plain_single_lambda": float(f"{max(err_p):.3e}"),
            "max_rel_err_batched_by_lambda": {f"{lam:.3g}": float(f"{e:.2e}") for lam, e in zip(lams, per_lam)},
            "oracle_s": round(time.time() - t0, 1)}
    for sk in handles:
        sk.close()
    return out


def run_dual(args, dev, ws, peaks, peak_src):
    """Dual M-IHS (Algorithm 2) on a wide problem: n = 2048 rows, d = 2¹⁸
    columns (A = 2.1 GB), σ_i = 1/i, λ = 1e-4 (sd ≈ 147), b = A x0 + ω at
    40 dB; CountSketch and Gaussian sketches of Aᵀ with m = 4·sd; stop at
    relative dual residual 1e-6.  One step = sketch + solve + x = Aᵀν.  The
    roofline is the dual gradient g = b − A(Aᵀν) − λν alone: two passes over A
    (8nd bytes)."""
    import numpy as np
    import torch

    from paper_1912_03514_gb300 import mihs
    from paper_1912_03514_gb300 import workloads as W
    n, d, lam = 2048, 1 << 18, 1e-4
    sigma = 1.0 / np.arange(1, n + 1, dtype=np.float64)
    q = W.make_problem(d, n, sigma, lam, 40.0, seed=1004, device=str(dev), device_rng=True)
    A = q.A.t().contiguous()           # n × d with singular values σ
    del q
    g = torch.Generator(device=dev).manual_seed(1005)
    x0 = torch.randn(d, generator=g, device=dev)
    Ax0 = A @ x0
    om = torch.randn(n, generator=g, device=dev)
    b = (Ax0 + om * (Ax0.norm() / om.norm()) / 100.0).contiguous()
    sd = W.nominal_sd(sigma, lam)
    m = int(math.ceil(4 * sd / 4)) * 4
    out = {"workload": f"dual-{n}x{d}-poly1-lam1e-4, SNR 40 dB, m = {m} (4·sd, sd = {sd:.2f}), tol 1e-6; "
                       f"A = {4 * n * d / 1e9:.2f} GB", "unit": "solves/s", "by_family": {}}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    for fam in ("countsketch", "gaussian"):
        dk = mihs.DualSketch(A, fam, m, seed=7)
        x = torch.empty(d, device=dev)
        nu = torch.empty(n, device=dev)

        def step(want_info=False):
            dk.resketch(A, 7)
            return dk.solve(A, b, lam, sd, tol=1e-6, max_outer=200, x=x, nu=nu, want_info=want_info)[2]
        info = step(want_info=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(3):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1) / 3, ws)
        out["by_family"][fam] = {"value": round(ws / (ms / 1e3), 3), "ms_per_step": round(ms, 3),
                                 "status": info.status, "outer_iters": info.outer_iters,
                                 "inner_iters": info.inner_iters_total, "rel_resid": float(f"{info.rel_resid:.3e}")}
        dk.close()
    # the dual gradient's two passes over A, timed alone
    nu = torch.randn(n, device=dev)
    gd = torch.empty(n, device=dev)
    for _ in range(3):
        mihs.gradient_dual(A, b, nu, lam, g=gd)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(10):
        mihs.gradient_dual(A, b, nu, lam, g=gd)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 10 / 1e3
    by = 8.0 * n * d + 4.0 * (3 * n + d)
    out["gradient_roofline"] = {"bound": "hbm", "kernels": "atnu_kernel + dual_resid_kernel",
                                "bytes_per_call": by, "avg_call_us": round(t * 1e6, 2),
                                "achieved": round(by / t / 1e9, 1), "peak": peaks.get("hbm_gbs"),
                                "unit": "GB/s", "frac": round(by / t / 1e9 / peaks.get("hbm_gbs"), 4)
                                if peaks.get("hbm_gbs") else None, "peak_source": peak_src}
    return out


def run_mixed(args, dev, ws):
    """2²¹ × 2048, σ_i = 10^(−8(i−1)/2047), λ = 1e-6 (sd ≈ 768, κ(H) ≈ 1e6),
    40 dB SNR, Gaussian sketch with m = 4·sd: compensated-refinement solves to
    a relative residual of --mixed-tol with SA stored in fp32, bf16 and fp8
    inside AAb_Solver (bf16 handles form S·A from bf16 operands, fp8 handles
    from e4m3 operands).  One
    step = sketch + refined solve.  The relative error against the oracle is
    measured on a sample with the same σ profile, λ and sketch size at
    --mixed-sample-rows rows (the oracle's fp64 Gram of all 2²¹ rows takes
    minutes on the host; --mixed-oracle does it for the full problem)."""
    import numpy as np
    import torch

    from paper_1912_03514_gb300 import mihs
    from paper_1912_03514_gb300 import workloads as W
    n, d, lam = 1 << 21, 2048, 1e-6
    tol = args.mixed_tol
    precs = ("fp32", "bf16", "fp8")

    def solve_all(p, A, b, timed, lam=lam, sd=None, m=None):
        sd = p.sd if sd is None else sd
        m = p.m if m is None else m
        res = {}
        sk = mihs.Sketch(A, "gaussian", m, seed=3)
        x = torch.empty(d, dtype=torch.float64, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream = torch.cuda.current_stream()
        for prec in precs:
            def step(want_info=False):
                sk.resketch(A, 3)
                return sk.solve_refined(A, b, lam, sd, tol=tol, max_outer=300, x=x, want_info=want_info)[1]
            sk.set_precision(prec)
            try:
                info = step(want_info=True)
            except mihs.MihsError as e:  # the library's guard: the quantised SA no longer preconditions
                res[prec] = {"status": e.code, "error": str(e)[:400]}
                continue
            r = {"status": info.status, "outer_iters": info.outer_iters, "inner_iters": info.inner_iters_total,
                 "rel_resid": float(f"{info.rel_resid:.3e}"), "x": x.cpu().numpy().copy()}
            if timed:
                torch.cuda.synchronize()
                e0.record(stream)
                step()
                e1.record(stream)
                torch.cuda.synchronize()
                ms = max_over_ranks(e0.elapsed_time(e1), ws)
                r.update({"value": round(ws / (ms / 1e3), 3), "ms_per_step": round(ms, 2)})
                # per-kernel event times of one more step (host-driven: the
                # library times each launch on the solve's stream)
                mihs.timing(True)
                step()
                torch.cuda.synchronize()
                r["kernel_ms"] = {k: round(mihs.timing_read(t)[0], 2) for k, t in
                                  (("sketch", mihs.TIMER_SKETCH), ("apass", mihs.TIMER_APASS),
                                   ("apass_dd", mihs.TIMER_APASS_DD), ("apass_corr", mihs.TIMER_APASS_CORR),
                                   ("aab", mihs.TIMER_AAB))}
                r["steps"] = {k: mihs.timing_read(t)[1] for k, t in
                              (("plain", mihs.TIMER_APASS), ("compensated", mihs.TIMER_APASS_DD),
                               ("correction", mihs.TIMER_APASS_CORR))}
                mihs.timing(False)
            res[prec] = r
        sk.close()
        return res

    p = W.make_problem(n, d, W.profile_exponential(d, 8.0), lam, 40.0, seed=1002, device=str(dev), device_rng=True)
    out = {"workload": f"{p.name}, SNR 40 dB, λ = 1e-6 (sd {p.sd:.1f}, κ(H) ≈ 1e6), Gaussian m = {p.m}, "
                       f"refinement to relative residual {tol:g}; A = {4 * n * d / 1e9:.1f} GB",
           "unit": "solves/s",
           "sketch_operands": "fp32 SA: tf32 S and A; bf16 SA: S·A formed from bf16 S and A; fp8 SA: "
                              "from e4m3 S and A (A scaled by a power of two); fp32 accumulation, then "
                              "stored in that precision",
           "by_sa_precision": solve_all(p, p.A, p.b, True)}
    if args.mixed_oracle:
        from oracle import mihs_oracle as o
        xs = o.exact_solve(p.A.cpu().numpy(), p.b.cpu().numpy(), lam, refine=2, dd=True)
        for r in out["by_sa_precision"].values():
            if "x" in r:
                r["rel_err_vs_oracle"] = float(f"{o.rel_error(r['x'], xs):.3e}")
    for r in out["by_sa_precision"].values():
        r.pop("x", None)
    # The same matrix at λ = 1e-3 (κ(H) ≈ 1e3), where fp8 and bf16 storage of
    # SA still precondition (the guard accepts them): m = 4·sd(1e-3).
    lam3 = 1e-3
    sd3 = W.nominal_sd(p.sigma, lam3)
    m3 = W.round_up(4.0 * sd3, 4)
    r3 = solve_all(p, p.A, p.b, True, lam=lam3, sd=sd3, m=m3)
    for r in r3.values():
        r.pop("x", None)
    out["lambda_1e-3"] = {"workload": f"the same A and b, λ = {lam3:g} (sd {sd3:.1f}, κ(H) ≈ 1e3), Gaussian m = {m3}, "
                                      f"refinement to relative residual {tol:g} (relative error ≤ κ(H)·residual "
                                      f"≈ {1e3 * tol:.0e})",
                          "by_sa_precision": r3}
    del p
    torch.cuda.empty_cache()
    if args.mixed_sample_rows > 0:
        from oracle import mihs_oracle as o
        ns = args.mixed_sample_rows
        q = W.make_problem(ns, d, W.profile_exponential(d, 8.0), lam, 40.0, seed=1012, device=str(dev),
                           device_rng=True)
        res = solve_all(q, q.A, q.b, False)
        # the plain fp32 path (fp32 iterate and gradient, no refinement) on the
        # same sample: its error floor at κ(H) ≈ 1e6
        with mihs.Sketch(q.A, "gaussian", q.m, seed=3) as skp:
            xp, ip = skp.solve(q.A, q.b, lam, q.sd, tol=1e-9, max_outer=150)
        res["plain_fp32_no_refinement"] = {"status": ip.status, "outer_iters": ip.outer_iters,
                                           "inner_iters": ip.inner_iters_total,
                                           "rel_resid": float(f"{ip.rel_resid:.3e}"),
                                           "x": xp.double().cpu().numpy()}
        t0 = time.time()
        xs = o.exact_solve(q.A.cpu().numpy(), q.b.cpu().numpy(), lam, refine=2, dd=True)
        t_or = time.time() - t0
        for r in res.values():
            if "x" in r:
                r["rel_err_vs_oracle"] = float(f"{o.rel_error(r.pop('x'), xs):.3e}")
        out["accuracy_sample"] = {
            "workload": f"{q.name}: the same σ profile, λ, SNR and m = {q.m} on {ns} rows",
            "oracle": "fp64 Gram + Cholesky, 2 refinement steps with a double-double residual (host C)",
            "oracle_s": round(t_or, 1), "by_sa_precision": res}
    return out


def run_profile_op(args, local):
    """W + K launches of one operation on the workload, timed with CUDA events."""
    import numpy as np
    import torch

    from paper_1912_03514_gb300 import mihs
    from paper_1912_03514_gb300 import workloads as W
    dev = torch.device("cuda", local)
    p = W.problem_bandwidth(device=str(dev), seed=1001, n=args.n, d=args.d)
    A, b = p.A, p.b
    x = W.randn((p.d,), seed=5, scale=0.01).to(dev)
    g = torch.empty(p.d, device=dev)
    op = args.profile_op
    if op == "dual-grad":
        # the Dual M-IHS gradient g = b − A(Aᵀν) − λν on a wide 2048 × (n·d/2048)
        # matrix (as many elements as the n × d workload)
        nd, dd = 2048, max(1024, args.n * args.d // 2048)
        Aw = W.randn((nd, dd), 11, scale=1.0 / math.sqrt(dd)).to(dev)
        bw = W.randn((nd,), 12).to(dev)
        nu = W.randn((nd,), 13).to(dev)
        gd = torch.empty(nd, device=dev)
        fn = lambda: mihs.gradient_dual(Aw, bw, nu, 1e-4, g=gd)
    elif op in ("aab-wide", "aab-wide-bf16"):
        # AAb_Solver on an SA of the mixed-precision workload's shape (m = 3076,
        # d = 2048, 25 MB in fp32, 12.6 MB in bf16: too large for one cluster,
        # so the grid form runs), a fixed 200 passes (per-pass latency =
        # ms_per_call / 200)
        m, d = 3076, 2048
        SA = W.randn((m, d), 7, scale=1.0 / math.sqrt(m)).to(dev)
        gw = W.randn((d,), 8).to(dev)
        delta = torch.empty(d, device=dev)
        if op == "aab-wide":
            fn = lambda: mihs.aab_solve(SA, gw, 1e-6, 0.0, max_inner=200, delta=delta)
        else:
            q, sc = mihs.quantize_sa(SA, "bf16")
            fn = lambda: mihs.aab_solve_q(q, "bf16", sc, d, gw, 1e-6, 0.0, max_inner=200, delta=delta)
    elif op in ("aab", "aab-late"):
        SA = mihs.sketch_apply(A, "countsketch", p.m, 3)
        x0 = torch.zeros_like(x)
        if op == "aab-late":  # a gradient from late in a solve (the typical inner solve)
            with mihs.Sketch(A, "countsketch", p.m, 3) as sk:
                sk.solve(A, b, p.lam, p.sd, tol=1e-6, x=x0)
        g = mihs.gradient(A, b, x0, p.lam)
        delta = torch.empty_like(g)
        fn = lambda: mihs.aab_solve(SA, g, p.lam, 0.1, delta=delta)
    elif op == "apass":
        fn = lambda: mihs.gradient(A, b, x, p.lam, g=g)
    elif op == "apass-dd":
        x64, g64 = x.double(), torch.empty(p.d, device=dev, dtype=torch.float64)
        fn = lambda: mihs.gradient_refined(A, b, x64, p.lam, g=g64)
    elif op == "path":
        # one λ-path solve (16 λ in [1e-6, 1e-1]) on an exponential profile of 3
        # decades with m = 4·sd(λ_min): the shape of the batched workload's
        # widest sketches (the AAb form follows MIHS_PATH_AAB)
        q = W.problem_scaled(args.n, args.d, seed=5, decades=3.0, sd_frac=0.9, device=str(dev))
        lams = list(np.logspace(-6, -1, 16))
        sds = [W.nominal_sd(q.sigma, l) for l in lams]
        m = min(q.n, int(np.ceil(max(sds))) * 4)
        skp = mihs.Sketch(q.A, "gaussian", m, seed=3)
        Xp = torch.empty(16, q.d, device=dev)
        fn = lambda: skp.solve_path(q.A, q.b, lams, sds=sds, tol=1e-6, max_outer=100, X=Xp, want_info=False)
    elif op in ("gaussian-bf16", "gaussian-fp8"):
        SA = torch.empty(p.m, p.d, device=dev)
        form = mihs.sketch_gaussian_bf16 if op == "gaussian-bf16" else mihs.sketch_gaussian_fp8
        fn = lambda: form(A, p.m, 3, SA=SA)
    elif op == "backward":
        v = W.randn((p.d,), seed=6, scale=0.01).to(dev)
        fn = lambda: mihs.backward_grads(A, b, x, v)
    else:
        SA = torch.empty(p.m, p.d, device=dev)
        fn = lambda: mihs.sketch_apply(A, op, p.m, 3, SA=SA)
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    print(json.dumps({"profile_op": op, "n": p.n, "d": p.d, "m": p.m,
                      "ms_per_call": round(e0.elapsed_time(e1) / args.steps, 4)}), flush=True)


def run_reference(args, ws, rank, families):
    """The oracle, as it stands, on the host cores (bounded sample per step)."""
    if rank != 0:
        return
    from paper_1912_03514_gb300 import workloads as W
    p = W.problem_bandwidth(device="cpu", seed=1001, n=args.n, d=args.d)
    # The first step times every piece of the oracle's work; each later step
    # re-times one piece in turn (a second or a few at 262144×1024), so that
    # the whole run stays within minutes for any --steps.  A step's value
    # combines the latest time of every piece.
    ot = OracleTimer(p.A, p.b, p, families, rows=ORACLE_ROWS)
    vals = []
    for k in range(args.warmup + args.steps):
        if k == 0:
            ot.measure_all()
        else:
            ot.measure(ot.parts[(k - 1) % len(ot.parts)])
        if k >= args.warmup:
            vals.append(ot.value())
    v = statistics.median(vals)
    sample = ot.sample() + "; one piece re-timed per step after the first"
    out = {"impl": "reference", "metric": METRIC, "value": round(v, 5), "unit": "solves/s",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{p.name}, SNR 40 dB, m={p.m}, one solve per family {families}",
                      "n": p.n, "d": p.d, "m": p.m, "families": families},
           "cpu_baseline": {"value": round(v, 5), "unit": "solves/s", "cores": os.cpu_count(),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": round(v, 5), "unit": "solves/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
