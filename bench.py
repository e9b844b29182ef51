"""Benchmark: space-time DOF/s of a full STMG solve to 1e-8 relative residual.

One step = one ``stmg_solve`` of the 4097 x 16385-node workload (N = 4096 elements,
NT = 16384 steps, box-filtered SIMP conductivity with k_ins = 1e-4, heat load on
x < 0.1) from u = 0 until ||J u - b|| / ||b|| < 1e-8, including the nodal load
assembly from element loads already resident in HBM.  Hierarchy set-up is timed
separately.  Every vector (537 MB in FP64) is larger than L2, so no flush is needed.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
    python bench.py --impl reference ...   # the FP64 CPU oracle on the host cores

Under torchrun every rank solves its own copy (replicas, weak scaling) and rank 0
prints one JSON line.  The roofline object is measured live on the dominant kernel.

Besides the headline solve the line carries (one GPU): `variant` -- the same grid with
k_ins = 1e-6 in the mixed scheme, with its error against the oracle's exact solution;
`variant_same_field` -- the headline field in the mixed scheme; `other_configs` -- the
128 x 128 two-phase rod (to 1e-10 in FP64, and to 1e-8 in both precisions) and one
gradient step of the 1024 x 4096 differentiation workload through torch.autograd;
`serving` -- the 512-request trace; `cpu_baseline` -- the oracle on the host cores.
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
sys.path.insert(0, ROOT)

METRIC = "space-time DOF/s solved to 1e-8 rel. residual (HBM GB/s %); serving p50/p99"
TOL = 1e-8
NOMINAL_FP64_TFLOPS = 1.25  # GB300 FP64 (vector and tensor), nominal


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    p.add_argument("--workload", default="filtered_simp", choices=sorted(WORKLOADS),
                   help="rod_blocks (128 x 128 two-phase blocks), filtered_simp (4096 x 16384, k_ins 1e-4), "
                        "filtered_simp_high_contrast (same grid, k_ins 1e-6), random_design (1024 x 4096, nu 20)")
    p.add_argument("--grid", default="", help="NxNT: the workload's recipe on another grid (not rod_blocks), "
                                                "e.g. a case small enough for a multi-pass ncu capture")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-variant", action="store_true", help="skip the other-precision solve of the same workload")
    p.add_argument("--mixed-inner", type=int, default=4, help="FP32 V-cycles per FP64 defect in the mixed scheme")
    p.add_argument("--mixed-first", type=int, default=4, help="FP32 V-cycles on the first defect in the mixed scheme")
    p.add_argument("--max-coarse-dofs", type=int, default=0, help="planner: stop at a level this small (0: default)")
    p.add_argument("--serving-requests", type=int, default=512,
                   help="requests of the 512-request serving trace to replay (0: skip serving)")
    p.add_argument("--no-all-cores", action="store_true", help="skip the all-cores oracle timing")
    p.add_argument("--no-other-configs", action="store_true",
                   help="skip the 128 x 128 rod and the differentiation workload legs")
    p.add_argument("--serving-workers", type=int, default=6)
    return p.parse_args()


WORKLOADS = ("rod_blocks", "filtered_simp", "filtered_simp_high_contrast", "random_design")


def load_workload(name, grid=""):
    from paper_2505_10168_gb300 import workloads as wl

    if grid:
        n, nt = (int(v) for v in grid.lower().split("x"))
        w = getattr(wl, name)(N=n, NT=nt)
    else:
        w = getattr(wl, name)()
    w["fn"] = name
    return w


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_id), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


class BusySampler(ClockSampler):
    """nvidia-smi utilization.gpu (the share of each sample period in which a kernel ran)."""

    Q = "utilization.gpu"

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        vals = []
        for ln in self.lines:
            try:
                vals.append(float(ln.split(",")[0]))
            except ValueError:
                continue
        if not vals:
            return None
        return {"median_pct": statistics.median(vals), "mean_pct": sum(vals) / len(vals), "samples": len(vals),
                "what": "nvidia-smi utilization.gpu every 100 ms over the closed-loop replay: the share of "
                        "time in which at least one kernel ran (not how many SMs it used)"}


def gpu_smi_id(dev):
    import torch

    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return 0


# ----------------------------------------------------------------------------- CPU oracle
def oracle_sample(w, nt_sample, tol=TOL):
    """Oracle STMG solve of the first nt_sample time steps of the workload (same dx, dt,
    material and load), timed on one host core."""
    import oracle

    N = w["N"]
    if w["k"] is None:
        k, c = oracle.simp(w["chi"], w["simp"])
    else:
        k, c = w["k"], w["c"]
    tT = w["tT"] * nt_sample / w["NT"]
    q = np.ascontiguousarray(w["q"][: nt_sample + 1])
    t0 = time.perf_counter()
    H = oracle.Hierarchy(N, nt_sample, w["L"], tT, k, c, nu=w.get("nu", 5))
    b = oracle.assemble_load(N, nt_sample, w["L"] / N, q)
    u, st, cyc, hist = H.solve(b, tol=tol)
    dt = time.perf_counter() - t0
    dofs = (N + 1) * (nt_sample + 1)
    return dict(value=dofs / dt, seconds=dt, dofs=dofs, cycles=cyc, status=st, relres=float(hist[-1]))


def _oracle_sample_task(args):
    """One oracle sample in a worker process (spawned: the parent holds a CUDA context)."""
    import importlib

    name, nt_sample = args
    sys.path.insert(0, ROOT)
    w = importlib.import_module("paper_2505_10168_gb300.workloads")
    return oracle_sample(getattr(w, name)(), nt_sample)


def cpu_model():
    """The host CPU's model name and core count (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model Name"):
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith("model name"):
                        model = ln.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    return {"model": model, "nproc": os.cpu_count()}


def oracle_all_cores(wname, nt_sample, procs=None):
    """The same oracle sample solved by one process per host core at once (the oracle is
    serial C; the cores work on independent copies): aggregate DOF/s = procs x DOFs / wall."""
    import multiprocessing as mp

    procs = procs or os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_sample_task, [(wname, 16)] * procs)  # start-up and imports, untimed
        t0 = time.perf_counter()
        res = pool.map(_oracle_sample_task, [(wname, nt_sample)] * procs)
        wall = time.perf_counter() - t0
    dofs = sum(r["dofs"] for r in res)
    return {"value": dofs / wall, "unit": "DOF/s", "cores": procs, "seconds": wall,
            "what": "%d concurrent oracle STMG processes, each solving the same %d-step sample" % (procs, nt_sample)}


def oracle_time_stepping(w):
    """Exact sequential implicit time stepping (the oracle's direct solver) on the full grid."""
    import oracle

    N, NT = w["N"], w["NT"]
    if w["k"] is None:
        k, c = oracle.simp(w["chi"], w["simp"])
    else:
        k, c = w["k"], w["c"]
    t0 = time.perf_counter()
    b = oracle.assemble_load(N, NT, w["L"] / N, w["q"])
    u = oracle.exact(N, NT, w["L"], w["tT"], k, c, b)
    dt = time.perf_counter() - t0
    return dict(value=(N + 1) * (NT + 1) / dt, seconds=dt, u=u)


def accuracy_against_exact(w, solutions):
    """max |u - u_exact| / max |u_exact| of each host solution of workload w against the
    oracle's exact time stepping on the full grid."""
    ts = oracle_time_stepping(w)
    ue = ts["u"]
    scale = float(np.abs(ue).max())
    acc = {name: float(np.abs(v - ue).max() / scale) for name, v in solutions.items()}
    acc["what"] = "max |u - u_exact| / max |u_exact| against the oracle's exact time stepping on the full grid"
    return acc, ts


def cpu_baseline_obj(w, nt_sample=256, solutions=None, all_cores=True):
    """The timed oracle legs; `solutions` (name -> host solution of the full workload) are
    compared with the oracle's exact solution, which the time-stepping leg produces."""
    nt_sample = min(nt_sample, w["NT"])
    s = oracle_sample(w, nt_sample)
    acc, ts = accuracy_against_exact(w, solutions or {})
    out = {"value": s["value"], "unit": "DOF/s", "cores": 1, "kind": "oracle",
           "sample": "oracle STMG (FP64 C, Alg. 1 with the same options) solving the first %d of %d time steps "
                     "of the workload (%d DOFs, same dx, dt, material and load) to %.0e: %d cycles in %.1f s"
                     % (nt_sample, w["NT"], s["dofs"], TOL, s["cycles"], s["seconds"]),
           "host": cpu_model(),
           "time_stepping": {"value": ts["value"], "unit": "DOF/s", "seconds": ts["seconds"],
                             "what": "oracle exact sequential time stepping (Thomas per step) on the full grid"},
           "accuracy": acc if solutions else None}
    if all_cores:
        try:
            out["all_cores"] = oracle_all_cores(w["fn"], nt_sample)
        except Exception as ex:  # report, do not hide
            out["all_cores"] = {"error": repr(ex)}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = load_workload(args.workload, args.grid)
    nt_sample = min(128, w["NT"])
    for _ in range(args.warmup):
        oracle_sample(w, nt_sample)
    vals, secs = [], []
    for _ in range(args.steps):
        s = oracle_sample(w, nt_sample)
        vals.append(s["value"])
        secs.append(s["seconds"])
    tot = sum(secs)
    dofs = (w["N"] + 1) * (nt_sample + 1)
    value = dofs * args.steps / tot
    sample = ("oracle STMG (FP64 C, one core) solving the first %d of %d time steps of %s to %.0e per step"
              % (nt_sample, w["NT"], w["name"], TOL))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "N": w["N"], "NT": w["NT"], "dofs": (w["N"] + 1) * (w["NT"] + 1),
                   "precision": "fp64", "tol": TOL, "sample": "first %d time steps per step" % nt_sample},
        "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ----------------------------------------------------------------------------- ranks
def max_over_ranks(x, world, device="cpu"):
    """The slowest rank's value (every rank gets it); identity on one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Aggregate throughput of independent replicas: every rank's units / the slowest rank's time."""
    return world * units_per_rank / seconds


# ----------------------------------------------------------------------------- serving
def precision_opts(args, precision):
    """Solver options that only the mixed scheme takes."""
    if precision != "mixed":
        return {}
    return {"mixed_inner_cycles": args.mixed_inner, "mixed_first_cycles": args.mixed_first}


def workload_opts(w, args=None):
    """Solver options the workload fixes (nu = 20 for the rough differentiation field), and
    the planner's coarsest-level size when given on the command line."""
    o = {"nu": w["nu"]} if "nu" in w else {}
    if args is not None and args.max_coarse_dofs > 0:
        o["max_coarse_dofs"] = args.max_coarse_dofs
    return o


# the serving trace's solver options; 3 FP32 cycles per FP64 defect measured best at nu = 60
SERVING_OPTS = dict(precision="mixed", tol=TOL, nu=60, max_cycles=300, mixed_first_cycles=3, mixed_inner_cycles=3)
SERVING_MAX_NU = 240  # a request that does not converge is solved again with 2x the sweeps, up to this


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture
# of the kernel on the named workload; a kernel changed since its capture has no entry.
NCU_TRAFFIC = {
    ("4096x16384", "k_sweep<double>"): 1.590e9,
    ("4096x16384", "k_defect (FP64, finest level)"): 1.3325e9,
    ("4096x16384", "k_stream UP + FP64 accumulate (finest level)"): 1.7477e9,
    ("4096x16384", "k_stream DOWN from zero (finest level)"): 0.6297e9,
    # captured on 2048 x 16384 (466.8 MB for 33.57 M DOFs) and scaled by the DOFs
    ("4096x16384", "k_stream UP into the FP32 iterate (finest level)"): 0.9335e9,
}


def mixed_rooflines(solver, stream, wname, dofs, nu, reps=20):
    """The mixed scheme's heaviest steps, each launched alone `reps` times on the solver's
    stream (after its timed solves) and timed with CUDA events there: the FP64 defect (6 FP64
    FMA, 20 B per DOF), the finest level's UP pass that adds into the FP64 iterate (26 B per
    DOF), its UP pass into the FP32 iterate (read u, b', z, write u: 14 B per DOF; the inner
    cycles' form) and its DOWN pass from zero (10 B per DOF).  Shares of the solve come from
    the launch list, not from here."""
    import torch

    if nu > 5:
        return [{"skipped": "nu > 5: each half of a level is several passes"}]
    hbm = measured_peaks().get("hbm_gbs", 6788.3)
    out = []
    for kind, name, nbytes, flops in (("defect", "k_defect (FP64, finest level)", 20.0, 12.0),
                                      ("up", "k_stream UP + FP64 accumulate (finest level)", 26.0, None),
                                      ("up32", "k_stream UP into the FP32 iterate (finest level)", 14.0, None),
                                      ("down", "k_stream DOWN from zero (finest level)", 10.0, None)):
        # an NVTX range per step, so that a profiler can select these launches alone
        torch.cuda.nvtx.range_push("roofline_" + kind)
        solver.mixed_pass(0, kind)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            solver.mixed_pass(0, kind)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        ms = e0.elapsed_time(e1) / reps
        gbs = nbytes * dofs / (ms * 1e-3) / 1e9
        if flops is None:
            r = {"kernel": name, "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm}
        else:
            tf = flops * dofs / (ms * 1e-3) / 1e12
            r = {"kernel": name, "bound": "alu", "achieved": tf, "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
                 "frac": tf / NOMINAL_FP64_TFLOPS, "hbm_gbs": gbs, "hbm_frac_of_measured": gbs / hbm}
        r.update({"traffic": NCU_TRAFFIC.get((wname, name)), "ms_per_launch": ms, "algorithmic_bytes_per_dof": nbytes,
                  "peak_source": "measured HBM copy" if flops is None else "nominal GB300 FP64"})
        out.append(r)
    return out


def run_serving(nreq, workers, compare=8, gpu_id=None):
    """Closed loop (all requests queued at once) for throughput, then the same requests
    with their Poisson gaps rescaled to 0.5x, 0.8x and 1.0x that throughput for latency
    (0.8x is the headline p50/p99)."""
    from paper_2505_10168_gb300 import serving as sv
    from paper_2505_10168_gb300 import workloads as wl

    reqs = wl.serving_requests()[:nreq]
    fields = lambda r: wl.request_fields(r)[:2]  # noqa: E731
    opts = dict(SERVING_OPTS)
    with sv.Server(workers=workers, max_nu=SERVING_MAX_NU) as srv:
        sv.replay(srv, reqs[: min(4, nreq)], fields, speed=1e9, **opts)  # warm-up
        busy = BusySampler(gpu_id) if gpu_id is not None else None
        if busy:
            busy.start()
        _, closed = sv.replay(srv, reqs, fields, speed=1e9, **opts)
        if busy:
            closed["gpu_busy"] = busy.stop()
        rate = closed["requests"] / closed["makespan_s"]  # requests per second
        mean_gap = (reqs[-1]["arrival"] - reqs[0]["arrival"]) / max(1, len(reqs) - 1)
        loads = {}
        for load in (0.5, 0.8, 1.0):  # Poisson arrivals at this fraction of that rate
            _, loads[load] = sv.replay(srv, reqs, fields, speed=load * rate * mean_gap, **opts)
        poisson = loads[0.8]
        # the same first requests, mixed and batched, against the plain FP64 single-solve
        # form: FP64 V-cycles, one request at a time (one worker), same tolerance and cap
        sub = reqs[: min(compare, nreq)]
        _, batched = sv.replay(srv, sub, fields, speed=1e9, **opts)
    fp64_opts = dict(opts, precision="fp64")
    fp64_opts.pop("mixed_inner_cycles")
    fp64_opts.pop("mixed_first_cycles")
    with sv.Server(workers=1, max_nu=SERVING_MAX_NU) as one:
        _, single = sv.replay(one, sub, fields, speed=1e9, **fp64_opts)
    vs = {"requests": len(sub), "mixed_batched": batched, "fp64_single": single,
          "speedup": batched["dofs_per_s"] / single["dofs_per_s"] if single["dofs_per_s"] > 0 else None}
    return {"requests": nreq, "of": 512, "workers": workers, "solver": opts, "max_nu": SERVING_MAX_NU,
            "closed_loop": closed, "poisson_0.8": poisson,
            "p50_p99_by_load": {str(l): [v["p50_s"], v["p99_s"]] for l, v in loads.items()},
            "p50_s": poisson["p50_s"], "p99_s": poisson["p99_s"], "dofs_per_s": closed["dofs_per_s"],
            "vs_fp64_single": vs}


# ----------------------------------------------------------------------------- other configs
def cuda_time(stream, fn, reps):
    """Average ms of fn() over reps calls, CUDA events on the stream (after one warm-up)."""
    import torch

    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = [fn() for _ in range(reps)]
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out[-1]


def rod_blocks_leg(pkg, dev, stream, reps=10):
    """The 128 x 128 two-phase rod (k in {1e-3, 1}, uniform load), solved to relative residual
    1e-10 in FP64 as the workload states, and to 1e-8 (the metric) in both precisions;
    errors against the oracle's exact time stepping."""
    import torch

    import oracle

    w = load_workload("rod_blocks")
    N, NT, L, tT = w["N"], w["NT"], w["L"], w["tT"]
    dofs = (N + 1) * (NT + 1)
    q = torch.tensor(w["q"], device=dev)
    u = torch.empty((NT + 1, N + 1), dtype=torch.float64, device=dev)
    ue = oracle.exact(N, NT, L, tT, w["k"], w["c"], oracle.assemble_load(N, NT, L / N, w["q"]))
    out = {"workload": w["name"], "dofs": dofs, "solves": {}}
    for name, prec, tol in (("fp64_1e-10", "fp64", 1e-10), ("fp64", "fp64", TOL), ("mixed", "mixed", TOL)):
        s = pkg.Solver(N, NT, L, tT, w["k"], w["c"], precision=prec, tol=tol)
        ms, st = cuda_time(stream, lambda: s.solve(u, q=q), reps)
        err = float(np.abs(u.cpu().numpy() - ue).max() / np.abs(ue).max())
        out["solves"][name] = {"precision": prec, "tol": tol, "value": dofs / (ms * 1e-3), "unit": "DOF/s",
                               "ms_per_solve": ms, "cycles": st[1], "relres": st[2], "converged": st[0] == "ok",
                               "error_vs_exact": err}
        s.close()
    return out


def differentiation_leg(pkg, dev, stream, reps=3):
    """The differentiation workload (1024 x 4096, densities U(0.05, 1), SIMP p = 3,
    k_min = 1e-3, nu = 20): one gradient step through torch.autograd -- SIMP material, forward
    STMG solve, compliance Theta = sum_n b_n^T u_n dt, adjoint STMG solve and the fused
    sensitivity -- to relative residual 1e-8 in each precision, against the oracle's gradient
    from exact time stepping (the central-difference check is in the tests)."""
    import torch

    import oracle
    from paper_2505_10168_gb300 import autograd as ag

    w = load_workload("random_design")
    N, NT, L, tT, s6 = w["N"], w["NT"], w["L"], w["tT"], w["simp"]
    dofs = (N + 1) * (NT + 1)
    q = torch.tensor(w["q"], device=dev)
    ko, co = oracle.simp(w["chi"], s6)
    bo = oracle.assemble_load(N, NT, L / N, w["q"])
    uo = oracle.exact(N, NT, L, tT, ko, co, bo)
    lo = oracle.exact(N, NT, L, tT, ko, co, bo * (tT / NT), adj=True)
    go = oracle.sensitivity(N, NT, L, tT, w["chi"], s6, uo, lo)
    out = {"workload": w["name"], "dofs": dofs, "nu": w["nu"], "tol": TOL, "steps": {}}
    for prec in ("fp64", "mixed"):
        solver = pkg.Solver(N, NT, L, tT, ko, co, precision=prec, tol=TOL, nu=w["nu"], max_cycles=300)
        b = torch.empty((NT + 1, N + 1), dtype=torch.float64, device=dev)
        solver.assemble_load(q, b)

        def step():
            chi = torch.tensor(w["chi"], device=dev).requires_grad_(True)
            u = ag.solve(chi, q, solver, s6)
            theta = ag.compliance(u, b, solver)
            theta.backward()
            return chi.grad

        ms, g = cuda_time(stream, step, reps)
        gerr = float(np.abs(g.cpu().numpy() - go).max() / np.abs(go).max())
        out["steps"][prec] = {"value": 2 * dofs / (ms * 1e-3), "unit": "DOF/s (forward + adjoint)",
                              "ms_per_gradient": ms, "gradient_error_vs_oracle": gerr}
        if prec == "fp64":
            # the sequential-in-time competitor on the same grid: exact time stepping of the
            # forward problem on the GPU (one block, a block-scan Thomas solve per step)
            row0 = torch.zeros((1, N + 1), dtype=torch.float64, device=dev)
            ut = torch.empty_like(b)
            ts_ms, _ = cuda_time(stream, lambda: solver.recompute_slabs(b, row0, NT, ut), reps)
            out["gpu_time_stepping"] = {"value": dofs / (ts_ms * 1e-3), "unit": "DOF/s", "ms_per_solve": ts_ms,
                                        "what": "exact forward solve by sequential time stepping on the GPU"}
        solver.close()
    return out


# ----------------------------------------------------------------------------- GPU arm
def timed_variant(pkg, w, k, c, q, u, precision, args, stream, world, rooflines=False):
    """Solves of workload w (material k, c and element loads q on the device) in the given
    precision, timed with CUDA events like the main leg; returns the record and the last
    solution on the host."""
    import torch

    N, NT, L, tT = w["N"], w["NT"], w["L"], w["tT"]
    dofs = (N + 1) * (NT + 1)
    s2 = pkg.Solver(N, NT, L, tT, k, c, precision=precision, tol=TOL, **precision_opts(args, precision),
                    **workload_opts(w, args))
    for _ in range(max(1, args.warmup)):
        s2.solve(u, q=q)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    st2 = [s2.solve(u, q=q) for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms2 = e0.elapsed_time(e1) / args.steps
    rec = {"config": {"workload": w["name"], "N": N, "NT": NT, "dofs": dofs, "precision": precision,
                      "k_ins": float(w["simp"][0]) if w.get("simp") is not None else None, "tol": TOL},
           "precision": precision, "value": world * dofs / (ms2 * 1e-3), "unit": "DOF/s", "ms_per_step": ms2,
           "cycles": st2[-1][1], "relres": st2[-1][2], "levels": s2.num_levels,
           "fine_sweep_dofs_per_s": world * dofs * st2[-1][1] * 2 * s2.opts.nu / (ms2 * 1e-3),
           "converged": all(x[0] == "ok" and x[2] < TOL for x in st2),
           "dtype": "f64" if precision == "fp64" else "f32+f64", **precision_opts(args, precision)}
    if precision == "mixed" and rooflines:
        rec["rooflines"] = mixed_rooflines(s2, stream, "%dx%d" % (N, NT), dofs, w.get("nu", 5))
    s2.close()
    return rec, u.cpu().numpy()


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    import paper_2505_10168_gb300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl")

    def barrier():
        if world > 1:
            dist.barrier()

    w = load_workload(args.workload, args.grid)
    N, NT, L, tT = w["N"], w["NT"], w["L"], w["tT"]
    dofs = (N + 1) * (NT + 1)
    stream = torch.cuda.current_stream(dev)
    if w["k"] is None:
        chi = torch.tensor(w["chi"], device=dev)
        k = torch.empty(N, dtype=torch.float64, device=dev)
        c = torch.empty_like(k)
        pkg.simp(chi, w["simp"], k, c)
    else:
        k = torch.tensor(w["k"], device=dev)
        c = torch.tensor(w["c"], device=dev)
    q = torch.tensor(w["q"], device=dev)
    u = torch.empty((NT + 1, N + 1), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    solver = pkg.Solver(N, NT, L, tT, k, c, precision=args.precision, tol=TOL, **precision_opts(args, args.precision),
                        **workload_opts(w, args))
    setup_ms = 1e3 * (time.perf_counter() - t0)
    levels, path = solver.num_levels, solver.path()

    for _ in range(args.warmup):
        st, cyc, rr = solver.solve(u, q=q)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(gpu_smi_id(dev))
    clk.start()
    time.sleep(0.3)
    l0 = pkg.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    statuses = []
    for _ in range(args.steps):
        statuses.append(solver.solve(u, q=q))
    ev1.record(stream)
    torch.cuda.synchronize()
    launches = pkg.kernel_launches() - l0
    clocks = clk.stop()
    barrier()
    ms = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    ms_per_step = ms / args.steps
    value = whole_job_rate(dofs * args.steps, world, ms * 1e-3)
    cycles = statuses[-1][1]
    fine_sweeps = world * dofs * cycles * 2 * solver.opts.nu / (ms_per_step * 1e-3)
    relres = statuses[-1][2]
    ok = all(s[0] == "ok" and s[2] < TOL for s in statuses)
    check = rank == 0 and world == 1 and not args.no_cpu_baseline
    solutions = {args.precision: u.cpu().numpy()} if check else {}

    # ---- end to end through the C ABI with host buffers (right after the timed region) ----
    e2e = None
    if not args.no_e2e:
        qh = torch.tensor(w["q"]).pin_memory()
        uh = torch.empty((NT + 1, N + 1), dtype=torch.float64).pin_memory()
        solver.solve(uh, q=qh)
        torch.cuda.synchronize()
        barrier()
        ksteps = max(1, min(args.steps, 5))
        each = []
        t1 = time.perf_counter()
        for _ in range(ksteps):
            ta = time.perf_counter()
            solver.solve(uh, q=qh)  # returns once u is in host memory
            each.append(1e3 * (time.perf_counter() - ta))
        torch.cuda.synchronize()
        el = max_over_ranks(time.perf_counter() - t1, world, dev)
        e2e = {"value": whole_job_rate(dofs * ksteps, world, el), "unit": "DOF/s", "h2d_bytes_per_step": int(qh.numel() * 8),
               "d2h_bytes_per_step": int(uh.numel() * 8 + 8 * (cycles + 2)), "steps": ksteps,
               "ms_per_step_each": each}
        del qh, uh

    # ---- dominant kernel: FP64 Jacobi sweep on the finest level, timed live ----
    roofline = None
    try:
        b = torch.empty_like(u)
        solver.assemble_load(q, b)
        uu = torch.zeros_like(u)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        solver.smooth(0, uu, b, 0)
        nsw = 20
        torch.cuda.nvtx.range_push("roofline_sweep")  # lets a profiler select these launches
        e[0].record(stream)
        solver.smooth(0, uu, b, 0)
        e[1].record(stream)
        e[2].record(stream)
        solver.smooth(0, uu, b, nsw)
        e[3].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        sweep_ms = (e[2].elapsed_time(e[3]) - e[0].elapsed_time(e[1])) / nsw
        flops = 12.0 * dofs  # 6 FMA per DOF: u <- (1 - w) u + b' + sum of 5 scaled neighbours
        bytes_alg = 24.0 * dofs  # read u, b; write u (FP64)
        ach = flops / (sweep_ms * 1e-3) / 1e12
        roofline = {"kernel": "k_sweep<double> (finest level)", "bound": "alu", "achieved": ach,
                    "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s", "frac": ach / NOMINAL_FP64_TFLOPS,
                    "traffic": NCU_TRAFFIC.get(("%dx%d" % (N, NT), "k_sweep<double>")), "ms_per_launch": sweep_ms,
                    "hbm_gbs": bytes_alg / (sweep_ms * 1e-3) / 1e9,
                    "hbm_frac_of_measured": bytes_alg / (sweep_ms * 1e-3) / 1e9 /
                    measured_peaks().get("hbm_gbs", 6788.3),
                    "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (FP64 FMA throughput measured 1.20)"}
        del b, uu
    except Exception as ex:  # report, do not hide
        roofline = {"error": repr(ex)}

    # ---- GPU competitor: exact sequential time stepping (one block, all NT steps) ----
    gpu_ts = None
    try:
        b = torch.empty_like(u)
        solver.assemble_load(q, b)
        row0 = torch.zeros((1, N + 1), dtype=torch.float64, device=dev)  # T = 0 at t = 0
        ut = torch.empty_like(u)
        solver.recompute_slabs(b, row0, NT, ut)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.recompute_slabs(b, row0, NT, ut)
        e1.record(stream)
        torch.cuda.synchronize()
        ts_ms = e0.elapsed_time(e1)
        gpu_ts = {"value": dofs / (ts_ms * 1e-3), "unit": "DOF/s", "ms_per_solve": ts_ms,
                  "what": "exact solution by sequential implicit time stepping on the GPU: one block, one "
                          "block-scan Thomas solve per time step (not STMG; the sequential-in-time competitor)"}
        del b, ut
    except Exception as ex:
        gpu_ts = {"error": repr(ex)}

    # ---- the other precision on the same workload, and the k_ins = 1e-6 field of the same
    # grid in the mixed scheme (same metric, same tolerance) ----
    variant, variant_same_field = None, None
    if not args.no_variant:
        other = "mixed" if args.precision == "fp64" else "fp64"
        variant_same_field, u2 = timed_variant(pkg, w, k, c, q, u, other, args, stream, world,
                                               rooflines=args.workload != "filtered_simp")
        if check:
            solutions[other] = u2
        if args.precision == "fp64" and args.workload == "filtered_simp":
            w3 = load_workload("filtered_simp_high_contrast", args.grid)
            chi3 = torch.tensor(w3["chi"], device=dev)
            k3, c3 = torch.empty_like(k), torch.empty_like(c)
            pkg.simp(chi3, w3["simp"], k3, c3)
            q3 = torch.tensor(w3["q"], device=dev)
            variant, u3 = timed_variant(pkg, w3, k3, c3, q3, u, "mixed", args, stream, world, rooflines=True)
            if check:
                variant["accuracy"], _ = accuracy_against_exact(w3, {"mixed": u3})
            del chi3, k3, c3, q3, u3
        else:
            variant, variant_same_field = variant_same_field, None
        del u2

    # ---- the other workloads: the 128 x 128 rod and the differentiation step ----
    other_configs = None
    if not args.no_other_configs and world == 1 and not args.grid:
        other_configs = {}
        for name, fn in (("rod_blocks", rod_blocks_leg), ("differentiation", differentiation_leg)):
            try:
                other_configs[name] = fn(pkg, dev, stream)
            except Exception as ex:  # report, do not hide
                other_configs[name] = {"error": repr(ex)}

    # ---- serving: continuous batching of the uneven forward/adjoint request trace ----
    serving = None
    if args.serving_requests > 0 and world == 1:  # one GPU's server; replicas under torchrun skip it
        del u, q
        solver.close()
        torch.cuda.empty_cache()
        serving = run_serving(args.serving_requests, args.serving_workers, gpu_id=gpu_smi_id(dev))

    cpu = None
    if check:
        cpu = cpu_baseline_obj(w, solutions=solutions, all_cores=not args.no_all_cores)
        del solutions

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": w["name"], "N": N, "NT": NT, "dofs": dofs, "precision": args.precision, **precision_opts(args, args.precision), **workload_opts(w, args),
                       "tol": TOL, "levels": levels, "path": path, "cycles": cycles,
                       "relres": relres, "converged": ok, "setup_ms": setup_ms,
                       "l2": "no flush: every vector (%d MB) exceeds the 129 MB L2" % (dofs * 8 // 2 ** 20),
                       "parallelism": "replicas" if world > 1 else "single"},
            "fine_sweep_dofs_per_s": fine_sweeps,
            "clocks": clocks, "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline,
            "cpu_baseline": cpu, "variant": variant, "variant_same_field": variant_same_field,
            "other_configs": other_configs,
            "gpu_time_stepping": gpu_ts, "serving": serving,
            "accuracy": cpu.pop("accuracy", None) if cpu else None,
        }
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
