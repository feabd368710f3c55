#!/usr/bin/env python
"""Benchmark of the FAS multigrid hot path on GB300.

Workload (one "step"): 2D backward-Euler heat on an 8192^2 cell-centred grid of [0,1]^2, Neumann
boundaries, kappa 1, dt 1e-4, 20 time steps from u0 = cos(pi x) cos(pi y) + 1e-2 U(-1,1) noise with a
source of 16 Gaussians (sigma 0.02), every time step solved to 1e-10 relative residual by V(2,2)
FAS cycles with X-MCGS smoothing (coarsest 4x4). Inputs are seeded synthetic fields (workloads/).

Metric: Mcells*V-cycles/s = fine cells x fine-grid V-cycles done / seconds / 1e6 for the whole
20-step run, mixed precision (float32 cycles inside float64 iterative refinement). The plain float64
solve of the same run is measured beside it, with its time-to-solution ratio.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the workload (the solver has no
cross-GPU step); value = cells x cycles summed over ranks / the slowest rank's time.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mcells*V-cycles/s to 1e-10 rel. residual (2D heat 8192^2, mixed precision)"
UNIT = "Mcells*V-cycles/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", "--grid", dest="n", type=int, default=8192,
                    help="cells per axis (--grid: the same, unambiguous behind torch.distributed.run)")
    ap.add_argument("--heat-steps", type=int, default=20)
    ap.add_argument("--inner", type=int, default=0, help="float32 cycles per refinement step (0: tune)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--no-fp64", action="store_true", help="skip the float64 comparison arm")
    ap.add_argument("--case", default="heat2d", choices=["heat2d", "heat3d", "ns"],
                    help="heat2d: the benchmark line; heat3d / ns: one small timed case of the 3D heat or the "
                         "cavity workload (for kernel profiles), printed as its own JSON line")
    ap.add_argument("--shape", default="256,512,512", help="--case heat3d: nz,ny,nx (planes of the 512^3 recipe)")
    ap.add_argument("--ns-n", type=int, default=128, help="--case ns: cells per axis of the 3D cavity")
    ap.add_argument("--ns-order", type=int, default=1, help="--case ns: projection scheme order")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch every kernel from the host instead of one CUDA graph per solve (the same "
                         "kernels; ncu cannot list kernel nodes of graphs with conditional nodes)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the other workloads (3D heat, NS cavity, batched solves, adjoint)")
    return ap.parse_args()


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                    power.append(float(parts[3]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        finally:
            os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


def traffic_table():
    """DRAM bytes per cell from the committed ncu summaries, valid only while the kernel sources are
    unchanged (profiles/traffic.json)."""
    import hashlib
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    except (OSError, ValueError):
        return {}
    out = {}
    for key, v in t.items():
        if not isinstance(v, dict):
            continue
        m = hashlib.sha256()
        try:
            for f in v["sources"]:
                m.update(open(os.path.join(ROOT, f), "rb").read())
        except OSError:
            continue
        if m.hexdigest()[:16] == v["hash"]:
            out[key] = v["bytes_per_cell"]
    return out


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------------------------------------
# algorithmic work per cell of each kernel family (bytes or float64 operations)
# ---------------------------------------------------------------------------------------------

def kernel_work(family, level, inner=1):
    """(bound, per-cell work, unit) of a kernel family on a level of the mixed-precision solver.
    Bytes that must cross HBM once (b = 4 for float32 fields, 8 for float64). inner = float32 cycles
    per refinement step: the first level-0 pre-smoothing of a step starts from zero (no u read), the
    others read u, so the family's per-launch bytes are their average."""
    b = 4.0
    if family == "smooth":  # fused pre-smoothing: f (+u, +R(r)) in, u and R(u), R(r) out
        if level == 0:
            return "hbm", (2.5 + 3.5 * (inner - 1)) / inner * b, "B"
        return "hbm", 4.5 * b, "B"
    if family == "prolong":  # fused post-smoothing: u, f, u_c in; u out
        return "hbm", 3.25 * b, "B"
    if family == "ir":  # r32 = (float)(b - A u): u, b in (float64), r32 out; the exact-difference kernel
        return "hbm", 8.0 + 8.0 + b, "B"  # also has a float64 floor of 2 DFMA per cell (fp64_work)
    if family == "update":  # fused post-smoothing + u += e: u, f, u_c in (float32), float64 u in/out
        return "hbm", 2.25 * b + 16.0, "B"
    return None, None, None


def fp64_work(family):
    """float64 FLOPs per cell (an FMA counts two) that a kernel family must execute on the FP64 pipe,
    or None: the refinement residual finishes r = fma(c, S, fma(-alpha, u, b)) with 2 DFMA per cell;
    the fused float64 update adds u += e with 1 DADD per cell."""
    return {"ir": 4.0, "update": 1.0}.get(family)


def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_2510_11152_gb300 as fas
    from workloads import heat2d_large

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fas.load()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(x):
        from paper_2510_11152_gb300.shard import max_over_ranks as mor
        return mor(x, ws, dev)

    n = args.n
    w = heat2d_large(n=n, nsteps=args.heat_steps)
    shape, h, dt, nsteps = w["shape"], w["h"], w["dt"], w["nsteps"]
    cells = n * n
    u0_d = torch.from_numpy(w["u0"]).to(dev)
    f_d = torch.from_numpy(w["fsrc"]).to(dev)
    u_d = torch.empty_like(u0_d)
    stream = torch.cuda.current_stream(dev)

    def make(precision, inner=1):
        return fas.fas_create(fas.make_params(shape, h, alpha=1.0, beta=dt, coarsest=4, precision=precision,
                                              inner_cycles=inner, use_graph=0 if args.no_graph else 1),
                              stream=stream)

    def one_run(ctx, inner):
        u_d.copy_(u0_d)
        infos = fas.fas_heat_run(ctx, u_d, f_d, dt, nsteps)
        return sum(i.cycles for i in infos) * inner, infos

    # tune the float32 cycles per refinement step on one run each (time to solution decides)
    inners = [args.inner] if args.inner > 0 else [1, 2, 3]
    best = None
    for inner in inners:
        ctx = make(fas.FAS_MIXED, inner)
        one_run(ctx, inner)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        one_run(ctx, inner)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        if best is None or t < best[0]:
            best = (t, inner, ctx)
        else:
            fas.fas_destroy(ctx)
    _, inner, ctx = best

    def timed(ctx, inner, steps, warmup):
        for _ in range(warmup):
            one_run(ctx, inner)
        barrier()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        fas.fas_launch_count(ctx, reset=True)
        cycles, infos_all = 0, []
        ev0.record(stream)
        for _ in range(steps):
            c, infos = one_run(ctx, inner)
            cycles += c
            infos_all.append(infos)
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = ev0.elapsed_time(ev1)
        return ms, cycles, fas.fas_launch_count(ctx), infos_all

    clocks = Clocks(local)
    clocks.start()
    ms, cycles, launches, infos_all = timed(ctx, inner, args.steps, args.warmup)
    clk = clocks.stop()
    ms_max = max_over_ranks(ms)
    value = ws * cells * cycles / (ms_max / 1e3) / 1e6
    last = infos_all[-1]
    converged = all(i.converged for infos in infos_all for i in infos)
    u_final = u_d.clone()

    # float64 arm
    fp64 = None
    if not args.no_fp64:
        ctx64 = make(fas.FAS_FP64)
        ms64, cyc64, _, inf64 = timed(ctx64, 1, max(1, args.steps), max(1, min(args.warmup, 3)))
        ms64 = max_over_ranks(ms64)
        u64 = u_d.clone()
        err = float((u_final - u64).abs().max().item() / u64.abs().max().item())
        fp64 = {"value": ws * cells * cyc64 / (ms64 / 1e3) / 1e6, "unit": UNIT,
                "ms_per_step": ms64 / max(1, args.steps),
                "vcycles_per_run": cyc64 / max(1, args.steps),
                "mixed_vs_fp64_rel_maxdiff": err,
                "speedup_mixed_vs_fp64_time": (ms64 / max(1, args.steps)) / (ms / args.steps)}
        fas.fas_destroy(ctx64)

    # kernel timings: one instrumented run, CUDA events on the solver's stream
    fas.fas_prof_enable(ctx, True)
    one_run(ctx, inner)
    recs = fas.fas_prof_read(ctx)
    fas.fas_prof_enable(ctx, False)
    total_ms = sum(r["ms"] for r in recs)
    dom = max(recs, key=lambda r: r["ms"])
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured (MEASURED_PEAKS.json hbm_gbs, copy bandwidth)" if "hbm_gbs" in peaks else "fallback"
    fp64_peak = fas.fas_probe_fp64_rate()  # TFLOP/s, measured on this device (independent DFMA chains)

    def roofline_of(r):
        """Both floors of a kernel family: HBM (algorithmic bytes) and, where it executes float64
        arithmetic, the FP64 pipe (algorithmic FLOPs); the binding one (the larger time floor) leads."""
        bound, work, unit = kernel_work(r["family"], r["level"], inner)
        if bound is None:
            return None
        per_launch_units = r["units"] / r["launches"]
        t = r["ms"] / r["launches"] / 1e3
        ach = work * per_launch_units / t / 1e9
        hbm = {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak,
               "peak_source": hbm_src, "algorithmic_bytes_per_cell": work}
        fw = fp64_work(r["family"])
        if fw is None:
            return dict(hbm, traffic=None)
        ach64 = fw * per_launch_units / t / 1e12
        f64 = {"bound": "alu", "achieved": ach64, "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach64 / fp64_peak,
               "peak_source": "measured on this GPU in this run (fas_probe_fp64_rate: DFMA chains, FMA = 2 FLOPs)",
               "pipe": "fp64", "algorithmic_flops_per_cell": fw}
        lead, other = (f64, hbm) if f64["frac"] > hbm["frac"] else (hbm, f64)
        out = dict(lead, traffic=None)
        out["hbm" if lead is f64 else "fp64"] = other
        return out

    roof = roofline_of(dom) or {"bound": "hbm", "achieved": None, "peak": hbm_peak, "unit": "GB/s",
                                "frac": None, "traffic": None}
    tt = traffic_table().get("%s@%d" % (dom["family"], dom["level"]))
    if tt is not None:
        roof["traffic"] = tt * dom["units"] / dom["launches"]
        roof["traffic_source"] = "ncu dram bytes per cell (profiles/traffic.json) x cells per launch"
    roof.update({"kernel": "%s@level%d" % (dom["family"], dom["level"]),
                 "share_of_kernel_time": dom["ms"] / total_ms if total_ms else None,
                 "ms_per_launch": dom["ms"] / dom["launches"]})
    kernels = sorted(({"kernel": "%s@L%d" % (r["family"], r["level"]), "launches": r["launches"],
                       "ms": round(r["ms"], 4), "share": round(r["ms"] / total_ms, 4)} for r in recs),
                     key=lambda d: -d["ms"])[:12]
    # X-MCGS sweeps on the finest level: sweep-equivalent bytes 3b per cell per sweep (u in/out, f in)
    xm = {}
    for fam, name in (("smooth", "pre"), ("prolong", "post"), ("update", "post_with_fp64_update")):
        r = [q for q in recs if q["family"] == fam and q["level"] == 0]
        if r:
            r = r[0]
            t = r["ms"] / r["launches"] / 1e3
            rf = roofline_of(r)
            hb = rf if rf["bound"] == "hbm" else rf["hbm"]
            xm[name] = {"ms_per_launch": r["ms"] / r["launches"],
                        "kernel_GBs": hb["achieved"], "kernel_frac": hb["frac"],
                        "algorithmic_bytes_per_cell": hb["algorithmic_bytes_per_cell"],
                        "traffic_bytes_per_cell": traffic_table().get("%s@0" % fam),
                        "sweep_equiv_GBs": 2 * 3 * 4 * cells / t / 1e9}

    # end to end through the host-buffer entry point (pinned host memory, copies inside the region)
    e2e = None
    try:
        u0_h = torch.from_numpy(w["u0"]).pin_memory()
        f_h = torch.from_numpy(w["fsrc"]).pin_memory()
        out_h = torch.empty_like(u0_h).pin_memory()
        a0, ah, fh = u0_h.numpy(), out_h.numpy(), f_h.numpy()
        fas.fas_heat_run_host(ctx, a0, ah, fh, dt, nsteps)
        barrier()
        t0 = time.perf_counter()
        cyc = 0
        for _ in range(args.steps):
            infos = fas.fas_heat_run_host(ctx, a0, ah, fh, dt, nsteps)
            cyc += sum(i.cycles for i in infos) * inner
        te = time.perf_counter() - t0
        te = max_over_ranks(te)
        e2e = {"value": ws * cells * cyc / te / 1e6, "unit": UNIT, "h2d_bytes_per_step": 2 * 8 * cells,
               "d2h_bytes_per_step": 8 * cells, "ms_per_step": te * 1e3 / args.steps,
               "matches_device_run": bool(np.array_equal(ah, u_final.cpu().numpy()))}
    except Exception as exc:  # pragma: no cover - reported, not hidden
        e2e = {"value": None, "unit": UNIT, "error": repr(exc)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(w)
        try:
            cpu["all_cores"] = cpu_baseline_all_cores()
        except Exception as exc:  # pragma: no cover - reported, not hidden
            cpu["all_cores"] = {"value": None, "error": repr(exc)}

    secondary = None
    if not args.no_secondary:
        del u0_d, f_d, u_d, u_final
        fas.fas_destroy(ctx)
        torch.cuda.empty_cache()
        secondary = secondary_workloads(dev, stream, ws, rank)

    if rank == 0 and secondary is not None:
        print(json.dumps({"kind": "secondary", "note": "other workloads of the method; the benchmark line follows",
                          "secondary": secondary}))
        sys.stdout.flush()
    if rank == 0:
        tts = {"mixed": ms_max / args.steps, "fp64": fp64["ms_per_step"] if fp64 else None}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "heat2d-8192x8192-neumann-dt1e-4-20steps-tol1e-10-V(2,2)-coarsest4",
                       "grid": [n, n], "time_steps_per_run": nsteps, "precision": "mixed",
                       "inner_float32_cycles": inner, "vcycles_per_run": cycles / args.steps,
                       "l2": "inputs larger than L2 (512 MiB per float64 field)",
                       "parallelism": "replicas" if ws > 1 else "single-gpu",
                       "launch": "host loop" if args.no_graph else "one CUDA graph per solve"},
            "converged_all": converged, "last_step_info": last[-1].as_dict(),
            "time_to_solution_ms": tts,
            "speedup_mixed_vs_fp64_time": fp64["speedup_mixed_vs_fp64_time"] if fp64 else None,
            "fp64": fp64, "roofline": roof, "xmcgs": xm, "kernels": kernels,
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "secondary": "printed on the line before this one" if secondary is not None else None,
        }
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _event_ms(stream, fn, warmup=1):
    """fn() after `warmup` untimed calls, timed with CUDA events on the solver's stream."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def tune_inner(stream, make, candidates=(1, 2, 3)):
    """The float32 cycles per refinement step with the shortest time to solution, the way the headline
    workload is tuned: make(inner) returns (run, cleanup); each candidate is run once untimed and once
    timed with CUDA events. Returns (inner, {inner: ms})."""
    times = {}
    for inner in candidates:
        run, cleanup = make(inner)
        ms, _ = _event_ms(stream, run)
        times[inner] = ms
        cleanup()
    best = min(times, key=times.get)
    return best, times


def secondary_workloads(dev, stream, ws=1, rank=0):
    """The other workloads of the method, each once after one warm-up run (float64 vs mixed where both
    apply; the mixed arm's float32 cycles per refinement step tuned by time to solution first, as for
    the headline workload): 3D heat 512^3, the 256^3 lid-driven cavity projection steps, 96 batched Helmholtz solves in
    one graph launch, the 512^2 grain-growth step with 1189 order parameters (periodic solves), the
    1024^2 adjoint heat run. Inputs are the seeded recipes of workloads/. Under
    several ranks the batched problems are shared out (cell-balanced, no data exchange) and the other
    workloads run as one replica per rank."""
    import numpy as np
    import torch

    import paper_2510_11152_gb300 as fas
    from workloads import (adjoint_heat, batched_helmholtz, batched_problem_rhs, heat3d, ns_cavity)

    out = {}
    mc = lambda cells, cycles, ms: cells * cycles / (ms / 1e3) / 1e6  # noqa: E731

    # 3D heat, 512^3, Neumann, dt 1e-4, 10 steps
    w = heat3d()
    shape, h, dt, nsteps = w["shape"], w["h"], w["dt"], w["nsteps"]
    cells = int(np.prod(shape))
    u0 = torch.from_numpy(w["u0"]).to(dev)
    f = torch.from_numpy(w["fsrc"]).to(dev) if w.get("fsrc") is not None else None
    u = torch.empty_like(u0)
    res = {}

    def make_heat(prec, inner):
        ctx = fas.fas_create(fas.make_params(shape, h, alpha=1.0, beta=dt, coarsest=4, precision=prec,
                                             inner_cycles=inner), stream=stream)

        def run():
            u.copy_(u0)
            return fas.fas_heat_run(ctx, u, f, dt, nsteps)
        return run, lambda: fas.fas_destroy(ctx)
    inner3, tune3 = tune_inner(stream, lambda k: make_heat(fas.FAS_MIXED, k))
    for prec, name in ((fas.FAS_MIXED, "mixed"), (fas.FAS_FP64, "fp64")):
        inner = inner3 if prec == fas.FAS_MIXED else 1
        run, done = make_heat(prec, inner)
        ms, infos = _event_ms(stream, run)
        cyc = sum(i.cycles for i in infos) * inner
        res[name] = {"ms_per_run": ms, "vcycles_per_run": cyc, "Mcells_vcycles_per_s": mc(cells, cyc, ms),
                     "converged_all": all(i.converged for i in infos), "u": u.clone()}
        if prec == fas.FAS_MIXED:
            res[name]["inner_float32_cycles"] = inner
            res[name]["ms_per_run_by_inner_cycles"] = {str(k): v for k, v in tune3.items()}
        done()
    out["heat3d_512"] = {
        "workload": "heat3d-512^3-neumann-dt1e-4-10steps-tol1e-10-V(2,2)-coarsest4",
        "mixed": {k: v for k, v in res["mixed"].items() if k != "u"},
        "fp64": {k: v for k, v in res["fp64"].items() if k != "u"},
        "speedup_mixed_vs_fp64_time": res["fp64"]["ms_per_run"] / res["mixed"]["ms_per_run"],
        "mixed_vs_fp64_rel_maxdiff": float((res["mixed"]["u"] - res["fp64"]["u"]).abs().max().item()
                                           / res["fp64"]["u"].abs().max().item())}
    del u0, f, u, res
    torch.cuda.empty_cache()

    # NS: first- and second-order projection, lid-driven cavity 256^3, Re 100, dt 1e-3, 20 steps from rest
    w = ns_cavity(n=256, dim=3, nsteps=20)
    shape, nsteps = w["shape"], w["nsteps"]
    cells = int(np.prod(shape))
    zero = torch.zeros(shape, dtype=torch.float64, device=dev)
    for order in (1, 2):
      ns_res = {}

      def make_ns(prec, inner):
        sp = fas.fas_default_params()
        sp.precision, sp.kmax, sp.coarsest, sp.inner_cycles = prec, 40, 4, inner
        pp = fas.fas_default_params()
        pp.precision, pp.kmax, pp.coarsest, pp.coarse_exact, pp.inner_cycles = prec, 60, 4, 1, inner
        ns = fas.ns_create(shape, w["h"], w["Re"], w["dt"], lid=w["lid"], order=order, solver=sp, pressure=pp,
                           stream=stream)
        flds = {k: zero.clone() for k in w["fields"]}

        def run():
            for t in flds.values():
                t.zero_()
            tot, div = [0, 0, 0, 0], 0.0
            for _ in range(nsteps):
                infos, div = fas.ns_projection_step(ns, flds, want_div=False)
                for k in range(4):
                    tot[k] += infos[k].cycles * inner
            return tot
        return ns, flds, run
      def ns_candidate(k):
        ns_k, _, run_k = make_ns(fas.FAS_MIXED, k)
        return run_k, lambda: fas.ns_destroy(ns_k)
      inner_ns, tune_ns = tune_inner(stream, ns_candidate)
      for prec, name in ((fas.FAS_MIXED, "mixed"), (fas.FAS_FP64, "fp64")):
        inner = inner_ns if prec == fas.FAS_MIXED else 1
        ns, flds, run = make_ns(prec, inner)
        fas.ns_launch_count(ns, reset=True)
        ms, tot = _event_ms(stream, run)
        _, dmax = fas.ns_projection_step(ns, flds, want_div=True)
        ns_res[name] = {"ms_per_step": ms / nsteps, "vcycles_per_step_u_v_w_p": [c / nsteps for c in tot],
                        "Mcells_vcycles_per_s": mc(cells, sum(tot), ms), "div_max_after": dmax,
                        "U": (flds["U_old"] if order == 1 else flds["U_new"]).clone()}
        if prec == fas.FAS_MIXED:
            ns_res[name]["inner_float32_cycles"] = inner
            ns_res[name]["ms_per_step_by_inner_cycles"] = {str(k): v / nsteps for k, v in tune_ns.items()}
        del flds
        fas.ns_destroy(ns)
      key = "ns_cavity_256" if order == 1 else "ns_cavity_256_order2"
      out[key] = {
        "workload": "ns-%s-order-projection-lid-cavity-256^3-Re100-dt1e-3-20steps-WENO3-tol1e-10"
                    % ("first" if order == 1 else "second"),
        "mixed": {k: v for k, v in ns_res["mixed"].items() if k != "U"},
        "fp64": {k: v for k, v in ns_res["fp64"].items() if k != "U"},
        "speedup_mixed_vs_fp64_time": ns_res["fp64"]["ms_per_step"] / ns_res["mixed"]["ms_per_step"],
        "mixed_vs_fp64_rel_maxdiff_U": float((ns_res["mixed"]["U"] - ns_res["fp64"]["U"]).abs().max().item()
                                             / ns_res["fp64"]["U"].abs().max().item()),
        "resident_fields": 8}
    del zero, ns_res
    torch.cuda.empty_cache()

    # batched: 96 independent 2D Helmholtz problems in one graph launch (per rank), mixed precision
    from paper_2510_11152_gb300.shard import gather_by_index, max_over_ranks, partition, sum_over_ranks
    probs_all = batched_helmholtz()
    mine = partition([p["n"] * p["n"] for p in probs_all], ws)[rank]
    probs = [probs_all[k] for k in mine]
    fs = [torch.from_numpy(batched_problem_rhs(p)).to(dev) for p in probs]
    ctxs = [fas.fas_create(fas.make_params((p["n"], p["n"]), 1.0 / p["n"], alpha=1.0, beta=p["dt"],
                                           kappa_const=p["kappa"], coarsest=4, precision=fas.FAS_MIXED),
                           stream=stream) for p in probs]
    us = [torch.zeros_like(t) for t in fs]

    def run_b():
        for t in us:
            t.zero_()
        return fas.fas_solve_batched(ctxs, us, fs, stream=stream) if ctxs else []

    def timed_b():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        ms, infos = _event_ms(stream, run_b)
        ms = max_over_ranks(ms, ws, dev)
        work = sum_over_ranks(sum(p["n"] * p["n"] * i.cycles for p, i in zip(probs, infos)), ws, dev)
        conv = gather_by_index({k: bool(i.converged) for k, i in zip(mine, infos)}, ws, len(probs_all))
        return {"ms": ms, "Mcells_vcycles_per_s": work / (ms / 1e3) / 1e6, "converged_all": all(conv)}
    default = timed_b()
    # autotuned: one tuning per size class (fas_autotune times whole solves of the class's first
    # problem; the other contexts of that size take the cached choice), then the same graph launch
    tuned_choice, t0 = {}, time.perf_counter()
    for p, c, f_ in zip(probs, ctxs, fs):
        scratch = torch.zeros_like(f_)
        r = fas.fas_autotune(c, scratch, f_)
        tuned_choice.setdefault(p["n"], (r["inner_cycles"], r["seg_rows"]))
    tune_s = time.perf_counter() - t0
    tuned = timed_b()
    out["batched_96"] = {"workload": "96 2D Helmholtz problems, n in 64..2048, kappa U(0.5,2), dt {1e-4,1e-3}, "
                                     "mixed, tol 1e-10, one graph launch per rank",
                         "ms": tuned["ms"], "Mcells_vcycles_per_s": tuned["Mcells_vcycles_per_s"],
                         "autotuned": True, "default_params": default,
                         "tuned_inner_cycles_seg_rows_by_n": {str(k): v for k, v in sorted(tuned_choice.items())},
                         "tuning_s": tune_s,
                         "fine_cells": sum(p["n"] * p["n"] for p in probs_all), "ranks": ws,
                         "converged_all": tuned["converged_all"] and default["converged_all"]}
    for c in ctxs:
        fas.fas_destroy(c)
    del fs, us, ctxs
    torch.cuda.empty_cache()

    # grain growth (Sec. 3.3.1): 512^2 periodic, q = 1189 order parameters, h 2, dt 0.25, from the
    # disordered start U(-0.001, 0.001); one step = the q right-hand sides and q periodic solves
    from workloads import grain_growth
    w = grain_growth()
    q, shape = w["q"], w["shape"]
    cells = int(np.prod(shape))
    eta0 = torch.from_numpy(w["etas"]).to(dev)
    del w["etas"]
    gsteps = 3
    ggr = {}
    eta = eta0.clone()

    def make_gg(prec, inner):
        sp = fas.fas_default_params()
        sp.precision, sp.kmax, sp.coarsest, sp.inner_cycles = prec, 40, 4, inner
        ctx = fas.gg_create(shape, w["h"], w["dt"], q, solver=sp, stream=stream)

        def run_g():  # the first call also builds the batch graphs
            eta.copy_(eta0)
            cyc = 0
            for _ in range(gsteps):
                cyc += sum(i.cycles for i in fas.gg_step(ctx, eta)) * inner
            return cyc
        return run_g, lambda: fas.gg_destroy(ctx)
    inner_gg, tune_gg = tune_inner(stream, lambda k: make_gg(fas.FAS_MIXED, k))
    for prec, name in ((fas.FAS_MIXED, "mixed"), (fas.FAS_FP64, "fp64")):
        inner = inner_gg if prec == fas.FAS_MIXED else 1
        run_g, done = make_gg(prec, inner)
        ms, cyc = _event_ms(stream, run_g)
        ggr[name] = {"ms_per_step": ms / gsteps, "vcycles_per_step": cyc / gsteps,
                     "Mcells_vcycles_per_s": mc(cells, cyc, ms), "eta": eta.clone()}
        if prec == fas.FAS_MIXED:
            ggr[name]["inner_float32_cycles"] = inner
            ggr[name]["ms_per_step_by_inner_cycles"] = {str(k): v / gsteps for k, v in tune_gg.items()}
        done()
    del eta
    out["grain_growth_512"] = {
        "workload": "grain growth 512^2 periodic, q=1189 order parameters, h 2, dt 0.25, %d steps from "
                    "U(-0.001,0.001), linearly implicit step, tol 1e-10" % gsteps,
        "mixed": {k: v for k, v in ggr["mixed"].items() if k != "eta"},
        "fp64": {k: v for k, v in ggr["fp64"].items() if k != "eta"},
        "speedup_mixed_vs_fp64_time": ggr["fp64"]["ms_per_step"] / ggr["mixed"]["ms_per_step"],
        "mixed_vs_fp64_rel_maxdiff": float((ggr["mixed"]["eta"] - ggr["fp64"]["eta"]).abs().max().item()
                                           / ggr["fp64"]["eta"].abs().max().item())}
    del eta0, ggr
    torch.cuda.empty_cache()

    # adjoint: 1024^2 heat with varying kappa, 50 steps, checkpoints every 10
    w = adjoint_heat()
    shape = w["shape"]
    kap = torch.from_numpy(w["kappa"]).to(dev)
    u0 = torch.from_numpy(w["u0"]).to(dev)
    fsrc = torch.from_numpy(w["fsrc"]).to(dev)
    tgt = torch.from_numpy(w["target"]).to(dev)
    adj = {}
    uT = torch.empty_like(u0)
    g = [torch.empty_like(u0) for _ in range(3)]
    fwd = torch.empty_like(u0)

    def make_adj(prec, inner):
        ctx = fas.fas_create(fas.make_params(shape, w["h"], alpha=1.0, beta=w["dt"], coarsest=4, precision=prec,
                                             inner_cycles=inner), stream=stream, kappa=kap)

        def run_a():
            fwd.copy_(u0)
            fas.fas_heat_run(ctx, fwd, fsrc, w["dt"], w["nsteps"])
            dl = 2.0 * (fwd - tgt)
            fas.fas_heat_adjoint(ctx, u0, fsrc, w["dt"], w["nsteps"], dl, uT, g[0], g[1], g[2], 10)
        return run_a, lambda: fas.fas_destroy(ctx)
    inner_adj, tune_adj = tune_inner(stream, lambda k: make_adj(fas.FAS_MIXED, k))
    for prec, name in ((fas.FAS_MIXED, "mixed"), (fas.FAS_FP64, "fp64")):
        run_a, done = make_adj(prec, inner_adj if prec == fas.FAS_MIXED else 1)
        ms, _ = _event_ms(stream, run_a)
        adj[name] = {"ms_forward_plus_adjoint": ms, "g_kappa": g[2].clone()}
        done()
    out["adjoint_1024"] = {"workload": "adjoint heat 1024^2, varying kappa, 50 steps, checkpoints every 10",
                           "mixed": {"ms_forward_plus_adjoint": adj["mixed"]["ms_forward_plus_adjoint"],
                                     "inner_float32_cycles": inner_adj,
                                     "ms_by_inner_cycles": {str(k): v for k, v in tune_adj.items()}},
                           "fp64": {"ms_forward_plus_adjoint": adj["fp64"]["ms_forward_plus_adjoint"]},
                           "mixed_vs_fp64_rel_maxdiff_g_kappa": float(
                               (adj["mixed"]["g_kappa"] - adj["fp64"]["g_kappa"]).abs().max().item()
                               / adj["fp64"]["g_kappa"].abs().max().item())}
    return out


def cpu_baseline(w, n_cycles=2):
    """The oracle as it stands, float64 V(2,2) cycles on the first time step's system at full size
    (bounded sample: two cycles, about 20 s of single-threaded numpy on the GB300 host's cores)."""
    from oracle import cell_centred as cc
    op = cc.heat_operator(w["shape"], w["h"], w["dt"])
    lev = cc.build_levels(op, 4)
    b = w["u0"] + w["dt"] * w["fsrc"]
    u = w["u0"].copy()
    t0 = time.perf_counter()
    for _ in range(n_cycles):
        cc.vcycle(lev, u, b, cc.Params(coarsest=4))
    t = time.perf_counter() - t0
    cells = w["shape"][0] * w["shape"][1]
    return {"value": cells * n_cycles / t / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d float64 V(2,2) cycle(s) of the numpy oracle on the first backward-Euler step of the "
                      "%dx%d workload (%.1f s)" % (n_cycles, w["shape"][0], w["shape"][1], t)}


def _oracle_cycles_worker(args):
    """One worker of the all-core CPU baseline: the oracle's float64 V(2,2) cycles on the first
    backward-Euler step's system of the heat recipe at n x n; returns (start, end, cells x cycles)."""
    n, n_cycles = args
    from oracle import cell_centred as cc
    from workloads import heat2d_large
    w = heat2d_large(n=n, nsteps=1)
    op = cc.heat_operator(w["shape"], w["h"], w["dt"])
    lev = cc.build_levels(op, 4)
    b = w["u0"] + w["dt"] * w["fsrc"]
    u = w["u0"].copy()
    t0 = time.time()
    for _ in range(n_cycles):
        cc.vcycle(lev, u, b, cc.Params(coarsest=4))
    return t0, time.time(), n * n * n_cycles


def cpu_baseline_all_cores(n=4096, n_cycles=2):
    """The oracle on every host core at once: one process per core (spawned, so no process is forked
    from one that holds a CUDA context), each running the same bounded sample; throughput = all the
    cells x cycles done / the wall time from the first start to the last end."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    env_keep = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env_keep:
        os.environ[k] = "1"  # one thread per worker process
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_cycles_worker, [(n, n_cycles)] * cores)
    finally:
        for k, v in env_keep.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    t = max(r[1] for r in res) - min(r[0] for r in res)
    work = sum(r[2] for r in res)
    return {"value": work / t / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d processes at once, each %d float64 V(2,2) cycles of the numpy oracle on the first "
                      "backward-Euler step of the heat recipe at %dx%d (%.1f s from first start to last end)"
                      % (cores, n_cycles, n, n, t)}


def run_reference(args, ws, rank):
    """The oracle timed on the host cores on the same metric; each step one oracle V-cycle on the
    first time step's system, at a grid size chosen so the whole run stays within a few minutes."""
    if rank != 0:
        return
    from oracle import cell_centred as cc
    from workloads import heat2d_large
    total = args.steps + args.warmup
    n = args.n if total <= 6 else (args.n // 2 if total <= 24 else args.n // 4)
    w = heat2d_large(n=n, nsteps=1)
    op = cc.heat_operator(w["shape"], w["h"], w["dt"])
    lev = cc.build_levels(op, 4)
    b = w["u0"] + w["dt"] * w["fsrc"]
    prm = cc.Params(coarsest=4)
    u = w["u0"].copy()
    for _ in range(args.warmup):
        cc.vcycle(lev, u, b, prm)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cc.vcycle(lev, u, b, prm)
    t = time.perf_counter() - t0
    value = n * n * args.steps / t / 1e6
    sample = "one float64 V(2,2) cycle of the numpy oracle per step on the first backward-Euler step of the " \
             "heat workload at %dx%d (same recipe as the 8192^2 workload)" % (n, n)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "heat2d-8192x8192-neumann-dt1e-4-20steps-tol1e-10-V(2,2)-coarsest4",
                       "sample_grid": [n, n]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_case(args):
    """One small timed case of the 3D heat or cavity workload (single GPU), e.g. for ncu captures."""
    import numpy as np
    import torch

    import paper_2510_11152_gb300 as fas
    from workloads import heat3d, ns_cavity
    fas.load()
    graph = 0 if args.no_graph else 1
    out = {"case": args.case, "launch": "host loop" if args.no_graph else "one CUDA graph per solve"}
    if args.case == "heat3d":
        nz, ny, nx = (int(v) for v in args.shape.split(","))
        w = heat3d(n=nx)
        u0 = torch.from_numpy(np.ascontiguousarray(w["u0"][:nz, :ny, :nx])).cuda()
        ctx = fas.fas_create(fas.make_params((nz, ny, nx), w["h"], alpha=1.0, beta=w["dt"], coarsest=4, precision=1,
                                             use_graph=graph))
        u = u0.clone()
        t0 = time.perf_counter()
        infos = fas.fas_heat_run(ctx, u, None, w["dt"], args.heat_steps)
        torch.cuda.synchronize()
        out.update({"shape": [nz, ny, nx], "steps": args.heat_steps, "ms": (time.perf_counter() - t0) * 1e3,
                    "cycles": [i.cycles for i in infos]})
    else:
        w = ns_cavity(n=args.ns_n, dim=3, nsteps=args.heat_steps)
        sp = fas.fas_default_params()
        sp.precision, sp.kmax, sp.coarsest, sp.use_graph = 1, 40, 4, graph
        pp = fas.fas_default_params()
        pp.precision, pp.kmax, pp.coarsest, pp.coarse_exact, pp.use_graph = 1, 60, 4, 1, graph
        ns = fas.ns_create(w["shape"], w["h"], w["Re"], w["dt"], lid=w["lid"], order=args.ns_order, solver=sp,
                           pressure=pp)
        flds = {k: torch.zeros(w["shape"], dtype=torch.float64, device="cuda") for k in w["fields"]}
        t0 = time.perf_counter()
        cyc = []
        for _ in range(args.heat_steps):
            infos, _ = fas.ns_projection_step(ns, flds, want_div=False)
            cyc.append([i.cycles for i in infos])
        torch.cuda.synchronize()
        out.update({"n": args.ns_n, "order": args.ns_order, "steps": args.heat_steps,
                    "ms": (time.perf_counter() - t0) * 1e3, "cycles_u_v_w_p": cyc})
    print(json.dumps(out))


def main():
    args = parse()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.case != "heat2d":
        if rank == 0:
            run_case(args)
        return
    run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
