"""Benchmark: time-to-gradient of closed-shell CD-CCSD on one GB300.

One step = one full gradient: cd_ccsd_init (inputs already in HBM) ->
ccsd_solve -> lambda_solve -> build_density -> contract_dL over all
displacements, through the C ABI.  Prints ONE JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config 1]
                    [--precision fp64|mixed] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (bounded sample, host cores).
With N > 1 (torchrun) every rank runs an independent replica (the method
does not shard across GPUs here); value is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("time-to-gradient & ladder TFLOP/s, mixed vs FP64 GPU, at "
          "|dE|<=1e-8 Eh; p50/p99")
WORKLOAD = {0: "c0: C1 o=4 v=20 nL=60, 6 displacements",
            1: "c1: D2h o=16 v=144 nL=640, 18 displacements",
            2: "c2: C2v o=40 v=360 nL=1600, 24 displacements",
            3: "c3: D2h o=60 v=540 nL=2400, 36 displacements"}
FP64_PEAK_GFLOPS = 1250.0      # GB300 FP64 nominal (profiling recipe table)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", type=int, default=1)
    ap.add_argument("--precision", default="fp64",
                    choices=["fp64", "mixed", "tc"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--others", default="all",
                    help="other schedules to time beside --precision: "
                         "'all', 'none' or a comma list")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--error-estimate", action="store_true",
                    help="after the timed steps, run cdcc_error_estimate "
                         "(one FP64 residual and density sweep, untimed)")
    ap.add_argument("--symmetry-ignored", action="store_true",
                    help="the same data with every irrep label set to 0 "
                         "(C1 twin): measures the speed-up symmetry gives")
    ap.add_argument("--serving", action="store_true",
                    help="run the serving workload (Poisson arrivals of "
                         "mixed requests) instead of a fixed workload")
    ap.add_argument("--jobs", type=int, default=64)
    ap.add_argument("--slots", type=int, default=4)
    return ap.parse_args()


def dist_init():
    from paper_2512_21909_gb300 import replicas
    return replicas.init()


def barrier(ws):
    from paper_2512_21909_gb300 import replicas
    replicas.barrier(ws)


def allmax(x, ws):
    from paper_2512_21909_gb300 import replicas
    return replicas.allmax(x, ws)


# ---------------------------------------------------------------- clocks
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,"
         "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device=0):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}",
                 f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no-smi"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle
def oracle_sample(cfg):
    """Time the FP64 oracle on a bounded sample of the workload: one CCSD
    residual and one Lambda (reverse-mode) evaluation at the MP2-like start,
    scaled by the oracle's own iteration counts stored with the golden
    values (tests/golden/c<cfg>.json, written by oracle-only code)."""
    import torch
    from synth import make_system, unpack_dense
    from oracle import model, ccsd, lagrangian
    s = make_system(cfg)
    o, v = s.nocc, s.nvir
    L = torch.as_tensor(unpack_dense(s, s.L))
    h = model.core_from_eps(torch.as_tensor(s.eps), L, o)
    z1 = torch.zeros(o, v, dtype=torch.float64)
    z2 = torch.zeros(o, o, v, v, dtype=torch.float64)
    t0 = time.perf_counter()
    with torch.no_grad():
        R1, R2, _ = ccsd.residual(z1, z2, h, L, o)
    t_cc = time.perf_counter() - t0
    f = model.fock(h, L, o)
    _, Dijab = ccsd.denominators(f, o)
    t2 = R2 / Dijab
    t0 = time.perf_counter()
    lagrangian.lambda_gradient(z1, t2, z1, t2, h, L, o)
    t_lam = time.perf_counter() - t0
    gold = os.path.join(ROOT, "tests", "golden", f"c{cfg}.json")
    n_cc, n_lam = 17, 15
    if os.path.exists(gold):
        g = json.load(open(gold))
        n_cc, n_lam = g["ccsd_iterations"], g["lambda_iterations"]
    est = n_cc * t_cc + (n_lam + 1) * t_lam     # +1: density sweep
    return dict(value=est, unit="s", cores=torch.get_num_threads(),
                kind="oracle",
                sample=(f"1 CCSD residual ({t_cc:.2f}s) + 1 Lambda "
                        f"reverse sweep ({t_lam:.2f}s) of {WORKLOAD[cfg]}, "
                        f"scaled by the oracle's {n_cc} CCSD + {n_lam} "
                        "Lambda iterations + 1 density sweep"),
                sample_seconds=t_cc + t_lam)


def run_reference(args, rank, ws):
    if rank != 0:
        return
    times = []
    for i in range(args.warmup + args.steps):
        r = oracle_sample(args.config)
        if i >= args.warmup:
            times.append(r["value"])
    v = float(np.median(times))
    r["value"] = v
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": v * 1e3, "higher_is_better": False,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD[args.config],
                                           "precision": "fp64"},
           "cpu_baseline": r,
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- GPU arm
def run_ours(args, rank, ws):
    import torch
    from synth import make_system, make_displacements
    from paper_2512_21909_gb300 import build as cbuild, cdcc

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    if rank == 0:
        cbuild.build()
    barrier(ws)
    cdcc.load()
    s = make_system(args.config)
    dL = make_displacements(s)
    if args.symmetry_ignored:
        from synth import as_c1
        s, extra = as_c1(s, list(dL))
        dL = np.stack(extra)
    nx = dL.shape[0]
    L_d = torch.as_tensor(s.L, device="cuda")
    dL_d = torch.as_tensor(dL, device="cuda")
    L_h = torch.as_tensor(s.L).pin_memory()
    dL_h = torch.as_tensor(dL).pin_memory()
    flush = torch.empty(int(512 * 2 ** 20) // 4, dtype=torch.float32,
                        device="cuda")
    stream = torch.cuda.current_stream()

    def options():
        o = cdcc.cdcc_default_options()
        o.device = dev
        o.precision = {"fp64": cdcc.PREC_FP64, "mixed": cdcc.PREC_MIXED,
                       "tc": cdcc.PREC_TC}[args.precision]
        return o

    def one(Lsrc, dLsrc, profile=False):
        ctx = cdcc.cd_ccsd_init(s.nirrep, s.nocc, s.nvir, s.nchol,
                                s.orb_irrep, s.eps, s.chol_irrep, Lsrc,
                                options=options())
        if profile:
            cdcc.cdcc_profile(ctx, True)
        e, g = cdcc.gradient(ctx, dLsrc)
        stats = None
        if profile:
            stats = [cdcc.cdcc_kernel_stats(ctx, k) for k in range(6)]
            stats.append(cdcc.cdcc_ladder_stats(ctx))
        nl = cdcc.cdcc_kernel_launches(ctx)
        ph = cdcc.cdcc_phase_times(ctx)
        cdcc.cd_ccsd_free(ctx)
        return e, g, nl, stats, ph

    for _ in range(args.warmup):
        one(L_d, dL_d)
    torch.cuda.synchronize()

    # ---- device-resident timing (inputs in HBM), L2 flushed between steps
    clk = ClockSampler(dev)
    clk.start()
    barrier(ws)
    torch.cuda.synchronize()
    times, launches = [], 0
    agg = np.zeros((7, 3))
    for _ in range(args.steps):
        flush.fill_(1.0)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        e, g, nl, stats, ph = one(L_d, dL_d, profile=True)
        ev1.record(stream)
        torch.cuda.synchronize()
        times.append(ev0.elapsed_time(ev1) * 1e-3)
        launches += nl
        agg += np.array(stats)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = clk.stop()
    t50 = allmax(float(np.median(times)), ws)
    t99 = allmax(float(np.percentile(times, 99)), ws)

    # ---- the other schedules on the same workload (mixed / TC vs FP64 GPU)
    saved = args.precision
    other_lines = []
    wanted = ("fp64", "mixed", "tc") if args.others == "all" else \
        tuple(x for x in args.others.split(",") if x and x != "none")
    for other in [p for p in wanted if p != saved]:
        args.precision = other
        one(L_d, dL_d)                   # warm-up of the other schedule
        o_times = []
        for _ in range(max(1, min(args.steps, 3))):
            flush.fill_(1.0)
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            o_e, o_g, _, o_stats, _ = one(L_d, dL_d, profile=True)
            ev1.record(stream)
            torch.cuda.synchronize()
            o_times.append(ev0.elapsed_time(ev1) * 1e-3)
        tc = o_stats[5]
        lad = o_stats[6]
        other_lines.append({
            "precision": other,
            "time_to_gradient_s": float(np.median(o_times)),
            "abs_dE_vs_this_run": abs(o_e - e),
            "max_abs_dg_vs_this_run": float(np.abs(o_g - g).max()),
            "tc_gemm_s": tc[0],
            "tc_gemm_tflops": tc[2] / tc[0] / 1e12 if tc[0] > 0 else None,
            "ladder_s": lad[0],
            "ladder_tflops": lad[1] / lad[0] / 1e12 if lad[0] > 0 else None})
    args.precision = saved

    # ---- error report of the --precision schedule (untimed)
    err_est = None
    if args.error_estimate:
        ctx = cdcc.cd_ccsd_init(s.nirrep, s.nocc, s.nvir, s.nchol,
                                s.orb_irrep, s.eps, s.chol_irrep, L_d,
                                options=options())
        cdcc.gradient(ctx, dL_d)
        t0 = time.perf_counter()
        dE, dg = cdcc.cdcc_error_estimate(ctx, dL_d)
        err_est = {"dE": dE, "max_dg": float(np.abs(dg).max()),
                   "seconds": time.perf_counter() - t0,
                   "what": "|E64(t)-E(t)| + |<lambda,R64(t)>| and "
                           "|<Gamma64-Gamma, dL>| against FP64 at the "
                           "converged t, lambda"}
        cdcc.cd_ccsd_free(ctx)

    # ---- end to end through the C ABI with host buffers
    e2e = []
    for _ in range(max(0, min(args.steps, args.e2e_steps))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        one(L_h.numpy(), dL_h.numpy())
        e2e.append(time.perf_counter() - t0)
    e2e50 = allmax(float(np.median(e2e)), ws) if e2e else None
    h2d = (s.L.nbytes + dL.nbytes + s.eps.nbytes + s.orb_irrep.nbytes
           + s.chol_irrep.nbytes)
    d2h = 8 * (nx + 1)

    if rank != 0:
        return
    # roofline of the dominant kernel class (FP64 GEMM) over the timed region
    gsec, gn, gfl = agg[0]
    achieved = gfl / gsec / 1e9 if gsec > 0 else 0.0
    # ladder flops (algorithmic) per application, for the ladder TFLOP/s line
    from synth.gen import packed_size  # noqa
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        try:
            cpu = oracle_sample(args.config)
        except Exception as ex:  # pragma: no cover
            cpu = {"error": str(ex)}
    classes = {}
    for k, nm in enumerate(["gemm64", "permute", "update", "contract_dL",
                            "other", "tc_gemm"]):
        sec, n, w = agg[k]
        classes[nm] = {"seconds": sec / args.steps, "launches": int(n /
                                                                    args.steps),
                       "work_per_step": w / args.steps}
    out = {
        "metric": METRIC, "value": t50, "unit": "s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t50 * 1e3,
        "p99_s": t99, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD[args.config] + (
                       " (C1 twin: irreps ignored)" if args.symmetry_ignored
                       else ""),
                   "precision": args.precision,
                   "l2": "flushed between steps (512 MiB write)",
                   "parallelism": "replicas" if ws > 1 else "1 GPU"},
        "e_corr": e, "gradients_per_s": ws / t50,
        "gpu_launches": int(launches / args.steps),
        "phases_s": {"ccsd": ph[0], "lambda": ph[1], "density": ph[2],
                     "contract_dL": ph[3]},
        "peak_device_gb": torch.cuda.max_memory_allocated(dev) / 1e9,
        "error_estimate": err_est,
        "kernel_classes": classes,
        "ladder": {"seconds_per_step": agg[6][0] / args.steps,
                   "flops_per_step": agg[6][1] / args.steps,
                   "tflops": (agg[6][1] / agg[6][0] / 1e12
                              if agg[6][0] > 0 else None),
                   "share_of_step": agg[6][0] / args.steps / t50,
                   "note": "algorithmic flops of the ladder products, "
                           "(ac|bd) builds and their adjoints"},
        "roofline": {"kernel": "gemm64_kernel (FP64 DFMA grouped GEMM)",
                     "bound": "alu", "achieved": achieved / 1e3,
                     "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_GFLOPS,
                     "peak_source": "nominal GB300 FP64 from the profiling "
                                    "recipe (not in MEASURED_PEAKS.json)",
                     "traffic": None},
        "other_precisions": other_lines,
        "e2e": {"value": e2e50, "unit": "s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(out), flush=True)


def run_serving(args, rank, ws):
    """Serving workload: requests arrive as a Poisson stream (mean 0.5 s),
    are admitted by device memory and slots, overlap on the GPU and report
    p50 / p99 time-to-gradient (completion - arrival) and jobs/s.  Each
    replica (N > 1) serves the whole stream on its own GPU."""
    import torch
    from synth import make_displacements
    from synth.serving import serving_jobs, job_system
    from paper_2512_21909_gb300 import build as cbuild, cdcc
    from paper_2512_21909_gb300.serve import (GradientServer, Request,
                                              latency_stats)
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    if rank == 0:
        cbuild.build()
    barrier(ws)
    prec = {"fp64": cdcc.PREC_FP64, "mixed": cdcc.PREC_MIXED,
            "tc": cdcc.PREC_TC}[args.precision]
    specs = serving_jobs()[:args.jobs]
    reqs = []
    for sp in specs:
        sysm = job_system(sp)
        reqs.append(Request.from_system(sp.index, sp.arrival, sysm,
                                        make_displacements(sysm, 2)))
        reqs[-1].extra.update(group=sp.group, o=sp.o)
    # warm-up: the smallest request alone
    small = min(specs, key=lambda j: j.o)
    ws_sys = job_system(small)
    warm = [Request.from_system(-1, 0.0, ws_sys,
                                make_displacements(ws_sys, 2))]
    srv = GradientServer(device=dev, precision=prec, max_active=args.slots)
    for _ in range(max(1, args.warmup)):
        srv.run([Request.from_system(-1, 0.0, ws_sys, warm[0].dL)],
                realtime=False)
    clk = ClockSampler(dev)
    clk.start()
    barrier(ws)
    srv.run(reqs, realtime=True)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = clk.stop()
    st = latency_stats(reqs, srv.wall)
    p50 = allmax(st["p50_s"] or float("nan"), ws)
    p99 = allmax(st["p99_s"] or float("nan"), ws)
    wall = allmax(srv.wall, ws)
    if rank != 0:
        return
    h2d = sum(r.L.nbytes + r.dL.nbytes for r in reqs)
    out = {
        "metric": "serving: time-to-gradient p50 (p99 and jobs/s beside) "
                  "under Poisson arrivals",
        "value": p50, "unit": "s", "n_gpus": ws, "steps": 1,
        "warmup": max(1, args.warmup), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "mixed": "bf16x3+f64",
                  "tc": "bf16x3+exact-slice"}[args.precision],
        "data": "synthetic",
        "config": {"workload": f"c4: {len(reqs)} requests, Poisson arrivals "
                               "mean 0.5 s, o~U{4..40}, v=9o, nL=40o, "
                               "C1/C2v/D2h, 2 displacements each",
                   "precision": args.precision, "slots": args.slots,
                   "parallelism": "replicas" if ws > 1 else "1 GPU"},
        "p50_s": p50, "p99_s": p99,
        "jobs_per_s": ws * len(reqs) / wall if wall > 0 else None,
        "done": st["done"], "failed": st["failed"], "wall_s": wall,
        "max_concurrent": srv.max_seen_active,
        "e2e": {"value": p50, "unit": "s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(sum(8 * (r.dL.shape[0] + 1)
                                              for r in reqs))},
        "requests": [{"i": r.index, "group": r.extra["group"],
                      "o": r.extra["o"], "latency_s": r.latency,
                      "admit_s": (r.t_admit - r.arrival
                                  if r.t_admit is not None else None),
                      "ladder": "stored" if r.ladder == cdcc.LADDER_STORED
                      else "otf", "status": r.status, "e_corr": r.e}
                     for r in reqs],
        "clocks": clocks,
    }
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank, ws = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, ws)
    elif args.serving:
        run_serving(args, rank, ws)
    else:
        run_ours(args, rank, ws)
    from paper_2512_21909_gb300 import replicas
    replicas.finalize(ws)


if __name__ == "__main__":
    main()
