"""Benchmark: time-to-gradient of closed-shell CD-CCSD on one GB300.

One step = one full gradient: cd_ccsd_init (inputs already in HBM) ->
ccsd_solve -> lambda_solve -> build_density -> contract_dL over all
displacements, through the C ABI.  Prints ONE JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config 3]
                    [--precision tc|mixed|fp64] [--compare 2|none]
                    [--impl ours|reference]
    python bench.py --gemm M,N,K[,ta,tb] [--gemm-modes 0,2,14]

Default workload: D2h o=60 v=540 nL=2400 with 36 displacements in the
tensor-core schedule (BF16x3 iterations, exact-slice accurate phase).  The
mixed-vs-FP64 comparison runs on the C2v o=40 v=360 nL=1600 workload (the
FP64 path would take about half an hour on the larger one).
--impl reference times the FP64 CPU oracle (bounded sample, host cores).
With N > 1 (torchrun) every rank runs an independent replica (the method
does not shard across GPUs here); value is the max over ranks.
--gemm times the library's contraction kernels on one product shape
through cdcc_dgemm (the command the kernel profiles were taken with).
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
DTYPE = {"fp64": "f64", "mixed": "bf16x3+f64", "tc": "bf16x3+exact-slice"}
PLAIN_LADDER = False   # --plain-ladder: cdcc_options.ladder_pm = 0
# FP64 pipe of GB300 (not in the measured peaks): 2 DFMA per clock per SM
# x 2 flop x 152 SMs x 2.07 GHz
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12
CLASSES = ["gemm64", "permute", "update", "contract_dL", "other",
           "tc_float_slices", "tc_exact_slices"]
# BF16 MMAs per algorithmic product: float slices (2 slices: i + j < 2) and
# exact slices (4 slices: i + j < 4)
MMA_PER_PRODUCT = {"tc_float_slices": 3, "tc_exact_slices": 10}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", type=int, default=3)
    ap.add_argument("--precision", default="tc",
                    choices=["fp64", "mixed", "tc"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--compare", default="2",
                    help="workload of the mixed-vs-FP64 comparison (both "
                         "schedules timed once each), or 'none'")
    ap.add_argument("--others", default="none",
                    help="other schedules timed on the --config workload: "
                         "'all', 'none' or a comma list")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-linearize", action="store_true",
                    help="every accurate-phase iteration fully accurate "
                         "(cdcc_options.ladder_linearize = 0)")
    ap.add_argument("--plain-ladder", action="store_true",
                    help="the on-the-fly ladder without the +/- packing "
                         "(cdcc_options.ladder_pm = 0)")
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
    ap.add_argument("--gemm", default=None,
                    help="M,N,K[,ta,tb]: time cdcc_dgemm on one shape")
    ap.add_argument("--gemm-modes", default="0,2,14")
    ap.add_argument("--ref-blocks", type=int, default=1,
                    help="oracle ladder blocks timed per reference step")
    ap.add_argument("--cd", action="store_true",
                    help="symmetry-adapted two-step Cholesky decomposition "
                         "(Algorithm 1) of a synthetic D2h pair-integral "
                         "matrix of the paper's 678-function basis size, "
                         "timed, with the oracle on the same input")
    ap.add_argument("--ladder-shape", action="store_true",
                    help="two tensor-core CCSD iterations of a D2h system "
                         "with the ladder batch shape of the o=60 v=540 "
                         "nL=2400 workload (68 virtuals and 300 Cholesky "
                         "vectors per irrep) but o=16: a small case for "
                         "kernel captures")
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


def peaks():
    """Roofline denominators: MEASURED_PEAKS.json if present, else the
    earlier GB300 measurement of the profiling notes (labelled)."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]),
                "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d["bf16_tflops_sustained"]),
                "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0,
                "bf16_tflops_sustained": 1700.0, "source": "fallback"}


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
class OracleSample:
    """The FP64 oracle on a bounded sample of a workload.

    The oracle's rate-determining step is its particle-particle ladder
    (Sec. 2.3), evaluated one block of the virtual index a at a time
    (oracle.ccsd.ladder_block: (ac|bd) for the block from L^P_ab, then the
    product with t2); the whole ladder is n_blocks such blocks.  A sample
    times `blocks` of them on the dense (symmetry-ignored) arrays of the
    workload and scales to a full gradient:
        t_grad = t_block * n_blocks * n_ladder,
        n_ladder = n_cc + 4 (n_lambda + 1),
    n_cc / n_lambda the iteration counts of the oracle's own c1 run
    (tests/golden/c1.json; 17 and 15): one ladder per CCSD residual and
    about four ladder-equivalents per reverse-mode Lambda or density sweep
    (checkpointed forward, recomputation and the two adjoint products).
    The oracle's O(o^3 v^3) terms are not counted, so this is a lower
    bound of the oracle's time-to-gradient."""

    def __init__(self, cfg):
        import torch
        from synth import make_system, unpack_dense
        s = make_system(cfg)
        o, v = s.nocc, s.nvir
        L = unpack_dense(s, s.L)
        self.vv = torch.as_tensor(np.ascontiguousarray(L[:, o:, o:]))
        del L
        rng = np.random.default_rng(20251221909 + 100 + cfg)
        t2 = rng.standard_normal((o, o, v, v)) * 1e-3
        self.t2 = torch.as_tensor(t2)
        self.o, self.v, self.cfg = o, v, cfg
        self.blk = max(1, min(v, int(2.0e7 // max(1, v ** 3))))
        self.n_blocks = -(-v // self.blk)
        gold = os.path.join(ROOT, "tests", "golden", "c1.json")
        self.n_cc, self.n_lam = 17, 15
        if os.path.exists(gold):
            g = json.load(open(gold))
            self.n_cc = g["ccsd_iterations"]
            self.n_lam = g["lambda_iterations"]
        self.n_ladder = self.n_cc + 4 * (self.n_lam + 1)
        self.next_a = 0
        self.threads = torch.get_num_threads()

    def time_blocks(self, nblocks):
        import torch
        from oracle import ccsd
        t = 0.0
        with torch.no_grad():
            for _ in range(nblocks):
                a0 = self.next_a
                a1 = min(self.v, a0 + self.blk)
                self.next_a = a1 % self.v
                t0 = time.perf_counter()
                ccsd.ladder_block(self.t2, self.vv, a0, a1)
                t += time.perf_counter() - t0
        return t / nblocks

    def estimate(self, nblocks):
        tb = self.time_blocks(nblocks)
        est = tb * self.n_blocks * self.n_ladder
        return dict(
            value=est, unit="s", cores=self.threads, kind="oracle",
            sample=(f"{nblocks} of the {self.n_blocks} a-blocks of the "
                    f"oracle's particle-particle ladder on {WORKLOAD[self.cfg]}"
                    f" (oracle.ccsd.ladder_block, dense FP64, {tb:.2f} s per "
                    f"block), scaled by {self.n_blocks} blocks x "
                    f"{self.n_ladder} ladder evaluations ({self.n_cc} CCSD + "
                    f"4 x ({self.n_lam} Lambda + 1 density)); O(o^3 v^3) "
                    "terms not counted (lower bound)"),
            seconds_per_block=tb, sample_seconds=tb * nblocks)


def run_reference(args, rank, ws):
    if rank != 0:
        return
    smp = OracleSample(args.config)
    smp.time_blocks(1)                   # untimed warm-up (thread pools)
    vals = []
    for i in range(args.warmup + args.steps):
        r = smp.estimate(args.ref_blocks)
        if i >= args.warmup:
            vals.append(r["value"])
    v = float(np.median(vals))
    r["value"] = v
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": v * 1e3, "p99_s": float(np.percentile(vals, 99)),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD[args.config],
                      "precision": "fp64 (CPU oracle)"},
           "cpu_baseline": r,
           "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------- GPU arm
# DRAM traffic of the dominant kernel from one ncu capture (dram__bytes_read
# + dram__bytes_write of one launch; the full gradient is too large to
# capture): the exact-slice kernel on a c3 ring block.
TRAFFIC = {
    "tc_exact_slices": {
        "traffic": 2017741312 + 129201152,
        "traffic_note": "ncu, one oz_gemm_kernel launch on a 4048 x 4048 x "
                        "4048 block (the size of a c3 ring block), 4 exact "
                        "slices: 1.390 ms, 95.4 TFLOP/s algorithmic; "
                        "algorithmic bytes of that launch 393 MB (slices of "
                        "both operands read once, C written once): the B "
                        "panels are re-read per row tile (262 MB of slices "
                        "exceed L2); command: ncu --metrics gpu__time_"
                        "duration.sum,dram__bytes_read.sum,dram__bytes_"
                        "write.sum --clock-control none -k regex:oz_gemm "
                        "-c 2 python bench.py --gemm 4048,4048,4048,0,0 "
                        "--gemm-modes 14",
        "traffic_algorithmic_bytes": 393400000,
    },
}


def prec_code(cdcc, name):
    return {"fp64": cdcc.PREC_FP64, "mixed": cdcc.PREC_MIXED,
            "tc": cdcc.PREC_TC}[name]


class Runner:
    """One workload resident in HBM; one() runs a full gradient."""

    def __init__(self, cfg, dev, symmetry_ignored=False):
        import torch
        from synth import make_system, make_displacements
        s = make_system(cfg)
        dL = make_displacements(s)
        if symmetry_ignored:
            from synth import as_c1
            s, extra = as_c1(s, list(dL))
            dL = np.stack(extra)
        self.s, self.dL, self.nx, self.dev = s, dL, dL.shape[0], dev
        self.L_d = torch.as_tensor(s.L, device="cuda")
        self.dL_d = torch.as_tensor(dL, device="cuda")
        self._host = None

    def host(self):
        import torch
        if self._host is None:
            self._host = (torch.as_tensor(self.s.L).pin_memory(),
                          torch.as_tensor(self.dL).pin_memory())
        return self._host

    def one(self, cdcc, prec, Lsrc=None, dLsrc=None, profile=False,
            linearize=True):
        s = self.s
        o = cdcc.cdcc_default_options()
        o.device = self.dev
        o.precision = prec_code(cdcc, prec)
        o.ladder_linearize = 1 if linearize else 0
        o.ladder_pm = 0 if PLAIN_LADDER else 1
        ctx = cdcc.cd_ccsd_init(s.nirrep, s.nocc, s.nvir, s.nchol,
                                s.orb_irrep, s.eps, s.chol_irrep,
                                self.L_d if Lsrc is None else Lsrc, options=o)
        if profile:
            cdcc.cdcc_profile(ctx, True)
        e, g = cdcc.gradient(ctx, self.dL_d if dLsrc is None else dLsrc)
        info = {"launches": cdcc.cdcc_kernel_launches(ctx),
                "phases": [float(x) for x in cdcc.cdcc_phase_times(ctx)],
                "solver": [int(x) for x in cdcc.cdcc_solver_info(ctx)]}
        if profile:
            info["stats"] = [cdcc.cdcc_kernel_stats(ctx, k)
                             for k in range(len(CLASSES))]
            info["ladder"] = cdcc.cdcc_ladder_stats(ctx)
        cdcc.cd_ccsd_free(ctx)
        return e, g, info


def timed_steps(torch, runner, cdcc, prec, n, flush, stream, linearize):
    times, infos, last = [], [], None
    for _ in range(n):
        flush.fill_(1.0)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        e, g, info = runner.one(cdcc, prec, profile=True, linearize=linearize)
        ev1.record(stream)
        torch.cuda.synchronize()
        times.append(ev0.elapsed_time(ev1) * 1e-3)
        infos.append(info)
        last = (e, g)
    return times, infos, last


def class_table(infos, steps):
    agg = np.zeros((len(CLASSES), 3))
    lad = np.zeros(3)
    for inf in infos:
        agg += np.array(inf["stats"], dtype=float)
        lad += np.array(inf["ladder"], dtype=float)
    out = {}
    for k, nm in enumerate(CLASSES):
        sec, n, w = agg[k] / steps
        out[nm] = {"seconds": sec, "launches": int(round(n)),
                   "work_per_step": w}
    return out, lad / steps


def rooflines(classes, pk):
    """Per kernel class: achieved rate over its device time against its
    bound.  Tensor-core classes: algorithmic flops (2MNK) and the BF16 MMA
    work they execute (x3 float slices, x10 exact slices) against the
    measured sustained BF16 peak; FP64 GEMM against the derived DFMA peak;
    the rest (bytes) against the measured HBM copy bandwidth."""
    out = {}
    for nm, c in classes.items():
        sec, work = c["seconds"], c["work_per_step"]
        if sec <= 0:
            continue
        if nm in MMA_PER_PRODUCT:
            alg = work / sec / 1e12
            exe = alg * MMA_PER_PRODUCT[nm]
            P = pk["bf16_tflops_sustained"]
            out[nm] = {"bound": "tensor", "achieved": alg, "peak": P,
                       "unit": "TFLOP/s", "frac": alg / P,
                       "executed_mma_tflops": exe, "frac_executed": exe / P,
                       "peak_source": pk["source"] + " bf16 sustained",
                       "seconds": sec}
        elif nm == "gemm64":
            a = work / sec / 1e12
            out[nm] = {"bound": "alu", "achieved": a,
                       "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                       "frac": a / FP64_PEAK_TFLOPS,
                       "peak_source": "derived: 2 DFMA/clk/SM x 2 flop x "
                                      "152 SMs x 2.07 GHz",
                       "seconds": sec}
        else:
            a = work / sec / 1e9
            out[nm] = {"bound": "hbm", "achieved": a, "peak": pk["hbm_gbs"],
                       "unit": "GB/s", "frac": a / pk["hbm_gbs"],
                       "peak_source": pk["source"] + " HBM copy",
                       "seconds": sec}
    return out


def run_ours(args, rank, ws):
    import torch
    from paper_2512_21909_gb300 import build as cbuild, cdcc

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    if rank == 0:
        cbuild.build()
    barrier(ws)
    cdcc.load()
    pk = peaks()
    global PLAIN_LADDER
    PLAIN_LADDER = bool(args.plain_ladder)
    lin = not args.no_linearize
    run = Runner(args.config, dev, args.symmetry_ignored)
    s, nx = run.s, run.nx
    # an L2 flush between steps (the workload inputs exceed L2 as well)
    flush = torch.empty(int(512 * 2 ** 20) // 4, dtype=torch.float32,
                        device="cuda")
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        run.one(cdcc, args.precision, linearize=lin)
    torch.cuda.synchronize()

    # ---- device-resident timing (inputs in HBM), L2 flushed between steps
    clk = ClockSampler(dev)
    clk.start()
    barrier(ws)
    torch.cuda.synchronize()
    times, infos, (e, g) = timed_steps(torch, run, cdcc, args.precision,
                                       args.steps, flush, stream, lin)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = clk.stop()
    t50 = allmax(float(np.median(times)), ws)
    t99 = allmax(float(np.percentile(times, 99)), ws)
    classes, lad = class_table(infos, args.steps)
    launches = int(np.mean([i["launches"] for i in infos]))

    # ---- end to end through the C ABI with pinned host buffers
    e2e = []
    if args.e2e_steps > 0:
        L_h, dL_h = run.host()
        for _ in range(max(1, min(args.steps, args.e2e_steps))):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            run.one(cdcc, args.precision, L_h.numpy(), dL_h.numpy(),
                    linearize=lin)
            e2e.append(time.perf_counter() - t0)
    e2e50 = allmax(float(np.median(e2e)), ws) if e2e else None
    h2d = (s.L.nbytes + run.dL.nbytes + s.eps.nbytes + s.orb_irrep.nbytes
           + s.chol_irrep.nbytes)
    d2h = 8 * (nx + 1)

    # ---- other schedules on the same workload (optional)
    other_lines = []
    wanted = ("fp64", "mixed", "tc") if args.others == "all" else \
        tuple(x for x in args.others.split(",") if x and x != "none")
    for other in [p for p in wanted if p != args.precision]:
        run.one(cdcc, other, linearize=lin)
        o_t, o_inf, (o_e, o_g) = timed_steps(torch, run, cdcc, other, 1,
                                             flush, stream, lin)
        ocls, olad = class_table(o_inf, 1)
        other_lines.append({
            "precision": other, "time_to_gradient_s": o_t[0],
            "abs_dE_vs_this_run": abs(o_e - e),
            "max_abs_dg_vs_this_run": float(np.abs(o_g - g).max()),
            "ladder_tflops": olad[1] / olad[0] / 1e12 if olad[0] else None})

    # ---- error report of the --precision schedule (untimed)
    err_est = None
    if args.error_estimate:
        o = cdcc.cdcc_default_options()
        o.precision = prec_code(cdcc, args.precision)
        o.ladder_linearize = 1 if lin else 0
        o.ladder_pm = 0 if PLAIN_LADDER else 1
        ctx = cdcc.cd_ccsd_init(s.nirrep, s.nocc, s.nvir, s.nchol,
                                s.orb_irrep, s.eps, s.chol_irrep, run.L_d,
                                options=o)
        cdcc.gradient(ctx, run.dL_d)
        t0 = time.perf_counter()
        dE, dg = cdcc.cdcc_error_estimate(ctx, run.dL_d)
        err_est = {"dE": dE, "max_dg": float(np.abs(dg).max()),
                   "seconds": time.perf_counter() - t0,
                   "what": "|E64(t)-E(t)| + |<lambda,R64(t)>| and "
                           "|<Gamma64-Gamma, dL>| against FP64 at the "
                           "converged t, lambda"}
        cdcc.cd_ccsd_free(ctx)

    # ---- mixed (this schedule) vs plain FP64 GPU path on the comparison
    # workload, one gradient each after one warm-up of each; the timed
    # workload's inputs leave the device first, so that each schedule picks
    # its ladder mode from the free memory of a dedicated device
    compare = None
    peak_gb = torch.cuda.max_memory_allocated(dev) / 1e9
    if args.compare not in ("none", "") and args.precision != "fp64" \
            and not args.symmetry_ignored:
        cfg2 = int(args.compare)
        if cfg2 != args.config:
            run.L_d = run.dL_d = None
            torch.cuda.empty_cache()
        r2 = run if cfg2 == args.config else Runner(cfg2, dev)
        res = {}
        for p in (args.precision, "fp64"):
            if p != "fp64":
                r2.one(cdcc, p, linearize=lin)   # warm-up (tile tuner, pools)
            t, inf, (ee, gg) = timed_steps(torch, r2, cdcc, p, 1, flush,
                                           stream, lin)
            _, l2 = class_table(inf, 1)
            res[p] = {"time_to_gradient_s": t[0], "e_corr": ee,
                      "ladder_s": l2[0],
                      "ladder_tflops": l2[1] / l2[0] / 1e12 if l2[0] else None,
                      "iterations": inf[0]["solver"], "g": gg}
        a, b = res[args.precision], res["fp64"]
        compare = {
            "workload": WORKLOAD[cfg2],
            args.precision: {k: v for k, v in a.items() if k != "g"},
            "fp64": {k: v for k, v in b.items() if k != "g"},
            "speedup_vs_fp64": b["time_to_gradient_s"] / a["time_to_gradient_s"],
            "abs_dE_vs_fp64": abs(a["e_corr"] - b["e_corr"]),
            "max_abs_dg_vs_fp64": float(np.abs(a["g"] - b["g"]).max()),
            "note": "the FP64 GPU path is not run on the D2h o=60 v=540 "
                    "workload: at its c2 rate (DFMA-bound ladder, 9.6e12 + "
                    "6.4e12 flop per application) it would take about half "
                    "an hour per gradient"}
        del r2

    if rank != 0:
        return
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        try:
            smp = OracleSample(args.config)
            smp.time_blocks(1)               # warm-up, as in the reference arm
            cpu = smp.estimate(1)
            del smp
        except Exception as ex:  # pragma: no cover
            cpu = {"error": str(ex)}
    roof = rooflines(classes, pk)
    dom = max(roof, key=lambda k: roof[k]["seconds"]) if roof else None
    roofline = None
    if dom:
        roofline = dict(roof[dom], kernel=dom, traffic=None,
                        traffic_note="no ncu DRAM capture of this kernel "
                                     "version at this workload")
        if dom in TRAFFIC:
            roofline.update(TRAFFIC[dom])
    info0 = infos[-1]
    out = {
        "metric": METRIC, "value": t50, "unit": "s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t50 * 1e3,
        "p50_s": t50, "p99_s": t99, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": WORKLOAD[args.config] + (
                       " (C1 twin: irreps ignored)" if args.symmetry_ignored
                       else ""),
                   "precision": args.precision,
                   "ladder_linearize": lin,
                   "ladder_pm": not PLAIN_LADDER,
                   "l2": "flushed between steps (512 MiB write); inputs "
                         "larger than L2",
                   "parallelism": "replicas" if ws > 1 else "1 GPU"},
        "e_corr": e, "gradients_per_s": ws / t50,
        "gpu_launches": launches,
        "phases_s": dict(zip(["ccsd", "lambda", "density", "contract_dL"],
                             info0["phases"])),
        "iterations": dict(zip(["ccsd_bf16x3", "ccsd_accurate",
                                "lambda_bf16x3", "lambda_accurate"],
                               info0["solver"])),
        "peak_device_gb": peak_gb,
        "ladder": {"seconds_per_step": lad[0], "flops_per_step": lad[1],
                   "tflops": lad[1] / lad[0] / 1e12 if lad[0] > 0 else None,
                   "share_of_step": lad[0] / t50,
                   "note": "flops of the ladder products as executed "
                           "(with the +/- packing: over canonical ij, ab, cd "
                           "pairs, about a quarter of the plain map's), the "
                           "(ac|bd) builds from L^P_ab and their adjoints"},
        "kernel_classes": classes,
        "roofline": roofline,
        "rooflines": roof,
        "mixed_vs_fp64": compare,
        "other_precisions": other_lines,
        "error_estimate": err_est,
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
    prec = prec_code(cdcc, args.precision)
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
        "dtype": DTYPE[args.precision], "data": "synthetic",
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
                      else "otf", "status": r.status, "e_corr": r.e,
                      "error_dE": r.extra.get("dE")}
                     for r in reqs],
        "clocks": clocks,
    }
    print(json.dumps(out), flush=True)


def run_gemm(args):
    """Time cdcc_dgemm (operand slicing included) on one product shape."""
    import torch
    from paper_2512_21909_gb300 import build as cbuild, cdcc
    cbuild.build()
    cdcc.load()
    f = [int(x) for x in args.gemm.split(",")]
    M, N, K = f[:3]
    ta = f[3] if len(f) > 3 else 0
    tb = f[4] if len(f) > 4 else 1
    modes = [int(x) for x in args.gemm_modes.split(",")]
    A = torch.randn((K, M) if ta else (M, K), dtype=torch.float64,
                    device="cuda")
    B = torch.randn((N, K) if tb else (K, N), dtype=torch.float64,
                    device="cuda")
    C = torch.zeros(M, N, dtype=torch.float64, device="cuda")
    for mode in modes:
        best = None
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            cdcc.cdcc_dgemm(ta, tb, M, N, K, 1.0, A, A.shape[1], B,
                            B.shape[1], 0.0, C, N, mode=mode)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        print(f"M{M} N{N} K{K} ta{ta} tb{tb} mode{mode}: {best * 1e3:.2f} ms "
              f"{2.0 * M * N * K / best / 1e12:.2f} TFLOP/s", flush=True)


def run_ladder_shape(args):
    """Two tensor-core CCSD iterations (ladder on the fly) of a D2h system
    whose ladder batches have the shape of the o=60 v=540 nL=2400 workload:
    8 build products of 4624 x 4624 x 300 per batch, at a small device
    footprint."""
    import torch
    from synth import random_system
    from paper_2512_21909_gb300 import build as cbuild, cdcc
    cbuild.build()
    cdcc.load()
    s = random_system([2] * 8, [68] * 8, [300] * 8, seed=5, scale=0.03)
    o = cdcc.cdcc_default_options()
    o.precision = cdcc.PREC_TC
    o.max_iter = 2
    o.ladder = cdcc.LADDER_OTF
    ctx = cdcc.init_from_system(s, options=o)
    try:
        cdcc.ccsd_solve(ctx)
    except cdcc.CdccError as err:
        if err.status != cdcc.CDCC_ENOCONV:
            raise
    torch.cuda.synchronize()
    print(json.dumps({"ladder_shape_case": "done",
                      "peak_device_gb": torch.cuda.max_memory_allocated()
                      / 1e9}))
    cdcc.cd_ccsd_free(ctx)


def run_cd(args):
    """Two-step CD of the synthetic D2h case: 678 basis functions (230,181
    pairs), a factor of rank 600 per irrep whose spectrum decays so that
    tau = 1e-4 keeps 3770 vectors (the paper: 3710 for this basis size),
    sigma = 1e-2,
    Q_max = 1000 (the paper's parameters); GPU time per decomposition
    (W warm-up runs, then `steps` timed ones), the oracle's time on the
    host, and their comparison (pivots, vectors, sampled residual rows)."""
    import torch
    from synth.cd import make_cd_system
    from paper_2512_21909_gb300 import build as cbuild, cdcc
    cbuild.build()
    cdcc.load()
    s = make_cd_system(678, 8, 600, seed=41, decay=19.5)
    tau, sigma, qmax = 1e-4, 1e-2, 1000
    dB = torch.as_tensor(s.B, device="cuda")
    for _ in range(max(1, args.warmup)):
        cdcc.cd_two_step(s.npair, s.naux, dB, tau, sigma, qmax)
    times, stats = [], None
    for _ in range(max(1, args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        piv, L, stats = cdcc.cd_two_step(s.npair, s.naux, dB, tau, sigma,
                                         qmax)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    ncv = [len(p) for p in piv]
    # second step FP64 work: metric, (Q|rs), K^-1 (Q|rs)
    fl2 = sum(2.0 * q * q * k + 2.0 * q * n * k + 2.0 * q * q * n
              for q, n, k in zip(ncv, s.npair, s.naux))
    peak64 = 2 * 2 * 152 * 2.07e9 / 1e12
    out = {"metric": "two-step CD time (s)", "value": float(np.median(times)),
           "unit": "s", "higher_is_better": False, "steps": len(times),
           "warmup": max(1, args.warmup), "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "two-step CD, D2h, 678 basis functions "
                                  "(230181 pairs), factor rank 600 per irrep, "
                                  "3770 vectors at tau = 1e-4",
                      "tau": tau, "sigma": sigma, "qmax": qmax},
           "ncv": ncv, "ncv_total": int(sum(ncv)),
           "macro_iterations": int(stats[0]),
           "micro_iterations": int(stats[1]),
           "first_step_s": float(stats[2]), "second_step_s": float(stats[3]),
           "roofline_second_step": {
               "bound": "alu", "achieved": fl2 / stats[3] / 1e12,
               "peak": peak64, "unit": "TFLOP/s",
               "frac": fl2 / stats[3] / 1e12 / peak64,
               "peak_source": "derived: 2 DFMA/clk/SM x 2 flop x 152 SMs x "
                              "2.07 GHz"}}
    if not args.no_cpu_baseline:
        from oracle import cd as ocd
        blocks = [s.block(g) for g in range(s.nirrep)]
        t0 = time.perf_counter()
        piv_o, _, _, info = ocd.first_step(blocks, tau, sigma, qmax)
        L_o = ocd.second_step(blocks, piv_o)
        t_o = time.perf_counter() - t0
        rng = np.random.default_rng(0)
        worst = 0.0
        for g in range(s.nirrep):
            B = s.block(g)
            rows = rng.choice(B.shape[0], 16, replace=False)
            R = B[rows] @ B.T - L[g][:, rows].T @ L[g]
            worst = max(worst, float(np.abs(R).max()))
        dl = max(float(np.abs(L[g] - L_o[g]).max()) if L[g].shape ==
                 L_o[g].shape else float("inf") for g in range(s.nirrep))
        out["cpu_baseline"] = {"value": t_o, "unit": "s", "kind": "oracle",
                               "cores": os.cpu_count(),
                               "sample": "the whole decomposition"}
        out["parity"] = {"pivots_equal": piv == piv_o,
                         "max_abs_dL": dl,
                         "max_residual_sampled_rows": worst,
                         "oracle_macro_micro": [info["macro"],
                                                info["micro"]]}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.gemm:
        run_gemm(args)
        return
    if args.cd:
        run_cd(args)
        return
    if args.ladder_shape:
        run_ladder_shape(args)
        return
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
