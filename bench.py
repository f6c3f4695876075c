#!/usr/bin/env python
"""Benchmark of the likelihood + cokriging hot path (arxiv 2008.07437).

Default workload "bivariate-n20000": the parsimonious bivariate Matern model
at n = 20,000 jittered-grid locations (N = 40,000), theta = (1, 1, 0.03, 0.5,
1.5, 0.5), dense FP64 tiled Cholesky (tile 512) whose trailing updates and
panel solves run emulated on the BF16 tensor cores (8 digit slices, FP64-class
accuracy, with the magnitude-aware level cut: ``--oz-cut 0`` turns it off),
plus cokriging of 2,000 held-out locations.  One step = one full
evaluation: Eq. 2 covariance generation, tiled Cholesky, L^-1 Z,
log-determinant and Eq. 1, backward solve and the Eq. 3 predictor at the
2,000 new locations.  Inputs are synthetic: locations from a seeded jittered
grid, Z = L e drawn once at setup from the joint 22,000-location covariance
(the held-out 2,000 give the MSPE).  The same step with native FP64 FMA
updates is timed once beside it (``fp64_dense``: time, l and |dl| / |l|).

Output: one JSON line (rank 0).  ``--impl reference`` times the CPU FP64
oracle on a bounded sample of the same workload instead (this repository has
no other reference implementation: the paper ships no code).

Other workloads (``--workload``): the reduced form at N = 100,000
(bivariate-n50000-mixed), tile low rank at N = 180,000 (trivariate-n60000-tlr;
``--mle K`` runs K Nelder-Mead steps instead, ``--mle-checkpoint F`` saves the
state after every step and resumes from F), serving, batch (also batched
cokriging), mloe, gemm (the emulated FP64 product alone).

Multi-GPU: one process per GPU under torchrun; each rank evaluates its own
replica (independent likelihood evaluations, no collective on the data path);
value = evaluations of all ranks / max over ranks of the timed region.
"""
from __future__ import annotations

import argparse
import ctypes
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2008_07437_gb300 import inputs  # noqa: E402

# FP64 peak derived from unit counts and clock: 152 SMs x 2 FP64 FMA / clock /
# SM x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s for GB300).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# FP32 SIMT peak: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def measured_peaks():
    import json as _json
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return _json.load(f)
    except (OSError, ValueError):
        return {}


# --------------------------------------------------------------------------
# replicas under torchrun: one process per GPU, no collective on the data path
# --------------------------------------------------------------------------
def max_over_ranks(x: float, device) -> float:
    """The largest x over the ranks (the timed region is the slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_over_ranks(obj) -> list:
    """Every rank's obj, in rank order."""
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out


def replica_value(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job throughput: the units all ranks processed / the slowest rank's time."""
    return world * units_per_rank / seconds


# Roofline of each kernel class: (bound, peak, unit, what the peak is).
# The tensor-core classes are timed inside long steps: the sustained bf16 rate.
def class_roofline(cls):
    mp = measured_peaks()
    if cls == "tcgemm":
        if "bf16_tflops_sustained" in mp:
            return ("tensor", float(mp["bf16_tflops_sustained"]),
                    "measured cuBLAS bf16 sustained (FP16 and BF16 MMAs run at the same rate)")
        return "tensor", 1700.0, "fallback 1.7 PFLOP/s bf16 sustained"
    if cls == "sgemm":
        return "alu", FP32_PEAK_TFLOPS, "derived: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz"
    return "alu", FP64_PEAK_TFLOPS, "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz"


KERNEL_NAMES = {"gemm": "k_dgemm_update (FP64 FMA trailing/panel updates)",
                "oz": "k_oz_update (tcgen05 BF16 digit products, exact FP32 accumulation: emulated FP64 "
                      "trailing updates and panel solves)",
                "sgemm": "k_sgemm_nt (FP32 SIMT diagonal/band and panel updates)",
                "tcgemm": "k_tc_update (tcgen05 FP16x2 updates beyond the band)",
                "covgen": "k_covgen_sym (FP64 Matern + Bessel K_nu)"}
TLR_KERNEL_NAMES = {"gemm": "k_bgemm + k_dgemm_update (FP64 low-rank updates of the tile column, diagonal tiles)",
                    "tlr": "k_house_qr + k_jacobi_svd_cl (FP64 compression of the tiles)",
                    "covgen": "k_covgen_block (FP64 Matern + Bessel K_nu)"}
METRIC = "loglik evals/s"


def DENSE_EMULATED(geo):
    """The dense FP64 form with tensor-core emulated updates, 8 slices (FP64-class accuracy)."""
    return geo.opts(nb=512, fp64_gemm=1, oz_slices=8)
UNIT = "evals/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bivariate-n20000",
                    choices=sorted(inputs.WORKLOADS) + ["serving", "batch", "mloe", "estimation", "gemm"])
    ap.add_argument("--n", type=int, default=0, help="override n (profiling runs on small cases only)")
    ap.add_argument("--n-pred", type=int, default=-1)
    ap.add_argument("--nb", type=int, default=0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-n", type=int, default=2000)
    # serving workload
    ap.add_argument("--requests", type=int, default=48, help="serving: requests in the stream")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: mean arrival rate (req/s)")
    ap.add_argument("--slots", type=int, default=4, help="serving: worker threads")
    ap.add_argument("--budget-gb", type=float, default=200.0, help="serving: device-memory budget (GiB)")
    ap.add_argument("--serving-prec", default="mixed", choices=["mixed", "fp64", "emulated"],
                    help="serving form: FP32 off-diagonal tiles (mixed), native FP64, or the 5-slice tensor-core form")
    ap.add_argument("--no-tune", action="store_true", help="serving: skip the tile-size autotuner")
    ap.add_argument("--batch-count", type=int, default=512, help="batch: problems per call")
    ap.add_argument("--mle", type=int, default=0, help="run this many Nelder-Mead steps instead of evaluations")
    ap.add_argument("--mle-checkpoint", default="",
                    help="MLE: save the Nelder-Mead state and the step times here after every step, and resume "
                         "from it when the file exists")
    ap.add_argument("--mle-budget-s", type=float, default=0.0,
                    help="MLE: stop (state saved) before a step that would end after this many seconds")
    ap.add_argument("--profile-lik", action="store_true",
                    help="mle: optimise the profile likelihood (marginal variances estimated, Sec. 4.2)")
    ap.add_argument("--mloe-m", type=int, default=100, help="mloe: prediction locations")
    ap.add_argument("--mloe-form", default="native", choices=["native", "emulated"],
                    help="mloe: FP64 factorisations with native FMA updates or on the tensor cores (8 slices)")
    ap.add_argument("--tlr-tol", type=float, default=0.0, help="tile low-rank accuracy (default: the workload's)")
    ap.add_argument("--est-a", default="0.03,0.09,0.2", help="estimation: range parameters (weak, moderate, strong)")
    ap.add_argument("--replicates", type=int, default=2, help="estimation: simulated fields per range")
    ap.add_argument("--est-full", action="store_true", help="estimation: full likelihood instead of the profile one")
    ap.add_argument("--est-methods", default="exact,TLR5,TLR7,TLR9,DST 40/60,DST 70/30",
                    help="estimation: comma-separated subset of the fits")
    ap.add_argument("--est-budget-s", type=float, default=600.0,
                    help="estimation: start no new MLE run after this many seconds")
    ap.add_argument("--fp64-ref", default="auto", choices=["auto", "on", "off"],
                    help="time one native FP64 step beside a reduced or emulated form (auto: when N <= 50,000)")
    ap.add_argument("--tlr-z", default="model", choices=["model", "white"],
                    help="tile low-rank workloads: Z drawn from the model (dense emulated factor) or white noise")
    ap.add_argument("--tlr-ref", action="store_true",
                    help="tile low-rank workloads: also l at the other accuracy (1e-7 / 1e-9) and the dense "
                         "emulated-FP64 l of the same Z")
    ap.add_argument("--oracle-subset", type=int, default=0,
                    help="also compare l with the oracle on the first this-many locations (0 = off)")
    ap.add_argument("--gemm-mnk", default="8192,8192,512", help="gemm: m,n,k of C -= A B' (FP64 emulated)")
    ap.add_argument("--gemm-slices", type=int, default=8, help="gemm: digit slices")
    ap.add_argument("--oz-cut", type=int, default=-1, choices=[-1, 0, 1],
                    help="emulated FP64 workloads: magnitude-aware level cut in the trailing updates "
                         "(-1: the workload's setting)")
    ap.add_argument("--dst", type=int, default=0,
                    help="tile low-rank workloads: Diagonal Super Tile, keep this many tile diagonals (Sec. 3.4)")
    return ap.parse_args()


def workload(args):
    w = inputs.WORKLOADS[args.workload]
    if args.n:
        w = inputs.Workload(w.name + "-n%d" % args.n, args.n, w.theta, n_pred=w.n_pred, nb=w.nb,
                            loc_seed=w.loc_seed, z_seed=w.z_seed, extra=dict(w.extra))
    if args.n_pred >= 0:
        w.n_pred = args.n_pred
    if args.nb:
        w.nb = args.nb
    if args.tlr_tol > 0 and w.extra.get("prec") == 2:
        w = inputs.Workload(w.name + "-tol%g" % args.tlr_tol, w.n, w.theta, n_pred=w.n_pred, nb=w.nb,
                            loc_seed=w.loc_seed, z_seed=w.z_seed, extra=dict(w.extra, tlr_tol=args.tlr_tol))
    if args.dst > 0 and w.extra.get("prec") == 2:
        w = inputs.Workload(w.name + "-dst%d" % args.dst, w.n, w.theta, n_pred=w.n_pred, nb=w.nb,
                            loc_seed=w.loc_seed, z_seed=w.z_seed, extra=dict(w.extra, dst=args.dst))
    if args.oz_cut >= 0 and w.extra.get("fp64_gemm") == 1 and args.oz_cut != w.extra.get("oz_cut", 0):
        w = inputs.Workload(w.name + ("-cut" if args.oz_cut else "-nocut"), w.n, w.theta, n_pred=w.n_pred, nb=w.nb,
                            loc_seed=w.loc_seed, z_seed=w.z_seed, extra=dict(w.extra, oz_cut=args.oz_cut))
    return w


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------
# CPU oracle on a bounded sample (cpu_baseline and --impl reference)
# --------------------------------------------------------------------------
def oracle_sample_run(w, n_s: int, m_s: int):
    """Time the oracle's phases on the first n_s observed and m_s held-out
    locations; return (extrapolated seconds per full evaluation, details)."""
    import oracle
    oracle.build()
    spec = w.theta
    th = oracle.Theta(list(spec.sigma2), spec.a, list(spec.nu), spec.beta_matrix())
    obs, pred = w.locations()
    n_s = min(n_s, w.n)
    m_s = min(m_s, max(w.n_pred, 0))
    ls, ps = obs[:n_s], pred[:m_s]
    p = spec.p
    Z = inputs.normals(w.z_seed, p * n_s)   # white noise stands in for data: the cost does not depend on it
    t0 = time.perf_counter()
    S = oracle.covgen(th, ls)
    t1 = time.perf_counter()
    L, info = oracle.cholesky(S)
    t2 = time.perf_counter()
    y = oracle.forward(L, Z)
    _ = float(np.sum(np.log(np.diag(L)))) * 2.0 + float(y @ y)
    t3 = time.perf_counter()
    if m_s:
        oracle.predict(th, ls, Z, ps, L=L)
    t4 = time.perf_counter()
    Ns, Nf = p * n_s, p * w.n
    r = Nf / Ns
    t_full = (t1 - t0) * r * r + (t2 - t1) * r ** 3 + (t3 - t2) * r * r
    if m_s and w.n_pred:
        t_full += (t4 - t3) * (w.n / n_s) * (w.n_pred / m_s)
    det = {"sample_s": t4 - t0, "covgen_s": t1 - t0, "cholesky_s": t2 - t1, "solve_s": t3 - t2,
           "predict_s": t4 - t3, "n_sample": n_s, "m_sample": m_s, "info": info}
    return t_full, det


def oracle_full_config0():
    """The oracle's full evaluation of the N = 800 workload (covariance, Cholesky, solve, Eq. 1), timed."""
    import oracle
    oracle.build()
    w0 = inputs.WORKLOADS["bivariate-n400"]
    spec = w0.theta
    th = oracle.Theta(list(spec.sigma2), spec.a, list(spec.nu), spec.beta_matrix())
    locs, _ = w0.locations()
    Z = inputs.normals(w0.z_seed, spec.p * w0.n)
    t0 = time.perf_counter()
    r = oracle.loglik(th, locs, Z)
    t = time.perf_counter() - t0
    # the same on one core
    cores = oracle.num_threads()
    oracle.set_threads(1)
    try:
        t1 = time.perf_counter()
        oracle.loglik(th, locs, Z)
        t_one = time.perf_counter() - t1
    finally:
        oracle.set_threads(cores)
    return {"workload": w0.name, "N": spec.p * w0.n, "seconds": t, "evals_per_s": 1.0 / t, "loglik": r.loglik,
            "cores": cores, "seconds_1_core": t_one}


def host_cpu() -> str:
    """The host's architecture and CPU model (the model name where the kernel reports one, else the
    implementer / part codes of an Arm core)."""
    import platform
    fields = {}
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    fields.setdefault(k.strip(), v.strip())
    except OSError:
        pass
    model = fields.get("model name") or ("implementer %s part %s" % (fields.get("CPU implementer", "?"),
                                                                     fields.get("CPU part", "?")))
    return "%s, %s, %d logical CPUs" % (platform.machine(), model, os.cpu_count() or 0)


def cpu_baseline_json(w, n_s, m_s, t_full, det, cores):
    return {"value": 1.0 / t_full, "unit": UNIT, "cores": cores, "kind": "oracle", "host": host_cpu(),
            "extrapolated": True, "sample_N": w.theta.p * det["n_sample"], "sample_m": det["m_sample"],
            "sample_seconds": det["sample_s"],
            "sample": ("oracle (C, OpenMP, FP64) on the first %d observed + %d held-out locations "
                       "(N = %d), timed: %.1f s; value extrapolated to N = %d by N^3 for the Cholesky, N^2 for "
                       "covariance generation and the solve, n*m for prediction"
                       % (det["n_sample"], det["m_sample"], w.theta.p * det["n_sample"], det["sample_s"],
                          w.theta.p * w.n)),
            "phases_s": {k: round(v, 3) for k, v in det.items() if k.endswith("_s")},
            "config0_full": oracle_full_config0()}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    w = workload(args)
    cores = oracle.num_threads()
    m_s = 200 if w.n_pred else 0
    for _ in range(args.warmup):
        oracle_sample_run(w, args.cpu_sample_n, m_s)
    ts, ss, det = [], [], None
    for _ in range(args.steps):
        t_full, det = oracle_sample_run(w, args.cpu_sample_n, m_s)
        ts.append(t_full)
        ss.append(det["sample_s"])
    t = sum(ts) / len(ts)
    value = 1.0 / t
    # steps / ms_per_step describe what ran: one bounded oracle sample per step;
    # value is the full workload's rate extrapolated from those samples
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(ss) / len(ss),
            "extrapolated": True, "extrapolated_ms_per_eval": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_json(w, args),
            "cpu_baseline": cpu_baseline_json(w, args.cpu_sample_n, m_s, t, det, cores),
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def config_json(w, args):
    p = w.theta.p
    form = "dense FP64 tiled Cholesky"
    if w.extra.get("prec") == 2:
        form = ("tile low-rank: dense FP64 diagonal tiles, off-diagonal tiles U V' at absolute accuracy %g, "
                "rank <= %d (dense beyond)" % (w.extra.get("tlr_tol", 1e-9), w.extra.get("tlr_kmax", 200)))
        if w.extra.get("dst"):
            form = ("Diagonal Super Tile: the %d tile diagonals nearest the diagonal kept dense, the other tiles "
                    "dropped" % w.extra["dst"])
    if w.extra.get("prec") == 1:
        form = ("mixed: FP64 diagonal tiles, FP32 band of %d tiles, %s tensor cores beyond, %d FP64 refinement sweeps"
                % (w.extra.get("band", 4), "BF16" if w.extra.get("lowp") else "FP16x2", w.extra.get("refine_iters", 2)))
    if w.extra.get("fp64_gemm") == 1:
        S = w.extra.get("oz_slices", 8)
        form = ("dense tiled Cholesky, FP64 diagonal tiles (native POTRF and inversion); trailing updates and panel "
                "solves on the BF16 tensor cores: %d 7-bit digit slices per operand row with a power-of-two row "
                "scale, exact FP32 accumulation, FP64 recombination (%s)%s"
                % (S, "FP64-class accuracy" if S >= 8 else "about %d bits per operand" % (7 * S),
                   "; level cut: each trailing-update tile keeps the digit levels its operands' magnitudes need "
                   "against the update's largest rows" if w.extra.get("oz_cut") else ""))
    return {"workload": w.name, "n": w.n, "p": p, "N": p * w.n, "nb": w.nb, "n_pred": w.n_pred,
            "form": form, "theta": {"sigma2": list(w.theta.sigma2), "a": w.theta.a,
                                                           "nu": list(w.theta.nu), "beta": list(w.theta.beta)},
            "l2": ("inputs larger than L2: every tile column (%.1f GB) is regenerated every step" % (
                8.0 * p * w.n * w.nb / 1e9) if w.extra.get("prec") == 2 else
                "inputs larger than L2: the %.1f GB matrix is regenerated every step" % (8.0 * (p * w.n) ** 2 / 1e9)),
            "z": ("white noise (cost does not depend on Z)" if w.extra.get("prec") == 2 and args.tlr_z == "white"
                  else "Z = L e, joint draw" + (" (L: dense emulated-FP64 factor)" if w.extra.get("prec") == 2
                                               else ""))}


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2008_07437_gb300 as geo
    from paper_2008_07437_gb300 import build as gbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    if rank == 0 or world == 1:
        gbuild.build()
    if world > 1:
        dist.barrier()
    dev = torch.device("cuda", torch.cuda.current_device())

    w = workload(args)
    p = w.theta.p
    N = p * w.n
    theta = geo.Theta.from_spec(w.theta)
    o = geo.opts(nb=w.nb, **w.extra)
    ctx = geo.geo_create(dev.index)

    # ---- setup (untimed): locations and one joint draw Z = L e -------------
    # (tile low-rank: the draw needs the dense factor of the full matrix; it
    # is taken with the emulated FP64 form in a context of its own, which is
    # destroyed afterwards so that the dense matrix does not stay cached)
    tlr = w.extra.get("prec") == 2
    obs, pred = w.locations()
    allp = np.vstack([obs, pred])
    e = w.white_noise()
    d_all = torch.as_tensor(allp, device=dev)
    d_e = torch.as_tensor(e, device=dev)
    d_zall = torch.empty(p * len(allp), dtype=torch.float64, device=dev)
    if tlr and args.tlr_z == "white":
        d_zall.copy_(d_e)
    elif tlr:
        sctx = geo.geo_create(dev.index)
        geo.geo_simulate(sctx, d_all, d_e, theta, d_zall, DENSE_EMULATED(geo))
        sctx.close()
    else:   # the draw takes an FP64-class factor whatever form is measured
        geo.geo_simulate(ctx, d_all, d_e, theta, d_zall, DENSE_EMULATED(geo))
    d_locs = torch.as_tensor(obs, device=dev).contiguous()
    d_pred = torch.as_tensor(pred, device=dev).contiguous()
    d_z = d_zall[:N].clone()
    z_true_pred = d_zall[N:].cpu().numpy()
    d_zhat = torch.empty(p * w.n_pred, dtype=torch.float64, device=dev)
    del d_all, d_e, d_zall

    if args.mle:
        return run_mle(args, w, ctx, d_locs, d_z, theta, o, dev)

    tlr_stats = {}

    def step():
        ll, fac = geo.geo_loglik(ctx, d_locs, d_z, theta, o, keep=True)
        if w.n_pred:
            geo.geo_predict(ctx, fac, d_pred, d_zhat)
        if tlr:
            fs = geo.geo_factor_stats_get(fac)
            tlr_stats.update(max_rank=fs.tlr_max_rank, dense_tiles=fs.tlr_dense_tiles,
                             bytes_vs_dense=fs.tlr_bytes_ratio)
        fac.free()
        return ll

    for _ in range(args.warmup):
        ll = step()
    torch.cuda.synchronize()

    # ---- timed region: inputs resident in HBM -----------------------------
    clocks = ClockSampler(dev.index)
    geo.geo_profile_enable(ctx, True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        ll = step()
    ev1.record()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = geo.geo_profile_read(ctx)
    geo.geo_profile_enable(ctx, False)
    ms = max_over_ranks(ms, dev)
    if world > 1:
        dist.barrier()
    zhat = d_zhat.cpu().numpy()
    mspe = float(np.mean(np.sum((zhat - z_true_pred).reshape(-1, p) ** 2, axis=1))) if w.n_pred else None

    # ---- end to end through the C ABI with host buffers -------------------
    e2e = None
    if not args.no_e2e:
        h_locs = torch.as_tensor(obs).pin_memory()
        h_z = d_z.cpu().pin_memory()
        h_pred = torch.as_tensor(pred).pin_memory()
        h_zhat = torch.empty(p * w.n_pred, dtype=torch.float64).pin_memory()
        e_locs = torch.empty_like(d_locs)
        e_z = torch.empty_like(d_z)
        e_pred = torch.empty_like(d_pred)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e_locs.copy_(h_locs, non_blocking=True)
            e_z.copy_(h_z, non_blocking=True)
            e_pred.copy_(h_pred, non_blocking=True)
            ll_e, fac = geo.geo_loglik(ctx, e_locs, e_z, theta, o, keep=True)
            if w.n_pred:
                geo.geo_predict(ctx, fac, e_pred, d_zhat)
                h_zhat.copy_(d_zhat, non_blocking=True)
            fac.free()
            torch.cuda.synchronize()
        t_e2e = max_over_ranks(time.perf_counter() - t0, dev)
        e2e = {"value": replica_value(args.steps, t_e2e, world), "unit": UNIT,
               "h2d_bytes_per_step": 8 * (2 * w.n + N + 2 * w.n_pred),
               "d2h_bytes_per_step": 8 * (p * w.n_pred + 1)}

    # ---- native FP64 beside a reduced or emulated form (same step, same inputs) ----
    emulated = w.extra.get("fp64_gemm") == 1
    fp64_dense = None
    want_ref = args.fp64_ref == "on" or (args.fp64_ref == "auto" and (emulated or w.extra.get("prec") == 1)
                                         and N <= 100000 and not tlr)
    if want_ref and (rank == 0 or world == 1):
        o_nat = geo.opts(nb=960)
        if N <= 50000:   # warm-up of the native kernels (negligible against a step beyond that)
            ll_ref, fac = geo.geo_loglik(ctx, d_locs, d_z, theta, o_nat, keep=True)
            fac.free()
        geo.geo_profile_enable(ctx, True)
        torch.cuda.synchronize()
        r0 = torch.cuda.Event(enable_timing=True)
        r1 = torch.cuda.Event(enable_timing=True)
        r0.record()
        ll_ref, fac = geo.geo_loglik(ctx, d_locs, d_z, theta, o_nat, keep=True)
        if w.n_pred:
            geo.geo_predict(ctx, fac, d_pred, d_zhat)
        fac.free()
        r1.record()
        torch.cuda.synchronize()
        pref = geo.geo_profile_read(ctx)
        geo.geo_profile_enable(ctx, False)
        ms_ref = r0.elapsed_time(r1)
        g = pref["gemm"]
        fp64_dense = {"form": "native FP64 FMA updates, tile 960", "ms_per_step": ms_ref,
                      "evals_per_s": 1e3 / ms_ref, "loglik": ll_ref,
                      "rel_dl": abs(ll - ll_ref) / abs(ll_ref),
                      "speedup": ms_ref / (ms / args.steps),
                      "k_dgemm_update_frac_of_fp64_peak": (g["flops"] / (g["ms"] * 1e-3) / 1e12 / FP64_PEAK_TFLOPS
                                                           if g["ms"] > 0 else None)}
    tlr_accuracy = None
    if tlr and args.tlr_ref and (rank == 0 or world == 1):
        tol = w.extra.get("tlr_tol", 1e-9)
        other = 1e-7 if tol < 1e-8 else 1e-9
        o_other = geo.opts(nb=w.nb, **dict(w.extra, tlr_tol=other))
        t0 = time.perf_counter()
        ll_other, _ = geo.geo_loglik(ctx, d_locs, d_z, theta, o_other)
        t_other = time.perf_counter() - t0
        ctx.close()   # release the TLR workspaces before the dense matrix
        dctx = geo.geo_create(dev.index)
        t0 = time.perf_counter()
        ll_dense, _ = geo.geo_loglik(dctx, d_locs, d_z, theta, DENSE_EMULATED(geo))
        t_dense = time.perf_counter() - t0
        dctx.close()
        ctx = geo.geo_create(dev.index)
        tlr_accuracy = {"reference": "dense FP64 form, tensor-core emulated updates (8 slices)",
                        "loglik_dense": ll_dense, "dense_seconds": t_dense,
                        "tol": tol, "loglik": ll, "rel_dl_vs_dense": abs(ll - ll_dense) / abs(ll_dense),
                        "other_tol": other, "loglik_other": ll_other, "other_seconds": t_other,
                        "rel_dl_other_vs_dense": abs(ll_other - ll_dense) / abs(ll_dense)}
    oracle_subset = None
    if args.oracle_subset > 0 and (rank == 0 or world == 1):
        import oracle
        k = min(args.oracle_subset, w.n)
        spec = w.theta
        th_o = oracle.Theta(list(spec.sigma2), spec.a, list(spec.nu), spec.beta_matrix())
        zs = d_z[: p * k].cpu().numpy()
        t0 = time.perf_counter()
        ref_sub = oracle.loglik(th_o, obs[:k], zs).loglik
        t_or = time.perf_counter() - t0
        ll_sub, _ = geo.geo_loglik(ctx, d_locs[:k].contiguous(), d_z[: p * k].contiguous(), theta,
                                   geo.opts(nb=min(w.nb, 256) if emulated else 256, **w.extra))
        oracle_subset = {"n": k, "N": p * k, "loglik_gpu": ll_sub, "loglik_oracle": ref_sub,
                         "rel_dl": abs(ll_sub - ref_sub) / abs(ref_sub), "oracle_seconds": t_or}

    # ---- report ------------------------------------------------------------
    launches = sum(v["launches"] for v in prof.values())
    # dominant kernel class of the step and its roofline
    dom = max(("gemm", "sgemm", "tcgemm", "covgen", "tlr"), key=lambda k: prof[k]["ms"])
    dk = prof[dom]
    bound, peak, peak_src = class_roofline(dom)
    dom_tflops = dk["flops"] / (dk["ms"] * 1e-3) / 1e12 if dk["ms"] > 0 and dk["flops"] > 0 else 0.0
    fp64eq_tflops = None
    kname = (TLR_KERNEL_NAMES if tlr else KERNEL_NAMES).get(dom, dom)
    if dom == "tcgemm" and emulated:
        # the class counts FP64-equivalent flops (2 K per output); the tensor-core work is
        # what the kernels issued (counted on the device): S (S + 1) / 2 digit products of
        # that size per output without the level cut, fewer with it
        fp64eq_tflops = dom_tflops
        dom_tflops = dk["tensor_flops"] / (dk["ms"] * 1e-3) / 1e12 if dk["ms"] > 0 else 0.0
        kname = KERNEL_NAMES["oz"]
    # Cholesky rate: N^3 / 3 over the step's time outside covariance generation,
    # reductions, solves and prediction (the lookahead overlaps the classes)
    other = sum(prof[k]["ms"] for k in ("covgen", "reduce", "solve", "predict")) / args.steps
    chol_ms = max(ms / args.steps - other, 1e-9)
    chol_tflops = (N ** 3 / 3.0) / (chol_ms * 1e-3) / 1e12
    # DRAM bytes per launch: an ncu capture of a full rank-960 trailing update
    # (N = 8,000) measured 0.822 x the algorithmic bytes; scaled to this run's
    # average launch (FP64 update kernel only)
    traffic = 0.822 * dk["bytes"] / max(dk["launches"], 1) if dom == "gemm" and not tlr else None
    if dom == "tcgemm" and emulated and w.extra.get("oz_cut") and w.extra.get("oz_slices", 8) == 8:
        # k_oz_update with the level cut: an ncu capture of every launch of one evaluation at
        # N = 16,000 measured DRAM read + write = 0.967 x the algorithmic bytes the library counts
        # (16 B per output written, the digit slices); scaled to this run's launches (8 slices, the
        # captured kernel; other slice counts have no capture: null)
        traffic = 0.967 * dk["bytes"] / max(dk["launches"], 1)
    dtype = "f64"
    if emulated:
        dtype = "f64 (emulated: bf16 digit products, exact fp32 accumulation, %d slices)" % w.extra.get("oz_slices", 8)
    out = {"metric": METRIC, "value": replica_value(args.steps, ms * 1e-3, world), "unit": UNIT, "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
           "data": "synthetic", "config": config_json(w, args),
           "cholesky_tflops": None if tlr else chol_tflops,
           "dense_equivalent_tflops": chol_tflops if tlr else None,
           "roofline": {"bound": bound, "kernel": kname,
                        "achieved": dom_tflops, "peak": peak,
                        "unit": "TFLOP/s", "frac": dom_tflops / peak, "peak_source": peak_src,
                        "traffic": traffic, "fp64_equivalent_tflops": fp64eq_tflops,
                        "algorithmic_bytes_per_launch": dk["bytes"] / max(dk["launches"], 1)},
           "gpu_launches": launches,
           "phases_ms_per_step": {k: v["ms"] / args.steps for k, v in prof.items()},
           "quality": {"loglik": ll, "mspe": mspe},
           "fp64_dense": fp64_dense, "oracle_subset": oracle_subset, "tlr_accuracy": tlr_accuracy,
           "tlr_factor": tlr_stats or None,
           "clocks": clk, "e2e": e2e}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        m_s = 200 if w.n_pred else 0
        t_full, det = oracle_sample_run(w, args.cpu_sample_n, m_s)
        out["cpu_baseline"] = cpu_baseline_json(w, args.cpu_sample_n, m_s, t_full, det, oracle.num_threads())
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------------
# serving: a Poisson stream of likelihood and cokriging requests
# --------------------------------------------------------------------------
SERVING_METRIC = "serving latency p50 (ms; p99 beside)"


def serving_opts(geo, prec):
    if prec == "fp64":
        return geo.opts(nb=0), "dense FP64"
    if prec == "emulated":
        return (geo.opts(nb=0, fp64_gemm=1, oz_slices=5),
                "FP64 diagonal tiles; every other tile's update and panel solve on the BF16 tensor cores, 5 digit "
                "slices (about 35 bits per operand, exact FP32 accumulation); no refinement, no FP64 re-run")
    return (geo.opts(nb=0, prec=1, band=1 << 20, refine_iters=2),
            "FP64 diagonal tiles, FP32 off-diagonal tiles (FP32 TRSM and updates), 2 FP64 refinement sweeps; "
            "run again in FP64 when the reduced form is not positive definite")


def serving_config(args, stream, form, tuned):
    nl = [r.n for r in stream if r.kind == "loglik"]
    return {"workload": "serving", "stream": "Poisson, mean %.0f req/s, seed 3000 + rank" % args.rate,
            "requests": len(stream), "loglik_requests": len(nl),
            "predict_requests": len(stream) - len(nl), "p": 2,
            "n_range": [1000, 20000], "m_range": [100, 2000], "form": form, "slots": args.slots,
            "hbm_budget_gib": args.budget_gb, "tuned_nb": tuned,
            "theta_box": "a in [0.03, 0.2], nu_i in [0.5, 1.5], beta in [-0.7, 0.7], sigma^2_i in [0.5, 2]",
            "z": "seeded standard normals (cost does not depend on Z)",
            "l2": "inputs larger than L2: every likelihood generates its own %d-%d MB matrix" % (
                8 * (2 * 1000) ** 2 // 2 ** 20, 8 * (2 * 20000) ** 2 // 2 ** 20)}


def fifo_latencies(arrivals, service, servers=1):
    """Latencies of a first-come first-served queue with identical servers."""
    import heapq
    free = [0.0] * servers
    out = []
    for a, sv in zip(arrivals, service):
        t = heapq.heappop(free)
        end = max(a, t) + sv
        heapq.heappush(free, end)
        out.append(end - a)
    return out


def serving_cpu_model(stream, n_s=1000, m_s=200):
    """Oracle service time per request, from one timed oracle evaluation at
    n_s locations (+ m_s predictions), extrapolated per request by N^3 / N^2 / n m."""
    import oracle
    w = inputs.Workload("serving-sample", n_s, inputs.THETA_FIG5, n_pred=m_s, nb=256, loc_seed=3999, z_seed=3998)
    _, det = oracle_sample_run(w, n_s, m_s)
    service = []
    for r in stream:
        if r.kind == "loglik":
            q = r.n / n_s
            service.append(det["covgen_s"] * q * q + det["cholesky_s"] * q ** 3 + det["solve_s"] * q * q)
        else:
            service.append(det["predict_s"] * (r.m / m_s))
    return service, det, oracle.num_threads()


def serving_cpu_json(stream, service, det, cores):
    lat = fifo_latencies([r.t_arrival for r in stream], service, 1)
    span = max(r.t_arrival + v for r, v in zip(stream, lat)) - stream[0].t_arrival
    return {"value": float(np.percentile(lat, 50)) * 1e3, "unit": "ms", "cores": cores, "kind": "oracle",
            "p99_ms": float(np.percentile(lat, 99)) * 1e3, "throughput_req_s": len(stream) / span,
            "sample": ("oracle (C, OpenMP, FP64) timed once at n = %d (N = %d) + %d predictions in %.1f s; each "
                       "request's service time extrapolated (N^3 Cholesky, N^2 generation and solve, m for "
                       "cokriging on a kept factor), the stream replayed through a one-server FIFO queue"
                       % (det["n_sample"], 2 * det["n_sample"], det["m_sample"], det["sample_s"]))}


def run_serving(args):
    import torch
    import torch.distributed as dist

    import paper_2008_07437_gb300 as geo
    from paper_2008_07437_gb300 import build as gbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    if rank == 0 or world == 1:
        gbuild.build()
    if world > 1:
        dist.barrier()
    dev = torch.device("cuda", torch.cuda.current_device())

    stream = inputs.serving_stream(args.requests, rate=args.rate, seed=3000 + rank)
    o, form = serving_opts(geo, args.serving_prec)
    # host inputs, prepared before the timed region
    prep = {}
    for r in stream:
        if r.kind == "loglik":
            prep[r.k] = (r.locations(), r.observations(), geo.Theta.from_spec(r.theta))
        else:
            prep[r.k] = r.new_locations()

    # tile sizes for the reduced form, one per order bucket of the stream (untimed)
    tuned = {}
    ctx = geo.geo_create(dev.index)
    if args.serving_prec != "fp64" and not args.no_tune:
        th_t = geo.Theta.from_spec(inputs.THETA_FIG5)
        by_bucket = {}
        for r in stream:
            if r.kind == "loglik":
                b = (2 * r.n).bit_length() - 1
                if r.n > by_bucket.get(b, 0):
                    by_bucket[b] = r.n
        for b, n in sorted(by_bucket.items()):
            locs = inputs.jittered_grid(n, 3997)
            dl = torch.as_tensor(locs, device=dev)
            dz = torch.as_tensor(inputs.normals(3996, 2 * n), device=dev)
            cands = ([c for c in (256, 512, 768) if c <= 2 * n] if args.serving_prec == "emulated"
                     else [c for c in (256, 512, 1024) if c <= 2 * n]) or [256]
            best, _ = geo.geo_autotune_nb(ctx, dl, dz, th_t, cands, o)
            tuned["N>=%d" % (1 << b)] = best

    srv = geo.Server(dev.index, int(args.budget_gb * 2 ** 30), args.slots)

    def collect(want, timeout=3600.0):
        got, t0 = {}, time.time()
        while len(got) < len(want) and time.time() - t0 < timeout:
            for x in srv.poll(256, wait_ms=100):
                if x["id"] in want:
                    got[x["id"]] = x
        return got

    # warm-up: small likelihoods on every worker
    wids = {}
    for i in range(max(args.warmup, 1) * args.slots):
        wr = inputs.ServingRequest(10 ** 6 + i, 0.0, "loglik", n=1000, theta=inputs.THETA_FIG5)
        wids[srv.submit_loglik(wr.locations(), wr.observations(), geo.Theta.from_spec(wr.theta), o,
                               escalate=args.serving_prec == "mixed")] = wr
    collect(wids)
    torch.cuda.synchronize()
    launches0 = sum(v["launches"] for v in srv.profile().values())

    # ---- timed region: the open-loop stream -------------------------------
    clocks = ClockSampler(dev.index)
    if world > 1:
        dist.barrier()
    clocks.start()
    t0 = time.perf_counter()
    ids = {}
    for r in stream:
        delay = t0 + r.t_arrival - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        if r.kind == "loglik":
            locs, z, th = prep[r.k]
            rid = srv.submit_loglik(locs, z, th, o, dataset=r.dataset, keep=r.keep,
                                    escalate=args.serving_prec == "mixed")
        else:
            rid, _ = srv.submit_predict(r.dataset, prep[r.k], 2, release=r.release)
        ids[rid] = r
    res = collect(ids)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = sum(v["launches"] for v in srv.profile().values()) - launches0
    srv.close()

    rows = []
    for rid, r in ids.items():
        x = res.get(rid)
        if x is None:
            continue
        rows.append((r, x))
    lat = [x["t_end"] - x["t_submit"] for _, x in rows]
    svc = [x["t_end"] - x["t_start"] for _, x in rows]
    span = max(x["t_end"] for _, x in rows) - min(x["t_submit"] for _, x in rows)
    n_ll = sum(1 for r, x in rows if r.kind == "loglik" and x["status"] == 0)
    escalated = sum(1 for r, x in rows if r.kind == "loglik" and x["prec"] == 0 and args.serving_prec == "mixed")
    failed = sum(1 for _, x in rows if x["status"] != 0)
    lat_k = {k: [x["t_end"] - x["t_submit"] for r, x in rows if r.kind == k] for k in ("loglik", "predict")}
    allv = gather_over_ranks({"lat": lat, "span": span, "n": len(rows), "n_ll": n_ll, "launches": launches})
    lat = [v for a in allv for v in a["lat"]]
    span = max(a["span"] for a in allv)
    total, n_ll = sum(a["n"] for a in allv), sum(a["n_ll"] for a in allv)
    launches = sum(a["launches"] for a in allv)

    # accuracy of the served reduced form: |dl| / |l| against FP64 on Z drawn
    # from the model, at the theta and locations of the smallest served likelihoods
    acc = None
    if args.serving_prec != "fp64":
        acc = []
        served_reduced = (lambda x: x["prec"] == 1) if args.serving_prec == "mixed" else (lambda x: x["status"] == 0)
        small = sorted((r for r, x in rows if r.kind == "loglik" and served_reduced(x)), key=lambda r: r.n)[:3]
        for r in small:
            locs, _, th = prep[r.k]
            dl = torch.as_tensor(locs, device=dev)
            de = torch.as_tensor(inputs.normals(45000 + r.k, 2 * r.n), device=dev)
            dz = torch.empty(2 * r.n, dtype=torch.float64, device=dev)
            geo.geo_simulate(ctx, dl, de, th, dz, geo.opts(nb=0))
            l64, _ = geo.geo_loglik(ctx, dl, dz, th, geo.opts(nb=0))
            try:
                lmx, _ = geo.geo_loglik(ctx, dl, dz, th, o)
                acc.append({"n": r.n, "rel": abs(lmx - l64) / abs(l64)})
            except geo.GeoError as e:
                acc.append({"n": r.n, "rel": None, "status": e.code})
    ctx.close()

    p50, p99 = float(np.percentile(lat, 50)) * 1e3, float(np.percentile(lat, 99)) * 1e3
    h2d = sum(32 * r.n if r.kind == "loglik" else 16 * r.m for r in stream) / len(stream)
    d2h = sum(16 * r.m if r.kind == "predict" else 8 for r in stream) / len(stream)
    out = {"metric": SERVING_METRIC, "value": p50, "unit": "ms", "n_gpus": world, "steps": total,
           "warmup": max(args.warmup, 1) * args.slots, "ms_per_step": span * 1e3 / max(total, 1),
           "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": {"mixed": "f64+f32", "fp64": "f64", "emulated": "f64 (emulated: bf16 digit products, 5 slices)"}[
               args.serving_prec], "data": "synthetic",
           "config": serving_config(args, stream, form, tuned),
           "p50_ms": p50, "p99_ms": p99,
           "p50_ms_by_kind": {k: float(np.percentile(v, 50)) * 1e3 for k, v in lat_k.items() if v},
           "p99_ms_by_kind": {k: float(np.percentile(v, 99)) * 1e3 for k, v in lat_k.items() if v},
           "service_p50_ms": float(np.percentile(svc, 50)) * 1e3, "service_p99_ms": float(np.percentile(svc, 99)) * 1e3,
           "throughput_req_s": total / span, "loglik_evals_s": n_ll / span, "offered_req_s": args.rate * world,
           "makespan_s": span, "escalated_to_fp64": escalated, "failed": failed,
           "accuracy_vs_fp64": acc, "gpu_launches": launches, "clocks": clk,
           "roofline": None,
           "e2e": {"value": p50, "unit": "ms", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "note": "the served latency is already end to end: host inputs, copies and the result read"}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        service, det, cores = serving_cpu_model(stream)
        out["cpu_baseline"] = serving_cpu_json(stream, service, det, cores)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------------
# MLE: Nelder-Mead steps (Sec. 5.1) on the workload's data and form
# --------------------------------------------------------------------------
def theta_rel_error(best, spec):
    """|estimate - truth| / |truth| per parameter (beta: absolute error)."""
    p = spec.p
    bt = np.asarray(best.beta, dtype=np.float64).reshape(p, p)
    true_b = list(spec.beta) if p > 1 else []
    est_b = [float(bt[i, j]) for i in range(p) for j in range(i + 1, p)]
    return {"sigma2": [abs(e - t) / t for e, t in zip(best.sigma2, spec.sigma2)],
            "a": abs(best.a - spec.a) / spec.a,
            "nu": [abs(e - t) / t for e, t in zip(best.nu, spec.nu)],
            "beta_abs": [abs(e - t) for e, t in zip(est_b, true_b)]}


def _mle_load(path, geo):
    """Nelder-Mead state and step records saved by an earlier run, or None."""
    if not path or not os.path.exists(path):
        return None, []
    with open(path, "rb") as f:
        blob = f.read()
    size = ctypes.sizeof(geo.geo_mle_state)
    st = geo.geo_mle_state.from_buffer_copy(blob[:size])
    return st, json.loads(blob[size:].decode())


def _mle_save(path, st, records):
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        f.write(bytes(st))
        f.write(json.dumps(records).encode())
    os.replace(tmp, path)


def run_mle(args, w, ctx, d_locs, d_z, theta, o, dev):
    import torch

    import paper_2008_07437_gb300 as geo
    spec = w.theta
    # start: a x 1.3, nu x 0.9, sigma^2 x 1.1, beta x 0.8
    th0 = geo.Theta(tuple(1.1 * v for v in spec.sigma2), 1.3 * spec.a, tuple(0.9 * v for v in spec.nu),
                    tuple(0.8 * v for v in spec.beta) if spec.p > 1 else None)
    st, records = _mle_load(args.mle_checkpoint, geo)
    resumed = len(records)
    if st is None:
        st = geo.geo_mle_init(th0, profile=args.profile_lik)
    ll_true, _ = geo.geo_loglik(ctx, d_locs, d_z, theta, o)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    clocks.start()
    t_call = time.perf_counter()
    while len(records) < args.mle:
        if args.mle_budget_s > 0 and records:
            # the first step evaluates the whole starting simplex: the later ones take one to a few
            # evaluations (a rare shrink more, and the per-step checkpoint bounds what it can lose)
            later = [r["seconds"] for r in records if r["step"] > 1]
            guess = max(later) if later else records[0]["seconds"] / max(records[0]["evals"], 1) * 2
            if time.perf_counter() - t_call + guess > args.mle_budget_s:
                break
        t0 = time.perf_counter()
        ev0 = st.evals
        geo.geo_mle_step(ctx, st, d_locs, d_z, o)
        torch.cuda.synchronize()
        records.append({"step": len(records) + 1, "seconds": time.perf_counter() - t0,
                        "evals": st.evals - ev0, "best_loglik": geo.geo_mle_best(st)[1]})
        if args.mle_checkpoint:
            _mle_save(args.mle_checkpoint, st, records)
        print("mle step %d: %.1f s, %d evaluations, best %.6f" % (
            records[-1]["step"], records[-1]["seconds"], records[-1]["evals"], records[-1]["best_loglik"]),
            file=sys.stderr, flush=True)
    clk = clocks.stop()
    t = sum(r["seconds"] for r in records)
    best, ll = geo.geo_mle_best(st)
    out = {"metric": "MLE wall time", "value": t, "unit": "s", "n_gpus": 1, "steps": len(records), "warmup": 0,
           "ms_per_step": 1e3 * t / max(len(records), 1), "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_json(w, args),
           "complete": len(records) >= args.mle, "steps_requested": args.mle,
           "resumed_after_step": resumed,
           "evals": st.evals, "evals_per_s": st.evals / t if t > 0 else None, "loglik_at_truth": ll_true,
           "best_loglik": ll, "best_loglik_by_step": [r["best_loglik"] for r in records],
           "seconds_by_step": [r["seconds"] for r in records], "evals_by_step": [r["evals"] for r in records],
           "best_theta": {"sigma2": list(best.sigma2), "a": best.a, "nu": list(best.nu),
                          "beta": [float(b) for b in np.asarray(best.beta).ravel()]},
           "start_theta": {"sigma2": list(th0.sigma2), "a": th0.a, "nu": list(th0.nu)},
           "objective": "profile" if args.profile_lik else "full",
           "theta_rel_error": theta_rel_error(best, spec),
           "clocks": clk}
    print(json.dumps(out), flush=True)
    ctx.close()
    return 0


# --------------------------------------------------------------------------
# batch: many small uneven likelihoods per call
# --------------------------------------------------------------------------
def predict_batch_sample(ctx, items, dev, count=128, m=100, reps=5):
    """Cokriging on `count` resident factors (m new locations each): one
    geo_predict_batch launch against one geo_predict call per factor."""
    import torch

    import paper_2008_07437_gb300 as geo
    facs, entries = [], []
    for k, (dl, dz, th) in enumerate(items[:count]):
        facs.append(geo.geo_loglik(ctx, dl, dz, th, geo.opts(nb=128), keep=True)[1])
        new = torch.as_tensor(inputs.jittered_grid(m, 5100 + k), device=dev)
        entries.append((facs[-1], new, torch.empty(2 * m, dtype=torch.float64, device=dev)))
    geo.geo_predict_batch(ctx, entries)          # weights Sigma^-1 Z computed here, untimed
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(reps):
        geo.geo_predict_batch(ctx, entries)
    ev1.record()
    torch.cuda.synchronize()
    t_batch = ev0.elapsed_time(ev1) * 1e-3 / reps
    got = [z.clone() for _, _, z in entries]
    ev0.record()
    for _ in range(reps):
        for f, new, z in entries:
            geo.geo_predict(ctx, f, new, z)
    ev1.record()
    torch.cuda.synchronize()
    t_single = ev0.elapsed_time(ev1) * 1e-3 / reps
    same = all(torch.equal(a, z) for a, (_, _, z) in zip(got, entries))
    for f in facs:
        f.free()
    return {"factors": count, "new_locations_each": m, "predictions_s": count * m / t_batch,
            "predictions_s_one_call_per_factor": count * m / t_single, "bit_identical": same,
            "timing": "CUDA events, mean of %d calls, factors resident" % reps}


def run_batch(args):
    import torch
    import torch.distributed as dist

    import paper_2008_07437_gb300 as geo
    from paper_2008_07437_gb300 import build as gbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    if rank == 0 or world == 1:
        gbuild.build()
    if world > 1:
        dist.barrier()
    dev = torch.device("cuda", torch.cuda.current_device())
    probs = inputs.batch_problems(args.batch_count, seed=3100 + rank)
    ctx = geo.geo_create(dev.index)
    # setup (untimed): locations and Z = L e for every problem
    items, host = [], []
    for n, th_spec, ls, zs in probs:
        th = geo.Theta.from_spec(th_spec)
        locs = inputs.jittered_grid(n, ls)
        dl = torch.as_tensor(locs, device=dev)
        de = torch.as_tensor(inputs.normals(zs, 2 * n), device=dev)
        dz = torch.empty(2 * n, dtype=torch.float64, device=dev)
        geo.geo_simulate(ctx, dl, de, th, dz, geo.opts(nb=128))
        items.append((dl, dz, th))
        host.append((locs, dz.cpu().numpy()))
    Ntot3 = sum((2.0 * n) ** 3 / 3.0 for n, _, _, _ in probs)
    for _ in range(args.warmup):
        geo.geo_loglik_batch(ctx, items)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    geo.geo_profile_enable(ctx, True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        vals, info = geo.geo_loglik_batch(ctx, items)
    ev1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    prof = geo.geo_profile_read(ctx)
    geo.geo_profile_enable(ctx, False)
    ms = max_over_ranks(ms, dev)
    # the same problems one geo_loglik call at a time (context, not the metric)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    single = [geo.geo_loglik(ctx, dl, dz, th, geo.opts(nb=128))[0] for dl, dz, th in items]
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    worst = max(abs(a - b) / abs(b) for a, b in zip(vals, single))
    pred = predict_batch_sample(ctx, items, dev) if rank == 0 else None
    # end to end: host inputs copied every step, results read back
    e2e = None
    if not args.no_e2e:
        pinned = [(torch.as_tensor(l).pin_memory(), torch.as_tensor(z).pin_memory()) for l, z in host]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for (hl, hz), (dl, dz, _) in zip(pinned, items):
                dl.copy_(hl, non_blocking=True)
                dz.copy_(hz, non_blocking=True)
            geo.geo_loglik_batch(ctx, items)   # returns host results (synchronises)
        t_e2e = max_over_ranks(time.perf_counter() - t0, dev)
        e2e = {"value": replica_value(args.steps * len(items), t_e2e, world), "unit": UNIT,
               "h2d_bytes_per_step": sum(8 * 4 * n for n, _, _, _ in probs),
               "d2h_bytes_per_step": 8 * len(items)}
    launches = sum(v["launches"] for v in prof.values())
    dom = max(("gemm", "covgen", "potrf", "trsm"), key=lambda k: prof[k]["ms"])
    bound, peak, peak_src = class_roofline("gemm")
    tflops = (Ntot3 * args.steps) / (ms * 1e-3) / 1e12
    out = {"metric": METRIC, "value": replica_value(args.steps * len(items), ms * 1e-3, world), "unit": UNIT,
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "batch", "problems": len(items), "p": 2, "n_range": [50, 1000],
                      "theta_box": "a in [0.03, 0.2], nu_i in [0.5, 1.5], beta in [-0.7, 0.7], sigma^2_i in [0.5, 2]",
                      "form": "dense FP64, one persistent launch over the units of every problem (progress counters, bounded waits), CUDA graph replay",
                      "l2": "inputs larger than L2: %.1f GB of matrices regenerated every step" % (
                          sum(8.0 * (2 * n) ** 2 for n, _, _, _ in probs) / 1e9)},
           "dense_equivalent_tflops": tflops,
           "roofline": {"bound": bound, "kernel": "whole batch (N^3/3 per problem over the call's time)",
                        "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                        "peak_source": peak_src, "traffic": None},
           "gpu_launches": launches, "dominant_class": dom,
           "phases_ms_per_step": {k: v["ms"] / args.steps for k, v in prof.items()},
           "single_call_evals_s": len(items) / t_single, "max_rel_diff_vs_single": worst,
           "predict_batch": pred, "clocks": clk, "e2e": e2e}
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------------
# MLOE / MMOM (Eq. 5 - Eq. 8, Algorithm 1) on the bivariate n = 20,000 locations
# --------------------------------------------------------------------------
def mloe_setup(args):
    w = inputs.WORKLOADS["bivariate-n20000"]
    n = args.n or w.n
    allp = inputs.jittered_grid(n + args.mloe_m, w.loc_seed)
    spec = w.theta
    th_a = inputs.ThetaSpec(tuple(1.1 * v for v in spec.sigma2), 1.2 * spec.a, tuple(0.9 * v for v in spec.nu),
                            tuple(0.8 * b for b in spec.beta))
    return w, n, allp[:n], allp[n:], spec, th_a


def mloe_config(args, n, spec, th_a):
    return {"workload": "mloe", "n": n, "p": 2, "N": 2 * n, "m": args.mloe_m,
            "theta_t": {"sigma2": list(spec.sigma2), "a": spec.a, "nu": list(spec.nu), "beta": list(spec.beta)},
            "theta_a": {"sigma2": list(th_a.sigma2), "a": th_a.a, "nu": list(th_a.nu), "beta": list(th_a.beta)},
            "form": "dense FP64; both factorisations carry the m cross-covariances as extra rows",
            "l2": "inputs larger than L2: two %.1f GB matrices generated every step" % (8.0 * (2 * n) ** 2 / 1e9)}


def run_mloe(args):
    import torch

    import paper_2008_07437_gb300 as geo
    from paper_2008_07437_gb300 import build as gbuild
    torch.cuda.set_device(0)
    gbuild.build()
    dev = torch.device("cuda", 0)
    w, n, locs, pred, spec, th_a_spec = mloe_setup(args)
    ctx = geo.geo_create(0)
    dl, dp = torch.as_tensor(locs, device=dev), torch.as_tensor(pred, device=dev)
    th_t, th_a = geo.Theta.from_spec(spec), geo.Theta.from_spec(th_a_spec)
    o = geo.opts(nb=960) if args.mloe_form == "native" else geo.opts(nb=512, fp64_gemm=1, oz_slices=8, oz_cut=1)
    for _ in range(args.warmup):
        geo.geo_mloe_mmom(ctx, dl, dp, th_t, th_a, o)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    geo.geo_profile_enable(ctx, True)
    clocks.start()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ml, mm, loe, mom = geo.geo_mloe_mmom(ctx, dl, dp, th_t, th_a, o)
    torch.cuda.synchronize()
    t = (time.perf_counter() - t0) / args.steps
    clk = clocks.stop()
    prof = geo.geo_profile_read(ctx)
    ph = {k: v["ms"] / args.steps for k, v in prof.items()}
    gen = ph["covgen"]
    fact = ph["potrf"] + ph["trsm"] + ph["gemm"] + ph["tcgemm"]
    comp = ph["solve"] + ph["reduce"] + ph["aux"]
    cls = "gemm" if args.mloe_form == "native" else "tcgemm"
    dk = prof[cls]
    bound, peak, peak_src = class_roofline(cls)
    ach = dk["flops"] / (dk["ms"] * 1e-3) / 1e12 if dk["ms"] > 0 else 0.0
    if cls == "tcgemm":
        # the tensor work the kernels issued (device-counted; the level cut lowers it)
        ach = dk["tensor_flops"] / (dk["ms"] * 1e-3) / 1e12 if dk["ms"] > 0 else 0.0
    out = {"metric": "MLOE/MMOM time", "value": t, "unit": "s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": mloe_config(args, n, spec, th_a_spec),
           "mloe": ml, "mmom": mm, "phases_ms": {"GEN": gen, "FACT": fact, "COMP": comp},
           "form": ("native FP64 FMA updates" if args.mloe_form == "native"
                    else "FP64 updates and panel solves on the tensor cores (8 digit slices, level cut)"),
           "roofline": {"bound": bound, "kernel": ("k_dgemm_update" if cls == "gemm" else "k_oz_update") +
                        " (both factorisations)", "achieved": ach,
                        "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "peak_source": peak_src,
                        "traffic": None},
           "gpu_launches": sum(v["launches"] for v in prof.values()), "clocks": clk}
    if not args.no_cpu_baseline:
        import oracle
        n_s = min(1000, n)
        tt0 = time.perf_counter()
        oracle.mloe_mmom(oracle.Theta(list(spec.sigma2), spec.a, list(spec.nu), spec.beta_matrix()),
                         oracle.Theta(list(th_a_spec.sigma2), th_a_spec.a, list(th_a_spec.nu), th_a_spec.beta_matrix()),
                         locs[:n_s], pred)
        ts = time.perf_counter() - tt0
        out["cpu_baseline"] = {"value": ts * (n / n_s) ** 3, "unit": "s", "cores": oracle.num_threads(),
                               "kind": "oracle",
                               "sample": "oracle at n = %d, m = %d in %.1f s, extrapolated by n^3" % (
                                   n_s, args.mloe_m, ts)}
    print(json.dumps(out), flush=True)
    ctx.close()
    return 0


# --------------------------------------------------------------------------
# estimation: parameter recovery of exact, TLR and DST fits (Sec. 6, Experiment 2)
# --------------------------------------------------------------------------
EST_METHODS = [("exact", {}), ("TLR5", {"tol": 1e-5}), ("TLR7", {"tol": 1e-7}), ("TLR9", {"tol": 1e-9}),
               ("DST 40/60", {"keep": 0.4}), ("DST 70/30", {"keep": 0.7})]


def dst_band(T: int, keep: float) -> int:
    """Tile diagonals d whose share of the T x T tiles of Sigma, (T + 2 sum_{k<d} (T - k)) / T^2, is closest
    to ``keep`` (DST 40/60 keeps 40 % of the tiles nearest the diagonal)."""
    best, best_err = 1, 2.0
    for d in range(1, T + 1):
        kept = T + 2 * sum(T - k for k in range(1, d))
        if abs(kept / T / T - keep) < best_err:
            best, best_err = d, abs(kept / T / T - keep)
    return best


def est_opts(geo, method, N, nb):
    kind = dict(EST_METHODS)[method]
    if "tol" in kind:
        return geo.opts(prec=geo.GEO_PREC_TLR, nb=nb, tlr_tol=kind["tol"], tlr_kmax=nb // 4)
    if "keep" in kind:
        return geo.opts(prec=geo.GEO_PREC_TLR, nb=nb, tlr_tol=1e-9, tlr_kmax=nb // 4,
                        dst=dst_band((N + nb - 1) // nb, kind["keep"]))
    return geo.opts(nb=nb)


def nm_converged(st, ftol=1e-6, xtol=1e-5):
    q = st.q
    if not st.initialized:
        return False
    fs = [st.f[v] for v in range(q + 1)]
    if not all(math.isfinite(f) for f in fs) or fs[-1] - fs[0] > ftol:
        return False
    return max(abs(st.x[v][d] - st.x[0][d]) for v in range(1, q + 1) for d in range(q)) < xtol


def run_estimation(args):
    import torch

    import paper_2008_07437_gb300 as geo
    from paper_2008_07437_gb300 import build as gbuild
    torch.cuda.set_device(0)
    gbuild.build()
    dev = torch.device("cuda", 0)
    n = args.n or 1600
    p = 2
    N = p * n
    nb = args.nb or 2 * ((N // 10 + 1) // 2)          # ten tile rows, nb a multiple of p
    max_iter = args.mle or 400
    ranges = [float(v) for v in args.est_a.split(",")]
    methods = [m.strip() for m in args.est_methods.split(",")]
    unknown = [m for m in methods if m not in dict(EST_METHODS)]
    if unknown:
        raise SystemExit("unknown estimation methods: %s" % unknown)
    ctx = geo.geo_create(0)
    clocks = ClockSampler(dev.index)
    clocks.start()
    t_start = time.perf_counter()
    results, runs, skipped = {}, 0, 0
    for a in ranges:
        truth = inputs.ThetaSpec((1.0, 1.0), a, (0.5, 1.0), (0.5,))
        th_true = geo.Theta.from_spec(truth)
        per = {m: [] for m in methods}
        for r in range(args.replicates):
            locs = inputs.jittered_grid(n, 3000 + r)
            dl = torch.as_tensor(locs, device=dev).contiguous()
            de = torch.as_tensor(inputs.normals(4000 + r, N), device=dev)
            dz = torch.empty(N, dtype=torch.float64, device=dev)
            geo.geo_simulate(ctx, dl, de, th_true, dz, geo.opts(nb=nb))
            start = geo.Theta((1.2, 0.8), 1.3 * a, (0.6, 0.9), 0.3)
            for m in methods:
                if time.perf_counter() - t_start > args.est_budget_s:
                    skipped += 1
                    continue
                o = est_opts(geo, m, N, nb)
                st = geo.geo_mle_init(start, 0.1, profile=not args.est_full)
                t0 = time.perf_counter()
                it = 0
                infeasible = False
                while it < max_iter and not nm_converged(st):
                    geo.geo_mle_step(ctx, st, dl, dz, o)
                    it += 1
                    if it == 1 and all(math.isinf(st.f[v]) for v in range(st.q + 1)):
                        infeasible = True    # no vertex of the initial simplex has a positive definite matrix
                        break
                dt = time.perf_counter() - t0
                best, ll = geo.geo_mle_best(st)
                per[m].append({"sigma2": list(best.sigma2), "a": best.a, "nu": list(best.nu),
                               "beta": float(np.asarray(best.beta).reshape(2, 2)[0, 1]), "loglik": ll,
                               "iters": st.iter, "evals": st.evals, "converged": nm_converged(st), "s": dt,
                               "infeasible": infeasible})
                runs += 1
                print("a=%g r=%d %-9s %3d it %4d ev %6.1f s  a=%.4f nu=(%.3f, %.3f) beta=%.3f s2=(%.3f, %.3f)" % (
                    a, r, m, st.iter, st.evals, dt, best.a, best.nu[0], best.nu[1], per[m][-1]["beta"],
                    best.sigma2[0], best.sigma2[1]), file=sys.stderr, flush=True)
        summary = {}
        tv = {"sigma2_1": 1.0, "sigma2_2": 1.0, "a": a, "nu_1": 0.5, "nu_2": 1.0, "beta": 0.5}
        for m, est in per.items():
            if not est:
                continue
            if all(e["infeasible"] for e in est):
                summary[m] = {"infeasible": "the matrix (or a marginal R_ii) with the dropped tiles is not positive "
                                            "definite at any vertex of the initial simplex", "runs": est}
                continue
            est = [e for e in est if not e["infeasible"]]
            vals = {"sigma2_1": [e["sigma2"][0] for e in est], "sigma2_2": [e["sigma2"][1] for e in est],
                    "a": [e["a"] for e in est], "nu_1": [e["nu"][0] for e in est],
                    "nu_2": [e["nu"][1] for e in est], "beta": [e["beta"] for e in est]}
            summary[m] = {"median": {k: float(np.median(v)) for k, v in vals.items()},
                          "std": {k: float(np.std(v)) for k, v in vals.items()},
                          "median_rel_err": {k: float(np.median([abs(x - tv[k]) / abs(tv[k]) for x in v]))
                                             for k, v in vals.items()},
                          "runs": est}
        results["a=%g" % a] = summary
    torch.cuda.synchronize()
    t = time.perf_counter() - t_start
    clk = clocks.stop()
    out = {"metric": "estimation study wall time", "value": t, "unit": "s", "n_gpus": 1, "steps": runs,
           "warmup": 0, "ms_per_step": 1e3 * t / max(runs, 1), "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "estimation", "n": n, "p": p, "N": N, "nb": nb, "tiles": (N + nb - 1) // nb,
                      "truth": {"sigma2": [1.0, 1.0], "nu": [0.5, 1.0], "beta": 0.5, "a": ranges},
                      "replicates": args.replicates, "objective": "full" if args.est_full else "profile",
                      "start": "sigma2 (1.2, 0.8), a x 1.3, nu (0.6, 0.9), beta 0.3; simplex step 0.1",
                      "stop": "f spread <= 1e-6 and vertex spread <= 1e-5, or %d iterations" % max_iter,
                      "tlr_kmax": nb // 4,
                      "dst_bands": {m: dst_band((N + nb - 1) // nb, k["keep"]) for m, k in EST_METHODS
                                    if "keep" in k}},
           "results": results, "runs_skipped_for_time": skipped, "clocks": clk}
    print(json.dumps(out), flush=True)
    ctx.close()
    return 0


def run_serving_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    stream = inputs.serving_stream(args.requests, rate=args.rate, seed=3000)
    service, det, cores = serving_cpu_model(stream)
    cb = serving_cpu_json(stream, service, det, cores)
    line = {"impl": "reference", "metric": SERVING_METRIC, "value": cb["value"], "unit": "ms", "n_gpus": args.gpus,
            "steps": len(stream), "warmup": 0, "ms_per_step": sum(service) * 1e3 / len(stream),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": serving_config(args, stream, "oracle FP64 (extrapolated)", {}),
            "p50_ms": cb["value"], "p99_ms": cb["p99_ms"], "throughput_req_s": cb["throughput_req_s"],
            "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gemm(args):
    """The emulated FP64 product alone (the GEMM tile task of Sec. 5.1 as one call):
    C (m x n) -= A (m x k) B (n x k)' through geo_gemm_f64e, inputs resident, CUDA events."""
    import torch

    import paper_2008_07437_gb300 as geo
    from paper_2008_07437_gb300 import build as gbuild
    gbuild.build()
    torch.cuda.set_device(0)
    m, n, k = (int(x) for x in args.gemm_mnk.split(","))
    S = args.gemm_slices
    ctx = geo.geo_create(0)
    g = torch.Generator(device="cuda").manual_seed(1)
    A = torch.randn((k, m), dtype=torch.float64, device="cuda", generator=g).t()
    B = torch.randn((k, n), dtype=torch.float64, device="cuda", generator=g).t()
    C = torch.zeros((n, m), dtype=torch.float64, device="cuda").t()
    for _ in range(args.warmup):
        geo.geo_gemm_f64e(ctx, A, B, C, slices=S)
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    geo.geo_profile_enable(ctx, True)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        geo.geo_gemm_f64e(ctx, A, B, C, slices=S)
    ev1.record()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    tc = geo.geo_profile_read(ctx)["tcgemm"]
    geo.geo_profile_enable(ctx, False)
    fl = 2.0 * m * n * k
    kernel_ms = tc["ms"] / args.steps
    bound, peak, peak_src = class_roofline("tcgemm")
    tensor = tc["tensor_flops"] / args.steps / (kernel_ms * 1e-3) / 1e12
    out = {"metric": "emulated FP64 GEMM FP64-equivalent TFLOP/s", "value": fl / (ms * 1e-3) / 1e12,
           "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64 (emulated: bf16 digit products, exact fp32 accumulation, %d slices)" % S,
           "data": "synthetic", "config": {"workload": "gemm", "m": m, "n": n, "k": k, "slices": S,
                                           "l2": "C (%.2f GB) larger than L2" % (8.0 * m * n / 1e9)},
           "roofline": {"bound": bound, "kernel": KERNEL_NAMES["oz"], "achieved": tensor, "peak": peak,
                        "unit": "TFLOP/s", "frac": tensor / peak, "peak_source": peak_src, "traffic": None,
                        "kernel_ms": kernel_ms, "fp64_equivalent_tflops": fl / (kernel_ms * 1e-3) / 1e12,
                        "algorithmic_bytes_per_launch": tc["bytes"] / max(tc["launches"], 1)},
           "gpu_launches": sum(v["launches"] for v in geo.geo_profile_read(ctx).values()), "clocks": clk}
    print(json.dumps(out), flush=True)
    ctx.close()
    return 0


def main():
    args = parse()
    if args.workload == "gemm":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "gemm mode: a kernel benchmark, no CPU arm"}))
            return 0
        return run_gemm(args)
    if args.workload == "serving":
        return run_serving_reference(args) if args.impl == "reference" else run_serving(args)
    if args.workload == "mloe":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "mloe mode: the oracle time is this mode's cpu_baseline"}))
            return 0
        return run_mloe(args)
    if args.workload == "estimation":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "estimation mode: a study of fits, not a timed path"}))
            return 0
        return run_estimation(args)
    if args.workload == "batch":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "batch mode: use the default workload's reference arm"}))
            return 0
        return run_batch(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
