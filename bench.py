"""Benchmark of the GB300 SRTM filter + smoother (fast-rate smoothed states/s).

One step = one srtm_smoother_batch call over the ragged batch (default
workload): 4096 independent 4-species chains (nx=4, ny=1, ratio in {5,10,20},
100..20000 slow steps each; about 4.9*10^8 fast steps), synthetic data from
the seeded generator.  Each step runs, for every sequence, the per-model
constants, the forward filter scan, the interval setup and smoother elements,
the reverse smoother scan and the fast-rate recovery (fast and slow smoothed
means and covariances written to HBM).  The call is captured in a CUDA graph
and replayed; inputs and outputs are resident in HBM (outputs of about 84 GB
per step, far above the 129 MB L2, so no flush).

Headline `value`: mixed precision (float32 scans with float64 solves,
symmetrisation and recovery), launch shapes chosen by the library's
autotuner.  The line also carries the plain FP64 batched number, the plain
FP64 single-sequence path looped over the sequences, the batched sequential
comparator, the end-to-end number with every output written to pinned host
memory, the recovery roofline with per-phase fractions against the measured
FP64 / FP32 peaks, the oracle on every host core, and chain4 (one 4-species
chain, nx=4, ny=2, ratio 20, 10^4 slow steps) as a nested line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload ragged_chains|chain4] [--peaks]
Multi-GPU (torchrun): the batch's sequences are split over the ranks in
contiguous ranges of nearly equal fast steps (no collective on the data
path; strong scaling); with --workload chain4 every rank runs its own
sequence (weak scaling).  Rank 0 prints.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fast-rate smoothed states/sec (filter+smoother) on 1 GB300, mixed vs FP64, at oracle tol"
UNIT = "fast states/s"
PEAKS_FILE = os.path.join(ROOT, "profiles", "fp64_fp32_peak.json")
NOMINAL_PEAKS = {"fp64_gflops": 1250.0, "fp32_gflops": 80500.0}   # GB300 nominal, used only without the file


def measured_peaks() -> dict:
    """FMA-throughput peaks (GFLOP/s) of this machine's GB300 from the committed
    calibration (``bench.py --peaks``: srtm_measure_peak, float64 and float32
    FMA chains on every SM), else the nominal figures, with their source."""
    try:
        d = json.load(open(PEAKS_FILE))
        return {"fp64_gflops": float(d["fp64_gflops"]), "fp32_gflops": float(d["fp32_gflops"]),
                "source": f"measured: profiles/{os.path.basename(PEAKS_FILE)} (srtm_measure_peak, {d.get('when', '')}, "
                          f"SM {d.get('sm_mhz_median')} MHz)"}
    except (OSError, ValueError, KeyError):
        return dict(NOMINAL_PEAKS, source="nominal (no committed calibration)")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64", "fp32"], default="mixed")
    ap.add_argument("--n-slow", type=int, default=10_000)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-extras", action="store_true", help="skip the fp64, e2e and cpu legs")
    ap.add_argument("--workload", choices=["chain4", "ragged_chains"], default="ragged_chains")
    ap.add_argument("--no-chain4", action="store_true", help="ragged_chains: skip the nested chain4 line")
    ap.add_argument("--peaks", action="store_true",
                    help="measure the FP64 and FP32 FMA peaks (srtm_measure_peak) with SM clocks sampled, print one "
                         "JSON line")
    ap.add_argument("--n-seq", type=int, default=4096, help="ragged_chains: sequences in the batch")
    ap.add_argument("--no-autotune", action="store_true", help="keep the built-in launch shapes")
    ap.add_argument("--tuning", default=None,
                    help="explicit launch shapes scan_groups,scan_elems,recover_threads,lookback_window"
                         "[,setup_mode,recover_split,batch_chunks,chunk_recover_bps,chunk_scan_bps,recover_form] "
                         "(for every precision; replaces the autotuner)")
    ap.add_argument("--tune-reps", type=int, default=2)
    ap.add_argument("--sweep", action="store_true",
                    help="chain4 over T = 10^2 .. 10^4 slow steps (x sqrt 10), FP64 and mixed, one JSON line each")
    ap.add_argument("--figure", action="store_true",
                    help="run time of the scan and the sequential forms (filter and smoother, FP64) over "
                         "T = 16 .. 6000 slow steps of chain4, one JSON line per T")
    ap.add_argument("--report-errors", action="store_true",
                    help="max relative errors of every mode against the FP64 oracle, every single-sequence "
                         "workload at full size")
    return ap.parse_args(argv)


def workload(args, rank=0):
    from paper_2410_00627_gb300 import synth
    return synth.chain4(seed=args.seed + rank, n_slow=args.n_slow, keep_states=False)


def config_dict(args, prob, precision):
    return {"workload": f"chain4: 4-species chain nx=4 ny=2 L={prob.ratio} T={prob.n_slow} slow "
                        f"({prob.n_slow * prob.ratio} fast steps)",
            "precision": precision, "nx": prob.nx, "ny": prob.ny, "ratio": prob.ratio,
            "n_slow": prob.n_slow, "l2": "flushed (256 MB write) before every timed step",
            "seed": args.seed}


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={','.join(self.FIELDS)}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in self.rows for j in range(4) if r[3 + j].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def reduce_over_ranks(mean_ms, units, dist, device):
    """Whole-job figures over the ranks: the slowest rank's mean step time and
    the units (fast states) all ranks processed per step.  Without a process
    group: this rank's own figures."""
    if dist is None:
        return float(mean_ms), float(units)
    import torch
    if dist.get_backend() == "gloo":
        device = "cpu"
    t = torch.tensor([float(mean_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# --------------------------------------------------------------------------- our arm
def run_ours(args, rank, world, dist):
    import torch

    from paper_2410_00627_gb300 import api, build
    build.build()
    api.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    prob = workload(args, rank)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)  # noqa: E731
    ins = [t(getattr(prob, k)) for k in ("F", "Q", "H", "R", "m0", "P0", "y")]
    n_fast = prob.n_slow * prob.ratio
    outs = {"fast_mean": torch.empty(n_fast, prob.nx, dtype=torch.float64, device=dev),
            "fast_cov": torch.empty(n_fast, prob.nx, prob.nx, dtype=torch.float64, device=dev),
            "slow_mean": torch.empty(prob.n_slow, prob.nx, dtype=torch.float64, device=dev),
            "slow_cov": torch.empty(prob.n_slow, prob.nx, prob.nx, dtype=torch.float64, device=dev)}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step(precision, st=None):
        api.smoother(*ins, prob.ratio, precision=precision, out=outs, stream=st)

    def timed_graph(precision, steps, warmup):
        """The call captured in a CUDA graph and replayed: flush L2, then the
        replay between two events, every step on one side stream."""
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            for _ in range(warmup):
                step(precision, side)
            api.status(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side, capture_error_mode="relaxed"):
            step(precision, side)
        launches = api.last_call_launches()
        ms = []
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        with torch.cuda.stream(side):   # replay() launches on the current stream
            for _ in range(steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(side)
                g.replay()
                e1.record(side)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        api.status(side)
        del g
        return ms, launches

    def timed(precision, steps, warmup, stage=False):
        for _ in range(warmup):
            step(precision)
        api.status()
        ms, rec_ms = [], []
        api.set_stage_timing(stage)
        try:
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
            for _ in range(steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step(precision)
                e1.record(stream)
                if stage:
                    rec_ms.append(api.stage_times())
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
        finally:
            api.set_stage_timing(False)
        api.status()
        return ms, rec_ms

    tuning = {}
    precs = [args.precision] + ([] if args.no_extras else ["fp64" if args.precision != "fp64" else "mixed"])
    if args.tuning:
        for p in precs:
            api.set_tuning(prob.nx, p, *[int(v) for v in args.tuning.split(",")])
            tuning[p] = api.get_tuning(prob.nx, p)
    elif not args.no_autotune:
        for p in precs:
            tuning[p], _ = api.autotune(*ins, prob.ratio, precision=p, reps=args.tune_reps, out=outs)
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
    ms, launches = timed_graph(args.precision, args.steps, args.warmup)
    clock_info = clocks.stop() if clocks else None
    parity = check_parity(prob, outs, args.precision) if rank == 0 else None
    ms_direct, stages = timed(args.precision, max(5, args.steps // 2), 2, stage=True)
    mean_ms, units = reduce_over_ranks(float(np.mean(ms)), n_fast, dist, dev)
    value = units / (mean_ms * 1e-3)
    if rank != 0:
        return None
    stage_mean = {k: float(np.mean([s[k] for s in stages])) for k in stages[0]}
    # roofline of the dominant kernel (fast-rate recovery): FP64 ALU bound.
    # With a split recovery its two halves are timed on their own streams and
    # their durations added.
    peaks = measured_peaks()
    roof = recovery_roofline(stage_mean, prob.nx, prob.ny, args.precision, prob.n_slow, n_fast,
                             recorded_traffic(args.precision, n_fast), peaks,
                             "stage events around the recovery launch(es) of direct calls, mean of the steps "
                             "(a split recovery adds its two halves)",
                             api.get_tuning(prob.nx, args.precision)["recover_form"])
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"mixed": "f32+f64", "fp64": "f64", "fp32": "f32"}[args.precision],
        "data": "synthetic (seeded generator, chain4 linear kinetics)",
        "config": dict(config_dict(args, prob, args.precision),
                       tuning=tuning.get(args.precision, api.get_tuning(prob.nx, args.precision)),
                       timing="CUDA-graph replay of the call, CUDA events on its stream, mean of the steps"),
        "ms_per_step_median": float(np.median(ms)),
        "parity": parity,
        "direct_calls": {"ms_per_step": float(np.mean(ms_direct)),
                         "note": "the same call issued through the C-ABI each step (host launch cost included)"},
        "stage_ms": stage_mean,
        "roofline": roof,
        "gpu_launches": args.steps * launches,
        "clocks": clock_info,
    }
    if not args.no_extras:
        other = "fp64" if args.precision != "fp64" else "mixed"
        ms2, _ = timed_graph(other, max(5, args.steps // 2), 3)
        line[other] = {"value": n_fast / (float(np.mean(ms2)) * 1e-3), "ms_per_step": float(np.mean(ms2)),
                       "tuning": tuning.get(other, api.get_tuning(prob.nx, other)),
                       "parity": check_parity(prob, outs, other)}
        line["e2e"] = run_e2e(args, prob, api, torch, flush)
        seq_ms = time_calls(lambda st: api.smoother(*ins, prob.ratio, precision=args.precision, out=outs, stream=st,
                                                    method="sequential"), 2, 1, stream, flush)
        line["sequential_comparator"] = {
            "value": n_fast / (float(np.mean(seq_ms)) * 1e-3), "ms_per_step": float(np.mean(seq_ms)),
            "call": "srtm_smoother_sequential (IMKF and IMS recursions over the slow steps on one thread), "
                    "direct calls, mean of 2 after 1 warm-up"}
        line["cpu_baseline"] = run_cpu_baseline(args, prob)
    return line


def recovery_fma(n, m, form=1):
    """FMAs per fast step of the smoothing recovery as the kernel executes them
    (a multiply counts as one).

    form 2 (two-point): the mean C1_i mu0 + C2_i mu1 + c3_i y_k (2 n^2 + n m),
    W = C1_i E_k + C2_i (n^3), and two factored quadratic forms W P^s_{k+1,1}
    W^T and C1_i S_k C1_i^T, each (W L) (n^2 (n-1)/2), its columns scaled by D
    (n^2) and the upper triangle (n(n+1)/2 n); per fast step of an interval
    with a successor (the last interval of a sequence, 1/N of the steps, takes
    one quadratic form and no W).

    form 1 (record form, Remarks 1 and 3): U_i (n^2 m), m^f_i (n^2 + n m),
    P^f_il (n^3 + n^2 m), U_i S_y^-1 (n m^2), A^i P A^iT with P = L D L^T from
    the record, (A^i L) D (A^i L)^T: A^i L (n^2 (n-1)/2), its columns scaled by
    D (n^2) and the upper triangle (n(n+1)/2 n, the n(n+1)/2 m of the gain term
    added); the smoothing correction P^f_il Om P^f_il^T the same way with
    Om = L D L^T (n^2 (n-1)/2 + n^2 + n(n+1)/2 n) and the smoothed mean (n^2).
    Products whose result is symmetric count their upper triangle only, as
    computed."""
    if form == 2:
        return 2 * n * n + n * m + n ** 3 + 2 * (n * n * (n - 1) // 2 + n * n + n * (n + 1) // 2 * n)
    return (n ** 3 + n * n * (n - 1) + n * (n + 1) // 2 * (2 * n + m) + 2 * n * n * m + n * m * m + 4 * n * n
            + n * m)


def recovery_roofline(stage_ms, n, m, precision, n_slow, n_fast, traffic, peaks, timing, form=1):
    """The roofline object of the dominant kernel (recover_kernel, bound by the
    float64 FMA pipe): algorithmic FLOPs per call over its event-timed duration,
    against the measured peak, with the per-phase fractions beside it."""
    key = "fp32" if precision == "fp32" else "fp64"
    rec_ms = stage_ms["recovery"] + stage_ms.get("recovery_filtered_half", 0.0)
    achieved = 2.0 * recovery_fma(n, m, form) * n_fast / (rec_ms * 1e-3) / 1e9
    peak = peaks[f"{key}_gflops"]
    return {"bound": "alu", "kernel": "recover_kernel", "achieved": achieved, "peak": peak, "unit": "GFLOP/s",
            "frac": achieved / peak, "traffic": traffic,
            "peak_source": f"{key.upper()} FMA peak, {peaks['source']}",
            "recover_form": {1: "record", 2: "two-point"}[form],
            "flops_per_fast_step": 2 * recovery_fma(n, m, form), "fast_steps_per_launch": n_fast, "timing": timing,
            "phases": roofline_phases(stage_ms, n, m, precision, n_slow, n_fast, peaks, form)}


def phase_fma(n, m, precision, form=1):
    """Algorithmic FMAs per slow step of the three slow-rate phases, split by
    the arithmetic type they run in (float64 or float32 in the mixed mode;
    every FMA in float64 in the FP64 mode, in float32 in the FP32 mode).

    filter scan (one Eq. 27 combine per element, the element build of Eq. 25-26
    and the interval setup run as its epilogue):
      combine with a generic element (m < n, the matrix inversion lemma):
      C_bar D_i, C_bar F_i (2 m n^2), D_i eta_j, J_j d_i (2 n^2), S (m^2 n),
      S^-1 C_bar D_i, S^-1 G (2 m^2 n), u (n m), D_i - K C_bar D_i and
      J_ij (upper, 2 n(n+1)/2 m), V (n^2 m), d_ij, eta_ij (2 n^2), F_j P,
      F_j V (2 n^3), D_ij upper (n(n+1)/2 n); its m x m solve (m = 1: a
      float32 reciprocal; m = 2: the float64 determinant, 2; m > 2: m^3) is
      float64 in the mixed mode.  (m >= n: the general combine,
      (25/3) n^3 + 5 n^2 with the n^3 inverse in float64.)  Element build 2 n m;
      setup record (float64): X = P C_bar^T (n^2 m), S_y (n m (m+1)/2),
      innovation (n m), kappa (m^2), U_l (n^2 m), S_y^-1 U_l^T (n m^2),
      m^f_l (n^2 + n m), P A^{lT} and A P_ll (2 n^3), P^- upper triangle
      (n^2 (n+1)/2), its inverse and Z (2 n^3);
      smoother element, Eq. 29 (float32 in the mixed mode): U_1 (n^2 m),
      m^f_1 (n^2 + n m), A m^f_l (n^2), U_1 S_y^-1 (n m^2), A P, P^f_1l, E and
      A P^f_1l^T (4 n^3 + n^2 m), P^f_11 upper (n(n+1)/2 (n + m)), g (n^2),
      S upper (n^2 (n+1)/2).
    smoother scan: one Eq. 30 combine 3 n^3 + n^2 (scan type) and, per result,
      the record form's smoothing terms Z dP, Om upper, om, dm
      (n^3 + n^2 (n+1)/2 + 2 n^2, float64 in the mixed mode), or the two-point
      form's LDL^T factors of P^s_{k+1,1} and S_k (2 x sum_j (j + (n-1-j)(j+1)),
      float64 in the mixed mode).
    The parallel scan's second combine per element (its re-walk) is overhead,
    not algorithmic work, and is not counted."""
    if m < n:
        solve = 0 if m == 1 else (2 if m == 2 else m ** 3)
        combine = (2 * m * n * n + 2 * n * n + m * m * n + 2 * m * m * n + n * m + n * (n + 1) * m + n * n * m
                   + 2 * n * n + 2 * n ** 3 + n * (n + 1) // 2 * n)
    else:
        solve = n ** 3
        combine = (25 * n ** 3) // 3 + 5 * n * n
    record = (n * n * m + n * m * (m + 1) // 2 + n * m + m * m + n * n * m + n * m * m + n * n + n * m + 2 * n ** 3
              + n * n * (n + 1) // 2 + 2 * n ** 3)
    element = (n * n * m + n * n + n * m + n * n + n * m * m + 4 * n ** 3 + n * n * m + n * (n + 1) // 2 * (n + m)
               + n * n + n * n * (n + 1) // 2)
    s_combine = 3 * n ** 3 + n * n
    s_terms = n ** 3 + n * n * (n + 1) // 2 + 2 * n * n
    if form == 2:
        s_terms = 2 * sum(j + (n - 1 - j) * (j + 1) for j in range(n))
    f32 = {"filter_scan": combine - solve + 2 * n * m + element, "smoother_scan": s_combine}
    f64 = {"filter_scan": solve + record, "smoother_scan": s_terms}
    if precision == "fp64":
        return {k: (0, f32[k] + f64[k]) for k in f32}
    if precision == "fp32":
        return {k: (f32[k] + f64[k], 0) for k in f32}
    return {k: (f32[k], f64[k]) for k in f32}


def roofline_phases(stage_ms, n, m, precision, n_slow, n_fast, peaks, form=1):
    """Per-phase achieved FLOP/s (algorithmic counts of phase_fma and
    recovery_fma) over the phase's event time, as fractions of the measured
    float32 and float64 FMA peaks."""
    out = {}
    pf = phase_fma(n, m, precision, form)
    times = {"filter_scan": stage_ms["filter_scan"] + stage_ms.get("interval_setup", 0.0),
             "smoother_scan": stage_ms["smoother_scan"]}
    for ph, (f32, f64) in pf.items():
        t = times[ph] * 1e-3
        if t <= 0:
            continue
        g32, g64 = 2.0 * f32 * n_slow / t / 1e9, 2.0 * f64 * n_slow / t / 1e9
        out[ph] = {"ms": times[ph], "fp32_gflops": g32, "fp32_frac": g32 / peaks["fp32_gflops"],
                   "fp64_gflops": g64, "fp64_frac": g64 / peaks["fp64_gflops"],
                   "fma_per_slow_step": {"fp32": f32, "fp64": f64}}
    rec_ms = stage_ms["recovery"] + stage_ms.get("recovery_filtered_half", 0.0)
    g = 2.0 * recovery_fma(n, m, form) * n_fast / (rec_ms * 1e-3) / 1e9
    key = "fp32" if precision == "fp32" else "fp64"
    out["recovery"] = {"ms": rec_ms, f"{key}_gflops": g, f"{key}_frac": g / peaks[f"{key}_gflops"],
                       "fma_per_fast_step": recovery_fma(n, m, form)}
    return out


def time_calls(call, steps, warmup, stream, flush=None):
    """Per-call device times (ms) of ``call(stream)`` by CUDA events on ``stream``
    after ``warmup`` untimed calls; L2 flushed before each call when given."""
    import torch

    from paper_2410_00627_gb300 import api
    for _ in range(warmup):
        call(stream)
    api.status(stream)
    ms = []
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call(stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    api.status(stream)
    return ms


def run_figure(args):
    """The scan forms against the sequential forms (the paper's figure of
    parallel vs sequential IMKF / IMS run time over the number of steps), on
    chain4 (l = 20) in FP64, each call timed on its own."""
    import torch

    from paper_2410_00627_gb300 import api, build, synth
    build.build()
    api.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    lines = []
    for n_slow in (16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 6000):
        prob = synth.chain4(seed=args.seed, n_slow=n_slow, keep_states=False)
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)  # noqa: E731
        ins = [t(getattr(prob, k)) for k in ("F", "Q", "H", "R", "m0", "P0", "y")]
        n_fast = n_slow * prob.ratio
        outs = {"fast_mean": torch.empty(n_fast, prob.nx, dtype=torch.float64, device=dev),
                "fast_cov": torch.empty(n_fast, prob.nx, prob.nx, dtype=torch.float64, device=dev),
                "slow_mean": torch.empty(n_slow, prob.nx, dtype=torch.float64, device=dev),
                "slow_cov": torch.empty(n_slow, prob.nx, prob.nx, dtype=torch.float64, device=dev)}
        row = {"figure": "chain4 scan vs sequential, fp64", "n_slow": n_slow, "fast_steps": n_fast, "unit": "us"}
        for method in ("scan", "sequential"):
            for kind in ("filter", "smoother"):
                fn = api.filter if kind == "filter" else api.smoother
                call = lambda st, fn=fn, method=method: fn(*ins, prob.ratio, precision="fp64", out=outs,  # noqa: E731
                                                            stream=st, method=method)
                ms = time_calls(call, 20, 3, stream)
                row[f"{method}_{kind}_us"] = float(np.median(ms)) * 1e3
        lines.append(row)
    return lines


# --------------------------------------------------------------------------- ragged batch
def batched_workload(args, rank=0, world=1):
    """The ragged batch, or under torchrun this rank's share of it: a
    contiguous range of sequences holding nearly 1/world of the fast steps.
    Returns (sequences, (first, end) index range in the whole batch)."""
    from paper_2410_00627_gb300 import synth
    workers = max(1, min(16, (os.cpu_count() or 1) // max(1, world)))
    rng = (0, args.n_seq)
    if world > 1:
        r, n = synth.ragged_shapes(args.seed, args.n_seq)
        rng = synth.balanced_ranges(r * n, world)[rank]
        if rng[1] <= rng[0]:
            raise RuntimeError(f"rank {rank} received no sequence of the batch")
    return synth.ragged_chains(seed=args.seed, n_seq=args.n_seq, workers=workers, seq_range=rng), rng


def batched_config(args, pk, precision, tuning, world=1, seq_range=None):
    d = {"workload": f"ragged_chains: {args.n_seq} ragged 4-species chains nx=4 ny=1 L in {{5,10,20}} "
                     f"N in [100,20000]" + (f" ({pk['total_slow']} slow / {pk['total_fast']} fast steps)"
                                            if world == 1 else ""),
         "precision": precision, "n_seq": args.n_seq, "call": "srtm_smoother_batch captured in a CUDA graph, replayed",
         "l2": "not flushed: each step writes 168 B per fast step (about 84 GB, far above the 129 MB L2)",
         "seed": args.seed, "tuning": tuning}
    if world == 1:
        d.update(total_slow=pk["total_slow"], total_fast=pk["total_fast"])
    else:
        d["partition"] = (f"sequences split over {world} ranks in contiguous ranges of nearly equal fast steps; "
                          f"rank 0 holds sequences {seq_range[0]}..{seq_range[1] - 1}")
    return d


def upload_batch(pk, api, torch, dev):
    t = lambda a: torch.as_tensor(a, device=dev)  # noqa: E731
    ten = {k: t(pk[k]) for k in ("F", "Q", "H", "R", "m0", "P0", "y", "ratio", "n_slow")}
    b = api.make_batch(ten["F"], ten["Q"], ten["H"], ten["R"], ten["m0"], ten["P0"], ten["y"], ten["ratio"],
                       ten["n_slow"], pk["max_ratio"], pk["total_slow"], pk["total_fast"])
    return b, ten


def batch_outputs(torch, dev, n_fast, n_slow, nx):
    return {"fast_mean": torch.empty(n_fast, nx, dtype=torch.float64, device=dev),
            "fast_cov": torch.empty(n_fast, nx, nx, dtype=torch.float64, device=dev),
            "slow_mean": torch.empty(n_slow, nx, dtype=torch.float64, device=dev),
            "slow_cov": torch.empty(n_slow, nx, nx, dtype=torch.float64, device=dev)}


def live_peaks(api):
    """FMA peaks measured now, on this GPU (srtm_measure_peak, 200 ms launches)."""
    return {k: api.measure_peak(k, 200.0)[0] for k in ("fp64", "fp32")}


def run_batched(args, rank, world, dist):
    import torch

    from paper_2410_00627_gb300 import api, build, synth
    build.build()
    api.load()
    t0 = time.perf_counter()
    probs, seq_range = batched_workload(args, rank, world)
    gen_s = time.perf_counter() - t0
    dev = torch.device("cuda", torch.cuda.current_device())
    pk = synth.pack(probs)
    batch, ten = upload_batch(pk, api, torch, dev)
    nx, ny = pk["F"].shape[1], pk["H"].shape[1]
    n_fast, n_slow = pk["total_fast"], pk["total_slow"]
    outs = batch_outputs(torch, dev, n_fast, n_slow, nx)
    peaks_now = live_peaks(api) if rank == 0 else None
    precs = [args.precision] + ([] if args.no_extras else ["fp64" if args.precision != "fp64" else "mixed"])
    tuning = {}
    if args.tuning:
        for p in precs:
            api.set_tuning(nx, p, *[int(v) for v in args.tuning.split(",")])
            tuning[p] = api.get_tuning(nx, p)
    elif not args.no_autotune:   # on the first 512 sequences (same distribution, ~1/8 of the work)
        sub = synth.pack(probs[:min(512, len(probs))])
        sb, sten = upload_batch(sub, api, torch, dev)
        so = batch_outputs(torch, dev, sub["total_fast"], sub["total_slow"], nx)
        for p in precs:
            tuning[p], _ = api.autotune_batch(sb, precision=p, reps=1, out=so)
        del sb, sten, so
    stream = torch.cuda.Stream()

    def graph_for(precision):
        with torch.cuda.stream(stream):
            for _ in range(max(1, args.warmup)):
                api.smoother_batch(batch, precision=precision, out=outs, stream=stream)
            api.status(stream)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream, capture_error_mode="relaxed"):
            api.smoother_batch(batch, precision=precision, out=outs, stream=stream)
        with torch.cuda.stream(stream):
            g.replay()
        stream.synchronize()
        api.status(stream)
        return g

    def timed_graph(g, steps):
        ms = []
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        with torch.cuda.stream(stream):   # replay() launches on the current stream
            for _ in range(steps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.replay()
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        api.status(stream)
        return ms

    def stage_call(precision, **tune):
        """Per-launch durations of one direct call (library stage events)."""
        saved = api.get_tuning(nx, precision)
        if tune:
            api.set_tuning(nx, precision, **dict(saved, **tune))
        api.set_stage_timing(True)
        try:
            with torch.cuda.stream(stream):
                api.smoother_batch(batch, precision=precision, out=outs, stream=stream)
                st = api.stage_times()
        finally:
            api.set_stage_timing(False)
            api.set_tuning(nx, precision, **saved)
        api.status(stream)
        return st

    g = graph_for(args.precision)
    launches = api.last_call_launches()
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if clocks:
        clocks.start()
    ms = timed_graph(g, args.steps)
    clock_info = clocks.stop() if clocks else None
    del g
    parity = check_parity_batch(probs, pk, outs, args.precision) if rank == 0 else None
    mean_ms, units = reduce_over_ranks(float(np.mean(ms)), n_fast, dist, dev)
    value = units / (mean_ms * 1e-3)
    stage = stage_call(args.precision)                      # the timed configuration
    stage_serial = stage_call(args.precision, batch_chunks=1)  # stages one after another
    line = None
    if rank == 0:
        peaks = measured_peaks()
        form = api.get_tuning(nx, args.precision)["recover_form"]
        roof = recovery_roofline(stage_serial, nx, ny, args.precision, n_slow, n_fast,
                                 recorded_traffic(args.precision, n_fast, "ragged_chains"), peaks,
                                 "stage events of a direct call with every stage over the whole batch "
                                 "(the recovery launch alone on the GPU)", form)
        key = "fp32" if args.precision == "fp32" else "fp64"
        rec_pipe = stage["recovery"] * 1e-3
        roof["achieved_in_timed_configuration"] = 2.0 * recovery_fma(nx, ny, form) * n_fast / rec_pipe / 1e9
        roof["note_in_timed_configuration"] = (
            "summed durations of the per-chunk recovery launches of the timed (chunked) configuration, which share "
            "the GPU with the scans of the next chunk" if api.get_tuning(nx, args.precision)["batch_chunks"] > 1
            else "same configuration")
        roof["peak_live"] = peaks_now[key]
        roof["peak_live_fp32"] = peaks_now["fp32"]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": mean_ms, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak",
            "vs_baseline": None, "dtype": {"mixed": "f32+f64", "fp64": "f64", "fp32": "f32"}[args.precision],
            "data": "synthetic (seeded generator, ragged batch of linear-kinetics chains)",
            "config": batched_config(args, pk, args.precision,
                                     tuning.get(args.precision, api.get_tuning(nx, args.precision)), world, seq_range),
            "ms_per_step_median": float(np.median(ms)),
            "parity": parity,
            "stage_ms": stage,
            "stage_ms_one_chunk": stage_serial,
            "roofline": roof,
            "gpu_launches": args.steps * launches,
            "clocks": clock_info,
            "generator_seconds": gen_s,
        }
    if not args.no_extras:
        other = precs[1]
        g2 = graph_for(other)
        ms2 = timed_graph(g2, max(3, args.steps // 2))
        del g2
        ms2_max, units2 = reduce_over_ranks(float(np.mean(ms2)), n_fast, dist, dev)
        par2 = check_parity_batch(probs, pk, outs, other) if rank == 0 else None
        loop = run_single_loop(probs, pk, ten, outs, api, torch, stream)
        loop_ms, loop_units = reduce_over_ranks(loop["ms_per_step"], n_fast, dist, dev)
        seq_ms = time_calls(lambda st: api.smoother_batch(batch, precision=args.precision, out=outs, stream=st,
                                                          method="sequential"), 2, 1, stream)
        seq_max, seq_units = reduce_over_ranks(float(np.mean(seq_ms)), n_fast, dist, dev)
        outs.clear()                 # the device outputs are not needed any more
        torch.cuda.empty_cache()
        e2e = run_batched_e2e(args, probs, pk, batch, ten, api, torch, stream, rank)
        e2e_ms, e2e_units = reduce_over_ranks(e2e["ms_per_step"], n_fast, dist, dev)
        if rank == 0:
            line[other + "_batched"] = {"value": units2 / (ms2_max * 1e-3), "ms_per_step": ms2_max,
                                        "tuning": tuning.get(other, api.get_tuning(nx, other)), "parity": par2}
            line["fp64_single_sequence_loop"] = dict(loop, value=loop_units / (loop_ms * 1e-3), ms_per_step=loop_ms)
            line["mixed_batched_over_fp64_single_sequence_loop"] = value / line["fp64_single_sequence_loop"]["value"]
            line["sequential_comparator"] = {
                "value": seq_units / (seq_max * 1e-3), "ms_per_step": seq_max,
                "call": "srtm_smoother_batch_sequential (IMKF and IMS recursions one thread per sequence), "
                        "direct calls, mean of 2 after 1 warm-up"}
            line["e2e"] = dict(e2e, value=e2e_units / (e2e_ms * 1e-3), ms_per_step=e2e_ms)
            if world == 1:
                line["cpu_baseline"] = run_cpu_baseline_batched(args, probs)
    return line


def check_parity_batch(probs, pk, outs, precision):
    """Sampled sequences of the timed batched call (the shortest, the first,
    the last) against the FP64 oracle, every output of each."""
    import oracle
    oracle.build()
    tol = {"fp64": (1e-9, 1e-8), "mixed": (1e-4, 1e-3), "fp32": (1e-4, 1e-3)}[precision]
    n = pk["n_slow"].astype(np.int64)
    off_f = np.concatenate([[0], np.cumsum(n * pk["ratio"])])
    pick = sorted({int(np.argmin(n)), 0, len(probs) - 1})
    e_mean = e_cov = 0.0
    for s_ in pick:
        o = oracle.sequential(probs[s_], slow=False)
        sl = slice(int(off_f[s_]), int(off_f[s_ + 1]))
        e_mean = max(e_mean, rel_err(outs["fast_mean"][sl].cpu().numpy(), o["fast_smooth_mean"]))
        e_cov = max(e_cov, rel_err(outs["fast_cov"][sl].cpu().numpy(), o["fast_smooth_cov"]))
    return {"max_rel_err_mean": e_mean, "max_rel_err_cov": e_cov, "tol": list(tol),
            "ok": bool(e_mean <= tol[0] and e_cov <= tol[1]),
            "checked": f"every fast output of sequences {pick}"}


def run_single_loop(probs, pk, ten, outs, api, torch, stream):
    """The plain FP64 single-sequence path (srtm_smoother) called once per
    sequence of the batch, into the same output buffers, timed as one loop."""
    off_s = np.concatenate([[0], np.cumsum(pk["n_slow"].astype(np.int64))])
    off_f = np.concatenate([[0], np.cumsum(pk["n_slow"].astype(np.int64) * pk["ratio"])])

    def one(s):
        sl_s, sl_f = slice(int(off_s[s]), int(off_s[s + 1])), slice(int(off_f[s]), int(off_f[s + 1]))
        o = {"fast_mean": outs["fast_mean"][sl_f], "fast_cov": outs["fast_cov"][sl_f],
             "slow_mean": outs["slow_mean"][sl_s], "slow_cov": outs["slow_cov"][sl_s]}
        api.smoother(ten["F"][s], ten["Q"][s], ten["H"][s], ten["R"][s], ten["m0"][s], ten["P0"][s],
                     ten["y"][sl_s], int(pk["ratio"][s]), precision="fp64", out=o, stream=stream)

    with torch.cuda.stream(stream):
        for s in range(min(32, len(probs))):
            one(s)
        api.status(stream)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s in range(len(probs)):
            one(s)
        e1.record(stream)
        e1.synchronize()
        api.status(stream)
    ms = e0.elapsed_time(e1)
    return {"value": pk["total_fast"] / (ms * 1e-3), "ms_per_step": ms, "calls": len(probs),
            "api": "srtm_smoother (FP64) once per sequence, same stream"}


def pinned_empty(shape):
    """A page-locked host float64 tensor from torch's pinned allocator
    (cudaHostAlloc: mapped, the device writes it at its host address).  Host
    memory merely registered with cudaHostRegister was measured much slower to
    write from the GPU at this size (~42 GB/s against ~193 GB/s)."""
    import torch
    return torch.empty(shape, dtype=torch.float64, pin_memory=True)


def release_pinned():
    """Hand torch's cached pinned host blocks back to the system."""
    import torch
    fn = getattr(torch._C, "_host_emptyCache", None)
    if fn is not None:
        fn()


def run_batched_e2e(args, probs, pk, batch, ten, api, torch, stream, rank=0):
    """The batched step end to end through the public API: every step copies
    the inputs from pinned host memory into the batch's device buffers and
    replays the captured srtm_smoother_batch call whose outputs -- all of them:
    fast and slow smoothed means and covariances -- are pinned host memory,
    written by the recovery kernel over the CPU-GPU link.  The timed host
    outputs of sampled sequences are checked against the oracle."""
    keys = ("F", "Q", "H", "R", "m0", "P0", "y", "ratio", "n_slow")
    host_in = {}
    for k in keys:
        h = torch.empty(pk[k].shape, dtype=ten[k].dtype, pin_memory=True)
        h.numpy()[...] = pk[k]
        host_in[k] = h
    nx, n_fast, n_slow = pk["F"].shape[1], pk["total_fast"], pk["total_slow"]
    shapes = {"fast_mean": (n_fast, nx), "fast_cov": (n_fast, nx, nx), "slow_mean": (n_slow, nx),
              "slow_cov": (n_slow, nx, nx)}
    t0 = time.perf_counter()
    host_out = {k: pinned_empty(shp) for k, shp in shapes.items()}
    pin_s = time.perf_counter() - t0
    try:
        with torch.cuda.stream(stream):
            api.smoother_batch(batch, precision=args.precision, out=host_out, stream=stream)
            api.status(stream)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream, capture_error_mode="relaxed"):
            api.smoother_batch(batch, precision=args.precision, out=host_out, stream=stream)
        ms = []
        steps = max(2, args.steps // 2)
        with torch.cuda.stream(stream):
            for _ in range(steps + 1):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for k in keys:
                    ten[k].copy_(host_in[k], non_blocking=True)
                g.replay()
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            api.status(stream)
        del g
        ms = ms[1:]
        parity = check_parity_batch(probs, pk, host_out, args.precision) if rank == 0 else None
    finally:
        host_out.clear()
        release_pinned()
    h2d = sum(h.numel() * h.element_size() for h in host_in.values())
    d2h = sum(int(np.prod(shp)) * 8 for shp in shapes.values())
    return {"value": n_fast / (float(np.mean(ms)) * 1e-3), "unit": UNIT, "ms_per_step": float(np.mean(ms)),
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "parity": parity,
            "pin_seconds": pin_s,
            "api": "pinned host inputs copied into the batch's device buffers, then srtm_smoother_batch (CUDA graph) "
                   "with every smoothed output (fast and slow means and covariances) in pinned (cudaHostAlloc) host "
                   "memory, written by the recovery kernel over the CPU-GPU link"}


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.machine()


def run_cpu_baseline_batched(args, probs, seconds=None, pool=None):
    """The oracle on every host core: one sequence per task on spawned worker
    processes (the sequences are independent), the first sequences of the
    batch in order, about ``seconds`` of wall time."""
    from oracle.pool import SequencePool
    seconds = args.cpu_seconds if seconds is None else seconds
    own = pool is None
    pool = SequencePool() if own else pool
    try:
        r = pool.run(probs, seconds)
    finally:
        if own:
            pool.close()
    return {"value": r["fast_steps"] / r["seconds"], "unit": UNIT, "cores": r["workers"], "kind": "oracle",
            "sample": f"the first {r['sequences']} sequences of the batch ({r['fast_steps']} fast steps) in "
                      f"{r['seconds']:.1f} s, one sequence per task on {r['workers']} spawned worker processes "
                      f"({cpu_model()}), FP64 C"}


def recorded_traffic(precision, n_fast, workload="chain4"):
    """DRAM bytes per call of the recovery from the committed ncu summary, if
    the recovery kernel's source is unchanged since the capture.  chain4 is
    captured at full size; the ragged batch (too large for a full ncu capture)
    on its first 64 sequences, scaled to the call by the number of fast steps."""
    import hashlib
    name = {"chain4": f"recover_kernel_chain4_T1e4_{precision}.json",
            "ragged_chains": f"recover_kernel_ragged_chains_first64_{precision}.json"}[workload]
    prof = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(prof):
        return None
    try:
        tr = json.load(open(prof))
        src = open(os.path.join(ROOT, "paper_2410_00627_gb300", "csrc", "kernels.cuh")).read()
        a = src.index("// fast-rate recovery (Remarks 1 and 3)")
        b = src.index("// host-side launch of the templated stages")
        if tr.get("source_sha1") != hashlib.sha1(src[a:b].encode()).hexdigest():
            return None
        if workload == "chain4":
            return float(tr["dram_bytes_per_launch"]) if tr.get("n_fast") == n_fast else None
        return float(tr["dram_bytes_per_launch"]) * n_fast / float(tr["n_fast"])
    except (ValueError, KeyError, OSError):
        return None


def run_e2e(args, prob, api, torch, flush):
    """Same metric through the host-buffer C-ABI entry point: pinned host
    inputs/outputs, H2D copies, the device path and D2H copies in the timed region."""
    def pinned(a):
        t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
        t.numpy()[...] = a
        return t
    ins = {k: pinned(np.ascontiguousarray(getattr(prob, k))) for k in ("F", "Q", "H", "R", "m0", "P0", "y")}
    n_fast = prob.n_slow * prob.ratio
    nx = prob.nx
    outs = {"fast_mean": torch.empty((n_fast, nx), dtype=torch.float64, pin_memory=True),
            "fast_cov": torch.empty((n_fast, nx, nx), dtype=torch.float64, pin_memory=True),
            "slow_mean": torch.empty((prob.n_slow, nx), dtype=torch.float64, pin_memory=True),
            "slow_cov": torch.empty((prob.n_slow, nx, nx), dtype=torch.float64, pin_memory=True)}
    on = {k: v.numpy() for k, v in outs.items()}
    stream = torch.cuda.current_stream()
    args_np = [ins[k].numpy() for k in ("F", "Q", "H", "R", "m0", "P0", "y")]
    for _ in range(3):
        api.smoother_host(*args_np, prob.ratio, precision=args.precision, out=on, stream=stream)
    ms = []
    steps = max(5, args.steps // 2)
    for _ in range(steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        api.smoother_host(*args_np, prob.ratio, precision=args.precision, out=on, stream=stream)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    h2d = sum(a.nbytes for a in args_np)
    d2h = sum(a.nbytes for a in on.values())
    return {"value": n_fast / (float(np.mean(ms)) * 1e-3), "unit": UNIT, "ms_per_step": float(np.mean(ms)),
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "api": "srtm_smoother_host (C-ABI, pinned host buffers: model arrays packed into one H2D copy, "
                   "y read and outputs written by the kernels directly over the CPU-GPU link)"}


def oracle_time(prob, seconds):
    """The FP64 CPU oracle as it stands (sequential IMKF + fast filter + the
    paper's sequential smoother, every fast output), single thread, timed on
    repeated passes over the whole workload for about `seconds`."""
    import oracle
    oracle.build()
    n_fast = prob.n_slow * prob.ratio
    oracle.sequential(prob)  # warm
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.sequential(prob)
        reps += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return reps * n_fast / el, reps, el


def run_cpu_baseline(args, prob):
    v, reps, el = oracle_time(prob, args.cpu_seconds)
    return {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{reps} full passes over the chain4 workload ({prob.n_slow} slow / "
                      f"{prob.n_slow * prob.ratio} fast steps) in {el:.1f} s, 1 thread ({cpu_model()}), FP64 C (-O2)"}


# --------------------------------------------------------------------------- parity of the timed outputs
def check_parity(prob, outs, precision, w=3):
    """The timed call's smoothed outputs against the FP64 oracle: every output
    when the workload has at most 2*10^6 fast steps, else every x_{k,1} and the
    fast outputs of the first and last w intervals.  The slow outputs must be
    the i = l fast rows exactly.  The bench line counts only within tolerance."""
    import oracle
    oracle.build()
    tol = {"fp64": (1e-9, 1e-8), "mixed": (1e-4, 1e-3), "fp32": (1e-4, 1e-3)}[precision]
    N, l = prob.n_slow, prob.ratio
    fm, fc = outs["fast_mean"].cpu().numpy(), outs["fast_cov"].cpu().numpy()
    sm, sc = outs["slow_mean"].cpu().numpy(), outs["slow_cov"].cpu().numpy()
    if N * l <= 2_000_000:
        o = oracle.sequential(prob, slow=False)
        e_mean, e_cov = rel_err(fm, o["fast_smooth_mean"]), rel_err(fc, o["fast_smooth_cov"])
        checked = f"every fast output ({N * l} fast steps)"
    else:
        w = min(w, N)
        head = oracle.sequential(prob, k_lo=0, k_hi=w, slow=False)
        tail = oracle.sequential(prob, k_lo=N - w, k_hi=N, slow=False)
        e_mean = max(rel_err(np.concatenate([fm[:w * l], fm[-w * l:]]),
                             np.concatenate([head["fast_smooth_mean"], tail["fast_smooth_mean"]])),
                     rel_err(fm[0::l], head["first_smooth_mean"]))
        e_cov = max(rel_err(np.concatenate([fc[:w * l], fc[-w * l:]]),
                            np.concatenate([head["fast_smooth_cov"], tail["fast_smooth_cov"]])),
                    rel_err(fc[0::l], head["first_smooth_cov"]))
        checked = f"x_(k,1) of all {N} intervals and every fast output of the first and last {w}"
    slow_views = bool(np.array_equal(sm, fm[l - 1::l]) and np.array_equal(sc, fc[l - 1::l]))
    return {"max_rel_err_mean": e_mean, "max_rel_err_cov": e_cov, "tol": list(tol),
            "ok": bool(e_mean <= tol[0] and e_cov <= tol[1] and slow_views), "checked": checked,
            "slow_outputs_are_the_i_l_rows": slow_views}


# --------------------------------------------------------------------------- error report
REPORT_SIZES = {"ab_kinetics": 100, "chain4": 10_000, "network8": 100_000, "stiff_chain6": 10_000}


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


def report_errors(name, precisions=("fp64", "mixed", "fp32"), n_slow=None, seed=0):
    """Max relative errors (max |x - x_oracle| / max |x_oracle|) of the smoothed
    outputs (a smoother call without filtered outputs, and the record form of a
    call that also asks for them) and the filtered outputs of each precision
    mode against the FP64 oracle, for
    workload `name` at full size: every slow-rate output and the fast-rate
    outputs of the first and last three intervals.  Also the time of the
    smoother call (smoothed outputs only, built-in launch shapes): median of 5
    direct calls after 2 warm-up calls, CUDA events on the calling stream."""
    import torch

    import oracle
    from paper_2410_00627_gb300 import api, build, synth
    build.build()
    api.load()
    oracle.build()
    N = REPORT_SIZES[name] if n_slow is None else n_slow
    prob = synth.WORKLOADS[name](seed=seed, n_slow=N, keep_states=False)
    l = prob.ratio
    w = min(3, N)
    head = oracle.sequential(prob, k_lo=0, k_hi=w)
    tail = oracle.sequential(prob, k_lo=N - w, k_hi=N, slow=False, smooth=True)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")  # noqa: E731
    ins = [dev(getattr(prob, k)) for k in ("F", "Q", "H", "R", "m0", "P0", "y")]
    res, timing = {}, {}
    for prec in precisions:
        try:
            # smoothed outputs only (the recovery form the tuning selects: two-point
            # by default), then with the filtered outputs (the record form)
            sm, _ = api.smoother(*ins, l, precision=prec)
            api.status()
            sr, fi = api.smoother(*ins, l, precision=prec, filtered=api.OUTPUT_KEYS)
            api.status()
        except api.SRTMError as err:   # reported, e.g. a singular solve in the float32 mode
            res[prec] = {"error": str(err)}
            continue
        ms = time_calls(lambda st: api.smoother(*ins, l, precision=prec, out=sm, stream=st), 5, 2,
                        torch.cuda.current_stream())
        timing[prec] = {"ms_per_call": float(np.median(ms)),
                        "fast_states_per_s": N * l / (float(np.median(ms)) * 1e-3)}
        sm = {k: v.cpu().numpy() for k, v in sm.items()}
        sr = {k: v.cpu().numpy() for k, v in sr.items()}
        fi = {k: v.cpu().numpy() for k, v in fi.items()}
        e = {}
        for key, got, ref in (
                ("smoothed fast mean", np.concatenate([sm["fast_mean"][:w * l], sm["fast_mean"][-w * l:]]),
                 np.concatenate([head["fast_smooth_mean"], tail["fast_smooth_mean"]])),
                ("smoothed fast cov", np.concatenate([sm["fast_cov"][:w * l], sm["fast_cov"][-w * l:]]),
                 np.concatenate([head["fast_smooth_cov"], tail["fast_smooth_cov"]])),
                ("smoothed first-state mean (all k)", sm["fast_mean"][0::l], head["first_smooth_mean"]),
                ("smoothed first-state cov (all k)", sm["fast_cov"][0::l], head["first_smooth_cov"]),
                ("smoothed fast mean, record form", np.concatenate([sr["fast_mean"][:w * l], sr["fast_mean"][-w * l:]]),
                 np.concatenate([head["fast_smooth_mean"], tail["fast_smooth_mean"]])),
                ("smoothed fast cov, record form", np.concatenate([sr["fast_cov"][:w * l], sr["fast_cov"][-w * l:]]),
                 np.concatenate([head["fast_smooth_cov"], tail["fast_smooth_cov"]])),
                ("filtered fast mean", np.concatenate([fi["fast_mean"][:w * l], fi["fast_mean"][-w * l:]]),
                 np.concatenate([head["fast_filt_mean"], tail["fast_filt_mean"]])),
                ("filtered fast cov", np.concatenate([fi["fast_cov"][:w * l], fi["fast_cov"][-w * l:]]),
                 np.concatenate([head["fast_filt_cov"], tail["fast_filt_cov"]])),
                ("filtered slow mean (all k)", fi["slow_mean"], head["slow_filt_mean"]),
                ("filtered slow cov (all k)", fi["slow_cov"], head["slow_filt_cov"])):
            e[key] = rel_err(got, ref)
        res[prec] = e
        del sm, sr, fi
        torch.cuda.empty_cache()
    return {"workload": name, "nx": prob.nx, "ny": prob.ny, "ratio": l, "n_slow": N, "n_fast": N * l,
            "errors": res, "timing": timing}


def run_peaks():
    """FP64 and FP32 FMA peaks of GPU 0 (srtm_measure_peak: 300 ms launches of
    independent FMA chains on every SM, fastest of three, three times each),
    with the SM clocks sampled by nvidia-smi while they run; and the CPU-GPU
    link's rates for 4 and 32 GiB moves (srtm_measure_link)."""
    import torch

    from paper_2410_00627_gb300 import api, build
    build.build()
    api.load()
    torch.cuda.init()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.5)
    res = {k: [api.measure_peak(k, 300.0)[0] for _ in range(3)] for k in ("fp64", "fp32")}
    time.sleep(0.3)
    ck = clocks.stop()
    link = {f"{k}_GBps": {f"{g}GiB": api.measure_link(k, g) for g in (4.0, 32.0)} for k in api.LINK_KINDS}
    return {"peaks": "FMA throughput (srtm_measure_peak)", "gpu": torch.cuda.get_device_name(),
            "fp64_gflops": max(res["fp64"]), "fp32_gflops": max(res["fp32"]), "runs": res,
            "sm_mhz_median": ck["sm_mhz"], "sm_max_mhz": ck["sm_max_mhz"], "reasons": ck["reasons"],
            "clock_samples": ck["samples"], "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
            "link": link}


def run_reference(args):
    """Reference arm: the FP64 CPU oracle on the host cores, same workload
    (ragged_chains: the first sequences of the batch, about --cpu-seconds of work
    per step)."""
    if args.workload == "ragged_chains":
        probs, _ = batched_workload(args)
        import oracle
        oracle.build()
        from paper_2410_00627_gb300 import synth
        pk = synth.pack(probs)
        from oracle.pool import SequencePool
        per_step = min(args.cpu_seconds / 2, 60.0 / max(1, args.steps))   # the whole run within a few minutes
        with SequencePool() as pool:
            vals = [run_cpu_baseline_batched(args, probs, per_step / 2, pool) for _ in range(args.warmup)]
            vals = [run_cpu_baseline_batched(args, probs, per_step, pool) for _ in range(args.steps)]
        value = float(np.mean([v["value"] for v in vals]))
        return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator)",
                "config": batched_config(args, pk, "fp64 (CPU oracle)", None),
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": vals[-1]["cores"], "kind": "oracle",
                                 "sample": vals[-1]["sample"]},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    from paper_2410_00627_gb300 import synth  # noqa: F401
    prob = workload(args)
    n_fast = prob.n_slow * prob.ratio
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle.sequential(prob)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.sequential(prob)
        ts.append(time.perf_counter() - t0)
    mean = float(np.mean(ts))
    value = n_fast / mean
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded generator)",
            "config": config_dict(args, prob, "fp64 (CPU oracle)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"the whole workload per step, {args.steps} steps, 1 thread ({cpu_model()})"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return
    if args.peaks:
        print(json.dumps(run_peaks()), flush=True)
        return
    if args.report_errors:
        for name in REPORT_SIZES:
            print(json.dumps(report_errors(name)), flush=True)
        return
    if args.figure:
        for ln in run_figure(args):
            print(json.dumps(ln), flush=True)
        return
    if args.sweep:
        import copy
        for n_slow in (100, 316, 1000, 3162, 10000):
            for prec in ("fp64", "mixed"):
                a = copy.copy(args)
                a.n_slow, a.precision, a.no_extras = n_slow, prec, True
                ln = run_ours(a, 0, 1, None)
                print(json.dumps({"sweep": "chain4", "n_slow": n_slow, "fast_steps": n_slow * 20, "precision": prec,
                                  "value": ln["value"], "unit": UNIT, "ms_per_step": ln["ms_per_step"],
                                  "us_per_call": ln["ms_per_step"] * 1e3, "parity_ok": ln["parity"]["ok"],
                                  "tuning": ln["config"]["tuning"]}), flush=True)
        return
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        torch.cuda.set_device(local % torch.cuda.device_count())
        # NCCL between GPUs; SRTM_DIST_BACKEND=gloo runs the ranks' host-side
        # reductions over gloo (e.g. several ranks sharing one GPU)
        dist.init_process_group(os.environ.get("SRTM_DIST_BACKEND", "nccl"), init_method="env://")
    line = (run_batched if args.workload == "ragged_chains" else run_ours)(args, rank, world, dist)
    if args.workload == "ragged_chains" and world == 1 and not args.no_chain4 and not args.no_extras:
        import copy
        a = copy.copy(args)
        a.workload, a.n_slow, a.tuning = "chain4", 10_000, None
        a.steps, a.warmup = max(5, args.steps), max(3, args.warmup)
        ln = run_ours(a, rank, world, dist)
        line["chain4"] = {k: v for k, v in ln.items() if k not in ("metric", "unit", "n_gpus", "higher_is_better",
                                                                   "scaling", "vs_baseline", "data")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
