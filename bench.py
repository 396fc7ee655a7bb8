#!/usr/bin/env python3
"""Throughput of the vegas+ hot path (one adaptive iteration = one step) on GB300.

Default workload (the largest single-GPU configuration): the 20-D indicator of
the ball of radius 0.5 centred in [0,1]^20 (§1 footnote), N_ev = 1e7 samples
per iteration, N_g = 1000, beta = 0.75, alpha = 0.5, 2^20 hypercubes; map and
integrand in FP32, per-hypercube moments Kahan-compensated FP32, estimate,
reallocation and refinement in FP64.  A step is one vp_step: sampling
(a1-a5), estimate (a6), reallocation (a7) and grid refinement (a8), replayed
from a CUDA graph.  The same JSON line carries, as extra keys, the 8-D
four-peak step (N_ev = 1e6), the 512-integral batch against one integral at a
time, and the served request stream with its p50/p99 latency.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the host cores instead (the reference arm), on whole iterations of the same
workload.

Multi-GPU (torchrun): one independent integral per rank (distinct Philox
counter word 3), no collective on the data path; value = all ranks' integrand
evaluations / max-over-ranks time ("scaling": "weak").
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "ball_d20"
L2_FLUSH_BYTES = 512 << 20   # > 129 MB of L2, written between timed steps
KERNEL_TIMING_ITERS = 10     # eager iterations timing the sampling kernel
# the library measures the sampling launch shape again once the grid has
# adapted (after 4 iterations): warm-up always covers that point
MIN_WARMUP = 5


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", choices=["four_peaks_d8", "ball_d20", "exp_origin_d16",
                                           "bayes_d3", "precond_d8", "batch_mix", "serve"],
                    default="ball_d20",
                    help="ball_d20 (default): the single-integral step on the 20-D ball "
                         "(N_ev = 1e7), with the four-peak, batched and served figures as extra "
                         "keys; four_peaks_d8: the step on the 8-D four peaks (N_ev = 1e6); "
                         "exp_origin_d16: exp(-50|x|) in 16-D "
                         "with the mixed stratification (N_ev = 2.5e5, 2^15 hypercubes); "
                         "bayes_d3: the 3-D posterior with the eight outputs of the Bayesian "
                         "example (means and second moments, FP64, N_ev = 1e5); precond_d8: "
                         "three sharp 8-D peaks with the map trained on 3000 sample points, "
                         "then frozen (N_ev = 1e6); batch_mix: 512 "
                         "integrals per launch against one at a time; serve: continuous batching "
                         "of a Poisson request stream")
    ap.add_argument("--requests", type=int, default=2000,
                    help="serve: requests of the stream served at their arrival times")
    ap.add_argument("--saturated-requests", type=int, default=20000,
                    help="serve: requests queued at once for the saturated rate (the whole "
                         "20k-request stream)")
    ap.add_argument("--no-extras", action="store_true",
                    help="ball_d20: leave out the four-peak, batched and served keys")
    ap.add_argument("--n-ev", type=float, default=None,
                    help="four_peaks_d8: samples per iteration other than the workload's 1e6 "
                         "(a sweep of the step's size; N_st follows Eq. Nst_vegasp)")
    ap.add_argument("--launch", default=None,
                    help="fix the sampling launch shape instead of autotuning it: "
                         "scheme:blocks:threads:cluster:run with scheme static-cluster or tasks")
    return ap.parse_args()


def flops_per_sample(dim, n_peaks):
    """Algorithmic FP32 flops per sample of the fused kernel: the map 4 per axis
    (y N_g, the fraction, the x multiply-add as 2, the J product), the Gaussian
    integrand 3 per axis per peak plus 2 per peak, and 10 for the compensated
    moments (2 plain + 8 Kahan)."""
    return 4 * dim + n_peaks * (3 * dim + 2) + 10


def ops_per_sample(dim, n_peaks, ball=False, expnorm=False):
    """Algorithmic lane operations per sample of the fused kernel (each one
    issue slot of one lane): Philox4x32-10 6 per round (the high and low words
    of two 32x32 products, two key XORs) x 10 rounds x ceil(D/4) calls; the map
    7 per axis (uniform from the bits, y N_g, floor, fraction, table load, x, J);
    the Gaussian integrand 2D + 3 per peak (difference and multiply-add per
    axis, scale, exp2, accumulate), the exponential 2D + 4 (the square root
    besides), the ball 2D + 2 (compare, select); the moments 10 (J f, v^2, two
    compensated adds of 4); the histograms 2 atomic adds per axis."""
    f = n_peaks * (2 * dim + (2 if ball else (4 if expnorm else 3)))
    return 60 * ((dim + 3) // 4) + 7 * dim + f + 10 + 2 * dim


def fp64_ops_per_sample(dim, n_pts, n_par, n_out):
    """Algorithmic FP64 operations per sample of the FP64 kernel on the
    posterior with n_out outputs, counted from the source with every add,
    multiply, division, conversion, floor and library call (exp, log, sqrt)
    as one operation: the map 14 per axis (uniform from the bits 3, y 2,
    y N_g 1, floor 1, fraction 2, increment width 1, x 2, J 2); the
    posterior 27 per point (the model 2 per coefficient, the residual and its
    square, the narrow and wide Gaussians with their normalisations, their
    sum, its log and the running sum) plus the prior 5 per coefficient and 3;
    the moments 5; the histograms 2 per axis; the outputs 3M + 2 M(M+1)/2
    (g_k, v_k, the sums and the products).  Library calls take many FP64
    instructions, so the fraction of the FP64 peak is a lower bound."""
    T = n_out * (n_out + 1) // 2
    post = n_pts * (2 * n_par + 23) + 5 * n_par + 3
    outs = (3 * n_out + 2 * T) if n_out > 1 else 0
    return 14 * dim + post + 5 + 2 * dim + outs


BAYES_OUTPUTS = [(0, -1), (1, -1), (2, -1), (0, 0), (0, 1), (1, 1), (2, 2)]


def ball_flops_per_sample(dim):
    """Algorithmic FP32 flops of the ball workload: the map 4 per axis, the
    ball test 2D + 1, the compensated moments 10."""
    return 4 * dim + 2 * dim + 1 + 10


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            p = [x.strip() for x in l.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ncu summaries of the sampling kernel, one per workload, under profiles/
PROFILE_FILES = {("ball_d20", 10 ** 7): "sample_kernel_ball_d20.txt",
                 ("four_peaks_d8", 10 ** 6): "sample_kernel_four_peaks_d8.txt",
                 ("four_peaks_d8", 10 ** 8): "sample_kernel_four_peaks_d8_n1e8.txt"}
# per-pipe figures the summaries carry, as percentages of the peak sustained
# over ELAPSED cycles (ncu's .pct_of_peak_sustained_elapsed)
PIPE_KEYS = ["sm__pipe_fma_cycles_active", "sm__pipe_alu_cycles_active",
             "sm__inst_executed_pipe_xu", "smsp__issue_active"]


def profile_figures(workload, kernel_src_hash, n_ev):
    """The committed ncu summary of the workload's sampling kernel at this N_ev
    (the traffic per sample grows with the hypercubes' moments, so it is kept
    per size), if it was taken on the current kernel source:
    {"traffic_per_sample": DRAM bytes per sample of the profiled launch,
    "pipes_pct_elapsed": {...}}; else None."""
    name = PROFILE_FILES.get((workload, int(n_ev)))
    if not name:
        return None
    try:
        text = open(os.path.join(ROOT, "profiles", name)).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_sha1") != kernel_src_hash:
        return None
    try:
        out = {"traffic_per_sample": float(vals["dram_bytes_per_launch"].split()[0]) /
               float(vals["profiled_samples"].split()[0])}
        out["pipes_pct_elapsed"] = {k: float(vals[k + "_pct_elapsed"].split()[0])
                                    for k in PIPE_KEYS if k + "_pct_elapsed" in vals}
        return out
    except (KeyError, ValueError, IndexError, ZeroDivisionError):
        return None


def kernel_source_hash():
    import hashlib
    h = hashlib.sha1()
    for f in ["sample_impl.cuh", "vp_internal.cuh"]:
        h.update(open(os.path.join(ROOT, "paper_2009_05112_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def cpu_baseline(prob, seconds=12.0, out_mono=None, data=None):
    """The FP64 CPU oracle, as it stands, on this host: whole iterations of the
    same workload until ~seconds of CPU time; one thread.  data: sample points
    the map is first trained on (untimed), the map then frozen."""
    import oracle
    o = oracle.VegasPlus(dim=prob.dim, lo=prob.lo, hi=prob.hi, n_g=prob.n_g, n_ev=prob.n_ev,
                         alpha=prob.alpha, beta=prob.beta, seed=prob.seed, kind=prob.kind,
                         prm=prob.prm, n_st_axis=prob.n_st_axis, mixed=prob.mixed,
                         out_mono=out_mono)
    if data is not None:
        o.precondition(data, n_iter=10)
        o.alpha = 0.0
    evals, t0, its = 0, time.perf_counter(), 0
    while True:
        n = int(o.offsets[-1])
        o.iterate()
        o.adapt()
        evals += n
        its += 1
        el = time.perf_counter() - t0
        if el >= seconds or its >= 400:
            break
    return {"value": evals / el, "unit": "integrand evals/s", "cores": 1, "kind": "oracle",
            "sample": "%d whole iterations (%s, N_ev=%d, D=%d, N_g=%d) of the FP64 C "
                      "oracle, single thread, %.1f s" % (its, prob.name, prob.n_ev, prob.dim,
                                                         prob.n_g, el),
            "host": host_cpu()}


def host_cpu():
    """The host's CPU as the system reports it: lscpu's model name (or
    /proc/cpuinfo's), the machine type and the logical CPU count."""
    import platform
    import subprocess
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"model": model, "machine": platform.machine(), "nproc": os.cpu_count()}


def _oracle_worker(job):
    """One process of the all-cores baseline: the single-thread oracle on the
    workload (its own Philox counter word 3) for ~seconds; (evals, seconds)."""
    name, seed_id, seconds = job
    import oracle
    from paper_2009_05112_gb300 import inputs
    prob = getattr(inputs, name)()
    o = oracle.VegasPlus(dim=prob.dim, lo=prob.lo, hi=prob.hi, n_g=prob.n_g, n_ev=prob.n_ev,
                         alpha=prob.alpha, beta=prob.beta, seed=prob.seed, kind=prob.kind,
                         prm=prob.prm, integral_id=seed_id)
    evals, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        evals += int(o.offsets[-1])
        o.iterate()
        o.adapt()
    return evals, time.perf_counter() - t0


def cpu_baseline_all_cores(name, seconds=12.0):
    """The oracle as it stands on every host core: one spawned process per
    core, each running the single-thread oracle on the workload; evals/s
    summed over the processes (each timed on its own)."""
    import multiprocessing as mp
    cores = max(1, min(os.cpu_count() or 1, 128))
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_worker, [(name, k, seconds) for k in range(cores)])
    value = sum(e / s for e, s in res)
    return {"value": value, "unit": "integrand evals/s", "cores": cores, "kind": "oracle",
            "sample": "%d processes, each the single-thread FP64 C oracle on whole iterations "
                      "of %s for ~%.0f s" % (cores, name, seconds)}


def cpu_baseline_batch(probs, n_it, seconds=12.0):
    """The oracle on the batch's integrals one after another (whole runs of
    n_it iterations) until ~seconds of CPU time: a bounded sample of the
    512-integral job; one thread."""
    import oracle
    evals, done, t0 = 0, 0, time.perf_counter()
    for p in probs:
        o = oracle.VegasPlus(dim=p.dim, lo=p.lo, hi=p.hi, n_g=p.n_g, n_ev=p.n_ev, alpha=p.alpha,
                             beta=p.beta, seed=p.seed, kind=p.kind, prm=p.prm,
                             integral_id=p.integral_id)
        for _ in range(n_it):
            evals += int(o.offsets[-1])
            o.iterate()
            o.adapt()
        done += 1
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    return {"value": evals / el, "unit": "integrand evals/s", "cores": 1, "kind": "oracle",
            "sample": "the first %d of the 512 integrals, %d iterations each, FP64 C oracle, "
                      "single thread, %.1f s" % (done, n_it, el)}


def cpu_baseline_serve(probs, rules, seconds=12.0):
    """The oracle serving the stream's requests one after another, each until
    its stop rule (the §2.5 combination of iterations >= discard reaching
    sdev <= rtol |mean| after min_meas of them, or max_it iterations), until
    ~seconds of CPU time; one thread."""
    import oracle
    done, evals, t0 = 0, 0, time.perf_counter()
    for p, r in zip(probs, rules):
        o = oracle.VegasPlus(dim=p.dim, lo=p.lo, hi=p.hi, n_g=p.n_g, n_ev=p.n_ev, alpha=p.alpha,
                             beta=p.beta, seed=p.seed, kind=p.kind, prm=p.prm,
                             integral_id=p.integral_id)
        for it in range(r["max_it"]):
            evals += int(o.offsets[-1])
            o.iterate()
            o.adapt()
            if it + 1 - r["discard"] >= r["min_meas"]:
                c = oracle.combine(o.I, o.var, r["discard"])
                if c["sdev"] <= r["rtol"] * abs(c["mean"]):
                    break
        done += 1
        if time.perf_counter() - t0 >= seconds:
            break
    el = time.perf_counter() - t0
    return {"value": done / el, "unit": "requests/s", "cores": 1, "kind": "oracle",
            "evals_per_s": evals / el,
            "sample": "the first %d requests of the stream served one at a time by the FP64 C "
                      "oracle, single thread, %.1f s" % (done, el)}


def run_reference(args):
    """The reference arm: the FP64 C oracle, as it stands, on this host, on
    whole iterations of the same workload as our arm (W untimed, then K
    timed); rank 0 alone."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2009_05112_gb300 import inputs
    name = args.workload if args.workload in ("ball_d20", "four_peaks_d8") else WORKLOAD
    prob = getattr(inputs, name)()
    o = oracle.VegasPlus(dim=prob.dim, lo=prob.lo, hi=prob.hi, n_g=prob.n_g, n_ev=prob.n_ev,
                         alpha=prob.alpha, beta=prob.beta, seed=prob.seed, kind=prob.kind,
                         prm=prob.prm)
    for _ in range(args.warmup):
        o.iterate()
        o.adapt()
    evals = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        evals += int(o.offsets[-1])
        o.iterate()
        o.adapt()
    el = time.perf_counter() - t0
    v = evals / el
    line = {"metric": "integrand evals/s", "value": v, "unit": "integrand evals/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": name, "dim": prob.dim, "n_ev": prob.n_ev, "n_g": prob.n_g,
                       "alpha": prob.alpha, "beta": prob.beta},
            "cpu_baseline": {"value": v, "unit": "integrand evals/s", "cores": 1,
                             "kind": "oracle",
                             "sample": "%d whole iterations of %s (N_ev=%d) after %d warm-up, "
                                       "single thread" % (args.steps, name, prob.n_ev,
                                                          args.warmup),
                             "host": host_cpu()},
            "e2e": {"value": v, "unit": "integrand evals/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _integral(g, prob, ball, late_half=False):
    """The combined estimate: all iterations, or for the ball (whose first
    iterations may see no sample inside it, i.e. exact zeros) the last 10, or
    (late_half: a peak the first iterations miss, with errors they
    underestimate, §3.2) the second half of them."""
    if ball or late_half:
        n_it = g.info()[2]  # (N_st, N_h, iterations done)
        keep = n_it // 2 if late_half else 10
        r = g.result(discard=max(0, n_it - keep))
        return {"mean": r["mean"], "sdev": r["sdev"], "iterations": "last %d" % keep}
    r = g.result()
    return {"mean": r["mean"], "sdev": r["sdev"]}


def rank_problem(prob, rank):
    """The integral a rank runs: the same problem with Philox counter word 3 =
    rank, so that the ranks draw independent samples (no data exchange)."""
    prob.integral_id = rank
    return prob


def reduce_over_ranks(total_ms, evals, dist, device):
    """Whole-job figures over the ranks: the slowest rank's time (MAX) and all
    ranks' integrand evaluations (SUM).  `device` holds the reduction tensors
    ("cuda" under NCCL, "cpu" under gloo)."""
    import torch
    t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    e = torch.tensor([float(evals)], device=device, dtype=torch.float64)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), float(e.item())


def _problem(workload, inputs, vegasp, n_ev=None):
    """(problem, peaks, extra outputs, precision) of a single-integral workload."""
    if workload == "ball_d20":
        return inputs.ball_d20(), 1, None, vegasp.VP_FP32
    if workload == "exp_origin_d16":
        return inputs.exp_origin(dim=16), 1, None, vegasp.VP_FP32
    if workload == "bayes_d3":
        return (inputs.posterior(dim=3, n_ev=100_000, n_g=1000), 1, BAYES_OUTPUTS,
                vegasp.VP_FP64)
    if workload == "precond_d8":
        return inputs.three_sharp_peaks_d8(n_ev=1_000_000), 3, None, vegasp.VP_FP32
    prob = inputs.four_peaks_d8(**({"n_ev": int(n_ev)} if n_ev else {}))
    return prob, 4, None, vegasp.VP_FP32


def _timed_steps(g, steps, stream, flush, clk_index, world=1, dist=None):
    """K steps, L2 flushed before each, CUDA events around each graph launch
    on the launching stream; (total ms, evaluations, clocks summary)."""
    import torch
    n0 = g.result()["n_eval"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(clk_index) as clk:
        for k in range(steps):
            flush.fill_(k & 0xff)           # evict L2 between timed steps
            ev[k][0].record(stream)
            g.step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    return total_ms, g.result()["n_eval"] - n0, clk.summary()


def _sampling_ms(g, flush):
    """The sampling kernel's own duration: CUDA events around its launch on
    its stream, in eager iterations of the same integral right after the timed
    steps (the step graph carries no events: as graph nodes they would add
    microseconds to every step); L2 flushed before each, as in the timed
    steps.  Mean over KERNEL_TIMING_ITERS."""
    import torch
    ms, whole = [], []
    s = torch.cuda.current_stream()
    for k in range(KERNEL_TIMING_ITERS):
        flush.fill_(k & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        g.iterate()
        g.adapt()
        e1.record(s)
        ms.append(g.last_sample_ms())
        e1.synchronize()
        whole.append(e0.elapsed_time(e1))
    # the same iterations' estimate -> allocation -> offsets (and k_refine beside
    # them): the eager iteration less its sampling launch
    _LAST_CHAIN_MS[0] = sum(w - m for w, m in zip(whole, ms)) / len(ms)
    return sum(ms) / len(ms)


_LAST_CHAIN_MS = [0.0]


def _chain_view(n_hc, dim, n_g, hbm_gbs):
    """The estimate -> allocation -> offsets chain (steps a6-a7) against HBM:
    algorithmic bytes per iteration -- per hypercube S1, S2, n_h read, d_h
    written and the other buffer's S1, S2 cleared (44 B), d_h read and n_h
    written (12 B), n_h read and the offset written (12 B); the other
    histogram buffer cleared (12 B per increment) -- over the chain's time:
    CUDA events around each eager iteration (iterate + adapt) less its
    sampling launch, in the iterations that time the sampling kernel (k_refine
    runs beside the chain on its side stream)."""
    nbytes = 68.0 * n_hc + 12.0 * dim * n_g
    ms = _LAST_CHAIN_MS[0]
    out = {"bytes_per_iteration": nbytes, "ms": ms, "peak_gbs": hbm_gbs,
           "note": "estimate, allocation and offsets, eager iterations less the sampling "
                   "launch: an upper bound on the chain in the step graph (eager launches "
                   "add host gaps and run k_refine after the estimate, not beside it), so "
                   "frac is a lower bound; peak = MEASURED_PEAKS.json hbm_gbs (of measured)"}
    if ms > 0:
        out["achieved_gbs"] = nbytes / (ms * 1e-3) / 1e9
        out["frac"] = out["achieved_gbs"] / hbm_gbs
    return out


_ATOMIC_RATES = {}


def _atomic_view(g, vegasp, dim, samples_per_step, k1_ms, n_sample=65536):
    """The sampling kernel against the shared-memory atomic bound of its
    histograms (§2.3 d_i): D 32-bit count adds per sample and D FP32 sum adds
    per sample whose J f is nonzero, at the rates the library's probe measures
    on this device; the share of nonzero samples from n_sample samples of the
    current allocation evaluated by the kernel's own code (vp_eval_samples)."""
    import numpy as np
    if not _ATOMIC_RATES:
        _ATOMIC_RATES["u32"] = vegasp.shared_atomic_rate(False)
        _ATOMIC_RATES["f32"] = vegasp.shared_atomic_rate(True)
    n_h, off = g.alloc()
    total = int(off[-1])
    rng = np.random.default_rng(12345)
    s = rng.integers(0, total, size=n_sample).astype(np.uint64)
    h = (np.searchsorted(off, s, side="right") - 1).astype(np.uint64)
    j = (s - off[h.astype(np.int64)]).astype(np.uint32)
    f = g.eval_samples(h, j, g.result()["n_it"])[3]
    nz = float(np.count_nonzero(f) / n_sample)
    counts, sums = dim * samples_per_step, dim * nz * samples_per_step
    bound_ms = (counts / _ATOMIC_RATES["u32"] + sums / _ATOMIC_RATES["f32"]) * 1e3
    return {"bound": "shared-memory atomics", "count_adds_per_launch": counts,
            "sum_adds_per_launch": sums, "nonzero_share": nz,
            "peak_u32_adds_per_s": _ATOMIC_RATES["u32"], "peak_f32_adds_per_s": _ATOMIC_RATES["f32"],
            "bound_ms": bound_ms, "frac": bound_ms / k1_ms,
            "note": "time the histogram adds alone would take at the rates measured live by "
                    "vp_shared_atomic_rate (random increments, 20 axes x 1000, one 768-thread "
                    "CTA per SM) over the kernel's CUDA-event time; the nonzero share sampled "
                    "from %d samples of the current allocation" % n_sample}


def _sample_roofline(workload, prob, n_peaks, samples_per_step, k1_ms, step_ms, n_sm,
                     clocks, max_mhz, atomics=None):
    """The sampling kernel against the FP32 roofline: algorithmic FP32 flops
    per sample (counted from the source, an FMA as 2) x samples per launch /
    its CUDA-event duration, over SMs x 128 lanes x 2 flops x the maximum SM
    clock; the issue-slot view (algorithmic lane operations over SMs x 128 x
    clock) and the ncu pipe figures of the committed summary beside it."""
    ball = workload == "ball_d20"
    expo = workload == "exp_origin_d16"
    flops = (ball_flops_per_sample(prob.dim) if ball else
             flops_per_sample(prob.dim, n_peaks) + (n_peaks if expo else 0))
    ops = ops_per_sample(prob.dim, n_peaks, ball, expnorm=expo)
    fp32_peak = n_sm * 128 * 2 * max_mhz * 1e6 / 1e12   # TFLOP/s at the maximum SM clock
    issue_peak = n_sm * 128 * max_mhz * 1e6 / 1e12      # lane operations/s, Tops/s
    tflops = flops * samples_per_step / (k1_ms / 1e3) / 1e12
    tops = ops * samples_per_step / (k1_ms / 1e3) / 1e12
    prof = profile_figures(workload, kernel_source_hash(), prob.n_ev)
    roof = {"bound": "alu", "achieved": tflops, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": tflops / fp32_peak,
            "traffic": (prof["traffic_per_sample"] * samples_per_step) if prof else None,
            "kernel": "k_sample (fused a1-a5)", "kernel_ms": k1_ms,
            "kernel_ms_note": "CUDA events around the sampling launch on its stream, mean of "
                              "%d eager iterations after the timed steps" % KERNEL_TIMING_ITERS,
            "kernel_share_of_step": k1_ms / step_ms,
            "flops_per_sample": flops,
            "peak_note": "FP32 peak = %d SMs x 128 lanes x 2 flops x %.0f MHz (maximum SM clock; "
                         "MEASURED_PEAKS.json records no FP32 figure); algorithmic FP32 flops "
                         "counted from the kernel source, an FMA as 2" % (n_sm, max_mhz),
            "issue_view": {"achieved_tops": tops, "peak_tops": issue_peak,
                           "frac": tops / issue_peak, "ops_per_sample": ops,
                           "note": "algorithmic lane operations (Philox, map, integrand, "
                                   "moments, histogram atomics) over issue slots"},
            "ncu_pct_of_peak_elapsed": prof["pipes_pct_elapsed"] if prof else None}
    if atomics is not None:
        roof["atomics_view"] = atomics
    if clocks.get("sm_mhz"):
        roof["frac_at_measured_clock"] = tflops / (n_sm * 128 * 2 * clocks["sm_mhz"] * 1e6 / 1e12)
    return roof


def _single_summary(workload, args, inputs, vegasp, flush, n_sm, max_mhz):
    """A secondary single-integral line: device-timed steps and the sampling
    kernel's FP32 fraction, as the main line measures them."""
    import torch
    prob, n_peaks, out_mono, precision = _problem(workload, inputs, vegasp)
    g = vegasp.Integrator.from_problem(prob, precision=precision, out_mono=out_mono)
    for _ in range(max(args.warmup, MIN_WARMUP)):
        g.step()
    total_ms, evals, clocks = _timed_steps(g, args.steps, torch.cuda.current_stream(), flush,
                                           int(os.environ.get("LOCAL_RANK", "0")))
    k1 = _sampling_ms(g, flush)
    roof = _sample_roofline(workload, prob, n_peaks, evals / args.steps, k1,
                            total_ms / args.steps, n_sm, clocks, max_mhz,
                            _atomic_view(g, vegasp, prob.dim, evals / args.steps, k1))
    out = {"value": evals / (total_ms / 1e3), "unit": "integrand evals/s",
           "ms_per_step": total_ms / args.steps, "steps": args.steps,
           "n_ev": prob.n_ev, "dim": prob.dim, "n_hc": g.n_hc,
           "kernel_ms": k1, "fp32_frac": roof["frac"], "issue_frac": roof["issue_view"]["frac"],
           "atomics_frac": roof["atomics_view"]["frac"],
           "chain": _chain_view(g.n_hc, prob.dim, prob.n_g,
                                measured_peaks().get("hbm_gbs", 6800.0)),
           "traffic": roof["traffic"], "ncu_pct_of_peak_elapsed": roof["ncu_pct_of_peak_elapsed"],
           "clocks": clocks, "sample_launch": g.tuning(),
           "integral": dict(_integral(g, prob, False), exact=prob.exact)}
    g.close()
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2009_05112_gb300 import build as _build
    from paper_2009_05112_gb300 import inputs, vegasp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    _build.build()
    vegasp.use_torch_allocator()
    ball = args.workload == "ball_d20"
    expo = args.workload == "exp_origin_d16"
    bayes = args.workload == "bayes_d3"
    precond = args.workload == "precond_d8"
    prob, n_peaks, out_mono, precision = _problem(args.workload, inputs, vegasp, args.n_ev)
    prob = rank_problem(prob, rank)
    stream = torch.cuda.current_stream()
    g = vegasp.Integrator.from_problem(prob, precision=precision, out_mono=out_mono)
    training = None
    data = None
    if precond:  # §4.2: the map trained on 3000 points, then frozen
        data = inputs.peak_samples(prob, 3000, seed=0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.precondition(data, n_iter=10)
        training = {"points": 3000, "passes": 10,
                    "ms": 1e3 * (time.perf_counter() - t0),
                    "note": "vp_precondition wall clock (host copies of the data included)"}
        g.set_damping(0.0, prob.beta)
    launch = None
    if args.launch:
        sch, blk, thr, cl, run = args.launch.split(":")
        launch = (sch, int(blk), int(thr), int(cl), int(run))
        g.set_tuning(*launch)
    for _ in range(max(args.warmup, MIN_WARMUP)):
        g.step()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    total_ms, evals, clocks = _timed_steps(g, args.steps, stream, flush, local, world, dist)
    t_max = total_ms
    evals_all = evals
    if world > 1:
        t_max, evals_all = reduce_over_ranks(total_ms, evals, dist, "cuda")
        dist.barrier()
    value = evals_all / (t_max / 1e3)

    k1_avg_ms = _sampling_ms(g, flush)

    # end to end through the public API with host buffers: create from host
    # parameters (H2D), steps each reading its estimate (I_j, sigma_j^2) back
    # into host memory (D2H; vp_step_read returns it one call later, so the
    # copy overlaps the next step), and the final combined result
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g2 = vegasp.Integrator.from_problem(prob, precision=precision, out_mono=out_mono)
    if precond:
        g2.precondition(data, n_iter=10)
        g2.set_damping(0.0, prob.beta)
    if launch:
        g2.set_tuning(*launch)
    reads = []
    for _ in range(args.steps):
        got = g2.step_read()
        if got is not None:
            reads.append(got)
    reads.append(g2.step_read_flush())
    r2 = g2.result()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_evals = r2["n_eval"]
    assert len(reads) == args.steps and reads[-1][0] == r2["last_i"]
    g2.close()
    h2d = (prob.prm.size * 8 + 2 * prob.dim * 8 + prob.dim * (prob.n_g + 1) * 8 +
           prob.dim * prob.n_g * 8 + g.n_hc * 8 + 64)  # blob, box, grid, FP32 table, d_h, state
    d2h = 16 + (64 + args.steps * 16) / args.steps      # the step's estimate + the final result

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    peaks = measured_peaks()
    max_mhz = peaks.get("sm_max_mhz", 2070.0)
    samples_per_step = evals / args.steps
    step_ms = total_ms / args.steps
    timing_note = ("CUDA events around the sampling launch on its stream, mean of %d eager "
                   "iterations after the timed steps" % KERNEL_TIMING_ITERS)
    if bayes:
        # FP64 path: bound by the FP64 pipe; peak from the nominal 1.25 TFLOP/s
        # (an FMA counted as 2 flops), i.e. 0.625e12 FP64 lane instructions/s
        n_pts, n_par = int(prob.prm[0]), int(prob.prm[1])
        ops = fp64_ops_per_sample(prob.dim, n_pts, n_par, 1 + len(out_mono))
        fp64_peak = 1.25 / 2
        k1_tops = ops * samples_per_step / (k1_avg_ms / 1e3) / 1e12
        roof = {"bound": "fp64", "achieved": k1_tops, "peak": fp64_peak, "unit": "Tops/s",
                "frac": k1_tops / fp64_peak, "traffic": None,
                "kernel": "k_sample (fused a1-a5, FP64, 8 outputs)", "kernel_ms": k1_avg_ms,
                "kernel_ms_note": timing_note,
                "kernel_share_of_step": k1_avg_ms / step_ms,
                "ops_per_sample": ops,
                "peak_note": "FP64 lane instructions per second from the nominal 1.25 TFLOP/s "
                             "(fallback figure; FMA = 2 flops); library calls counted as one "
                             "operation each, so frac is a lower bound"}
    else:
        roof = _sample_roofline(args.workload, prob, n_peaks, samples_per_step, k1_avg_ms,
                                step_ms, n_sm, clocks, max_mhz,
                                _atomic_view(g, vegasp, prob.dim, samples_per_step, k1_avg_ms))
    if precond:
        h2d += data.size * 8
    integrand = ("ball" if ball else "exp(-50|x|), mixed strata %s" % list(g.strata()) if expo
                 else "three exp(-1e4 (x - r_i)^2) peaks, map trained on 3000 points then frozen"
                 if precond
                 else "App. B posterior (50 points), outputs f, f p1, f p2, f w, f p1^2, "
                      "f p1 p2, f p2^2, f w^2" if bayes else "gaussian peaks")
    prec_note = ("fp64 map, integrand, moments and outputs" if bayes else
                 "fp32 map/integrand, Kahan fp32 moments, fp64 estimate")
    line = {"metric": "integrand evals/s", "value": value, "unit": "integrand evals/s",
            "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, MIN_WARMUP),
            "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if bayes else "f32", "data": "synthetic",
            "config": {"workload": args.workload, "dim": prob.dim, "n_ev": prob.n_ev,
                       "n_g": prob.n_g, "alpha": prob.alpha, "beta": prob.beta,
                       "peaks": n_peaks, "integrand": integrand, "n_hc": g.n_hc,
                       "precision": prec_note,
                       "l2": "flushed between timed steps (512 MiB write)",
                       "parallelism": "one integral per GPU" if world > 1 else "single GPU"},
            "e2e": {"value": e2e_evals / e2e_s, "unit": "integrand evals/s",
                    "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h,
                    "note": "create from host parameters + %d steps, each step's estimate "
                            "copied to host memory (vp_step_read, read one call later) + the "
                            "final result, wall clock" % args.steps},
            "roofline": roof, "clocks": clocks,
            "chain": _chain_view(g.n_hc, prob.dim, prob.n_g, peaks.get("hbm_gbs", 6800.0)),
            # sample, estimate, alloc, offsets, refine (+ the task prefix for the task
            # kernel, + the several-outputs estimate)
            "gpu_launches": (5 + (g.tuning()["scheme"] == "tasks") + bayes) * args.steps,
            "sample_launch": g.tuning(),
            "integral": dict(_integral(g, prob, ball, late_half=expo), exact=prob.exact)}
    if bayes:
        r = g.result_multi()
        line["integral"]["means (p1, p2, w)"] = [float(v) for v in r["mean"][1:4] / r["mean"][0]]
    if training:
        line["training"] = training
    g.close()
    if ball and world == 1 and not args.no_extras:
        # the other terms of the metric, measured in the same run
        line["four_peaks_d8"] = _single_summary("four_peaks_d8", args, inputs, vegasp, flush,
                                                n_sm, max_mhz)
        del flush
        torch.cuda.empty_cache()
        line["batched_vs_plain"] = batch_summary(args, inputs, vegasp)
        line["served"] = serve_summary(args, inputs, vegasp)
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(prob, out_mono=out_mono, data=data)
        if args.workload in ("four_peaks_d8", "ball_d20"):
            line["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores(args.workload)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def batch_summary(args, inputs, vegasp):
    """512 integrals (D 2..12, N_ev 1e4..1e6, 1-4 Gaussian peaks, N_g = 500,
    15 iterations) in one persistent launch per iteration: device-timed steps
    of the batch, then the whole batched job against the same integrals run
    one at a time through the single-integral path (wall clock, same samples,
    so equal relative error)."""
    import torch
    probs = inputs.batch_mix(n=512, seed=1)
    n_it = 15
    stream = torch.cuda.current_stream()
    # device-timed steps of the batched job (the first W iterations warm up)
    bt = vegasp.Batch(probs, precision=vegasp.VP_FP32)
    for _ in range(max(args.warmup, MIN_WARMUP)):
        bt.step()
    n0 = sum(r["n_eval"] for r in bt.results())
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    torch.cuda.synchronize()
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for k in range(args.steps):
            flush.fill_(k & 0xff)
            ev[k][0].record(stream)
            bt.step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    evals = sum(r["n_eval"] for r in bt.results()) - n0
    bt.close()
    del flush
    # whole jobs, wall clock: batched and one integral at a time (same samples)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    bt = vegasp.Batch(probs, precision=vegasp.VP_FP32).run(n_it)
    rb = bt.results()
    torch.cuda.synchronize()
    wall_b = time.perf_counter() - t0
    evals_b = sum(r["n_eval"] for r in rb)
    bt.close()
    t0 = time.perf_counter()
    evals_p = 0
    rel_p, rel_b = [], []
    for i, p in enumerate(probs):
        g = vegasp.Integrator.from_problem(p, precision=vegasp.VP_FP32).run(n_it)
        r = g.result()
        evals_p += r["n_eval"]
        rel_p.append(r["sdev"] / abs(r["mean"]) if r["mean"] else float("inf"))
        rel_b.append(rb[i]["sdev"] / abs(rb[i]["mean"]) if rb[i]["mean"] else float("inf"))
        g.close()
    torch.cuda.synchronize()
    wall_p = time.perf_counter() - t0
    return {"workload": "batch_mix_512", "integrals": 512, "iterations": n_it,
            "device_evals_per_s": evals / (total_ms / 1e3),
            "device_ms_per_step": total_ms / args.steps, "steps": args.steps,
            "wall_s_batched": wall_b, "wall_s_plain": wall_p,
            "speedup_wall": wall_p / wall_b,
            "evals_per_s_batched": evals_b / wall_b,
            "evals_per_s_plain": evals_p / wall_p,
            "median_rel_err_batched": statistics.median(rel_b),
            "median_rel_err_plain": statistics.median(rel_p),
            "note": "device: graph steps of all 512 integrals, L2 flushed between; wall: whole "
                    "jobs (create from host parameters, 15 iterations, host read of every "
                    "result), batched vs one integral at a time through the single-integral "
                    "path, same samples",
            "clocks": clk.summary()}


def run_batch(args):
    """The batched workload on its own line."""
    import torch
    from paper_2009_05112_gb300 import build as _build
    from paper_2009_05112_gb300 import inputs, vegasp
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    _build.build()
    vegasp.use_torch_allocator()
    b = batch_summary(args, inputs, vegasp)
    line = {"metric": "integrand evals/s", "value": b["device_evals_per_s"],
            "unit": "integrand evals/s", "n_gpus": 1, "steps": args.steps,
            "warmup": max(args.warmup, MIN_WARMUP),
            "ms_per_step": b["device_ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch_mix_512", "integrals": 512, "dim": "2..12",
                       "n_ev": "log-uniform 1e4..1e6", "n_g": 500, "iterations": 15,
                       "l2": "flushed between timed steps (512 MiB write)"},
            "e2e": {"value": b["evals_per_s_batched"], "unit": "integrand evals/s",
                    "note": "whole batched job (create from host parameters, 15 graph steps, "
                            "host read of all results), wall clock"},
            "batched_vs_plain": b, "clocks": b["clocks"]}
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_batch(inputs.batch_mix(n=512, seed=1), 15)
    print(json.dumps(line), flush=True)


def _serve_once(vegasp, stream_t, probs, rules, max_active, paced):
    """Feeds the request stream to a server whose worker thread steps while the
    caller submits: at the stream's arrival times (paced) or all at once.
    Returns (per-request results, wall seconds first submit -> last done, stats)."""
    srv = vegasp.Server(max_active=max_active)
    srv.start()
    t0 = vegasp.clock()
    for k, (p, r) in enumerate(zip(probs, rules)):
        if paced:
            delay = t0 + stream_t[k] - vegasp.clock()
            if delay > 0:
                time.sleep(delay)
        srv.submit(p, precision=vegasp.VP_FP32, tag=k, **r)
    srv.wait(len(probs), timeout_s=600)
    got = []
    while len(got) < len(probs):
        got += srv.poll()
    srv.stop()
    stats = srv.stats()
    srv.close()
    wall = max(r["t_done"] for r in got) - t0
    return got, wall, stats


def _serve_figures(got, wall, st, probs):
    import numpy as np
    lat = np.array([r["t_done"] - r["t_submit"] for r in got]) * 1e3
    d21 = np.array([probs[r["tag"]].dim == 21 for r in got])
    rel = np.array([r["sdev"] / abs(r["mean"]) if r["mean"] else float("inf") for r in got])
    return {"requests": len(got), "requests_per_s": len(got) / wall, "wall_s": wall,
            "evals_per_s": sum(r["n_eval"] for r in got) / wall,
            "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)),
            "p50_ms_d3": float(np.percentile(lat[~d21], 50)),
            "p50_ms_d21": float(np.percentile(lat[d21], 50)),
            "converged_frac": float(np.mean([r["converged"] for r in got])),
            "zero_estimates": int(sum(1 for r in got if not r["mean"])),
            "median_rel_err": float(np.median(rel)),
            "mean_iterations": float(np.mean([r["n_iter"] for r in got])),
            "steps": st["steps"], "busy_s": st["busy_s"],
            "peak_state_mib": st["bytes_peak"] / 2 ** 20}


def serve_summary(args, inputs, vegasp):
    """A Poisson stream of integration requests (mean 200/s; 70% D = 3, 30%
    D = 21 Bayesian-posterior integrands, 50 points each, rtol 1e-3): the
    first args.requests served at their arrival times by continuous batching
    (every admitted request advances one iteration per server step) and one
    request at a time (max_active = 1), with p50/p99 latency; the saturated
    rates with requests queued at once (the whole stream of
    args.saturated_requests batched; the first args.requests one at a time)."""
    rate = 200.0
    n_all = max(args.requests, args.saturated_requests)
    stream_t, probs, rules = inputs.serve_stream(n_all, rate=rate, seed=0)
    n = args.requests
    # warm-up: a few requests through both configurations
    _serve_once(vegasp, stream_t[:8], probs[:8], rules[:8], 0, False)
    _serve_once(vegasp, stream_t[:8], probs[:8], rules[:8], 1, False)
    out = {}
    with Clocks(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        for name, max_active, paced, m in [("served", 0, True, n), ("plain", 1, True, n),
                                           ("served_saturated", 0, False,
                                            args.saturated_requests),
                                           ("plain_saturated", 1, False, n)]:
            got, wall, st = _serve_once(vegasp, stream_t[:m], probs[:m], rules[:m], max_active,
                                        paced)
            out[name] = _serve_figures(got, wall, st, probs)
    out["config"] = {"arrivals": "Poisson, mean %g/s" % rate, "mix": "70% D=3, 30% D=21",
                     "n_ev": "1e4 (D=3), 3e4 (D=21)", "n_g": 1000, "rtol": 1e-3,
                     "stop": {str(k): v for k, v in inputs.SERVE_RULE.items()},
                     "paced_requests": n, "saturated_requests": args.saturated_requests,
                     "note": "paced: the first %d requests of the stream submitted at their "
                             "arrival times (latency = submit to result); saturated: requests "
                             "queued at once, wall clock from first submit to last result" % n}
    out["p50_ms"] = out["served"]["p50_ms"]
    out["p99_ms"] = out["served"]["p99_ms"]
    out["latency_speedup_p99"] = out["plain"]["p99_ms"] / out["served"]["p99_ms"]
    out["clocks"] = clk.summary()
    return out


def run_serve(args):
    """The served workload on its own line (value: the saturated rate)."""
    import torch
    from paper_2009_05112_gb300 import build as _build
    from paper_2009_05112_gb300 import inputs, vegasp
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    _build.build()
    out = serve_summary(args, inputs, vegasp)
    sat = out["served_saturated"]
    line = {"metric": "served requests/s", "value": sat["requests_per_s"],
            "unit": "requests/s", "n_gpus": 1, "steps": sat["steps"], "warmup": 8,
            "ms_per_step": 1e3 * sat["busy_s"] / max(1, sat["steps"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": dict(out["config"], workload="serve_posteriors",
                           l2="each step touches a few MB of request state (fits L2); "
                              "latency, not bandwidth, bounds this workload"),
            "served": out, "clocks": out["clocks"]}
    if not args.no_cpu_baseline:
        _, probs, rules = inputs.serve_stream(args.requests, rate=200.0, seed=0)
        line["cpu_baseline"] = cpu_baseline_serve(probs, rules)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch_mix":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
