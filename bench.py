#!/usr/bin/env python
"""Benchmark: converged steady-PSR solves/s on GB300, mixed-precision vs FP64 form.

One step = one persistent-kernel solve of the whole batch (B = 4096 reactors per GPU of
the K = 53 / I = 325 synthetic mechanism with 10 third-body and 15 Troe reactions,
adiabatic, 1 atm, guess = inlet at 2000 K), inputs resident in HBM. The headline value
is the mixed form (FP64 residual, FP32 Jacobian and LU); the FP64 form is timed on the
same inputs. `e2e` times the host-pointer C entry (copies in, solve, copies out).
Multi-GPU: one process per GPU, each solving its own seeded shard (no collective).

The default run also times the other workloads of the scope (K = 10, the sooting batch,
K = 200 and the uneven batch) in both forms, under `workloads`, and measures the pipe
peaks the roofline is reported against (FP64 and FP32 FMA, double exp, log and division)
with the library's probe kernels, under `peaks`.

Roofline: the work of a solve is counted per category (FP64 flops, FP32 flops, exp, log
and division calls) from the per-reactor Newton iteration and residual-evaluation counts
the kernel reports; each category's time at its measured peak gives the pipe-time lower
bound t_min = max(t_fp64_pipe, t_fp32_pipe), with exp/log/division on the FP64 pipe.
frac = t_min / measured time; `achieved` expresses t_min as FP64-FMA-pipe flops per
second, so achieved / peak = frac.

`--impl reference` times the CPU oracle (plain numpy FP64) on a bounded sample of the
same workload instead, one reactor per host core per step.
"""
import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

# the CPU oracle runs one BLAS thread per process (the all-core baseline uses processes)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "k53_b4096"
MIXED = "mixed_b32768"       # the uneven batch: 50/35/15 % of K = 10 / 53 / 200 reactors
RATES = "k101_rates"         # the paper's timed unit: one rate evaluation per state
PEAKS = "peaks"              # the pipe probes alone
EXTRA = ("k10_b64", "k53soot_b16384", "k200_b2048", MIXED)
METRIC = "converged PSR solves/s, mixed vs FP64 form on one GB300 at ‖F‖∞≤1e-8; roofline %"
RATES_METRIC = "rate evaluations/s (kf, kr, q, wdot per state; Eqs. (4)-(9)) at T = 1800 K"
UNIT = "solves/s"
# dram__bytes_read.sum + dram__bytes_write.sum of one mixed-form launch of
# solve_kernel<float> on k53_b4096 (stragglers handed over at 90 % idle warps), from an ncu
# capture of the current build; set to None whenever that kernel changes, until it is
# captured again
K53_TRAFFIC_BYTES = 5176576 + 5269760


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extra", action="store_true", help="skip the other workloads of the default run")
    p.add_argument("--batch", type=int, default=0,
                   help="solve only the first N reactors of the workload's batch (profiling captures)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------- pipe peaks
def measure_peaks(torch, dev):
    """Sustained rates of the pipes the solver runs on, from the library's probe kernels
    (psr_pipe_probe): FP64 and FP32 FMA (TFLOP/s), FP64 exp, log and division (G calls/s).
    Each probe: one warm-up launch, then the best of three CUDA-event-timed launches of
    ~10-30 ms over 8 x 256-thread blocks per SM."""
    from paper_2005_11468_gb300 import psr
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads = 8 * nsm, 256
    sink = torch.empty(blocks * threads, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    iters = {psr.PROBE_FMA64: 4000, psr.PROBE_FMA32: 60000, psr.PROBE_EXP64: 200, psr.PROBE_LOG64: 100,
             psr.PROBE_DIV64: 300}
    out = {}
    for kind, it in iters.items():
        psr.pipe_probe(kind, max(1, it // 10), blocks, threads, sink)
        best = None
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ops = psr.pipe_probe(kind, it, blocks, threads, sink)
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b)
            best = ms if best is None else min(best, ms)
        out[kind] = ops / (best / 1e3)
    return {"fp64_tflops": out[psr.PROBE_FMA64] / 1e12, "fp32_tflops": out[psr.PROBE_FMA32] / 1e12,
            "exp64_gps": out[psr.PROBE_EXP64] / 1e9, "log64_gps": out[psr.PROBE_LOG64] / 1e9,
            "div64_gps": out[psr.PROBE_DIV64] / 1e9,
            "how": f"psr_pipe_probe, {blocks} x {threads} threads, best of 3 CUDA-event-timed launches"}


# ---------------------------------------------------------------------------- work model
def mech_counts(spec):
    K, I = spec.K, spec.I
    n_tb = sum(r.kind == "tb" for r in spec.reactions)
    n_troe = sum(r.kind == "troe" for r in spec.reactions)
    n_t2 = sum(r.kind == "troe" and r.troe is not None and r.troe[3] != 0.0 for r in spec.reactions)
    n_eff = sum(len(r.eff) for r in spec.reactions)
    parts = [len(set(r.reac) | set(r.prod)) for r in spec.reactions]
    nnz = sum(parts)                       # species -> reaction entries of the wdot gather
    pairs = sum(p * p for p in parts)      # entries a reaction adds to the Jacobian
    return K, I, n_tb, n_troe, n_t2, n_eff, nnz, pairs


def work_counts(spec, nfev, iters, precision):
    """Algorithmic work of the solves, summed over reactors, in the categories of the
    scope's measurement section: FP64 flops, FP32 flops, and exp, log and division calls
    counted as calls (an FMA is two flops; an FP32 division is counted as 8 FP32 flops).
    Each piece is counted in the precision the solver computes it in: the residual, its
    exponentials and the species sums in FP64; the Jacobian's per-reaction pieces, the Troe
    derivatives, the scatter, transform, LU and substitutions in the Jacobian's precision
    (FP32 in the mixed form).

    Per residual evaluation (nfev per reactor): per species NASA-7 c_p, H, S and dc_p
    (37 flops), concentration and the energy sums (16), residual (4); wdot gather 2 per
    entry; per reaction ln k (4), ln K_c (8), slot products (4), q (3) and two exp; per
    third-body efficiency 2 flops; per Troe row 4-5 exp (P_r, F_cent terms, F), two log10,
    2 divisions and ~30 flops for the value, 6 divisions and ~35 flops for the derivatives;
    per evaluation 2 log and 4 divisions. With soot: one MOMIC source evaluation (39 exp,
    29 log, ~600 flops) and six moment balances (6 exp, ~40 flops).
    Per Newton iteration (iters per reactor): per reaction ~85 flops of derivative pieces
    and 2 flops per Jacobian entry it adds, 3 per efficiency entry and participant; species
    sums 4 per gather entry and ~15 per species (FP64); transform 4 K^2 and energy-row column
    sums 2 K^2; the LU 2 n^3 / 3. With soot, the soot block adds 17 source evaluations and
    9 n chained entries (12 flops each, FP64). Per residual one pair of triangular solves,
    2 n^2 flops and n divisions."""
    K, I, n_tb, n_troe, n_t2, n_eff, nnz, pairs = mech_counts(spec)
    soot = spec.soot is not None
    n = K + 1 + (6 if soot else 0)
    nf, it = float(np.sum(nfev)), float(np.sum(iters))
    mixed = precision == "mixed"
    # per residual evaluation: FP64 parts, and the Troe derivatives in the Jacobian's precision
    f64_F = K * (37 + 16 + 4) + 2 * nnz + I * 19 + 2 * n_eff + n_tb + n_troe * 30
    exp_F = 2 * I + 4 * n_troe + n_t2
    log_F = 2 + 2 * n_troe
    div_F = 4 + 2 * n_troe
    jac_F, jdiv_F = n_troe * 35, n_troe * 6
    if soot:
        f64_F += 600 + 40
        exp_F += 39 + 6
        log_F += 29
    # per Newton iteration
    f64_J = 4 * nnz + 15 * K
    jac_J = I * 85 + 2 * pairs + 3 * n_eff * 3 + 4 * K * K + 2 * K * K + 2.0 * n ** 3 / 3.0
    exp_J = log_J = 0.0
    if soot:
        f64_J += 17 * 600 + 9 * n * 12
        exp_J += 17 * 39
        log_J += 17 * 29
    jac_S, jdiv_S = 2.0 * n * n, n
    c = {"fp64_flop": nf * f64_F + it * f64_J, "fp32_flop": 0.0, "exp": nf * exp_F + it * exp_J,
         "log": nf * log_F + it * log_J, "div": nf * div_F}
    if mixed:
        c["fp32_flop"] += nf * (jac_F + 8 * jdiv_F + jac_S + 8 * jdiv_S) + it * jac_J
    else:
        c["fp64_flop"] += nf * (jac_F + jac_S) + it * jac_J
        c["div"] += nf * (jdiv_F + jdiv_S)
    return c


def roofline(counts, seconds, peaks, traffic=None):
    """The roofline object of a timed step: pipe times at the measured peaks, the bound
    t_min = max(FP64 pipe, FP32 pipe), frac = t_min / measured time."""
    t64 = (counts["fp64_flop"] / (peaks["fp64_tflops"] * 1e12) + counts["exp"] / (peaks["exp64_gps"] * 1e9)
           + counts["log"] / (peaks["log64_gps"] * 1e9) + counts["div"] / (peaks["div64_gps"] * 1e9))
    t32 = counts["fp32_flop"] / (peaks["fp32_tflops"] * 1e12)
    tmin = max(t64, t32)
    return {"bound": "alu", "pipe": "fp64" if t64 >= t32 else "fp32",
            "achieved": tmin * peaks["fp64_tflops"] / seconds, "peak": peaks["fp64_tflops"],
            "unit": "TFLOP/s (FP64-FMA-pipe equivalent)", "frac": tmin / seconds, "traffic": traffic,
            "peak_source": "measured in this run (psr_pipe_probe, see peaks)",
            "pipe_ms": {"fp64_pipe": 1e3 * t64, "fp32_pipe": 1e3 * t32, "measured": 1e3 * seconds},
            "work_per_step": {k: float(v) for k, v in counts.items()}}


# ---------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (SM clock, throttle reasons) while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


# ---------------------------------------------------------------------------- oracle timing
def _oracle_solve(arg):
    """One oracle solve (a pool task): (name, class index or -1, reactor) -> converged?"""
    import warnings
    from oracle import psr_oracle as O
    from paper_2005_11468_gb300 import synth
    warnings.filterwarnings("ignore", category=RuntimeWarning)
    name, c, b = arg
    if c >= 0:
        specs = [synth.workload_mechanism(nm) for nm in synth.MIXED_WORKLOAD["parts"]]
        spec, batch = specs[c], synth.mixed_batch(specs)["batches"][c]
    else:
        spec = synth.workload_mechanism(name)
        batch = synth.workload_batch(name, spec)
    mech = O.Mechanism(synth.mechanism_text(spec))
    t0 = time.perf_counter()
    if spec.soot is not None:
        from oracle import momic_oracle as S
        r, _ = S.solve_soot_reactor(mech, O.inlet_of(batch, b), batch.Y0[b], batch.T0[b], batch.M_in[b])
    else:
        r = O.solve_reactor(mech, O.inlet_of(batch, b), np.r_[batch.Y0[b], batch.T0[b]])
    return int(r.status == O.CONVERGED), time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_pool_time(tasks, procs):
    """Wall time and converged count of the oracle on `tasks` in a spawn pool of `procs`
    processes (one BLAS thread each); the pool is started before the timed region."""
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_oracle_solve, [("k10_b64", -1, 0)] * procs)     # start-up (imports) outside the timing
        t0 = time.perf_counter()
        res = pool.map(_oracle_solve, tasks, chunksize=1)
        dt = time.perf_counter() - t0
    return sum(c for c, _ in res), dt, sum(t for _, t in res)


def cpu_baseline(name, n_all, n_one):
    """The oracle on all host cores (n_all reactors of the workload, a process pool) and
    on one core (the first n_one of them, in this process)."""
    procs = host_cores()
    tasks = [(name, -1, b) for b in range(n_all)]
    conv, wall, _ = oracle_pool_time(tasks, procs)
    c1, t1 = 0, 0.0
    for t in tasks[:n_one]:
        c, dt = _oracle_solve(t)
        c1 += c
        t1 += dt
    return {"value": conv / wall, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"reactors 0..{n_all - 1} of {name} on {procs} processes ({conv} converged, {wall:.1f} s wall)",
            "single_core": {"value": c1 / t1 if t1 > 0 else 0.0, "cores": 1,
                            "sample": f"reactors 0..{n_one - 1} ({c1} converged, {t1:.1f} s)"}}


def cpu_baseline_mixed(per_class):
    """The oracle on the uneven batch: `per_class` reactors of each mechanism class on all
    host cores, class times weighted by the class fractions (solves/s of the batch)."""
    from paper_2005_11468_gb300 import synth
    procs = host_cores()
    tasks = [(MIXED, c, b) for c, n in enumerate(per_class) for b in range(n)]
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_oracle_solve, [("k10_b64", -1, 0)] * procs)
        t0 = time.perf_counter()
        res = pool.map(_oracle_solve, tasks, chunksize=1)
        wall = time.perf_counter() - t0
    # CPU seconds per reactor of each class, then the batch's mean over the class mix
    sec, conv, k = [], 0.0, 0
    for c, n in enumerate(per_class):
        part = res[k:k + n]
        k += n
        sec.append(sum(t for _, t in part) / n)
        conv += synth.MIXED_WORKLOAD["fractions"][c] * sum(cc for cc, _ in part) / n
    mean_s = sum(f * s for f, s in zip(synth.MIXED_WORKLOAD["fractions"], sec))
    v = conv * procs / mean_s
    return {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{'/'.join(map(str, per_class))} reactors of the K=10/53/200 classes on {procs} processes "
                      f"({wall:.1f} s wall); CPU s per reactor {', '.join(f'{s:.2f}' for s in sec)}, "
                      f"weighted 50/35/15 %, times {procs} cores"}


def workload_config(name, world, B=None, spec=None):
    """The `config` object of a workload's JSON line; both arms print the same one (the
    reference arm's sample is described in its cpu_baseline)."""
    from paper_2005_11468_gb300 import synth
    dp = f"dp{world} (independent reactors)"
    flushed = "flushed (256 MB write) between timed steps"
    if name == RATES:
        spec = spec if spec is not None else synth.workload_mechanism(RATES)
        B = 1000000 if B is None else B
        return {"workload": f"{RATES}: K={spec.K}, I={spec.I} ({spec.n_tb} third-body, {spec.n_troe} Troe), "
                            f"B={B} states at T=1800 K, outputs q and wdot",
                "l2": flushed}
    if name == MIXED:
        B = synth.MIXED_WORKLOAD["B"] if B is None else B
        return {"workload": f"{MIXED}: {B} reactors per GPU, 50/35/15 % of K=10/53/200 mechanisms "
                            f"(I=24/325/1500), shuffled, one psr_batch_solve_multi call replayed as a CUDA graph",
                "global_batch": B * world, "precision": "mixed", "parallelism": dp, "l2": flushed}
    spec = spec if spec is not None else synth.workload_mechanism(name)
    B = synth.WORKLOADS[name]["B"] if B is None else B
    if spec.soot is not None:
        return {"workload": f"{name}: K={spec.K} + 6 MOMIC moments, I={spec.I}, B={B}",
                "global_batch": B * world, "precision": "mixed", "parallelism": dp, "l2": flushed}
    return {"workload": f"{name}: K={spec.K} species, I={spec.I} reactions "
                        f"({spec.n_tb} third-body, {spec.n_troe} Troe), B={B} reactors per GPU, adiabatic, 1 atm",
            "global_batch": B * world, "precision": "mixed", "parallelism": dp, "l2": flushed}


# ---------------------------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle as it stands, on the host cores: each step solves one reactor per core
    (a spawn process pool, one BLAS thread per process)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    K, W = args.steps, args.warmup
    procs = host_cores()
    base = {"impl": "reference", "n_gpus": args.gpus, "steps": K, "warmup": W, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic"}
    if args.workload == RATES:
        from paper_2005_11468_gb300 import synth
        tc = oracle_rates_time(synth.workload_mechanism(RATES), 20000)
        v = 1.0 / tc
        print(json.dumps({**base, "metric": RATES_METRIC, "value": v, "unit": "states/s",
                          "ms_per_step": 1e3 * tc * 20000, "config": workload_config(RATES, world),
                          "cpu_baseline": {"value": v, "unit": "states/s", "cores": 1, "kind": "oracle",
                                           "sample": "20000 states"},
                          "e2e": {"value": v, "unit": "states/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    if args.workload == MIXED:
        cb = cpu_baseline_mixed((procs, procs, max(1, procs // 4)))
        v = cb["value"]
        print(json.dumps({**base, "metric": METRIC, "value": v, "unit": UNIT, "ms_per_step": 1e3 * procs / v,
                          "config": workload_config(MIXED, world), "cpu_baseline": cb,
                          "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    from paper_2005_11468_gb300 import synth
    B = synth.WORKLOADS[args.workload]["B"]
    conv_total, t_total = 0, 0.0
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_oracle_solve, [("k10_b64", -1, 0)] * procs)
        for s in range(W + K):
            tasks = [(args.workload, -1, (s * procs + j) % B) for j in range(procs)]
            t0 = time.perf_counter()
            res = pool.map(_oracle_solve, tasks, chunksize=1)
            dt = time.perf_counter() - t0
            if s >= W:
                conv_total += sum(c for c, _ in res)
                t_total += dt
    v = conv_total / t_total if t_total > 0 else 0.0
    print(json.dumps({**base, "metric": METRIC, "value": v, "unit": UNIT, "ms_per_step": 1e3 * t_total / K,
                      "config": workload_config(args.workload, world),
                      "cpu_baseline": {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle",
                                       "sample": f"{procs} reactors of {args.workload} per step (one per core), "
                                                 f"timed steps {W}..{W + K - 1}"},
                      "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


# ---------------------------------------------------------------------------- our arm
class Ctx:
    """Device, process group and helpers shared by the measurements of one run."""

    def __init__(self):
        import torch
        self.torch = torch
        self.rank, self.world, self.local = dist_env()
        torch.cuda.set_device(self.local)
        self.dev = torch.device("cuda", self.local)
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl", device_id=self.dev)
            self.pg = dist
        from paper_2005_11468_gb300 import _build, psr
        if not os.path.exists(psr.LIB_PATH):
            _build.build()
        self.flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=self.dev)   # > L2 (129 MB)
        self.stream = torch.cuda.current_stream()

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()
        self.torch.cuda.synchronize()

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()


def shard_batch(ctx, name, spec, batch_cap=0):
    from paper_2005_11468_gb300 import shard, synth
    w = synth.WORKLOADS[name]
    batch = synth.make_batch(spec, w["B"], seed=shard.shard_seed(synth.MECH_SEED_BASE + 10 * w["tag"] + 1, ctx.rank),
                             tau_range=w.get("tau_range", (1e-4, 1e-2)))
    if batch_cap:
        batch = batch.subset(range(min(batch_cap, batch.B)))
    return batch


def measure_solves(ctx, name, steps, warmup, steps64, sampler=None, batch_cap=0, keep=False):
    """Time the mixed form (steps after warmup, L2 flushed before each) and the FP64 form
    (steps64 after one warm-up) on one seeded batch of a gas or sooting workload."""
    torch = ctx.torch
    from paper_2005_11468_gb300 import psr, shard, synth
    spec = synth.workload_mechanism(name)
    mech = psr.Mechanism(synth.mechanism_text(spec))
    batch = shard_batch(ctx, name, spec, batch_cap)
    t = {k: torch.tensor(getattr(batch, k), dtype=torch.float64, device=ctx.dev)
         for k in ("Y_in", "T_in", "tau", "P", "Y0", "T0")}
    soot = spec.soot is not None
    if soot:
        t["M_in"] = torch.tensor(batch.M_in, dtype=torch.float64, device=ctx.dev)

    def solve(opts, out):
        if soot:
            return psr.batch_solve_soot(mech, t["Y_in"], t["T_in"], t["tau"], t["P"], t["M_in"], t["Y0"], t["T0"],
                                        opts=opts, out=out)
        return psr.batch_solve(mech, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"], opts=opts, out=out)

    def timed(precision, k, w, smp):
        opts = psr.Options(precision=precision)
        out = None
        for _ in range(w):
            out = solve(opts, out)
        ctx.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        with (smp if smp is not None else _Null()):
            for s in range(k):
                ctx.flush.fill_(float(s))                      # evict the inputs from L2 between steps
                ev[s][0].record(ctx.stream)
                out = solve(opts, out)
                ev[s][1].record(ctx.stream)
            ctx.barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        st = out["status"].cpu().numpy()
        return dict(ms=ms, total_ms=shard.reduce_max(ctx.pg, [sum(ms)], ctx.dev)[0],
                    conv=int(np.isin(st, psr.CONVERGED_STATES).sum()), fallback=int(np.sum(st == psr.PSR_REFINE_FALLBACK)),
                    nfev=out["nfev"].cpu().numpy(), iters=out["iters"].cpu().numpy())

    mixed = timed(psr.PSR_MIXED, steps, warmup, sampler)
    fp64 = timed(psr.PSR_FP64, steps64, 1, None)
    res = dict(spec=spec, batch=batch, mech=mech, t=t, soot=soot, mixed=mixed, fp64=fp64, solve=solve)
    if not keep:
        mech.close()
    return res


def solve_summary(ctx, r, peaks, traffic=None):
    """mixed / FP64 throughput, convergence, iteration counts and rooflines of a measure_solves result."""
    from paper_2005_11468_gb300 import shard
    m, f = r["mixed"], r["fp64"]
    k, k64 = len(m["ms"]), len(f["ms"])
    conv_all, conv64 = shard.reduce_sum(ctx.pg, [m["conv"] * k, f["conv"] * k64], ctx.dev)
    value = shard.job_throughput(conv_all, m["total_ms"] / 1e3)
    value64 = shard.job_throughput(conv64, f["total_ms"] / 1e3)
    B = r["batch"].B
    s_m, s_f = m["total_ms"] / k / 1e3, f["total_ms"] / k64 / 1e3
    roof = roofline(work_counts(r["spec"], m["nfev"], m["iters"], "mixed"), s_m, peaks, traffic)
    roof64 = roofline(work_counts(r["spec"], f["nfev"], f["iters"], "fp64"), s_f, peaks)
    return {"value": value, "unit": UNIT, "ms_per_step": 1e3 * s_m, "steps": k,
            "ms_steps": [round(x, 3) for x in m["ms"]],
            "converged_fraction": m["conv"] / B, "refine_fallback": m["fallback"],
            "newton_iters_mean": float(np.mean(m["iters"])), "newton_iters_median": float(np.median(m["iters"])),
            "residual_evals_mean": float(np.mean(m["nfev"])),
            "roofline": roof,
            "fp64_form": {"value": value64, "unit": UNIT, "ms_per_step": 1e3 * s_f, "steps": k64,
                          "converged_fraction": f["conv"] / B,
                          "newton_iters_mean": float(np.mean(f["iters"])),
                          "residual_evals_mean": float(np.mean(f["nfev"])), "roofline": roof64},
            "mixed_vs_fp64": value / value64 if value64 > 0 else None}


def measure_multi(ctx, steps, warmup, steps64, peaks, sampler=None, e2e=False):
    """The uneven batch through psr_batch_solve_multi, captured once in a CUDA graph and
    replayed per step (mixed form); the FP64 form by direct calls; optionally e2e through
    the call with the packed inputs copied from pinned host memory and results read back."""
    torch = ctx.torch
    from paper_2005_11468_gb300 import psr, shard, synth
    specs = [synth.workload_mechanism(nm) for nm in synth.MIXED_WORKLOAD["parts"]]
    gms = [psr.Mechanism(synth.mechanism_text(sp)) for sp in specs]
    mb = synth.mixed_batch(specs, seed=shard.shard_seed(synth.MECH_SEED_BASE + 10 * synth.MIXED_WORKLOAD["tag"] + 1,
                                                        ctx.rank))
    B = len(mb["mech_id"])
    keys = ("Y_in", "Y0", "T_in", "tau", "P", "T0")
    host = {k: torch.tensor(mb[k], dtype=torch.float64).pin_memory() for k in keys}
    host["mech_id"] = torch.tensor(mb["mech_id"], dtype=torch.int32).pin_memory()
    host["row_off"] = torch.tensor(mb["row_off"], dtype=torch.int64).pin_memory()
    t = {k: v.to(ctx.dev) for k, v in host.items()}

    def call(opts, out=None):
        return psr.batch_solve_multi(gms, t["mech_id"], t["row_off"], t["Y_in"], t["T_in"], t["tau"], t["P"],
                                     t["Y0"], t["T0"], opts=opts, out=out)

    mixed_opts = psr.Options(precision=psr.PSR_MIXED)
    out = None
    for _ in range(warmup):
        out = call(mixed_opts, out)
    ctx.barrier()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        call(mixed_opts, out)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="thread_local"):
        call(mixed_opts, out)
    ctx.barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    with (sampler if sampler is not None else _Null()):
        for s in range(steps):
            ctx.flush.fill_(float(s))
            ev[s][0].record(ctx.stream)
            graph.replay()
            ev[s][1].record(ctx.stream)
        ctx.barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    st = out["status"].cpu().numpy()
    nfev, iters = out["nfev"].cpu().numpy(), out["iters"].cpu().numpy()
    conv = int(np.isin(st, psr.CONVERGED_STATES).sum())
    fp64_opts = psr.Options(precision=psr.PSR_FP64)
    o64 = call(fp64_opts)
    ctx.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(steps64):
        call(fp64_opts, o64)
    e1.record(ctx.stream)
    ctx.barrier()
    ms64 = e0.elapsed_time(e1) / steps64
    st64 = o64["status"].cpu().numpy()
    conv64 = int(np.isin(st64, psr.CONVERGED_STATES).sum())
    nfev64, iters64 = o64["nfev"].cpu().numpy(), o64["iters"].cpu().numpy()
    # the same mixed-form call as one persistent launch over all mechanisms (persistent = 1)
    pers_opts = psr.Options(precision=psr.PSR_MIXED, persistent=1)
    o_pers = call(pers_opts)
    ctx.barrier()
    e0.record(ctx.stream)
    call(pers_opts, o_pers)
    e1.record(ctx.stream)
    ctx.barrier()
    ms_pers = e0.elapsed_time(e1)
    conv_pers = int(np.isin(o_pers["status"].cpu().numpy(), psr.CONVERGED_STATES).sum())
    e_conv = e_t = 0.0
    h2d = d2h = 0
    if e2e:
        hout = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()}
        for s in range(steps):
            ctx.flush.fill_(float(s))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k, v in host.items():
                t[k].copy_(v, non_blocking=True)
            o = call(mixed_opts, out)
            for k in ("Y", "T", "status"):
                hout[k].copy_(o[k], non_blocking=True)
            torch.cuda.synchronize()
            e_t += time.perf_counter() - t0
            e_conv += int(np.isin(hout["status"].numpy(), psr.CONVERGED_STATES).sum())
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        d2h = sum(hout[k].numel() * hout[k].element_size() for k in ("Y", "T", "status"))
    total = sum(ms)
    conv_all, conv64_all, e_conv, conv_pers = shard.reduce_sum(ctx.pg, [conv * steps, conv64, e_conv, conv_pers],
                                                                 ctx.dev)
    total, ms64, e_t, ms_pers = shard.reduce_max(ctx.pg, [total, ms64, e_t, ms_pers], ctx.dev)
    value = conv_all / (total / 1e3)
    value64 = conv64_all / (ms64 / 1e3)

    def class_roof(nf, it, prec, seconds):
        counts = None
        for c, sp in enumerate(specs):
            w = work_counts(sp, nf[mb["members"][c]], it[mb["members"][c]], prec)
            counts = w if counts is None else {k: counts[k] + w[k] for k in w}
        return roofline(counts, seconds, peaks)

    res = {"value": value, "unit": UNIT, "ms_per_step": total / steps, "steps": steps,
           "converged_fraction": conv / B, "newton_iters_mean": float(np.mean(iters)),
           "newton_iters_median": float(np.median(iters)), "residual_evals_mean": float(np.mean(nfev)),
           "roofline": class_roof(nfev, iters, "mixed", total / steps / 1e3),
           "fp64_form": {"value": value64, "unit": UNIT, "ms_per_step": ms64, "steps": steps64,
                         "converged_fraction": conv64 / B, "newton_iters_mean": float(np.mean(iters64)),
                         "residual_evals_mean": float(np.mean(nfev64)),
                         "roofline": class_roof(nfev64, iters64, "fp64", ms64 / 1e3)},
           "mixed_vs_fp64": value / value64 if value64 > 0 else None,
           "persistent_launch": {"value": conv_pers / (ms_pers / 1e3), "unit": UNIT, "ms_per_step": ms_pers,
                                 "steps": 1, "gpu_launches_per_step": 2,
                                 "how": "persistent = 1: the bucketing kernel and one multi_solve_kernel over "
                                        "all mechanisms, FP64 re-solves inside (direct call)"},
           # per step: the bucketing kernel, then per mechanism the solver launch and the FP64
           # re-solve passes (warp path: the handoff list and continuation, then two
           # list/re-solve pairs; block path: one pair)
           "gpu_launches_per_step": 1 + sum(7 if sp.K + 1 <= 64 else 3 for sp in specs)}
    if e2e:
        res["e2e"] = {"value": e_conv / e_t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    for g in gms:
        g.close()
    return res


def e2e_host(ctx, r, steps):
    """The same metric through psr_batch_solve_host (pinned host arrays in and out, copies
    inside the timed call) on the workload's batch."""
    torch = ctx.torch
    from paper_2005_11468_gb300 import psr, shard
    spec, batch, mech = r["spec"], r["batch"], r["mech"]
    B = batch.B
    host = {k: torch.tensor(getattr(batch, k), dtype=torch.float64).pin_memory()
            for k in ("Y_in", "T_in", "tau", "P", "Y0", "T0")}
    hout = dict(Y=torch.empty((B, spec.K), dtype=torch.float64).pin_memory(),
                T=torch.empty(B, dtype=torch.float64).pin_memory(),
                iters=torch.empty(B, dtype=torch.int32).pin_memory(),
                ts_steps=torch.empty(B, dtype=torch.int32).pin_memory(),
                status=torch.empty(B, dtype=torch.int32).pin_memory(),
                fnorm=torch.empty(B, dtype=torch.float64).pin_memory(),
                nfev=torch.empty(B, dtype=torch.int32).pin_memory())
    eopts = psr.Options(precision=psr.PSR_MIXED)
    psr.batch_solve_host(mech, host["Y_in"], host["T_in"], host["tau"], host["P"], host["Y0"], host["T0"],
                         opts=eopts, out=hout)
    ctx.barrier()
    e_conv, e_t = 0, 0.0
    for s in range(steps):
        ctx.flush.fill_(float(s))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        psr.batch_solve_host(mech, host["Y_in"], host["T_in"], host["tau"], host["P"], host["Y0"], host["T0"],
                             opts=eopts, out=hout)
        e_t += time.perf_counter() - t0
        e_conv += int(np.isin(hout["status"], psr.CONVERGED_STATES).sum())
    e_t = shard.reduce_max(ctx.pg, [e_t], ctx.dev)[0]
    e_conv = shard.reduce_sum(ctx.pg, [e_conv], ctx.dev)[0]
    h2d = B * spec.K * 8 * 2 + B * 8 * 4
    d2h = B * spec.K * 8 + B * 8 * 2 + B * 4 * 4
    return {"value": shard.job_throughput(e_conv, e_t), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h}


def e2e_soot(ctx, r, steps):
    """e2e of the sooting workload (no host-pointer entry): inputs copied from pinned host
    memory with torch, the device entry, outputs read back, all inside the timed region."""
    torch = ctx.torch
    from paper_2005_11468_gb300 import psr
    B, spec = r["batch"].B, r["spec"]
    host = {k: v.cpu().pin_memory() for k, v in r["t"].items()}
    opts = psr.Options(precision=psr.PSR_MIXED)
    e_conv, e_t = 0, 0.0
    for s in range(steps):
        ctx.flush.fill_(float(s))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r["t"].update({k: v.to(ctx.dev, non_blocking=True) for k, v in host.items()})
        out = r["solve"](opts, None)
        st = out["status"].to("cpu")
        out["Y"].to("cpu")
        out["M"].to("cpu")
        e_t += time.perf_counter() - t0
        e_conv += int(np.isin(st.numpy(), psr.CONVERGED_STATES).sum())
    h2d = B * spec.K * 8 * 2 + B * 8 * 4 + B * 6 * 8
    d2h = B * spec.K * 8 + B * 4 + B * 6 * 8
    return {"value": e_conv / e_t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}


def launches_per_step(r):
    """Our kernels per timed mixed step of a warp-path gas workload (K + 1 <= 64): the
    FP32-Jacobian warp solve, the list of the stragglers it handed over and their block-
    solver continuation, then for the FP64 re-solve of what is left the list kernel and the
    continuation from its iterate, and the list kernel and the restart from the guess (all
    always enqueued, lists built on the device; the ncu launch list counts the same)."""
    return 7


def run_ours(args):
    ctx = Ctx()
    torch = ctx.torch
    K, W = args.steps, args.warmup
    sampler = ClockSampler(ctx.local)
    with sampler:
        peaks = measure_peaks(torch, ctx.dev)
    peak_clocks = sampler.summary()
    sampler = ClockSampler(ctx.local)
    if args.workload == MIXED:
        head = measure_multi(ctx, K, W, max(1, min(K, 2)), peaks, sampler=sampler, e2e=True)
        B = None
    else:
        r = measure_solves(ctx, args.workload, K, W, max(1, min(K, 3)), sampler, args.batch, keep=True)
        traffic = K53_TRAFFIC_BYTES if (args.workload == WORKLOAD and not args.batch) else None
        head = solve_summary(ctx, r, peaks, traffic)
        head["e2e"] = e2e_soot(ctx, r, K) if r["soot"] else e2e_host(ctx, r, K)
        B = r["batch"].B
        r["mech"].close()
    clocks = sampler.summary()
    extra = {}
    if not args.no_extra and not args.batch and args.workload == WORKLOAD:
        for name in EXTRA:
            if name == MIXED:
                extra[name] = measure_multi(ctx, 2, 1, 1, peaks)
            elif name == "k53soot_b16384":
                extra[name] = solve_summary(ctx, measure_solves(ctx, name, 1, 1, 1), peaks)
            else:
                extra[name] = solve_summary(ctx, measure_solves(ctx, name, 3 if name == "k10_b64" else 2, 1,
                                                                3 if name == "k10_b64" else 1), peaks)
            extra[name]["config"] = workload_config(name, ctx.world)
            extra[name]["timing"] = "warm-up 1, then the steps shown, L2 flushed before each, CUDA events"
    if ctx.rank != 0:
        ctx.close()
        return
    from paper_2005_11468_gb300 import synth
    line = {
        "metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": ctx.world, "steps": K, "warmup": W,
        "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 residual / f32 Jacobian+LU", "data": "synthetic",
        "config": workload_config(args.workload, ctx.world, B),
        **{k: head[k] for k in ("ms_steps",) if k in head},
        **{k: head[k] for k in ("fp64_form", "mixed_vs_fp64", "converged_fraction", "newton_iters_mean",
                                "newton_iters_median", "residual_evals_mean", "roofline")},
        "e2e": head["e2e"],
        "gpu_launches": head.get("gpu_launches_per_step", launches_per_step(None)) * K,
        "clocks": clocks,
        "peaks": {**peaks, "clocks": peak_clocks},
    }
    if "persistent_launch" in head:
        line["persistent_launch"] = head["persistent_launch"]
    if extra:
        line["workloads"] = extra
    if not args.no_cpu_baseline and not args.batch:
        if args.workload == MIXED:
            line["cpu_baseline"] = cpu_baseline_mixed((host_cores(), host_cores(), max(1, host_cores() // 4)))
        else:
            spec = synth.workload_mechanism(args.workload)
            B_w = synth.WORKLOADS[args.workload]["B"]
            n_all = min(B_w, 256 if spec.K <= 60 and spec.soot is None else 2 * host_cores())
            line["cpu_baseline"] = cpu_baseline(args.workload, n_all, min(B_w, 8 if spec.soot is None else 2))
    print(json.dumps(line))
    ctx.close()


def run_peaks(args):
    """The pipe probes alone, with the SM clock sampled while they run."""
    ctx = Ctx()
    sampler = ClockSampler(ctx.local)
    with sampler:
        peaks = measure_peaks(ctx.torch, ctx.dev)
    if ctx.rank == 0:
        print(json.dumps({"metric": "pipe peaks", "peaks": peaks, "clocks": sampler.summary(),
                          "gpu": ctx.torch.cuda.get_device_name(ctx.dev)}))
    ctx.close()


# ---------------------------------------------------------------------------- rate unit
def _rate_states(spec, B, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    Y = rng.dirichlet(np.full(spec.K, 0.7), size=B)
    return Y, np.full(B, 1800.0), np.full(B, 101325.0 * 10.0)


def oracle_rates_time(spec, B):
    """Seconds per state of the oracle's vectorised rate functions (one core)."""
    import warnings
    from oracle import psr_oracle as O
    from paper_2005_11468_gb300 import synth
    warnings.filterwarnings("ignore", category=RuntimeWarning)
    mech = O.Mechanism(synth.mechanism_text(spec))
    Y, T, P = _rate_states(spec, B, 7)
    t0 = time.perf_counter()
    _, _, C = O.mixture_state(mech, Y, T, P)
    q = O.rates_of_progress(mech, T, C)
    O.net_production_rates(mech, q)
    return (time.perf_counter() - t0) / B


def run_rates(args):
    """Rate evaluation (psr_eval_rates) of a 101-species / 542-reaction synthetic mechanism
    at B = 1e2 ... 1e6 states, T = 1800 K, the unit the paper times on its GPU; the value
    is states/s at the largest batch, timed with the states resident."""
    ctx = Ctx()
    torch, dev = ctx.torch, ctx.dev
    from paper_2005_11468_gb300 import psr, synth
    with ClockSampler(ctx.local) as s0:
        peaks = measure_peaks(torch, dev)
    spec = synth.workload_mechanism(RATES)
    mech = psr.Mechanism(synth.mechanism_text(spec))
    K, W = args.steps, args.warmup
    per_b, ms_big, B_big = {}, 0.0, 0
    sampler = ClockSampler(ctx.local)
    for B in (100, 1000, 10000, 100000, 1000000):
        Y, T, P = _rate_states(spec, B, 1 + ctx.rank)
        d = dict(Y=torch.tensor(Y, device=dev), T=torch.tensor(T, device=dev), P=torch.tensor(P, device=dev))
        out = dict(q=torch.empty((B, spec.I), dtype=torch.float64, device=dev),
                   wdot=torch.empty((B, spec.K), dtype=torch.float64, device=dev))
        for _ in range(W):
            psr.eval_rates(mech, d["Y"], d["T"], d["P"], out=out)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        with (sampler if B == 1000000 else _Null()):
            for s in range(K):
                ctx.flush.fill_(float(s))
                ev[s][0].record(ctx.stream)
                psr.eval_rates(mech, d["Y"], d["T"], d["P"], out=out)
                ev[s][1].record(ctx.stream)
            torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / K
        per_b[B] = B / (ms / 1e3)
        ms_big, B_big = ms, B
        del d, out
    # end to end at B = 1e5: states from pinned host memory, rates back to the host
    B = 100000
    Y, T, P = _rate_states(spec, B, 1 + ctx.rank)
    host = dict(Y=torch.tensor(Y).pin_memory(), T=torch.tensor(T).pin_memory(), P=torch.tensor(P).pin_memory())
    hq = torch.empty((B, spec.I), dtype=torch.float64).pin_memory()
    hw = torch.empty((B, spec.K), dtype=torch.float64).pin_memory()
    d = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    out = dict(q=torch.empty((B, spec.I), dtype=torch.float64, device=dev),
               wdot=torch.empty((B, spec.K), dtype=torch.float64, device=dev))
    e_t = 0.0
    for s in range(K):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in d:
            d[k].copy_(host[k], non_blocking=True)
        psr.eval_rates(mech, d["Y"], d["T"], d["P"], out=out)
        hq.copy_(out["q"], non_blocking=True)
        hw.copy_(out["wdot"], non_blocking=True)
        torch.cuda.synchronize()
        e_t += time.perf_counter() - t0
    value = per_b[B_big]
    # per state: one residual evaluation's rate part (no residual rows, no energy sums)
    Kk, I, n_tb, n_troe, n_t2, n_eff, nnz, _ = mech_counts(spec)
    counts = {"fp64_flop": B_big * (Kk * 45 + 2 * nnz + I * 19 + 2 * n_eff + n_tb + n_troe * 30),
              "fp32_flop": 0.0, "exp": B_big * (2 * I + 4 * n_troe + n_t2), "log": B_big * (2 + 2 * n_troe),
              "div": B_big * (3 + 8 * n_troe)}
    line = {"metric": RATES_METRIC, "value": value, "unit": "states/s", "n_gpus": ctx.world, "steps": K, "warmup": W,
            "ms_per_step": ms_big, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": workload_config(RATES, ctx.world, B_big, spec),
            "states_per_s_by_batch": {str(b): v for b, v in per_b.items()},
            "roofline": roofline(counts, ms_big / 1e3, peaks),
            "e2e": {"value": B * K / e_t, "unit": "states/s", "h2d_bytes_per_step": B * (spec.K + 2) * 8,
                    "d2h_bytes_per_step": B * (spec.I + spec.K) * 8},
            "gpu_launches": K * 5, "clocks": sampler.summary(), "peaks": {**peaks, "clocks": s0.summary()}}
    if not args.no_cpu_baseline:
        tc = oracle_rates_time(spec, 20000)
        line["cpu_baseline"] = {"value": 1.0 / tc, "unit": "states/s", "cores": 1, "kind": "oracle",
                                "sample": "20000 states, the oracle's vectorised numpy rate functions"}
        line["gpu_over_oracle_by_batch"] = {str(b): v * tc for b, v in per_b.items()}
    if ctx.rank == 0:
        print(json.dumps(line))
    ctx.close()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == PEAKS:
        run_peaks(args)
    elif args.workload == RATES:
        run_rates(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
