#!/usr/bin/env python
"""Benchmark: converged steady-PSR solves/s on GB300, mixed-precision vs FP64 form.

One step = one persistent-kernel solve of the whole batch (B = 4096 reactors per GPU of
the K = 53 / I = 325 synthetic mechanism with 10 third-body and 15 Troe reactions,
adiabatic, 1 atm, guess = inlet at 2000 K), inputs resident in HBM. The headline value
is the mixed form (FP64 residual, FP32 Jacobian and LU); the FP64 form is timed on the
same inputs. `e2e` times the host-pointer C entry (copies in, solve, copies out).
Multi-GPU: one process per GPU, each solving its own seeded shard (no collective).

`--impl reference` times the CPU oracle (plain numpy FP64) on a bounded sample of the
same workload instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

# the CPU oracle legs run single-threaded (reported as cores = 1)
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "k53_b4096"
MIXED = "mixed_b32768"       # the uneven batch: 50/35/15 % of K = 10 / 53 / 200 reactors
METRIC = "converged PSR solves/s, mixed vs FP64 form on one GB300 at ‖F‖∞≤1e-8; roofline %"
UNIT = "solves/s"
FP64_PEAK_TFLOPS = 1.25          # nominal GB300 FP64 (non-tensor) rate
# FP64-pipe cost of one transcendental in flop slots (measured GB300 throughput of CUDA's
# double exp / log relative to the FP64 FMA rate: 1.2 TFLOP/s / 29.6 G exp/s, / 16.3 G log/s)
EXP_FLOPS, LOG_FLOPS, DIV_FLOPS = 40.0, 73.0, 16.0
# dram__bytes_read + write of one mixed-form launch on k53_b4096, from the ncu capture of
# the current solver build (to be re-measured whenever the kernel changes)
K53_TRAFFIC_BYTES = 5050112


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default=WORKLOAD)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--batch", type=int, default=0,
                   help="solve only the first N reactors of the workload's batch (profiling captures)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------- work model
def fp64_work(mech_spec, nfev, iters, precision):
    """FP64-pipe work (flops, transcendentals at their measured pipe cost) of the solver:
    per residual evaluation W_F, per Newton iteration the Jacobian's FP64 part W_J and,
    in the FP64 form, the LU (2n^3/3) and per residual one triangular solve pair (2n^2)."""
    K, I = mech_spec.K, mech_spec.I
    n = K + 1
    n_tb = sum(r.kind == "tb" for r in mech_spec.reactions)
    n_troe = sum(r.kind == "troe" for r in mech_spec.reactions)
    n_eff = sum(len(r.eff) for r in mech_spec.reactions)
    nnz = sum(len(set(r.reac) | set(r.prod)) for r in mech_spec.reactions)   # wdot gather entries
    W_F = (K * 45 + I * (20 + 2 * EXP_FLOPS) + 2 * n_eff + 2 * nnz + K * 4
           + n_troe * (4 * EXP_FLOPS + 2 * LOG_FLOPS + 30) + 2 * LOG_FLOPS + 4 * DIV_FLOPS)
    W_J = I * 80 + 4 * nnz + 2 * K * K + 4 * K * K + (n_tb + n_troe) * 12 + n_troe * (60 + 4 * EXP_FLOPS + 2 * LOG_FLOPS)
    if mech_spec.soot is not None:
        # one MOMIC source evaluation: 29 fractional moments (exp), 28 grid-function logs,
        # 7 interpolated f(1/2) (exp) and the nucleation/growth rates; the Jacobian's soot
        # block takes 17 of them plus 9 (K + 7) chained entries
        n = K + 7
        W_S_EVAL = 36 * EXP_FLOPS + 30 * LOG_FLOPS + 400
        W_F += W_S_EVAL + 6 * (EXP_FLOPS + 10)
        W_J += 17 * W_S_EVAL + 9 * n * 12
    W_LU = 2.0 * n ** 3 / 3.0 if precision == "fp64" else 0.0
    W_S = 2.0 * n * n if precision == "fp64" else 0.0
    nf, it = float(np.sum(nfev)), float(np.sum(iters))
    return nf * (W_F + W_S) + it * (W_J + W_LU)


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


# ---------------------------------------------------------------------------- oracle timing
def oracle_sample_size(spec):
    """Reactors the oracle solves for the CPU baseline: about 10-30 s of one core."""
    return 6 if spec.K <= 60 else 1


def oracle_time(name, indices):
    """Converged count and seconds of the oracle on reactors `indices` of a workload
    (gas, or gas + MOMIC soot for a sooting mechanism)."""
    import warnings
    from oracle import psr_oracle as O
    from paper_2005_11468_gb300 import synth
    warnings.filterwarnings("ignore", category=RuntimeWarning)   # trial states of the damped Newton
    spec = synth.workload_mechanism(name)
    mech = O.Mechanism(synth.mechanism_text(spec))
    batch = synth.workload_batch(name, spec)
    t0 = time.perf_counter()
    if spec.soot is not None:
        from oracle import momic_oracle as S
        conv = 0
        for b in indices:
            r, _ = S.solve_soot_reactor(mech, O.inlet_of(batch, b), batch.Y0[b], batch.T0[b], batch.M_in[b])
            conv += int(r.status == O.CONVERGED)
    else:
        res = O.solve_batch(mech, batch, indices=list(indices))
        conv = int(np.sum(res["status"] == O.CONVERGED))
    return conv, time.perf_counter() - t0


def oracle_time_mixed(per_class):
    """Oracle seconds per reactor of the uneven batch: `per_class` reactors of each
    mechanism class timed, weighted by the class fractions. Returns (solves/s, detail)."""
    from oracle import psr_oracle as O
    from paper_2005_11468_gb300 import synth
    specs = [synth.workload_mechanism(nm) for nm in synth.MIXED_WORKLOAD["parts"]]
    mb = synth.mixed_batch(specs, B=512)
    t_avg, conv_frac, detail = 0.0, 0.0, []
    for c, (spec, frac, n) in enumerate(zip(specs, synth.MIXED_WORKLOAD["fractions"], per_class)):
        mech = O.Mechanism(synth.mechanism_text(spec))
        bc = mb["batches"][c]
        t0 = time.perf_counter()
        res = O.solve_batch(mech, bc, indices=list(range(n)))
        dt = (time.perf_counter() - t0) / n
        t_avg += frac * dt
        conv_frac += frac * float(np.mean(res["status"] == O.CONVERGED))
        detail.append(f"{n} K={spec.K} reactors {dt:.2f} s each")
    return conv_frac / t_avg, "; ".join(detail)


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
                "global_batch": B * world, "precision": "mixed", "l2": "flushed between timed steps"}
    return {"workload": f"{name}: K={spec.K} species, I={spec.I} reactions "
                        f"({spec.n_tb} third-body, {spec.n_troe} Troe), B={B} reactors per GPU, adiabatic, 1 atm",
            "global_batch": B * world, "precision": "mixed", "parallelism": dp, "l2": flushed}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    K, W = args.steps, args.warmup
    if args.workload == RATES:
        from paper_2005_11468_gb300 import synth
        tc = oracle_rates_time(synth.workload_mechanism(RATES), 20000)
        v = 1.0 / tc
        print(json.dumps({"impl": "reference", "metric": RATES_METRIC, "value": v, "unit": "states/s",
                          "n_gpus": args.gpus, "steps": K, "warmup": W, "ms_per_step": 1e3 * tc * 20000,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": workload_config(RATES, world),
                          "cpu_baseline": {"value": v, "unit": "states/s", "cores": 1, "kind": "oracle",
                                           "sample": "20000 states"},
                          "e2e": {"value": v, "unit": "states/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))
        return
    if args.workload == MIXED:
        v, detail = oracle_time_mixed((2, 1, 1))
        line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
                "steps": K, "warmup": W, "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload_config(MIXED, world),
                "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": detail},
                "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    conv_total, t_total = 0, 0.0
    for s in range(W + K):
        c, dt = oracle_time(args.workload, [s])
        if s >= W:
            conv_total += c
            t_total += dt
    v = conv_total / t_total if t_total > 0 else 0.0
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * t_total / K, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, world),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"reactors 0..{W + K - 1} of {args.workload}, one per step, "
                                       f"timed steps {W}..{W + K - 1}"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    from paper_2005_11468_gb300 import _build, psr, synth
    if not os.path.exists(psr.LIB_PATH):
        _build.build()
    w = synth.WORKLOADS[args.workload]
    spec = synth.workload_mechanism(args.workload)
    mech = psr.Mechanism(synth.mechanism_text(spec))
    from paper_2005_11468_gb300 import shard
    batch = synth.make_batch(spec, w["B"], seed=shard.shard_seed(synth.MECH_SEED_BASE + 10 * w["tag"] + 1, rank),
                             tau_range=w.get("tau_range", (1e-4, 1e-2)))
    if args.batch:
        batch = batch.subset(range(min(args.batch, batch.B)))
    t = {k: torch.tensor(getattr(batch, k), dtype=torch.float64, device=dev)
         for k in ("Y_in", "T_in", "tau", "P", "Y0", "T0")}
    soot = spec.soot is not None
    if soot:
        t["M_in"] = torch.tensor(batch.M_in, dtype=torch.float64, device=dev)
    B = batch.B

    def solve(opts, out):
        if soot:
            return psr.batch_solve_soot(mech, t["Y_in"], t["T_in"], t["tau"], t["P"], t["M_in"], t["Y0"], t["T0"],
                                        opts=opts, out=out)
        return psr.batch_solve(mech, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"], opts=opts, out=out)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    def timed(precision, steps, warmup, sampler=None):
        opts = psr.Options(precision=precision)
        out = None
        for _ in range(warmup):
            out = solve(opts, out)
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        conv = 0
        nfev = iters = None
        ctx = sampler if sampler is not None else _Null()
        with ctx:
            for s in range(steps):
                flush.fill_(float(s))                     # evict the inputs from L2 between steps
                ev[s][0].record(stream)
                out = solve(opts, out)
                ev[s][1].record(stream)
            barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        st = out["status"].cpu().numpy()
        conv = int(np.isin(st, psr.CONVERGED_STATES).sum())
        nfev = out["nfev"].cpu().numpy()
        iters = out["iters"].cpu().numpy()
        total = shard.reduce_max(pg, [sum(ms)], dev)[0]   # the slowest rank's time
        return dict(ms=ms, total_ms=total, conv=conv, nfev=nfev, iters=iters)

    K, W = args.steps, args.warmup
    sampler = ClockSampler(local)
    mixed = timed(psr.PSR_MIXED, K, W, sampler)
    fp64 = timed(psr.PSR_FP64, max(1, min(K, 3)), 1)

    # end to end through the host-pointer entry (inputs from pinned host memory); the
    # soot workload has no host-pointer entry, so its e2e copies through torch
    if soot:
        return run_soot_tail(args, spec, batch, mixed, fp64, t, solve, flush, barrier, pg, rank, world, sampler)
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
    barrier()
    e_conv, e_t = 0, 0.0
    for s in range(K):
        flush.fill_(float(s))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        psr.batch_solve_host(mech, host["Y_in"], host["T_in"], host["tau"], host["P"], host["Y0"], host["T0"],
                             opts=eopts, out=hout)
        e_t += time.perf_counter() - t0
        e_conv += int(np.isin(hout["status"], psr.CONVERGED_STATES).sum())
    e_t = shard.reduce_max(pg, [e_t], dev)[0]
    h2d = B * spec.K * 8 * 2 + B * 8 * 4
    d2h = B * spec.K * 8 + B * 8 * 2 + B * 4 * 4

    conv_all = mixed["conv"] * K
    conv64 = fp64["conv"] * len(fp64["ms"])
    conv_all, conv64, e_conv = shard.reduce_sum(pg, [conv_all, conv64, e_conv], dev)
    value = shard.job_throughput(conv_all, mixed["total_ms"] / 1e3)
    value64 = shard.job_throughput(conv64, fp64["total_ms"] / 1e3)
    e2e_value = shard.job_throughput(e_conv, e_t)

    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return
    avg_ms = mixed["total_ms"] / K
    work = fp64_work(spec, mixed["nfev"], mixed["iters"], "mixed")
    achieved = work / (avg_ms / 1e3) / 1e12
    work64 = fp64_work(spec, fp64["nfev"], fp64["iters"], "fp64")
    achieved64 = work64 / (fp64["total_ms"] / len(fp64["ms"]) / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": avg_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 residual / f32 Jacobian+LU", "data": "synthetic",
        "config": workload_config(args.workload, world, B, spec),
        "fp64_form": {"value": value64, "unit": UNIT, "ms_per_step": fp64["total_ms"] / len(fp64["ms"]),
                      "converged": fp64["conv"], "roofline_frac": achieved64 / FP64_PEAK_TFLOPS},
        "mixed_vs_fp64": value / value64 if value64 > 0 else None,
        "converged_fraction": mixed["conv"] / B,
        "newton_iters_median": float(np.median(mixed["iters"])),
        "roofline": {"bound": "alu", "pipe": "fp64", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                     "traffic": K53_TRAFFIC_BYTES if args.workload == WORKLOAD else None,
                     "traffic_unit": "DRAM bytes per mixed launch (ncu capture, profiles/solve_kernel_k53_b4096.md)",
                     "peak_source": "nominal GB300 FP64 rate (recipe table); measured FMA loop 1.198",
                     "work_model": "FP64 flops with exp=40, log=73, div=16 flop slots"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        # per step: the FP32-Jacobian solve, the unconverged-list kernel, the FP64 re-solve
        "gpu_launches": 3 * K,
        "clocks": sampler.summary(),
    }
    if not args.no_cpu_baseline:
        n_cpu = oracle_sample_size(spec)
        idx = list(range(n_cpu))
        c, dt = oracle_time(args.workload, idx)
        line["cpu_baseline"] = {"value": c / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"reactors 0..{n_cpu - 1} of {args.workload} ({c} converged, {dt:.1f} s)"}
    print(json.dumps(line))
    if pg is not None:
        pg.destroy_process_group()


def run_soot_tail(args, spec, batch, mixed, fp64, t, solve, flush, barrier, pg, rank, world, sampler):
    import torch
    from paper_2005_11468_gb300 import psr
    K, W = args.steps, args.warmup
    B = batch.B
    host = {k: v.cpu().pin_memory() for k, v in t.items()}
    opts = psr.Options(precision=psr.PSR_MIXED)
    e_conv, e_t = 0, 0.0
    for s in range(K):
        flush.fill_(float(s))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d = {k: v.to(t[k].device, non_blocking=True) for k, v in host.items()}
        t.update(d)
        out = solve(opts, None)
        st = out["status"].to("cpu")
        Y = out["Y"].to("cpu")
        M = out["M"].to("cpu")
        e_t += time.perf_counter() - t0
        e_conv += int(np.isin(st.numpy(), psr.CONVERGED_STATES).sum())
    h2d = B * spec.K * 8 * 2 + B * 8 * 4 + B * 6 * 8
    d2h = B * spec.K * 8 + B * 4 + B * 6 * 8
    conv_all = mixed["conv"] * K
    conv64 = fp64["conv"] * len(fp64["ms"])
    value = conv_all / (mixed["total_ms"] / 1e3)
    value64 = conv64 / (fp64["total_ms"] / 1e3)
    if rank != 0:
        return
    avg_ms = mixed["total_ms"] / K
    achieved = fp64_work(spec, mixed["nfev"], mixed["iters"], "mixed") / (avg_ms / 1e3) / 1e12
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": mixed["total_ms"] / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 residual / f32 Jacobian+LU", "data": "synthetic",
            "config": workload_config(args.workload, world, B, spec),
            "fp64_form": {"value": value64, "unit": UNIT, "ms_per_step": fp64["total_ms"] / len(fp64["ms"]),
                          "converged": fp64["conv"]},
            "mixed_vs_fp64": value / value64 if value64 > 0 else None,
            "converged_fraction": mixed["conv"] / B,
            "newton_iters_median": float(np.median(mixed["iters"])),
            "roofline": {"bound": "alu", "pipe": "fp64", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                         "peak_source": "nominal GB300 FP64 rate (recipe table); measured FMA loop 1.198",
                         "work_model": "FP64 flops with exp=40, log=73, div=16 flop slots, MOMIC terms"},
            "e2e": {"value": e_conv / e_t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": 3 * K, "clocks": sampler.summary()}
    if not args.no_cpu_baseline:
        n_cpu = 2
        c, dt = oracle_time(args.workload, list(range(n_cpu)))
        line["cpu_baseline"] = {"value": c / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"reactors 0..{n_cpu - 1} of {args.workload} ({c} converged, {dt:.1f} s)"}
    print(json.dumps(line))


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def run_multi(args):
    """The uneven batch through psr_batch_solve_multi, captured once in a CUDA graph and
    replayed per step (mixed form); the FP64 form by direct calls; e2e through the call
    with the packed inputs copied from pinned host memory and the results read back."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    from paper_2005_11468_gb300 import _build, psr, synth
    if not os.path.exists(psr.LIB_PATH):
        _build.build()
    specs = [synth.workload_mechanism(nm) for nm in synth.MIXED_WORKLOAD["parts"]]
    gms = [psr.Mechanism(synth.mechanism_text(sp)) for sp in specs]
    from paper_2005_11468_gb300 import shard
    mb = synth.mixed_batch(specs, seed=shard.shard_seed(synth.MECH_SEED_BASE + 10 * synth.MIXED_WORKLOAD["tag"] + 1,
                                                        rank))
    B = len(mb["mech_id"])
    keys = ("Y_in", "Y0", "T_in", "tau", "P", "T0")
    host = {k: torch.tensor(mb[k], dtype=torch.float64).pin_memory() for k in keys}
    host["mech_id"] = torch.tensor(mb["mech_id"], dtype=torch.int32).pin_memory()
    host["row_off"] = torch.tensor(mb["row_off"], dtype=torch.int64).pin_memory()
    t = {k: v.to(dev) for k, v in host.items()}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    K, W = args.steps, args.warmup

    def call(opts, out=None):
        return psr.batch_solve_multi(gms, t["mech_id"], t["row_off"], t["Y_in"], t["T_in"], t["tau"], t["P"],
                                     t["Y0"], t["T0"], opts=opts, out=out)

    def barrier():
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize()

    mixed_opts = psr.Options(precision=psr.PSR_MIXED)
    out = None
    for _ in range(W):
        out = call(mixed_opts, out)
    barrier()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        call(mixed_opts, out)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="thread_local"):
        call(mixed_opts, out)
    barrier()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    sampler = ClockSampler(local)
    with sampler:
        for s in range(K):
            flush.fill_(float(s))
            ev[s][0].record(stream)
            graph.replay()
            ev[s][1].record(stream)
        barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    st = out["status"].cpu().numpy()
    nfev, iters = out["nfev"].cpu().numpy(), out["iters"].cpu().numpy()
    conv = int(np.isin(st, psr.CONVERGED_STATES).sum())
    # FP64 form, direct calls
    fp64_opts = psr.Options(precision=psr.PSR_FP64)
    o64 = call(fp64_opts)
    barrier()
    n64 = max(1, min(K, 2))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n64):
        call(fp64_opts, o64)
    e1.record(stream)
    barrier()
    ms64 = e0.elapsed_time(e1) / n64
    conv64 = int(np.isin(o64["status"].cpu().numpy(), psr.CONVERGED_STATES).sum())
    # end to end: pinned host -> device, the call, results -> host
    hout = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items()}
    e_conv, e_t = 0, 0.0
    for s in range(K):
        flush.fill_(float(s))
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
    vals = torch.tensor([conv * K, total, conv64, ms64, e_conv, e_t], dtype=torch.float64, device=dev)
    if pg is not None:
        mx = vals.clone()
        pg.all_reduce(mx, op=pg.ReduceOp.MAX)
        pg.all_reduce(vals)
        vals[1], vals[3], vals[5] = mx[1], mx[3], mx[5]
    conv_all, total, conv64_all, ms64, e_conv, e_t = vals.tolist()
    if rank != 0:
        if pg is not None:
            pg.destroy_process_group()
        return
    value = conv_all / (total / 1e3)
    value64 = conv64_all / (ms64 / 1e3)
    work = sum(fp64_work(sp, nfev[mb["members"][c]], iters[mb["members"][c]], "mixed") for c, sp in enumerate(specs))
    achieved = work / (total / K / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": total / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64 residual / f32 Jacobian+LU", "data": "synthetic",
        "config": workload_config(MIXED, world, B),
        "fp64_form": {"value": value64, "unit": UNIT, "ms_per_step": ms64, "converged": int(conv64)},
        "mixed_vs_fp64": value / value64 if value64 > 0 else None,
        "converged_fraction": conv / B,
        "newton_iters_median": float(np.median(iters)),
        "roofline": {"bound": "alu", "pipe": "fp64", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                     "peak_source": "nominal GB300 FP64 rate (recipe table); measured FMA loop 1.198",
                     "work_model": "FP64 flops with exp=40, log=73, div=16 flop slots, summed over classes"},
        "e2e": {"value": e_conv / e_t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        # per step: bucketing, and per class the solver, the unconverged list and the FP64 re-solve
        "gpu_launches": K * (1 + 3 * len(specs)),
        "clocks": sampler.summary(),
    }
    if not args.no_cpu_baseline:
        v, detail = oracle_time_mixed((2, 1, 1))
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": f"class-weighted: {detail}"}
    print(json.dumps(line))
    if pg is not None:
        pg.destroy_process_group()


RATES = "k101_rates"   # the paper's timed unit: one rate evaluation per state
RATES_METRIC = "rate evaluations/s (kf, kr, q, wdot per state; Eqs. (4)-(9)) at T = 1800 K"


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
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2005_11468_gb300 import _build, psr, synth
    if not os.path.exists(psr.LIB_PATH):
        _build.build()
    spec = synth.workload_mechanism(RATES)
    mech = psr.Mechanism(synth.mechanism_text(spec))
    K, W = args.steps, args.warmup
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    per_b, ms_big, B_big = {}, 0.0, 0
    sampler = ClockSampler(local)
    for B in (100, 1000, 10000, 100000, 1000000):
        Y, T, P = _rate_states(spec, B, 1 + rank)
        d = dict(Y=torch.tensor(Y, device=dev), T=torch.tensor(T, device=dev), P=torch.tensor(P, device=dev))
        out = dict(q=torch.empty((B, spec.I), dtype=torch.float64, device=dev),
                   wdot=torch.empty((B, spec.K), dtype=torch.float64, device=dev))
        for _ in range(W):
            psr.eval_rates(mech, d["Y"], d["T"], d["P"], out=out)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        ctx = sampler if B == 1000000 else _Null()
        with ctx:
            for s in range(K):
                flush.fill_(float(s))
                ev[s][0].record(stream)
                psr.eval_rates(mech, d["Y"], d["T"], d["P"], out=out)
                ev[s][1].record(stream)
            torch.cuda.synchronize()
        ms = sum(a.elapsed_time(b) for a, b in ev) / K
        per_b[B] = B / (ms / 1e3)
        ms_big, B_big = ms, B
        del d, out
    # end to end at B = 1e5: states from pinned host memory, rates back to the host
    B = 100000
    Y, T, P = _rate_states(spec, B, 1 + rank)
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
    work = spec.I * (20 + 2 * EXP_FLOPS) + spec.K * 45 + (spec.n_troe) * (4 * EXP_FLOPS + 2 * LOG_FLOPS + 30)
    achieved = work * value / 1e12
    line = {"metric": RATES_METRIC, "value": value, "unit": "states/s", "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_big, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": workload_config(RATES, world, B_big, spec),
            "states_per_s_by_batch": {str(b): v for b, v in per_b.items()},
            "roofline": {"bound": "alu", "pipe": "fp64", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None,
                         "work_model": "per state: I (20 + 2 exp) + 45 K + Troe terms, exp=40 flop slots"},
            "e2e": {"value": B * K / e_t, "unit": "states/s", "h2d_bytes_per_step": B * (spec.K + 2) * 8,
                    "d2h_bytes_per_step": B * (spec.I + spec.K) * 8},
            "gpu_launches": K * 5, "clocks": sampler.summary()}
    if not args.no_cpu_baseline:
        tc = oracle_rates_time(spec, 20000)
        line["cpu_baseline"] = {"value": 1.0 / tc, "unit": "states/s", "cores": 1, "kind": "oracle",
                                "sample": "20000 states, the oracle's vectorised numpy rate functions"}
        line["gpu_over_oracle_by_batch"] = {str(b): v * tc for b, v in per_b.items()}
    if rank == 0:
        print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == MIXED:
        run_multi(args)
    elif args.workload == RATES:
        run_rates(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
