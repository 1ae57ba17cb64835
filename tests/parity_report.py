"""Per-output error of the GPU solves against the FP64 oracle (test infrastructure).

The GPU tests assert the parity bar (Y_k > 1e-10 to 1e-6 relative, T to 1e-8 K, soot
moments to 1e-5 relative); this script measures how far inside the bar each output lands,
per workload and per form, and counts the reactors that miss it. It runs in two phases,
so that the GPU machine only solves:

  python tests/parity_report.py gpu OUT.npz
      needs a GPU: solves each workload's full batch in both forms (PSR_MIXED, PSR_FP64)
      through the C ABI and keeps the outputs of a seeded sample of reactors. Imports
      nothing from the oracle.
  python tests/parity_report.py cpu OUT.npz [--procs N]
      anywhere: solves the sampled reactors with the oracle (a process pool, one reactor
      per task) and prints a markdown table per workload and form.

Classification of a sampled reactor the oracle converged (the multiple-root reading of the
steady problem): "pass" = the GPU converged on the same branch (|dT| <= 1 K) within the
bar; "branch" = the GPU converged on another branch and its state is a root of the
oracle's residual (||F||inf <= 1e-7); "off" = same branch but outside the bar, reported
with the condition number of the oracle's Jacobian at its root (an FP64 solve cannot fix a
component better than about cond * 1e-16 relative); "gpu-unconv" = the GPU did not
converge. Reactors the oracle did not converge are counted apart.
"""
import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2005_11468_gb300 import synth  # noqa: E402
from tests import oracle_pool  # noqa: E402

Y_REL, Y_MIN, T_ABS, M_REL = 1e-6, 1e-10, 1e-8, 1e-5
SAMPLE_SEED = 20051146 + 97
# sampled reactors per workload (the oracle takes ~0.05 s (K = 10), ~0.7 s (K = 53),
# ~5-12 s (K = 53 + soot) and ~10 s (K = 200) per reactor on one core)
SAMPLES = {"k10_b64": 64, "k53_b4096": 96, "k200_b2048": 24, "k53soot_b16384": 48}
MIXED_SAMPLES = (16, 16, 8)      # per mechanism class of the uneven batch (K = 10, 53, 200)
FORMS = (("mixed", 1), ("fp64", 0))     # PSR_MIXED = 1, PSR_FP64 = 0


def sample(B, m, salt):
    rng = np.random.Generator(np.random.PCG64(SAMPLE_SEED + salt))
    return np.sort(rng.choice(B, size=min(m, B), replace=False))


# ------------------------------------------------------------------------------ GPU phase
def gpu_results(samples=SAMPLES, mixed_samples=MIXED_SAMPLES):
    """Solve each workload's full batch in both forms on cuda:0 through the C ABI and keep
    the outputs of the seeded sample (the first `samples[name]` of the report's sample, so
    that a smaller sample is a subset of the larger one). Returns the arrays by key."""
    import torch
    from paper_2005_11468_gb300 import _build, psr
    _build.build()
    dev = torch.device("cuda:0")
    out = {}

    def dv(a, dtype=torch.float64):
        return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device=dev)

    for salt, name in enumerate(SAMPLES):
        if name not in samples:
            continue
        spec = synth.workload_mechanism(name)
        gm = psr.Mechanism(synth.mechanism_text(spec))
        batch = synth.workload_batch(name, spec)
        idx = sample(batch.B, SAMPLES[name], salt)[:samples[name]]
        t = {k: dv(getattr(batch, k)) for k in ("Y_in", "T_in", "tau", "P", "Y0", "T0")}
        for form, prec in FORMS:
            t0 = time.time()
            if spec.soot is not None:
                r = psr.batch_solve_soot(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], dv(batch.M_in), t["Y0"],
                                         t["T0"], opts=psr.Options(precision=prec))
            else:
                r = psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"],
                                    opts=psr.Options(precision=prec))
            torch.cuda.synchronize()
            key = f"{name}|{form}"
            st = r["status"].cpu().numpy()
            out[key + "|idx"] = idx
            out[key + "|Y"] = r["Y"].cpu().numpy()[idx]
            out[key + "|T"] = r["T"].cpu().numpy()[idx]
            out[key + "|status"] = st[idx]
            out[key + "|conv_all"] = np.array([np.isin(st, psr.CONVERGED_STATES).mean()])
            if "M" in r:
                out[key + "|M"] = r["M"].cpu().numpy()[idx]
            print(f"{key}: {time.time() - t0:.1f} s, converged {out[key + '|conv_all'][0]:.4f}", flush=True)
        gm.close()

    if mixed_samples is None:
        return out
    specs = [synth.workload_mechanism(nm) for nm in synth.MIXED_WORKLOAD["parts"]]
    gms = [psr.Mechanism(synth.mechanism_text(sp)) for sp in specs]
    mb = synth.mixed_batch(specs)
    td = {k: dv(mb[k]) for k in ("Y_in", "Y0", "T_in", "tau", "P", "T0")}
    mid, off = dv(mb["mech_id"], torch.int32), dv(mb["row_off"], torch.int64)
    for form, prec in FORMS:
        r = psr.batch_solve_multi(gms, mid, off, td["Y_in"], td["T_in"], td["tau"], td["P"], td["Y0"], td["T0"],
                                  opts=psr.Options(precision=prec))
        torch.cuda.synchronize()
        Y, T, st = r["Y"].cpu().numpy(), r["T"].cpu().numpy(), r["status"].cpu().numpy()
        for c, spec in enumerate(specs):
            mem = mb["members"][c]
            j = sample(len(mem), MIXED_SAMPLES[c], 50 + c)[:mixed_samples[c]]
            rows = mem[j]
            key = f"mixed_b32768:{synth.MIXED_WORKLOAD['parts'][c]}|{form}"
            out[key + "|idx"] = j
            out[key + "|Y"] = np.stack([Y[mb["row_off"][g]:mb["row_off"][g] + spec.K] for g in rows])
            out[key + "|T"] = T[rows]
            out[key + "|status"] = st[rows]
            out[key + "|conv_all"] = np.array([np.isin(st[mem], psr.CONVERGED_STATES).mean()])
        print(f"mixed_b32768|{form}: converged {np.isin(st, psr.CONVERGED_STATES).mean():.4f}", flush=True)
    for g in gms:
        g.close()
    return out


def gpu_phase(path):
    np.savez(path, **gpu_results())


# ------------------------------------------------------------------------------ CPU phase
def oracle_tasks(d, want_cond=True):
    keys = sorted({k.rsplit("|", 2)[0] for k in d})
    return sorted({(k, int(b), want_cond) for k in keys for b in d[f"{k}|mixed|idx"]})


def classify(d, res):
    """One row per workload and form: counts of pass / other branch / off bar / GPU
    unconverged / oracle unconverged among the sampled reactors, and the error maxima."""
    from oracle import psr_oracle as O
    from paper_2005_11468_gb300.psr import CONVERGED_STATES
    keys = sorted({k.rsplit("|", 2)[0] for k in d})
    rows = []
    for key in keys:
        mech, batch, soot = oracle_pool.problem(key)
        K = mech.K
        for form, _ in FORMS:
            p = f"{key}|{form}"
            idx, Y, T, st = d[p + "|idx"], d[p + "|Y"], d[p + "|T"], d[p + "|status"]
            M = d.get(p + "|M")
            row = dict(key=key, form=form, sampled=len(idx), n_pass=0, branch=0, off=0, gpu_unconv=0,
                       oracle_unconv=0, ey=[], et=[], em=[], conds=[], conv_all=float(d[p + "|conv_all"][0]),
                       soot=M is not None)
            for j, b in enumerate(idx):
                x, s, Mo, cond = res[(key, int(b))]
                if s != O.CONVERGED:
                    row["oracle_unconv"] += 1
                    continue
                if st[j] not in CONVERGED_STATES:
                    row["gpu_unconv"] += 1
                    continue
                if abs(T[j] - x[K]) > 1.0:
                    fr = oracle_pool.root_residual(key, int(b), Y[j], T[j], None if M is None else M[j])
                    row["branch" if fr <= 1e-7 else "off"] += 1
                    continue
                big = x[:K] > Y_MIN
                rel = float(np.max(np.abs(Y[j][big] - x[:K][big]) / x[:K][big]))
                dT = float(abs(T[j] - x[K]))
                rm = float(np.max(np.abs(M[j] - Mo) / Mo)) if M is not None else 0.0
                row["ey"].append(rel)
                row["et"].append(dT)
                row["em"].append(rm)
                if rel <= Y_REL and dT <= T_ABS and rm <= M_REL:
                    row["n_pass"] += 1
                else:
                    row["off"] += 1
                    row["conds"].append(cond)
            rows.append(row)
    return rows


def table(rows):
    lines = ["| workload | form | sampled | pass | other branch | off bar (max cond J) | GPU unconv. | "
             "oracle unconv. | max rel err Y (Y>1e-10) | median | max abs err T (K) | max rel err M | "
             "converged (full batch) |",
             "|---|---|---|---|---|---|---|---|---|---|---|---|---|"]
    for r in rows:
        ey = r["ey"]
        offs = f"{r['off']}" + (f" ({max(r['conds']):.1e})" if r["conds"] else "")
        fmt = (lambda v: f"{max(v):.1e}") if ey else (lambda v: "–")
        lines.append(f"| {r['key']} | {r['form']} | {r['sampled']} | {r['n_pass']} | {r['branch']} | {offs} | "
                     f"{r['gpu_unconv']} | {r['oracle_unconv']} | {fmt(ey)} | "
                     f"{np.median(ey) if ey else float('nan'):.1e} | {fmt(r['et'])} | "
                     f"{fmt(r['em']) if r['soot'] else '–'} | {r['conv_all']:.4f} |")
    return "\n".join(lines)


def cpu_phase(path, procs):
    d = dict(np.load(path))
    tasks = oracle_tasks(d)
    t0 = time.time()
    res = oracle_pool.solve(tasks, procs)
    print(f"oracle: {len(tasks)} reactors in {time.time() - t0:.0f} s on {procs} processes\n")
    print(table(classify(d, res)))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("phase", choices=["gpu", "cpu"])
    ap.add_argument("path")
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    a = ap.parse_args()
    if a.phase == "gpu":
        gpu_phase(a.path)
    else:
        cpu_phase(a.path, a.procs)


if __name__ == "__main__":
    main()
