"""Oracle solves of seeded workload reactors in a pool of worker processes (test
infrastructure: GPU parity tests and the per-output error report use it).

The pool is started with the `spawn` method, so it is safe to open after the parent has
used the GPU (a process forked after the first CUDA call can hang), and each worker runs
with one BLAS thread: with a thread pool in each of several processes the oracle's small
matrix products ran about 20x slower on oversubscribed cores.

A task is (key, b): reactor b of the workload `key`, or of one mechanism class of the
uneven batch (`"mixed_b32768:<class workload>"`, b indexing that class's own batch).
"""
import math
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2005_11468_gb300 import synth  # noqa: E402

_CACHE = {}


def problem(key):
    """Oracle mechanism, batch and soot flag of a task key."""
    from oracle import psr_oracle as O
    if key not in _CACHE:
        if key.startswith("mixed_b32768:"):
            part = key.split(":")[1]
            specs = [synth.workload_mechanism(nm) for nm in synth.MIXED_WORKLOAD["parts"]]
            c = synth.MIXED_WORKLOAD["parts"].index(part)
            mb = synth.mixed_batch(specs)
            spec, batch = specs[c], mb["batches"][c]
        else:
            spec = synth.workload_mechanism(key)
            batch = synth.workload_batch(key, spec)
        _CACHE[key] = (O.Mechanism(synth.mechanism_text(spec)), batch, spec.soot is not None)
    return _CACHE[key]


def oracle_task(arg):
    """One oracle solve: (key, b, x = (Y, T), status, moments or None, cond(J) or nan).
    The condition number of the oracle's Jacobian at its root is computed only when the
    task asks for it (a third element True)."""
    import warnings
    from oracle import momic_oracle as S
    from oracle import psr_oracle as O
    warnings.filterwarnings("ignore", category=RuntimeWarning)
    key, b = arg[0], int(arg[1])
    want_cond = len(arg) > 2 and arg[2]
    mech, batch, soot = problem(key)
    inlet = O.inlet_of(batch, b)
    if soot:
        r, M = S.solve_soot_reactor(mech, inlet, batch.Y0[b], batch.T0[b], batch.M_in[b])
        system = S.SootSystem(mech, inlet, batch.M_in[b])
    else:
        r = O.solve_reactor(mech, inlet, np.r_[batch.Y0[b], batch.T0[b]])
        M = None
        system = O.GasSystem(mech, inlet)
    cond = math.nan
    if want_cond and r.status == O.CONVERGED:
        cond = float(np.linalg.cond(O.jacobian_cs(system, r.x)))
    return key, b, r.x[:mech.K + 1].copy(), int(r.status), M, cond


def solve(tasks, procs=None):
    """{(key, b): (x, status, M, cond)} for every task, solved in a spawn pool."""
    tasks = sorted(set(tuple(t) for t in tasks))
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    procs = max(1, min(procs or os.cpu_count() or 1, len(tasks)))
    # the slowest classes first, so that the pool does not end on one long task
    order = sorted(tasks, key=lambda t: -problem(t[0])[0].K - (100 if problem(t[0])[2] else 0))
    with mp.get_context("spawn").Pool(procs) as pool:
        return {(k, b): (x, s, M, c) for k, b, x, s, M, c in pool.imap_unordered(oracle_task, order)}


def root_residual(key, b, Y, T, M=None):
    """||F||_inf of the oracle's residual at a GPU state (a root on another branch?)."""
    from oracle import momic_oracle as S
    from oracle import psr_oracle as O
    mech, batch, soot = problem(key)
    inlet = O.inlet_of(batch, b)
    if soot:
        system = S.SootSystem(mech, inlet, batch.M_in[b])
        x = np.r_[Y, T, np.log(M / system.soot.scale)]
    else:
        system = O.GasSystem(mech, inlet)
        x = np.r_[Y, T]
    return float(np.max(np.abs(system.F(x[None])[0])))
