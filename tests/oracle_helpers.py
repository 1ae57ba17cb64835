"""Shared helpers for the oracle tests: golden mechanisms and seeded workloads."""
import functools
import os

import numpy as np

from oracle import psr_oracle as O
from paper_2005_11468_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_text(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return fh.read()


def golden(name):
    return O.Mechanism(golden_text(name))


@functools.lru_cache(maxsize=None)
def workload(name):
    spec = synth.workload_mechanism(name)
    text = synth.mechanism_text(spec)
    return spec, O.Mechanism(text), synth.workload_batch(name, spec)


def random_states(mech, m, seed, T_range=(600.0, 2500.0), y_small=False):
    """Seeded states (m, K+1): mass fractions on the simplex (some species tiny),
    temperatures uniform."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Y = rng.dirichlet(np.full(mech.K, 0.7), size=m)
    if y_small:
        Y = np.where(rng.random(Y.shape) < 0.3, Y * 1e-9, Y)
        Y /= Y.sum(1, keepdims=True)
    T = rng.uniform(*T_range, m)
    return np.concatenate([Y, T[:, None]], axis=1)


def inlet_for(mech, seed, tau=1e-3, T_in=500.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    Y_in = np.zeros(mech.K)
    Y_in[:min(4, mech.K)] = rng.dirichlet([1.0] * min(4, mech.K))
    return O.Inlet(Y_in, T_in, tau, synth.ONE_ATM)
