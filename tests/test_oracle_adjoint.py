"""Pins of the oracle's sensitivities d(Y, T)/d ln(rate multiplier): central finite
differences of re-solved roots (h = 1e-6 on the parameter), each perturbed solve
polished to the rounding floor; and the closed form of the isomerisation toy."""
import math

import numpy as np
import pytest

from oracle import psr_oracle as O
from paper_2005_11468_gb300 import synth
from tests.oracle_helpers import golden, workload

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

TIGHT = O.Options(step_rtol=1e-13, step_atol_y=1e-18, step_atol_t=1e-12)


def test_isomerisation_sensitivity_closed_form():
    """A <=> B at fixed T: Y_A = (Y_A,in + tau k_r s)/(1 + tau (k_f + k_r)), s = Y_A,in + Y_B,in;
    one multiplier m scales both k_f and k_r, so dY_A/d ln m follows in closed form."""
    mech = golden("isomer_ab.psrmech")
    T, tau = 1500.0, 1e-3
    Y_in = np.array([0.5, 0.4, 0.1])
    inlet = O.Inlet(Y_in, 500.0, tau, synth.ONE_ATM, T_spec=T)
    r = O.solve_reactor(mech, inlet, np.r_[Y_in, T], TIGHT, energy="fixed")
    kf = 1000.0
    kr = kf / math.exp((5.5 - 6.0) - (1500.0 - 2000.0) / T)
    s = 0.5
    # d/d ln m at m = 1 of (a + tau kr m s)/(1 + tau m (kf + kr))
    num, den = 0.4 + tau * kr * s, 1 + tau * (kf + kr)
    dYA = (tau * kr * s * den - num * tau * (kf + kr)) / den**2
    S = O.sensitivities(mech, inlet, r.x, energy="fixed")
    np.testing.assert_allclose(S[1, 0], dYA, rtol=1e-10)
    np.testing.assert_allclose(S[2, 0], -dYA, rtol=1e-10)
    assert S[3, 0] == 0.0 and abs(S[0, 0]) < 1e-18


def test_sensitivities_match_finite_differences_of_resolved_roots():
    _, mech, batch = workload("k10_b64")
    rng = np.random.Generator(np.random.PCG64(2))
    for b in (1, 2):
        inlet = O.inlet_of(batch, b)
        x0 = np.r_[batch.Y0[b], batch.T0[b]]
        r = O.solve_reactor(mech, inlet, x0, TIGHT)
        assert r.status == O.CONVERGED
        S = O.sensitivities(mech, inlet, r.x)
        h = 1e-6
        for i in rng.choice(mech.I, 4, replace=False):
            lp = np.zeros(mech.I); lp[i] = h
            xp = O.solve_reactor(mech, inlet, r.x, TIGHT, lnmult=lp).x
            xm = O.solve_reactor(mech, inlet, r.x, TIGHT, lnmult=-lp).x
            fd = (xp - xm) / (2 * h)
            scale = np.abs(S).max()
            big = np.abs(S[:, i]) > 1e-6 * scale
            # a root is known to about one ulp, so the difference quotient carries up to
            # ulp(x)/h of rounding on top of its O(h^2) truncation
            floor = 4 * np.finfo(float).eps * np.abs(r.x[big]) / h
            np.testing.assert_array_less(np.abs(fd[big] - S[big, i]), 1e-4 * np.abs(S[big, i]) + 1e-7 * scale + floor)


def test_adjoint_is_g_times_sensitivities():
    _, mech, batch = workload("k10_b64")
    inlet = O.inlet_of(batch, 3)
    r = O.solve_reactor(mech, inlet, np.r_[batch.Y0[3], batch.T0[3]], TIGHT)
    g = np.random.Generator(np.random.PCG64(4)).standard_normal(mech.K + 1)
    np.testing.assert_allclose(O.adjoint_gradient(mech, inlet, r.x, g),
                               g @ O.sensitivities(mech, inlet, r.x), rtol=1e-13)
