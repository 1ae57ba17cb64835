"""Pins of the CPU oracle against what the paper and the mathematics fix.

The paper prints no worked example values (its figures are absent and it has no
tables), so every pin here is a closed form, an exact identity, a special case that
reduces to a textbook or library routine, or a brute-force search. Each targets a
plausible mistake: a dropped term, a wrong sign or index, a transposed operand, a
wrong standard-state factor.
"""
import math
import types

import numpy as np
import pytest
import scipy.linalg
from scipy.optimize import brentq

from oracle import psr_oracle as O
from paper_2005_11468_gb300 import synth
from tests.oracle_helpers import golden, golden_text, inlet_for, random_states, workload

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ------------------------------------------------------------------ LU (Sec. 1, Sec. 3)
@pytest.mark.parametrize("n", [1, 2, 5, 11, 54, 60])
def test_lu_matches_lapack(n):
    """Partial-pivot LU equals LAPACK getrf (same pivot rule: first largest |a|)."""
    rng = np.random.Generator(np.random.PCG64(n))
    A = rng.standard_normal((n, n)) * np.exp(rng.uniform(-3, 3, (n, 1)))
    b = rng.standard_normal(n)
    LU, piv, ok = O.lu_factor(A)
    assert ok
    lu_ref, ipiv = scipy.linalg.lu_factor(A)
    perm = np.arange(n)
    for k, p in enumerate(ipiv):
        perm[[k, p]] = perm[[p, k]]
    np.testing.assert_array_equal(piv, perm)
    np.testing.assert_allclose(LU, lu_ref, rtol=1e-12, atol=1e-12 * np.abs(lu_ref).max())
    x = O.lu_solve(LU, piv, b)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-12)
    # backward error of the solve
    assert np.max(np.abs(A @ x - b)) <= 50 * n * 2.2e-16 * np.abs(A).max() * np.abs(x).max()


def test_lu_flags_singular():
    A = np.array([[1.0, 2.0], [2.0, 4.0]])
    _, _, ok = O.lu_factor(A)
    assert not ok


# ------------------------------------------------------------------ NASA-7 thermo
@pytest.mark.parametrize("split", [False, True])
def test_nasa_enthalpy_and_entropy_derivatives(split):
    """dH/dT = c_p and dS/dT = c_p / T for the polynomials, both ranges."""
    spec = synth.make_mechanism(10, 24, seed=7, split_ranges=split)
    mech = O.Mechanism(synth.mechanism_text(spec))
    for T in (350.0, 800.0, 1500.0, 3200.0):
        h = 1e-3
        Ts = np.array([T - h, T, T + h])
        cp, h_RT, s_R = O.species_thermo(mech, Ts)
        H = h_RT * Ts[:, None]                    # H / R in kelvin
        np.testing.assert_allclose((H[2] - H[0]) / (2 * h), cp[1], rtol=1e-8)
        np.testing.assert_allclose((s_R[2] - s_R[0]) / (2 * h), cp[1] / T, rtol=1e-8)


def test_nasa_range_switch():
    """The low-range set applies below T_mid, the high-range set at and above it:
    a species with c_p/R = 3 below 1000 K and 5 above."""
    text = golden_text("isomer_ab.psrmech").replace("0 N2 0 0 0 2 200 1000 5000 3.5 0 0 0 0 -1000 4 3.5 0 0 0 0 -1000 4",
                        "0 N2 0 0 0 2 200 1000 5000 3 0 0 0 0 -1000 4 5 0 0 0 0 -1000 4")
    mech = O.Mechanism(text)
    cp, h_RT, _ = O.species_thermo(mech, np.array([999.0, 1000.0, 1500.0]))
    assert cp[0, 0] == 3.0 and cp[1, 0] == 5.0 and cp[2, 0] == 5.0
    assert h_RT[2, 0] == 5.0 - 1000.0 / 1500.0


# ------------------------------------------------------------------ Eq. (6)
def test_arrhenius_special_cases():
    mech = golden("arrhenius_cases.psrmech")
    kf1000 = O.forward_rate_constants(mech, np.array([1000.0]))[0]
    kf2000 = O.forward_rate_constants(mech, np.array([2000.0]))[0]
    assert kf1000[0] == 2500.0 and kf2000[0] == 2500.0
    np.testing.assert_allclose(kf1000[1], 3.0 * 1000.0, rtol=1e-15)
    np.testing.assert_allclose(kf2000[2], 7.0 * 2000.0**2, rtol=1e-15)
    np.testing.assert_allclose(kf1000[3], 6.0e8 / 2.0, rtol=1e-14)
    np.testing.assert_allclose(kf2000[4], 8.0e9 / (2000.0 * 10.0), rtol=1e-14)


# ------------------------------------------------------------------ Eqs. (8)-(9)
def test_van_t_hoff():
    """d ln K_p / dT = sum nu H / (R T^2): K_c = K_p (P_atm/RT)^dnu, so
    d ln K_c / dT = sum nu H/(R T^2) - dnu / T."""
    _, mech, _ = workload("k10_b64")
    for T in (700.0, 1800.0, 3000.0):
        h = 1e-3
        lnK = np.log(O.equilibrium_constants(mech, np.array([T - h, T + h])))
        d = (lnK[1] - lnK[0]) / (2 * h)
        _, h_RT, _ = O.species_thermo(mech, np.array([T]))
        expect = (h_RT[0] @ mech.nu) / T - mech.nu.sum(0) / T
        np.testing.assert_allclose(d, expect, rtol=1e-6, atol=1e-9)


def test_isomerisation_closed_form():
    """A <=> B, fixed T: the steady balance is linear (see the golden file)."""
    mech = golden("isomer_ab.psrmech")
    T, tau = 1500.0, 1e-3
    Y_in = np.array([0.5, 0.4, 0.1])
    inlet = O.Inlet(Y_in, 500.0, tau, synth.ONE_ATM, T_spec=T)
    r = O.solve_reactor(mech, inlet, np.r_[Y_in, T], energy="fixed")
    assert r.status == O.CONVERGED
    kf = 1000.0
    Kc = math.exp((5.5 - 6.0) - (1500.0 - 2000.0) / T)
    kr = kf / Kc
    YA = (Y_in[1] + tau * kr * (Y_in[1] + Y_in[2])) / (1 + tau * (kf + kr))
    np.testing.assert_allclose(r.x[1], YA, rtol=1e-12)
    np.testing.assert_allclose(r.x[2], Y_in[1] + Y_in[2] - YA, rtol=1e-12)
    np.testing.assert_allclose(r.x[0], Y_in[0], rtol=1e-14)


def test_dimerisation_closed_form():
    """2 A <=> A2, fixed T: one scalar balance solved by bracketing (golden file)."""
    mech = golden("dimer.psrmech")
    T, tau, P = 1500.0, 1e-4, synth.ONE_ATM
    Y_in = np.array([0.7, 0.3, 0.0])
    inlet = O.Inlet(Y_in, 500.0, tau, P, T_spec=T)
    r = O.solve_reactor(mech, inlet, np.r_[Y_in, T], energy="fixed")
    assert r.status == O.CONVERGED
    W = mech.W
    kf = 3.0e12
    Kc = math.exp((1 - 2 * 3) - (-2000.0 - 2 * 4000.0) / T) * (O.P_ATM / (O.R_U * T)) ** (-1)
    kr = kf / Kc

    def g(yA):
        yA2 = Y_in[1] + Y_in[2] - yA
        rho = P / (O.R_U * T) / (Y_in[0] / W[0] + yA / W[1] + yA2 / W[2])
        cA, cA2 = rho * yA / W[1], rho * yA2 / W[2]
        return yA - Y_in[1] + 2 * tau * W[1] * (kf * cA**2 - kr * cA2) / rho

    yA = brentq(g, 0.0, Y_in[1], xtol=1e-16, rtol=1e-15)
    np.testing.assert_allclose(r.x[1], yA, rtol=1e-10)


def _isomer_constants(mech, T, P, Y_in):
    """rho, W_A and the mass fraction sum S of the A/B pair of the isomerisation goldens
    (W_A = W_B, so both stay constant at fixed T and P)."""
    W = mech.comp @ np.array([12.011, 1.008, 15.999, 14.007])
    S = Y_in[1] + Y_in[2]
    rho = P / (O.R_U * T) / (Y_in[0] / W[0] + S / W[1])
    return rho, W, S


def test_third_body_isomerisation_closed_form():
    """A + M <=> B + M with distinct efficiencies, fixed T: the steady balance of A is a
    quadratic in Y_A (golden file). Catches a dropped [M] factor, efficiencies of the
    wrong species or default efficiencies where the file lists others."""
    mech = golden("tb_isomer.psrmech")
    T, tau, P = 1500.0, 1e-3, synth.ONE_ATM
    Y_in = np.array([0.5, 0.4, 0.1])
    inlet = O.Inlet(Y_in, 500.0, tau, P, T_spec=T)
    r = O.solve_reactor(mech, inlet, np.r_[Y_in, T], energy="fixed")
    assert r.status == O.CONVERGED
    rho, W, S = _isomer_constants(mech, T, P, Y_in)
    kf = 1.0e8
    kr = kf / math.exp((5.5 - 6.0) - (1500.0 - 2000.0) / T)
    m0 = 2.5 * rho * Y_in[0] / W[0] + 1.5 * rho * S / W[1]
    m1 = (0.5 - 1.5) * rho / W[1]
    a = tau * m1 * (kf + kr)
    b = 1.0 + tau * m0 * (kf + kr) - tau * m1 * kr * S
    c = -(Y_in[1] + tau * m0 * kr * S)
    roots = np.roots([a, b, c]).real
    YA = roots[(roots >= 0) & (roots <= S)]
    assert YA.size == 1
    # the [M] factor matters here: tau k_f [M] is of order one
    assert 0.1 < tau * kf * (m0 + m1 * YA[0]) < 10
    np.testing.assert_allclose(r.x[1], YA[0], rtol=1e-12)
    np.testing.assert_allclose(r.x[2], S - YA[0], rtol=1e-12)


def _falloff_isomer_closed_form(fixture):
    """Fixed-T steady state of the falloff isomerisation fixtures (F = F_cent = 1/2 at the
    centre of the broadening curve): the oracle's root and the closed-form Y_A, Y_B."""
    mech = golden(fixture)
    T, tau, P = 1500.0, 1e-3, synth.ONE_ATM
    Y_in = np.array([0.5, 0.4, 0.1])
    inlet = O.Inlet(Y_in, 500.0, tau, P, T_spec=T)
    r = O.solve_reactor(mech, inlet, np.r_[Y_in, T], energy="fixed")
    assert r.status == O.CONVERGED
    rho, W, S = _isomer_constants(mech, T, P, Y_in)
    k_inf, k_0 = 2000.0, 257582561.28170544
    M = 2.0 * rho * Y_in[0] / W[0] + rho * S / W[1]
    Pr = k_0 * M / k_inf
    # the fixture sits at the centre: log10 P_r + c = 0 with c = -0.4 - 0.67 log10(1/2)
    assert abs(math.log10(Pr) - 0.4 - 0.67 * math.log10(0.5)) < 1e-9
    kf = k_inf * Pr / (1.0 + Pr) * 0.5
    kr = kf / math.exp((5.5 - 6.0) - (1500.0 - 2000.0) / T)
    YA = (Y_in[1] + tau * kr * S) / (1.0 + tau * (kf + kr))
    return r, YA, S


def test_falloff_isomerisation_at_the_troe_centre():
    """A (+M) <=> B (+M), Troe falloff at the centre of the broadening curve (F = F_cent
    = 1/2, golden file): k_f = k_inf P_r / (1 + P_r) / 2 with P_r = k_0 [M] / k_inf, then
    the linear isomerisation closed form. Catches a missing Lindemann blend, a missing F,
    [M] without efficiencies, and an extra [M] factor on a falloff rate of progress."""
    r, YA, S = _falloff_isomer_closed_form("troe_isomer.psrmech")
    np.testing.assert_allclose(r.x[1], YA, rtol=1e-12)
    np.testing.assert_allclose(r.x[2], S - YA, rtol=1e-12)


def test_falloff_isomerisation_t2_term():
    """The same closed form with F_cent = 1/2 made by the four-parameter T** term alone
    (alpha = 0, T*** -> 0+, T** = T ln 2; golden file). Catches the T** term read as
    exp(-T/T**) (F_cent = 0.236) or dropped (F_cent = 0)."""
    r, YA, S = _falloff_isomer_closed_form("troe_t2_isomer.psrmech")
    np.testing.assert_allclose(r.x[1], YA, rtol=1e-12)
    np.testing.assert_allclose(r.x[2], S - YA, rtol=1e-12)


# ------------------------------------------------------------------ Troe falloff
def _troe(alpha, T3, T1, T2):
    return types.SimpleNamespace(troe=np.array([[alpha, T3, T1, T2]]))


def test_troe_fcent_one_is_lindemann():
    m = _troe(1.0, 100.0, np.inf, 0.0)        # F_cent = exp(-T/inf) = 1
    Pr = np.logspace(-8, 8, 17)[None, :].T
    F = O.troe_broadening(m, np.full(17, 1500.0), Pr)
    np.testing.assert_allclose(F, 1.0, rtol=0, atol=1e-15)


@pytest.mark.parametrize("T", [800.0, 1500.0, 2600.0])
def test_troe_t2_term_alone(T):
    """alpha = 0 and T*** -> 0+ leave F_cent = exp(-T**/T); with T** = T ln 2 that is 1/2,
    and at the centre log10 P_r = -c the broadening factor equals F_cent. A second T**
    (= T ln 4, F_cent = 1/4) checks the exponent's scaling, and the centre of each lies
    where F is smallest."""
    for t2, fc in ((T * math.log(2.0), 0.5), (T * math.log(4.0), 0.25)):
        m = _troe(0.0, 1e-30, 1.0, t2)
        c = -0.4 - 0.67 * math.log10(fc)
        F = O.troe_broadening(m, np.array([T]), np.array([[10.0 ** (-c)]]))[0, 0]
        np.testing.assert_allclose(F, fc, rtol=1e-13)
        pr = 10.0 ** (-c + np.linspace(-3, 3, 61))
        Fs = O.troe_broadening(m, np.full(1, T), pr[None, :])[0]
        assert np.all(Fs >= fc * (1 - 1e-13)) and np.argmin(Fs) == 30


def test_troe_centre_and_limits():
    T = 1200.0
    m = _troe(0.0, T / math.log(2.0), 1.0, 0.0)   # F_cent = exp(-ln 2) = 1/2 exactly
    lf = math.log10(0.5)
    c = -0.4 - 0.67 * lf
    F_mid = O.troe_broadening(m, np.array([T]), np.array([[10.0 ** (-c)]]))[0, 0]
    np.testing.assert_allclose(F_mid, 0.5, rtol=1e-14)
    # log10 F = log10 F_cent / (1 + f1^2) with 1 + f1^2 >= 1: F_cent <= F <= 1, the
    # minimum F_cent sits at f1 = 0, and F -> F_cent^(1/(1 + (1/0.14)^2)) far away
    pr = np.logspace(-40, 40, 801)
    F = O.troe_broadening(m, np.full(1, T), pr[None, :])[0]
    assert np.all(F >= 0.5 - 1e-15) and np.all(F <= 1.0)
    j = int(np.argmin(F))
    assert abs(math.log10(pr[j]) + c) <= 0.1
    # the denominator n - 0.14 (log10 P_r + c) vanishes at log10 P_r = n/0.14 - c,
    # where f1 is unbounded and F reaches 1
    n = 0.75 - 1.27 * lf
    F_pole = O.troe_broadening(m, np.array([T]), np.array([[10.0 ** (n / 0.14 - c) * (1 + 1e-12)]]))
    np.testing.assert_allclose(F_pole, 1.0, atol=1e-9)
    lim = 0.5 ** (1.0 / (1.0 + (1.0 / 0.14) ** 2))
    assert abs(F[0] - lim) < 0.02 and abs(F[-1] - lim) < 0.02


# ------------------------------------------------------------------ Eq. (4): conservation
@pytest.mark.parametrize("name", ["k10_b64", "k53_b4096", "k200_b2048", "k53soot_b16384"])
def test_wdot_conserves_mass_and_elements(name):
    _, mech, _ = workload(name)
    X = random_states(mech, 16, seed=3)
    Y, T = X[:, :-1], X[:, -1]
    _, rho, C = O.mixture_state(mech, Y, T, synth.ONE_ATM)
    q = O.rates_of_progress(mech, T, C)
    wdot = O.net_production_rates(mech, q)
    gross = np.abs(q) @ np.abs(mech.nu.T)          # (m, K) sum_i |nu_ki q_i|
    mass = wdot @ mech.W
    assert np.all(np.abs(mass) <= 1e-13 * (gross @ mech.W))
    elem = wdot @ mech.comp
    assert np.all(np.abs(elem) <= 1e-13 * (gross @ mech.comp) + 1e-300)


@pytest.mark.parametrize("name", ["k10_b64", "k53_b4096", "k200_b2048", "k53soot_b16384"])
def test_residual_identities(name):
    """For any state: sum_k F_k = sum_k (Y_k - Y_k,in); the element combinations of F
    equal those of Y - Y_in; and the energy row obeys
    F_T c_p T + sum_k h_k F_k = h(T, Y) - h_in (Eq. (3) against Eq. (2))."""
    _, mech, _ = workload(name)
    inlet = inlet_for(mech, seed=5, tau=3e-3, T_in=450.0)
    X = random_states(mech, 12, seed=4)
    F = O.gas_residual(mech, X, inlet)
    Y, T = X[:, :-1], X[:, -1]
    scale = 1.0 + np.abs(F[:, :-1]).sum(1)
    assert np.all(np.abs(F[:, :-1].sum(1) - (Y.sum(1) - inlet.Y_in.sum())) <= 1e-13 * scale)
    e_F = (F[:, :-1] / mech.W) @ mech.comp
    e_Y = ((Y - inlet.Y_in) / mech.W) @ mech.comp
    escale = ((np.abs(F[:, :-1]) + np.abs(Y)) / mech.W) @ mech.comp + 1e-30
    assert np.all(np.abs(e_F - e_Y) <= 1e-13 * escale)
    cp_R, h_RT, _ = O.species_thermo(mech, T)
    h = h_RT * O.R_U * T[:, None] / mech.W
    cp = np.sum(Y * cp_R * O.R_U / mech.W, axis=1)
    lhs = F[:, -1] * cp * T + np.sum(h * F[:, :-1], axis=1)
    rhs = O.mixture_enthalpy(mech, Y, T) - O.mixture_enthalpy(mech, inlet.Y_in[None], np.array([inlet.T_in]))
    hscale = np.abs(F[:, -1] * cp * T) + np.sum(np.abs(h * F[:, :-1]), axis=1) + np.abs(rhs)
    assert np.all(np.abs(lhs - rhs) <= 1e-12 * hscale)


# ------------------------------------------------------------------ Jacobian
def test_jacobian_complex_step_vs_central_differences():
    _, mech, _ = workload("k53_b4096")
    inlet = inlet_for(mech, seed=6, tau=1e-3)
    S = O.GasSystem(mech, inlet)
    for x in random_states(mech, 3, seed=8):
        Jc = O.jacobian_cs(S, x)
        Jf = O.jacobian_fd(S, x, O.Options(fd_rel=1e-5))
        big = np.abs(Jc) > 1e-6 * np.abs(Jc).max(axis=1, keepdims=True)
        rel = np.abs(Jc - Jf)[big] / np.abs(Jc)[big]
        assert np.quantile(rel, 0.99) < 1e-5


def test_jacobian_element_rows():
    """sum_k a_ek/W_k dF_k/dY_j = a_ej/W_j and sum_k a_ek/W_k dF_k/dT = 0."""
    _, mech, _ = workload("k53_b4096")
    inlet = inlet_for(mech, seed=9, tau=2e-3)
    S = O.GasSystem(mech, inlet)
    for x in random_states(mech, 3, seed=10, y_small=True):
        J = O.jacobian_cs(S, x)
        lhs = (mech.comp / mech.W[:, None]).T @ J[:-1]          # (E, n)
        rhs = np.zeros_like(lhs)
        rhs[:, :-1] = (mech.comp / mech.W[:, None]).T
        scale = (np.abs(mech.comp) / mech.W[:, None]).T @ np.abs(J[:-1]) + 1e-300
        assert np.all(np.abs(lhs - rhs) <= 1e-12 * scale)


# ------------------------------------------------------------------ whole root
def test_tau_to_zero_gives_inlet():
    _, mech, batch = workload("k10_b64")
    for b in range(4):
        inlet = O.inlet_of(batch, b)
        inlet.tau = 1e-20                  # tau k_f << 1e-9 for every reaction
        r = O.solve_reactor(mech, inlet, np.r_[batch.Y0[b], batch.T0[b]])
        assert r.status == O.CONVERGED
        np.testing.assert_allclose(r.x[:-1], inlet.Y_in, atol=1e-10)
        np.testing.assert_allclose(r.x[-1], inlet.T_in, rtol=1e-9)


def test_tau_to_infinity_is_gibbs_equilibrium():
    """tau -> infinity at fixed T and P: the root is chemical equilibrium. Checked
    against Eqs. (8)-(9) (every reaction at K_c) and, independently of them, against
    the Gibbs-minimum condition: g_k/RT + ln(x_k P/P_atm) is a combination of the
    element rows (the golden reactions span every element-preserving change). The
    distance from equilibrium falls as 1/tau (1e-5 at tau = 1 s here)."""
    mech = golden("h2o2_equilibrium.psrmech")
    assert np.linalg.matrix_rank(mech.nu) == mech.K - 1 - np.linalg.matrix_rank(mech.comp[1:])
    T = 2600.0
    for Y_in in ([0.7, 0.03, 0.27, 0, 0, 0, 0], [0.6, 0.02, 0.3, 0, 0, 0, 0.08]):
        Y_in = np.array(Y_in, dtype=float)
        inlet = O.Inlet(Y_in, 500.0, 100.0, synth.ONE_ATM, T_spec=T)
        r = O.solve_reactor(mech, inlet, np.r_[Y_in, T], energy="fixed")
        assert r.status == O.CONVERGED
        Y = r.x[:-1]
        _, rho, C = O.mixture_state(mech, Y[None], np.array([T]), inlet.P)
        lnKc = np.log(O.equilibrium_constants(mech, np.array([T]))[0])
        for i in range(mech.I):
            lnQ = np.sum(np.log(C[0][mech.prod[i]])) - np.sum(np.log(C[0][mech.reac[i]]))
            assert abs(lnQ - lnKc[i]) <= 1e-6
        _, h_RT, s_R = O.species_thermo(mech, np.array([T]))
        n = Y / mech.W
        x = n / n.sum()
        mu = h_RT[0] - s_R[0] + np.log(x) + math.log(inlet.P / O.P_ATM)
        lam, *_ = np.linalg.lstsq(mech.comp, mu, rcond=None)
        assert np.max(np.abs(mech.comp @ lam - mu)) <= 1e-6


def test_element_conservation_at_roots():
    _, mech, batch = workload("k10_b64")
    res = O.solve_batch(mech, batch, indices=range(10))
    conv = res["status"] == O.CONVERGED
    assert conv.sum() >= 5
    dY = res["Y"][conv] - batch.Y_in[:10][conv]
    elem = (dY / mech.W) @ mech.comp
    assert np.max(np.abs(elem)) <= 1e-12
    assert np.max(res["fnorm"][conv]) <= 1e-8


def test_newton_finds_only_true_roots_adiabatic_s_curve():
    """Brute force: scan T, solve the (linear in Y_A) species balance by bisection
    on the oracle residual, and bracket sign changes of the energy row -> all roots.
    Newton from many guesses must land on one of them, and all three are reachable."""
    mech = golden("adiabatic_isomer.psrmech")
    Y_in = np.array([0.8, 0.2, 0.0])
    inlet = O.Inlet(Y_in, 400.0, 2e-2, synth.ONE_ATM)
    S = O.GasSystem(mech, inlet)

    def state(T, yA):
        return np.array([Y_in[0], yA, Y_in[1] + Y_in[2] - yA, T])

    def yA_of(T):
        return brentq(lambda y: S.F(state(T, y))[0][1], -1e-12, 0.2 + 1e-12, xtol=1e-17, rtol=1e-15)

    def g(T):
        return S.F(state(T, yA_of(T)))[0][-1]

    Ts = np.linspace(400.0, 1800.0, 1401)
    gs = np.array([g(t) for t in Ts])
    roots = []
    for j in np.nonzero(np.sign(gs[:-1]) != np.sign(gs[1:]))[0]:
        Tr = brentq(g, Ts[j], Ts[j + 1], xtol=1e-12)
        roots.append(state(Tr, yA_of(Tr)))
    assert len(roots) == 3
    found = set()
    for T0 in (400.0, 700.0, 900.0, 1100.0, 1300.0, 1500.0, 1700.0, 2000.0):
        r = O.solve_reactor(mech, inlet, np.r_[Y_in, T0])
        if r.status != O.CONVERGED:
            continue
        d = [np.max(np.abs(r.x - rt) / np.r_[1, 1, 1, rt[-1]]) for rt in roots]
        assert min(d) <= 1e-9
        found.add(int(np.argmin(d)))
    assert {0, 2} <= found


# ------------------------------------------------------------------ Sec. 1: finite-difference Jacobian
@pytest.mark.parametrize("name,n", [("k10_b64", 16), ("k53_b4096", 3)])
def test_fd_jacobian_newton_reaches_the_same_roots(name, n):
    """Newton steered by the paper's central-difference Jacobian (Sec. 1) converges to
    the roots the complex-step Jacobian reaches: J only steers the iteration, the root is
    fixed by the residual."""
    _, mech, batch = workload(name)
    cs = O.solve_batch(mech, batch, indices=range(n))
    fd = O.solve_batch(mech, batch, O.Options(jacobian="fd"), indices=range(n))
    assert np.all(cs["status"] == O.CONVERGED) and np.all(fd["status"] == O.CONVERGED)
    assert np.all(np.abs(fd["T"] - cs["T"]) <= 1e-8)
    big = cs["Y"] > 1e-10
    rel = np.abs(fd["Y"] - cs["Y"])[big] / cs["Y"][big]
    assert np.max(rel) <= 1e-6
    with pytest.raises(ValueError):
        O.solve_batch(mech, batch, O.Options(jacobian="exact"), indices=range(1))
