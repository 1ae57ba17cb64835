"""The oracle's pins catch plausible mistakes: each case below plants one mistake in the
oracle (on the CPU, by wrapping one of its functions for the duration of the test) and
checks that the pins named beside it fail. A mistake no pin caught would be a mistake
the oracle could carry into every parity comparison unseen.

The mistakes are the kinds the pins were chosen against: a dropped term or factor, a
wrong sign, a wrong operand, a missing pivot search.
"""
import math

import numpy as np
import pytest

from oracle import momic_oracle as S
from oracle import psr_oracle as O
from tests import test_oracle_adjoint as adjoint_pins
from tests import test_oracle_momic as momic_pins
from tests import test_oracle_pins as pins

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

_orig = {name: getattr(O, name) for name in (
    "equilibrium_constants", "forward_rate_constants", "rates_of_progress", "third_body_concentrations",
    "troe_broadening", "net_production_rates", "species_thermo", "mixture_state", "gas_residual", "lu_factor",
    "sensitivities")}
_orig_soot = {name: getattr(S, name) for name in ("fractional_moment", "soot_sources", "f_half", "grid_f")}


# ---------------------------------------------------------------- planted mistakes
def kc_without_pressure_factor(mech, T):
    """K_c = K_p: the (P_atm / RT)^(sum nu) factor of Eq. (8) dropped."""
    T = np.asarray(T)
    return _orig["equilibrium_constants"](mech, T) / (O.P_ATM / (O.R_U * T[:, None])) ** mech.nu.sum(0)[None]


def kc_enthalpy_sign(mech, T):
    """K_p = exp(sum nu S/R + sum nu H/RT): the sign of the enthalpy term of Eq. (9) flipped."""
    _, h_RT, _ = _orig["species_thermo"](mech, np.asarray(T))
    return _orig["equilibrium_constants"](mech, T) * np.exp(2.0 * (h_RT @ mech.nu))


def kf_activation_sign(mech, T):
    """k_f = A T^beta exp(+E/RT): the sign of the exponent of Eq. (6) flipped."""
    T = np.asarray(T)
    return _orig["forward_rate_constants"](mech, T) * np.exp(2.0 * mech.theta[None] / T[:, None])


def q_without_third_body(mech, T, C, lnmult=None):
    """Third-body rows not multiplied by [M]."""
    q = _orig["rates_of_progress"](mech, T, C, lnmult)
    M = _orig["third_body_concentrations"](mech, C)
    return np.where(mech.is_tb[None], q / M, q)


def q_falloff_times_m(mech, T, C, lnmult=None):
    """Falloff rows multiplied by [M] as well (the Lindemann form already holds it)."""
    q = _orig["rates_of_progress"](mech, T, C, lnmult)
    M = _orig["third_body_concentrations"](mech, C)
    return np.where(mech.is_troe[None], q * M, q)


def m_without_efficiencies(mech, C):
    """[M] = sum_k [X_k]: the collision efficiencies ignored."""
    return np.repeat(C.sum(axis=1, keepdims=True), mech.I, axis=1)


def troe_without_broadening(mech, T, Pr):
    """F = 1: the Troe broadening factor left out of the falloff rate."""
    return np.ones_like(np.asarray(Pr))


def _troe_with_t2_term(mech, T, Pr, t2_term):
    """The Troe form of the oracle's docstring with the T** term of F_cent replaced by
    t2_term(T, T2) (the planted mistakes below differ only there)."""
    T = np.asarray(T)[:, None]
    alpha, T3, T1, T2 = (mech.troe[None, :, j] for j in range(4))
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        Fcent = (1 - alpha) * np.exp(-T / T3) + alpha * np.exp(-T / T1) + t2_term(T, T2)
        lf = np.log10(Fcent)
        c = -0.4 - 0.67 * lf
        n = 0.75 - 1.27 * lf
        u = np.log10(Pr) + c
        f1 = u / (n - 0.14 * u)
        return 10.0 ** (lf / (1 + f1 * f1))


def troe_t2_inverted(mech, T, Pr):
    """The T** term of F_cent written exp(-T/T**) instead of exp(-T**/T)."""
    return _troe_with_t2_term(mech, T, Pr, lambda T_, T2: np.where(T2 != 0, np.exp(-T_ / T2), 0.0))


def troe_t2_dropped(mech, T, Pr):
    """F_cent without its T** term (the three-parameter form for every row)."""
    return _troe_with_t2_term(mech, T, Pr, lambda T_, T2: 0.0 * T2)


def wdot_sign(mech, q):
    """wdot = sum nu' q (reactant minus product): the sign of nu in Eq. (4) flipped."""
    return -_orig["net_production_rates"](mech, q)


def wdot_reactants_only(mech, q):
    """wdot = -sum nu' q: the products' coefficients nu'' left out of nu in Eq. (4)."""
    return -(q @ mech.nu_f.T)


def entropy_without_log_term(mech, T):
    """S/R without the a1 ln T term of the NASA-7 entropy."""
    cp, h, s = _orig["species_thermo"](mech, T)
    T = np.asarray(T)[:, None]
    a1 = np.where((np.real(T) < mech.t_mid[None, :]), mech.nasa_low[None, :, 0], mech.nasa_high[None, :, 0])
    return cp, h, s - a1 * np.log(T)


def density_without_mean_weight(mech, Y, T, P):
    """rho = P / (R T): the mean molecular weight left out of the ideal-gas density."""
    Wbar, rho, C = _orig["mixture_state"](mech, Y, T, P)
    return Wbar, rho / Wbar, C / Wbar[:, None]


def energy_without_inlet_enthalpy(mech, X, inlet, energy="adiabatic", lnmult=None):
    """Energy row without the inlet term sum_k Y_k,in (h_k(T) - h_k(T_in)) of Eq. (3)."""
    F = _orig["gas_residual"](mech, X, inlet, energy, lnmult)
    if energy == "fixed":
        return F
    X = np.atleast_2d(X)
    Y, T = X[:, :mech.K], X[:, mech.K]
    cp_R, h_RT, _ = _orig["species_thermo"](mech, T)
    _, h_RT_in, _ = _orig["species_thermo"](mech, np.array([inlet.T_in]))
    h = h_RT * O.R_U * T[:, None] / mech.W[None]
    h_in = h_RT_in * O.R_U * inlet.T_in / mech.W[None]
    cp = np.sum(Y * cp_R * O.R_U / mech.W[None], axis=1)
    F = F.copy()
    F[:, mech.K] -= np.sum(inlet.Y_in[None] * (h - h_in), axis=1) / (cp * T)
    return F


def lu_without_pivoting(A):
    """Doolittle LU with no row interchanges."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    for k in range(n):
        if A[k, k] == 0 or not np.isfinite(A[k, k]):
            return A, np.arange(n), False
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    return A, np.arange(n), True


def moment_interpolation_linear(logmu, p):
    """log mu_p interpolated linearly between the neighbouring integer moments (and
    extrapolated linearly from r = 0, 1 below zero) instead of by the Lagrange polynomials."""
    lo = int(min(max(math.floor(p), 0), 4))
    t = p - lo
    return 10.0 ** ((1 - t) * logmu[..., lo] + t * logmu[..., lo + 1])


def coagulation_sign(soot, M, CP, T):
    """Coagulation sources with the wrong sign (G_0 > 0: coagulation creating particles)."""
    R, W, G, s = _orig_soot["soot_sources"](soot, M, CP, T)
    return R, W, -G, s


def soot_without_gas_sink(soot, M, CP, T):
    """Nucleation and growth take no precursor out of the gas."""
    R, W, G, s = _orig_soot["soot_sources"](soot, M, CP, T)
    return R, W, G, 0.0 * s


def nucleation_without_size(soot, M, CP, T):
    """Nuclei added to every moment as C_min, not C_min^r."""
    R, W, G, s = _orig_soot["soot_sources"](soot, M, CP, T)
    return np.broadcast_to(R[..., 1:2], R.shape).copy(), W, G, s


def growth_per_particle(soot, M, CP, T):
    """Surface growth per particle: the M_0 factor of the total surface left out."""
    R, W, G, s = _orig_soot["soot_sources"](soot, M, CP, T)
    return R, W / np.asarray(M)[..., :1], G, s


def coagulation_grid_linear(logmu, x, y):
    """f(1/2) interpolated in f(l) rather than in log f(l)."""
    w = S.lagrange_weights(range(4), 0.5)
    return sum(w[l] * _orig_soot["grid_f"](logmu, l, x, y) for l in range(4))


def coagulation_without_binomial(soot, M, CP, T):
    """G_r = ½ K_f M_0² sum_k f(1/2)_{k,r-k}: the binomial weights C(r, k) of the
    coagulation sums dropped (G_0 and G_1 unchanged)."""
    R, W, G, s = _orig_soot["soot_sources"](soot, M, CP, T)
    M = np.asarray(M)
    logmu = np.log10(M / M[..., :1])
    Kf = soot.eps * (3 * S.M_C / (4 * math.pi * soot.rho_s)) ** (1 / 6) * (6 * S.K_B * np.asarray(T) / soot.rho_s) ** 0.5
    beta = Kf * M[..., 0] ** 2
    G = np.array(G, copy=True)
    for rr in range(2, S.NMOM):
        G[..., rr] = 0.5 * beta * sum(S.f_half(logmu, k, rr - k) for k in range(1, rr))
    return R, W, G, s


def sensitivity_sign(mech, inlet, x, energy="adiabatic", lnmult=None):
    """S = +J^-1 dF/dp: the minus sign of the implicit-function theorem dropped."""
    return -_orig["sensitivities"](mech, inlet, x, energy, lnmult)


# ---------------------------------------------------------------- the pins that must fail
def _call(name, *args, module=pins):
    return lambda: getattr(module, name)(*args)


def _momic(name):
    return _call(name, module=momic_pins)


CASES = [
    ("equilibrium_constants", kc_without_pressure_factor,
     [_call("test_dimerisation_closed_form"), _call("test_van_t_hoff")]),
    ("equilibrium_constants", kc_enthalpy_sign,
     [_call("test_isomerisation_closed_form"), _call("test_van_t_hoff"),
      _call("test_tau_to_infinity_is_gibbs_equilibrium")]),
    ("forward_rate_constants", kf_activation_sign, [_call("test_arrhenius_special_cases")]),
    ("rates_of_progress", q_without_third_body, [_call("test_third_body_isomerisation_closed_form")]),
    ("rates_of_progress", q_falloff_times_m, [_call("test_falloff_isomerisation_at_the_troe_centre")]),
    ("third_body_concentrations", m_without_efficiencies,
     [_call("test_third_body_isomerisation_closed_form"), _call("test_falloff_isomerisation_at_the_troe_centre")]),
    ("troe_broadening", troe_without_broadening,
     [_call("test_falloff_isomerisation_at_the_troe_centre"), _call("test_troe_centre_and_limits")]),
    ("troe_broadening", troe_t2_inverted,
     [_call("test_falloff_isomerisation_t2_term"), _call("test_troe_t2_term_alone", 1500.0)]),
    ("troe_broadening", troe_t2_dropped,
     [_call("test_falloff_isomerisation_t2_term"), _call("test_troe_t2_term_alone", 800.0)]),
    ("net_production_rates", wdot_sign, [_call("test_isomerisation_closed_form"),
                                         _call("test_dimerisation_closed_form")]),
    ("net_production_rates", wdot_reactants_only, [_call("test_wdot_conserves_mass_and_elements", "k10_b64")]),
    ("species_thermo", entropy_without_log_term, [_call("test_nasa_enthalpy_and_entropy_derivatives", False)]),
    ("mixture_state", density_without_mean_weight, [_call("test_dimerisation_closed_form")]),
    ("gas_residual", energy_without_inlet_enthalpy, [_call("test_residual_identities", "k10_b64"),
                                                     _call("test_newton_finds_only_true_roots_adiabatic_s_curve")]),
    ("lu_factor", lu_without_pivoting, [_call("test_lu_matches_lapack", 11)]),
    ("sensitivities", sensitivity_sign,
     [_call("test_isomerisation_sensitivity_closed_form", module=adjoint_pins),
      _call("test_sensitivities_match_finite_differences_of_resolved_roots", module=adjoint_pins)]),
]
# MOMIC soot (wrapped in oracle/momic_oracle.py)
SOOT_CASES = [
    ("fractional_moment", moment_interpolation_linear, [_momic("test_lognormal_interpolation_is_exact")]),
    ("soot_sources", coagulation_sign, [_momic("test_monodisperse_coagulation_and_growth_closed_forms"),
                                        _momic("test_coagulation_conserves_carbon_and_reduces_number")]),
    ("soot_sources", soot_without_gas_sink, [_momic("test_carbon_conservation_gas_plus_soot")]),
    ("soot_sources", nucleation_without_size, [_momic("test_nucleation_only_steady_state")]),
    ("soot_sources", growth_per_particle, [_momic("test_monodisperse_coagulation_and_growth_closed_forms")]),
    ("f_half", coagulation_grid_linear, [_momic("test_monodisperse_coagulation_and_growth_closed_forms")]),
    ("soot_sources", coagulation_without_binomial,
     [_call("test_monodisperse_coagulation_higher_moments", 500.0, module=momic_pins)]),
]


ALL = [(O, *c) for c in CASES] + [(S, *c) for c in SOOT_CASES]


# The named pins pass on the oracle as it is (their own modules run them unmodified);
# each must fail once the mistake is planted.
@pytest.mark.parametrize("module,target,mistake,catchers", ALL, ids=[c[2].__name__ for c in ALL])
def test_pins_catch_the_planted_mistake(monkeypatch, module, target, mistake, catchers):
    monkeypatch.setattr(module, target, mistake)
    for pin in catchers:
        with pytest.raises(AssertionError):
            pin()
