"""Pins of the MOMIC soot part of the oracle: exactness of the log-moment interpolation
for a lognormal population, monodisperse closed forms of free-molecular coagulation and
of surface growth, G_1 = 0, the nucleation-only steady state, and carbon conservation
(gas + soot) at the coupled roots."""
import math

import numpy as np
import pytest

from oracle import momic_oracle as S
from oracle import psr_oracle as O
from paper_2005_11468_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _soot_mech():
    spec = synth.workload_mechanism("k53soot_b16384")
    return spec, O.Mechanism(synth.mechanism_text(spec)), synth.workload_batch("k53soot_b16384", spec)


def test_lognormal_interpolation_is_exact():
    """log mu_r of a lognormal is quadratic in r, so both interpolants reproduce
    mu_p = exp(p a + p^2 s^2 / 2) for every p."""
    a, s2 = 4.0, 0.6
    r = np.arange(6)
    logmu = (r * a + r * r * s2 / 2) / math.log(10)
    for p in (-0.5, -1 / 6, 1 / 6, 2 / 3, 1.5, 3.7, 5.0, 7 + 1 / 6):
        np.testing.assert_allclose(S.fractional_moment(logmu, p), math.exp(p * a + p * p * s2 / 2), rtol=1e-11)


def test_monodisperse_coagulation_and_growth_closed_forms():
    """All particles of m carbons: mu_r = m^r. Free-molecular coagulation of equal
    spheres: dN/dt = -beta N^2 / 2 with beta = K_f (2/m)^(1/2) (2 m^(1/3))^2; growth adds
    2 carbons per step at k_g [P] chi_alpha pi d_C^2 m^(2/3) steps per particle."""
    spec, mech, _ = _soot_mech()
    sp = S.Soot(mech.soot)
    m, N, T, CP = 500.0, 3e10, 1700.0, 2e-7
    M = N * m ** np.arange(6.0)
    R, W, G, s = S.soot_sources(sp, M[None], np.array([CP]), np.array([T]))
    Kf = sp.eps * (3 * S.M_C / (4 * math.pi * sp.rho_s)) ** (1 / 6) * (6 * S.K_B * T / sp.rho_s) ** 0.5
    beta = Kf * math.sqrt(2.0 / m) * (2 * m ** (1 / 3)) ** 2
    np.testing.assert_allclose(G[0, 0], -0.5 * beta * N * N, rtol=1e-10)
    assert G[0, 1] == 0.0
    kg = sp.grow_A * T ** sp.grow_beta * math.exp(-sp.grow_theta / T)
    steps = kg * CP * sp.chi_alpha * math.pi * sp.dC ** 2 * m ** (2 / 3)      # per particle per s
    np.testing.assert_allclose(W[0, 1], 2.0 * steps * N, rtol=1e-10)
    # W_r for a monodisperse population: N steps ((m + 2)^r - m^r), first order in the step
    for r in range(2, 6):
        exact = N * steps * ((m + 2) ** r - m ** r)
        np.testing.assert_allclose(W[0, r], exact, rtol=1e-10)


@pytest.mark.parametrize("m", [32.0, 500.0, 2.0e4])
def test_monodisperse_coagulation_higher_moments(m):
    """Equal particles of m carbons: each free-molecular collision takes two m-particles
    and makes one 2m-particle, at ½ β N² collisions per unit volume and time with
    β = K_f (2/m)^(1/2) (2 m^(1/3))^2. So dM_r/dt = ½ β N² ((2m)^r − 2 m^r)
    = ½ β N² m^r (2^r − 2) for every r: −½ β N² at r = 0, 0 at r = 1, and the
    binomial sums of G_2..G_5 must add up to 2^r − 2."""
    spec, mech, _ = _soot_mech()
    sp = S.Soot(mech.soot)
    N, T = 4e9, 1900.0
    M = N * m ** np.arange(6.0)
    _, _, G, _ = S.soot_sources(sp, M[None], np.array([1e-7]), np.array([T]))
    Kf = sp.eps * (3 * S.M_C / (4 * math.pi * sp.rho_s)) ** (1 / 6) * (6 * S.K_B * T / sp.rho_s) ** 0.5
    beta = Kf * math.sqrt(2.0 / m) * (2 * m ** (1 / 3)) ** 2
    for r in range(6):
        np.testing.assert_allclose(G[0, r], 0.5 * beta * N * N * m ** r * (2.0 ** r - 2.0), rtol=1e-10,
                                   atol=1e-12 * beta * N * N * m ** r)


def test_coagulation_conserves_carbon_and_reduces_number():
    spec, mech, _ = _soot_mech()
    sp = S.Soot(mech.soot)
    rng = np.random.Generator(np.random.PCG64(3))
    for _ in range(5):
        a, s2, N = rng.uniform(3, 7), rng.uniform(0.1, 1.0), 10 ** rng.uniform(8, 12)
        r = np.arange(6)
        M = N * np.exp(r * a + r * r * s2 / 2)
        _, _, G, _ = S.soot_sources(sp, M[None], np.array([1e-7]), np.array([1800.0]))
        assert G[0, 1] == 0.0 and G[0, 0] < 0 and np.all(G[0, 2:] > 0)


def test_nucleation_only_steady_state():
    """Growth and coagulation off, fixed T: M_r = M_r,in + tau J([P]) C_min^r at the root."""
    spec, mech, batch = _soot_mech()
    mech.soot = dict(mech.soot, grow_A=0.0, coag_eps=0.0)
    sp = S.Soot(mech.soot)
    for b in (3, 6):
        inlet = O.inlet_of(batch, b, "fixed")
        inlet.T_spec = 1600.0
        r, M = S.solve_soot_reactor(mech, inlet, batch.Y0[b], 1600.0, batch.M_in[b], energy="fixed")
        assert r.status == O.CONVERGED
        _, rho, C = O.mixture_state(mech, r.x[None, :mech.K], np.array([1600.0]), inlet.P)
        J = sp.nuc_A * math.exp(-sp.nuc_theta / 1600.0) * C[0, sp.P] * S.N_A
        np.testing.assert_allclose(M, batch.M_in[b] + inlet.tau * J * sp.cmin ** np.arange(6), rtol=1e-9)


def test_carbon_conservation_gas_plus_soot():
    """sum_k a_Ck (Y_k - Y_k,in)/W_k + (M_1 - M_1,in)/(rho N_A) = 0 at every root: the
    carbon that leaves the gas is the soot carbon flowing out."""
    spec, mech, batch = _soot_mech()
    iC = 0
    for b in (1, 3, 6):
        inlet = O.inlet_of(batch, b)
        r, M = S.solve_soot_reactor(mech, inlet, batch.Y0[b], batch.T0[b], batch.M_in[b])
        assert r.status == O.CONVERGED
        Y, T = r.x[:mech.K], r.x[mech.K]
        _, rho, _ = O.mixture_state(mech, Y[None], np.array([T]), inlet.P)
        gas = np.sum(mech.comp[:, iC] * (Y - inlet.Y_in) / mech.W)
        soot = (M[1] - batch.M_in[b][1]) / (rho[0] * S.N_A)
        scale = np.sum(mech.comp[:, iC] * (Y + inlet.Y_in) / mech.W)
        assert abs(gas + soot) <= 1e-12 * scale


def test_soot_jacobian_complex_step_vs_central_differences():
    spec, mech, batch = _soot_mech()
    inlet = O.inlet_of(batch, 3)
    sys_ = S.SootSystem(mech, inlet, batch.M_in[3])
    M = batch.M_in[3] + 1e10 * 80.0 ** np.arange(6)
    x = np.r_[batch.Y_in[3] * 0.9 + 0.1 / mech.K, 1500.0, np.log(M / sys_.soot.scale)]
    Jc = O.jacobian_cs(sys_, x)
    Jf = O.jacobian_fd(sys_, x, O.Options(fd_rel=1e-6))
    blk = Jc[mech.K + 1:]                   # soot rows
    rel = np.abs(blk - Jf[mech.K + 1:]) / (np.abs(blk).max(axis=1, keepdims=True) + 1e-300)
    assert np.max(rel) < 1e-5
