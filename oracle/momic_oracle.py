"""MOMIC soot moments coupled to the steady PSR, plain float64 (TEST INFRASTRUCTURE ONLY).

The paper couples its PSR solver to the Method of Moments with Interpolative Closure
(MOMIC) for soot (Abstract, Sec. 1, Sec. 5, Sec. 7) but prints none of its equations;
this module writes the model out from the published method (Frenklach's moment method):

* moments M_r = sum_i m_i^r N_i, r = 0..5 (m in carbon atoms, N per cm^3); reduced
  moments mu_r = M_r / M_0; fractional moments mu_p from Lagrange interpolation of
  log10 mu_r over r = 0..5 (p >= 0) or quadratic extrapolation over r = 0, 1, 2 (p < 0);
* nucleation from the precursor P (C2H2-like): J = A_n exp(-theta_n/T) [P] N_A nuclei of
  C_min carbon atoms, R_r = J C_min^r;
* surface growth by C2H2 addition (2 carbon atoms per step) to active sites:
  W_r = k_g(T) [P] chi_alpha pi d_C^2 M_0 sum_{l<r} C(r, l) mu_{l+2/3} 2^(r-l),
  k_g = A_g T^beta_g exp(-theta_g/T), d_C the diameter of a one-carbon sphere;
* free-molecular coagulation: G_0 = -K_f M_0^2 f(1/2)_{0,0} / 2, G_1 = 0,
  G_r = K_f M_0^2 / 2 sum_{k=1}^{r-1} C(r, k) f(1/2)_{k,r-k}, with the grid functions
  f(l)_{x,y} = sum_k C(l, k) [mu_{k+x+1/6} mu_{l-k+y-1/2} + 2 mu_{k+x-1/6} mu_{l-k+y-1/6}
  + mu_{k+x-1/2} mu_{l-k+y+1/6}] for l = 0..3, f(1/2) by Lagrange interpolation of their
  log10 at l = 1/2, and K_f = eps (3 m_C / (4 pi rho_s))^(1/6) (6 k_B T / rho_s)^(1/2);
* gas coupling: each nucleus and each growth step turn C2H2 into two soot carbons and H2:
  wdot_P -= s, wdot_H2 += s with s = (J C_min + W_1) / (2 N_A);
* steady moment balances F_r = (M_r - M_r,in - tau (R_r + W_r + G_r)) / (M_r + s_r) with
  unknowns zeta_r = ln(M_r / s_r), s_r = M0_floor C_min^r.
"""
from __future__ import annotations

import math

import numpy as np

from oracle import psr_oracle as O

N_A = 6.02214076e23       # 1/mol
K_B = 1.380649e-16        # erg/K
M_C = 12.011 / N_A        # g per carbon atom
NMOM = 6
ZETA_STEP = 3.0           # largest change of a log moment ln(M_r/s_r) in one Newton step


class Soot:
    """Soot constants of a mechanism's `soot` record."""

    def __init__(self, d: dict):
        self.P = int(d["precursor"])
        self.H2 = int(d["h2"])
        self.nuc_A, self.nuc_theta = d["nuc_A"], d["nuc_theta"]
        self.cmin = d["cmin"]
        self.grow_A, self.grow_beta, self.grow_theta = d["grow_A"], d["grow_beta"], d["grow_theta"]
        self.chi_alpha = d["chi_alpha"]
        self.rho_s = d["rho_s"]
        self.eps = d["coag_eps"]
        self.m0_floor = d["m0_floor"]
        self.scale = self.m0_floor * self.cmin ** np.arange(NMOM)          # s_r
        self.dC = (6.0 * M_C / (math.pi * self.rho_s)) ** (1.0 / 3.0)


def lagrange_weights(nodes, p):
    """Weights l_j(p) of the Lagrange polynomial through `nodes` evaluated at p."""
    w = []
    for j, xj in enumerate(nodes):
        v = 1.0
        for k, xk in enumerate(nodes):
            if k != j:
                v *= (p - xk) / (xj - xk)
        w.append(v)
    return np.array(w)


def fractional_moment(logmu, p):
    """mu_p from log10 mu_r (r = 0..5, last axis): interpolation over all six for p >= 0,
    quadratic extrapolation over r = 0, 1, 2 for p < 0."""
    if p >= 0:
        w = lagrange_weights(range(NMOM), p)
        return 10.0 ** (logmu @ w)
    w = lagrange_weights(range(3), p)
    return 10.0 ** (logmu[..., :3] @ w)


def grid_f(logmu, l, x, y):
    """f(l)_{x,y} of free-molecular coagulation."""
    tot = 0.0
    for k in range(l + 1):
        c = math.comb(l, k)
        a1 = fractional_moment(logmu, k + x + 1 / 6) * fractional_moment(logmu, l - k + y - 1 / 2)
        a2 = fractional_moment(logmu, k + x - 1 / 6) * fractional_moment(logmu, l - k + y - 1 / 6)
        a3 = fractional_moment(logmu, k + x - 1 / 2) * fractional_moment(logmu, l - k + y + 1 / 6)
        tot = tot + c * (a1 + 2 * a2 + a3)
    return tot


def f_half(logmu, x, y):
    """f(1/2)_{x,y}: Lagrange interpolation of log10 f(l) over l = 0..3 at l = 1/2."""
    w = lagrange_weights(range(4), 0.5)
    lf = sum(w[l] * np.log10(grid_f(logmu, l, x, y)) for l in range(4))
    return 10.0 ** lf


def soot_sources(soot: Soot, M, CP, T):
    """Moment sources (R, W, G each (..., 6)) and the precursor sink s (mol/cm^3/s) for
    moments M (..., 6), precursor concentration CP (mol/cm^3) and temperature T."""
    M = np.asarray(M)
    logmu = np.log10(M / M[..., :1])
    r = np.arange(NMOM)
    J = soot.nuc_A * np.exp(-soot.nuc_theta / T) * CP * N_A
    R = J[..., None] * soot.cmin ** r
    kg = soot.grow_A * T ** soot.grow_beta * np.exp(-soot.grow_theta / T)
    pref = kg * CP * soot.chi_alpha * math.pi * soot.dC ** 2 * M[..., 0]
    Wl = []
    for rr in range(NMOM):
        acc = 0.0 * pref
        for l in range(rr):
            acc = acc + math.comb(rr, l) * fractional_moment(logmu, l + 2 / 3) * 2.0 ** (rr - l)
        Wl.append(pref * acc)
    W = np.stack(Wl, axis=-1)
    Kf = soot.eps * (3 * M_C / (4 * math.pi * soot.rho_s)) ** (1 / 6) * (6 * K_B * T / soot.rho_s) ** 0.5
    beta = Kf * M[..., 0] ** 2
    Gl = [-0.5 * beta * f_half(logmu, 0, 0), 0.0 * beta]
    for rr in range(2, NMOM):
        acc = 0.0 * beta
        for k in range(1, rr):
            acc = acc + math.comb(rr, k) * f_half(logmu, k, rr - k)
        Gl.append(0.5 * beta * acc)
    G = np.stack(Gl, axis=-1)
    s = (J * soot.cmin + W[..., 1]) / (2 * N_A)
    return R, W, G, s


class SootSystem(O.GasSystem):
    """Gas + soot unknowns x = (Y_1..Y_K, T, zeta_0..zeta_5), zeta_r = ln(M_r / s_r)."""

    def __init__(self, mech, inlet, M_in, energy="adiabatic", lnmult=None):
        super().__init__(mech, inlet, energy, lnmult)
        self.soot = Soot(mech.soot)
        self.M_in = np.asarray(M_in, dtype=np.float64)
        self.n = mech.K + 1 + NMOM

    def F(self, X):
        mech, sp = self.mech, self.soot
        X = np.atleast_2d(O._arr(X))
        K = mech.K
        Y, T, z = X[:, :K], X[:, K], X[:, K + 1:]
        M = np.exp(z) * sp.scale
        _, rho, C = O.mixture_state(mech, Y, T, self.inlet.P)
        q = O.rates_of_progress(mech, T, C, self.lnmult)
        wdot = O.net_production_rates(mech, q)
        R, W, G, s = soot_sources(sp, M, C[:, sp.P], T)
        wdot = wdot.copy()
        wdot[:, sp.P] = wdot[:, sp.P] - s
        wdot[:, sp.H2] = wdot[:, sp.H2] + s
        out = np.empty_like(X)
        out[:, :K] = Y - self.inlet.Y_in[None] - self.inlet.tau * wdot * mech.W[None] / rho[:, None]
        if self.energy == "fixed":
            out[:, K] = T - self.inlet.T_spec
        else:
            cp_R, h_RT, _ = O.species_thermo(mech, T)
            _, h_RT_in, _ = O.species_thermo(mech, np.array([self.inlet.T_in]))
            h = h_RT * O.R_U * T[:, None] / mech.W[None]
            h_in = h_RT_in * O.R_U * self.inlet.T_in / mech.W[None]
            cp = np.sum(Y * cp_R * O.R_U / mech.W[None], axis=1)
            N = np.sum(self.inlet.Y_in[None] * (h - h_in), axis=1) \
                + self.inlet.tau / rho * np.sum(h * mech.W[None] * wdot, axis=1)
            out[:, K] = N / (cp * T)
        out[:, K + 1:] = (M - self.M_in[None] - self.inlet.tau * (R + W + G)) / (M + sp.scale[None])
        return out

    def fd_scale(self, x):
        s = super().fd_scale(x)
        return np.r_[s, np.ones(NMOM)]

    def step_tol(self, x, opts):
        t = super().step_tol(x[:self.K + 1], opts)
        return np.r_[t, np.full(NMOM, opts.step_rtol)]        # zeta: absolute in log space

    def ts_tol(self, x, opts):
        t = super().ts_tol(x[:self.K + 1], opts)
        return np.r_[t, np.full(NMOM, opts.ts_rtol)]

    def norm_weights(self, x):
        return np.r_[super().norm_weights(x[:self.K + 1]), np.ones(NMOM)]

    def max_in_bounds(self, x, dx, opts):
        """The gas bounds, and no log moment moving by more than ZETA_STEP in one step:
        larger moves (undamped pseudo-time steps at large dt) can leave a moment set outside
        the range where the interpolative closure is defined."""
        lam = super().max_in_bounds(x[:self.K + 1], dx[:self.K + 1], opts)
        dz = float(np.max(np.abs(dx[self.K + 1:])))
        return min(lam, ZETA_STEP / dz) if dz > ZETA_STEP else lam

    def in_bounds(self, x, opts):
        return super().in_bounds(x[:self.K + 1], opts)

    def transient_weights(self, x):
        return np.r_[super().transient_weights(x[:self.K + 1]), np.ones(NMOM)]


def initial_moments(mech, inlet, Y0, T0, M_in):
    """Nucleation-only steady moments at the initial gas state: M_r = M_r,in + tau J C_min^r."""
    sp = Soot(mech.soot)
    _, _, C = O.mixture_state(mech, np.asarray(Y0)[None], np.array([T0]), inlet.P)
    J = sp.nuc_A * math.exp(-sp.nuc_theta / T0) * C[0, sp.P] * N_A
    return np.asarray(M_in) + inlet.tau * J * sp.cmin ** np.arange(NMOM)


def solve_soot_reactor(mech, inlet, Y0, T0, M_in, M0=None, opts=O.Options(), energy="adiabatic", lnmult=None):
    """Gas + MOMIC PSR: x = (Y, T, zeta); returns (Result, M)."""
    S = SootSystem(mech, inlet, M_in, energy, lnmult)
    M0 = initial_moments(mech, inlet, Y0, T0, M_in) if M0 is None else np.asarray(M0)
    x0 = np.r_[Y0, T0, np.log(M0 / S.soot.scale)]
    r = O.solve_system(S, x0, opts)
    return r, np.exp(r.x[mech.K + 1:]) * S.soot.scale
