"""Plain FP64 CPU oracle for the batched steady-state perfectly-stirred-reactor solve.

TEST INFRASTRUCTURE ONLY. Nothing in the library imports this module; only the test
suite, the smoke check and the benchmark's CPU-baseline leg do. It shares no code
with the CUDA path: it parses the `.psrmech` text itself and evaluates every
formula below with numpy in float64, one reactor at a time, with no blocking,
fusion or reordering beyond what the equations state.

What it computes (Adhikari, Sayre & Chandy, "Towards using GPGPU units for
accelerating the batched perfectly stirred reactor (PSR) calculations"):

* Sec. 2, Eqs. (1)-(3): steady PSR balances. With d/dt = 0 and tau = rho V / mdot,
  Eq. (2) times tau gives the species residual
      F_k = Y_k - Y_k,in - tau wdot_k W_k / rho,
  and Eq. (3) (Q = 0, dP/dt = 0) times -tau gives
      N = sum_k Y_k,in (h_k(T) - h_k(T_in)) + (tau / rho) sum_k h_k(T) W_k wdot_k,
  which is reported as the dimensionless F_T = N / (c_p,mix T).
* Sec. 3, Eq. (4): wdot_k = sum_i nu_ki q_i, nu = nu'' - nu'.
* Eq. (5): q_i = k_f,i prod_k [X_k]^nu'_ki - k_r,i prod_k [X_k]^nu''_ki with [X_k]
  molar concentrations (the printed product bound is read as running over species).
* Eq. (6): k_f = A T^beta exp(-E / RT)  (E/R stored in kelvin).
* Eq. (7): k_r = k_f / K_c.  Eq. (8): K_c = K_p (P_atm / RT)^(sum_k nu_ki).
* Eq. (9): K_p = exp(sum_k nu_ki S_k/R - sum_k nu_ki H_k/RT).
* S and H from NASA 7-coefficient polynomials; third-body reactions multiply q_i
  by [M] = sum_k eps_ki [X_k]; falloff reactions replace k_f by the Lindemann form
  k_inf P_r / (1 + P_r) F with the Troe broadening F (Gilbert, Luther & Troe 1983),
  P_r = k_0 [M] / k_inf (the paper's mechanisms contain such reactions; it gives no
  formula for them).
* Sec. 1 and Sec. 3: Newton iteration on the error vector with a Jacobian obtained by
  finite differences, LU decomposition with partial pivoting and back-solving; the
  hybrid scheme of Sec. 3: when Newton fails, the estimate is conditioned by
  pseudo-transient time integration of Eqs. (2)-(3) and Newton is tried again.
* MOMIC soot moments (the paper couples the PSR to MOMIC, Abstract and Sec. 1):
  see `oracle/momic_oracle.py`.

Units are CGS: concentrations mol/cm^3, rho g/cm^3, P dyn/cm^2, energies erg.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

R_U = 8.314462618e7      # erg / (mol K)
P_ATM = 1.01325e6        # dyn / cm^2, standard-state pressure of Eq. (8)

# per-reactor status codes
CONVERGED, MAX_ITER, NONFINITE, SINGULAR, TS_EXHAUSTED = 0, 1, 2, 3, 4


# ----------------------------------------------------------------------------- mechanism
class Mechanism:
    """A parsed `.psrmech` mechanism (own parser; format described in the generator)."""

    def __init__(self, text: str):
        toks = []
        for line in text.splitlines():
            line = line.strip()
            if line and not line.startswith("#"):
                toks.append(line.split())
        it = iter(toks)
        head = next(it)
        if head[0] != "psrmech" or head[1] != "1":
            raise ValueError("not a psrmech v1 file")
        row = next(it)
        assert row[0] == "elements"
        E = int(row[1])
        self.elem_names, self.elem_w = [], np.zeros(E)
        for e in range(E):
            r = next(it)
            self.elem_names.append(r[0]); self.elem_w[e] = float(r[1])
        row = next(it)
        assert row[0] == "species"
        K = int(row[1])
        self.K = K
        self.names = []
        self.comp = np.zeros((K, E))
        self.t_low = np.zeros(K); self.t_mid = np.zeros(K); self.t_high = np.zeros(K)
        self.nasa_low = np.zeros((K, 7)); self.nasa_high = np.zeros((K, 7))
        for k in range(K):
            r = next(it)
            assert int(r[0]) == k
            self.names.append(r[1])
            self.comp[k] = [float(v) for v in r[2:2 + E]]
            vals = [float(v) for v in r[2 + E:]]
            self.t_low[k], self.t_mid[k], self.t_high[k] = vals[0:3]
            self.nasa_low[k] = vals[3:10]
            self.nasa_high[k] = vals[10:17]
        # molecular weights W_k = sum_e a_ek W_e
        self.W = self.comp @ self.elem_w
        row = next(it)
        assert row[0] == "reactions"
        I = int(row[1])
        self.I = I
        self.kind = []
        self.reac, self.prod = [], []
        self.A = np.zeros(I); self.beta = np.zeros(I); self.theta = np.zeros(I)
        self.low = np.zeros((I, 3)); self.troe = np.zeros((I, 4))
        self.eff = np.ones((I, K))
        for i in range(I):
            r = next(it)
            assert int(r[0]) == i
            self.kind.append(r[1])
            p = 2
            nr = int(r[p]); self.reac.append([int(v) for v in r[p + 1:p + 1 + nr]]); p += 1 + nr
            npr = int(r[p]); self.prod.append([int(v) for v in r[p + 1:p + 1 + npr]]); p += 1 + npr
            self.A[i], self.beta[i], self.theta[i] = float(r[p]), float(r[p + 1]), float(r[p + 2])
            p += 3
            while p < len(r):
                key = r[p]
                if key == "low":
                    self.low[i] = [float(v) for v in r[p + 1:p + 4]]; p += 4
                elif key == "troe":
                    self.troe[i] = [float(v) for v in r[p + 1:p + 5]]; p += 5
                elif key == "eff":
                    m = int(r[p + 1]); p += 2
                    for _ in range(m):
                        self.eff[i, int(r[p])] = float(r[p + 1]); p += 2
                else:
                    raise ValueError(f"unknown reaction field {key!r}")
        self.kind = np.array(self.kind)
        self.is_tb = self.kind == "tb"
        self.is_troe = self.kind == "troe"
        # stoichiometric coefficients nu' (reactants), nu'' (products), nu = nu'' - nu'
        self.nu_f = np.zeros((K, I)); self.nu_r = np.zeros((K, I))
        for i in range(I):
            for k in self.reac[i]:
                self.nu_f[k, i] += 1
            for k in self.prod[i]:
                self.nu_r[k, i] += 1
        self.nu = self.nu_r - self.nu_f
        self.soot = None
        for r in it:
            if r[0] == "soot":
                d = {}
                for j in range(1, len(r), 2):
                    d[r[j]] = float(r[j + 1])
                self.soot = d
            elif r[0] == "end":
                break

    @classmethod
    def from_file(cls, path):
        with open(path) as fh:
            return cls(fh.read())

    @property
    def n_gas(self):
        return self.K + 1


def _arr(x):
    """float64 array, or complex128 when x is complex (complex-step derivatives)."""
    x = np.asarray(x)
    return x.astype(np.complex128 if np.iscomplexobj(x) else np.float64, copy=False)


# ----------------------------------------------------------------------------- thermo
def species_thermo(mech: Mechanism, T):
    """NASA 7-coefficient polynomials at temperatures T (shape (m,)); returns
    c_p/R, H/(R T), S/R, each (m, K). The low-range set applies below T_mid."""
    T = _arr(T)[:, None]
    a = np.where((T.real < mech.t_mid[None, :])[..., None], mech.nasa_low[None], mech.nasa_high[None])
    a1, a2, a3, a4, a5, a6, a7 = (a[..., j] for j in range(7))
    cp_R = a1 + a2 * T + a3 * T**2 + a4 * T**3 + a5 * T**4
    h_RT = a1 + a2 * T / 2 + a3 * T**2 / 3 + a4 * T**3 / 4 + a5 * T**4 / 5 + a6 / T
    s_R = a1 * np.log(T) + a2 * T + a3 * T**2 / 2 + a4 * T**3 / 3 + a5 * T**4 / 4 + a7
    return cp_R, h_RT, s_R


def mixture_state(mech: Mechanism, Y, T, P):
    """Mean molecular weight, density (ideal gas) and molar concentrations [X_k]."""
    Wbar = 1.0 / np.sum(Y / mech.W[None, :], axis=1)
    rho = P * Wbar / (R_U * T)
    C = rho[:, None] * Y / mech.W[None, :]
    return Wbar, rho, C


# ----------------------------------------------------------------------------- rates
def forward_rate_constants(mech: Mechanism, T):
    """Eq. (6): k_f = A T^beta exp(-E/RT), (m, I)."""
    T = _arr(T)[:, None]
    return mech.A[None] * T ** mech.beta[None] * np.exp(-mech.theta[None] / T)


def equilibrium_constants(mech: Mechanism, T):
    """Eqs. (8)-(9): K_p = exp(sum nu S/R - sum nu H/RT); K_c = K_p (P_atm/RT)^(sum nu)."""
    T = _arr(T)
    _, h_RT, s_R = species_thermo(mech, T)
    Kp = np.exp(s_R @ mech.nu - h_RT @ mech.nu)
    dnu = mech.nu.sum(axis=0)
    return Kp * (P_ATM / (R_U * T[:, None])) ** dnu[None]


def third_body_concentrations(mech: Mechanism, C):
    """[M]_i = sum_k eps_ki [X_k] for every reaction (used by tb and falloff rows)."""
    return C @ mech.eff.T


def troe_broadening(mech: Mechanism, T, Pr):
    """Troe falloff broadening factor F(T, P_r) (Gilbert, Luther & Troe 1983):
    F_cent = (1 - alpha) exp(-T/T3) + alpha exp(-T/T1) + exp(-T2/T) (last term only
    when T2 != 0); c = -0.4 - 0.67 log10 F_cent; n = 0.75 - 1.27 log10 F_cent;
    f1 = (log10 P_r + c) / (n - 0.14 (log10 P_r + c)); log10 F = log10 F_cent / (1 + f1^2).
    T: (m,), Pr: (m, I); returns (m, I) (rows of non-falloff reactions are meaningless)."""
    T = _arr(T)[:, None]
    alpha, T3, T1, T2 = (mech.troe[None, :, j] for j in range(4))
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        Fcent = (1 - alpha) * np.exp(-T / T3) + alpha * np.exp(-T / T1) \
            + np.where(T2 != 0, np.exp(-T2 / T), 0.0)
        lf = np.log10(Fcent)
        c = -0.4 - 0.67 * lf
        n = 0.75 - 1.27 * lf
        u = np.log10(Pr) + c
        f1 = u / (n - 0.14 * u)
        return 10.0 ** (lf / (1 + f1 * f1))


def rates_of_progress(mech: Mechanism, T, C, lnmult=None):
    """Eq. (5) with the third-body and falloff forms. T (m,), C (m, K) -> q (m, I).
    lnmult (I,) or (m, I), optional: ln of a multiplier applied to each q_i (the
    parameter whose sensitivities the adjoint computes)."""
    T = _arr(T)
    m = len(T)
    kf = forward_rate_constants(mech, T)
    Kc = equilibrium_constants(mech, T)
    M = third_body_concentrations(mech, C)
    if mech.is_troe.any():
        Tc = T[:, None]
        k0 = mech.low[None, :, 0] * Tc ** mech.low[None, :, 1] * np.exp(-mech.low[None, :, 2] / Tc)
        with np.errstate(divide="ignore", invalid="ignore"):
            Pr = k0 * M / kf
        F = troe_broadening(mech, T, Pr)
        kf = np.where(mech.is_troe[None], kf * Pr / (1 + Pr) * F, kf)
    kr = kf / Kc                                            # Eq. (7)
    Cx = np.concatenate([C, np.ones((m, 1))], axis=1)        # index K = "no species" -> 1
    fwd = np.ones((m, mech.I), dtype=Cx.dtype); rev = np.ones((m, mech.I), dtype=Cx.dtype)
    for i in range(mech.I):
        for k in mech.reac[i]:
            fwd[:, i] *= Cx[:, k]
        for k in mech.prod[i]:
            rev[:, i] *= Cx[:, k]
    q = kf * fwd - kr * rev
    q = np.where(mech.is_tb[None], q * M, q)
    if lnmult is not None:
        q = q * np.exp(_arr(lnmult))
    return q


def net_production_rates(mech: Mechanism, q):
    """Eq. (4): wdot_k = sum_i nu_ki q_i. q (m, I) -> (m, K)."""
    return q @ mech.nu.T


# ----------------------------------------------------------------------------- residual
@dataclasses.dataclass
class Inlet:
    """One reactor's inlet and operating point."""
    Y_in: np.ndarray
    T_in: float
    tau: float
    P: float
    T_spec: float = 0.0      # reactor temperature in the fixed-temperature mode


def gas_residual(mech: Mechanism, X, inlet: Inlet, energy="adiabatic", lnmult=None):
    """Steady residual of Eqs. (2)-(3) at states X (m, K+1) = (Y_1..Y_K, T)."""
    X = np.atleast_2d(_arr(X))
    Y, T = X[:, :mech.K], X[:, mech.K]
    _, rho, C = mixture_state(mech, Y, T, inlet.P)
    q = rates_of_progress(mech, T, C, lnmult)
    wdot = net_production_rates(mech, q)
    F = np.empty_like(X)
    F[:, :mech.K] = Y - inlet.Y_in[None] - inlet.tau * wdot * mech.W[None] / rho[:, None]
    if energy == "fixed":
        F[:, mech.K] = T - inlet.T_spec
    else:
        cp_R, h_RT, _ = species_thermo(mech, T)
        _, h_RT_in, _ = species_thermo(mech, np.array([inlet.T_in]))
        h = h_RT * R_U * T[:, None] / mech.W[None]            # erg/g
        h_in = h_RT_in * R_U * inlet.T_in / mech.W[None]      # erg/g at T_in
        cp = np.sum(Y * cp_R * R_U / mech.W[None], axis=1)    # c_p,mix, erg/(g K)
        N = np.sum(inlet.Y_in[None] * (h - h_in), axis=1) \
            + inlet.tau / rho * np.sum(h * mech.W[None] * wdot, axis=1)
        F[:, mech.K] = N / (cp * T)
    return F


def mixture_enthalpy(mech: Mechanism, Y, T):
    """h(T, Y) = sum_k Y_k h_k(T), erg/g."""
    _, h_RT, _ = species_thermo(mech, T)
    return np.sum(Y * h_RT * R_U * np.asarray(T)[:, None] / mech.W[None], axis=1)


# ----------------------------------------------------------------------------- linear algebra
def lu_factor(A):
    """LU decomposition with partial pivoting (row interchanges), P A = L U with unit
    lower L. Returns (LU packed, piv, ok); ok is False when a pivot is 0 or not finite."""
    A = np.array(A, dtype=np.float64, copy=True)
    n = A.shape[0]
    piv = np.arange(n)
    for k in range(n):
        p = k + int(np.argmax(np.abs(A[k:, k])))
        if not np.isfinite(A[p, k]) or A[p, k] == 0.0:
            return A, piv, False
        if p != k:
            A[[k, p]] = A[[p, k]]
            piv[[k, p]] = piv[[p, k]]
        A[k + 1:, k] /= A[k, k]
        A[k + 1:, k + 1:] -= np.outer(A[k + 1:, k], A[k, k + 1:])
    return A, piv, True


def lu_solve(LU, piv, b):
    """Solve A x = b from lu_factor's output: forward then back substitution."""
    n = LU.shape[0]
    y = np.asarray(b, dtype=np.float64)[piv].copy()
    for i in range(n):
        y[i] -= LU[i, :i] @ y[:i]
    x = y
    for i in range(n - 1, -1, -1):
        x[i] = (x[i] - LU[i, i + 1:] @ x[i + 1:]) / LU[i, i]
    return x


# ----------------------------------------------------------------------------- solver
@dataclasses.dataclass
class Options:
    """Solver controls (the same meaning as the library's options)."""
    ftol: float = 1e-8          # ||F||_inf target
    step_rtol: float = 1e-10    # polish: last undamped Newton step |dx_j| <= rtol |x_j| + atol_j
    step_atol_y: float = 1e-14
    step_atol_t: float = 1e-10  # kelvin
    max_newton: int = 500       # all Newton iterations, steady and inside time steps
    max_damp: int = 8           # halvings of the damping factor
    max_ts_rounds: int = 100    # Newton attempts that may be followed by time stepping
    ts_steps: int = 12          # pseudo-time steps per round before Newton is retried
    ts_newton: int = 8          # Newton iterations allowed per pseudo-time step
    ts_linear: int = 150        # pseudo-time steps are linearised (one Newton iteration each)
                                #   while fewer iterations than this have been used; later
                                #   ones (all when 0) are solved by damped Newton to ts_rtol
    ts_rtol: float = 1e-4       # a time step is solved when its undamped step is below
    ts_atol_y: float = 1e-10    #   ts_rtol |x_j| + ts_atol_j
    dt0_over_tau: float = 1e-6    # first pseudo-time step / tau
    dt_shrink: float = 0.25     # dt factor after a failed pseudo-time step
    y_floor: float = 1e-10      # iterates keep Y_k >= -y_floor
    t_min: float = 200.0
    t_max: float = 5000.0
    fd_rel: float = 1e-6        # central-difference step h_j = fd_rel * max(|x_j|, s_j)
    jacobian: str = "cs"        # Newton's Jacobian: "cs" complex step, "fd" central
                                #   differences (the paper's choice, Sec. 1)


@dataclasses.dataclass
class Result:
    x: np.ndarray
    status: int
    iters: int
    ts_steps: int
    fnorm: float


class GasSystem:
    """The K+1 gas-phase unknowns of one reactor: residual, bounds, scales."""

    def __init__(self, mech, inlet, energy="adiabatic", lnmult=None):
        self.mech, self.inlet, self.energy, self.lnmult = mech, inlet, energy, lnmult
        self.n = mech.K + 1
        self.K = mech.K

    def F(self, X):
        return gas_residual(self.mech, X, self.inlet, self.energy, self.lnmult)

    def fd_scale(self, x):
        s = np.full(self.K + 1, 0.1)
        s[self.K] = 1000.0
        return s

    def step_tol(self, x, opts):
        atol = np.full(self.K + 1, opts.step_atol_y)
        atol[self.K] = opts.step_atol_t
        return opts.step_rtol * np.abs(x) + atol

    def ts_tol(self, x, opts):
        atol = np.full(self.K + 1, opts.ts_atol_y)
        atol[self.K] = opts.ts_rtol
        return opts.ts_rtol * np.abs(x) + atol

    def norm_weights(self, x):
        """Scaling of the step norm: mass fractions absolute, temperature relative."""
        w = np.ones(self.K + 1)
        w[self.K] = 1.0 / abs(x[self.K])
        return w

    def max_in_bounds(self, x, dx, opts):
        """Largest lambda with x + lambda dx inside the bounds (inf if unlimited)."""
        lam = math.inf
        lo = np.full(self.K + 1, -opts.y_floor); hi = np.full(self.K + 1, math.inf)
        lo[self.K], hi[self.K] = opts.t_min, opts.t_max
        for j in range(self.K + 1):
            if dx[j] < 0 and x[j] + dx[j] < lo[j]:
                lam = min(lam, (lo[j] - x[j]) / dx[j])
            elif dx[j] > 0 and x[j] + dx[j] > hi[j]:
                lam = min(lam, (hi[j] - x[j]) / dx[j])
        return lam

    def in_bounds(self, x, opts):
        T = x[self.K]
        return bool(np.all(x[:self.K] >= -opts.y_floor) and opts.t_min <= T <= opts.t_max)

    def transient_weights(self, x):
        """Inverse mass-matrix diagonal of the pseudo-transient form dx/dt = -D F / tau:
        1 for the species rows, 1/T for the (dimensionless) energy row."""
        w = np.ones(self.K + 1)
        if self.energy != "fixed":
            w[self.K] = 1.0 / x[self.K]
        return w


def jacobian_fd(system, x, opts: Options):
    """Central finite-difference Jacobian dF/dx, h_j = fd_rel max(|x_j|, s_j); all 2n
    perturbed states are evaluated in one call. Kept for checks; the solver uses the
    complex-step form below."""
    n = len(x)
    h = opts.fd_rel * np.maximum(np.abs(x), system.fd_scale(x))
    X = np.repeat(x[None], 2 * n, axis=0)
    X[np.arange(n), np.arange(n)] += h
    X[n + np.arange(n), np.arange(n)] -= h
    Fx = system.F(X)
    return ((Fx[:n] - Fx[n:]) / (2 * h)[:, None]).T


def jacobian_cs(system, x, h=1e-30):
    """Jacobian by complex-step differentiation: J[:, j] = Im F(x + i h e_j) / h.
    Like the finite differences the paper uses to build its Jacobian (Sec. 1), it
    perturbs one unknown at a time, but it has no subtractive cancellation, so the
    columns are exact to rounding for any small h (Squire & Trapp 1998)."""
    n = len(x)
    X = np.repeat(np.asarray(x, dtype=np.complex128)[None], n, axis=0)
    X[np.arange(n), np.arange(n)] += 1j * h
    return (system.F(X).imag / h).T


def newton_jacobian(system, x, opts: Options):
    """The Jacobian Newton uses: complex step (default) or the paper's central
    finite differences (Sec. 1), per opts.jacobian. Both reach the same roots."""
    if opts.jacobian == "fd":
        return jacobian_fd(system, x, opts)
    if opts.jacobian != "cs":
        raise ValueError(f"unknown Jacobian option {opts.jacobian!r}")
    return jacobian_cs(system, x)


def _damped_newton(system, x, c, x_ref, max_it, opts, steady, counter, fnorm=None):
    """Damped Newton on R(y) = F(y) + c (y - x_ref) from y = x (c = 0: the steady
    problem; c = tau/dt D^-1: one backward-Euler step of dx/dt = -D F / tau).

    Each iteration solves (J + diag(c)) dy = -R by LU. The damping factor lambda
    starts at the largest value <= 1 that keeps the iterate in bounds and is halved
    until the natural monotonicity test holds: the simplified correction
    -(J + diag(c))^-1 R(y + lambda dy), computed with the same LU factors, is smaller
    than dy in the scaled max-norm (species absolute, temperature relative).
    Steady: converged when ||F||_inf <= ftol and the undamped step is below the
    polish tolerance; that step is applied. Time step: converged when the undamped
    step is below ts_rtol. Returns (y, F(y), converged); fnorm, when given, receives
    ||F||_inf (the steady residual, not R) at the first and at the last evaluated point."""
    def residual(v):
        Fv = system.F(v)[0]
        if fnorm is not None:
            f = float(np.max(np.abs(Fv)))
            if fnorm[0] is None:
                fnorm[0] = f
            fnorm[1] = f
        return Fv + c * (v - x_ref)

    y = x.copy()
    R = residual(y)
    dn_prev = math.inf
    for _ in range(max_it):
        if counter[0] >= opts.max_newton:
            break
        counter[0] += 1
        J = newton_jacobian(system, y, opts) + np.diag(c)
        LU, piv, ok = lu_factor(J)
        if not ok:
            break
        dy = lu_solve(LU, piv, -R)
        if not np.all(np.isfinite(dy)):
            break
        if steady:
            if np.max(np.abs(R)) <= opts.ftol and np.all(np.abs(dy) <= system.step_tol(y, opts)):
                y = y + dy
                return y, system.F(y)[0], True
        elif np.all(np.abs(dy) <= system.ts_tol(y, opts)):
            y = y + dy
            return y, system.F(y)[0], True
        w = system.norm_weights(y)
        dn = float(np.max(np.abs(dy) * w))
        if dn >= dn_prev:
            break                                   # corrections stopped shrinking: give up
        dn_prev = dn
        lam = min(1.0, system.max_in_bounds(y, dy, opts))
        accepted = False
        for _ in range(opts.max_damp):
            yt = y + lam * dy
            if system.in_bounds(yt, opts):
                Rt = residual(yt)
                if np.all(np.isfinite(Rt)):
                    dbar = lu_solve(LU, piv, -Rt)
                    if float(np.max(np.abs(dbar) * w)) < dn:
                        accepted = True
                        break
            lam *= 0.5
        if not accepted:
            break
        y, R = yt, Rt
    return y, system.F(y)[0], False


def _linearised_step(system, x, c, opts, counter):
    """One linearised backward-Euler step of dx/dt = -D F(x) / tau (pseudo-transient
    continuation, Kelley & Keyes 1998): solve (J(x) + diag(c)) dx = -F(x) and take the
    full step when it keeps the iterate in bounds and F finite. Returns (x_new,
    ||F(x_new)||_inf, accepted)."""
    if counter[0] >= opts.max_newton:
        return x, None, False
    counter[0] += 1
    F = system.F(x)[0]
    LU, piv, ok = lu_factor(newton_jacobian(system, x, opts) + np.diag(c))
    if not ok:
        return x, None, False
    dx = lu_solve(LU, piv, -F)
    if not np.all(np.isfinite(dx)) or system.max_in_bounds(x, dx, opts) < 1.0:
        return x, None, False
    y = x + dx
    if not system.in_bounds(y, opts):
        return x, None, False
    Fy = system.F(y)[0]
    if not np.all(np.isfinite(Fy)):
        return x, None, False
    return y, float(np.max(np.abs(Fy))), True


def solve_system(system, x0, opts: Options = Options()):
    """Hybrid Newton / pseudo-transient solve of F(x) = 0 (Sec. 3): a damped Newton
    iteration on the steady problem; when it fails (damping exhausted, corrections
    not shrinking, singular J) the estimate it started from is conditioned by
    ts_steps backward-Euler steps of the transient form dx/dt = -D F(x) / tau; then
    Newton is tried again.

    While fewer than ts_linear Newton iterations have been used, each step is one
    linearised Newton iteration (pseudo-transient continuation, Kelley & Keyes 1998); after
    an accepted step dt grows by 2 times the factor by which the step changed ||F||_inf,
    clipped to [0.1, 8] (switched evolution relaxation, Mulder & van Leer 1985), and shrinks
    by dt_shrink after a rejected one.
    Later steps are solved by damped Newton (<= ts_newton iterations, to ts_rtol);
    after an accepted step dt grows by 2 if it took <= 3 iterations (1.25 after 4, 1
    after more), times the ||F||_inf reduction clipped to [1, 4] (||F||_inf at the last
    point each Newton evaluated).
    iters counts every Newton iteration (one Jacobian and LU each), ts_steps the
    accepted pseudo-time steps."""
    tau = system.inlet.tau
    x = np.array(x0, dtype=np.float64)
    F = system.F(x)[0]
    if not np.all(np.isfinite(F)):
        return Result(x, NONFINITE, 0, 0, math.inf)
    counter = [0]
    ts = rounds = 0
    dt = opts.dt0_over_tau * tau
    zero = np.zeros(system.n)
    while True:
        fn = [None, None]
        y, Fy, conv = _damped_newton(system, x, zero, x, opts.max_newton, opts, True, counter, fn)
        if conv:
            return Result(y, CONVERGED, counter[0], ts, float(np.max(np.abs(Fy))))
        if counter[0] >= opts.max_newton:
            return Result(y, MAX_ITER, counter[0], ts, float(np.max(np.abs(Fy))))
        # a failed Newton attempt leaves the estimate where it was: the time steps
        # condition the estimate from which Newton started
        rounds += 1
        if rounds > opts.max_ts_rounds:
            return Result(x, TS_EXHAUSTED, counter[0], ts, float(np.max(np.abs(system.F(x)[0]))))
        taken = 0
        f_prev = fn[0]                      # ||F(x)||_inf of the estimate being conditioned
        while taken < opts.ts_steps:
            c = tau / dt * system.transient_weights(x)
            used = counter[0]
            linear = counter[0] < opts.ts_linear
            if linear:
                y, f_new, conv = _linearised_step(system, x, c, opts, counter)
            else:
                fs = [None, None]
                y, Fy, conv = _damped_newton(system, x, c, x, opts.ts_newton, opts, False, counter, fs)
                f_new = fs[1]
            used = counter[0] - used
            if counter[0] >= opts.max_newton:
                return Result(x, MAX_ITER, counter[0], ts, float(np.max(np.abs(system.F(x)[0]))))
            if conv:
                x = y
                taken += 1
                ts += 1
                if linear:
                    g = 2.0 * (min(8.0, max(0.1, f_prev / f_new)) if f_new > 0.0 else 1.0)
                else:
                    # grow dt by how easily the step was solved and how much it reduced ||F||
                    g = 2.0 if used <= 3 else (1.25 if used == 4 else 1.0)
                    if f_new is not None and f_new > 0.0 and f_prev is not None:
                        g *= min(4.0, max(1.0, f_prev / f_new))
                f_prev = f_new
                dt = min(g * dt, 1e6 * tau)
            else:
                dt *= opts.dt_shrink
                if dt < 1e-16 * tau:
                    return Result(x, TS_EXHAUSTED, counter[0], ts,
                                  float(np.max(np.abs(system.F(x)[0]))))


def solve_reactor(mech: Mechanism, inlet: Inlet, x0, opts: Options = Options(),
                  energy="adiabatic", lnmult=None):
    """Gas-only PSR: x = (Y, T)."""
    return solve_system(GasSystem(mech, inlet, energy, lnmult), x0, opts)


def inlet_of(batch, b, energy="adiabatic"):
    return Inlet(np.asarray(batch.Y_in[b], dtype=np.float64), float(batch.T_in[b]),
                 float(batch.tau[b]), float(batch.P[b]),
                 float(batch.T0[b]) if energy == "fixed" else 0.0)


def solve_batch(mech: Mechanism, batch, opts: Options = Options(), energy="adiabatic",
                indices=None):
    """Solve the reactors `indices` (default all) of a batch one after another."""
    idx = range(batch.B) if indices is None else indices
    out = dict(Y=[], T=[], status=[], iters=[], ts_steps=[], fnorm=[])
    for b in idx:
        x0 = np.concatenate([batch.Y0[b], [batch.T0[b]]])
        r = solve_reactor(mech, inlet_of(batch, b, energy), x0, opts, energy)
        out["Y"].append(r.x[:mech.K]); out["T"].append(r.x[mech.K])
        out["status"].append(r.status); out["iters"].append(r.iters)
        out["ts_steps"].append(r.ts_steps); out["fnorm"].append(r.fnorm)
    return {k: np.array(v) for k, v in out.items()}


# ----------------------------------------------------------------------------- sensitivities
def rate_parameter_jacobian(mech: Mechanism, inlet: Inlet, x, energy="adiabatic", lnmult=None, h=1e-30):
    """dF/dp at state x for p_i = ln(multiplier of q_i), one complex-step column per
    reaction (the multiplier scales the whole rate of progress of reaction i)."""
    I = mech.I
    base = np.zeros(I) if lnmult is None else np.asarray(lnmult, dtype=np.float64)
    P = np.repeat(base[None].astype(np.complex128), I, axis=0)
    P[np.arange(I), np.arange(I)] += 1j * h
    X = np.repeat(np.asarray(x, dtype=np.complex128)[None], I, axis=0)
    Fp = gas_residual(mech, X, inlet, energy, P)
    return (Fp.imag / h).T                        # (n, I)


def sensitivities(mech: Mechanism, inlet: Inlet, x, energy="adiabatic", lnmult=None):
    """Dense S = dx*/dp = -J^-1 dF/dp at a root x* (implicit function theorem), with the
    complex-step Jacobian and the oracle's own LU."""
    S_sys = GasSystem(mech, inlet, energy, lnmult)
    J = jacobian_cs(S_sys, x)
    Fp = rate_parameter_jacobian(mech, inlet, x, energy, lnmult)
    LU, piv, ok = lu_factor(J)
    if not ok:
        raise ArithmeticError("singular Jacobian at the root")
    return -np.stack([lu_solve(LU, piv, Fp[:, i]) for i in range(mech.I)], axis=1)


def adjoint_gradient(mech: Mechanism, inlet: Inlet, x, g, energy="adiabatic", lnmult=None):
    """dL/dp_i = g^T dx*/dp_i for a loss with dL/dx* = g, from the dense sensitivities."""
    return np.asarray(g, dtype=np.float64) @ sensitivities(mech, inlet, x, energy, lnmult)
