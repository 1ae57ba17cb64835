"""Seeded synthetic workloads for the batched steady-state PSR solve.

This module only draws numbers and writes them out: reaction mechanisms (species,
elementary / third-body / Troe-falloff reactions, NASA-7 thermo coefficients, MOMIC
soot constants) and inlet batches. It holds none of the reactor arithmetic. Both the
CPU oracle and the CUDA library read the `.psrmech` text written here, each with its
own parser, so the two share inputs and nothing else.

The mechanisms stand in for the paper's ethylene mechanisms (101 species / 542
reactions for the speed runs of Sec. 6, the Wang-Frenklach mechanism for Sec. 5),
which are not available: species over {C, H, O, N} with integer compositions 0..4,
element-balanced reversible reactions with at most three reactants and three
products, Arrhenius parameters A log-uniform in [1e6, 1e14] (CGS), beta in [-1, 2],
activation energy in [0, 250] kJ/mol, ideal-gas heat capacities between 3.5 R and
8 R. The drawn A is the magnitude of a bimolecular rate coefficient at 1000 K; the
file stores the equivalent A of the standard A T^beta exp(-E/RT) form for the
reaction's order (A_file = A_1000 C_REF^(2 - order) / 1000^beta), which keeps the
fastest pseudo-first-order rates near 1e9 /s, as in real combustion mechanisms, so
that the steady residual stays resolvable in FP64.

File format (`.psrmech`, whitespace-separated text, one record per line, '#'
starts a comment line)::

    psrmech 1
    elements <E>
    <symbol> <atomic weight g/mol>                      (E lines)
    species <K>
    <idx> <name> <a_C a_H a_O a_N> <T_low T_mid T_high> <7 low-range coeffs> <7 high-range coeffs>
    reactions <I>
    <idx> <type> <n_r> <reactant idx ...> <n_p> <product idx ...> <A> <beta> <E/R [K]> [extras]
    soot <key value pairs>                               (optional, one line)
    end

`type` is `elem`, `tb` (third body) or `troe` (falloff). Reactant and product
lists repeat a species once per unit of stoichiometric coefficient. Extras, in this
order when present: `low <A0> <beta0> <E0/R>` and `troe <alpha> <T3> <T1> <T2>`
(falloff only; T2 = 0 means the three-parameter form), then
`eff <m> <species idx> <efficiency> ...` (tb and troe). Units are CGS with
concentrations in mol/cm^3: A in (cm^3/mol)^(order-1)/s, E/R in kelvin.
"""
from __future__ import annotations

import dataclasses
import io
from typing import Optional

import numpy as np

ELEMENTS = ("C", "H", "O", "N")
ELEMENT_WEIGHTS = (12.011, 1.008, 15.999, 14.007)
ONE_ATM = 1.01325e6          # dyn/cm^2; every reactor of the synthetic batches runs at 1 atm
GAS_CONSTANT_J = 8.314462618  # J/(mol K), only to express the activation-energy range as E/R
C_REF = 1e-5                  # mol/cm^3, concentration scale that sets A's units per reaction order
MECH_SEED_BASE = 20051146
MAX_HEAT_K = 60000.0          # largest |heat of reaction| / R drawn, K (about 500 kJ/mol)
ANCHOR_BIAS = 0.5             # share of elementary reactions drawn with an inlet species as reactant

# anchor species 0..3: N2-like, O2-like, H2-like, C2H2-like (the soot precursor)
_ANCHORS = ((0, 0, 0, 2), (0, 0, 2, 0), (0, 2, 0, 0), (2, 2, 0, 0))
_ANCHOR_NAMES = ("N2", "O2", "H2", "C2H2")


@dataclasses.dataclass
class Reaction:
    kind: str                      # "elem" | "tb" | "troe"
    reac: list                     # species indices, repeated per unit coefficient
    prod: list
    A: float
    beta: float
    theta: float                   # E/R in K
    eff: dict = dataclasses.field(default_factory=dict)   # species -> efficiency
    low: Optional[tuple] = None    # (A0, beta0, theta0) for falloff
    troe: Optional[tuple] = None   # (alpha, T3, T1, T2)


@dataclasses.dataclass
class MechanismSpec:
    names: list
    comp: np.ndarray               # (K, 4) int
    t_range: np.ndarray            # (K, 3) T_low, T_mid, T_high
    nasa_low: np.ndarray           # (K, 7)
    nasa_high: np.ndarray          # (K, 7)
    reactions: list
    soot: Optional[dict] = None

    @property
    def K(self):
        return len(self.names)

    @property
    def I(self):
        return len(self.reactions)

    @property
    def n_tb(self):
        return sum(r.kind == "tb" for r in self.reactions)

    @property
    def n_troe(self):
        return sum(r.kind == "troe" for r in self.reactions)


def _name(c):
    s = ""
    for sym, n in zip(ELEMENTS, c):
        if n:
            s += sym + (str(n) if n > 1 else "")
    return s


def _species(K, rng):
    comps = list(_ANCHORS)
    seen = set(comps)
    frags = []
    for e in range(4):                       # monatomic fragments
        c = [0, 0, 0, 0]; c[e] = 1; frags.append(tuple(c))
    for e1 in range(4):                      # diatomic fragments
        for e2 in range(e1, 4):
            c = [0, 0, 0, 0]; c[e1] += 1; c[e2] += 1
            if tuple(c) not in seen:
                frags.append(tuple(c))
    order = rng.permutation(len(frags))
    for j in order:
        if len(comps) >= K:
            break
        comps.append(frags[j]); seen.add(frags[j])
    tries = 0
    while len(comps) < K:                    # constructive sums, each element capped at 4
        tries += 1
        if tries > 200000:
            raise RuntimeError(f"cannot build {K} distinct species")
        a, b = rng.integers(0, len(comps), 2)
        c = tuple(int(x) for x in np.add(comps[a], comps[b]))
        if max(c) <= 4 and c not in seen:
            comps.append(c); seen.add(c)
    comp = np.array(comps[:K], dtype=np.int64)
    names = []
    for k, c in enumerate(comp):
        names.append(_ANCHOR_NAMES[k] if k < 4 else _name(c) + f"_{k}")
    return names, comp


# gas-phase heats of formation of the free atoms C, H, O, N (kJ/mol) and valences
_ATOM_HF = np.array([717.0, 218.0, 249.0, 473.0])
_VALENCE = np.array([4, 1, 2, 3])
_K_PER_KJ = 1000.0 / GAS_CONSTANT_J      # 1 kJ/mol expressed as E/R in kelvin


def _thermo(comp, rng, split_ranges):
    """NASA-7 coefficients: c_p/R linear in T between 3.5 and 8 (a3..a5 = 0); heats of
    formation from bond additivity: atoms' formation heats minus the number of bond
    pairs (valences / 2, 0 for a free atom) times a per-species mean bond energy of
    300..420 kJ/mol (up to 60 kJ/mol stronger for oxidised C/H species), so that
    molecules are stable at flame temperatures and oxidation releases heat; N2, O2 and
    H2 are the reference states (0) and C2H2 gets +228 kJ/mol. Standard entropies grow
    with size as for real species: S(298)/R = 14 + 5 (atoms - 1) + U[-2, 3], at most
    45. a6 and a7 place H and S at about 298 K."""
    K = len(comp)
    low = np.zeros((K, 7)); t_range = np.tile([200.0, 1000.0, 5000.0], (K, 1))
    a1 = rng.uniform(3.5, 5.5, K)
    cp3000 = rng.uniform(a1, 8.0)
    low[:, 0] = a1
    low[:, 1] = (cp3000 - a1) / 3000.0
    natoms = comp.sum(1)
    bonds = np.where(natoms > 1, np.maximum(natoms - 1, (comp @ _VALENCE) // 2), 0)
    nC, nH, nO = comp[:, 0], comp[:, 1], comp[:, 2]
    oxid = (nO > 0) & ((nC + nH) > 0)
    bond_e = rng.uniform(300.0, 420.0, K) + np.where(oxid, rng.uniform(0.0, 60.0, K), 0.0)
    hf = comp @ _ATOM_HF - bonds * bond_e                   # kJ/mol
    hf[:3] = 0.0                                             # N2, O2, H2
    hf[3] = 228.0                                            # C2H2-like
    s298 = np.minimum(14.0 + 5.0 * (natoms - 1) + rng.uniform(-2.0, 3.0, K), 45.0)
    low[:, 5] = hf * _K_PER_KJ - 298.15 * a1
    low[:, 6] = s298 - a1 * np.log(298.15)
    high = low.copy()
    if split_ranges:
        # different low-range coefficients, so that evaluations must pick the right range
        low[:, 0] = low[:, 0] + rng.uniform(-0.3, 0.3, K)
        low[:, 5] = low[:, 5] + rng.uniform(-300.0, 300.0, K)
        low[:, 6] = low[:, 6] + rng.uniform(-0.5, 0.5, K)
    return t_range, low, high


def _products_with(v, comp_index, pair_index, comp):
    """All multisets (size 1..3) of species whose summed composition is v."""
    out = []
    k = comp_index.get(v)
    if k is not None:
        out.append((k,))
    for pr in pair_index.get(v, ()):
        out.append(pr)
    for b in range(len(comp)):
        r = tuple(int(x) for x in np.subtract(v, comp[b]))
        if min(r) < 0:
            continue
        for pr in pair_index.get(r, ()):
            if pr[0] >= b:
                out.append((b,) + pr)
    return out


def make_mechanism(K, I, n_tb=0, n_troe=0, seed=MECH_SEED_BASE, soot=False, split_ranges=False):
    """Draw a mechanism of K species and I reversible reactions (n_tb third-body and
    n_troe falloff among them), all element-balanced. Fails loudly if the species set
    cannot supply I distinct balanced reactions."""
    rng = np.random.Generator(np.random.PCG64(seed))
    names, comp = _species(K, rng)
    t_range, low, high = _thermo(comp, rng, split_ranges)
    comp_index = {tuple(int(x) for x in c): k for k, c in enumerate(comp)}
    pair_index = {}
    for a in range(K):
        for b in range(a, K):
            v = tuple(int(x) for x in comp[a] + comp[b])
            pair_index.setdefault(v, []).append((a, b))
    recomb = [(a, b) for (v, lst) in pair_index.items() if v in comp_index for (a, b) in lst]
    seen = set()
    reactions = []
    a6 = low[:, 5]

    def heat_ok(r, p):
        # no reaction with a heat of reaction above about 500 kJ/mol, so that
        # equilibrium constants stay within the FP64 range down to 200 K
        return abs(a6[list(p)].sum() - a6[list(r)].sum()) <= MAX_HEAT_K

    def exothermic_first(r, p):
        # write each reaction in the direction in which the summed a6 parameters
        # (heats of formation / R) fall, so that neither direction has a negative
        # effective barrier once the reverse rate is taken from the equilibrium constant
        return (r, p) if a6[list(p)].sum() <= a6[list(r)].sum() else (p, r)

    def draw_arrhenius(order):
        # A is drawn as the magnitude of a bimolecular rate coefficient at 1000 K,
        # then written in the file's A T^beta form for the reaction's true order:
        # file A = A_1000 * C_REF^(2 - order) / 1000^beta.
        a_ref = 10.0 ** rng.uniform(6.0, 14.0)
        beta = float(rng.uniform(-1.0, 2.0))
        theta = float(rng.uniform(0.0, 250e3) / GAS_CONSTANT_J)
        return float(a_ref * C_REF ** (2 - order) / 1000.0 ** beta), beta, theta

    def draw_eff():
        m = int(rng.integers(0, 5))
        sp = rng.choice(K, size=m, replace=False) if m else []
        return {int(s): float(rng.uniform(0.5, 5.0)) for s in sp}

    def key(r, p):
        r, p = tuple(sorted(r)), tuple(sorted(p))
        return min(r, p), max(r, p)

    n_special = n_tb + n_troe
    if n_special > len(recomb):
        raise RuntimeError("not enough recombination pairs for third-body/falloff reactions")
    tries = 0
    while len(reactions) < n_special:
        tries += 1
        if tries > 100000:
            raise RuntimeError("cannot draw distinct recombination reactions")
        a, b = recomb[int(rng.integers(len(recomb)))]
        p = comp_index[tuple(int(x) for x in comp[a] + comp[b])]
        kk = key((a, b), (p,))
        if kk in seen or not heat_ok([a, b], [p]):
            continue
        seen.add(kk)
        r_, p_ = exothermic_first([a, b], [p])
        if len(reactions) < n_tb:
            A, beta, theta = draw_arrhenius(len(r_) + 1)      # the third body adds one order
            reactions.append(Reaction("tb", r_, p_, A, beta, theta, eff=draw_eff()))
        else:
            A, beta, theta = draw_arrhenius(len(r_))          # high-pressure limit
            # low-pressure limit (one order higher) placed so that the reduced pressure
            # k0 [M] / k_inf at [M] = C_REF and 1000 K is 10^U[-2, 2]
            beta0 = float(rng.uniform(-2.0, 0.0))
            theta0 = float(rng.uniform(0.0, 0.5) * theta)
            pr_ref = 10.0 ** rng.uniform(-2.0, 2.0)
            k_inf_1000 = A * 1000.0 ** beta
            A0 = pr_ref * k_inf_1000 / C_REF / 1000.0 ** beta0   # k0 C_REF = pr_ref k_inf
            low_p = (float(A0), beta0, theta0)
            T2 = float(rng.uniform(1000.0, 8000.0)) if rng.random() < 0.5 else 0.0
            troe = (float(rng.uniform(0.1, 0.9)), float(rng.uniform(50.0, 300.0)),
                    float(rng.uniform(500.0, 5000.0)), T2)
            reactions.append(Reaction("troe", r_, p_, A, beta, theta, eff=draw_eff(),
                                      low=low_p, troe=troe))
    tries = 0
    while len(reactions) < I:
        tries += 1
        if tries > 200000:
            raise RuntimeError(f"cannot draw {I} distinct balanced reactions over {K} species")
        rs = int(rng.choice([1, 2, 3], p=[0.1, 0.7, 0.2]))
        reac = [int(x) for x in rng.integers(0, K, rs)]
        if rng.random() < ANCHOR_BIAS:
            # fuel and oxidiser take part in many reactions, as in real mechanisms
            reac[0] = int(rng.integers(0, 4))
        reac = sorted(reac)
        v = tuple(int(x) for x in comp[reac].sum(0))
        cands = [c for c in _products_with(v, comp_index, pair_index, comp)
                 if tuple(sorted(c)) != tuple(reac)]
        if not cands:
            continue
        prod = sorted(cands[int(rng.integers(len(cands)))])
        kk = key(reac, prod)
        if kk in seen or not heat_ok(reac, prod):
            continue
        seen.add(kk)
        reac, prod = exothermic_first(reac, prod)
        A, beta, theta = draw_arrhenius(len(reac))
        reactions.append(Reaction("elem", reac, prod, A, beta, theta))
    order = rng.permutation(len(reactions))          # interleave special and elementary
    reactions = [reactions[j] for j in order]
    soot_p = None
    if soot:
        soot_p = dict(
            precursor=3, h2=2,
            nuc_A=float(10.0 ** rng.uniform(5.0, 6.0)),       # 1/s on the precursor concentration
            nuc_theta=float(rng.uniform(10000.0, 14000.0)),
            cmin=32.0,                                         # carbon atoms per nucleus
            grow_A=float(10.0 ** rng.uniform(13.0, 14.0)),     # cm^3/(mol s) per active site
            grow_beta=0.0,
            grow_theta=float(rng.uniform(3000.0, 6000.0)),
            chi_alpha=float(rng.uniform(1e13, 5e14)),          # active sites per cm^2 x alpha
            rho_s=1.8, coag_eps=2.2, m0_floor=1.0,
        )
    return MechanismSpec(names, comp, t_range, low, high, reactions, soot_p)


def mechanism_text(m: MechanismSpec) -> str:
    f = io.StringIO()
    w = f.write
    w("psrmech 1\n")
    w(f"elements {len(ELEMENTS)}\n")
    for s, wt in zip(ELEMENTS, ELEMENT_WEIGHTS):
        w(f"{s} {wt!r}\n")
    w(f"species {m.K}\n")
    for k in range(m.K):
        vals = [*m.t_range[k], *m.nasa_low[k], *m.nasa_high[k]]
        w(f"{k} {m.names[k]} " + " ".join(str(int(x)) for x in m.comp[k]) + " "
          + " ".join(f"{float(v):.17g}" for v in vals) + "\n")
    w(f"reactions {m.I}\n")
    for i, r in enumerate(m.reactions):
        s = f"{i} {r.kind} {len(r.reac)} " + " ".join(map(str, r.reac))
        s += f" {len(r.prod)} " + " ".join(map(str, r.prod))
        s += f" {r.A:.17g} {r.beta:.17g} {r.theta:.17g}"
        if r.kind == "troe":
            s += " low " + " ".join(f"{v:.17g}" for v in r.low)
            s += " troe " + " ".join(f"{v:.17g}" for v in r.troe)
        if r.kind in ("tb", "troe"):
            s += f" eff {len(r.eff)}" + "".join(f" {k} {v:.17g}" for k, v in sorted(r.eff.items()))
        w(s + "\n")
    if m.soot is not None:
        w("soot " + " ".join(f"{k} {v:.17g}" if isinstance(v, float) else f"{k} {v}"
                             for k, v in m.soot.items()) + "\n")
    w("end\n")
    return f.getvalue()


def write_mechanism(m: MechanismSpec, path):
    with open(path, "w") as fh:
        fh.write(mechanism_text(m))


@dataclasses.dataclass
class Batch:
    """Inlet conditions and initial guesses for B reactors of one mechanism.
    Row-major [B][K] mass fractions, [B] scalars; P in dyn/cm^2, tau in s."""
    Y_in: np.ndarray
    T_in: np.ndarray
    tau: np.ndarray
    P: np.ndarray
    Y0: np.ndarray
    T0: np.ndarray
    M_in: Optional[np.ndarray] = None      # [B][6] inlet soot moments (sooting mechanisms)

    @property
    def B(self):
        return self.Y_in.shape[0]

    def subset(self, idx):
        idx = np.asarray(idx, dtype=np.int64)
        return Batch(*(None if getattr(self, f.name) is None else getattr(self, f.name)[idx]
                       for f in dataclasses.fields(self)))


SEED_PARTICLES = 1e-6      # nuclei per cm^3 in the inlet of a sooting batch (a trace of seeds)


def make_batch(m: MechanismSpec, B, seed, tau_range=(1e-4, 1e-2), T_in_range=(300.0, 800.0),
               T_guess=2000.0, alpha=0.5):
    """Inlets: Y_in ~ Dirichlet(alpha) over the four anchor species (others zero),
    T_in uniform, tau log-uniform, P = 1 atm; guess = inlet composition at T_guess."""
    rng = np.random.Generator(np.random.PCG64(seed))
    K = m.K
    Y_in = np.zeros((B, K))
    Y_in[:, :4] = rng.dirichlet([alpha] * 4, size=B)
    T_in = rng.uniform(*T_in_range, B)
    tau = np.exp(rng.uniform(np.log(tau_range[0]), np.log(tau_range[1]), B))
    P = np.full(B, ONE_ATM)
    b = Batch(Y_in, T_in, tau, P, Y_in.copy(), np.full(B, float(T_guess)))
    if m.soot is not None:
        # inlet moments of SEED_PARTICLES nuclei of C_min carbon atoms: M_r = N C_min^r
        b.M_in = np.tile(SEED_PARTICLES * m.soot["cmin"] ** np.arange(6.0), (B, 1))
    return b


# Named workloads (shapes of the paper's batched runs, scaled to the synthetic mechanisms).
WORKLOADS = {
    "k10_b64": dict(K=10, I=24, n_tb=0, n_troe=0, B=64, soot=False, tag=1),
    "k53_b4096": dict(K=53, I=325, n_tb=10, n_troe=15, B=4096, soot=False, tag=2),
    "k53soot_b16384": dict(K=53, I=325, n_tb=10, n_troe=15, B=16384, soot=True, tag=3,
                           tau_range=(1e-5, 1e-1)),
    "k200_b2048": dict(K=200, I=1500, n_tb=60, n_troe=40, B=2048, soot=False, tag=4),
    # the size of the ethylene mechanism the paper times its rate kernel on (101 species,
    # 542 reactions), for the rate-evaluation measurement
    "k101_rates": dict(K=101, I=542, n_tb=20, n_troe=20, B=100000, soot=False, tag=6),
}
# uneven batch: 50/35/15 % of reactors from the K=10 / K=53 / K=200 mechanisms
MIXED_WORKLOAD = dict(B=32768, parts=("k10_b64", "k53_b4096", "k200_b2048"),
                      fractions=(0.50, 0.35, 0.15), tag=5)


def workload_mechanism(name):
    w = WORKLOADS[name]
    return make_mechanism(w["K"], w["I"], w["n_tb"], w["n_troe"],
                          seed=MECH_SEED_BASE + 10 * w["tag"], soot=w["soot"])


def workload_batch(name, mech=None, B=None):
    w = WORKLOADS[name]
    mech = mech if mech is not None else workload_mechanism(name)
    return make_batch(mech, w["B"] if B is None else B, seed=MECH_SEED_BASE + 10 * w["tag"] + 1,
                      tau_range=w.get("tau_range", (1e-4, 1e-2)))


def mixed_assignment(B=None, seed=None):
    """Mechanism id (0, 1, 2 for K = 10, 53, 200) of each reactor of the uneven batch,
    in a seeded shuffled order."""
    B = MIXED_WORKLOAD["B"] if B is None else B
    seed = MECH_SEED_BASE + 10 * MIXED_WORKLOAD["tag"] + 1 if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = [int(round(f * B)) for f in MIXED_WORKLOAD["fractions"]]
    counts[0] = B - counts[1] - counts[2]
    ids = np.concatenate([np.full(c, j, dtype=np.int32) for j, c in enumerate(counts)])
    return ids[rng.permutation(B)]


def mixed_batch(specs, B=None, seed=None):
    """The uneven batch: mech ids from mixed_assignment, and for each mechanism class a
    batch of its own (make_batch, seed base + 10 tag + 2 + class) whose rows go, in order,
    to that class's reactors. Returns a dict with mech_id [B], row_off [B] (offsets into the
    packed rows), packed Y_in / Y0, per-reactor T_in, tau, P, T0, and per class the
    reactor indices and its Batch."""
    ids = mixed_assignment(B, seed)
    B = ids.shape[0]
    K = np.array([s.K for s in specs])
    row_len = K[ids]
    row_off = np.zeros(B, dtype=np.int64)
    row_off[1:] = np.cumsum(row_len)[:-1]
    L = int(row_len.sum())
    out = dict(mech_id=ids, row_off=row_off, Y_in=np.zeros(L), Y0=np.zeros(L), T_in=np.zeros(B),
               tau=np.zeros(B), P=np.zeros(B), T0=np.zeros(B), members=[], batches=[])
    base = MECH_SEED_BASE + 10 * MIXED_WORKLOAD["tag"] + 2
    for c, spec in enumerate(specs):
        members = np.flatnonzero(ids == c)
        bc = make_batch(spec, max(len(members), 1), seed=base + c)
        bc = bc.subset(range(len(members)))
        for j, r in enumerate(members):
            o = row_off[r]
            out["Y_in"][o:o + spec.K] = bc.Y_in[j]
            out["Y0"][o:o + spec.K] = bc.Y0[j]
        for k in ("T_in", "tau", "P", "T0"):
            out[k][members] = getattr(bc, k)
        out["members"].append(members)
        out["batches"].append(bc)
    return out
