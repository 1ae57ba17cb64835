"""GPU parity of the gas + MOMIC soot path against the oracle: residual, Jacobian, full
solves (sampled at the full 16384-reactor size) and carbon conservation gas + soot."""
import numpy as np
import pytest

from oracle import momic_oracle as S
from oracle import psr_oracle as O
from paper_2005_11468_gb300 import psr, synth

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]
NAME = "k53soot_b16384"
M_REL = 1e-5          # moments: relative parity bar
Y_REL, Y_MIN, T_ABS = 1e-6, 1e-10, 1e-8


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_11468_gb300 import _build
    _build.build()
    spec = synth.workload_mechanism(NAME)
    text = synth.mechanism_text(spec)
    return dict(dev=torch.device("cuda:0"), spec=spec, mech=O.Mechanism(text), gm=psr.Mechanism(text),
                batch=synth.workload_batch(NAME, spec))


_ROOTS = {}


def _oracle_roots(idx):
    """Oracle solves of sampled reactors of the sooting batch, cached across both forms."""
    key = tuple(idx)
    if key not in _ROOTS:
        from tests import oracle_pool
        _ROOTS[key] = oracle_pool.solve([(NAME, b) for b in idx])
    return _ROOTS[key]


def _t(env, b, keys=("Y_in", "T_in", "tau", "P", "Y0", "T0", "M_in")):
    import torch
    return {k: torch.tensor(getattr(b, k), dtype=torch.float64, device=env["dev"]) for k in keys}


def _states(env, m, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    mech = env["mech"]
    Y = rng.dirichlet(np.full(mech.K, 0.7), size=m)
    T = rng.uniform(900, 2400, m)
    N = 10 ** rng.uniform(6, 12, m)
    a = rng.uniform(3.5, 6.5, m)
    s2 = rng.uniform(0.05, 0.8, m)
    r = np.arange(6)
    M = N[:, None] * np.exp(a[:, None] * r + s2[:, None] * r * r / 2)
    return Y, T, M


def test_soot_residual_parity(env):
    import torch
    m = 16
    Y, T, M = _states(env, m, 1)
    sub = env["batch"].subset(range(m))
    t = _t(env, sub)
    dv = lambda a: torch.tensor(a, dtype=torch.float64, device=env["dev"])
    F = psr.eval_residual_soot(env["gm"], t["Y_in"], t["T_in"], t["tau"], t["P"], t["M_in"], dv(Y), dv(T), dv(M))
    F = F.cpu().numpy()
    for b in range(m):
        sysb = S.SootSystem(env["mech"], O.inlet_of(sub, b), sub.M_in[b])
        x = np.r_[Y[b], T[b], np.log(M[b] / sysb.soot.scale)]
        Fo = sysb.F(x)[0]
        scale = 1.0 + np.abs(Fo)
        scale[:env["mech"].K + 1] += 1e3          # gas rows: gross-rate cancellation (checked elsewhere)
        assert np.max(np.abs(F[b] - Fo) / scale) <= 1e-10


@pytest.mark.parametrize("precision", [psr.PSR_FP64, psr.PSR_MIXED])
def test_soot_jacobian_parity(env, precision):
    import torch
    m = 6
    Y, T, M = _states(env, m, 2)
    sub = env["batch"].subset(range(m))
    t = _t(env, sub)
    dv = lambda a: torch.tensor(a, dtype=torch.float64, device=env["dev"])
    J = psr.eval_jacobian_soot(env["gm"], t["Y_in"], t["T_in"], t["tau"], t["P"], t["M_in"], dv(Y), dv(T), dv(M),
                               precision=precision).cpu().numpy()
    tol = 1e-6 if precision == psr.PSR_FP64 else 2e-5
    for b in range(m):
        sysb = S.SootSystem(env["mech"], O.inlet_of(sub, b), sub.M_in[b])
        x = np.r_[Y[b], T[b], np.log(M[b] / sysb.soot.scale)]
        Jo = O.jacobian_cs(sysb, x)
        rowmax = np.max(np.abs(Jo), axis=1, keepdims=True)
        err = np.abs(J[b] - Jo) / rowmax
        assert np.max(err) <= tol, (b, np.unravel_index(np.argmax(err), err.shape), np.max(err))


@pytest.mark.parametrize("precision", [psr.PSR_FP64, psr.PSR_MIXED])
def test_soot_full_size_solve(env, precision):
    """The 16384-reactor launch: every converged reactor has ||F|| <= 1e-8 and conserves
    carbon (gas + soot) to 1e-12; eight sampled reactors (oracle in a process pool) match
    the oracle, at least six of them on the same branch."""
    batch, mech = env["batch"], env["mech"]
    t = _t(env, batch)
    out = psr.batch_solve_soot(env["gm"], t["Y_in"], t["T_in"], t["tau"], t["P"], t["M_in"], t["Y0"], t["T0"],
                               opts=psr.Options(precision=precision))
    st = out["status"].cpu().numpy()
    conv = np.isin(st, psr.CONVERGED_STATES)
    assert conv.mean() >= 0.9
    assert np.all(out["fnorm"].cpu().numpy()[conv] <= 1e-8)
    Y, T, M = out["Y"].cpu().numpy(), out["T"].cpu().numpy(), out["M"].cpu().numpy()
    _, rho, _ = O.mixture_state(mech, Y[conv], T[conv], batch.P[conv])
    gas = ((Y[conv] - batch.Y_in[conv]) / mech.W) @ mech.comp[:, 0]
    soot = (M[conv, 1] - batch.M_in[conv, 1]) / (rho * S.N_A)
    scale = ((Y[conv] + batch.Y_in[conv]) / mech.W) @ mech.comp[:, 0]
    assert np.max(np.abs(gas + soot) / scale) <= 1e-12
    idx = (3, 6, 11, 257, 1900, 4711, 9001, 16000)
    res = _oracle_roots(idx)
    compared = 0
    for b in idx:
        x, status, Mo, _ = res[(NAME, b)]
        if status != O.CONVERGED:
            continue
        assert st[b] in psr.CONVERGED_STATES, f"reactor {b}: GPU status {st[b]}, the oracle converged"
        if abs(T[b] - x[mech.K]) > 1.0:
            # another branch: it must be a root of the oracle's residual
            from tests import oracle_pool
            assert oracle_pool.root_residual(NAME, b, Y[b], T[b], M[b]) <= 1e-7, f"reactor {b}: not a root"
            continue
        big = x[:mech.K] > Y_MIN
        assert np.max(np.abs(Y[b][big] - x[:mech.K][big]) / x[:mech.K][big]) <= Y_REL
        assert abs(T[b] - x[mech.K]) <= T_ABS
        assert np.max(np.abs(M[b] - Mo) / Mo) <= M_REL
        compared += 1
    assert compared >= 6, f"only {compared} of {len(idx)} sampled sooting reactors compared within the bar"


def test_mixed_fallback_resolves_in_fp64(env):
    """PSR_MIXED with the FP64 fallback on 2048 sooting reactors (where the FP32-Jacobian
    launch leaves ~20 % unconverged): reactors the first launch converged are bit-identical
    with and without the fallback; the others are re-solved with the FP64 Jacobian
    (status PSR_REFINE_FALLBACK, counters adding up) and reach the FP64 form's root."""
    import torch
    batch = env["batch"].subset(range(2048))
    t = _t(env, batch)
    args = (env["gm"], t["Y_in"], t["T_in"], t["tau"], t["P"], t["M_in"], t["Y0"], t["T0"])
    # the fallback's first launch stops at mixed_max_newton; the same cap without fallback
    # is that launch on its own
    cap = 200                                  # the FP32 launch's default cap with soot moments
    one = psr.batch_solve_soot(*args, opts=psr.Options(precision=psr.PSR_MIXED, mixed_fallback=0, max_newton=cap))
    fb = psr.batch_solve_soot(*args, opts=psr.Options(precision=psr.PSR_MIXED, mixed_fallback=1))
    f64 = psr.batch_solve_soot(*args, opts=psr.Options(precision=psr.PSR_FP64))
    s1, sf, s64 = (o["status"].cpu().numpy() for o in (one, fb, f64))
    first = s1 == psr.PSR_CONVERGED
    assert np.all(sf[first] == psr.PSR_CONVERGED)
    keep = torch.tensor(first, device=env["dev"])
    assert torch.equal(one["Y"][keep], fb["Y"][keep]) and torch.equal(one["M"][keep], fb["M"][keep])
    redo = ~first
    assert redo.sum() >= 20, "the FP32-Jacobian launch should leave reactors to the fallback"
    assert not np.any(sf[redo] == psr.PSR_CONVERGED)
    won = sf == psr.PSR_REFINE_FALLBACK
    assert won.sum() >= 0.8 * np.sum(redo & (s64 == psr.PSR_CONVERGED))
    assert np.all(fb["fnorm"].cpu().numpy()[won] <= 1e-8)
    assert np.all(fb["iters"].cpu().numpy()[won] > one["iters"].cpu().numpy()[won])
    Yf, Y64 = fb["Y"].cpu().numpy(), f64["Y"].cpu().numpy()
    Tf, T64 = fb["T"].cpu().numpy(), f64["T"].cpu().numpy()
    Mf, M64 = fb["M"].cpu().numpy(), f64["M"].cpu().numpy()
    for b in np.flatnonzero(won & (s64 == psr.PSR_CONVERGED) & (np.abs(Tf - T64) < 1.0)):
        big = Y64[b] > Y_MIN
        assert np.max(np.abs(Yf[b][big] - Y64[b][big]) / Y64[b][big]) <= Y_REL
        assert abs(Tf[b] - T64[b]) <= T_ABS
        assert np.max(np.abs(Mf[b] - M64[b]) / M64[b]) <= M_REL
    assert np.isin(sf, psr.CONVERGED_STATES).mean() >= np.mean(s64 == psr.PSR_CONVERGED) - 0.01


def test_mixed_fallback_continues_then_restarts(env):
    """The default fallback (mixed_fallback = 2) on 2048 sooting reactors: the reactors the
    FP32-Jacobian launch leaves are first continued in FP64 from its final iterate, then
    restarted from the guess where that fails. It converges at least as many reactors as the
    restart alone (within 0.5 %), and its roots are the FP64 form's on the same branch."""
    batch = env["batch"].subset(range(2048))
    t = _t(env, batch)
    args = (env["gm"], t["Y_in"], t["T_in"], t["tau"], t["P"], t["M_in"], t["Y0"], t["T0"])
    two = psr.batch_solve_soot(*args, opts=psr.Options(precision=psr.PSR_MIXED, mixed_fallback=2))
    one = psr.batch_solve_soot(*args, opts=psr.Options(precision=psr.PSR_MIXED, mixed_fallback=1))
    f64 = psr.batch_solve_soot(*args, opts=psr.Options(precision=psr.PSR_FP64))
    s2, s1, s64 = (o["status"].cpu().numpy() for o in (two, one, f64))
    c2, c1 = np.isin(s2, psr.CONVERGED_STATES), np.isin(s1, psr.CONVERGED_STATES)
    assert c2.mean() >= c1.mean() - 0.005
    assert np.sum(s2 == psr.PSR_REFINE_FALLBACK) >= 20
    assert np.all(two["fnorm"].cpu().numpy()[c2] <= 1e-8)
    Y2, Y64 = two["Y"].cpu().numpy(), f64["Y"].cpu().numpy()
    T2, T64 = two["T"].cpu().numpy(), f64["T"].cpu().numpy()
    M2, M64 = two["M"].cpu().numpy(), f64["M"].cpu().numpy()
    both = c2 & (s64 == psr.PSR_CONVERGED) & (np.abs(T2 - T64) < 1.0)
    assert both.mean() >= 0.95
    for b in np.flatnonzero(both):
        big = Y64[b] > Y_MIN
        assert np.max(np.abs(Y2[b][big] - Y64[b][big]) / Y64[b][big]) <= Y_REL
        assert abs(T2[b] - T64[b]) <= T_ABS
        assert np.max(np.abs(M2[b] - M64[b]) / M64[b]) <= M_REL
