"""GPU parity of the block-per-reactor path (K = 200, I = 1500, 60 third-body and 40
falloff reactions; n = 201 unknowns) against the oracle: residual, Jacobian, LU beyond one
warp's 64 rows, full solves of the 2048-reactor batch (sampled against the oracle,
properties on every converged reactor) and adjoint sensitivities."""
import numpy as np
import pytest

from oracle import psr_oracle as O
from paper_2005_11468_gb300 import psr, synth
from tests.oracle_helpers import random_states, workload

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]
NAME = "k200_b2048"
Y_REL, Y_MIN, T_ABS = 1e-6, 1e-10, 1e-8


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_11468_gb300 import _build
    _build.build()
    spec, mech, batch = workload(NAME)
    return dict(dev=torch.device("cuda:0"), mech=mech, batch=batch,
                gm=psr.Mechanism(synth.mechanism_text(spec)))


def _t(env, b):
    import torch
    return {k: torch.tensor(np.ascontiguousarray(getattr(b, k)), dtype=torch.float64, device=env["dev"])
            for k in ("Y_in", "T_in", "tau", "P", "Y0", "T0")}


@pytest.mark.parametrize("energy", ["adiabatic", "fixed"])
def test_k200_residual_parity(env, energy):
    import torch
    mech, batch = env["mech"], env["batch"]
    m = 6
    X = random_states(mech, m, seed=21, y_small=True)
    sub = batch.subset(range(m))
    t = _t(env, sub)
    Yd = torch.tensor(X[:, :-1], device=env["dev"])
    Td = torch.tensor(X[:, -1], device=env["dev"])
    e = psr.PSR_FIXED_T if energy == "fixed" else psr.PSR_ADIABATIC
    F = psr.eval_residual(env["gm"], t["Y_in"], t["T_in"], t["tau"], t["P"], Yd, Td, energy=e).cpu().numpy()
    for b in range(m):
        inlet = O.inlet_of(sub, b)
        inlet.T_spec = X[b, -1]
        Fo = O.gas_residual(mech, X[b][None], inlet, energy)[0]
        _, rho, C = O.mixture_state(mech, X[b:b + 1, :-1], X[b:b + 1, -1], inlet.P)
        q = O.rates_of_progress(mech, X[b:b + 1, -1], C)[0]
        gross = np.abs(mech.nu) @ np.abs(q) * inlet.tau * mech.W / rho[0]
        scale = np.r_[1.0 + gross, 1.0 + np.max(np.abs(Fo)) + gross.max() * 50]
        err = np.abs(F[b] - Fo) / scale
        assert np.max(err) <= 1e-11, (b, np.argmax(err), F[b][np.argmax(err)], Fo[np.argmax(err)])


@pytest.mark.parametrize("precision", [psr.PSR_FP64, psr.PSR_MIXED])
def test_k200_jacobian_parity(env, precision):
    import torch
    mech, batch = env["mech"], env["batch"]
    m = 3
    X = random_states(mech, m, seed=22, y_small=True)
    sub = batch.subset(range(m))
    t = _t(env, sub)
    J = psr.eval_jacobian(env["gm"], t["Y_in"], t["T_in"], t["tau"], t["P"],
                          torch.tensor(X[:, :-1], device=env["dev"]), torch.tensor(X[:, -1], device=env["dev"]),
                          precision=precision).cpu().numpy()
    tol = 1e-8 if precision == psr.PSR_FP64 else 5e-5
    for b in range(m):
        Jo = O.jacobian_cs(O.GasSystem(mech, O.inlet_of(sub, b)), X[b])
        err = np.abs(J[b] - Jo) / np.max(np.abs(Jo), axis=1, keepdims=True)
        assert np.max(err) <= tol, (b, np.unravel_index(np.argmax(err), err.shape), np.max(err))


@pytest.mark.parametrize("n", [65, 130, 201, 256, 512])
def test_block_lu_parity(env, n):
    """Rows beyond one warp: same pivots and solution as the oracle's LAPACK-order LU;
    the FP32 form to its backward-error bound. n = 512 holds the matrix in global slots."""
    import torch
    rng = np.random.Generator(np.random.PCG64(1000 + n))
    B = 5
    A = rng.standard_normal((B, n, n)) * np.exp(rng.uniform(-4, 4, (B, n, 1)))
    r = rng.standard_normal((B, n))
    x, ok = psr.batch_lu_solve(torch.tensor(A, device=env["dev"]), torch.tensor(r, device=env["dev"]), psr.PSR_FP64)
    x, ok = x.cpu().numpy(), ok.cpu().numpy()
    assert np.all(ok == 1)
    for b in range(B):
        LU, piv, good = O.lu_factor(A[b])
        xo = O.lu_solve(LU, piv, r[b])
        np.testing.assert_allclose(x[b], xo, rtol=1e-8, atol=1e-11 * np.abs(xo).max())
    xm, okm = psr.batch_lu_solve(torch.tensor(A, device=env["dev"]), torch.tensor(r, device=env["dev"]),
                                 psr.PSR_MIXED)
    xm = xm.cpu().numpy()
    assert np.all(okm.cpu().numpy() == 1)
    for b in range(B):
        res = np.abs(A[b] @ xm[b] - r[b]).max() / (np.abs(A[b]).max() * np.abs(xm[b]).max() + np.abs(r[b]).max())
        assert res <= 1e-5 * n


_REF = {}
_POOL = {}


def _oracle_pool(idx):
    key = tuple(idx)
    if key not in _POOL:
        from tests import oracle_pool
        _POOL[key] = oracle_pool.solve([(NAME, b) for b in idx])
    return _POOL[key]


def _oracle(env, idx):
    key = tuple(idx)
    if key not in _REF:
        _REF[key] = O.solve_batch(env["mech"], env["batch"], indices=list(idx))
    return _REF[key]


@pytest.mark.parametrize("precision", [psr.PSR_FP64, psr.PSR_MIXED])
def test_k200_full_size_solve(env, precision):
    """The 2048-reactor launch the benchmark times: every converged reactor has
    ||F|| <= 1e-8 and conserves elements to 1e-12; eight sampled reactors (oracle in a
    process pool) match the oracle, at least six on the same branch."""
    mech, batch = env["mech"], env["batch"]
    t = _t(env, batch)
    out = psr.batch_solve(env["gm"], t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"],
                          opts=psr.Options(precision=precision))
    st = out["status"].cpu().numpy()
    conv = np.isin(st, psr.CONVERGED_STATES)
    assert conv.mean() >= 0.8
    assert np.all(out["fnorm"].cpu().numpy()[conv] <= 1e-8)
    Y, T = out["Y"].cpu().numpy(), out["T"].cpu().numpy()
    elem = ((Y[conv] - batch.Y_in[conv]) / mech.W) @ mech.comp
    assert np.max(np.abs(elem)) <= 1e-12
    idx = [0, 1, 97, 500, 1024, 1500, 1999, 2047]
    res = _oracle_pool(idx)
    compared = 0
    for b in idx:
        x, status, _, _ = res[(NAME, b)]
        if status != O.CONVERGED:
            continue
        assert st[b] in psr.CONVERGED_STATES
        if abs(T[b] - x[-1]) > 1.0:
            Fo = O.gas_residual(mech, np.r_[Y[b], T[b]][None], O.inlet_of(batch, b))[0]
            assert np.max(np.abs(Fo)) <= 1e-7
            continue
        big = x[:-1] > Y_MIN
        assert np.max(np.abs(Y[b][big] - x[:-1][big]) / x[:-1][big]) <= Y_REL
        assert abs(T[b] - x[-1]) <= T_ABS
        compared += 1
    assert compared >= 6, f"only {compared} of {len(idx)} sampled K = 200 reactors compared"


def test_k200_adjoint(env):
    """At K = 200 the Jacobian at a root can have a condition number near 1e16 (a reaction
    faster than the residence time by 13 orders next to trace species), so lambda is not
    compared element by element. Instead: lambda solves J^T lambda = g to FP64 backward
    error (the oracle's complex-step J), and the gradient equals the oracle's
    -dF/d ln m^T lambda for that lambda, entry by entry at its rounding scale."""
    import torch
    mech, batch = env["mech"], env["batch"]
    idx = [0, 1, 2]
    sub = batch.subset(idx)
    t = _t(env, sub)
    out = psr.batch_solve(env["gm"], t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"])
    g = np.random.Generator(np.random.PCG64(2)).standard_normal((len(idx), mech.K + 1))
    grad, lam, ok = psr.batch_adjoint(env["gm"], t["Y_in"], t["T_in"], t["tau"], t["P"], out["Y"], out["T"],
                                      torch.tensor(g, device=env["dev"]))
    grad, lam, ok = grad.cpu().numpy(), lam.cpu().numpy(), ok.cpu().numpy()
    Y, T, st = out["Y"].cpu().numpy(), out["T"].cpu().numpy(), out["status"].cpu().numpy()
    checked = 0
    for j in range(len(idx)):
        if st[j] != 0:
            continue
        assert ok[j] == 1
        x = np.r_[Y[j], T[j]]
        inlet = O.inlet_of(sub, j)
        J = O.jacobian_cs(O.GasSystem(mech, inlet), x)
        res = np.abs(J.T @ lam[j] - g[j]).max()
        scale = np.abs(J.T).sum(axis=1).max() * np.abs(lam[j]).max() + np.abs(g[j]).max()
        assert res <= 1e-12 * scale, (j, res / scale)
        Fp = O.rate_parameter_jacobian(mech, inlet, x)
        go = -Fp.T @ lam[j]
        rnd = np.abs(Fp.T) @ np.abs(lam[j])
        bound = 1e-12 * rnd + 1e-14 * rnd.max()
        assert np.all(np.abs(grad[j] - go) <= bound), (j, np.max(np.abs(grad[j] - go) - bound))
        checked += 1
    assert checked >= 1


@pytest.mark.parametrize("K", [63, 64])
def test_warp_block_boundary(env, K):
    """K + 1 = 64 is the largest system of the warp-per-reactor path and K + 1 = 65 the
    smallest of the block-per-reactor path: both solve to the oracle's roots."""
    import torch
    spec = synth.make_mechanism(K, 4 * K, n_tb=4, n_troe=4, seed=synth.MECH_SEED_BASE + 700 + K)
    text = synth.mechanism_text(spec)
    mech, gm = O.Mechanism(text), psr.Mechanism(text)
    batch = synth.make_batch(spec, 8, seed=synth.MECH_SEED_BASE + 701 + K)
    t = _t(env, batch)
    for prec in (psr.PSR_FP64, psr.PSR_MIXED):
        out = psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"],
                              opts=psr.Options(precision=prec))
        st, Y, T = out["status"].cpu().numpy(), out["Y"].cpu().numpy(), out["T"].cpu().numpy()
        assert np.isin(st, psr.CONVERGED_STATES).mean() >= 0.75
        for b in (0, 1):
            r = O.solve_reactor(mech, O.inlet_of(batch, b), np.r_[batch.Y0[b], batch.T0[b]])
            if r.status != O.CONVERGED or abs(T[b] - r.x[-1]) > 1.0:
                continue
            assert st[b] in psr.CONVERGED_STATES
            big = r.x[:-1] > Y_MIN
            assert np.max(np.abs(Y[b][big] - r.x[:-1][big]) / r.x[:-1][big]) <= Y_REL
            assert abs(T[b] - r.x[-1]) <= T_ABS


def test_k200_autotune_and_block_threads(env):
    """psr_autotune on 608 reactors of the K = 200 batch picks one of its block-path shapes
    (512 or 256 threads per reactor, 0-2 blocks per SM); the 256-thread solver on the same
    reactors converges as the 512-thread one does and reaches the same roots within the bar,
    in both forms."""
    import torch
    batch = env["batch"].subset(range(608))
    t = _t(env, batch)
    args = (env["gm"], t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"])
    tuned = psr.autotune(*args, opts=psr.Options(precision=psr.PSR_MIXED))
    assert (tuned.path, tuned.warps_per_block) == (psr.PSR_PATH_BLOCK, 0)
    assert tuned.block_threads in (256, 512) and tuned.blocks_per_sm in (0, 1, 2)
    for prec in (psr.PSR_FP64, psr.PSR_MIXED):
        a = psr.batch_solve(*args, opts=psr.Options(precision=prec, block_threads=512))
        b = psr.batch_solve(*args, opts=psr.Options(precision=prec, block_threads=256))
        ca = np.isin(a["status"].cpu().numpy(), psr.CONVERGED_STATES)
        cb = np.isin(b["status"].cpu().numpy(), psr.CONVERGED_STATES)
        assert cb.mean() >= 0.99 and np.sum(ca != cb) <= 3
        Ta, Tb = a["T"].cpu().numpy(), b["T"].cpu().numpy()
        both = ca & cb & (np.abs(Ta - Tb) <= 1.0)
        assert both.mean() >= 0.98
        Ya, Yb = a["Y"].cpu().numpy()[both], b["Y"].cpu().numpy()[both]
        big = Ya > Y_MIN
        assert (np.abs(Yb - Ya)[big] / Ya[big]).max() <= Y_REL
        assert np.abs(Ta[both] - Tb[both]).max() <= T_ABS
    with pytest.raises(psr.PsrError):
        psr.batch_solve(*args, opts=psr.Options(block_threads=300))
