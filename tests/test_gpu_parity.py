"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by element,
on seeded inputs (residual, Jacobian, LU, full solves), plus edge cases and properties
that hold at any size (element conservation, residual norm) for the full batches."""
import math

import numpy as np
import pytest

from oracle import psr_oracle as O
from paper_2005_11468_gb300 import psr, synth
from tests.oracle_helpers import golden_text, random_states, workload

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

Y_REL, Y_MIN, T_ABS = 1e-6, 1e-10, 1e-8        # parity bar: Y_k > 1e-10 to 1e-6 relative, T to 1e-8 K


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_11468_gb300 import _build
    _build.build()
    return torch.device("cuda:0")


_MECH = {}


def gpu_mech(name):
    if name not in _MECH:
        spec, _, _ = workload(name)
        _MECH[name] = psr.Mechanism(synth.mechanism_text(spec))
    return _MECH[name]


def to_dev(batch, dev):
    import torch
    return {k: torch.tensor(np.ascontiguousarray(getattr(batch, k)), dtype=torch.float64, device=dev)
            for k in ("Y_in", "T_in", "tau", "P", "Y0", "T0")}


_ORACLE = {}


def oracle_solution(name, indices, energy="adiabatic"):
    key = (name, tuple(indices), energy)
    if key not in _ORACLE:
        _, mech, batch = workload(name)
        _ORACLE[key] = O.solve_batch(mech, batch, energy=energy, indices=list(indices))
    return _ORACLE[key]


def oracle_solution_pool(name, indices):
    """oracle_solution computed in a spawn process pool (one reactor per task)."""
    key = (name, tuple(indices), "adiabatic")
    if key not in _ORACLE:
        from tests import oracle_pool
        res = oracle_pool.solve([(name, b) for b in indices])
        _ORACLE[key] = {"status": np.array([res[(name, b)][1] for b in indices]),
                        "Y": np.stack([res[(name, b)][0][:-1] for b in indices]),
                        "T": np.array([res[(name, b)][0][-1] for b in indices])}
    return _ORACLE[key]


def compare_roots(name, idx, ref, Y, T, st, what):
    """Parity on reactors the oracle converged: same status, Y and T within the bar; a
    different branch (|dT| > 1 K) counts only if the GPU state is a root of the oracle."""
    _, mech, batch = workload(name)
    n_ok = n_branch = 0
    for j, b in enumerate(idx):
        if ref["status"][j] != O.CONVERGED:
            continue
        assert st[j] in psr.CONVERGED_STATES, f"{what}: reactor {b} status {st[j]} (oracle converged)"
        if abs(T[j] - ref["T"][j]) > 1.0:
            F = O.gas_residual(mech, np.r_[Y[j], T[j]][None], O.inlet_of(batch, b))[0]
            assert np.max(np.abs(F)) <= 1e-7, f"{what}: reactor {b} on another branch and not a root"
            n_branch += 1
            continue
        big = ref["Y"][j] > Y_MIN
        rel = np.max(np.abs(Y[j][big] - ref["Y"][j][big]) / ref["Y"][j][big])
        assert rel <= Y_REL, f"{what}: reactor {b} Y rel err {rel:.3e}"
        assert abs(T[j] - ref["T"][j]) <= T_ABS, f"{what}: reactor {b} T err {T[j] - ref['T'][j]:.3e}"
        n_ok += 1
    return n_ok, n_branch


# ------------------------------------------------------------------ residual, Eqs. (2)-(9)
@pytest.mark.parametrize("name", ["k10_b64", "k53_b4096"])
@pytest.mark.parametrize("energy", ["adiabatic", "fixed"])
def test_residual_parity(dev, name, energy):
    import torch
    _, mech, batch = workload(name)
    m = 40
    X = random_states(mech, m, seed=11, y_small=True)
    sub = batch.subset(range(m))
    t = to_dev(sub, dev)
    Yd = torch.tensor(X[:, :-1], dtype=torch.float64, device=dev)
    Td = torch.tensor(X[:, -1], dtype=torch.float64, device=dev)
    e = psr.PSR_FIXED_T if energy == "fixed" else psr.PSR_ADIABATIC
    F = psr.eval_residual(gpu_mech(name), t["Y_in"], t["T_in"], t["tau"], t["P"], Yd, Td, energy=e).cpu().numpy()
    for b in range(m):
        inlet = O.inlet_of(sub, b)
        inlet.T_spec = X[b, -1]
        Fo = O.gas_residual(mech, X[b][None], inlet, energy)[0]
        # rounding scale: the gross production terms that cancel in each row
        _, rho, C = O.mixture_state(mech, X[b:b + 1, :-1], X[b:b + 1, -1], inlet.P)
        q = O.rates_of_progress(mech, X[b:b + 1, -1], C)[0]
        gross = np.abs(mech.nu) @ np.abs(q) * inlet.tau * mech.W / rho[0]
        scale = np.r_[1.0 + gross, 1.0 + np.max(np.abs(Fo)) + gross.max() * 50]
        err = np.abs(F[b] - Fo) / scale
        assert np.max(err) <= 1e-11, (b, np.argmax(err), F[b][np.argmax(err)], Fo[np.argmax(err)])


# ------------------------------------------------------------------ Jacobian
@pytest.mark.parametrize("name", ["k10_b64", "k53_b4096"])
@pytest.mark.parametrize("precision", [psr.PSR_FP64, psr.PSR_MIXED])
def test_jacobian_parity(dev, name, precision):
    import torch
    _, mech, batch = workload(name)
    m = 12
    X = random_states(mech, m, seed=12, y_small=True)
    sub = batch.subset(range(m))
    t = to_dev(sub, dev)
    Yd = torch.tensor(X[:, :-1], dtype=torch.float64, device=dev)
    Td = torch.tensor(X[:, -1], dtype=torch.float64, device=dev)
    J = psr.eval_jacobian(gpu_mech(name), t["Y_in"], t["T_in"], t["tau"], t["P"], Yd, Td,
                          precision=precision).cpu().numpy()
    tol = 1e-8 if precision == psr.PSR_FP64 else 2e-5
    for b in range(m):
        S = O.GasSystem(mech, O.inlet_of(sub, b))
        Jo = O.jacobian_cs(S, X[b])
        rowmax = np.max(np.abs(Jo), axis=1, keepdims=True)
        err = np.abs(J[b] - Jo) / rowmax
        assert np.max(err) <= tol, (b, np.unravel_index(np.argmax(err), err.shape), np.max(err))


# ------------------------------------------------------------------ LU
@pytest.mark.parametrize("n", [1, 11, 33, 54, 64])
def test_lu_parity(dev, n):
    import torch
    rng = np.random.Generator(np.random.PCG64(n))
    B = 37
    A = rng.standard_normal((B, n, n)) * np.exp(rng.uniform(-4, 4, (B, n, 1))) + 0 * np.eye(n)
    r = rng.standard_normal((B, n))
    x, ok = psr.batch_lu_solve(torch.tensor(A, device=dev), torch.tensor(r, device=dev), psr.PSR_FP64)
    x, ok = x.cpu().numpy(), ok.cpu().numpy()
    assert np.all(ok == 1)
    for b in range(B):
        LU, piv, good = O.lu_factor(A[b])
        xo = O.lu_solve(LU, piv, r[b])
        np.testing.assert_allclose(x[b], xo, rtol=1e-9, atol=1e-12 * np.abs(xo).max())
    xm, okm = psr.batch_lu_solve(torch.tensor(A, device=dev), torch.tensor(r, device=dev), psr.PSR_MIXED)
    xm = xm.cpu().numpy()
    for b in range(B):
        res = np.abs(A[b] @ xm[b] - r[b]).max() / (np.abs(A[b]).max() * np.abs(xm[b]).max() + np.abs(r[b]).max())
        assert res <= 1e-5 * n


def test_lu_singular(dev):
    import torch
    A = np.zeros((2, 3, 3))
    A[0] = np.eye(3)
    A[1] = [[1, 2, 3], [2, 4, 6], [1, 1, 1]]
    x, ok = psr.batch_lu_solve(torch.tensor(A, device=dev), torch.ones((2, 3), dtype=torch.float64, device=dev))
    assert ok.cpu().tolist() == [1, 0]


# ------------------------------------------------------------------ full solves
@pytest.mark.parametrize("precision", [psr.PSR_FP64, psr.PSR_MIXED])
def test_solve_parity_k10_full_batch(dev, precision):
    _, mech, batch = workload("k10_b64")
    idx = list(range(batch.B))
    ref = oracle_solution("k10_b64", idx)
    t = to_dev(batch, dev)
    out = psr.batch_solve(gpu_mech("k10_b64"), t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"],
                          opts=psr.Options(precision=precision))
    Y, T, st = out["Y"].cpu().numpy(), out["T"].cpu().numpy(), out["status"].cpu().numpy()
    n_ok, n_branch = compare_roots("k10_b64", idx, ref, Y, T, st, f"k10 prec={precision}")
    assert n_ok >= 0.9 * np.sum(ref["status"] == O.CONVERGED)
    fn = out["fnorm"].cpu().numpy()
    assert np.all(fn[np.isin(st, psr.CONVERGED_STATES)] <= 1e-8)


@pytest.mark.parametrize("precision", [psr.PSR_FP64, psr.PSR_MIXED])
def test_solve_parity_k53_full_size_sampled(dev, precision):
    """The B = 4096 launch the benchmark times; 32 sampled reactors against the oracle,
    element conservation and ||F|| for every converged reactor."""
    _, mech, batch = workload("k53_b4096")
    t = to_dev(batch, dev)
    out = psr.batch_solve(gpu_mech("k53_b4096"), t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"],
                          opts=psr.Options(precision=precision))
    Y, T, st = out["Y"].cpu().numpy(), out["T"].cpu().numpy(), out["status"].cpu().numpy()
    conv = np.isin(st, psr.CONVERGED_STATES)
    assert conv.mean() >= 0.8
    assert np.all(out["fnorm"].cpu().numpy()[conv] <= 1e-8)
    elem = ((Y[conv] - batch.Y_in[conv]) / mech.W) @ mech.comp
    assert np.max(np.abs(elem)) <= 1e-12
    idx = [int(i) for i in np.random.Generator(np.random.PCG64(5)).choice(batch.B, 32, replace=False)]
    ref = oracle_solution_pool("k53_b4096", idx)
    n_ok, n_branch = compare_roots("k53_b4096", idx, ref, Y[idx], T[idx], st[idx], f"k53 prec={precision}")
    assert n_ok >= 28, f"only {n_ok} of 32 sampled reactors compared within the bar"


def test_mixed_fallback_through_the_block_solver_k53(dev):
    """The mixed form's FP64 re-solve of the reactors its FP32-Jacobian launch left runs one
    block per reactor (n = 54 here, below the sizes the block solver otherwise takes): with
    the FP32 launch capped at 40 iterations most reactors take that path, and the sampled
    ones match the oracle."""
    _, mech, batch = workload("k53_b4096")
    t = to_dev(batch, dev)
    out = psr.batch_solve(gpu_mech("k53_b4096"), t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"],
                          opts=psr.Options(precision=psr.PSR_MIXED, mixed_max_newton=40))
    Y, T, st = out["Y"].cpu().numpy(), out["T"].cpu().numpy(), out["status"].cpu().numpy()
    assert np.mean(st == psr.PSR_REFINE_FALLBACK) >= 0.5
    conv = np.isin(st, psr.CONVERGED_STATES)
    assert conv.mean() >= 0.999
    assert np.all(out["fnorm"].cpu().numpy()[conv] <= 1e-8)
    idx = [int(i) for i in np.random.Generator(np.random.PCG64(5)).choice(batch.B, 6, replace=False)]
    ref = oracle_solution("k53_b4096", idx)
    assert np.any(st[idx] == psr.PSR_REFINE_FALLBACK)
    compare_roots("k53_b4096", idx, ref, Y[idx], T[idx], st[idx], "k53 block re-solve")


def test_fixed_temperature_closed_forms(dev):
    """Golden isomerisation and dimerisation (fixed T) against their closed forms."""
    import torch
    mech = psr.Mechanism(golden_text("isomer_ab.psrmech"))
    T, tau = 1500.0, 1e-3
    Y_in = np.array([[0.5, 0.4, 0.1]])
    args = [torch.tensor(v, dtype=torch.float64, device=dev) for v in
            (Y_in, [500.0], [tau], [synth.ONE_ATM], Y_in, [T])]
    for prec in (psr.PSR_FP64, psr.PSR_MIXED):
        out = psr.batch_solve(mech, *args, opts=psr.Options(energy=psr.PSR_FIXED_T, precision=prec))
        kf = 1000.0
        kr = kf / math.exp((5.5 - 6.0) - (1500.0 - 2000.0) / T)
        YA = (0.4 + tau * kr * 0.5) / (1 + tau * (kf + kr))
        assert out["status"].item() == 0
        np.testing.assert_allclose(out["Y"][0, 1].item(), YA, rtol=1e-12)
        assert out["T"].item() == T


@pytest.mark.parametrize("fixture", ["troe_isomer.psrmech", "troe_t2_isomer.psrmech"])
def test_falloff_closed_forms(dev, fixture):
    """The falloff isomerisation fixtures at the centre of the Troe curve (F = F_cent =
    1/2, made by the T*** term or by the four-parameter T** term alone) against their
    closed form, in both forms: k_f = k_inf P_r / (1 + P_r) / 2, k_r = k_f / K_c."""
    import torch
    mech = psr.Mechanism(golden_text(fixture))
    T, tau, P = 1500.0, 1e-3, synth.ONE_ATM
    Y_in = np.array([[0.5, 0.4, 0.1]])
    args = [torch.tensor(v, dtype=torch.float64, device=dev) for v in (Y_in, [500.0], [tau], [P], Y_in, [T])]
    W = O.Mechanism(golden_text(fixture)).W          # element-weight sums of the file's compositions
    S = 0.5
    rho = P / (O.R_U * T) / (0.5 / W[0] + S / W[1])
    M = 2.0 * rho * 0.5 / W[0] + rho * S / W[1]
    Pr = 257582561.28170544 * M / 2000.0
    kf = 2000.0 * Pr / (1.0 + Pr) * 0.5
    kr = kf / math.exp((5.5 - 6.0) - (1500.0 - 2000.0) / T)
    YA = (0.4 + tau * kr * S) / (1.0 + tau * (kf + kr))
    for prec in (psr.PSR_FP64, psr.PSR_MIXED):
        out = psr.batch_solve(mech, *args, opts=psr.Options(energy=psr.PSR_FIXED_T, precision=prec))
        assert out["status"].item() == 0
        np.testing.assert_allclose(out["Y"][0, 1].item(), YA, rtol=1e-12)
        np.testing.assert_allclose(out["Y"][0, 2].item(), S - YA, rtol=1e-12)


def test_rate_multipliers(dev):
    """rate_mult = 1 equals NULL; a perturbed multiplier vector matches the oracle's."""
    import torch
    _, mech, batch = workload("k10_b64")
    idx = list(range(8))
    sub = batch.subset(idx)
    t = to_dev(sub, dev)
    gm = gpu_mech("k10_b64")
    det = psr.Options(handoff=0)          # bit-reproducible: no timing-dependent handoff
    a = psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"], opts=det)
    ones = torch.ones(mech.I, dtype=torch.float64, device=dev)
    b = psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"], rate_mult=ones, opts=det)
    assert torch.equal(a["Y"], b["Y"]) and torch.equal(a["T"], b["T"])
    lnm = np.random.Generator(np.random.PCG64(3)).uniform(-0.5, 0.5, mech.I)
    c = psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"],
                        rate_mult=torch.tensor(np.exp(lnm), device=dev))
    compared = 0
    for j, bi in enumerate(idx):
        r = O.solve_reactor(mech, O.inlet_of(sub, j), np.r_[sub.Y0[j], sub.T0[j]], lnmult=lnm)
        if r.status == O.CONVERGED and c["status"][j].item() == 0 and abs(c["T"][j].item() - r.x[-1]) < 1:
            big = r.x[:-1] > Y_MIN
            Yg = c["Y"][j].cpu().numpy()
            assert np.max(np.abs(Yg[big] - r.x[:-1][big]) / r.x[:-1][big]) <= Y_REL
            assert abs(c["T"][j].item() - r.x[-1]) <= T_ABS
            compared += 1
    assert compared >= 6, f"only {compared} of 8 reactors compared with perturbed multipliers"


def test_host_entry_matches_device(dev):
    _, mech, batch = workload("k10_b64")
    sub = batch.subset(range(16))
    t = to_dev(sub, dev)
    gm = gpu_mech("k10_b64")
    det = psr.Options(handoff=0)          # bit-reproducible: no timing-dependent handoff
    a = psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"], opts=det)
    h = psr.batch_solve_host(gm, sub.Y_in, sub.T_in, sub.tau, sub.P, sub.Y0, sub.T0, opts=det)
    np.testing.assert_array_equal(h["Y"], a["Y"].cpu().numpy())
    np.testing.assert_array_equal(h["status"], a["status"].cpu().numpy())


def test_edge_cases(dev):
    import torch
    _, mech, batch = workload("k10_b64")
    gm = gpu_mech("k10_b64")
    # empty batch: nothing launched, success
    e = to_dev(batch.subset([]), dev)
    out = psr.batch_solve(gm, e["Y_in"], e["T_in"], e["tau"], e["P"], e["Y0"], e["T0"])
    assert out["Y"].shape == (0, mech.K)
    # ragged sizes give the same per-reactor answers as the full batch (without the
    # timing-dependent handoff of stragglers, the warp path is bit-reproducible)
    det = psr.Options(handoff=0)
    full = to_dev(batch, dev)
    ref = psr.batch_solve(gm, full["Y_in"], full["T_in"], full["tau"], full["P"], full["Y0"], full["T0"], opts=det)
    for B in (1, 3, 33):
        s = to_dev(batch.subset(range(B)), dev)
        o = psr.batch_solve(gm, s["Y_in"], s["T_in"], s["tau"], s["P"], s["Y0"], s["T0"], opts=det)
        assert torch.equal(o["Y"], ref["Y"][:B]) and torch.equal(o["status"], ref["status"][:B])
    # tau -> 0: outlet = inlet
    s = to_dev(batch.subset(range(8)), dev)
    s["tau"] = torch.full_like(s["tau"], 1e-20)
    o = psr.batch_solve(gm, s["Y_in"], s["T_in"], s["tau"], s["P"], s["Y0"], s["T0"])
    assert torch.all(o["status"] == 0)
    torch.testing.assert_close(o["Y"], s["Y_in"], rtol=0, atol=1e-10)
    torch.testing.assert_close(o["T"], s["T_in"], rtol=1e-9, atol=0)
    # non-finite initial guess is reported per reactor, not as a call error
    bad = {k: v.clone() for k, v in s.items()}
    bad["T0"][2] = float("nan")
    o = psr.batch_solve(gm, bad["Y_in"], bad["T_in"], bad["tau"], bad["P"], bad["Y0"], bad["T0"])
    assert o["status"][2].item() == psr.PSR_NONFINITE
    # invalid options are call errors
    with pytest.raises(psr.PsrError):
        psr.batch_solve(gm, s["Y_in"], s["T_in"], s["tau"], s["P"], s["Y0"], s["T0"], opts=psr.Options(ftol=-1))



def test_autotune_picks_a_shape_with_identical_results(dev):
    """psr_autotune returns one of its candidate launch shapes; solving with it gives the
    default shape's results: bit for bit where the warp solver converged in both (one warp
    per reactor either way) when it keeps the warp path, and to the parity bar otherwise
    (the block path and the FP64 re-solve sum the Jacobian's contributions with
    shared-memory atomics from several warps, in an order that varies)."""
    import torch
    _, mech, batch = workload("k53_b4096")
    sub = batch.subset(range(1024))
    t = to_dev(sub, dev)
    gm = gpu_mech("k53_b4096")
    base = psr.Options(precision=psr.PSR_MIXED, handoff=0)
    tuned = psr.autotune(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"], base)
    shapes = {(psr.PSR_PATH_WARP, w, b, 0) for w, b in ((1, 0), (2, 0), (3, 0), (4, 0), (2, 2), (2, 3), (2, 4))}
    shapes |= {(psr.PSR_PATH_BLOCK, 0, 0, 512), (psr.PSR_PATH_BLOCK, 0, 0, 256)}
    assert (tuned.path, tuned.warps_per_block, tuned.blocks_per_sm, tuned.block_threads) in shapes
    assert tuned.precision == base.precision and tuned.ftol == base.ftol
    a = psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"], opts=base)
    b = psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"], opts=tuned)
    sa, sb = a["status"].cpu().numpy(), b["status"].cpu().numpy()
    ca, cb = np.isin(sa, psr.CONVERGED_STATES), np.isin(sb, psr.CONVERGED_STATES)
    assert cb.mean() >= 0.99 and np.sum(ca != cb) <= 4
    both = ca & cb
    if tuned.path == psr.PSR_PATH_WARP:
        warp = (sa == psr.PSR_CONVERGED) & (sb == psr.PSR_CONVERGED)
        assert warp.mean() >= 0.95
        assert torch.equal(a["Y"][torch.from_numpy(warp).to(dev)], b["Y"][torch.from_numpy(warp).to(dev)])
    Ya, Yb = a["Y"].cpu().numpy()[both], b["Y"].cpu().numpy()[both]
    same = np.abs(a["T"].cpu().numpy()[both] - b["T"].cpu().numpy()[both]) <= 1.0
    assert same.mean() >= 0.99
    Ya, Yb = Ya[same], Yb[same]
    big = Ya > Y_MIN
    assert np.max(np.where(big, np.abs(Yb - Ya) / np.where(big, Ya, 1.0), 0.0)) <= Y_REL
    with pytest.raises(psr.PsrError):
        psr.autotune(gm, t["Y_in"][:0], t["T_in"][:0], t["tau"][:0], t["P"][:0], t["Y0"][:0], t["T0"][:0])


@pytest.mark.parametrize("block_threads", [512, 256])
@pytest.mark.parametrize("precision", [psr.PSR_FP64, psr.PSR_MIXED])
def test_block_path_on_the_k53_batch(dev, precision, block_threads):
    """The same 4096-reactor K = 53 batch with one block of 512 or 256 threads per reactor
    (the path larger mechanisms take) instead of one warp: every converged reactor has
    ||F|| <= 1e-8 and conserves elements, 32 sampled reactors match the oracle."""
    _, mech, batch = workload("k53_b4096")
    t = to_dev(batch, dev)
    out = psr.batch_solve(gpu_mech("k53_b4096"), t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"],
                          opts=psr.Options(precision=precision, path=psr.PSR_PATH_BLOCK,
                                           block_threads=block_threads))
    Y, T, st = out["Y"].cpu().numpy(), out["T"].cpu().numpy(), out["status"].cpu().numpy()
    conv = np.isin(st, psr.CONVERGED_STATES)
    assert conv.mean() >= 0.99
    assert np.all(out["fnorm"].cpu().numpy()[conv] <= 1e-8)
    elem = ((Y[conv] - batch.Y_in[conv]) / mech.W) @ mech.comp
    assert np.max(np.abs(elem)) <= 1e-12
    idx = [int(i) for i in np.random.Generator(np.random.PCG64(5)).choice(batch.B, 32, replace=False)]
    ref = oracle_solution_pool("k53_b4096", idx)          # the sample of the warp-path test (cached)
    n_ok, _ = compare_roots("k53_b4096", idx, ref, Y[idx], T[idx], st[idx], f"k53 block path prec={precision} bt={block_threads}")
    assert n_ok >= 28


@pytest.mark.parametrize("name", ["k53_b4096", "k200_b2048"])
def test_eval_rates_match_oracle(dev, name):
    """psr_eval_rates (the paper's timed unit: k_f, K_c -> k_r, q, wdot) against the
    oracle's Eqs. (4)-(9) at seeded states, on the warp (K = 53) and block (K = 200) paths."""
    import torch
    _, mech, batch = workload(name)
    m = 8
    X = random_states(mech, m, seed=31)
    P = np.full(m, synth.ONE_ATM)
    gm = gpu_mech(name)
    lnm = np.random.Generator(np.random.PCG64(4)).uniform(-0.3, 0.3, mech.I)
    out = psr.eval_rates(gm, torch.tensor(X[:, :-1], device=dev), torch.tensor(X[:, -1], device=dev),
                         torch.tensor(P, device=dev), rate_mult=torch.tensor(np.exp(lnm), device=dev))
    kf, kr, q, wd = (out[k].cpu().numpy() for k in ("kf", "kr", "q", "wdot"))
    T = X[:, -1]
    _, rho, C = O.mixture_state(mech, X[:, :-1], T, P)
    q_o = O.rates_of_progress(mech, T, C, lnmult=lnm)
    wd_o = O.net_production_rates(mech, q_o)
    kf_o = O.forward_rate_constants(mech, T)
    Kc_o = O.equilibrium_constants(mech, T)
    plain = ~mech.is_troe
    np.testing.assert_allclose(kf[:, plain], kf_o[:, plain], rtol=1e-12)
    np.testing.assert_allclose(kf / kr, np.broadcast_to(Kc_o, kf.shape), rtol=1e-10)
    gross = np.abs(q_o).max(axis=1, keepdims=True)
    assert np.max(np.abs(q - q_o) / gross) <= 1e-11
    scale = (np.abs(q_o) @ np.abs(mech.nu.T)).max(axis=1, keepdims=True)
    assert np.max(np.abs(wd - wd_o) / scale) <= 1e-11


def test_fixed_t_sweep_with_continuation(dev):
    """The paper's run mode: a fixed-T grid (1500-2000 K in 50 K steps x tau 5-95 ms in
    5 ms steps) solved column by column with the previous temperature's roots as guesses.
    Warm and cold starts reach the same roots where both converge on the same branch,
    continuation needs fewer Newton iterations in all, and two grid points match the
    oracle."""
    from paper_2005_11468_gb300 import sweep
    spec, mech, batch = workload("k53_b4096")
    gm = gpu_mech("k53_b4096")
    Y_in = batch.Y_in[0]
    T_grid = np.arange(1500.0, 2001.0, 50.0)
    tau_grid = np.arange(5e-3, 95.1e-3, 5e-3)
    Yw, sw, iw = sweep.fixed_t_sweep(gm, Y_in, T_grid, tau_grid, warm=True)
    Yc, sc, ic = sweep.fixed_t_sweep(gm, Y_in, T_grid, tau_grid, warm=False)
    cw, cc = np.isin(sw, psr.CONVERGED_STATES), np.isin(sc, psr.CONVERGED_STATES)
    assert cw.mean() >= 0.95 and cc.mean() >= 0.95
    both = cw & cc
    big = Yc > Y_MIN
    rel = np.where(big, np.abs(Yw - Yc) / np.where(big, Yc, 1.0), 0.0).max(axis=2)
    assert np.mean(rel[both] <= Y_REL) >= 0.95     # other points sit on another root (a valid one)
    assert iw[both].sum() < ic[both].sum()
    for a, j in ((0, 0), (len(T_grid) - 1, len(tau_grid) - 1)):
        inlet = O.Inlet(Y_in, 300.0, tau_grid[j], synth.ONE_ATM)
        inlet.T_spec = T_grid[a]
        r = O.solve_reactor(mech, inlet, np.r_[Y_in, T_grid[a]], energy="fixed")
        assert r.status == O.CONVERGED
        big = r.x[:-1] > Y_MIN
        assert np.max(np.abs(Yc[a, j][big] - r.x[:-1][big]) / r.x[:-1][big]) <= Y_REL


@pytest.mark.parametrize("name", ["k10_b64", "k53_b4096"])
def test_fd_jacobian_matches_oracle_differences(dev, name):
    """psr_eval_jacobian_fd (the paper's finite-difference Jacobian; mass-fraction columns
    with frozen rate constants) against the oracle's central differences with the same
    steps, and against the analytic Jacobian to the differences' truncation level."""
    import torch
    _, mech, batch = workload(name)
    m = 6
    X = random_states(mech, m, seed=41)
    sub = batch.subset(range(m))
    t = to_dev(sub, dev)
    Yd = torch.tensor(X[:, :-1], device=dev)
    Td = torch.tensor(X[:, -1], device=dev)
    Jf = psr.eval_jacobian_fd(gpu_mech(name), t["Y_in"], t["T_in"], t["tau"], t["P"], Yd, Td).cpu().numpy()
    Ja = psr.eval_jacobian(gpu_mech(name), t["Y_in"], t["T_in"], t["tau"], t["P"], Yd, Td).cpu().numpy()
    for b in range(m):
        S = O.GasSystem(mech, O.inlet_of(sub, b))
        Jo = O.jacobian_fd(S, X[b], O.Options())
        rowmax = np.max(np.abs(Jo), axis=1, keepdims=True)
        assert np.max(np.abs(Jf[b] - Jo) / rowmax) <= 1e-6
        assert np.max(np.abs(Jf[b] - Ja[b]) / np.max(np.abs(Ja[b]), axis=1, keepdims=True)) <= 1e-3


def test_fd_jacobian_solves_reach_the_same_roots(dev):
    """Newton with the finite-difference Jacobian converges to the analytic-Jacobian roots."""
    _, mech, batch = workload("k10_b64")
    t = to_dev(batch, dev)
    gm = gpu_mech("k10_b64")
    a = psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"])
    f = psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"],
                        opts=psr.Options(jacobian=psr.PSR_JAC_FD))
    sa, sf = a["status"].cpu().numpy(), f["status"].cpu().numpy()
    both = (sa == 0) & (sf == 0) & (np.abs(a["T"].cpu().numpy() - f["T"].cpu().numpy()) < 1.0)
    assert both.mean() >= 0.8
    Ya, Yf = a["Y"].cpu().numpy()[both], f["Y"].cpu().numpy()[both]
    big = Ya > Y_MIN
    assert np.max(np.where(big, np.abs(Yf - Ya) / np.where(big, Ya, 1.0), 0.0)) <= Y_REL
    assert np.all(f["fnorm"].cpu().numpy()[sf == 0] <= 1e-8)
    with pytest.raises(psr.PsrError):
        psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"], opts=psr.Options(jacobian=7))


@pytest.mark.parametrize("name,n", [("k10_b64", 64), ("k200_b2048", 12)])
def test_jacobian_reuse_reaches_roots_of_the_oracle(dev, name, n):
    """Newton with factors kept for up to `jac_age` iterations (warp path at K = 10, block
    path at K = 200) stops only at points the oracle's residual calls steady states."""
    _, mech, batch = workload(name)
    batch = batch.subset(range(n))
    t = to_dev(batch, dev)
    gm = gpu_mech(name)
    a = psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"])
    r = psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"], opts=psr.Options(jac_age=2))
    sr = r["status"].cpu().numpy()
    Yr, Tr = r["Y"].cpu().numpy(), r["T"].cpu().numpy()
    ok = np.isin(sr, psr.CONVERGED_STATES)
    assert ok.mean() >= 0.9
    for b in np.flatnonzero(ok):
        F = O.gas_residual(mech, np.r_[Yr[b], Tr[b]][None], O.inlet_of(batch, b))[0]
        assert np.max(np.abs(F)) <= 1e-7, f"reactor {b}: |F| {np.max(np.abs(F)):.2e}"
    same = ok & (np.abs(Tr - a["T"].cpu().numpy()) <= 1e-6)
    assert same.sum() >= 0.8 * ok.sum()
    with pytest.raises(psr.PsrError):
        psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"], opts=psr.Options(jac_age=65))
