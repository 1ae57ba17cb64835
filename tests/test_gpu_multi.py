"""The uneven batch (50/35/15 % of K = 10 / 53 / 200 reactors, 32768 in all, shuffled) in
one call of psr_batch_solve_multi: the persistent launch against per-mechanism solves of
the same reactors, against one launch sequence per mechanism and, on sampled reactors,
against the oracle; the block path and the bounded wait inside the persistent launch;
out-of-range mechanism ids; and a CUDA graph capture of the call replayed."""
import numpy as np
import pytest

from oracle import psr_oracle as O
from paper_2005_11468_gb300 import psr, synth
from tests.oracle_helpers import workload

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]
Y_REL, Y_MIN, T_ABS = 1e-6, 1e-10, 1e-8


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_11468_gb300 import _build
    _build.build()
    parts = synth.MIXED_WORKLOAD["parts"]
    specs, mechs, gms = [], [], []
    for name in parts:
        spec, mech, _ = workload(name)
        specs.append(spec)
        mechs.append(mech)
        gms.append(psr.Mechanism(synth.mechanism_text(spec)))
    return dict(dev=torch.device("cuda:0"), specs=specs, mechs=mechs, gms=gms)


def _dev(env, mb):
    import torch
    d = env["dev"]
    t = {k: torch.tensor(mb[k], dtype=torch.float64, device=d) for k in ("Y_in", "Y0", "T_in", "tau", "P", "T0")}
    t["mech_id"] = torch.tensor(mb["mech_id"], dtype=torch.int32, device=d)
    t["row_off"] = torch.tensor(mb["row_off"], dtype=torch.int64, device=d)
    return t


def _multi(env, t, opts=None):
    return psr.batch_solve_multi(env["gms"], t["mech_id"], t["row_off"], t["Y_in"], t["T_in"], t["tau"], t["P"],
                                 t["Y0"], t["T0"], opts=opts)


def _rows(mb, Y, c, K):
    return np.stack([Y[o:o + K] for o in mb["row_off"][mb["members"][c]]]) if len(mb["members"][c]) else \
        np.zeros((0, K))


@pytest.mark.parametrize("persistent", [0, 1])
def test_uneven_batch_full_size(env, persistent):
    """The 32768-reactor call the benchmark times, in both layouts (one launch sequence per
    mechanism, and the one persistent launch): each mechanism's reactors equal a separate
    psr_batch_solve of that mechanism on the same reactors; sampled reactors of every
    mechanism match the oracle."""
    import torch
    mb = synth.mixed_batch(env["specs"])
    t = _dev(env, mb)
    # without the timing-dependent handoff of stragglers, so that the per-mechanism layout's
    # warp-path statuses equal those of the one-mechanism solves
    opts = psr.Options(precision=psr.PSR_MIXED, persistent=persistent, handoff=0)
    out = _multi(env, t, opts)
    Y, T, st = out["Y"].cpu().numpy(), out["T"].cpu().numpy(), out["status"].cpu().numpy()
    fn = out["fnorm"].cpu().numpy()
    conv = np.isin(st, psr.CONVERGED_STATES)
    assert conv.mean() >= 0.95
    assert np.all(fn[conv] <= 1e-8)
    for c, (spec, mech, gm) in enumerate(zip(env["specs"], env["mechs"], env["gms"])):
        mem = mb["members"][c]
        bc = mb["batches"][c]
        d = {k: torch.tensor(np.ascontiguousarray(getattr(bc, k)), dtype=torch.float64, device=env["dev"])
             for k in ("Y_in", "T_in", "tau", "P", "Y0", "T0")}
        ref = psr.batch_solve(gm, d["Y_in"], d["T_in"], d["tau"], d["P"], d["Y0"], d["T0"],
                              opts=psr.Options(precision=psr.PSR_MIXED, handoff=0))
        Yr, Tr, sr = ref["Y"].cpu().numpy(), ref["T"].cpu().numpy(), ref["status"].cpu().numpy()
        Yc = _rows(mb, Y, c, spec.K)
        # the block-per-reactor path accumulates its Jacobian with atomics from several
        # warps, so a reactor's iterates can differ in rounding between two launches and a
        # marginal reactor may converge in the other precision's launch (status 0 vs 5)
        cm, cr = np.isin(st[mem], psr.CONVERGED_STATES), np.isin(sr, psr.CONVERGED_STATES)
        assert np.mean(cm == cr) >= 0.99, f"class {c}: convergence differs"
        if spec.K + 1 <= 64 and not persistent:
            assert np.array_equal(st[mem], sr), f"class {c}: statuses differ"
        both = np.isin(st[mem], psr.CONVERGED_STATES) & np.isin(sr, psr.CONVERGED_STATES) & \
            (np.abs(T[mem] - Tr) < 1.0)
        big = Yr[both] > Y_MIN
        rel = np.max(np.where(big, np.abs(Yc[both] - Yr[both]) / np.where(big, Yr[both], 1.0), 0.0), axis=1)
        off = (rel > Y_REL) | (np.abs(T[mem][both] - Tr[both]) > T_ABS)
        if spec.K + 1 <= 64:
            assert not off.any(), f"class {c}: {off.sum()} reactors off the parity bar"
        else:
            # Jacobians with condition numbers near 1e16 leave some minor species of a
            # root undetermined beyond ~1e-4 at ||F|| <= 1e-8 (both rows are roots)
            assert off.mean() <= 0.01, f"class {c}: {off.sum()} of {off.size} reactors off the parity bar"
        elem = ((Yc[conv[mem]] - bc.Y_in[conv[mem]]) / mech.W) @ mech.comp
        assert np.max(np.abs(elem)) <= 1e-12
        # sampled against the oracle: two reactors of the small mechanisms, one of K = 200
        for j in range(2 if spec.K < 100 else 1):
            r = O.solve_reactor(mech, O.inlet_of(bc, j), np.r_[bc.Y0[j], bc.T0[j]])
            if r.status != O.CONVERGED or abs(T[mem[j]] - r.x[-1]) > 1.0:
                continue
            assert st[mem[j]] in psr.CONVERGED_STATES
            bigo = r.x[:-1] > Y_MIN
            assert np.max(np.abs(Yc[j][bigo] - r.x[:-1][bigo]) / r.x[:-1][bigo]) <= Y_REL
            assert abs(T[mem[j]] - r.x[-1]) <= T_ABS


def _agree(st_a, st_b, Ta, Tb, min_frac=0.99):
    """Two solves of the same reactors: convergence agrees on >= min_frac of them, and rows
    both converged on the same branch match within the parity bar."""
    ca, cb = np.isin(st_a, psr.CONVERGED_STATES), np.isin(st_b, psr.CONVERGED_STATES)
    assert np.mean(ca == cb) >= min_frac
    both = ca & cb & (np.abs(Ta - Tb) < 1.0)
    assert both.mean() >= min_frac - 0.01
    return both


@pytest.mark.parametrize("precision", [psr.PSR_MIXED, psr.PSR_FP64])
def test_persistent_launch_matches_per_class_launches(env, precision):
    """The one persistent launch (block-solver classes first, then warp-solver classes, the
    FP64 re-solve in the same kernel) against one launch sequence per mechanism on forked
    streams, on 4096 reactors of the uneven batch: the same convergence and, row by row, the
    same roots within the parity bar. (Not bit for bit: the same solver code compiled into
    another kernel may contract and order its floating-point operations differently.)"""
    mb = synth.mixed_batch(env["specs"], B=4096)
    t = _dev(env, mb)
    a = _multi(env, t, psr.Options(precision=precision, persistent=1, handoff=0))
    b = _multi(env, t, psr.Options(precision=precision, persistent=0, handoff=0))
    sa, sb = a["status"].cpu().numpy(), b["status"].cpu().numpy()
    Ya, Yb, Ta, Tb = (x.cpu().numpy() for x in (a["Y"], b["Y"], a["T"], b["T"]))
    assert np.isin(sa, psr.CONVERGED_STATES).mean() >= 0.95
    _agree(sa, sb, Ta, Tb)
    for c, spec in enumerate(env["specs"]):
        mem = mb["members"][c]
        Yc_a, Yc_b = _rows(mb, Ya, c, spec.K), _rows(mb, Yb, c, spec.K)
        both = _agree(sa[mem], sb[mem], Ta[mem], Tb[mem], 0.98)
        big = Yc_b[both] > Y_MIN
        rel = np.where(big, np.abs(Yc_a[both] - Yc_b[both]) / np.where(big, Yc_b[both], 1.0), 0.0).max(axis=1)
        off = (rel > Y_REL) | (np.abs(Ta[mem][both] - Tb[mem][both]) > T_ABS)
        assert off.mean() <= (0.0 if spec.K + 1 <= 64 else 0.01), f"class {c}: {off.sum()} rows off the bar"


def test_persistent_launch_on_the_block_path(env):
    """PSR_PATH_BLOCK puts every class on the block solver inside the persistent launch
    (phase 2 empty): converged rows at ||F|| <= 1e-8 that conserve elements and match the
    default launch's roots."""
    mb = synth.mixed_batch(env["specs"], B=2048)
    t = _dev(env, mb)
    a = _multi(env, t, psr.Options(precision=psr.PSR_MIXED, path=psr.PSR_PATH_BLOCK, persistent=1))
    b = _multi(env, t, psr.Options(precision=psr.PSR_MIXED))
    sa, sb = a["status"].cpu().numpy(), b["status"].cpu().numpy()
    Ta, Tb = a["T"].cpu().numpy(), b["T"].cpu().numpy()
    conv = np.isin(sa, psr.CONVERGED_STATES)
    assert conv.mean() >= 0.95
    assert np.all(a["fnorm"].cpu().numpy()[conv] <= 1e-8)
    both = _agree(sa, sb, Ta, Tb, 0.98)
    assert np.abs(Ta[both] - Tb[both]).max() <= T_ABS
    Ya = a["Y"].cpu().numpy()
    for c, (spec, mech) in enumerate(zip(env["specs"], env["mechs"])):
        mem = mb["members"][c]
        bc = mb["batches"][c]
        Yc = _rows(mb, Ya, c, spec.K)
        ok = conv[mem]
        elem = ((Yc[ok] - bc.Y_in[ok]) / mech.W) @ mech.comp
        assert np.max(np.abs(elem)) <= 1e-12


def test_spin_limit_bounds_the_wait(env):
    """With spin_limit = 1 a block of the persistent launch that finds no re-solve entry
    published yet gives up at once instead of waiting: the call still completes, every
    status is a valid code, and what converged meets the tolerance."""
    mb = synth.mixed_batch(env["specs"], B=1024)
    t = _dev(env, mb)
    out = _multi(env, t, psr.Options(precision=psr.PSR_MIXED, persistent=1, spin_limit=1, mixed_max_newton=20))
    st = out["status"].cpu().numpy()
    assert np.all(np.isin(st, [psr.PSR_CONVERGED, psr.PSR_REFINE_FALLBACK, psr.PSR_MAX_ITER,
                               psr.PSR_NONFINITE, psr.PSR_TS_EXHAUSTED]))
    conv = np.isin(st, psr.CONVERGED_STATES)
    assert np.all(out["fnorm"].cpu().numpy()[conv] <= 1e-8)
    with pytest.raises(psr.PsrError):
        _multi(env, t, psr.Options(spin_limit=-1))
    with pytest.raises(psr.PsrError):
        _multi(env, t, psr.Options(persistent=2))


def test_bad_mechanism_id_is_reported(env):
    mb = synth.mixed_batch(env["specs"], B=96)
    t = _dev(env, mb)
    t["mech_id"][5] = 7
    t["mech_id"][9] = -1
    out = _multi(env, t)
    st = out["status"].cpu().numpy()
    assert st[5] == psr.PSR_BAD_INPUT and st[9] == psr.PSR_BAD_INPUT
    others = np.ones(96, bool)
    others[[5, 9]] = False
    assert np.isin(st[others], psr.CONVERGED_STATES).mean() >= 0.9
    with pytest.raises(psr.PsrError):
        psr.batch_solve_multi([], t["mech_id"], t["row_off"], t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"])


@pytest.mark.parametrize("persistent", [0, 1])
def test_graph_capture_replays_the_call(env, persistent):
    """The call captured into a CUDA graph (bucketing, then three solver launches on forked
    streams and the FP64 re-solves, or the one persistent launch) and replayed gives the
    eager call's results."""
    import torch
    mb = synth.mixed_batch(env["specs"], B=384)
    t = _dev(env, mb)
    # without the handoff of stragglers, which depends on timing, so that warp-path rows
    # are bit-reproducible
    opts = psr.Options(precision=psr.PSR_MIXED, handoff=0, persistent=persistent)
    eager = _multi(env, t, opts)
    torch.cuda.synchronize()
    out = {k: torch.empty_like(v) for k, v in eager.items()}
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        psr.batch_solve_multi(env["gms"], t["mech_id"], t["row_off"], t["Y_in"], t["T_in"], t["tau"], t["P"],
                              t["Y0"], t["T0"], opts=opts, out=out)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        psr.batch_solve_multi(env["gms"], t["mech_id"], t["row_off"], t["Y_in"], t["T_in"], t["tau"], t["P"],
                              t["Y0"], t["T0"], opts=opts, out=out)
    for v in out.values():
        v.zero_()
    g.replay()
    torch.cuda.synchronize()
    cs = torch.tensor(psr.CONVERGED_STATES, device=env["dev"], dtype=torch.int32)
    ok_e, ok_g = torch.isin(eager["status"], cs), torch.isin(out["status"], cs)
    assert ok_g.float().mean().item() >= 0.95
    assert (ok_e == ok_g).float().mean().item() >= 0.98
    both = ok_e & ok_g & ((out["T"] - eager["T"]).abs() < 1.0)
    torch.testing.assert_close(out["T"][both], eager["T"][both], rtol=0, atol=1e-8)
    # warp-path mechanisms are reproducible launch to launch: identical rows
    small = torch.tensor(mb["mech_id"] < 2, device=env["dev"])
    assert torch.equal(out["status"][small], eager["status"][small])
    assert torch.equal(out["T"][small], eager["T"][small])


@pytest.mark.parametrize("cls", [0, 1])
def test_uneven_batch_adjoint_matches_central_differences(env, cls):
    """Adjoint gradients (torch.autograd over psr_batch_adjoint) of reactors of the uneven
    batch's K = 10 and K = 53 classes against central differences (h = 1e-6 on ln m_i) of
    tightly converged re-solves; the K = 200 class is checked against the oracle by
    backward error in test_gpu_k200.py (its Jacobians are too ill-conditioned for
    differences of re-solved roots)."""
    import torch
    from paper_2005_11468_gb300.autograd import psr_solve
    mb = synth.mixed_batch(env["specs"], B=512)
    bc = mb["batches"][cls].subset(range(3))
    dev = env["dev"]
    t = {k: torch.tensor(np.ascontiguousarray(getattr(bc, k)), dtype=torch.float64, device=dev)
         for k in ("Y_in", "T_in", "tau", "P", "Y0", "T0")}
    gm, spec = env["gms"][cls], env["specs"][cls]
    tight = psr.Options(step_rtol=1e-13, step_atol_y=1e-18, step_atol_t=1e-12)
    w = torch.tensor(np.random.Generator(np.random.PCG64(11 + cls)).standard_normal(spec.K), device=dev)
    lnm = torch.zeros(spec.I, dtype=torch.float64, device=dev, requires_grad=True)
    Y, T, st = psr_solve(lnm, gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"], tight)
    ok = torch.isin(st, torch.tensor(psr.CONVERGED_STATES, device=dev, dtype=torch.int32))
    assert ok.all()
    loss = (Y * w).sum() + 1e-3 * T.sum()
    loss.backward()
    gr = lnm.grad.cpu().numpy()
    h = 1e-6
    Ys, Ts = Y.detach(), T.detach()
    for i in np.random.Generator(np.random.PCG64(21 + cls)).choice(spec.I, 4, replace=False):
        vals = []
        for sgn in (+1, -1):
            lp = torch.zeros(spec.I, dtype=torch.float64, device=dev)
            lp[i] = sgn * h
            o = psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], Ys, Ts, rate_mult=torch.exp(lp),
                                opts=tight)
            vals.append(((o["Y"] * w).sum() + 1e-3 * o["T"].sum()).item())
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - gr[i]) <= 1e-4 * np.abs(gr).max() + 1e-4 * abs(gr[i]), (i, fd, gr[i])
