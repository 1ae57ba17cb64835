"""Handoff of stragglers: once the warp launch's work queue has drained and a given share
of its warps is idle, the reactors still running stop at their next Newton iteration and a
second launch continues them from their iterates with one thread block each (options
`handoff`). The roots must be those of the solve without handoff (and of the oracle), the
Newton budget stays the reactor's total, and the capture of the whole call in a CUDA graph
replays it."""
import numpy as np
import pytest

from paper_2005_11468_gb300 import psr, synth
from tests.oracle_helpers import workload
from tests.test_gpu_parity import T_ABS, Y_MIN, Y_REL, compare_roots, gpu_mech, oracle_solution_pool, to_dev

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_11468_gb300 import _build
    _build.build()
    return torch.device("cuda:0")


def _solve(dev, precision, handoff, B=4096):
    _, mech, batch = workload("k53_b4096")
    t = to_dev(batch.subset(range(B)), dev)
    out = psr.batch_solve(gpu_mech("k53_b4096"), t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"],
                          opts=psr.Options(precision=precision, handoff=handoff))
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize("precision", [psr.PSR_FP64, psr.PSR_MIXED])
def test_handoff_reaches_the_same_roots(dev, precision):
    """K = 53, 4096 reactors: no handoff, one at 50 % of the working warps idle and an eager
    one (1 %): the same converged set within a few reactors, roots within the parity
    bar of each other, every converged reactor at ||F|| <= 1e-8, no Newton budget overrun,
    and the eager handoff visibly moves reactors to the block solver."""
    ref = _solve(dev, precision, 0)
    # the reactor's budget: max_newton, or in the mixed form the FP32 launch's gas cap (300)
    # plus an FP64 continuation and an FP64 restart of max_newton each
    cap = psr.Options().max_newton * (2 if precision == psr.PSR_MIXED else 1) + \
        (300 if precision == psr.PSR_MIXED else 0)
    for h in (50, 1):
        got = _solve(dev, precision, h)
        c0, c1 = np.isin(ref["status"], psr.CONVERGED_STATES), np.isin(got["status"], psr.CONVERGED_STATES)
        assert c1.mean() >= c0.mean() - 0.002
        assert np.all(got["fnorm"][c1] <= 1e-8)
        assert np.all(got["iters"] <= cap)
        assert not np.any(got["status"] == 8), "an internal handoff status reached the caller"
        both = c0 & c1 & (np.abs(ref["T"] - got["T"]) <= 1.0)
        assert both.mean() >= 0.99
        big = ref["Y"][both] > Y_MIN
        rel = np.abs(got["Y"][both] - ref["Y"][both])[big] / ref["Y"][both][big]
        assert rel.max() <= Y_REL
        assert np.abs(got["T"][both] - ref["T"][both]).max() <= T_ABS
        if h == 1:
            moved = np.any(got["Y"] != ref["Y"], axis=1)
            assert moved.sum() >= 10, "the eager handoff left every reactor on the warp path"


def test_handoff_roots_match_the_oracle(dev):
    """The eager handoff's roots on the 32 sampled reactors of the K = 53 parity test."""
    _, mech, batch = workload("k53_b4096")
    got = _solve(dev, psr.PSR_FP64, 1)
    idx = [int(i) for i in np.random.Generator(np.random.PCG64(5)).choice(batch.B, 32, replace=False)]
    ref = oracle_solution_pool("k53_b4096", idx)
    n_ok, _ = compare_roots("k53_b4096", idx, ref, got["Y"][idx], got["T"][idx], got["status"][idx], "handoff")
    assert n_ok >= 28


def test_handoff_call_replays_from_a_cuda_graph(dev):
    """psr_batch_solve with the handoff (warp launch, list kernel, block continuation)
    captured in a CUDA graph and replayed: the eager call's converged set and roots."""
    import torch
    _, mech, batch = workload("k53_b4096")
    t = to_dev(batch, dev)            # the handoff needs at least two reactors per warp
    gm = gpu_mech("k53_b4096")
    opts = psr.Options(precision=psr.PSR_FP64, handoff=1)
    eager = psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"], opts=opts)
    torch.cuda.synchronize()
    out = {k: torch.empty_like(v) for k, v in eager.items()}
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"], opts=opts, out=out)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="thread_local"):
        psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"], opts=opts, out=out)
    for v in out.values():
        v.zero_()
    g.replay()
    torch.cuda.synchronize()
    cs = torch.tensor(psr.CONVERGED_STATES, device=dev, dtype=torch.int32)
    ok_e, ok_g = torch.isin(eager["status"], cs), torch.isin(out["status"], cs)
    assert ok_g.float().mean().item() >= 0.99 and (ok_e != ok_g).sum().item() <= 8
    both = ok_e & ok_g & ((out["T"] - eager["T"]).abs() < 1.0)
    torch.testing.assert_close(out["T"][both], eager["T"][both], rtol=0, atol=T_ABS)
