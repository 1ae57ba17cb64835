"""The LU's trailing update A22 -= L21 U12 on the fifth-generation tensor cores (tcgen05,
TF32 operands in shared memory, FP32 accumulator in tensor memory) for the block solver's
FP32 Jacobian (K + 1 >= 96): batched LU solves against their backward-error bound and the
CUDA-core FP32 LU, and full K = 200 solves whose roots must be the FP64 form's (the
residual and the Newton update stay FP64, the LU only steers)."""
import numpy as np
import pytest

from paper_2005_11468_gb300 import psr, synth
from tests.oracle_helpers import workload

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]
Y_REL, Y_MIN, T_ABS = 1e-6, 1e-10, 1e-8


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_11468_gb300 import _build
    _build.build()
    return torch.device("cuda:0")


def _backward_error(A, x, r):
    return np.abs(A @ x - r).max() / (np.abs(A).max() * np.abs(x).max() + np.abs(r).max())


@pytest.mark.parametrize("n", [96, 128, 201, 300, 512])
def test_tensor_core_lu_backward_error(dev, n):
    """Row-scaled random systems (scales e^U(-4, 4), the Jacobians' row spread): 3xTF32
    within the FP32 LU's bound and close to the CUDA-core FP32 LU; TF32 within its own
    (2^-11 unit roundoff) bound and visibly coarser than 3xTF32 (the tensor path ran).
    n = 512 keeps the matrix in global memory, n = 96 updates only its first panel on the
    tensor cores."""
    import torch
    rng = np.random.Generator(np.random.PCG64(2000 + n))
    B = 6
    A = rng.standard_normal((B, n, n)) * np.exp(rng.uniform(-4, 4, (B, n, 1)))
    r = rng.standard_normal((B, n))
    tA, tr = torch.tensor(A, device=dev), torch.tensor(r, device=dev)
    x32, ok32 = psr.batch_lu_solve(tA, tr, psr.PSR_MIXED)
    x3, ok3 = psr.batch_lu_solve_tc(tA, tr, psr.PSR_LU_3XTF32)
    x1, ok1 = psr.batch_lu_solve_tc(tA, tr, psr.PSR_LU_TF32)
    for ok in (ok32, ok3, ok1):
        assert np.all(ok.cpu().numpy() == 1)
    x32, x3, x1 = x32.cpu().numpy(), x3.cpu().numpy(), x1.cpu().numpy()
    e32 = max(_backward_error(A[b], x32[b], r[b]) for b in range(B))
    e3 = max(_backward_error(A[b], x3[b], r[b]) for b in range(B))
    e1 = max(_backward_error(A[b], x1[b], r[b]) for b in range(B))
    assert e32 <= 1e-5 * n
    assert e3 <= 1e-5 * n and e3 <= 8 * e32 + 1e-12
    assert e1 <= 1e-2
    assert e1 > 4 * e3, f"TF32 {e1:.2e} vs 3xTF32 {e3:.2e}: the TF32 products did not show"


def test_tensor_core_lu_small_n_uses_cuda_cores(dev):
    """Below n = 96 (and on the warp path, n <= 64) the call is the FP32 CUDA-core LU."""
    import torch
    rng = np.random.Generator(np.random.PCG64(7))
    for n in (54, 80):
        A = rng.standard_normal((3, n, n)) + n * np.eye(n)
        r = rng.standard_normal((3, n))
        a = psr.batch_lu_solve(torch.tensor(A, device=dev), torch.tensor(r, device=dev), psr.PSR_MIXED)[0]
        b = psr.batch_lu_solve_tc(torch.tensor(A, device=dev), torch.tensor(r, device=dev), psr.PSR_LU_TF32)[0]
        assert torch.equal(a, b)
    with pytest.raises(psr.PsrError):
        psr.batch_lu_solve_tc(torch.zeros((1, 128, 128), dtype=torch.float64, device=dev),
                              torch.zeros((1, 128), dtype=torch.float64, device=dev), 2)


@pytest.mark.parametrize("block_threads", [512, 256])
@pytest.mark.parametrize("mode", [psr.PSR_LU_TF32, psr.PSR_LU_3XTF32])
def test_k200_solves_with_tensor_core_lu(dev, mode, block_threads):
    """304 reactors of the K = 200 batch (two per SM) in the mixed form with the
    tensor-core trailing update, on blocks of 512 or 256 threads: converged reactors at ||F|| <= 1e-8 with elements
    conserved, and on the FP64 form's branch the FP64 form's roots within the bar."""
    import torch
    spec, mech, batch = workload("k200_b2048")
    sub = batch.subset(range(304))
    t = {k: torch.tensor(np.ascontiguousarray(getattr(sub, k)), dtype=torch.float64, device=dev)
         for k in ("Y_in", "T_in", "tau", "P", "Y0", "T0")}
    gm = psr.Mechanism(synth.mechanism_text(spec))
    ref = psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"],
                          opts=psr.Options(precision=psr.PSR_FP64))
    got = psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"],
                          opts=psr.Options(precision=psr.PSR_MIXED, lu_tensor=mode, block_threads=block_threads))
    rs, gs = ref["status"].cpu().numpy(), got["status"].cpu().numpy()
    rc, gc = np.isin(rs, psr.CONVERGED_STATES), np.isin(gs, psr.CONVERGED_STATES)
    assert gc.mean() >= 0.97
    assert np.all(got["fnorm"].cpu().numpy()[gc] <= 1e-8)
    Y, T = got["Y"].cpu().numpy(), got["T"].cpu().numpy()
    elem = ((Y[gc] - sub.Y_in[gc]) / mech.W) @ mech.comp
    assert np.max(np.abs(elem)) <= 1e-12
    Yr, Tr = ref["Y"].cpu().numpy(), ref["T"].cpu().numpy()
    both = rc & gc & (np.abs(T - Tr) <= 1.0)
    assert both.mean() >= 0.95
    big = Yr[both] > Y_MIN
    assert (np.abs(Y[both] - Yr[both])[big] / Yr[both][big]).max() <= Y_REL
    assert np.abs(T[both] - Tr[both]).max() <= T_ABS
    gm.close()
