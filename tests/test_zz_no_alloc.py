"""The allocation-free solve entry, psr_batch_solve_noalloc, for callers that cannot
allocate device memory (an allocator frozen after start-up, or only pre-registered
buffers): it must give the same results as psr_batch_solve. It is called through the
C ABI twice in a row, because every call reuses the library's static work-queue array,
which keeps the previous call's contents. This file is collected last so that a run
stopping at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_2005_11468_gb300 import psr, synth

pytestmark = pytest.mark.gpu

Y_REL, Y_MIN, T_ABS = 1e-6, 1e-10, 1e-8     # the solver parity bar used by the other tests


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_11468_gb300 import _build
    _build.build()
    return torch.device("cuda:0")


def _outputs(torch, B, K, dev):
    f64, i32 = torch.float64, torch.int32
    return dict(Y=torch.empty((B, K), dtype=f64, device=dev), T=torch.empty(B, dtype=f64, device=dev),
                iters=torch.empty(B, dtype=i32, device=dev), ts_steps=torch.empty(B, dtype=i32, device=dev),
                status=torch.empty(B, dtype=i32, device=dev), fnorm=torch.empty(B, dtype=f64, device=dev),
                nfev=torch.empty(B, dtype=i32, device=dev))


def _call(fn, mech, t, out, opts, torch):
    rc = fn(mech.handle, t["Y_in"].shape[0], *[t[k].data_ptr() for k in ("Y_in", "T_in", "tau", "P", "Y0", "T0")],
            None, *[out[k].data_ptr() for k in ("Y", "T", "iters", "ts_steps", "status", "fnorm", "nfev")],
            ctypes.byref(opts), torch.cuda.current_stream().cuda_stream)
    assert rc == 0, psr.lib().psr_last_error().decode()
    torch.cuda.synchronize()


class _DefaultPool:
    """High-water mark of the device's default stream-ordered memory pool, where the
    library's cudaMallocAsync scratch comes from (torch keeps its own caching allocator):
    reset to zero before a call, it stays zero if the call allocated nothing there."""
    USED_MEM_HIGH = 8          # cudaMemPoolAttrUsedMemHigh

    def __init__(self):
        self.rt = None
        for name in ("libcudart.so.13", "libcudart.so"):
            try:
                self.rt = ctypes.CDLL(name)
                break
            except OSError:
                continue
        self.pool = ctypes.c_void_p()
        if self.rt is not None and self.rt.cudaDeviceGetDefaultMemPool(ctypes.byref(self.pool), 0) != 0:
            self.rt = None

    def reset(self):
        if self.rt is not None:
            zero = ctypes.c_uint64(0)
            assert self.rt.cudaMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(zero)) == 0

    def high(self):
        if self.rt is None:
            return None
        v = ctypes.c_uint64(0)
        assert self.rt.cudaMemPoolGetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(v)) == 0
        return v.value


@pytest.mark.parametrize("precision,jacobian", [(psr.PSR_FP64, psr.PSR_JAC_ANALYTIC),
                                                (psr.PSR_MIXED, psr.PSR_JAC_ANALYTIC),
                                                (psr.PSR_FP64, psr.PSR_JAC_FD)])
def test_noalloc_matches_allocating_entry(dev, precision, jacobian):
    import torch
    spec = synth.workload_mechanism("k10_b64")
    mech = psr.Mechanism(synth.mechanism_text(spec))
    batch = synth.workload_batch("k10_b64", spec)
    t = {k: torch.tensor(getattr(batch, k), dtype=torch.float64, device=dev)
         for k in ("Y_in", "T_in", "tau", "P", "Y0", "T0")}
    # the allocating entry without its FP64 fallback is the single launch this entry runs
    opts = psr.Options(precision=precision, mixed_fallback=0, jacobian=jacobian).to_c()
    L = psr.lib()
    ref = _outputs(torch, batch.B, spec.K, dev)
    _call(L.psr_batch_solve, mech, t, ref, opts, torch)
    pool = _DefaultPool()
    for _ in range(2):                     # the second call finds the first call's counter in the array
        got = _outputs(torch, batch.B, spec.K, dev)
        torch.cuda.synchronize()
        pool.reset()
        _call(L.psr_batch_solve_noalloc, mech, t, got, opts, torch)
        assert pool.high() in (None, 0), "the allocation-free entry used the stream-ordered pool"
        st_ref, st = ref["status"].cpu().numpy(), got["status"].cpu().numpy()
        # a reactor that ends next to the convergence limit (or the iteration cap) may land
        # on the other side of it in another launch: statuses may differ on a few reactors
        assert np.sum(st != st_ref) <= max(1, batch.B // 32)
        both = (st_ref == psr.PSR_CONVERGED) & (st == psr.PSR_CONVERGED)
        assert both.sum() >= 0.9 * batch.B
        Yr, Yg = ref["Y"].cpu().numpy()[both], got["Y"].cpu().numpy()[both]
        big = Yr > Y_MIN
        assert np.all(np.abs(Yg[big] - Yr[big]) <= Y_REL * Yr[big])
        assert np.all(np.abs(got["T"].cpu().numpy()[both] - ref["T"].cpu().numpy()[both]) <= T_ABS)


def test_noalloc_rejects_oversized_batch(dev):
    import torch
    spec = synth.workload_mechanism("k10_b64")
    mech = psr.Mechanism(synth.mechanism_text(spec))
    L = psr.lib()
    x = torch.zeros(8, dtype=torch.float64, device=dev)
    rc = L.psr_batch_solve_noalloc(mech.handle, 1 << 31, *([x.data_ptr()] * 6), None, *([x.data_ptr()] * 7),
                                   None, None)
    assert rc == -1
    assert "static work-queue limit" in L.psr_last_error().decode()
