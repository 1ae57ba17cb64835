"""The per-output error report against the FP64 oracle, run as a test: every workload's
full batch solved on the GPU in both forms (mixed and FP64), a seeded sample of its
reactors solved by the oracle in a process pool in the same job, and each sampled reactor
classified. Every reactor the oracle converged must be within the parity bar (Y_k > 1e-10
to 1e-6 relative, T to 1e-8 K, soot moments to 1e-5 relative) or on another steady branch
that is a root of the oracle's residual; none may be off the bar or left unconverged by
the GPU. The sample is the first part of the full report's sample (tests/parity_report.py)."""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

SAMPLES = {"k10_b64": 32, "k53_b4096": 16, "k200_b2048": 6, "k53soot_b16384": 8}
MIXED_SAMPLES = (8, 8, 3)


def test_per_output_errors_within_the_bar():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from tests import oracle_pool, parity_report
    d = parity_report.gpu_results(SAMPLES, MIXED_SAMPLES)
    res = oracle_pool.solve(parity_report.oracle_tasks(d, want_cond=False))
    rows = parity_report.classify(d, res)
    print("\n" + parity_report.table(rows))
    assert len(rows) == 2 * (len(SAMPLES) + len(MIXED_SAMPLES))
    for r in rows:
        what = f"{r['key']} {r['form']}"
        assert r["off"] == 0, f"{what}: {r['off']} reactors off the bar"
        assert r["gpu_unconv"] == 0, f"{what}: {r['gpu_unconv']} reactors the oracle converged are unconverged"
        assert r["n_pass"] + r["branch"] + r["oracle_unconv"] == r["sampled"]
        assert r["n_pass"] >= 0.75 * r["sampled"], f"{what}: only {r['n_pass']} of {r['sampled']} compared"
        assert max(r["ey"]) <= parity_report.Y_REL and max(r["et"]) <= parity_report.T_ABS
        if r["soot"]:
            assert max(r["em"]) <= parity_report.M_REL
        assert r["conv_all"] >= 0.99
