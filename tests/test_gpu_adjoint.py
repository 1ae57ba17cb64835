"""GPU adjoint sensitivities against the oracle's dense sensitivities, and the autograd
wrapper against central differences of GPU re-solves."""
import numpy as np
import pytest

from oracle import psr_oracle as O
from paper_2005_11468_gb300 import psr, synth
from tests.oracle_helpers import workload

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


@pytest.fixture(scope="module")
def dev():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_11468_gb300 import _build
    _build.build()
    return torch.device("cuda:0")


def _setup(dev, name, idx):
    import torch
    spec, mech, batch = workload(name)
    sub = batch.subset(idx)
    gm = psr.Mechanism(synth.mechanism_text(spec))
    t = {k: torch.tensor(getattr(sub, k), dtype=torch.float64, device=dev)
         for k in ("Y_in", "T_in", "tau", "P", "Y0", "T0")}
    return mech, sub, gm, t


@pytest.mark.parametrize("name", ["k10_b64", "k53_b4096"])
def test_adjoint_matches_oracle_sensitivities(dev, name):
    import torch
    idx = list(range(6))
    mech, sub, gm, t = _setup(dev, name, idx)
    out = psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"])
    g = torch.tensor(np.random.Generator(np.random.PCG64(1)).standard_normal((len(idx), mech.K + 1)), device=dev)
    grad, lam, ok = psr.batch_adjoint(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], out["Y"], out["T"], g)
    grad, lam, ok = grad.cpu().numpy(), lam.cpu().numpy(), ok.cpu().numpy()
    Y, T, st = out["Y"].cpu().numpy(), out["T"].cpu().numpy(), out["status"].cpu().numpy()
    for j in range(len(idx)):
        if st[j] != 0:
            continue
        assert ok[j] == 1
        x = np.r_[Y[j], T[j]]
        inlet = O.inlet_of(sub, j)
        J = O.jacobian_cs(O.GasSystem(mech, inlet), x)
        lam_o = np.linalg.solve(J.T, g[j].cpu().numpy())
        np.testing.assert_allclose(lam[j], lam_o, rtol=1e-7, atol=1e-9 * np.abs(lam_o).max())
        go = O.adjoint_gradient(mech, inlet, x, g[j].cpu().numpy())
        np.testing.assert_allclose(grad[j], go, rtol=1e-6, atol=1e-8 * np.abs(go).max())


def test_autograd_matches_central_differences(dev):
    import torch
    from paper_2005_11468_gb300.autograd import psr_solve
    idx = [1, 2, 3]
    mech, sub, gm, t = _setup(dev, "k10_b64", idx)
    tight = psr.Options(step_rtol=1e-13, step_atol_y=1e-18, step_atol_t=1e-12)
    w = torch.tensor(np.random.Generator(np.random.PCG64(7)).standard_normal(mech.K), device=dev)
    lnm = torch.zeros(mech.I, dtype=torch.float64, device=dev, requires_grad=True)
    Y, T, st = psr_solve(lnm, gm, t["Y_in"], t["T_in"], t["tau"], t["P"], t["Y0"], t["T0"], tight)
    assert torch.all(st == 0)
    loss = (Y * w).sum() + 1e-3 * T.sum()
    loss.backward()
    gr = lnm.grad.cpu().numpy()
    h = 1e-6
    Ydev = (Y.detach(), T.detach())
    for i in np.random.Generator(np.random.PCG64(8)).choice(mech.I, 5, replace=False):
        vals = []
        for s in (+1, -1):
            lp = torch.zeros(mech.I, dtype=torch.float64, device=dev)
            lp[i] = s * h
            o = psr.batch_solve(gm, t["Y_in"], t["T_in"], t["tau"], t["P"], Ydev[0], Ydev[1],
                                rate_mult=torch.exp(lp), opts=tight)
            vals.append(((o["Y"] * w).sum() + 1e-3 * o["T"].sum()).item())
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - gr[i]) <= 1e-4 * np.abs(gr).max() + 1e-4 * abs(gr[i]), (i, fd, gr[i])
