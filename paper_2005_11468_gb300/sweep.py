"""Fixed-temperature PSR sweeps with continuation (the paper's run mode: the reactor
temperature is specified and swept together with the residence time, Secs. 5-6).

Orchestration only: each temperature of the grid is one batched fixed-T solve of all
residence times in libpsr; with `warm=True` the solutions at the previous temperature are
the initial guesses of the next (continuation along T), else every column starts from the
inlet composition.
"""
import numpy as np

from . import psr


def fixed_t_sweep(mech: psr.Mechanism, Y_in, T_grid, tau_grid, P=1013250.0, T_in=300.0, opts: psr.Options = None,
                  warm=True, device="cuda"):
    """Y [nT, ntau, K], status [nT, ntau], iters [nT, ntau] of the steady fixed-T PSRs at
    every (T, tau) of the grid with inlet Y_in [K] at T_in and pressure P (dyn/cm^2)."""
    import torch
    T_grid = np.asarray(T_grid, dtype=np.float64)
    tau_grid = np.asarray(tau_grid, dtype=np.float64)
    nT, nt, K = len(T_grid), len(tau_grid), mech.K
    base = opts or psr.Options()
    o = psr.Options(**{**base.__dict__, "energy": psr.PSR_FIXED_T})
    f64 = torch.float64
    Yin = torch.tensor(np.tile(np.asarray(Y_in, dtype=np.float64), (nt, 1)), dtype=f64, device=device)
    Tin = torch.full((nt,), float(T_in), dtype=f64, device=device)
    tau = torch.tensor(tau_grid, dtype=f64, device=device)
    Pd = torch.full((nt,), float(P), dtype=f64, device=device)
    Y = np.empty((nT, nt, K))
    status = np.empty((nT, nt), dtype=np.int32)
    iters = np.empty((nT, nt), dtype=np.int32)
    guess = Yin.clone()
    for a, T in enumerate(T_grid):
        Ts = torch.full((nt,), float(T), dtype=f64, device=device)
        out = psr.batch_solve(mech, Yin, Tin, tau, Pd, guess if warm else Yin, Ts, opts=o)
        st = out["status"]
        Y[a] = out["Y"].cpu().numpy()
        status[a] = st.cpu().numpy()
        iters[a] = out["iters"].cpu().numpy()
        conv = torch.isin(st, torch.tensor(psr.CONVERGED_STATES, dtype=st.dtype, device=st.device))
        guess = torch.where(conv[:, None], out["Y"], Yin)   # continue from converged columns only
    return Y, status, iters
