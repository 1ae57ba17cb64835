"""Host-side checks of the C ABI (no GPU needed): the library builds, loads and exports
every function include/psr.h declares; parse errors and bad arguments come back as
status codes with messages; option defaults agree across the header, the binding and
the oracle."""
import ctypes
import dataclasses
import os
import re

import pytest

from oracle import psr_oracle as O
from paper_2005_11468_gb300 import _build, psr, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    _build.build()
    return psr.lib()


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(psr_\w+)\s*\(", text))
    return sorted(names)


def test_exports_every_declared_symbol(L):
    names = declared_functions()
    assert "psr_batch_solve" in names and "psr_mech_load" in names and "psr_pipe_probe" in names
    for n in names:
        assert hasattr(L, n), n


@pytest.mark.parametrize("text,needle", [
    ("hello", "header"),
    ("psrmech 1\nelements 0\n", "elements"),
    ("psrmech 1\nelements 1\nC 12\nspecies 1\n0 X 1 200 1000 5000 1 2 3\n", "species record 0"),
    ("psrmech 1\nelements 1\nC 12\nspecies 1\n0 X 1 200 1000 5000 " + "1 " * 14 + "\nreactions 1\n"
     "0 elem 1 0 1 5 1 0 0\nend\n", "bad species index"),
    ("psrmech 1\nelements 1\nC 12\nspecies 1\n0 X 1 200 1000 5000 " + "1 " * 14 + "\nreactions 1\n"
     "0 troe 1 0 1 0 1 0 0\nend\n", "needs low and troe"),
    ("psrmech 1\nelements 1\nC 12\nspecies 1\n0 X 1 200 1000 5000 " + "1 " * 14 + "\nreactions 1\n"
     "0 elem 1 0 1 0 -1 0 0\nend\n", "Arrhenius"),
])
def test_parse_errors(L, text, needle):
    h = ctypes.c_void_p()
    raw = text.encode()
    rc = L.psr_mech_load_mem(raw, len(raw), ctypes.byref(h))
    assert rc == -3                                        # PSR_E_FORMAT
    assert needle in L.psr_last_error().decode()
    assert not h.value


def test_null_arguments(L):
    assert L.psr_mech_load(None, None) == -1
    assert L.psr_mech_load(b"/nonexistent/file.psrmech", ctypes.byref(ctypes.c_void_p())) == -2
    L.psr_mech_free(None)
    assert L.psr_batch_solve(None, 1, *([None] * 14), None, None) == -1


def test_generated_mechanisms_parse_up_to_upload(L):
    """Workload text passes the C parser: with no GPU the load fails only at upload."""
    for name in ("k10_b64", "k53_b4096"):
        raw = synth.mechanism_text(synth.workload_mechanism(name)).encode()
        h = ctypes.c_void_p()
        rc = L.psr_mech_load_mem(raw, len(raw), ctypes.byref(h))
        if rc == 0:
            L.psr_mech_free(h)
        else:
            assert rc in (-4, -5), L.psr_last_error().decode()   # CUDA / allocation only


def test_option_defaults_agree(L):
    c = psr.COptions()
    L.psr_options_default(ctypes.byref(c))
    py = psr.Options()
    for f in dataclasses.fields(py):
        assert getattr(c, f.name) == getattr(py, f.name), f.name
    o = O.Options()
    for name in ("ftol", "step_rtol", "step_atol_y", "step_atol_t", "ts_rtol", "ts_atol_y", "dt0_over_tau",
                 "dt_shrink", "y_floor", "t_min", "t_max", "max_newton", "max_damp", "max_ts_rounds",
                 "ts_steps", "ts_newton"):
        assert getattr(o, name) == getattr(c, name), name


def test_batch_limit_is_checked_before_anything_else(L):
    """Persistent solvers take one work-queue ticket per reactor plus one overshoot per
    resident warp on an int32 counter: batches above 2^31 - 2^22 are refused with
    PSR_E_ARG before the mechanism or any pointer is looked at."""
    for B in ((1 << 31) - 64, (1 << 31) - (1 << 22) + 1):
        assert L.psr_batch_solve(None, B, *([None] * 14), None, None) == -1
        assert "work-queue limit" in L.psr_last_error().decode()
        assert L.psr_batch_solve_noalloc(None, B, *([None] * 14), None, None) == -1
        assert "work-queue limit" in L.psr_last_error().decode()
        assert L.psr_batch_solve_soot(None, B, *([None] * 17), None, None) == -1
        assert "work-queue limit" in L.psr_last_error().decode()
        mechs = (ctypes.c_void_p * 1)(None)
        assert L.psr_batch_solve_multi(mechs, 1, B, *([None] * 15), None, None) == -1
        assert "work-queue limit" in L.psr_last_error().decode()
    # at the limit the call goes on to the mechanism check
    assert L.psr_batch_solve(None, (1 << 31) - (1 << 22), *([None] * 14), None, None) == -1
    assert "mechanism is NULL" in L.psr_last_error().decode()
