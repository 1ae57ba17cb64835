"""Builds libpsr.so in-tree with nvcc for sm_103a (no cmake; translation units in parallel)."""
import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpsr.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["psr_solve.cu", "psr_block.cu", "mech.cpp", "pipe_probe.cu"]
# psr_solve_inst.cu is built once per solve_kernel instantiation (Jacobian precision,
# soot, finite-difference Jacobian): six objects that compile in parallel.
INSTANCES = [(tj, soot, fdj) for soot, fdj in ((0, 0), (0, 1), (1, 0)) for tj in ("float", "double")]
HEADERS = ["psr_internal.h", "psr_device.cuh", "psr_warp.cuh", "psr_block.cuh", "psr_tc.cuh"]


def _nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is needed to build libpsr")
    return exe


def _compile(unit, nvcc):
    src, defines, tag = unit
    obj = os.path.join(BUILD, os.path.basename(src) + tag + ".o")
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", *defines,
           f"-I{INCLUDE}", f"-I{CSRC}", "-c", os.path.join(CSRC, src), "-o", obj]
    if src.endswith(".cpp"):
        cmd.insert(1, "-x")
        cmd.insert(2, "cu")
    subprocess.run(cmd, check=True)
    return obj


def build(force=False):
    """Compile every translation unit and link libpsr.so; returns the library path."""
    srcs = ([os.path.join(CSRC, s) for s in SOURCES + ["psr_solve_inst.cu", "psr_multi.cu"] + HEADERS]
            + [os.path.join(INCLUDE, h) for h in ("psr.h", "psr_probe.h")])
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= t for s in srcs) and os.path.getmtime(__file__) <= t:
            return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    units = [(s, [], "") for s in SOURCES]
    units.append(("psr_block.cu", ["-DPSR_BLOCK_THREADS=256"], ".bt256"))   # the 256-thread block solver
    # the persistent multi-mechanism kernel, once per first-pass Jacobian precision: one
    # block per SM with the FP32 Jacobian (its K = 200 Jacobian fills the shared memory),
    # two at 128 registers with the FP64 one (measured 1.34x faster than one at 255)
    units += [("psr_multi.cu", [f"-DPSR_MULTI_TJ={tj}", f"-DPSR_MULTI_ENTRY=multi_persistent_{tag}",
                                f"-DPSR_MULTI_MINB={minb}"], f".{tag}")
              for tj, tag, minb in (("float", "f32", 1), ("double", "f64", 2))]
    units += [("psr_solve_inst.cu", [f"-DPSR_INST_TJ={tj}", f"-DPSR_INST_SOOT={soot}", f"-DPSR_INST_FDJ={fdj}"],
               f".{tj}{soot}{fdj}") for tj, soot, fdj in INSTANCES]
    # the slowest units first, so that they start before the small ones take the cores
    units.sort(key=lambda u: 0 if u[0] in ("psr_multi.cu", "psr_solve_inst.cu", "psr_block.cu") else 1)
    with concurrent.futures.ThreadPoolExecutor(min(len(units), max(2, os.cpu_count() or 2))) as ex:
        objs = list(ex.map(lambda u: _compile(u, nvcc), units))
    tmp = LIB + ".tmp"
    subprocess.run([nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
