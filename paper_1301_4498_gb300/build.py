"""Build libnyxhydro.so for sm_103a with nvcc (no cmake, no torch extension
machinery): each translation unit is compiled in parallel with its own
floating-point flags, then linked into one shared library in this package.

* FP64 translation units (per-box stage kernels, fused FP64 advance) use
  ``--fmad=false`` so every operation is a separately rounded IEEE op.
* The mixed-precision fused advance allows FMA contraction and the
  approximate FP32 division and square root.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libnyxhydro.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
          "-I", os.path.join(ROOT, "include"), "-I", CSRC, "--expt-relaxed-constexpr"]

UNITS = {
    "nyx_api.cu": [],
    "nyx_fill.cu": [],
    "nyx_staged.cu": ["--fmad=false"],
    "nyx_fused_f64.cu": ["--fmad=false"],
    "nyx_fused_mixed.cu": ["--fmad=true", "-prec-div=false", "-prec-sqrt=false", "-ftz=true"],
    "nyx_noalloc.cu": [],
    "nyx_probe.cu": [],
    "nyx_amr.cu": ["--fmad=false"],
    "nyx_poisson.cu": ["--fmad=false"],
}


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(obj: str, src: str) -> bool:
    if not os.path.exists(obj):
        return True
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    deps.append(os.path.join(ROOT, "include", "nyx_hydro.h"))
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for unit, flags in UNITS.items():
        src = os.path.join(CSRC, unit)
        obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
        if force or _stale(obj, src):
            cmd = [nvcc] + ARCH + COMMON + flags + ["-c", src, "-o", obj]
            if ptxas_info:
                cmd += ["-Xptxas", "-v"]
            jobs.append((unit, cmd))

    def run(job):
        unit, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        return unit, cmd, r

    relink = bool(jobs) or not os.path.exists(LIB)
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 1))) as ex:
        for unit, cmd, r in ex.map(run, jobs):
            if verbose or ptxas_info:
                sys.stderr.write(r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {unit}:\n{' '.join(cmd)}\n{r.stderr}")
    if relink:
        objs = [os.path.join(BUILD, u.replace(".cu", ".o")) for u in UNITS]
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-ldl"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{' '.join(cmd)}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
