"""Build and run the unit-throughput microbenchmarks of peaks.cu (FP64 FMA,
FP32 FMA, tcgen05 BF16 and TF32 MMA issue) on the current GPU.

    python -m paper_1708_03340_gb300.peaks.peaks      # prints one JSON line per unit

The results are the roofline denominators of the kernel families whose unit
the measured peak file of the GPU pool does not cover (it holds the HBM copy
rate and the cuBLAS BF16 rate only).
"""
from __future__ import annotations

import json
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(os.path.dirname(HERE), "_build")
EXE = os.path.join(BUILD, "peaks")


def build() -> str:
    os.makedirs(BUILD, exist_ok=True)
    src = os.path.join(HERE, "peaks.cu")
    if os.path.exists(EXE) and os.path.getmtime(EXE) >= os.path.getmtime(src):
        return EXE
    cmd = ["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", src, "-o", EXE]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed:\n{r.stdout}\n{r.stderr}")
    return EXE


def run() -> dict:
    out = subprocess.run([build()], capture_output=True, text=True, timeout=300)
    if out.returncode != 0:
        raise RuntimeError(out.stderr)
    res = {}
    for line in out.stdout.splitlines():
        rec = json.loads(line)
        res[rec["unit_test"]] = rec
    return res


if __name__ == "__main__":
    for k, v in run().items():
        print(json.dumps(v))
    sys.exit(0)
