"""The tcgen05 main loop of the sliced products, checked bit for bit.

`tc_mainloop_check.cu` runs the shared main loop (`tc_sliced.cuh`: TMA copies into the
64-byte-swizzled ring, one wide tcgen05.mma per A digit plane, one tensor-memory accumulator per
digit order, tcgen05.ld of the accumulators) on random digit planes small enough that every FP32
accumulator holds an exact integer, and compares each accumulator of each digit order with the
integer product computed on the host.  Shapes: those of the Krylov-chain kernel (6 and 5 digits,
N = 48) and of the pair kernel (5 digits, N = 96), with one to fourteen K stages, two K chunks,
K not a multiple of the 32-wide stage, and zero rows in A.  Integer work, so the bar is exact.
"""
import os
import subprocess

import pytest
import torch

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_tc05_mainloop_products_are_exact(tmp_path):
    from paper_2407_06409_gb300 import build
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    exe = tmp_path / "tc_mainloop_check"
    cmd = [build._nvcc(), *build.ARCH, "-O2", "-std=c++17", "-o", str(exe),
           os.path.join(HERE, "tc_mainloop_check.cu")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = [ln for ln in r.stdout.splitlines() if "mismatches" in ln]
    assert len(lines) == 5 and all("status 0 mismatches 0 of" in ln for ln in lines), r.stdout
    assert r.stdout.strip().endswith("all exact")
