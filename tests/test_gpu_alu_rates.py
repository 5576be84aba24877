"""Measures the ALU rates the double-float roofline is derived from (FP32 FMA scalar and paired,
native FP64 FMA, double-float multiply-add) with a standalone probe; asserts only that the probe
ran and that FP64 on this GPU is far slower than FP32 (the reason for the double-float path)."""
import os
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_alu_rates():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "alu_rates")
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                        os.path.join(HERE, "probes", "alu_rates.cu")], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    print(out)
    vals = {k: float(v) for k, v in (line.split()[:2] for line in out.splitlines() if line and line.split()[0] != "status")}
    assert vals["fp32_fma_tflops"] > 0 and vals["df64_mad_tper_s"] > 0
    assert vals["fp64_dfma_tflops"] < vals["fp32_fma_tflops"] / 8
