"""The library's table-driven FP64 exp (Tang 1989) against CUDA's exp on the GPU:
at most a few units in the last place over the whole argument range used."""
import json
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_table_driven_exp_matches_cuda_exp(tmp_path):
    exe = str(tmp_path / "fexp_check")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                           "-std=c++17", os.path.join(HERE, "cuda", "fexp_check.cu"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    rec = json.loads(out.stdout.strip().splitlines()[-1])
    assert rec["max_ulp"] <= 4.0, rec
    assert rec["max_rel"] <= 1e-15, rec
