"""The library's integer-pipeline FP64 exp on the GPU: bit for bit the same as
the host build of the same function, and within 0.6 units in the last place of
the exact value (expl in extended precision) over the argument range used;
CUDA's own exp is measured beside it for reference. The mixed variant's table
logarithm on the GPU: bit for bit its host build and within 1.5 units in the
last place of logl; its Newton-Raphson reciprocal within 2^-44 of 1/x, and the
two-step one within 2^-51. The integer-pipe split of a double into a float
pair: the high part is the double rounded to float, and the pair is within
2^-47 of the double, for magnitudes from 2^-97 to the float maximum. The
integer-pipe double -> float conversion at the edges of the float range (zeros,
subnormal results and their ties, overflow, infinities, NaN) equals the host's
conversion bit for bit."""
import json
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_integer_exp_on_gpu_matches_host_and_exact(tmp_path):
    exe = str(tmp_path / "iexp_check")
    subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                           "-std=c++17", os.path.join(HERE, "cuda", "iexp_check.cu"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    rec = json.loads(out.stdout.strip().splitlines()[-1])
    assert rec["host_mismatch"] == 0, rec
    assert rec["max_ulp"] <= 0.6, rec
    assert rec["log_host_mismatch"] == 0, rec
    assert rec["log_max_ulp"] <= 1.5, rec
    assert rec["recip_max_rel"] <= 2.0 ** -44, rec
    assert rec["recip2_max_rel"] <= 2.0 ** -51, rec
    assert rec["split_hi_mismatch"] == 0, rec
    assert rec["split_max_rel"] <= 2.0 ** -47, rec
    assert rec["edge_n"] > 2 ** 18 and rec["edge_mismatch"] == 0, rec
