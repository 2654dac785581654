"""The library's integer-pipeline FP64 exp (csrc/adg_math.cuh), compiled for the
host, against expl in extended precision: within 0.6 units in the last place
over the whole range |x| <= 700, the Arrhenius arguments, small and tiny
arguments and the table nodes, and correctly rounded almost everywhere; its
float variant (exact reduction, 32-bit polynomial good to ~2^-29, one rounding)
within 0.53 float ulp. The FP32-pipe exp of a float-float argument (the mixed
chemistry: Tang's reduction in df32, the table as float pairs, one final
rounding dominant) within 0.55 float ulp over [-87, 88] and correctly rounded for
99 % of the arguments. The table-driven logarithm of the mixed variant's ln T
(Tang's method, 128 nodes, series to u^7) within 1.5 units in the last place
over temperatures, the table nodes and their neighbours, the whole normal range
and both sides of 1, and within 3e-15 absolute over temperatures 50-10000 K."""
import json
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_integer_exp_host_build_against_extended_precision(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "iexp_host")
    subprocess.check_call([nvcc, "-O2", "-std=c++17",
                           os.path.join(HERE, "cuda", "iexp_host_check.cu"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    rec = json.loads(out.stdout.strip().splitlines()[-1])
    assert rec["max_ulp"] <= 0.6, rec
    assert rec["correctly_rounded"] >= 0.99, rec
    assert rec["float_max_ulp"] <= 0.53, rec
    assert rec["df_max_ulp"] <= 0.55, rec
    assert rec["df_correctly_rounded"] >= 0.99, rec
    assert rec["log_max_ulp"] <= 1.5, rec
    assert rec["log_max_abs_T"] <= 3e-15, rec


def test_integer_float_conversion_at_the_range_edges_host_build(tmp_path):
    """The integer double -> float conversion of the doubles outside the normal
    float range (zeros, subnormal results with exact ties, overflow, infinities,
    NaN; `d2f_edge_bits`), compiled for the host, equals the host's IEEE
    round-to-nearest-even conversion bit for bit on about a million values."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "d2f_host")
    subprocess.check_call([nvcc, "-O2", "-std=c++17",
                           os.path.join(HERE, "cuda", "d2f_host_check.cu"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    rec = json.loads(out.stdout.strip().splitlines()[-1])
    assert rec["checked"] > 10 ** 6, rec
    assert rec["mismatch"] == 0 and rec["nan_bad"] == 0, rec
