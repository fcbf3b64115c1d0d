"""The integer-pipe TwoSum error term (csrc/mp_eft_int.cuh), compiled for the host
with g++, against the host's binary64 arithmetic (Algorithm 2): every accepted
pair must give Algorithm 2's error term bit for bit, and every pair inside the
documented domain must be accepted -- for the default form, for the variant
that also packs subnormal error terms (whose domain takes in tiny and subnormal
operands), and for the TwoProd error term.  Independent of the oracle and of the
GPU."""

import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("eft") / "eft_int_check")
    # -ffp-contract=off keeps the reference sequence free of fused multiply-adds
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", os.path.join(HERE, "eft_int_check.cpp"),
                    "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_two_sum_error_term_matches_binary64(checker, seed):
    r = subprocess.run([checker, "2000000", str(seed)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    lines = [ln for ln in r.stdout.splitlines() if "checked" in ln]
    assert len(lines) == 3 and all("wrong 0 refused-in-domain 0" in ln for ln in lines), r.stdout
