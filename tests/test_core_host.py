"""The GPU arithmetic on the host: its fast forms against its general forms,
and its general forms against the oracle.

tests/c/core_identities.cpp compiles paper_2401_14117_gb300/csrc/posit_core.cuh
with g++ (tests/c/core_host.h stands in for the CUDA intrinsics) and checks,
over 2e7 operand pairs from several families, that the serial-chain addition,
the table and in-band multiplies (sticky bit in the tie bit), the in-band
additions (select and multiply-add operand pick) and the table rounding give
the same decoded results as pz_add_fast / pz_mul_fast / pz_round.  These are
the rewrites the Rgemm, trsm, batched and solve kernels rely on; the GPU
parity tests compare the kernels themselves with the oracle."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_fast_forms_equal_general_forms(tmp_path):
    exe = tmp_path / "core_identities"
    subprocess.run(["g++", "-O2", "-std=c++17", "-o", str(exe),
                    os.path.join(HERE, "c", "core_identities.cpp")], check=True)
    r = subprocess.run([str(exe), "20000000"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "serial add 0, multiply 0, in-band add 0, rounding 0, chains 0" in r.stdout, r.stdout


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_general_ops_equal_the_oracle_on_the_host(tmp_path):
    """tests/c/core_vs_oracle.cpp: the device core's general add, sub, mul,
    div, sqrt and FP64 conversion, compiled on the host, give the oracle's
    word on 5e6 operand pairs (any word, |x| near 1, long regimes, few
    fraction bits, special words, cancellations)."""
    import oracle
    libdir = os.path.dirname(oracle.build())
    exe = tmp_path / "core_vs_oracle"
    subprocess.run(["g++", "-O2", "-std=c++17", "-o", str(exe),
                    os.path.join(HERE, "c", "core_vs_oracle.cpp"), f"-L{libdir}", "-loracle",
                    f"-Wl,-rpath,{libdir}"], check=True)
    r = subprocess.run([str(exe), "5000000"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "add 0 sub 0 mul 0 div 0 sqrt 0 from_double 0" in r.stdout, r.stdout
