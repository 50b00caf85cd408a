"""The integer-pipe binary64 operations match IEEE 754 arithmetic bit for bit.

paper_1510_05218_gb300/csrc/thiim_i64f.cuh computes binary64 sums and
products in integer arithmetic so that the FP64 sweep can move work off the
FP64 pipe without changing a single result bit.  The header also compiles as
plain C++; tests/i64f_check.cpp runs its integer path on random and
constructed operands (every exponent, close exponents with carries and
cancellation, exact ties of sums and products, the overflow and underflow
edges, zeros, subnormals, infinities and NaNs) and compares each result with
the host CPU's IEEE double arithmetic (round to nearest even; NaN results
only as NaN).  Sums never leave the integer path; products of normal
operands with a normal result must take it every time.
"""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1510_05218_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    exe = str(tmp_path_factory.mktemp("i64f") / "i64f_check")
    cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-I", CSRC,
           os.path.join(ROOT, "tests", "i64f_check.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_integer_path_is_bit_exact(checker):
    r = subprocess.run([checker, "1000000"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:]
    rows = {}
    for line in r.stdout.splitlines():
        name, cases, hits, bad = line.split()
        rows[name] = (int(cases), int(hits), int(bad))
    assert len(rows) == 9
    for name, (cases, hits, bad) in rows.items():
        assert bad == 0, name
        assert cases > 0
    # operands and results inside the normal range never leave the integer path
    for name in ("close_exponents", "cancellation", "add_ties", "mul_short", "sweep_range"):
        cases, hits, _ = rows[name]
        assert hits == cases, name
