"""The library's double-double and quad-double arithmetic (csrc/mp.cuh) built for the
host and checked against exact rationals on adversarial operands.

The device code rounds every operation with an explicit IEEE round-to-nearest intrinsic;
the host build maps each intrinsic to the same IEEE operation (and FMA to std::fma), so
it computes the same bits.  Checked: the error of each result is within 2^(-52 L) times
the operands' magnitude (the bound of this arithmetic), and the result is normalised --
each limb at most a unit in the last place of the one above -- so that the leading
limb is the value rounded to double.  That last property failed for quad-double sums
whose top components cancel exactly (the leading limb came out zero with the value in
the lower limbs), which misled the FP64 refinement solve that reads only leading limbs.
"""
import os
import re
import shutil
import subprocess
from fractions import Fraction as Fr

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MP = os.path.join(ROOT, "paper_1109_0545_gb300", "csrc", "mp.cuh")
SHIM = """#pragma once
#include <cmath>
#include <cstdint>
#include <cstring>
static inline double __dadd_rn(double a, double b) { return a + b; }
static inline double __dsub_rn(double a, double b) { return a - b; }
static inline double __dmul_rn(double a, double b) { return a * b; }
static inline double __ddiv_rn(double a, double b) { return a / b; }
static inline double __fma_rn(double a, double b, double c) { return std::fma(a, b, c); }
static inline long long __double_as_longlong(double x) { long long b; std::memcpy(&b, &x, 8); return b; }
static inline double __longlong_as_double(long long b) { double x; std::memcpy(&x, &b, 8); return x; }
static inline int __double2hiint(double x) { return (int)(__double_as_longlong(x) >> 32); }
static inline int __clz(int x) { return x ? __builtin_clz((unsigned)x) : 32; }
static inline int __ffs(int x) { return __builtin_ffs(x); }
using std::isfinite;
"""


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("mp_host")
    src = open(MP).read()
    src = src.replace("#include <cuda_runtime.h>", '#include "shim.h"')
    src = src.replace("__device__ __forceinline__", "static inline")
    src = re.sub(r"template <> static inline", "template <> inline", src)
    (d / "mp_host.h").write_text(src)
    (d / "shim.h").write_text(SHIM)
    exe = d / "check"
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", str(d),
                    os.path.join(ROOT, "tests", "mp_host_check.cpp"), "-o", str(exe)], check=True)
    return str(exe)


def _cases(exe, L, mode, count):
    out = subprocess.run([exe, str(L), str(mode), str(count)], capture_output=True, text=True, check=True).stdout
    for line in out.splitlines():
        v = [float.fromhex(t) for t in line.split()]
        yield v[:L], v[L:2 * L], v[2 * L:]


def _separated(r):
    """Each nonzero limb at most one unit in the last place of the limb above it."""
    import math
    for hi, lo in zip(r, r[1:]):
        if lo == 0.0:
            continue
        if hi == 0.0 or abs(lo) > math.ulp(hi):
            return False
    return True


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_host_build_of_the_device_arithmetic(checker, L, mode):
    bound = 2.0 ** (-52 * L + 2)
    worst, unsep = 0.0, 0
    for a, b, r in _cases(checker, L, mode, 3000):
        A, B, R = (sum(Fr(x) for x in v) for v in (a, b, r))
        exact = A * B if mode == 2 else A + B
        scale = abs(A) * abs(B) if mode == 2 else max(abs(A), abs(B))
        if scale:
            worst = max(worst, abs(float((R - exact) / scale)))
        if L == 4 and not _separated(r):
            unsep += 1
    assert worst <= bound, worst
    assert unsep == 0


@pytest.mark.parametrize("L", [2, 4])
def test_running_sums_within_bound_and_settled(checker, L):
    """r_acc over m terms (some of them cancelling the sum so far, exactly or up to a
    small remainder), then r_settle: the error is within m 2^(-52 L + 2) of the largest
    partial sum, and the settled result is normalised."""
    out = subprocess.run([checker, str(L), "3", "400"], capture_output=True, text=True, check=True).stdout
    worst = 0.0
    for line in out.splitlines():
        tok = line.split()
        m = int(tok[0])
        v = [float.fromhex(t) for t in tok[1:]]
        assert len(v) == (m + 1) * L
        total, biggest = Fr(0), Fr(0)
        for q in range(m):
            total += sum(Fr(x) for x in v[q * L:(q + 1) * L])
            biggest = max(biggest, abs(total))
        r = v[m * L:]
        if biggest:
            worst = max(worst, abs(float((sum(Fr(x) for x in r) - total) / biggest)) / m)
        assert _separated(r), r
    assert worst <= 2.0 ** (-52 * L + 2), worst
