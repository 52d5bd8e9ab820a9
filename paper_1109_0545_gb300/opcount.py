"""Static count of the FP64 instructions the evaluation kernel issues per point.

The roofline of the evaluation kernel is the FP64 pipe, so its algorithmic work is the
number of FP64 instructions (DADD, DMUL, DFMA, each one instruction) that the kernel's
arithmetic executes for one point.  The per-operation counts below are those of
``csrc/mp.cuh`` (stated there beside each routine); the per-monomial and per-row
structure is that of ``csrc/points.cuh``.  ncu's per-thread FP64 instruction counters
(``smsp__sass_thread_inst_executed_op_{dadd,dmul,dfma}_pred_on.sum``) check the total.
"""
from __future__ import annotations

import numpy as np

# FP64 instructions per operation, per limb count L
C_MUL = {1: 4, 2: 32, 4: 2 * 141}      # normalised complex product
C_MUL_NN = {1: 4, 2: 26, 4: 2 * 141}   # product feeding a product or a sum
C_ADD = {1: 2, 2: 16, 4: 2 * 47}
R_ADD = {1: 1, 2: 8, 4: 47}
C_ACC = {1: 2, 2: 10, 4: 2 * 47}       # a term of a running sum (c_acc)
C_SETTLE = {1: 0, 2: 6, 4: 0}          # the running sum renormalised at its end
C_MUL_D = {1: 2, 2: 12, 4: 2 * 40}


def scale_int(L: int, k: int) -> int:
    """c_scale_int: free for 1 and for powers of two (exponent arithmetic on the bit
    pattern), c_mul_d otherwise."""
    if k == 1 or k & (k - 1) == 0:
        return 0
    return C_MUL_D[L]


def pow_mults(e: int) -> int:
    """Multiplications of c_pow (binary powering) for exponent e."""
    if e <= 0:
        return 0
    return (bin(e).count("1") - 1) + (e.bit_length() - 1)


def eval_ops_per_point(s, L: int, homotopy: bool = True, jac: bool = True) -> int:
    """FP64 instructions of the evaluation kernel for one point of system ``s``."""
    cm, cn, ca = C_MUL[L], C_MUL_NN[L], C_ACC[L]
    total = 0
    vp, ve = s.var_ptr, s.var_exp
    for m in range(s.nmon):
        k = int(vp[m + 1] - vp[m])
        ex = ve[vp[m]:vp[m + 1]]
        if k == 0:
            total += ca
            continue
        n2 = int(np.sum(ex >= 2))
        if not jac:
            total += (n2 + k) * cn + ca
            continue
        nmul = n2 + (3 * k - 3 if k >= 2 else 1)
        total += nmul * cn + (k + 1) * ca + sum(scale_int(L, int(a)) for a in ex)
    # f_i and the row of J are running sums, renormalised once per row
    total += s.npoly * (1 + (s.n if jac else 0)) * C_SETTLE[L]
    if homotopy:
        deg = np.zeros(s.npoly, dtype=np.int64)
        for i in range(s.npoly):
            for m in range(s.mon_ptr[i], s.mon_ptr[i + 1]):
                deg[i] = max(deg[i], int(ve[vp[m]:vp[m + 1]].sum()))
        for i in range(s.npoly):
            d = int(deg[i])
            row = (pow_mults(d - 1) + 2) * cm + R_ADD[L] + C_MUL_D[L] + C_ADD[L]
            if jac:
                row += s.n * C_MUL_D[L] + scale_int(L, d) + cm + C_ADD[L]
            total += row
    return total


def powers_ops_per_point(s, L: int) -> int:
    """FP64 instructions of the power-table kernel for one point."""
    emax = int(s.var_exp.max()) if len(s.var_exp) else 1
    return s.n * max(emax - 2, 0) * C_MUL[L]


def lu64_ops(n: int) -> int:
    """FP64 instructions of the block FP64 LU (`block_lu64`) of an n x n complex matrix:
    per column k the pivot moduli (3 per row), the multipliers (4 each) and the trailing
    update (4 per entry, a complex FMA)."""
    return sum(3 * (n - k) + 4 * (n - k - 1) + 4 * (n - k - 1) ** 2 for k in range(n))


def lu64_solve_ops(n: int) -> int:
    """FP64 instructions of one solve with the FP64 factors: forward and back substitution,
    4 per complex multiply-add, 4 per diagonal product."""
    return 4 * (n * (n - 1) // 2) * 2 + 4 * n


def newton_iteration_ops(s, L: int) -> int:
    """FP64 instructions of one Newton iteration of the path tracker's FP64-LU mode, refinement
    sweeps not counted (so a lower bound): evaluation of h and its Jacobian, the FP64 LU and
    the first solve."""
    return eval_ops_per_point(s, L) + lu64_ops(s.n) + lu64_solve_ops(s.n)
