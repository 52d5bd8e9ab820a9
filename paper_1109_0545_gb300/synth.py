"""Seeded synthetic inputs shaped like the paper's experiments.

This module draws random sparse polynomial systems, evaluation points and the homotopy
constant gamma.  It holds none of the method's arithmetic: it only draws numbers, and
both the CUDA library's tests and the CPU oracle consume what it draws.

Recipe (the paper's own generator is not specified, Sec. 4, 5 and 7 describe only shapes):
  * the support of a monomial is a uniform random k-subset of {0..n-1}, sorted increasing
    (the normalised form of Sec. 6);
  * exponents are uniform integers in [e_lo, e_hi];
  * coefficients are exp(i theta), theta uniform in [0, 2 pi), leading limb cos/sin in
    double, lower limbs zero;
  * points are uniform on the unit torus |x_j| = 1;
  * gamma is exp(i theta) for one more uniform theta.
Draw order for one random system (vectorised over the whole system): the monomial count
of every polynomial (if ranged), the k of every monomial (if ranged), one uniform key per
(monomial, variable) (the support is the k variables with the smallest keys, sorted), the
exponents, the coefficient angles, then the constant-term angles if requested.  numpy's
default_rng(seed) generates everything; a family of systems uses default_rng([seed, j])
for system j, so system j can be drawn without the others.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class System:
    """A sparse polynomial system in the CSR form the library's loader takes."""
    n: int
    npoly: int
    mon_ptr: np.ndarray  # int32 [npoly+1]
    var_ptr: np.ndarray  # int32 [nmon+1]
    var_idx: np.ndarray  # int32 [nvar]
    var_exp: np.ndarray  # int32 [nvar]
    coef: np.ndarray     # complex128 [nmon], leading limbs (lower limbs are zero)

    @property
    def nmon(self) -> int:
        return int(self.mon_ptr[-1])

    @property
    def nvar(self) -> int:
        return int(self.var_ptr[-1])

    def as_dict(self) -> dict:
        return {"n": self.n, "npoly": self.npoly, "mon_ptr": self.mon_ptr,
                "var_ptr": self.var_ptr, "var_idx": self.var_idx, "var_exp": self.var_exp}

    def coef_limbs(self, L: int) -> np.ndarray:
        """coef[m][2][L]: re limbs then im limbs, leading limb first."""
        return limbs(self.coef, L)


def limbs(z: np.ndarray, L: int) -> np.ndarray:
    """Complex doubles -> [..., 2, L] with the lower limbs zero."""
    z = np.asarray(z, dtype=np.complex128)
    out = np.zeros(z.shape + (2, L), dtype=np.float64)
    out[..., 0, 0] = z.real
    out[..., 1, 0] = z.imag
    return out


def _draw(rng, v):
    if isinstance(v, tuple):
        return int(rng.integers(v[0], v[1] + 1))
    return int(v)


def random_system(rng: np.random.Generator, n: int, mons_per_poly, k, exps,
                  const_term: bool = False, npoly: int | None = None) -> System:
    """One random system.  mons_per_poly and k are ints or inclusive (lo, hi) ranges,
    exps is an inclusive (lo, hi) range.  Drawn whole-system at a time (vectorised): the
    monomial counts of all polynomials, the k of every monomial, one uniform key per
    (monomial, variable) whose k smallest give the support (a uniform k-subset), the
    exponents, the coefficient angles, then the constant terms' angles."""
    npoly = n if npoly is None else npoly
    if isinstance(mons_per_poly, tuple):
        m = rng.integers(mons_per_poly[0], mons_per_poly[1] + 1, size=npoly)
    else:
        m = np.full(npoly, int(mons_per_poly))
    mt = int(m.sum())
    if isinstance(k, tuple):
        ks = rng.integers(k[0], k[1] + 1, size=mt)
    else:
        ks = np.full(mt, int(k))
    keys = rng.random((mt, n))
    order = np.argsort(keys, axis=1)
    kmax = int(ks.max()) if mt else 0
    sup = np.sort(np.where(np.arange(kmax)[None, :] < ks[:, None], order[:, :kmax], n), axis=1)
    var_idx = sup[sup < n].astype(np.int32)      # row by row, each row sorted
    var_exp = rng.integers(exps[0], exps[1] + 1, size=int(ks.sum())).astype(np.int32)
    th = rng.uniform(0.0, 2.0 * np.pi, size=mt)
    coef = np.cos(th) + 1j * np.sin(th)
    var_ptr = np.concatenate([[0], np.cumsum(ks)])
    if not const_term:
        mon_ptr = np.concatenate([[0], np.cumsum(m)])
        return System(n=n, npoly=npoly, mon_ptr=mon_ptr.astype(np.int32), var_ptr=var_ptr.astype(np.int32),
                      var_idx=var_idx, var_exp=var_exp, coef=coef)
    # a constant term (k = 0) closes every polynomial
    thc = rng.uniform(0.0, 2.0 * np.pi, size=npoly)
    ends = np.cumsum(m)
    pos = ends + np.arange(1, npoly + 1) - 1           # index of polynomial i's constant
    mon_ptr = np.concatenate([[0], ends + np.arange(1, npoly + 1)])
    kk = np.insert(ks, ends, 0)
    allc = np.insert(coef, ends, np.cos(thc) + 1j * np.sin(thc))
    assert np.all(kk[pos] == 0)
    return System(n=n, npoly=npoly, mon_ptr=mon_ptr.astype(np.int32),
                  var_ptr=np.concatenate([[0], np.cumsum(kk)]).astype(np.int32),
                  var_idx=var_idx, var_exp=var_exp, coef=allc)


def torus_points(rng: np.random.Generator, npts: int, n: int) -> np.ndarray:
    """npts points uniform on the unit torus, complex128 [npts][n]."""
    th = rng.uniform(0.0, 2.0 * np.pi, size=(npts, n))
    return np.cos(th) + 1j * np.sin(th)


def unit_complex(rng: np.random.Generator) -> complex:
    th = rng.uniform(0.0, 2.0 * np.pi)
    return complex(np.cos(th), np.sin(th))


def fixed_degree_system(rng: np.random.Generator, n: int, mons_per_poly, degree: int, kmax: int = 8,
                        const_term: bool = False) -> System:
    """A random system whose monomials all have total degree `degree` (the shapes of the
    paper's experiments, "monomials of degree D", Sec. 5 and 7): per monomial k uniform in
    {1..min(degree, kmax, n)}, a uniform random k-subset of the variables, and exponents a
    uniform random composition of `degree` into k positive parts (k-1 distinct cut points
    drawn from {1..degree-1}); theta uniform.  Draw order per monomial: k, support, cut
    points, theta; then a constant-term theta if requested."""
    mon_ptr = [0]
    var_ptr = [0]
    idx: list[np.ndarray] = []
    ex: list[np.ndarray] = []
    thetas: list[float] = []
    kk_max = max(1, min(degree, kmax, n))
    for _ in range(n):
        m_i = _draw(rng, mons_per_poly)
        for _ in range(m_i):
            kk = int(rng.integers(1, kk_max + 1))
            sup = np.sort(rng.choice(n, size=kk, replace=False)).astype(np.int32)
            cuts = np.sort(rng.choice(np.arange(1, degree), size=kk - 1, replace=False)) if kk > 1 else np.zeros(0)
            e = np.diff(np.concatenate([[0], cuts, [degree]])).astype(np.int32)
            idx.append(sup)
            ex.append(e)
            var_ptr.append(var_ptr[-1] + kk)
            thetas.append(rng.uniform(0.0, 2.0 * np.pi))
        cnt = m_i
        if const_term:
            var_ptr.append(var_ptr[-1])
            thetas.append(rng.uniform(0.0, 2.0 * np.pi))
            cnt += 1
        mon_ptr.append(mon_ptr[-1] + cnt)
    th = np.array(thetas)
    return System(n=n, npoly=n, mon_ptr=np.array(mon_ptr, dtype=np.int32),
                  var_ptr=np.array(var_ptr, dtype=np.int32),
                  var_idx=np.concatenate(idx).astype(np.int32), var_exp=np.concatenate(ex).astype(np.int32),
                  coef=np.cos(th) + 1j * np.sin(th))


def _with_leading_powers(s: System, lead: int) -> System:
    """s plus, in polynomial i, the monomial x_i^D with coefficient 1, D = max(lead, 1 + the
    largest total degree in s), placed last in the polynomial."""
    cs = np.concatenate([[0], np.cumsum(s.var_exp, dtype=np.int64)])
    top = int((cs[s.var_ptr[1:]] - cs[s.var_ptr[:-1]]).max()) if s.nmon else 0
    lead = max(lead, top + 1)
    ends = s.mon_ptr[1:]                      # the new monomial goes after these
    ks = np.insert(np.diff(s.var_ptr), ends, 1)
    vpos = s.var_ptr[ends]
    return System(n=s.n, npoly=s.npoly, mon_ptr=(s.mon_ptr + np.arange(s.npoly + 1)).astype(np.int32),
                  var_ptr=np.concatenate([[0], np.cumsum(ks)]).astype(np.int32),
                  var_idx=np.insert(s.var_idx, vpos, np.arange(s.npoly)).astype(np.int32),
                  var_exp=np.insert(s.var_exp, vpos, lead).astype(np.int32),
                  coef=np.insert(s.coef, ends, 1.0 + 0j))


def regular_system(rng: np.random.Generator, n: int, mons_per_poly, k, exps,
                   lead: int) -> System:
    """A random system (as random_system) plus, in polynomial i, the monomial x_i^D with
    coefficient 1, D = max(lead, 1 + the largest total degree of the other monomials).
    Its leading forms then vanish together only at 0, so no path of the total-degree
    homotopy goes to infinity: test systems whose paths should end at roots.  Each
    polynomial also gets a constant term, so that x = 0 (a singular root of a system
    without constants) is not a root."""
    return _with_leading_powers(random_system(rng, n, mons_per_poly, k, exps, const_term=True), lead)


# ---------------------------------------------------------------------------------------
# The workloads.  Each returns plain data; sizes can be reduced for tests.
# ---------------------------------------------------------------------------------------

def single_path_dd(seed: int = 1):
    """One path, complex DD: n = 8, 8 polynomials of 12 monomials plus a constant term,
    3 distinct variables per monomial, exponents in {1,2,3}.  Returns (system, gamma)."""
    rng = np.random.default_rng(seed)
    s = random_system(rng, 8, 12, 3, (1, 3), const_term=True)
    return s, unit_complex(rng)


def eval_throughput(seed: int = 2, npts: int = 65536, n: int = 32, mons: int = 128,
                    k: int = 6, exps=(1, 4)):
    """Eval+Jacobian throughput workload: n = 32, 32 x 128 monomials, k = 6, exponents
    in {1..4}; npts points on the unit torus.  Returns (system, points, gamma)."""
    rng = np.random.default_rng(seed)
    s = random_system(rng, n, mons, k, exps)
    gamma = unit_complex(rng)
    pts = torus_points(rng, npts, n)
    return s, pts, gamma


def uneven_path_system(seed: int, j: int):
    """System j of the batched uneven-path family: n in {10..64}, monomials per
    polynomial in {20..200}, variables per monomial in {2..8}, exponents in {1..3}.
    Returns (system, gamma)."""
    rng = np.random.default_rng([seed, j])
    n = int(rng.integers(10, 65))
    s = random_system(rng, n, (20, 200), (2, 8), (1, 3))
    return s, unit_complex(rng)


def large_path_qd(seed: int = 4, n: int = 96, mons: int = 1024, k: int = 12, exps=(1, 5)):
    """Large single path, complex QD: n = 96, 96 x 1024 monomials, k = 12, exponents in
    {1..5}.  Returns (system, gamma)."""
    rng = np.random.default_rng(seed)
    s = random_system(rng, n, mons, k, exps)
    return s, unit_complex(rng)


def paper_dim_degree(seed: int, n: int, mons: int, degree: int, regular: bool = True):
    """One system of the shapes of the paper's one-path experiments (Tables 2-5): n x n,
    `mons` monomials of total degree `degree` per polynomial.  regular: plus a constant
    and x_i^(degree+1) in polynomial i (the leading powers make every path of the
    total-degree homotopy end at a regular root).  Returns (system, gamma)."""
    rng = np.random.default_rng([seed, n, mons, degree])
    s = fixed_degree_system(rng, n, mons, degree, const_term=regular)
    if regular:
        s = _with_leading_powers(s, degree + 1)
    return s, unit_complex(rng)


def common_support_system(seed: int, n: int = 40, nuniq: int = 200, dmax: int = 80, kmax: int = 32):
    """A system whose n polynomials share one support of `nuniq` monomials (the system
    behind the cost split of Table 1, Sec. 4: 40 variables, 200 monomials of degree 40 on
    average and 80 at most): per monomial a degree d uniform in {1..dmax}, k uniform in
    {1..min(d, n, kmax)}, a uniform random k-subset, exponents a uniform random
    composition of d into k parts; then a coefficient theta per (polynomial, monomial),
    polynomial by polynomial.  Returns (system, gamma)."""
    rng = np.random.default_rng([seed, n, nuniq, dmax])
    sup, exps = [], []
    for _ in range(nuniq):
        d = int(rng.integers(1, dmax + 1))
        kk = int(rng.integers(1, min(d, n, kmax) + 1))
        sup.append(np.sort(rng.choice(n, size=kk, replace=False)).astype(np.int32))
        cuts = np.sort(rng.choice(np.arange(1, d), size=kk - 1, replace=False)) if kk > 1 else np.zeros(0)
        exps.append(np.diff(np.concatenate([[0], cuts, [d]])).astype(np.int32))
    th = rng.uniform(0.0, 2.0 * np.pi, size=(n, nuniq))
    var_ptr = np.concatenate([[0], np.cumsum([len(x) for x in sup] * n)]).astype(np.int32)
    s = System(n=n, npoly=n, mon_ptr=(np.arange(n + 1) * nuniq).astype(np.int32), var_ptr=var_ptr,
               var_idx=np.concatenate(sup * n).astype(np.int32), var_exp=np.concatenate(exps * n).astype(np.int32),
               coef=(np.cos(th) + 1j * np.sin(th)).ravel())
    return s, unit_complex(rng)
