"""The seeded generators: shapes the paper's experiments name, and determinism."""
import numpy as np

from paper_1109_0545_gb300 import synth


def _degrees(s):
    return [int(s.var_exp[s.var_ptr[m]:s.var_ptr[m + 1]].sum()) for m in range(s.nmon)]


def test_fixed_degree_monomials_have_the_stated_degree():
    for deg in (1, 2, 10, 20):
        s, g = synth.paper_dim_degree(3, 12, 9, deg, regular=False)
        assert s.nmon == 12 * 9
        assert all(d == deg for d in _degrees(s))
        assert np.all(s.var_exp >= 1)
        for m in range(s.nmon):
            sup = s.var_idx[s.var_ptr[m]:s.var_ptr[m + 1]]
            assert np.all(np.diff(sup) > 0) and len(sup) <= min(deg, 8)
        assert abs(abs(g) - 1) < 1e-15 and np.allclose(np.abs(s.coef), 1)


def test_regular_variant_adds_a_constant_and_a_leading_power_per_polynomial():
    s, _ = synth.paper_dim_degree(4, 10, 6, 5)
    for i in range(s.n):
        ms = range(s.mon_ptr[i], s.mon_ptr[i + 1])
        degs = [_degrees(s)[m] for m in ms]
        assert degs.count(0) == 1 and degs.count(5) == 6
        last = s.mon_ptr[i + 1] - 1
        assert s.var_idx[s.var_ptr[last]] == i and s.var_exp[s.var_ptr[last]] == 6
        assert s.coef[last] == 1.0


def test_generators_are_deterministic():
    a, ga = synth.paper_dim_degree(7, 20, 20, 10)
    b, gb = synth.paper_dim_degree(7, 20, 20, 10)
    assert ga == gb
    for f in ("mon_ptr", "var_ptr", "var_idx", "var_exp", "coef"):
        assert np.array_equal(getattr(a, f), getattr(b, f))


def test_common_support_shape():
    s, g = synth.common_support_system(1)
    assert s.n == s.npoly == 40 and s.nmon == 40 * 200
    degs = _degrees(s)
    assert max(degs) <= 80 and 35 <= np.mean(degs) <= 45
    first = [tuple(s.var_idx[s.var_ptr[m]:s.var_ptr[m + 1]]) + tuple(s.var_exp[s.var_ptr[m]:s.var_ptr[m + 1]])
             for m in range(200)]
    for i in range(1, 40):
        for u in range(200):
            m = i * 200 + u
            assert tuple(s.var_idx[s.var_ptr[m]:s.var_ptr[m + 1]]) + \
                tuple(s.var_exp[s.var_ptr[m]:s.var_ptr[m + 1]]) == first[u]
