"""The C ABI on the host: the library loads, exports every symbol the header declares,
and rejects malformed input with HC_EINVAL before touching the device."""
import ctypes as ct
import os
import re

import numpy as np
import pytest

from paper_1109_0545_gb300 import hc, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(hc_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_symbols()
    for want in ("hc_system_load", "hc_system_free", "hc_eval_jac", "hc_newton_step",
                 "hc_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol():
    lib = hc.load()
    for name in declared_symbols():
        assert hasattr(lib, name), name


def _load(s, prec=2, **over):
    d = dict(n=s.n, npoly=s.npoly, mon_ptr=s.mon_ptr.copy(), var_ptr=s.var_ptr.copy(),
             var_idx=s.var_idx.copy(), var_exp=s.var_exp.copy(),
             coef=s.coef_limbs(prec if prec in (1, 2, 4) else 2),
             prec=prec, gamma=(0.6, 0.8))
    d.update(over)
    return hc.hc_system_load(d["n"], d["npoly"], d["mon_ptr"], d["var_ptr"], d["var_idx"],
                             d["var_exp"], d["coef"], d["prec"], d["gamma"])


@pytest.fixture
def small():
    return synth.random_system(np.random.default_rng(5), 4, 3, 2, (1, 3), const_term=True)


def test_rejects_unsorted_indices(small):
    vi = small.var_idx.copy()
    vi[0], vi[1] = vi[1], vi[0]
    with pytest.raises(hc.HCError) as e:
        _load(small, var_idx=vi)
    assert e.value.code == hc.HC_EINVAL and "increasing" in str(e.value)


def test_rejects_zero_exponent(small):
    ve = small.var_exp.copy()
    ve[2] = 0
    with pytest.raises(hc.HCError) as e:
        _load(small, var_exp=ve)
    assert e.value.code == hc.HC_EINVAL


def test_rejects_index_out_of_range(small):
    vi = small.var_idx.copy()
    vi[-1] = small.n
    with pytest.raises(hc.HCError) as e:
        _load(small, var_idx=vi)
    assert e.value.code == hc.HC_EINVAL


def test_rejects_nonfinite_coefficient(small):
    c = small.coef_limbs(2)
    c[1, 0, 1] = np.nan
    with pytest.raises(hc.HCError) as e:
        _load(small, coef=c)
    assert e.value.code == hc.HC_EINVAL and "finite" in str(e.value)


@pytest.mark.parametrize("prec", [0, 3, 8])
def test_rejects_bad_precision(small, prec):
    with pytest.raises(hc.HCError) as e:
        _load(small, prec=prec, coef=small.coef_limbs(2))
    assert e.value.code == hc.HC_EINVAL


def test_rejects_too_many_variables_per_monomial():
    n = 70
    s = synth.System(n=n, npoly=1, mon_ptr=np.array([0, 1], np.int32),
                     var_ptr=np.array([0, 33], np.int32), var_idx=np.arange(33, dtype=np.int32),
                     var_exp=np.ones(33, np.int32), coef=np.array([1.0 + 0j]))
    with pytest.raises(hc.HCError) as e:
        _load(s)
    assert e.value.code == hc.HC_EINVAL


def test_null_handle_calls_fail_cleanly():
    lib = hc.load()
    assert lib.hc_eval_jac(None, 1, 0.5, None, None, None, None) == hc.HC_EINVAL
    assert lib.hc_newton_step(None, 1, 0.5, None, 0, 1, None, None, None, None) == hc.HC_EINVAL
    lib.hc_system_free(None)  # no-op
    assert lib.hc_system_set_eval_mode(None, hc.HC_EVAL_SHARED) == hc.HC_EINVAL
    assert lib.hc_system_eval_mode(None, None, None) == hc.HC_EINVAL
    assert lib.hc_system_info(None, None, None, None, None, None, None, None) == hc.HC_EINVAL
    # the tracker validates its arguments (and options) before touching the device
    opts = hc.hc_track_opts_default()
    stats = (hc.PathStats * 1)()
    assert lib.hc_track_path(None, 1, None, None, ct.byref(opts), stats, None, 0, None) == hc.HC_EINVAL
    states = hc.new_states(1)
    assert lib.hc_track_resume(None, 1, None, None, states, 1, ct.byref(opts), stats, None, 0, None) == hc.HC_EINVAL
    assert lib.hc_last_error()  # a message says why


@pytest.mark.gpu
def test_resume_rejects_bad_states_before_any_launch(small):
    """hc_track_resume checks its arguments and every saved state on the host: a NULL
    buffer, max_stages < 1, an unknown phase, a history of 0 or 4 points, an end game
    before t = 1, tracking at t = 1.  Every case returns HC_EINVAL without a device."""
    s = synth.regular_system(np.random.default_rng(6), 3, 4, (1, 2), (1, 2), lead=3)
    h = hc.system_from(s, 2, 0.6 + 0.8j)   # loading a system needs the device
    lib = hc.load()
    opts = hc.hc_track_opts_default()
    stats = (hc.PathStats * 1)()
    handles = (ct.c_void_p * 1)(h.handle)
    fake = ct.c_void_p(256)   # never dereferenced: the checks come first

    def call(state, max_stages=1, x=fake, hist=fake):
        return lib.hc_track_resume(handles, 1, x, hist, state, max_stages, ct.byref(opts), stats, None, 0, None)

    st = hc.new_states(1)
    assert call(st, x=None) == hc.HC_EINVAL
    assert call(st, hist=None) == hc.HC_EINVAL
    assert call(st, max_stages=0) == hc.HC_EINVAL
    for field, value, phase, t in (("phase", 7, 7, 0.5), ("nhist", 0, 1, 0.5), ("nhist", 4, 1, 0.5),
                                   ("t", 0.5, 2, 0.5), ("t", 1.0, 1, 1.0)):
        st = hc.new_states(1)
        st[0].phase, st[0].nhist, st[0].lambda_, st[0].t = phase, 2, 0.01, t
        setattr(st[0], field, value)
        assert call(st) == hc.HC_EINVAL, (field, value)
    h.free()


def test_option_defaults_follow_the_readings():
    """The defaults of hc_track_opts_default are the readings of Alg. 3.1's constants:
    lambda0 0.01, halve on failure, double after 3 successes up to 0.08 (the 0.01 2^j
    lattice of Tables 2-3), lambda_min 1e-12, 3 Newton iterations per stage."""
    o = hc.hc_track_opts_default()
    assert (o.lambda0, o.shrink, o.grow, o.grow_after, o.lambda_max) == (0.01, 0.5, 2.0, 3, 0.08)
    assert (o.lambda_min, o.max_it, o.max_steps) == (1e-12, 3, 100000)
    assert o.predictor == hc.HC_PRED_SECANT and o.explore == 0.0 and not o.proposer


def test_layout_round_trip():
    rng = np.random.default_rng(3)
    limbs = rng.normal(size=(7, 5, 3, 2, 2))
    soa = hc.to_soa(None, 2, limbs)
    assert soa.shape == (2, 2, 5, 3, 7)
    assert soa[1, 0, 4, 2, 6] == limbs[6, 4, 2, 1, 0]
    assert np.array_equal(hc.from_soa(soa), limbs)


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the option, statistics and log structs have the sizes and
    field offsets that a C compiler gives the declarations in include/hc.h."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"hc_track_opts": hc.TrackOpts, "hc_path_stats": hc.PathStats, "hc_path_state": hc.PathState}
    cnames = {"lambda_": "lambda"}   # a Python keyword in the ctypes mirror
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hc.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {cnames.get(fname, fname)}));')
    lines.append('printf("hc_step_record size %zu\\n", sizeof(hc_step_record));')
    for fname, cfield in (("t", "t"), ("lam", "lambda"), ("res_first", "res_first"), ("res_last", "res_last"),
                          ("pc_dist", "pc_dist"), ("cond_log10", "cond_log10"), ("iters", "iters"),
                          ("accepted", "accepted")):
        lines.append(f'printf("hc_step_record {fname} %zu\\n", offsetof(hc_step_record, {cfield}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ct.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
    rec = hc.STEP_RECORD_DTYPE
    assert got[("hc_step_record", "size")] == rec.itemsize
    for fname in rec.names:
        assert got[("hc_step_record", fname)] == rec.fields[fname][1], fname


def test_track_tiles_reject_bad_shapes():
    """hc_set_track_tiles accepts 0 (automatic) or 64 / 128 / 256 / 512 threads per block, 0..32
    blocks per SM, factor placement 0..2 and a chunk of 0..4096; anything else is HC_EINVAL
    and leaves the setting as it was.  Host-side only."""
    lib = hc.load()
    assert lib.hc_set_track_tiles(128, 4, 2, 64) == hc.HC_SUCCESS
    assert lib.hc_set_track_tiles(512, 1, 0, 0) == hc.HC_SUCCESS
    assert lib.hc_set_track_tiles(128, 4, 2, 64) == hc.HC_SUCCESS
    for bad in ((96, 0, 0, 0), (-1, 0, 0, 0), (1024, 0, 0, 0), (0, 33, 0, 0), (0, 0, 3, 0), (0, 0, 0, -1),
                (0, 0, 0, 5000)):
        assert lib.hc_set_track_tiles(*bad) == hc.HC_EINVAL, bad
    assert hc.hc_get_track_tiles() == {"threads_per_block": 128, "blocks_per_sm": 4, "factors": 2, "grid_chunk": 64}
    hc.hc_set_track_tiles(0, 0, 0, 0)
