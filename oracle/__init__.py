"""CPU oracle for the DD/QD path tracker's hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It shares no code with the CUDA library: its arithmetic lives in
``hc_oracle.c`` (exact floating-point expansions rounded once per operation), compiled
here with gcc, and its Python side only marshals numpy arrays.

Layout of all arrays handed to or returned by the oracle: point-major, complex parts
split into limbs -- x[p][j][2][L], f[p][i][2][L], J[p][i][j][2][L], coef[m][2][L].
"""
from .wrap import (  # noqa: F401
    build, lib, r_add, r_mul, r_div, c_mul, c_div, degrees, validate, evaluate,
    evaluate_threads, solve, newton_step, newton_threads, track, track_replay, track_resume, predict,
    TrackOpts, PathState, STATUS,
)
