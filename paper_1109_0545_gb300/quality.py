"""Quality up (Sec. 2): at fixed time, how much more precision p processors buy.

The paper counts quality as correct decimal places, assumes optimal speedup, and takes
the ratio of qualities y(p) = Q_p / Q_1 to be linear in p.  With a base precision that
runs in t_base on one processor and a higher precision that runs in t_high on p_high
processors, the higher precision matches t_base on p* = ceil(p_high t_high / t_base)
processors, where y(p*) is the ratio of the two precisions' qualities.
"""
from __future__ import annotations

import math


def processors_for_fixed_time(t_base: float, t_high: float, p_high: int) -> tuple[float, int]:
    """(p_high t_high / t_base, that number rounded up): the processors the higher precision
    needs, at optimal speedup, to finish in the base precision's one-processor time."""
    ratio = p_high * t_high / t_base
    return ratio, math.ceil(ratio - 1e-12)


def quality_up(p: float, p_star: float, y_star: float) -> float:
    """y(p) on the line through y(1) = 1 and y(p*) = y_star, and y_star from p* on (the
    higher precision's quality is all there is to gain)."""
    if p >= p_star:
        return y_star
    return 1.0 + (y_star - 1.0) * (p - 1.0) / (p_star - 1.0)
