"""Benchmark aggregates.

shifted_geometric_mean: the paper's aggregate of solve times over a test set
(Sec. 4.1 reports SGM10: the geometric mean of t_i + 10 s, minus 10 s), which
damps the weight of the many very short solves.
"""

from __future__ import annotations

import math


def shifted_geometric_mean(values, shift: float = 10.0) -> float:
    """exp(mean(log(v_i + shift))) - shift; 0.0 for an empty sequence."""
    vals = [float(v) for v in values]
    if not vals:
        return 0.0
    if any(v + shift <= 0.0 for v in vals):
        raise ValueError("every value must exceed -shift")
    return math.exp(sum(math.log(v + shift) for v in vals) / len(vals)) - shift
