"""GB300-native restarted-PDHG (PDLP) linear-programming solver.

The solver is the C-ABI library libpdlp_gb300.so (include/pdlp.h) built from
csrc/ for sm_103a; ``pdlp`` is its ctypes binding.
"""

from . import _build
from .pdlp import (
    ITER_LIMIT,
    NUMERICAL,
    OPTIMAL,
    TIME_LIMIT,
    PdlpError,
    Solver,
    pdlp_default_params,
    pdlp_params,
)

__all__ = [
    "Solver",
    "PdlpError",
    "pdlp_params",
    "pdlp_default_params",
    "OPTIMAL",
    "ITER_LIMIT",
    "TIME_LIMIT",
    "NUMERICAL",
    "build",
]


def build(force: bool = False) -> str:
    return _build.build(force=force)
