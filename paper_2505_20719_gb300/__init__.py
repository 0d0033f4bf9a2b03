"""F3R nested Krylov solver (arXiv 2505.20719) for GB300 / sm_103a.

The solver lives in the CUDA library libf3r.so (C ABI: include/f3r.h); this
package is its thin Python binding.  Build it with
``python -c "import __graft_entry__ as g; g.build()"`` or
``python paper_2505_20719_gb300/build.py``.
"""
from .f3r import (  # noqa: F401
    BF16, F16, F32, F64, PC_IDENTITY, PC_JACOBI, F3RError, Params, Result, Solver, Stats, default_params,
    lib, preset,
)
