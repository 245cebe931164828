"""Plain FP64 CPU oracle for the Cox / Fine-Gray CCD hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the product package imports this
module. The only callers allowed are the tests under ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``.

The oracle shares no code, constants or helpers with the CUDA path.  It is
written from the paper's equations (Sections 2.1-2.4 and 2.7) in float64
with numpy, as slow and plain as possible so that it can be checked against
the paper by eye.  Every function cites the passage it follows.

Parity status of each function is listed in ``oracle/survival.py``'s header.
"""
from .survival import *  # noqa: F401,F403
from .nll import *  # noqa: F401,F403
from .cv import *  # noqa: F401,F403
from .sparse_numerator import *  # noqa: F401,F403
