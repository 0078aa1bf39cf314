"""Plain, slow FP64 CPU oracle for the Burton-Miller collocation BEM (arXiv 2312.12787).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The CUDA library never calls it and shares no code with it.

Every function cites the passage of the paper it follows.  Parity status of each function is listed
at the top of ``bem_oracle.py``.  ``parallel.py`` only splits the rows of the oracle's assembly over
processes; it adds no arithmetic.
"""
from .bem_oracle import *  # noqa: F401,F403
from .mie import *  # noqa: F401,F403
from .parallel import assemble_parallel, default_workers  # noqa: F401
