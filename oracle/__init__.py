"""FP64 CPU oracle (test infrastructure only; see ``ptycho_oracle``).

Only ``tests/``, ``__graft_entry__.smoke`` and the CPU-baseline / reference legs of
``bench.py`` use this package.  The GPU library neither imports nor links it.
"""
from . import ptycho_oracle  # noqa: F401
