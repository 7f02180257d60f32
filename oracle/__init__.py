"""SFHK oracle: a plain FP64 CPU restatement of the paper's trajectory path.

Test infrastructure only.  ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  It shares no code with the
CUDA library under ``paper_2601_17164_gb300/``.
"""
from .oracle import *  # noqa: F401,F403
