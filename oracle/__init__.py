"""FP64 CPU oracle of the OPO split-step hot path (test infrastructure).

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline legs may
import this package.  It shares no code with ``paper_2410_02532_gb300``.
"""
