"""FP64 CPU oracle for OS-LALM PWLS CT reconstruction.

TEST INFRASTRUCTURE: only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` may import this package.  It shares no code with
the CUDA path (``paper_1402_4381_gb300``); both consume the same seeded inputs
from ``paper_1402_4381_gb300.synth``.
"""
