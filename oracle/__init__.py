"""CPU oracle for the fused preprocessing path -- TEST INFRASTRUCTURE ONLY.

Imported by the tests, by ``__graft_entry__.smoke()`` and by the CPU-baseline
legs of ``bench.py``; never by the library. See ``fkl_oracle`` for what each
function computes and which passage of the paper it follows.
"""
from .fkl_oracle import *  # noqa: F401,F403
from . import fkl_oracle  # noqa: F401
