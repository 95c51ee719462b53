"""FP64 CPU oracle -- test infrastructure only.

Imported by tests/, __graft_entry__.smoke() and the CPU-baseline leg of
bench.py; never by the product package.  See oracle/oracle.py.
"""
from .oracle import *  # noqa: F401,F403
from .oracle import Oracle, Tallies  # noqa: F401
