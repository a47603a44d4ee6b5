"""FP64 CPU oracle of nonlinear FEAST.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline / reference leg of bench.py.  The GPU library never uses it.
"""
from .nlfeast_ref import *  # noqa: F401,F403
