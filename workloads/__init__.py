"""Seeded synthetic inputs shared by the oracle and the GPU library's tests/bench.

This package holds no arithmetic of the nonlinear FEAST method: it only draws
random numbers and builds the coefficient matrices of the test problems.
"""
from .generators import *  # noqa: F401,F403
