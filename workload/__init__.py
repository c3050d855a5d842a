"""Seeded synthetic workloads for the coherent F-statistic.

This package draws random numbers and lays out shapes; it holds none of the
method's arithmetic (no timing, antenna patterns, phases or Dirichlet sums).
Both the oracle tests and the GPU path read the inputs it produces.
"""
from .generate import *  # noqa: F401,F403
