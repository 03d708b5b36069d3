"""Seeded synthetic inputs shared by the GPU path's tests/bench and by the oracle.

This package holds only input generation (counter-based random numbers and flat
phase-space sampling).  It contains none of the matrix-element arithmetic: the
paper's method starts from momenta (the third step of the event-generation chain
described in Sec. 2: random numbers -> momenta -> matrix element).
"""
from .philox import philox4x32_10, uniform01, uniform_open01
from .rambo import rambo, incoming_beams, rambo_massless_weight
from .workloads import Workload, WORKLOADS, make_inputs

__all__ = ["philox4x32_10", "uniform01", "uniform_open01", "rambo", "incoming_beams",
           "rambo_massless_weight", "Workload", "WORKLOADS", "make_inputs"]
