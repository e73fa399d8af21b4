"""Seeded synthetic inputs for the Helmholtz workloads (shared by the CUDA
library's tests/bench and by the oracle).

Holds none of the solver's arithmetic: it only evaluates wave-speed fields,
sources and boundary data at node coordinates that the CALLER supplies (each
side computes its own node positions), and samples problem parameters.
"""

from . import fields, configs  # noqa: F401
