"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA path.

This package produces the *inputs* of the method — the time sequence of sparse
matrices A(t_i) and right-hand sides b(t_i) of a 2-D variable-coefficient
elliptic problem (the kind of sequence the paper's Section 1, eq. (1), and
Sections 4-5 consider) and the random draws of the batched and learned
workloads.  It contains none of the method's arithmetic: no sketch, no least
squares, no Krylov step.
"""
from .pde import (PDEParams, assemble, rhs, csr_system, time_grid, pattern,
                  plain_spd, plain_nonsym,
                  batched_params, learned_amplitudes, splitmix64_stream)

__all__ = ["PDEParams", "assemble", "rhs", "csr_system", "time_grid", "pattern",
           "plain_spd", "plain_nonsym",
           "batched_params", "learned_amplitudes", "splitmix64_stream"]
