"""GB300-native subspace acceleration for sequences of sparse linear systems.

Python face of libseqaccel (include/seqaccel.h).  Each call marshals torch
tensors (device memory, current stream) into the C-ABI; all arithmetic runs
in the library's CUDA kernels.  There is no CPU path: using this package
without the built library or without a CUDA device raises.

Paper: Guido, Kressner, Ricci, "Subspace acceleration for a sequence of
linear systems and application to plasma simulation" (arXiv 2309.02156):
the guess of Algorithm 1 over span(X) of the last M solutions, here with the
reduced least-squares problem row-sketched by a sparse-sign S, followed by
CG or GMRES from that guess.
"""
from ._binding import (Batch, CSR, MLP, Sequence, SeqError, lib_path, load, probe_fp64_peak,
                       sketch_block_noalloc, sketch_columns, STATUS)

__all__ = ["Batch", "CSR", "MLP", "Sequence", "SeqError", "lib_path", "load", "probe_fp64_peak",
           "sketch_block_noalloc", "sketch_columns", "STATUS"]
