"""CPU oracle for the sketched subspace-acceleration hot path.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of
what the GPU library computes, written so that a reader can check it against
the paper (Guido, Kressner, Ricci, "Subspace acceleration for a sequence of
linear systems and application to plasma simulation", arXiv 2309.02156) by
eye.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the product library never does, and the
two share no code.  Inputs come from the separate ``workloads`` package.

Modules
-------
sketch   sparse-sign row sketch S (s x n, zeta nonzeros of +-1/sqrt(zeta) per
         column) generated from SplitMix64 counters, and W = S [A X | b].
lsq      column-scaled, column-pivoted Householder least squares with rank
         truncation (the reduced problem of Algorithm 1).
krylov   CSR products, CG (Hestenes-Stiefel), restarted GMRES with CGS2
         Arnoldi, and mixed-precision iterative refinement.
method   Algorithm 1 of the paper with the subspace S = span(X) and the
         least-squares problem sketched by S; the previous-solution guess.
basis    Algorithm 2 (POD basis) and Algorithm 4 (randomized range finder with
         progressive updates), the paper's compressed subspaces.
mlp      the learned coefficient predictor (forward, backward, Adam).

Parity status of each function is stated in its docstring; every function
listed above is pinned by a ``-m "not gpu"`` test unless its docstring says
"parity unpinned".
"""
