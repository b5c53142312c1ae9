"""FP64 CPU oracle for FastTT (Li, Yu, Batselier, "Faster Tensor Train
Decomposition for Sparse Data").

TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this package; only
the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` (its CPU-baseline leg and its reference arm) may import or run it.  It shares no code with the CUDA path.

Modules
-------
fasttt   the sparse decomposition (Theorem 1, Alg. 4/5, value-aware Alg. 3,
         Alg. 6, Alg. 8, Alg. 9, eq. (5)-(8)) in plain numpy/scipy FP64.
dense    dense brute force: Alg. 1 TT-SVD, unfoldings, TT contraction,
         the TT sum of Lemma 2, TT norms of differences and Alg. 2 TT-rounding.
tteval   TT entry evaluation (Section 2.3 entry formula), its exact gradient and
         gradient-descent fitting of a fixed-rank TT to entries.
"""
from . import dense, fasttt, tteval  # noqa: F401
