"""CPU float64 oracle of the randomized range finder and randomized SVD.

TEST INFRASTRUCTURE.  Only tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of bench.py may import or run
anything in this package.  It shares no code with the CUDA library: the two
meet only through the seeded input generators in ``synth`` and through the
published definition of the Philox4x32-10 generator that each side implements
on its own.

Modules (each cites the passage of Halko, Martinsson and Tropp,
"Finding structure with randomness", that it follows):
  philox       -- Philox4x32-10 + Box-Muller Gaussian test matrices (Alg. 4.1 step 1)
  rsvd64       -- Algorithms 4.1, 4.3, 4.4 (Stage A) and 5.1 + Remark 5.1 (Stage B)
  jacobi       -- one-sided Jacobi SVD, a second route to Algorithm 5.1 step 2
  srft         -- SRFT test matrix and the FFT sketch (Section 4.6, Algorithm 4.5)
  single_pass  -- two-sided one-pass sketch and min-residual B (Section 5.5)
  grad         -- gradient of the rank-k reconstruction loss, Omega fixed
  metrics      -- error norms and comparison helpers
  bounds       -- the error bounds of Theorems 1.1, 1.2, 9.1, 10.5, 10.6, Cor. 10.10

Every function is pinned by tests/test_oracle_*.py against facts fixed by the
paper or by mathematics (closed forms, exact-rank recovery, the deterministic
bound of Theorem 9.1, brute force on tiny inputs, published known-answer
vectors).  Parity status of each function is listed in the design notes.
"""
