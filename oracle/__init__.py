"""Plain FP64 CPU oracle for the H_h matrix-vector product.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package imports, calls or
links this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.

It is written from the paper (Khan & Carson, "Hybrid hierarchical matrices
with adaptive mixed precision storage") step by step, in float64 NumPy, with
no blocking, fusion or reordering beyond what the paper states:

  formats.py    Table 1 unit roundoffs; round-to-nearest-even into fp32, fp16,
                bf16 and fp8-e4m3; power-of-two block scales.
  tree.py       cluster tree (binary KD bisection, Section 2.1 adapted) and
                bounding-box geometry.
  partition.py  standard / weak / hybrid admissibility (Eqs. 2.2, 2.4, 3.1)
                and the block partition of Algorithm 1; sparsity constants
                (Eqs. 2.3, 2.5, 2.8).
  compress.py   kernel functions (Eq. 5.1) and LRcompression: truncated SVD
                (Section 2.2) and ACA with SVD recompression.
  build.py      Algorithm 1 + Algorithm 5 (Frobenius norms) + Algorithm 3
                (adaptive precision assignment) + storage formulas.
  matvec.py     Algorithm 4 (b = H_hat x), its transpose, dense assembly.
  switch.py     Algorithm 2 (the switching level with the largest storage
                gain over the H_s matrix).
  solve.py      conjugate gradients for (H_hat + shift I) x = b on
                Algorithm 4's product.
  bounds.py     Theorem 4.2 / 4.4 error bounds and Lemma 3.1.
  hhfile.py     reader/writer of the serialized H_h file (the input both the
                oracle and the CUDA path consume).

Parity status of every function is stated in its module docstring.
"""
