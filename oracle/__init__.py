"""CPU oracle for the arrow-decomposition SpMM (test infrastructure only).

Plain, slow, obviously correct restatements of what the paper computes:

* :mod:`oracle.spmm` -- the product the method reaches exactly, Y = A X
  (Eq. 1 is an identity, so the plain FP64 CSR product is the value oracle),
  its iteration X_{t+1} = sigma(A X_t) (Section 2, "Matrices"), and the
  decomposed product sum_i P_i (B_i (P_i^T X)) of Eq. 1 written out.
* :mod:`oracle.cspmm` -- the same FP64 product and iteration as a plain C loop
  (oracle/c/csr_spmm.c, compiled by the project's build step) whose rows run on all host
  cores; the timed CPU baseline.
* :mod:`oracle.decompose` -- LA-Decompose (Section 4.1) with the random
  spanning forest linear arrangement (Section 4.3) and the smallest-first tree
  layout (Section 4.4), step by step in the paper's order.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA path (``paper_2402_19364_gb300``) and imports nothing
from it; inputs come from the seeded generators in :mod:`workloads`.
"""
