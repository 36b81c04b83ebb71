"""CPU oracle for the AZ least-squares solver of arXiv 2308.14490 (Zhou & Huybrechs).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 NumPy/SciPy
restatement of the method, written from the paper's equations.  It shares no
code with the CUDA library: it imports nothing from ``paper_2308_14490_gb300``
and the library imports nothing from here.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference leg of
``bench.py`` may import it.  The seeded problem data (grids, masks, right-hand
sides) comes from ``workloads``, which holds none of the method's arithmetic.

Modules
-------
``philox``     Philox4x32-10 counter-based generator and the Rademacher test
               matrix R (Sec. 3.2.3, the random matrix of the low-rank solver).
``rbf``        Gaussian kernel, its second derivative, periodised samples on
               the oversampled grid and the diagonal symbols (Sec. 2.1,
               Eqs. rbf / periodic_rbf; Sec. 3.1 Eq. explicit_d; Lemma 4.2).
``operators``  The full-box operator A^c applied through the FFT and formed
               densely, the plain inverse Z* (Eq. B_pinv, Sec. 3.2.2), the
               restriction to Omega, the boundary rows of Sec. 6.2.
``az``         Algorithm 1 (AZ) with a randomised truncated-SVD step 1, the
               residual refinement, and the dense truncated-SVD least-squares
               solve used as the direct comparison.

Parity status: every function here is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py`` except where its docstring says "parity unpinned".
"""
