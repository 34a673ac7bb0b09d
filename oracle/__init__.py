"""FP64 CPU oracle for the polymer-flooding Newton step (arXiv 1807.05298).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import, call or execute anything
under ``oracle/``.  The CUDA path (``paper_1807_05298_gb300``) shares no code
with it and never calls it.

Contents:
  dual.py    forward-mode dual numbers (exact Jacobians)
  model.py   properties, set-up, residual/Jacobian, wells, Newton (Alg. 1),
             forcing term (Sec. 3.3), time loop
  linalg.py  dense LU with partial pivoting (Golub and Van Loan, Alg.
             3.4.1), the check on the sparse direct solve that model.py uses
"""
