"""FP64 CPU oracle for the FastLRNR / SPInProp hot path.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; never by the product library.

Parity status per function (what pins it is in ``tests/test_oracle_*.py``):

* ``lrnr64.full_forward``   pinned: central finite differences in x and t;
  torch.autograd FP64 on the dense network ``W = U diag(s) V^T``; closed-form
  convection solution ``u = h(x - beta t)``.
* ``lrnr64.full_backward``  pinned: central finite differences in s and b;
  torch.autograd FP64.
* ``lrnr64.fast_forward`` / ``fast_backward``  pinned: identity with the full
  network when every row is selected; exact agreement with the full network at
  the snapshot points; finite differences; closed-form convection solution.
* ``lrnr64.cdr_residual``   pinned: three closed-form solutions of Eq. 4.1.
* ``eim64.eim_greedy``      pinned: scaled unit vectors, unit lower-triangular
  ``P^T Xi``, exact interpolation of spanned snapshots, brute-force rule replay.
* ``deim64.pod_basis``      pinned: planted spectrum (known singular vectors and
  values, rank cut); eigenvectors of ``S S^T`` and the Eckart-Young projection
  error, both against a symmetric eigen-solver.
* ``deim64.deim_rows``      pinned: equal to the pivot order of LU with partial
  pivoting (LAPACK); unit-vector bases; tie rule; exact interpolation of the span
  and the DEIM bound on ``||(P^T Xi)^{-1}||``; invariance to column scaling and
  equivariance under row relabelling; reduced network exact at the snapshot points
  and equal to the full network when every row is kept.
* ``adam64.adam_step``      pinned: ``torch.optim.Adam`` in FP64.
"""
