"""FP64 CPU oracle of the multilevel Monte-Carlo trace estimator (arXiv 2108.11281).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with
the CUDA library in ``paper_2108_11281_gb300/``; the only module both sides use
is the seeded input generator ``paper_2108_11281_gb300/workloads.py``, which
holds none of the method's arithmetic.

Modules:
  philox      Philox4x64-10 and the Rademacher / Z4 noise maps (Sec. 3, Eqs. iid_components1/2)
  operators   2-D Laplacian (Example 5.1) and 2-spin Wilson/Schwinger operator (Example 5.3)
  hierarchy   aggregation hierarchy with orthonormal P and Galerkin coarsening (Sec. 4.1, Ex. 5.3)
  solver      exact level solves; FGMRES + multigrid cycle (Remark 4.1, Ex. 5.3)
  estimator   difference samples, exact coarse trace, estimate, stopping rule and the
              Sec. 2 optimal allocation (Secs. 2, 4, 5)

Parity pins live in tests/test_oracle_pins.py.  The stopping rule's tau / rho
split (Sec. 5 prints no values) is pinned against a hand-derived closed form on
synthetic sample streams (test_stopping_rule_closed_form).
"""
