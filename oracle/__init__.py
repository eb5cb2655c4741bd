"""Plain FP64 CPU oracle for the Lagrange-dual DCOPF method (test infrastructure).

This package is test infrastructure.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA path and never imports the product package.

Modules:
  dcopf   -- network operators by dense Laplacian solves, the dual function in three
             forms, the supergradient, and the GDM / Adam / AdaGrad ascent rules.
  exact   -- an exact LP/QP solver (dense primal-dual interior point with a
             weak-duality sandwich) and brute-force vertex enumeration for tiny LPs.
  primal  -- primal recovery: a balanced box minimiser (uniform price shift by
             bisection) repaired towards a feasible reference dispatch, whose cost
             is an upper bound on gamma* (weak duality, Remarks 1-2).
  mlp     -- the warm-start perceptron: forward pass, mean-squared-error gradient
             and Adam, in FP64 (the paper has no learned part; any dual proposal
             is a valid bound by Remarks 1-2).

Every function names the passage of "GPU-Accelerated DCOPF using Gradient-Based
Optimization" (arXiv 2406.13191) it follows.  All functions are pinned by
``tests/test_oracle_*.py`` against closed forms, hand-solved cases, brute force and
invariants; none is marked "parity unpinned".
"""
