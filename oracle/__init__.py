"""FP64 CPU oracle for the primal-dual symmetric-cone MWU framework.

TEST INFRASTRUCTURE ONLY. This package is the slow, plain reference that the
CUDA path is checked against. Only the test suite, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it. The product path (the C-ABI library and its Python binding) never imports,
calls or links anything here, and nothing here imports the product path.

Every function follows the paper (Zheng, Varvitsiotis, Tan, Lin, "A
Primal-Dual Framework for Symmetric Cone Programming", arXiv 2405.09157) and
cites the section, equation or theorem it writes out. Arithmetic is IEEE
float64 through numpy; inputs are promoted to float64 on entry.

Modules
  eja     Jordan-algebra primitives of the second-order cone and R^n_+ (Sec. 2.1)
  ses     Smallest Enclosing Sphere: SCMWU weights, closed-form ORACLE, the
          alpha-FTP loop of Theorem 2 and the search of Sec. 3 (Sec. 4.1)
  svm     Hard-margin SVM / polytope distance, the minimisation variant
          (Theorem 3) with the closed-form ORACLE of Sec. 4.2
  exact   Textbook exact solvers used to pin the oracle on tiny inputs
          (Welzl-style minimum enclosing circle, support-set enumeration for
          balls, active-set enumeration for polytope distance)

Parity status: every function here is pinned by a test under ``tests/``
(closed forms, invariants, brute force); none is "parity unpinned" except
where a docstring says so explicitly.
"""

from . import eja, ses, svm, exact  # noqa: F401
