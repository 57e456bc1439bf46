"""Plain FP64 CPU oracle for the IgA-SGBEM weighted-quadrature assembly.

TEST INFRASTRUCTURE ONLY.  This package exists so that the tests, the smoke
check and the benchmark's CPU-baseline leg can compare the CUDA path against
an obviously-correct restatement of the paper's method.  Nothing in the
product path (the C-ABI library and its Python binding) imports, links or
executes it, and it shares no code with the CUDA path: the two meet only in
the seeded input generators of ``paper_1703_10016_gb300.workloads``, which
hold no arithmetic of the method.

Source: Aimi, Calabro, Diligenti, Sampoli, Sangalli, Sestini, "Efficient
assembly based on B-spline tailored quadrature rules for the IgA-SGBEM"
(arXiv:1703.10016).  Each function cites the section / equation / algorithm
it follows.

Modules
  bspline        Cox-de Boor values and derivatives, NURBS curve evaluation (Sect. 3)
  discretization test space, exactness space, node vector eta, index sets (Sect. 3, 4, 4.1)
  rules          Algorithm 1 (regular weighted rules), modified moments (eq. mod_mom_gen),
                 Algorithm 2 (singular weighted rules)
  assembly       I_K1 (eq. IK1e2), I_K2 (eq. IK1e2_bis), right-hand side (Sect. 5),
                 Cholesky solve and the error measures E_R, E_M (Sect. 6),
                 representation formula (Sect. 2)
  collocation    collocation form of the single-layer equation with the same rules
                 (Sect. 7 remark), LU solve
  sampled        single entries A[i, j] from local pieces of the same definitions
                 (parity at sizes where the dense arrays do not fit)

Pins: every function is checked in ``tests/test_oracle_*.py`` against
quantities the paper or mathematics fixes (exactness, closed forms, adaptive
quadrature, circle eigenvalues, manufactured solutions, Table 2 condition
numbers).  Functions without such a pin say "parity unpinned" in their
docstring; at present there are none.
"""
from . import bspline, discretization, rules, assembly, collocation, sampled  # noqa: F401
