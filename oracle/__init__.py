"""Plain FP64 CPU oracle for the isogeometric PCG + fast-diagonalization path.

TEST INFRASTRUCTURE ONLY. Nothing in the product library imports, links or
executes this package; only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may use it. It shares no code
with the CUDA path: the only common module is ``synth`` (seeded inputs, no
arithmetic of the method).

Every function follows the paper (Sangalli & Tani, "Isogeometric
preconditioners based on fast solvers for the Sylvester equation") step by
step, in FP64, with numpy/scipy primitives (matmul, Cholesky, triangular
solve, symmetric eigen-solve, sparse solve) as building blocks and no
blocking, fusion or reordering beyond what the definitions state.

Modules
  spline    Section 2.1: open knot vectors, Cox-de Boor recursion, Gauss rule
  assemble  Eqs. (A), (Q), (prec): 1D pencils, geometry map, stiffness matrix A
            in a (2p+1)^d offset layout, right-hand side, dense Kronecker P
  fd        Algorithms 1 and 3: generalized eigendecomposition via Cholesky,
            fast-diagonalization solve of P s = r
  pcg       preconditioned conjugate gradients (the paper's outer solver)
  learned   span scalings of the pencils: features of Q, separable log-fit,
            and the scaling network with its gradient
  adi       Algorithms 2 and 4: two- and three-variable ADI solvers of
            P s = r, their parameters and error operators
  multipatch  Section 6: the C^0 three-patch L-shaped domain, its subdomain
            restrictions and the additive Schwarz preconditioners of
            Eqs. (Peas), (Pias)

Readings where the paper is silent or garbled are stated at each function.
"""
from . import spline, assemble, fd, pcg, learned, adi, multipatch  # noqa: F401
