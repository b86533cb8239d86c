"""FP64 CPU oracle for the adaptive multigrid CP-ALS method (De Sterck & Miller).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
NumPy restatement of the paper's mathematics, used to check the CUDA path.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The product library never imports or calls it,
and it shares no code with the CUDA path (only the seeded input generators in
``paper_1111_6091_gb300.synth`` feed both sides).

All arithmetic is float64.  Library primitives used as single steps: matrix
products, ``numpy.linalg.cholesky``/``solve``/``pinv``, and
``scipy.optimize.linear_sum_assignment`` for factor alignment.

Modules
-------
tensor     matricization, n-mode product, Khatri-Rao, MTTKRP, f, gradient, g
           (Sections 2-3; Eqs. for Phi, Gamma, G, f and g)
als        ALS (block nonlinear Gauss-Seidel with pseudoinverse), normalization,
           sorting, and the BNGS relaxation with inner Gauss-Seidel (Sections 3, 5.2)
multigrid  coarsening, least-squares interpolation, Cholesky-transformed
           Galerkin coarse tensors, CP-AMG-mult (Algorithm 1), CP-FAS
           (Algorithm 2), FMG-CP-FAS (Algorithm 3) and the setup/solve driver
           (Sections 4, 5, 6.1)
align      permutation/scaling alignment of two CP solutions (Section 1
           indeterminacies) for error reporting

Parity status: every function is pinned by ``tests/test_oracle_*.py`` except
where a module header says "parity unpinned".
"""
from . import tensor, als, multigrid, align  # noqa: F401
