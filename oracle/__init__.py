"""CPU float64 oracle for the low-rank Matrix Exponentiated Gradient method.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check
and the CPU-baseline leg of the benchmark may import, call or execute
anything here; the product path (the CUDA library and its binding) never
does, and this package never imports the product path.

Modules:
  meg      -- Algorithm 1 (exact MEG), Algorithm 2 (low-rank MEG, exact
              and subspace-iteration eigensolvers), the Lemma 2
              certificate, eq. (exp:init) warm start, objectives.
  linalg   -- eigh wrapper, textbook cyclic Jacobi, simplex and
              spectrahedron projections (eq. euclidProj).
  diag_mp  -- the diagonal special case of Algorithm 2 at 50 digits.

Pins (tests marked "not gpu" check each against something other than
itself): trace/PSD invariants; the factored Frobenius identity; the
closed form of exact MEG for linear objectives; the diagonal recursion
(mpmath golden file); rotation equivariance; the exact spectrum of
log Z+ - log X+ from the proof of Lemma 2 and the Lemma 2 bound;
certificate monotonicity b_{r+1} <= b_n; Lemma 1 optimality of the
quadratic and linear optima; agreement of the exact and subspace
eigensolvers; brute force (Jacobi, sphere sampling) at n <= 16.
Parity unpinned: the paper's Tables 1-4 are averages over unpublished
random seeds and are used as context only.
"""
from . import linalg, meg  # noqa: F401
