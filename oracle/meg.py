"""Matrix Exponentiated Gradient, exact and low-rank: the CPU float64 oracle.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with the CUDA path and is deliberately plain: dense NumPy/SciPy in
float64, no blocking, fusion or reordering beyond what the paper states.

What it computes (paper: Garber & Kaplan, "On the Efficient Implementation
of the Matrix Exponentiated Gradient Algorithm for Low-Rank Matrix
Optimization"):

* ``full_meg_step`` -- Algorithm 1 (exact MEG), eq. (MDvonNeumannUpdate):
  Z+ = exp(log Z - eta grad) / Tr(exp(...)).
* ``lowrank_step`` -- one iteration of Algorithm 2 / Definition 2
  (eq. LowRankMDvonNeumannUpdate): top-r eigen-decomposition of
  M_t = log X_t - eta_t grad f(X_t), then
  X_{t+1} = (1 - eps_t) Y^r / a_t + eps_t/(n - r) (I - V V^T), stored in the
  factored form of eq. (eigenFastUpdate).  Two eigensolvers:
  "exact" (dense eigh of M_t, any n the machine can hold) and "subspace"
  (its own orthogonal iteration + Rayleigh-Ritz, Section 3, run to a
  residual of 1e-12, for large or sparse cases).
* ``certificate`` -- the sufficient condition of Lemma 2,
  eq. (convergenceCondition), with b = b_{r+1} (eq.
  convergenceGuaranteeExperiment2) and, when every eigenvalue is known,
  with the exact b = b_n (eq. convergenceGuaranteeExperiment).
* ``init_X1`` -- Algorithm 2's initialization X_1 = (1-eps_0) X_0 + eps_0/n I.
* ``warm_start`` -- eq. (exp:init) with U = 0: the top-r eigenpairs of
  -grad f(0), eigenvalues projected onto the unit simplex.
* objectives: dense quadratic 1/2||X - M||_F^2, linear <C, X>, matrix
  completion on a mirrored sample Omega, stochastic quadratic
  measurements with minibatches drawn by SplitMix64, and the experiments'
  bilinear measurements 1/2 sum (a^T X b - y)^2 on the tau-spectrahedron
  (Section 7), with ``warm_start_at`` for their initialization.

Readings of points the paper leaves open are listed with the code that
takes them (eps schedule, shift of the subspace iteration, minibatch
sampling, sign of eq. exp:init).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .linalg import eigh_desc, logsumexp, project_simplex

MASK64 = (1 << 64) - 1
SPLITMIX_GAMMA = 0x9E3779B97F4A7C15


# ---------------------------------------------------------------- schedules
def eps_schedule(t: int, a: float = 0.8, c: float = 10.0, q: float = 2.0) -> float:
    """eps_t = a / (t + c + 1)^q; Section 7 uses a = 4/5, c = 10, q = 2.

    Reading: X_1 takes eps_0 and the step that produces X_{t+1} takes eps_t.
    """
    return a / float(t + c + 1) ** q


# ---------------------------------------------------------------- factored iterate
@dataclasses.dataclass
class Factored:
    """X = V diag(mu) V^T + s (I - V V^T), eq. (eigenFastUpdate).

    V is n x r with orthonormal columns; the spectrum of X is mu (on V)
    and s (with multiplicity n - r).
    """
    V: np.ndarray
    mu: np.ndarray
    s: float

    @property
    def n(self) -> int:
        return int(self.V.shape[0])

    @property
    def r(self) -> int:
        return int(self.V.shape[1])

    def trace(self) -> float:
        return float(np.sum(self.mu) + (self.n - self.r) * self.s)

    def dense(self) -> np.ndarray:
        X = (self.V * (self.mu - self.s)) @ self.V.T
        X[np.diag_indices(self.n)] += self.s
        return X

    def apply(self, W: np.ndarray) -> np.ndarray:
        """X W without forming X."""
        return self.V @ ((self.mu - self.s)[:, None] * (self.V.T @ W)) + self.s * W

    def log_coeffs(self):
        """log X = V diag(log mu - log s) V^T + log s I  (Section 3)."""
        ls = math.log(self.s)
        return np.log(self.mu) - ls, ls

    def log_apply(self, W: np.ndarray) -> np.ndarray:
        d, ls = self.log_coeffs()
        return self.V @ (d[:, None] * (self.V.T @ W)) + ls * W

    def log_dense(self) -> np.ndarray:
        d, ls = self.log_coeffs()
        L = (self.V * d) @ self.V.T
        L[np.diag_indices(self.n)] += ls
        return L

    def entries(self, rows: np.ndarray, cols: np.ndarray) -> np.ndarray:
        """X_ij for the listed positions."""
        val = np.einsum("kr,kr->k", self.V[rows] * (self.mu - self.s), self.V[cols])
        return val + np.where(rows == cols, self.s, 0.0)


def frob_inner(a: Factored, b: Factored) -> float:
    """<X_a, X_b> from the factors.

    With D = diag(mu - s): X = V D V^T + s I, so
    <X_a, X_b> = sum_ij D_a,i D_b,j (v_a,i . v_b,j)^2 + s_b Tr D_a + s_a Tr D_b + n s_a s_b.
    """
    Da = a.mu - a.s
    Db = b.mu - b.s
    P = a.V.T @ b.V
    return float(Da @ (P * P) @ Db + b.s * Da.sum() + a.s * Db.sum() + a.n * a.s * b.s)


def frob_dist(a: Factored, b: Factored) -> float:
    """||X_a - X_b||_F without cancellation between the two iterates.

    With B = [V_a, V_b] = Q R: X_a - X_b = Q K Q^T + (s_a - s_b) I where
    K = R_a D_a R_a^T - R_b D_b R_b^T is small, hence
    ||X_a - X_b||^2 = ||K||^2 + 2 (s_a - s_b) Tr K + n (s_a - s_b)^2.
    """
    Q, R = np.linalg.qr(np.concatenate([a.V, b.V], axis=1))
    Ra, Rb = R[:, : a.r], R[:, a.r:]
    K = (Ra * (a.mu - a.s)) @ Ra.T - (Rb * (b.mu - b.s)) @ Rb.T
    ds = a.s - b.s
    d2 = float(np.sum(K * K)) + 2.0 * ds * float(np.trace(K)) + a.n * ds * ds
    return math.sqrt(max(d2, 0.0))


def init_X1(V0: np.ndarray, lam0: np.ndarray, eps0: float) -> Factored:
    """Algorithm 2, Initialization: X_1 = (1 - eps_0) X_0 + (eps_0/n) I.

    X_0 = V0 diag(lam0) V0^T with lam0 on the unit simplex, so X_1 has
    mu = (1 - eps_0) lam0 + eps_0/n on V0 and s = eps_0/n elsewhere.
    """
    n = V0.shape[0]
    lam0 = np.asarray(lam0, dtype=np.float64)
    return Factored(V=np.array(V0, dtype=np.float64), mu=(1.0 - eps0) * lam0 + eps0 / n,
                    s=eps0 / n)


# ---------------------------------------------------------------- SplitMix64
def splitmix64(x: int) -> int:
    """SplitMix64 output function (Steele, Lea & Flood, OOPSLA 2014)."""
    z = x & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def minibatch_indices(seed: int, t: int, L: int, m: int) -> np.ndarray:
    """L i.i.d. uniform indices in [0, m), with replacement (Section 6).

    Reading: draw j of step t is splitmix64(seed + (t*L + j + 1) * gamma) mod m,
    i.e. the (t*L + j + 1)-th output of a SplitMix64 stream started at seed.
    """
    out = np.empty(L, dtype=np.int64)
    for j in range(L):
        ctr = (t * L + j + 1) & MASK64
        out[j] = splitmix64((seed + ctr * SPLITMIX_GAMMA) & MASK64) % m
    return out


# ---------------------------------------------------------------- objectives
class DenseQuadratic:
    """f(X) = 1/2 ||X - M||_F^2, grad f(X) = X - M."""
    kind = "dense_quadratic"

    def __init__(self, M: np.ndarray):
        self.M = np.asarray(M, dtype=np.float64)
        self.n = self.M.shape[0]

    def value(self, X: Factored) -> float:
        R = X.dense() - self.M
        return 0.5 * float(np.sum(R * R))

    def value_dense(self, X: np.ndarray) -> float:
        R = X - self.M
        return 0.5 * float(np.sum(R * R))

    def grad_dense(self, X, t: int = 0) -> np.ndarray:
        Xd = X.dense() if isinstance(X, Factored) else X
        return Xd - self.M

    def grad_apply(self, X: Factored, W: np.ndarray, t: int = 0) -> np.ndarray:
        return X.apply(W) - self.M @ W

    def grad_norm_bound(self, X: Factored, t: int = 0) -> float:
        return math.sqrt(2.0 * self.value(X))

    def neg_grad0_apply(self, W):
        return self.M @ W


class Linear:
    """f(X) = <C, X>, grad f = C."""
    kind = "linear"

    def __init__(self, C: np.ndarray):
        self.C = np.asarray(C, dtype=np.float64)
        self.n = self.C.shape[0]

    def value(self, X: Factored) -> float:
        return float(np.sum(X.dense() * self.C))

    def value_dense(self, X: np.ndarray) -> float:
        return float(np.sum(X * self.C))

    def grad_dense(self, X, t: int = 0) -> np.ndarray:
        return self.C.copy()

    def grad_apply(self, X: Factored, W: np.ndarray, t: int = 0) -> np.ndarray:
        return self.C @ W

    def grad_norm_bound(self, X: Factored, t: int = 0) -> float:
        return float(np.linalg.norm(self.C))

    def neg_grad0_apply(self, W):
        return -(self.C @ W)


class Completion:
    """f(X) = 1/2 sum_{(i,j) in Omega} (X_ij - M_ij)^2 with Omega mirrored.

    Reading: the sample is stored for both (i, j) and (j, i), so the sum
    counts an off-diagonal pair twice and grad f = P_Omega(X - M) is
    symmetric (footnote to eq. Model).
    """
    kind = "completion"

    def __init__(self, n: int, rowptr, col, val):
        self.n = n
        self.rowptr = np.asarray(rowptr, dtype=np.int64)
        self.col = np.asarray(col, dtype=np.int64)
        self.val = np.asarray(val, dtype=np.float64)
        self.row = np.repeat(np.arange(n), np.diff(self.rowptr))

    def residual(self, X: Factored) -> np.ndarray:
        return X.entries(self.row, self.col) - self.val

    def value(self, X: Factored) -> float:
        R = self.residual(X)
        return 0.5 * float(R @ R)

    def value_dense(self, X: np.ndarray) -> float:
        R = X[self.row, self.col] - self.val
        return 0.5 * float(R @ R)

    def grad_sparse(self, X: Factored) -> sp.csr_matrix:
        return sp.csr_matrix((self.residual(X), self.col, self.rowptr), shape=(self.n, self.n))

    def grad_dense(self, X, t: int = 0) -> np.ndarray:
        if isinstance(X, Factored):
            return self.grad_sparse(X).toarray()
        R = X[self.row, self.col] - self.val
        return sp.csr_matrix((R, self.col, self.rowptr), shape=(self.n, self.n)).toarray()

    def grad_apply(self, X: Factored, W: np.ndarray, t: int = 0) -> np.ndarray:
        return self.grad_sparse(X) @ W

    def grad_norm_bound(self, X: Factored, t: int = 0) -> float:
        return float(np.linalg.norm(self.residual(X)))

    def neg_grad0_apply(self, W):
        return sp.csr_matrix((self.val, self.col, self.rowptr), shape=(self.n, self.n)) @ W


class Measurements:
    """f(X) = (1/m) sum_i (a_i^T X a_i - y_i)^2 with a minibatch oracle.

    Full gradient (2/m) sum_i r_i a_i a_i^T; the stochastic gradient of
    step t is (2/L) sum over L indices drawn i.i.d. with replacement
    (Section 6: L i.i.d. queries), r_i = a_i^T X a_i - y_i.
    """
    kind = "measurements"

    def __init__(self, A: np.ndarray, y: np.ndarray, L: int, seed: int):
        self.A = np.asarray(A, dtype=np.float64)
        self.y = np.asarray(y, dtype=np.float64)
        self.m, self.n = self.A.shape
        self.L = int(L)
        self.seed = int(seed)

    def batch(self, t: int) -> np.ndarray:
        return minibatch_indices(self.seed, t, self.L, self.m)

    def quad(self, X: Factored, idx) -> np.ndarray:
        """a_i^T X a_i = sum_l (mu_l - s) (v_l . a_i)^2 + s ||a_i||^2."""
        a = self.A[idx]
        p = a @ X.V
        return (p * p) @ (X.mu - X.s) + X.s * np.einsum("ij,ij->i", a, a)

    def value(self, X: Factored) -> float:
        total = 0.0
        for s in range(0, self.m, 8192):
            idx = np.arange(s, min(self.m, s + 8192))
            r = self.quad(X, idx) - self.y[idx]
            total += float(r @ r)
        return total / self.m

    def value_dense(self, X: np.ndarray) -> float:
        r = np.einsum("ij,jk,ik->i", self.A, X, self.A) - self.y
        return float(r @ r) / self.m

    def _batch_resid(self, X, t):
        idx = self.batch(t)
        a = self.A[idx]
        if isinstance(X, Factored):
            r = self.quad(X, idx) - self.y[idx]
        else:
            r = np.einsum("ij,jk,ik->i", a, X, a) - self.y[idx]
        return a, r

    def grad_dense(self, X, t: int = 0) -> np.ndarray:
        a, r = self._batch_resid(X, t)
        return (2.0 / self.L) * (a.T * r) @ a

    def grad_apply(self, X: Factored, W: np.ndarray, t: int = 0) -> np.ndarray:
        a, r = self._batch_resid(X, t)
        return (2.0 / self.L) * (a.T @ (r[:, None] * (a @ W)))

    def grad_norm_bound(self, X: Factored, t: int = 0) -> float:
        a, r = self._batch_resid(X, t)
        return (2.0 / self.L) * float(np.sum(np.abs(r) * np.einsum("ij,ij->i", a, a)))

    def neg_grad0_apply(self, W):
        # -grad f(0) = (2/m) sum_i y_i a_i a_i^T  (full data)
        return (2.0 / self.m) * (self.A.T @ (self.y[:, None] * (self.A @ W)))


class BilinearMeasurements:
    """The paper's experiment objective (Section 7, eq. recoveryProb) in
    trace-1 variables: f(X) = 1/2 sum_i (a_i^T X b_i - y_i)^2 over the
    tau-spectrahedron, written for X' = X / tau on the unit spectrahedron,
    f'(X') = f(tau X') = 1/2 sum_i (tau a_i^T X' b_i - y_i)^2 (the library is
    trace-1 only).  For symmetric X, a^T X b = <X, (a b^T + b a^T)/2>, so
    grad f'(X') = tau sum_i r_i (a_i b_i^T + b_i a_i^T)/2 with
    r_i = tau a_i^T X' b_i - y_i (full gradients: the experiments' setting).
    """
    kind = "bilinear"

    def __init__(self, A: np.ndarray, B: np.ndarray, y: np.ndarray, tau: float = 1.0):
        self.A = np.asarray(A, dtype=np.float64)
        self.B = np.asarray(B, dtype=np.float64)
        self.y = np.asarray(y, dtype=np.float64)
        self.m, self.n = self.A.shape
        self.tau = float(tau)

    def bil(self, X) -> np.ndarray:
        """tau a_i^T X b_i for every i; Factored X: sum_l (mu_l - s)(a_i.v_l)(b_i.v_l) + s a_i.b_i."""
        if isinstance(X, Factored):
            pa, pb = self.A @ X.V, self.B @ X.V
            q = (pa * pb) @ (X.mu - X.s) + X.s * np.einsum("ij,ij->i", self.A, self.B)
        else:
            q = np.einsum("ij,ij->i", self.A @ np.asarray(X), self.B)      # (a_i^T X) . b_i
        return self.tau * q

    def residual(self, X) -> np.ndarray:
        return self.bil(X) - self.y

    def value(self, X: Factored) -> float:
        r = self.residual(X)
        return 0.5 * float(r @ r)

    def value_dense(self, X: np.ndarray) -> float:
        r = self.residual(X)
        return 0.5 * float(r @ r)

    def grad_dense(self, X, t: int = 0) -> np.ndarray:
        r = self.residual(X)
        G = (self.A.T * r) @ self.B
        return 0.5 * self.tau * (G + G.T)

    def grad_apply(self, X: Factored, W: np.ndarray, t: int = 0) -> np.ndarray:
        r = self.residual(X)[:, None]
        return 0.5 * self.tau * (self.A.T @ (r * (self.B @ W)) + self.B.T @ (r * (self.A @ W)))

    def grad_norm_bound(self, X: Factored, t: int = 0) -> float:
        # ||(a b^T + b a^T)/2||_2 <= ||a|| ||b||
        r = self.residual(X)
        na, nb = np.linalg.norm(self.A, axis=1), np.linalg.norm(self.B, axis=1)
        return self.tau * float(np.sum(np.abs(r) * na * nb))

    def neg_grad0_apply(self, W):
        # -grad f'(0) = tau sum_i y_i (a_i b_i^T + b_i a_i^T)/2
        y = self.y[:, None]
        return 0.5 * self.tau * (self.A.T @ (y * (self.B @ W)) + self.B.T @ (y * (self.A @ W)))


class RankPMeasurements:
    """The experiments' objective with measurement matrices of rank p > 1
    (Section 7, higher-rank measurements): f(X) = 1/2 sum_i (Tr(A_i^T X B_i)
    - y_i)^2 with A_i, B_i in R^{n x p}, in trace-1 variables X' = X / tau as
    for ``BilinearMeasurements``.  For symmetric X, Tr(A^T X B) =
    <X, (A B^T + B A^T)/2>, so grad f'(X') = tau sum_i r_i (A_i B_i^T +
    B_i A_i^T)/2 with r_i = tau Tr(A_i^T X' B_i) - y_i.  As, Bs: m x n x p.
    """
    kind = "rank_p"

    def __init__(self, As: np.ndarray, Bs: np.ndarray, y: np.ndarray, tau: float = 1.0):
        self.As = np.asarray(As, dtype=np.float64)
        self.Bs = np.asarray(Bs, dtype=np.float64)
        self.y = np.asarray(y, dtype=np.float64)
        self.m, self.n, self.p = self.As.shape
        self.tau = float(tau)

    def trace_form(self, X) -> np.ndarray:
        """tau Tr(A_i^T X B_i) for every i; Factored X: sum_l (mu_l - s) <A_i^T v_l, B_i^T v_l>
        + s <A_i, B_i>."""
        if isinstance(X, Factored):
            pa = np.einsum("inp,nl->ipl", self.As, X.V)
            pb = np.einsum("inp,nl->ipl", self.Bs, X.V)
            q = np.einsum("ipl,ipl->il", pa, pb) @ (X.mu - X.s) + X.s * np.einsum("inp,inp->i", self.As, self.Bs)
        else:
            q = np.einsum("inp,nk,ikp->i", self.As, np.asarray(X), self.Bs, optimize=True)
        return self.tau * q

    def residual(self, X) -> np.ndarray:
        return self.trace_form(X) - self.y

    def value(self, X: Factored) -> float:
        r = self.residual(X)
        return 0.5 * float(r @ r)

    def value_dense(self, X: np.ndarray) -> float:
        r = self.residual(X)
        return 0.5 * float(r @ r)

    def grad_dense(self, X, t: int = 0) -> np.ndarray:
        r = self.residual(X)
        G = np.einsum("i,inp,ikp->nk", r, self.As, self.Bs, optimize=True)
        return 0.5 * self.tau * (G + G.T)

    def grad_apply(self, X: Factored, W: np.ndarray, t: int = 0) -> np.ndarray:
        r = self.residual(X)
        bw = np.einsum("ikp,kj->ipj", self.Bs, W)
        aw = np.einsum("ikp,kj->ipj", self.As, W)
        return 0.5 * self.tau * (np.einsum("i,inp,ipj->nj", r, self.As, bw) + np.einsum("i,inp,ipj->nj", r, self.Bs, aw))

    def grad_norm_bound(self, X: Factored, t: int = 0) -> float:
        # ||(A B^T + B A^T)/2||_2 <= ||A||_2 ||B||_2
        r = self.residual(X)
        na = np.array([np.linalg.norm(a, 2) for a in self.As])
        nb = np.array([np.linalg.norm(b, 2) for b in self.Bs])
        return self.tau * float(np.sum(np.abs(r) * na * nb))

    def neg_grad0_apply(self, W):
        y = self.y
        bw = np.einsum("ikp,kj->ipj", self.Bs, W)
        aw = np.einsum("ikp,kj->ipj", self.As, W)
        return 0.5 * self.tau * (np.einsum("i,inp,ipj->nj", y, self.As, bw) + np.einsum("i,inp,ipj->nj", y, self.Bs, aw))


def warm_start_at(obj, r: int, U: np.ndarray, printed_sign: bool = False):
    """eq. (exp:init) at a given U (||U||_F = 1), in trace-1 variables:
    X_0 = V_r diag(Pi_{Delta_tau}(w)) V_r^T with (V_r, Lambda_r) the top-r
    eigenpairs of -grad f(tau U U^T), and X'_0 = X_0 / tau =
    V_r diag(Pi_Delta(w / tau)) V_r^T.  With grad f(tau U U^T) =
    grad f'(U U^T) / tau, Lambda_r / tau are the top eigenvalues of
    -grad f'(U U^T) / tau^2.  w = Lambda_r is the reading of ``warm_start``;
    printed_sign=True takes the equation as printed, w = -Lambda_r, which is
    what reproduces the initialization errors of the paper's Table 1 (rank 5
    and 20, where the projection of -Lambda_r weights the r-th eigenvector
    most).  Returns (V0 n x r, lam0 on the unit simplex).
    """
    tau = getattr(obj, "tau", 1.0)
    G = obj.grad_dense(U @ U.T)
    lam, V = eigh_desc(-0.5 * (G + G.T) / (tau * tau))
    w = -lam[:r] if printed_sign else lam[:r]
    return V[:, :r], project_simplex(w)


# ---------------------------------------------------------------- trace of exp(M) by sampling
def lanczos_quadrature(apply_M: Callable, u: np.ndarray, steps: int, fn: Callable = np.exp) -> float:
    """u^T fn(M) u by `steps` Lanczos steps on the symmetric operator M from u
    (Gauss quadrature): with the tridiagonal T_k of the Lanczos basis Q_k,
    u^T fn(M) u ~ ||u||^2 e_1^T fn(T_k) e_1, exact for polynomials of degree
    < 2k and for any fn once k reaches the dimension of the Krylov space.
    Full re-orthogonalization keeps the basis orthonormal in floating point."""
    nrm = float(np.linalg.norm(u))
    Q = [u / nrm]
    alpha, beta = [], []
    for j in range(steps):
        w = apply_M(Q[j])
        a = float(Q[j] @ w)
        alpha.append(a)
        w = w - a * Q[j] - (beta[-1] * Q[j - 1] if j > 0 else 0.0)
        Qm = np.array(Q)
        w = w - Qm.T @ (Qm @ w)                         # re-orthogonalize against the basis
        b = float(np.linalg.norm(w))
        if j == steps - 1 or b <= 1e-14 * max(1.0, abs(a)):
            break
        beta.append(b)
        Q.append(w / b)
    T = np.diag(alpha) + np.diag(beta[: len(alpha) - 1], 1) + np.diag(beta[: len(alpha) - 1], -1)
    th, S = np.linalg.eigh(T)
    return nrm * nrm * float(np.sum(S[0, :] ** 2 * fn(th)))


def hutchinson_trace_exp(apply_M: Callable, n: int, samples: int, steps: int, seed: int) -> float:
    """Tr(exp(M)) = E_u[u^T exp(M) u], u ~ N(0, I) (the alternative for the
    scalar b of the certificate that Section 4 notes after Lemma 2), as the
    mean over `samples` Gaussian vectors of Lanczos quadratures."""
    rng = np.random.default_rng(seed)
    total = 0.0
    for _ in range(samples):
        total += lanczos_quadrature(apply_M, rng.standard_normal(n), steps)
    return total / samples


# ---------------------------------------------------------------- certificate
def certificate(sig: np.ndarray, n: int, r: int, eps: float) -> float:
    """log((n - r) lambda_{r+1}(Y) / (eps b)) with lambda_i(Y) = exp(sigma_i).

    ``sig`` holds the leading eigenvalues of M = log X - eta grad in
    non-increasing order: sig[:r+1] gives b_{r+1}, eq.
    (convergenceGuaranteeExperiment2); all n of them give the exact b_n,
    eq. (convergenceGuaranteeExperiment).  The certificate holds when the
    value is <= 2 eps (Lemma 2).
    """
    sig = np.asarray(sig, dtype=np.float64)
    return math.log(n - r) + float(sig[r]) - math.log(eps) - logsumexp(sig)


def lemma2_D_spectrum(sig_all: np.ndarray, r: int, eps: float) -> np.ndarray:
    """Eigenvalues of D = log Z+ - log X+ in the proof of Lemma 2.

    j <= r: log(a/b) - log(1 - eps);  j > r: log((n - r) lambda_j / (eps b)),
    with a = sum_{i<=r} lambda_i(Y), b = sum_i lambda_i(Y), lambda = exp(sig).
    """
    n = sig_all.size
    lse_a = logsumexp(sig_all[:r])
    lse_b = logsumexp(sig_all)
    top = np.full(r, lse_a - lse_b - math.log(1.0 - eps))
    low = math.log(n - r) + sig_all[r:] - math.log(eps) - lse_b
    return np.concatenate([top, low])


# ---------------------------------------------------------------- exact MEG
def full_meg_step(Z: np.ndarray, G: np.ndarray, eta: float):
    """Algorithm 1: Y = exp(log Z - eta G), b = Tr Y, Z+ = Y / b.

    Returns (Z+, sig) with sig the eigenvalues of log Z - eta G,
    non-increasing.
    """
    w, U = np.linalg.eigh(0.5 * (Z + Z.T))
    logZ = (U * np.log(w)) @ U.T
    sig, V = eigh_desc(logZ - eta * G)
    lse = logsumexp(sig)
    Zp = (V * np.exp(sig - lse)) @ V.T
    return 0.5 * (Zp + Zp.T), sig


def bregman(X: np.ndarray, Y: np.ndarray) -> float:
    """B(X, Y) = Tr(X log X - X log Y) for trace-one X, Y, eq. (bregmanInSpectrahedron)."""
    def logm(A):
        w, U = np.linalg.eigh(0.5 * (A + A.T))
        lw = np.where(w > 0, np.log(np.maximum(w, 1e-300)), 0.0)
        return (U * lw) @ U.T
    return float(np.sum(X * (logm(X) - logm(Y))))


def dual_gap(X: np.ndarray, G: np.ndarray, tau: float = 1.0) -> float:
    """Tr((X - tau v_n v_n^T) G), v_n the bottom eigenvector of G (Section 7)."""
    lam_min = float(np.linalg.eigvalsh(0.5 * (G + G.T))[0])
    return float(np.sum(X * G)) - tau * lam_min


# ---------------------------------------------------------------- low-rank step
@dataclasses.dataclass
class StepInfo:
    sig: np.ndarray          # leading eigenvalues of M_t (r+1 for subspace, all for exact)
    cert: float              # certificate value with b_{r+1}
    cert_exact: Optional[float]
    eps: float
    holds: bool
    products: int = 0        # subspace iteration products used


def _mirror_map(sig: np.ndarray, V: np.ndarray, eps: float, r: int, n: int) -> Factored:
    """X_{t+1} = (1-eps) Y^r / a + eps/(n-r) (I - V^r V^r^T)  (Def. 2 / Alg. 2).

    mu_i = (1 - eps) exp(sigma_i) / sum_{j<=r} exp(sigma_j), evaluated via
    log-sum-exp; s = eps / (n - r).
    """
    lse = logsumexp(sig[:r])
    mu = (1.0 - eps) * np.exp(sig[:r] - lse)
    return Factored(V=V[:, :r].copy(), mu=mu, s=eps / (n - r))


def orth_iteration(apply: Callable, W0: np.ndarray, need: int, shift: float,
                   tol: float = 1e-12, max_products: int = 5000):
    """Orthogonal (subspace) iteration with Rayleigh-Ritz (Section 3).

    Iterates W <- QR((A - shift I) W) and extracts Ritz pairs of A from
    W^T A W until the first ``need`` residuals ||A x - theta x|| fall below
    tol * max|theta|.  Returns (theta non-increasing, Ritz vectors, products).
    """
    W, _ = np.linalg.qr(W0)
    for it in range(1, max_products + 1):
        AW = apply(W)
        H = W.T @ AW
        th, Q = eigh_desc(0.5 * (H + H.T))
        X = W @ Q
        R = AW @ Q - X * th
        res = np.linalg.norm(R[:, :need], axis=0)
        if np.max(res) <= tol * max(1.0, float(np.max(np.abs(th[:need])))):
            return th, X, it
        W, _ = np.linalg.qr(AW @ Q - shift * X)
    return th, X, max_products


def block_krylov(apply: Callable, W0: np.ndarray, need: int, tol: float = 1e-12, max_blocks: int = 200):
    """Block Krylov (block Lanczos with full re-orthogonalization) for the
    top eigenpairs, the faster alternative to subspace iteration that
    Section 3 points to: the basis of span[W0, A W0, A^2 W0, ...] grows one
    block per product; after each block, Rayleigh-Ritz on the whole basis
    gives Ritz pairs, and the run stops when the first ``need`` residuals
    ||A x - theta x|| fall below tol * max|theta|.  Returns (theta
    non-increasing, Ritz vectors, products)."""
    n = W0.shape[0]
    Q, _ = np.linalg.qr(W0)
    basis = Q
    AB = apply(Q)
    prods = 1
    while True:
        H = basis.T @ AB
        th, S = eigh_desc(0.5 * (H + H.T))
        X = basis @ S[:, :need]
        R = AB @ S[:, :need] - X * th[:need]
        res = np.linalg.norm(R, axis=0)
        if np.max(res) <= tol * max(1.0, float(np.max(np.abs(th[:need])))) or prods >= max_blocks \
                or basis.shape[1] + Q.shape[1] > n:
            return th, basis @ S, prods
        Z = AB[:, -Q.shape[1]:]
        for _ in range(2):                              # re-orthogonalize twice
            Z = Z - basis @ (basis.T @ Z)
        Q, _ = np.linalg.qr(Z)
        basis = np.concatenate([basis, Q], axis=1)
        AB = np.concatenate([AB, apply(Q)], axis=1)
        prods += 1


def mirror_matrix(X: Factored, obj, t: int, eta: float) -> np.ndarray:
    """M_t = log X_t - eta_t grad f(X_t), dense (Algorithm 2, first line)."""
    return X.log_dense() - eta * obj.grad_dense(X, t)


def lowrank_step(X: Factored, obj, t: int, eta: float, eps: float, method: str = "exact",
                 k: Optional[int] = None, W0: Optional[np.ndarray] = None,
                 need_r1: bool = False):
    """One iteration of Algorithm 2 from X_t; returns (X_{t+1}, StepInfo, W_next).

    method "exact": dense eigh of M_t (gives every eigenvalue and the exact
    certificate).  method "subspace": orthogonal iteration on M_t - c I.
    Reading of the shift (the paper's subspace iteration finds eigenvalues
    largest in magnitude, while the wanted ones are the algebraically
    largest of an operator whose spectrum is negative): c = min(log s,
    min log mu) - eta * g with g >= ||grad f||_2, which makes M_t - c I
    positive semidefinite.
    """
    n, r = X.n, X.r
    if method == "exact":
        sig, V = eigh_desc(mirror_matrix(X, obj, t, eta))
        Xn = _mirror_map(sig, V, eps, r, n)
        c1 = certificate(sig[: r + 1], n, r, eps)
        ce = certificate(sig, n, r, eps)
        return Xn, StepInfo(sig=sig, cert=c1, cert_exact=ce, eps=eps, holds=c1 <= 2 * eps), V[:, : (k or r + 1)]
    if method == "krylov":
        k = k or (r + 1)

        def apply_k(W):
            return X.log_apply(W) - eta * obj.grad_apply(X, W, t)

        if W0 is None:
            rng = np.random.default_rng(12345 + t)
            W0 = np.concatenate([X.V, rng.standard_normal((n, k - r))], axis=1)
        th, Xr, prods = block_krylov(apply_k, W0, need=r + 1)
        Xn = _mirror_map(th, Xr, eps, r, n)
        c1 = certificate(th[: r + 1], n, r, eps)
        return Xn, StepInfo(sig=th[: r + 1].copy(), cert=c1, cert_exact=None, eps=eps,
                            holds=c1 <= 2 * eps, products=prods), Xr[:, :k]
    if method != "subspace":
        raise ValueError(method)
    k = k or (r + 1)
    d, ls = X.log_coeffs()
    g = obj.grad_norm_bound(X, t)
    shift = min(ls, float(np.min(np.log(X.mu)))) - eta * g

    def apply(W):
        return X.log_apply(W) - eta * obj.grad_apply(X, W, t)

    if W0 is None:
        rng = np.random.default_rng(12345 + t)
        W0 = np.concatenate([X.V, rng.standard_normal((n, k - r))], axis=1)
    th, Xr, prods = orth_iteration(apply, W0, need=(r + 1) if need_r1 else r, shift=shift)
    Xn = _mirror_map(th, Xr, eps, r, n)
    c1 = certificate(th[: r + 1], n, r, eps)
    return Xn, StepInfo(sig=th[: r + 1].copy(), cert=c1, cert_exact=None, eps=eps,
                        holds=c1 <= 2 * eps, products=prods), Xr


def lowrank_meg(obj, V0: np.ndarray, lam0: np.ndarray, T: int, eta,
                eps_fn: Callable[[int], float] = eps_schedule, method: str = "exact",
                k: Optional[int] = None, record: Optional[Callable] = None,
                need_r1: bool = False):
    """Algorithm 2 for T iterations; returns (X_{T+1}, [StepInfo]).

    ``eta`` is a constant or a function of t.  ``record(t, X_{t+1}, info)``
    is called after each iteration.
    """
    X = init_X1(V0, lam0, eps_fn(0))
    infos = []
    W = None
    for t in range(1, T + 1):
        e = eta(t) if callable(eta) else eta
        X, info, W = lowrank_step(X, obj, t, e, eps_fn(t), method=method, k=k, W0=W,
                                  need_r1=need_r1)
        infos.append(info)
        if record is not None:
            record(t, X, info)
    return X, infos


def full_meg(obj, Z1: np.ndarray, T: int, eta, record: Optional[Callable] = None):
    """Algorithm 1 for T iterations from Z_1 (dense)."""
    Z = np.array(Z1, dtype=np.float64)
    for t in range(1, T + 1):
        e = eta(t) if callable(eta) else eta
        Z, sig = full_meg_step(Z, obj.grad_dense(Z, t), e)
        if record is not None:
            record(t, Z, sig)
    return Z


# ---------------------------------------------------------------- warm start
def warm_start(obj, r: int, dense_limit: int = 2500):
    """eq. (exp:init) with U = 0: X_0 = V_r diag(Pi_Delta(lambda_1..r)) V_r^T.

    (V_r, lambda) are the top-r eigenpairs of -grad f(0).  Reading: the
    printed diag(-Lambda_r) would flip the sign of eigenvalues that are
    already those of -grad f, so the eigenvalues are used as they are.
    Returns (V0 n x r, lam0 on the unit simplex).
    """
    n = obj.n
    if n <= dense_limit:
        G = obj.neg_grad0_apply(np.eye(n))
        lam, V = eigh_desc(0.5 * (G + G.T))
        lam, V = lam[:r], V[:, :r]
    else:
        op = spla.LinearOperator((n, n), matvec=lambda x: obj.neg_grad0_apply(x[:, None])[:, 0],
                                 dtype=np.float64)
        lam, V = spla.eigsh(op, k=r, which="LA", tol=1e-13)
        order = np.argsort(-lam)
        lam, V = lam[order], V[:, order]
    return V, project_simplex(lam)
