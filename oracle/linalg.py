"""Small dense linear-algebra helpers for the oracle (float64, NumPy).

Test infrastructure only: nothing in the product path may import this.
"""
from __future__ import annotations

import math

import numpy as np


def eigh_desc(A: np.ndarray):
    """Eigen-decomposition of a symmetric matrix, eigenvalues non-increasing.

    The paper indexes eigenvalues so that lambda_1 is the largest
    (Section 2.1, Notation).  LAPACK returns them ascending; we flip.
    """
    A = 0.5 * (A + A.T)
    w, V = np.linalg.eigh(A)
    return w[::-1].copy(), V[:, ::-1].copy()


def logsumexp(x) -> float:
    x = np.asarray(x, dtype=np.float64)
    m = float(np.max(x))
    return m + math.log(float(np.sum(np.exp(x - m))))


def sym_fun(A: np.ndarray, fun) -> np.ndarray:
    """f(A) = V diag(f(lambda)) V^T for symmetric A (Section 2.1)."""
    w, V = np.linalg.eigh(0.5 * (A + A.T))
    return (V * fun(w)) @ V.T


def project_simplex(v, tau: float = 1.0) -> np.ndarray:
    """Euclidean projection onto {z >= 0, sum z = tau}.

    Sort-based method of Held, Wolfe and Crowder (1974): with u sorted
    non-increasingly, rho is the largest j with u_j > (sum_{i<=j} u_i - tau)/j
    and the threshold is theta = (sum_{i<=rho} u_i - tau)/rho.
    """
    v = np.asarray(v, dtype=np.float64)
    u = np.sort(v)[::-1]
    css = np.cumsum(u)
    j = np.arange(1, v.size + 1)
    cond = u - (css - tau) / j > 0
    rho = int(j[cond][-1])
    theta = (css[rho - 1] - tau) / rho
    return np.maximum(v - theta, 0.0)


def project_spectrahedron(Y: np.ndarray) -> np.ndarray:
    """Euclidean projection onto S_n = {X >= 0, Tr X = 1}, eq. (euclidProj).

    Keeps the eigenvectors of Y and replaces its eigenvalues lambda_i by
    max(0, lambda_i - theta) with theta chosen so that they sum to one,
    i.e. projects the spectrum onto the unit simplex.
    """
    w, V = np.linalg.eigh(0.5 * (Y + Y.T))
    return (V * project_simplex(w)) @ V.T


def jacobi_eigh(A: np.ndarray, tol: float = 1e-15, max_sweeps: int = 100):
    """Cyclic Jacobi eigenvalue method (Golub & Van Loan, Section 8.5).

    A textbook implementation that shares nothing with LAPACK; used to
    brute-force small cases independently of ``numpy.linalg.eigh``.
    Returns (eigenvalues non-increasing, eigenvectors).
    """
    A = np.array(0.5 * (A + A.T), dtype=np.float64)
    n = A.shape[0]
    V = np.eye(n)
    for _ in range(max_sweeps):
        off = math.sqrt(float(np.sum(np.tril(A, -1) ** 2)))
        if off <= tol * max(1.0, float(np.linalg.norm(A))):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                # symmetric Schur 2x2: choose (c, s) zeroing A[p, q]
                tau = (A[q, q] - A[p, p]) / (2.0 * apq)
                t = (1.0 if tau >= 0 else -1.0) / (abs(tau) + math.sqrt(1.0 + tau * tau))
                c = 1.0 / math.sqrt(1.0 + t * t)
                s = t * c
                # A <- J^T A J on rows/cols p, q
                ap = A[:, p].copy()
                aq = A[:, q].copy()
                A[:, p] = c * ap - s * aq
                A[:, q] = s * ap + c * aq
                ap = A[p, :].copy()
                aq = A[q, :].copy()
                A[p, :] = c * ap - s * aq
                A[q, :] = s * ap + c * aq
                vp = V[:, p].copy()
                vq = V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
    w = np.diag(A).copy()
    order = np.argsort(-w, kind="stable")
    return w[order], V[:, order]
