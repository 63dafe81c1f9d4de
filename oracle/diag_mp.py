"""Low-rank MEG on diagonal data, in 50-digit arithmetic (mpmath).

TEST INFRASTRUCTURE ONLY (see ``oracle/meg.py``).

When the gradient is diagonal whenever X is (linear f with diagonal C,
or 1/2||X - M||^2 with diagonal M) and X_0 is diagonal, every iterate of
Algorithm 2 is diagonal: log X_t - eta grad f(X_t) is the diagonal vector
m_j = log x_j - eta g_j, its top-r eigenvalues are the r largest entries,
X_{t+1} puts (1 - eps_t) exp(m_j) / sum_{top r} exp(m) on those r
coordinates and eps_t/(n - r) on the others (Definition 2).  This module
runs that scalar recursion at high precision; it is the closed form the
general oracle is pinned to.
"""
from __future__ import annotations

import mpmath as mp


def lowrank_meg_diagonal(c_or_m, kind: str, x1, r: int, T: int, eta, eps_fn, dps: int = 50):
    """Iterate the diagonal recursion T times from the diagonal of X_1.

    kind "linear": g = c.  kind "dense_quadratic": g = x - m.
    Returns a list of (x_{t+1} as mpf list, top-(r+1) m values, certificate)
    for t = 1..T, with the certificate log((n-r) e^{m_(r+1)} / (eps b_{r+1})).
    """
    mp.mp.dps = dps
    n = len(x1)
    c = [mp.mpf(v) for v in c_or_m]
    x = [mp.mpf(v) for v in x1]
    out = []
    for t in range(1, T + 1):
        e = mp.mpf(eta(t) if callable(eta) else eta)
        eps = mp.mpf(eps_fn(t))
        if kind == "linear":
            g = c
        elif kind == "dense_quadratic":
            g = [x[j] - c[j] for j in range(n)]
        else:
            raise ValueError(kind)
        m = [mp.log(x[j]) - e * g[j] for j in range(n)]
        order = sorted(range(n), key=lambda j: (-m[j], j))
        top = order[:r]
        a = mp.fsum(mp.exp(m[j]) for j in top)
        b1 = a + mp.exp(m[order[r]])
        cert = mp.log(n - r) + m[order[r]] - mp.log(eps) - mp.log(b1)
        xn = [eps / (n - r)] * n
        for j in top:
            xn[j] = (1 - eps) * mp.exp(m[j]) / a
        x = xn
        out.append((list(x), [m[j] for j in order[: r + 1]], cert))
    return out
