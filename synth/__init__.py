"""Seeded synthetic inputs for the low-rank MEG workloads.

This module only draws data: planted matrices, noise, sampling masks,
measurement vectors, arrival traces.  It holds none of the method's
arithmetic (no gradient, no eigensolver, no mirror step), so both the
CPU oracle and the CUDA path may take their inputs from here.

Every array that the GPU stores in reduced precision is rounded here, at
generation time, so that both sides see bit-identical data:

* dense data for the mixed-precision path is rounded to bfloat16
  (round-to-nearest-even) and returned as float64 values together with
  the raw uint16 bit patterns;
* CSR values are rounded to float32;
* measurement vectors are rounded to bfloat16.

Workload recipes (the paper's experiments, Section 7, are synthetic):

* ``dense_quadratic``: M = U diag(w) U^T + E, U orthonormal (QR of a
  Gaussian matrix), E symmetric with i.i.d. N(0, sigma^2) entries on and
  above the diagonal, mirrored below.
* ``completion``: planted trace-1 rank-r PSD M, Omega a uniform sample of
  upper-triangle positions (diagonal included), mirrored.
* ``measurements``: a_i ~ N(0, I_n), X* trace-1 rank-r PSD,
  y_i = a_i^T X* a_i (noiseless).
* ``linear``: C symmetric with i.i.d. N(0,1) upper triangle.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

__all__ = [
    "bf16_round", "bf16_bits", "sym_noise", "orthonormal", "dense_quadratic",
    "completion", "measurements", "linear", "arrival_trace", "serving_trace", "ServingRequest",
    "DenseQuadratic",
    "Completion", "Measurements", "Linear", "config",
]


# ---------------------------------------------------------------- rounding
def bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (nearest, ties to even); uint16 bits."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    bias = ((u >> np.uint64(16)) & np.uint64(1)) + np.uint64(0x7FFF)
    u = ((u + bias) >> np.uint64(16)) & np.uint64(0xFFFF)
    return u.astype(np.uint16)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Values of ``bf16_bits(x)`` as float64."""
    b = bf16_bits(x).astype(np.uint32) << np.uint32(16)
    return b.view(np.float32).astype(np.float64)


def _round(x: np.ndarray, storage: str) -> np.ndarray:
    if storage == "f64":
        return np.asarray(x, dtype=np.float64)
    if storage == "f32":
        return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)
    if storage == "bf16":
        return bf16_round(x)
    raise ValueError(f"unknown storage {storage!r}")


# ---------------------------------------------------------------- pieces
def orthonormal(rng: np.random.Generator, n: int, r: int) -> np.ndarray:
    """Orthonormal n x r matrix: the Q factor of a Gaussian n x r matrix."""
    q, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return q


def sym_noise(rng: np.random.Generator, n: int, sigma: float) -> np.ndarray:
    """Symmetric noise: i.i.d. N(0, sigma^2) on and above the diagonal."""
    e = np.triu(rng.standard_normal((n, n)) * sigma)
    return e + np.triu(e, 1).T


@dataclasses.dataclass
class DenseQuadratic:
    """f(X) = 1/2 ||X - M||_F^2 over the spectrahedron."""
    n: int
    M: np.ndarray            # float64 values (already rounded to `storage`)
    storage: str             # "f64" | "f32" | "bf16"
    U: np.ndarray            # planted factor (for diagnostics only)
    w: np.ndarray            # planted weights

    def bits(self) -> np.ndarray:
        """Row-major data in the storage format (bf16 -> uint16 bits)."""
        if self.storage == "bf16":
            return bf16_bits(self.M)
        if self.storage == "f32":
            return self.M.astype(np.float32)
        return self.M


def dense_quadratic(n: int, r: int, seed: int, weights=None, sigma: float = 1e-5,
                    storage: str = "f64") -> DenseQuadratic:
    """Planted rank-r trace-1 PSD matrix plus symmetric Gaussian noise.

    ``weights`` None draws w ~ Dirichlet(1_r); otherwise the given weights.
    """
    rng = np.random.default_rng(seed)
    U = orthonormal(rng, n, r)
    if weights is None:
        w = rng.dirichlet(np.ones(r))
    else:
        w = np.asarray(weights, dtype=np.float64)
    M = (U * w) @ U.T + sym_noise(rng, n, sigma)
    M = 0.5 * (M + M.T)
    return DenseQuadratic(n=n, M=_round(M, storage), storage=storage, U=U, w=w)


@dataclasses.dataclass
class Linear:
    """f(X) = <C, X>."""
    n: int
    C: np.ndarray
    storage: str

    def bits(self) -> np.ndarray:
        if self.storage == "bf16":
            return bf16_bits(self.C)
        if self.storage == "f32":
            return self.C.astype(np.float32)
        return self.C


def linear(n: int, seed: int, scale: float = 1.0, storage: str = "f64") -> Linear:
    rng = np.random.default_rng(seed)
    C = sym_noise(rng, n, scale)
    return Linear(n=n, C=_round(C, storage), storage=storage)


@dataclasses.dataclass
class Completion:
    """f(X) = 1/2 sum_{(i,j) in Omega} (X_ij - M_ij)^2, Omega mirrored.

    CSR arrays hold every stored (i, j) once per direction: an off-diagonal
    sample appears as (i, j) and (j, i); a diagonal sample once.
    """
    n: int
    rowptr: np.ndarray       # int32 [n+1]
    col: np.ndarray          # int32 [nnz], sorted within each row
    val: np.ndarray          # float64 values of M_ij rounded to float32
    U: np.ndarray
    w: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])


def completion(n: int, r: int, frac: float, seed: int) -> Completion:
    """Planted trace-1 rank-r PSD M, a uniform fraction of the upper triangle."""
    rng = np.random.default_rng(seed)
    U = orthonormal(rng, n, r)
    w = rng.dirichlet(np.ones(r))
    n_up = n * (n + 1) // 2
    cnt = int(round(frac * n_up))
    # sample distinct linear indices of the upper triangle (incl. diagonal)
    lin = np.unique(rng.integers(0, n_up, size=int(cnt * 1.02) + 16, dtype=np.int64))
    lin = rng.permutation(lin)[:cnt]
    lin.sort()
    # row i of the upper triangle starts at i*n - i*(i-1)/2
    starts = np.arange(n, dtype=np.int64) * n - (np.arange(n, dtype=np.int64) * (np.arange(n, dtype=np.int64) - 1)) // 2
    i = np.searchsorted(starts, lin, side="right") - 1
    j = i + (lin - starts[i])
    off = i != j
    rows = np.concatenate([i, j[off]])
    cols = np.concatenate([j, i[off]])
    order = np.lexsort((cols, rows))
    rows, cols = rows[order], cols[order]
    vals = np.einsum("kr,kr->k", U[rows] * w, U[cols])
    vals = vals.astype(np.float32).astype(np.float64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return Completion(n=n, rowptr=rowptr.astype(np.int32), col=cols.astype(np.int32),
                      val=vals, U=U, w=w)


@dataclasses.dataclass
class Measurements:
    """f(X) = (1/m) sum_i (a_i^T X a_i - y_i)^2, sampled L at a time."""
    n: int
    A: np.ndarray            # m x n, float64 values rounded to bf16
    y: np.ndarray            # m, float64
    L: int                   # minibatch size
    U: np.ndarray
    w: np.ndarray

    @property
    def m(self) -> int:
        return int(self.A.shape[0])

    def bits(self) -> np.ndarray:
        return bf16_bits(self.A)


def measurements(n: int, r: int, m: int, L: int, seed: int,
                 chunk: int = 4096) -> Measurements:
    """a_i ~ N(0, I_n) rounded to bf16, y_i = a_i^T X* a_i in float64."""
    rng = np.random.default_rng(seed)
    U = orthonormal(rng, n, r)
    w = rng.dirichlet(np.ones(r))
    A = np.empty((m, n), dtype=np.float64)
    y = np.empty(m, dtype=np.float64)
    for s in range(0, m, chunk):
        e = min(m, s + chunk)
        a = bf16_round(rng.standard_normal((e - s, n)))
        A[s:e] = a
        p = a @ U
        y[s:e] = (p * p) @ w
    return Measurements(n=n, A=A, y=y, L=L, U=U, w=w)


@dataclasses.dataclass
class BilinearRecovery:
    """Recovery from bilinear measurements (the paper's experiment, Section 7):
    ground truth M = (sqrt(n) G)(sqrt(n) G)^T with G Gaussian, ||G||_F = 1;
    m pairs of uniform unit vectors (a_i, b_i); y = y0 + kappa ||y0|| v with
    y0_i = a_i^T M b_i and v a uniform unit vector; trace bound tau; U the
    Gaussian, ||U||_F = 1, matrix of the initialization."""
    n: int
    r: int
    A: np.ndarray        # m x n
    B: np.ndarray        # m x n
    y: np.ndarray        # m
    G: np.ndarray        # n x r, M = n G G^T
    tau: float
    U: np.ndarray        # n x r

    @property
    def M(self) -> np.ndarray:
        return self.n * (self.G @ self.G.T)


def _unit_rows(rng: np.random.Generator, m: int, n: int) -> np.ndarray:
    x = rng.standard_normal((m, n))
    return x / np.linalg.norm(x, axis=1, keepdims=True)


def bilinear_recovery(n: int, r: int, seed: int, kappa: float = 0.5, m: Optional[int] = None,
                      tau_frac: Optional[float] = None, r_svd: Optional[int] = None) -> BilinearRecovery:
    """The instance of Section 7: ground truth of rank r, noise level kappa,
    tau = 0.5 tr(M) for rank 1 and 5 and 0.65 tr(M) for rank 20 (unless
    given), m = 20 n r_svd measurements and U with r_svd columns, r_svd the
    algorithm's rank parameter (r unless the rank is overestimated)."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, r))
    G /= np.linalg.norm(G)
    r_svd = r if r_svd is None else int(r_svd)
    m = 20 * n * r_svd if m is None else int(m)
    A = _unit_rows(rng, m, n)
    B = _unit_rows(rng, m, n)
    y0 = n * np.einsum("ij,ij->i", A @ G, B @ G)
    v = rng.standard_normal(m)
    v /= np.linalg.norm(v)
    y = y0 + kappa * np.linalg.norm(y0) * v
    if tau_frac is None:
        tau_frac = 0.65 if r >= 20 else 0.5
    tau = tau_frac * float(n)          # tr(M) = n ||G||_F^2 = n
    U = rng.standard_normal((n, r_svd))
    U /= np.linalg.norm(U)
    return BilinearRecovery(n=n, r=r, A=A, B=B, y=y, G=G, tau=tau, U=U)


@dataclasses.dataclass
class RankPRecovery:
    """The higher-rank-measurement instance of Section 7: as
    ``BilinearRecovery`` with A_i, B_i in R^{n x p} with orthonormal columns
    and y0_i = Tr(A_i^T M B_i)."""
    n: int
    r: int
    p: int
    As: np.ndarray       # m x n x p
    Bs: np.ndarray       # m x n x p
    y: np.ndarray
    G: np.ndarray
    tau: float
    U: np.ndarray

    @property
    def M(self) -> np.ndarray:
        return self.n * (self.G @ self.G.T)


def _orthonormal_blocks(rng: np.random.Generator, m: int, n: int, p: int) -> np.ndarray:
    return np.linalg.qr(rng.standard_normal((m, n, p)))[0]


def rank_p_recovery(n: int, r: int, p: int, m: int, seed: int, kappa: float = 0.5,
                    tau_frac: float = 0.5) -> RankPRecovery:
    """Section 7 with measurement matrices of rank p (orthonormal columns);
    ground truth and noise as in ``bilinear_recovery``; m given (the paper's
    runs take m = 20 n r)."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, r))
    G /= np.linalg.norm(G)
    As = _orthonormal_blocks(rng, m, n, p)
    Bs = _orthonormal_blocks(rng, m, n, p)
    y0 = n * np.einsum("ipl,ipl->i", np.einsum("inp,nl->ipl", As, G), np.einsum("inp,nl->ipl", Bs, G))
    v = rng.standard_normal(m)
    v /= np.linalg.norm(v)
    y = y0 + kappa * np.linalg.norm(y0) * v
    U = rng.standard_normal((n, r))
    U /= np.linalg.norm(U)
    return RankPRecovery(n=n, r=r, p=p, As=As, Bs=Bs, y=y, G=G, tau=tau_frac * float(n), U=U)


def arrival_trace(count: int, rate: float, seed: int, n_lo: int = 64, n_hi: int = 1024,
                  r_max: int = 8):
    """Poisson arrivals: (time_s, n, r, kind) with n log-uniform, r uniform."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    times = np.cumsum(gaps)
    n = np.floor(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))).astype(int)
    r = rng.integers(1, r_max + 1, size=count)
    kind = rng.integers(0, 2, size=count)   # 0: dense quadratic, 1: measurements
    return [(float(times[i]), int(n[i]), int(r[i]), int(kind[i])) for i in range(count)]


@dataclasses.dataclass
class ServingRequest:
    """One request of the serving trace (host data)."""
    t: float                 # arrival time, seconds from the start of the trace
    n: int
    r: int
    kind: int                # 0: dense quadratic (float64), 1: measurements (bf16)
    M: Optional[np.ndarray] = None       # dense: n x n float64
    M32: Optional[np.ndarray] = None     # dense: the same matrix rounded to float32
    A_bits: Optional[np.ndarray] = None  # measurements: m x n bf16 bits (a view of the pool)
    A: Optional[np.ndarray] = None       # the same values as float64 (a view of the pool)
    y: Optional[np.ndarray] = None       # m float64
    L: int = 256


def serving_trace(count: int, rate: float, seed: int, m: int = 50000, L: int = 256,
                  sigma: float = 1e-4, n_lo: int = 64, n_hi: int = 1024, r_max: int = 8):
    """Poisson trace of config-0-type and config-3-type requests.

    Dense requests: M = U diag(w) U^T + E, w ~ Dirichlet(1_r), U orthonormal
    of the request's own seed, E the leading n x n block of one seeded
    symmetric N(0, sigma^2) matrix (a block of a symmetric matrix with i.i.d.
    upper triangle has the same distribution).  Measurement requests: m
    vectors a_i ~ N(0, I_n) rounded to bf16, taken as a contiguous window of
    one seeded pool of i.i.d. values at a request-specific offset, and
    y_i = a_i^T X* a_i (float64) for the request's own trace-1 rank-r X*.
    Sharing the pools keeps the trace's host memory and generation time
    bounded; every request still has its own planted solution.
    """
    arr = arrival_trace(count, rate, seed, n_lo, n_hi, r_max)
    rng = np.random.default_rng(seed + 1)
    E = sym_noise(rng, n_hi, sigma)
    need_meas = any(k == 1 for _, _, _, k in arr)
    pool_len = m * n_hi + 64 * 1024
    if need_meas:
        pool_bits = bf16_bits(rng.standard_normal(pool_len))
        pool = (pool_bits.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)
    out = []
    for j, (t, n, r, kind) in enumerate(arr):
        rj = np.random.default_rng([seed, j])
        U = orthonormal(rj, n, r)
        w = rj.dirichlet(np.ones(r))
        if kind == 0:
            M = (U * w) @ U.T + E[:n, :n]
            M = 0.5 * (M + M.T)
            out.append(ServingRequest(t=t, n=n, r=r, kind=0, M=M, M32=M.astype(np.float32)))
        else:
            off = int(rj.integers(0, (pool_len - m * n) // 8 + 1)) * 8
            A = pool[off:off + m * n].reshape(m, n)
            p = A @ U
            y = (p * p) @ w
            out.append(ServingRequest(t=t, n=n, r=r, kind=1, A_bits=pool_bits[off:off + m * n].reshape(m, n),
                                      A=A, y=y, L=L))
    return out


# ---------------------------------------------------------------- named workloads
CONFIG0_WEIGHTS = (0.4, 0.25, 0.15, 0.12, 0.08)


def config(i: int, scale: Optional[int] = None, storage: Optional[str] = None):
    """The named workloads, seeds 1000 + i.

    ``scale`` replaces n by a smaller value with the same recipe (test sizes).
    0: dense quadratic n=200 r=5, fixed weights, sigma=1e-4, float64.
    1: dense quadratic n=4096 r=10, Dirichlet weights, sigma=1e-5, bf16.
    2: completion n=20000 r=8, 1% of the upper triangle.
    3: measurements n=2048 r=4, m=50000, L=256.
    """
    seed = 1000 + i
    if i == 0:
        n = scale or 200
        return dense_quadratic(n, 5, seed, weights=CONFIG0_WEIGHTS, sigma=1e-4,
                               storage=storage or "f64")
    if i == 1:
        n = scale or 4096
        return dense_quadratic(n, 10, seed, sigma=1e-5, storage=storage or "bf16")
    if i == 2:
        n = scale or 20000
        return completion(n, 8, 0.01 if scale is None else max(0.01, 200.0 / n), seed)
    if i == 3:
        n = scale or 2048
        m = 50000 if scale is None else 20 * n
        return measurements(n, 4, m, 256 if scale is None else 64, seed)
    raise ValueError(i)
