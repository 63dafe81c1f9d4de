"""The estimate of Tr exp(M_t) by sampling on the GPU (the note after Lemma 2:
the scalar b of the exact certificate, eq. convergenceGuaranteeExperiment,
estimated with Hutchinson's estimator and Lanczos quadrature), against the
oracle's quadrature (`oracle.meg.lanczos_quadrature`) on the same probe
vectors and the same mirror matrix M_t = log X_t - eta grad f(X_t) of the
GPU's own iterate.
"""
import numpy as np
import pytest

import synth
from oracle import meg

from meg_cases import gpu_factored, make_gpu_solve

pytestmark = pytest.mark.gpu


def _mirror(obj, X, eta):
    """M_t = log X_t - eta grad f(X_t), dense, float64."""
    w, U = np.linalg.eigh(X.dense())
    G = obj.grad_dense(X.dense())
    return (U * np.log(w)) @ U.T - eta * 0.5 * (G + G.T)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_trace_exp_matches_oracle_quadrature(prec):
    """n = 256, r = 3, k = 8 Gaussian probes, 20 Lanczos steps, after 4 MEG
    iterations (float32 data on the CUDA cores, bf16 data on the tensor
    cores): the GPU's estimate equals the oracle's mean of quadratures to
    1e-4 (the products are float32), and the iterate is left as it was: the
    next iteration is bitwise that of a solve that never ran the estimate."""
    from paper_2012_10469_gb300 import binding as B
    n, r, p = 256, 3, 5
    prob = synth.dense_quadratic(n, r, seed=77, sigma=1e-4, storage={"fp32": "f32", "bf16": "bf16"}[prec])
    obj = meg.DenseQuadratic(prob.M)
    V0, lam0 = meg.warm_start(obj, r)
    a = make_gpu_solve("dense_quadratic", prob, r, p, 2, B.PRECISION[prec], 1.0, 3, V0=V0, lam0=lam0)
    b = make_gpu_solve("dense_quadratic", prob, r, p, 2, B.PRECISION[prec], 1.0, 3, V0=V0, lam0=lam0)
    a.meg_step(4)
    b.meg_step(4)
    M = _mirror(obj, gpu_factored(a), 1.0)
    U = np.random.default_rng(5).standard_normal((n, r + p))
    steps = 20
    est_g = a.meg_trace_exp_estimate(U, steps)
    est_o = float(np.mean([meg.lanczos_quadrature(lambda v: M @ v, U[:, j], steps) for j in range(r + p)]))
    exact = float(np.sum(np.exp(np.linalg.eigvalsh(M))))
    print(f"{prec}: GPU {est_g:.9e}  oracle quadrature {est_o:.9e}  exact Tr exp(M) {exact:.9e}")
    assert abs(est_g - est_o) <= 1e-4 * abs(est_o), (est_g, est_o)
    a.meg_step(1)
    b.meg_step(1)
    for x, y in zip(a.meg_get_iterate(), b.meg_get_iterate()):
        assert np.array_equal(np.asarray(x), np.asarray(y))
    with pytest.raises(B.MegError):
        a.meg_trace_exp_estimate(U, 33)                      # at most 32 steps
    a.meg_destroy()
    b.meg_destroy()
