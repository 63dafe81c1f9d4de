"""CPU emulation, in float32 arithmetic, of the numerical method the CUDA path
uses for the float-storage modes' single CholeskyQR pass (no GPU, no oracle):
the Gram S = Z^T Z is known to double-word accuracy; M1 is the float Cholesky
factor of S rounded to float; B = M1^T S M1 is formed exactly and rounded to
float; M2 is the float factor of B; M = M1 M2 is applied to the float rows of
Z with exact products and W is rounded once.  The claim checked: W is
orthonormal to a few float rounding units whatever the conditioning of Z,
where one plain float factor leaves about kappa(Z)^2 units (which is why the
refinement replaces the second pass over the rows)."""
import numpy as np


def _pass(Z32, refine):
    Zd = Z32.astype(np.float64)
    S = Zd.T @ Zd
    M1 = np.linalg.inv(np.linalg.cholesky(S.astype(np.float32))).T.astype(np.float32)
    M = M1.astype(np.float64)
    if refine:
        B = (M.T @ S @ M).astype(np.float32)
        M2 = np.linalg.inv(np.linalg.cholesky(B)).T.astype(np.float32)
        M = M @ M2.astype(np.float64)
    W = (Zd @ M).astype(np.float32).astype(np.float64)
    return np.linalg.norm(W.T @ W - np.eye(W.shape[1]), 2)


def test_one_pass_refined_factor_orthonormality():
    u = 2.0 ** -24
    n, k = 2048, 14
    for kappa in (1e1, 1e2, 1e3, 1e4):
        for seed in range(2):
            rng = np.random.default_rng(seed)
            U = np.linalg.qr(rng.standard_normal((n, k)))[0]
            Vt = np.linalg.qr(rng.standard_normal((k, k)))[0]
            Z32 = ((U * np.logspace(0, -np.log10(kappa), k)) @ Vt).astype(np.float32)
            refined, plain = _pass(Z32, True), _pass(Z32, False)
            assert refined <= 16 * u * np.sqrt(k), (kappa, refined)
            if kappa >= 1e3:
                assert plain >= 1e-3 * kappa ** 2 * u, (kappa, plain)   # what the refinement removes


def test_bilinear_shift_estimate_bounds_the_gradient():
    """The bilinear kind's size of grad f for the shift (the Wishart form of
    the Cauchy-Schwarz bound, g = (tau/n)(1 + sqrt(n/m))^2 (m sum_i r_i^2
    ||a_i||^2 ||b_i||^2)^(1/2)) lies above ||grad f||_2 on the Section 7
    instance at X = 0 (the warm start's operator) and along the iterates, as
    the shift of subspace iteration needs (a lower bound of the spectrum)."""
    import math
    import synth
    from oracle import meg
    n, rank = 96, 3
    p = synth.bilinear_recovery(n, rank, seed=4)
    obj = meg.BilinearMeasurements(p.A, p.B, p.y, p.tau)
    m = obj.m
    na2, nb2 = np.sum(p.A ** 2, 1), np.sum(p.B ** 2, 1)

    def est(r):
        return p.tau * (1 + math.sqrt(n / m)) ** 2 / n * math.sqrt(m * np.sum(r * r * na2 * nb2))

    assert est(-obj.y) >= np.abs(np.linalg.eigvalsh(-obj.neg_grad0_apply(np.eye(n)))).max()
    V0, lam0 = meg.warm_start_at(obj, rank, p.U, printed_sign=True)
    X = meg.init_X1(V0, lam0, meg.eps_schedule(0))
    eta = 1.0 / (p.tau * 0.4 * math.sqrt(rank * n))
    for t in range(1, 6):
        G = obj.grad_dense(X)
        assert est(obj.residual(X)) >= np.abs(np.linalg.eigvalsh(0.5 * (G + G.T))).max(), t
        X, _, _ = meg.lowrank_step(X, obj, t, eta, meg.eps_schedule(t), method="exact")
