"""CUDA path vs the float64 oracle, element by element, on the same seeded
inputs, through the C ABI.  Tolerances: relative Frobenius error of X_t
<= 1e-5, relative error of the objective <= 1e-6 and of the top-r Ritz
values sigma_1..r <= 1e-6.  The certificate's sigma_{r+1} is a Ritz value
of a k-dimensional subspace: it never exceeds the exact eigenvalue
(Cauchy interlacing) and matches it where the (r+1)-th eigenvalue is
separated from the rest; the reported certificate must equal the paper's
formula on the reported Ritz values, and the "holds" flags must agree
unless the oracle's certificate is within the sigma_{r+1} gap of 2 eps_t.
"""
import numpy as np
import pytest

import synth
from oracle import meg

from meg_cases import gpu_factored, make_gpu_solve, oracle_objective, rel_frob, run_pair

pytestmark = pytest.mark.gpu

TOL_X, TOL_F, TOL_SIG = 1e-5, 1e-6, 1e-6


def _check(rows, r, tol_x=TOL_X, tol_f=TOL_F, tol_sig=TOL_SIG, tol_r1=None, tol_eval=None,
           r1_from=10, r1_slack=1e-9):
    """Objective: the kernel's f(X_t) must equal the oracle's f on the same
    (GPU) iterate to tol_eval (relative), and the GPU iterate's f must match
    the oracle iterate's f to tol_f relative to the run's objective scale
    f(X_1) (f -> f* = 0 for noiseless measurements, where an error relative
    to f(X_t) itself is undefined).
    tol_r1: when given, sigma_{r+1} must match to that relative error from
    iteration r1_from on (cases whose (r+1)-th eigenvalue is separated from
    the rest; the extra subspace vectors start random).  Always: the GPU's
    sigma_{r+1} is a Ritz value of a k-dimensional subspace, so it never
    exceeds the exact eigenvalue (up to r1_slack relative: the rounding of the
    storage precision)."""
    for row in rows:
        ex = rel_frob(row["Xg"], row["Xo"])
        es = np.max(np.abs(row["sig_g"][:r] - row["sig_o"][:r]) / np.abs(row["sig_o"][:r]))
        scale = max(abs(row["fo"]), abs(row["f1"]))
        ef = abs(row["fo_at_g"] - row["fo"]) / scale
        ee = abs(row["fg"] - row["fo_at_g"]) / max(abs(row["fo_at_g"]), 1e-300)
        assert ex <= tol_x, f"t={row['t']}: X rel err {ex:.3e}"
        assert es <= tol_sig, f"t={row['t']}: sigma rel err {es:.3e}"
        assert ef <= tol_f, f"t={row['t']}: f rel err {ef:.3e} ({row['fo_at_g']!r} vs {row['fo']!r})"
        assert ee <= (tol_eval or 1e-7), f"t={row['t']}: f evaluation rel err {ee:.3e}"
        dr1 = row["sig_g"][r] - row["sig_o"][r]
        if r1_slack is not None:     # None: the oracle's sigma_r+1 is itself a Ritz value
            assert dr1 <= r1_slack * abs(row["sig_o"][r]), f"t={row['t']}: Ritz sigma_r+1 above the eigenvalue"
        if tol_r1 is not None and row["t"] >= r1_from:
            assert abs(dr1) <= tol_r1 * abs(row["sig_o"][r]), f"t={row['t']}: sigma_r+1 err {dr1:.3e}"
        # the certificate the GPU reports is the paper's formula on its own Ritz values
        c_self = (np.log(row["Xg"].n - r) + row["sig_g"][r] - np.log(row["eps"])
                  - np.logaddexp.reduce(row["sig_g"][: r + 1]))
        assert abs(row["cert_g"] - c_self) <= 1e-10 * max(1.0, abs(c_self)), (row["cert_g"], c_self)
        if abs(row["cert_o"] - 2 * row["eps"]) > abs(dr1) + 1e-6:
            assert row["holds_g"] == row["holds_o"]


def test_config0_fp64_full_run():
    """Dense quadratic n=200 r=5 (weights .4 .25 .15 .12 .08, noise 1e-4), FP64, 200 iterations."""
    from paper_2012_10469_gb300 import binding as B
    prob = synth.config(0)
    rows = run_pair("dense_quadratic", prob, 5, 4, 2, B.MEG_FP64, 1.0, 200, {1, 2, 10, 100, 200})
    _check(rows, 5, tol_eval=1e-12)
    for row in rows:      # float64 throughout: the objective also matches relative to f(X_t)
        assert abs(row["fg"] - row["fo"]) <= 1e-10 * abs(row["fo"])


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_separated_r_plus_1(prec):
    """Planted rank r + 1 with a distinct (r+1)-th weight: sigma_{r+1} is
    separated from the bulk, so the certificate's eigenvalue must match too."""
    from paper_2012_10469_gb300 import binding as B
    n, r = 256, 3
    prob = synth.dense_quadratic(n, r + 1, seed=60, sigma=1e-5, weights=(0.45, 0.3, 0.2, 0.05),
                                 storage={"fp64": "f64", "fp32": "f32", "bf16": "bf16"}[prec])
    obj = meg.DenseQuadratic(prob.M)
    V0, lam0 = meg.warm_start(obj, r)
    rows = run_pair("dense_quadratic", prob, r, 4, 2, B.PRECISION[prec], 1.0, 25, {1, 10, 25},
                    warm=(V0, lam0))
    _check(rows, r, tol_r1=1e-6)


def test_checkpoint_resume_bitwise():
    """T steps, save, restore into a fresh solve, T more == 2T steps, bit for bit."""
    from paper_2012_10469_gb300 import binding as B
    prob = synth.config(0, scale=120)
    obj = meg.DenseQuadratic(prob.M)
    V0, lam0 = meg.warm_start(obj, 5)
    a = make_gpu_solve("dense_quadratic", prob, 5, 3, 2, B.MEG_FP32, 1.0, 4, V0=V0, lam0=lam0)
    a.meg_step(14)
    Va, mua, sa = a.meg_get_iterate()
    b = make_gpu_solve("dense_quadratic", prob, 5, 3, 2, B.MEG_FP32, 1.0, 4, V0=V0, lam0=lam0)
    b.meg_step(7)
    state = b.meg_get_state()
    c = make_gpu_solve("dense_quadratic", prob, 5, 3, 2, B.MEG_FP32, 1.0, 4, V0=V0, lam0=lam0)
    c.meg_set_state(state)
    c.meg_step(7)
    Vc, muc, sc = c.meg_get_iterate()
    assert np.array_equal(Va, Vc) and np.array_equal(mua, muc) and sa == sc
    for s_ in (a, b, c):
        s_.meg_destroy()


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_config1_scaled(prec):
    """Dense quadratic recipe of the n=4096 workload at n=384 (several tiles, ragged tail)."""
    from paper_2012_10469_gb300 import binding as B
    prob = synth.config(1, scale=384, storage="bf16" if prec == "bf16" else "f32")
    rows = run_pair("dense_quadratic", prob, 10, 6, 2, B.PRECISION[prec], 1.0, 30, {1, 5, 30})
    _check(rows, 10)
    s = make_gpu_solve("dense_quadratic", prob, 10, 6, 2, B.PRECISION[prec], 1.0, 1)
    assert np.frombuffer(s.meg_get_state()[:64], dtype=np.int64)[7] == (1 if prec == "bf16" else 0)
    s.meg_destroy()


@pytest.mark.parametrize("n", [392, 250])
def test_bf16_ragged_sizes(n):
    """bf16 dense product at sizes with partial 128-row tiles and 64-column K
    blocks (n = 392, tensor-core path) and with n not a multiple of 8 (n = 250,
    where the CUDA-core product is used)."""
    from paper_2012_10469_gb300 import binding as B
    prob = synth.dense_quadratic(n, 5, seed=80 + n, sigma=1e-5, storage="bf16")
    rows = run_pair("dense_quadratic", prob, 5, 3, 2, B.MEG_MIXED_BF16, 1.0, 12, {1, 12})
    _check(rows, 5)
    s = make_gpu_solve("dense_quadratic", prob, 5, 3, 2, B.MEG_MIXED_BF16, 1.0, 1)
    tc = np.frombuffer(s.meg_get_state()[:64], dtype=np.int64)[7]
    assert tc == (1 if n % 8 == 0 else 0)      # tcgen05 product where TMA can address the rows
    s.meg_destroy()


def test_linear_fp64():
    """<C, X> with a separated bottom eigenvalue of C."""
    from paper_2012_10469_gb300 import binding as B
    prob = synth.linear(150, seed=31, scale=0.05)
    u = synth.orthonormal(np.random.default_rng(45), 150, 1)
    prob.C = prob.C - 2.0 * u @ u.T
    rows = run_pair("linear", prob, 1, 4, 2, B.MEG_FP64, 0.3, 40, {1, 20, 40})
    _check(rows, 1)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_completion(prec):
    """Matrix completion, n=300, 30% of the upper triangle, 6 products per iteration."""
    from paper_2012_10469_gb300 import binding as B
    prob = synth.completion(300, 4, 0.3, seed=32)
    rows = run_pair("completion", prob, 4, 4, 6, B.PRECISION[prec], 1.0, 20, {1, 10, 20})
    _check(rows, 4)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_measurements(prec):
    """Stochastic quadratic measurements (minibatch L=128 of m=40n), warm start
    X_0 = the planted rank-3 point (a valid input of Algorithm 2); eta = 1/(4(1+n/L))."""
    from paper_2012_10469_gb300 import binding as B
    n = 96
    prob = synth.measurements(n, 3, 40 * n, 128, seed=33)
    eta = 1.0 / (4 * (1 + n / prob.L))
    rows = run_pair("measurements", prob, 3, 4, 6, B.PRECISION[prec], eta, 15, {1, 8, 15}, seed=77,
                    warm=(prob.U, prob.w))
    _check(rows, 3)


@pytest.mark.parametrize("kind", ["dense_quadratic", "completion", "measurements", "linear"])
def test_warm_start(kind):
    """eq. (exp:init) computed on the device vs the oracle."""
    from paper_2012_10469_gb300 import binding as B
    n, r = 160, 3
    if kind == "dense_quadratic":
        prob = synth.dense_quadratic(n, r, seed=40, sigma=1e-4)
    elif kind == "linear":
        # C with a separated bottom eigenvalue (the optimum of <C, X> is its eigenvector)
        prob, r = synth.linear(n, seed=41, scale=0.05), 1
        u = synth.orthonormal(np.random.default_rng(44), n, 1)
        prob.C = prob.C - 2.0 * u @ u.T
    elif kind == "completion":
        prob = synth.completion(n, r, 0.4, seed=42)
    else:
        prob = synth.measurements(n, r, 20 * n, 32, seed=43)
    obj = oracle_objective(kind, prob, seed=3)
    V0, lam0 = meg.warm_start(obj, r)
    Xo = meg.init_X1(V0, lam0, meg.eps_schedule(0))
    s = make_gpu_solve(kind, prob, r, 6, 2, B.MEG_FP64, 1.0, 3)
    s.meg_warm_start(3000)
    Xg = gpu_factored(s)
    assert rel_frob(Xg, Xo) <= 1e-6
    s.meg_destroy()


def test_group_equals_alone():
    """Solves stepped together by grouped kernels give the results of each alone."""
    import torch
    from paper_2012_10469_gb300 import binding as B
    probs = [synth.dense_quadratic(n, r, seed=50 + n, sigma=1e-4) for n, r in ((130, 2), (257, 4), (64, 3))]
    rs = (2, 4, 3)
    alone, grouped = [], []
    for prob, r in zip(probs, rs):
        obj = meg.DenseQuadratic(prob.M)
        V0, lam0 = meg.warm_start(obj, r)
        a = make_gpu_solve("dense_quadratic", prob, r, 3, 2, B.MEG_FP64, 1.0, 9, V0=V0, lam0=lam0)
        a.meg_step(12)
        alone.append(gpu_factored(a))
        a.meg_destroy()
        grouped.append(make_gpu_solve("dense_quadratic", prob, r, 3, 2, B.MEG_FP64, 1.0, 9, V0=V0, lam0=lam0))
    g = B.Group(grouped, stream=torch.cuda.current_stream().cuda_stream)
    g.meg_group_step(12)
    for s, Xa in zip(grouped, alone):
        assert rel_frob(gpu_factored(s), Xa) <= 1e-12
    g.meg_group_destroy()


@pytest.mark.parametrize("prec", ["fp64", "bf16"])
def test_group_time_chain_leaves_iterates(prec):
    """meg_group_time_chain runs the chain kernels many times on the group's
    current block; W, its split and the small state are restored, so a group
    timed mid-run reaches bitwise the iterate of an untimed twin."""
    import torch
    from paper_2012_10469_gb300 import binding as B
    precision = B.PRECISION[prec]
    storage = {"fp64": "f64", "bf16": "bf16"}[prec]
    probs = [synth.dense_quadratic(n, r, seed=70 + n, sigma=1e-4, storage=storage) for n, r in ((256, 3), (384, 5))]
    rs = (3, 5)
    stream = torch.cuda.current_stream().cuda_stream

    def group():
        ss = [make_gpu_solve("dense_quadratic", p, r, 4, 3, precision, 1.0, 13, V0=p.U, lam0=p.w)
              for p, r in zip(probs, rs)]
        return ss, B.Group(ss, stream=stream)

    timed, gt = group()
    plain, gp = group()
    try:
        gt.meg_group_step(3)
        us = gt.meg_group_time_chain(5)
        assert len(us) == 6 and all(v > 0 for v in (us[0], us[1], us[2], us[5]))
        assert (us[3] > 0 and us[4] > 0) if prec == "fp64" else (us[3] == 0 and us[4] == 0)
        gt.meg_group_step(3)
        gp.meg_group_step(6)
        for a, b in zip(timed, plain):
            Xa, Xb = gpu_factored(a), gpu_factored(b)
            assert np.array_equal(Xa.V, Xb.V) and np.array_equal(Xa.mu, Xb.mu) and Xa.s == Xb.s
    finally:
        gt.meg_group_destroy()
        gp.meg_group_destroy()
        for x in timed + plain:
            x.meg_destroy()


def test_invalid_arguments_rejected():
    from paper_2012_10469_gb300 import binding as B
    with pytest.raises(B.MegError) as e:
        B.Solve(10, 10, p=1)
    assert e.value.status == B.MEG_ERR_INVALID_ARG
    with pytest.raises(B.MegError):
        B.Solve(100, 5, p=40)
    with pytest.raises(B.MegError):
        B.Solve(100, 5, eps=(0.9, 0.0, 2.0))          # eps_0 > 3/4 violates Lemma 2
    s = B.Solve(50, 2, p=2)
    with pytest.raises(B.MegError) as e:
        s.meg_step(1)                                  # no objective yet
    assert e.value.status == B.MEG_ERR_STATE
