"""CUDA path vs the float64 oracle over the workloads' configured horizons.

The per-iteration parity tests check a few iterations; these run each
full-size workload, as benchmarked (grouped kernels, CUDA graph, autotuned
p and q), for hundreds of iterations and compare with the oracle at
checkpoints spread over the run:

* n = 4096 dense quadratic, bf16 data, the batch of 8 that the benchmark
  times; two sampled instances at t = 1, 100, 250, 500 (the horizon);
* n = 2048 stochastic measurements (m = 50000, L = 256), bf16 data, at
  t = 1, 100, 250, 500;
* n = 20000 matrix completion, float32 data, at t = 1, 25, 50.

The oracle's eigensolver runs to a residual of 1e-12 (subspace iteration
for the dense and sparse problems, its block Krylov solver for the
measurement problem, whose bulk of nearly equal eigenvalues makes subspace
iteration slow), so its iterates are those of exact low-rank MEG.
Tolerances: X_t relative Frobenius <= 1e-5, sigma_1..r
relative <= 1e-6, f relative <= 1e-6 (the denominator per workload is
stated at each test).  Each test prints its measured errors.
"""
import numpy as np
import pytest

import synth
from oracle import meg

from meg_cases import gpu_factored, make_gpu_solve, oracle_objective, rel_frob, to_device_dense

pytestmark = pytest.mark.gpu

TOL_X, TOL_F, TOL_SIG = 1e-5, 1e-6, 1e-6


def _errors(t, s, Xo, info, obj, r, f1):
    Xg = gpu_factored(s)
    sig, tg = s.meg_get_ritz()
    assert tg == t
    fo, fg = obj.value(Xo), obj.value(Xg)
    return dict(t=t, x=rel_frob(Xg, Xo),
                sig=float(np.max(np.abs(sig[:r] - info.sig[:r]) / np.abs(info.sig[:r]))),
                f_rel_ft=abs(fg - fo) / abs(fo), f_rel_f1=abs(fg - fo) / abs(f1),
                trace=abs(Xg.trace() - 1.0), pos=bool(np.all(Xg.mu > 0) and Xg.s > 0))


def _report(name, rows):
    for e in rows:
        print(f"{name} t={e['t']:4d}  X {e['x']:.2e}  sigma {e['sig']:.2e}  "
              f"f/f_t {e['f_rel_ft']:.2e}  f/f_1 {e['f_rel_f1']:.2e}")


@pytest.mark.parametrize("scheme", ["benchmarked", "subspace_q3"])
def test_config1_batch_to_the_horizon(scheme):
    """n = 4096, r = 10, the benchmark's batch: with the eigensolver, p and q
    the benchmark's autotuner chooses, and with subspace iteration at
    (p, q) = (4, 3).  f* > 0 here (the noise puts M outside the
    spectrahedron), so f is compared relative to f(X_t) itself."""
    import torch
    from paper_2012_10469_gb300 import binding as B
    from test_gpu_fullsize import AUTOTUNE
    N, R = 4096, 10
    probs = [synth.dense_quadratic(N, R, seed=1001 + i, sigma=1e-5, storage="bf16") for i in range(8)]
    stream = torch.cuda.current_stream().cuda_stream
    if scheme == "benchmarked":
        P, Q, _, ok, eig = B.meg_autotune(N, R, B.MEG_MIXED_BF16, B.MEG_DENSE_QUAD, probs[0].U, probs[0].w,
                                          dense=to_device_dense(probs[0], B.MEG_MIXED_BF16), seed=1001,
                                          stream=stream, **AUTOTUNE)
        assert ok
    else:
        P, Q, eig = 4, 3, B.MEG_EIG_SUBSPACE
    solves = [make_gpu_solve("dense_quadratic", p, R, P, Q, B.MEG_MIXED_BF16, 1.0, 1001 + i,
                             V0=p.U, lam0=p.w, eigensolver=eig) for i, p in enumerate(probs)]
    g = B.Group(solves, stream=stream)
    sampled = (0, 5)
    objs = {i: oracle_objective("dense_quadratic", probs[i]) for i in sampled}
    Xo = {i: meg.init_X1(probs[i].U, probs[i].w, meg.eps_schedule(0)) for i in sampled}
    f1 = {i: objs[i].value(Xo[i]) for i in sampled}
    Wo = {i: None for i in sampled}
    rows = {i: [] for i in sampled}
    checkpoints = (1, 100, 250, 500)
    try:
        t = 0
        for cp in checkpoints:
            g.meg_group_step(cp - t)
            for i in sampled:
                for tt in range(t + 1, cp + 1):
                    Xo[i], info, Wo[i] = meg.lowrank_step(Xo[i], objs[i], tt, 1.0, meg.eps_schedule(tt),
                                                          method="subspace", k=R + P, W0=Wo[i])
                rows[i].append(_errors(cp, solves[i], Xo[i], info, objs[i], R, f1[i]))
            t = cp
    finally:
        g.meg_group_destroy()
        for s in solves:
            s.meg_destroy()
    for i in sampled:
        _report(f"n=4096 seed {1001 + i} (eigensolver {eig}, p={P}, q={Q})", rows[i])
    for i in sampled:
        for e in rows[i]:
            assert e["trace"] <= 1e-12 and e["pos"]
            assert e["x"] <= TOL_X, (i, e)
            assert e["sig"] <= TOL_SIG, (i, e)
            assert e["f_rel_ft"] <= TOL_F, (i, e)


def test_config3_measurements_to_500():
    """n = 2048, r = 4, m = 50000, L = 256, bf16 data, the autotuned (p, q).
    The measurements are noiseless, f* = 0 and f(X_t) -> 0, so the f error
    is taken relative to f(X_1), the scale of the relative gap the serving
    rule uses; relative to f(X_t) it is printed."""
    import torch
    from paper_2012_10469_gb300 import binding as B
    prob = synth.config(3)
    eta = 1.0 / (4 * (1 + prob.n / prob.L))
    obj = oracle_objective("measurements", prob, seed=1003)
    V0, lam0 = prob.U, np.full(4, 0.25)
    A = torch.from_numpy(np.ascontiguousarray(synth.bf16_bits(prob.A).view(np.int16))).cuda()
    y = torch.from_numpy(prob.y).cuda()
    P, Q, _, ok, _eig = B.meg_autotune(prob.n, 4, B.MEG_MIXED_BF16, B.MEG_MEAS_STOCH, V0, lam0, A=A, y=y,
                                  L=prob.L, eta=eta, seed=1003, q_max=7, pilot_iters=20, horizon=2000, tol_x=1e-5,
                                  stream=torch.cuda.current_stream().cuda_stream)
    assert ok, (P, Q)
    s = make_gpu_solve("measurements", prob, 4, P, Q, B.MEG_MIXED_BF16, eta, 1003, V0=V0, lam0=lam0)
    X = meg.init_X1(V0, lam0, meg.eps_schedule(0))
    f1 = obj.value(X)
    rows, W, t = [], None, 0
    for cp in (1, 100, 250, 500):
        s.meg_step(cp - t)
        for tt in range(t + 1, cp + 1):
            X, info, W = meg.lowrank_step(X, obj, tt, eta, meg.eps_schedule(tt), method="krylov", k=4 + P, W0=W)
        rows.append(_errors(cp, s, X, info, obj, 4, f1))
        t = cp
    s.meg_destroy()
    _report(f"n=2048 measurements (p={P}, q={Q})", rows)
    for e in rows:
        assert e["trace"] <= 1e-12 and e["pos"]
        assert e["x"] <= TOL_X, e
        assert e["sig"] <= TOL_SIG, e
        assert e["f_rel_f1"] <= TOL_F, e


def test_config2_completion_to_50():
    """n = 20000, r = 8, 1% of the upper triangle mirrored, float32 data, the
    workload's (p, q) = (8, 6).  M is planted in the spectrahedron (f* = 0),
    so the f error is taken relative to f(X_1); relative to f(X_t) it is
    printed."""
    from paper_2012_10469_gb300 import binding as B
    prob = synth.config(2)
    obj = oracle_objective("completion", prob)
    X = meg.init_X1(prob.U, prob.w, meg.eps_schedule(0))
    f1 = obj.value(X)
    s = make_gpu_solve("completion", prob, 8, 8, 6, B.MEG_FP32, 1.0, 1002, V0=prob.U, lam0=prob.w)
    rows, W, t = [], None, 0
    for cp in (1, 25, 50):
        s.meg_step(cp - t)
        for tt in range(t + 1, cp + 1):
            X, info, W = meg.lowrank_step(X, obj, tt, 1.0, meg.eps_schedule(tt), method="subspace", k=16, W0=W)
        rows.append(_errors(cp, s, X, info, obj, 8, f1))
        t = cp
    s.meg_destroy()
    _report("n=20000 completion (p=8, q=6)", rows)
    for e in rows:
        assert e["trace"] <= 1e-12 and e["pos"]
        assert e["x"] <= TOL_X, e
        assert e["sig"] <= TOL_SIG, e
        assert e["f_rel_f1"] <= TOL_F, e
