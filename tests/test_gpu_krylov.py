"""Block Krylov Rayleigh-Ritz on the GPU (MEG_EIG_BLOCK_KRYLOV) against the
float64 oracle.

Section 3 computes the top-r eigenpairs of M_t by subspace iteration and
names Lanczos-type methods as the faster alternative.  The GPU's block
Krylov eigensolver makes two products per MEG iteration, A W0 and A W1 with
W1 the orthonormalised part of A W0 outside span W0 (A = M_t - c I), and runs
the Rayleigh-Ritz step on span [W0 W1] (2k columns); the next iteration
starts from the top-k Ritz vectors.  The oracle's iterates are those of
exact low-rank MEG: its exact eigensolver (dense eigh) at small n, its own
block Krylov solver run to a residual of 1e-12 (`lowrank_step(method=
"krylov")`) and its subspace solver at n = 4096.  Tolerances as in the
other parity tests: X_t 1e-5 relative Frobenius, sigma_1..r 1e-6 relative,
f 1e-6 (denominator per workload, stated at each test).
"""
import numpy as np
import pytest

import synth
from oracle import meg

from meg_cases import gpu_factored, make_gpu_solve, oracle_objective, rel_frob, run_pair, to_device_dense
from test_gpu_parity import _check

pytestmark = pytest.mark.gpu

KRY = 1


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_krylov_dense_scaled(prec):
    """Dense quadratic recipe of the n = 4096 workload at n = 384 (several
    tensor-core tiles), r = 6, k = 10 (a 20-column Krylov space), against the
    oracle's exact eigensolver."""
    from paper_2012_10469_gb300 import binding as B
    prob = synth.config(1, scale=384, storage="bf16" if prec == "bf16" else "f32")
    rows = run_pair("dense_quadratic", prob, 6, 4, 2, B.PRECISION[prec], 1.0, 30, {1, 5, 30}, eigensolver=KRY)
    _check(rows, 6, r1_slack=1e-7)


@pytest.mark.parametrize("kind", ["completion", "measurements", "linear"])
def test_krylov_other_objectives(kind):
    """The sparse, minibatch and linear gradient products under the block
    Krylov eigensolver (float32 storage), against the oracle's own block
    Krylov solver (converged) or its exact one."""
    from paper_2012_10469_gb300 import binding as B
    if kind == "completion":
        prob = synth.completion(300, 4, 0.2, seed=91)
        r, eta, method = 4, 1.0, "krylov"
    elif kind == "measurements":
        prob = synth.measurements(96, 3, 40 * 96, 128, seed=33)
        r, eta, method = 3, 1.0 / (4 * (1 + 96 / 128)), "exact"
    else:
        prob = synth.linear(200, seed=93)
        r, eta, method = 1, 0.3, "exact"
    obj = oracle_objective(kind, prob, seed=7)
    if kind == "measurements":
        warm = (prob.U, prob.w)        # the planted point (a valid X_0 of Algorithm 2)
    elif kind == "completion":
        warm = (prob.U, prob.w)
    else:
        warm = meg.warm_start(obj, r)
    rows = run_pair(kind, prob, r, 5, 2, B.MEG_FP32, eta, 12, {1, 12}, method=method, warm=warm,
                    eigensolver=KRY)
    _check(rows, r, r1_slack=None if method == "krylov" else 1e-7, tol_eval=1e-6)


def test_krylov_config1_batch_to_the_horizon():
    """The n = 4096 batch of 8 with the block Krylov eigensolver (p = 4,
    k = 14, a 28-column Krylov space, two tensor-core products per
    iteration), two sampled instances at t = 1, 100, 250, 500: one against
    the oracle's block Krylov solver, one against its subspace solver (both
    converged).  f* > 0: f is compared relative to f(X_t)."""
    import torch
    from paper_2012_10469_gb300 import binding as B
    from test_gpu_horizon import TOL_F, TOL_SIG, TOL_X, _errors, _report
    N, R, P = 4096, 10, 4
    probs = [synth.dense_quadratic(N, R, seed=1001 + i, sigma=1e-5, storage="bf16") for i in range(8)]
    stream = torch.cuda.current_stream().cuda_stream
    solves = [make_gpu_solve("dense_quadratic", p, R, P, 2, B.MEG_MIXED_BF16, 1.0, 1001 + i,
                             V0=p.U, lam0=p.w, eigensolver=KRY) for i, p in enumerate(probs)]
    for s in solves:
        assert np.frombuffer(s.meg_get_state()[:64], dtype=np.int64)[7] == 1     # tensor-core product
    g = B.Group(solves, stream=stream)
    sampled = {0: "krylov", 5: "subspace"}
    objs = {i: oracle_objective("dense_quadratic", probs[i]) for i in sampled}
    Xo = {i: meg.init_X1(probs[i].U, probs[i].w, meg.eps_schedule(0)) for i in sampled}
    f1 = {i: objs[i].value(Xo[i]) for i in sampled}
    Wo = {i: None for i in sampled}
    rows = {i: [] for i in sampled}
    try:
        t = 0
        for cp in (1, 100, 250, 500):
            g.meg_group_step(cp - t)
            for i, method in sampled.items():
                for tt in range(t + 1, cp + 1):
                    Xo[i], info, Wo[i] = meg.lowrank_step(Xo[i], objs[i], tt, 1.0, meg.eps_schedule(tt),
                                                          method=method, k=R + P, W0=Wo[i])
                rows[i].append(_errors(cp, solves[i], Xo[i], info, objs[i], R, f1[i]))
            t = cp
        for s in solves:
            X = gpu_factored(s)
            assert abs(X.trace() - 1.0) <= 1e-12 and np.all(X.mu > 0) and X.s > 0
    finally:
        g.meg_group_destroy()
        for s in solves:
            s.meg_destroy()
    for i, method in sampled.items():
        _report(f"n=4096 seed {1001 + i} block Krylov (p={P}) vs oracle {method}", rows[i])
    for i in sampled:
        for e in rows[i]:
            assert e["x"] <= TOL_X, (i, e)
            assert e["sig"] <= TOL_SIG, (i, e)
            assert e["f_rel_ft"] <= TOL_F, (i, e)


def test_krylov_group_equals_alone():
    """Solves of different n, r and kinds stepped in one group with the
    block Krylov eigensolver give the bits of stepping each alone."""
    from paper_2012_10469_gb300 import binding as B
    import torch
    cases = [("dense_quadratic", synth.dense_quadratic(200, 3, seed=94, sigma=1e-4, storage="bf16"), 3),
             ("dense_quadratic", synth.dense_quadratic(136, 5, seed=95, sigma=1e-4, storage="bf16"), 5),
             ("dense_quadratic", synth.dense_quadratic(96, 2, seed=96, sigma=1e-4, storage="bf16"), 2)]
    alone, grouped = [], []
    for kind, prob, r in cases:
        for dst in (alone, grouped):
            dst.append(make_gpu_solve(kind, prob, r, 4, 2, B.MEG_MIXED_BF16, 1.0, 11, V0=prob.U, lam0=prob.w,
                                      eigensolver=KRY))
    for s in alone:
        s.meg_step(7)
    g = B.Group(grouped, stream=torch.cuda.current_stream().cuda_stream)
    g.meg_group_step(7)
    g.meg_group_destroy()
    for a, b in zip(alone, grouped):
        Va, ma, sa = a.meg_get_iterate()
        Vb, mb, sb = b.meg_get_iterate()
        assert np.array_equal(Va, Vb) and np.array_equal(ma, mb) and sa == sb
        a.meg_destroy()
        b.meg_destroy()


def test_krylov_argument_checks():
    """Block Krylov needs q = 2, a 2k <= 32 column space and float storage."""
    from paper_2012_10469_gb300 import binding as B
    for kw in (dict(q=3, precision=B.MEG_FP32, p=4), dict(q=2, precision=B.MEG_FP64, p=4),
               dict(q=2, precision=B.MEG_FP32, p=8)):
        with pytest.raises(B.MegError) as ei:
            B.Solve(256, 10, eigensolver=KRY, **kw)
        assert ei.value.status == B.MEG_ERR_INVALID_ARG


def test_autotune_chooses_between_the_eigensolvers():
    """With krylov=True, meg_autotune tries q = 1 (subspace), then at q = 2
    subspace iteration, then the block Krylov candidates, then q = 3 ...; the
    returned (eigensolver, q, p) is the first within tol_x sqrt(pilot/horizon)
    of the reference, checked by running the candidates through the C ABI."""
    import torch
    from paper_2012_10469_gb300 import binding as B
    n, r = 384, 6
    prob = synth.dense_quadratic(n, r, seed=1500, sigma=1e-5, storage="bf16")
    D = to_device_dense(prob, B.MEG_MIXED_BF16)
    ps, q_max, pilot, horizon, tol = (2, 4, 8), 3, 12, 400, 1e-5
    stream = torch.cuda.current_stream().cuda_stream
    p, q, err, ok, eig = B.meg_autotune(n, r, B.MEG_MIXED_BF16, B.MEG_DENSE_QUAD, prob.U, prob.w, dense=D, seed=3,
                                        q_max=q_max, p_cand=ps, pilot_iters=pilot, horizon=horizon, tol_x=tol,
                                        stream=stream, krylov=True)
    accept = tol * np.sqrt(pilot / horizon)

    def run(pp, qq, ee):
        s = B.Solve(n, r, p=pp, q=qq, precision=B.MEG_MIXED_BF16, seed=3, V0=prob.U, lam0=prob.w, stream=stream,
                    eigensolver=ee)
        s.meg_set_objective(B.MEG_DENSE_QUAD, dense=D)
        s.meg_step(pilot)
        X = gpu_factored(s)
        s.meg_destroy()
        return X

    ref = run(min(32 - r, 2 * max(ps)), q_max + 2, 0)
    order = [(1, pp, 0) for pp in ps] + [(2, pp, 0) for pp in ps] + \
            [(2, pp, KRY) for pp in ps if 2 * (r + pp) <= 32] + [(3, pp, 0) for pp in ps]
    found = None
    for qq, pp, ee in order:
        e = rel_frob(run(pp, qq, ee), ref)
        if e <= accept:
            found = (pp, qq, ee, e)
            break
    assert ok and found is not None
    assert (p, q, eig) == found[:3] and abs(err - found[3]) <= 1e-6 * found[3] + 1e-15
