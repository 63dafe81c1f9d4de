"""meg_solve and the failure paths of the C ABI, on the GPU.

meg_solve runs Algorithm 2 until the relative objective gap
(f(X_t) - f*) / (f(X_1) - f*) <= tol (problem statement, eq. Model), testing
the gap every 10 iterations on the device.  The instance is the config-0
recipe without noise: M = U diag(.4, .25, .15, .12, .08) U^T lies in the
spectrahedron, so X* = M and f* = 0 exactly, and the oracle gives the
iteration at which the gap first falls below tol.

Failure detection (all made on the host side or by the input data; no
test here hangs or faults the GPU): CSR structure checks, the footprint
refusal (MEG_ERR_OOM before any allocation), and a non-finite input that
the k x k island reports as MEG_ERR_NUMERIC, after which the solve answers
MEG_ERR_STATE to every call but meg_destroy.
"""
import numpy as np
import pytest

import synth
from oracle import meg

from meg_cases import gpu_factored, make_gpu_solve, rel_frob

pytestmark = pytest.mark.gpu

W0 = (0.4, 0.25, 0.15, 0.12, 0.08)


def _noiseless_config0(n=200, seed=1000):
    prob = synth.dense_quadratic(n, 5, seed=seed, weights=W0, sigma=0.0)
    assert abs(np.trace(prob.M) - 1.0) < 1e-12
    return prob


def _oracle_solve(obj, V0, lam0, t0, tol, max_iters, chunk=10):
    """Oracle run of meg_solve's rule after t0 plain steps: (iterations of the
    solve, X after them, gaps at the chunk ends)."""
    X = meg.init_X1(V0, lam0, meg.eps_schedule(0))
    f1 = obj.value(X)
    W = None
    t = 0
    for _ in range(t0):
        t += 1
        X, _, W = meg.lowrank_step(X, obj, t, 1.0, meg.eps_schedule(t), method="exact", k=9, W0=W)
    gaps = []
    done = 0
    while done < max_iters:
        step = min(chunk, max_iters - done)
        for _ in range(step):
            t += 1
            X, _, W = meg.lowrank_step(X, obj, t, 1.0, meg.eps_schedule(t), method="exact", k=9, W0=W)
        done += step
        gaps.append(obj.value(X) / f1)
        if gaps[-1] <= tol:
            return done, X, gaps, True
    return done, X, gaps, False


def test_meg_solve_stops_where_the_oracle_gap_falls_below_tol():
    """After 3 meg_step calls, meg_solve(tol=1e-4) must stop at the first
    10-iteration boundary where the oracle's gap, measured against f(X_1)
    (not f at the call's entry), is <= tol, with X equal to the oracle's."""
    from paper_2012_10469_gb300 import binding as B
    prob = _noiseless_config0()
    obj = meg.DenseQuadratic(prob.M)
    V0, lam0 = meg.warm_start(obj, 5)
    tol = 1e-4
    exp_iters, Xo, gaps, conv = _oracle_solve(obj, V0, lam0, 3, tol, 400)
    assert conv
    # with f at the call's entry as the denominator the rule would stop elsewhere
    f1 = obj.value(meg.init_X1(V0, lam0, meg.eps_schedule(0)))
    s = make_gpu_solve("dense_quadratic", prob, 5, 4, 2, B.MEG_FP64, 1.0, 3, V0=V0, lam0=lam0)
    s.meg_step(3)
    f_entry = s.meg_objective()
    assert f_entry < 0.5 * f1
    it, ok = s.meg_solve(tol, 400)
    assert ok
    near = any(abs(g - tol) <= 1e-6 * tol for g in gaps[-2:])
    if near:
        assert abs(it - exp_iters) <= 10
    else:
        assert it == exp_iters, (it, exp_iters, gaps[-3:])
        assert rel_frob(gpu_factored(s), Xo) <= 1e-9
    # the iteration counter of the solve advanced by exactly the reported count
    _, t = s.meg_get_ritz()
    assert t == 3 + it
    s.meg_destroy()


def test_meg_solve_remainder_and_not_converged():
    """max_iters not a multiple of the 10-iteration check: 25 iterations run
    (two device chunks, then 5 plain steps), MEG_ERR_NOT_CONVERGED for an
    unreachable tol, and X equals the oracle's after 25 iterations."""
    from paper_2012_10469_gb300 import binding as B
    prob = _noiseless_config0(n=160, seed=1007)
    obj = meg.DenseQuadratic(prob.M)
    V0, lam0 = meg.warm_start(obj, 5)
    exp_iters, Xo, _, conv = _oracle_solve(obj, V0, lam0, 0, 1e-300, 25)
    assert exp_iters == 25 and not conv
    s = make_gpu_solve("dense_quadratic", prob, 5, 4, 2, B.MEG_FP64, 1.0, 3, V0=V0, lam0=lam0)
    it, ok = s.meg_solve(1e-300, 25)
    assert (it, ok) == (25, False)
    assert rel_frob(gpu_factored(s), Xo) <= 1e-9
    # a second call continues from X_26 with the same f(X_1)
    it2, ok2 = s.meg_solve(1e-300, 7)
    assert (it2, ok2) == (7, False)
    s.meg_destroy()


def test_meg_solve_rejects_an_undefined_gap():
    """A linear objective whose f(X_1) is negative: with the default f* = 0
    the relative gap is undefined and meg_solve refuses (MEG_ERR_INVALID_ARG);
    with f* = lambda_min(C) (Lemma 1) below f(X_1) it runs."""
    from paper_2012_10469_gb300 import binding as B
    n = 64
    rng = np.random.default_rng(71)
    C = rng.standard_normal((n, n))
    C = 0.5 * (C + C.T) - 3.0 * np.eye(n)          # every eigenvalue well below 0
    prob = synth.Linear(n=n, C=C, storage="f64")
    obj = meg.Linear(C)
    V0, lam0 = meg.warm_start(obj, 1)
    f1 = obj.value(meg.init_X1(V0, lam0, meg.eps_schedule(0)))
    assert f1 < 0
    s = make_gpu_solve("linear", prob, 1, 3, 2, B.MEG_FP64, 0.5, 5, V0=V0, lam0=lam0)
    with pytest.raises(B.MegError) as ei:
        s.meg_solve(1e-3, 50)
    assert ei.value.status == B.MEG_ERR_INVALID_ARG
    s.meg_set_fstar(float(np.linalg.eigvalsh(C)[0]))
    it, _ = s.meg_solve(1e-3, 50)
    assert 10 <= it <= 50
    s.meg_destroy()


def test_meg_solve_f1_survives_a_checkpoint():
    """f(X_1) is part of the small state: a solve restored from a checkpoint
    taken after 5 steps stops where the original does."""
    from paper_2012_10469_gb300 import binding as B
    prob = _noiseless_config0(n=128, seed=1003)
    obj = meg.DenseQuadratic(prob.M)
    V0, lam0 = meg.warm_start(obj, 5)
    a = make_gpu_solve("dense_quadratic", prob, 5, 4, 2, B.MEG_FP64, 1.0, 3, V0=V0, lam0=lam0)
    a.meg_step(5)
    state = a.meg_get_state()
    b = make_gpu_solve("dense_quadratic", prob, 5, 4, 2, B.MEG_FP64, 1.0, 3, V0=V0, lam0=lam0)
    b.meg_set_state(state)
    assert b.small_state()[B.SM_F1] == a.small_state()[B.SM_F1]
    ia, _ = a.meg_solve(1e-4, 400)
    ib, _ = b.meg_solve(1e-4, 400)
    assert ia == ib
    for s_ in (a, b):
        s_.meg_destroy()


# ---------------------------------------------------------------- failure detection
def test_csr_structure_is_validated():
    """Malformed CSR structure is refused by meg_set_objective before any
    kernel reads it: rowptr not monotone, rowptr[n] != nnz, a column index
    outside [0, n)."""
    import torch
    from paper_2012_10469_gb300 import binding as B
    prob = synth.completion(60, 3, 0.3, seed=72)
    s = B.Solve(prob.n, 3, p=3, q=2, precision=B.MEG_FP32, seed=1,
                stream=torch.cuda.current_stream().cuda_stream)
    val = torch.from_numpy(prob.val.astype(np.float32)).cuda()

    def attempt(rowptr, col):
        with pytest.raises(B.MegError) as ei:
            s.meg_set_objective(B.MEG_CSR_QUAD, rowptr=torch.from_numpy(rowptr.astype(np.int32)).cuda(),
                                col=torch.from_numpy(col.astype(np.int32)).cuda(), val=val)
        assert ei.value.status == B.MEG_ERR_INVALID_ARG

    rp = prob.rowptr.copy()
    i = int(np.argmax(np.diff(rp) > 1)) + 1
    rp[i] = rp[i + 1] + 1                          # rowptr[i] > rowptr[i + 1]
    attempt(rp, prob.col)
    rp = prob.rowptr.copy()
    rp[-1] -= 1                                    # rowptr[n] != nnz
    attempt(rp, prob.col)
    col = prob.col.copy()
    col[len(col) // 2] = prob.n                    # column index out of range
    attempt(prob.rowptr, col)
    col[len(col) // 2] = -1
    attempt(prob.rowptr, col)
    # the well-formed structure is accepted by the same solve afterwards
    s.meg_set_objective(B.MEG_CSR_QUAD, rowptr=torch.from_numpy(prob.rowptr.astype(np.int32)).cuda(),
                        col=torch.from_numpy(prob.col.astype(np.int32)).cuda(), val=val)
    s.meg_destroy()


def test_oversized_solve_is_refused_before_allocating():
    """A solve whose buffers (meg_footprint) exceed the device's free memory
    gets MEG_ERR_OOM without any allocation; n above 2^28 is an argument
    error."""
    import torch
    from paper_2012_10469_gb300 import binding as B
    n = 1 << 28
    free, _ = torch.cuda.mem_get_info()
    need = B.meg_footprint(n, 30, 2, B.MEG_FP64, -1)
    assert need > free
    with pytest.raises(B.MegError) as ei:
        B.Solve(n, 30, p=2, q=2, precision=B.MEG_FP64)
    assert ei.value.status == B.MEG_ERR_OOM
    with pytest.raises(B.MegError) as ei:
        B.Solve(n + 1, 3, p=2, q=2, precision=B.MEG_FP64)
    assert ei.value.status == B.MEG_ERR_INVALID_ARG
    # the device is still usable: an ordinary solve runs
    prob = _noiseless_config0(n=96, seed=1009)
    obj = meg.DenseQuadratic(prob.M)
    V0, lam0 = meg.warm_start(obj, 5)
    s = make_gpu_solve("dense_quadratic", prob, 5, 3, 2, B.MEG_FP64, 1.0, 3, V0=V0, lam0=lam0)
    s.meg_step(2)
    s.meg_get_iterate()
    s.meg_destroy()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_non_finite_data_latches_the_solve(prec):
    """Data with a NaN entry: the island finds non-finite Ritz values and
    records MEG_ERR_NUMERIC; the first synchronising call reports it and
    every later call but meg_destroy answers MEG_ERR_STATE."""
    from paper_2012_10469_gb300 import binding as B
    prob = _noiseless_config0(n=64, seed=1011)
    obj = meg.DenseQuadratic(prob.M)
    V0, lam0 = meg.warm_start(obj, 5)
    M = prob.M.copy()
    M[3, 5] = M[5, 3] = np.nan
    bad = synth.DenseQuadratic(n=prob.n, M=M, storage=prob.storage, U=prob.U, w=prob.w)
    s = make_gpu_solve("dense_quadratic", bad, 5, 3, 2, B.PRECISION[prec], 1.0, 3, V0=V0, lam0=lam0)
    s.meg_step(2)                                   # enqueued; nothing is known yet
    with pytest.raises(B.MegError) as ei:
        s.meg_get_iterate()
    assert ei.value.status == B.MEG_ERR_NUMERIC
    for call in (s.meg_get_iterate, s.meg_objective, lambda: s.meg_step(1), s.meg_certificate,
                 s.meg_get_ritz, lambda: s.meg_solve(1e-3, 10), s.meg_get_state, lambda: s.meg_warm_start(2)):
        with pytest.raises(B.MegError) as ei:
            call()
        assert ei.value.status == B.MEG_ERR_STATE
    s.meg_destroy()
    # other solves are unaffected
    good = make_gpu_solve("dense_quadratic", prob, 5, 3, 2, B.PRECISION[prec], 1.0, 3, V0=V0, lam0=lam0)
    good.meg_step(2)
    good.meg_get_iterate()
    good.meg_destroy()
