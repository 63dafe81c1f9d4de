"""The bilinear-measurement objective of Section 7 (eq. recoveryProb) on the
GPU, against the float64 oracle.

f(X) = 1/2 sum_i (tau a_i^T X b_i - y_i)^2 in trace-1 variables, the full
gradient every iteration.  The library computes it as two tcgen05 passes
over the stacked rows [A; B] (bf16 data): P = [A; B] [V | W], then
Y = [A; B]^T S with S_i = (tau/2) r_i b_i^T W, S_{m+i} = (tau/2) r_i a_i^T W.
The instances are the paper's (unit a_i, b_i rounded to bf16 so that both
sides see the same data; kappa = 1/2; m = 20 n r; tau = 0.5 tr M for ranks 1
and 5, 0.65 tr M for rank 20), the start is eq. (exp:init) as printed at a
random U (computed by the oracle), the step size 1 / (tau beta) with
beta = 0.4 sqrt(r n), and eps_t = 0.8 / (t + 11)^2.
"""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import meg

from meg_cases import gpu_factored, rel_frob
from test_gpu_parity import _check

pytestmark = pytest.mark.gpu


def _instance(n, rank, seed, r_svd=None):
    """The Section 7 instance with A and B rounded to bf16 (y as generated)."""
    p = synth.bilinear_recovery(n, rank, seed=seed, r_svd=r_svd)
    A, Bm = synth.bf16_round(p.A), synth.bf16_round(p.B)
    obj = meg.BilinearMeasurements(A, Bm, p.y, p.tau)
    return p, obj


def _gpu(p, obj, r, pp, q, precision, seed, V0, lam0):
    import torch
    from paper_2012_10469_gb300 import binding as B
    n = obj.n
    eta = 1.0 / (p.tau * 0.4 * math.sqrt(r * n))
    A = torch.from_numpy(np.ascontiguousarray(synth.bf16_bits(obj.A).view(np.int16))).cuda()
    Bm = torch.from_numpy(np.ascontiguousarray(synth.bf16_bits(obj.B).view(np.int16))).cuda()
    y = torch.from_numpy(obj.y).cuda()
    assert A.data_ptr() % 16 == 0 and Bm.data_ptr() % 16 == 0
    s = B.Solve(n, r, p=pp, q=q, precision=precision, eta=eta, seed=seed, V0=V0, lam0=lam0,
                stream=torch.cuda.current_stream().cuda_stream)
    s.meg_set_objective(B.MEG_BILINEAR, A=A, B=Bm, y=y, tau=p.tau)
    return s, eta


def _run(n, rank, r_svd, seed, pp, q, precision, T, checkpoints):
    p, obj = _instance(n, rank, seed, r_svd=r_svd)
    r = r_svd
    V0, lam0 = meg.warm_start_at(obj, r, p.U, printed_sign=True)
    s, eta = _gpu(p, obj, r, pp, q, precision, seed, V0, lam0)
    s.meg_refine_subspace(32)          # the start block: V_0 and random columns
    X = meg.init_X1(V0, lam0, meg.eps_schedule(0))
    f1 = obj.value(X)
    assert abs(s.meg_objective() - f1) <= 1e-7 * f1        # the kernel's f(X_1)
    rows, first_g, first_o = [], None, None
    for t in range(1, T + 1):
        X, info, _ = meg.lowrank_step(X, obj, t, eta, meg.eps_schedule(t), method="exact")
        s.meg_step(1)
        cert, holds, _ = s.meg_certificate()
        if first_g is None and holds:
            first_g = t
        if first_o is None and info.holds:
            first_o = t
        if t in checkpoints:
            Xg = gpu_factored(s)
            sig, tg = s.meg_get_ritz()
            assert tg == t
            rows.append(dict(t=t, Xg=Xg, Xo=X, sig_g=sig, sig_o=info.sig, fg=s.meg_objective(),
                             fo=obj.value(X), f1=f1, fo_at_g=obj.value(Xg), cert_g=cert, holds_g=holds,
                             cert_o=info.cert, holds_o=info.holds, eps=info.eps))
        if first_g is not None and first_o is not None and t >= max(checkpoints, default=0):
            break
    s.meg_destroy()
    return rows, first_g, first_o


@pytest.mark.parametrize("rank", [1, 5])
@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_bilinear_matches_oracle_n200(rank, prec):
    """n = 200, ranks 1 and 5 (m = 4000 and 20000 measurement pairs), 12
    iterations: X_t, sigma_1..r, f and the certificate against the oracle's
    exact low-rank MEG.  The bulk of M_t's spectrum (log s - eta times the
    gradient's noise spectrum) lies close below the top r eigenvalues, so the
    subspace iteration takes q = 8 products per iteration to reach the
    tolerances."""
    from paper_2012_10469_gb300 import binding as B
    rows, _, _ = _run(200, rank, rank, seed=31 + rank, pp=5, q=8, precision=B.PRECISION[prec], T=12,
                      checkpoints={1, 2, 6, 12})
    for e in rows:
        print(f"rank {rank} {prec} t={e['t']:3d}  X {rel_frob(e['Xg'], e['Xo']):.2e}  "
              f"f {e['fg']:.6e} vs {e['fo']:.6e}")
    _check(rows, rank, r1_slack=1e-7)


def test_bilinear_certificate_onset_table2():
    """Table 2 (n = 200, ranks 1 and 5): on 4 seeded instances the GPU's
    b^{r+1} certificate (eq. convergenceGuaranteeExperiment2) first holds at
    the same iteration as the oracle's on the same data, and the average is
    within 1 of the printed one."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "table23_certificate.json")) as fh:
        gold = json.load(fh)
    from paper_2012_10469_gb300 import binding as B
    for row in gold["table2"]:
        got = []
        for seed in range(4):
            _, fg, fo = _run(row["n"], row["rank"], row["rank"], seed, pp=5, q=8, precision=B.MEG_FP32, T=30,
                             checkpoints=set())
            assert fg == fo, (row, seed, fg, fo)
            got.append(fg if fg is not None else 31)
        print(f"Table 2 rank {row['rank']}: first hold {got} (printed {row['first_r1']})")
        assert abs(np.mean(got) - row["first_r1"]) <= 1.0, (row, got)


@pytest.mark.parametrize("rank,r_svd", [(1, 3), (5, 10)])
def test_bilinear_rank_overestimated(rank, r_svd):
    """Table 3's setting (n = 200, SVD rank r above rank M, m = 20 n r): the
    GPU's b^{r+1} certificate first holds at the oracle's iteration; over 10
    iterations X_t and f follow the oracle's to 1e-4, sigma_1..rank M to
    1e-5 and sigma_{rank M + 1..r} to 1e-2.

    Why the looser bounds: the r - rank M extra directions of M_t's top r
    sit in or just above the bulk of its spectrum (the gradient's noise),
    where neighbouring eigenvalues lie close together and subspace iteration
    resolves them slowly; their weights mu are small, so X_t is still close,
    and the MEG dynamics amplify the eigensolver's error when those
    eigenvalues move up through the spectrum (about 50x near t = 3 for
    r = 10).  A float64 restatement of the library's iteration (same q, 32
    start products) stays within 4e-5 of exact MEG here, so the bound is the
    eigensolver's, not the arithmetic's."""
    from paper_2012_10469_gb300 import binding as B
    rows, fg, fo = _run(200, rank, r_svd, seed=41 + rank, pp=4, q=8, precision=B.MEG_FP32, T=10,
                        checkpoints={1, 2, 3, 5, 10})
    for e in rows:
        rel = np.abs(e["sig_g"][:r_svd] - e["sig_o"][:r_svd]) / np.abs(e["sig_o"][:r_svd])
        ex = rel_frob(e["Xg"], e["Xo"])
        ef = abs(e["fo_at_g"] - e["fo"]) / max(abs(e["fo"]), abs(e["f1"]))
        print(f"rank {rank}, r = {r_svd}: t={e['t']:2d}  X {ex:.2e}  f {ef:.2e}  "
              f"sigma top {rel[:rank].max():.2e}  extra {rel[rank:].max():.2e}")
        assert ex <= 1e-4 and ef <= 1e-4, e["t"]
        assert rel[:rank].max() <= 1e-5 and rel[rank:].max() <= 1e-2, e["t"]
        # the certificate the GPU reports is the paper's formula on its own Ritz values
        c_self = (np.log(e["Xg"].n - r_svd) + e["sig_g"][r_svd] - np.log(e["eps"])
                  - np.logaddexp.reduce(e["sig_g"][: r_svd + 1]))
        assert abs(e["cert_g"] - c_self) <= 1e-10 * max(1.0, abs(c_self))
    print(f"rank {rank}, r = {r_svd}: first hold GPU {fg}, oracle {fo}")
    assert fg == fo


def test_bilinear_full_size_n600_r20():
    """n = 600, rank 20 (m = 240000 pairs, 2 x 288 MB of bf16 data), the
    configuration whose iteration the benchmark times (p = 8, q = 6): 2
    iterations against the oracle."""
    from paper_2012_10469_gb300 import binding as B
    rows, _, _ = _run(600, 20, 20, seed=7, pp=8, q=6, precision=B.MEG_FP32, T=2, checkpoints={1, 2})
    for e in rows:
        print(f"n=600 r=20 t={e['t']}  X {rel_frob(e['Xg'], e['Xo']):.2e}")
    _check(rows, 20, r1_slack=1e-7)


def test_bilinear_warm_start_and_arguments():
    """meg_warm_start (eq. (exp:init) at U = 0, the top eigenvectors of
    -grad f(0)) through the two passes matches the oracle; the kind rejects
    float64 storage, n % 8 != 0, misaligned data and tau <= 0."""
    import torch
    from paper_2012_10469_gb300 import binding as B
    n, rank = 96, 3
    p, obj = _instance(n, rank, seed=5)
    V0, lam0 = meg.warm_start(obj, rank)
    X1 = meg.init_X1(V0, lam0, meg.eps_schedule(0))
    s, _ = _gpu(p, obj, rank, 5, 2, B.MEG_FP32, 3, None, None)
    s.meg_warm_start(400)
    assert rel_frob(gpu_factored(s), X1) <= 1e-5, rel_frob(gpu_factored(s), X1)
    s.meg_destroy()
    A = torch.from_numpy(np.ascontiguousarray(synth.bf16_bits(obj.A).view(np.int16))).cuda()
    Bm = torch.from_numpy(np.ascontiguousarray(synth.bf16_bits(obj.B).view(np.int16))).cuda()
    y = torch.from_numpy(obj.y).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    U = np.linalg.qr(np.random.default_rng(0).standard_normal((n, rank)))[0]
    lam = np.full(rank, 1.0 / rank)
    buf = torch.zeros(A.numel() + 8, dtype=torch.int16, device="cuda")
    buf[1:1 + A.numel()] = A.view(-1)
    A_mis = buf[1:1 + A.numel()].view(A.shape)                # rows no longer 16-byte aligned
    assert A_mis.data_ptr() % 16 != 0
    bad = [(B.MEG_FP64, A, p.tau), (B.MEG_FP32, A, 0.0), (B.MEG_FP32, A, -1.0), (B.MEG_FP32, A_mis, p.tau)]
    for precision, Ac, tau in bad:
        s = B.Solve(n, rank, p=3, q=2, precision=precision, eta=1e-3, seed=1, V0=U, lam0=lam, stream=stream)
        with pytest.raises(B.MegError):
            s.meg_set_objective(B.MEG_BILINEAR, A=Ac, B=Bm, y=y, tau=tau)
        s.meg_destroy()
    # n % 8 != 0
    n2 = 100
    s = B.Solve(n2, 2, p=3, q=2, precision=B.MEG_FP32, eta=1e-3, seed=1,
                V0=np.linalg.qr(np.random.default_rng(1).standard_normal((n2, 2)))[0], lam0=np.array([.5, .5]),
                stream=stream)
    A2 = torch.zeros((16, n2), dtype=torch.int16, device="cuda")
    with pytest.raises(B.MegError):
        s.meg_set_objective(B.MEG_BILINEAR, A=A2, B=A2.clone(), y=torch.zeros(16, dtype=torch.float64,
                                                                              device="cuda"), tau=1.0)
    s.meg_destroy()


def test_rank_p_measurements_match_oracle():
    """Section 7's higher-rank measurements: A_i, B_i in R^{n x p} with
    orthonormal columns (rounded to bf16), r_i = tau Tr(A_i^T X B_i) - y_i.
    The library takes the p columns of A_i (B_i) as p consecutive rows of A
    (B) with mrank = p, and the p pairs of a measurement share its residual.
    n = 96, rank 3, p = 2, m = 20 n r measurements, start eq. (exp:init) as
    printed, 10 iterations against the oracle's exact low-rank MEG.

    The eigenvalue r of M_t lies close to the top of the unwanted spectrum
    relative to how far the library's lower bound of the spectrum (the shift
    estimate of grad f, loose by about 2 sqrt(p) here) lies below it, so
    subspace iteration converges slowly: 32 products per iteration (q = 8
    plus 24 by meg_refine_subspace before each step) reach the tolerances.
    At p = 4 the gap lambda_3 - lambda_4 is about 0.8 against a spread of 50
    under that bound and the iterates are not resolved (one step from the
    same iterate is exact to float rounding: f to 1e-14, sigma_1 to 3e-7)."""
    import torch
    from paper_2012_10469_gb300 import binding as B
    n, rank = 96, 3
    pm = 2
    prob = synth.rank_p_recovery(n, rank, pm, 20 * n * rank, seed=50 + pm)
    As, Bs = synth.bf16_round(prob.As), synth.bf16_round(prob.Bs)
    obj = meg.RankPMeasurements(As, Bs, prob.y, prob.tau)
    m = obj.m
    V0, lam0 = meg.warm_start_at(obj, rank, prob.U, printed_sign=True)
    eta = 1.0 / (prob.tau * 0.4 * math.sqrt(rank * n))

    def rows_of(T):              # row i p + c = column c of T_i
        return torch.from_numpy(np.ascontiguousarray(
            synth.bf16_bits(np.ascontiguousarray(T.transpose(0, 2, 1)).reshape(m * pm, n)).view(np.int16))).cuda()

    A, Bm = rows_of(As), rows_of(Bs)
    bad = B.Solve(n, rank, p=5, q=2, precision=B.MEG_FP32, eta=eta, seed=9, V0=V0, lam0=lam0,
                  stream=torch.cuda.current_stream().cuda_stream)
    with pytest.raises(B.MegError):          # mrank must be a power of two
        bad.meg_set_objective(B.MEG_BILINEAR, A=A, B=Bm, y=torch.from_numpy(obj.y).cuda(), tau=prob.tau, mrank=3)
    bad.meg_destroy()
    s = B.Solve(n, rank, p=5, q=8, precision=B.MEG_FP32, eta=eta, seed=9, V0=V0, lam0=lam0,
                stream=torch.cuda.current_stream().cuda_stream)
    s.meg_set_objective(B.MEG_BILINEAR, A=A, B=Bm, y=torch.from_numpy(obj.y).cuda(), tau=prob.tau, mrank=pm)
    s.meg_refine_subspace(32)
    X = meg.init_X1(V0, lam0, meg.eps_schedule(0))
    f1 = obj.value(X)
    assert abs(s.meg_objective() - f1) <= 1e-7 * f1
    rows = []
    for t in range(1, 11):
        X, info, _ = meg.lowrank_step(X, obj, t, eta, meg.eps_schedule(t), method="exact")
        if t > 1:
            s.meg_refine_subspace(24)
        s.meg_step(1)
        if t in (1, 2, 5, 10):
            Xg = gpu_factored(s)
            sig, _ = s.meg_get_ritz()
            cert, holds, _ = s.meg_certificate()
            rows.append(dict(t=t, Xg=Xg, Xo=X, sig_g=sig, sig_o=info.sig, fg=s.meg_objective(), fo=obj.value(X),
                             f1=f1, fo_at_g=obj.value(Xg), cert_g=cert, holds_g=holds, cert_o=info.cert,
                             holds_o=info.holds, eps=info.eps))
            print(f"rank-{pm} measurements t={t:2d}  X {rel_frob(Xg, X):.2e}")
    s.meg_destroy()
    # sigma to 5e-5: the Ritz values come from float32 work on M_t - c I with the
    # shift c about 25 below sigma_1 here, so their absolute error is about
    # 1e-7 |sigma - c| (2.5e-6 of sigma_3, about -1.3), and sigma_3 is the one
    # the slow convergence above leaves furthest (1.9e-5 at t = 10)
    _check(rows, rank, tol_sig=5e-5, r1_slack=1e-7)
