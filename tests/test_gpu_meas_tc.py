"""Minibatch gradient of the measurement objective on the tcgen05 tensor
cores, against the float64 oracle and against the CUDA-core kernels.

Section 6's stochastic first-order oracle: step t's gradient is
(2/L) sum_b r_b a_b a_b^T over L i.i.d. draws.  In float storage with bf16
measurement vectors (rows of A 16-byte aligned) the library applies it as two
tcgen05 contractions (A_B [V | W], then A_B^T S); with A at an address that
is not 16-byte aligned it uses the CUDA-core kernels.  Both must match the
oracle at the parity tolerances, on the same seeded inputs, and each other.
"""
import numpy as np
import pytest

import synth
from oracle import meg

from meg_cases import gpu_factored, oracle_objective, rel_frob
from test_gpu_parity import _check

pytestmark = pytest.mark.gpu


def _solve(prob, r, p, q, precision, eta, seed, V0, lam0, aligned):
    import torch
    from paper_2012_10469_gb300 import binding as B
    bits = synth.bf16_bits(prob.A).view(np.int16).ravel()
    buf = torch.zeros(bits.size + 8, dtype=torch.int16, device="cuda")
    off = 0 if aligned else 1                     # one element = 2 bytes: rows no longer 16-byte aligned
    buf[off:off + bits.size] = torch.from_numpy(bits).cuda()
    A = buf[off:off + bits.size].view(prob.A.shape)
    assert (A.data_ptr() % 16 == 0) == aligned
    s = B.Solve(prob.n, r, p=p, q=q, precision=precision, eta=eta, seed=seed, V0=V0, lam0=lam0,
                stream=torch.cuda.current_stream().cuda_stream)
    s.meg_set_objective(B.MEG_MEAS_STOCH, A=A, y=torch.from_numpy(prob.y).cuda(), L=prob.L)
    s._keep.append(buf)
    return s


def _meas_kernels(s):
    """Minibatch kernels per iteration of a one-member group: 4 on the tensor
    cores (operand split, batch pass, its finish, apply pass) x q, 2 on the
    CUDA cores."""
    import torch
    from paper_2012_10469_gb300 import binding as B
    g = B.Group([s], stream=torch.cuda.current_stream().cuda_stream)
    kps = g.meg_group_kernels_per_step()
    g.meg_group_destroy()
    return kps


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_tensor_core_minibatch_matches_oracle_and_cuda_cores(prec):
    from paper_2012_10469_gb300 import binding as B
    n, r, p, q = 136, 3, 5, 4
    prob = synth.measurements(n, r, 40 * n, 200, seed=81)        # L = 200: a ragged last 128-row tile
    # noisy y (f* > 0): near the planted start f then stays well above its float32
    # floor, where a relative error of f is meaningful
    noise = np.random.default_rng(83).normal(0.0, 0.05, prob.y.shape)
    prob = synth.Measurements(n=prob.n, A=prob.A, y=prob.y + noise, L=prob.L, U=prob.U, w=prob.w)
    eta = 1.0 / (4 * (1 + n / prob.L))
    obj = oracle_objective("measurements", prob, seed=7)
    V0, lam0 = prob.U, prob.w
    tc = _solve(prob, r, p, q, B.PRECISION[prec], eta, 7, V0, lam0, aligned=True)
    cc = _solve(prob, r, p, q, B.PRECISION[prec], eta, 7, V0, lam0, aligned=False)
    assert _meas_kernels(tc) - _meas_kernels(cc) == 2 * q        # two more kernels per product
    X = meg.init_X1(V0, lam0, meg.eps_schedule(0))
    f1 = obj.value(X)
    rows = []
    for t in range(1, 13):
        X, info, _ = meg.lowrank_step(X, obj, t, eta, meg.eps_schedule(t), method="exact")
        tc.meg_step(1)
        cc.meg_step(1)
        if t in (1, 6, 12):
            Xt, Xc = gpu_factored(tc), gpu_factored(cc)
            assert rel_frob(Xt, Xc) <= 2e-6, (t, rel_frob(Xt, Xc))
            sig, tg = tc.meg_get_ritz()
            assert tg == t
            cert, holds, _ = tc.meg_certificate()
            rows.append(dict(t=t, Xg=Xt, Xo=X, sig_g=sig, sig_o=info.sig, fg=tc.meg_objective(), fo=obj.value(X),
                             f1=f1, fo_at_g=obj.value(Xt), cert_g=cert, holds_g=holds, cert_o=info.cert,
                             holds_o=info.holds, eps=info.eps))
    _check(rows, r, r1_slack=1e-7)
    tc.meg_destroy()
    cc.meg_destroy()


def test_tensor_core_warm_start_over_all_measurements():
    """The warm start's pass over all m measurements (m = 3000: many
    128-row tiles, the apply pass over several batch chunks) on the tensor
    cores gives the oracle's eq. (exp:init) start."""
    from paper_2012_10469_gb300 import binding as B
    n, r = 160, 3
    prob = synth.measurements(n, r, 3000, 64, seed=82)
    obj = oracle_objective("measurements", prob, seed=3)
    V0, lam0 = meg.warm_start(obj, r)
    X1 = meg.init_X1(V0, lam0, meg.eps_schedule(0))
    s = _solve(prob, r, 5, 2, B.MEG_FP32, 1.0 / (4 * (1 + n / 64)), 3, None, None, aligned=True)
    s.meg_warm_start(600)
    Xg = gpu_factored(s)
    assert rel_frob(Xg, X1) <= 1e-5, rel_frob(Xg, X1)
    s.meg_destroy()
