"""Shared set-up of parity cases: the same seeded inputs for the CUDA path
(through the C ABI binding) and for the oracle."""
from __future__ import annotations

import numpy as np

import synth
from oracle import meg


def to_device_dense(prob, precision):
    import torch
    from paper_2012_10469_gb300 import binding as B
    M = prob.M if hasattr(prob, "M") else prob.C
    if precision == B.MEG_FP64:
        return torch.from_numpy(np.ascontiguousarray(M)).cuda()
    if precision == B.MEG_FP32:
        return torch.from_numpy(np.ascontiguousarray(M.astype(np.float32))).cuda()
    bits = synth.bf16_bits(M).view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(bits)).cuda()


def oracle_objective(kind, prob, seed=0):
    if kind == "dense_quadratic":
        return meg.DenseQuadratic(prob.M)
    if kind == "linear":
        return meg.Linear(prob.C)
    if kind == "completion":
        return meg.Completion(prob.n, prob.rowptr, prob.col, prob.val)
    if kind == "measurements":
        return meg.Measurements(prob.A, prob.y, prob.L, seed=seed)
    raise ValueError(kind)


def make_gpu_solve(kind, prob, r, p, q, precision, eta, seed, V0=None, lam0=None, eigensolver=0):
    """Create a solve through the C ABI and attach the objective."""
    import torch
    from paper_2012_10469_gb300 import binding as B
    s = B.Solve(prob.n, r, p=p, q=q, precision=precision, eta=eta, seed=seed, V0=V0, lam0=lam0,
                stream=torch.cuda.current_stream().cuda_stream, eigensolver=eigensolver)
    if kind in ("dense_quadratic", "linear"):
        s.meg_set_objective(B.MEG_DENSE_QUAD if kind == "dense_quadratic" else B.MEG_LINEAR,
                            dense=to_device_dense(prob, precision))
    elif kind == "completion":
        vt = np.float64 if precision == B.MEG_FP64 else np.float32
        s.meg_set_objective(B.MEG_CSR_QUAD,
                            rowptr=torch.from_numpy(prob.rowptr.astype(np.int32)).cuda(),
                            col=torch.from_numpy(prob.col.astype(np.int32)).cuda(),
                            val=torch.from_numpy(prob.val.astype(vt)).cuda())
    elif kind == "measurements":
        if precision == B.MEG_FP64:
            A = torch.from_numpy(np.ascontiguousarray(prob.A)).cuda()
        else:
            A = torch.from_numpy(np.ascontiguousarray(synth.bf16_bits(prob.A).view(np.int16))).cuda()
        s.meg_set_objective(B.MEG_MEAS_STOCH, A=A, y=torch.from_numpy(prob.y).cuda(), L=prob.L)
    return s


def gpu_factored(s) -> meg.Factored:
    V, mu, sv = s.meg_get_iterate()
    return meg.Factored(V=V, mu=mu, s=sv)


def rel_frob(Xg: meg.Factored, Xo: meg.Factored) -> float:
    return meg.frob_dist(Xg, Xo) / np.sqrt(meg.frob_inner(Xo, Xo))


def run_pair(kind, prob, r, p, q, precision, eta, T, checkpoints, seed=7, method="exact",
             warm=None, eigensolver=0):
    """Run oracle and GPU side by side from the same X_0; return per-checkpoint
    (t, X_gpu, X_oracle, sigma_gpu, sigma_oracle, f_gpu, f_oracle, cert pairs)."""
    obj = oracle_objective(kind, prob, seed=seed)
    if warm is None:
        V0, lam0 = meg.warm_start(obj, r)
    else:
        V0, lam0 = warm
    s = make_gpu_solve(kind, prob, r, p, q, precision, eta, seed, V0=V0, lam0=lam0, eigensolver=eigensolver)
    X = meg.init_X1(V0, lam0, meg.eps_schedule(0))
    f1 = obj.value(X)
    out = []
    W = None
    for t in range(1, T + 1):
        X, info, W = meg.lowrank_step(X, obj, t, eta, meg.eps_schedule(t), method=method,
                                      k=r + p, W0=W)
        s.meg_step(1)
        if t in checkpoints:
            Xg = gpu_factored(s)
            sig, tg = s.meg_get_ritz()
            assert tg == t
            cert, holds, _ = s.meg_certificate()
            fg = s.meg_objective()
            fo = obj.value(X)
            out.append(dict(t=t, Xg=Xg, Xo=X, sig_g=sig, sig_o=info.sig, fg=fg, fo=fo, f1=f1,
                            fo_at_g=obj.value(Xg),
                            cert_g=cert, holds_g=holds, cert_o=info.cert, holds_o=info.holds,
                            eps=info.eps))
    s.meg_destroy()
    return out
