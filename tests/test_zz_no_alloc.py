"""meg_objective_dense_noalloc (for callers that cannot allocate device
memory: graph-capture contexts, fixed-budget serving loops, hosts that
manage device memory themselves) must give meg_objective's result for the
same iterate and data, through the C ABI, on two calls in a row -- the
second call reuses the library's fixed scratch array left by the first."""
import ctypes

import numpy as np
import pytest

import synth
from oracle import meg

from meg_cases import make_gpu_solve

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-7), ("bf16", 1e-7)])
def test_noalloc_objective_matches_meg_objective(prec, tol):
    import torch
    from paper_2012_10469_gb300 import binding as B
    lib = B.load()
    storage = {"fp64": "f64", "fp32": "f32", "bf16": "bf16"}[prec]
    prob = synth.dense_quadratic(300, 4, seed=71, sigma=1e-4, storage=storage)
    V0, lam0 = meg.warm_start(meg.DenseQuadratic(prob.M), 4)
    s = make_gpu_solve("dense_quadratic", prob, 4, 3, 2, B.PRECISION[prec], 1.0, 5, V0=V0, lam0=lam0)
    s.meg_step(6)
    f_ref = s.meg_objective()
    V, mu, sv = s.meg_get_iterate()
    dense = s._keep[0]                       # the objective's device data
    Vd = torch.from_numpy(V).cuda()
    out = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    mu_c = np.ascontiguousarray(mu)
    for _ in range(2):
        out.fill_(-1.0)
        st = lib.meg_objective_dense_noalloc(Vd.data_ptr(), mu_c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             sv, prob.n, 4, dense.data_ptr(), B.PRECISION[prec],
                                             out.data_ptr(), stream)
        assert st == B.MEG_OK, B.meg_last_error()
        torch.cuda.synchronize()
        f = float(out.item())
        assert abs(f - f_ref) <= tol * abs(f_ref), (f, f_ref)
    s.meg_destroy()


def test_noalloc_rejects_sizes_beyond_the_scratch():
    from paper_2012_10469_gb300 import binding as B
    lib = B.load()
    mu = (ctypes.c_double * 2)(0.5, 0.5)
    st = lib.meg_objective_dense_noalloc(16, mu, 0.0, B_MAX_N() + 1, 2, 16, 0, 16, None)
    assert st == B.MEG_ERR_INVALID_ARG
    assert "MEG_NOALLOC_MAX_N" in B.meg_last_error()


def B_MAX_N():
    import os
    import re
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "meg.h")
    return int(re.search(r"#define MEG_NOALLOC_MAX_N (\d+)", open(hdr).read()).group(1))
