"""Benchmark of the low-rank MEG iteration (Algorithm 2) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Workload (dense quadratic recipe with n = 4096, r = 10): f(X) = 1/2||X - M||_F^2
with M = U diag(w) U^T + E, w ~ Dirichlet(1), E symmetric N(0, 1e-5^2),
data stored in bfloat16.  One step = one MEG iteration (gradient product,
mirror operator, subspace iteration with CholeskyQR2, Rayleigh-Ritz,
exp-map, certificate) for a batch of B = 8 independent instances stepped
together by grouped kernels; the batch's data (268 MB) is larger than L2,
so no step re-reads data from L2.  value = instance-iterations per second
over all ranks.  Under torchrun every rank runs its own batch (weak
scaling, no data-path collective).

--impl reference times the CPU float64 oracle on the same workload (a
bounded sample of iterations, on the host cores).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MEG iters/s at n=4096 and solves/s p50/p99 vs plain FP32 GPU form at 1e-6 gap"
N, R = 4096, 10
P, Q, EIG = 6, 3, 0  # extra subspace vectors, products per iteration, eigensolver: set by meg_autotune
AUTOTUNE = dict(q_max=4, p_cand=(2, 4, 6, 8, 12, 16), pilot_iters=20, horizon=500, tol_x=1e-5, krylov=True)
EIG_NAME = {0: "subspace iteration", 1: "block Krylov"}
BATCH = 8
SEED0 = 1001


def bf16_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"])
    return 1900.0


BF16_TFLOPS = None


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d["hbm_gbs"], "measured"
    return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, device) -> float:
    """The largest value over all ranks (the slowest rank's time); the value
    itself when not distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- workload
def make_batch(batch: int, seed0: int):
    import synth
    return [synth.dense_quadratic(N, R, seed=seed0 + i, sigma=1e-5, storage="bf16") for i in range(batch)]


def autotune_pq(prob, device, stream):
    """meg_autotune on one instance of the batch: the cheapest (eigensolver, p,
    q) whose iterate stays within 1e-5 of a more resolved reference over 500
    iterations."""
    import torch
    from paper_2012_10469_gb300 import binding as B
    global P, Q, EIG
    bits = torch.from_numpy(np.ascontiguousarray(prob.bits().view(np.int16))).to(device)
    p, q, err, ok, eig = B.meg_autotune(N, R, B.MEG_MIXED_BF16, B.MEG_DENSE_QUAD, prob.U, prob.w, dense=bits,
                                        seed=SEED0, stream=stream, **AUTOTUNE)
    P, Q, EIG = p, q, eig
    return {"p": p, "q": q, "eigensolver": EIG_NAME[eig], "pilot_distance": err, "met_target": ok,
            **{k: v for k, v in AUTOTUNE.items()}}


def gpu_solves(probs, device, stream):
    """Create the batch's solves through the C ABI, X_0 = each instance's planted point."""
    import torch
    from paper_2012_10469_gb300 import binding as B
    solves, dense = [], []
    for i, prob in enumerate(probs):
        bits = torch.from_numpy(np.ascontiguousarray(prob.bits().view(np.int16))).to(device)
        s = B.Solve(N, R, p=P, q=Q, precision=B.MEG_MIXED_BF16, eta=1.0, seed=SEED0 + i, stream=stream,
                    V0=prob.U, lam0=prob.w, eigensolver=EIG)
        s.meg_set_objective(B.MEG_DENSE_QUAD, dense=bits)
        solves.append(s)
        dense.append(bits)
    return solves, dense


# DRAM bytes (read + write) of one k_dense_tc launch on this workload, from one
# ncu capture of it (dram__bytes_read.sum + dram__bytes_write.sum; the summary
# is kept with the other ncu summaries).  None whenever the kernel has changed
# since that capture.
DENSE_TC_TRAFFIC_BYTES = 273.977600e6 + 3.698944e6


def algorithmic_bytes_dense_product():
    """Minimum HBM traffic of one grouped dense product Y = M W over the batch:
    M once (n^2 bf16) + W read + Y written (n k float32 each)."""
    k = R + P
    return BATCH * (N * N * 2 + 2 * N * k * 4)


# --------------------------------------------------------------------------- CPU baseline (oracle)
ERR_CHECKPOINTS = (1, 10, 100, 200)


def oracle_sample(seconds: float, record: dict = None):
    """Time the float64 oracle's low-rank MEG iterations (subspace-iteration
    eigensolver) on one instance of the workload, for about `seconds` (at most
    200 iterations).  `record` (a dict) receives the oracle's iterate and
    Ritz values at the checkpoints reached, for the error report."""
    import synth
    from oracle import meg
    prob = synth.dense_quadratic(N, R, seed=SEED0, sigma=1e-5, storage="bf16")
    obj = meg.DenseQuadratic(prob.M)
    # warm start from the planted factors: the sample times iterations, not the start-up
    X = meg.init_X1(prob.U, prob.w, meg.eps_schedule(0))
    W = None
    iters, t0 = 0, time.perf_counter()
    while True:
        X, info, W = meg.lowrank_step(X, obj, iters + 1, 1.0, meg.eps_schedule(iters + 1), method="subspace",
                                      k=R + P, W0=W)
        iters += 1
        if record is not None and iters in ERR_CHECKPOINTS:
            record[iters] = ((X.V.copy(), X.mu.copy(), float(X.s)), info.sig[:R].copy())
        el = time.perf_counter() - t0
        if el >= seconds or iters >= 200:
            break
    try:
        from threadpoolctl import threadpool_info
        cores = max([d.get("num_threads", 1) for d in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count() or 1
    return iters / el, cores, iters, el


def mode_errors(device, stream, record: dict):
    """Error of each precision mode against the float64 oracle on the
    oracle-sample instance (seed 1001): the GPU solve runs the same
    iterations through the C ABI in MEG_FP64 (subspace iteration, q = 3),
    MEG_FP32 (float32 data, the benchmark's eigensolver, p and q) and
    MEG_MIXED_BF16 (the benchmarked mode); relative Frobenius error of X_t,
    largest relative error of sigma_1..r and relative error of f(X_t) at each
    checkpoint the oracle sample reached."""
    import torch
    import synth
    from paper_2012_10469_gb300 import binding as B
    prob = synth.dense_quadratic(N, R, seed=SEED0, sigma=1e-5, storage="bf16")

    def dense(V, mu, sv):                 # X = V diag(mu - s) V^T + s I
        X = (V * (mu - sv)) @ V.T
        X[np.diag_indices_from(X)] += sv
        return X

    def fval(X):
        D = X - prob.M
        return 0.5 * float(np.sum(D * D))

    out = {}
    modes = (("fp64", B.MEG_FP64, 3, 0, np.float64), ("fp32", B.MEG_FP32, Q, EIG, np.float32),
             ("bf16", B.MEG_MIXED_BF16, Q, EIG, None))
    for name, prec, q, eig, dt in modes:
        if dt is None:
            data = torch.from_numpy(np.ascontiguousarray(prob.bits().view(np.int16))).to(device)
        else:
            data = torch.from_numpy(np.ascontiguousarray(prob.M.astype(dt))).to(device)
        s = B.Solve(N, R, p=P, q=q, precision=prec, eta=1.0, seed=SEED0, stream=stream, V0=prob.U, lam0=prob.w,
                    eigensolver=eig)
        s.meg_set_objective(B.MEG_DENSE_QUAD, dense=data)
        rows, t = {}, 0
        for cp in sorted(record):
            s.meg_step(cp - t)
            t = cp
            Xg = dense(*s.meg_get_iterate())
            (Vo, muo, so_), sig_o = record[cp]
            Xo = dense(Vo, muo, so_)
            sig, _ = s.meg_get_ritz()
            fo = fval(Xo)
            rows[str(cp)] = {"x": float(np.linalg.norm(Xg - Xo) / np.linalg.norm(Xo)),
                             "sigma": float(np.max(np.abs(sig[:R] - sig_o) / np.abs(sig_o))),
                             "f": abs(fval(Xg) - fo) / abs(fo)}
        s.meg_destroy()
        out[name] = {"eigensolver": EIG_NAME[eig], "q": q, "p": P, "checkpoints": rows}
    out["what"] = ("relative Frobenius error of X_t, max relative error of sigma_1..r, relative error of f(X_t), "
                   "against the float64 oracle (subspace eigensolver to a 1e-12 residual), n=4096 seed 1001")
    return out


# --------------------------------------------------------------------------- plain FP32 torch form
def torch_fp32_form(prob, device, iters: int):
    """The same iteration with plain float32 torch ops (cuBLAS/cuSOLVER), one
    solve at a time, no graphs, no batching: the comparator the metric names."""
    import torch
    M = torch.from_numpy(prob.M.astype(np.float32)).to(device)
    k = R + P
    g = torch.Generator(device="cpu").manual_seed(7)
    V = torch.from_numpy(prob.U.astype(np.float32)).to(device)
    eps0 = 0.8 / 121.0
    mu = torch.tensor(prob.w, dtype=torch.float32, device=device) * (1 - eps0) + eps0 / N
    s = eps0 / N
    W, _ = torch.linalg.qr(torch.cat([V, torch.randn(N, P, generator=g).to(device)], 1))
    torch.linalg.eigh(W.T @ W)          # load cuSOLVER before timing
    # the library's shift bound: 1.25 sqrt(2 f) with f from the factors
    frod2 = float((M.double() ** 2).sum())
    trm = float(torch.trace(M.double()))
    X0 = (V * (mu - s)) @ V.T
    f0 = 0.5 * float(((X0 + s * torch.eye(N, device=device) - M) ** 2).sum())
    gnorm = 1.25 * math.sqrt(2.0 * max(f0, 0.0))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for t in range(1, iters + 1):
        eps = 0.8 / (t + 11.0) ** 2
        logs = math.log(s)
        d = torch.log(mu) - logs - (mu - s)
        c0 = logs - s
        shift = min(logs, float(torch.log(mu).min())) - gnorm
        if EIG == 1:
            # block Krylov: Rayleigh-Ritz on [W, orth(A W - W (W^T A W))], next block = top-k Ritz vectors
            Y1 = M @ W
            Z1 = V @ (d[:, None] * (V.T @ W)) + (c0 - shift) * W + Y1
            Zp = Z1 - W @ (W.T @ Z1)
            Zp = Zp - W @ (W.T @ Zp)        # second Gram-Schmidt pass: Zp is small, the first leaves u |Z1| along W
            W1, _ = torch.linalg.qr(Zp)
            Y2 = M @ W1
            Z2 = V @ (d[:, None] * (V.T @ W1)) + (c0 - shift) * W1 + Y2
            Bk = torch.cat([W, W1], 1)
            H = Bk.T @ torch.cat([Z1, Z2], 1)
            th, Qm = torch.linalg.eigh(0.5 * (H + H.T))
            th, Qm = th.flip(0), Qm.flip(1)
            sig = th + shift
            mu = (1 - eps) * torch.exp(sig[:R] - torch.logsumexp(sig[:R], 0))
            s = eps / (N - R)
            pdg = torch.einsum("ai,ab,bi->i", Qm[:, :R], Bk.T @ torch.cat([Y1, Y2], 1), Qm[:, :R])
            xd = float(((mu - s) * pdg).sum()) + s * trm
            x2 = float((mu * mu).sum()) + (N - R) * s * s
            gnorm = 1.25 * math.sqrt(2.0 * max(0.5 * x2 - xd + 0.5 * frod2, 0.0))
            V = Bk @ Qm[:, :R]
            W = Bk @ Qm[:, :k]
            continue
        for j in range(Q):
            Y = M @ W
            Z = V @ (d[:, None] * (V.T @ W)) + (c0 - shift) * W + Y
            if j < Q - 1:
                W, _ = torch.linalg.qr(Z)
        H = W.T @ Z
        th, Qm = torch.linalg.eigh(0.5 * (H + H.T))
        th, Qm = th.flip(0), Qm.flip(1)
        sig = th + shift
        lse = torch.logsumexp(sig[:R], 0)
        mu = (1 - eps) * torch.exp(sig[:R] - lse)
        s = eps / (N - R)
        # f(X_{t+1}) from the factors: v_i^T M v_i = (Q^T W^T Y Q)_ii
        pdg = torch.einsum("ai,ab,bi->i", Qm[:, :R], W.T @ Y, Qm[:, :R])
        xd = float(((mu - s) * pdg).sum()) + s * trm
        x2 = float((mu * mu).sum()) + (N - R) * s * s
        gnorm = 1.25 * math.sqrt(2.0 * max(0.5 * x2 - xd + 0.5 * frod2, 0.0))
        V = W @ Qm[:, :R]
        W, _ = torch.linalg.qr(Z @ Qm)
    e1.record()
    torch.cuda.synchronize()
    return iters / (e0.elapsed_time(e1) / 1e3)


# --------------------------------------------------------------------------- serving
SERVE_P, SERVE_Q, SERVE_TOL, SERVE_MAX_ITERS = 4, 2, 1e-6, 5000


def serve_request_args(B, q):
    """Server request for one trace entry (config-0 type: float32 dense data, f*
    unknown, plateau rule; config-3 type: bf16 measurements, f* = 0)."""
    common = dict(n=q.n, r=q.r, p=SERVE_P, q=SERVE_Q, seed=17 + q.n, warm_start_products=40,
                  tol=SERVE_TOL, max_iters=SERVE_MAX_ITERS)
    if q.kind == 0:
        return dict(kind=B.MEG_DENSE_QUAD, data=q.M32, precision=B.MEG_FP32, eta=1.0, **common)
    return dict(kind=B.MEG_MEAS_STOCH, data=q.A_bits, y=q.y, L=q.L, precision=B.MEG_MIXED_BF16,
                eta=1.0 / (4.0 * (1.0 + q.n / q.L)), fstar=0.0, **common)


def run_serving(trace, budget_bytes: int, max_active: int = 1024):
    """Replay the trace's Poisson arrivals into meg_server; returns the summary."""
    import threading
    from paper_2012_10469_gb300 import binding as B
    srv = B.Server(budget_bytes, max_active=max_active, check_every=10, meas_check_every=250)
    results, errors = [], []
    kind_of, index_of = {}, {}         # request id -> 0 (dense quadratic) or 1 (measurements); trace index

    def submitter():
        try:
            base = srv.meg_server_now()
            for j, q in enumerate(trace):
                delay = base + q.t - srv.meg_server_now()
                if delay > 0:
                    time.sleep(delay)
                rid = srv.meg_server_submit(**serve_request_args(B, q))
                kind_of[rid], index_of[rid] = q.kind, j
        except Exception as ex:  # surfaced below
            errors.append(ex)

    th = threading.Thread(target=submitter)
    th.start()
    deadline = time.time() + 900
    while len(results) < len(trace) and time.time() < deadline and not errors:
        for rec, _V, _mu, _s in srv.meg_server_poll(max_out=512, timeout_ms=20):
            results.append(rec)
    th.join()
    ticks, graph_ticks = srv.meg_server_tick_counts()
    srv.meg_server_destroy()
    if errors:
        raise errors[0]
    lat = np.array([r["t_done"] - r["t_submit"] for r in results])
    t_first = min(r["t_submit"] for r in results)
    t_last = max(r["t_done"] for r in results)
    st = [r["status"] for r in results]
    its = np.array([r["iters"] for r in results])
    return {
        "requests": len(trace), "finished": len(results),
        "solves_per_s": len(results) / (t_last - t_first),
        "latency_p50_ms": 1e3 * float(np.percentile(lat, 50)),
        "latency_p99_ms": 1e3 * float(np.percentile(lat, 99)),
        "iters_p50": float(np.percentile(its, 50)), "iters_p99": float(np.percentile(its, 99)),
        "converged": int(sum(1 for x in st if x == 0)),
        "hit_max_iters": int(sum(1 for x in st if x == 5)),
        "failed": int(sum(1 for x in st if x not in (0, 5))),
        "makespan_s": t_last - t_first,
        "ticks": ticks, "graph_ticks": graph_ticks,
        "service_by_index": {index_of[r["id"]]: r["t_done"] - r["t_admit"] for r in results},
        "per_class": {name: serving_class_stats([r for r in results if kind_of.get(r["id"]) == kind])
                      for kind, name in ((0, "dense_quadratic"), (1, "measurements"))},
    }


def serving_class_stats(results):
    """Service time (admission to result) and queueing (submission to admission)
    percentiles, iterations and outcome counts of one request class."""
    if not results:
        return {"requests": 0}
    svc = np.array([r["t_done"] - r["t_admit"] for r in results])
    que = np.array([r["t_admit"] - r["t_submit"] for r in results])
    its = np.array([r["iters"] for r in results])
    st = [r["status"] for r in results]
    pct = lambda a, q: float(np.percentile(a, q))
    return {"requests": len(results),
            "service_p50_ms": 1e3 * pct(svc, 50), "service_p99_ms": 1e3 * pct(svc, 99),
            "queue_p50_ms": 1e3 * pct(que, 50), "queue_p99_ms": 1e3 * pct(que, 99),
            "iters_p50": pct(its, 50), "iters_p99": pct(its, 99),
            "converged": int(sum(1 for x in st if x == 0)),
            "hit_max_iters": int(sum(1 for x in st if x == 5)),
            "failed": int(sum(1 for x in st if x not in (0, 5)))}


def torch_fp32_solve(q, device, max_iters=SERVE_MAX_ITERS, tol=SERVE_TOL):
    """One serving request with plain float32 torch ops (cuBLAS/cuSOLVER), the
    same algorithm, warm start and stopping rule, no batching, no graphs."""
    import torch
    n, r, k = q.n, q.r, q.r + SERVE_P
    gen = torch.Generator(device="cpu").manual_seed(q.n)
    dense = q.kind == 0
    if dense:
        M = torch.from_numpy(q.M32).to(device)
        G0 = M
        eta, check = 1.0, 10
    else:
        A = torch.from_numpy(q.A.astype(np.float32)).to(device)
        y = torch.from_numpy(q.y.astype(np.float32)).to(device)
        G0 = (2.0 / A.shape[0]) * (A.T @ (y[:, None] * A))
        eta, check = 1.0 / (4.0 * (1.0 + n / q.L)), 50
    lam, U = torch.linalg.eigh(0.5 * (G0 + G0.T))
    lam, V = lam.flip(0)[:r], U.flip(1)[:, :r]
    srt, _ = torch.sort(lam, descending=True)           # simplex projection of lam
    css = torch.cumsum(srt, 0) - 1.0
    ind = torch.arange(1, r + 1, device=device, dtype=torch.float32)
    rho = int(torch.nonzero(srt - css / ind > 0).max()) + 1
    lam = torch.clamp(lam - css[rho - 1] / rho, min=0.0)
    eps0 = 0.8 / 121.0
    mu = (1 - eps0) * lam + eps0 / n
    s = eps0 / n

    def fval(V, mu, s):
        if dense:
            X = (V * (mu - s)) @ V.T + s * torch.eye(n, device=device)
            return 0.5 * float(((X - M) ** 2).sum())
        P = A @ V
        qv = (P * P) @ (mu - s) + s * (A * A).sum(1)
        return float(((qv - y) ** 2).mean())

    def grad_apply(V, mu, s, W):
        if dense:
            return V @ ((mu - s)[:, None] * (V.T @ W)) + s * W - M @ W, None
        idx = torch.randint(0, A.shape[0], (q.L,), device=device)
        Ab = A[idx]
        P = Ab @ V
        res = (P * P) @ (mu - s) + s * (Ab * Ab).sum(1) - y[idx]
        return (2.0 / q.L) * (Ab.T @ (res[:, None] * (Ab @ W))), res

    f1 = fval(V, mu, s)
    f_prev, f = f1, f1
    W, _ = torch.linalg.qr(torch.cat([V, torch.randn(n, SERVE_P, generator=gen).to(device)], 1))
    gb = 1.25 * math.sqrt(2 * f1) if dense else 1.0
    it = 0
    while it < max_iters:
        for _ in range(check):
            it += 1
            eps = 0.8 / (it + 11.0) ** 2
            logs = math.log(s)
            dlog = torch.log(mu) - logs
            shift = min(logs, float(torch.log(mu).min())) - eta * gb
            for j in range(SERVE_Q):
                GW, res = grad_apply(V, mu, s, W)
                Z = V @ (dlog[:, None] * (V.T @ W)) + (logs - shift) * W - eta * GW
                if j < SERVE_Q - 1:
                    W, _ = torch.linalg.qr(Z)
            if res is not None:
                gb = float((2.0 / q.L) * res.abs().max() * (A[:1] * A[:1]).sum() * (1 + math.sqrt(q.L / n)) ** 2)
            H = W.T @ Z
            th, Qm = torch.linalg.eigh(0.5 * (H + H.T))
            th, Qm = th.flip(0), Qm.flip(1)
            sig = th + shift
            mu = (1 - eps) * torch.exp(sig[:r] - torch.logsumexp(sig[:r], 0))
            s = eps / (n - r)
            V = W @ Qm[:, :r]
            W, _ = torch.linalg.qr(Z @ Qm)
            if it >= max_iters:
                break
        f_prev, f = f, fval(V, mu, s)
        if dense:
            gb = 1.25 * math.sqrt(2 * max(f, 0.0))
            if f1 - f > 0 and f_prev - f <= tol * (f1 - f):
                return it, True
        elif f <= tol * f1:
            return it, True
    return it, False


def torch_fp32_serve_sample(trace, device, seconds: float, count: int = 50, gpu_service=None):
    """The plain float32 form on `count` requests spread evenly over the trace
    (every len/count-th arrival, both classes in their trace proportions), one
    at a time, for at most about `seconds`; latency from a FIFO replay of
    those arrivals with the measured service times; beside it the serving
    loop's own service times of the same requests."""
    import torch
    torch_fp32_solve(trace[0], device, max_iters=20)        # load cuBLAS/cuSOLVER
    torch.cuda.synchronize()
    pick = list(range(0, len(trace), max(1, len(trace) // count)))[:count]
    serv, its, kinds, t_all = [], [], [], time.perf_counter()
    for j in pick:
        t0 = time.perf_counter()
        it, _ok = torch_fp32_solve(trace[j], device)
        torch.cuda.synchronize()
        serv.append(time.perf_counter() - t0)
        its.append(it)
        kinds.append(trace[j].kind)
        if time.perf_counter() - t_all > seconds:
            break
    done, lat = 0.0, []
    for j, sv in zip(pick, serv):
        done = max(done, trace[j].t) + sv
        lat.append(done - trace[j].t)
    out = {"requests": len(serv), "requests_dense": kinds.count(0), "requests_measurements": kinds.count(1),
           "solves_per_s": len(serv) / sum(serv),
           "service_p50_ms": 1e3 * float(np.percentile(serv, 50)),
           "service_p99_ms": 1e3 * float(np.percentile(serv, 99)),
           "latency_p50_ms": 1e3 * float(np.percentile(lat, 50)),
           "latency_p99_ms": 1e3 * float(np.percentile(lat, 99)),
           "iters_p50": float(np.percentile(its, 50)),
           "what": "same algorithm and stopping rule in plain float32 torch ops, one request at a time "
                   "(FIFO replay of the same arrivals for latency), on requests spread over the trace"}
    if gpu_service:
        same = [gpu_service[j] for j in pick[:len(serv)] if j in gpu_service]
        if same:
            out["serving_loop_service_p50_ms_same_requests"] = 1e3 * float(np.percentile(same, 50))
            out["service_ratio_p50"] = float(np.percentile(serv, 50)) / float(np.percentile(same, 50))
    return out


# --------------------------------------------------------------------------- main
def run_reference(args):
    """The oracle on the workload: each step is one float64 low-rank MEG
    iteration of one instance (subspace-iteration eigensolver), on the host
    cores; capped at about 150 s of stepping."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import synth
    from oracle import meg
    prob = synth.dense_quadratic(N, R, seed=SEED0, sigma=1e-5, storage="bf16")
    obj = meg.DenseQuadratic(prob.M)
    X = meg.init_X1(prob.U, prob.w, meg.eps_schedule(0))
    W = None
    t = 0
    for _ in range(args.warmup):
        t += 1
        X, _, W = meg.lowrank_step(X, obj, t, 1.0, meg.eps_schedule(t), method="subspace", k=R + P, W0=W)
    done, t0 = 0, time.perf_counter()
    while done < args.steps and time.perf_counter() - t0 < 150.0:
        t += 1
        X, _, W = meg.lowrank_step(X, obj, t, 1.0, meg.eps_schedule(t), method="subspace", k=R + P, W0=W)
        done += 1
    el = time.perf_counter() - t0
    value = done / el
    try:
        from threadpoolctl import threadpool_info
        cores = max([d.get("num_threads", 1) for d in threadpool_info()] + [1])
    except Exception:
        cores = os.cpu_count() or 1
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": args.gpus,
            "steps": done, "warmup": args.warmup, "ms_per_step": 1e3 * el / done,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"dense quadratic n={N} r={R}, one instance, oracle subspace-iteration "
                                   f"eigensolver in float64", "global_batch": 1},
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": cores, "kind": "oracle",
                             "sample": f"{done} of {args.steps} requested iterations (150 s cap)"},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    from paper_2012_10469_gb300 import binding as B

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    B.load()
    stream = torch.cuda.Stream(device)
    probs = make_batch(BATCH, SEED0 + 100 * rank)
    with torch.cuda.stream(stream):
        tuned = autotune_pq(probs[0], device, stream.cuda_stream)
        solves, dense = gpu_solves(probs, device, stream.cuda_stream)
    group = B.Group(solves, stream=stream.cuda_stream)
    kps = group.meg_group_kernels_per_step()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    group.meg_group_step(max(3, args.warmup))
    stream.synchronize()
    # ---- timed region: K iterations of the whole batch, device-resident inputs
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        # the sampler reads the clocks every 200 ms: the same iterations run for
        # about 2 s (untimed, the warm state continues) so that it sees this load,
        # then the timed region follows inside the same sampling window
        t_soak = time.perf_counter()
        while time.perf_counter() - t_soak < 2.0:
            group.meg_group_step(200)
            stream.synchronize()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("meg_timed")
        e0.record(stream)
        group.meg_group_step(args.steps)
        e1.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    barrier()
    ms = e0.elapsed_time(e1)
    clocks = clk.summary()
    clocks["window"] = "2 s of the same grouped iterations directly before the timed region, and the timed region"

    ms = max_over_ranks(ms, device)
    value = ws * BATCH * args.steps / (ms / 1e3)

    # ---- dominant kernel: grouped dense product, timed alone with CUDA events
    prod_ms = group.meg_group_time_product(20)
    # ---- the kernels after an intermediate product, each timed alone (warm)
    chain_us = group.meg_group_time_chain(20)
    hbm_peak, peak_kind = peaks()
    global BF16_TFLOPS
    BF16_TFLOPS = bf16_peak()
    alg = algorithmic_bytes_dense_product()
    achieved = alg / (prod_ms / 1e3) / 1e9

    # ---- end to end through the public API: each step uploads the batch's
    # data from pinned host memory, runs the iteration, reads back each
    # solve's certificate and Ritz values
    pinned = [torch.from_numpy(np.ascontiguousarray(p.bits().view(np.int16))).pin_memory() for p in probs]
    e2e_steps = max(3, min(args.steps, 50))
    h2d = sum(p.numel() * 2 for p in pinned)
    d2h = BATCH * (8 * 3 + 8 * (R + P) + 4)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        with torch.cuda.stream(stream):
            for dd, pp in zip(dense, pinned):
                dd.copy_(pp, non_blocking=True)
        group.meg_group_step(1)
        for s_ in solves:
            s_.meg_certificate()
            s_.meg_get_ritz()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_value = ws * BATCH * e2e_steps / e2e_s

    line = None
    if rank == 0:
        try:
            torch_fp32_form(probs[0], device, 2)
            fp32_form = {"value": torch_fp32_form(probs[0], device, 30), "unit": "iters/s",
                         "what": "same iteration (eigensolver, p, q, shift bound) in plain float32 torch ops, one "
                                 "solve, no graphs"}
        except Exception as ex:  # reported, never fatal
            fp32_form = {"error": repr(ex)[:200]}
        single = None
        try:
            single = single_solve_rate(probs[0], device)
        except Exception as ex:  # reported, never fatal
            single = {"error": repr(ex)}
        try:
            others = other_kernel_rooflines(device, stream.cuda_stream, hbm_peak)
        except Exception as ex:  # reported, never fatal
            others = {"error": repr(ex)[:300]}
        record = {}
        cpu_rate, cores, it, el = oracle_sample(args.cpu_seconds, record)
        try:
            errors = mode_errors(device, stream.cuda_stream, record)
        except Exception as ex:  # reported, never fatal
            errors = {"error": repr(ex)[:300]}
        try:
            fp32_arm = fp32_data_arm(device, stream.cuda_stream, hbm_peak, args.steps)
        except Exception as ex:  # reported, never fatal
            fp32_arm = {"error": repr(ex)[:300]}
        serving = None
        if args.serve_requests > 0:
            try:
                import synth
                trace = synth.serving_trace(args.serve_requests, args.serve_rate, 2000)
                free, _tot = torch.cuda.mem_get_info()
                serving = run_serving(trace, budget_bytes=int(free * 0.6))
                serving["arrival_rate_per_s"] = args.serve_rate
                serving["workload"] = ("Poisson arrivals, n log-uniform [64, 1024], r uniform 1..8, 50/50 "
                                       "dense quadratic (float32 data, noise 1e-4, plateau rule) / measurements "
                                       "(bf16 A, m=50000, L=256, f*=0), tol 1e-6, max_iters 5000, p=4, q=2, objective checked every "
                                       "10 (dense) / 250 (measurements) iterations")
                serving["plain_fp32_form"] = torch_fp32_serve_sample(
                    trace, device, args.serve_fp32_seconds, gpu_service=serving.pop("service_by_index", None))
            except Exception as ex:  # reported, never fatal
                serving = {"error": repr(ex)[:300]}
        line = {
            "metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"dense quadratic n={N} r={R} k={R + P} q={Q} ({EIG_NAME[EIG]} eigensolver), "
                                   f"{BATCH} independent instances per step (grouped kernels, CUDA graph), bf16 data, "
                                   f"tcgen05 product, float32 subspace blocks (CholeskyQR with a factor refined in Gram "
                                   f"space), float32 k x k island with double-word refinement, X_0 = planted point",
                       "autotune": tuned,
                       "global_batch": ws * BATCH, "l2": "inputs larger than L2 (268 MB bf16 per rank)",
                       "parallelism": f"replicas x{ws}"},
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": "iters/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "what": "per step: the batch's bf16 data copied from pinned host memory into the device tensors "
                            "the solves borrow (torch copy_ on the solves' stream), one meg_group_step, then "
                            "meg_certificate and meg_get_ritz of every solve (host read-back)"},
            "errors": errors,
            "fp32_data_arm": fp32_arm,
            "gpu_launches": kps * args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": DENSE_TC_TRAFFIC_BYTES,
                         "kernel": "grouped dense product k_dense_tc (bf16 tcgen05, TMA)",
                         "peak_kind": f"{peak_kind} burst copy bandwidth", "ms_per_launch": prod_ms,
                         "bytes_per_launch": alg},
            "cpu_baseline": {"value": cpu_rate, "unit": "iters/s", "cores": cores, "kind": "oracle",
                             "sample": f"{it} oracle iterations (float64, subspace eigensolver) of one "
                                       f"n={N} instance in {el:.1f} s"},
            "chain_us": {"what": "warm microseconds per launch of the kernels after an intermediate product, "
                                 "each timed alone (back-to-back launches), all 8 solves; one CholeskyQR pass "
                                 "(float storage)",
                         **{name: round(v, 2) for name, v in
                            zip(("combine", "factor", "orth", "factor_2", "orth_2", "reduce_U_G"), chain_us)
                            if v > 0}},
            "fp32_torch_form": fp32_form,
            "single_solve": single,
            "other_kernels": others,
            "serving": serving,
        }
    group.meg_group_destroy()
    for s_ in solves:
        s_.meg_destroy()
    if line is not None:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def other_kernel_rooflines(device, stream, hbm_peak):
    """Gradient-product kernels of the other workloads at their full sizes, each
    timed alone (CUDA events around back-to-back launches, warm):
      * n = 20000 matrix completion (1% of the upper triangle, mirrored): the
        fused SDDMM + SpMM pass reads each stored entry's column index and
        value once (8 bytes); the rows of V and W it gathers (n (r + k) words)
        stay in L2;
      * n = 2048 stochastic measurements (m = 50000, L = 256): the implicit
        minibatch product A_B^T (r o (A_B W)) reads the L gathered rows of A
        (bf16) twice, 4 L n k flops; the explicit SYRK form would be n(n+1)L."""
    import torch
    import synth
    from paper_2012_10469_gb300 import binding as B
    out = {}
    prob = synth.config(2)
    nnz = int(len(prob.col))
    s = B.Solve(prob.n, 8, p=8, q=6, precision=B.MEG_FP32, seed=1002, stream=stream, V0=prob.U, lam0=prob.w)
    rp = torch.from_numpy(prob.rowptr.astype(np.int32)).to(device)
    cl = torch.from_numpy(prob.col.astype(np.int32)).to(device)
    vl = torch.from_numpy(prob.val.astype(np.float32)).to(device)
    s.meg_set_objective(B.MEG_CSR_QUAD, rowptr=rp, col=cl, val=vl)
    g = B.Group([s], stream=stream)
    ms = g.meg_group_time_product(50)
    alg = nnz * 8 + (prob.n + 1) * 4
    out["csr_product_n20000"] = {"bound": "hbm", "ms_per_launch": ms, "bytes_per_launch": alg,
                                 "achieved_GBs": alg / (ms / 1e3) / 1e9,
                                 "frac": alg / (ms / 1e3) / 1e9 / hbm_peak, "nnz": nnz}
    g.meg_group_destroy()
    s.meg_destroy()
    out["minibatch_product_n2048"] = minibatch_timing(device, stream)
    out["bilinear_n600_r20"] = bilinear_timing(device, stream, hbm_peak)
    return out


def minibatch_timing(device, stream):
    """The n = 2048 stochastic-measurement workload (m = 50000, L = 256, bf16 A,
    r = 4, p = 8): one minibatch product (operand split, batch pass, finish and
    apply pass on the tensor cores) timed alone, warm, back to back."""
    import torch
    import synth
    from paper_2012_10469_gb300 import binding as B
    prob = synth.config(3)
    n, L, k = prob.n, prob.L, 4 + 8
    s = B.Solve(n, 4, p=8, q=6, precision=B.MEG_MIXED_BF16, eta=1.0 / (4 * (1 + n / L)), seed=1003, stream=stream,
                V0=prob.U, lam0=np.full(4, 0.25))
    A = torch.from_numpy(np.ascontiguousarray(prob.bits().view(np.int16))).to(device)
    y = torch.from_numpy(prob.y).to(device)
    s.meg_set_objective(B.MEG_MEAS_STOCH, A=A, y=y, L=L)
    g = B.Group([s], stream=stream)
    ms = g.meg_group_time_product(50)
    g.meg_group_destroy()
    s.meg_destroy()
    alg = 2 * L * n * 2
    # tensor-core work of the two passes: bf16 A times the three bf16 pieces of the
    # float operands, [V | W] (2 k_bucket(k) columns) and S (k padded to 16 columns)
    kb = 8 if k <= 8 else 16 if k <= 16 else 32
    tflop = 2 * L * n * 3 * 2 * kb + 2 * n * L * 3 * ((k + 15) // 16 * 16)
    return {"bound": "latency (L2-resident batch)", "engine": "tcgen05 (bf16, float pieces)",
            "ms_per_launch": ms, "kernels": 4,
            "bytes_per_launch": alg, "achieved_GBs": alg / (ms / 1e3) / 1e9,
            "flops_implicit": 4 * L * n * k, "flops_explicit_syrk": n * (n + 1) * L,
            "tensor_flops": tflop,
            "tensor_TFLOPs": tflop / (ms / 1e3) / 1e12,
            "tensor_frac_of_bf16_peak": tflop / (ms / 1e3) / 1e12 / (BF16_TFLOPS or bf16_peak())}


def bilinear_timing(device, stream, hbm_peak):
    """Section 7's experiment at its largest size: n = 600, rank 20, m = 20 n r
    = 240000 pairs of unit bf16 measurement vectors (2 x 288 MB), full
    gradient every iteration, p = 8 and q = 6 (the products the parity test
    at this size uses).  Per product the two tensor-core passes read the
    stacked rows [A; B] twice: 4 m n bf16 values.  Iterations/s of meg_step
    (a captured graph) and the product's fraction of the HBM copy bandwidth."""
    import torch
    import synth
    from paper_2012_10469_gb300 import binding as B
    n, rank, p_, q_ = 600, 20, 8, 6
    prob = synth.bilinear_recovery(n, rank, seed=7)
    A = torch.from_numpy(np.ascontiguousarray(synth.bf16_bits(prob.A).view(np.int16))).to(device)
    Bm = torch.from_numpy(np.ascontiguousarray(synth.bf16_bits(prob.B).view(np.int16))).to(device)
    y = torch.from_numpy(prob.y).to(device)
    m = prob.A.shape[0]
    del prob.A, prob.B
    U = np.linalg.qr(prob.U)[0]
    eta = 1.0 / (prob.tau * 0.4 * np.sqrt(rank * n))
    s = B.Solve(n, rank, p=p_, q=q_, precision=B.MEG_FP32, eta=eta, seed=7, stream=stream, V0=U,
                lam0=np.full(rank, 1.0 / rank))
    s.meg_set_objective(B.MEG_BILINEAR, A=A, B=Bm, y=y, tau=prob.tau)
    s.meg_refine_subspace(8)
    st = torch.cuda.ExternalStream(stream)
    s.meg_step(3)
    torch.cuda.synchronize()
    iters = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    s.meg_step(iters)
    e1.record(st)
    torch.cuda.synchronize()
    ms_iter = e0.elapsed_time(e1) / iters
    g = B.Group([s], stream=stream)
    ms = g.meg_group_time_product(20)
    alg = 4 * m * n * 2
    g.meg_group_destroy()
    s.meg_destroy()
    return {"bound": "hbm", "engine": "tcgen05 (bf16 data, float pieces)", "n": n, "rank": rank, "m": m,
            "p": p_, "q": q_, "ms_per_iteration": ms_iter, "iterations_per_s": 1e3 / ms_iter,
            "ms_per_product": ms, "kernels_per_product": 3, "bytes_per_product": alg,
            "achieved_GBs": alg / (ms / 1e3) / 1e9, "frac": alg / (ms / 1e3) / 1e9 / hbm_peak,
            "product_share_of_iteration": q_ * ms / ms_iter}


def fp32_data_arm(device, stream, hbm_peak, steps):
    """The same batch with float32 data (MEG_FP32: the product on CUDA cores,
    k_dense, 537 MB of data per step) with the benchmark's eigensolver, p and
    q: iterations/s and the product's fraction of the HBM copy bandwidth."""
    import torch
    import synth
    from paper_2012_10469_gb300 import binding as B
    probs = [synth.dense_quadratic(N, R, seed=SEED0 + i, sigma=1e-5, storage="bf16") for i in range(BATCH)]
    solves, keep = [], []
    for i, prob in enumerate(probs):
        M32 = torch.from_numpy(np.ascontiguousarray(prob.M.astype(np.float32))).to(device)
        s = B.Solve(N, R, p=P, q=Q, precision=B.MEG_FP32, eta=1.0, seed=SEED0 + i, stream=stream,
                    V0=prob.U, lam0=prob.w, eigensolver=EIG)
        s.meg_set_objective(B.MEG_DENSE_QUAD, dense=M32)
        solves.append(s)
        keep.append(M32)
    g = B.Group(solves, stream=stream)
    g.meg_group_step(20)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    st = torch.cuda.ExternalStream(stream)
    e0.record(st)
    g.meg_group_step(steps)
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    prod_ms = g.meg_group_time_product(20)
    k = R + P
    alg = BATCH * (N * N * 4 + 2 * N * k * 4)
    g.meg_group_destroy()
    for s in solves:
        s.meg_destroy()
    return {"value": BATCH / (ms / 1e3), "unit": "iters/s", "ms_per_step": ms, "product_ms": prod_ms,
            "product_GBs": alg / (prod_ms / 1e3) / 1e9, "product_frac": alg / (prod_ms / 1e3) / 1e9 / hbm_peak,
            "what": "8 x n=4096 with float32 data (the same bf16-valued matrices), MEG_FP32: float32 CUDA-core "
                    "product k_dense, same eigensolver and (p, q) as the bf16 arm"}


def single_solve_rate(prob, device, iters: int = 200):
    """One instance alone (its 33.5 MB of data stays in L2): iterations/s."""
    import torch
    from paper_2012_10469_gb300 import binding as B
    stream = torch.cuda.Stream(device)
    bits = torch.from_numpy(np.ascontiguousarray(prob.bits().view(np.int16))).to(device)
    s = B.Solve(N, R, p=P, q=Q, precision=B.MEG_MIXED_BF16, eta=1.0, seed=SEED0, stream=stream.cuda_stream,
                V0=prob.U, lam0=prob.w, eigensolver=EIG)
    s.meg_set_objective(B.MEG_DENSE_QUAD, dense=bits)
    s.meg_step(20)
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.meg_step(iters)
    e1.record(stream)
    torch.cuda.synchronize()
    rate = iters / (e0.elapsed_time(e1) / 1e3)
    s.meg_destroy()
    return {"value": rate, "unit": "iters/s", "note": "one n=4096 instance; its data fits in L2"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--serve-requests", type=int, default=2000, help="serving trace length (0: skip)")
    ap.add_argument("--serve-rate", type=float, default=500.0, help="mean arrivals per second")
    ap.add_argument("--serve-fp32-seconds", type=float, default=180.0,
                    help="time cap on the plain float32 form's 50 requests spread over the trace")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
