// meg_autotune: choose the oversampling p, the products per iteration q and
// (optionally) the eigensolver -- subspace iteration or block Krylov, both
// of Section 3 -- for one problem.
//
// The subspace iteration is warm-started from the previous iteration's Ritz
// vectors, so each MEG iteration only has to follow the rotation of the
// top-r eigenvectors of M_t; with too few products (or too few extra
// vectors) the iterate drifts from the exact-eigenpair iterate of
// Definition 2 by a small amount per iteration.  The autotuner measures that
// drift directly: a reference solve with more products and extra vectors
// than any candidate, and pilot solves for the candidates, all from the same
// X_1 and in the same precision, run `pilot_iters` iterations; a candidate is
// accepted when its relative Frobenius distance to the reference is at most
// tol_x * sqrt(pilot_iters / horizon) (rounding differences grow like the
// square root of the iteration count; an under-resolved subspace drifts
// linearly and is rejected).  Candidates are tried in order of cost -- q
// first, then p -- so the first accepted one is the cheapest, and the choice
// depends only on the (bitwise reproducible) results, not on timings.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "../../include/meg.h"

namespace meg_internal {
void set_last_error(const std::string& msg);
}

namespace {

meg_status afail(meg_status st, const std::string& msg) {
    meg_internal::set_last_error("meg_autotune: " + msg);
    return st;
}

struct Iter {
    std::vector<double> V, mu;
    double s = 0.0;
    int n = 0, r = 0;
};

// ||X_a - X_b||_F / ||X_b||_F for X = V diag(mu) V^T + s (I - V V^T), without
// forming n x n matrices and without the cancellation of expanding the
// square: with B = [V_a | V_b] = Q R (Householder QR, Q n x 2r orthonormal),
// C = diag(mu_a - s_a, -(mu_b - s_b)) and d = s_a - s_b,
//   X_a - X_b = Q (R C R^T + d I) Q^T + d (I - Q Q^T),
//   ||X_a - X_b||^2 = ||R C R^T + d I||_F^2 + d^2 (n - 2r).
double rel_dist(const Iter& a, const Iter& b) {
    const int n = a.n, r = a.r, m = 2 * r;
    std::vector<double> A((size_t)n * m);          // column-major n x m
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < r; ++j) {
            A[(size_t)j * n + i] = a.V[(size_t)i * r + j];
            A[(size_t)(r + j) * n + i] = b.V[(size_t)i * r + j];
        }
    // Householder QR, R kept in the upper triangle of the leading m x m block
    for (int j = 0; j < m; ++j) {
        double* x = &A[(size_t)j * n];
        double nrm = 0.0;
        for (int i = j; i < n; ++i) nrm += x[i] * x[i];
        nrm = std::sqrt(nrm);
        if (nrm == 0.0) continue;
        const double alpha = x[j] > 0 ? -nrm : nrm;
        std::vector<double> v(x + j, x + n);
        v[0] -= alpha;
        double vn = 0.0;
        for (double e : v) vn += e * e;
        if (vn > 0.0)
            for (int c = j; c < m; ++c) {
                double* y = &A[(size_t)c * n];
                double dot = 0.0;
                for (int i = j; i < n; ++i) dot += v[i - j] * y[i];
                const double f = 2.0 * dot / vn;
                for (int i = j; i < n; ++i) y[i] -= f * v[i - j];
            }
    }
    auto R = [&](int i, int j) { return i <= j ? A[(size_t)j * n + i] : 0.0; };
    std::vector<double> c(m);
    for (int j = 0; j < r; ++j) { c[j] = a.mu[j] - a.s; c[r + j] = -(b.mu[j] - b.s); }
    const double d = a.s - b.s;
    double d2 = d * d * (double)(n - m);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) {
            double v = (i == j) ? d : 0.0;
            for (int l = 0; l < m; ++l) v += R(i, l) * c[l] * R(j, l);
            d2 += v * v;
        }
    // ||X_b||_F^2 = sum (mu - s)^2 + 2 s sum (mu - s) + n s^2
    double nb = (double)n * b.s * b.s;
    for (int j = 0; j < r; ++j) {
        const double e = b.mu[j] - b.s;
        nb += e * e + 2.0 * b.s * e;
    }
    return std::sqrt(d2 / nb);
}

meg_status run_pilot(const meg_options& o, const meg_objective_desc* obj, const double* V0, const double* lam0,
                     int iters, Iter* out) {
    meg_handle h = nullptr;
    meg_status st = meg_create(&o, V0, lam0, &h);
    if (st == MEG_OK) st = meg_set_objective(h, obj);
    if (st == MEG_OK) st = meg_step(h, iters);
    if (st == MEG_OK) {
        out->n = o.n;
        out->r = o.r;
        out->V.resize((size_t)o.n * o.r);
        out->mu.resize(o.r);
        st = meg_get_iterate(h, out->V.data(), out->mu.data(), &out->s);
    }
    meg_destroy(h);
    return st;
}

}  // namespace

extern "C" meg_status meg_autotune(const meg_options* base, const meg_objective_desc* obj, const double* V0,
                                   const double* lam0, const meg_autotune_options* ao, int* p_out, int* q_out,
                                   double* err_out, int* eig_out) {
    if (!base || !obj || !V0 || !lam0 || !ao || !p_out || !q_out) return afail(MEG_ERR_INVALID_ARG, "null argument");
    const int n = base->n, r = base->r;
    const int kmax = std::min(32, n);
    if (ao->q_max < 1 || ao->q_max > 7 || ao->pilot_iters < 1 || ao->horizon < ao->pilot_iters || !(ao->tol_x > 0.0))
        return afail(MEG_ERR_INVALID_ARG, "need 1 <= q_max <= 7, 1 <= pilot_iters <= horizon, tol_x > 0");
    std::vector<int> ps;
    if (ao->p_cand && ao->n_p > 0) ps.assign(ao->p_cand, ao->p_cand + ao->n_p);
    else ps = {2, 4, 6, 8, 12, 16};
    std::sort(ps.begin(), ps.end());
    ps.erase(std::remove_if(ps.begin(), ps.end(), [&](int p) { return p < 1 || r + p > kmax; }), ps.end());
    if (ps.empty()) return afail(MEG_ERR_INVALID_ARG, "no candidate p with r + p <= min(n, 32)");
    // reference: more extra vectors and more products than any candidate
    meg_options ro = *base;
    ro.p = std::min(kmax - r, std::max(ps.back(), 2 * ps.back()));
    ro.q = std::min(8, ao->q_max + 2);
    ro.eigensolver = MEG_EIG_SUBSPACE;
    Iter ref;
    meg_status st = run_pilot(ro, obj, V0, lam0, ao->pilot_iters, &ref);
    if (st != MEG_OK) return st;
    const double accept = ao->tol_x * std::sqrt((double)ao->pilot_iters / (double)ao->horizon);
    double best_err = INFINITY;
    int best_p = ps.back(), best_q = ao->q_max, best_eig = MEG_EIG_SUBSPACE;
    // with two products the block Krylov eigensolver (Rayleigh-Ritz on
    // [W, A W]) costs a little more than subspace iteration (its 2k x 2k
    // island) and less than a third product: it is tried after subspace
    // iteration at q = 2 and before q = 3
    const bool kry = ao->krylov && base->precision != MEG_FP64;
    for (int q = 1; q <= ao->q_max; ++q)
        for (int eig = MEG_EIG_SUBSPACE; eig <= ((kry && q == 2) ? MEG_EIG_BLOCK_KRYLOV : MEG_EIG_SUBSPACE); ++eig)
            for (int p : ps) {
                if (eig == MEG_EIG_BLOCK_KRYLOV && 2 * (r + p) > 32) continue;
                meg_options o = *base;
                o.p = p;
                o.q = q;
                o.eigensolver = eig;
                Iter it;
                if ((st = run_pilot(o, obj, V0, lam0, ao->pilot_iters, &it)) != MEG_OK) return st;
                const double e = rel_dist(it, ref);
                if (e < best_err) { best_err = e; best_p = p; best_q = q; best_eig = eig; }
                if (e <= accept) {
                    *p_out = p;
                    *q_out = q;
                    if (err_out) *err_out = e;
                    if (eig_out) *eig_out = eig;
                    return MEG_OK;
                }
            }
    // nothing met the target: the most accurate candidate, and say so
    *p_out = best_p;
    *q_out = best_q;
    if (err_out) *err_out = best_err;
    if (eig_out) *eig_out = best_eig;
    return afail(MEG_ERR_NOT_CONVERGED, "no candidate met the target; the most accurate one is returned");
}
