// Row kernels of one low-rank MEG iteration (Algorithm 2, Garber & Kaplan),
// grouped over solves, and the float64 k x k island run by the last block of
// each reduction.
//
// Per iteration t, for each solve (X_t = V diag(mu) V^T + s (I - V V^T)):
//   begin    : eps_t, the operator M_t - c I = V diag(d) V^T + (c0 - c) I + alpha * G_f
//              with G_f the gradient part (Section 3, closed-form log X), and
//              the shift c (see k_begin)
//   product  : Y = G_f W (dense, CSR or measurement kernel)
//   combine  : Z = alpha Y + V (d o U) + (c0 - c) W,  U = V^T W;  Z^T Z, W^T Y
//              last block: Rayleigh-Ritz on span W (final product), exp-map
//              (Definition 2), certificate (Lemma 2), CholeskyQR factor
//   orth1/2  : float64 storage: W <- CholeskyQR2(Z) (two passes), V_{t+1} = W Q_r;
//              V^T W, W^T W
//   orth     : float storage: W <- Z L^{-T}, one CholeskyQR pass whose factor is
//              computed in float64 from the double-word Gram, V_{t+1} = W Q_r;
//              V^T W, W^T W (the Rayleigh-Ritz step uses the exact Gram of W)
#include <algorithm>
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <math.h>

namespace cg = cooperative_groups;

#include "island_f32.cuh"
#include "kxk.cuh"
#include <cstdlib>

#include "meg_dev.cuh"

namespace {

constexpr int NT = 256;              // threads of every row kernel

// sum of entry e over the partials of blocks [b0, b1), in block order; loads are
// issued eight at a time so that a chain of L2 round trips is not serialised
__device__ __forceinline__ dw sum_partials(const float* part, size_t stride, int e, int b0, int b1) {
    dw acc = {0.f, 0.f};
    int b = b0;
    for (; b + 8 <= b1; b += 8) {
        float hv[8], lv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            hv[u] = __ldcg(part + (size_t)(b + u) * stride + 2 * e);
            lv[u] = __ldcg(part + (size_t)(b + u) * stride + 2 * e + 1);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) dw_add(acc, dw{hv[u], lv[u]});
    }
    for (; b < b1; ++b) dw_add(acc, dw{__ldcg(part + (size_t)b * stride + 2 * e), __ldcg(part + (size_t)b * stride + 2 * e + 1)});
    return acc;
}

// --------------------------------------------------------------------------
// Two-level deterministic last-block reduction of per-block double-word
// partials.  Every block of a solve passes its E entries in `mine`; the last
// block of each group of RED_GROUP blocks sums the group in block order, the
// last group-finisher sums the groups in order and gets the totals in `out`.
// Returns true in exactly one block per solve.  No block waits on another.
__device__ bool red_two_level(const SolveDev& s, int lb, const dw* mine, dw* out, int E) {
    const int tid = threadIdx.x;
    const int stride = 2 * RED_MAX_ENTRIES;
    float* part = s.part;
    const int ngroups = (s.nb_red + RED_GROUP - 1) / RED_GROUP;
    __shared__ int am_last;
    for (int e = tid; e < E; e += blockDim.x) {
        part[(size_t)lb * stride + 2 * e] = mine[e].hi;
        part[(size_t)lb * stride + 2 * e + 1] = mine[e].lo;
    }
    __threadfence();
    __syncthreads();
    if (s.nb_red <= 128) {
        // one level: the last block sums every block's partial in block order
        if (tid == 0) am_last = (atomicAdd(&s.ctr[ngroups], 1u) == (unsigned)(s.nb_red - 1));
        __syncthreads();
        if (!am_last) return false;
        if (tid == 0) s.ctr[ngroups] = 0u;
        for (int e = tid; e < E; e += blockDim.x) out[e] = sum_partials(part, stride, e, 0, s.nb_red);
        __syncthreads();
        return true;
    }
    const int g = lb / RED_GROUP;
    const int g0 = g * RED_GROUP, gsz = min(RED_GROUP, s.nb_red - g0);
    if (tid == 0) am_last = (atomicAdd(&s.ctr[g], 1u) == (unsigned)(gsz - 1));
    __syncthreads();
    if (!am_last) return false;
    if (tid == 0) s.ctr[g] = 0u;
    for (int e = tid; e < E; e += blockDim.x) {
        const dw acc = sum_partials(part, stride, e, g0, g0 + gsz);
        part[(size_t)(s.nb_red + g) * stride + 2 * e] = acc.hi;
        part[(size_t)(s.nb_red + g) * stride + 2 * e + 1] = acc.lo;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) am_last = (atomicAdd(&s.ctr[ngroups], 1u) == (unsigned)(ngroups - 1));
    __syncthreads();
    if (!am_last) return false;
    if (tid == 0) s.ctr[ngroups] = 0u;
    for (int e = tid; e < E; e += blockDim.x) out[e] = sum_partials(part, stride, e, s.nb_red, s.nb_red + ngroups);
    __syncthreads();
    return true;
}

// The RED_CLUSTER blocks of a cluster add their E double-word entries through
// distributed shared memory (in rank order) and rank 0 writes one partial per
// cluster to the solve's partial buffer.  Every block of the cluster must call
// this (blocks past the solve's rows contribute zeros).
__device__ __forceinline__ void write_partial(const SolveDev& s, int lb, dw* ent, int E) {
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();
    if (cluster.block_rank() == 0) {
        float* p = s.part + (size_t)(lb / RED_CLUSTER) * 2 * RED_MAX_ENTRIES;
        for (int e = threadIdx.x; e < E; e += blockDim.x) {
            dw acc = ent[e];
            for (int rk = 1; rk < RED_CLUSTER; ++rk) dw_add(acc, cluster.map_shared_rank(ent, rk)[e]);
            p[2 * e] = acc.hi;
            p[2 * e + 1] = acc.lo;
        }
    }
    cluster.sync();    // the other blocks' shared memory must stay until rank 0 has read it
}

// Island kernels: sum the nb_red partials of every entry in a fixed order.
// Items (entry, chunk of blocks) are spread over the threads, each chunk
// summed with batched loads; chunks are then added in chunk order.  The
// result does not depend on timing (deterministic).
__device__ void reduce_partials(const SolveDev& s, dw* out, int E, dw* scratch, int scratch_cap) {
    const int nb = (s.nb_red + RED_CLUSTER - 1) / RED_CLUSTER;     // one partial per cluster
    int C = scratch_cap / E;
    const int cmax = (nb + 15) / 16;               // at least 16 partials per chunk
    C = C < 1 ? 1 : (C > cmax ? cmax : C);
    const size_t stride = 2 * RED_MAX_ENTRIES;
    for (int it = threadIdx.x; it < C * E; it += blockDim.x) {
        const int e = it % E, c = it / E;
        const int b0 = (int)((long long)nb * c / C), b1 = (int)((long long)nb * (c + 1) / C);
        scratch[c * E + e] = sum_partials(s.part, stride, e, b0, b1);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < E; e += blockDim.x) {
        dw acc = scratch[e];
        for (int c = 1; c < C; ++c) dw_add(acc, scratch[c * E + e]);
        out[e] = acc;
    }
    __syncthreads();
}

// index e of the packed upper triangle (column by column) -> (i, j), i <= j
__device__ __forceinline__ void tri_decode(int e, int& i, int& j) {
    int jj = (int)((sqrtf(8.f * e + 1.f) - 1.f) * 0.5f);
    while ((jj + 1) * (jj + 2) / 2 <= e) ++jj;
    while (jj * (jj + 1) / 2 > e) --jj;
    j = jj;
    i = e - jj * (jj + 1) / 2;
}

__device__ __forceinline__ void unpack_sym(const dw* src, double* dst, int k) {
    const int nsym = k * (k + 1) / 2;
    for (int e = threadIdx.x; e < nsym; e += blockDim.x) {
        int i, j;
        tri_decode(e, i, j);
        double v = dw_value(src[e]);
        dst[i * MEG_LDK + j] = v;
        dst[j * MEG_LDK + i] = v;
    }
    __syncthreads();
}

__device__ __forceinline__ void store_kxk(double* g, const double* s, int m, int n) {
    for (int e = threadIdx.x; e < m * n; e += blockDim.x) g[(e / n) * 32 + e % n] = s[(e / n) * MEG_LDK + e % n];
}

__device__ __forceinline__ void load_kxk(const double* g, double* s, int m, int n) {
    for (int e = threadIdx.x; e < m * n; e += blockDim.x) s[(e / n) * MEG_LDK + e % n] = g[(e / n) * 32 + e % n];
    __syncthreads();
}

__device__ __forceinline__ double lse(const double* x, int cnt) {
    double m = x[0];
    for (int i = 1; i < cnt; ++i) m = fmax(m, x[i]);
    double acc = 0.0;
    for (int i = 0; i < cnt; ++i) acc += exp(x[i] - m);
    return m + log(acc);
}

}  // namespace

// ==========================================================================
// begin: per-iteration scalars (one block of 32 threads per solve).
//
// M_t = log X_t - eta grad f(X_t) in closed form (Section 3):
//   log X_t = V diag(log mu - log s) V^T + log s I.
// Dense quadratic: grad f = X - M, so M_t = V diag(log mu - log s - eta (mu - s)) V^T
//   + (log s - eta s) I + eta M  (alpha = +eta, gradient part Y = M W).
// Other kinds: the gradient part enters with alpha = -eta.
// Shift: subspace iteration finds the eigenvalues largest in magnitude, the
// wanted ones are the algebraically largest of M_t, whose spectrum is
// negative.  Reading adopted: iterate on M_t - c I with
// c = min(log s, min log mu) - eta * g, g a bound on ||grad f||_2 (Frobenius
// norm of the gradient or of its minibatch form), which makes M_t - c I
// positive semidefinite; the Ritz values are shifted back exactly.
// Warm start (mode 1) runs the same machinery on -grad f(0) - c I.
__global__ void k_begin(const SolveDev* sds, int ns) {
    pdl_wait();
    pdl_trigger();
    const int si = blockIdx.x;
    if (si >= ns) return;
    const SolveDev& s = sds[si];
    double* sm = s.sm;
    const int r = s.r, lane = threadIdx.x;
    if (s.mode == 1) {
        if (lane < r) sm[SM_DCOEF + lane] = 0.0;
        if (lane == 0) {
            sm[SM_C0] = 0.0;
            sm[SM_ALPHA] = (s.kind == MEG_DENSE_QUAD) ? 1.0 : -1.0;
            double g0;
            if (s.kind == MEG_MEAS_STOCH || s.kind == MEG_BILINEAR) g0 = sm[SM_RESID_BOUND];
            else if (s.kind == MEG_CSR_QUAD) g0 = sm[SM_RSS];
            else g0 = sqrt(sm[SM_FROD2]);
            sm[SM_SHIFT] = -1.0001 * g0 - 1e-300;
        }
        return;
    }
    const double t = sm[SM_T];
    const double sv = sm[SM_S];
    const double eta = s.eta;
    // log s and log mu were stored with s and mu (no logarithm here)
    const double logs = sm[SM_LOGS];
    double lmu = logs;
    if (lane < r) {
        const double mu = sm[SM_MU + lane];
        lmu = sm[SM_LOGMU + lane];
        double d = lmu - logs;
        if (s.kind == MEG_DENSE_QUAD) d -= eta * (mu - sv);
        sm[SM_DCOEF + lane] = d;
    }
    double lmin = fmin(lmu, logs);
    for (int o = 16; o > 0; o >>= 1) lmin = fmin(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
    if (lane == 0) {
        // eps_t = a / (t + c + 1)^q; integer q by repeated multiplication
        const double x = t + s.eps_c + 1.0;
        double xp;
        if (s.eps_pow == 2.0) xp = x * x;
        else if (s.eps_pow == 1.0) xp = x;
        else if (s.eps_pow == 3.0) xp = x * x * x;
        else xp = pow(x, s.eps_pow);
        sm[SM_EPS] = s.eps_a / xp;
        sm[SM_C0] = (s.kind == MEG_DENSE_QUAD) ? logs - eta * sv : logs;
        sm[SM_ALPHA] = (s.kind == MEG_DENSE_QUAD) ? eta : -eta;
        double g;
        switch (s.kind) {
            case MEG_DENSE_QUAD: g = sm[SM_GNORM]; break;
            case MEG_LINEAR: g = sqrt(sm[SM_FROD2]); break;
            case MEG_CSR_QUAD: g = sm[SM_RSS]; break;
            default: g = sm[SM_RESID_BOUND]; break;
        }
        double c = lmin - eta * g - 1e-12 * fabs(lmin);
        // Subspace iteration after a Rayleigh-Ritz step.  c above is a lower
        // bound of the spectrum; the previous step's lowest Ritz value
        // sigma_k, carried to this iterate's bulk level (sigma_k - log s moves
        // with log s: e = log s + SM_SKREL), estimates the top of the unwanted
        // part.  Their midpoint centres the unwanted eigenvalues of M_t - c I
        // around zero, halving their largest magnitude, while every wanted
        // eigenvalue (above e) stays the larger: per product the error of
        // eigenvector i shrinks by (e - c) / (2 lambda_i - c - e) instead of
        // (lambda_{k+1} - c) / (lambda_i - c).  The shift stays at least
        // (sigma_1 - e) / 64 below e, so that (M_t - c I) W keeps its rank in
        // float arithmetic when the unwanted spectrum is one narrow cluster.
        const double e = logs + sm[SM_SKREL], s1 = sm[SM_SIGMA];
        if (s.eig == MEG_EIG_SUBSPACE && t > 1.0 && sm[SM_LAST_T] == t - 1.0 && isfinite(e) && isfinite(s1)) {
            const double cm = fmin(0.5 * (c + e), e - (s1 - e) * (1.0 / 64.0));
            if (cm > c) c = cm;
        }
        sm[SM_SHIFT] = c;
    }
}


// ---------------------------------------------------------------------------
// Rayleigh-Ritz for float storage (float64 results from float32 work).
//   Ht = G^{-1/2} H G^{-1/2},  E = G - I (|E| < 1e-3: W is orthonormal to a few
//        float32 units after its CholeskyQR pass, at most about kappa(Z) of
//        them; with q > 1 the final product's plain float factor leaves up to
//        kappa(Z)^2 units for the next iteration's first product), to second order:
//        G^{-1/2} = I - E/2 + 3 E^2/8 + O(E^3), so
//        Ht = H - (E H + H E)/2 + 3 (E^2 H + H E^2)/8 + E H E/4 + O(E^3 |H|)
//        (the second-order terms in float32: they are below 1e-6 |H|)
//   float32 Jacobi on Ht -> Q
//   theta_i = q_i^T Ht q_i / q_i^T q_i  with exact (Dot2) products
//   top r vectors: q_i + sum_j q_j (q_j^T Ht q_i)/(theta_i - theta_j)  (first order;
//        pairs closer than 100 |q_j^T Ht q_i| are left as they are),
//        Lowdin re-orthonormalisation, map back x = (I - E/2 + 3 E^2/8) q
// Scratch: F (4 float matrices), the double regions C, JB, Bm (G), H.
// Writes sigma, mu, s, t, certificate, objective estimate, QV, M1 like the
// float64 island.  kk is the dimension of the pencil: the block size k for
// subspace iteration, 2k for the block Krylov space [W0 W1], whose tail
// (krylov = true) writes the next block's coordinates QW (kk x k: the top-k
// Ritz vectors, the first r of them as in QV) instead of a CholeskyQR factor.
__device__ void rr_fast_f32(const SolveDev& s, double* smw, const double* S1, const double* P, double* G,
                            double* H, double* C, double* JB, float* F, double* wv, double* pr, double* pdg,
                            double* sig, double* mun, double shift, int kk, bool krylov) {
    const int tid = threadIdx.x, nt = blockDim.x, k = kk, r = s.r, n = s.n;
    constexpr int FM = 32 * MEG_LDK;        // floats per float matrix
    float* F0 = F;
    float* F1 = F + FM;
    float* F2 = F + 2 * FM;
    float* F3 = F + 3 * FM;
    float* Bh = (float*)G;                  // two float matrices in the G region
    float* Bl = Bh + FM;
    __shared__ int perm[MEG_KMAX];
    __shared__ int flag2;
    // 1. E, H in float; Ht = H - (T + T^T)/2 + 3 (E T + (E T)^T)/8 + T E/4 in
    //    float64, T = E H (T E = E H E is symmetric)
    for (int e = tid; e < k * k; e += nt) {
        const int i = e / k, j = e % k;
        F0[i * MEG_LDK + j] = (float)(G[i * MEG_LDK + j] - (i == j ? 1.0 : 0.0));
        F1[i * MEG_LDK + j] = (float)H[i * MEG_LDK + j];
    }
    __syncthreads();
    mm_f32(F0, false, F1, F2, k, k, k);                       // T = E H
    mm_f32(F0, false, F2, F1, k, k, k);                       // E T = E^2 H
    mm_f32(F2, false, F0, F3, k, k, k);                       // T E = E H E
    for (int e = tid; e < k * k; e += nt) {
        const int i = e / k, j = e % k;
        const double t1 = (double)F2[i * MEG_LDK + j] + (double)F2[j * MEG_LDK + i];
        const double t2 = (double)F1[i * MEG_LDK + j] + (double)F1[j * MEG_LDK + i];
        const double t3 = (double)F3[i * MEG_LDK + j] + (double)F3[j * MEG_LDK + i];
        H[i * MEG_LDK + j] += -0.5 * t1 + 0.375 * t2 + 0.125 * t3;
    }
    __syncthreads();
    // 2. float32 Jacobi on Ht
    for (int e = tid; e < k * k; e += nt) F1[(e / k) * MEG_LDK + e % k] = (float)H[(e / k) * MEG_LDK + e % k];
    __syncthreads();
    // the double-word refinement below corrects the remaining rotations to first
    // order, so Jacobi only has to reach about 1e-5 relative off-diagonal size
    __shared__ float* jA;
    if (tid == 0) jA = F1;
    __syncthreads();
    // the 2k x 2k pencils of the block Krylov step are swept by the whole block
    const int nsw = k > 16 ? jacobi_block_f32(&jA, F3, F2, (float*)pr, k, 4, 1e-5f)
                           : jacobi_warp_f32(&jA, F3, F2, (float*)pr, k, 4, 1e-5f);   // Q in F2; F1/F3 free
    if (tid == 0) smw[SM_JSWEEPS] = nsw;
    // 3. Ht as hi/lo floats; Tq = Ht Q exactly (Dot2), as hi/lo floats in F1/F3
    for (int e = tid; e < k * k; e += nt) {
        const int i = e / k, j = e % k;
        float hi, lo;
        dw_split(H[i * MEG_LDK + j], hi, lo);
        Bh[i * MEG_LDK + j] = hi;
        Bl[i * MEG_LDK + j] = lo;
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += nt) {
        const int a = e / k, i = e % k;
        dw acc = {0.f, 0.f};
        for (int b = 0; b < k; ++b) {
            const float q = F2[b * MEG_LDK + i];
            dot2_acc(acc, Bh[a * MEG_LDK + b], q);
            dot2_acc(acc, Bl[a * MEG_LDK + b], q);
        }
        F1[a * MEG_LDK + i] = acc.hi;
        F3[a * MEG_LDK + i] = acc.lo;
    }
    __syncthreads();
    // 4. Rayleigh quotients theta_i (exact products) and the descending order
    if (tid < k) {
        dw num = {0.f, 0.f}, den = {0.f, 0.f};
        for (int a = 0; a < k; ++a) {
            const float q = F2[a * MEG_LDK + tid];
            dot2_acc(num, q, F1[a * MEG_LDK + tid]);
            dot2_acc(num, q, F3[a * MEG_LDK + tid]);
            dot2_acc(den, q, q);
        }
        wv[tid] = dw_value(num) * rcp_newton(dw_value(den));
    }
    __syncthreads();
    if (tid < k) {
        int rank = 0;
        const double v = wv[tid];
        for (int j = 0; j < k; ++j) rank += ranks_before(wv[j], j, v, tid);
        perm[rank] = tid;
    }
    __syncthreads();
    if (tid < k) sig[tid] = wv[perm[tid]] + shift;
    // 5. perturbation theory in the Jacobi basis, h_ji = q_j^T Ht q_i (exact
    //    products): first-order correction of the top r vectors, coefficients
    //    h_ji / (theta_i - theta_j) in Bh (k x r); second-order correction of
    //    the top r + 1 Ritz values, sum_j h_ji^2 / (theta_i - theta_j), its terms
    //    in Bl (the Rayleigh quotient of a vector that Jacobi left a relative
    //    1e-5 off is low by up to that squared times the spread; without this
    //    term the Ritz values carry that bias from one iteration to the next)
    const int rc = min(r + 1, k);
    for (int e = tid; e < k * rc; e += nt) {
        const int j = e / rc, i = e % rc, ci = perm[i];
        float cf = 0.f, c2 = 0.f;
        if (j != ci) {
            dw h = {0.f, 0.f};
            for (int a = 0; a < k; ++a) {
                const float q = F2[a * MEG_LDK + j];
                dot2_acc(h, q, F1[a * MEG_LDK + ci]);
                dot2_acc(h, q, F3[a * MEG_LDK + ci]);
            }
            const double hv = dw_value(h), gap = wv[ci] - wv[j];
            if (fabs(gap) > 100.0 * fabs(hv)) {
                // float quotients: the coefficients are stored as floats
                const float hf = (float)hv, gf = (float)gap;
                cf = hf / gf;
                c2 = hf * cf;
            }
        }
        if (i < r) Bh[j * MEG_LDK + i] = cf;
        Bl[j * MEG_LDK + i] = c2;
    }
    __syncthreads();
    if (tid < rc) {
        double c = 0.0;
        for (int j = 0; j < k; ++j) c += (double)Bl[j * MEG_LDK + tid];
        sig[tid] += c;
    }
    __syncthreads();
    mm_f32(F2, false, Bh, Bl, k, k, r);                        // corr = Q coef  (k x r)
    for (int e = tid; e < k * r; e += nt) {
        const int a = e / r, i = e % r;
        H[a * MEG_LDK + i] = (double)F2[a * MEG_LDK + perm[i]] + (double)Bl[a * MEG_LDK + i];
    }
    __syncthreads();
    // 6. Lowdin: QV <- QV (I - (QV^T QV - I)/2), float64 (k r^2)
    for (int e = tid; e < r * r; e += nt) {
        const int i = e / r, j = e % r;
        double g = 0.0;
        for (int a = 0; a < k; ++a) g = fma(H[a * MEG_LDK + i], H[a * MEG_LDK + j], g);
        C[i * MEG_LDK + j] = g - (i == j ? 1.0 : 0.0);
    }
    __syncthreads();
    for (int e = tid; e < k * r; e += nt) {
        const int a = e / r, i = e % r;
        double v = H[a * MEG_LDK + i];
        for (int j = 0; j < r; ++j) v -= 0.5 * H[a * MEG_LDK + j] * C[j * MEG_LDK + i];
        JB[a * MEG_LDK + i] = v;
        Bh[a * MEG_LDK + i] = (float)v;
    }
    __syncthreads();
    // 7. back to the W basis: x = (I - E/2 + 3 E^2/8) q
    mm_f32(F0, false, Bh, Bl, k, k, r);                        // E QV (k x r)
    mm_f32(F0, false, Bl, F1, k, k, r);                        // E^2 QV
    for (int e = tid; e < k * r; e += nt) {
        const int a = e / r, i = e % r;
        const double v = JB[a * MEG_LDK + i] - 0.5 * (double)Bl[a * MEG_LDK + i] + 0.375 * (double)F1[a * MEG_LDK + i];
        smw[SM_QV + a * 32 + i] = v;
        Bh[a * MEG_LDK + i] = (float)v;
    }
    __syncthreads();
    // 8. objective estimate v_i^T D v_i (float32 suffices: it only sets the shift bound)
    for (int e = tid; e < k * k; e += nt) F3[(e / k) * MEG_LDK + e % k] = (float)P[(e / k) * MEG_LDK + e % k];
    __syncthreads();
    mm_f32(F3, false, Bh, Bl, k, k, r);                        // P QV
    if (tid < r) {
        float acc = 0.f;
        for (int a = 0; a < k; ++a) acc = fmaf(Bh[a * MEG_LDK + tid], Bl[a * MEG_LDK + tid], acc);
        pdg[tid] = acc;
    }
    // 9. scalars: exp-map (Definition 2), certificate (Lemma 2), objective estimate.
    //    The transcendental functions run side by side on different lanes; the
    //    state they read is loaded at once (one lane per slot), and float64
    //    operations are kept few: GB300 issues a warp's float64 instruction at
    //    about 1/60 of the float32 rate.
    if (tid < 32) {
        const int lane = tid;
        const int slot = lane == 0 ? SM_T : lane == 1 ? SM_EPS : lane == 2 ? SM_FIRST_HOLD : lane == 3 ? SM_TRD
                                                                                          : SM_FROD2;
        const double ld = lane < 5 ? smw[slot] : 0.0;
        const double t = __shfl_sync(0xffffffffu, ld, 0);
        const double eps = __shfl_sync(0xffffffffu, ld, 1);
        const double first_hold = __shfl_sync(0xffffffffu, ld, 2);
        const double trd = __shfl_sync(0xffffffffu, ld, 3);
        const double frod2 = __shfl_sync(0xffffffffu, ld, 4);
        double m = (lane <= r && lane < k) ? sig[lane] : -1e300;
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        const double ex = (lane <= r && lane < k) ? exp(sig[lane] - m) : 0.0;
        double a_r = lane < r ? ex : 0.0, a_r1 = ex;
        for (int o = 16; o > 0; o >>= 1) {
            a_r += __shfl_xor_sync(0xffffffffu, a_r, o);
            a_r1 += __shfl_xor_sync(0xffffffffu, a_r1, o);
        }
        // lane 0: log a_r, lane 1: log a_{r+1}, lane 2: log eps, lane 3: log(1 - eps)
        const double lg = log(lane == 0 ? a_r : (lane == 1 ? a_r1 : (lane == 2 ? eps : lane == 3 ? 1.0 - eps : 1.0)));
        const double lse_r = m + __shfl_sync(0xffffffffu, lg, 0);
        const double lse_r1 = m + __shfl_sync(0xffffffffu, lg, 1);
        const double log_eps = __shfl_sync(0xffffffffu, lg, 2);
        const double log_1meps = __shfl_sync(0xffffffffu, lg, 3);
        if (s.mode == 1) {
            if (lane == 0) {
                for (int i = 0; i < r; ++i) mun[i] = sig[i];
                simplex_project(mun, r);
                const double eps0 = eps_of(s, 0.0);
                for (int i = 0; i < r; ++i) {
                    const double mu0 = (1.0 - eps0) * mun[i] + eps0 / n;
                    smw[SM_MU + i] = mu0;
                    smw[SM_LOGMU + i] = log(mu0);
                }
                smw[SM_S] = eps0 / n;
                smw[SM_LOGS] = log(eps0 / n);
                smw[SM_T] = 1.0;
                smw[SM_LAST_T] = 0.0;
                smw[SM_CERT] = 0.0;
                smw[SM_HOLDS] = 0.0;
                smw[SM_FIRST_HOLD] = 0.0;
            }
        } else {
            const double s_new = eps * rcp_newton((double)(n - r));
            // mu_i = (1 - eps) e^{sigma_i - m} / a_r: the exponentials already formed;
            // log mu_i = log(1 - eps) + sigma_i - lse_r, log s = log eps - log(n - r)
            const double mu = lane < r ? (1.0 - eps) * ex * rcp_newton(a_r) : 0.0;
            if (lane < r) smw[SM_LOGMU + lane] = log_1meps + (sig[lane] - lse_r);
            double xd = lane < r ? (mu - s_new) * pdg[lane] : 0.0, x2 = mu * mu;
            for (int o = 16; o > 0; o >>= 1) {
                xd += __shfl_xor_sync(0xffffffffu, xd, o);
                x2 += __shfl_xor_sync(0xffffffffu, x2, o);
            }
            if (lane < r) smw[SM_MU + lane] = mu;
            if (lane == 0) {
                const double cert = s.log_nr + sig[r] - log_eps - lse_r1;
                const int holds = cert <= 2.0 * eps;
                smw[SM_LSE] = lse_r;
                smw[SM_CERT] = cert;
                smw[SM_HOLDS] = holds;
                if (holds && first_hold == 0.0) smw[SM_FIRST_HOLD] = t;
                smw[SM_LAST_T] = t;
                if (s.kind == MEG_DENSE_QUAD || s.kind == MEG_LINEAR) {
                    xd += s_new * trd;
                    x2 += (double)(n - r) * s_new * s_new;
                    if (s.kind == MEG_DENSE_QUAD) {
                        const double f = 0.5 * x2 - xd + 0.5 * frod2;
                        smw[SM_FEST] = f;
                        smw[SM_GNORM] = 1.25 * sqrt(fmax(2.0 * f, 0.0));
                    } else {
                        smw[SM_FEST] = xd;
                    }
                }
                smw[SM_S] = s_new;
                smw[SM_SKREL] = sig[s.k - 1] - smw[SM_LOGS];
                smw[SM_LOGS] = log_eps - s.log_nr;
                smw[SM_T] = t + 1.0;
            }
        }
        if (lane < k) {
            smw[SM_SIGMA + lane] = sig[lane];
            if (!isfinite(sig[lane])) smw[SM_STATUS] = MEG_ERR_NUMERIC;
        }
    }
    __syncthreads();
    if (krylov) {
        // 10'. next block [W0 W1] QW: the top k = s.k Ritz vectors, columns r.. as
        //      the sorted Jacobi vectors mapped back, x = (I - E/2 + 3 E^2/8) q
        //      (orthonormal to float accuracy; the next Rayleigh-Ritz step uses
        //      the exact Gram of the stored block)
        const int kb = s.k;
        for (int e = tid; e < k * kb; e += nt) {
            const int a = e / kb, i = e % kb;
            Bh[a * MEG_LDK + i] = i < r ? 0.f : F2[a * MEG_LDK + perm[i]];
        }
        __syncthreads();
        mm_f32(F0, false, Bh, Bl, k, k, kb);                   // E q
        mm_f32(F0, false, Bl, F1, k, k, kb);                   // E^2 q
        for (int e = tid; e < k * kb; e += nt) {
            const int a = e / kb, i = e % kb;
            smw[SM_QW + a * 32 + i] = i < r ? smw[SM_QV + a * 32 + i]
                                            : (double)Bh[a * MEG_LDK + i] - 0.5 * (double)Bl[a * MEG_LDK + i] +
                                                  0.375 * (double)F1[a * MEG_LDK + i];
        }
        return;
    }
    // 10. next block W = Z Q M (Ritz-ordered), M^T (Q^T S1 Q) M = I.  With q > 1
    //     the next product's CholeskyQR pass restores orthonormality before any
    //     Rayleigh-Ritz step, so a float32 factor suffices (it changes how
    //     orthonormal W is, not its span); with q = 1 the Gram Q^T S1 Q is formed
    //     with exact products and factored by gram_factor_f32, Q M in float64.
    for (int e = tid; e < k * k; e += nt) {
        const int a = e / k, i = e % k;
        F1[a * MEG_LDK + i] = F2[a * MEG_LDK + perm[i]];       // Q, sorted columns
        if (s.q > 1) F3[a * MEG_LDK + i] = (float)S1[a * MEG_LDK + i];
    }
    __syncthreads();
    if (s.q > 1) {
        mm_f32(F3, false, F1, Bh, k, k, k);                    // S1 Q
        mm_f32(F1, true, Bh, Bl, k, k, k);                     // Q^T S1 Q
        if (!chol_inv_f32(Bl, F3, (float*)pr, k, &flag2) && tid == 0) smw[SM_STATUS] = MEG_ERR_NUMERIC;
        mm_f32(F1, false, F3, Bh, k, k, k);                    // M1 = Q L^{-T}
        for (int e = tid; e < k * k; e += nt) smw[SM_M1 + (e / k) * 32 + e % k] = (double)Bh[(e / k) * MEG_LDK + e % k];
        return;
    }
    for (int e = tid; e < k * k; e += nt) {                     // C = S1 Q (exact products)
        const int i = e / k, j = e % k;
        dw acc = {0.f, 0.f};
        for (int a = 0; a < k; ++a) {
            float hi, lo;
            dw_split(S1[i * MEG_LDK + a], hi, lo);
            const float q = F1[a * MEG_LDK + j];
            dot2_acc(acc, hi, q);
            dot2_acc(acc, lo, q);
        }
        C[i * MEG_LDK + j] = dw_value(acc);
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += nt) {                     // H = Q^T C
        const int i = e / k, j = e % k;
        dw acc = {0.f, 0.f};
        for (int a = 0; a < k; ++a) {
            float hi, lo;
            dw_split(C[a * MEG_LDK + j], hi, lo);
            const float q = F1[a * MEG_LDK + i];
            dot2_acc(acc, q, hi);
            dot2_acc(acc, q, lo);
        }
        H[i * MEG_LDK + j] = dw_value(acc);
    }
    __syncthreads();
    if (!gram_factor_f32(H, F0, F2, F3, Bh, C, JB, (float*)pr, k, &flag2) && tid == 0)
        smw[SM_STATUS] = MEG_ERR_NUMERIC;
    for (int e = tid; e < k * k; e += nt) {                     // M1 = Q M (exact products)
        const int i = e / k, j = e % k;
        dw acc = {0.f, 0.f};
        for (int a = 0; a < k; ++a) {
            float hi, lo;
            dw_split(JB[a * MEG_LDK + j], hi, lo);
            const float q = F1[i * MEG_LDK + a];
            dot2_acc(acc, q, hi);
            dot2_acc(acc, q, lo);
        }
        smw[SM_M1 + i * 32 + j] = dw_value(acc);
    }
}

// ==========================================================================
// combine: Z = (M_t - c I) W for the block's rows, reductions, last block.
template <typename T>
__global__ void __launch_bounds__(NT) k_combine(const SolveDev* sds, int ns, int phase) {
    pdl_wait();
    pdl_trigger();
    const int si = find_solve(sds, ns, PK_RED, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_RED];     // blocks past nb_red pad the last cluster
    const int n = s.n, k = s.k, r = s.r, tid = threadIdx.x;
    const int row0 = min(n, lb * s.rows_red), row1 = min(n, row0 + s.rows_red), nr = row1 - row0;

    extern __shared__ __align__(16) unsigned char smraw[];
    // layout: Bc[r*k] Coef, sW/sZ/sY [rows_red*k] T, ent dw[2*528], then k x k doubles
    Coef<T>* Bc = (Coef<T>*)smraw;
    T* sW = (T*)(Bc + MEG_RMAX * MEG_KMAX);
    T* sZ = sW + s.rows_red * k;
    T* sY = sZ + s.rows_red * k;
    dw* ent = (dw*)(((uintptr_t)(sY + s.rows_red * k) + 15) & ~(uintptr_t)15);
    __shared__ Coef<T> c_id, c_al;

    const double* sm = s.sm;
    const bool init = (phase == PH_INIT);
    if (!init) {
        for (int e = tid; e < r * k; e += NT) {
            int l = e / k, j = e % k;
            Bc[e].set(sm[SM_DCOEF + l] * sm[SM_U + l * 32 + j]);
        }
        if (tid == 0) {
            c_id.set(sm[SM_C0] - sm[SM_SHIFT]);
            c_al.set(sm[SM_ALPHA]);
        }
    }
    __syncthreads();

    const T* W = (const T*)s.W;
    const double* V = s.V;
    T* Z = (T*)s.Z;
    const bool dense = (s.kind == MEG_DENSE_QUAD || s.kind == MEG_LINEAR);
    // block Krylov, second product: Z is not needed, its row buffer holds W0
    const bool kry2 = (phase == PH_KRY2);
    const T* W0 = (const T*)s.Wp;
    __shared__ T sVt[ROWS_MAX * MEG_RMAX];     // this block's rows of V in storage precision
    if (!init)
        for (int e = tid; e < nr * r; e += NT) sVt[e] = (T)V[(size_t)(row0 + e / r) * r + e % r];
    __syncthreads();
    for (int idx = tid; idx < nr * k; idx += NT) {
        const int i = row0 + idx / k, j = idx % k;
        const T w = W[(size_t)i * k + j];
        T z, y = 0;
        if (init) {
            z = w;
        } else {
            if (dense) {
                const T* Ys = (const T*)s.Ys;
                const int np = s.tc ? tc_tile_slots(s, i / 128) : s.nb_ds;   // slots in order
                for (int p = 0; p < np; ++p) y += Ys[((size_t)p * n + i) * k + j];
            } else if (s.kind == MEG_MEAS_STOCH || s.kind == MEG_BILINEAR) {
                const T* Ys = (const T*)s.Ys;
                const int np = apply_slots(s.kind, s.nb_meas, n, s.mtc);    // chunks in order
                for (int p = 0; p < np; ++p) y += Ys[((size_t)p * n + i) * k + j];
            } else {
                y = ((const T*)s.Y)[(size_t)i * k + j];
            }
            if (kry2) {
                z = W0[(size_t)i * k + j];
            } else {
                z = c_al.mul(y);
                z = c_id.fma_(w, z);
                for (int l = 0; l < r; ++l) z = Bc[l * k + j].fma_(sVt[(idx / k) * r + l], z);
            }
        }
        if (!kry2) Z[(size_t)i * k + j] = z;
        sW[idx] = w;
        sZ[idx] = z;
        sY[idx] = y;
    }
    __syncthreads();

    // Gram entries, by phase:
    //   advance / init : Z^T Z
    //   final          : Z^T Z, W^T Y
    //   block Krylov 1 : W^T Y, W^T Z (k x k, for the projection on W)
    //   block Krylov 2 : W1^T Y, W0^T Y (k x k)
    const int nsym = k * (k + 1) / 2;
    const bool fin = (phase == PH_FINAL), kry1 = (phase == PH_KRY1);
    const int E = (kry1 || kry2) ? nsym + k * k : fin ? 2 * nsym : nsym;
    for (int e = tid; e < E; e += NT) {
        int i, j;
        const T* X;
        const T* Yv;
        if (kry1 || kry2) {
            if (e < nsym) { tri_decode(e, i, j); X = sW; Yv = sY; }
            else { i = (e - nsym) / k; j = (e - nsym) % k; X = kry1 ? sW : sZ; Yv = kry1 ? sZ : sY; }
        } else if (e < nsym) {
            tri_decode(e, i, j); X = sZ; Yv = sZ;
        } else if (e < 2 * nsym) {
            tri_decode(e - nsym, i, j); X = sW; Yv = sY;
        } else {
            i = (e - 2 * nsym) / k; j = (e - 2 * nsym) % k; X = sW; Yv = sZ;
        }
        Acc<T> a, b;
        a.zero();
        b.zero();
        int q = 0;
        for (; q + 1 < nr; q += 2) {          // two independent chains for ILP
            a.add_prod(X[q * k + i], Yv[q * k + j]);
            b.add_prod(X[(q + 1) * k + i], Yv[(q + 1) * k + j]);
        }
        if (q < nr) a.add_prod(X[q * k + i], Yv[q * k + j]);
        dw r0 = a.as_dw();
        dw_add(r0, b.as_dw());
        ent[e] = r0;
    }
    __syncthreads();
    write_partial(s, lb, ent, E);
}

// ==========================================================================
// island after combine (one block per solve): Z^T Z (and W^T Y) from the
// partials; CholeskyQR factor, and on the final product the Rayleigh-Ritz
// step, exp-map (Definition 2) and certificate (Lemma 2).
template <typename T>
__global__ void __launch_bounds__(NT) k_island_c(const SolveDev* sds, int ns, int phase) {
    pdl_wait();
    pdl_trigger();
    const int si = blockIdx.x;
    if (si >= ns) return;
    const SolveDev& s = sds[si];
    const int n = s.n, k = s.k, r = s.r, tid = threadIdx.x;
    extern __shared__ __align__(16) unsigned char smraw[];
    // four float matrices (the reduction's scratch first), the entries, the k x k doubles
    constexpr int FBYTES = 4 * 32 * MEG_LDK * (int)sizeof(float);
    dw* ent = (dw*)(smraw + FBYTES);
    double* kx = (double*)(ent + RED_MAX_ENTRIES);
    const int nsym = k * (k + 1) / 2;
    const bool fin = (phase == PH_FINAL);
    const int E = fin ? 2 * nsym : nsym;
    reduce_partials(s, ent, E, (dw*)smraw, FBYTES / (int)sizeof(dw));
    // ---------------- last block of this solve: k x k island (float64)
    double* S1 = kx;
    double* A = S1 + 32 * MEG_LDK;
    double* Bm = A + 32 * MEG_LDK;
    double* C = Bm + 32 * MEG_LDK;
    double* Qg = C + 32 * MEG_LDK;
    double* JB = Qg + 32 * MEG_LDK;     // Jacobi scratch
    double* wv = JB + 32 * MEG_LDK;     // [32]
    double* pr = wv + 32;               // [96]
    double* pdg = pr + 96;              // [32] v_i^T D v_i
    __shared__ int flag;
    double* smw = s.sm;
    unpack_sym(ent, S1, k);
    if (!fin) {
        // W' = Z L^{-T}, L = chol(Z^T Z)
        if constexpr (sizeof(T) == 4) {
            // the only CholeskyQR pass of the float-storage modes: a factor of the
            // double-word Gram refined in Gram space, so that W = Z M1 (exact
            // products, one rounding) is orthonormal to a few float rounding units
            // (a plain float factor would leave about kappa(Z)^2 of them and need
            // a second pass over the rows)
            float* F = (float*)smraw;                  // the reduction's scratch, free again
            constexpr int FM = 32 * MEG_LDK;
            if (!gram_factor_f32(S1, F, F + FM, F + 2 * FM, F + 3 * FM, A, C, (float*)pr, k, &flag) && tid == 0)
                smw[SM_STATUS] = MEG_ERR_NUMERIC;
            store_kxk(smw + SM_M1, C, k, k);
        } else {
            for (int e = tid; e < k * k; e += NT) A[(e / k) * MEG_LDK + e % k] = S1[(e / k) * MEG_LDK + e % k];
            __syncthreads();
            if (!kxk_chol(A, k, &flag) && tid == 0) smw[SM_STATUS] = MEG_ERR_NUMERIC;
            kxk_inv_lower_T(A, C, k);
            store_kxk(smw + SM_M1, C, k, k);
        }
        return;
    }
    // ---- Rayleigh-Ritz on span W (Section 3, three steps):
    //   H = W^T (M_t - c I) W = U^T diag(d) U + (c0 - c) G + alpha P,  G = W^T W,
    //   eigenpairs of the pencil (H, G) -> Ritz values theta, G-orthonormal Qg.
    double* P = A;
    unpack_sym(ent + nsym, P, k);
    double* G = Bm;
    load_kxk(smw + SM_G, G, k, k);
    double* U = C;
    load_kxk(smw + SM_U, U, r, k);
    const double d_id = smw[SM_C0] - smw[SM_SHIFT], alpha = smw[SM_ALPHA], shift = smw[SM_SHIFT];
    double* H = Qg;
    __shared__ double dco[MEG_RMAX];
    if (tid < r) dco[tid] = smw[SM_DCOEF + tid];
    __syncthreads();
    for (int e = tid; e < k * k; e += NT) {
        int i = e / k, j = e % k;
        double h = d_id * G[i * MEG_LDK + j] + alpha * P[i * MEG_LDK + j];
        for (int l = 0; l < r; ++l) h += U[l * MEG_LDK + i] * dco[l] * U[l * MEG_LDK + j];
        H[i * MEG_LDK + j] = h;
    }
    __syncthreads();
    __shared__ double sig[MEG_KMAX];
    __shared__ double mun[MEG_KMAX];
    __shared__ int use_fast;
    if constexpr (sizeof(T) == 4) {
        // E = G - I; after the CholeskyQR pass ||E|| is a few float32 rounding
        // units, so the second-order treatment below is exact to O(E^3)
        if (tid < 32) {
            float em = 0.f;
            for (int e = tid; e < k * k; e += 32)
                em = fmaxf(em, fabsf((float)(G[(e / k) * MEG_LDK + e % k] - ((e / k == e % k) ? 1.0 : 0.0))));
            for (int o = 16; o > 0; o >>= 1) em = fmaxf(em, __shfl_xor_sync(0xffffffffu, em, o));
            if (tid == 0) use_fast = em < 1e-3f;
        }
        __syncthreads();
        if (use_fast) {
            rr_fast_f32(s, smw, S1, P, G, H, C, JB, (float*)smraw, wv, pr, pdg, sig, mun, shift, k, false);
            return;
        }
    }
    // G = L L^T; Ht = L^{-1} H L^{-T}
    if (!kxk_chol(G, k, &flag) && tid == 0) smw[SM_STATUS] = MEG_ERR_NUMERIC;
    double* Li = U;                       // U no longer needed (H is built)
    kxk_inv_lower_T(G, Li, k);            // Li = L^{-T} (upper)
    double* T1 = G;                       // L no longer needed
    kxk_mm(H, false, Li, T1, k, k, k);    // T1 = H L^{-T}
    kxk_mm(Li, true, T1, H, k, k, k);     // H <- L^{-1} H L^{-T}
    double* Qt = T1;
    kxk_jacobi(H, Qt, JB, wv, pr, k, 30);
    kxk_mm(Li, false, Qt, Qg, k, k, k);   // Qg = L^{-T} Qt  (G-orthonormal Ritz coordinates)
    // v_i^T D v_i = (Qg^T P Qg)_ii for the objective estimate (dense data)
    kxk_mm(P, false, Qg, JB, k, k, r);    // JB = P Qg[:, :r]
    if (tid < r) {
        double acc = 0.0;
        for (int a = 0; a < k; ++a) acc += Qg[a * MEG_LDK + tid] * JB[a * MEG_LDK + tid];
        pdg[tid] = acc;
    }
    __syncthreads();

    // Ritz values sigma_i = theta_i + c, kept in shared memory
    if (tid < k) {
        sig[tid] = wv[tid] + shift;
        smw[SM_SIGMA + tid] = sig[tid];
    }
    __syncthreads();
    if (tid == 0) {
        for (int i = 0; i < k; ++i)
            if (!isfinite(sig[i])) smw[SM_STATUS] = MEG_ERR_NUMERIC;
        const double t = smw[SM_T];
        if (s.mode == 1) {
            // eq. (exp:init), U = 0: eigenvalues of -grad f(0) projected on the simplex
            for (int i = 0; i < r; ++i) mun[i] = sig[i];
            simplex_project(mun, r);
            const double eps0 = eps_of(s, 0.0);
            for (int i = 0; i < r; ++i) {
                const double mu0 = (1.0 - eps0) * mun[i] + eps0 / n;
                smw[SM_MU + i] = mu0;
                smw[SM_LOGMU + i] = log(mu0);
            }
            smw[SM_S] = eps0 / n;
            smw[SM_LOGS] = log(eps0 / n);
            smw[SM_T] = 1.0;
            smw[SM_LAST_T] = 0.0;
            smw[SM_CERT] = 0.0;
            smw[SM_HOLDS] = 0.0;
            smw[SM_FIRST_HOLD] = 0.0;
        } else {
            const double eps = smw[SM_EPS];
            // Lemma 2 certificate with b_{r+1} (eq. convergenceGuaranteeExperiment2):
            //   C_t = log((n - r) e^{sigma_{r+1}} / (eps_t b_{r+1})),  b_{r+1} = sum_{i<=r+1} e^{sigma_i}
            const double lse_r1 = lse(sig, r + 1);
            const double cert = log((double)(n - r)) + sig[r] - log(eps) - lse_r1;
            const int holds = cert <= 2.0 * eps;
            // Definition 2: mu_i = (1 - eps) e^{sigma_i} / sum_{j<=r} e^{sigma_j}, s = eps/(n - r)
            const double lse_r = lse(sig, r);
            for (int i = 0; i < r; ++i) mun[i] = (1.0 - eps) * exp(sig[i] - lse_r);
            const double s_new = eps / (double)(n - r);
            smw[SM_LSE] = lse_r;
            smw[SM_CERT] = cert;
            smw[SM_HOLDS] = holds;
            if (holds && smw[SM_FIRST_HOLD] == 0.0) smw[SM_FIRST_HOLD] = t;
            smw[SM_LAST_T] = t;
            if (s.kind == MEG_DENSE_QUAD || s.kind == MEG_LINEAR) {
                // <X_{t+1}, D> = sum_i (mu_i - s) v_i^T D v_i + s Tr D
                double xd = s_new * smw[SM_TRD], x2 = (double)(n - r) * s_new * s_new;
                for (int i = 0; i < r; ++i) {
                    xd += (mun[i] - s_new) * pdg[i];
                    x2 += mun[i] * mun[i];
                }
                if (s.kind == MEG_DENSE_QUAD) {
                    const double f = 0.5 * x2 - xd + 0.5 * smw[SM_FROD2];
                    smw[SM_FEST] = f;
                    smw[SM_GNORM] = 1.25 * sqrt(fmax(2.0 * f, 0.0));
                } else {
                    smw[SM_FEST] = xd;
                }
            }
            const double log_1meps = log1p(-eps);
            for (int i = 0; i < r; ++i) {
                smw[SM_MU + i] = mun[i];
                smw[SM_LOGMU + i] = log_1meps + (sig[i] - lse_r);
            }
            smw[SM_S] = s_new;
            smw[SM_SKREL] = sig[s.k - 1] - smw[SM_LOGS];
            smw[SM_LOGS] = log(eps) - log((double)(n - r));
            smw[SM_T] = t + 1.0;
        }
    }
    __syncthreads();
    // V_{t+1} = W Qg[:, :r];  next block W' from CholQR of Z Qg (Ritz-ordered)
    store_kxk(smw + SM_QV, Qg, k, r);
    kxk_mm(S1, false, Qg, Bm, k, k, k);   // S1 Qg
    kxk_mm(Qg, true, Bm, A, k, k, k);     // Qg^T S1 Qg
    if (!kxk_chol(A, k, &flag) && tid == 0) smw[SM_STATUS] = MEG_ERR_NUMERIC;
    kxk_inv_lower_T(A, C, k);             // L^{-T}
    kxk_mm(Qg, false, C, Bm, k, k, k);    // M1 = Qg L^{-T}
    store_kxk(smw + SM_M1, Bm, k, k);
}

// ==========================================================================
// Block Krylov Rayleigh-Ritz (Section 3 names Lanczos-type methods as the
// faster alternative to subspace iteration).  One MEG iteration makes two
// products with A = M_t - c I: A W0 with the warm-started block W0, then
// A W1 with W1 the orthonormalised part of Z = A W0 outside span W0; the
// Rayleigh-Ritz step runs on the 2k-dimensional Krylov space span [W0 W1]
// and the next block is its top-k Ritz vectors.  Float storage only.
//
// island after the block Krylov combines (one block per solve).
//   PH_KRY1 (Z = A W0, entries W0^T Y, B = W0^T Z):
//     H00 = W0^T A W0 = U0^T diag(d) U0 + (c0 - c) G0 + alpha W0^T Y (kept for
//     the Rayleigh-Ritz step) and the projection coefficients C = G0^{-1} B
//     (G0 = I + E0, |E0| a few float units: C = B - E0 B).  U0, G0 and W0^T Y
//     move to their own slots (the reduction after the orth pass overwrites
//     U, G with those of W1).  The rest of Z, Z' = Z - W0 C, is formed by the
//     projection pass on the rows, and its Gram taken there: near convergence
//     the columns of Z' shrink to the rounding of the stored Z, below what a
//     Gram-space difference Z^T Z - B^T C resolves.
//   PH_KRY2 (entries P2 = W1^T Y2, Q2 = W0^T Y2): the 2k x 2k pencil
//     H = [H00 H01; H01^T H11], G = [G0 G01; G01^T G11] with
//     H11 = U1^T diag(d) U1 + (c0 - c) G11 + alpha P2,
//     H01 = U0^T diag(d) U1 + (c0 - c) G01 + alpha Q2,
//     Rayleigh-Ritz (rr_fast_f32 on 2k), exp-map, certificate, and the next
//     block's coordinates QW.
template <typename T>
__global__ void __launch_bounds__(NT) k_island_kry(const SolveDev* sds, int ns, int phase) {
    pdl_wait();
    pdl_trigger();
    const int si = blockIdx.x;
    if (si >= ns) return;
    const SolveDev& s = sds[si];
    const int k = s.k, r = s.r, tid = threadIdx.x;
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int FBYTES = 4 * 32 * MEG_LDK * (int)sizeof(float);
    constexpr int FM = 32 * MEG_LDK;
    dw* ent = (dw*)(smraw + FBYTES);
    double* kx = (double*)(ent + RED_MAX_ENTRIES);
    double* R0 = kx;                    // six double k x k regions
    double* R1 = R0 + FM;
    double* R2 = R1 + FM;
    double* R3 = R2 + FM;
    double* R4 = R3 + FM;
    double* R5 = R4 + FM;
    double* wv = R5 + FM;               // [32]
    double* pr = wv + 32;               // [96]
    double* pdg = pr + 96;              // [32]
    __shared__ int flag;
    __shared__ double dco[MEG_RMAX];
    double* smw = s.sm;
    const int nsym = k * (k + 1) / 2;
    const bool kry1 = (phase == PH_KRY1);
    const int E = kry1 ? 2 * nsym + k * k : nsym + k * k;
    reduce_partials(s, ent, E, (dw*)smraw, FBYTES / (int)sizeof(dw));
    if (tid < r) dco[tid] = smw[SM_DCOEF + tid];
    const double d_id = smw[SM_C0] - smw[SM_SHIFT], alpha = smw[SM_ALPHA], shift = smw[SM_SHIFT];
    __syncthreads();
    if (kry1) {
        double* P1 = R1;
        double* B = R2;
        double* G0 = R3;
        double* U0 = R4;
        unpack_sym(ent, P1, k);
        for (int e = tid; e < k * k; e += NT) B[(e / k) * MEG_LDK + e % k] = dw_value(ent[nsym + e]);
        load_kxk(smw + SM_G, G0, k, k);
        load_kxk(smw + SM_U, U0, r, k);
        for (int e = tid; e < k * k; e += NT) {
            const int i = e / k, j = e % k;
            double h = d_id * G0[i * MEG_LDK + j] + alpha * P1[i * MEG_LDK + j];
            for (int l = 0; l < r; ++l) h += U0[l * MEG_LDK + i] * dco[l] * U0[l * MEG_LDK + j];
            smw[SM_H00 + i * 32 + j] = h;
            smw[SM_G0 + i * 32 + j] = G0[i * MEG_LDK + j];
            smw[SM_P + i * 32 + j] = P1[i * MEG_LDK + j];
        }
        for (int e = tid; e < r * k; e += NT) smw[SM_U0 + (e / k) * 32 + e % k] = U0[(e / k) * MEG_LDK + e % k];
        // C = B - E0 B  (E0 = G0 - I; the E0^2 term is below 1e-13 of B)
        float* F = (float*)smraw;       // the reduction's scratch, free again
        float* Fe = F;
        float* Fb = F + FM;
        float* Fc = F + 2 * FM;
        for (int e = tid; e < k * k; e += NT) {
            const int i = e / k, j = e % k;
            Fe[i * MEG_LDK + j] = (float)(G0[i * MEG_LDK + j] - (i == j ? 1.0 : 0.0));
            Fb[i * MEG_LDK + j] = (float)B[i * MEG_LDK + j];
        }
        __syncthreads();
        mm_f32(Fe, false, Fb, Fc, k, k, k);
        for (int e = tid; e < k * k; e += NT)
            smw[SM_KC + (e / k) * 32 + e % k] = B[(e / k) * MEG_LDK + e % k] - (double)Fc[(e / k) * MEG_LDK + e % k];
        return;
    }
    // ---- PH_KRY2: Rayleigh-Ritz on span [W0 W1]
    const int kk = 2 * k;
    double* H = R0;
    double* G = R1;
    double* P = R2;
    double* U1 = R3;                    // scratch until the pencil is built
    double* U0 = R4;
    {
        // P2 (sym) and Q2 = W0^T Y2 from the entries
        for (int e = tid; e < nsym; e += NT) {
            int i, j;
            tri_decode(e, i, j);
            const double v = dw_value(ent[e]);
            P[(k + i) * MEG_LDK + k + j] = v;
            P[(k + j) * MEG_LDK + k + i] = v;
        }
        for (int e = tid; e < k * k; e += NT) {
            const int i = e / k, j = e % k;          // (W0^T Y2)_ij: row i of W0, column j of W1's product
            const double v = dw_value(ent[nsym + e]);
            P[i * MEG_LDK + k + j] = v;
            P[(k + j) * MEG_LDK + i] = v;
            P[i * MEG_LDK + j] = smw[SM_P + i * 32 + j];
            G[i * MEG_LDK + j] = smw[SM_G0 + i * 32 + j];
            G[(k + i) * MEG_LDK + k + j] = smw[SM_G + i * 32 + j];
            const double g01 = smw[SM_G01 + i * 32 + j];
            G[i * MEG_LDK + k + j] = g01;
            G[(k + j) * MEG_LDK + i] = g01;
            H[i * MEG_LDK + j] = smw[SM_H00 + i * 32 + j];
        }
        load_kxk(smw + SM_U, U1, r, k);
        load_kxk(smw + SM_U0, U0, r, k);
        for (int e = tid; e < k * k; e += NT) {
            const int i = e / k, j = e % k;
            double h11 = d_id * G[(k + i) * MEG_LDK + k + j] + alpha * P[(k + i) * MEG_LDK + k + j];
            double h01 = d_id * G[i * MEG_LDK + k + j] + alpha * P[i * MEG_LDK + k + j];
            for (int l = 0; l < r; ++l) {
                h11 += U1[l * MEG_LDK + i] * dco[l] * U1[l * MEG_LDK + j];
                h01 += U0[l * MEG_LDK + i] * dco[l] * U1[l * MEG_LDK + j];
            }
            H[(k + i) * MEG_LDK + k + j] = h11;
            H[i * MEG_LDK + k + j] = h01;
            H[(k + j) * MEG_LDK + i] = h01;
        }
        __syncthreads();
    }
    // E = G - I must be small for the second-order treatment of rr_fast_f32:
    // W0 and W1 are orthonormal to a few float units, W0^T W1 to the
    // rounding of Z' relative to its size
    __shared__ float em_s;
    if (tid < 32) {
        float em = 0.f;
        for (int e = tid; e < kk * kk; e += 32)
            em = fmaxf(em, fabsf((float)(G[(e / kk) * MEG_LDK + e % kk] - ((e / kk == e % kk) ? 1.0 : 0.0))));
        for (int o = 16; o > 0; o >>= 1) em = fmaxf(em, __shfl_xor_sync(0xffffffffu, em, o));
        if (tid == 0) em_s = em;
    }
    __syncthreads();
    if (!(em_s < 1e-2f) && tid == 0) smw[SM_STATUS] = MEG_ERR_NUMERIC;
    __shared__ double sig[MEG_KMAX];
    __shared__ double mun[MEG_KMAX];
    rr_fast_f32(s, smw, nullptr, P, G, H, R3, R4, (float*)smraw, wv, pr, pdg, sig, mun, shift, kk, true);
}

// ==========================================================================
// orth1: W' = Z M1 (first CholeskyQR pass); final phase also V_{t+1} = W Qv.
template <typename T>
__global__ void __launch_bounds__(NT) k_orth1(const SolveDev* sds, int ns, int phase) {
    pdl_wait();
    pdl_trigger();
    const int si = find_solve(sds, ns, PK_RED, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_RED];     // blocks past nb_red pad the last cluster
    const int n = s.n, k = s.k, r = s.r, tid = threadIdx.x;
    const int row0 = min(n, lb * s.rows_red), row1 = min(n, row0 + s.rows_red), nr = row1 - row0;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* M1 = (T*)smraw;                                  // k x k
    Coef<T>* Qv = (Coef<T>*)(M1 + MEG_KMAX * MEG_KMAX); // k x r
    T* sW = (T*)(Qv + MEG_KMAX * MEG_RMAX);
    dw* ent = (dw*)(((uintptr_t)(sW + s.rows_red * k) + 15) & ~(uintptr_t)15);
    const double* sm = s.sm;
    const bool fin = (phase == PH_FINAL);
    for (int e = tid; e < k * k; e += NT) M1[e] = (T)sm[SM_M1 + (e / k) * 32 + e % k];
    if (fin)
        for (int e = tid; e < k * r; e += NT) Qv[e].set(sm[SM_QV + (e / r) * 32 + e % r]);
    __syncthreads();
    const T* Z = (const T*)s.Z;
    const T* W = (const T*)s.W;
    T* Wp = (T*)s.Wp;
    double* Vn = s.Vn;
    // the block's rows of Z are one contiguous span: stage it (coalesced), then W' = Z M1
    T* sZ = (T*)(ent + 528);
    for (int idx = tid; idx < nr * k; idx += NT) sZ[idx] = Z[(size_t)row0 * k + idx];
    __syncthreads();
    for (int idx = tid; idx < nr * k; idx += NT) {
        const int q = idx / k, j = idx % k;
        T acc = 0;
        for (int l = 0; l < k; ++l) acc += sZ[q * k + l] * M1[l * k + j];
        Wp[(size_t)row0 * k + idx] = acc;
        sW[idx] = acc;
    }
    if (fin) {
        for (int idx = tid; idx < nr * r; idx += NT) {
            const int i = row0 + idx / r, j = idx % r;
            // V_{t+1} = W Qv evaluated exactly enough to keep X_{t+1} at float64 accuracy
            if constexpr (sizeof(T) == 8) {
                double acc = 0.0;
                for (int l = 0; l < k; ++l) acc = Qv[l * r + j].fma_(W[(size_t)i * k + l], acc);
                Vn[(size_t)i * r + j] = acc;
            } else {
                dw acc = {0.f, 0.f};
                for (int l = 0; l < k; ++l) {
                    const float w = W[(size_t)i * k + l];
                    dot2_acc(acc, w, Qv[l * r + j].hi);
                    dot2_acc(acc, w, Qv[l * r + j].lo);
                }
                Vn[(size_t)i * r + j] = dw_value(acc);
            }
        }
    }
    __syncthreads();
    const int nsym = k * (k + 1) / 2;
    for (int e = tid; e < nsym; e += NT) {
        int i, j;
        tri_decode(e, i, j);
        Acc<T> a, b;
        a.zero();
        b.zero();
        int q = 0;
        for (; q + 1 < nr; q += 2) {
            a.add_prod(sW[q * k + i], sW[q * k + j]);
            b.add_prod(sW[(q + 1) * k + i], sW[(q + 1) * k + j]);
        }
        if (q < nr) a.add_prod(sW[q * k + i], sW[q * k + j]);
        dw r0 = a.as_dw();
        dw_add(r0, b.as_dw());
        ent[e] = r0;
    }
    __syncthreads();
    write_partial(s, lb, ent, nsym);
}

// ==========================================================================
// island after orth1: W'^T W' from the partials -> second CholeskyQR factor.
template <typename T>
__global__ void __launch_bounds__(NT) k_island_o1(const SolveDev* sds, int ns, int phase) {
    pdl_wait();
    pdl_trigger();
    const int si = blockIdx.x;
    if (si >= ns) return;
    const SolveDev& s = sds[si];
    const int k = s.k, tid = threadIdx.x;
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int FBYTES = 4 * 32 * MEG_LDK * (int)sizeof(float);
    dw* ent = (dw*)(smraw + FBYTES);
    double* kx = (double*)(ent + RED_MAX_ENTRIES);
    const int nsym = k * (k + 1) / 2;
    reduce_partials(s, ent, nsym, (dw*)smraw, FBYTES / (int)sizeof(dw));
    double* A = kx;
    double* C = A + 32 * MEG_LDK;
    __shared__ int flag;
    __shared__ float dsc[MEG_KMAX];
    unpack_sym(ent, A, k);
    if constexpr (sizeof(T) == 4) {
        float* Af = (float*)C;
        float* Mf = Af + 32 * MEG_LDK;
        for (int e = tid; e < k * k; e += NT) Af[(e / k) * MEG_LDK + e % k] = (float)A[(e / k) * MEG_LDK + e % k];
        __syncthreads();
        if (!chol_inv_f32(Af, Mf, dsc, k, &flag) && tid == 0) s.sm[SM_STATUS] = MEG_ERR_NUMERIC;
        for (int e = tid; e < k * k; e += NT) s.sm[SM_M2 + (e / k) * 32 + e % k] = (double)Mf[(e / k) * MEG_LDK + e % k];
    } else {
        if (!kxk_chol(A, k, &flag) && tid == 0) s.sm[SM_STATUS] = MEG_ERR_NUMERIC;
        kxk_inv_lower_T(A, C, k);
        store_kxk(s.sm + SM_M2, C, k, k);
    }
}

// ==========================================================================
// orth2: W = W' M2 (second CholeskyQR pass); final phase commits V = V_{t+1}.
// Reductions U = V^T W and G = W^T W for the next product's operator and
// Rayleigh-Ritz step.
template <typename T>
__global__ void __launch_bounds__(NT) k_orth2(const SolveDev* sds, int ns, int phase) {
    pdl_wait();
    pdl_trigger();
    const int si = find_solve(sds, ns, PK_RED, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_RED];     // blocks past nb_red pad the last cluster
    const int n = s.n, k = s.k, r = s.r, tid = threadIdx.x;
    const int row0 = min(n, lb * s.rows_red), row1 = min(n, row0 + s.rows_red), nr = row1 - row0;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* M2 = (T*)smraw;
    T* sW = M2 + MEG_KMAX * MEG_KMAX;
    double* sV = (double*)(((uintptr_t)(sW + s.rows_red * k) + 7) & ~(uintptr_t)7);
    dw* ent = (dw*)(((uintptr_t)(sV + s.rows_red * r) + 15) & ~(uintptr_t)15);
    __shared__ float sVh[ROWS_MAX * MEG_RMAX], sVl[ROWS_MAX * MEG_RMAX];
    const double* sm = s.sm;
    const bool fin = (phase == PH_FINAL);
    for (int e = tid; e < k * k; e += NT) M2[e] = (T)sm[SM_M2 + (e / k) * 32 + e % k];
    __syncthreads();
    const T* Wp = (const T*)s.Wp;
    T* W = (T*)s.W;
    double* V = s.V;
    const double* Vn = s.Vn;
    // the block's rows of W' are one contiguous span: stage it (coalesced), then W = W' M2;
    // in float storage the staging area is the entries' buffer (unused until the Gram)
    T* sIn = sizeof(T) == 4 ? (T*)ent : (T*)(ent + RED_MAX_ENTRIES);
    for (int idx = tid; idx < nr * k; idx += NT) sIn[idx] = Wp[(size_t)row0 * k + idx];
    __syncthreads();
    for (int idx = tid; idx < nr * k; idx += NT) {
        const int q = idx / k, j = idx % k;
        T acc = 0;
        for (int l = 0; l < k; ++l) acc += sIn[q * k + l] * M2[l * k + j];
        W[(size_t)row0 * k + idx] = acc;
        sW[idx] = acc;
    }
    for (int idx = tid; idx < nr * r; idx += NT) {
        const int i = row0 + idx / r, j = idx % r;
        double v;
        if (fin) {
            v = Vn[(size_t)i * r + j];
            V[(size_t)i * r + j] = v;
        } else {
            v = V[(size_t)i * r + j];
        }
        sV[idx] = v;
        const float vh = (float)v;
        sVh[idx] = vh;
        sVl[idx] = (float)(v - (double)vh);
    }
    __syncthreads();
    if (s.Wsp) {
        // exact split for the tensor-core product, W = hi + mid + lo in bf16; Wsp is
        // K-major (row j of a piece holds column j of W), so consecutive threads
        // take consecutive rows i of W for coalesced stores
        const size_t kp = (size_t)s.tc_kpad;
        const size_t P = (size_t)(s.tc_npad / 3);        // rows per piece (k rounded up to 16)
        for (int idx = tid; idx < nr * k; idx += NT) {
            const int j = idx / nr, q = idx % nr, i = row0 + q;
            const float w = (float)sW[q * k + j];
            const __nv_bfloat16 hi = __float2bfloat16_rn(w);
            const float r1 = w - __bfloat162float(hi);
            const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
            const float r2 = r1 - __bfloat162float(mid);
            const __nv_bfloat16 lo = __float2bfloat16_rn(r2);
            s.Wsp[(size_t)j * kp + i] = __bfloat16_as_ushort(hi);
            s.Wsp[(P + j) * kp + i] = __bfloat16_as_ushort(mid);
            s.Wsp[(2 * P + j) * kp + i] = __bfloat16_as_ushort(lo);
        }
    }
    const int nsym = k * (k + 1) / 2;
    const int E = nsym + r * k;
    for (int e = tid; e < E; e += NT) {
        Acc<T> a, b;
        a.zero();
        b.zero();
        if (e < nsym) {
            int i, j;
            tri_decode(e, i, j);
            int q = 0;
            for (; q + 1 < nr; q += 2) {
                a.add_prod(sW[q * k + i], sW[q * k + j]);
                b.add_prod(sW[(q + 1) * k + i], sW[(q + 1) * k + j]);
            }
            if (q < nr) a.add_prod(sW[q * k + i], sW[q * k + j]);
        } else {
            int l = (e - nsym) / k, j = (e - nsym) % k;
            for (int q = 0; q < nr; ++q) {
                if constexpr (sizeof(T) == 8) {
                    a.add_prod(sV[q * r + l], sW[q * k + j]);
                } else {      // V is float64: two floats per entry, both products exact in Dot2
                    a.add_prod(sVh[q * r + l], sW[q * k + j]);
                    b.add_prod(sVl[q * r + l], sW[q * k + j]);
                }
            }
        }
        dw r0 = a.as_dw();
        dw_add(r0, b.as_dw());
        ent[e] = r0;
    }
    __syncthreads();
    write_partial(s, lb, ent, E);
}

// ==========================================================================
// orth (float storage): W = Z M1, the single CholeskyQR pass (M1 = L^{-T} of
// the double-word Gram of Z, factored in float64); on the final product
// M1 = Qg L^{-T} and V_{t+1} = W Qv is formed from the block's rows of the
// previous W and committed.  Reductions U = V^T W and G = W^T W for the next
// product's operator and Rayleigh-Ritz step, and the bf16 split of W for the
// tensor-core product.
template <typename T>
__global__ void __launch_bounds__(NT) k_orth(const SolveDev* sds, int ns, int phase) {
    pdl_wait();
    pdl_trigger();
    const int si = find_solve(sds, ns, PK_RED, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_RED];     // blocks past nb_red pad the last cluster
    const int n = s.n, k = s.k, r = s.r, tid = threadIdx.x;
    const int row0 = min(n, lb * s.rows_red), row1 = min(n, row0 + s.rows_red), nr = row1 - row0;
    extern __shared__ __align__(16) unsigned char smraw[];
    Coef<T>* M1 = (Coef<T>*)smraw;                      // k x k, float64 values as (hi, lo)
    Coef<T>* Qv = M1 + MEG_KMAX * MEG_KMAX;             // k x r
    T* sW = (T*)(Qv + MEG_KMAX * MEG_RMAX);             // rows of W (first the previous W)
    double* sV = (double*)(((uintptr_t)(sW + s.rows_red * k) + 7) & ~(uintptr_t)7);
    dw* ent = (dw*)(((uintptr_t)(sV + s.rows_red * r) + 15) & ~(uintptr_t)15);
    // float storage: V as (hi, lo) floats in the area of sV
    float* sVh = (float*)sV;
    float* sVl = sVh + s.rows_red * r;
    const double* sm = s.sm;
    const bool fin = (phase == PH_FINAL);
    for (int e = tid; e < k * k; e += NT) M1[e].set(sm[SM_M1 + (e / k) * 32 + e % k]);
    if (fin)
        for (int e = tid; e < k * r; e += NT) Qv[e].set(sm[SM_QV + (e / r) * 32 + e % r]);
    const T* Z = (const T*)s.Z;
    T* W = (T*)s.W;
    double* V = s.V;
    // the block's rows of Z (and of the previous W) are contiguous spans: stage
    // them (coalesced); Z goes to the entries' buffer, unused until the Gram
    T* sZ = (T*)ent;
    for (int idx = tid; idx < nr * k; idx += NT) sZ[idx] = Z[(size_t)row0 * k + idx];
    if (fin)
        for (int idx = tid; idx < nr * k; idx += NT) sW[idx] = W[(size_t)row0 * k + idx];
    __syncthreads();
    for (int idx = tid; idx < nr * r; idx += NT) {
        const int q = idx / r, j = idx % r;
        double v;
        if (fin) {
            // V_{t+1} = W Qv evaluated exactly enough to keep X_{t+1} at float64 accuracy
            if constexpr (sizeof(T) == 8) {
                v = 0.0;
                for (int l = 0; l < k; ++l) v = Qv[l * r + j].fma_(sW[q * k + l], v);
            } else {
                dw acc = {0.f, 0.f};
                for (int l = 0; l < k; ++l) {
                    const float w = sW[q * k + l];
                    dot2_acc(acc, w, Qv[l * r + j].hi);
                    dot2_acc(acc, w, Qv[l * r + j].lo);
                }
                v = dw_value(acc);
            }
            V[(size_t)row0 * r + idx] = v;
        } else {
            v = V[(size_t)row0 * r + idx];
        }
        if constexpr (sizeof(T) == 8) {
            sV[idx] = v;
        } else {
            const float vh = (float)v;
            sVh[idx] = vh;
            sVl[idx] = (float)(v - (double)vh);
        }
    }
    __syncthreads();      // the previous W rows are read
    for (int idx = tid; idx < nr * k; idx += NT) {
        const int q = idx / k, j = idx % k;
        // W = Z M1 with exact products (Dot2) over the high part of M1: the
        // entries of Z and M1 reach kappa(Z) times those of W, and a float sum
        // would leave k kappa(Z) rounding units in W instead of one; the low
        // part (a float rounding unit of M1) adds in plain float arithmetic
        T acc;
        if constexpr (sizeof(T) == 4) {
            dw a2 = {0.f, 0.f};
            float lo = 0.f;
            for (int l = 0; l < k; ++l) {
                const float z = sZ[q * k + l];
                dot2_acc(a2, z, M1[l * k + j].hi);
                lo = fmaf(z, M1[l * k + j].lo, lo);
            }
            acc = a2.hi + (a2.lo + lo);
        } else {
            acc = 0;
            for (int l = 0; l < k; ++l) acc = M1[l * k + j].fma_(sZ[q * k + l], acc);
        }
        W[(size_t)row0 * k + idx] = acc;
        sW[idx] = acc;
    }
    __syncthreads();
    if (s.Wsp) {
        // exact split for the tensor-core product, W = hi + mid + lo in bf16; Wsp is
        // K-major (row j of a piece holds column j of W), so consecutive threads
        // take consecutive rows i of W for coalesced stores
        const size_t kp = (size_t)s.tc_kpad;
        const size_t P = (size_t)(s.tc_npad / 3);        // rows per piece (k rounded up to 16)
        for (int idx = tid; idx < nr * k; idx += NT) {
            const int j = idx / nr, q = idx % nr, i = row0 + q;
            const float w = (float)sW[q * k + j];
            const __nv_bfloat16 hi = __float2bfloat16_rn(w);
            const float r1 = w - __bfloat162float(hi);
            const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
            const float r2 = r1 - __bfloat162float(mid);
            const __nv_bfloat16 lo = __float2bfloat16_rn(r2);
            s.Wsp[(size_t)j * kp + i] = __bfloat16_as_ushort(hi);
            s.Wsp[(P + j) * kp + i] = __bfloat16_as_ushort(mid);
            s.Wsp[(2 * P + j) * kp + i] = __bfloat16_as_ushort(lo);
        }
    }
    const int nsym = k * (k + 1) / 2;
    const int E = nsym + r * k;
    for (int e = tid; e < E; e += NT) {
        Acc<T> a, b;
        a.zero();
        b.zero();
        if (e < nsym) {
            int i, j;
            tri_decode(e, i, j);
            int q = 0;
            for (; q + 1 < nr; q += 2) {
                a.add_prod(sW[q * k + i], sW[q * k + j]);
                b.add_prod(sW[(q + 1) * k + i], sW[(q + 1) * k + j]);
            }
            if (q < nr) a.add_prod(sW[q * k + i], sW[q * k + j]);
        } else {
            int l = (e - nsym) / k, j = (e - nsym) % k;
            if constexpr (sizeof(T) == 8) {
                for (int q = 0; q < nr; ++q) a.add_prod(sV[q * r + l], sW[q * k + j]);
            } else {
                // V is float64, held as (hi, lo) floats: the high part in Dot2, the
                // low part (a float rounding unit of V) in plain float arithmetic
                float lo = 0.f;
                for (int q = 0; q < nr; ++q) {
                    const float w = sW[q * k + j];
                    a.add_prod(sVh[q * r + l], w);
                    lo = fmaf(sVl[q * r + l], w, lo);
                }
                dw r0 = a.as_dw();
                dw_add(r0, dw{lo, 0.f});
                ent[e] = r0;
                continue;
            }
        }
        dw r0 = a.as_dw();
        dw_add(r0, b.as_dw());
        ent[e] = r0;
    }
    __syncthreads();
    write_partial(s, lb, ent, E);
}

// ==========================================================================
// projection pass of the block Krylov iteration (float storage): the rest of
// Z = A W0 outside span W0, Z' = Z - W0 C (C = G0^{-1} W0^T Z), with exact
// products and one rounding, written over Z; Gram entries Z'^T Z' for its
// CholeskyQR factor (k_island_c's single-pass factor).
__global__ void __launch_bounds__(NT) k_kry_proj(const SolveDev* sds, int ns, int phase) {
    pdl_wait();
    pdl_trigger();
    const int si = find_solve(sds, ns, PK_RED, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_RED];
    const int n = s.n, k = s.k, tid = threadIdx.x;
    const int row0 = min(n, lb * s.rows_red), row1 = min(n, row0 + s.rows_red), nr = row1 - row0;
    extern __shared__ __align__(16) unsigned char smraw[];
    Coef<float>* Cc = (Coef<float>*)smraw;              // C (k x k)
    float* sA = (float*)(Cc + MEG_KMAX * MEG_KMAX);     // rows of W0
    float* sB = sA + ROWS_MAX * MEG_KMAX;               // rows of Z, then of Z'
    dw* ent = (dw*)(sB + ROWS_MAX * MEG_KMAX);
    const double* sm = s.sm;
    for (int e = tid; e < k * k; e += NT) Cc[e].set(sm[SM_KC + (e / k) * 32 + e % k]);
    const float* W = (const float*)s.W;
    float* Z = (float*)s.Z;
    for (int idx = tid; idx < nr * k; idx += NT) {
        sA[idx] = W[(size_t)row0 * k + idx];
        sB[idx] = Z[(size_t)row0 * k + idx];
    }
    __syncthreads();
    float zp[(ROWS_MAX * MEG_KMAX + NT - 1) / NT];
    int c = 0;
    for (int idx = tid; idx < nr * k; idx += NT, ++c) {
        const int q = idx / k, j = idx % k;
        dw a2 = {sB[idx], 0.f};
        float lo = 0.f;
        for (int l = 0; l < k; ++l) {
            const float w = sA[q * k + l];
            dot2_acc(a2, -w, Cc[l * k + j].hi);
            lo = fmaf(-w, Cc[l * k + j].lo, lo);
        }
        zp[c] = a2.hi + (a2.lo + lo);
    }
    __syncthreads();                                    // every row of Z is read
    c = 0;
    for (int idx = tid; idx < nr * k; idx += NT, ++c) {
        sB[idx] = zp[c];
        Z[(size_t)row0 * k + idx] = zp[c];
    }
    __syncthreads();
    const int nsym = k * (k + 1) / 2;
    for (int e = tid; e < nsym; e += NT) {
        int i, j;
        tri_decode(e, i, j);
        Acc<float> a, b;
        a.zero();
        b.zero();
        int q = 0;
        for (; q + 1 < nr; q += 2) {
            a.add_prod(sB[q * k + i], sB[q * k + j]);
            b.add_prod(sB[(q + 1) * k + i], sB[(q + 1) * k + j]);
        }
        if (q < nr) a.add_prod(sB[q * k + i], sB[q * k + j]);
        dw r0 = a.as_dw();
        dw_add(r0, b.as_dw());
        ent[e] = r0;
    }
    __syncthreads();
    write_partial(s, lb, ent, nsym);
}

// ==========================================================================
// orth pass of the block Krylov iteration (float storage), per row block:
//   PH_KRY1: W1 = Z' M (Z' = Z - W0 C from the projection pass, M its refined
//     CholeskyQR factor), exact products; W0 moves to Wp and W1 becomes the
//     current block W; the bf16 split of W1 for the second product; Gram
//     entries W1^T W1, V^T W1, W0^T W1.
//   PH_KRY2: V_{t+1} = [W0 W1] QV (exact products, float64 result) and the
//     next block W = [W0 W1] QW; its bf16 split; Gram entries W^T W and
//     V_{t+1}^T W for the next iteration (as k_orth's final phase).
__global__ void __launch_bounds__(NT) k_orth_kry(const SolveDev* sds, int ns, int phase) {
    pdl_wait();
    pdl_trigger();
    const int si = find_solve(sds, ns, PK_RED, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_RED];     // blocks past nb_red pad the last cluster
    const int n = s.n, k = s.k, r = s.r, tid = threadIdx.x;
    const int row0 = min(n, lb * s.rows_red), row1 = min(n, row0 + s.rows_red), nr = row1 - row0;
    const bool kry1 = (phase == PH_KRY1);
    extern __shared__ __align__(16) unsigned char smraw[];
    Coef<float>* A1 = (Coef<float>*)smraw;             // KRY1: M (k x k)   KRY2: QW (2k x k)
    Coef<float>* A2 = A1 + MEG_KMAX * MEG_KMAX;         //                   KRY2: QV (2k x r)
    float* sA = (float*)(A2 + MEG_KMAX * MEG_KMAX);     // rows of W0
    float* sB = sA + ROWS_MAX * MEG_KMAX;               // rows of Z (KRY1) / W1 (KRY2)
    float* sC = sB + ROWS_MAX * MEG_KMAX;               // rows of the new block
    float* sVh = sC + ROWS_MAX * MEG_KMAX;              // V as (hi, lo) floats
    float* sVl = sVh + ROWS_MAX * MEG_RMAX;
    dw* ent = (dw*)(sVl + ROWS_MAX * MEG_RMAX);
    const double* sm = s.sm;
    float* W = (float*)s.W;
    float* Wp = (float*)s.Wp;
    if (kry1) {
        for (int e = tid; e < k * k; e += NT) A1[e].set(sm[SM_M1 + (e / k) * 32 + e % k]);
    } else {
        for (int e = tid; e < 2 * k * k; e += NT) A1[e].set(sm[SM_QW + (e / k) * 32 + e % k]);
        for (int e = tid; e < 2 * k * r; e += NT) A2[e].set(sm[SM_QV + (e / r) * 32 + e % r]);
    }
    const float* Z = (const float*)s.Z;
    for (int idx = tid; idx < nr * k; idx += NT) {
        if (kry1) {
            sA[idx] = W[(size_t)row0 * k + idx];
            sB[idx] = Z[(size_t)row0 * k + idx];
        } else {
            sA[idx] = Wp[(size_t)row0 * k + idx];
            sB[idx] = W[(size_t)row0 * k + idx];
        }
    }
    __syncthreads();
    double* V = s.V;
    if (!kry1) {
        // V_{t+1} = W0 QV[:k] + W1 QV[k:], exact products, float64 result
        for (int idx = tid; idx < nr * r; idx += NT) {
            const int q = idx / r, j = idx % r;
            dw acc = {0.f, 0.f};
            for (int l = 0; l < k; ++l) {
                const float w0 = sA[q * k + l], w1 = sB[q * k + l];
                dot2_acc(acc, w0, A2[l * r + j].hi);
                dot2_acc(acc, w0, A2[l * r + j].lo);
                dot2_acc(acc, w1, A2[(k + l) * r + j].hi);
                dot2_acc(acc, w1, A2[(k + l) * r + j].lo);
            }
            V[(size_t)row0 * r + idx] = dw_value(acc);
        }
    }
    // the new block, exact products over the high parts, low parts in float
    for (int idx = tid; idx < nr * k; idx += NT) {
        const int q = idx / k, j = idx % k;
        dw a2 = {0.f, 0.f};
        float lo = 0.f;
        for (int l = 0; l < k; ++l) {
            const float x0 = sA[q * k + l], x1 = sB[q * k + l];
            if (kry1) {                         // Z' M
                dot2_acc(a2, x1, A1[l * k + j].hi);
                lo = fmaf(x1, A1[l * k + j].lo, lo);
            } else {                            // W0 QW[:k] + W1 QW[k:]
                dot2_acc(a2, x0, A1[l * k + j].hi);
                lo = fmaf(x0, A1[l * k + j].lo, lo);
                dot2_acc(a2, x1, A1[(k + l) * k + j].hi);
                lo = fmaf(x1, A1[(k + l) * k + j].lo, lo);
            }
        }
        const float w = a2.hi + (a2.lo + lo);
        sC[idx] = w;
        W[(size_t)row0 * k + idx] = w;
        if (kry1) Wp[(size_t)row0 * k + idx] = sA[idx];
    }
    __syncthreads();
    // V (the current one for KRY1, V_{t+1} for KRY2) as (hi, lo) floats
    for (int idx = tid; idx < nr * r; idx += NT) {
        const double v = V[(size_t)row0 * r + idx];
        const float vh = (float)v;
        sVh[idx] = vh;
        sVl[idx] = (float)(v - (double)vh);
    }
    if (s.Wsp) {
        // exact split W = hi + mid + lo in bf16, K-major, for the tensor-core product
        const size_t kp = (size_t)s.tc_kpad;
        const size_t P = (size_t)(s.tc_npad / 3);
        for (int idx = tid; idx < nr * k; idx += NT) {
            const int j = idx / nr, q = idx % nr, i = row0 + q;
            const float w = sC[q * k + j];
            const __nv_bfloat16 hi = __float2bfloat16_rn(w);
            const float r1 = w - __bfloat162float(hi);
            const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
            const float r2 = r1 - __bfloat162float(mid);
            const __nv_bfloat16 lo = __float2bfloat16_rn(r2);
            s.Wsp[(size_t)j * kp + i] = __bfloat16_as_ushort(hi);
            s.Wsp[(P + j) * kp + i] = __bfloat16_as_ushort(mid);
            s.Wsp[(2 * P + j) * kp + i] = __bfloat16_as_ushort(lo);
        }
    }
    __syncthreads();
    const int nsym = k * (k + 1) / 2;
    const int E = nsym + r * k + (kry1 ? k * k : 0);
    for (int e = tid; e < E; e += NT) {
        Acc<float> a;
        a.zero();
        if (e < nsym) {
            int i, j;
            tri_decode(e, i, j);
            for (int q = 0; q < nr; ++q) a.add_prod(sC[q * k + i], sC[q * k + j]);
        } else if (e < nsym + r * k) {
            const int l = (e - nsym) / k, j = (e - nsym) % k;
            float lo = 0.f;
            for (int q = 0; q < nr; ++q) {
                const float w = sC[q * k + j];
                a.add_prod(sVh[q * r + l], w);
                lo = fmaf(sVl[q * r + l], w, lo);
            }
            dw r0 = a.as_dw();
            dw_add(r0, dw{lo, 0.f});
            ent[e] = r0;
            continue;
        } else {
            const int f = e - nsym - r * k, i = f / k, j = f % k;     // (W0^T W1)_ij
            for (int q = 0; q < nr; ++q) a.add_prod(sA[q * k + i], sC[q * k + j]);
        }
        ent[e] = a.as_dw();
    }
    __syncthreads();
    write_partial(s, lb, ent, E);
}

// ==========================================================================
// island after orth2: G = W^T W and U = V^T W from the partials.
template <typename T>
__global__ void __launch_bounds__(NT) k_island_o2(const SolveDev* sds, int ns, int phase) {
    pdl_wait();
    pdl_trigger();
    const int si = blockIdx.x;
    if (si >= ns) return;
    const SolveDev& s = sds[si];
    const int k = s.k, r = s.r, tid = threadIdx.x;
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int FBYTES = 4 * 32 * MEG_LDK * (int)sizeof(float);
    dw* ent = (dw*)(smraw + FBYTES);
    const int nsym = k * (k + 1) / 2;
    const bool kry1 = (phase == PH_KRY1);          // block Krylov: also W0^T W1
    const int E = nsym + r * k + (kry1 ? k * k : 0);
    reduce_partials(s, ent, E, (dw*)smraw, FBYTES / (int)sizeof(dw));
    double* smw = s.sm;
    for (int e = tid; e < nsym; e += NT) {
        int i, j;
        tri_decode(e, i, j);
        double v = dw_value(ent[e]);
        smw[SM_G + i * 32 + j] = v;
        smw[SM_G + j * 32 + i] = v;
    }
    for (int e = tid; e < r * k; e += NT) smw[SM_U + (e / k) * 32 + e % k] = dw_value(ent[nsym + e]);
    if (kry1)
        for (int e = tid; e < k * k; e += NT) smw[SM_G01 + (e / k) * 32 + e % k] = dw_value(ent[nsym + r * k + e]);
}

// ==========================================================================
// Dense gradient part: Ys[split] = D[:, Ks] W[Ks, :]  (FFMA, T = double/float).
// 64-row tiles, K tiles of 32, k <= 32 columns; each split of K writes its
// own partial (summed in k_combine).
template <typename T> __device__ __forceinline__ T load_d(const void* D, size_t idx, int prec) {
    if (prec == MEG_MIXED_BF16) {
        unsigned short b = ((const unsigned short*)D)[idx];
        return (T)__uint_as_float(((unsigned)b) << 16);
    }
    return ((const T*)D)[idx];
}

template <typename T, typename TD> __device__ __forceinline__ T load_dt(const TD* D, size_t idx) {
    return (T)D[idx];
}
template <> __device__ __forceinline__ float load_dt<float, unsigned short>(const unsigned short* D, size_t idx) {
    return __uint_as_float(((unsigned)D[idx]) << 16);
}

template <typename T, typename TD>
__global__ void __launch_bounds__(NT) k_dense(const SolveDev* sds, int ns) {
    pdl_wait();
    pdl_trigger();
    const int si = find_solve(sds, ns, PK_DENSE, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_DENSE];
    if (lb < 0 || lb >= s.nb_dm * s.nb_ds) return;
    const int n = s.n, k = s.k, tid = threadIdx.x;
    const int mt = lb % s.nb_dm, sp = lb / s.nb_dm;
    const int m0 = mt * 64;
    const int k0 = sp * s.ks_len, k1 = min(n, k0 + s.ks_len);
    __shared__ T Ds[32][64 + 1];
    __shared__ __align__(16) T Ws[32][32];
    const TD* D = (const TD*)s.D;
    const T* W = (const T*)s.W;
    const int ty = tid >> 3, tx = tid & 7;     // rows ty, ty+32; cols 4 tx .. 4 tx + 3
    T acc[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    for (int kb = k0; kb < k1; kb += 32) {
        for (int e = tid; e < 64 * 32; e += NT) {
            int row = e >> 5, col = e & 31;
            int gi = m0 + row, gk = kb + col;
            Ds[col][row] = (gi < n && gk < k1) ? load_dt<T, TD>(D, (size_t)gi * n + gk) : (T)0;
        }
        for (int e = tid; e < 32 * 32; e += NT) {
            int kk = e >> 5, c = e & 31;
            int gk = kb + kk;
            Ws[kk][c] = (gk < k1 && c < k) ? W[(size_t)gk * k + c] : (T)0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            T d0 = Ds[kk][ty], d1 = Ds[kk][ty + 32];
            T w0 = Ws[kk][4 * tx], w1 = Ws[kk][4 * tx + 1], w2 = Ws[kk][4 * tx + 2], w3 = Ws[kk][4 * tx + 3];
            acc[0][0] += d0 * w0; acc[0][1] += d0 * w1; acc[0][2] += d0 * w2; acc[0][3] += d0 * w3;
            acc[1][0] += d1 * w0; acc[1][1] += d1 * w1; acc[1][2] += d1 * w2; acc[1][3] += d1 * w3;
        }
        __syncthreads();
    }
    T* Ys = (T*)s.Ys + (size_t)sp * n * k;
    for (int a = 0; a < 2; ++a) {
        int gi = m0 + ty + 32 * a;
        if (gi >= n) continue;
        for (int b = 0; b < 4; ++b) {
            int c = 4 * tx + b;
            if (c < k) Ys[(size_t)gi * k + c] = acc[a][b];
        }
    }
}

// ==========================================================================
// CSR gradient part (matrix completion): Y = P_Omega(X - M) W, the residual
// R_ij = X_ij - M_ij formed on the fly from the factors (never stored).
// One warp per row.  Also sum of R_ij^2 (for the shift bound of the next
// iteration), reduced deterministically through per-block partials.
// Float rows [V_j | W_j] for the sparse product of the float-storage modes,
// each part padded to a multiple of 4 floats (16-byte slots: a row is
// pad4(r)/4 + pad4(k)/4 vector loads), in the solve's scratch after the
// row-block maxima.
__host__ __device__ __forceinline__ int csr_pad4(int x) { return (x + 3) & ~3; }
constexpr int CSR_CAP = 256;        // entries of a row staged at a time (per warp)
__device__ __forceinline__ float* csr_vw(const SolveDev& s) { return (float*)(s.meas + ((s.nb_csr + 1) & ~1)); }

// One row i of the sparse product in float64 storage, KB = k_bucket(k) >= k > r:
// each lane takes every 32nd stored entry (i, j) of the row, forms R = X_ij -
// M_ij from the gathered row j of V and adds R W[j][:] into its own k running
// sums; the warp then sums the lanes' vectors.  Returns sum_j |R_ij| (on
// every lane).
template <typename T, int KB>
__device__ __forceinline__ double csr_row(const SolveDev& s, int i, const double* coef, int lane) {
    const int r = s.r, k = s.k;
    const T* val = (const T*)s.val;
    T vi[KB], z[KB];
#pragma unroll
    for (int l = 0; l < KB; ++l) {
        // V_il (mu_l - s) formed in float64 and rounded once: the rounding errors are
        // independent across (i, l) instead of a shared error in (mu_l - s)
        vi[l] = l < r ? (T)(s.V[(size_t)i * r + l] * coef[l]) : (T)0;
        z[l] = 0;
    }
    const T sd = (T)coef[MEG_RMAX];
    double rabs = 0.0;
    const int b = s.rowptr[i], e = s.rowptr[i + 1];
#pragma unroll 2
    for (int p = b + lane; p < e; p += 32) {
        const int j = s.col[p];
        T x = (j == i) ? sd : (T)0;
        T R;
        {
            const T* vj = (const T*)s.V + (size_t)j * r;
#pragma unroll
            for (int l = 0; l < KB; ++l)
                if (l < r) x += vi[l] * vj[l];
            R = x - val[p];
            const T* wj = (const T*)s.W + (size_t)j * k;
#pragma unroll
            for (int c = 0; c < KB; ++c)
                if (c < k) z[c] += R * wj[c];
        }
        rabs += fabs((double)R);
    }
    T mine = 0;
#pragma unroll
    for (int c = 0; c < KB; ++c)
        if (c < k) {
            T v = z[c];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == c) mine = v;
        }
    if (lane < k) ((T*)s.Y)[(size_t)i * k + lane] = mine;
    for (int o = 16; o > 0; o >>= 1) rabs += __shfl_xor_sync(0xffffffffu, rabs, o);
    return rabs;
}

// One row i of the sparse product in float storage.  The warp's lanes form
// groups of GS; a group takes one stored entry (i, j) at a time, each of its
// lanes one 16-byte slot of the padded row [V_j | W_j] (vs slots of V, ws of
// W), so that each lane holds a few registers and a warp keeps 32/GS entries
// (two per group, unrolled) of gathers in flight: the product is bound by the
// latency of these L2 gathers.  The V lanes form partial dots with their
// slot of V_i (mu - s); the group adds them (shuffles), R = X_ij - M_ij, and
// the W lanes add R W_j into their slot's running sums.  The groups' sums are
// added at the end (fixed shuffle order).  Returns sum_j |R_ij| (every lane).
template <int GS>
__device__ __forceinline__ double csr_row_coop(const SolveDev& s, int i, const double* coef, int lane, int* scol,
                                               float* sval) {
    const int r = s.r, k = s.k, vs = csr_pad4(r) / 4, ws = csr_pad4(k) / 4, rw = vs + ws;
    constexpr int NG = 32 / GS, U = 4;                       // groups per warp, entries per group and step
    const int g = lane / GS, l = lane % GS;
    const float4* F = (const float4*)csr_vw(s);
    const float* val = (const float*)s.val;
    float4 vi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (l < vs) {
        float t[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int idx = 4 * l + c;
            // V_il (mu_l - s) formed in float64 and rounded once
            t[c] = idx < r ? (float)(s.V[(size_t)i * r + idx] * coef[idx]) : 0.f;
        }
        vi = make_float4(t[0], t[1], t[2], t[3]);
    }
    const float sd = (float)coef[MEG_RMAX];
    const bool vlane = l < vs, wlane = l >= vs && l < rw;
    float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    float rabs = 0.f;
    const int b = s.rowptr[i], e = s.rowptr[i + 1];
    // the row in pieces of CSR_CAP entries: indices and values staged in the
    // warp's shared buffer with all loads in flight at once, then the gathers
    // of [V_j | W_j], U per group and step (independent loads); every loop
    // bound is warp-uniform, so the shuffles always have the whole warp
    for (int cb = b; cb < e; cb += CSR_CAP) {
        const int cn = min(CSR_CAP, e - cb);
        __syncwarp();
        for (int q = lane; q < cn; q += 32) {
            scol[q] = s.col[cb + q];
            sval[q] = val[cb + q];
        }
        __syncwarp();
        for (int pb = 0; pb < cn; pb += U * NG) {
            int j[U];
            float4 f[U];
            float x[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = pb + u * NG + g;
                j[u] = q < cn ? scol[q] : -1;
                f[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (j[u] >= 0 && l < rw) f[u] = F[(size_t)j[u] * rw + l];
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                x[u] = vlane ? vi.x * f[u].x + vi.y * f[u].y + vi.z * f[u].z + vi.w * f[u].w : 0.f;
#pragma unroll
            for (int o = GS / 2; o > 0; o >>= 1)
#pragma unroll
                for (int u = 0; u < U; ++u) x[u] += __shfl_xor_sync(0xffffffffu, x[u], o);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = pb + u * NG + g;
                if (j[u] == i) x[u] += sd;
                const float R = j[u] >= 0 ? x[u] - sval[q] : 0.f;
                if (wlane) {
                    z.x += R * f[u].x; z.y += R * f[u].y; z.z += R * f[u].z; z.w += R * f[u].w;
                }
                if (l == 0) rabs += fabsf(R);
            }
        }
    }
#pragma unroll
    for (int o = GS; o < 32; o <<= 1) {
        z.x += __shfl_xor_sync(0xffffffffu, z.x, o);
        z.y += __shfl_xor_sync(0xffffffffu, z.y, o);
        z.z += __shfl_xor_sync(0xffffffffu, z.z, o);
        z.w += __shfl_xor_sync(0xffffffffu, z.w, o);
    }
    if (g == 0 && wlane) {
        float* Y = (float*)s.Y + (size_t)i * k;
        const int c0 = 4 * (l - vs);
        const float zz[4] = {z.x, z.y, z.z, z.w};
#pragma unroll
        for (int c = 0; c < 4; ++c)
            if (c0 + c < k) Y[c0 + c] = zz[c];
    }
    for (int o = 16; o > 0; o >>= 1) rabs += __shfl_xor_sync(0xffffffffu, rabs, o);
    return (double)rabs;
}

// The padded float rows of V and W for the block's rows (one pass per product).
__global__ void __launch_bounds__(NT) k_csr_prep(const SolveDev* sds, int ns) {
    pdl_wait();
    pdl_trigger();
    const int si = find_solve(sds, ns, PK_CSR, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_CSR];
    if (lb < 0 || lb >= s.nb_csr) return;
    const int r = s.r, k = s.k, rs = csr_pad4(r), ks = csr_pad4(k), w = rs + ks;
    const int row0 = lb * (NT / 32), nr = min(NT / 32, s.n - row0);
    float* F = csr_vw(s);
    const float* W = (const float*)s.W;
    for (int e = threadIdx.x; e < nr * w; e += NT) {
        const int q = e / w, c = e % w, i = row0 + q;
        float x = 0.f;
        if (c < rs) { if (c < r) x = (float)s.V[(size_t)i * r + c]; }
        else if (c - rs < k) x = W[(size_t)i * k + (c - rs)];
        F[(size_t)i * w + c] = x;
    }
}

// Matrix completion: Y = P_Omega(X - M) W, fused (the residual of each stored
// entry is formed on the fly and never stored), one warp per row; also the
// row abs-sums of the residual, whose maximum bounds ||P_Omega(X - M)||_2.
template <typename T>
__global__ void __launch_bounds__(NT) k_csr(const SolveDev* sds, int ns) {
    pdl_wait();
    pdl_trigger();
    const int si = find_solve(sds, ns, PK_CSR, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_CSR];
    if (lb < 0 || lb >= s.nb_csr) return;
    const int n = s.n, r = s.r;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = lb * (NT / 32) + warp;
    __shared__ double coef[MEG_RMAX + 1];
    __shared__ double wsum[NT / 32];
    const bool warm = (s.mode == 1);
    if (threadIdx.x < r) coef[threadIdx.x] = warm ? 0.0 : s.sm[SM_MU + threadIdx.x] - s.sm[SM_S];
    if (threadIdx.x == 0) coef[MEG_RMAX] = warm ? 0.0 : s.sm[SM_S];
    __syncthreads();
    double rabs = 0.0;        // sum_j |R_ij| of this row: ||P_Omega(X - M)||_2 <= max_i of it
    if (i < n) {
        if constexpr (sizeof(T) == 4) {
            __shared__ int scol[NT / 32][CSR_CAP];
            __shared__ float sval[NT / 32][CSR_CAP];
            // 16-byte slots of [V_j | W_j]: at most 8 -> groups of 8 lanes, else 16
            if (csr_pad4(r) / 4 + csr_pad4(s.k) / 4 <= 8)
                rabs = csr_row_coop<8>(s, i, coef, lane, scol[warp], sval[warp]);
            else
                rabs = csr_row_coop<16>(s, i, coef, lane, scol[warp], sval[warp]);
        } else {
            switch (k_bucket(s.k)) {
                case 8: rabs = csr_row<T, 8>(s, i, coef, lane); break;
                case 16: rabs = csr_row<T, 16>(s, i, coef, lane); break;
                default: rabs = csr_row<T, 32>(s, i, coef, lane); break;
            }
        }
    }
    if (lane == 0) wsum[warp] = rabs;
    __syncthreads();
    __shared__ int am_last;
    double* pr = s.meas;                      // CSR kinds use the scratch for row-block maxima
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < NT / 32; ++w) t = fmax(t, wsum[w]);
        pr[lb] = t;
        __threadfence();
        unsigned* c = s.ctr + (s.nb_red + RED_GROUP - 1) / RED_GROUP + 1;
        am_last = (atomicAdd(c, 1u) == (unsigned)(s.nb_csr - 1));
        if (am_last) *c = 0u;
    }
    __syncthreads();
    if (!am_last) return;
    // last block: the maximum over every block, all threads (a max is order-free)
    __shared__ double red[NT];
    double t = 0.0;
    for (int q = threadIdx.x; q < s.nb_csr; q += NT) t = fmax(t, __ldcg(pr + q));
    red[threadIdx.x] = t;
    __syncthreads();
    for (int h = NT / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + h]);
        __syncthreads();
    }
    if (threadIdx.x == 0) s.sm[SM_RSS] = red[0];
}

// ==========================================================================
// Measurement objective.  Minibatch of step t: L indices drawn with
// replacement by SplitMix64 (index j: splitmix64(seed + (t L + j + 1) gamma)
// mod m); mode 1 (warm start) uses every measurement once.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

template <typename T> __device__ __forceinline__ T load_a(const void* A, size_t idx);
template <> __device__ __forceinline__ double load_a<double>(const void* A, size_t idx) {
    return ((const double*)A)[idx];
}
template <> __device__ __forceinline__ float load_a<float>(const void* A, size_t idx) {
    unsigned short b = ((const unsigned short*)A)[idx];
    return __uint_as_float(((unsigned)b) << 16);
}

// Minibatch pass over MB_ROWS batch rows b per block:
//   r_b = a_b^T X a_b - y_b (mode 0) or -y_b (mode 1, the warm start's
//   -grad f(0)), ||a_b||^2 and T_b = a_b^T W (k values).
// The block computes the small product [a_b rows] x [V | W] (2B columns, B =
// k_bucket(k) >= k > r, zero columns beyond r and k) in tiles of MB_TILE
// elements: the tile of the gathered rows of A and the tile of V (converted
// to the storage type) and W are staged in shared memory; thread (row,
// column group) accumulates C/8 consecutive columns of one row, so a staged
// value of V/W serves four rows by broadcast and no cross-lane reduction is
// needed.  The last block of the solve turns the per-block partial bounds
// into the shift bound.
template <typename T, int B>
__device__ __forceinline__ void meas_batch_tile(const SolveDev& s, int lb, bool warm, const int64_t* sidx,
                                                T* As, T* Xs, double (&out)[B / 4], T& aa) {
    constexpr int C = 2 * B, CPT = C / 8;               // columns, columns per thread
    constexpr int TL = sizeof(T) == 8 ? MB_TILE / 2 : MB_TILE, EPT = TL / 8;   // elements per tile / thread
    constexpr int LDA = TL + 1, LDX = C + 1;
    const int n = s.n, k = s.k, r = s.r, tid = threadIdx.x;
    const int row = tid >> 3, c0 = (tid & 7) * CPT;
    const int Lb = s.nb_meas;
    const double* V = s.V;
    const T* W = (const T*)s.W;
    const int b0 = lb * MB_ROWS;
    T acc[CPT];
#pragma unroll
    for (int j = 0; j < CPT; ++j) acc[j] = 0;
    for (int i0 = 0; i0 < n; i0 += TL) {
        const int tn = min(TL, n - i0);
        __syncthreads();
        {   // rows of A: thread (row, EPT consecutive elements); ||a||^2 on the way
            const int e0 = (tid & 7) * EPT;
            const bool live = b0 + row < Lb;
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                T a = 0;
                if (live && e0 + e < tn) a = load_a<T>(s.A, (size_t)sidx[row] * n + i0 + e0 + e);
                As[row * LDA + e0 + e] = a;
                aa += a * a;
            }
        }
        for (int e = tid; e < tn * C; e += NT) {
            const int j = e / C, c = e % C;
            T x = 0;
            if (c < B) { if (!warm && c < r) x = (T)V[(size_t)(i0 + j) * r + c]; }
            else if (c - B < k) x = W[(size_t)(i0 + j) * k + (c - B)];
            Xs[j * LDX + c] = x;
        }
        __syncthreads();
        for (int i = 0; i < tn; ++i) {
            const T a = As[row * LDA + i];
#pragma unroll
            for (int j = 0; j < CPT; ++j) acc[j] += a * Xs[i * LDX + c0 + j];
        }
    }
#pragma unroll
    for (int j = 0; j < CPT; ++j) out[j] = (double)acc[j];
    // the eight threads of a row hold pieces of ||a||^2 (consecutive lanes)
    for (int o = 4; o > 0; o >>= 1) aa += __shfl_xor_sync(0xffffffffu, aa, o);
}

// Second half of the minibatch pass, for the MB_ROWS batch rows of block lb
// whose products Ps[row] = [a_b^T V (B columns) | a_b^T W (B columns) | ||a_b||^2]
// are in shared memory: residuals r_b = a_b^T X a_b - y_b, ||a_b||^2, T_b =
// a_b^T W and the indices to the solve's scratch, and the shift bound (the
// last block of the solve combines the per-block parts in a fixed order).
__device__ void meas_batch_tail(const SolveDev& s, int lb, bool warm, const int64_t* sidx,
                                double (*Ps)[2 * MEG_KMAX + 1]) {
    const int n = s.n, k = s.k, r = s.r, tid = threadIdx.x;
    const int Lb = s.nb_meas, nblk = (Lb + MB_ROWS - 1) / MB_ROWS;
    const int B = k_bucket(k);
    double* sc = s.meas;              // [Lb] residual, [Lb] ||a||^2, [Lb x 32] T_b, [nblk] bounds
    // T_b: one thread per (row, column)
    for (int e = tid; e < MB_ROWS * k; e += NT) {
        const int rr = e / k, c = e % k, b = lb * MB_ROWS + rr;
        if (b < Lb) sc[2 * (size_t)Lb + (size_t)b * MEG_KMAX + c] = Ps[rr][B + c];
    }
    __shared__ double bsum;
    __shared__ float srs[MB_ROWS];
    static_assert(MB_ROWS == 32, "one warp per block's rows");
    if (tid < MB_ROWS) {
        const int b = lb * MB_ROWS + tid;
        double contrib = 0.0;
        srs[tid] = 0.f;
        if (b < Lb) {
            const double aav = Ps[tid][2 * MEG_KMAX];
            const double sv = warm ? 0.0 : s.sm[SM_S];
            double q = sv * aav;
            if (!warm)
                for (int l = 0; l < r; ++l) q += (s.sm[SM_MU + l] - sv) * Ps[tid][l] * Ps[tid][l];
            const double res = q - s.y[sidx[tid]];
            sc[b] = res;
            sc[Lb + b] = aav;
            if (!warm) s.bidx[b] = (int)sidx[tid];
            srs[tid] = (2.f / (float)Lb) * (float)res;   // S_b = srs T_b for the tensor-core apply pass
            // Minibatch (mode 0): the spectral size of (2/L) sum r_b a_b a_b^T is
            // estimated as for a weighted Wishart matrix,
            //   (2/L) rms_b(|r_b| ||a_b||^2) (1 + sqrt(L/n))^2.
            // It only sets the shift c, whose job is to centre the bulk of M_t near
            // log s: the top-r eigenvalues sit log(mu_r / s) (about 10) above it, far
            // beyond the gradient's spread, so a direction the estimate misses (one
            // large residual) only converges more slowly.  Rayleigh-Ritz is exact.
            // Warm start (mode 1, r_b = -y_b): lambda_min(-grad f(0)) >= -(2/m) sum_{y<0} |y| ||a||^2.
            contrib = warm ? (res > 0.0 ? res * aav : 0.0) : (res * aav) * (res * aav);
        }
        for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
        if (tid == 0) bsum = contrib;
    }
    __syncthreads();
    if (s.mtc) {
        // the block's 32 rows of S (0 past the batch) as 16-byte pieces of the image
        __shared__ float Sx[MB_ROWS][MEG_KMAX + 1];
        for (int e = tid; e < MB_ROWS * k; e += NT) {
            const int rr = e / k, c = e % k;
            Sx[rr][c] = srs[rr] * (float)Ps[rr][B + c];
        }
        __syncthreads();
        mts_put32(s.mts, k, (int64_t)lb * MB_ROWS, &Sx[0][0], MEG_KMAX + 1);
    }
    __shared__ int am_last;
    if (tid == 0) {
        const double v = bsum;
        sc[(size_t)Lb * (2 + MEG_KMAX) + lb] = v;
        __threadfence();
        unsigned* c = s.ctr + (s.nb_red + RED_GROUP - 1) / RED_GROUP + 2;
        am_last = (atomicAdd(c, 1u) == (unsigned)(nblk - 1));
        if (am_last) *c = 0u;
    }
    __syncthreads();
    if (!am_last) return;
    // last block: combine the per-block bounds (fixed order per thread, then a fixed tree)
    __shared__ double red[NT];
    const double* bp = sc + (size_t)Lb * (2 + MEG_KMAX);
    double v = 0.0;
    for (int q2 = tid; q2 < nblk; q2 += NT) v += __ldcg(bp + q2);
    red[tid] = v;
    __syncthreads();
    for (int h = NT / 2; h > 0; h >>= 1) {
        if (tid < h) red[tid] = red[tid] + red[tid + h];
        __syncthreads();
    }
    if (tid == 0) {
        // an estimate that only centres the shift: float arithmetic (a float64
        // square root or division costs thousands of cycles on GB300)
        const float sum = (float)red[0], fL = (float)Lb;
        float bound;
        if (warm) {
            bound = sum * (2.f / fL);
        } else {
            const float f = 1.f + sqrtf(fL / (float)n);
            bound = (2.f / fL) * sqrtf(sum / fL) * f * f;
        }
        s.sm[SM_RESID_BOUND] = (double)bound;
    }
}

template <typename T>
__global__ void __launch_bounds__(NT) k_meas_batch(const SolveDev* sds, int ns) {
    pdl_wait();
    pdl_trigger();
    const int si = find_solve(sds, ns, PK_MEAS, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_MEAS];
    const int Lb = s.nb_meas, nblk = (Lb + MB_ROWS - 1) / MB_ROWS;
    if (lb < 0 || lb >= nblk || s.mtc) return;              // tensor-core members: k_meas_tc_batch
    const int n = s.n, k = s.k, r = s.r, tid = threadIdx.x;
    const bool warm = (s.mode == 1);
    __shared__ int64_t sidx[MB_ROWS];
    if (tid < MB_ROWS) {
        const int b = lb * MB_ROWS + tid;
        int64_t idx = 0;
        if (b < Lb)
            idx = warm ? (int64_t)b
                       : (int64_t)(splitmix64(s.seed + ((uint64_t)s.sm[SM_T] * (uint64_t)s.L + (uint64_t)b + 1ull) *
                                                           0x9E3779B97F4A7C15ull) %
                                   (uint64_t)s.m);
        sidx[tid] = idx;
    }
    // shared tiles: rows of A (MB_ROWS x (MB_TILE+1)), V|W (MB_TILE x (2*32+1)), products
    constexpr int TL = sizeof(T) == 8 ? MB_TILE / 2 : MB_TILE;
    __shared__ T As[MB_ROWS * (TL + 1)];
    __shared__ T Xs[TL * (2 * MEG_KMAX + 1)];
    __shared__ double Ps[MB_ROWS][2 * MEG_KMAX + 1];
    __syncthreads();
    const int row = tid >> 3;
    T aa = 0;
    switch (k_bucket(k)) {
        case 8: {
            double out[2];
            meas_batch_tile<T, 8>(s, lb, warm, sidx, As, Xs, out, aa);
            for (int j = 0; j < 2; ++j) Ps[row][(tid & 7) * 2 + j] = out[j];
            if ((tid & 7) == 0) Ps[row][2 * MEG_KMAX] = (double)aa;
            break;
        }
        case 16: {
            double out[4];
            meas_batch_tile<T, 16>(s, lb, warm, sidx, As, Xs, out, aa);
            for (int j = 0; j < 4; ++j) Ps[row][(tid & 7) * 4 + j] = out[j];
            if ((tid & 7) == 0) Ps[row][2 * MEG_KMAX] = (double)aa;
            break;
        }
        default: {
            double out[8];
            meas_batch_tile<T, 32>(s, lb, warm, sidx, As, Xs, out, aa);
            for (int j = 0; j < 8; ++j) Ps[row][(tid & 7) * 8 + j] = out[j];
            if ((tid & 7) == 0) Ps[row][2 * MEG_KMAX] = (double)aa;
            break;
        }
    }
    __syncthreads();
    meas_batch_tail(s, lb, warm, sidx, Ps);
}

// Second half of the minibatch pass of the tensor-core members: the parts of
// the batch pass (k_meas_tc_batch: 2B products and ||a_b||^2 per row and part)
// are added in part order, then meas_batch_tail as for the CUDA-core pass.
__global__ void __launch_bounds__(NT) k_meas_finish(const SolveDev* sds, int ns) {
    pdl_wait();
    pdl_trigger();
    const int si = find_solve(sds, ns, PK_MEAS, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_MEAS];
    const int Lb = s.nb_meas, nblk = (Lb + MB_ROWS - 1) / MB_ROWS;
    if (lb < 0 || lb >= nblk || !s.mtc || s.kind != MEG_MEAS_STOCH) return;
    const int tid = threadIdx.x;
    const bool warm = (s.mode == 1);
    const int B = k_bucket(s.k), NC = 2 * B, KS = meas_ks(Lb, s.n);
    __shared__ int64_t sidx[MB_ROWS];
    __shared__ double Ps[MB_ROWS][2 * MEG_KMAX + 1];
    if (tid < MB_ROWS) {
        const int b = lb * MB_ROWS + tid;
        int64_t idx = 0;
        if (b < Lb)
            idx = warm ? (int64_t)b
                       : (int64_t)(splitmix64(s.seed + ((uint64_t)s.sm[SM_T] * (uint64_t)s.L + (uint64_t)b + 1ull) *
                                                           0x9E3779B97F4A7C15ull) %
                                   (uint64_t)s.m);
        sidx[tid] = idx;
    }
    // each entry adds its KS parts in part order; the parts of an entry are
    // contiguous ([row][column][part]): with KS a multiple of 4 they are read
    // as 16-byte vectors, all in flight together (one L2 round trip)
    for (int e = tid; e < MB_ROWS * (NC + 1); e += NT) {
        const int rr = e / (NC + 1), c = e % (NC + 1), b = lb * MB_ROWS + rr;
        float acc = 0.f;
        if (b < Lb) {
            const float* p0 = s.mtp + ((size_t)b * (NC + 1) + c) * KS;
            if ((KS & 3) == 0) {
                float4 v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (4 * u < KS) v[u] = __ldcg((const float4*)p0 + u);
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (4 * u < KS) acc = (((acc + v[u].x) + v[u].y) + v[u].z) + v[u].w;
            } else {
                for (int p = 0; p < KS; ++p) acc += __ldcg(p0 + p);
            }
        }
        Ps[rr][c == NC ? 2 * MEG_KMAX : c] = (double)acc;
    }
    __syncthreads();
    meas_batch_tail(s, lb, warm, sidx, Ps);
}

// c_i = a_i^T b_i of the bilinear pairs (bf16 products are exact in float;
// sums in float64), one warp per pair, into meas[i].
__global__ void __launch_bounds__(NT) k_bil_prep(const SolveDev* sd, int64_t m) {
    const SolveDev& s = *sd;
    const int n = s.n, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (NT / 32) + (threadIdx.x >> 5);
    if (i >= m) return;
    const unsigned short* a = (const unsigned short*)s.A + (size_t)i * n;
    const unsigned short* b = (const unsigned short*)s.Bm + (size_t)i * n;
    double acc = 0.0;
    for (int j = lane; j < n; j += 32)
        acc += (double)(__uint_as_float((unsigned)a[j] << 16) * __uint_as_float((unsigned)b[j] << 16));
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) s.meas[i] = acc;
}

// ==========================================================================
// Tr exp(M_t) by sampling (the note after Lemma 2: the scalar b of the exact
// certificate can be estimated instead of computed): Hutchinson's estimator
// Tr exp(M) = E[u^T exp(M) u] over the k probe vectors u (the columns of the
// solve's block), each quadrature u^T exp(M) u = ||u||^2 e_1^T exp(T) e_1 from
// `steps` Lanczos steps on A = M_t - c I (the operator the products apply)
// with full reorthogonalisation (two classical Gram-Schmidt passes per step),
// T the tridiagonal of the Lanczos coefficients, and exp(M) = e^c exp(A).
// One block per probe column; the basis is kept column-major per slot:
// column j of slot i at Qb + (i k + j) n.  ab per column: [0] ||u||^2,
// [1 + i] alpha_i, [1 + LZ_MAX + i] beta_i.

// block sum of one double (every thread gets the result)
__device__ double lz_block_sum(double v, double* red) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += red[w];
    return t;
}

// column col of W (float storage) and of its bf16 split (tensor-core path) set to
// the float vector q; U = V^T W for the combine's log X part
__device__ void lz_set_w(const SolveDev& s, int col, const float* q, double* red) {
    const int n = s.n, k = s.k, r = s.r, tid = threadIdx.x;
    float* W = (float*)s.W;
    for (int i = tid; i < n; i += NT) {
        const float w = q[i];
        W[(size_t)i * k + col] = w;
        if (s.Wsp) {
            const size_t kp = (size_t)s.tc_kpad, P = (size_t)(s.tc_npad / 3);
            const __nv_bfloat16 hi = __float2bfloat16_rn(w);
            const float r1 = w - __bfloat162float(hi);
            const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
            const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
            s.Wsp[(size_t)col * kp + i] = __bfloat16_as_ushort(hi);
            s.Wsp[(P + col) * kp + i] = __bfloat16_as_ushort(mid);
            s.Wsp[(2 * P + col) * kp + i] = __bfloat16_as_ushort(lo);
        }
    }
    for (int l = 0; l < r; ++l) {
        double u = 0.0;
        for (int i = tid; i < n; i += NT) u += s.V[(size_t)i * r + l] * (double)q[i];
        u = lz_block_sum(u, red);
        if (tid == 0) s.sm[SM_U + l * 32 + col] = u;
    }
}

// q_0 = u / ||u|| for probe column col of U (n x k, float64, row-major)
__global__ void __launch_bounds__(NT) k_lz_start(const SolveDev* sd, const double* U, float* Qb, double* ab) {
    pdl_wait();
    pdl_trigger();
    const SolveDev& s = *sd;
    const int n = s.n, k = s.k, col = blockIdx.x, tid = threadIdx.x;
    if (col >= k) return;
    __shared__ double red[NT / 32];
    double a = 0.0;
    for (int i = tid; i < n; i += NT) a += U[(size_t)i * k + col] * U[(size_t)i * k + col];
    const double nrm2 = lz_block_sum(a, red);
    const double inv = nrm2 > 0.0 ? 1.0 / sqrt(nrm2) : 0.0;
    float* q = Qb + (size_t)col * n;
    for (int i = tid; i < n; i += NT) q[i] = (float)(U[(size_t)i * k + col] * inv);
    if (tid == 0) ab[(size_t)col * (2 * LZ_MAX + 1)] = nrm2;
    __syncthreads();
    lz_set_w(s, col, q, red);
}

// Lanczos step j of column col, after Z = (M_t - c I) W: alpha_j = q_j^T z,
// w = z - alpha_j q_j - beta_{j-1} q_{j-1}, two classical Gram-Schmidt passes
// against q_0..q_j, beta_j = ||w||, q_{j+1} = w / beta_j into slot j + 1 and
// W (a zero vector if w vanished)
__global__ void __launch_bounds__(NT) k_lz_step(const SolveDev* sd, float* Qb, double* ab, int j, int steps) {
    pdl_wait();
    pdl_trigger();
    const SolveDev& s = *sd;
    const int n = s.n, k = s.k, col = blockIdx.x, tid = threadIdx.x;
    if (col >= k || j < 0 || j >= steps || steps > LZ_MAX) return;
    const size_t slot = (size_t)k * n;
    const float* q0 = Qb + (size_t)col * n;                 // slot i at q0 + i * slot
    const float* z = (const float*)s.Z;
    double* abc = ab + (size_t)col * (2 * LZ_MAX + 1);
    __shared__ double red[NT / 32];
    __shared__ double hred[NT / 32][LZ_MAX];
    __shared__ double hs[LZ_MAX];
    double a = 0.0;
    for (int i = tid; i < n; i += NT) a += (double)q0[(size_t)j * slot + i] * (double)z[(size_t)i * k + col];
    const double alpha = lz_block_sum(a, red);
    const double bprev = j > 0 ? abc[1 + LZ_MAX + j - 1] : 0.0;
    float* w = (float*)q0 + (size_t)(j + 1) * slot;
    for (int i = tid; i < n; i += NT) {
        double v = (double)z[(size_t)i * k + col] - alpha * (double)q0[(size_t)j * slot + i];
        if (j > 0) v -= bprev * (double)q0[(size_t)(j - 1) * slot + i];
        w[i] = (float)v;
    }
    __syncthreads();
    for (int pass = 0; pass < 2; ++pass) {
        double h[LZ_MAX];
#pragma unroll
        for (int l = 0; l < LZ_MAX; ++l) h[l] = 0.0;
        for (int i = tid; i < n; i += NT) {
            const double wi = (double)w[i];
#pragma unroll
            for (int l = 0; l < LZ_MAX; ++l)
                if (l <= j) h[l] += (double)q0[(size_t)l * slot + i] * wi;
        }
        const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
        for (int l = 0; l < LZ_MAX; ++l) {
            if (l > j) break;
            double v = h[l];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) hred[wid][l] = v;
        }
        __syncthreads();
        if (tid <= j) {
            double t = 0.0;
            for (int ww = 0; ww < NT / 32; ++ww) t += hred[ww][tid];
            hs[tid] = t;
        }
        __syncthreads();
        for (int i = tid; i < n; i += NT) {
            double v = (double)w[i];
            for (int l = 0; l <= j; ++l) v -= hs[l] * (double)q0[(size_t)l * slot + i];
            w[i] = (float)v;
        }
        __syncthreads();
    }
    double b2 = 0.0;
    for (int i = tid; i < n; i += NT) b2 += (double)w[i] * (double)w[i];
    const double beta = sqrt(lz_block_sum(b2, red));
    if (tid == 0) {
        abc[1 + j] = alpha;
        abc[1 + LZ_MAX + j] = beta;
    }
    if (j + 1 < steps) {
        const double inv = beta > 1e-300 ? 1.0 / beta : 0.0;
        for (int i = tid; i < n; i += NT) w[i] = (float)((double)w[i] * inv);
        __syncthreads();
        lz_set_w(s, col, w, red);
    }
}

// the estimate: per column the tridiagonal T (cut at the first beta_j below
// 1e-10 of the local scale: an invariant subspace), its eigenpairs by Jacobi,
// ||u||^2 sum_i (e_1^T y_i)^2 exp(theta_i + c); the mean over the columns
__global__ void __launch_bounds__(NT) k_lz_quad(const SolveDev* sd, const double* ab, int steps, double* out) {
    pdl_wait();
    pdl_trigger();
    const SolveDev& s = *sd;
    const int k = s.k, tid = threadIdx.x;
    __shared__ double A[MEG_KMAX * MEG_LDK], Qm[MEG_KMAX * MEG_LDK], Bm[MEG_KMAX * MEG_LDK];
    __shared__ double wv[MEG_KMAX], pr[3 * MEG_KMAX + 8];
    __shared__ int len_s;
    const double c = s.sm[SM_SHIFT];
    double total = 0.0;                                      // thread 0
    for (int col = 0; col < k; ++col) {
        const double* abc = ab + (size_t)col * (2 * LZ_MAX + 1);
        if (tid == 0) {
            int len = steps;
            for (int j = 0; j + 1 < steps; ++j) {
                const double scale = fabs(abc[1 + j]) + (j > 0 ? abc[1 + LZ_MAX + j - 1] : 0.0);
                if (!(abc[1 + LZ_MAX + j] > 1e-10 * scale)) { len = j + 1; break; }
            }
            len_s = len;
        }
        __syncthreads();
        const int len = len_s;
        for (int e = tid; e < len * len; e += NT) {
            const int a = e / len, b = e % len;
            double v = 0.0;
            if (a == b) v = abc[1 + a];
            else if (b == a + 1) v = abc[1 + LZ_MAX + a];
            else if (a == b + 1) v = abc[1 + LZ_MAX + b];
            A[a * MEG_LDK + b] = v;
        }
        __syncthreads();
        kxk_jacobi(A, Qm, Bm, wv, pr, len, 60);
        if (tid == 0) {
            double v = 0.0;
            for (int i = 0; i < len; ++i) v += Qm[i] * Qm[i] * exp(wv[i] + c);   // row 0 of the eigenvectors
            total += abc[0] * v;
        }
        __syncthreads();
    }
    if (tid == 0) out[0] = total / (double)k;
}

cudaError_t launch_lz_start(const GroupLaunch& g, const double* U, float* Qb, double* ab, int k) {
    return launch_k(k_lz_start, dim3(k), dim3(NT), 0, g.stream, 1, g.d_solves, U, Qb, ab);
}
cudaError_t launch_lz_step(const GroupLaunch& g, float* Qb, double* ab, int j, int steps, int k) {
    return launch_k(k_lz_step, dim3(k), dim3(NT), 0, g.stream, 1, g.d_solves, Qb, ab, j, steps);
}
cudaError_t launch_lz_quad(const GroupLaunch& g, const double* ab, int steps, double* out) {
    return launch_k(k_lz_quad, dim3(1), dim3(NT), 0, g.stream, 1, g.d_solves, ab, steps, out);
}

// Y = (2/Lb) sum_b r_b a_b (a_b^T W): block = MA_ROWS rows of Y times one chunk
// of the batch.  Thread (row i, column group of 8) accumulates over the
// chunk's rows; a warp reads 32 consecutive elements of a row of A per step,
// and the scaled r_b T_b are staged in shared memory (broadcast reads).
// Chunk c's partial goes to slot c of Ys; k_combine sums the slots in order.
template <typename T>
__global__ void __launch_bounds__(NT) k_meas_apply(const SolveDev* sds, int ns) {
    pdl_wait();
    pdl_trigger();
    constexpr int CH = sizeof(T) == 8 ? 128 : 256;        // staged batch rows (shared memory)
    const int si = find_solve(sds, ns, PK_MAP, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_MAP];
    const int n = s.n, k = s.k, tid = threadIdx.x;
    const int Lb = s.nb_meas, nch = meas_chunks(Lb);
    const int ntile = (n + MA_ROWS - 1) / MA_ROWS;
    if (lb < 0 || lb >= ntile * nch || s.kind != MEG_MEAS_STOCH || s.mtc) return;
    const int tile = lb % ntile, ch = lb / ntile;
    const int b_lo = (int)((int64_t)ch * Lb / nch), b_hi = (int)((int64_t)(ch + 1) * Lb / nch);
    const bool warm = (s.mode == 1);
    const double scale = 2.0 / (double)Lb;
    const double* sc = s.meas;
    const int i = tile * MA_ROWS + (tid & (MA_ROWS - 1)), cg = tid / MA_ROWS;     // 4 groups x 8 columns
    __shared__ T S[CH][MEG_KMAX + 1];
    __shared__ int sidx[CH];
    T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b0 = b_lo; b0 < b_hi; b0 += CH) {
        const int bn = min(CH, b_hi - b0);
        __syncthreads();
        for (int e = tid; e < bn * k; e += NT) {
            const int bb = e / k, c = e % k;
            S[bb][c] = (T)(scale * sc[b0 + bb] * sc[2 * (size_t)Lb + (size_t)(b0 + bb) * MEG_KMAX + c]);
        }
        for (int e = tid; e < bn; e += NT) sidx[e] = warm ? b0 + e : s.bidx[b0 + e];
        __syncthreads();
        if (i < n) {
            for (int bb = 0; bb < bn; ++bb) {
                const T a = load_a<T>(s.A, (size_t)sidx[bb] * n + i);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (cg * 8 + q < k) acc[q] += a * S[bb][cg * 8 + q];
            }
        }
    }
    if (i < n) {
        T* Ys = (T*)s.Ys + ((size_t)ch * n + i) * k;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (cg * 8 + q < k) Ys[cg * 8 + q] = acc[q];
    }
}

// ==========================================================================
// Accurate objective f(X_t): dense pass / Omega pass / all measurements.
// The quantities that cancel (X_ij - M_ij, a^T X a - y) are formed in
// double-word arithmetic from float64 V (Dot2 with both factors split into
// float pairs), then squared and summed with compensation; deterministic
// last-block total.  Float64 storage uses plain float64 arithmetic.
struct XdotDw {
    // x += w * v with w, v float64 values, both split into float pairs
    __device__ __forceinline__ static void acc(dw& x, double w, double v) {
        const float wh = (float)w, wl = (float)(w - (double)wh);
        const float vh = (float)v, vl = (float)(v - (double)vh);
        dot2_acc(x, wh, vh);
        dot2_acc(x, wh, vl);
        dot2_acc(x, wl, vh);
    }
};

template <typename T>
__device__ __forceinline__ double load_val(const void* val, int64_t p) { return (double)((const T*)val)[p]; }

// Measurement part of the objective for bf16 A (exact in float), the block's
// slice of the m measurements, one warp per row.  V is split once per block
// into hi/lo floats in shared memory (RB columns, zero beyond r, rows padded
// to RB + 1 floats: conflict-free); a^T v_l = Dot2(a, v_hi) + sum a v_lo, the
// second sum in plain float (its terms are 2^-24 of the first), ||a||^2 exact.
template <int RB, typename A>
__device__ void obj_meas_rows(const SolveDev& s, int lb, float* vsm, const double* coef, A& acc) {
    const int n = s.n, r = s.r, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    constexpr int rp = RB + 1;
    float* vhi = vsm;
    float* vlo = vsm + (size_t)n * rp;
    for (int e = tid; e < n * RB; e += NT) {
        const int j = e / RB, l = e % RB;
        const double v = l < r ? s.V[(size_t)j * r + l] : 0.0;
        const float h = (float)v;
        vhi[j * rp + l] = h;
        vlo[j * rp + l] = (float)(v - (double)h);
    }
    __syncthreads();
    const int64_t per = (s.m + s.nb_red - 1) / s.nb_red;
    const int64_t i0 = (int64_t)lb * per, i1 = min((int64_t)s.m, i0 + per);
    for (int64_t i = i0 + warp; i < i1; i += NT / 32) {
        dw ph[RB], paa = {0.f, 0.f};
        float pl[RB];
#pragma unroll
        for (int l = 0; l < RB; ++l) { ph[l] = {0.f, 0.f}; pl[l] = 0.f; }
        for (int j = lane; j < n; j += 32) {
            const float a = load_a<float>(s.A, (size_t)i * n + j);
#pragma unroll
            for (int l = 0; l < RB; ++l) {
                dot2_acc(ph[l], a, vhi[j * rp + l]);
                pl[l] = fmaf(a, vlo[j * rp + l], pl[l]);
            }
            dot2_acc(paa, a, a);
        }
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int l = 0; l < RB; ++l) {
                dw t = {__shfl_xor_sync(0xffffffffu, ph[l].hi, o), __shfl_xor_sync(0xffffffffu, ph[l].lo, o)};
                dw_add(ph[l], t);
                pl[l] += __shfl_xor_sync(0xffffffffu, pl[l], o);
            }
            dw t = {__shfl_xor_sync(0xffffffffu, paa.hi, o), __shfl_xor_sync(0xffffffffu, paa.lo, o)};
            dw_add(paa, t);
        }
        if (lane == 0) {
            double q = coef[MEG_RMAX] * dw_value(paa);
#pragma unroll
            for (int l = 0; l < RB; ++l)
                if (l < r) {
                    const double pv = dw_value(ph[l]) + (double)pl[l];
                    q += coef[l] * pv * pv;
                }
            const double R = q - s.y[i];
            const double w = R * R / (double)s.m;
            const float wh = (float)w;
            acc.add_prod(wh, 1.f);
            acc.add_prod((float)(w - (double)wh), 1.f);
        }
    }
}

// a_i^T X b_i of pair i (valid in lane 0; the whole warp takes part):
// sum_l (mu_l - s)(a_i^T v_l)(b_i^T v_l) + s a_i^T b_i, a_i^T b_i from meas[i]
__device__ double bil_pair_q(const SolveDev& s, int64_t i, const float* vsm, const double* coef) {
    const int n = s.n, r = s.r, lane = threadIdx.x & 31, rp = rank_bucket(r) + 1;
    const unsigned short* Aa = (const unsigned short*)s.A;
    const unsigned short* Bb = (const unsigned short*)s.Bm;
    double q = 0.0;
    for (int l0 = 0; l0 < r; l0 += 8) {
        dw pa[8], pb[8];
        float la[8], lbv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) { pa[u] = pb[u] = {0.f, 0.f}; la[u] = lbv[u] = 0.f; }
        for (int j = lane; j < n; j += 32) {
            const float a = __uint_as_float((unsigned)Aa[(size_t)i * n + j] << 16);
            const float b = __uint_as_float((unsigned)Bb[(size_t)i * n + j] << 16);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int l = l0 + u;
                float vh = 0.f, vl = 0.f;
                if (l < r) {
                    if (vsm) {
                        vh = vsm[j * rp + l];
                        vl = vsm[(size_t)n * rp + j * rp + l];
                    } else {
                        const double v = s.V[(size_t)j * r + l];
                        vh = (float)v;
                        vl = (float)(v - (double)vh);
                    }
                }
                dot2_acc(pa[u], a, vh);
                la[u] = fmaf(a, vl, la[u]);
                dot2_acc(pb[u], b, vh);
                lbv[u] = fmaf(b, vl, lbv[u]);
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                dw t = {__shfl_xor_sync(0xffffffffu, pa[u].hi, o), __shfl_xor_sync(0xffffffffu, pa[u].lo, o)};
                dw_add(pa[u], t);
                t = {__shfl_xor_sync(0xffffffffu, pb[u].hi, o), __shfl_xor_sync(0xffffffffu, pb[u].lo, o)};
                dw_add(pb[u], t);
                la[u] += __shfl_xor_sync(0xffffffffu, la[u], o);
                lbv[u] += __shfl_xor_sync(0xffffffffu, lbv[u], o);
            }
        }
        if (lane == 0)
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (l0 + u < r)
                    q += coef[l0 + u] * (dw_value(pa[u]) + (double)la[u]) * (dw_value(pb[u]) + (double)lbv[u]);
    }
    return lane == 0 ? q + coef[MEG_RMAX] * s.meas[i] : 0.0;
}

// Bilinear measurements: f = 1/2 sum_i (tau a_i^T X b_i - y_i)^2 with
// a_i^T X b_i = sum_l (mu_l - s)(a_i^T v_l)(b_i^T v_l) + s a_i^T b_i, a_i^T b_i
// from meas[i] (rank-p measurement matrices: Tr(A_i^T X B_i), the sum of this
// over the p column pairs).  One warp per measurement, 8 columns of V at a time; a_i^T v_l is a
// double-word sum of the bf16 data times the float hi piece of v_l plus a
// float sum with its lo piece (V staged as hi/lo floats in shared memory when
// vsm is given, else split from the float64 V as it is read).  Adds r_i^2
// to acc (the caller halves the total).
template <typename A>
__device__ void obj_bil_rows(const SolveDev& s, int lb, float* vsm, const double* coef, A& acc) {
    const int n = s.n, r = s.r, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int RB = rank_bucket(r), rp = RB + 1;
    if (vsm) {
        for (int e = tid; e < n * RB; e += NT) {
            const int j = e / RB, l = e % RB;
            const double v = l < r ? s.V[(size_t)j * r + l] : 0.0;
            const float h = (float)v;
            vsm[j * rp + l] = h;
            vsm[(size_t)n * rp + j * rp + l] = (float)(v - (double)h);
        }
        __syncthreads();
    }
    const int G = s.mrank;                                  // pairs per measurement
    const int64_t mm = s.m / G;
    const int64_t per = (mm + s.nb_red - 1) / s.nb_red;
    const int64_t g0 = (int64_t)lb * per, g1 = min(mm, g0 + per);
    for (int64_t gm = g0 + warp; gm < g1; gm += NT / 32) {
        double q = 0.0;                                     // lane 0: Tr(A^T X B) of measurement gm
        for (int64_t i = gm * G; i < (gm + 1) * G; ++i) q += bil_pair_q(s, i, vsm, coef);
        if (lane == 0) {
            const double R = s.tau * q - s.y[gm];
            const double w = R * R;
            const float wh = (float)w;
            acc.add_prod(wh, 1.f);
            acc.add_prod((float)(w - (double)wh), 1.f);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(NT) k_objective(const SolveDev* sds, int ns, double* out, int vcap) {
    pdl_wait();
    pdl_trigger();
    const int si = find_solve(sds, ns, PK_RED, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_RED];
    if (lb < 0 || lb >= s.nb_red) return;
    const int n = s.n, r = s.r, tid = threadIdx.x;
    const double* V = s.V;
    __shared__ double coef[MEG_RMAX + 1];
    if (tid < r) coef[tid] = s.sm[SM_MU + tid] - s.sm[SM_S];
    if (tid == 0) coef[MEG_RMAX] = s.sm[SM_S];
    __syncthreads();
    Acc<T> acc;
    acc.zero();
    const int row0 = lb * s.rows_red, row1 = min(n, row0 + s.rows_red);
    const bool dense = (s.kind == MEG_DENSE_QUAD || s.kind == MEG_LINEAR);
    if (dense || s.kind == MEG_CSR_QUAD) {
        for (int i = row0; i < row1; ++i) {
            double wi[MEG_RMAX];
            for (int l = 0; l < r; ++l) wi[l] = V[(size_t)i * r + l] * coef[l];
            const int64_t pb = dense ? 0 : s.rowptr[i], pe = dense ? n : s.rowptr[i + 1];
            for (int64_t p = pb + tid; p < pe; p += NT) {
                const int j = dense ? (int)p : s.col[p];
                const double d = dense ? (double)load_d<T>(s.D, (size_t)i * n + j, s.prec) : load_val<T>(s.val, p);
                if constexpr (sizeof(T) == 8) {
                    double x = (j == i) ? coef[MEG_RMAX] : 0.0;
                    for (int l = 0; l < r; ++l) x = fma(wi[l], V[(size_t)j * r + l], x);
                    if (s.kind == MEG_LINEAR) acc.add_prod(x, d);
                    else { const double R = x - d; acc.add_prod(R, R); }
                } else {
                    dw x = dw_from_double((j == i) ? coef[MEG_RMAX] : 0.0);
                    for (int l = 0; l < r; ++l) XdotDw::acc(x, wi[l], V[(size_t)j * r + l]);
                    if (s.kind == MEG_LINEAR) {
                        dot2_acc(acc.v, x.hi, (float)d);
                        dot2_acc(acc.v, x.lo, (float)d);
                    } else {
                        float e, hi;
                        two_sum(x.hi, -(float)d, hi, e);       // d is exactly a float
                        const float R = __fadd_rn(hi, __fadd_rn(e, x.lo));
                        acc.add_prod(R, R);
                    }
                }
            }
        }
    } else if (s.kind == MEG_BILINEAR) {
        // float storage only (the kind needs bf16 A and B)
        if constexpr (sizeof(T) == 4) {
            extern __shared__ __align__(16) unsigned char bsm[];
            obj_bil_rows(s, lb, vcap >= 2 * n * (rank_bucket(r) + 1) ? (float*)bsm : nullptr, coef, acc);
        }
    } else if (sizeof(T) == 4 && vcap >= 2 * n * (rank_bucket(r) + 1)) {
        // measurements, bf16 A: see obj_meas_rows
        extern __shared__ __align__(16) unsigned char dsm[];
        switch (rank_bucket(r)) {
            case 2: obj_meas_rows<2>(s, lb, (float*)dsm, coef, acc); break;
            case 4: obj_meas_rows<4>(s, lb, (float*)dsm, coef, acc); break;
            case 8: obj_meas_rows<8>(s, lb, (float*)dsm, coef, acc); break;
            case 16: obj_meas_rows<16>(s, lb, (float*)dsm, coef, acc); break;
            default: obj_meas_rows<32>(s, lb, (float*)dsm, coef, acc); break;
        }
    } else {
        // measurements: rows of this block index measurement blocks over m
        const int64_t per = (s.m + s.nb_red - 1) / s.nb_red;
        const int64_t i0 = (int64_t)lb * per, i1 = min((int64_t)s.m, i0 + per);
        const int warp = tid >> 5, lane = tid & 31;
        for (int64_t i = i0 + warp; i < i1; i += NT / 32) {
            dw p[MEG_RMAX + 1];
            for (int l = 0; l <= r; ++l) p[l] = {0.f, 0.f};
            for (int j = lane; j < n; j += 32) {
                const double a = (double)load_a<T>(s.A, (size_t)i * n + j);
                for (int l = 0; l < r; ++l) XdotDw::acc(p[l], a, V[(size_t)j * r + l]);
                XdotDw::acc(p[r], a, a);
            }
            double pv[MEG_RMAX + 1];
            for (int l = 0; l <= r; ++l) {
                double v = dw_value(p[l]);
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                pv[l] = v;
            }
            if (lane == 0) {
                double q = coef[MEG_RMAX] * pv[r];
                for (int l = 0; l < r; ++l) q += coef[l] * pv[l] * pv[l];
                const double R = q - s.y[i];
                const double w = R * R / (double)s.m;
                if constexpr (sizeof(T) == 8) acc.add_prod(w, 1.0);
                else {
                    const float wh = (float)w;
                    acc.add_prod(wh, 1.f);
                    acc.add_prod((float)(w - (double)wh), 1.f);
                }
            }
        }
    }
    __shared__ dw ent[NT];
    ent[tid] = acc.as_dw();
    __syncthreads();
    if (tid == 0) {
        dw a = {0.f, 0.f};
        for (int q = 0; q < NT; ++q) dw_add(a, ent[q]);
        ent[0] = a;
    }
    __syncthreads();
    __shared__ dw fin;
    if (!red_two_level(s, lb, ent, &fin, 1)) return;
    if (tid == 0) {
        double v = dw_value(fin);
        if (s.kind == MEG_DENSE_QUAD || s.kind == MEG_CSR_QUAD || s.kind == MEG_BILINEAR) v *= 0.5;
        out[si] = v;
    }
}

// ==========================================================================
// host launch wrappers
namespace {
constexpr size_t OBJ_SMEM_MAX = 200 * 1024;   // k_objective: V hi/lo of measurement members
size_t combine_smem(int prec) {
    size_t tsz = prec == MEG_FP64 ? 8 : 4;
    return 8 * MEG_RMAX * MEG_KMAX + 3 * ROWS_MAX * MEG_KMAX * tsz + 2 * 528 * sizeof(dw) + 16;
}
size_t orth1_smem(int prec) {      // M1, Qv, rows of W', entries, rows of Z
    size_t tsz = prec == MEG_FP64 ? 8 : 4;
    return MEG_KMAX * MEG_KMAX * tsz + 8 * MEG_KMAX * MEG_RMAX + ROWS_MAX * MEG_KMAX * tsz + 528 * sizeof(dw) + 16 +
           ROWS_MAX * MEG_KMAX * tsz;
}
size_t orth2_smem(int prec) {      // M2, rows of W, V, entries (float: also the rows of W'), rows of W' (double)
    size_t tsz = prec == MEG_FP64 ? 8 : 4;
    return MEG_KMAX * MEG_KMAX * tsz + ROWS_MAX * MEG_KMAX * tsz + 8 + ROWS_MAX * MEG_RMAX * 8 + RED_MAX_ENTRIES * sizeof(dw) + 16 +
           (prec == MEG_FP64 ? ROWS_MAX * MEG_KMAX * tsz : 0);
}
size_t orth_smem(int prec) {       // M1, Qv, rows of W, rows of V, entries (first the rows of Z)
    size_t tsz = prec == MEG_FP64 ? 8 : 4;
    return 8 * MEG_KMAX * MEG_KMAX + 8 * MEG_KMAX * MEG_RMAX + ROWS_MAX * MEG_KMAX * tsz + 8 +
           ROWS_MAX * MEG_RMAX * 8 + 16 + std::max<size_t>(RED_MAX_ENTRIES * sizeof(dw), ROWS_MAX * MEG_KMAX * tsz);
}
size_t kry_proj_smem() {          // C (Coef k x k), rows of W0 and Z, entries
    return 8 * MEG_KMAX * MEG_KMAX + 2 * ROWS_MAX * MEG_KMAX * 4 + 528 * sizeof(dw) + 16;
}
size_t orth_kry_smem() {          // two Coef k x k areas, three row blocks, V hi/lo, entries
    return 2 * 8 * MEG_KMAX * MEG_KMAX + 3 * ROWS_MAX * MEG_KMAX * 4 + 2 * ROWS_MAX * MEG_RMAX * 4 +
           RED_MAX_ENTRIES * sizeof(dw) + 16;
}
size_t island_smem() {
    return 4 * 32 * MEG_LDK * sizeof(float) + RED_MAX_ENTRIES * sizeof(dw) + (6 * 32 * MEG_LDK + 32 + 96 + 32) * sizeof(double);
}
template <typename K>
cudaError_t set_smem(K kern, size_t bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
}  // namespace

// row-reduction kernels run in clusters of RED_CLUSTER blocks (grid padded per solve)
template <typename T>
cudaError_t launch_clustered(void (*kern)(const SolveDev*, int, int), const GroupLaunch& g, size_t smem, int phase) {
    return launch_k(kern, dim3(g.blocks[PK_RED]), dim3(NT), smem, g.stream, RED_CLUSTER, g.d_solves, g.ns, phase);
}

cudaError_t init_kernel_attributes() {
    cudaError_t e;
    if ((e = set_smem(k_combine<double>, combine_smem(MEG_FP64))) != cudaSuccess) return e;
    if ((e = set_smem(k_combine<float>, combine_smem(MEG_FP32))) != cudaSuccess) return e;
    if ((e = set_smem(k_orth1<double>, orth1_smem(MEG_FP64))) != cudaSuccess) return e;
    if ((e = set_smem(k_orth2<double>, orth2_smem(MEG_FP64))) != cudaSuccess) return e;
    if ((e = set_smem(k_orth<float>, orth_smem(MEG_FP32))) != cudaSuccess) return e;
    if ((e = set_smem(k_island_c<double>, island_smem())) != cudaSuccess) return e;
    if ((e = set_smem(k_island_c<float>, island_smem())) != cudaSuccess) return e;
    if ((e = set_smem(k_island_o1<double>, island_smem())) != cudaSuccess) return e;
    if ((e = set_smem(k_island_o2<double>, island_smem())) != cudaSuccess) return e;
    if ((e = set_smem(k_island_o2<float>, island_smem())) != cudaSuccess) return e;
    if ((e = set_smem(k_island_kry<float>, island_smem())) != cudaSuccess) return e;
    if ((e = set_smem(k_orth_kry, orth_kry_smem())) != cudaSuccess) return e;
    if ((e = set_smem(k_kry_proj, kry_proj_smem())) != cudaSuccess) return e;
    if ((e = set_smem(k_objective<float>, OBJ_SMEM_MAX)) != cudaSuccess) return e;
    if ((e = meas_tc_init()) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t launch_begin(const GroupLaunch& g) {
    return launch_k(k_begin, dim3(g.ns), dim3(32), 0, g.stream, 1, g.d_solves, g.ns);
}

cudaError_t launch_dense(const GroupLaunch& g) {
    for (int c = 0; c < g.tc_chunks; ++c) {
        cudaError_t e = launch_dense_tc(g.tc_desc[c], g.tc_ns[c], g.tc_T[c], g.tc_G[c], g.tc_npad[c], *g.tc_maps[c],
                                        g.stream);
        if (e != cudaSuccess) return e;
    }
    const dim3 grid(g.blocks[PK_DENSE]), blk(NT);
    if (g.prec == MEG_FP64) return launch_k(k_dense<double, double>, grid, blk, 0, g.stream, 1, g.d_solves, g.ns);
    if (g.prec == MEG_FP32) return launch_k(k_dense<float, float>, grid, blk, 0, g.stream, 1, g.d_solves, g.ns);
    return launch_k(k_dense<float, unsigned short>, grid, blk, 0, g.stream, 1, g.d_solves, g.ns);
}

cudaError_t launch_csr(const GroupLaunch& g) {
    const dim3 grid(g.blocks[PK_CSR]), blk(NT);
    if (g.prec == MEG_FP64) return launch_k(k_csr<double>, grid, blk, 0, g.stream, 1, g.d_solves, g.ns);
    cudaError_t e = launch_k(k_csr_prep, grid, blk, 0, g.stream, 1, g.d_solves, g.ns);
    if (e != cudaSuccess) return e;
    return launch_k(k_csr<float>, grid, blk, 0, g.stream, 1, g.d_solves, g.ns);
}

cudaError_t launch_meas_batch(const GroupLaunch& g) {
    const dim3 grid(g.blocks[PK_MEAS]), blk(NT);
    if (g.prec == MEG_FP64) return launch_k(k_meas_batch<double>, grid, blk, 0, g.stream, 1, g.d_solves, g.ns);
    cudaError_t e = cudaSuccess;
    // tensor-core members: the batch pass, then its finish (minibatch and bilinear kinds)
    if ((g.meas_tc || g.meas_bil) && (e = launch_meas_tc_batch(g)) != cudaSuccess) return e;
    if (g.meas_tc && (e = launch_k(k_meas_finish, grid, blk, 0, g.stream, 1, g.d_solves, g.ns)) != cudaSuccess)
        return e;
    if (g.meas_plain) e = launch_k(k_meas_batch<float>, grid, blk, 0, g.stream, 1, g.d_solves, g.ns);
    return e;
}

cudaError_t launch_meas_apply(const GroupLaunch& g) {
    if (g.blocks[PK_MAP] == 0) return cudaSuccess;
    const dim3 grid(g.blocks[PK_MAP]), blk(NT);
    if (g.prec == MEG_FP64) return launch_k(k_meas_apply<double>, grid, blk, 0, g.stream, 1, g.d_solves, g.ns);
    cudaError_t e = cudaSuccess;
    if ((g.meas_tc || g.meas_bil) && (e = launch_meas_tc_apply(g)) != cudaSuccess) return e;
    if (g.meas_plain) e = launch_k(k_meas_apply<float>, grid, blk, 0, g.stream, 1, g.d_solves, g.ns);
    return e;
}

cudaError_t launch_bil_prep(const SolveDev* d_solve, int64_t m, cudaStream_t st) {
    const int64_t blocks = (m + NT / 32 - 1) / (NT / 32);
    return launch_k(k_bil_prep, dim3((unsigned)blocks), dim3(NT), 0, st, 1, d_solve, m);
}

// a row kernel (clusters) followed by its per-solve island kernel
template <typename T>
cudaError_t launch_row_island(void (*row)(const SolveDev*, int, int), void (*island)(const SolveDev*, int, int),
                              const GroupLaunch& g, size_t smem, int phase) {
    cudaError_t e = launch_clustered<T>(row, g, smem, phase);
    if (e != cudaSuccess) return e;
    return launch_k(island, dim3(g.ns), dim3(NT), island_smem(), g.stream, 1, g.d_solves, g.ns, phase);
}

// Z = (M_t - c I) W for float storage, without the factor step (Lanczos products)
cudaError_t launch_combine_rows(const GroupLaunch& g) {
    if (g.prec == MEG_FP64) return cudaErrorNotSupported;
    return launch_clustered<float>(k_combine<float>, g, combine_smem(g.prec), PH_ADVANCE);
}

cudaError_t launch_combine(const GroupLaunch& g, int phase) {
    if (phase == PH_KRY1 || phase == PH_KRY2) {
        if (g.prec == MEG_FP64) return cudaErrorNotSupported;   // float storage only
        return launch_row_island<float>(k_combine<float>, k_island_kry<float>, g, combine_smem(g.prec), phase);
    }
    if (g.prec == MEG_FP64)
        return launch_row_island<double>(k_combine<double>, k_island_c<double>, g, combine_smem(g.prec), phase);
    return launch_row_island<float>(k_combine<float>, k_island_c<float>, g, combine_smem(g.prec), phase);
}

// the subspace block after combine's factor: float64 storage runs both
// CholeskyQR passes (orth1, its factor, orth2: the two-pass kernels exist
// for float64 only); the float-storage modes run the single pass k_orth
// (their factor refined in Gram space by combine's factor kernel); both end
// with the reduction of U and G
cudaError_t launch_orthonormalise(const GroupLaunch& g, int phase) {
    if (phase == PH_KRY1 || phase == PH_KRY2) {
        if (g.prec == MEG_FP64) return cudaErrorNotSupported;
        if (phase == PH_KRY1) {
            // Z' = Z - W0 C and its Gram, then the single-pass CholeskyQR factor of Z'
            cudaError_t e = launch_row_island<float>(k_kry_proj, k_island_c<float>, g, kry_proj_smem(), PH_ADVANCE);
            if (e != cudaSuccess) return e;
        }
        return launch_row_island<float>(k_orth_kry, k_island_o2<float>, g, orth_kry_smem(),
                                        phase == PH_KRY1 ? PH_KRY1 : PH_FINAL);
    }
    if (g.prec == MEG_FP64) {
        cudaError_t e =
            launch_row_island<double>(k_orth1<double>, k_island_o1<double>, g, orth1_smem(MEG_FP64), phase);
        if (e != cudaSuccess) return e;
        return launch_row_island<double>(k_orth2<double>, k_island_o2<double>, g, orth2_smem(MEG_FP64), phase);
    }
    return launch_row_island<float>(k_orth<float>, k_island_o2<float>, g, orth_smem(g.prec), phase);
}

// one kernel of the chain after a product, for timing: 0 combine, 1 its island,
// 2 orth1 (float storage: k_orth), 3 its island, 4 orth2 (float64 storage
// only), 5 the reduction of U and G
cudaError_t launch_chain_kernel(const GroupLaunch& g, int which, int phase) {
    void (*isl)(const SolveDev*, int, int) = nullptr;
    if (g.prec == MEG_FP64) {
        switch (which) {
        case 0: return launch_clustered<double>(k_combine<double>, g, combine_smem(MEG_FP64), phase);
        case 2: return launch_clustered<double>(k_orth1<double>, g, orth1_smem(MEG_FP64), phase);
        case 4: return launch_clustered<double>(k_orth2<double>, g, orth2_smem(MEG_FP64), phase);
        case 1: isl = k_island_c<double>; break;
        case 3: isl = k_island_o1<double>; break;
        default: isl = k_island_o2<double>; break;
        }
    } else {
        switch (which) {
        case 0: return launch_clustered<float>(k_combine<float>, g, combine_smem(g.prec), phase);
        case 2: return launch_clustered<float>(k_orth<float>, g, orth_smem(g.prec), phase);
        case 3:
        case 4: return cudaErrorNotSupported;                  // single pass
        case 1: isl = k_island_c<float>; break;
        default: isl = k_island_o2<float>; break;
        }
    }
    return launch_k(isl, dim3(g.ns), dim3(NT), island_smem(), g.stream, 1, g.d_solves, g.ns, phase);
}

cudaError_t launch_objective(const GroupLaunch& g, double* out_f) {
    const dim3 grid(g.blocks[PK_RED]), blk(NT);
    if (g.prec == MEG_FP64) return launch_k(k_objective<double>, grid, blk, 0, g.stream, 1, g.d_solves, g.ns, out_f, 0);
    // measurement members stage V as hi/lo floats (2 n (rank_bucket(r) + 1) floats) when they fit
    const size_t need = g.meas_vr > 0 ? (size_t)g.meas_vr * 8 : 0;
    const bool fits = need > 0 && need <= OBJ_SMEM_MAX;
    return launch_k(k_objective<float>, grid, blk, fits ? need : 0, g.stream, 1, g.d_solves, g.ns, out_f,
                    fits ? (int)(need / 4) : 0);
}

// ==========================================================================
// meg_solve's stopping test (problem statement: the relative objective gap
// (f(X_t) - f*) / (f(X_1) - f*) <= tol), one thread, after each chunk of
// iterations of the device loop.  It counts the chunk, records f, and ends
// the loop (conditional graph node) when the test holds, when f is not
// finite, when a kernel recorded an error, or when the chunk limit is reached,
// so the loop always ends after at most SM_SOLVE_LIMIT chunks.
__global__ void k_solve_check(double* sm, const double* f, cudaGraphConditionalHandle cond) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double fv = *f, fstar = sm[SM_SOLVE_FSTAR];
    const double chunks = sm[SM_SOLVE_CHUNKS] + 1.0;
    sm[SM_SOLVE_CHUNKS] = chunks;
    sm[SM_SOLVE_F] = fv;
    const bool conv = (fv - fstar) <= sm[SM_SOLVE_TOL] * (sm[SM_F1] - fstar);
    if (conv) sm[SM_SOLVE_DONE] = 1.0;
    if (conv || !isfinite(fv) || sm[SM_STATUS] != 0.0 || chunks >= sm[SM_SOLVE_LIMIT])
        cudaGraphSetConditional(cond, 0u);
}

cudaError_t launch_solve_check(double* sm, const double* f, cudaGraphConditionalHandle cond, cudaStream_t st) {
    k_solve_check<<<1, 32, 0, st>>>(sm, f, cond);
    return cudaGetLastError();
}

// Programmatic dependent launch is opt-in (MEG_PDL=1): on the n = 4096 batch
// it measured 5% slower than plain launches (the early-placed dependent
// blocks compete with the running kernel's clusters).
bool meg_pdl_enabled() {
    static const bool on = [] {
        const char* v = getenv("MEG_PDL");
        return v && v[0] == '1';
    }();
    return on;
}
