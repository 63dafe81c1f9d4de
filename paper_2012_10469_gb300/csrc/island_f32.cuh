// k x k island in float32 with double-word refinement, for the float-storage
// precision modes.  GB300 runs float64 at about 1/58 of the float32 rate, so
// the k x k work stays in one warp's registers: the CholeskyQR factor
// (equilibrated; float64 for the single pass of the float-storage modes,
// float32 where a second pass follows) and the Rayleigh-Ritz eigenproblem,
// solved by float32 Jacobi
// rotations followed by a refinement whose products are exact (Dot2):
// Rayleigh quotients for the Ritz values and a first-order correction of
// the top-r Ritz vectors.  All routines are called by every thread of the
// block; matrices live in shared memory with leading dimension MEG_LDK.
#pragma once

#include "meg_dev.cuh"

// ---------------------------------------------------------------------------
// A (k x k SPD) -> M = L^{-T} with A = L L^T, computed on the equilibrated
// matrix B = D A D (D = diag(A)^{-1/2}): B = Lb Lb^T, L = D^{-1} Lb,
// L^{-T} = D Lb^{-T}.  Warp 0 only, in registers: lane i holds row i of B
// (then of Lb) and column i of X = Lb^{-1}; the entries other lanes need
// travel by warp shuffles.  The order KP is k rounded up to a multiple of 8
// and fixed at compile time, B padded with the identity, so every loop is
// straight-line code.  F = float: pivots from the hardware reciprocal square
// root (one or two units in the last place; used where a second CholeskyQR
// pass follows); F = double: correctly rounded square roots and divisions,
// for the single CholeskyQR pass of the float-storage modes, whose factor
// must hold the accuracy of a double-word Gram.  Returns false on a
// non-positive pivot (M then holds the identity).  A is not modified.
template <typename F> __device__ __forceinline__ F chol_rsqrt(F d);
template <> __device__ __forceinline__ float chol_rsqrt<float>(float d) { return rsqrtf(d); }
template <> __device__ __forceinline__ double chol_rsqrt<double>(double d) { return 1.0 / sqrt(d); }
template <typename F> __device__ __forceinline__ F chol_rcp(F d);
template <> __device__ __forceinline__ float chol_rcp<float>(float d) { return __frcp_rn(d); }
template <> __device__ __forceinline__ double chol_rcp<double>(double d) { return 1.0 / d; }

template <typename F, int KP>
__device__ __forceinline__ void chol_inv_k(const F* A, F* M, F* dsc, int k, int* flag) {
    const int lane = threadIdx.x & 31;
    const unsigned full = 0xffffffffu;
    const F one = (F)1, zero = (F)0;
    const F dl = (lane < k) ? A[lane * MEG_LDK + lane] : one;
    const F sl = (lane < k && dl > zero) ? chol_rsqrt<F>(dl) : zero;
    if (lane < k) dsc[lane] = sl;
    F a[KP];
#pragma unroll
    for (int c = 0; c < KP; ++c) {
        const F sc = __shfl_sync(full, sl, c);
        a[c] = (lane < k && c < k) ? A[lane * MEG_LDK + c] * sl * sc : (c == lane ? one : zero);
    }
    int bad = 0;
    // right-looking Cholesky: column j of Lb, then the trailing update
#pragma unroll
    for (int j = 0; j < KP; ++j) {
        F d = __shfl_sync(full, a[j], j);
        if (!(d > zero)) { bad = 1; d = one; }
        const F inv = chol_rsqrt<F>(d), pj = d * inv;
        a[j] = (lane == j) ? pj : (lane > j ? a[j] * inv : a[j]);
#pragma unroll
        for (int c = j + 1; c < KP; ++c) {
            const F lcj = __shfl_sync(full, a[j], c);
            a[c] = (lane > j) ? fma(-a[j], lcj, a[c]) : a[c];
        }
    }
    // X = Lb^{-1}, lane = column: X_ic = (delta_ic - sum_{m<i} L_im X_mc) / L_ii
    F x[KP];
#pragma unroll
    for (int i = 0; i < KP; ++i) {
        F acc = (lane == i) ? one : zero;
#pragma unroll
        for (int m = 0; m < i; ++m) acc = fma(-__shfl_sync(full, a[m], i), x[m], acc);
        x[i] = acc * chol_rcp<F>(__shfl_sync(full, a[i], i));
    }
    // M = D X^T: lane c writes row c (zero left of the diagonal since X is lower)
    if (lane < k) {
#pragma unroll
        for (int i = 0; i < KP; ++i)
            if (i < k) M[lane * MEG_LDK + i] = bad ? (i == lane ? one : zero) : sl * x[i];
    }
    if (lane == 0) *flag = bad;
}

template <typename F>
__device__ inline bool chol_inv(const F* A, F* M, F* dsc, int k, int* flag) {
    if (threadIdx.x < 32) {
        switch ((k + 7) >> 3) {
            case 1: chol_inv_k<F, 8>(A, M, dsc, k, flag); break;
            case 2: chol_inv_k<F, 16>(A, M, dsc, k, flag); break;
            case 3: chol_inv_k<F, 24>(A, M, dsc, k, flag); break;
            default: chol_inv_k<F, 32>(A, M, dsc, k, flag); break;
        }
    }
    __syncthreads();
    return *flag == 0;
}

__device__ inline bool chol_inv_f32(const float* A, float* M, float* dsc, int k, int* flag) {
    return chol_inv<float>(A, M, dsc, k, flag);
}

// C = op(A) B in float32 (k x k or given shapes)
__device__ inline void mm_f32(const float* A, bool transA, const float* B, float* C, int m, int inner, int nc) {
    for (int e = threadIdx.x; e < m * nc; e += blockDim.x) {
        const int i = e / nc, j = e % nc;
        float s = 0.f;
        for (int l = 0; l < inner; ++l) s = fmaf(transA ? A[l * MEG_LDK + i] : A[i * MEG_LDK + l], B[l * MEG_LDK + j], s);
        C[i * MEG_LDK + j] = s;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Jacobi eigen-decomposition of a symmetric float matrix by one warp (lane i
// owns row i; k <= 32).  Round-robin ordering: the k/2 disjoint rotations of
// a round are applied together, each an exact 2 x 2 symmetric Schur step
// (Golub & Van Loan, Section 8.5).  Rows are double-buffered (A <-> B) so a
// round needs only warp synchronisation.  On return *pA points at the nearly
// diagonal matrix and Q holds the accumulated rotations.  Stops when the
// off-diagonal norm is below tol times the diagonal norm or stops falling.
__device__ inline int jacobi_warp_f32(float** pA, float* B, float* Q, float* pr, int k, int max_sweeps, float tol) {
    __shared__ int nsw;
    const int tid = threadIdx.x, lane = tid & 31;
    const int kk = (k + 1) & ~1;
    int* partner = (int*)(pr + 2 * MEG_KMAX);
    float* cs = pr;
    float* sg = pr + MEG_KMAX;
    if (tid < 32) {
        float* A = *pA;
        if (lane < k)
            for (int j = 0; j < k; ++j) Q[lane * MEG_LDK + j] = (j == lane) ? 1.f : 0.f;
        float prev_off = 3.4e38f;
        int sweep = 0;
        for (; sweep < max_sweeps; ++sweep) {
            __syncwarp();
            float off = 0.f, dia = 0.f;
            if (lane < k)
                for (int j = 0; j < k; ++j) {
                    const float v = A[lane * MEG_LDK + j];
                    if (j == lane) dia += v * v; else off += v * v;
                }
            for (int o = 16; o > 0; o >>= 1) {
                off += __shfl_xor_sync(0xffffffffu, off, o);
                dia += __shfl_xor_sync(0xffffffffu, dia, o);
            }
            if (off <= tol * tol * dia || off >= prev_off) break;
            prev_off = off;
            for (int round = 0; round < kk - 1; ++round) {
                if (lane < kk / 2) {
                    const int a = lane == 0 ? 0 : 1 + (lane - 1 + round) % (kk - 1);
                    const int bpos = kk - 1 - lane;
                    const int b = bpos == 0 ? 0 : 1 + (bpos - 1 + round) % (kk - 1);
                    const int p = min(a, b), q = max(a, b);
                    float c = 1.f, s = 0.f;
                    if (q < k) {
                        const float apq = A[p * MEG_LDK + q];
                        if (apq != 0.f) {
                            const float th = (A[q * MEG_LDK + q] - A[p * MEG_LDK + p]) / (2.f * apq);
                            const float t = (th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(1.f + th * th));
                            c = rsqrtf(1.f + t * t);
                            s = t * c;
                        }
                    }
                    if (p < k) { partner[p] = q < k ? q : p; cs[p] = c; sg[p] = q < k ? -s : 0.f; }
                    if (q < k) { partner[q] = p; cs[q] = c; sg[q] = s; }
                }
                __syncwarp();
                if (lane < k) {
                    const int i = lane, pi = partner[i];
                    const float ci = cs[i], si = sg[i];
                    for (int j = 0; j < k; ++j) {
                        const int pj = partner[j];
                        const float cj = cs[j], sj = sg[j];
                        B[i * MEG_LDK + j] = ci * (cj * A[i * MEG_LDK + j] + sj * A[i * MEG_LDK + pj]) +
                                             si * (cj * A[pi * MEG_LDK + j] + sj * A[pi * MEG_LDK + pj]);
                    }
                    // Q <- Q J on row i: columns j and partner(j) mix; process each pair once
                    for (int j = 0; j < k; ++j) {
                        const int pj = partner[j];
                        if (pj < j) continue;
                        const float qj = Q[i * MEG_LDK + j], qp = Q[i * MEG_LDK + pj];
                        Q[i * MEG_LDK + j] = cs[j] * qj + sg[j] * qp;
                        if (pj != j) Q[i * MEG_LDK + pj] = cs[pj] * qp + sg[pj] * qj;
                    }
                }
                __syncwarp();
                float* t = A; A = B; B = t;
            }
        }
        if (lane == 0) { *pA = A; nsw = sweep; }
    }
    __syncthreads();
    return nsw;
}

// ---------------------------------------------------------------------------
// The same Jacobi sweeps (round-robin ordering, the same 2 x 2 Schur steps,
// the same stopping rule) with the whole block updating the matrix: for the
// 2k x 2k pencils of the block Krylov Rayleigh-Ritz step, where one warp's
// k-cubed work per sweep would dominate the iteration.  Each round computes
// the k/2 rotations, then every thread updates its entries of A (into B) and
// of Q (through registers).  Requires blockDim.x * 4 >= k * k.
__device__ inline int jacobi_block_f32(float** pA, float* B, float* Q, float* pr, int k, int max_sweeps,
                                       float tol) {
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
    const int kk = (k + 1) & ~1;
    int* partner = (int*)(pr + 2 * MEG_KMAX);
    float* cs = pr;
    float* sg = pr + MEG_KMAX;
    __shared__ float red[2][32];
    __shared__ int s_stop;
    __shared__ float s_prev;
    // the (up to four) entries this thread owns, fixed for the whole run
    int ei[4], ej[4];
    bool ev[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int e = tid + m * nt;
        ev[m] = e < k * k;
        ei[m] = ev[m] ? e / k : 0;
        ej[m] = ev[m] ? e - (e / k) * k : 0;
    }
    float* A = *pA;
#pragma unroll
    for (int m = 0; m < 4; ++m)
        if (ev[m]) Q[ei[m] * MEG_LDK + ej[m]] = (ei[m] == ej[m]) ? 1.f : 0.f;
    if (tid == 0) s_prev = 3.4e38f;
    __syncthreads();
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        float off = 0.f, dia = 0.f;
#pragma unroll
        for (int m = 0; m < 4; ++m)
            if (ev[m]) {
                const float v = A[ei[m] * MEG_LDK + ej[m]];
                if (ei[m] == ej[m]) dia += v * v; else off += v * v;
            }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            dia += __shfl_xor_sync(0xffffffffu, dia, o);
        }
        if (lane == 0) { red[0][wid] = off; red[1][wid] = dia; }
        __syncthreads();
        if (tid == 0) {
            float o2 = 0.f, d2 = 0.f;
            for (int w = 0; w < (nt + 31) / 32; ++w) { o2 += red[0][w]; d2 += red[1][w]; }
            s_stop = (o2 <= tol * tol * d2 || o2 >= s_prev);
            s_prev = o2;
        }
        __syncthreads();
        if (s_stop) break;
        for (int round = 0; round < kk - 1; ++round) {
            if (tid < kk / 2) {
                const int a = tid == 0 ? 0 : 1 + (tid - 1 + round) % (kk - 1);
                const int bpos = kk - 1 - tid;
                const int b = bpos == 0 ? 0 : 1 + (bpos - 1 + round) % (kk - 1);
                const int p = min(a, b), q = max(a, b);
                float c = 1.f, sn = 0.f;
                if (q < k) {
                    const float apq = A[p * MEG_LDK + q];
                    if (apq != 0.f) {
                        const float th = (A[q * MEG_LDK + q] - A[p * MEG_LDK + p]) / (2.f * apq);
                        const float t = (th >= 0.f ? 1.f : -1.f) / (fabsf(th) + sqrtf(1.f + th * th));
                        c = rsqrtf(1.f + t * t);
                        sn = t * c;
                    }
                }
                if (p < k) { partner[p] = q < k ? q : p; cs[p] = c; sg[p] = q < k ? -sn : 0.f; }
                if (q < k) { partner[q] = p; cs[q] = c; sg[q] = sn; }
            }
            __syncthreads();
            float qn[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                qn[m] = 0.f;
                if (ev[m]) {
                    const int i = ei[m], j = ej[m], pi = partner[i], pj = partner[j];
                    const float ci = cs[i], si = sg[i], cj = cs[j], sj = sg[j];
                    B[i * MEG_LDK + j] = ci * (cj * A[i * MEG_LDK + j] + sj * A[i * MEG_LDK + pj]) +
                                         si * (cj * A[pi * MEG_LDK + j] + sj * A[pi * MEG_LDK + pj]);
                    qn[m] = cj * Q[i * MEG_LDK + j] + sj * Q[i * MEG_LDK + pj];
                }
            }
            __syncthreads();
#pragma unroll
            for (int m = 0; m < 4; ++m)
                if (ev[m]) Q[ei[m] * MEG_LDK + ej[m]] = qn[m];
            float* t = A; A = B; B = t;
        }
    }
    __syncthreads();
    if (tid == 0) *pA = A;
    __syncthreads();
    return sweep;
}

// ---------------------------------------------------------------------------
// Double-word helpers for exact products of float32 operands with a
// float64 matrix held as hi/lo floats.
__device__ __forceinline__ void dw_split(double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}

// ---------------------------------------------------------------------------
// M (k x k, float) with M^T S M = I to float32 accuracy for a Gram matrix S
// known to double-word accuracy (given in float64, leading dimension
// MEG_LDK): the second CholeskyQR pass carried out in Gram space instead of
// on the n rows.  M1 = L1^{-T} from the float32 Cholesky of S leaves
// M1^T S M1 = I + E with ||E|| about kappa(S) float rounding units;
// B = M1^T S M1 is formed with exact products (Dot2 over the (hi, lo) float
// split of S, then of T = S M1), M2 = L_B^{-T} from the float32 Cholesky of
// the well-conditioned B, and M = M1 M2 (exact products, returned in
// float64 to be applied as a (hi, lo) pair) gives M^T S M = M2^T B M2 = I to
// float accuracy.  F0..F3: four float k x k work matrices; T: a float64 one
// (it holds T = S M1 as a normalised (hi, lo) float pair, so that no float64
// arithmetic runs in the k^3 loops); M may alias none of them.  Returns false
// on a non-positive pivot.
__device__ inline bool gram_factor_f32(const double* S, float* F0, float* F1, float* F2, float* F3, double* T,
                                       double* M, float* dsc, int k, int* flag) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < k * k; e += nt) {
        const int i = e / k, j = e - i * k;
        float hi, lo;
        dw_split(S[i * MEG_LDK + j], hi, lo);
        F0[i * MEG_LDK + j] = hi;
        F1[i * MEG_LDK + j] = lo;
    }
    __syncthreads();
    bool ok = chol_inv<float>(F0, F2, dsc, k, flag);             // M1 in F2
    float* Th = (float*)T;                                      // T = S M1 as (hi, lo) floats
    float* Tl = Th + 32 * MEG_LDK;
    for (int e = tid; e < k * k; e += nt) {                     // T = S M1 (exact products)
        const int i = e / k, j = e - i * k;
        dw acc = {0.f, 0.f};
        for (int a = 0; a < k; ++a) {
            const float m = F2[a * MEG_LDK + j];
            dot2_acc(acc, F0[i * MEG_LDK + a], m);
            dot2_acc(acc, F1[i * MEG_LDK + a], m);
        }
        // normalise: hi = fl(acc.hi + acc.lo), lo its exact error -- the pair
        // that rounding the float64 value hi + lo to float and back gives
        float hi, lo;
        two_sum(acc.hi, acc.lo, hi, lo);
        Th[i * MEG_LDK + j] = hi;
        Tl[i * MEG_LDK + j] = lo;
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += nt) {                     // B = M1^T T (exact products)
        const int i = e / k, j = e - i * k;
        dw acc = {0.f, 0.f};
        for (int a = 0; a < k; ++a) {
            const float m = F2[a * MEG_LDK + i];
            dot2_acc(acc, m, Th[a * MEG_LDK + j]);
            dot2_acc(acc, m, Tl[a * MEG_LDK + j]);
        }
        F3[i * MEG_LDK + j] = (float)dw_value(acc);
    }
    __syncthreads();
    ok = chol_inv<float>(F3, F1, dsc, k, flag) && ok;            // M2 in F1
    for (int e = tid; e < k * k; e += nt) {                     // M = M1 M2 (exact products)
        const int i = e / k, j = e - i * k;
        dw acc = {0.f, 0.f};
        for (int a = 0; a < k; ++a) dot2_acc(acc, F2[i * MEG_LDK + a], F1[a * MEG_LDK + j]);
        M[i * MEG_LDK + j] = dw_value(acc);
    }
    __syncthreads();
    return ok;
}
