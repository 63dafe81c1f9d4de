// k x k float64 routines run by one thread block (the "last block" of a
// reduction): Cholesky, triangular inverse, Jacobi eigen-decomposition,
// products.  Matrices live in shared memory with leading dimension MEG_LDK.
// All routines must be called by every thread of the block.
#pragma once

// Order of a non-increasing sort by rank: element (u, j) comes before (v, i)
// when u > v, or u == v and j < i.  NaN counts as -infinity, so the relation
// is a strict total order and the ranks of k values are a permutation of
// 0..k-1 even when the values are not finite.
__device__ __forceinline__ int ranks_before(double u, int j, double v, int i) {
    u = isnan(u) ? -INFINITY : u;
    v = isnan(v) ? -INFINITY : v;
    return (u > v) || (u == v && j < i);
}

#include "meg_dev.cuh"

// A (k x k, SPD) -> lower Cholesky factor L in place (upper part zeroed).
// Right-looking, one column per round.  Returns false on a non-positive pivot.
__device__ inline bool kxk_chol(double* A, int k, int* flag) {
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) *flag = 0;
    __syncthreads();
    for (int j = 0; j < k; ++j) {
        if (tid == 0) {
            double d = A[j * MEG_LDK + j];
            if (!(d > 0.0)) { *flag = 1; d = 1.0; }
            A[j * MEG_LDK + j] = sqrt(d);
        }
        __syncthreads();
        double djj = A[j * MEG_LDK + j];
        for (int i = j + 1 + tid; i < k; i += nt) A[i * MEG_LDK + j] /= djj;
        __syncthreads();
        int m = k - j - 1;
        for (int e = tid; e < m * m; e += nt) {
            int i = j + 1 + e / m, c = j + 1 + e % m;
            if (c <= i) A[i * MEG_LDK + c] -= A[i * MEG_LDK + j] * A[c * MEG_LDK + j];
        }
        __syncthreads();
    }
    for (int e = tid; e < k * k; e += nt) {
        int i = e / k, c = e % k;
        if (c > i) A[i * MEG_LDK + c] = 0.0;
    }
    __syncthreads();
    return *flag == 0;
}

// M = L^{-T} for lower-triangular L (M upper-triangular).  Column c of L^{-1}
// by forward substitution in thread c.
__device__ inline void kxk_inv_lower_T(const double* L, double* M, int k) {
    const int tid = threadIdx.x;
    for (int e = tid; e < k * k; e += blockDim.x) M[(e / k) * MEG_LDK + e % k] = 0.0;
    __syncthreads();
    if (tid < k) {
        const int c = tid;
        double x[MEG_KMAX];
        for (int i = 0; i < k; ++i) x[i] = 0.0;
        x[c] = 1.0 / L[c * MEG_LDK + c];
        for (int i = c + 1; i < k; ++i) {
            double s = 0.0;
            for (int m = c; m < i; ++m) s = fma(L[i * MEG_LDK + m], x[m], s);
            x[i] = -s / L[i * MEG_LDK + i];
        }
        // (L^{-1})_{i c} = x[i]  ->  M_{c i} = x[i]
        for (int i = c; i < k; ++i) M[c * MEG_LDK + i] = x[i];
    }
    __syncthreads();
}

// C = op(A) * B with op = A or A^T; all k x k (or the given shapes).
// C must not alias A or B.
__device__ inline void kxk_mm(const double* A, bool transA, const double* B, double* C,
                              int m, int inner, int ncols) {
    for (int e = threadIdx.x; e < m * ncols; e += blockDim.x) {
        int i = e / ncols, j = e % ncols;
        double s = 0.0;
        for (int l = 0; l < inner; ++l) {
            double a = transA ? A[l * MEG_LDK + i] : A[i * MEG_LDK + l];
            s = fma(a, B[l * MEG_LDK + j], s);
        }
        C[i * MEG_LDK + j] = s;
    }
    __syncthreads();
}

// Symmetric eigen-decomposition by Jacobi rotations in parallel (round-robin)
// ordering: k/2 disjoint rotations per round, each an exact 2 x 2 symmetric
// Schur step (Golub & Van Loan, Section 8.5).  A (k x k) is destroyed; on
// return w holds the eigenvalues in non-increasing order and Q the
// corresponding eigenvectors as columns.  Scratch: B (k x k), pr (>= 3*32).
__device__ inline void kxk_jacobi(double* A, double* Q, double* B, double* w, double* pr, int k,
                                  int max_sweeps) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int kk = (k + 1) & ~1;              // even number of positions (one dummy if k odd)
    int* partner = (int*)(pr + 2 * MEG_KMAX); // [32]
    double* cs = pr;                          // c_i
    double* sg = pr + MEG_KMAX;               // sigma_i (signed s)
    __shared__ int s_done;
    for (int e = tid; e < k * k; e += nt) Q[(e / k) * MEG_LDK + e % k] = (e / k == e % k) ? 1.0 : 0.0;
    __syncthreads();
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (tid == 0) {
            double off = 0.0, dia = 0.0;
            for (int i = 0; i < k; ++i)
                for (int j = 0; j < k; ++j) {
                    double v = A[i * MEG_LDK + j];
                    if (i == j) dia += v * v; else off += v * v;
                }
            s_done = (off <= 1e-30 * dia) || off == 0.0;
        }
        __syncthreads();
        if (s_done) break;
        for (int round = 0; round < kk - 1; ++round) {
            // chess-tournament pairing: position 0 fixed, others rotate
            if (tid < kk / 2) {
                auto pos = [&](int j) { return j == 0 ? 0 : 1 + (j - 1 + round) % (kk - 1); };
                int a = pos(tid), b = pos(kk - 1 - tid);
                int p = min(a, b), q = max(a, b);
                double c = 1.0, s = 0.0;
                if (q < k) {
                    double apq = A[p * MEG_LDK + q];
                    if (apq != 0.0) {
                        double th = (A[q * MEG_LDK + q] - A[p * MEG_LDK + p]) / (2.0 * apq);
                        double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                    }
                }
                if (p < k) { partner[p] = q < k ? q : p; cs[p] = c; sg[p] = q < k ? -s : 0.0; }
                if (q < k) { partner[q] = p; cs[q] = c; sg[q] = s; }
            }
            __syncthreads();
            for (int e = tid; e < k * k; e += nt) {
                int i = e / k, j = e % k;
                int pi = partner[i], pj = partner[j];
                double v = cs[i] * cs[j] * A[i * MEG_LDK + j] + cs[i] * sg[j] * A[i * MEG_LDK + pj] +
                           sg[i] * cs[j] * A[pi * MEG_LDK + j] + sg[i] * sg[j] * A[pi * MEG_LDK + pj];
                B[i * MEG_LDK + j] = v;
            }
            __syncthreads();
            for (int e = tid; e < k * k; e += nt) {
                int i = e / k, j = e % k;
                A[i * MEG_LDK + j] = B[i * MEG_LDK + j];
                B[i * MEG_LDK + j] = cs[j] * Q[i * MEG_LDK + j] + sg[j] * Q[i * MEG_LDK + partner[j]];
            }
            __syncthreads();
            for (int e = tid; e < k * k; e += nt) Q[(e / k) * MEG_LDK + e % k] = B[(e / k) * MEG_LDK + e % k];
            __syncthreads();
        }
    }
    // sort eigenpairs, non-increasing (selection by rank; ties by index, NaN
    // last, so the ranks always form a permutation)
    if (tid < k) {
        double v = A[tid * MEG_LDK + tid];
        int rank = 0;
        for (int j = 0; j < k; ++j) rank += ranks_before(A[j * MEG_LDK + j], j, v, tid);
        partner[tid] = rank;
        w[rank] = v;
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += nt) {
        int i = e / k, j = e % k;
        B[i * MEG_LDK + partner[j]] = Q[i * MEG_LDK + j];
    }
    __syncthreads();
    for (int e = tid; e < k * k; e += nt) Q[(e / k) * MEG_LDK + e % k] = B[(e / k) * MEG_LDK + e % k];
    __syncthreads();
}

// Euclidean projection of v[0..r) onto the unit simplex (sort-based, Held,
// Wolfe & Crowder 1974); thread 0 only.
__device__ inline void simplex_project(double* v, int r) {
    double u[MEG_KMAX];
    for (int i = 0; i < r; ++i) u[i] = v[i];
    for (int i = 1; i < r; ++i) {            // insertion sort, non-increasing
        double x = u[i];
        int j = i - 1;
        while (j >= 0 && u[j] < x) { u[j + 1] = u[j]; --j; }
        u[j + 1] = x;
    }
    double css = 0.0, theta = 0.0;
    for (int j = 0; j < r; ++j) {
        css += u[j];
        double th = (css - 1.0) / (j + 1);
        if (u[j] - th > 0.0) theta = th;
    }
    for (int i = 0; i < r; ++i) v[i] = fmax(v[i] - theta, 0.0);
}
