// k x k island in float32 with double-word refinement, for the float-storage
// precision modes.  GB300 runs float64 at about 1/58 of the float32 rate, so
// the Cholesky factors of CholeskyQR2 are computed in float32 (equilibrated,
// one warp) and the Rayleigh-Ritz eigenproblem is solved by float32 Jacobi
// rotations followed by a refinement whose products are exact (Dot2):
// Rayleigh quotients for the Ritz values and a first-order correction of
// the top-r Ritz vectors.  All routines are called by every thread of the
// block; matrices live in shared memory with leading dimension MEG_LDK.
#pragma once

#include "meg_dev.cuh"

// ---------------------------------------------------------------------------
// A (k x k SPD, float) -> M = L^{-T} with A = L L^T, computed on the
// equilibrated matrix B = D A D (D = diag(A)^{-1/2}): B = Lb Lb^T,
// L = D^{-1} Lb, L^{-T} = D Lb^{-T}.  Warp 0 only; returns false on a
// non-positive pivot (M then holds the identity).  A is destroyed.
__device__ inline bool chol_inv_f32(float* A, float* M, float* dsc, int k, int* flag) {
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid < 32) {
        if (lane == 0) *flag = 0;
        if (lane < k) {
            const float d = A[lane * MEG_LDK + lane];
            dsc[lane] = d > 0.f ? rsqrtf(d) : 0.f;
        }
        __syncwarp();
        if (lane < k)
            for (int c = 0; c < k; ++c) A[lane * MEG_LDK + c] *= dsc[lane] * dsc[c];
        __syncwarp();
        for (int j = 0; j < k; ++j) {
            if (lane == j) {
                float d = A[j * MEG_LDK + j];
                if (!(d > 0.f)) { *flag = 1; d = 1.f; }
                A[j * MEG_LDK + j] = sqrtf(d);
            }
            __syncwarp();
            const float ljj = A[j * MEG_LDK + j];
            if (lane > j && lane < k) A[lane * MEG_LDK + j] /= ljj;
            __syncwarp();
            if (lane > j && lane < k) {
                const float lij = A[lane * MEG_LDK + j];
                for (int c = j + 1; c <= lane; ++c) A[lane * MEG_LDK + c] -= lij * A[c * MEG_LDK + j];
            }
            __syncwarp();
        }
        // column c of Lb^{-1} by forward substitution in lane c; M_{c i} = d_c (Lb^{-1})_{i c}
        if (lane < k) {
            const int c = lane;
            float x[MEG_KMAX];
            for (int i = 0; i < k; ++i) x[i] = 0.f;
            x[c] = 1.f / A[c * MEG_LDK + c];
            for (int i = c + 1; i < k; ++i) {
                float s = 0.f;
                for (int m = c; m < i; ++m) s = fmaf(A[i * MEG_LDK + m], x[m], s);
                x[i] = -s / A[i * MEG_LDK + i];
            }
            for (int i = 0; i < k; ++i) M[i * MEG_LDK + c] = 0.f;
            for (int i = c; i < k; ++i) M[i * MEG_LDK + c] = 0.f;
            __syncwarp(__activemask());
            for (int i = c; i < k; ++i) M[c * MEG_LDK + i] = dsc[c] * x[i];
        }
        __syncwarp();
        if (*flag && lane < k)
            for (int i = 0; i < k; ++i) M[lane * MEG_LDK + i] = (i == lane) ? 1.f : 0.f;
    }
    __syncthreads();
    return *flag == 0;
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
// Jacobi eigen-decomposition of a symmetric float matrix (parallel,
// round-robin ordering of the k/2 disjoint rotations of a round; exact 2 x 2
// symmetric Schur step, Golub & Van Loan Section 8.5).  A is overwritten by
// a nearly diagonal matrix, Q accumulates the rotations (starts at I).
// Stops when the off-diagonal norm falls below tol * ||diag|| or stalls.
__device__ inline void jacobi_f32(float* A, float* Q, float* B, float* pr, int k, int max_sweeps, float tol) {
    const int tid = threadIdx.x, nt = blockDim.x;
    const int kk = (k + 1) & ~1;
    int* partner = (int*)(pr + 2 * MEG_KMAX);
    float* cs = pr;
    float* sg = pr + MEG_KMAX;
    __shared__ float s_off, s_dia;
    for (int e = tid; e < k * k; e += nt) Q[(e / k) * MEG_LDK + e % k] = (e / k == e % k) ? 1.f : 0.f;
    __syncthreads();
    float prev_off = 3.4e38f;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (tid < 32) {
            float off = 0.f, dia = 0.f;
            for (int e = tid; e < k * k; e += 32) {
                const float v = A[(e / k) * MEG_LDK + e % k];
                if (e / k == e % k) dia += v * v; else off += v * v;
            }
            for (int o = 16; o > 0; o >>= 1) {
                off += __shfl_xor_sync(0xffffffffu, off, o);
                dia += __shfl_xor_sync(0xffffffffu, dia, o);
            }
            if (tid == 0) { s_off = off; s_dia = dia; }
        }
        __syncthreads();
        const float off = s_off;
        if (off <= tol * tol * s_dia || off >= prev_off) break;
        prev_off = off;
        for (int round = 0; round < kk - 1; ++round) {
            if (tid < kk / 2) {
                const int a = tid == 0 ? 0 : 1 + (tid - 1 + round) % (kk - 1);
                const int bpos = kk - 1 - tid;
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
            __syncthreads();
            for (int e = tid; e < k * k; e += nt) {
                const int i = e / k, j = e % k, pi = partner[i], pj = partner[j];
                B[i * MEG_LDK + j] = cs[i] * (cs[j] * A[i * MEG_LDK + j] + sg[j] * A[i * MEG_LDK + pj]) +
                                     sg[i] * (cs[j] * A[pi * MEG_LDK + j] + sg[j] * A[pi * MEG_LDK + pj]);
            }
            __syncthreads();
            for (int e = tid; e < k * k; e += nt) {
                const int i = e / k, j = e % k;
                A[i * MEG_LDK + j] = B[i * MEG_LDK + j];
                B[i * MEG_LDK + j] = cs[j] * Q[i * MEG_LDK + j] + sg[j] * Q[i * MEG_LDK + partner[j]];
            }
            __syncthreads();
            for (int e = tid; e < k * k; e += nt) Q[(e / k) * MEG_LDK + e % k] = B[(e / k) * MEG_LDK + e % k];
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Double-word helpers for exact products of float32 operands with a
// float64 matrix held as hi/lo floats.
__device__ __forceinline__ void dw_split(double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
}
