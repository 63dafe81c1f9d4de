// Minibatch gradient of the stochastic measurement objective on the tcgen05
// tensor cores (float storage, bf16 measurement vectors); the same two passes
// give the full gradient of the bilinear objective (Section 7, eq.
// recoveryProb) over the stacked rows [A; B], see the end of this comment.
//
// Step t draws the minibatch B_t (Section 6: L i.i.d. queries) and applies the
// gradient (2/L) sum_b r_b a_b a_b^T to the subspace block in implicit form,
//   Y = A_B^T (s o (A_B W)),  s_b = (2/L) r_b,  r_b = a_b^T X a_b - y_b,
// as two dense contractions:
//   batch pass  P = A_B [V | W]   (Lb x n times n x 2B): a_b^T v_l gives r_b,
//                                 a_b^T W the rows T_b; also ||a_b||^2;
//   apply pass  Y = A_B^T S       (n x Lb times Lb x k), S_b = s_b T_b.
// The operands of the tensor cores are bf16: A is bf16 already; the float
// operands ([V | W] and S) are split exactly into three bf16 pieces
// (x = hi + mid + lo, 24 mantissa bits), so each product equals the float
// product up to the float32 accumulation.  Each accumulation covers 32 of a
// chunk's 64 K (two MMAs; two accumulators per chunk, one commit) and the
// accumulations are added in registers as compensated float32 sums (an
// accumulation's error grows with its length on the tensor cores, where
// partial sums are rounded toward zero; a plain float sum's with the number
// of terms).
//
// Tiles are staged by the CTA's threads (asynchronous 16-byte copies of the
// gathered rows of A and of the operand images that k_meas_tc_split and the
// finish kernels write; the apply pass transposes A through registers) into
// the canonical K-major layout with the 128-byte swizzle: row q of a
// tile is 128 bytes (64 bf16 of K), its 16-byte piece c sits at position
// c xor (q mod 8), rows grouped by 8 into 1024-byte atoms.  Both passes keep
// two tile stages: the next chunk's copies are in flight while one thread
// issues the current chunk's four MMAs (M = 128, N = 3 x columns, K = 16) into
// tensor memory and commits them to an mbarrier; the block waits (bounded: about 1 s,
// then MEG_ERR_TIMEOUT is recorded, the CTA waits for its own MMAs, frees its
// tensor memory and returns) and drains the accumulator with tcgen05.ld.
//
// Bilinear kind: the batch rows are the stacked rows of [A; B] in 128-row
// tiles of 64 pairs (their a, then their b), every step; the batch pass's
// epilogue pairs the two halves into r_i = tau a_i^T X b_i - y_i and writes the
// S of row a_i, (tau/2) r_i b_i^T W, and of row b_i, (tau/2) r_i a_i^T W, so the
// apply pass over the stacked rows gives (tau/2) sum_i r_i (a_i b_i^T +
// b_i a_i^T) W = grad f W.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "meg_dev.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int MT_THREADS = 256;
constexpr int MT_TMEM_COLS = 64;                              // apply pass: two accumulators of P <= 32
constexpr int MT_BATCH_COLS = 128;                            // two accumulators of NC <= 64 columns
constexpr int MT_A_BYTES = MT_BM * MT_BK * 2;                 // 16 KB
constexpr int MT_B_MAX = 192 * MT_BK * 2;                     // N <= 192 (B = 32: 3 x 64 columns)

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// row index of batch row b: the b-th draw of step t (SplitMix64, as the
// CUDA-core kernels draw it), or b itself for the warm start's full pass and
// for the bilinear kind (a full pass over the stacked rows [A; B] every step)
__device__ __forceinline__ int64_t batch_row(const SolveDev& s, bool warm, int b) {
    if (warm || s.kind == MEG_BILINEAR) return b;
    return (int64_t)(splitmix64(s.seed + ((uint64_t)s.sm[SM_T] * (uint64_t)s.L + (uint64_t)b + 1ull) *
                                             0x9E3779B97F4A7C15ull) %
                     (uint64_t)s.m);
}

// start of batch row j: row j of A; for the bilinear kind row j of tile j / 128
// (a of pair 64 (j / 128) + j mod 64 in its first 64 rows, b in the others),
// nullptr for a padding pair past the last one
__device__ __forceinline__ const unsigned short* stacked_row(const SolveDev& s, int64_t j) {
    if (s.kind != MEG_BILINEAR) return (const unsigned short*)s.A + (size_t)j * s.n;
    const int64_t i = (j >> 7) * 64 + (j & 63);
    if (i >= s.m) return nullptr;
    return (const unsigned short*)((j & 64) ? s.Bm : s.A) + (size_t)i * s.n;
}

// byte offset of element (row q, k) of a K-major 128-byte-swizzled tile
__device__ __forceinline__ uint32_t sw_off(int q, int kk) {
    return (uint32_t)(q * 128 + ((((kk >> 3) ^ (q & 7))) << 4) + (kk & 7) * 2);
}

// Compensated running sum: hi + lo, each addition's rounding error (Knuth's
// TwoSum, exact in round-to-nearest) collected in lo.  The apply pass adds
// thousands of slice results per output, where a plain float sum would lose
// about 6e-8 sqrt(count) relative.
__device__ __forceinline__ void csum_add(float& hi, float& lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
}

// 16-byte asynchronous global -> shared copy (zero fill when !pred; nothing is
// read then, src only has to be a valid address) and its group operations
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool pred) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(pred ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// exact three-piece bf16 split of a float: piece 0, 1 or 2
__device__ __forceinline__ unsigned short bf16_piece(float x, int p) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    if (p == 0) return __bfloat16_as_ushort(hi);
    const float r1 = x - __bfloat162float(hi);
    const __nv_bfloat16 mid = __float2bfloat16_rn(r1);
    if (p == 1) return __bfloat16_as_ushort(mid);
    return __bfloat16_as_ushort(__float2bfloat16_rn(r1 - __bfloat162float(mid)));
}

// Shared state of one CTA: tile buffers (1024-byte aligned), the mbarrier of
// the MMA commits, the tensor-memory address, an error flag.
struct MtSmem {
    unsigned char* a;
    unsigned char* b;
    uint64_t* bar;
    uint32_t* tslot;
    int* err;
};

// stages: tile buffers one after the other (stage st: a + st MT_STAGE, b + st MT_STAGE)
constexpr int MT_STAGE = MT_A_BYTES + MT_B_MAX;
__device__ __forceinline__ MtSmem mt_carve(unsigned char* raw, int stages = 1) {
    MtSmem m;
    unsigned char* base = (unsigned char*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
    m.a = base;
    m.b = base + MT_A_BYTES;
    m.bar = (uint64_t*)(base + stages * MT_STAGE);
    m.tslot = (uint32_t*)(m.bar + 2);
    m.err = (int*)(m.tslot + 1);
    return m;
}

__device__ __forceinline__ uint32_t mt_setup(const MtSmem& m, uint32_t cols = MT_TMEM_COLS) {
    if (threadIdx.x == 0) {
        mbar_init(m.bar, 1);
        mbar_init(m.bar + 1, 1);
        *m.err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(m.tslot)),
                     "r"(cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *m.tslot;
}

// End of a CTA: on error, wait (bounded) for every MMA this CTA issued and
// flag the solve; free the tensor memory.
__device__ __forceinline__ void mt_teardown(const MtSmem& m, uint32_t tmem, const SolveDev& s, bool bad,
                                            uint32_t cols = MT_TMEM_COLS) {
    tc_fence_before();
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) {
            umma_commit(m.bar + 1);
            mbar_wait(m.bar + 1, 0);
            *m.err = 1;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && *m.err) s.sm[SM_STATUS] = MEG_ERR_TIMEOUT;
    if (threadIdx.x < 32) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols)
                     : "memory");
    }
}

// ==========================================================================
// Split image of the batch pass's B operand, once per product: for each
// 64-wide K chunk c, the N = 3 x 2B rows of [V | W] (B columns each, zero
// beyond r and k; piece p of column col at row p 2B + col) as the chunk's 64
// bf16 values, laid out byte for byte as the swizzled shared-memory tile
// (N x 128 bytes per chunk), so that every CTA of the batch pass copies it
// with 16-byte loads instead of splitting the same values again.  The blocks
// of the batch-pass grid take the chunks in turn.
__global__ void __launch_bounds__(MT_THREADS) k_meas_tc_split(const SolveDev* sds, int ns) {
    pdl_wait();
    pdl_trigger();
    const int si = find_solve(sds, ns, PK_MTB, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_MTB];
    const int Lb = s.nb_meas, n = s.n, k = s.k, r = s.r, tid = threadIdx.x;
    const int G = (Lb + MT_BM - 1) / MT_BM * batch_ks(s.kind, Lb, n);
    if (!s.mtc || (s.kind != MEG_MEAS_STOCH && s.kind != MEG_BILINEAR) || lb < 0 || lb >= G) return;
    const int nch = (n + MT_BK - 1) / MT_BK;
    const bool warm = (s.mode == 1);
    const int B = k_bucket(k), NC = 2 * B, N = 3 * NC;
    const float* W = (const float*)s.W;
    const double* V = s.V;
    for (int c = lb; c < nch; c += G) {
        unsigned char* img = (unsigned char*)(s.mtb + (size_t)c * N * 64);
        const int k0 = c * MT_BK;
        for (int it = tid; it < N * 8; it += MT_THREADS) {
            const int q = it >> 3, kc = it & 7;
            const int p = q / NC, col = q % NC;
            unsigned short e[8];
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                const int i = k0 + kc * 8 + h;
                float x = 0.f;
                if (i < n) {
                    if (col < B) { if (!warm && col < r) x = (float)V[(size_t)i * r + col]; }
                    else if (col - B < k) x = W[(size_t)i * k + (col - B)];
                }
                e[h] = bf16_piece(x, p);
            }
            uint4 val;
            val.x = (unsigned)e[0] | ((unsigned)e[1] << 16);
            val.y = (unsigned)e[2] | ((unsigned)e[3] << 16);
            val.z = (unsigned)e[4] | ((unsigned)e[5] << 16);
            val.w = (unsigned)e[6] | ((unsigned)e[7] << 16);
            *(uint4*)(img + q * 128 + ((kc ^ (q & 7)) << 4)) = val;
        }
    }
}

// ==========================================================================
// Bilinear kind (Section 7, eq. recoveryProb, trace-1 variables): the end of a
// batch-pass tile, whose rows 0-63 hold a_i^T [V | W] and ||a_i||^2 and rows
// 64-127 the same for b_i (Ps, 128 x (NC + 1) floats), i = 64 tile + row:
//   r_i = tau (sum_l (mu_l - s)(a_i^T v_l)(b_i^T v_l) + s a_i^T b_i) - y_i
//   (mode 1, the warm start's -grad f(0): r_i = -y_i; rank-p measurement
//   matrices: the p pairs of a measurement sum to tau Tr(A^T X B) and share
//   its residual), with a_i^T b_i from meas[i];
//   S of row a_i = (tau/2) r_i b_i^T W, S of row b_i = (tau/2) r_i a_i^T W, as
//   16-byte pieces of the S image (the tile is image chunks 2 tile, 2 tile + 1);
// and the shift estimate: grad f = (tau/2)(A^T D B + B^T D A), D = diag(r), so
// ||grad f|| <= tau (||A^T |D| A|| ||B^T |D| B||)^(1/2), each factor estimated
// as for a weighted Wishart matrix:
//   g = (tau / n) (1 + sqrt(n/m))^2 (m sum_i r_i^2 ||a_i||^2 ||b_i||^2)^(1/2)
// (m pairs).  Like the minibatch estimate it only centres the shift; Rayleigh-
// Ritz is exact.  The last tile to finish combines the per-tile sums in a
// fixed order.  Every thread of the block takes part.
__device__ void bil_tile_finish(const SolveDev& s, int tile, const float* Ps, float* Sx) {
    const int tid = threadIdx.x, n = s.n, k = s.k, r = s.r;
    const int B = k_bucket(k), NC = 2 * B, ld = NC + 1;
    const int64_t m = s.m, i0 = (int64_t)tile * 64;
    const bool warm = (s.mode == 1);
    double* sc = s.meas;                                    // [m] a_i^T b_i, then one partial per tile
    __shared__ float sr_s[64];
    __shared__ double bs[2];
    if (tid < 64) {
        const int64_t i = i0 + tid;
        double q = 0.0;
        if (i < m && !warm) {
            // float terms: each product a_i^T v_l is a float-accurate sum
            const double sv = s.sm[SM_S];
            float qf = 0.f;
            for (int l = 0; l < r; ++l)
                qf = fmaf((float)(s.sm[SM_MU + l] - sv), Ps[tid * ld + l] * Ps[(64 + tid) * ld + l], qf);
            q = (double)qf + sv * sc[i];
        }
        for (int o = 1; o < s.mrank; o <<= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        double contrib = 0.0;
        float sr = 0.f;
        if (i < m) {
            const double res = s.tau * q - s.y[i / s.mrank];
            sr = (float)(0.5 * s.tau * res);
            const float rf = (float)res;
            contrib = (double)(rf * rf * Ps[tid * ld + NC] * Ps[(64 + tid) * ld + NC]);
        }
        sr_s[tid] = sr;
        for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
        if ((tid & 31) == 0) bs[tid >> 5] = contrib;
    }
    __syncthreads();
    // S rows of the tile: row p < 64 (a_p) takes b_p^T W, row 64 + p (b_p) takes a_p^T W
    for (int e = tid; e < 128 * k; e += MT_THREADS) {
        const int rr = e / k, c = e % k, pp = rr & 63;
        Sx[rr * (MEG_KMAX + 1) + c] = sr_s[pp] * Ps[(rr < 64 ? 64 + pp : pp) * ld + B + c];
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 4; ++h)
        mts_put32(s.mts, k, (int64_t)tile * 128 + 32 * h, Sx + 32 * h * (MEG_KMAX + 1), MEG_KMAX + 1);
    __shared__ int am_last;
    const int ntiles = (int)((m + 63) / 64);
    if (tid == 0) {
        sc[(size_t)m + tile] = bs[0] + bs[1];
        __threadfence();
        unsigned* c = s.ctr + (s.nb_red + RED_GROUP - 1) / RED_GROUP + 2;
        am_last = (atomicAdd(c, 1u) == (unsigned)(ntiles - 1));
        if (am_last) *c = 0u;
    }
    __syncthreads();
    if (!am_last) return;
    __shared__ double red[MT_THREADS];
    double v = 0.0;
    for (int q2 = tid; q2 < ntiles; q2 += MT_THREADS) v += __ldcg(sc + m + q2);
    red[tid] = v;
    __syncthreads();
    for (int h = MT_THREADS / 2; h > 0; h >>= 1) {
        if (tid < h) red[tid] = red[tid] + red[tid + h];
        __syncthreads();
    }
    if (tid == 0) {
        const float fm = (float)m, fn = (float)n;
        const float f = 1.f + sqrtf(fn / fm);
        s.sm[SM_RESID_BOUND] = (double)((float)s.tau / fn * f * f * sqrtf(fm * (float)red[0]));
    }
}

// ==========================================================================
// Batch pass.  CTA (tile, part): 128 batch rows b times the columns [V | W]
// (B each, zero beyond r and k), the part's K chunks of the n-long
// contraction.  The B operand holds the three pieces of the float values,
// N = 3 x 2B rows: piece p of column c is row p 2B + c.  Warps w and w + 4
// share the tensor-memory lanes of rows 32 (w mod 4) ...; each takes every
// other 16-column group.  Output: per row and part, the 2B products and the
// part's ||a_b||^2, as floats in mtp, parts innermost ([row][column][part]) so
// that the finish kernel reads an entry's parts as contiguous vectors.
__global__ void __launch_bounds__(MT_THREADS, 2) k_meas_tc_batch(const SolveDev* sds, int ns) {
    pdl_wait();
    pdl_trigger();
    const int si = find_solve(sds, ns, PK_MTB, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_MTB];
    const int Lb = s.nb_meas, n = s.n, k = s.k, tid = threadIdx.x;
    const int mtiles = (Lb + MT_BM - 1) / MT_BM, KS = batch_ks(s.kind, Lb, n);
    if (!s.mtc || (s.kind != MEG_MEAS_STOCH && s.kind != MEG_BILINEAR) || lb < 0 || lb >= mtiles * KS) return;
    const int mt = lb % mtiles, part = lb / mtiles;
    const int nch = (n + MT_BK - 1) / MT_BK;
    const int c_lo = (int)((int64_t)part * nch / KS), c_hi = (int)((int64_t)(part + 1) * nch / KS);
    const bool warm = (s.mode == 1);
    const int B = k_bucket(k), NC = 2 * B, N = 3 * NC;
    extern __shared__ __align__(1024) unsigned char smraw[];
    const MtSmem m = mt_carve(smraw, 2);
    __shared__ int64_t rowidx[MT_BM];
    if (tid < MT_BM) {
        const int b = mt * MT_BM + tid;
        rowidx[tid] = b < Lb ? batch_row(s, warm, b) : -1;
    }
    const uint32_t tmem = mt_setup(m, MT_BATCH_COLS);       // (synchronises the block)
    const uint32_t idesc = idesc_bf16(MT_BM, NC);
    // A tile: thread = (row, half of the 64 columns), four 16-byte vectors
    const int arow = tid >> 1, ahalf = tid & 1;
    const int64_t ar = rowidx[arow];
    const unsigned short* rowp = ar >= 0 ? stacked_row(s, ar) : nullptr;
    const bool live = rowp != nullptr;                      // a row of data (not past the batch)
    const unsigned short* arp = live ? rowp : (const unsigned short*)s.A;
    float aa = 0.f;                                         // this thread's part of ||a||^2
    // accumulator drain: rows (lanes) and 16-column groups of this warp
    const int warp = tid >> 5, quarter = warp & 3, lane = tid & 31;
    const int grow = quarter * 32 + lane;                   // tile row of this thread's results
    const int ngroups = NC / 16;                            // 1, 2 or 4
    float run[2][16], rlo[2][16];
#pragma unroll
    for (int g = 0; g < 2; ++g)
#pragma unroll
        for (int j = 0; j < 16; ++j) run[g][j] = rlo[g][j] = 0.f;
    // chunk c into stage st: the gathered rows of A (zero beyond n) and the chunk's
    // image of the split [V | W] (k_meas_tc_split), asynchronous 16-byte copies
    auto stage = [&](int c, int st) {
        unsigned char* As = m.a + st * MT_STAGE;
        unsigned char* Bs = m.b + st * MT_STAGE;
        const int k0 = c * MT_BK;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int kc = ahalf * 4 + v;                   // 16-byte piece of the row
            const bool pred = live && k0 + kc * 8 < n;
            cp_async16(As + arow * 128 + ((kc ^ (arow & 7)) << 4), pred ? arp + k0 + kc * 8 : arp, pred);
        }
        const unsigned short* src = s.mtb + (size_t)c * N * 64;
        for (int it = tid; it < N * 8; it += MT_THREADS) cp_async16(Bs + it * 16, src + it * 8, true);
        cp_async_commit();
    };
    bool ok = true;
    uint32_t parity = 0;
    if (c_lo < c_hi) stage(c_lo, 0);
    for (int c = c_lo; c < c_hi && ok; ++c) {
        const int st = (c - c_lo) & 1;
        // the next chunk's copies run while this chunk is multiplied
        if (c + 1 < c_hi) stage(c + 1, st ^ 1);
        else cp_async_commit();                             // an empty group: wait_group 1 still means chunk c
        cp_async_wait1();
        __syncthreads();
        const unsigned char* As = m.a + st * MT_STAGE;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int kc = ahalf * 4 + v;
            const uint4 val = *(const uint4*)(As + arow * 128 + ((kc ^ (arow & 7)) << 4));
            const unsigned wds[4] = {val.x, val.y, val.z, val.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float lo = __uint_as_float(wds[h] << 16), hi = __uint_as_float(wds[h] & 0xffff0000u);
                aa = fmaf(lo, lo, aa);
                aa = fmaf(hi, hi, aa);
            }
        }
        // slices 0 and 1 accumulate in columns 0.., slices 2 and 3 in columns 64..
        // (32-wide accumulations).  Within an accumulation the lo pieces of [V | W]
        // (sub-tile 2 NC rows into the image) go first, then mid (NC), then hi (0):
        // the small terms are added while the accumulator is small, so only the
        // hi MMAs round at its full magnitude.  One commit for the chunk.
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(m.a + st * MT_STAGE), b0 = smem_u32(m.b + st * MT_STAGE);
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int p = 2; p >= 0; --p)
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const int kk = 2 * h + j;
                        umma_bf16(tmem + (uint32_t)(h * 64), sdesc_sw128(a0 + kk * 32),
                                  sdesc_sw128(b0 + (uint32_t)(p * NC * 128 + kk * 32)), idesc,
                                  (uint32_t)(p != 2 || j != 0));
                    }
            umma_commit(m.bar);
        }
        const bool done = mbar_wait(m.bar, parity);
        parity ^= 1u;
        ok = __syncthreads_or(done ? 0 : 1) == 0;
        tc_fence_after();
        if (!ok) break;
        // ---- drain: each output column of both accumulators
        const uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
        for (int acc = 0; acc < 2; ++acc)
#pragma unroll
            for (int gi = 0; gi < 2; ++gi) {
                const int g = (warp >> 2) + 2 * gi;         // this warp's 16-column groups
                if (g < ngroups) {
                    uint32_t v[16];
                    tmem_ld16(tb + (uint32_t)(acc * 64 + 16 * g), v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) csum_add(run[gi][j], rlo[gi][j], __uint_as_float(v[j]));
                }
            }
        tc_fence_before();
        __syncthreads();                                    // the stage and the accumulators are reused
    }
    cp_async_wait0();                                       // no copy in flight when the CTA ends
    // ---- partials of this part: columns, then ||a||^2 (the two threads of a row add theirs)
    aa += __shfl_xor_sync(0xffffffffu, aa, 1);
    if (s.kind == MEG_BILINEAR) {
        // the tile's 64 pairs are finished here: products through shared memory
        // (the stage buffers are free: no copy in flight, the last MMA waited for)
        float* Ps = (float*)m.a;
        __syncthreads();
        if (ok) {
#pragma unroll
            for (int gi = 0; gi < 2; ++gi) {
                const int g = (warp >> 2) + 2 * gi;
                if (g < ngroups)
#pragma unroll
                    for (int j = 0; j < 16; ++j) Ps[grow * (NC + 1) + 16 * g + j] = run[gi][j] + rlo[gi][j];
            }
            if (ahalf == 0) Ps[arow * (NC + 1) + NC] = aa;
        }
        __syncthreads();
        if (ok) bil_tile_finish(s, mt, Ps, Ps + MT_BM * (NC + 1));
        mt_teardown(m, tmem, s, !ok, MT_BATCH_COLS);
        return;
    }
    const int b = mt * MT_BM + grow;
    if (ok && b < Lb) {
        float* out = s.mtp + (size_t)b * (NC + 1) * KS + part;
#pragma unroll
        for (int gi = 0; gi < 2; ++gi) {
            const int g = (warp >> 2) + 2 * gi;
            if (g < ngroups)
#pragma unroll
                for (int j = 0; j < 16; ++j) out[(size_t)(16 * g + j) * KS] = run[gi][j] + rlo[gi][j];
        }
    }
    if (ok && ahalf == 0 && mt * MT_BM + arow < Lb)
        s.mtp[((size_t)(mt * MT_BM + arow) * (NC + 1) + NC) * KS + part] = aa;
    mt_teardown(m, tmem, s, !ok, MT_BATCH_COLS);
}

// ==========================================================================
// Apply pass.  CTA (tile, slot of the batch): 128 rows i of Y = A_B^T S over
// the slot's batch rows, 64-row chunks (slots start on chunk boundaries).  The
// A operand is A_B^T: element (i, b) = A[idx_b, i], loaded 8 consecutive i
// at a time (16 bytes of one row of A) into registers one chunk ahead and
// scattered into the K-major tile (2-byte stores).  The B operand is the
// chunk's image of S (mts_put: the three pieces of S_bj, N = 3 P rows, P = k
// padded to 16), copied asynchronously one chunk ahead.  Slices 0-1 and 2-3
// of a chunk accumulate in two accumulators, one commit per chunk.  Output:
// the slot's partial of Y in slot `chunk` of Ys (k_combine adds the slots in
// order).
__global__ void __launch_bounds__(MT_THREADS, 2) k_meas_tc_apply(const SolveDev* sds, int ns) {
    pdl_wait();
    pdl_trigger();
    const int si = find_solve(sds, ns, PK_MAP, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_MAP];
    const int Lb = s.nb_meas, n = s.n, k = s.k, tid = threadIdx.x;
    const int ntile = (n + MT_BM - 1) / MT_BM, nchk = apply_slots(s.kind, Lb, n, 1);
    if (!s.mtc || (s.kind != MEG_MEAS_STOCH && s.kind != MEG_BILINEAR) || lb < 0 || lb >= ntile * nchk) return;
    const int tile = lb % ntile, chunk = lb / ntile;
    const int nc64 = (Lb + MT_BK - 1) / MT_BK;
    const int c_lo = (int)((int64_t)chunk * nc64 / nchk), c_hi = (int)((int64_t)(chunk + 1) * nc64 / nchk);
    const bool full = (s.mode == 1) || s.kind == MEG_BILINEAR;    // batch row b is stacked row b
    const int P = (k + 15) / 16 * 16, N = 3 * P;
    extern __shared__ __align__(1024) unsigned char smraw[];
    const MtSmem m = mt_carve(smraw, 2);
    const uint32_t tmem = mt_setup(m);
    const uint32_t idesc = idesc_bf16(MT_BM, P);
    const int i0 = tile * MT_BM;
    const int warp = tid >> 5, quarter = warp & 3, lane = tid & 31;
    const int grow = quarter * 32 + lane;
    const int ngroups = P / 16;                             // 1 or 2: warps 0-3 take group 0, 4-7 group 1
    const int g = warp >> 2;
    float run[16], rlo[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) run[j] = rlo[j] = 0.f;
    // A^T items of this thread: (batch row kk, 8 consecutive i); consecutive lanes
    // take consecutive kk, so their 2-byte stores to one tile row i fall in
    // different banks
    constexpr int NIT = MT_BK * (MT_BM / 8) / MT_THREADS;   // 4
    uint4 pv[NIT];
    auto fetch = [&](int c) {
#pragma unroll
        for (int j = 0; j < NIT; ++j) {
            const int it = tid + j * MT_THREADS, kk = it % MT_BK, ii = (it / MT_BK) * 8;
            const int b = c * MT_BK + kk;
            pv[j] = make_uint4(0u, 0u, 0u, 0u);
            if (b < Lb && i0 + ii < n) {
                const int64_t row = full ? (int64_t)b : (int64_t)s.bidx[b];
                const unsigned short* rp = stacked_row(s, row);
                if (rp) pv[j] = *(const uint4*)(rp + i0 + ii);
            }
        }
    };
    auto put = [&](int st) {
        unsigned char* As = m.a + st * MT_STAGE;
#pragma unroll
        for (int j = 0; j < NIT; ++j) {
            const int it = tid + j * MT_THREADS, kk = it % MT_BK, ii = (it / MT_BK) * 8;
            const unsigned wds[4] = {pv[j].x, pv[j].y, pv[j].z, pv[j].w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                *(unsigned short*)(As + sw_off(ii + 2 * h, kk)) = (unsigned short)(wds[h] & 0xffffu);
                *(unsigned short*)(As + sw_off(ii + 2 * h + 1, kk)) = (unsigned short)(wds[h] >> 16);
            }
        }
    };
    auto stage_s = [&](int c, int st) {
        unsigned char* Bs = m.b + st * MT_STAGE;
        const unsigned short* src = s.mts + (size_t)c * N * 64;
        for (int it = tid; it < N * 8; it += MT_THREADS) cp_async16(Bs + it * 16, src + it * 8, true);
        cp_async_commit();
    };
    bool ok = true;
    uint32_t parity = 0;
    if (c_lo < c_hi) {
        fetch(c_lo);
        stage_s(c_lo, 0);
    }
    for (int c = c_lo; c < c_hi && ok; ++c) {
        const int st = (c - c_lo) & 1;
        put(st);                                            // chunk c's A^T, from the registers
        if (c + 1 < c_hi) {                                 // chunk c + 1 is read while c is multiplied
            fetch(c + 1);
            stage_s(c + 1, st ^ 1);
        } else {
            cp_async_commit();                              // an empty group: wait_group 1 still means chunk c
        }
        cp_async_wait1();
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {   // pieces of S per accumulation: lo, mid, hi (sub-tiles 2P, P, 0), small first
            tc_fence_after();
            const uint32_t a0 = smem_u32(m.a + st * MT_STAGE), b0 = smem_u32(m.b + st * MT_STAGE);
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int p = 2; p >= 0; --p)
#pragma unroll
                    for (int j = 0; j < 2; ++j) {
                        const int kk = 2 * h + j;
                        umma_bf16(tmem + (uint32_t)(h * 32), sdesc_sw128(a0 + kk * 32),
                                  sdesc_sw128(b0 + (uint32_t)(p * P * 128 + kk * 32)), idesc,
                                  (uint32_t)(p != 2 || j != 0));
                    }
            umma_commit(m.bar);
        }
        const bool done = mbar_wait(m.bar, parity);
        parity ^= 1u;
        ok = __syncthreads_or(done ? 0 : 1) == 0;
        tc_fence_after();
        if (!ok) break;
        if (g < ngroups) {
            const uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
            for (int acc = 0; acc < 2; ++acc) {
                uint32_t v[16];
                tmem_ld16(tb + (uint32_t)(acc * 32 + 16 * g), v);
#pragma unroll
                for (int j = 0; j < 16; ++j) csum_add(run[j], rlo[j], __uint_as_float(v[j]));
            }
        }
        tc_fence_before();
        __syncthreads();                                    // the stage and the accumulators are reused
    }
    cp_async_wait0();                                       // no copy in flight when the CTA ends
    const int i = i0 + grow;
    if (ok && g < ngroups && i < n) {
        float* Ys = (float*)s.Ys + ((size_t)chunk * n + i) * k;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (16 * g + j < k) Ys[16 * g + j] = run[j] + rlo[j];
    }
    mt_teardown(m, tmem, s, !ok);
}

constexpr size_t MT_SMEM = 1024 + 2 * (size_t)MT_STAGE + 64;   // two stages (both passes)

}  // namespace

cudaError_t meas_tc_init() {
    cudaError_t e =
        cudaFuncSetAttribute(k_meas_tc_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MT_SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_meas_tc_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MT_SMEM);
}

cudaError_t launch_meas_tc_batch(const GroupLaunch& g) {
    if (g.blocks[PK_MTB] == 0) return cudaSuccess;
    cudaError_t e = launch_k(k_meas_tc_split, dim3(g.blocks[PK_MTB]), dim3(MT_THREADS), 0, g.stream, 1, g.d_solves,
                             g.ns);
    if (e != cudaSuccess) return e;
    return launch_k(k_meas_tc_batch, dim3(g.blocks[PK_MTB]), dim3(MT_THREADS), MT_SMEM, g.stream, 1, g.d_solves,
                    g.ns);
}

cudaError_t launch_meas_tc_apply(const GroupLaunch& g) {
    if (g.blocks[PK_MAP] == 0) return cudaSuccess;
    return launch_k(k_meas_tc_apply, dim3(g.blocks[PK_MAP]), dim3(MT_THREADS), MT_SMEM, g.stream, 1, g.d_solves,
                    g.ns);
}
