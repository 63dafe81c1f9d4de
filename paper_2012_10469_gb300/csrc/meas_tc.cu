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
// product up to the float32 accumulation.  Each accumulation covers one
// 16-wide K slice (one MMA) and the slices are added in registers as
// compensated float32 sums (an accumulation's error grows with its length on
// the tensor cores, a plain float sum's with the number of terms).
//
// Tiles are staged by the CTA's threads with ordinary loads (the rows of A
// are gathered by the minibatch indices; the apply pass transposes them)
// into the canonical K-major layout with the 128-byte swizzle: row q of a
// tile is 128 bytes (64 bf16 of K), its 16-byte piece c sits at position
// c xor (q mod 8), rows grouped by 8 into 1024-byte atoms.  One thread issues
// each MMA of a chunk (M = 128, N = 3 x columns, K = 16) into tensor memory
// and commits it to an mbarrier; the block waits (bounded: about 1 s,
// then MEG_ERR_TIMEOUT is recorded, the CTA waits for its own MMAs, frees its
// tensor memory and returns) and drains the accumulator with tcgen05.ld.
//
// Bilinear kind: the batch rows are the 2m stacked rows (row i = a_i, row
// m + i = b_i), every step; the finish kernel pairs rows i and m + i into
// r_i = tau a_i^T X b_i - y_i and writes S_i = (tau/2) r_i b_i^T W and
// S_{m+i} = (tau/2) r_i a_i^T W, so the apply pass over the stacked rows gives
// (tau/2) sum_i r_i (a_i b_i^T + b_i a_i^T) W = grad f W.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "meg_dev.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int MT_THREADS = 256;
constexpr int MT_TMEM_COLS = 256;
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

// start of stacked row j: a_j for j < m; for the bilinear kind b_{j - m} for j >= m
__device__ __forceinline__ const unsigned short* stacked_row(const SolveDev& s, int64_t j) {
    if (j < s.m) return (const unsigned short*)s.A + (size_t)j * s.n;
    return (const unsigned short*)s.Bm + (size_t)(j - s.m) * s.n;
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

__device__ __forceinline__ MtSmem mt_carve(unsigned char* raw) {
    MtSmem m;
    unsigned char* base = (unsigned char*)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
    m.a = base;
    m.b = base + MT_A_BYTES;
    m.bar = (uint64_t*)(m.b + MT_B_MAX);
    m.tslot = (uint32_t*)(m.bar + 2);
    m.err = (int*)(m.tslot + 1);
    return m;
}

__device__ __forceinline__ uint32_t mt_setup(const MtSmem& m) {
    if (threadIdx.x == 0) {
        mbar_init(m.bar, 1);
        mbar_init(m.bar + 1, 1);
        *m.err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(m.tslot)),
                     "r"(MT_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return *m.tslot;
}

// One 16-wide K slice of the staged chunk as a fresh accumulation.  The
// tensor cores round each partial sum of an accumulation toward zero, so its
// error grows with the accumulation's length (about 4e-8 K relative for sums
// that cancel, as dot products of random-sign data do); every MMA therefore
// starts afresh and the slices are added in registers as compensated sums.
// Slice 0 makes the staged tiles (generic-proxy stores) visible
// to the tensor cores; a later slice first orders the previous slice's drain
// before the accumulator is overwritten.  One thread issues and commits; the
// block waits for the commit (bounded).  Returns false on timeout.
__device__ __forceinline__ bool mt_mma_slice(const MtSmem& m, uint32_t tmem, uint32_t idesc, uint32_t parity,
                                             int kk) {
    if (kk == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    else tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc_fence_after();
        umma_bf16(tmem, sdesc_sw128(smem_u32(m.a) + kk * 32), sdesc_sw128(smem_u32(m.b) + kk * 32), idesc, 0u);
        umma_commit(m.bar);
    }
    const bool ok = mbar_wait(m.bar, parity);
    const bool bad = __syncthreads_or(ok ? 0 : 1) != 0;      // the same verdict in every thread
    tc_fence_after();
    return !bad;
}

// End of a CTA: on error, wait (bounded) for every MMA this CTA issued and
// flag the solve; free the tensor memory.
__device__ __forceinline__ void mt_teardown(const MtSmem& m, uint32_t tmem, const SolveDev& s, bool bad) {
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
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(MT_TMEM_COLS)
                     : "memory");
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
__global__ void __launch_bounds__(MT_THREADS, 1) k_meas_tc_batch(const SolveDev* sds, int ns) {
    pdl_wait();
    pdl_trigger();
    const int si = find_solve(sds, ns, PK_MTB, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_MTB];
    const int Lb = s.nb_meas, n = s.n, k = s.k, r = s.r, tid = threadIdx.x;
    const int mtiles = (Lb + MT_BM - 1) / MT_BM, KS = meas_ks(Lb, n);
    if (!s.mtc || (s.kind != MEG_MEAS_STOCH && s.kind != MEG_BILINEAR) || lb < 0 || lb >= mtiles * KS) return;
    const int mt = lb % mtiles, part = lb / mtiles;
    const int nch = (n + MT_BK - 1) / MT_BK;
    const int c_lo = (int)((int64_t)part * nch / KS), c_hi = (int)((int64_t)(part + 1) * nch / KS);
    const bool warm = (s.mode == 1);
    const int B = k_bucket(k), NC = 2 * B, N = 3 * NC;
    extern __shared__ __align__(1024) unsigned char smraw[];
    const MtSmem m = mt_carve(smraw);
    __shared__ int64_t rowidx[MT_BM];
    if (tid < MT_BM) {
        const int b = mt * MT_BM + tid;
        rowidx[tid] = b < Lb ? batch_row(s, warm, b) : -1;
    }
    const uint32_t tmem = mt_setup(m);                      // (synchronises the block)
    const uint32_t idesc = idesc_bf16(MT_BM, N);
    const float* W = (const float*)s.W;
    const double* V = s.V;
    // A tile: thread = (row, half of the 64 columns), four 16-byte vectors
    const int arow = tid >> 1, ahalf = tid & 1;
    const int64_t ar = rowidx[arow];
    const unsigned short* arp = ar >= 0 ? stacked_row(s, ar) : nullptr;
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
    bool ok = true;
    uint32_t parity = 0;
    for (int c = c_lo; c < c_hi && ok; ++c) {
        const int k0 = c * MT_BK;
        // ---- A tile (gathered rows)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int kc = ahalf * 4 + v;                   // 16-byte piece of the row
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (ar >= 0 && k0 + kc * 8 < n) val = *(const uint4*)(arp + k0 + kc * 8);
            *(uint4*)(m.a + arow * 128 + ((kc ^ (arow & 7)) << 4)) = val;
            const unsigned wds[4] = {val.x, val.y, val.z, val.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float lo = __uint_as_float(wds[h] << 16), hi = __uint_as_float(wds[h] & 0xffff0000u);
                aa = fmaf(lo, lo, aa);
                aa = fmaf(hi, hi, aa);
            }
        }
        // ---- B tile: N rows (piece, column) x 64 K, one 16-byte vector per item
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
            *(uint4*)(m.b + q * 128 + ((kc ^ (q & 7)) << 4)) = val;
        }
        // K slices beyond n multiply zero columns: skipped
        const int nsl = min(MT_BK / 16, (n - k0 + 15) / 16);
        for (int kk = 0; kk < nsl; ++kk) {
            ok = mt_mma_slice(m, tmem, idesc, parity, kk);
            parity ^= 1u;
            if (!ok) break;
            // ---- drain: hi + mid + lo of each output column, added to the running sums
            const uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16);
#pragma unroll
            for (int gi = 0; gi < 2; ++gi) {
                const int g = (warp >> 2) + 2 * gi;         // this warp's 16-column groups
                if (g < ngroups) {
                    uint32_t vh[16], vm[16], vl[16];
                    tmem_ld16(tb + (uint32_t)(16 * g), vh);
                    tmem_ld16(tb + (uint32_t)(NC + 16 * g), vm);
                    tmem_ld16(tb + (uint32_t)(2 * NC + 16 * g), vl);
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        csum_add(run[gi][j], rlo[gi][j],
                                 (__uint_as_float(vh[j]) + __uint_as_float(vm[j])) + __uint_as_float(vl[j]));
                }
            }
        }
        if (!ok) break;
        tc_fence_before();
        __syncthreads();                                    // tiles and accumulator are reused
    }
    // ---- partials of this part: columns, then ||a||^2 (the two threads of a row add theirs)
    aa += __shfl_xor_sync(0xffffffffu, aa, 1);
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
    mt_teardown(m, tmem, s, !ok);
}

// ==========================================================================
// Apply pass.  CTA (tile, chunk of the batch): 128 rows i of Y = A_B^T S over
// the chunk's batch rows, 64 at a time.  The A operand is A_B^T: element
// (i, b) = A[idx_b, i], loaded 8 consecutive i at a time (16 bytes of one
// row of A) and scattered into the K-major tile (2-byte stores).  The B
// operand holds the pieces of S_bj = (2/Lb) r_b T_bj, N = 3 P rows (P = k
// padded to 16): piece p of column j is row p P + j.  Output: the chunk's
// partial of Y in slot `chunk` of Ys (k_combine adds the slots in order).
__global__ void __launch_bounds__(MT_THREADS, 1) k_meas_tc_apply(const SolveDev* sds, int ns) {
    pdl_wait();
    pdl_trigger();
    const int si = find_solve(sds, ns, PK_MAP, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_MAP];
    const int Lb = s.nb_meas, n = s.n, k = s.k, tid = threadIdx.x;
    const int ntile = (n + MT_BM - 1) / MT_BM, nchk = meas_slots(Lb, 1);
    if (!s.mtc || (s.kind != MEG_MEAS_STOCH && s.kind != MEG_BILINEAR) || lb < 0 || lb >= ntile * nchk) return;
    const int tile = lb % ntile, chunk = lb / ntile;
    const int b_lo = (int)((int64_t)chunk * Lb / nchk), b_hi = (int)((int64_t)(chunk + 1) * Lb / nchk);
    const bool full = (s.mode == 1) || s.kind == MEG_BILINEAR;    // batch row b is stacked row b
    const int P = (k + 15) / 16 * 16, N = 3 * P;
    const float* S = s.mts;                                 // S_b = (2/Lb) r_b T_b (bilinear: see above), rows x k
    extern __shared__ __align__(1024) unsigned char smraw[];
    const MtSmem m = mt_carve(smraw);
    __shared__ int64_t bidx[MT_BK];
    const uint32_t tmem = mt_setup(m);
    const uint32_t idesc = idesc_bf16(MT_BM, N);
    const int i0 = tile * MT_BM;
    const int warp = tid >> 5, quarter = warp & 3, lane = tid & 31;
    const int grow = quarter * 32 + lane;
    const int ngroups = P / 16;                             // 1 or 2: warps 0-3 take group 0, 4-7 group 1
    const int g = warp >> 2;
    float run[16], rlo[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) run[j] = rlo[j] = 0.f;
    bool ok = true;
    uint32_t parity = 0;
    for (int b0 = b_lo; b0 < b_hi && ok; b0 += MT_BK) {
        const int bn = min(MT_BK, b_hi - b0);
        if (tid < MT_BK) bidx[tid] = tid < bn ? (full ? (int64_t)(b0 + tid) : (int64_t)s.bidx[b0 + tid]) : -1;
        __syncthreads();
        // ---- A^T tile: 64 batch rows x 16 vectors of 8 consecutive i
        for (int it = tid; it < MT_BK * (MT_BM / 8); it += MT_THREADS) {
            const int kk = it / (MT_BM / 8), iv = it % (MT_BM / 8);
            const int64_t row = bidx[kk];
            const int ii = iv * 8;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (row >= 0 && i0 + ii < n) val = *(const uint4*)(stacked_row(s, row) + i0 + ii);
            const unsigned wds[4] = {val.x, val.y, val.z, val.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                *(unsigned short*)(m.a + sw_off(ii + 2 * h, kk)) = (unsigned short)(wds[h] & 0xffffu);
                *(unsigned short*)(m.a + sw_off(ii + 2 * h + 1, kk)) = (unsigned short)(wds[h] >> 16);
            }
        }
        // ---- S tile: N rows (piece, column j) x 64 batch rows, 16-byte vectors
        for (int it = tid; it < N * 8; it += MT_THREADS) {
            const int q = it >> 3, kc = it & 7;
            const int p = q / P, j = q % P;
            unsigned short e[8];
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                const int bb = kc * 8 + h;
                const float x = (bb < bn && j < k) ? S[(size_t)(b0 + bb) * k + j] : 0.f;
                e[h] = bf16_piece(x, p);
            }
            uint4 val;
            val.x = (unsigned)e[0] | ((unsigned)e[1] << 16);
            val.y = (unsigned)e[2] | ((unsigned)e[3] << 16);
            val.z = (unsigned)e[4] | ((unsigned)e[5] << 16);
            val.w = (unsigned)e[6] | ((unsigned)e[7] << 16);
            *(uint4*)(m.b + q * 128 + ((kc ^ (q & 7)) << 4)) = val;
        }
        // K slices beyond the chunk's rows multiply zero rows: skipped
        for (int kk = 0; kk < (bn + 15) / 16; ++kk) {
            ok = mt_mma_slice(m, tmem, idesc, parity, kk);
            parity ^= 1u;
            if (!ok) break;
            if (g < ngroups) {
                const uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16);
                uint32_t vh[16], vm[16], vl[16];
                tmem_ld16(tb + (uint32_t)(16 * g), vh);
                tmem_ld16(tb + (uint32_t)(P + 16 * g), vm);
                tmem_ld16(tb + (uint32_t)(2 * P + 16 * g), vl);
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    csum_add(run[j], rlo[j], (__uint_as_float(vh[j]) + __uint_as_float(vm[j])) + __uint_as_float(vl[j]));
            }
        }
        if (!ok) break;
        tc_fence_before();
        __syncthreads();
    }
    const int i = i0 + grow;
    if (ok && g < ngroups && i < n) {
        float* Ys = (float*)s.Ys + ((size_t)chunk * n + i) * k;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (16 * g + j < k) Ys[16 * g + j] = run[j] + rlo[j];
    }
    mt_teardown(m, tmem, s, !ok);
}

constexpr size_t MT_SMEM = 1024 + MT_A_BYTES + MT_B_MAX + 64;

}  // namespace

cudaError_t meas_tc_init() {
    cudaError_t e = cudaFuncSetAttribute(k_meas_tc_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MT_SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_meas_tc_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MT_SMEM);
}

cudaError_t launch_meas_tc_batch(const GroupLaunch& g) {
    if (g.blocks[PK_MTB] == 0) return cudaSuccess;
    return launch_k(k_meas_tc_batch, dim3(g.blocks[PK_MTB]), dim3(MT_THREADS), MT_SMEM, g.stream, 1, g.d_solves,
                    g.ns);
}

cudaError_t launch_meas_tc_apply(const GroupLaunch& g) {
    if (g.blocks[PK_MAP] == 0) return cudaSuccess;
    return launch_k(k_meas_tc_apply, dim3(g.blocks[PK_MAP]), dim3(MT_THREADS), MT_SMEM, g.stream, 1, g.d_solves,
                    g.ns);
}
