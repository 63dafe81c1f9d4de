// Dense gradient part Y = D W on the 5th-generation tensor cores (tcgen05)
// for the mixed-precision path: D is the objective's n x n bfloat16 matrix,
// W the float32 subspace block, split exactly into three bfloat16 pieces
// W = W_hi + W_mid + W_lo (24 mantissa bits) by k_orth2 and stored K-major
// as Wsp[3k padded to 16][n padded to 64].
//
// Persistent stream-K schedule: the launch's work is the sequence of 64-wide
// K chunks of every 128-row tile of every solve (solve by solve, tile by
// tile); CTA c of G (one per SM) takes chunks [cT/G, (c+1)T/G).  Where a
// CTA's range cuts a tile, each piece (segment) is written as its own
// float32 partial (slot = the CTA's index among the tile's CTAs) and
// k_combine sums the tile's slots in slot order, so the result does not
// depend on timing.  Roles inside the CTA (192 threads):
//   - warp 0, one lane: TMA producer, D tiles (128 x 64) and Wsp tiles
//     (N x 64), 128-byte swizzle, into an S-stage mbarrier ring that runs on
//     across segment and tile boundaries (D is streamed once: L2 evict-first);
//   - warp 1, one lane: issues tcgen05.mma kind::f16 (bf16 x bf16 -> fp32),
//     M = 128, N = 3k padded to 16, K = 16, into one of two tensor-memory
//     accumulators (segment i uses accumulator i mod 2);
//   - warps 2-5: epilogue of the other accumulator: tcgen05.ld, the sum
//     hi + mid + lo per column added to a running sum in registers,
//     coalesced float32 stores of the partial at the end of a segment.
// Every mbarrier wait is bounded (about one second of globaltimer); on
// timeout the CTA flags its solves with MEG_ERR_TIMEOUT, waits (bounded) for
// its own copies and MMAs, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "dense_tc.cuh"
#include "meg_dev.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int TC_THREADS = 192;
constexpr int TC_STAGES_MAX = 8;
constexpr int TC_BM = 128;
constexpr int TC_BK = 64;                       // bf16 elements per 128-byte row
constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;   // 16 KB
constexpr int TC_TMEM_COLS = 256;               // two accumulators, 128 columns apart
constexpr int TC_EPI_LD = 33;                   // epilogue staging row (k <= 32 floats)
// The tensor cores add each MMA's products into the float32 accumulator
// with less than round-to-nearest accuracy (the result of each MMA is biased
// toward zero by a fraction of a unit in its last place), so the error of one
// accumulation grows with its length.  An accumulation is therefore
// restarted every TC_SUB chunks and the epilogue adds the sub-results in
// float32 round-to-nearest arithmetic.  Measured on the n = 4096 batch: with
// restarts every 8 chunks (K = 512, 32 MMAs) the top Ritz values were
// 1.6-3e-7 (relative) off the float64 oracle after one iteration and 1.5-3e-6
// after 500; restarting every chunk (K = 64, 4 MMAs) gives 2-5e-8 after one
// iteration (the float32-data path: 1e-9) for 3% more product time.
constexpr int TC_SUB = 1;
constexpr int TC_EPI_BYTES = TC_BM * TC_EPI_LD * 4;
constexpr int TC_SMEM_LIMIT = 227 * 1024;

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

__device__ __forceinline__ void tma_load_2d_hint(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                                 uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%3, %4}], [%2], %5;"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y), "l"(policy)
        : "memory");
}

__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// One segment of a CTA's chunk range: solve, tile, first chunk, chunk count,
// partial slot.
struct TcSeg {
    int si, m0, kb0, len, slot;
};

// Segment of CTA c that starts at chunk g (g < end of the CTA's range).
__device__ __forceinline__ TcSeg tc_segment(const SolveDev* sds, int ns, long long g, long long gend, long long T,
                                            int G, int c) {
    TcSeg q;
    q.si = find_solve(sds, ns, PK_DTC, (int)g);
    const SolveDev& s = sds[q.si];
    const int nkb = s.tc_kpad / TC_BK;
    const long long local = g - s.off[PK_DTC];
    const int mt = (int)(local / nkb);
    q.kb0 = (int)(local % nkb);
    q.m0 = mt * TC_BM;
    q.len = (int)min((long long)(nkb - q.kb0), gend - g);
    q.slot = c - tc_cta_of(g - q.kb0, G, T);
    return q;
}

__global__ void __launch_bounds__(TC_THREADS, 1)
k_dense_tc(const SolveDev* sds, int ns, const __grid_constant__ TcMaps maps, long long T, int S, int b_stride) {
    pdl_wait();
    pdl_trigger();
    const int G = gridDim.x, c = blockIdx.x;
    const long long g_begin = tc_chunk_start(c, G, T), g_end = tc_chunk_start(c + 1, G, T);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = base;                                   // S x 16 KB
    unsigned char* sB = base + (size_t)S * TC_A_BYTES;          // S x b_stride
    float* stage = (float*)(sB + (size_t)S * b_stride);         // 128 x TC_EPI_LD
    uint64_t* full = (uint64_t*)(stage + TC_BM * TC_EPI_LD);
    uint64_t* empty = full + S;
    uint64_t* tfull = empty + S;                                // accumulator ready [2]
    uint64_t* tempty = tfull + 2;                               // accumulator drained [2]
    uint64_t* mdone = tempty + 2;
    uint32_t* tslot = (uint32_t*)(mdone + 1);
    volatile int* err = (volatile int*)(tslot + 1);

    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&tfull[i], 1);
            mbar_init(&tempty[i], 4);
        }
        mbar_init(mdone, 1);
        *err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer
            const uint64_t pol = policy_evict_first();
            int it = 0;
            for (long long g = g_begin; g < g_end && !*err;) {
                const TcSeg q = tc_segment(sds, ns, g, g_end, T, G, c);
                const uint32_t bytes = TC_A_BYTES + (uint32_t)sds[q.si].tc_npad * TC_BK * 2;
                for (int j = 0; j < q.len; ++j, ++it) {
                    const int st = it % S;
                    if (!mbar_wait(&empty[st], ((it / S) & 1) ^ 1)) { *err = 1; break; }
                    mbar_arrive_expect_tx(&full[st], bytes);
                    const int kx = (q.kb0 + j) * TC_BK;
                    tma_load_2d_hint(sA + (size_t)st * TC_A_BYTES, &maps.a[q.si], &full[st], kx, q.m0, pol);
                    tma_load_2d(sB + (size_t)st * b_stride, &maps.b[q.si], &full[st], kx, 0);
                }
                g += q.len;
            }
            if (*err) {
                // drain: wait (bounded) for the copies that may still be in flight
                for (int j = (it > S ? it - S : 0); j < it; ++j) mbar_wait(&full[j % S], (j / S) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            int it = 0, u = 0;                      // u: sub-accumulation counter
            bool ok = true;
            for (long long g = g_begin; g < g_end && ok && !*err;) {
                const TcSeg q = tc_segment(sds, ns, g, g_end, T, G, c);
                const uint32_t idesc = idesc_bf16(TC_BM, sds[q.si].tc_npad);
                for (int j0 = 0; j0 < q.len && ok; j0 += TC_SUB, ++u) {
                    const int ab = u & 1;
                    if (!mbar_wait(&tempty[ab], ((u >> 1) & 1) ^ 1)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t acc = tmem + (uint32_t)(ab * 128);
                    const int j1 = min(q.len, j0 + TC_SUB);
                    for (int j = j0; j < j1; ++j, ++it) {
                        const int st = it % S;
                        if (!mbar_wait(&full[st], (it / S) & 1)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t a0 = smem_u32(sA + (size_t)st * TC_A_BYTES),
                                       b0 = smem_u32(sB + (size_t)st * b_stride);
#pragma unroll
                        for (int kk = 0; kk < TC_BK / 16; ++kk)
                            umma_bf16(acc, sdesc_sw128(a0 + kk * 32), sdesc_sw128(b0 + kk * 32), idesc,
                                      (j > j0 || kk > 0) ? 1u : 0u);
                        umma_commit(&empty[st]);    // frees the stage once these MMAs have read it
                    }
                    if (ok) umma_commit(&tfull[ab]);   // sub-accumulation ab complete
                }
                g += q.len;
            }
            if (!ok) *err = 1;
            umma_commit(mdone);                     // every MMA issued by this thread
            mbar_wait(mdone, 0);
        }
    } else {
        // ---------------- epilogue: warp w reads accumulator lanes 32 (w mod 4) ...
        // The three pieces of W occupy columns [0, P), [P, 2P), [2P, 3P) of the
        // accumulator (P = k rounded up to 16), so one 16-column load holds one
        // piece of 16 output columns and the running sums stay in registers.
        const int quarter = warp & 3;
        const int row = quarter * 32 + lane;
        float* srow = stage + row * TC_EPI_LD;
        int u = 0;
        bool ok = true;
        for (long long g = g_begin; g < g_end && ok && !*err;) {
            const TcSeg q = tc_segment(sds, ns, g, g_end, T, G, c);
            const SolveDev& s = sds[q.si];
            const int n = s.n, k = s.k, P = s.tc_npad / 3;
            float run[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) run[j] = 0.f;
            for (int j0 = 0; j0 < q.len; j0 += TC_SUB, ++u) {
                const int ab = u & 1;
                if (!mbar_wait(&tfull[ab], (u >> 1) & 1)) { ok = false; break; }
                tc_fence_after();
                const uint32_t tb = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ab * 128);
#pragma unroll
                for (int h = 0; h < 2; ++h) {            // output columns [16h, 16h + 16)
                    if (16 * h < P) {
                        uint32_t vh[16], vm[16], vl[16];
                        tmem_ld16(tb + (uint32_t)(16 * h), vh);
                        tmem_ld16(tb + (uint32_t)(P + 16 * h), vm);
                        tmem_ld16(tb + (uint32_t)(2 * P + 16 * h), vl);
#pragma unroll
                        for (int j = 0; j < 16; ++j)      // (hi + mid) + lo, then the running sum
                            run[16 * h + j] += (__uint_as_float(vh[j]) + __uint_as_float(vm[j])) + __uint_as_float(vl[j]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[ab]);
            }
            if (!ok) break;
#pragma unroll
            for (int j = 0; j < 32; ++j)
                if (j < k) srow[j] = run[j];
            __syncwarp();
            // this warp's 32 rows are k * 32 consecutive floats of the partial
            float* Ys = (float*)s.Ys + ((size_t)q.slot * n + q.m0 + quarter * 32) * k;
            const int rows = min(32, n - (q.m0 + quarter * 32));
            for (int e = lane; e < rows * k; e += 32) Ys[e] = stage[(quarter * 32 + e / k) * TC_EPI_LD + e % k];
            __syncwarp();
            g += q.len;
        }
        if (!ok) *err = 1;
    }
    tc_fence_before();
    __syncthreads();
    if (*err && threadIdx.x == 0)
        for (int i = 0; i < ns; ++i) sds[i].sm[SM_STATUS] = MEG_ERR_TIMEOUT;
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
int g_sms = 1;

}  // namespace

// Two resident CTAs per SM (each with half the ring) overlap one CTA's start
// and end of range with the other's streaming: 51.3 -> 47.4 us per launch on
// 8 x n = 4096 (GB300).  With few chunks per CTA the shallower ring costs more
// than it gains, so a launch uses two per SM only when every CTA still gets
// at least TC_TWO_MIN chunks.
constexpr long long TC_TWO_MIN = 32;
int tc_ctas_per_sm(long long T, int sms) { return T >= 2LL * sms * TC_TWO_MIN ? 2 : 1; }

// stages of the ring for a B tile of b_stride bytes, and the dynamic shared memory
int tc_stages(int b_stride, int cps) {
    const int fixed = 1024 + TC_EPI_BYTES + 256;
    const int limit = cps == 1 ? TC_SMEM_LIMIT : (228 * 1024) / 2 - 1024;
    return std::min(TC_STAGES_MAX, (limit - fixed) / (TC_A_BYTES + b_stride));
}

size_t tc_smem_bytes(int S, int b_stride) {
    return 1024 + (size_t)S * (TC_A_BYTES + b_stride) + TC_EPI_BYTES + (2 * S + 5) * 8 + 16;
}

cudaError_t tc_init() {
    if (!g_encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            g_sms = v;
    }
    return cudaFuncSetAttribute(k_dense_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM_LIMIT);
}

// Tensor maps of one solve: A over D (n x n bf16, rows of n elements), B over
// Wsp (npad x kpad bf16).  Both tiles use the 128-byte swizzle; boxes 64 x 128
// and 64 x npad.  Requires n % 8 == 0 (row stride a multiple of 16 bytes).
bool tc_make_maps(const void* D, int n, const void* Wsp, int kpad, int npad, CUtensorMap* a, CUtensorMap* b) {
    if (!g_encode || (n % 8) != 0 || ((uintptr_t)D % 16) != 0 || ((uintptr_t)Wsp % 16) != 0) return false;
    cuuint64_t dimsA[2] = {(cuuint64_t)n, (cuuint64_t)n};
    cuuint64_t strA[1] = {(cuuint64_t)n * 2};
    cuuint32_t boxA[2] = {TC_BK, TC_BM};
    cuuint32_t es[2] = {1, 1};
    CUresult r = g_encode(a, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(D), dimsA, strA, boxA, es,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return false;
    cuuint64_t dimsB[2] = {(cuuint64_t)kpad, (cuuint64_t)npad};
    cuuint64_t strB[1] = {(cuuint64_t)kpad * 2};
    cuuint32_t boxB[2] = {TC_BK, (cuuint32_t)npad};
    r = g_encode(b, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(Wsp), dimsB, strB, boxB, es,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

cudaError_t launch_dense_tc(const SolveDev* d_solves, int ns, long long T, int G, int npad_max, const TcMaps& maps,
                            cudaStream_t st) {
    if (T <= 0 || G <= 0) return cudaSuccess;
    const int b_stride = npad_max * TC_BK * 2;      // a multiple of 2048: keeps 1024-byte tile alignment
    const int S = tc_stages(b_stride, G > g_sms ? 2 : 1);
    return launch_k(k_dense_tc, dim3(G), dim3(TC_THREADS), tc_smem_bytes(S, b_stride), st, 1, d_solves, ns, maps, T,
                    S, b_stride);
}
