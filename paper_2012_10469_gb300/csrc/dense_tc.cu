// Dense gradient part Y = D W on the 5th-generation tensor cores (tcgen05)
// for the mixed-precision path: D is the objective's n x n bfloat16 matrix,
// W the float32 subspace block, split exactly into three bfloat16 pieces
// W = W_hi + W_mid + W_lo (24 mantissa bits) by k_orth2 and stored K-major
// as Wsp[3k padded to 16][n padded to 64].  One CTA computes a 128-row tile
// of [D W_hi | D W_mid | D W_lo] over one K split:
//   - warp 0, one lane: TMA producer, 64-column K blocks of D (128 x 64) and
//     Wsp (N x 64), 128-byte swizzle, into a 3-stage mbarrier ring;
//   - warp 1, one lane: issues tcgen05.mma kind::f16 (bf16 x bf16 -> fp32 in
//     tensor memory), M = 128, N = 3k padded to 16, K = 16 per instruction;
//   - all four warps: tcgen05.ld of the accumulator, sum of the three pieces,
//     float32 partial of this K split written to Ys (summed in k_combine).
// Every mbarrier wait is bounded (about one second of globaltimer); on
// timeout the CTA flags the solve with MEG_ERR_TIMEOUT, drains its own copies
// and MMAs (again bounded), frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "dense_tc.cuh"
#include "meg_dev.cuh"

namespace {

constexpr int TC_THREADS = 128;
constexpr int TC_STAGES = 3;
constexpr int TC_BM = 128;
constexpr int TC_BK = 64;                       // bf16 elements per 128-byte row
constexpr int TC_A_BYTES = TC_BM * TC_BK * 2;   // 16 KB
constexpr int TC_B_MAX = TC_NMAX * TC_BK * 2;   // 12 KB
constexpr int TC_TMEM_COLS = 128;
constexpr unsigned long long TC_WAIT_NS = 1000000000ull;   // 1 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait: false after about TC_WAIT_NS without completion
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (gtimer() - t0 > TC_WAIT_NS) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];"
        ::"r"(smem_u32(dst)), "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// tcgen05 shared-memory matrix descriptor: K-major, 128-byte swizzle,
// 8-row groups 1024 bytes apart (stride byte offset), version bits 46-48 = 1.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride byte offset
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
    return d;
}

// instruction descriptor, kind::f16: D f32, A bf16, B bf16, both K-major, N, M
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__global__ void __launch_bounds__(TC_THREADS, 1)
k_dense_tc(const SolveDev* sds, int ns, const __grid_constant__ TcMaps maps) {
    const int si = find_solve(sds, ns, PK_DTC, blockIdx.x);
    const SolveDev& s = sds[si];
    const int lb = blockIdx.x - s.off[PK_DTC];
    const int nblk = s.nb_tm * s.nb_ds;
    if (lb < 0 || lb >= nblk) return;
    const int n = s.n, k = s.k, npad = s.tc_npad;
    const int mt = lb % s.nb_tm, sp = lb / s.nb_tm;
    const int m0 = mt * TC_BM;
    const int k0 = sp * s.ks_len, k1 = min(n, k0 + s.ks_len);
    const int nkb = (k1 - k0 + TC_BK - 1) / TC_BK;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t b_bytes = (uint32_t)npad * TC_BK * 2;

    extern __shared__ __align__(1024) unsigned char smraw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = base;                                   // TC_STAGES x 16 KB
    unsigned char* sB = base + TC_STAGES * TC_A_BYTES;          // TC_STAGES x 12 KB
    uint64_t* full = (uint64_t*)(sB + TC_STAGES * TC_B_MAX);
    uint64_t* empty = full + TC_STAGES;
    uint64_t* accb = empty + TC_STAGES;
    uint32_t* tslot = (uint32_t*)(accb + 1);
    int* err = (int*)(tslot + 1);

    if (threadIdx.x == 0) {
        for (int i = 0; i < TC_STAGES; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        mbar_init(accb, 1);
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
    const CUtensorMap* mapA = &maps.a[si];
    const CUtensorMap* mapB = &maps.b[si];

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer
        int issued = 0;
        for (int it = 0; it < nkb; ++it) {
            const int st = it % TC_STAGES;
            const uint32_t par = ((it / TC_STAGES) & 1) ^ 1;
            if (!mbar_wait(&empty[st], par)) { *err = 1; break; }
            mbar_arrive_expect_tx(&full[st], TC_A_BYTES + b_bytes);
            const int kx = k0 + it * TC_BK;
            tma_load_2d(sA + st * TC_A_BYTES, mapA, &full[st], kx, m0);
            tma_load_2d(sB + st * TC_B_MAX, mapB, &full[st], kx, 0);
            ++issued;
        }
        if (*err) {
            // drain: wait (bounded) for the copies already in flight
            for (int it = (issued > TC_STAGES ? issued - TC_STAGES : 0); it < issued; ++it)
                mbar_wait(&full[it % TC_STAGES], (it / TC_STAGES) & 1);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer
        const uint32_t idesc = idesc_bf16(TC_BM, npad);
        int done = 0;
        for (int it = 0; it < nkb; ++it) {
            const int st = it % TC_STAGES;
            if (!mbar_wait(&full[st], (it / TC_STAGES) & 1)) { *err = 1; break; }
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA + st * TC_A_BYTES), b0 = smem_u32(sB + st * TC_B_MAX);
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk)
                umma_bf16(tmem, sdesc_sw128(a0 + kk * 32), sdesc_sw128(b0 + kk * 32), idesc,
                          (it > 0 || kk > 0) ? 1u : 0u);
            umma_commit(&empty[st]);        // frees the stage once these MMAs have read it
            ++done;
        }
        umma_commit(accb);                  // accumulator complete (all MMAs issued so far)
    }
    __syncwarp();
    // ---------------- epilogue: every thread owns one accumulator row
    const bool ok_acc = mbar_wait(accb, 0);
    tc_fence_after();
    float* stage = (float*)sA;              // reuse the A ring: 128 rows x (npad + 1) floats
    const int ld = npad + 1;
    const int row = warp * 32 + lane;
    if (ok_acc) {
        for (int c0 = 0; c0 < npad; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) stage[row * ld + c0 + j] = __uint_as_float(v[j]);
        }
    }
    const int gi = m0 + row;
    if (ok_acc && !*err && gi < n) {
        float* Ys = (float*)s.Ys + ((size_t)sp * n + gi) * k;
        for (int c = 0; c < k; ++c)
            Ys[c] = stage[row * ld + c] + stage[row * ld + k + c] + stage[row * ld + 2 * k + c];
    }
    tc_fence_before();
    __syncthreads();
    if ((!ok_acc || *err) && threadIdx.x == 0) s.sm[SM_STATUS] = MEG_ERR_TIMEOUT;
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                     : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

}  // namespace

size_t tc_smem_bytes() { return 1024 + TC_STAGES * (TC_A_BYTES + TC_B_MAX) + (2 * TC_STAGES + 1) * 8 + 16; }

cudaError_t tc_init() {
    if (!g_encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    }
    return cudaFuncSetAttribute(k_dense_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes());
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

cudaError_t launch_dense_tc(const SolveDev* d_solves, int ns, int blocks, const TcMaps& maps, cudaStream_t st) {
    if (blocks == 0) return cudaSuccess;
    k_dense_tc<<<blocks, TC_THREADS, tc_smem_bytes(), st>>>(d_solves, ns, maps);
    return cudaGetLastError();
}
