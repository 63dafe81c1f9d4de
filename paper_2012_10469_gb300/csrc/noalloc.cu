// meg_objective_dense_noalloc: the dense-quadratic objective pass for
// callers that cannot allocate device memory.
//
// Who cannot allocate: code that runs while a CUDA graph is being captured
// in global or thread-local capture mode (cudaMalloc/cudaFree may
// synchronise the device and are refused during such a capture), serving
// loops that admitted a solve against a fixed device-memory budget and
// must not grow it afterwards, and hosts that hand this library a context
// whose memory is managed by someone else.  They pass only their own
// inputs and output; the reduction scratch lives in a fixed device array
// of this library.
//
// The scratch array is a file-scope __device__ symbol: every GPU that
// loads the library holds it until the process exits.  In host code its
// name is only a stand-in, so the device address is looked up with
// cudaGetSymbolAddress once per device (on the first call made on that
// device, with the device current) and cached together with the CUDA
// context it belongs to.  A device reset or a new primary context reloads
// the module, which may move the array: a call that finds another current
// context than the cached one looks the address up again.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "meg_dev.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_ROWS = 16;                                    // rows per block
constexpr int NA_MAX_BLOCKS = MEG_NOALLOC_MAX_N / NA_ROWS;     // 4096
constexpr int NA_GROUP = 16;
constexpr int NA_MAX_GROUPS = NA_MAX_BLOCKS / NA_GROUP;        // 256
constexpr size_t NA_PART_BYTES = sizeof(dw) * (NA_MAX_BLOCKS + NA_MAX_GROUPS);
constexpr size_t NA_CTR_BYTES = sizeof(unsigned) * (NA_MAX_GROUPS + 1);
constexpr size_t NA_BYTES = NA_PART_BYTES + NA_CTR_BYTES;      // about 35 KB

struct MuArg { double c[MEG_RMAX + 1]; };                      // mu_l - s, then s

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

namespace {

template <typename T>
__device__ __forceinline__ double na_load(const void* M, size_t idx, int prec) {
    if (prec == MEG_MIXED_BF16) {
        unsigned short b = ((const unsigned short*)M)[idx];
        return (double)__uint_as_float(((unsigned)b) << 16);
    }
    return (double)((const T*)M)[idx];
}

// f = 1/2 sum_ij (X_ij - M_ij)^2, X = V diag(mu - s) V^T + s I; X_ij - M_ij in
// double-word (float storage) or float64 arithmetic, compensated sums, and a
// two-level last-block reduction through the fixed scratch array.
template <typename T>
__global__ void __launch_bounds__(NA_THREADS)
k_objective_noalloc(const double* __restrict__ V, MuArg coef, int n, int r, const void* M, int prec,
                    unsigned char* scratch, double* f_out) {
    const int tid = threadIdx.x, lb = blockIdx.x, nb = gridDim.x;
    dw* part = (dw*)scratch;
    unsigned* ctr = (unsigned*)(scratch + NA_PART_BYTES);
    Acc<T> acc;
    acc.zero();
    const int row0 = lb * NA_ROWS, row1 = min(n, row0 + NA_ROWS);
    for (int i = row0; i < row1; ++i) {
        double wi[MEG_RMAX];
        for (int l = 0; l < r; ++l) wi[l] = V[(size_t)i * r + l] * coef.c[l];
        for (int j = tid; j < n; j += NA_THREADS) {
            const double d = na_load<T>(M, (size_t)i * n + j, prec);
            if constexpr (sizeof(T) == 8) {
                double x = (j == i) ? coef.c[MEG_RMAX] : 0.0;
                for (int l = 0; l < r; ++l) x = fma(wi[l], V[(size_t)j * r + l], x);
                const double R = x - d;
                acc.add_prod(R, R);
            } else {
                dw x = dw_from_double((j == i) ? coef.c[MEG_RMAX] : 0.0);
                for (int l = 0; l < r; ++l) {
                    const double w = wi[l], v = V[(size_t)j * r + l];
                    const float wh = (float)w, wl = (float)(w - (double)wh);
                    const float vh = (float)v, vl = (float)(v - (double)vh);
                    dot2_acc(x, wh, vh);
                    dot2_acc(x, wh, vl);
                    dot2_acc(x, wl, vh);
                }
                float hi, e;
                two_sum(x.hi, -(float)d, hi, e);
                const float R = __fadd_rn(hi, __fadd_rn(e, x.lo));
                acc.add_prod(R, R);
            }
        }
    }
    __shared__ dw ent[NA_THREADS];
    __shared__ int am_last;
    ent[tid] = acc.as_dw();
    __syncthreads();
    if (tid == 0) {
        dw a = {0.f, 0.f};
        for (int q = 0; q < NA_THREADS; ++q) dw_add(a, ent[q]);
        part[lb] = a;
        __threadfence();
        const int g = lb / NA_GROUP, g0 = g * NA_GROUP, gsz = min(NA_GROUP, nb - g0);
        am_last = (atomicAdd(&ctr[g], 1u) == (unsigned)(gsz - 1));
    }
    __syncthreads();
    if (!am_last || tid != 0) return;
    const int g = lb / NA_GROUP, g0 = g * NA_GROUP, gsz = min(NA_GROUP, nb - g0);
    const int ngroups = (nb + NA_GROUP - 1) / NA_GROUP;
    dw a = {0.f, 0.f};
    for (int b = g0; b < g0 + gsz; ++b) {
        dw v = {__ldcg(&part[b].hi), __ldcg(&part[b].lo)};
        dw_add(a, v);
    }
    part[NA_MAX_BLOCKS + g] = a;
    __threadfence();
    if (atomicAdd(&ctr[NA_MAX_GROUPS], 1u) != (unsigned)(ngroups - 1)) return;
    dw tot = {0.f, 0.f};
    for (int q = 0; q < ngroups; ++q) {
        dw v = {__ldcg(&part[NA_MAX_BLOCKS + q].hi), __ldcg(&part[NA_MAX_BLOCKS + q].lo)};
        dw_add(tot, v);
    }
    *f_out = 0.5 * dw_value(tot);
}

std::mutex g_na_mu;
void* g_na_ptr[128] = {nullptr};
CUcontext g_na_ctx[128] = {nullptr};

// the calling thread's current context (driver entry point, looked up once)
typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
CUcontext current_context() {
    static PfnCtxGetCurrent fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        return (PfnCtxGetCurrent)p;
    }();
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

}  // namespace

namespace meg_internal {
void set_last_error(const std::string& msg);   // meg_api.cu: message returned by meg_last_error()
}

static meg_status na_fail(meg_status st, const std::string& msg) {
    meg_internal::set_last_error("meg_objective_dense_noalloc: " + msg);
    return st;
}

extern "C" meg_status meg_objective_dense_noalloc(const double* V, const double* mu, double s, int n, int r,
                                                  const void* M, int precision, double* f_out, void* stream) {
    if (!V || !mu || !M || !f_out) return na_fail(MEG_ERR_INVALID_ARG, "null argument");
    if (n < 2 || n > MEG_NOALLOC_MAX_N)
        return na_fail(MEG_ERR_INVALID_ARG, "n must lie in [2, MEG_NOALLOC_MAX_N = 65536] (fixed scratch size)");
    if (r < 1 || r > MEG_RMAX || r >= n) return na_fail(MEG_ERR_INVALID_ARG, "need 1 <= r <= min(n - 1, 30)");
    if (precision < MEG_FP64 || precision > MEG_MIXED_BF16) return na_fail(MEG_ERR_INVALID_ARG, "unknown precision");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return na_fail(MEG_ERR_CUDA, "cudaGetDevice");
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        CUcontext ctx = g_na_ptr[dev] ? current_context() : nullptr;
        if (!g_na_ptr[dev] || ctx != g_na_ctx[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess) return na_fail(MEG_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_na_ptr[dev] = p;
            g_na_ctx[dev] = current_context();   // the lookup made the device's context current
        }
        scratch = g_na_ptr[dev];
    }
    MuArg coef;
    for (int l = 0; l < r; ++l) coef.c[l] = mu[l] - s;
    coef.c[MEG_RMAX] = s;
    cudaStream_t st = (cudaStream_t)stream;
    // the counters must start at zero; partial sums are overwritten before use
    cudaError_t e = cudaMemsetAsync((unsigned char*)scratch + NA_PART_BYTES, 0, NA_CTR_BYTES, st);
    if (e != cudaSuccess) return na_fail(MEG_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
    const int blocks = (n + NA_ROWS - 1) / NA_ROWS;
    if (precision == MEG_FP64)
        k_objective_noalloc<double><<<blocks, NA_THREADS, 0, st>>>(V, coef, n, r, M, precision,
                                                                   (unsigned char*)scratch, f_out);
    else
        k_objective_noalloc<float><<<blocks, NA_THREADS, 0, st>>>(V, coef, n, r, M, precision,
                                                                  (unsigned char*)scratch, f_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(MEG_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return MEG_OK;
}
