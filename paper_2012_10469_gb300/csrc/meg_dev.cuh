// Device-side structures and helpers of the low-rank MEG library.
//
// One "solve" is one instance of Algorithm 2 (Garber & Kaplan).  Kernels are
// grouped: a launch covers every solve of a group, each block finds its solve
// from per-solve block offsets.  Storage type T of the n x k blocks is double
// (MEG_FP64) or float (MEG_FP32, MEG_MIXED_BF16).  The k x k "island" (Gram
// matrices, Cholesky factors, Rayleigh-Ritz matrix, Ritz values, log-sum-exp,
// certificate) is float64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/meg.h"
#include <cuda_bf16.h>

#include "dense_tc.cuh"

#define MEG_KMAX 32
#define MEG_RMAX 30
#define MEG_NMAX (1 << 28)      // largest n of a solve (sizes stay within int arithmetic)
#define MEG_LDK 33              // leading dimension of k x k matrices in shared memory

// ---------------------------------------------------------------------------
// Small float64 state of a solve: scalars followed by k x k blocks (ld 32).
enum SmallSlot : int {
    SM_T = 0,          // index t of the next iteration (X_t is the current iterate)
    SM_EPS,            // eps_t of the iteration in progress
    SM_S,              // s of X_t (spectrum value off span V)
    SM_LOGS,           // log s of X_t (set with s: by the exp-map, meg_create, checkpoints)
    SM_SHIFT,          // c: the subspace iteration runs on M_t - c I
    SM_C0,             // identity coefficient of M_t (without the shift)
    SM_ALPHA,          // coefficient of the gradient product Y in M_t W
    SM_GNORM,          // bound on ||grad f(X_t)||_2 used for the shift
    SM_FEST,           // objective estimate (DENSE_QUAD, LINEAR)
    SM_CERT,           // certificate of the last iteration
    SM_HOLDS,          // 1 if it held
    SM_FIRST_HOLD,     // first iteration at which it held (0 = never)
    SM_STATUS,         // MEG_OK or an error code set on the device
    SM_TRD,            // Tr D of the dense objective data
    SM_FROD2,          // ||D||_F^2
    SM_LAST_T,         // t of the iteration that produced the stored Ritz values
    SM_LSE,            // log-sum-exp of sigma_1..r of the last iteration
    SM_RSS,            // CSR: max_i sum_j |R_ij| of the last gradient pass (bounds ||grad f||_2)
    SM_RESID_BOUND,    // MEAS: spectral estimate of the minibatch gradient (see k_meas_batch)
    SM_ETA,            // eta
    SM_JSWEEPS,        // Jacobi sweeps of the last Rayleigh-Ritz step (diagnostic)
    SM_F1,             // f(X_1), the denominator of meg_solve's relative gap (NaN = unknown)
    SM_SOLVE_TOL,      // meg_solve: gap tolerance
    SM_SOLVE_FSTAR,    //   known optimal value f*
    SM_SOLVE_LIMIT,    //   chunks of iterations the device loop may run
    SM_SOLVE_CHUNKS,   //   chunks run so far
    SM_SOLVE_DONE,     //   1 once the gap test held
    SM_SOLVE_F,        //   f(X_t) at the last check
    SM_SKREL,          // sigma_k - log s of the last Rayleigh-Ritz step (the block's lowest Ritz value
                       //   relative to the bulk level log s of the iterate it was computed at)
    SM_MU = 32,        // [32] mu of X_t
    SM_DCOEF = 64,     // [32] coefficients of V diag(.) V^T in M_t
    SM_SIGMA = 96,     // [32] Ritz values of the last Rayleigh-Ritz, unshifted
    SM_U = 128,        // V^T W       (r x k)
    SM_G = SM_U + 1024,     // W^T W  (k x k)
    SM_P = SM_G + 1024,     // W^T Y  (k x k)
    SM_S1 = SM_P + 1024,    // Z^T Z  (k x k)
    SM_M1 = SM_S1 + 1024,   // first CholQR right factor (k x k), W' = Z M1
    SM_M2 = SM_M1 + 1024,   // second CholQR right factor, W = W' M2
    SM_QV = SM_M2 + 1024,   // rotation to the Ritz vectors: V_{t+1} = W QV[:, :r]
    // block Krylov (two blocks W0, W1 of one iteration; W1 is current after the
    // first product's orthonormalisation)
    SM_U0 = SM_QV + 1024,   // V^T W0      (r x k)
    SM_G0 = SM_U0 + 1024,   // W0^T W0     (k x k)
    SM_G01 = SM_G0 + 1024,  // W0^T W1     (k x k)
    SM_H00 = SM_G01 + 1024, // W0^T (M_t - c I) W0
    SM_KC = SM_H00 + 1024,  // C M, C = G0^{-1} W0^T Z the projection of Z = (M_t - c I) W0 on W0
    SM_QW = SM_KC + 1024,   // [W0 W1] QW = the next block (2k x k)
    SM_LOGMU = SM_QW + 1024, // [32] log mu of X_t, set with mu (the next iteration needs no logarithm)
    SM_TOTAL = SM_LOGMU + 32
};

// Work-partition kinds (one offset table per kind in a group).
enum PartKind : int { PK_RED = 0, PK_DENSE = 1, PK_CSR = 2, PK_MEAS = 3, PK_DTC = 4, PK_MAP = 5, PK_MTB = 6,
                     PK_COUNT = 7 };

// Minibatch kernels (MEAS_STOCH).  k_meas_batch: MB_ROWS batch rows per
// block as a small tiled product [rows of A] x [V | W], MB_TILE elements of
// the rows staged at a time.
// k_meas_apply: MA_ROWS rows of Y per block times one chunk of the batch;
// a batch of more than MA_CHUNK rows (the warm start's full set of m
// measurements) is split into up to MEAS_CHUNKS chunks whose partial
// products k_combine sums in chunk order.
#define MB_ROWS 32
#define MB_TILE 64
#define MA_ROWS 64
#define MA_CHUNK 256
#define MEAS_CHUNKS 16
// compile-time widths the minibatch and objective kernels specialise on
__host__ __device__ __forceinline__ int rank_bucket(int r) { return r <= 2 ? 2 : r <= 4 ? 4 : r <= 8 ? 8 : r <= 16 ? 16 : 32; }
__host__ __device__ __forceinline__ int k_bucket(int k) { return k <= 8 ? 8 : k <= 16 ? 16 : 32; }
__host__ __device__ __forceinline__ int meas_chunks(int Lb) {
    const int c = (Lb + MA_CHUNK - 1) / MA_CHUNK;
    return c < MEAS_CHUNKS ? (c > 0 ? c : 1) : MEAS_CHUNKS;
}
// Minibatch products on the tensor cores (meas_tc.cu), float storage: the
// batch pass tiles the Lb gathered rows of A by 128 and splits the n-long
// contraction into meas_ks(Lb, n) parts (for a 256-row minibatch one
// 64-wide K chunk per CTA); its float partials, (2 B + 1) per row and part,
// go to mtp.  The apply pass splits the batch into meas_slots partial slots
// (64 batch rows each for a minibatch), which k_combine adds in order.
#define MT_BM 128
#define MT_BK 64
__host__ __device__ __forceinline__ int meas_ks(int Lb, int n) {
    const int mtiles = (Lb + MT_BM - 1) / MT_BM, nch = (n + MT_BK - 1) / MT_BK;
    int ks = (64 + mtiles - 1) / mtiles;
    if (ks > 32) ks = 32;
    if (ks > nch) ks = nch;
    return ks < 1 ? 1 : ks;
}
__host__ __device__ __forceinline__ int meas_slots(int Lb, int mtc) {
    if (!mtc) return meas_chunks(Lb);
    const int c = (Lb + MT_BK - 1) / MT_BK;
    return c < MEAS_CHUNKS ? (c > 0 ? c : 1) : MEAS_CHUNKS;
}
// The bilinear kind's apply pass runs over all 2 m stacked rows every
// product: it is split into enough slots that the grid (row tiles of Y times
// slots) holds about four CTAs per SM, at most BIL_SLOTS_MAX.
#define BIL_SLOTS_MAX 256
__host__ __device__ __forceinline__ int bil_slots(int Lb, int n) {
    const int ntile = (n + MT_BM - 1) / MT_BM, c = (Lb + MT_BK - 1) / MT_BK;
    int sl = (4 * 152 + ntile - 1) / ntile;
    if (sl > BIL_SLOTS_MAX) sl = BIL_SLOTS_MAX;
    if (sl > c) sl = c;
    return sl > 0 ? sl : 1;
}
// Image of the tensor-core apply pass's S operand: per 64-row chunk of the
// batch rows, 3 P rows (P = k padded to 16; the exact three-piece bf16 split,
// piece p of column j at row p P + j) of 64 bf16 values, laid out byte for
// byte as the 128-byte-swizzled K-major shared-memory tile (3 P x 128 bytes
// per chunk), so that the apply pass copies it with 16-byte loads.
__host__ __device__ __forceinline__ size_t mts_image_bytes(int64_t rows, int k) {
    return (size_t)((rows + 63) / 64) * 3 * ((k + 15) / 16 * 16) * 128;
}
#ifdef __CUDACC__
// piece p (0: hi, 1: mid, 2: lo) of the exact three-piece bf16 split of x
__device__ __forceinline__ unsigned short split_piece(float x, int p) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    if (p == 0) return __bfloat16_as_ushort(h);
    const float r1 = x - __bfloat162float(h);
    const __nv_bfloat16 md = __float2bfloat16_rn(r1);
    if (p == 1) return __bfloat16_as_ushort(md);
    return __bfloat16_as_ushort(__float2bfloat16_rn(r1 - __bfloat162float(md)));
}
// Rows b0 .. b0 + 31 of S (b0 a multiple of 32) from shared memory, sx[rr * ld + j]
// for row b0 + rr and column j < k (rows past the batch hold 0), written as
// 16-byte pieces: half of one chunk's 64 K positions in all 3 P image rows.
// Every thread of the block takes part.
__device__ __forceinline__ void mts_put32(unsigned short* img, int k, int64_t b0, const float* sx, int ld) {
    const int P = (k + 15) / 16 * 16, kc0 = (int)(b0 & 63) >> 3;
    unsigned char* base = (unsigned char*)img + (size_t)(b0 >> 6) * 3 * P * 128;
    for (int e = threadIdx.x; e < 3 * P * 4; e += blockDim.x) {
        const int q = e >> 2, v = e & 3, p = q / P, j = q % P;
        unsigned short h[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) h[t] = split_piece(j < k ? sx[(v * 8 + t) * ld + j] : 0.f, p);
        uint4 val;
        val.x = (unsigned)h[0] | ((unsigned)h[1] << 16);
        val.y = (unsigned)h[2] | ((unsigned)h[3] << 16);
        val.z = (unsigned)h[4] | ((unsigned)h[5] << 16);
        val.w = (unsigned)h[6] | ((unsigned)h[7] << 16);
        *(uint4*)(base + q * 128 + (((kc0 + v) ^ (q & 7)) << 4)) = val;
    }
}
// one element of S (any row)
__device__ __forceinline__ void mts_put(unsigned short* img, int k, int64_t b, int j, float x) {
    const int P = (k + 15) / 16 * 16, kk = (int)(b & 63);
    unsigned char* base = (unsigned char*)img + (size_t)(b >> 6) * 3 * P * 128;
    unsigned short pc[3];
    const float h = __bfloat162float(__float2bfloat16_rn(x));
    const float r1 = x - h, md = __bfloat162float(__float2bfloat16_rn(r1));
    pc[0] = __bfloat16_as_ushort(__float2bfloat16_rn(x));
    pc[1] = __bfloat16_as_ushort(__float2bfloat16_rn(r1));
    pc[2] = __bfloat16_as_ushort(__float2bfloat16_rn(r1 - md));
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const int q = p * P + j;
        *(unsigned short*)(base + q * 128 + ((((kk >> 3) ^ (q & 7))) << 4) + (kk & 7) * 2) = pc[p];
    }
}
#endif

// Bilinear kind: the stacked batch rows come in 128-row tiles, tile t holding
// the 64 pairs 64 t .. 64 t + 63: its rows 0-63 are their a, rows 64-127 their b
// (pairs past the last one are zero rows), so that one batch-pass CTA sees
// both halves of its pairs and finishes them in its epilogue; the CTA covers
// all of n (one part).
__host__ __device__ __forceinline__ int64_t bil_rows(int64_t pairs) { return 128 * ((pairs + 63) / 64); }
__host__ __device__ __forceinline__ int batch_ks(int kind, int Lb, int n) {
    return kind == MEG_BILINEAR ? 1 : meas_ks(Lb, n);
}
// partial-product slots of a member's apply pass (k_combine adds them in order)
__host__ __device__ __forceinline__ int apply_slots(int kind, int Lb, int n, int mtc) {
    return kind == MEG_BILINEAR ? bil_slots(Lb, n) : meas_slots(Lb, mtc);
}

#define RED_GROUP 16            // blocks per first-level group of a reduction
#define ROWS_MAX 64             // rows per block of the row-reduction kernels, at most
#define RED_CLUSTER 8           // row blocks of a thread-block cluster; one partial per cluster
#define RED_MAX_ENTRIES 1536    // >= k(k+1)/2 + r k for k <= 32, r <= 30 (orth2: 528 + 960)

// Device descriptor of one solve.  Read-only for kernels (state lives in the
// arrays it points to).
struct SolveDev {
    int n, r, k, kind, prec, q;
    int mode;            // 0: MEG iterations, 1: warm start (operator -grad f(0))
    int nb_red;          // blocks of the row-reduction kernels
    int rows_red;        // rows per reduction block
    int nb_dm, nb_ds;    // dense product: row tiles, K splits
    int ks_len;          // K extent of one split (multiple of the K tile)
    int nb_csr, nb_meas; // blocks of the CSR / measurement kernels
    int tc;              // 1: dense product on tcgen05 (bf16 data, n % 8 == 0)
    int eig;             // MEG_EIG_SUBSPACE or MEG_EIG_BLOCK_KRYLOV
    int mtc;             // 1: minibatch products on tcgen05 (bf16 A, n % 8 == 0, float storage)
    float* mtp;          // partials of the tensor-core batch pass (meas_ks parts x rows x (2 B + 1))
    unsigned short* mts; // the apply pass's operand S (S_b = (2/Lb) r_b a_b^T W) as its split image (mts_put)
    unsigned short* mtb; // split [V | W] image of the batch pass's B operand (ceil(n/64) x 3 2B x 64 bf16)
    int nb_tm;           // tensor-core path: 128-row tiles
    int tc_npad, tc_kpad;// Wsp: (3k padded to 16) x (n padded to 64) bf16
    int tc_G;            // tensor-core launch holding this solve: CTAs
    long long tc_T;      //   and total K chunks (this solve's first chunk is off[PK_DTC])
    int off[PK_COUNT];   // first block of this solve in a grouped launch
    double* V;           // n x r   float64 in every mode: V of X_t
    double* Vn;          // n x r   float64: V of X_{t+1} being formed
    void* W;             // n x k   (T)  current subspace block
    void* Wp;            // n x k   (T)  after the first CholQR pass
    void* Z;             // n x k   (T)  (M_t - c I) W
    void* Y;             // n x k   (T)  gradient-part product
    void* Ys;            // nb_ds x n x k (T) split-K partials of the dense product
    unsigned short* Wsp; // bf16 bits of W = W_hi + W_mid + W_lo, K-major (tensor-core path)
    float* part;         // reduction partials: [nb_red + groups][2 * RED_MAX_ENTRIES]
    unsigned* ctr;       // reduction counters: [groups + 1]
    double* sm;          // SmallSlot state
    double* meas;        // measurement scratch: [L] residuals, [L] ||a||^2, [L x k] A_B W
    int* bidx;           // [L] minibatch indices of the iteration in progress
    // objective (borrowed)
    const void* D;
    const int* rowptr;
    const int* col;
    const void* val;
    int64_t nnz;
    const void* A;
    const double* y;
    int64_t m;
    int L;
    const void* Bm;      // BILINEAR: the b_i (m x n bf16); A holds the a_i
    double tau;          // BILINEAR: trace scale of the tau-spectrahedron
    int mrank;           // BILINEAR: rank p of the measurement matrices; m counts the m p (a, b) pairs,
                         //   and the p consecutive pairs of measurement i share r_i and y_i
    // schedule
    double eta, eps_a, eps_c, eps_pow;
    double log_nr;       // log(n - r), used by the certificate
    uint64_t seed;
};

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  Every kernel of the library begins with
// pdl_wait() -- it returns once the preceding kernel on the stream has
// completed and its memory is visible, before any global data is touched --
// and then pdl_trigger(), which lets the next kernel's blocks be launched and
// placed while this one runs.  The attribute is set only with MEG_PDL=1 in
// the environment; without it both instructions are no-ops and the launches
// are plain stream-ordered launches.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

bool meg_pdl_enabled();

// Launch with the programmatic-serialization attribute and, for cluster > 1,
// thread-block clusters of that size.
template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, int cluster,
                     Args... args) {
    if (grid.x == 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    unsigned na = 0;
    if (cluster > 1) {
        attr[na].id = cudaLaunchAttributeClusterDimension;
        attr[na].val.clusterDim.x = cluster;
        attr[na].val.clusterDim.y = 1;
        attr[na].val.clusterDim.z = 1;
        ++na;
    }
    if (meg_pdl_enabled()) {
        attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[na].val.programmaticStreamSerializationAllowed = 1;
        ++na;
    }
    cfg.attrs = attr;
    cfg.numAttrs = na;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// ---------------------------------------------------------------------------
// Block -> solve lookup for grouped launches.
__device__ __forceinline__ int find_solve(const SolveDev* sd, int ns, int kind, int b) {
    int lo = 0, hi = ns - 1;
    while (lo < hi) {                       // last solve with off[kind] <= b
        int mid = (lo + hi + 1) >> 1;
        if (sd[mid].off[kind] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Stream-K split of T work chunks over G CTAs: CTA c owns [start(c), start(c+1)),
// start(c) = floor(c T / G); tc_cta_of(g) is the CTA owning chunk g (the last c
// with start(c) <= g, i.e. ceil((g + 1) G / T) - 1).
__host__ __device__ __forceinline__ long long tc_chunk_start(int c, int G, long long T) {
    return (long long)c * T / G;
}
__host__ __device__ __forceinline__ int tc_cta_of(long long g, int G, long long T) {
    return (int)(((g + 1) * G + T - 1) / T) - 1;
}
// partial slots of the 128-row tile mt of a tensor-core solve (one per CTA that touches it)
__device__ __forceinline__ int tc_tile_slots(const SolveDev& s, int mt) {
    const int nkb = s.tc_kpad / 64;
    const long long t0 = s.off[PK_DTC] + (long long)mt * nkb;
    return tc_cta_of(t0 + nkb - 1, s.tc_G, s.tc_T) - tc_cta_of(t0, s.tc_G, s.tc_T) + 1;
}

// ---------------------------------------------------------------------------
// Double-word (float + float) arithmetic for compensated reductions.
// Error-free transformations: TwoSum (Knuth), TwoProduct via FMA; the
// accumulation is Ogita, Rump & Oishi's Dot2 ("Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005).  __fadd_rn/__fmul_rn keep the
// compiler from contracting the transformations into FMAs.
struct dw { float hi, lo; };

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// acc += x * y (Dot2 step)
__device__ __forceinline__ void dot2_acc(dw& acc, float x, float y) {
    float p = __fmul_rn(x, y);
    float pe = fmaf(x, y, -p);
    float s, se;
    two_sum(acc.hi, p, s, se);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(pe, se));
}

// acc += (b.hi + b.lo)
__device__ __forceinline__ void dw_add(dw& acc, dw b) {
    float s, e;
    two_sum(acc.hi, b.hi, s, e);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(e, b.lo));
}

__device__ __forceinline__ double dw_value(dw a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ dw dw_from_double(double v) {
    dw r;
    r.hi = (float)v;
    r.lo = (float)(v - (double)r.hi);
    return r;
}

// Accumulator type per storage type: float64 sums for double storage,
// double-word sums for float storage.
template <typename T> struct Acc;
template <> struct Acc<double> {
    double v;
    __device__ __forceinline__ void zero() { v = 0.0; }
    __device__ __forceinline__ void add_prod(double x, double y) { v = fma(x, y, v); }
    __device__ __forceinline__ dw as_dw() const { return dw_from_double(v); }
};
template <> struct Acc<float> {
    dw v;
    __device__ __forceinline__ void zero() { v.hi = 0.f; v.lo = 0.f; }
    __device__ __forceinline__ void add_prod(float x, float y) { dot2_acc(v, x, y); }
    __device__ __forceinline__ dw as_dw() const { return v; }
};

// A float64 coefficient applied to T data: a plain double for T = double,
// a (hi, lo) float pair for T = float so that x * c keeps ~48 bits of c.
template <typename T> struct Coef;
template <> struct Coef<double> {
    double c;
    __device__ __forceinline__ void set(double v) { c = v; }
    __device__ __forceinline__ double mul(double x) const { return x * c; }
    __device__ __forceinline__ double fma_(double x, double acc) const { return fma(x, c, acc); }
};
template <> struct Coef<float> {
    float hi, lo;
    __device__ __forceinline__ void set(double v) { hi = (float)v; lo = (float)(v - (double)hi); }
    __device__ __forceinline__ float mul(float x) const { return fmaf(x, lo, x * hi); }
    __device__ __forceinline__ float fma_(float x, float acc) const { return fmaf(x, hi, fmaf(x, lo, acc)); }
};

// 1/x for a positive double within the float range, without a float64
// division (a float64 division costs thousands of cycles on GB300): the float
// reciprocal refined by two Newton-Raphson steps y <- y (2 - x y), each of
// which squares the relative error (2^-23 -> 2^-46 -> the float64 rounding).
__device__ __forceinline__ double rcp_newton(double x) {
    double y = (double)__frcp_rn((float)x);
    y = y * fma(-x, y, 2.0);
    return y * fma(-x, y, 2.0);
}

// eps_t = a / (t + c + 1)^q  (Section 7 schedule, parameters of the solve)
__device__ __forceinline__ double eps_of(const SolveDev& s, double t) {
    return s.eps_a / pow(t + s.eps_c + 1.0, s.eps_pow);
}

// ---------------------------------------------------------------------------
// Host-side launch wrappers (defined in the kernel translation units).
#define TC_MAX_CHUNKS 8
struct GroupLaunch {
    const SolveDev* d_solves;   // device array of descriptors
    int ns;                     // number of solves
    int blocks[PK_COUNT];       // total blocks per partition kind
    int prec;                   // storage precision of the group
    cudaStream_t stream;
    // tensor-core dense product: chunks of at most TC_MAXG solves, each with
    // its own descriptor sub-array (PK_DTC offsets relative to the chunk)
    int meas_vr;                // largest n*(rank_bucket(r)+1) of a MEAS_STOCH member (objective staging), 0 if none
    int meas_tc, meas_plain;    // members whose minibatch products run on the tensor cores / on CUDA cores
    int meas_bil;               // members of the bilinear kind (tensor-core passes over [A; B])
    int tc_chunks;
    const SolveDev* tc_desc[TC_MAX_CHUNKS];
    int tc_ns[TC_MAX_CHUNKS];
    long long tc_T[TC_MAX_CHUNKS];   // K chunks of the launch
    int tc_G[TC_MAX_CHUNKS];         // CTAs of the launch
    int tc_npad[TC_MAX_CHUNKS];      // largest N tile of the launch
    const TcMaps* tc_maps[TC_MAX_CHUNKS];
};

// mode of a reduction-kernel launch within an iteration
enum RedPhase : int {
    PH_INIT = 0,        // orthonormalise the initial block (W <- CholQR2(W))
    PH_ADVANCE = 1,     // a product that only advances the subspace
    PH_FINAL = 2,       // the product whose W gets the Rayleigh-Ritz step
    // block Krylov, two products per iteration (float storage)
    PH_KRY1 = 3,        // after A W0: project Z = A W0 on W0, CholeskyQR of the rest -> W1
    PH_KRY2 = 4         // after A W1: Rayleigh-Ritz on span [W0 W1] (2k x 2k), next block
};

cudaError_t launch_begin(const GroupLaunch& g);
cudaError_t launch_dense(const GroupLaunch& g);
cudaError_t launch_csr(const GroupLaunch& g);
cudaError_t launch_meas_batch(const GroupLaunch& g);
cudaError_t launch_meas_apply(const GroupLaunch& g);
// tensor-core minibatch products (meas_tc.cu)
cudaError_t launch_meas_tc_batch(const GroupLaunch& g);
cudaError_t launch_meas_tc_apply(const GroupLaunch& g);
cudaError_t meas_tc_init();
// bilinear measurements: c_i = a_i^T b_i of the m pairs of one solve into meas[0, m)
cudaError_t launch_bil_prep(const SolveDev* d_solve, int64_t m, cudaStream_t st);
cudaError_t launch_combine(const GroupLaunch& g, int phase);
cudaError_t launch_combine_rows(const GroupLaunch& g);
// Hutchinson + Lanczos estimate of Tr exp(M_t) (one solve, float storage): at most LZ_MAX steps
#define LZ_MAX 32
cudaError_t launch_lz_start(const GroupLaunch& g, const double* U, float* Qb, double* ab, int k);
cudaError_t launch_lz_step(const GroupLaunch& g, float* Qb, double* ab, int j, int steps, int k);
cudaError_t launch_lz_quad(const GroupLaunch& g, const double* ab, int steps, double* out);
cudaError_t launch_orthonormalise(const GroupLaunch& g, int phase);
cudaError_t launch_chain_kernel(const GroupLaunch& g, int which, int phase);
cudaError_t launch_objective(const GroupLaunch& g, double* out_f);
// meg_solve's stopping test after a chunk of iterations (one solve); ends the
// enclosing conditional (while) graph node through `cond`
cudaError_t launch_solve_check(double* sm, const double* f, cudaGraphConditionalHandle cond, cudaStream_t st);
cudaError_t init_kernel_attributes();
