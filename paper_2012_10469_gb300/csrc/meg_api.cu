// C ABI of the low-rank MEG library (declared in include/meg.h).
//
// Host-side responsibilities: argument checks, device buffers of each solve,
// the order of kernel launches in one iteration of Algorithm 2, CUDA graphs
// of an iteration, grouped launches over several solves.  Every arithmetic
// step of the method runs in the kernels of kernels.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <random>
#include <string>
#include <vector>

#include "meg_dev.cuh"

namespace {

thread_local std::string g_last_error;

meg_status fail(meg_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

#define CU(expr)                                                                              \
    do {                                                                                      \
        cudaError_t _e = (expr);                                                              \
        if (_e != cudaSuccess)                                                                \
            return fail(MEG_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e));   \
    } while (0)

std::once_flag g_attr_once;
cudaError_t g_attr_err = cudaSuccess;
bool g_tc_ok = false;        // tcgen05 product available (driver entry point for TMA maps found)

cudaError_t ensure_attributes() {
    std::call_once(g_attr_once, [] {
        g_attr_err = init_kernel_attributes();
        g_tc_ok = (tc_init() == cudaSuccess);
        cudaGetLastError();
    });
    return g_attr_err;
}

int round_up(int a, int b) { return (a + b - 1) / b * b; }

int g_num_sms = 0;           // SMs of the device the first solve was created on

int num_sms() {
    if (g_num_sms <= 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            g_num_sms = v;
        else
            g_num_sms = 1;
    }
    return g_num_sms;
}

// K chunks (64 wide) of one tensor-core solve: 128-row tiles x chunks per tile
long long tc_chunks_of(const SolveDev& d) { return (long long)d.nb_tm * (d.tc_kpad / 64); }

// CTAs of a stream-K launch over T chunks whose tiles have at most nkb_max
// chunks: one or two per SM, fewer when a CTA's share would be so short that a tile
// could be cut into more than TC_YS_SLOTS segments (a share of at least
// ceil(nkb_max / (slots - 1)) chunks meets at most `slots` CTAs per tile).
int tc_grid(long long T, int nkb_max) {
    const long long need = (nkb_max + TC_YS_SLOTS - 2) / (TC_YS_SLOTS - 1);
    const long long G = std::min<long long>((long long)num_sms() * tc_ctas_per_sm(T, num_sms()),
                                            T / std::max<long long>(1, need));
    return (int)std::max<long long>(1, G);
}

void tc_partition(SolveDev& d) {
    d.nb_tm = (d.n + 127) / 128;
    d.nb_ds = TC_YS_SLOTS;                 // partial slots of Ys
    d.ks_len = d.tc_kpad;
    d.off[PK_DTC] = 0;                     // stand-alone launch: this solve only
    d.tc_T = tc_chunks_of(d);
    d.tc_G = tc_grid(d.tc_T, d.tc_kpad / 64);
}

// rows per reduction block: many small blocks for small n, up to ROWS_MAX for
// large n (fewer waves of the row kernels, whose last block needs the island's
// shared memory)
int rows_red_for(int n) { return n >= 4096 ? ROWS_MAX : (n >= 2048 ? 32 : 16); }

size_t tsize(int prec) { return prec == MEG_FP64 ? 8 : 4; }

int dense_splits(int n) {
    const int nb_dm = (n + 63) / 64;
    int target = 2 * 152;
    int s = std::max(1, (target + nb_dm - 1) / nb_dm);
    s = std::min(s, std::max(1, n / 128));
    return std::max(1, s);
}

}  // namespace

struct meg_solve_s {
    meg_options opt{};
    int n = 0, r = 0, k = 0, q = 0, prec = 0;
    cudaStream_t stream = nullptr;
    // device buffers (owned)
    void *V = nullptr, *Vn = nullptr, *W = nullptr, *Wp = nullptr, *Z = nullptr, *Y = nullptr, *Ys = nullptr;
    void* Wsp = nullptr;                   // split W for the tensor-core product (MEG_MIXED_BF16)
    TcMaps* solo_maps = nullptr;           // this solve's TMA maps at index 0
    float* part = nullptr;
    unsigned* ctr = nullptr;
    double* sm = nullptr;
    double* meas = nullptr;
    int* bidx = nullptr;
    float* mtp = nullptr;                  // partials of the tensor-core minibatch pass
    double* d_f = nullptr;
    SolveDev desc{};
    SolveDev* d_desc = nullptr;   // solo descriptor (offsets 0)
    bool has_obj = false, has_x = false;
    meg_objective_desc obj{};
    double fstar = 0.0;
    // solo graph of one iteration
    cudaGraphExec_t gexec = nullptr;
    // meg_solve's device loop: a conditional (while) node whose body runs a
    // chunk of iterations, the objective pass and the stopping test
    cudaGraphExec_t solve_gexec = nullptr;
    // set once the device reported an error (MEG_ERR_NUMERIC / TIMEOUT): every
    // later call except meg_destroy answers MEG_ERR_STATE
    bool failed = false;
    bool in_group = false;
    cudaStream_t group_stream = nullptr;   // stream of the group while in one
    bool own_stream = false;               // created by the library (caller gave NULL)
};

struct meg_group_s {
    std::vector<meg_solve_s*> solves;
    SolveDev* d_desc = nullptr;
    SolveDev* d_tc_desc = nullptr;         // descriptors of the tensor-core solves, chunk by chunk
    double* d_f = nullptr;                 // objective of each member (meg_group_objective)
    std::vector<TcMaps> tc_maps;           // one per chunk (addresses stable after creation)
    GroupLaunch gl{};
    bool has_dense = false, has_csr = false, has_meas = false;
    int q = 0;
    bool krylov = false;                   // block Krylov eigensolver (warm starts use subspace iteration)
    cudaStream_t stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool own_stream = false;
};

namespace {

void compute_partition(meg_solve_s* h, SolveDev& d) {
    d.rows_red = rows_red_for(h->n);
    d.nb_red = (h->n + d.rows_red - 1) / d.rows_red;
    d.nb_dm = (h->n + 63) / 64;
    d.nb_ds = dense_splits(h->n);
    int kl = (h->n + d.nb_ds - 1) / d.nb_ds;
    d.ks_len = ((kl + 31) / 32) * 32;
    d.nb_ds = (h->n + d.ks_len - 1) / d.ks_len;
    d.nb_csr = (h->n + 7) / 8;
    d.nb_meas = 0;
}

bool meas_kind(int kind) { return kind == MEG_MEAS_STOCH || kind == MEG_BILINEAR; }

int blocks_of(const SolveDev& d, int kind) {
    const bool dense = (d.kind == MEG_DENSE_QUAD || d.kind == MEG_LINEAR);
    const bool bil = d.kind == MEG_BILINEAR;
    switch (kind) {
        case PK_RED: return (d.nb_red + RED_CLUSTER - 1) / RED_CLUSTER * RED_CLUSTER;
        case PK_DENSE: return (dense && !d.tc) ? d.nb_dm * d.nb_ds : 0;
        case PK_CSR: return d.kind == MEG_CSR_QUAD ? d.nb_csr : 0;
        case PK_DTC: return (dense && d.tc) ? (int)tc_chunks_of(d) : 0;
        // minibatch: blocks of batch rows of the finish (the bilinear kind finishes
        // its pairs in the batch pass's epilogue)
        case PK_MEAS:
            if (bil) return 0;
            return d.kind == MEG_MEAS_STOCH ? (d.nb_meas + MB_ROWS - 1) / MB_ROWS : 0;
        case PK_MAP:
            if (!meas_kind(d.kind)) return 0;
            return (d.mtc ? (d.n + MT_BM - 1) / MT_BM : (d.n + MA_ROWS - 1) / MA_ROWS) *
                   apply_slots(d.kind, d.nb_meas, d.n, d.mtc);
        case PK_MTB:
            return (meas_kind(d.kind) && d.mtc) ? (d.nb_meas + MT_BM - 1) / MT_BM * batch_ks(d.kind, d.nb_meas, d.n)
                                                : 0;
        default: return 0;
    }
}

GroupLaunch solo_launch(meg_solve_s* h) {
    GroupLaunch g{};
    g.d_solves = h->d_desc;
    g.ns = 1;
    for (int p = 0; p < PK_COUNT; ++p) g.blocks[p] = blocks_of(h->desc, p);
    g.prec = h->prec;
    g.stream = h->stream;
    g.meas_vr = meas_kind(h->desc.kind) ? h->n * (rank_bucket(h->r) + 1) : 0;
    g.meas_tc = h->desc.kind == MEG_MEAS_STOCH && h->desc.mtc;
    g.meas_plain = h->desc.kind == MEG_MEAS_STOCH && !h->desc.mtc;
    g.meas_bil = h->desc.kind == MEG_BILINEAR;
    if (g.blocks[PK_DTC] > 0) {
        g.tc_chunks = 1;
        g.tc_desc[0] = h->d_desc;
        g.tc_ns[0] = 1;
        g.tc_T[0] = h->desc.tc_T;
        g.tc_G[0] = h->desc.tc_G;
        g.tc_npad[0] = h->desc.tc_npad;
        g.tc_maps[0] = h->solo_maps;
    }
    return g;
}

meg_status upload_desc(meg_solve_s* h, const SolveDev& d) {
    CU(cudaMemcpyAsync(h->d_desc, &d, sizeof(SolveDev), cudaMemcpyHostToDevice, h->stream));
    return MEG_OK;
}

// One iteration of Algorithm 2 (or one warm-start product set), enqueued.
// Subspace iteration: q products, each followed by the orthonormalisation of
// its block, the last one by the Rayleigh-Ritz step.  Block Krylov (q = 2):
// the first product's block is projected against W0 and orthonormalised, the
// second ends in the Rayleigh-Ritz step on span [W0 W1].
meg_status enqueue_iteration(const GroupLaunch& g, bool has_dense, bool has_csr, bool has_meas, int q,
                             bool krylov = false) {
    for (int j = 0; j < q; ++j) {
        const int phase = krylov ? (j == 0 ? PH_KRY1 : PH_KRY2) : (j == q - 1) ? PH_FINAL : PH_ADVANCE;
        if (has_meas) CU(launch_meas_batch(g));
        if (j == 0) CU(launch_begin(g));
        if (has_dense) CU(launch_dense(g));
        if (has_csr) CU(launch_csr(g));
        if (has_meas) CU(launch_meas_apply(g));
        CU(launch_combine(g, phase));
        CU(launch_orthonormalise(g, phase));
    }
    return MEG_OK;
}

meg_status enqueue_init_orth(const GroupLaunch& g) {
    CU(launch_combine(g, PH_INIT));
    CU(launch_orthonormalise(g, PH_INIT));
    return MEG_OK;
}

template <typename T>
void to_storage(const std::vector<double>& src, std::vector<unsigned char>& out) {
    out.resize(src.size() * sizeof(T));
    T* p = (T*)out.data();
    for (size_t i = 0; i < src.size(); ++i) p[i] = (T)src[i];
}

meg_status upload_T(meg_solve_s* h, void* dst, const std::vector<double>& src) {
    std::vector<unsigned char> buf;
    if (h->prec == MEG_FP64) to_storage<double>(src, buf);
    else to_storage<float>(src, buf);
    CU(cudaMemcpyAsync(dst, buf.data(), buf.size(), cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));   // buf is a local
    return MEG_OK;
}

meg_status upload_f64(meg_solve_s* h, void* dst, const std::vector<double>& src) {
    CU(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return MEG_OK;
}

// Work of a group runs on the group's stream: order the solve's stream after it.
meg_status join_group_stream(meg_solve_s* h) {
    if (h->in_group && h->group_stream != h->stream) CU(cudaStreamSynchronize(h->group_stream));
    return MEG_OK;
}

meg_status check_device_status(meg_solve_s* h) {
    if (h->failed) return fail(MEG_ERR_STATE, "the solve failed earlier on the device; only meg_destroy remains");
    if (meg_status js = join_group_stream(h); js != MEG_OK) return js;
    double st = 0.0;
    CU(cudaMemcpyAsync(&st, h->sm + SM_STATUS, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (st != 0.0) {
        h->failed = true;
        char msg[128];
        snprintf(msg, sizeof msg, "device reported status %d (numeric breakdown in a k x k step)", (int)st);
        return fail((meg_status)(int)st, msg);
    }
    return MEG_OK;
}

// f(X_t) by the accurate pass; also refreshes the shift bounds that depend on it.
meg_status eval_objective(meg_solve_s* h, double* f) {
    GroupLaunch g = solo_launch(h);
    CU(launch_objective(g, h->d_f));
    double v = 0.0;
    CU(cudaMemcpyAsync(&v, h->d_f, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    *f = v;
    return MEG_OK;
}

// f(X_1), the denominator of meg_solve's relative gap, kept in the small state
// (so it travels with a checkpoint): evaluated when X_1 and the objective are
// both known and the solve has not stepped yet (t = 1).
meg_status record_f1(meg_solve_s* h) {
    if (!h->has_obj || !h->has_x) return MEG_OK;
    double t = 0.0;
    CU(cudaMemcpyAsync(&t, h->sm + SM_T, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (t != 1.0) return MEG_OK;
    double f = 0.0;
    meg_status st = eval_objective(h, &f);
    if (st != MEG_OK) return st;
    CU(cudaMemcpyAsync(h->sm + SM_F1, &f, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return MEG_OK;
}

meg_status refresh_bounds(meg_solve_s* h) {
    if (!h->has_obj || !h->has_x) return MEG_OK;
    if (h->obj.kind == MEG_CSR_QUAD) {
        // one CSR gradient pass at X_t leaves max_i sum_j |R_ij| in the state
        CU(launch_csr(solo_launch(h)));
        CU(cudaStreamSynchronize(h->stream));
        return MEG_OK;
    }
    if (h->obj.kind != MEG_DENSE_QUAD) return MEG_OK;
    double f = 0.0;
    meg_status st = eval_objective(h, &f);
    if (st != MEG_OK) return st;
    double vals[1];
    int slot;
    vals[0] = 1.25 * std::sqrt(std::max(2.0 * f, 0.0));
    slot = SM_GNORM;
    CU(cudaMemcpyAsync(h->sm + slot, vals, sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return MEG_OK;
}

}  // namespace

namespace meg_internal {
void set_last_error(const std::string& msg) { g_last_error = msg; }

cudaStream_t group_stream(meg_group g) { return g->stream; }
cudaStream_t solve_stream(meg_handle h) { return h->stream; }

// every member's f(X_t) (meg_objective's accurate pass, one launch for the
// group) copied to host memory f[count]; enqueued on the group's stream
meg_status group_objective_enqueue(meg_group g, double* f) {
    CU(launch_objective(g->gl, g->d_f));
    CU(cudaMemcpyAsync(f, g->d_f, sizeof(double) * g->gl.ns, cudaMemcpyDeviceToHost, g->stream));
    return MEG_OK;
}

// device status of a member (MEG_OK or the error a kernel recorded); the
// group's stream must be idle
meg_status solve_status(meg_handle h) { return check_device_status(h); }
}

// ============================================================================
extern "C" {

const char* meg_last_error(void) { return g_last_error.c_str(); }

int64_t meg_footprint(int n, int r, int p, int precision, int kind) {
    if (n <= 0 || r <= 0 || p <= 0) return -1;
    const int64_t k = r + p;
    const int64_t ts = precision == MEG_FP64 ? 8 : 4;
    const int64_t nb_red = (n + rows_red_for(n) - 1) / rows_red_for(n);
    const int64_t groups = (nb_red + RED_GROUP - 1) / RED_GROUP;
    int64_t b = 0;
    b += ts * (int64_t)n * (2 * r + 4 * k);
    if (kind == MEG_DENSE_QUAD || kind == MEG_LINEAR) b += ts * (int64_t)std::max(dense_splits(n), 16) * n * k;
    if (kind == MEG_MEAS_STOCH)
        b += ts * (int64_t)MEAS_CHUNKS * n * k;   // (+ scratch of 8 (34 m + m/8) bytes and
                                                  //  4 (2 k_bucket(k) + 1) m tensor-core partials)
    if (kind == MEG_BILINEAR)                     // apply-pass slots for large m (+ 8 (m + m/32) bytes of
        b += ts * (int64_t)std::min(BIL_SLOTS_MAX, (4 * 152 + (n + MT_BM - 1) / MT_BM - 1) / ((n + MT_BM - 1) / MT_BM)) *
             n * k;                               //  scratch and the S image, 12 P bytes per pair)
    if (precision == MEG_MIXED_BF16 && n % 8 == 0) b += 2 * (int64_t)((3 * k + 15) / 16 * 16) * ((n + 63) / 64 * 64);
    b += 4 * (nb_red + groups) * 2 * RED_MAX_ENTRIES;
    b += 4 * (groups + 3) + 8 * SM_TOTAL + 8;
    return b;
}

meg_status meg_create(const meg_options* opt, const double* V0, const double* lam0, meg_handle* out) {
    if (!opt || !out) return fail(MEG_ERR_INVALID_ARG, "meg_create: null argument");
    *out = nullptr;
    const int n = opt->n, r = opt->r, p = opt->p, q = opt->q;
    if (n < 2 || n > MEG_NMAX || r < 1 || r > MEG_RMAX || r > n - 1)
        return fail(MEG_ERR_INVALID_ARG, "meg_create: need 2 <= n <= 2^28 and 1 <= r <= min(n - 1, 30)");
    if (p < 1 || r + p > MEG_KMAX || r + p > n)
        return fail(MEG_ERR_INVALID_ARG, "meg_create: need p >= 1 and r + p <= min(n, 32)");
    if (q < 1 || q > 8) return fail(MEG_ERR_INVALID_ARG, "meg_create: need 1 <= q <= 8");
    if (opt->precision < MEG_FP64 || opt->precision > MEG_MIXED_BF16)
        return fail(MEG_ERR_INVALID_ARG, "meg_create: unknown precision");
    if (!(opt->eta > 0.0) || !std::isfinite(opt->eta)) return fail(MEG_ERR_INVALID_ARG, "meg_create: eta must be > 0");
    if (!(opt->eps_a > 0.0) || !(opt->eps_c >= 0.0) || !(opt->eps_pow >= 0.0))
        return fail(MEG_ERR_INVALID_ARG, "meg_create: eps schedule parameters");
    const double eps0 = opt->eps_a / std::pow(opt->eps_c + 1.0, opt->eps_pow);
    if (!(eps0 > 0.0 && eps0 <= 0.75))
        return fail(MEG_ERR_INVALID_ARG, "meg_create: eps_t must lie in (0, 3/4] (Lemma 2)");
    if ((V0 == nullptr) != (lam0 == nullptr))
        return fail(MEG_ERR_INVALID_ARG, "meg_create: give both V0 and lam0 or neither");
    if (lam0) {
        double sum = 0.0;
        for (int i = 0; i < r; ++i) {
            if (!(lam0[i] >= 0.0)) return fail(MEG_ERR_INVALID_ARG, "meg_create: lam0 must be >= 0");
            sum += lam0[i];
        }
        if (std::fabs(sum - 1.0) > 1e-9) return fail(MEG_ERR_INVALID_ARG, "meg_create: lam0 must sum to 1");
    }
    if (cudaError_t e = ensure_attributes(); e != cudaSuccess)
        return fail(MEG_ERR_CUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
    // a solve whose own buffers cannot fit the device's free memory is refused
    // before anything is allocated
    {
        size_t freeb = 0, totb = 0;
        const int64_t need = meg_footprint(n, r, p, opt->precision, -1);
        if (cudaMemGetInfo(&freeb, &totb) == cudaSuccess && need > (int64_t)freeb)
            return fail(MEG_ERR_OOM, "meg_create: the solve needs " + std::to_string(need) +
                                         " device bytes, " + std::to_string(freeb) + " are free");
        cudaGetLastError();
    }

    if (opt->eigensolver != MEG_EIG_SUBSPACE && opt->eigensolver != MEG_EIG_BLOCK_KRYLOV)
        return fail(MEG_ERR_INVALID_ARG, "meg_create: unknown eigensolver");
    if (opt->eigensolver == MEG_EIG_BLOCK_KRYLOV &&
        (q != 2 || 2 * (r + p) > MEG_KMAX || opt->precision == MEG_FP64))
        return fail(MEG_ERR_INVALID_ARG,
                    "meg_create: block Krylov needs q = 2, 2 (r + p) <= 32 and float storage (MEG_FP32, MEG_MIXED_BF16)");

    meg_solve_s* h = new meg_solve_s();
    h->opt = *opt;
    h->n = n; h->r = r; h->k = r + p; h->q = q; h->prec = opt->precision;
    h->stream = (cudaStream_t)opt->stream;
    if (!h->stream) {
        // CUDA graphs cannot be captured on the legacy default stream: use a
        // blocking stream of our own, which stays ordered with the legacy stream.
        if (cudaStreamCreate(&h->stream) != cudaSuccess) {
            delete h;
            return fail(MEG_ERR_CUDA, "meg_create: stream creation failed");
        }
        h->own_stream = true;
    }
    SolveDev& d = h->desc;
    d.n = n; d.r = r; d.k = h->k; d.kind = -1; d.prec = h->prec; d.q = q; d.mode = 0;
    d.eig = opt->eigensolver;
    d.eta = opt->eta; d.eps_a = opt->eps_a; d.eps_c = opt->eps_c; d.eps_pow = opt->eps_pow; d.seed = opt->seed;
    d.log_nr = std::log((double)(n - r));
    compute_partition(h, d);
    const size_t ts = tsize(h->prec);
    const int k = h->k;
    const int groups = (d.nb_red + RED_GROUP - 1) / RED_GROUP;
    // stream-ordered allocations: creating or destroying a solve never
    // synchronises the device, so other solves' work keeps running
    auto alloc = [&](void** ptr, size_t bytes) -> bool {
        return cudaMallocAsync(ptr, std::max<size_t>(bytes, 16), h->stream) == cudaSuccess;
    };
    const size_t nr8 = (size_t)8 * n * r, nkt = ts * n * k;    // sizes in size_t: n * r * 8 can pass 2^31
    bool ok = alloc(&h->V, nr8) && alloc(&h->Vn, nr8) && alloc(&h->W, nkt) &&
              alloc(&h->Wp, nkt) && alloc(&h->Z, nkt) && alloc(&h->Y, nkt) &&
              alloc((void**)&h->part, sizeof(float) * (d.nb_red + groups) * 2 * RED_MAX_ENTRIES) &&
              alloc((void**)&h->ctr, sizeof(unsigned) * (groups + 3)) &&
              alloc((void**)&h->sm, sizeof(double) * SM_TOTAL) && alloc((void**)&h->d_f, sizeof(double)) &&
              alloc((void**)&h->d_desc, sizeof(SolveDev));
    if (!ok) {
        cudaGetLastError();
        meg_destroy(h);
        return fail(MEG_ERR_OOM, "meg_create: device allocation failed");
    }
    if (h->prec == MEG_MIXED_BF16 && (n % 8) == 0) {
        d.tc_npad = 3 * round_up(k, 16);     // three bf16 pieces of W, each padded to 16 rows
        d.tc_kpad = round_up(n, 64);
        const size_t wsb = (size_t)2 * d.tc_npad * d.tc_kpad;
        h->solo_maps = new TcMaps();
        if (cudaMallocAsync(&h->Wsp, wsb, h->stream) != cudaSuccess ||
            cudaMemsetAsync(h->Wsp, 0, wsb, h->stream) != cudaSuccess) {
            cudaGetLastError();
            meg_destroy(h);
            return fail(MEG_ERR_OOM, "meg_create: split block");
        }
    }
    d.Wsp = (unsigned short*)h->Wsp;
    d.V = (double*)h->V; d.Vn = (double*)h->Vn; d.W = h->W; d.Wp = h->Wp; d.Z = h->Z; d.Y = h->Y; d.Ys = nullptr;
    d.part = h->part; d.ctr = h->ctr; d.sm = h->sm; d.meas = nullptr; d.bidx = nullptr;
    meg_status st;
    std::vector<double> smh(SM_TOTAL, 0.0);
    smh[SM_T] = 1.0;
    smh[SM_ETA] = opt->eta;
    smh[SM_F1] = std::nan("");
    if (V0) {
        for (int i = 0; i < r; ++i) {
            smh[SM_MU + i] = (1.0 - eps0) * lam0[i] + eps0 / n;
            smh[SM_LOGMU + i] = std::log(smh[SM_MU + i]);
        }
        smh[SM_S] = eps0 / n;
        smh[SM_LOGS] = std::log(smh[SM_S]);
    }
    if (cudaMemsetAsync(h->ctr, 0, sizeof(unsigned) * (groups + 3), h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->V, 0, nr8, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->W, 0, nkt, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(h->sm, smh.data(), sizeof(double) * SM_TOTAL, cudaMemcpyHostToDevice, h->stream) !=
            cudaSuccess) {
        meg_destroy(h);
        return fail(MEG_ERR_CUDA, "meg_create: initial copies failed");
    }
    if ((st = upload_desc(h, d)) != MEG_OK) { meg_destroy(h); return st; }
    if (V0) {
        // W_1 = [V0 | P], P Gaussian (seeded); orthonormalised on the device
        std::vector<double> vh((size_t)n * r), wh((size_t)n * k);
        std::mt19937_64 gen(opt->seed ^ 0x5EEDC0DEull);
        std::normal_distribution<double> nd(0.0, 1.0);
        for (int i = 0; i < n; ++i) {
            for (int j = 0; j < r; ++j) vh[(size_t)i * r + j] = wh[(size_t)i * k + j] = V0[(size_t)i * r + j];
            for (int j = r; j < k; ++j) wh[(size_t)i * k + j] = nd(gen);
        }
        if ((st = upload_f64(h, h->V, vh)) != MEG_OK || (st = upload_T(h, h->W, wh)) != MEG_OK ||
            (st = enqueue_init_orth(solo_launch(h))) != MEG_OK) {
            meg_destroy(h);
            return st;
        }
        h->has_x = true;
    }
    *out = h;
    return MEG_OK;
}

meg_status meg_set_objective(meg_handle h, const meg_objective_desc* o) {
    if (!h || !o) return fail(MEG_ERR_INVALID_ARG, "meg_set_objective: null argument");
    if (h->failed) return fail(MEG_ERR_STATE, "meg_set_objective: the solve failed earlier on the device");
    if (h->in_group) return fail(MEG_ERR_STATE, "meg_set_objective: solve belongs to a group");
    SolveDev& d = h->desc;
    const int n = h->n, k = h->k;
    if (o->kind == MEG_DENSE_QUAD || o->kind == MEG_LINEAR) {
        if (!o->dense) return fail(MEG_ERR_INVALID_ARG, "meg_set_objective: dense data missing");
    } else if (o->kind == MEG_CSR_QUAD) {
        if (!o->rowptr || !o->col || !o->val || o->nnz < 0)
            return fail(MEG_ERR_INVALID_ARG, "meg_set_objective: CSR arrays missing");
        std::vector<int> rp(n + 1);
        CU(cudaMemcpyAsync(rp.data(), o->rowptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        if (rp[0] != 0 || rp[n] != o->nnz)
            return fail(MEG_ERR_INVALID_ARG, "meg_set_objective: rowptr[0] must be 0 and rowptr[n] == nnz");
        for (int i = 0; i < n; ++i)
            if (rp[i + 1] < rp[i]) return fail(MEG_ERR_INVALID_ARG, "meg_set_objective: rowptr not monotone");
        // column indices address rows of V and W in the kernels: all must lie in [0, n)
        std::vector<int> cols((size_t)o->nnz);
        if (o->nnz > 0) {
            CU(cudaMemcpyAsync(cols.data(), o->col, sizeof(int) * (size_t)o->nnz, cudaMemcpyDeviceToHost, h->stream));
            CU(cudaStreamSynchronize(h->stream));
        }
        for (int64_t e = 0; e < o->nnz; ++e)
            if (cols[e] < 0 || cols[e] >= n) return fail(MEG_ERR_INVALID_ARG, "meg_set_objective: column index out of range");
    } else if (o->kind == MEG_MEAS_STOCH) {
        if (!o->A || !o->y || o->m < 1 || o->L < 1)
            return fail(MEG_ERR_INVALID_ARG, "meg_set_objective: measurement arrays missing");
        if (o->m > 0x7fffffff) return fail(MEG_ERR_INVALID_ARG, "meg_set_objective: m too large");
    } else if (o->kind == MEG_BILINEAR) {
        if (!o->A || !o->B || !o->y || o->m < 1)
            return fail(MEG_ERR_INVALID_ARG, "meg_set_objective: bilinear arrays missing");
        const int pr = o->mrank <= 1 ? 1 : o->mrank;
        if (pr > 32 || (pr & (pr - 1)) != 0)
            return fail(MEG_ERR_INVALID_ARG, "meg_set_objective: mrank must be 0, 1 or a power of two up to 32");
        if (o->m > 0x3fffff00 / pr)
            return fail(MEG_ERR_INVALID_ARG, "meg_set_objective: m mrank too large (2 m mrank stacked rows)");
        if (!(o->tau > 0.0) || !std::isfinite(o->tau))
            return fail(MEG_ERR_INVALID_ARG, "meg_set_objective: tau must be positive and finite");
        // both products run on the tensor cores over 16-byte rows of bf16 data
        if (h->prec == MEG_FP64 || n % 8 != 0 || ((uintptr_t)o->A % 16) != 0 || ((uintptr_t)o->B % 16) != 0)
            return fail(MEG_ERR_INVALID_ARG,
                        "meg_set_objective: bilinear kind needs float storage, n % 8 == 0 and 16-byte aligned A, B");
    } else {
        return fail(MEG_ERR_INVALID_ARG, "meg_set_objective: unknown kind");
    }
    h->obj = *o;
    d.kind = o->kind;
    d.D = o->dense; d.rowptr = o->rowptr; d.col = o->col; d.val = o->val; d.nnz = o->nnz;
    // bilinear: the pair count m p (rank-p measurement matrices: p pairs per measurement)
    const int mrank = (o->kind == MEG_BILINEAR && o->mrank > 1) ? o->mrank : 1;
    const int64_t mp = o->m * mrank;
    d.A = o->A; d.y = o->y; d.m = o->kind == MEG_BILINEAR ? mp : o->m; d.L = o->L;
    d.Bm = o->kind == MEG_BILINEAR ? o->B : nullptr;
    d.tau = o->kind == MEG_BILINEAR ? o->tau : 1.0;
    d.mrank = mrank;
    const size_t ts = tsize(h->prec);
    const bool dense_kind = (o->kind == MEG_DENSE_QUAD || o->kind == MEG_LINEAR);
    d.tc = 0;
    if (dense_kind && h->Wsp && g_tc_ok &&
        tc_make_maps(o->dense, n, h->Wsp, d.tc_kpad, d.tc_npad, &h->solo_maps->a[0], &h->solo_maps->b[0])) {
        d.tc = 1;
        tc_partition(d);
    } else {
        compute_partition(h, d);
    }
    if (dense_kind || meas_kind(o->kind)) {
        // partial products: K splits of the dense product, or batch chunks of the minibatch product
        const size_t slots = dense_kind                    ? (size_t)d.nb_ds
                             : o->kind == MEG_BILINEAR ? (size_t)bil_slots((int)bil_rows(mp), n)
                                                       : (size_t)MEAS_CHUNKS;
        if (h->Ys) { cudaFreeAsync(h->Ys, h->stream); h->Ys = nullptr; }
        if (cudaMallocAsync(&h->Ys, ts * slots * n * k, h->stream) != cudaSuccess)
            return fail(MEG_ERR_OOM, "meg_set_objective: partial products");
    }
    d.Ys = h->Ys;
    if (meas_kind(o->kind) || o->kind == MEG_CSR_QUAD) {
        // minibatch scratch: [Lb] residuals, [Lb] ||a||^2, [Lb x 32] a^T W, one partial bound per block;
        // bilinear: [m] a_i^T b_i, one partial bound per block of MB_ROWS pairs
        const size_t lbm = (size_t)std::max<int64_t>(o->m, o->L);
        // CSR: one maximum per row block (rounded up to 16 bytes), then V and W as
        // float rows padded to a multiple of 4 for the sparse product
        const size_t pad4r = (size_t)((h->r + 3) & ~3), pad4k = (size_t)((k + 3) & ~3);
        size_t cnt = o->kind == MEG_MEAS_STOCH ? lbm * (2 + MEG_KMAX) + lbm / MB_ROWS + 1
                     : o->kind == MEG_BILINEAR ? (size_t)mp + (size_t)mp / MB_ROWS + 1
                                               : (size_t)((d.nb_csr + 1) & ~1) + ((size_t)n * (pad4r + pad4k) + 1) / 2;
        if (h->meas) cudaFreeAsync(h->meas, h->stream);
        if (h->bidx) cudaFreeAsync(h->bidx, h->stream);
        h->meas = nullptr; h->bidx = nullptr;
        if (cudaMallocAsync((void**)&h->meas, sizeof(double) * cnt, h->stream) != cudaSuccess ||
            cudaMallocAsync((void**)&h->bidx, sizeof(int) * std::max(1, o->L), h->stream) != cudaSuccess)
            return fail(MEG_ERR_OOM, "meg_set_objective: scratch");
    }
    d.meas = h->meas; d.bidx = h->bidx;
    d.nb_meas = o->kind == MEG_MEAS_STOCH ? o->L : o->kind == MEG_BILINEAR ? (int)bil_rows(mp) : 0;
    // minibatch products on the tensor cores: float storage (bf16 A), rows of A
    // 16-byte aligned (n % 8 == 0, aligned base); partials for the larger of
    // the minibatch pass and the warm start's pass over all m measurements
    d.mtc = 0;
    d.mtp = nullptr;
    d.mts = nullptr;
    d.mtb = nullptr;
    if (h->mtp) { cudaFreeAsync(h->mtp, h->stream); h->mtp = nullptr; }
    if (o->kind == MEG_BILINEAR ||
        (o->kind == MEG_MEAS_STOCH && h->prec != MEG_FP64 && n % 8 == 0 && ((uintptr_t)o->A % 16) == 0)) {
        const size_t cols = (size_t)2 * k_bucket(k) + 1;
        const size_t rows = o->kind == MEG_BILINEAR     // (no partials: the batch pass finishes its tiles)
                                ? 0
                                : std::max((size_t)meas_ks(o->L, n) * o->L, (size_t)meas_ks((int)o->m, n) * o->m);
        // S: one row per batch row (bilinear: per stacked row)
        const size_t srows = o->kind == MEG_BILINEAR ? (size_t)d.nb_meas : (size_t)std::max<int64_t>(o->L, o->m);
        // + the split images of the apply pass's S (zeroed: columns k..P-1 are never written)
        // and of the batch pass's [V | W] (ceil(n/64) chunks of 3 x (cols - 1) rows x 64 bf16)
        const size_t sfl = (rows * cols + 3) & ~(size_t)3;               // 16-byte aligned images
        const size_t sim = mts_image_bytes((int64_t)srows, k) / 4;
        const size_t img = (size_t)((n + MT_BK - 1) / MT_BK) * 3 * (cols - 1) * MT_BK / 2;
        if (cudaMallocAsync((void**)&h->mtp, sizeof(float) * (sfl + sim + img), h->stream) != cudaSuccess)
            return fail(MEG_ERR_OOM, "meg_set_objective: tensor-core partials");
        CU(cudaMemsetAsync(h->mtp + sfl, 0, sizeof(float) * sim, h->stream));
        d.mtc = 1;
        d.mtp = h->mtp;
        d.mts = (unsigned short*)(h->mtp + sfl);
        d.mtb = (unsigned short*)(h->mtp + sfl + sim);
    }
    meg_status st = upload_desc(h, d);
    if (st != MEG_OK) return st;
    if (o->kind == MEG_BILINEAR) CU(launch_bil_prep(h->d_desc, mp, h->stream));   // a^T b of every pair
    // statistics of the data used by the objective estimate and the shift: Tr D, ||D||_F^2
    // (computed by the objective kernel on X = 0 and X = I/n would need two passes;
    //  the k_objective pass on a zero iterate gives 1/2 ||D||^2 directly)
    if (o->kind == MEG_DENSE_QUAD || o->kind == MEG_LINEAR || o->kind == MEG_CSR_QUAD) {
        // evaluate with mu = s = 0 (X = 0): dense quadratic -> 1/2||D||^2, CSR -> 1/2 sum val^2
        std::vector<double> smh(SM_TOTAL);
        CU(cudaMemcpyAsync(smh.data(), h->sm, sizeof(double) * SM_TOTAL, cudaMemcpyDeviceToHost, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        std::vector<double> z = smh;
        for (int i = 0; i < h->r; ++i) z[SM_MU + i] = 0.0;
        z[SM_S] = 0.0;
        SolveDev dq = d;
        if (o->kind == MEG_LINEAR) dq.kind = MEG_DENSE_QUAD;      // same pass, sum of squares
        CU(cudaMemcpyAsync(h->sm, z.data(), sizeof(double) * SM_TOTAL, cudaMemcpyHostToDevice, h->stream));
        if ((st = upload_desc(h, dq)) != MEG_OK) return st;
        double half_sq = 0.0;
        if ((st = eval_objective(h, &half_sq)) != MEG_OK) return st;
        // X = I/n: <X, D> = Tr D / n for the linear form
        double trd = 0.0;
        if (o->kind != MEG_CSR_QUAD) {
            SolveDev dl = d;
            dl.kind = MEG_LINEAR;
            for (int i = 0; i < h->r; ++i) z[SM_MU + i] = 1.0 / n;   // X = I / n
            z[SM_S] = 1.0 / n;
            CU(cudaMemcpyAsync(h->sm, z.data(), sizeof(double) * SM_TOTAL, cudaMemcpyHostToDevice, h->stream));
            if ((st = upload_desc(h, dl)) != MEG_OK) return st;
            double v = 0.0;
            if ((st = eval_objective(h, &v)) != MEG_OK) return st;
            trd = v * n;
        }
        smh[SM_FROD2] = 2.0 * half_sq;
        smh[SM_TRD] = trd;
        CU(cudaMemcpyAsync(h->sm, smh.data(), sizeof(double) * SM_TOTAL, cudaMemcpyHostToDevice, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        if ((st = upload_desc(h, d)) != MEG_OK) return st;
    }
    h->has_obj = true;
    if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; }
    if (h->solve_gexec) { cudaGraphExecDestroy(h->solve_gexec); h->solve_gexec = nullptr; }
    if ((st = refresh_bounds(h)) != MEG_OK) return st;
    return record_f1(h);
}

meg_status meg_warm_start(meg_handle h, int products) {
    if (!h) return fail(MEG_ERR_INVALID_ARG, "meg_warm_start: null handle");
    if (h->failed) return fail(MEG_ERR_STATE, "meg_warm_start: the solve failed earlier on the device");
    if (!h->has_obj) return fail(MEG_ERR_STATE, "meg_warm_start: objective not set");
    if (products < 1) return fail(MEG_ERR_INVALID_ARG, "meg_warm_start: products >= 1");
    if (h->in_group) return fail(MEG_ERR_STATE, "meg_warm_start: solve belongs to a group");
    const int n = h->n, r = h->r, k = h->k;
    meg_status st;
    std::vector<double> vh((size_t)n * r), wh((size_t)n * k);
    std::mt19937_64 gen(h->opt.seed ^ 0xA11CE5ull);
    std::normal_distribution<double> nd(0.0, 1.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < k; ++j) {
            double v = nd(gen);
            wh[(size_t)i * k + j] = v;
            if (j < r) vh[(size_t)i * r + j] = v;
        }
    if ((st = upload_f64(h, h->V, vh)) != MEG_OK || (st = upload_T(h, h->W, wh)) != MEG_OK) return st;
    SolveDev dw = h->desc;
    dw.mode = 1;
    if (dw.kind == MEG_MEAS_STOCH) dw.nb_meas = (int)dw.m;
    CU(cudaMemcpyAsync(h->d_desc, &dw, sizeof(SolveDev), cudaMemcpyHostToDevice, h->stream));
    GroupLaunch g{};
    g.d_solves = h->d_desc;
    g.ns = 1;
    for (int p = 0; p < PK_COUNT; ++p) g.blocks[p] = blocks_of(dw, p);
    g.prec = h->prec;
    g.stream = h->stream;
    g.meas_vr = meas_kind(dw.kind) ? n * (rank_bucket(r) + 1) : 0;
    g.meas_tc = dw.kind == MEG_MEAS_STOCH && dw.mtc;
    g.meas_plain = dw.kind == MEG_MEAS_STOCH && !dw.mtc;
    g.meas_bil = dw.kind == MEG_BILINEAR;
    if ((st = enqueue_init_orth(g)) != MEG_OK) return st;
    if (dw.kind == MEG_CSR_QUAD) CU(launch_csr(g));   // bound max_i sum_j |M_ij| for the shift
    const bool dense = dw.kind == MEG_DENSE_QUAD || dw.kind == MEG_LINEAR;
    for (int j = 0; j < products; ++j) {
        const int phase = (j == products - 1) ? PH_FINAL : PH_ADVANCE;
        if (meas_kind(dw.kind)) CU(launch_meas_batch(g));
        if (j == 0) CU(launch_begin(g));
        if (dense) CU(launch_dense(g));
        if (dw.kind == MEG_CSR_QUAD) CU(launch_csr(g));
        if (meas_kind(dw.kind)) CU(launch_meas_apply(g));
        CU(launch_combine(g, phase));
        CU(launch_orthonormalise(g, phase));
    }
    if ((st = upload_desc(h, h->desc)) != MEG_OK) return st;
    CU(cudaStreamSynchronize(h->stream));
    h->has_x = true;
    if ((st = check_device_status(h)) != MEG_OK) return st;
    if ((st = refresh_bounds(h)) != MEG_OK) return st;
    return record_f1(h);
}

static meg_status ready(meg_handle h, const char* who) {
    if (!h) return fail(MEG_ERR_INVALID_ARG, std::string(who) + ": null handle");
    if (h->failed) return fail(MEG_ERR_STATE, std::string(who) + ": the solve failed earlier on the device");
    if (!h->has_obj || !h->has_x) return fail(MEG_ERR_STATE, std::string(who) + ": objective or X_1 not set");
    return MEG_OK;
}

meg_status meg_refine_subspace(meg_handle h, int products) {
    meg_status st = ready(h, "meg_refine_subspace");
    if (st != MEG_OK) return st;
    if (h->in_group) return fail(MEG_ERR_STATE, "meg_refine_subspace: solve belongs to a group");
    if (products < 0 || products > 4096) return fail(MEG_ERR_INVALID_ARG, "meg_refine_subspace: products in 0..4096");
    const GroupLaunch g = solo_launch(h);
    const int kind = h->desc.kind;
    const bool dense = kind == MEG_DENSE_QUAD || kind == MEG_LINEAR;
    for (int j = 0; j < products; ++j) {
        if (meas_kind(kind)) CU(launch_meas_batch(g));
        if (j == 0) CU(launch_begin(g));
        if (dense) CU(launch_dense(g));
        if (kind == MEG_CSR_QUAD) CU(launch_csr(g));
        if (meas_kind(kind)) CU(launch_meas_apply(g));
        CU(launch_combine(g, PH_ADVANCE));
        CU(launch_orthonormalise(g, PH_ADVANCE));
    }
    CU(cudaStreamSynchronize(h->stream));
    return check_device_status(h);
}

meg_status meg_trace_exp_estimate(meg_handle h, const double* U, int steps, double* estimate) {
    meg_status st = ready(h, "meg_trace_exp_estimate");
    if (st != MEG_OK) return st;
    if (h->in_group) return fail(MEG_ERR_STATE, "meg_trace_exp_estimate: solve belongs to a group");
    if (!U || !estimate) return fail(MEG_ERR_INVALID_ARG, "meg_trace_exp_estimate: null argument");
    if (steps < 1 || steps > LZ_MAX || steps > h->n)
        return fail(MEG_ERR_INVALID_ARG, "meg_trace_exp_estimate: need 1 <= steps <= min(32, n)");
    if (h->prec == MEG_FP64) return fail(MEG_ERR_INVALID_ARG, "meg_trace_exp_estimate: float storage only");
    const int n = h->n, k = h->k;
    const SolveDev& d = h->desc;
    const size_t wbytes = sizeof(float) * (size_t)n * k;
    const size_t spbytes = h->Wsp ? (size_t)2 * d.tc_npad * d.tc_kpad : 0;
    const size_t nab = (size_t)k * (2 * LZ_MAX + 1);
    // scratch: the probes, the Lanczos basis (steps + 1 slots of n x k), the coefficients,
    // the result, and copies of W, its split and the small state (restored at the end)
    char* buf = nullptr;
    const size_t b_U = sizeof(double) * (size_t)n * k, b_Q = sizeof(float) * (size_t)(steps + 1) * n * k;
    const size_t b_ab = sizeof(double) * (nab + 1), b_sm = sizeof(double) * SM_TOTAL;
    const size_t off_Q = (b_U + 255) & ~(size_t)255, off_ab = (off_Q + b_Q + 255) & ~(size_t)255;
    const size_t off_W = (off_ab + b_ab + 255) & ~(size_t)255, off_sp = (off_W + wbytes + 255) & ~(size_t)255;
    const size_t off_sm = (off_sp + spbytes + 255) & ~(size_t)255, total = off_sm + b_sm;
    if (cudaMallocAsync((void**)&buf, total, h->stream) != cudaSuccess)
        return fail(MEG_ERR_OOM, "meg_trace_exp_estimate: scratch");
    double* dU = (double*)buf;
    float* Qb = (float*)(buf + off_Q);
    double* ab = (double*)(buf + off_ab);
    double* dout = ab + nab;
    auto body = [&]() -> meg_status {
        CU(cudaMemcpyAsync(buf + off_W, h->W, wbytes, cudaMemcpyDeviceToDevice, h->stream));
        if (spbytes) CU(cudaMemcpyAsync(buf + off_sp, h->Wsp, spbytes, cudaMemcpyDeviceToDevice, h->stream));
        CU(cudaMemcpyAsync(buf + off_sm, h->sm, b_sm, cudaMemcpyDeviceToDevice, h->stream));
        CU(cudaMemcpyAsync(dU, U, b_U, cudaMemcpyHostToDevice, h->stream));
        const GroupLaunch g = solo_launch(h);
        const int kind = d.kind;
        const bool dense = kind == MEG_DENSE_QUAD || kind == MEG_LINEAR;
        CU(launch_lz_start(g, dU, Qb, ab, k));
        for (int j = 0; j < steps; ++j) {
            if (meas_kind(kind)) CU(launch_meas_batch(g));
            if (j == 0) CU(launch_begin(g));
            if (dense) CU(launch_dense(g));
            if (kind == MEG_CSR_QUAD) CU(launch_csr(g));
            if (meas_kind(kind)) CU(launch_meas_apply(g));
            CU(launch_combine_rows(g));
            CU(launch_lz_step(g, Qb, ab, j, steps, k));
        }
        CU(launch_lz_quad(g, ab, steps, dout));
        CU(cudaMemcpyAsync(estimate, dout, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        return MEG_OK;
    };
    st = body();
    // the iterate's block, its split and the small state as they were
    cudaMemcpyAsync(h->W, buf + off_W, wbytes, cudaMemcpyDeviceToDevice, h->stream);
    if (spbytes) cudaMemcpyAsync(h->Wsp, buf + off_sp, spbytes, cudaMemcpyDeviceToDevice, h->stream);
    cudaMemcpyAsync(h->sm, buf + off_sm, b_sm, cudaMemcpyDeviceToDevice, h->stream);
    cudaFreeAsync(buf, h->stream);
    if (st != MEG_OK) return st;
    CU(cudaStreamSynchronize(h->stream));
    return check_device_status(h);
}

meg_status meg_step(meg_handle h, int nsteps) {
    meg_status st = ready(h, "meg_step");
    if (st != MEG_OK) return st;
    if (h->in_group) return fail(MEG_ERR_STATE, "meg_step: solve belongs to a group");
    if (nsteps < 0) return fail(MEG_ERR_INVALID_ARG, "meg_step: nsteps < 0");
    if (!h->gexec) {
        cudaGraph_t graph;
        CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        const int kind = h->desc.kind;
        st = enqueue_iteration(solo_launch(h), kind == MEG_DENSE_QUAD || kind == MEG_LINEAR,
                               kind == MEG_CSR_QUAD, meas_kind(kind), h->q,
                               h->desc.eig == MEG_EIG_BLOCK_KRYLOV);
        cudaError_t ce = cudaStreamEndCapture(h->stream, &graph);
        if (st != MEG_OK) return st;
        if (ce != cudaSuccess) return fail(MEG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&h->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return fail(MEG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
    }
    for (int i = 0; i < nsteps; ++i) CU(cudaGraphLaunch(h->gexec, h->stream));
    return MEG_OK;
}

meg_status meg_set_fstar(meg_handle h, double fstar) {
    if (!h) return fail(MEG_ERR_INVALID_ARG, "meg_set_fstar: null handle");
    h->fstar = fstar;
    return MEG_OK;
}

meg_status meg_objective(meg_handle h, double* f) {
    meg_status st = ready(h, "meg_objective");
    if (st != MEG_OK) return st;
    if (!f) return fail(MEG_ERR_INVALID_ARG, "meg_objective: null output");
    if ((st = check_device_status(h)) != MEG_OK) return st;
    return eval_objective(h, f);
}

namespace {
// The device loop of meg_solve: a graph whose only node is a conditional
// while-loop; its body runs SOLVE_CHUNK iterations, the accurate objective
// pass and k_solve_check, which ends the loop.  Parameters (tol, f*, chunk
// limit) live in the small state, so one instantiated graph serves every call.
constexpr int SOLVE_CHUNK = 10;

meg_status build_solve_graph(meg_solve_s* h) {
    cudaGraph_t graph = nullptr;
    CU(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle cond;
    cudaError_t e = cudaGraphConditionalHandleCreate(&cond, graph, 1u, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
    meg_status st = MEG_OK;
    if (e == cudaSuccess) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        e = cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const int kind = h->desc.kind;
            const GroupLaunch g = solo_launch(h);
            for (int i = 0; i < SOLVE_CHUNK && st == MEG_OK; ++i)
                st = enqueue_iteration(g, kind == MEG_DENSE_QUAD || kind == MEG_LINEAR, kind == MEG_CSR_QUAD,
                                       meas_kind(kind), h->q, h->desc.eig == MEG_EIG_BLOCK_KRYLOV);
            cudaError_t le = cudaSuccess;
            if (st == MEG_OK) le = launch_objective(g, h->d_f);
            if (st == MEG_OK && le == cudaSuccess) le = launch_solve_check(h->sm, h->d_f, cond, h->stream);
            cudaGraph_t out = nullptr;
            e = cudaStreamEndCapture(h->stream, &out);
            if (e == cudaSuccess) e = le;
        }
    }
    if (e == cudaSuccess && st == MEG_OK) e = cudaGraphInstantiate(&h->solve_gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (st != MEG_OK) return st;
    if (e != cudaSuccess) return fail(MEG_ERR_CUDA, std::string("meg_solve graph: ") + cudaGetErrorString(e));
    return MEG_OK;
}
}  // namespace

meg_status meg_solve(meg_handle h, double tol, int max_iters, int* iters_out) {
    meg_status st = ready(h, "meg_solve");
    if (st != MEG_OK) return st;
    if (iters_out) *iters_out = 0;
    if (h->in_group) return fail(MEG_ERR_STATE, "meg_solve: solve belongs to a group");
    if (!(tol > 0.0) || max_iters < 0) return fail(MEG_ERR_INVALID_ARG, "meg_solve: need tol > 0, max_iters >= 0");
    if ((st = check_device_status(h)) != MEG_OK) return st;
    double f1 = 0.0;
    CU(cudaMemcpyAsync(&f1, h->sm + SM_F1, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (!std::isfinite(f1))
        return fail(MEG_ERR_STATE, "meg_solve: f(X_1) unknown (the objective was set after the first step)");
    const double denom = f1 - h->fstar;
    if (!(denom > 0.0))
        return fail(MEG_ERR_INVALID_ARG, "meg_solve: f* must lie below f(X_1); give it with meg_set_fstar");
    const int full = max_iters / SOLVE_CHUNK, rem = max_iters % SOLVE_CHUNK;
    double par[6] = {tol, h->fstar, (double)full, 0.0, 0.0, 0.0};   // SM_SOLVE_TOL .. SM_SOLVE_F
    int done_iters = 0;
    bool converged = false;
    if (full > 0) {
        if (!h->solve_gexec && (st = build_solve_graph(h)) != MEG_OK) return st;
        CU(cudaMemcpyAsync(h->sm + SM_SOLVE_TOL, par, sizeof(par), cudaMemcpyHostToDevice, h->stream));
        CU(cudaGraphLaunch(h->solve_gexec, h->stream));
        CU(cudaMemcpyAsync(par, h->sm + SM_SOLVE_TOL, sizeof(par), cudaMemcpyDeviceToHost, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        done_iters = SOLVE_CHUNK * (int)par[3];
        converged = par[4] != 0.0;
        if (iters_out) *iters_out = done_iters;
        if ((st = check_device_status(h)) != MEG_OK) return st;
        if (!std::isfinite(par[5])) {
            h->failed = true;
            return fail(MEG_ERR_NUMERIC, "meg_solve: the objective is not finite");
        }
    }
    if (!converged && rem > 0) {
        if ((st = meg_step(h, rem)) != MEG_OK) return st;
        done_iters += rem;
        if (iters_out) *iters_out = done_iters;
        double f = 0.0;
        if ((st = meg_objective(h, &f)) != MEG_OK) return st;
        converged = (f - h->fstar) <= tol * denom;
    }
    if (converged) return MEG_OK;
    return fail(MEG_ERR_NOT_CONVERGED, "meg_solve: max_iters reached");
}

meg_status meg_certificate(meg_handle h, double* C_t, int* holds, int* first_hold_iter) {
    meg_status st = ready(h, "meg_certificate");
    if (st != MEG_OK) return st;
    if ((st = check_device_status(h)) != MEG_OK) return st;
    double v[SM_LAST_T + 1];
    CU(cudaMemcpyAsync(v, h->sm, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (C_t) *C_t = v[SM_CERT];
    if (holds) *holds = (int)v[SM_HOLDS];
    if (first_hold_iter) *first_hold_iter = (int)v[SM_FIRST_HOLD];
    return MEG_OK;
}

meg_status meg_get_ritz(meg_handle h, double* sigma, int* t) {
    meg_status st = ready(h, "meg_get_ritz");
    if (st != MEG_OK) return st;
    if ((st = join_group_stream(h)) != MEG_OK) return st;
    std::vector<double> v(SM_SIGMA + MEG_KMAX);
    CU(cudaMemcpyAsync(v.data(), h->sm, sizeof(double) * v.size(), cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (sigma) for (int i = 0; i < h->k; ++i) sigma[i] = v[SM_SIGMA + i];
    if (t) *t = (int)v[SM_LAST_T];
    return check_device_status(h);
}

meg_status meg_get_iterate(meg_handle h, double* V, double* mu, double* s) {
    if (!h) return fail(MEG_ERR_INVALID_ARG, "meg_get_iterate: null handle");
    if (h->failed) return fail(MEG_ERR_STATE, "meg_get_iterate: the solve failed earlier on the device");
    if (!h->has_x) return fail(MEG_ERR_STATE, "meg_get_iterate: X_1 not set");
    if (meg_status js = join_group_stream(h); js != MEG_OK) return js;
    const int n = h->n, r = h->r;
    std::vector<double> smh(SM_MU + MEG_KMAX);
    CU(cudaMemcpyAsync(smh.data(), h->sm, sizeof(double) * smh.size(), cudaMemcpyDeviceToHost, h->stream));
    if (V) CU(cudaMemcpyAsync(V, h->V, sizeof(double) * n * r, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    if (mu) for (int i = 0; i < r; ++i) mu[i] = smh[SM_MU + i];
    if (s) *s = smh[SM_S];
    return check_device_status(h);
}

// ---------------------------------------------------------------------------- checkpoint
namespace {
constexpr int64_t STATE_MAGIC = 0x4D45475354415445LL;   // "MEGSTATE"
constexpr int STATE_HDR = 8;
}

int64_t meg_state_size(meg_handle h) {
    if (!h) return -1;
    return 8 * (STATE_HDR + (int64_t)SM_TOTAL + (int64_t)h->n * h->r) + (int64_t)tsize(h->prec) * h->n * h->k;
}

meg_status meg_get_state(meg_handle h, void* buf, int64_t bytes) {
    if (!h || !buf) return fail(MEG_ERR_INVALID_ARG, "meg_get_state: null argument");
    if (h->failed) return fail(MEG_ERR_STATE, "meg_get_state: the solve failed earlier on the device");
    if (bytes < meg_state_size(h)) return fail(MEG_ERR_INVALID_ARG, "meg_get_state: buffer too small");
    if (meg_status js = join_group_stream(h); js != MEG_OK) return js;
    int64_t* hdr = (int64_t*)buf;
    hdr[0] = STATE_MAGIC; hdr[1] = h->n; hdr[2] = h->r; hdr[3] = h->k; hdr[4] = h->prec;
    hdr[5] = h->desc.kind; hdr[6] = h->has_x; hdr[7] = h->desc.tc;
    char* p = (char*)buf + 8 * STATE_HDR;
    CU(cudaMemcpyAsync(p, h->sm, 8 * SM_TOTAL, cudaMemcpyDeviceToHost, h->stream));
    p += 8 * SM_TOTAL;
    CU(cudaMemcpyAsync(p, h->V, 8 * (size_t)h->n * h->r, cudaMemcpyDeviceToHost, h->stream));
    p += 8 * (size_t)h->n * h->r;
    CU(cudaMemcpyAsync(p, h->W, tsize(h->prec) * (size_t)h->n * h->k, cudaMemcpyDeviceToHost, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    return MEG_OK;
}

meg_status meg_set_state(meg_handle h, const void* buf, int64_t bytes) {
    if (!h || !buf) return fail(MEG_ERR_INVALID_ARG, "meg_set_state: null argument");
    if (bytes < meg_state_size(h)) return fail(MEG_ERR_INVALID_ARG, "meg_set_state: buffer too small");
    const int64_t* hdr = (const int64_t*)buf;
    if (h->failed) return fail(MEG_ERR_STATE, "meg_set_state: the solve failed earlier on the device");
    if (hdr[0] != STATE_MAGIC || hdr[1] != h->n || hdr[2] != h->r || hdr[3] != h->k || hdr[4] != h->prec)
        return fail(MEG_ERR_INVALID_ARG, "meg_set_state: state of a different solve shape or precision");
    // the small state carries constants of the objective (Tr D, ||D||_F^2, shift
    // bounds) and of the product path: a solve with an objective accepts only a
    // state saved under the same objective kind and dense-product path
    if (h->has_obj && (hdr[5] != h->desc.kind || hdr[7] != h->desc.tc))
        return fail(MEG_ERR_INVALID_ARG, "meg_set_state: state saved under another objective kind or product path");
    if (meg_status js = join_group_stream(h); js != MEG_OK) return js;
    const char* p = (const char*)buf + 8 * STATE_HDR;
    CU(cudaMemcpyAsync(h->sm, p, 8 * SM_TOTAL, cudaMemcpyHostToDevice, h->stream));
    p += 8 * SM_TOTAL;
    CU(cudaMemcpyAsync(h->V, p, 8 * (size_t)h->n * h->r, cudaMemcpyHostToDevice, h->stream));
    p += 8 * (size_t)h->n * h->r;
    CU(cudaMemcpyAsync(h->W, p, tsize(h->prec) * (size_t)h->n * h->k, cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    h->has_x = hdr[6] != 0;
    return MEG_OK;
}

meg_status meg_destroy(meg_handle h) {
    if (!h) return MEG_OK;
    cudaStreamSynchronize(h->stream);
    if (h->in_group) cudaStreamSynchronize(h->group_stream);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->solve_gexec) cudaGraphExecDestroy(h->solve_gexec);
    void* bufs[] = {h->V, h->Vn, h->W, h->Wp, h->Z, h->Y, h->Ys, h->Wsp, h->part, h->ctr,
                    h->sm, h->meas, h->bidx, h->mtp, h->d_f, h->d_desc};
    for (void* b : bufs)
        if (b) cudaFreeAsync(b, h->stream);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h->solo_maps;
    delete h;
    return MEG_OK;
}

// ---------------------------------------------------------------------------- groups
namespace {
// warm: the descriptors get the warm-start mode (operator -grad f(0), the
// measurement pass over all m measurements) and X_1 need not be set yet
meg_status group_create_impl(const meg_handle* solves, int count, void* stream, bool warm, meg_group* out);
}  // namespace

meg_status meg_group_create(const meg_handle* solves, int count, void* stream, meg_group* out) {
    return group_create_impl(solves, count, stream, false, out);
}

namespace {
meg_status group_create_impl(const meg_handle* solves, int count, void* stream, bool warm, meg_group* out) {
    if (!solves || count < 1 || !out) return fail(MEG_ERR_INVALID_ARG, "meg_group_create: arguments");
    *out = nullptr;
    if (!solves[0]) return fail(MEG_ERR_INVALID_ARG, "meg_group_create: null handle");
    const int prec = solves[0]->prec, q = solves[0]->q;
    for (int i = 0; i < count; ++i) {
        meg_solve_s* h = solves[i];
        if (!h || !h->has_obj || (!warm && !h->has_x)) return fail(MEG_ERR_STATE, "meg_group_create: solve not ready");
        if (h->failed) return fail(MEG_ERR_STATE, "meg_group_create: a solve failed earlier on the device");
        if (h->in_group) return fail(MEG_ERR_STATE, "meg_group_create: solve already in a group");
        if (h->prec != prec || h->q != q || h->desc.eig != solves[0]->desc.eig)
            return fail(MEG_ERR_INVALID_ARG, "meg_group_create: solves must share precision, q and eigensolver");
    }
    meg_group_s* g = new meg_group_s();
    g->stream = (cudaStream_t)stream;
    if (!g->stream) {
        if (cudaStreamCreate(&g->stream) != cudaSuccess) {
            delete g;
            return fail(MEG_ERR_CUDA, "meg_group_create: stream creation failed");
        }
        g->own_stream = true;
    }
    g->q = q;
    g->krylov = solves[0]->desc.eig == MEG_EIG_BLOCK_KRYLOV;
    std::vector<SolveDev> descs(count);
    int tot[PK_COUNT] = {};
    for (int i = 0; i < count; ++i) {
        meg_solve_s* h = solves[i];
        g->solves.push_back(h);
        descs[i] = h->desc;
        if (warm) {
            descs[i].mode = 1;
            if (descs[i].kind == MEG_MEAS_STOCH) descs[i].nb_meas = (int)descs[i].m;
        }
        for (int p = 0; p < PK_COUNT; ++p) {
            descs[i].off[p] = tot[p];
            tot[p] += blocks_of(descs[i], p);
        }
        const int kind = h->desc.kind;
        g->has_dense |= (kind == MEG_DENSE_QUAD || kind == MEG_LINEAR);
        g->has_csr |= kind == MEG_CSR_QUAD;
        g->has_meas |= meas_kind(kind);
    }
    // tensor-core solves: chunks of at most TC_MAXG solves, one stream-K launch
    // each; offsets, chunk totals and grids go into both descriptor copies
    // (the product reads the chunk's copy, k_combine the group's)
    std::vector<int> tc_idx;
    for (int i = 0; i < count; ++i)
        if (blocks_of(descs[i], PK_DTC) > 0) tc_idx.push_back(i);
    const int nch = ((int)tc_idx.size() + TC_MAXG - 1) / TC_MAXG;
    if (nch > TC_MAX_CHUNKS) {
        if (g->own_stream) cudaStreamDestroy(g->stream);
        delete g;
        return fail(MEG_ERR_INVALID_ARG, "meg_group_create: too many tensor-core solves in one group");
    }
    g->tc_maps.resize(nch);
    for (int c = 0; c < nch; ++c) {
        long long off = 0;
        int nkb_max = 1, npad_max = 16;
        const int first = c * TC_MAXG, cnt = std::min(TC_MAXG, (int)tc_idx.size() - first);
        for (int j = 0; j < cnt; ++j) {
            SolveDev& d = descs[tc_idx[first + j]];
            d.off[PK_DTC] = (int)off;
            off += tc_chunks_of(d);
            nkb_max = std::max(nkb_max, d.tc_kpad / 64);
            npad_max = std::max(npad_max, d.tc_npad);
            g->tc_maps[c].a[j] = solves[tc_idx[first + j]]->solo_maps->a[0];
            g->tc_maps[c].b[j] = solves[tc_idx[first + j]]->solo_maps->b[0];
        }
        const int G = tc_grid(off, nkb_max);
        for (int j = 0; j < cnt; ++j) {
            descs[tc_idx[first + j]].tc_T = off;
            descs[tc_idx[first + j]].tc_G = G;
        }
        g->gl.tc_ns[c] = cnt;
        g->gl.tc_T[c] = off;
        g->gl.tc_G[c] = G;
        g->gl.tc_npad[c] = npad_max;
    }
    std::vector<SolveDev> tcd;
    for (int i : tc_idx) tcd.push_back(descs[i]);
    // the group's stream waits (on the device) for each member's queued work
    cudaEvent_t ready = nullptr;
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess) {
        if (g->own_stream) cudaStreamDestroy(g->stream);
        delete g;
        return fail(MEG_ERR_CUDA, "meg_group_create: event");
    }
    for (auto* h : g->solves) {
        cudaEventRecord(ready, h->stream);
        cudaStreamWaitEvent(g->stream, ready, 0);
    }
    cudaEventDestroy(ready);
    auto undo = [&](meg_status st, const char* msg) {
        if (g->d_desc) cudaFreeAsync(g->d_desc, g->stream);
        if (g->d_tc_desc) cudaFreeAsync(g->d_tc_desc, g->stream);
        if (g->d_f) cudaFreeAsync(g->d_f, g->stream);
        cudaStreamSynchronize(g->stream);
        if (g->own_stream) cudaStreamDestroy(g->stream);
        delete g;
        return fail(st, msg);
    };
    if (cudaMallocAsync((void**)&g->d_desc, sizeof(SolveDev) * count, g->stream) != cudaSuccess ||
        cudaMallocAsync((void**)&g->d_f, sizeof(double) * count, g->stream) != cudaSuccess)
        return undo(MEG_ERR_OOM, "meg_group_create: descriptors");
    if (cudaMemcpyAsync(g->d_desc, descs.data(), sizeof(SolveDev) * count, cudaMemcpyHostToDevice, g->stream) !=
        cudaSuccess)
        return undo(MEG_ERR_CUDA, "meg_group_create: descriptor copy");
    g->gl.d_solves = g->d_desc;
    g->gl.ns = count;
    for (int p = 0; p < PK_COUNT; ++p) g->gl.blocks[p] = tot[p];
    g->gl.prec = prec;
    g->gl.stream = g->stream;
    g->gl.meas_vr = 0;
    g->gl.meas_tc = g->gl.meas_plain = g->gl.meas_bil = 0;
    for (auto* h : g->solves)
        if (meas_kind(h->desc.kind)) {
            g->gl.meas_vr = std::max(g->gl.meas_vr, h->n * (rank_bucket(h->r) + 1));
            if (h->desc.kind == MEG_BILINEAR) g->gl.meas_bil = 1;
            else if (h->desc.mtc) g->gl.meas_tc = 1;
            else g->gl.meas_plain = 1;
        }
    if (!tcd.empty()) {
        if (cudaMallocAsync((void**)&g->d_tc_desc, sizeof(SolveDev) * tcd.size(), g->stream) != cudaSuccess ||
            cudaMemcpyAsync(g->d_tc_desc, tcd.data(), sizeof(SolveDev) * tcd.size(), cudaMemcpyHostToDevice,
                            g->stream) != cudaSuccess)
            return undo(MEG_ERR_CUDA, "meg_group_create: tensor-core descriptors");
    }
    // the host vectors above go out of scope: finish the copies first
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) return undo(MEG_ERR_CUDA, "meg_group_create: copies");
    g->gl.tc_chunks = nch;
    for (int c = 0; c < nch; ++c) {
        g->gl.tc_desc[c] = g->d_tc_desc + c * TC_MAXG;
        g->gl.tc_maps[c] = &g->tc_maps[c];
    }
    for (auto* h : g->solves) { h->in_group = true; h->group_stream = g->stream; }
    *out = g;
    return MEG_OK;
}
}  // namespace

meg_status meg_warm_start_many(const meg_handle* solves, int count, int products, void* stream, double* f1) {
    if (!solves || count < 1 || products < 1) return fail(MEG_ERR_INVALID_ARG, "meg_warm_start_many: arguments");
    for (int i = 0; i < count; ++i) {
        meg_solve_s* h = solves[i];
        if (!h) return fail(MEG_ERR_INVALID_ARG, "meg_warm_start_many: null handle");
        if (!h->has_obj) return fail(MEG_ERR_STATE, "meg_warm_start_many: objective not set");
        if (h->in_group) return fail(MEG_ERR_STATE, "meg_warm_start_many: solve belongs to a group");
        if (h->failed) return fail(MEG_ERR_STATE, "meg_warm_start_many: a solve failed earlier on the device");
    }
    // random start block, as meg_warm_start draws it
    for (int i = 0; i < count; ++i) {
        meg_solve_s* h = solves[i];
        const int n = h->n, r = h->r, k = h->k;
        std::vector<double> vh((size_t)n * r), wh((size_t)n * k);
        std::mt19937_64 gen(h->opt.seed ^ 0xA11CE5ull);
        std::normal_distribution<double> nd(0.0, 1.0);
        for (int a = 0; a < n; ++a)
            for (int j = 0; j < k; ++j) {
                const double v = nd(gen);
                wh[(size_t)a * k + j] = v;
                if (j < r) vh[(size_t)a * r + j] = v;
            }
        meg_status st;
        if ((st = upload_f64(h, h->V, vh)) != MEG_OK || (st = upload_T(h, h->W, wh)) != MEG_OK) return st;
    }
    meg_group g = nullptr;
    meg_status st = group_create_impl(solves, count, stream, true, &g);
    if (st != MEG_OK) return st;
    st = enqueue_init_orth(g->gl);
    if (st == MEG_OK && g->has_csr) st = launch_csr(g->gl) == cudaSuccess ? MEG_OK : MEG_ERR_CUDA;
    if (st == MEG_OK) st = enqueue_iteration(g->gl, g->has_dense, g->has_csr, g->has_meas, products);
    if (st == MEG_OK && f1) st = meg_internal::group_objective_enqueue(g, f1);
    if (st == MEG_OK && cudaStreamSynchronize(g->stream) != cudaSuccess) st = fail(MEG_ERR_CUDA, "meg_warm_start_many");
    meg_group_destroy(g);
    if (st != MEG_OK) return st;
    for (int i = 0; i < count; ++i) {
        meg_solve_s* h = solves[i];
        cudaStreamSynchronize(h->stream);
        h->has_x = true;
        if ((st = check_device_status(h)) != MEG_OK) return st;
        if ((st = refresh_bounds(h)) != MEG_OK) return st;
        if (f1) {
            CU(cudaMemcpyAsync(h->sm + SM_F1, f1 + i, sizeof(double), cudaMemcpyHostToDevice, h->stream));
            CU(cudaStreamSynchronize(h->stream));
        } else if ((st = record_f1(h)) != MEG_OK) {
            return st;
        }
    }
    return MEG_OK;
}

meg_status meg_group_step(meg_group g, int nsteps) {
    if (!g) return fail(MEG_ERR_INVALID_ARG, "meg_group_step: null group");
    if (!g->gexec) {
        cudaGraph_t graph;
        CU(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
        meg_status st = enqueue_iteration(g->gl, g->has_dense, g->has_csr, g->has_meas, g->q, g->krylov);
        cudaError_t ce = cudaStreamEndCapture(g->stream, &graph);
        if (st != MEG_OK) return st;
        if (ce != cudaSuccess) return fail(MEG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&g->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return fail(MEG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
    }
    for (int i = 0; i < nsteps; ++i) CU(cudaGraphLaunch(g->gexec, g->stream));
    return MEG_OK;
}

meg_status meg_group_launch(meg_group g, int nsteps) {
    if (!g || nsteps < 0) return fail(MEG_ERR_INVALID_ARG, "meg_group_launch: arguments");
    for (int i = 0; i < nsteps; ++i) {
        meg_status st = enqueue_iteration(g->gl, g->has_dense, g->has_csr, g->has_meas, g->q, g->krylov);
        if (st != MEG_OK) return st;
    }
    return MEG_OK;
}

meg_status meg_group_objective(meg_group g, double* f) {
    if (!g || !f) return fail(MEG_ERR_INVALID_ARG, "meg_group_objective: arguments");
    meg_status st = meg_internal::group_objective_enqueue(g, f);
    if (st != MEG_OK) return st;
    CU(cudaStreamSynchronize(g->stream));
    return MEG_OK;
}

meg_status meg_group_time_product(meg_group g, int reps, float* ms_per_launch) {
    if (!g || reps < 1 || !ms_per_launch) return fail(MEG_ERR_INVALID_ARG, "meg_group_time_product: arguments");
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    // one untimed launch, then `reps` back-to-back launches between two events
    auto product = [&]() -> cudaError_t {
        cudaError_t e = cudaSuccess;
        if (g->has_dense && (e = launch_dense(g->gl)) != cudaSuccess) return e;
        if (g->has_csr && (e = launch_csr(g->gl)) != cudaSuccess) return e;
        if (g->has_meas && (e = launch_meas_batch(g->gl)) != cudaSuccess) return e;
        if (g->has_meas && (e = launch_meas_apply(g->gl)) != cudaSuccess) return e;
        return e;
    };
    CU(product());
    CU(cudaEventRecord(e0, g->stream));
    for (int i = 0; i < reps; ++i) CU(product());
    CU(cudaEventRecord(e1, g->stream));
    CU(cudaEventSynchronize(e1));
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_per_launch = ms / reps;
    return MEG_OK;
}

meg_status meg_group_time_chain(meg_group g, int reps, float* us) {
    if (!g || reps < 1 || !us) return fail(MEG_ERR_INVALID_ARG, "meg_group_time_chain: arguments");
    // the kernels rewrite W, its bf16 split and the small-slot state: copy them
    // aside and put them back afterwards (the other buffers they write are scratch)
    std::vector<std::pair<void*, size_t>> regions;
    for (auto* h : g->solves) {
        regions.push_back({h->W, tsize(h->prec) * h->n * h->k});
        regions.push_back({h->sm, sizeof(double) * SM_TOTAL});
        if (h->Wsp) regions.push_back({h->Wsp, (size_t)2 * h->desc.tc_npad * h->desc.tc_kpad});
    }
    size_t total = 0;
    for (auto& r : regions) total += (r.second + 255) / 256 * 256;
    char* keep = nullptr;
    if (cudaMallocAsync((void**)&keep, total, g->stream) != cudaSuccess) {
        cudaGetLastError();
        return fail(MEG_ERR_OOM, "meg_group_time_chain: scratch");
    }
    auto copy = [&](bool back) -> cudaError_t {
        size_t o = 0;
        for (auto& r : regions) {
            cudaError_t e = back ? cudaMemcpyAsync(r.first, keep + o, r.second, cudaMemcpyDeviceToDevice, g->stream)
                                 : cudaMemcpyAsync(keep + o, r.first, r.second, cudaMemcpyDeviceToDevice, g->stream);
            if (e != cudaSuccess) return e;
            o += (r.second + 255) / 256 * 256;
        }
        return cudaSuccess;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = copy(false);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int w = 0; w < 6 && e == cudaSuccess; ++w) {
        us[w] = 0.f;
        if (g->gl.prec != MEG_FP64 && (w == 3 || w == 4)) continue;   // single CholeskyQR pass
        for (int i = 0; i <= reps && e == cudaSuccess; ++i) {      // one untimed launch first
            if (i == 1) e = cudaEventRecord(e0, g->stream);
            if (e == cudaSuccess) e = launch_chain_kernel(g->gl, w, PH_ADVANCE);
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, g->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        us[w] = 1000.f * ms / reps;
    }
    const cudaError_t e2 = copy(true);
    if (e == cudaSuccess) e = e2;
    cudaFreeAsync(keep, g->stream);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess) return fail(MEG_ERR_CUDA, std::string("meg_group_time_chain: ") + cudaGetErrorString(e));
    return MEG_OK;
}

int meg_group_kernels_per_step(meg_group g) {
    if (!g) return -1;
    // per product: the gradient-part kernels (one tensor-core launch per chunk of
    // tensor-core solves, one FFMA launch for the other dense solves), CSR,
    // the two minibatch passes, and combine plus the orthonormalisation, each a
    // row kernel followed by an island kernel (float64 storage: combine, orth1,
    // orth2; float storage: combine, orth); plus the begin kernel once per iteration
    const int dense = g->gl.tc_chunks + (g->gl.blocks[PK_DENSE] > 0 ? 1 : 0);
    const int csr = g->has_csr ? (g->gl.prec == MEG_FP64 ? 1 : 2) : 0;   // float modes: V cast + product
    // minibatch: batch and apply passes (tensor cores: the operand split, batch pass, its
    // finish, apply pass; the bilinear kind shares the tensor-core passes and has its own finish)
    const bool tcp = g->gl.meas_tc || g->gl.meas_bil;
    const int meas = g->has_meas ? (tcp ? 3 : 0) + (g->gl.meas_tc ? 1 : 0) +
                                       (g->gl.meas_plain ? 2 : 0)
                                 : 0;
    const int per = dense + csr + meas + (g->gl.prec == MEG_FP64 ? 6 : 4);
    // block Krylov: the projection pass and its factor kernel after the first product
    return g->q * per + 1 + (g->krylov ? 2 : 0);
}

meg_status meg_group_destroy(meg_group g) {
    if (!g) return MEG_OK;
    // members' later work (and frees) on their own streams follows the group's
    cudaEvent_t done = nullptr;
    if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(done, g->stream);
        for (auto* h : g->solves) cudaStreamWaitEvent(h->stream, done, 0);
    } else {
        cudaStreamSynchronize(g->stream);
    }
    if (g->gexec) cudaGraphExecDestroy(g->gexec);
    if (g->d_desc) cudaFreeAsync(g->d_desc, g->stream);
    if (g->d_tc_desc) cudaFreeAsync(g->d_tc_desc, g->stream);
    if (g->d_f) cudaFreeAsync(g->d_f, g->stream);
    if (done) cudaEventDestroy(done);
    for (auto* h : g->solves) { h->in_group = false; h->group_stream = nullptr; }
    if (g->own_stream) cudaStreamDestroy(g->stream);
    delete g;
    return MEG_OK;
}

}  // extern "C"
