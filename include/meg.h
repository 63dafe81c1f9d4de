/*
 * meg.h -- C ABI of the GB300 low-rank Matrix Exponentiated Gradient library.
 *
 * The library minimises a convex f over the spectrahedron
 *     S_n = { X symmetric, X >= 0, Tr X = 1 }                (eq. Model)
 * with the low-rank MEG method of Garber & Kaplan (Algorithm 2): each
 * iteration takes the top-r eigen-decomposition of the mirror matrix
 *     M_t = log X_t - eta_t grad f(X_t)
 * and sets
 *     X_{t+1} = (1 - eps_t) Y^r / a_t + eps_t/(n - r) (I - V V^T),
 *     Y^r = V diag(exp sigma_1..r) V^T,  a_t = sum_{i<=r} exp sigma_i
 * (Definition 2, eq. LowRankMDvonNeumannUpdate).  X_t is held in the
 * factored form of eq. (eigenFastUpdate): V (n x r, orthonormal), mu (r)
 * and s, X = V diag(mu) V^T + s (I - V V^T).  The eigenpairs come from a
 * warm-started block subspace iteration (CholeskyQR: two passes in float64
 * storage, one pass with a factor refined in Gram space in the float
 * storage modes) and a Rayleigh-Ritz step (Section 3).
 *
 * Conventions for every call:
 *   - Matrices are row-major.  "host" pointers are ordinary CPU memory,
 *     "device" pointers are CUDA global memory of the current device.
 *   - All calls are ordered on the solve's CUDA stream (meg_options.stream,
 *     NULL = the legacy default stream).  meg_create, meg_set_objective
 *     and meg_step only enqueue work; meg_certificate, meg_get_iterate,
 *     meg_get_ritz, meg_objective and meg_solve synchronise that stream.
 *   - Errors are returned as meg_status; nothing throws across the ABI.
 *     meg_last_error() gives a thread-local message for the last failure.
 *   - A solve that hit MEG_ERR_NUMERIC or MEG_ERR_TIMEOUT on the device
 *     answers MEG_ERR_STATE to every later call except meg_destroy.
 */
#ifndef MEG_H
#define MEG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct meg_solve_s* meg_handle;   /* one solve; owned by the library */
typedef struct meg_group_s* meg_group;    /* several solves stepped together */

typedef enum {
    MEG_OK = 0,
    MEG_ERR_INVALID_ARG = 1,
    MEG_ERR_OOM = 2,
    MEG_ERR_CUDA = 3,
    MEG_ERR_NUMERIC = 4,       /* Cholesky breakdown, non-finite Ritz value */
    MEG_ERR_NOT_CONVERGED = 5, /* meg_solve reached max_iters */
    MEG_ERR_TIMEOUT = 6,       /* a bounded device wait gave up */
    MEG_ERR_STATE = 7          /* handle unusable (earlier error, wrong order) */
} meg_status;

/* Arithmetic of the path (precision modes). */
enum {
    MEG_FP64 = 0,        /* every array and operation in float64 */
    MEG_FP32 = 1,        /* float32 arrays and products; compensated
                            (double-word) reductions; float32 k x k island
                            (Cholesky, Jacobi) with double-word refinement,
                            float64 Ritz values, exp-map and certificate */
    MEG_MIXED_BF16 = 2   /* as MEG_FP32, dense data in bfloat16 and the dense
                            product on tcgen05 tensor cores (fp32 accumulate) */
};

/* Eigensolver of the top-r eigenpairs of M_t (meg_options.eigensolver),
 * both warm-started from the previous iteration's Ritz vectors (Section 3:
 * block subspace iteration, or the faster Lanczos-type methods it names). */
enum {
    MEG_EIG_SUBSPACE = 0,      /* q products, each followed by CholeskyQR; the
                                  Rayleigh-Ritz step on the last block */
    MEG_EIG_BLOCK_KRYLOV = 1   /* q = 2 products: Rayleigh-Ritz on the block
                                  Krylov space span [W, (M_t - cI) W] (2k <= 32
                                  columns); float-storage precisions only */
};

/* Objective kinds (meg_objective_desc.kind). */
enum {
    MEG_DENSE_QUAD = 0,  /* f = 1/2 ||X - M||_F^2,  grad f = X - M            */
    MEG_CSR_QUAD = 1,    /* f = 1/2 sum_{(i,j) in Omega} (X_ij - M_ij)^2,
                            Omega mirrored, grad f = P_Omega(X - M)           */
    MEG_MEAS_STOCH = 2,  /* f = (1/m) sum_i (a_i^T X a_i - y_i)^2; step t uses
                            the minibatch gradient (2/L) sum_b r_b a_b a_b^T   */
    MEG_LINEAR = 3,      /* f = <C, X>,  grad f = C                          */
    MEG_BILINEAR = 4     /* Section 7, eq. recoveryProb, in trace-1 variables:
                            f = 1/2 sum_i (tau a_i^T X b_i - y_i)^2,
                            grad f = (tau/2) sum_i r_i (a_i b_i^T + b_i a_i^T),
                            r_i = tau a_i^T X b_i - y_i (full gradient); with
                            measurement matrices of rank p (mrank):
                            r_i = tau Tr(A_i^T X B_i) - y_i and
                            grad f = (tau/2) sum_i r_i (A_i B_i^T + B_i A_i^T) */
};

/*
 * Options of one solve (Algorithm 2 inputs).
 *   n, r       : dimension and SVD rank, 2 <= n <= 2^28, 1 <= r <= n - 1,
 *                r <= 30.
 *   p          : extra subspace vectors, k = r + p, 1 <= p, k <= min(n, 32).
 *                (p >= 1 because the certificate needs sigma_{r+1}.)
 *   q          : subspace-iteration products per MEG iteration, 1..8.
 *   precision  : MEG_FP64 | MEG_FP32 | MEG_MIXED_BF16.
 *   eta        : constant step size eta_t = eta > 0.
 *   eps_a, eps_c, eps_pow : eps_t = eps_a / (t + eps_c + 1)^eps_pow
 *                (Section 7: 0.8, 10, 2); every eps_t must lie in (0, 3/4]
 *                (Lemma 2).
 *   max_iters, tol : defaults for meg_solve.
 *   seed       : seeds the extra subspace vectors and the minibatch stream.
 *   stream     : cudaStream_t (NULL = default stream).
 *   eigensolver: MEG_EIG_SUBSPACE (0, the default of a zeroed struct) or
 *                MEG_EIG_BLOCK_KRYLOV (needs q = 2, 2 (r + p) <= 32 and
 *                MEG_FP32 or MEG_MIXED_BF16; MEG_ERR_INVALID_ARG otherwise).
 */
typedef struct {
    int n, r, p, q;
    int precision;
    double eta;
    double eps_a, eps_c, eps_pow;
    int max_iters;
    double tol;
    uint64_t seed;
    void* stream;
    int eigensolver;
} meg_options;

/*
 * Objective data.  Every array is a caller-owned DEVICE pointer, borrowed
 * for the lifetime of the handle (the library never frees or writes it).
 *   dense  (DENSE_QUAD: M; LINEAR: C): n x n row-major symmetric;
 *          element type double (MEG_FP64), float (MEG_FP32) or bfloat16
 *          bit patterns, uint16 (MEG_MIXED_BF16).
 *   rowptr, col, val, nnz (CSR_QUAD): CSR of the mirrored sample Omega,
 *          int32 rowptr[n+1], int32 col[nnz] (sorted within a row),
 *          val[nnz] = M_ij as double (MEG_FP64) or float (otherwise).
 *   A, y, m, L (MEAS_STOCH): A m x n row-major, double (MEG_FP64) or
 *          bfloat16 bits (otherwise); y[m] double; minibatch size L.
 *   A, B, y, m, tau, mrank (BILINEAR): m measurements; mrank = p, the
 *          rank of the measurement matrices A_i, B_i in R^{n x p} (0 or 1:
 *          vectors a_i, b_i; else a power of two up to 32); A and B hold
 *          m p rows of n bfloat16 bits, row i p + c being column c of A_i
 *          (of B_i); y[m] double; trace scale tau > 0 (the tau-spectrahedron
 *          of the problem is mapped to the unit one, X' = X / tau); L is
 *          ignored.  Needs MEG_FP32 or MEG_MIXED_BF16, n % 8 == 0, A and B
 *          16-byte aligned and 1 <= m p <= 2^30 - 256 (both products run on
 *          the tensor cores over the 2 m p stacked rows [A; B]);
 *          MEG_ERR_INVALID_ARG otherwise.
 * Fields a kind does not use are ignored (zero them).
 */
typedef struct {
    int kind;
    const void* dense;
    const int* rowptr;
    const int* col;
    const void* val;
    int64_t nnz;
    const void* A;
    const double* y;
    int64_t m;
    int L;
    const void* B;
    double tau;
    int mrank;
} meg_objective_desc;

/*
 * meg_create -- allocate a solve and set X_1 (Algorithm 2, Initialization):
 *   X_1 = (1 - eps_0) X_0 + (eps_0/n) I,  X_0 = V0 diag(lam0) V0^T.
 * V0: host, n x r row-major, orthonormal columns; lam0: host, r values on
 * the unit simplex.  V0 == NULL leaves X_1 unset until meg_warm_start.
 * The library copies V0/lam0; the caller keeps ownership.
 * Errors: MEG_ERR_INVALID_ARG (sizes, schedule), MEG_ERR_OOM (also when
 * meg_footprint of the solve exceeds the device's free memory, checked
 * before anything is allocated), MEG_ERR_CUDA.
 */
meg_status meg_create(const meg_options* opt, const double* V0, const double* lam0,
                      meg_handle* out);

/* meg_set_objective -- attach f (problem statement, eq. Model).  The
 * descriptor is copied, the arrays are borrowed.  The CSR structure is
 * validated on host copies the call makes: rowptr[0] = 0, rowptr[n] = nnz,
 * rowptr monotone, every column index in [0, n).
 * Errors: MEG_ERR_INVALID_ARG, MEG_ERR_CUDA. */
meg_status meg_set_objective(meg_handle h, const meg_objective_desc* d);

/* meg_warm_start -- X_0 of eq. (exp:init) with U = 0: the top-r
 * eigenpairs of -grad f(0) by `products` subspace-iteration products on
 * the device, eigenvalues projected onto the unit simplex, then X_1 as in
 * meg_create.  Needs the objective.  Synchronises the stream. */
meg_status meg_warm_start(meg_handle h, int products);

/* meg_warm_start_many -- meg_warm_start for `count` solves at once (one
 * precision and one q): the products run as grouped kernels on `stream`,
 * with the same results as warming each alone.  f1 (host, count values,
 * may be NULL) receives f(X_1) of each solve.  Synchronises. */
meg_status meg_warm_start_many(const meg_handle* solves, int count, int products, void* stream, double* f1);

/* meg_refine_subspace -- `products` extra subspace-iteration products of
 * the next iteration's operator M_t - c I (Algorithm 2's eigensolver),
 * each followed by the orthonormalisation of the block W; X_t and t are
 * unchanged, so the next meg_step computes the same iterate from a better
 * start block.  Meant for t = 1, where W holds V_0 and random columns
 * (the top-r eigenvectors of M_1 can lie outside span V_0, e.g. after
 * eq. (exp:init) gave some of its directions zero weight).  Needs the
 * objective and X_t; a solve in a group answers MEG_ERR_STATE.
 * products in 0..4096 (MEG_ERR_INVALID_ARG otherwise).  Synchronises the
 * stream and reports a device error as meg_step's callers see it. */
meg_status meg_refine_subspace(meg_handle h, int products);

/* meg_trace_exp_estimate -- an estimate of b = Tr exp(M_t), the scalar of the
 * exact certificate (eq. convergenceGuaranteeExperiment), by sampling as the
 * note after Lemma 2 suggests: Hutchinson's estimator over the k = r + p
 * probe vectors u_j, the columns of U (host, n x k row-major float64, e.g.
 * Gaussian or +-1 entries; the caller draws them), each u^T exp(M_t) u by
 * `steps` Lanczos steps (Gauss quadrature, full reorthogonalisation) on
 * the operator of the solve's next iteration, M_t = log X_t - eta grad f(X_t)
 * (the minibatch gradient of step t for MEAS_STOCH).  *estimate receives
 * (1/k) sum_j ||u_j||^2 e_1^T exp(T_j) e_1.  The iterate, its subspace block
 * and t are unchanged.  Needs the objective and X_t, float storage
 * (MEG_FP32 or MEG_MIXED_BF16) and 1 <= steps <= min(32, n); a solve in a
 * group answers MEG_ERR_STATE.  Allocates (stream-ordered) and frees its
 * scratch; synchronises the stream. */
meg_status meg_trace_exp_estimate(meg_handle h, const double* U, int steps, double* estimate);

/* meg_step -- run `nsteps` iterations of Algorithm 2 (t -> t + nsteps),
 * enqueued on the stream without a host synchronisation. */
meg_status meg_step(meg_handle h, int nsteps);

/* meg_solve -- iterate until the relative objective gap
 * (f(X_t) - fstar)/(f(X_1) - fstar) <= tol or max_iters iterations
 * (problem statement, eq. Model; Algorithm 2 run to a tolerance).
 * fstar = 0 unless meg_set_fstar gave one.  f(X_1) is the objective at
 * the solve's first iterate, recorded when X_1 and the objective are both
 * set (meg_create with V0, meg_set_objective, meg_warm_start) and kept in
 * the checkpoint state.  f is evaluated every 10 iterations with
 * meg_objective's accurate pass and tested on the device: the iterations,
 * the objective pass and the test run as one CUDA graph with a
 * conditional while-node, launched once; the host waits once (and once
 * more for a final max_iters % 10 iterations).  *iters_out (may be NULL)
 * receives the iterations run by this call.
 * Errors: MEG_ERR_INVALID_ARG for tol <= 0, max_iters < 0, or
 * f(X_1) - fstar <= 0 (the gap is undefined: give f* below f(X_1) with
 * meg_set_fstar, e.g. for a linear objective whose f can be negative);
 * MEG_ERR_STATE when f(X_1) is unknown (objective set after the first
 * step) or the solve belongs to a group; MEG_ERR_NUMERIC when f is not
 * finite; MEG_ERR_NOT_CONVERGED when max_iters is reached first. */
meg_status meg_solve(meg_handle h, double tol, int max_iters, int* iters_out);

/* meg_set_fstar -- known optimal value for meg_solve's relative gap. */
meg_status meg_set_fstar(meg_handle h, double fstar);

/* meg_certificate -- certificate of the last iteration t (Lemma 2 with
 * b = b_{r+1}, eq. convergenceGuaranteeExperiment2):
 *   C_t = log((n - r) lambda_{r+1}(Y_t) / (eps_t b_{r+1})),
 * *holds = (C_t <= 2 eps_t); *first_hold_iter = first t at which it held
 * (0 if never).  Any output pointer may be NULL. */
meg_status meg_certificate(meg_handle h, double* C_t, int* holds, int* first_hold_iter);

/* meg_get_iterate -- copy X_t's factors to host memory: V n x r row-major
 * (float64), mu[r], s.  Any output pointer may be NULL. */
meg_status meg_get_iterate(meg_handle h, double* V, double* mu, double* s);

/* meg_get_ritz -- the k leading Ritz values sigma_1 >= ... >= sigma_k of
 * M_t from the last iteration (host, float64) and that iteration's t. */
meg_status meg_get_ritz(meg_handle h, double* sigma, int* t);

/* meg_objective -- f(X_t) for the current iterate, by a dense pass over
 * the objective data (DENSE_QUAD, LINEAR), over Omega (CSR_QUAD) or over
 * all m measurements (MEAS_STOCH), accumulated with compensation. */
meg_status meg_objective(meg_handle h, double* f);

/* Checkpoint / resume.  The state of a solve is everything the next
 * iteration reads: the float64 small state (t, mu, s, shift bounds,
 * certificate history, V^T W, W^T W), V (n x r) and the subspace block W.
 * meg_state_size gives the byte count; meg_get_state copies it to host
 * memory `buf`, meg_set_state restores it into a solve created with the
 * same n, r, p and precision (objective data are not part of the state).
 * The buffer starts with eight int64 header words: a magic number, n, r,
 * k, precision, objective kind, 1 if X_1 is set, and 1 if the dense
 * product runs on the tensor cores (tcgen05) for this solve.  A solve
 * that has an objective accepts only a state saved under the same
 * objective kind and product path (MEG_ERR_INVALID_ARG otherwise): the
 * small state carries constants of the objective data.
 * Iterating T steps, saving, restoring and iterating T more gives the
 * same bits as 2T steps.  Both calls synchronise the stream. */
int64_t meg_state_size(meg_handle h);
meg_status meg_get_state(meg_handle h, void* buf, int64_t bytes);
meg_status meg_set_state(meg_handle h, const void* buf, int64_t bytes);

/* meg_destroy -- free the solve (waits for its stream). NULL is a no-op. */
meg_status meg_destroy(meg_handle h);

/* meg_last_error -- message of the calling thread's last failure. */
const char* meg_last_error(void);

/*
 * Groups: step several solves (any n, r, kind; one precision and one q)
 * with grouped kernels, one launch per kernel for the whole group, the
 * step captured once as a CUDA graph.  The solves keep their own state;
 * results equal those of stepping each alone.  A solve belongs to at
 * most one group at a time; the group borrows the handles.
 */
meg_status meg_group_create(const meg_handle* solves, int count, void* stream, meg_group* out);
meg_status meg_group_step(meg_group g, int nsteps);
meg_status meg_group_destroy(meg_group g);

/* Profiling: average device time of the group's gradient-product kernels
 * (the dense or CSR product, or the two minibatch passes), from `reps`
 * back-to-back launches between two CUDA events on the group's stream.
 * The launches compute the product for the current W and leave the
 * solves' iterates unchanged.  Synchronises the stream. */
meg_status meg_group_time_product(meg_group g, int reps, float* ms_per_launch);

/* meg_group_time_chain -- profiling aid: the warm duration, in microseconds,
 * of each kernel of the chain that follows an intermediate product of the
 * subspace iteration (Section 3: the mirror operator, then CholeskyQR):
 * us[0] the row kernel forming Z = (M_t - c I) W and the partials of Z^T Z,
 * us[1] its per-solve kernel (the CholeskyQR factor).  Float64 storage
 * (two CholeskyQR passes): us[2] W' = Z M1 with the partials of W'^T W',
 * us[3] the second factor, us[4] W = W' M2 with the partials of V^T W and
 * W^T W.  Float storage (one pass): us[2] W = Z M1 with those partials,
 * us[3] = us[4] = 0 (not launched).  us[5] the reduction of V^T W and
 * W^T W.  Each kernel is
 * launched `reps` times back-to-back between two CUDA events on the group's
 * stream after one untimed launch.  W, its split and the solves' small
 * state are copied aside first and restored afterwards, so the iterates and
 * the next step are unchanged.  us must hold 6 floats.  Synchronises the
 * group's stream.  MEG_ERR_OOM if the copies cannot be allocated. */
meg_status meg_group_time_chain(meg_group g, int reps, float* us);

/* Number of kernels one meg_group_step iteration launches. */
int meg_group_kernels_per_step(meg_group g);

/* meg_group_launch -- enqueue `nsteps` iterations of every member like
 * meg_group_step, but as plain kernel launches (no graph capture), for
 * groups that live only a few steps.  Same results. */
meg_status meg_group_launch(meg_group g, int nsteps);

/* meg_group_objective -- f(X_t) of every member (meg_objective's accurate
 * pass, one launch for the group), written to host f[count] in member
 * order.  Synchronises the group's stream. */
meg_status meg_group_objective(meg_group g, double* f);

/*
 * Serving: continuous batching of independent solves on one GPU.  The
 * paper has no counterpart (it runs one solve at a time); each request
 * is an ordinary run of Algorithm 2 from X_1 until its stopping rule.
 * A worker thread of the library admits requests in submission order
 * when a slot is free and their device footprint -- meg_footprint plus a
 * copy of the request's objective data -- fits the memory budget, groups
 * the admitted solves by (precision, q, objective family), runs each
 * group `check_every` iterations at a time on its own stream (groups
 * overlap on the device), evaluates every member's f after each such
 * tick, and retires members whose stopping rule holds:
 *   f* known (finite): (f(X_t) - f*) <= tol (f(X_1) - f*)   (relative gap);
 *   f* unknown (NaN):  f(X_{t-c}) - f(X_t) <= tol (f(X_1) - f(X_t)), c the
 *                      check interval (the iteration's progress has stalled
 *                      at tol of the progress made);
 *   t = max_iters:     status MEG_ERR_NOT_CONVERGED.
 * Results do not depend on which other requests share the GPU: grouped
 * kernels compute each member exactly as it would run alone.
 */
typedef struct meg_server_s* meg_server;

typedef struct {
    int64_t hbm_budget;       /* device bytes the admitted requests may hold */
    int max_active;           /* most requests admitted at once, >= 1 */
    int check_every;          /* iterations per tick (objective check), dense */
    int meas_check_every;     /* same for MEAS_STOCH requests (the full
                                 objective reads all m measurements) */
} meg_server_options;

/* One request.  meg_server_submit copies this struct, not the arrays it
 * points to: the host arrays data, y, V0 and lam0 are read later, when
 * the worker thread admits the request, so they must stay valid and
 * unchanged until the request's result comes back from meg_server_poll;
 * out_V (n x r), out_mu (r) and out_s (1) are written before the result
 * is returned (each may be NULL). */
typedef struct {
    meg_options opt;          /* sizes, precision, schedule, seed; stream ignored */
    int kind;                 /* MEG_DENSE_QUAD, MEG_LINEAR or MEG_MEAS_STOCH */
    const void* data;         /* host: dense n x n, or A m x n (MEAS_STOCH); element
                                 type by precision as in meg_objective_desc */
    const double* y;          /* host: y[m] (MEAS_STOCH) */
    int64_t m;
    int L;
    int warm_start_products;  /* > 0: X_0 by meg_warm_start(products); 0: V0, lam0 */
    const double* V0;
    const double* lam0;
    double fstar;             /* optimal value, or NaN when unknown */
    double tol;               /* > 0 */
    int max_iters;            /* >= 1 */
    double* out_V;
    double* out_mu;
    double* out_s;
} meg_request;

typedef struct {
    uint64_t id;
    meg_status status;        /* MEG_OK, MEG_ERR_NOT_CONVERGED, or the failure */
    int iters;                /* iterations run */
    double f1, f;             /* f(X_1) and f at the last check */
    double t_submit, t_admit, t_done;   /* seconds on the server clock */
} meg_result;

/* Errors: MEG_ERR_INVALID_ARG (non-positive budget, slots or intervals). */
meg_status meg_server_create(const meg_server_options* opt, meg_server* out);
/* Queue a request; *id receives its id.  MEG_ERR_OOM when the request
 * alone exceeds the budget, MEG_ERR_INVALID_ARG for a malformed one. */
meg_status meg_server_submit(meg_server s, const meg_request* rq, uint64_t* id);
/* Move up to max_out finished results into out (oldest first), waiting up
 * to timeout_ms for at least one; *n_out receives the count. */
meg_status meg_server_poll(meg_server s, meg_result* out, int max_out, int* n_out, int timeout_ms);
/* Requests submitted and finished so far. */
meg_status meg_server_counts(meg_server s, int64_t* submitted, int64_t* finished);
/* Ticks launched so far, and how many of them ran as a captured CUDA graph
 * (a class's tick is captured once its group has held for a tick and is
 * relaunched while the membership and the tick length stay the same). */
meg_status meg_server_tick_counts(meg_server s, int64_t* ticks, int64_t* graph_ticks);
/* The server clock (seconds since meg_server_create). */
double meg_server_now(meg_server s);
/* Stop the worker and free everything; unfinished requests are dropped. */
meg_status meg_server_destroy(meg_server s);

/*
 * meg_objective_dense_noalloc -- f(X) = 1/2 ||X - M||_F^2 for
 * X = V diag(mu) V^T + s (I - V V^T), computed without allocating any
 * device memory.  The paper has no counterpart: this serves callers that
 * cannot call cudaMalloc -- code running while a CUDA graph is captured
 * in global or thread-local mode (allocation calls are refused there),
 * serving loops bound to the device-memory budget they were admitted
 * with, and hosts whose device memory is managed elsewhere.
 *   V     : device, n x r row-major float64 (orthonormal columns)
 *   mu    : host, r values;  s : the value of X off span V
 *   M     : device, n x n row-major; double (MEG_FP64), float (MEG_FP32)
 *           or bfloat16 bits (MEG_MIXED_BF16), as in meg_objective_desc
 *   f_out : device, one double, written when the work on `stream` ends
 * The reduction scratch is one fixed array of the library (about 35 KB
 * per GPU that loads it, kept until the process exits), so n is limited
 * to MEG_NOALLOC_MAX_N; larger n returns MEG_ERR_INVALID_ARG.  The first
 * call on a device looks up that array's device address (with the
 * device current) and caches it with the current CUDA context; a call
 * under another context (after a device reset) looks it up again.  Make
 * the first call, and the first after a reset, before any stream capture.
 * Each call enqueues two operations on `stream`: a memset that zeroes the
 * array's counters, then the reduction kernel (a captured call records
 * two graph nodes); *f_out is valid once both have run.
 * Every call shares the array: calls whose work overlaps on the GPU
 * (different streams, or different host threads) race -- order them.
 * The result equals meg_objective's for the same iterate and data.
 */
#define MEG_NOALLOC_MAX_N 65536
meg_status meg_objective_dense_noalloc(const double* V, const double* mu, double s, int n, int r,
                                       const void* M, int precision, double* f_out, void* stream);

/*
 * meg_autotune -- choose p (extra subspace vectors) and q (products per
 * iteration) for one problem (Section 3's subspace iteration; the paper
 * fixes neither).  A reference solve with more vectors and products than
 * any candidate and one pilot solve per candidate run `pilot_iters`
 * iterations from X_1 (V0, lam0 as in meg_create; host) on the objective
 * `obj` (device data, borrowed), all in base->precision.  Candidates are
 * tried in order of cost, q = 1..q_max, then p ascending; the first whose
 * iterate is within tol_x * sqrt(pilot_iters / horizon) of the reference
 * (relative Frobenius distance) is returned in *p_out, *q_out, its
 * distance in *err_out (may be NULL).  The choice depends on results, not
 * timings.  If none qualifies the most accurate candidate is returned with
 * MEG_ERR_NOT_CONVERGED.  With ao->krylov set (float storage), the block
 * Krylov eigensolver is a candidate too: at q = 2 it is tried after
 * subspace iteration and before q = 3 (two products and a 2k x 2k
 * Rayleigh-Ritz step; p with 2 (r + p) <= 32);
 * *eig_out (may be NULL) receives the chosen eigensolver.  The reference
 * solve always uses subspace iteration.  The paper has no counterpart.
 */
typedef struct {
    int q_max;            /* largest q tried, 1..7 (the reference uses q_max + 2, at most 8) */
    const int* p_cand;    /* candidate p values (host), or NULL for {2, 4, 6, 8, 12, 16} */
    int n_p;
    int pilot_iters;      /* iterations of each pilot run */
    int horizon;          /* iterations the solve will run */
    double tol_x;         /* target relative Frobenius error of X_t at the horizon */
    int krylov;           /* 1: also try MEG_EIG_BLOCK_KRYLOV (q = 2) */
} meg_autotune_options;

meg_status meg_autotune(const meg_options* base, const meg_objective_desc* obj, const double* V0,
                        const double* lam0, const meg_autotune_options* ao, int* p_out, int* q_out,
                        double* err_out, int* eig_out);

/* Device-memory footprint in bytes of one solve (library-owned buffers,
 * not the caller's objective data), for admission control. */
int64_t meg_footprint(int n, int r, int p, int precision, int kind);

#ifdef __cplusplus
}
#endif

#endif /* MEG_H */
