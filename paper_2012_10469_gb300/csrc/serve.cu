// Serving loop: continuous batching of independent low-rank MEG solves on one
// GPU.  The paper has no counterpart (it runs one solve at a time); every
// request is an ordinary run of Algorithm 2.
//
// One worker thread owns all device work:
//   admission  -- requests wait in FIFO order until a slot is free and their
//                 device footprint (solve state from meg_footprint plus a
//                 copy of their objective data) fits the memory budget; the
//                 data are copied in on the request's own stream, X_1 is set
//                 (given X_0 or the warm start of eq. exp:init) and f(X_1) is
//                 evaluated;
//   classes    -- admitted solves of one (precision, q, eigensolver, objective family)
//                 form a group (grouped kernels, one launch per kernel for
//                 all members) on the class's own stream, so classes overlap
//                 on the device;
//   ticks      -- a class runs `check` iterations of all members, then the
//                 grouped objective pass; the host polls an event and never
//                 blocks on a running tick.  From the second tick of an
//                 unchanged group the tick is a captured CUDA graph, relaunched
//                 until the membership or the tick length changes;
//   retirement -- a member stops when (f - f*) <= tol (f(X_1) - f*) for a
//                 known f*, or, when f* is unknown, when the decrease over
//                 the last check interval is <= tol (f(X_1) - f(X_t)); also at
//                 max_iters or on a numeric failure.  Its factors are copied
//                 to the caller's buffers, its memory released, and the group
//                 is rebuilt with the remaining and newly admitted members.
// Allocations are stream-ordered, so admitting or retiring a request never
// synchronises the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/meg.h"
#include "meg_dev.cuh"

namespace meg_internal {
void set_last_error(const std::string& msg);
cudaStream_t group_stream(meg_group g);
meg_status group_objective_enqueue(meg_group g, double* f);
meg_status solve_status(meg_handle h);
}  // namespace meg_internal

namespace {

meg_status sfail(meg_status st, const std::string& msg) {
    meg_internal::set_last_error(msg);
    return st;
}

size_t elem_bytes(int precision) { return precision == MEG_FP64 ? 8 : (precision == MEG_FP32 ? 4 : 2); }

struct Req {
    uint64_t id = 0;
    meg_request rq{};
    double t_submit = 0.0, t_admit = 0.0;
    int64_t footprint = 0;
    int cls = -1;
    meg_handle h = nullptr;
    cudaStream_t stream = nullptr;
    void* d_data = nullptr;
    double* d_y = nullptr;
    int iters = 0;
    double f1 = 0.0, f_prev = NAN, f = NAN;
    bool finished = false;
    meg_status status = MEG_OK;
};

struct Class {
    int precision = 0, q = 0, meas = 0, eig = 0, check = 10;
    std::vector<Req*> members;         // the running group, in member order
    std::vector<Req*> joining;         // admitted while a tick was running
    meg_group g = nullptr;
    bool dirty = false;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    bool inflight = false;
    int tick_len = 0;
    double* f_host = nullptr;          // pinned, one per member of the running tick
    int f_cap = 0;
    // CUDA graph of a tick (its iterations and the objective pass with the copy of f):
    // captured on the second tick of an unchanged group and relaunched while the
    // group and the tick length stay the same
    unsigned gen = 0;                  // bumped whenever the group is rebuilt
    int ticks_same = 0;                // ticks launched since then
    cudaGraphExec_t gexec = nullptr;
    unsigned gexec_gen = 0;
    int gexec_len = 0;
};

}  // namespace

struct meg_server_s {
    meg_server_options opt{};
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> pending;
    std::vector<meg_result> done;
    std::atomic<bool> stop{false};
    uint64_t next_id = 1;
    int64_t submitted = 0, finished = 0;
    std::atomic<int64_t> ticks{0}, graph_ticks{0};   // ticks launched; of them from a captured graph
    // worker-owned
    std::vector<Class> classes;
    int active = 0;
    int64_t used = 0;
    std::thread worker;
    std::string worker_error;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    cudaStream_t admit_stream = nullptr;
    void run();
    bool admit(Req* q);
    void admit_batch(std::vector<Req*>& ready);
    int class_of(const meg_request& rq);
    void launch_tick(Class& c);
    meg_status capture_tick(Class& c, int len);
    void finish_tick(Class& c);
    void retire(Req* q);
};

int meg_server_s::class_of(const meg_request& rq) {
    const int meas = rq.kind == MEG_MEAS_STOCH;
    for (size_t i = 0; i < classes.size(); ++i)
        if (classes[i].precision == rq.opt.precision && classes[i].q == rq.opt.q && classes[i].meas == meas &&
            classes[i].eig == rq.opt.eigensolver)
            return (int)i;
    Class c;
    c.precision = rq.opt.precision;
    c.q = rq.opt.q;
    c.eig = rq.opt.eigensolver;
    c.meas = meas;
    c.check = meas ? opt.meas_check_every : opt.check_every;
    cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&c.ev, cudaEventDisableTiming);
    classes.push_back(c);
    return (int)classes.size() - 1;
}

// First half of admission: stream, device copy of the data, solve, objective.
bool meg_server_s::admit(Req* q) {
    const meg_request& rq = q->rq;
    const int n = rq.opt.n;
    meg_status st = MEG_OK;
    q->t_admit = now();                       // its memory is reserved from here on
    cudaStreamCreateWithFlags(&q->stream, cudaStreamNonBlocking);
    meg_options o = rq.opt;
    o.stream = q->stream;
    meg_objective_desc d{};
    d.kind = rq.kind;
    size_t bytes = 0;
    if (rq.kind == MEG_MEAS_STOCH) bytes = (size_t)rq.m * n * elem_bytes(rq.opt.precision);
    else bytes = (size_t)n * n * elem_bytes(rq.opt.precision);
    if (cudaMallocAsync(&q->d_data, bytes, q->stream) != cudaSuccess ||
        cudaMemcpyAsync(q->d_data, rq.data, bytes, cudaMemcpyHostToDevice, q->stream) != cudaSuccess) {
        st = MEG_ERR_OOM;
    }
    if (st == MEG_OK && rq.kind == MEG_MEAS_STOCH) {
        if (cudaMallocAsync((void**)&q->d_y, sizeof(double) * rq.m, q->stream) != cudaSuccess ||
            cudaMemcpyAsync(q->d_y, rq.y, sizeof(double) * rq.m, cudaMemcpyHostToDevice, q->stream) != cudaSuccess)
            st = MEG_ERR_OOM;
        d.A = q->d_data;
        d.y = q->d_y;
        d.m = rq.m;
        d.L = rq.L;
    } else {
        d.dense = q->d_data;
    }
    const bool warm = rq.warm_start_products > 0;
    if (st == MEG_OK) st = meg_create(&o, warm ? nullptr : rq.V0, warm ? nullptr : rq.lam0, &q->h);
    if (st == MEG_OK) st = meg_set_objective(q->h, &d);
    if (st == MEG_OK && std::isfinite(rq.fstar)) st = meg_set_fstar(q->h, rq.fstar);
    if (st == MEG_OK && !warm) st = meg_objective(q->h, &q->f1);
    if (st != MEG_OK) {
        q->status = st;
        retire(q);
        return false;
    }
    return true;
}

// Second half for a batch of prepared requests: warm starts run together
// (grouped kernels, one pass for every solve of the same precision, q and
// product count), f(X_1) from the same grouped pass; then each request joins
// its class at the next tick boundary.
void meg_server_s::admit_batch(std::vector<Req*>& ready) {
    std::map<std::tuple<int, int, int, int>, std::vector<Req*>> warm;
    for (Req* q : ready)
        if (q->rq.warm_start_products > 0)
            warm[std::make_tuple(q->rq.opt.precision, q->rq.opt.q, q->rq.warm_start_products, q->rq.opt.eigensolver)]
                .push_back(q);
    for (auto& kv : warm) {
        std::vector<Req*>& v = kv.second;
        std::vector<meg_handle> hs;
        for (Req* q : v) hs.push_back(q->h);
        std::vector<double> f1(v.size(), NAN);
        const meg_status st =
            meg_warm_start_many(hs.data(), (int)hs.size(), std::get<2>(kv.first), admit_stream, f1.data());
        for (size_t i = 0; i < v.size(); ++i) {
            v[i]->f1 = f1[i];
            if (st != MEG_OK) v[i]->status = st;
        }
    }
    for (Req* q : ready) {
        if (q->status != MEG_OK || !std::isfinite(q->f1)) {
            if (q->status == MEG_OK) q->status = MEG_ERR_NUMERIC;
            retire(q);
            continue;
        }
        q->f = q->f1;
        q->cls = class_of(q->rq);
        classes[q->cls].joining.push_back(q);     // enters the group at the next tick boundary
    }
}

void meg_server_s::launch_tick(Class& c) {
    if (!c.joining.empty()) {
        c.members.insert(c.members.end(), c.joining.begin(), c.joining.end());
        c.joining.clear();
        c.dirty = true;
    }
    if (c.dirty || !c.g) {
        if (c.g) { meg_group_destroy(c.g); c.g = nullptr; }
        if (c.gexec) { cudaGraphExecDestroy(c.gexec); c.gexec = nullptr; }
        ++c.gen;
        c.ticks_same = 0;
        c.dirty = false;
        if (c.members.empty()) return;
        std::vector<meg_handle> hs;
        for (Req* q : c.members) hs.push_back(q->h);
        if (meg_group_create(hs.data(), (int)hs.size(), c.stream, &c.g) != MEG_OK) {
            for (Req* q : c.members) { q->status = MEG_ERR_CUDA; q->finished = true; }
            return;
        }
        if ((int)c.members.size() > c.f_cap) {
            if (c.f_host) cudaFreeHost(c.f_host);
            c.f_cap = std::max<int>(64, 2 * (int)c.members.size());
            cudaMallocHost((void**)&c.f_host, sizeof(double) * c.f_cap);
        }
    }
    // every member runs the same number of iterations in this tick
    int len = c.check;
    for (Req* q : c.members) len = std::min(len, std::max(1, q->rq.max_iters - q->iters));
    c.tick_len = len;
    meg_status st = MEG_OK;
    if (c.gexec && c.gexec_gen == c.gen && c.gexec_len == len) {
        st = cudaGraphLaunch(c.gexec, c.stream) == cudaSuccess ? MEG_OK : MEG_ERR_CUDA;
        if (st == MEG_OK) ++graph_ticks;
    } else if (c.ticks_same >= 1) {                     // the group held for a tick: capture this one
        if (c.gexec) { cudaGraphExecDestroy(c.gexec); c.gexec = nullptr; }
        st = capture_tick(c, len);
        if (st == MEG_OK) ++graph_ticks;
    } else {
        st = meg_group_launch(c.g, len);
        if (st == MEG_OK) st = meg_internal::group_objective_enqueue(c.g, c.f_host);
    }
    ++c.ticks_same;
    ++ticks;
    if (st != MEG_OK) {
        for (Req* q : c.members) { q->status = st; q->finished = true; }
        return;
    }
    cudaEventRecord(c.ev, c.stream);
    c.inflight = true;
}

// Capture the tick's grouped iterations and objective pass (kernels and the
// copy of f to pinned host memory, no allocation) on the class's stream, then
// launch the graph.
meg_status meg_server_s::capture_tick(Class& c, int len) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MEG_ERR_CUDA;
    meg_status st = meg_group_launch(c.g, len);
    if (st == MEG_OK) st = meg_internal::group_objective_enqueue(c.g, c.f_host);
    const cudaError_t ce = cudaStreamEndCapture(c.stream, &graph);
    if (st != MEG_OK || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return st != MEG_OK ? st : MEG_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&c.gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        c.gexec = nullptr;
        return MEG_ERR_CUDA;
    }
    c.gexec_gen = c.gen;
    c.gexec_len = len;
    return cudaGraphLaunch(c.gexec, c.stream) == cudaSuccess ? MEG_OK : MEG_ERR_CUDA;
}

void meg_server_s::finish_tick(Class& c) {
    c.inflight = false;
    bool any = false;
    for (size_t i = 0; i < c.members.size(); ++i) {
        Req* q = c.members[i];
        const double f = c.f_host[i];
        q->iters += c.tick_len;
        q->f_prev = q->f;
        q->f = f;
        const meg_request& rq = q->rq;
        if (!std::isfinite(f)) {
            q->status = MEG_ERR_NUMERIC;
            q->finished = true;
        } else if (std::isfinite(rq.fstar)) {
            const double den = q->f1 - rq.fstar;
            if (!(den > 0.0) || f - rq.fstar <= rq.tol * den) q->finished = true;
        } else {
            // f* unknown: stop when the last interval's decrease is below tol of the total
            // decrease (at the first check the two are equal, so it never stops there)
            const double total = q->f1 - f;
            if (total > 0.0 && q->f_prev - f <= rq.tol * total) q->finished = true;
        }
        if (!q->finished && q->iters >= rq.max_iters) {
            q->status = MEG_ERR_NOT_CONVERGED;
            q->finished = true;
        }
        any |= q->finished;
    }
    if (!any) return;
    // members leave the group before they are released
    if (c.g) { meg_group_destroy(c.g); c.g = nullptr; }
    std::vector<Req*> keep;
    for (Req* q : c.members) {
        if (q->finished) retire(q);
        else keep.push_back(q);
    }
    c.members.swap(keep);
    c.dirty = true;
}

void meg_server_s::retire(Req* q) {
    if (q->h) {
        if (q->status == MEG_OK || q->status == MEG_ERR_NOT_CONVERGED) {
            meg_status st = meg_internal::solve_status(q->h);
            if (st == MEG_OK) st = meg_get_iterate(q->h, q->rq.out_V, q->rq.out_mu, q->rq.out_s);
            if (st != MEG_OK) q->status = st;
        }
        meg_destroy(q->h);
        q->h = nullptr;
    }
    if (q->d_data) cudaFreeAsync(q->d_data, q->stream);
    if (q->d_y) cudaFreeAsync(q->d_y, q->stream);
    if (q->stream) cudaStreamDestroy(q->stream);
    meg_result r{};
    r.id = q->id;
    r.status = q->status;
    r.iters = q->iters;
    r.f1 = q->f1;
    r.f = q->f;
    r.t_submit = q->t_submit;
    r.t_admit = q->t_admit;
    r.t_done = now();
    used -= q->footprint;
    active -= 1;
    {
        std::lock_guard<std::mutex> lk(mu);
        done.push_back(r);
        finished += 1;
    }
    cv_done.notify_all();
    delete q;
}

void meg_server_s::run() {
    cudaSetDevice(device);
    cudaStreamCreateWithFlags(&admit_stream, cudaStreamNonBlocking);
    while (!stop.load()) {
        // admission, FIFO
        std::vector<Req*> take;
        {
            std::lock_guard<std::mutex> lk(mu);
            while (!pending.empty() && active + (int)take.size() < opt.max_active) {
                Req* q = pending.front();
                int64_t need = used;
                for (Req* t : take) need += t->footprint;
                if (need + q->footprint > opt.hbm_budget) break;
                pending.pop_front();
                take.push_back(q);
            }
        }
        std::vector<Req*> ready;
        for (Req* q : take) {
            used += q->footprint;
            active += 1;
            if (admit(q)) ready.push_back(q);
        }
        if (!ready.empty()) admit_batch(ready);
        bool busy = false;
        for (Class& c : classes) {
            if (c.inflight) {
                const cudaError_t e = cudaEventQuery(c.ev);
                if (e == cudaSuccess) finish_tick(c);
                else if (e != cudaErrorNotReady) {
                    cudaGetLastError();
                    c.inflight = false;
                    if (c.g) { meg_group_destroy(c.g); c.g = nullptr; }
                    for (Req* q : c.members) { q->status = MEG_ERR_CUDA; retire(q); }
                    c.members.clear();
                }
            }
            if (!c.inflight && (!c.members.empty() || !c.joining.empty())) launch_tick(c);
            // members flagged during launch (group or launch failure) leave now
            if (!c.inflight && !c.members.empty()) {
                if (c.g) { meg_group_destroy(c.g); c.g = nullptr; }
                for (Req* q : c.members) retire(q);
                c.members.clear();
            }
            busy |= c.inflight;
        }
        std::unique_lock<std::mutex> lk(mu);
        if (!busy && pending.empty()) {
            cv_work.wait_for(lk, std::chrono::milliseconds(2));
        } else if (!busy || take.empty()) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        }
    }
    for (Class& c : classes) {
        if (c.inflight) cudaEventSynchronize(c.ev);
        if (c.g) meg_group_destroy(c.g);
        c.members.insert(c.members.end(), c.joining.begin(), c.joining.end());
        c.joining.clear();
        for (Req* q : c.members) {
            if (q->h) meg_destroy(q->h);
            if (q->d_data) cudaFreeAsync(q->d_data, q->stream);
            if (q->d_y) cudaFreeAsync(q->d_y, q->stream);
            if (q->stream) cudaStreamDestroy(q->stream);
            delete q;
        }
        if (c.f_host) cudaFreeHost(c.f_host);
        if (c.gexec) cudaGraphExecDestroy(c.gexec);
        if (c.ev) cudaEventDestroy(c.ev);
        if (c.stream) cudaStreamDestroy(c.stream);
    }
    classes.clear();
    if (admit_stream) cudaStreamDestroy(admit_stream);
}

extern "C" {

meg_status meg_server_create(const meg_server_options* opt, meg_server* out) {
    if (!opt || !out) return sfail(MEG_ERR_INVALID_ARG, "meg_server_create: null argument");
    *out = nullptr;
    if (opt->hbm_budget <= 0 || opt->max_active < 1 || opt->check_every < 1 || opt->meas_check_every < 1)
        return sfail(MEG_ERR_INVALID_ARG, "meg_server_create: budget, max_active and check intervals must be positive");
    meg_server_s* s = new meg_server_s();
    s->opt = *opt;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return sfail(MEG_ERR_CUDA, "meg_server_create: cudaGetDevice");
    }
    // keep freed pool memory for the next request instead of returning it
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
        uint64_t keep = (uint64_t)opt->hbm_budget;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    s->t0 = std::chrono::steady_clock::now();
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return MEG_OK;
}

meg_status meg_server_submit(meg_server s, const meg_request* rq, uint64_t* id) {
    if (!s || !rq) return sfail(MEG_ERR_INVALID_ARG, "meg_server_submit: null argument");
    const int n = rq->opt.n, r = rq->opt.r;
    if (rq->kind != MEG_DENSE_QUAD && rq->kind != MEG_LINEAR && rq->kind != MEG_MEAS_STOCH)
        return sfail(MEG_ERR_INVALID_ARG, "meg_server_submit: kind must be DENSE_QUAD, LINEAR or MEAS_STOCH");
    if (!rq->data || (rq->kind == MEG_MEAS_STOCH && (!rq->y || rq->m < 1 || rq->L < 1)))
        return sfail(MEG_ERR_INVALID_ARG, "meg_server_submit: objective data missing");
    if (rq->warm_start_products <= 0 && (!rq->V0 || !rq->lam0))
        return sfail(MEG_ERR_INVALID_ARG, "meg_server_submit: give V0 and lam0 or warm_start_products > 0");
    if (!(rq->tol > 0.0) || rq->max_iters < 1)
        return sfail(MEG_ERR_INVALID_ARG, "meg_server_submit: tol > 0 and max_iters >= 1 required");
    const int64_t fp = meg_footprint(n, r, rq->opt.p, rq->opt.precision, rq->kind);
    if (fp < 0) return sfail(MEG_ERR_INVALID_ARG, "meg_server_submit: sizes");
    // the objective data copied in, and for measurements the per-measurement scratch
    // (residual, ||a||^2, a^T W) that meg_footprint cannot size without m, and the
    // partials of the tensor-core minibatch pass and its split operand image (float storage)
    const int64_t mtp = rq->kind == MEG_MEAS_STOCH && rq->opt.precision != MEG_FP64
                            ? 4 * (int64_t)(2 * k_bucket(r + rq->opt.p) + 1) *
                                      std::max((int64_t)meas_ks(rq->L, n) * rq->L, (int64_t)meas_ks((int)rq->m, n) * rq->m) +
                                  (int64_t)mts_image_bytes(std::max<int64_t>(rq->L, rq->m), r + rq->opt.p) + 16 +
                                  (int64_t)((n + MT_BK - 1) / MT_BK) * 3 * 2 * k_bucket(r + rq->opt.p) * MT_BK * 2
                            : 0;
    int64_t data = rq->kind == MEG_MEAS_STOCH
                       ? rq->m * (int64_t)n * (int64_t)elem_bytes(rq->opt.precision) + 8 * rq->m +
                             8 * (rq->m * 34 + rq->m / 8 + 1) + 4 * (int64_t)rq->L + mtp
                       : (int64_t)n * n * (int64_t)elem_bytes(rq->opt.precision);
    Req* q = new Req();
    q->rq = *rq;
    q->footprint = fp + data;
    if (q->footprint > s->opt.hbm_budget) {
        delete q;
        return sfail(MEG_ERR_OOM, "meg_server_submit: request larger than the whole memory budget");
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        q->id = s->next_id++;
        q->t_submit = s->now();
        s->pending.push_back(q);
        s->submitted += 1;
        if (id) *id = q->id;
    }
    s->cv_work.notify_one();
    return MEG_OK;
}

meg_status meg_server_poll(meg_server s, meg_result* out, int max_out, int* n_out, int timeout_ms) {
    if (!s || !n_out || (max_out > 0 && !out)) return sfail(MEG_ERR_INVALID_ARG, "meg_server_poll: arguments");
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && timeout_ms > 0)
        s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [s] { return !s->done.empty(); });
    const int cnt = std::min<int>(max_out, (int)s->done.size());
    for (int i = 0; i < cnt; ++i) out[i] = s->done[i];
    s->done.erase(s->done.begin(), s->done.begin() + cnt);
    *n_out = cnt;
    return MEG_OK;
}

meg_status meg_server_counts(meg_server s, int64_t* submitted, int64_t* finished) {
    if (!s) return sfail(MEG_ERR_INVALID_ARG, "meg_server_counts: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (submitted) *submitted = s->submitted;
    if (finished) *finished = s->finished;
    return MEG_OK;
}

meg_status meg_server_tick_counts(meg_server s, int64_t* ticks, int64_t* graph_ticks) {
    if (!s) return sfail(MEG_ERR_INVALID_ARG, "meg_server_tick_counts: null server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (ticks) *ticks = s->ticks.load();
    if (graph_ticks) *graph_ticks = s->graph_ticks.load();
    return MEG_OK;
}

double meg_server_now(meg_server s) { return s ? s->now() : -1.0; }

meg_status meg_server_destroy(meg_server s) {
    if (!s) return MEG_OK;
    s->stop.store(true);
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (Req* q : s->pending) delete q;
    delete s;
    return MEG_OK;
}

}  // extern "C"
