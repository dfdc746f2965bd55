// server.cu -- a request loop for NNFFT and fast sinc transform requests of mixed sizes
// and tolerances on one GPU (continuous batching).
//
// Requests arrive from any host thread (nnfft_server_submit) and queue in FIFO order.  One
// worker thread owns S slots, each a CUDA stream with device buffers for one request's
// inputs and outputs.  Whenever a slot is free and the plans the head request needs are
// available within the device-memory budget, the request is admitted: its inputs go up,
// its transform(s) run and its output comes back on that slot's stream, so requests in
// different slots overlap on the device while new ones keep being admitted as slots free
// up.  Completion is detected from a CUDA event per slot; the latency of a request runs
// from submit to that detection.
//
// Plans stay resident between requests (window fits, tables, sort buffers) in a cache
// keyed by (bandwidth bucket, dtype, m): a plan made for bandwidth N' and capacities
// (M1', M2') serves any request with N <= N', M1 <= M1', M2 <= M2' through
// nnfft_set_bandwidth / nnfft_set_sizes, with the results of a plan made for the exact
// sizes.  Plans are made with the server's full capacity (max_points) on their data
// sides, so one plan per bucket serves every request size.  A sinc request (Algorithm 6.1) takes two such plans (nodes a -> quadrature
// nodes, quadrature nodes -> b) and the quadrature rule of its bandwidth bucket.  Idle
// plans are evicted least recently used first when a new plan would exceed the budget.
//
// Tolerance -> arithmetic: tol >= 1e-6 runs the fp32 path, smaller tolerances the fp64
// path; m is the smallest with (24 m^{3/2} + 10) exp(-2 pi m sqrt(1 - 1/sigma)) <= tol
// (the first term of Theorem 4.1 at sigma = 2), at least 2 and at most 12.
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
#include <thread>
#include <tuple>
#include <vector>

#include "hostmath.h"
#include "internal.h"
#include "nnfft.h"

using namespace nnfft;

namespace {

using Clock = std::chrono::steady_clock;

int64_t pow2_at_least(int64_t x, int64_t lo) {
    int64_t c = lo;
    while (c < x) c *= 2;
    return c;
}

struct PlanEntry {
    nnfft_plan_t p = nullptr;
    int64_t Ncap = 0, cap1 = 0, cap2 = 0;
    int dtype = 0, m = 0;
    size_t bytes = 0;          // device bytes (the admission estimate while building)
    bool busy = false;
    bool ready = false;        // false while the builder thread makes the plan
    uint64_t last = 0;
};

struct BuildDone {             // a plan the builder thread finished (or failed to make)
    PlanEntry *e;
    nnfft_plan_t p;
    int rc;
};

struct Rule {                       // quadrature rule of a sinc bandwidth bucket (device)
    double *x1 = nullptr, *v2 = nullptr, *w = nullptr;   // nodes of NNFFT #1 / #2, weights
    int64_t nq = 0;
};

struct Req {
    nnfft_request r{};
    int64_t id = 0;
    int dtype = 0, m = 0;
    int64_t Ncap = 0;
    Clock::time_point t_submit, t_done;
    double dev_ms[4] = {-1, -1, -1, -1};   // device times since the epoch: first upload,
                                           // first kernel, after the last kernel, download end
    int status = NNFFT_OK;
    bool done = false;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    cudaEvent_t ev_t[4] = {};   // timing: before the uploads, before the first kernel, after
                                // the last kernel, after the download
    double *d1 = nullptr, *d2 = nullptr;   // nodes (v or a / x or b)
    void *c1 = nullptr, *c2 = nullptr;     // values (f or c / y or h), complex128-sized
    void *g = nullptr;                     // sinc: the quadrature-node values
    Req *req = nullptr;
    PlanEntry *pa = nullptr, *pb = nullptr;
};

int sfail(int code, const char *msg) { return report_error(code, msg); }

}  // namespace

struct nnfft_server_s {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req *> pending;
    std::map<int64_t, Req *> reqs;
    std::vector<Slot> slots;
    std::vector<PlanEntry *> plans;
    std::map<std::tuple<int64_t, int, int>, Rule> rules;   // (Ncap, rule, dtype)
    std::thread worker, builder;
    bool stop = false;
    // plan builds run on the builder thread so that admission never waits for one
    std::mutex mu_build;
    std::condition_variable cv_build;
    std::deque<PlanEntry *> build_jobs;
    std::vector<BuildDone> built;
    bool stop_build = false;
    int builds_in_flight = 0;                 // worker only
    std::map<std::tuple<int64_t, int, int>, int> build_error;   // (Ncap, dtype, m) -> status
    int64_t next_id = 1;
    uint64_t tick = 0;
    int64_t budget = 0, max_points = 0;
    std::atomic<size_t> fixed_bytes{0};   // slot buffers and rules (worker writes)
    std::atomic<size_t> plan_bytes{0};    // cached plans (worker writes)
    std::atomic<int64_t> plans_cached{0}, plans_made{0}, plans_evicted{0};
    // statistics
    std::vector<double> lat_ms;
    double points = 0;
    int64_t completed = 0, failed = 0;
    Clock::time_point t_first{}, t_last{};
    bool any = false;
    int device = 0;
    cudaEvent_t epoch = nullptr;          // device time origin of the kernel intervals
};

namespace {

double window_term(int m) {
    return (24.0 * std::pow((double)m, 1.5) + 10.0) * std::exp(-2.0 * M_PI * m * std::sqrt(0.5));
}

void tolerance_class(double tol, int *dtype, int *m) {
    *dtype = tol >= 1e-6 ? NNFFT_C64 : NNFFT_C128;
    int mm = 2;
    while (mm < 12 && window_term(mm) > tol) ++mm;
    *m = mm;
}

// An idle plan's last work has completed (its slot's event was seen): detach it from the
// slot stream it last ran on (which may be destroyed before the plan) and free it.
void destroy_idle_plan(nnfft_plan_t p) {
    nnfft_set_stream(p, nullptr);
    nnfft_destroy(p);
}

// An idle cached plan for (Ncap, dtype, m) with capacities >= (M1, M2).  Without one, a
// build of a new plan with capacities (c1, c2) is queued for the builder thread (one at a
// time per key; idle plans are evicted least recently used first to fit the budget) and
// nullptr is returned with *err == OK: not now.  *err != OK: the request fails.
PlanEntry *acquire_plan(nnfft_server_s *S, int64_t Ncap, int dtype, int m, int64_t M1,
                        int64_t M2, int64_t c1, int64_t c2, int *err) {
    *err = NNFFT_OK;
    PlanEntry *best = nullptr;
    bool building = false;
    for (PlanEntry *e : S->plans) {
        if (e->Ncap != Ncap || e->dtype != dtype || e->m != m) continue;
        if (!e->ready) {
            building = building || (e->cap1 >= M1 && e->cap2 >= M2);
            continue;
        }
        if (!e->busy && e->cap1 >= M1 && e->cap2 >= M2 &&
            (!best || e->cap1 + e->cap2 < best->cap1 + best->cap2))
            best = e;
    }
    if (best) {
        best->busy = true;
        best->last = ++S->tick;
        return best;
    }
    if (building) return nullptr;               // one build per key at a time
    auto berr = S->build_error.find(std::make_tuple(Ncap, dtype, m));
    if (berr != S->build_error.end()) {
        *err = berr->second;
        return nullptr;
    }
    // rough size for admission: sort and coordinate buffers, moments, cells, grids
    const size_t est = (size_t)(c1 + c2) * 64 + (size_t)Ncap * 2048 + (64u << 20);
    auto over = [&](size_t extra) {
        return (int64_t)(S->fixed_bytes + S->plan_bytes + extra) > S->budget;
    };
    while (over(est)) {
        PlanEntry *victim = nullptr;
        for (PlanEntry *e : S->plans)
            if (e->ready && !e->busy && (!victim || e->last < victim->last)) victim = e;
        if (!victim) {
            bool any_busy = S->builds_in_flight > 0;
            for (PlanEntry *e : S->plans) any_busy = any_busy || e->busy;
            if (!any_busy) {                    // nothing will ever free up: cannot serve
                *err = sfail(NNFFT_ENOMEM, "request does not fit the server's device budget");
                return nullptr;
            }
            return nullptr;                     // everything in use: wait
        }
        S->plan_bytes -= victim->bytes;
        destroy_idle_plan(victim->p);
        S->plans.erase(std::find(S->plans.begin(), S->plans.end(), victim));
        delete victim;
        ++S->plans_evicted;
        --S->plans_cached;
    }
    PlanEntry *e = new PlanEntry();
    e->Ncap = Ncap;
    e->cap1 = c1;
    e->cap2 = c2;
    e->dtype = dtype;
    e->m = m;
    e->bytes = est;                             // reserved until the plan exists
    e->busy = true;
    e->ready = false;
    e->last = ++S->tick;
    S->plan_bytes += est;
    S->plans.push_back(e);
    ++S->builds_in_flight;
    {
        std::lock_guard<std::mutex> g(S->mu_build);
        S->build_jobs.push_back(e);
    }
    S->cv_build.notify_one();
    return nullptr;
}

// Take in the plans the builder thread finished (worker thread).
void integrate_builds(nnfft_server_s *S) {
    std::vector<BuildDone> done;
    {
        std::lock_guard<std::mutex> g(S->mu_build);
        done.swap(S->built);
    }
    for (BuildDone &d : done) {
        PlanEntry *e = d.e;
        --S->builds_in_flight;
        S->plan_bytes -= e->bytes;
        if (d.rc) {
            S->build_error[std::make_tuple(e->Ncap, e->dtype, e->m)] = d.rc;
            S->plans.erase(std::find(S->plans.begin(), S->plans.end(), e));
            delete e;
            continue;
        }
        e->p = d.p;
        e->bytes = plan_bytes(d.p);
        S->plan_bytes += e->bytes;
        e->ready = true;
        e->busy = false;
        ++S->plans_made;
        ++S->plans_cached;
    }
}

void builder_loop(nnfft_server_s *S) {
    cudaSetDevice(S->device);
    for (;;) {
        PlanEntry *e = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu_build);
            S->cv_build.wait(lk, [&] { return S->stop_build || !S->build_jobs.empty(); });
            if (S->build_jobs.empty()) return;
            e = S->build_jobs.front();
            S->build_jobs.pop_front();
        }
        nnfft_plan_t p = nullptr;
        const int rc = nnfft_plan(&p, e->Ncap, e->cap1, e->cap2, 2.0, 2.0, e->m, e->m,
                                  (nnfft_dtype)e->dtype, nullptr);
        std::lock_guard<std::mutex> g(S->mu_build);
        S->built.push_back(BuildDone{e, rc ? nullptr : p, rc});
    }
}

void release_plan(PlanEntry *&e) {
    if (e) e->busy = false;
    e = nullptr;
}

// Quadrature rule of the sinc bandwidth bucket (GL: 2 Ncap nodes; CC: 4 Ncap intervals).
int get_rule(nnfft_server_s *S, int64_t Ncap, int rule, Rule **out) {
    auto key = std::make_tuple(Ncap, rule, 0);
    auto it = S->rules.find(key);
    if (it != S->rules.end()) {
        *out = &it->second;
        return NNFFT_OK;
    }
    int64_t nq = 0;
    int rc = sinc_quadrature(rule, Ncap, 0, nullptr, nullptr, &nq);
    if (rc) return rc;
    std::vector<double> t((size_t)nq), w((size_t)nq), x1((size_t)nq), v2((size_t)nq);
    if ((rc = sinc_quadrature(rule, Ncap, 0, t.data(), w.data(), &nq))) return rc;
    for (int64_t j = 0; j < nq; ++j) {         // the sign conventions of sinc_exec_rule
        x1[(size_t)j] = rule == SINC_RULE_CC ? t[(size_t)j] : -t[(size_t)j];
        v2[(size_t)j] = rule == SINC_RULE_CC ? -t[(size_t)j] : t[(size_t)j];
    }
    Rule R;
    R.nq = nq;
    cudaError_t e = cudaMalloc(&R.x1, sizeof(double) * 3 * (size_t)nq);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return sfail(NNFFT_ENOMEM, "server: quadrature rule");
    }
    R.v2 = R.x1 + nq;
    R.w = R.v2 + nq;
    cudaMemcpy(R.x1, x1.data(), sizeof(double) * nq, cudaMemcpyHostToDevice);
    cudaMemcpy(R.v2, v2.data(), sizeof(double) * nq, cudaMemcpyHostToDevice);
    cudaMemcpy(R.w, w.data(), sizeof(double) * nq, cudaMemcpyHostToDevice);
    S->fixed_bytes += sizeof(double) * 3 * (size_t)nq;
    *out = &(S->rules[key] = R);
    return NNFFT_OK;
}

#define SV_CUDA(call)                                   \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) {                        \
            cudaGetLastError();                         \
            return sfail(NNFFT_ECUDA, "server: CUDA call failed"); \
        }                                               \
    } while (0)

// Queue one NNFFT request on a slot (plans acquired by the caller).
int launch_nnfft(Slot &sl, Req *q) {
    const nnfft_request &r = q->r;
    const size_t cs = q->dtype == NNFFT_C128 ? 16 : 8;
    nnfft_plan_t p = sl.pa->p;
    int rc;
    if ((rc = nnfft_set_stream(p, sl.st)) || (rc = nnfft_set_sizes(p, r.M1, r.M2)) ||
        (rc = nnfft_set_bandwidth(p, r.N)))
        return rc;
    SV_CUDA(cudaEventRecord(sl.ev_t[0], sl.st));
    if (r.M1) SV_CUDA(cudaMemcpyAsync(sl.d1, r.v, 8 * (size_t)r.M1, cudaMemcpyHostToDevice, sl.st));
    if (r.M2) SV_CUDA(cudaMemcpyAsync(sl.d2, r.x, 8 * (size_t)r.M2, cudaMemcpyHostToDevice, sl.st));
    if (r.M1) SV_CUDA(cudaMemcpyAsync(sl.c1, r.f, cs * (size_t)r.M1, cudaMemcpyHostToDevice, sl.st));
    SV_CUDA(cudaEventRecord(sl.ev_t[1], sl.st));
    if ((rc = nnfft_set_nodes(p, sl.d1, sl.d2)) || (rc = nnfft_exec(p, sl.c1, sl.c2))) return rc;
    SV_CUDA(cudaEventRecord(sl.ev_t[2], sl.st));
    if (r.M2) SV_CUDA(cudaMemcpyAsync(r.y, sl.c2, cs * (size_t)r.M2, cudaMemcpyDeviceToHost, sl.st));
    SV_CUDA(cudaEventRecord(sl.ev_t[3], sl.st));
    return NNFFT_OK;
}

// Queue one fast sinc transform request (Algorithm 6.1) on a slot.
int launch_sinc(nnfft_server_s *S, Slot &sl, Req *q, Rule *R) {
    const nnfft_request &r = q->r;      // M1 = L1 (a, c), M2 = L2 (b, h)
    const bool dbl = q->dtype == NNFFT_C128;
    const size_t rs = dbl ? 8 : 4, cs = 2 * rs;
    const size_t vs = r.is_complex ? cs : rs;
    (void)S;
    int rc;
    nnfft_plan_t p1 = sl.pa->p, p2 = sl.pb->p;
    if ((rc = nnfft_set_stream(p1, sl.st)) || (rc = nnfft_set_sizes(p1, r.M1, R->nq)) ||
        (rc = nnfft_set_bandwidth(p1, r.N)) || (rc = nnfft_set_stream(p2, sl.st)) ||
        (rc = nnfft_set_sizes(p2, R->nq, r.M2)) || (rc = nnfft_set_bandwidth(p2, r.N)))
        return rc;
    SV_CUDA(cudaEventRecord(sl.ev_t[0], sl.st));
    if (r.M1) SV_CUDA(cudaMemcpyAsync(sl.d1, r.v, 8 * (size_t)r.M1, cudaMemcpyHostToDevice, sl.st));
    if (r.M2) SV_CUDA(cudaMemcpyAsync(sl.d2, r.x, 8 * (size_t)r.M2, cudaMemcpyHostToDevice, sl.st));
    if (r.M1) SV_CUDA(cudaMemcpyAsync(sl.c2, r.f, vs * (size_t)r.M1, cudaMemcpyHostToDevice, sl.st));
    SV_CUDA(cudaEventRecord(sl.ev_t[1], sl.st));
    const void *cin = sl.c2;
    if (!r.is_complex) {
        SV_CUDA(dbl ? launch_real_to_complex<double>(static_cast<const double *>(sl.c2), (int)r.M1, sl.c1, sl.st)
                    : launch_real_to_complex<float>(static_cast<const float *>(sl.c2), (int)r.M1, sl.c1, sl.st));
        cin = sl.c1;
    }
    if ((rc = nnfft_set_nodes(p1, sl.d1, R->x1)) || (rc = nnfft_exec(p1, cin, sl.g))) return rc;
    SV_CUDA(dbl ? launch_scale_by_weights<double>(sl.g, R->w, (int)R->nq, sl.st)
                : launch_scale_by_weights<float>(sl.g, R->w, (int)R->nq, sl.st));
    if ((rc = nnfft_set_nodes(p2, R->v2, sl.d2)) || (rc = nnfft_exec(p2, sl.g, sl.c1))) return rc;
    if (!r.is_complex) {
        SV_CUDA(dbl ? launch_complex_to_real<double>(sl.c1, (int)r.M2, static_cast<double *>(sl.c2), sl.st)
                    : launch_complex_to_real<float>(sl.c1, (int)r.M2, static_cast<float *>(sl.c2), sl.st));
        SV_CUDA(cudaEventRecord(sl.ev_t[2], sl.st));
        if (r.M2) SV_CUDA(cudaMemcpyAsync(r.y, sl.c2, rs * (size_t)r.M2, cudaMemcpyDeviceToHost, sl.st));
    } else {
        SV_CUDA(cudaEventRecord(sl.ev_t[2], sl.st));
        if (r.M2) SV_CUDA(cudaMemcpyAsync(r.y, sl.c1, cs * (size_t)r.M2, cudaMemcpyDeviceToHost, sl.st));
    }
    SV_CUDA(cudaEventRecord(sl.ev_t[3], sl.st));
    return NNFFT_OK;
}

// The slot's request is over (its event has completed, or it failed to start): collect
// device-side status, release the plans and the slot.  No lock: slots and plans belong to
// the worker thread.  Returns the request and its status.
Req *retire(Slot &sl, int &status, cudaEvent_t epoch) {
    Req *q = sl.req;
    if (status == NNFFT_OK && sl.pa) status = nnfft_sync(sl.pa->p);
    if (status == NNFFT_OK && sl.pb) status = nnfft_sync(sl.pb->p);
    for (int k = 0; k < 4 && status == NNFFT_OK && epoch; ++k) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, epoch, sl.ev_t[k]) == cudaSuccess) q->dev_ms[k] = t;
    }
    cudaGetLastError();
    release_plan(sl.pa);
    release_plan(sl.pb);
    sl.req = nullptr;
    return q;
}

// Publish a finished request (caller holds the lock).
void record_done(nnfft_server_s *S, Req *q, int status) {
    q->status = status;
    q->t_done = Clock::now();
    q->done = true;
    if (status == NNFFT_OK) {
        ++S->completed;
        S->lat_ms.push_back(std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count());
        S->points += (double)(q->r.M1 + q->r.M2);
    } else {
        ++S->failed;
    }
    S->t_last = q->t_done;
}

enum Admit { ADMITTED, WAIT, FAILED };

// Try to start request q on the free slot sl (no lock held).  WAIT: plans or memory will
// free up when other slots finish; FAILED: *status says why.
Admit admit(nnfft_server_s *S, Slot &sl, Req *q, int *status) {
    int err = NNFFT_OK;
    Rule *R = nullptr;
    if (q->r.kind == NNFFT_REQ_SINC) {
        if ((err = get_rule(S, q->Ncap, q->r.rule, &R)) == NNFFT_OK) {
            // data sides get the server's full capacity, the quadrature side its rule size
            const int64_t cq = pow2_at_least(R->nq, 64);
            sl.pa = acquire_plan(S, q->Ncap, q->dtype, q->m, q->r.M1, R->nq, S->max_points, cq, &err);
            if (sl.pa)
                sl.pb = acquire_plan(S, q->Ncap, q->dtype, q->m, R->nq, q->r.M2, cq, S->max_points, &err);
            if (sl.pa && !sl.pb) release_plan(sl.pa);
        }
    } else {
        sl.pa = acquire_plan(S, q->Ncap, q->dtype, q->m, q->r.M1, q->r.M2, S->max_points,
                             S->max_points, &err);
    }
    if (err == NNFFT_OK && !sl.pa) {
        // waiting helps only if a plan is being built or another slot will release
        // plans or memory
        if (S->builds_in_flight > 0) return WAIT;
        for (const Slot &o : S->slots)
            if (&o != &sl && o.req) return WAIT;
        err = sfail(NNFFT_ENOMEM, "request does not fit the server's device budget");
    }
    sl.req = q;
    int rc = err;
    if (rc == NNFFT_OK)
        rc = q->r.kind == NNFFT_REQ_SINC ? launch_sinc(S, sl, q, R) : launch_nnfft(sl, q);
    if (rc == NNFFT_OK && cudaEventRecord(sl.ev, sl.st) != cudaSuccess) {
        cudaGetLastError();
        rc = NNFFT_ECUDA;
    }
    if (rc == NNFFT_OK) return ADMITTED;
    if (sl.pa) cudaStreamSynchronize(sl.st);
    retire(sl, rc, nullptr);
    *status = rc;
    return FAILED;
}

// Requests the worker looks at past a waiting one (whose plan is being built).
constexpr size_t LOOKAHEAD = 64;

void worker_loop(nnfft_server_s *S) {
    cudaSetDevice(S->device);
    for (;;) {
        integrate_builds(S);
        bool busy = S->builds_in_flight > 0;
        for (Slot &sl : S->slots) {                 // retire finished requests
            if (!sl.req) continue;
            const cudaError_t e = cudaEventQuery(sl.ev);
            if (e == cudaErrorNotReady) {
                busy = true;
                continue;
            }
            if (e != cudaSuccess) cudaGetLastError();
            int st = e == cudaSuccess ? NNFFT_OK : NNFFT_ECUDA;
            Req *q = retire(sl, st, S->epoch);
            {
                std::lock_guard<std::mutex> g(S->mu);
                record_done(S, q, st);
            }
            S->cv_done.notify_all();
        }
        // admit in arrival order; a request whose plan is not ready yet keeps its place
        // while later ones (up to LOOKAHEAD) may start
        for (Slot &sl : S->slots) {
            if (sl.req) {
                busy = true;
                continue;
            }
            size_t i = 0;
            while (!sl.req) {
                Req *q = nullptr;
                {
                    std::lock_guard<std::mutex> g(S->mu);
                    if (i >= S->pending.size() || i >= LOOKAHEAD) break;
                    q = S->pending[i];
                }
                int st = NNFFT_OK;
                const Admit a = admit(S, sl, q, &st);
                if (a == WAIT) {
                    ++i;
                    continue;
                }
                {
                    std::lock_guard<std::mutex> g(S->mu);
                    S->pending.erase(S->pending.begin() + (std::ptrdiff_t)i);
                    if (a == FAILED) record_done(S, q, st);
                }
                if (a == FAILED) S->cv_done.notify_all();
                else busy = true;
            }
        }
        std::unique_lock<std::mutex> lk(S->mu);
        if (busy || !S->pending.empty()) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            continue;
        }
        if (S->stop) break;
        S->cv_work.wait(lk);
    }
}

}  // namespace

extern "C" {

int nnfft_tolerance_params(double tol, int *dtype, int *m) {
    if (!(tol > 0) || !dtype || !m) return sfail(NNFFT_EINVAL, "tolerance must be > 0");
    tolerance_class(tol, dtype, m);
    return NNFFT_OK;
}

int nnfft_server_create(nnfft_server_t *out, int64_t mem_budget_bytes, int nslots,
                        int64_t max_points) {
    if (!out) return sfail(NNFFT_EINVAL, "null server pointer");
    *out = nullptr;
    if (nslots < 1 || nslots > 64 || max_points < 1 || mem_budget_bytes <= 0)
        return sfail(NNFFT_EINVAL, "invalid server parameters");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return sfail(NNFFT_ECUDA, "no CUDA device");
    }
    nnfft_server_s *S = new nnfft_server_s();
    cudaGetDevice(&S->device);
    S->budget = mem_budget_bytes;
    S->max_points = max_points;
    S->slots.resize((size_t)nslots);
    const size_t mp = (size_t)max_points;
    for (Slot &sl : S->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        for (int k = 0; k < 4 && e == cudaSuccess; ++k) e = cudaEventCreate(&sl.ev_t[k]);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d1, 8 * mp);
        if (e == cudaSuccess) e = cudaMalloc(&sl.d2, 8 * mp);
        if (e == cudaSuccess) e = cudaMalloc(&sl.c1, 16 * mp);
        if (e == cudaSuccess) e = cudaMalloc(&sl.c2, 16 * mp);
        if (e == cudaSuccess) e = cudaMalloc(&sl.g, 16 * (8 * 16384 + 1));
        if (e != cudaSuccess) {
            cudaGetLastError();
            nnfft_server_destroy(S);
            return sfail(NNFFT_ENOMEM, "server: slot buffers");
        }
        S->fixed_bytes += 48 * mp + 16 * (8 * 16384 + 1);
    }
    if (cudaEventCreate(&S->epoch) != cudaSuccess || cudaEventRecord(S->epoch, nullptr) != cudaSuccess ||
        cudaEventSynchronize(S->epoch) != cudaSuccess) {
        cudaGetLastError();
        nnfft_server_destroy(S);
        return sfail(NNFFT_ECUDA, "server: timing event");
    }
    S->builder = std::thread(builder_loop, S);
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return NNFFT_OK;
}

int nnfft_server_submit(nnfft_server_t S, const nnfft_request *r, int64_t *id) {
    if (!S || !r) return sfail(NNFFT_EINVAL, "null argument");
    if (r->kind != NNFFT_REQ_NNFFT && r->kind != NNFFT_REQ_SINC)
        return sfail(NNFFT_EINVAL, "unknown request kind");
    if (r->N < 1 || r->N > 65536 || r->M1 < 0 || r->M2 < 0 || r->M1 > S->max_points ||
        r->M2 > S->max_points)
        return sfail(NNFFT_EINVAL, "request sizes outside the server's limits");
    if ((r->M1 > 0 && (!r->v || !r->f)) || (r->M2 > 0 && (!r->x || !r->y)))
        return sfail(NNFFT_EINVAL, "null data pointer");
    if (r->kind == NNFFT_REQ_SINC && r->rule != SINC_RULE_GL && r->rule != SINC_RULE_CC)
        return sfail(NNFFT_EINVAL, "unknown quadrature rule");
    const Clock::time_point t0 = Clock::now();
    Req *q = new Req();
    q->r = *r;
    if (!(r->tol > 0)) {
        delete q;
        return sfail(NNFFT_EINVAL, "tolerance must be > 0");
    }
    tolerance_class(r->tol, &q->dtype, &q->m);
    q->Ncap = pow2_at_least(r->N, 64);
    if (r->kind == NNFFT_REQ_SINC && q->Ncap > 16384) {
        delete q;
        return sfail(NNFFT_EINVAL, "sinc requests need N <= 16384");
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        q->id = S->next_id++;
        q->t_submit = t0;
        if (!S->any) {
            S->t_first = q->t_submit;
            S->any = true;
        }
        S->reqs[q->id] = q;
        S->pending.push_back(q);
    }
    S->cv_work.notify_one();
    if (id) *id = q->id;
    return NNFFT_OK;
}

int nnfft_server_wait(nnfft_server_t S, int64_t id, double *latency_ms) {
    return nnfft_server_wait_device(S, id, latency_ms, nullptr);
}

int nnfft_server_wait_device(nnfft_server_t S, int64_t id, double *latency_ms, double *device_ms) {
    if (!S) return sfail(NNFFT_EINVAL, "null server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return sfail(NNFFT_EINVAL, "unknown request id");
    Req *q = it->second;
    S->cv_done.wait(lk, [&] { return q->done; });
    const int st = q->status;
    if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count();
    if (device_ms)
        for (int k = 0; k < 4; ++k) device_ms[k] = q->dev_ms[k];
    S->reqs.erase(it);
    delete q;
    return st == NNFFT_OK ? NNFFT_OK : sfail(st, "request failed");
}

int nnfft_server_stats(nnfft_server_t S, nnfft_server_report *out, int reset) {
    if (!S || !out) return sfail(NNFFT_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof(*out));
    std::vector<double> l = S->lat_ms;
    std::sort(l.begin(), l.end());
    auto pct = [&](double p) {
        if (l.empty()) return 0.0;
        const size_t k = (size_t)std::ceil(p * (double)l.size()) - 1;
        return l[std::min(k, l.size() - 1)];
    };
    out->completed = S->completed;
    out->failed = S->failed;
    out->pending = (int64_t)S->pending.size();
    out->in_flight = (int64_t)S->reqs.size() - (int64_t)S->pending.size();
    for (const auto &kv : S->reqs) out->in_flight -= kv.second->done ? 1 : 0;
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = l.empty() ? 0.0 : l.back();
    double sum = 0;
    for (double v : l) sum += v;
    out->mean_ms = l.empty() ? 0.0 : sum / (double)l.size();
    out->points = S->points;
    out->seconds = S->any ? std::chrono::duration<double>(S->t_last - S->t_first).count() : 0.0;
    out->plans_cached = S->plans_cached.load();
    out->plans_made = S->plans_made;
    out->plans_evicted = S->plans_evicted;
    out->device_bytes = (int64_t)(S->fixed_bytes + S->plan_bytes);
    if (reset) {
        S->lat_ms.clear();
        S->points = 0;
        S->completed = S->failed = 0;
        S->any = false;
    }
    return NNFFT_OK;
}

int nnfft_server_destroy(nnfft_server_t S) {
    if (!S) return NNFFT_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    {
        std::lock_guard<std::mutex> g(S->mu_build);
        S->stop_build = true;
        for (PlanEntry *e : S->build_jobs) {   // queued, never started
            S->plans.erase(std::find(S->plans.begin(), S->plans.end(), e));
            delete e;
        }
        S->build_jobs.clear();
    }
    S->cv_build.notify_all();
    if (S->builder.joinable()) S->builder.join();
    integrate_builds(S);
    for (Slot &sl : S->slots)
        if (sl.st) cudaStreamSynchronize(sl.st);
    // plans first: they may still name a slot stream
    for (PlanEntry *e : S->plans) {
        if (e->p) destroy_idle_plan(e->p);
        delete e;
    }
    S->plans.clear();
    for (Slot &sl : S->slots) {
        cudaFree(sl.d1);
        cudaFree(sl.d2);
        cudaFree(sl.c1);
        cudaFree(sl.c2);
        cudaFree(sl.g);
        if (sl.ev) cudaEventDestroy(sl.ev);
        for (cudaEvent_t t : sl.ev_t)
            if (t) cudaEventDestroy(t);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    for (auto &kv : S->rules) cudaFree(kv.second.x1);
    if (S->epoch) cudaEventDestroy(S->epoch);
    for (auto &kv : S->reqs) delete kv.second;
    delete S;
    return NNFFT_OK;
}

}  // extern "C"
