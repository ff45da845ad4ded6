// server.cpp -- continuous-batching request loop for repeated mobility applies.
//
// A request is one suspension (N points, box L, tolerance, precision) that
// issues `napplies` successive applies with updated forces, as an iterative
// solve would: positions are binned once (cell lists and grid-tile order stay
// on the device, ewald_set_positions) and each apply after the first starts
// from the previous forces plus a seeded perturbation (k_serve.cu).  Only the
// last apply's velocities go back to the caller.
//
// A scheduler thread admits queued requests while the sum of the admitted
// requests' device footprints (the planner's estimate plus the request
// buffers) stays within the budget and a slot is free.  Order: shortest
// expected work first (N x applies x the planner's precision weight), so a
// small request does not wait behind a large one; a request queued longer
// than the age limit goes first (oldest first), and while such a request
// does not fit, nothing overtakes it.  Each admitted request runs on its own
// stream, with a CUDA stream priority that falls with its expected work, so
// the block scheduler serves the small requests' kernels first when several
// are ready; the work of different requests overlaps on the GPU.  The thread
// polls the requests' completion events, releases their plans and memory, and
// admits the next ones as room frees up.
// The paper has no counterpart: it applies one suspension at a time.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"

#define EW_ST_RET(call)                                  \
    do {                                                 \
        ewald_status s_ = (call);                        \
        if (s_ != EWALD_OK)                              \
            return s_;                                   \
    } while (0)

using namespace ewg;

namespace {

enum ReqState { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3, kCancelled = 4 };

struct Req {
    ewald_request r;
    ReqState state = kQueued;
    ewald_status status = EWALD_OK;
    int64_t footprint = 0;
    double work = 0.0;  // expected work: N x applies x precision weight
    double t_arrival = 0.0, t_done = 0.0;
    ewald_plan_t plan = nullptr;
    double *dbuf = nullptr;  // x, f, u (9 N doubles) and 3 doubles of sums
    double *hbuf = nullptr;  // pinned staging: x, f in, u out (9 N doubles)
    int slot = -1;
    cudaEvent_t done = nullptr;
};

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct ewald_server_s {
    int device = 0;
    int64_t budget = 0;
    int max_active = 1;
    std::mutex mu;
    std::condition_variable cv_done;   // waiters
    std::condition_variable cv_sched;  // scheduler wake-ups
    std::deque<int64_t> queue;
    std::map<int64_t, Req *> reqs;
    int64_t next_id = 1;
    int64_t fp_active = 0, fp_peak = 0;
    int active = 0;
    bool paused = false, stop = false;
    std::vector<cudaStream_t> slots;   // per admission slot, one stream per priority level
    std::vector<bool> slot_busy;
    int prio_least = 0, prio_greatest = 0;  // CUDA stream priority range (greatest = most urgent)
    double age_limit_s = 2.0;
    std::thread sched;
    std::vector<double> lat_ms;
    double pa = 0.0, t_first = -1.0, t_last = -1.0;
    int64_t n_sub = 0, n_done = 0, n_failed = 0, n_cancel = 0;
};

namespace {

void release(Req *q)
{
    if (q->plan)
        ewald_destroy(q->plan);
    q->plan = nullptr;
    if (q->dbuf)
        cudaFree(q->dbuf);
    q->dbuf = nullptr;
    if (q->hbuf)
        cudaFreeHost(q->hbuf);
    q->hbuf = nullptr;
    if (q->done)
        cudaEventDestroy(q->done);
    q->done = nullptr;
}

// Plan, buffers, copies and every apply of one request, enqueued on `s`.
ewald_status start(Req *q, cudaStream_t s, int priority)
{
    const ewald_request &r = q->r;
    const int64_t N = r.N;
    EW_ST_RET(ewald_plan(N, r.L, r.tol, (ewald_dtype)r.dtype, &q->plan));
    // the plan's near-field side stream at the request's priority too
    EW_ST_RET(plan_set_stream_priority(q->plan, priority));
    if (cudaMalloc(&q->dbuf, sizeof(double) * (9 * (size_t)N + 3)) != cudaSuccess) {
        cudaGetLastError();
        q->dbuf = nullptr;
        return EWALD_ENOMEM;
    }
    // pinned staging, so that every copy is asynchronous and this thread
    // never waits on the GPU
    if (cudaMallocHost(&q->hbuf, sizeof(double) * 9 * (size_t)N) != cudaSuccess) {
        cudaGetLastError();
        q->hbuf = nullptr;
        return EWALD_ENOMEM;
    }
    if (cudaEventCreateWithFlags(&q->done, cudaEventDisableTiming) != cudaSuccess)
        return EWALD_ECUDA;
    double *x = q->dbuf, *f = x + 3 * N, *u = f + 3 * N, *sums = u + 3 * N;
    const size_t bytes = sizeof(double) * 3 * (size_t)N;
    memcpy(q->hbuf, r.x_host, bytes);
    memcpy(q->hbuf + 3 * N, r.f_host, bytes);
    if (cudaMemcpyAsync(x, q->hbuf, 2 * bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return EWALD_ECUDA;
    EW_ST_RET(ewald_set_positions(q->plan, x, s));
    for (int t = 0; t < r.napplies; ++t) {
        if (t > 0 && launch_perturb_forces(f, N, r.perturb, (uint32_t)t, r.seed, sums, s) != cudaSuccess)
            return EWALD_ECUDA;
        EW_ST_RET(ewald_apply_forces(q->plan, f, u, s));
    }
    if (cudaMemcpyAsync(q->hbuf + 6 * N, u, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaEventRecord(q->done, s) != cudaSuccess)
        return EWALD_ECUDA;
    return EWALD_OK;
}

void finish(ewald_server_s *sv, Req *q, ReqState st, ewald_status status)
{
    // caller holds sv->mu
    q->state = st;
    q->status = status;
    q->t_done = now_s();
    if (q->slot >= 0)
        sv->slot_busy[q->slot] = false;
    sv->fp_active -= q->footprint;
    sv->active -= 1;
    if (st == kDone) {
        sv->n_done += 1;
        sv->lat_ms.push_back(1e3 * (q->t_done - q->t_arrival));
        sv->pa += (double)q->r.N * q->r.napplies;
        sv->t_last = std::max(sv->t_last, q->t_done);
    } else {
        sv->n_failed += 1;
    }
    sv->cv_done.notify_all();
}

// Relative cost of one point-apply in the plan's precision (FP32 = 1), from
// the GB300 stage weights the planner uses.
double precision_weight(const ewald_params &p)
{
    if (p.near_ds)
        return 5.0;
    if (p.near_f64)
        return 40.0;
    return p.fft_f64 ? 1.5 : 1.0;
}

// Stream priority of a request: log-spaced over expected work from 2e4 (a
// thousand points, 20 FP32 applies) to 5e9, the smallest the most urgent.
int priority_for(const ewald_server_s *sv, double work)
{
    const int levels = sv->prio_least - sv->prio_greatest + 1;
    if (levels <= 1)
        return sv->prio_least;
    double t = (std::log10(std::max(work, 1.0)) - std::log10(2e4)) / (std::log10(5e9) - std::log10(2e4));
    t = std::min(1.0, std::max(0.0, t));
    return sv->prio_greatest + (int)std::lround(t * (levels - 1));
}

// The next queued request to admit (index into sv->queue), or -1: the oldest
// one past the age limit if any (and -1 if it does not fit, so that nothing
// overtakes it), else the smallest expected work among those that fit.
// Caller holds sv->mu.
int pick_next(ewald_server_s *sv, double now)
{
    int oldest = -1;
    for (int k = 0; k < (int)sv->queue.size(); ++k) {
        const Req *q = sv->reqs[sv->queue[k]];
        if (now - q->t_arrival > sv->age_limit_s &&
            (oldest < 0 || q->t_arrival < sv->reqs[sv->queue[oldest]]->t_arrival))
            oldest = k;
    }
    if (oldest >= 0)
        return sv->fp_active + sv->reqs[sv->queue[oldest]]->footprint <= sv->budget ? oldest : -1;
    int best = -1;
    for (int k = 0; k < (int)sv->queue.size(); ++k) {
        const Req *q = sv->reqs[sv->queue[k]];
        if (sv->fp_active + q->footprint > sv->budget)
            continue;
        if (best < 0 || q->work < sv->reqs[sv->queue[best]]->work)
            best = k;
    }
    return best;
}

void scheduler(ewald_server_s *sv)
{
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        // completions
        for (auto &kv : sv->reqs) {
            Req *q = kv.second;
            if (q->state != kRunning)
                continue;
            const cudaError_t e = cudaEventQuery(q->done);
            if (e == cudaErrorNotReady)
                continue;
            if (e == cudaSuccess)
                memcpy(q->r.u_host, q->hbuf + 6 * q->r.N, sizeof(double) * 3 * (size_t)q->r.N);
            else
                cudaGetLastError();
            release(q);
            finish(sv, q, e == cudaSuccess ? kDone : kFailed, e == cudaSuccess ? EWALD_OK : EWALD_ECUDA);
        }
        // admissions: shortest expected work first, the age limit first of all
        while (!sv->paused && !sv->stop && !sv->queue.empty() && sv->active < sv->max_active) {
            const int k = pick_next(sv, now_s());
            if (k < 0)
                break;
            Req *q = sv->reqs[sv->queue[k]];
            sv->queue.erase(sv->queue.begin() + k);
            int slot = 0;
            while (sv->slot_busy[slot])
                ++slot;
            sv->slot_busy[slot] = true;
            q->slot = slot;
            q->state = kRunning;
            sv->active += 1;
            sv->fp_active += q->footprint;
            sv->fp_peak = std::max(sv->fp_peak, sv->fp_active);
            const int prio = priority_for(sv, q->work);
            const int levels = sv->prio_least - sv->prio_greatest + 1;
            cudaStream_t &ss = sv->slots[slot * levels + (prio - sv->prio_greatest)];
            lk.unlock();
            ewald_status st = EWALD_OK;
            if (!ss && cudaStreamCreateWithPriority(&ss, cudaStreamNonBlocking, prio) != cudaSuccess) {
                cudaGetLastError();
                ss = nullptr;
                st = EWALD_ECUDA;
            }
            if (st == EWALD_OK)
                st = start(q, ss, prio);
            lk.lock();
            if (st != EWALD_OK) {
                if (ss)
                    cudaStreamSynchronize(ss);
                cudaGetLastError();
                release(q);
                finish(sv, q, kFailed, st);
            }
        }
        if (sv->stop && sv->active == 0)
            break;
        if (sv->active > 0)
            sv->cv_sched.wait_for(lk, std::chrono::microseconds(100));
        else
            sv->cv_sched.wait(lk, [&] { return sv->stop || (!sv->paused && !sv->queue.empty()); });
    }
}

}  // namespace

extern "C" {

ewald_status ewald_server_create(int64_t hbm_budget_bytes, int32_t max_active, int32_t start_paused,
                                 ewald_server_t *out)
{
    if (!out || hbm_budget_bytes <= 0 || max_active < 1 || max_active > 256)
        return EWALD_EINVAL;
    ewald_server_s *sv = new (std::nothrow) ewald_server_s;
    if (!sv)
        return EWALD_ENOMEM;
    if (cudaGetDevice(&sv->device) != cudaSuccess) {
        cudaGetLastError();  // no device yet: requests fail at admission, not here
        sv->device = 0;
    }
    sv->budget = hbm_budget_bytes;
    sv->max_active = max_active;
    sv->paused = start_paused != 0;
    if (cudaDeviceGetStreamPriorityRange(&sv->prio_least, &sv->prio_greatest) != cudaSuccess) {
        cudaGetLastError();
        sv->prio_least = sv->prio_greatest = 0;
    }
    // streams made at a slot's first use at a priority level
    sv->slots.assign((size_t)max_active * (sv->prio_least - sv->prio_greatest + 1), nullptr);
    sv->slot_busy.assign(max_active, false);
    try {
        sv->sched = std::thread(scheduler, sv);
    } catch (...) {
        delete sv;
        return EWALD_ENOMEM;
    }
    *out = sv;
    return EWALD_OK;
}

ewald_status ewald_server_submit(ewald_server_t sv, const ewald_request *r, int64_t *ticket)
{
    if (!sv || !r || !ticket || r->N < 1 || r->napplies < 1 || !r->x_host || !r->f_host ||
        !r->u_host || !(r->perturb >= 0.0))
        return EWALD_EINVAL;
    ewald_params prm;
    const ewald_status st = ewald_choose_params(r->N, r->L, r->tol, (ewald_dtype)r->dtype, nullptr, &prm);
    if (st != EWALD_OK)
        return st;
    const int64_t fp = prm.footprint_bytes + (int64_t)sizeof(double) * (9 * r->N + 3);
    if (fp > sv->budget)
        return EWALD_ENOMEM;  // would never fit: refused at the door
    Req *q = new (std::nothrow) Req;
    if (!q)
        return EWALD_ENOMEM;
    q->r = *r;
    q->footprint = fp;
    q->work = (double)r->N * r->napplies * precision_weight(prm);
    q->t_arrival = now_s();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        const int64_t id = sv->next_id++;
        sv->reqs[id] = q;
        sv->queue.push_back(id);
        sv->n_sub += 1;
        if (sv->t_first < 0)
            sv->t_first = q->t_arrival;
        *ticket = id;
    }
    sv->cv_sched.notify_one();
    return EWALD_OK;
}

ewald_status ewald_server_poll(ewald_server_t sv, int64_t ticket, int32_t *state, double *latency_ms)
{
    if (!sv)
        return EWALD_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end())
        return EWALD_EINVAL;
    const Req *q = it->second;
    if (state)
        *state = (int32_t)q->state;
    if (latency_ms)
        *latency_ms = (q->state == kDone || q->state == kFailed) ? 1e3 * (q->t_done - q->t_arrival) : -1.0;
    return q->state == kFailed ? q->status : EWALD_OK;
}

ewald_status ewald_server_wait(ewald_server_t sv, int64_t ticket, double timeout_s)
{
    if (!sv || !(timeout_s >= 0.0))
        return EWALD_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end())
        return EWALD_EINVAL;
    Req *q = it->second;
    const bool ok = sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] {
        return q->state == kDone || q->state == kFailed || q->state == kCancelled;
    });
    if (!ok)
        return EWALD_ETIMEOUT;
    return q->state == kFailed ? q->status : EWALD_OK;
}

ewald_status ewald_server_cancel(ewald_server_t sv, int64_t ticket)
{
    if (!sv)
        return EWALD_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end())
        return EWALD_EINVAL;
    Req *q = it->second;
    if (q->state != kQueued)
        return EWALD_EINVAL;  // running requests finish; done ones are done
    sv->queue.erase(std::find(sv->queue.begin(), sv->queue.end(), ticket));
    q->state = kCancelled;
    sv->n_cancel += 1;
    sv->cv_done.notify_all();
    return EWALD_OK;
}

ewald_status ewald_server_resume(ewald_server_t sv)
{
    if (!sv)
        return EWALD_EINVAL;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->paused = false;
    }
    sv->cv_sched.notify_one();
    return EWALD_OK;
}

ewald_status ewald_server_stats(ewald_server_t sv, ewald_server_summary *out)
{
    if (!sv || !out)
        return EWALD_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = sv->n_sub;
    out->completed = sv->n_done;
    out->failed = sv->n_failed;
    out->cancelled = sv->n_cancel;
    out->queued = (int64_t)sv->queue.size();
    out->active = sv->active;
    out->peak_footprint_bytes = sv->fp_peak;
    out->particle_applies = sv->pa;
    std::vector<double> l = sv->lat_ms;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) {
            const double k = p * (double)(l.size() - 1);
            const size_t a = (size_t)k, b = std::min(a + 1, l.size() - 1);
            return l[a] + (k - (double)a) * (l[b] - l[a]);
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double s = 0;
        for (double v : l)
            s += v;
        out->mean_ms = s / (double)l.size();
    }
    if (sv->t_last > sv->t_first && sv->t_first >= 0)
        out->throughput = sv->pa / (sv->t_last - sv->t_first);
    return EWALD_OK;
}

void ewald_server_destroy(ewald_server_t sv)
{
    if (!sv)
        return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        // queued requests are dropped; running ones complete first
        for (int64_t id : sv->queue) {
            sv->reqs[id]->state = kCancelled;
            sv->n_cancel += 1;
        }
        sv->queue.clear();
    }
    sv->cv_sched.notify_one();
    if (sv->sched.joinable())
        sv->sched.join();
    for (auto &kv : sv->reqs) {
        release(kv.second);
        delete kv.second;
    }
    for (auto s : sv->slots)
        if (s)
            cudaStreamDestroy(s);
    sv->cv_done.notify_all();
    delete sv;
}

}  // extern "C"
