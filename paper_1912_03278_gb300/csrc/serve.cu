// serve.cu -- continuous-batching request loop for HMC ensemble jobs.
//
// A server owns a worker thread and ADMIT_THREADS admission threads.  Requests
// (a model configuration, a number of trajectories, a seed) are queued from any
// host thread; the admission threads take them in arrival order while their
// device memory fits the budget and create their handles (host set-up and
// uploads) while the worker keeps the device busy; the worker keeps every admitted request's state resident (one
// simulation handle per request) and advances all active FP32 lattice
// requests together by one CUDA-graph launch per quantum (other requests on
// their own streams, overlapping on the device).  A request
// leaves the batch when its trajectories are done: its observables are kept,
// its handle destroyed, and waiting requests are admitted into the freed
// memory before the next quantum.  Results of a request do not depend on the
// mix: random numbers depend only on (seed, chain, trajectory) and every
// chain's arithmetic is independent of the launch it runs in.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ising_hmc.h"

namespace {

using clk = std::chrono::steady_clock;

struct Request {
    int64_t id = 0;
    ising_hmc_config cfg{};
    std::vector<double> J, h, beta_c, C_c, eps_c, h0_c;  // owned copies of the config arrays
    int64_t n_traj = 0;
    uint64_t seed = 0;
    int64_t bytes = 0;
    ising_hmc_t *sim = nullptr;
    int64_t target = 0;
    clk::time_point t_submit, t_admit, t_done;
    int state = 0;  // 0 queued, 1 active, 2 done, 3 rejected
    ising_status status = ISING_OK;
    ising_obs obs{};
    int64_t site_steps = 0;
};

}  // namespace

struct ising_server {
    int64_t budget = 0, in_use = 0;
    int admitting = 0;   // taken off the queue, handle being created (not yet active)
    int quantum = 1;
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_admit, cv_work, cv_done;
    std::deque<int64_t> queue;
    std::map<int64_t, Request> req;
    std::vector<int64_t> ready;    // handle created, joins the batch at the next quantum
    std::vector<int64_t> active;
    int64_t next_id = 1;
    bool stop = false;
    std::vector<std::thread> admitters;   // handle creation runs on several host threads
    std::thread worker;
    // statistics
    int64_t admitted = 0, completed = 0, rejected = 0, group_launches = 0, quanta = 0;
    double site_steps = 0.0;
    // seconds spent: creating handles (admission thread), building group
    // graphs, queueing and waiting for quanta, retiring requests (worker)
    double t_create = 0.0, t_graph = 0.0, t_quanta = 0.0, t_retire = 0.0;
    clk::time_point t0;
    char err[512] = {0};
};

static thread_local char g_server_err[512];

// Admission threads: requests leave the queue in arrival order, but their
// handles (host set-up, uploads, the dense forms' Lanczos check) are created
// concurrently.
constexpr int ADMIT_THREADS = 4;

static ising_status sfail(ising_server *s, ising_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(s ? s->err : g_server_err, 512, fmt, ap);
    va_end(ap);
    return st;
}

static void copy_cfg(Request &r, const ising_hmc_config *c) {
    r.cfg = *c;
    r.cfg.stream = nullptr;
    const int64_t N = c->kind != ISING_KIND_LATTICE
                          ? c->n_sites
                          : (int64_t)c->L[0] * (c->dim > 1 ? c->L[1] : 1) * (c->dim > 2 ? c->L[2] : 1);
    auto cp = [&](std::vector<double> &dst, const double *src, int64_t n) -> const double * {
        if (!src) return nullptr;
        dst.assign(src, src + n);
        return dst.data();
    };
    r.cfg.J = cp(r.J, c->J, c->kind == ISING_KIND_DENSE ? N * N : 0);
    r.cfg.h = cp(r.h, c->h, N);
    r.cfg.beta_chain = cp(r.beta_c, c->beta_chain, c->n_chains);
    r.cfg.C_chain = cp(r.C_c, c->C_chain, c->n_chains);
    r.cfg.eps_chain = cp(r.eps_c, c->eps_chain, c->n_chains);
    r.cfg.h0_chain = cp(r.h0_c, c->h0_chain, c->n_chains);
}

// Admission: in arrival order while the budget allows; a request larger than
// the whole budget is rejected.  Handle creation runs outside the lock.
static void admit_loop(ising_server *s) {
    cudaSetDevice(s->device);
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_admit.wait(lk, [&] {
                if (s->stop) return true;
                if (s->queue.empty()) return false;
                const Request &q = s->req[s->queue.front()];
                return q.bytes > s->budget || s->in_use + q.bytes <= s->budget;
            });
            if (s->stop) break;
            Request &q = s->req[s->queue.front()];
            s->queue.pop_front();
            if (q.bytes > s->budget) {  // can never fit
                q.state = 3;
                q.status = ISING_ENOMEM;
                q.t_done = clk::now();
                s->rejected += 1;
                s->cv_done.notify_all();
                continue;
            }
            s->in_use += q.bytes;
            s->admitting += 1;
            r = &q;
            if (!s->queue.empty()) s->cv_admit.notify_one();   // another admission thread
        }
        ising_hmc_t *sim = nullptr;
        const auto tc0 = clk::now();
        nvtxRangePushA("server admission");
        const ising_status st = ising_hmc_create(&r->cfg, &sim);
        nvtxRangePop();
        const double tc = std::chrono::duration<double>(clk::now() - tc0).count();
        std::lock_guard<std::mutex> lk(s->mu);
        s->t_create += tc;
        s->admitting -= 1;
        if (st != ISING_OK) {
            r->state = 3;
            r->status = st;
            r->t_done = clk::now();
            s->in_use -= r->bytes;
            s->rejected += 1;
            s->cv_done.notify_all();
            continue;
        }
        r->sim = sim;
        r->state = 1;
        r->t_admit = clk::now();
        r->target = ising_hmc_traj_index(sim) + r->n_traj;
        s->ready.push_back(r->id);
        s->admitted += 1;
        s->cv_work.notify_one();
    }
}

// Worker: take in the newly admitted requests, advance one quantum, retire.
// Holds the lock only for bookkeeping, never across device work.
static void worker_loop(ising_server *s) {
    cudaSetDevice(s->device);
    ising_group_t *grp = nullptr;
    std::vector<int64_t> grp_members;
    for (;;) {
        std::vector<Request *> act;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->ready.empty() || !s->active.empty(); });
            if (s->stop) break;
            s->active.insert(s->active.end(), s->ready.begin(), s->ready.end());
            s->ready.clear();
            for (int64_t id : s->active) act.push_back(&s->req[id]);
        }
        if (act.empty()) continue;
        const auto tq0 = clk::now();
        nvtxRangePushA("server quantum");
        double tg = 0.0;
        // quantum: the same number of trajectories for every active request
        int64_t k = s->quantum;
        for (Request *r : act) k = std::min(k, r->target - ising_hmc_traj_index(r->sim));
        if (k <= 0) k = 1;
        // shared launch for the FP32 lattice requests, individual launches for the rest
        std::vector<ising_hmc_t *> lat;
        std::vector<int64_t> lat_ids;
        std::vector<uint64_t> seeds;
        for (Request *r : act) {
            if (r->cfg.kind == ISING_KIND_LATTICE && r->cfg.precision == ISING_PREC_FP32) {
                lat.push_back(r->sim);
                lat_ids.push_back(r->id);
                seeds.push_back(r->seed);
            } else {
                if (ising_hmc_trajectories(r->sim, k, r->seed) != ISING_OK) r->status = ISING_ECUDA;
            }
        }
        if (!lat.empty()) {
            if (lat_ids != grp_members) {
                const auto tg0 = clk::now();
                if (grp) ising_group_destroy(grp);
                grp = nullptr;
                if (ising_group_create(lat.data(), (int)lat.size(), &grp) != ISING_OK) grp = nullptr;
                grp_members = lat_ids;
                tg = std::chrono::duration<double>(clk::now() - tg0).count();
            }
            if (grp) {
                const bool ok = ising_group_trajectories_seeds(grp, k, seeds.data()) == ISING_OK;
                ising_group_sync(grp);
                if (ok) {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->group_launches += 1;
                }
            } else {
                for (Request *r : act)
                    if (r->cfg.kind == ISING_KIND_LATTICE && r->cfg.precision == ISING_PREC_FP32)
                        ising_hmc_trajectories(r->sim, k, r->seed);
            }
        }
        for (Request *r : act) ising_hmc_sync(r->sim);
        nvtxRangePop();
        const auto tr0 = clk::now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->quanta += 1;
            s->t_graph += tg;
            s->t_quanta += std::chrono::duration<double>(tr0 - tq0).count() - tg;
        }
        // retire finished requests
        for (Request *r : act) {
            const int64_t steps = (int64_t)k * r->cfg.n_md * r->cfg.n_chains *
                                  ising_hmc_n_sites(r->sim);
            {
                std::lock_guard<std::mutex> lk(s->mu);
                r->site_steps += steps;
                s->site_steps += (double)steps;
            }
            if (ising_hmc_traj_index(r->sim) >= r->target) {
                ising_obs o{};
                ising_status st = ising_hmc_observables(r->sim, &o);
                ising_group_t *g_old = nullptr;
                if (std::find(grp_members.begin(), grp_members.end(), r->id) != grp_members.end()) {
                    g_old = grp;  // the group refers to this handle: drop it first
                    grp = nullptr;
                    grp_members.clear();
                }
                if (g_old) ising_group_destroy(g_old);
                ising_hmc_destroy(r->sim);
                r->sim = nullptr;
                std::lock_guard<std::mutex> lk(s->mu);
                r->obs = o;
                r->status = st;
                r->state = 2;
                r->t_done = clk::now();
                s->in_use -= r->bytes;
                s->completed += 1;
                s->active.erase(std::find(s->active.begin(), s->active.end(), r->id));
                s->cv_done.notify_all();
                s->cv_admit.notify_all();   // memory freed
            }
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->t_retire += std::chrono::duration<double>(clk::now() - tr0).count();
        }
    }
    if (grp) ising_group_destroy(grp);
}

extern "C" {

ising_status ising_server_create(int64_t budget_bytes, int quantum_traj, ising_server_t **out) {
    g_server_err[0] = 0;
    if (!out || budget_bytes <= 0 || quantum_traj < 1)
        return sfail(nullptr, ISING_EINVAL, "server: need budget > 0 and quantum >= 1");
    ising_server *s = new (std::nothrow) ising_server();
    if (!s) return sfail(nullptr, ISING_ENOMEM, "server: host allocation failed");
    s->budget = budget_bytes;
    s->quantum = quantum_traj;
    cudaGetDevice(&s->device);
    s->t0 = clk::now();
    for (int i = 0; i < ADMIT_THREADS; ++i) s->admitters.emplace_back(admit_loop, s);
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return ISING_OK;
}

ising_status ising_server_submit(ising_server_t *s, const ising_hmc_config *cfg, int64_t n_traj,
                                 uint64_t seed, int64_t *request_id) {
    if (!s || !cfg || !request_id || n_traj < 1)
        return sfail(s, ISING_EINVAL, "submit: need config, id pointer and n_traj >= 1");
    const int64_t bytes = ising_hmc_estimate_bytes(cfg);
    if (bytes <= 0) return sfail(s, ISING_EINVAL, "submit: invalid configuration");
    std::lock_guard<std::mutex> lk(s->mu);
    const int64_t id = s->next_id++;
    Request &r = s->req[id];
    r.id = id;
    copy_cfg(r, cfg);
    r.n_traj = n_traj;
    r.seed = seed;
    r.bytes = bytes;
    r.t_submit = clk::now();
    s->queue.push_back(id);
    *request_id = id;
    s->cv_admit.notify_one();
    return ISING_OK;
}

ising_status ising_server_poll(ising_server_t *s, int64_t id, int *state, ising_obs *obs,
                               double *latency_s, double *queue_s) {
    if (!s || !state) return ISING_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->req.find(id);
    if (it == s->req.end()) return sfail(s, ISING_EINVAL, "poll: unknown request %lld", (long long)id);
    const Request &r = it->second;
    *state = r.state;
    if (r.state >= 2) {
        if (obs) *obs = r.obs;
        if (latency_s) *latency_s = std::chrono::duration<double>(r.t_done - r.t_submit).count();
        if (queue_s)
            *queue_s = r.state == 2 ? std::chrono::duration<double>(r.t_admit - r.t_submit).count() : -1.0;
        return r.status;
    }
    return ISING_OK;
}

ising_status ising_server_wait(ising_server_t *s, int64_t id, double timeout_s) {
    if (!s) return ISING_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->req.find(id);
    if (it == s->req.end()) return sfail(s, ISING_EINVAL, "wait: unknown request");
    const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                        [&] { return it->second.state >= 2; });
    return ok ? ISING_OK : sfail(s, ISING_ETIMEOUT, "wait: request %lld not done", (long long)id);
}

ising_status ising_server_drain(ising_server_t *s, double timeout_s) {
    if (!s) return ISING_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                        [&] {
                                            return s->queue.empty() && s->admitting == 0 &&
                                                   s->ready.empty() && s->active.empty();
                                        });
    return ok ? ISING_OK : sfail(s, ISING_ETIMEOUT, "drain: work remains");
}

ising_status ising_server_stats(ising_server_t *s, double *out /* ISING_SERVER_NSTATS */) {
    if (!s || !out) return ISING_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    out[0] = (double)s->admitted;
    out[1] = (double)s->completed;
    out[2] = (double)s->rejected;
    out[3] = (double)s->queue.size();
    out[4] = (double)(s->active.size() + s->ready.size());
    out[5] = (double)s->in_use;
    out[6] = s->site_steps;
    out[7] = (double)s->group_launches;
    out[8] = (double)s->quanta;
    out[9] = std::chrono::duration<double>(clk::now() - s->t0).count();
    out[10] = s->t_create;
    out[11] = s->t_graph;
    out[12] = s->t_quanta;
    out[13] = s->t_retire;
    return ISING_OK;
}

const char *ising_server_last_error(const ising_server_t *s) { return s ? s->err : g_server_err; }

void ising_server_destroy(ising_server_t *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_admit.notify_all();
    s->cv_work.notify_all();
    for (std::thread &t : s->admitters)
        if (t.joinable()) t.join();
    if (s->worker.joinable()) s->worker.join();
    for (auto &kv : s->req)
        if (kv.second.sim) ising_hmc_destroy(kv.second.sim);
    delete s;
}

}  // extern "C"
