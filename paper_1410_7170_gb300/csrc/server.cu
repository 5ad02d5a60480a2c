// Serving loop: overlap solves of different lattices, masses and right-hand-side counts
// submitted as they arrive, run concurrently on one GPU.
//
//   * slots: `slots` worker threads; every context runs on a CUDA stream of its own (a
//     cached context moves between workers, and a stream must never be driven by two
//     threads, one of them possibly capturing a graph on it), so the kernels of
//     concurrent requests overlap on the device;
//   * admission: a queued request starts as soon as a slot is idle and its estimated
//     device memory fits the HBM budget next to the requests already running and the
//     cached contexts (first fit in arrival order, so one large request does not hold up
//     smaller ones behind it);
//   * residency: the context of a finished request (gauge field in both precisions,
//     spectral interval, Zolotarev coefficients, autotuned stencils, Krylov workspaces) is
//     kept, keyed by the caller's gauge key and the operator parameters; a later request
//     with the same key reuses it without upload or set-up. Idle contexts are evicted,
//     least recently used first, when a new request needs their memory;
//   * accounting: per request the time queued, the time running and the latency
//     (submission to completion); over the server p50/p99 latency, completed solves per
//     second of wall time, and the high-water mark of reserved device memory.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/ovl.h"
#include "solver.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    long ticket;
    ovl_request req;
    ovl_params params;
    bool has_params;
    size_t est_bytes;
    Clock::time_point t_submit, t_start, t_end;
    ovl_result res;
    bool done = false;
    ovl_ctx *claimed = nullptr;   // cached context taken for this request at admission
    size_t claimed_bytes = 0;
};

struct CachedCtx {
    ovl_ctx *ctx;
    long key;
    int dims[4];
    double rho, mu;
    ovl_params params;
    size_t bytes;
    long last_use;
};

bool same_params(const ovl_params &a, const ovl_params &b) { return memcmp(&a, &b, sizeof(ovl_params)) == 0; }

}  // namespace

struct ovl_server {
    int slots;
    size_t budget;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> queue;
    std::map<long, Job *> jobs;
    std::list<CachedCtx> idle;   // cached contexts not in use
    size_t reserved = 0;         // running requests' estimates
    size_t cached = 0;           // idle contexts' bytes
    size_t high_water = 0;
    long next_ticket = 1, use_clock = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    std::vector<double> latencies;
    Clock::time_point t_first, t_last;
    bool any_done = false;
    long completed = 0, failed = 0;
    int device = 0;
};

namespace {

// Device memory of one request: the context's fields and workspaces for its lattice,
// precision, preconditioner and right-hand sides (an upper estimate of what ovl_create
// and ovl_solve allocate).
size_t estimate_bytes(const ovl_request &r, const ovl_params &p) {
    const double V = (double)r.dims[0] * r.dims[1] * r.dims[2] * r.dims[3];
    const double v64 = 24.0 * V * 8.0, v32 = 24.0 * V * 4.0;
    double b = V * 4 * (9 * 16 + 3 * 16);                 // links: FP64 18 reals + FP32 12 reals
    b += 3 * v64 + 6 * v32;                               // staging, Lanczos / tuning vectors
    b += 24 * v32;                                        // multi-RHS stencil tuning (12 RHS in and out)
    b += (p.n_poles + 3) * v64;                           // FP64 (or float-float) multishift
    const bool mixed = p.precision != OVL_FP64 || p.precond == OVL_PREC_RECURSIVE;
    if (mixed) b += (p.n_poles + 4) * v32;                 // FP32 multishift
    if (mixed && p.ff_outer) b += V * 4 * 9 * 16;          // float-float links
    if (p.sign_method == OVL_SIGN_KRYLOV) b += (p.krylov_m + p.krylov_keep + 3) * v64;   // Krylov sign basis
    if (p.n_deflate > 0) {
        // eigenvectors xi, gamma5 xi (FP64 and FP32) and scratch, plus the eigensolver's basis
        // while the context is created (basis m + 1, kept Ritz vectors, one scratch vector)
        const int k = p.n_deflate, mmax = std::min(2 * (k + 1) + 32, 120);
        const int nkeep = std::min(k + 17, mmax - 16);
        b += (2 * k + 1) * v64 + (2 * k + 1) * v32 + (mmax + nkeep + 2) * v64;
    }
    const int nrhs = r.n_rhs;
    if (nrhs > 1 && p.rhs_block > 1) {
        const int nb = std::min(std::min(p.rhs_block, nrhs), 12);
        const int mo = std::min(p.restart, 32), mi = std::min(p.restart_inner, 32), mw = std::min(p.prec_restart, 16);
        b += nb * ((2 * mo + 5) * v64 + (p.n_poles + 3) * v64);
        if (mixed) b += nb * ((2 * mi + 3) * v32 + (2 * mw + 3) * v32 + (p.n_poles + 3) * v32 + 2 * v32);
    } else {
        b += (2 * p.restart + 5) * v64;                   // outer FGMRES basis (V and Z)
        if (p.precond == OVL_PREC_RECURSIVE) b += (2 * p.restart_inner + 3) * v32;
        if (p.precond != OVL_PREC_NONE) b += (2 * p.prec_restart + 4) * (mixed ? v32 : v64) + 2 * v32;
    }
    return (size_t)(b * 1.1) + ((size_t)64 << 20);
}

// Frees every idle cached context. Called with the lock held.
void evict_idle(ovl_server *s) {
    for (auto &cc : s->idle) {
        s->cached -= cc.bytes;
        ovl_destroy(cc.ctx);
    }
    s->idle.clear();
}

void run_job(ovl_server *s, Job *j) {
    // context: the cached one claimed at admission, or a new one
    ovl_ctx *ctx = j->claimed;
    const size_t cbytes = j->claimed_bytes;
    ovl_status st = OVL_OK;
    if (!ctx) st = ovl_create(&ctx, j->req.gauge, j->req.dims, j->req.rho, j->req.mu, &j->params, nullptr);
    // the admission estimate reserved the batch workspaces: batch by rhs_block alone
    if (ctx) reinterpret_cast<ovl::Ctx *>(ctx)->fixed_batch = true;
    ovl_stats stats;
    memset(&stats, 0, sizeof(stats));
    if (st == OVL_OK) st = ovl_solve(ctx, j->req.x, j->req.b, j->req.n_rhs, j->req.tol, &stats);
    if (st == OVL_ENOMEM) {
        // the device ran out although the estimates fitted the budget (a running request using
        // more than its estimate): free every idle resident context and try once more from a new
        // context (the solve starts again from whatever x holds)
        if (ctx) {
            ovl_destroy(ctx);
            ctx = nullptr;
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            evict_idle(s);
        }
        st = ovl_create(&ctx, j->req.gauge, j->req.dims, j->req.rho, j->req.mu, &j->params, nullptr);
        if (ctx) reinterpret_cast<ovl::Ctx *>(ctx)->fixed_batch = true;
        if (st == OVL_OK) st = ovl_solve(ctx, j->req.x, j->req.b, j->req.n_rhs, j->req.tol, &stats);
    }
    if (st != OVL_OK && ctx) {
        strncpy(j->res.message, ovl_last_error(ctx), sizeof(j->res.message) - 1);
    } else if (st != OVL_OK) {
        strncpy(j->res.message, ovl_last_error(nullptr), sizeof(j->res.message) - 1);
    }
    size_t held = 0;
    if (ctx) held = reinterpret_cast<ovl::Ctx *>(ctx)->bytes_held;
    j->t_end = Clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    s->reserved -= cbytes ? cbytes : j->est_bytes;
    if (ctx) {
        if (j->req.gauge_key && st == OVL_OK) {
            CachedCtx cc;
            cc.ctx = ctx;
            cc.key = j->req.gauge_key;
            memcpy(cc.dims, j->req.dims, sizeof(cc.dims));
            cc.rho = j->req.rho;
            cc.mu = j->req.mu;
            cc.params = j->params;
            cc.bytes = std::max(held, j->est_bytes);
            cc.last_use = ++s->use_clock;
            s->idle.push_back(cc);
            s->cached += cc.bytes;
        } else {
            ovl_destroy(ctx);
        }
    }
    j->res.done = 1;
    j->res.status = st;
    j->res.stats = stats;
    j->res.queue_s = std::chrono::duration<double>(j->t_start - j->t_submit).count();
    j->res.run_s = std::chrono::duration<double>(j->t_end - j->t_start).count();
    j->res.latency_s = std::chrono::duration<double>(j->t_end - j->t_submit).count();
    j->res.device_bytes = std::max(held, j->est_bytes);
    j->done = true;
    if (st == OVL_OK) {
        s->completed++;
        s->latencies.push_back(j->res.latency_s);
    } else {
        s->failed++;
    }
    s->any_done = true;
    s->t_last = j->t_end;
    s->cv_done.notify_all();
    s->cv_work.notify_all();
}

// Frees idle cached contexts (least recently used first) until `need` more bytes fit.
// Called with the lock held.
bool make_room(ovl_server *s, size_t need) {
    while (s->reserved + s->cached + need > s->budget && !s->idle.empty()) {
        auto lru = std::min_element(s->idle.begin(), s->idle.end(),
                                    [](const CachedCtx &a, const CachedCtx &b) { return a.last_use < b.last_use; });
        s->cached -= lru->bytes;
        ovl_destroy(lru->ctx);
        s->idle.erase(lru);
    }
    return s->reserved + s->cached + need <= s->budget;
}

void worker(ovl_server *s) {
    cudaSetDevice(s->device);
    while (true) {
        Job *j = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            while (true) {
                if (s->stop && s->queue.empty()) break;
                // first queued request whose memory fits (reusing a cached context needs none)
                for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
                    Job *c = *it;
                    auto hit = s->idle.end();
                    if (c->req.gauge_key)
                        for (auto ci = s->idle.begin(); ci != s->idle.end(); ++ci)
                            if (ci->key == c->req.gauge_key && !memcmp(ci->dims, c->req.dims, sizeof(ci->dims)) &&
                                ci->rho == c->req.rho && ci->mu == c->req.mu && same_params(ci->params, c->params)) {
                                hit = ci;
                                break;
                            }
                    if (hit != s->idle.end()) {
                        // claim the resident context: its memory moves from cached to reserved
                        c->claimed = hit->ctx;
                        c->claimed_bytes = hit->bytes;
                        s->cached -= hit->bytes;
                        s->reserved += hit->bytes;
                        s->idle.erase(hit);
                    } else if (make_room(s, c->est_bytes)) {
                        s->reserved += c->est_bytes;
                    } else {
                        continue;
                    }
                    j = c;
                    s->queue.erase(it);
                    s->high_water = std::max(s->high_water, s->reserved + s->cached);
                    break;
                }
                if (j) break;
                s->cv_work.wait(lk);
            }
            if (!j) break;
            j->t_start = Clock::now();
        }
        run_job(s, j);
    }
}

}  // namespace

extern "C" ovl_status ovl_server_create(ovl_server **srv, int slots, size_t hbm_budget) {
    if (!srv || slots < 1 || slots > 64) return OVL_EINVAL;
    *srv = nullptr;
    ovl_server *s = new ovl_server();
    s->slots = slots;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return OVL_ECUDA;
    }
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return OVL_ECUDA;
    }
    s->budget = hbm_budget ? std::min(hbm_budget, fr) : (size_t)(0.9 * (double)fr);
    for (int k = 0; k < slots; k++) s->workers.emplace_back(worker, s);
    *srv = s;
    return OVL_OK;
}

extern "C" ovl_status ovl_request_bytes(const ovl_request *req, size_t *bytes) {
    if (!req || !bytes || req->n_rhs < 1) return OVL_EINVAL;
    for (int m = 0; m < 4; m++)
        if (req->dims[m] < 1) return OVL_EINVAL;
    ovl_params p;
    if (req->params) p = *req->params;
    else ovl_params_default(&p);
    *bytes = estimate_bytes(*req, p);
    return OVL_OK;
}

extern "C" ovl_status ovl_server_submit(ovl_server *s, const ovl_request *req, long *ticket) {
    if (!s || !req || !ticket || !req->gauge || !req->b || !req->x || req->n_rhs < 1) return OVL_EINVAL;
    Job *j = new Job();
    j->req = *req;
    if (req->params) j->params = *req->params;
    else ovl_params_default(&j->params);
    j->req.params = nullptr;
    j->est_bytes = estimate_bytes(j->req, j->params);
    memset(&j->res, 0, sizeof(j->res));
    std::lock_guard<std::mutex> lk(s->mu);
    if (j->est_bytes > s->budget) {
        delete j;
        return OVL_ENOMEM;   // can never be admitted under this budget
    }
    j->ticket = s->next_ticket++;
    j->t_submit = Clock::now();
    if (j->ticket == 1) s->t_first = j->t_submit;   // throughput counts from the first submission
    s->jobs[j->ticket] = j;
    s->queue.push_back(j);
    *ticket = j->ticket;
    s->cv_work.notify_one();
    return OVL_OK;
}

extern "C" ovl_status ovl_server_query(ovl_server *s, long ticket, ovl_result *res) {
    if (!s || !res) return OVL_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return OVL_EINVAL;
    *res = it->second->res;
    return OVL_OK;
}

extern "C" ovl_status ovl_server_wait(ovl_server *s, long ticket, ovl_result *res) {
    if (!s) return OVL_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(ticket);
    if (it == s->jobs.end()) return OVL_EINVAL;
    Job *j = it->second;
    s->cv_done.wait(lk, [&] { return j->done; });
    if (res) *res = j->res;
    return OVL_OK;
}

extern "C" ovl_status ovl_server_report(ovl_server *s, double *p50, double *p99, double *solves_per_s,
                                        size_t *hbm_high_water, long *completed, long *failed) {
    if (!s) return OVL_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    std::vector<double> l = s->latencies;
    std::sort(l.begin(), l.end());
    auto pct = [&](double q) {
        if (l.empty()) return 0.0;
        const double pos = q * (double)(l.size() - 1);
        const size_t i = (size_t)pos;
        const double f = pos - (double)i;
        return i + 1 < l.size() ? l[i] * (1 - f) + l[i + 1] * f : l[i];
    };
    if (p50) *p50 = pct(0.50);
    if (p99) *p99 = pct(0.99);
    if (solves_per_s) {
        const double wall = s->any_done ? std::chrono::duration<double>(s->t_last - s->t_first).count() : 0.0;
        *solves_per_s = wall > 0 ? (double)s->completed / wall : 0.0;
    }
    if (hbm_high_water) *hbm_high_water = s->high_water;
    if (completed) *completed = s->completed;
    if (failed) *failed = s->failed;
    return OVL_OK;
}

extern "C" ovl_status ovl_server_destroy(ovl_server *s) {
    if (!s) return OVL_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    for (auto &cc : s->idle) ovl_destroy(cc.ctx);
    for (auto &kv : s->jobs) delete kv.second;
    delete s;
    return OVL_OK;
}
