// Continuous-batching solve server.
//
// Requests (multipatch Poisson problems of any size) are queued as they
// arrive.  Setup workers, each owning one non-blocking CUDA stream, admit
// queued requests while the estimated device memory of the admitted requests
// stays within the budget (first come first served; a request that does not
// fit lets later, smaller ones pass) and run assembly and IETI-DP setup on
// their stream.  A set-up request joins the solve loop's batch engine at the
// next outer-iteration boundary: from then on its local solves share the
// merged launches of every other request in flight, and it leaves the batch
// when its dual PCG has converged.  Its operator, multigrid hierarchy, primal
// basis and multipliers stay resident until its solution has been copied to
// the host; then its memory returns to the stream-ordered pool and its budget
// share to the admission queue.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "engine.h"

void ieti_set_error(const std::string& msg);   // ietidp_host.cu

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
    unsigned long long ticket = 0;
    int dim = 0;
    std::vector<iga_patch_desc> patches;
    std::vector<iga_interface_desc> ifs;
    int rhs_kind = 0;
    std::vector<double> ma;
    std::vector<int> mk, ml;
    const double* quad_values = nullptr;
    long long est_bytes = 0;
    long long ntorn = 0;
    double t_submit = 0, t_start = 0, t_setup = 0, t_done = 0;
    iga_problem* prob = nullptr;
    ietidp_handle* h = nullptr;
    double* h_u_dev = nullptr;   // the handle's device output buffer
    int state = 0;   // 0 queued, 1 running, 2 done
    int rc = 0;
    std::string err;
    std::vector<double> u;
    ietidp_stats stats{};
};

// Upper bound of the device memory one request holds (problem + handle +
// assembly scratch), from its patch sizes.
long long estimate_bytes(const Request& r, const ietidp_options& o) {
    long long b = 0;
    const int d = r.dim;
    const bool mixed = o.precision == IETIDP_PREC_MIXED;
    long long ntorn = 0, qp = 0;
    for (const auto& p : r.patches) {
        long long n = 1, S = 1, q = 1;
        for (int k = 0; k < d; ++k) {
            n *= p.nelem[k] + p.degree[k];
            S *= 2 * p.degree[k] + 1;
            q *= (long long)p.nelem[k] * (p.degree[k] + 1);
        }
        ntorn += n;
        qp += q;
        const long long lev = d == 2 ? 2 : 2;       // all levels <= 4/3 (2D), 8/7 (3D) of the fine
        long long per_val = 8 + (mixed ? 4 : 0);     // K64 (+ K32)
        per_val += 8 + (mixed ? 4 : 0);              // K + alpha M^ copies (floating patches; bound)
        b += n * S * per_val * lev;
        b += n * S * 8;                              // the problem's fine stiffness
        b += n * 26 * 8 * 2;                         // primal basis and SZ W (<= 26 constraints per patch)
        b += n * 8 * 8 * 4;                          // CG vectors of patch and basis slots
        if (o.method == IETIDP_METHOD_DMG) {         // banded Cholesky factor
            const int d = r.dim;
            const long long m0 = p.nelem[0] + p.degree[0], m1 = d > 1 ? p.nelem[1] + p.degree[1] : 1;
            const long long bw = p.degree[0] + m0 * ((d > 1 ? p.degree[1] : 0) + m1 * (d > 2 ? p.degree[2] : 0));
            b += n * (bw + 1) * 8;
        }
        b += n * 4 * 8 * lev;                        // level vectors
    }
    b += ntorn * 12 * 8;                             // torn buffers
    if (o.method == IETIDP_METHOD_SADDLE) b += ntorn * 11 * 8;   // BPCG vectors
    b += qp * 7 * 8;                                 // assembly scratch (geometry factors, loads)
    b += 64LL << 20;                                 // tables, coarse matrices, dual vectors, slack
    return b;
}

}  // namespace

struct ietidp_server {
    long long budget = 0;
    int max_concurrent = 1;
    ietidp_options opt{};
    std::mutex mu;
    std::condition_variable cv;
    std::deque<unsigned long long> queue;                  // submitted, not admitted
    std::map<unsigned long long, std::shared_ptr<Request>> reqs;
    std::deque<std::shared_ptr<Request>> ready;            // set up, waiting to join the solve batch
    long long in_flight = 0;
    int running = 0;
    bool stop = false;
    unsigned long long next_ticket = 1;
    std::vector<std::thread> workers;
    // one stream per setup worker; a request's handle and problem stay
    // ordered on it until the solve loop releases them, so the streams are
    // destroyed only after the solve loop has ended
    std::vector<cudaStream_t> wstreams;
    std::thread solver;
    int device = 0;
    int completed = 0;

    void worker(int wid);
    void solve_loop();
    void release(const std::shared_ptr<Request>& r);
};

// a request leaves: its device memory goes back to the pool and the budget
void ietidp_server::release(const std::shared_ptr<Request>& r) {
    if (r->h) ietidp_destroy(r->h);
    if (r->prob) iga_problem_free(r->prob);
    r->h = nullptr;
    r->prob = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        r->t_done = now_s();
        r->state = 2;
        in_flight -= r->est_bytes;
        running -= 1;
        completed += 1;
    }
    cv.notify_all();
}

// setup workers: admit by budget, assemble and set up on the worker's own
// stream, then hand the request to the solve loop
void ietidp_server::worker(int wid) {
    cudaSetDevice(device);
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return;
    wstreams[wid] = st;
    for (;;) {
        std::shared_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lk(mu);
            for (;;) {
                if (stop) return;   // the stream outlives the worker (see wstreams)
                // first queued request that fits the budget
                auto it = queue.begin();
                for (; it != queue.end(); ++it) {
                    auto& q = reqs[*it];
                    if (in_flight + q->est_bytes <= budget || running == 0) break;
                }
                if (it != queue.end()) {
                    r = reqs[*it];
                    queue.erase(it);
                    in_flight += r->est_bytes;
                    running += 1;
                    r->state = 1;
                    r->t_start = now_s();
                    break;
                }
                cv.wait(lk);
            }
        }
        iga_domain_desc dd;
        std::memset(&dd, 0, sizeof(dd));
        dd.dim = r->dim;
        dd.npatch = (int)r->patches.size();
        dd.patches = r->patches.data();
        dd.ninterface = (int)r->ifs.size();
        dd.interfaces = r->ifs.data();
        dd.rhs_kind = r->rhs_kind;
        dd.nmodes = (int)r->ma.size();
        dd.mode_a = r->ma.data();
        dd.mode_k = r->mk.data();
        dd.mode_l = r->ml.data();
        dd.quad_values = r->quad_values;
        int rc = iga_assemble_patches(&dd, st, &r->prob);
        if (rc == IETIDP_OK) rc = ietidp_setup(r->prob, &opt, st, &r->h);
        if (rc == IETIDP_OK) {
            ietidp_info info;
            ietidp_info_get(r->h, &info);
            r->ntorn = info.n_torn;
            r->u.assign((size_t)info.n_torn, 0.0);
            r->h_u_dev = r->h->uH;
            if (cudaStreamSynchronize(st) != cudaSuccess) rc = IETIDP_E_CUDA;
        }
        r->t_setup = now_s();
        if (rc != IETIDP_OK) {
            r->rc = rc;
            r->err = ietidp_last_error();
            release(r);
            continue;
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            ready.push_back(r);
        }
        cv.notify_all();
    }
}

// solve loop: one batch engine; requests join between outer iterations and
// leave when converged, so the local solves of every admitted request share
// the same launches
void ietidp_server::solve_loop() {
    cudaSetDevice(device);
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return;
    ieti_engine* E = nullptr;
    if (ieti_engine_create(st, &E) != IETIDP_OK) {
        cudaStreamDestroy(st);
        return;
    }
    std::vector<std::shared_ptr<Request>> active;
    std::vector<std::unique_ptr<EngineJob>> jobs;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(mu);
            if (active.empty()) cv.wait(lk, [&] { return stop || !ready.empty(); });
            if (stop && active.empty() && ready.empty()) break;
            while (!ready.empty()) {
                auto r = ready.front();
                ready.pop_front();
                auto j = std::make_unique<EngineJob>();
                ieti_engine_job_init(*j, r->h, nullptr, r->h_u_dev);
                active.push_back(r);
                jobs.push_back(std::move(j));
            }
        }
        std::vector<EngineJob*> ptr;
        for (auto& j : jobs) ptr.push_back(j.get());
        int rc = opt.method == IETIDP_METHOD_SADDLE ? ieti_saddle_tick(E, ptr) : ieti_engine_tick(E, ptr);
        std::string terr = rc == IETIDP_OK ? "" : ietidp_last_error();
        // finished (or failed) requests: copy the solution out and release
        std::vector<std::shared_ptr<Request>> keep_r;
        std::vector<std::unique_ptr<EngineJob>> keep_j;
        for (size_t i = 0; i < active.size(); ++i) {
            auto& r = active[i];
            EngineJob& j = *jobs[i];
            if (rc != IETIDP_OK) {
                j.rc = rc;
                j.err = terr;
                j.phase = EngineJob::DONE;
            }
            if (j.phase != EngineJob::DONE) {
                keep_r.push_back(r);
                keep_j.push_back(std::move(jobs[i]));
                continue;
            }
            r->stats = j.S;
            r->rc = j.rc;
            r->err = j.err;
            if (j.rc == IETIDP_OK || j.rc == IETIDP_E_NOT_CONVERGED) {
                if (cudaMemcpyAsync(r->u.data(), r->h_u_dev, sizeof(double) * r->ntorn, cudaMemcpyDeviceToHost,
                                    st) != cudaSuccess ||
                    cudaStreamSynchronize(st) != cudaSuccess) {
                    r->rc = IETIDP_E_CUDA;
                    r->err = "copy of the solution to the host failed";
                }
            }
            release(r);
        }
        active.swap(keep_r);
        jobs.swap(keep_j);
    }
    ieti_engine_destroy(E);
    cudaStreamDestroy(st);
}

extern "C" int ietidp_server_create(long long budget_bytes, int max_concurrent, const ietidp_options* opt,
                                    ietidp_server** out) {
    if (!out || budget_bytes <= 0 || max_concurrent < 1 || max_concurrent > 64) return IETIDP_E_INVALID_ARG;
    auto* s = new ietidp_server();
    s->budget = budget_bytes;
    s->max_concurrent = max_concurrent;
    if (opt) s->opt = *opt;
    else ietidp_default_options(&s->opt);
    cudaGetDevice(&s->device);
    s->wstreams.assign(max_concurrent, nullptr);
    for (int i = 0; i < max_concurrent; ++i) s->workers.emplace_back([s, i] { s->worker(i); });
    s->solver = std::thread([s] { s->solve_loop(); });
    *out = s;
    return IETIDP_OK;
}

extern "C" int ietidp_server_submit(ietidp_server* s, const iga_domain_desc* dom, unsigned long long* ticket) {
    if (!s || !dom || !ticket || dom->npatch < 1 || !dom->patches || (dom->dim != 2 && dom->dim != 3))
        return IETIDP_E_INVALID_ARG;
    auto r = std::make_shared<Request>();
    r->dim = dom->dim;
    r->patches.assign(dom->patches, dom->patches + dom->npatch);
    if (dom->ninterface > 0) r->ifs.assign(dom->interfaces, dom->interfaces + dom->ninterface);
    r->rhs_kind = dom->rhs_kind;
    if (dom->rhs_kind == IGA_RHS_MODES && dom->nmodes > 0) {
        r->ma.assign(dom->mode_a, dom->mode_a + dom->nmodes);
        r->mk.assign(dom->mode_k, dom->mode_k + dom->nmodes);
        r->ml.assign(dom->mode_l, dom->mode_l + dom->nmodes);
    }
    r->quad_values = dom->quad_values;
    r->est_bytes = estimate_bytes(*r, s->opt);
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (r->est_bytes > s->budget) return IETIDP_E_BUDGET;
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        s->queue.push_back(r->ticket);
        *ticket = r->ticket;
    }
    s->cv.notify_all();
    return IETIDP_OK;
}

// Poll (wait = 0) or wait for (wait = 1) a request.  *state: 0 queued,
// 1 running, 2 done.  When done, u (n_torn doubles, may be NULL) and stats
// are filled, the request's return code is returned and the request is
// forgotten; timing: t[0] = queue time, t[1] = run time, t[2] = latency (s).
extern "C" int ietidp_server_poll(ietidp_server* s, unsigned long long ticket, int wait, int* state, double* u,
                                  long long n_u, ietidp_stats* stats, double* t) {
    if (!s || !state) return IETIDP_E_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return IETIDP_E_INVALID_ARG;
    auto r = it->second;
    if (wait)
        s->cv.wait(lk, [&] { return r->state == 2; });
    *state = r->state;
    if (r->state != 2) return IETIDP_OK;
    if (u) {
        if (n_u < r->ntorn) return IETIDP_E_INVALID_ARG;
        std::copy(r->u.begin(), r->u.end(), u);
    }
    if (stats) *stats = r->stats;
    if (t) {
        t[0] = r->t_start - r->t_submit;
        t[1] = r->t_done - r->t_start;
        t[2] = r->t_done - r->t_submit;
    }
    int rc = r->rc;
    if (rc != IETIDP_OK) ieti_set_error("request " + std::to_string(ticket) + ": " + r->err);
    s->reqs.erase(it);
    return rc;
}

// Current occupancy: admitted requests, their estimated bytes, queued count.
extern "C" int ietidp_server_status(ietidp_server* s, int* running, long long* in_flight_bytes, int* queued) {
    if (!s) return IETIDP_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (running) *running = s->running;
    if (in_flight_bytes) *in_flight_bytes = s->in_flight;
    if (queued) *queued = (int)s->queue.size();
    return IETIDP_OK;
}

extern "C" long long ietidp_server_estimate(ietidp_server* s, const iga_domain_desc* dom) {
    if (!s || !dom || dom->npatch < 1 || !dom->patches) return -1;
    Request r;
    r.dim = dom->dim;
    r.patches.assign(dom->patches, dom->patches + dom->npatch);
    return estimate_bytes(r, s->opt);
}

extern "C" int ietidp_server_destroy(ietidp_server* s) {
    if (!s) return IETIDP_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    for (auto& w : s->workers) w.join();
    s->solver.join();
    // the solve loop has released every request: no handle uses these now
    for (cudaStream_t st : s->wstreams)
        if (st) cudaStreamDestroy(st);
    delete s;
    return IETIDP_OK;
}
