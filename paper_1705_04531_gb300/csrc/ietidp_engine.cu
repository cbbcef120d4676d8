// Batched solve engine: the dual PCG of Sec. 2 (F lambda = d with the scaled
// Dirichlet preconditioner, Eq. 4) for several jobs -- a job is one handle and
// one right-hand side -- advanced in lockstep.  One tick is one outer
// iteration of every job:
//
//   stage A  local Neumann solves  (u0 = K~^{-1} f, F p, or the recovery
//            u = K~^{-1}(f - B^T lambda), whichever each job needs next);
//            all patches of all jobs run in ONE launch per kernel
//            specialisation
//   sync     one stream synchronisation reads every job's dual residual
//   stage B  scaled Dirichlet preconditioner of the jobs that continue,
//            again one launch per specialisation over all their patches
//
// Jobs join and leave the set between ticks (ietidp_solve is a batch of one;
// the server feeds the engine as requests are admitted).  The patch-to-CTA
// order of a merged launch is longest-first, and the block size and
// shared-memory budget of each merged launch are picked by an autotuner that
// times the candidate configurations once per launch shape.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <cstdint>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <tuple>
#include <vector>

#include "host_internal.h"
#include "engine.h"

using namespace ieti_host;

namespace {

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
struct TuneKey {
    int dim, p0, p1, p2, kind, mixed;   // kind: 0 specialised, 1 global-memory vectors, 2 run-time degree
    int waves;                          // ceil(slots / SMs)
    long long max_cost;                 // largest patch (rows x stencil)
    int clok;                           // every launch of the stage may run as clusters
    bool operator<(const TuneKey& o) const {
        return std::tie(dim, p0, p1, p2, kind, mixed, waves, max_cost, clok) <
               std::tie(o.dim, o.p0, o.p1, o.p2, o.kind, o.mixed, o.waves, o.max_cost, o.clok);
    }
};

struct TuneCfg {
    int threads;
    size_t smem;
    int ctas_per_sm;
    float ms;
    int xg;      // V-cycle vectors in global memory (fewer bytes of shared memory per CTA)
    int csize;   // CTAs per slot as one thread-block cluster (0 or 1: one CTA)
};

std::mutex g_tune_mu;
std::map<TuneKey, TuneCfg> g_tune;

bool autotune_enabled() {
    const char* e = std::getenv("IETIDP_AUTOTUNE");
    return !(e && e[0] == '0');
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// one merged launch: the slots of every job that share a kernel specialisation
struct MGroup {
    int dim = 0, p0 = 0, p1 = 0, p2 = 0, kind = 0, mixed = 0;
    std::vector<SlotDesc> s;
    std::vector<long long> cost;
    size_t smem = 0;       // shared memory of the handles' own plan (max)
    size_t smem_min = 0;   // shared memory the kernel cannot do without (max)
    size_t tab_min = 0;    // color tables alone (minimum of the global-vector variant)
    int max_bw = 0;        // direct Neumann solves: largest half band width
    int clok = 0;          // the stage's modes all run as clusters (solve-phase modes)
    TuneCfg cfg{512, 0, 1, 0.f, 0, 1};
};

}  // namespace

// ---------------------------------------------------------------------------
// engine state
// ---------------------------------------------------------------------------
struct Staging {   // pinned and device copies of one launch stage's arguments and slots
    SolveArgs* h_args = nullptr;
    SolveArgs* d_args = nullptr;
    size_t cap_args = 0;
    SlotDesc* h_slots = nullptr;
    SlotDesc* d_slots = nullptr;
    size_t cap_slots = 0;
};

struct GraphEntry {   // one captured launch segment
    cudaGraphExec_t exec = nullptr;   // null: the segment could not be captured
    std::vector<long long> dl;        // per job: kernel launches of one replay
    std::vector<long long> dn;        // per job: merged Neumann launches of one replay
    long long total = 0;              // kernels of one replay
    void* d_args = nullptr;           // merged launch arguments and slots owned by the graph
    void* d_slots = nullptr;
};

struct ieti_engine {
    bool own_stream = false;   // the stream was created for the engine (destroyed with it)
    std::map<std::vector<uintptr_t>, std::unique_ptr<GraphEntry>> graphs;
    std::map<std::vector<uintptr_t>, int> seen;
    cudaStream_t st = nullptr;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr, e0 = nullptr, e1 = nullptr;   // e0/e1: bracket of stage A
    cudaEvent_t t0 = nullptr, t1 = nullptr;                   // autotuner timing
    Staging stA, stB, stT;
    double* h_rb = nullptr;   // pinned read-back, one block per job
    size_t cap_rb = 0;
    unsigned long long* d_span = nullptr;   // [start, end] of the merged Neumann stage (globaltimer ns)
};

namespace {

int reserve(ieti_engine* E, Staging& S, size_t nargs, size_t nslots) {
    if (nargs <= S.cap_args && nslots <= S.cap_slots) return IETIDP_OK;
    // earlier copies from the pinned buffers must have completed
    CU(cudaStreamSynchronize(E->st));
    size_t na = std::max(nargs, 2 * S.cap_args), ns = std::max(nslots, 2 * S.cap_slots);
    if (S.h_args) cudaFreeHost(S.h_args);
    if (S.h_slots) cudaFreeHost(S.h_slots);
    if (S.d_args) cudaFreeAsync(S.d_args, E->st);
    if (S.d_slots) cudaFreeAsync(S.d_slots, E->st);
    S = Staging{};
    CU(cudaMallocHost((void**)&S.h_args, sizeof(SolveArgs) * na));
    CU(cudaMallocHost((void**)&S.h_slots, sizeof(SlotDesc) * ns));
    CU(cudaMallocAsync((void**)&S.d_args, sizeof(SolveArgs) * na, E->st));
    CU(cudaMallocAsync((void**)&S.d_slots, sizeof(SlotDesc) * ns, E->st));
    S.cap_args = na;
    S.cap_slots = ns;
    return IETIDP_OK;
}

void free_staging(ieti_engine* E, Staging& S) {
    if (S.h_args) cudaFreeHost(S.h_args);
    if (S.h_slots) cudaFreeHost(S.h_slots);
    if (S.d_args) cudaFreeAsync(S.d_args, E->st);
    if (S.d_slots) cudaFreeAsync(S.d_slots, E->st);
    S = Staging{};
}

void clear_graphs(ieti_engine* E) {
    for (auto& kv : E->graphs) {
        if (kv.second->exec) cudaGraphExecDestroy(kv.second->exec);
        if (kv.second->d_args) cudaFree(kv.second->d_args);
        if (kv.second->d_slots) cudaFree(kv.second->d_slots);
    }
    E->graphs.clear();
    E->seen.clear();
}

int ensure_side(ieti_engine* E, size_t n) {
    while (E->side.size() < std::min<size_t>(n, 8)) {
        cudaStream_t s;
        cudaEvent_t ev;
        CU(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        E->side.push_back(s);
        E->join.push_back(ev);
    }
    return IETIDP_OK;
}

cudaError_t launch_cfg(const SolveArgs& a, const MGroup& g, const TuneCfg& c, cudaStream_t st) {
    SolveArgs b = a;
    b.smem_bytes = c.smem;
    b.csize = c.csize;
    if (g.kind == 3) return launch_direct_neumann(b, g.max_bw, st);
    if (g.kind == 2) return launch_solve(b, c.threads, st);
    return launch_solve_variant(b, g.dim, g.p0, g.p1, g.p2, c.threads, st, g.kind == 1 || c.xg);
}

// candidate configurations of a merged launch: 512 threads with the full
// budget, or fewer threads with a budget that lets 2 or 3 CTAs share an SM
std::vector<TuneCfg> candidates(const MGroup& g) {
    std::vector<TuneCfg> c;
    c.push_back(TuneCfg{512, g.smem, 1, 0.f, 0});
    if (g.kind == 2) return c;
    // (threads, CTAs per SM, vectors in global memory): the vectors of a
    // patch need shared memory only in the shared-vector variant, so the
    // global-vector variant reaches more CTAs per SM
    const int thr[5] = {256, 128, 256, 128, 128};
    const int want[5] = {2, 3, 2, 3, 4};
    const int xg[5] = {0, 0, 1, 1, 1};
    for (int k = 0; k < 5; ++k) {
        const bool gx = g.kind == 1 || xg[k];
        if (g.kind == 1 && !xg[k]) continue;   // global-vector groups: listed once
        const size_t lo = gx ? g.tab_min : g.smem_min;
        // largest budget (in 4 KB steps) at which `want` CTAs fit on an SM
        for (size_t b = std::min(g.smem, (size_t)kSmemCap / want[k]); b >= 16 * 1024; b -= 4 * 1024) {
            if (b < lo) break;
            int occ = solve_variant_ctas_per_sm(g.dim, g.p0, g.p1, g.p2, g.mixed, gx, thr[k], b);
            if (occ >= want[k]) {
                c.push_back(TuneCfg{thr[k], b, occ, 0.f, xg[k], 1});
                break;
            }
        }
    }
    // a thread-block cluster of 2, 4 or 8 CTAs per slot (global-vector
    // variant, 512 threads, the full budget): several SMs on one patch, for
    // launches with fewer slots than SMs (one problem at a time, or the
    // largest patches of an uneven batch)
    if (g.clok && (g.kind == 0 || g.kind == 1)) {
        const size_t b = std::max(std::min(g.smem, (size_t)kSmemCap), g.tab_min);
        for (int cs = 2; cs <= 8; cs *= 2)
            if ((long long)g.s.size() * cs <= 2LL * sm_count()) c.push_back(TuneCfg{512, b, 1, 0.f, 1, cs});
    }
    return c;
}

// time each candidate on one V-cycle per slot (zero data, same work as a
// real launch) and keep the fastest; cached per launch shape
int tune(ieti_engine* E, MGroup& g, const std::vector<ietidp_handle*>& hs, long long* nlaunch) {
    g.cfg = TuneCfg{512, g.smem, 1, 0.f, 0, 1};
    if (g.kind >= 2 || !autotune_enabled()) return IETIDP_OK;
    TuneKey key{g.dim, g.p0, g.p1, g.p2, g.kind, g.mixed,
                (int)((g.s.size() + sm_count() - 1) / sm_count()),
                *std::max_element(g.cost.begin(), g.cost.end()), g.clok};
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            if (it->second.smem >= (it->second.xg ? g.tab_min : g.smem_min)) {
                g.cfg = it->second;
                g.cfg.smem = std::min(g.cfg.smem, g.smem);
            }
            return IETIDP_OK;
        }
    }
    std::vector<TuneCfg> cand = candidates(g);
    if (cand.size() > 1) {
        // scratch input/output vectors of every handle (zero)
        long long tot = 0;
        std::vector<long long> off(hs.size());
        for (size_t i = 0; i < hs.size(); ++i) {
            off[i] = tot;
            tot += hs[i]->prob->ntorn;
        }
        double* buf = nullptr;
        CU(cudaMallocAsync((void**)&buf, sizeof(double) * 2 * tot, E->st));
        CU(cudaMemsetAsync(buf, 0, sizeof(double) * 2 * tot, E->st));
        CHK(reserve(E, E->stT, hs.size(), g.s.size()));
        for (size_t i = 0; i < hs.size(); ++i) {
            SolveArgs a = ieti_solve_args(hs[i], MODE_VCYCLE, buf + off[i], buf + tot + off[i], 0.0, 0, nullptr);
            a.ncycles = 1;
            E->stT.h_args[i] = a;
        }
        std::copy(g.s.begin(), g.s.end(), E->stT.h_slots);
        CU(cudaMemcpyAsync(E->stT.d_args, E->stT.h_args, sizeof(SolveArgs) * hs.size(), cudaMemcpyHostToDevice,
                           E->st));
        CU(cudaMemcpyAsync(E->stT.d_slots, E->stT.h_slots, sizeof(SlotDesc) * g.s.size(), cudaMemcpyHostToDevice,
                           E->st));
        SolveArgs a0 = E->stT.h_args[0];
        a0.batch = E->stT.d_args;
        a0.slots = E->stT.d_slots;
        a0.nslots = (int)g.s.size();
        a0.mixed = g.mixed;
        float best = 1e30f;
        size_t bi = 0;
        for (size_t c = 0; c < cand.size(); ++c) {
            cudaError_t e = launch_cfg(a0, g, cand[c], E->st);   // warm-up
            if (e == cudaSuccess) {
                cudaEventRecord(E->t0, E->st);
                e = launch_cfg(a0, g, cand[c], E->st);
                cudaEventRecord(E->t1, E->st);
            }
            *nlaunch += 2;
            if (e != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            CU(cudaEventSynchronize(E->t1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, E->t0, E->t1);
            cand[c].ms = ms;
            if (ms < best) {
                best = ms;
                bi = c;
            }
        }
        CU(cudaFreeAsync(buf, E->st));
        g.cfg = cand[bi];
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = g.cfg;
    return IETIDP_OK;
}

// one local-solve stage prepared for launch: every item's slots, merged per
// kernel specialisation (longest patches first), each group's launch shape
// tuned, and the kernel arguments and slot lists as they go to the device
struct MergedPrep {
    std::vector<MGroup> groups;
    std::vector<SolveArgs> args;    // per item
    std::vector<SlotDesc> slots;    // the groups' slots, group after group
};

int merged_prepare(ieti_engine* E, std::vector<std::pair<ietidp_handle*, SolveArgs>>& items, MergedPrep& MP,
                   long long* nlaunch) {
    MP = MergedPrep{};
    if (items.empty()) return IETIDP_OK;
    std::map<std::tuple<int, int, int, int, int, int>, MGroup> by;
    for (size_t i = 0; i < items.size(); ++i) {
        ietidp_handle* h = items[i].first;
        const int mixed = h->opt.precision == IETIDP_PREC_MIXED;
        const bool direct = items[i].second.mode == MODE_NEUMANN_DIRECT;
        for (const SlotGroup& sg : h->gpatch) {
            // kind 3: direct Neumann solves (one kernel for every degree)
            const int kind = direct ? 3 : (sg.generic ? 2 : (sg.xg ? 1 : 0));
            MGroup& m = direct ? by[std::make_tuple(0, 0, 0, 0, 3, mixed)]
                               : by[std::make_tuple(sg.dim, sg.p0, sg.p1, sg.p2, kind, mixed)];
            m.dim = sg.dim;
            m.p0 = sg.p0;
            m.p1 = sg.p1;
            m.p2 = sg.p2;
            m.kind = kind;
            m.mixed = mixed;
            m.smem = std::max(m.smem, direct ? h->direct_smem : sg.smem);
            m.max_bw = std::max(m.max_bw, h->max_bw);
            for (SlotDesc sd : sg.hs) {
                sd.handle = (int)i;
                const PatchDesc& P = h->pd[sd.patch];
                m.s.push_back(sd);
                m.cost.push_back((long long)P.n * P.lev[P.L - 1].S);
                m.smem_min = std::max(m.smem_min, kind == 1 ? solve_smem_tables(P) : solve_smem_min(P, mixed));
                m.tab_min = std::max(m.tab_min, solve_smem_tables(P));
            }
        }
    }
    std::vector<ietidp_handle*> hs(items.size());
    for (size_t i = 0; i < items.size(); ++i) hs[i] = items[i].first;
    // cluster launches serve the solve-phase modes only (the kernel refuses
    // the others); IETIDP_CLUSTERS=0 keeps one CTA per slot, IETIDP_CLUSTERS=
    // 2, 4 or 8 forces clusters of that size on every group that can take
    // them (tests of the cluster path)
    int clok = 1, cforce = 0;
    {
        const char* ce = std::getenv("IETIDP_CLUSTERS");
        if (ce && ce[0] == '0') clok = 0;
        if (ce && (ce[0] == '2' || ce[0] == '4' || ce[0] == '8')) cforce = ce[0] - '0';
    }
    for (const auto& it : items) {
        const int md = it.second.mode;
        if (!(md == MODE_NEUMANN || md == MODE_SCHUR || md == MODE_VCYCLE || md == MODE_VCYCLE_DIR)) clok = 0;
    }
    for (auto& kv : by) {
        MGroup& m = kv.second;
        m.clok = clok;
        // longest patches first, so that uneven batches finish together
        std::vector<size_t> ord(m.s.size());
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](size_t x, size_t y) { return m.cost[x] > m.cost[y]; });
        std::vector<SlotDesc> s2(m.s.size());
        std::vector<long long> c2(m.s.size());
        for (size_t k = 0; k < ord.size(); ++k) {
            s2[k] = m.s[ord[k]];
            c2[k] = m.cost[ord[k]];
        }
        m.s.swap(s2);
        m.cost.swap(c2);
        CHK(tune(E, m, hs, nlaunch));
        if (cforce && clok && (m.kind == 0 || m.kind == 1))
            m.cfg = TuneCfg{512, std::max(std::min(m.smem, (size_t)kSmemCap), m.tab_min), 1, 0.f, 1, cforce};
        MP.slots.insert(MP.slots.end(), m.s.begin(), m.s.end());
        MP.groups.push_back(std::move(m));
    }
    for (auto& it : items) MP.args.push_back(it.second);
    return IETIDP_OK;
}

// the launches of a prepared stage (groups of several specialisations run
// concurrently on side streams); d_args / d_slots hold MP.args / MP.slots on
// the device; tspan (or null): [first CTA start, last CTA end] in
// globaltimer nanoseconds, widened by every launch of the stage
int merged_issue(ieti_engine* E, const MergedPrep& MP, const SolveArgs* d_args, const SlotDesc* d_slots,
                 unsigned long long* tspan, long long* nlaunch) {
    if (MP.groups.empty()) return IETIDP_OK;
    SolveArgs a0 = MP.args[0];
    a0.batch = d_args;
    a0.tspan = tspan;
    const bool multi = MP.groups.size() > 1;
    if (multi) {
        CHK(ensure_side(E, MP.groups.size()));
        CU(cudaEventRecord(E->fork, E->st));
    }
    size_t off = 0, gi = 0;
    for (const MGroup& m : MP.groups) {
        a0.slots = d_slots + off;
        a0.nslots = (int)m.s.size();
        a0.mixed = m.mixed;
        off += m.s.size();
        cudaStream_t s = E->st;
        if (multi) {
            s = E->side[gi % E->side.size()];
            CU(cudaStreamWaitEvent(s, E->fork, 0));
        }
        cudaError_t e = launch_cfg(a0, m, m.cfg, s);
        *nlaunch += 1;
        if (e != cudaSuccess) return fail(IETIDP_E_CUDA, std::string("local solve kernel: ") + cudaGetErrorString(e));
        ++gi;
    }
    if (multi) {
        for (size_t i = 0; i < std::min(MP.groups.size(), E->side.size()); ++i) {
            CU(cudaEventRecord(E->join[i], E->side[i]));
            CU(cudaStreamWaitEvent(E->st, E->join[i], 0));
        }
    }
    return IETIDP_OK;
}

// copy a prepared stage's arguments through the pinned staging buffers
int merged_stage_copy(ieti_engine* E, Staging& S, const MergedPrep& MP) {
    CHK(reserve(E, S, MP.args.size(), MP.slots.size()));
    std::copy(MP.args.begin(), MP.args.end(), S.h_args);
    std::copy(MP.slots.begin(), MP.slots.end(), S.h_slots);
    CU(cudaMemcpyAsync(S.d_args, S.h_args, sizeof(SolveArgs) * MP.args.size(), cudaMemcpyHostToDevice, E->st));
    CU(cudaMemcpyAsync(S.d_slots, S.h_slots, sizeof(SlotDesc) * MP.slots.size(), cudaMemcpyHostToDevice, E->st));
    return IETIDP_OK;
}

// one local-solve stage, eager: prepare, copy, launch
int merged_launch(ieti_engine* E, Staging& S, std::vector<std::pair<ietidp_handle*, SolveArgs>>& items,
                  long long* nlaunch) {
    if (items.empty()) return IETIDP_OK;
    MergedPrep MP;
    CHK(merged_prepare(E, items, MP, nlaunch));
    CHK(merged_stage_copy(E, S, MP));
    return merged_issue(E, MP, S.d_args, S.d_slots, nullptr, nlaunch);
}

double lanczos_kappa(const std::vector<double>& al, const std::vector<double>& be) {
    int n = (int)al.size();
    if (n == 0) return 1.0;
    // eigenvalues of the Lanczos tridiagonal matrix of the CG coefficients by
    // bisection on Sturm sequence counts
    std::vector<double> dd(n), ee(n, 0.0);
    for (int k = 0; k < n; ++k) {
        dd[k] = 1.0 / al[k] + (k > 0 ? be[k - 1] / al[k - 1] : 0.0);
        if (k < n - 1 && k < (int)be.size()) ee[k] = std::sqrt(std::max(0.0, be[k])) / al[k];
    }
    double lo = 1e300, hi = -1e300;
    for (int k = 0; k < n; ++k) {
        double rad = std::fabs(k > 0 ? ee[k - 1] : 0.0) + std::fabs(ee[k]);
        lo = std::min(lo, dd[k] - rad);
        hi = std::max(hi, dd[k] + rad);
    }
    auto count_below = [&](double x) {
        int c = 0;
        double q = 1.0;
        for (int k = 0; k < n; ++k) {
            double e2 = k > 0 ? ee[k - 1] * ee[k - 1] : 0.0;
            q = dd[k] - x - (k > 0 ? e2 / q : 0.0);
            if (q == 0.0) q = -1e-300;
            if (q < 0) ++c;
        }
        return c;
    };
    auto eig = [&](int idx) {
        double a = lo, b = hi;
        for (int it = 0; it < 200; ++it) {
            double mid = 0.5 * (a + b);
            if (count_below(mid) > idx) b = mid;
            else a = mid;
        }
        return 0.5 * (a + b);
    };
    return eig(n - 1) / eig(0);
}

constexpr int kRb = 16;   // read-back doubles per job before its CG history

// small per-job launches count for the job and for the process-wide counter
void count(EngineJob& j, long long k) {
    j.S.launches += k;
    ieti_host::g_kernel_launches += k;
}

size_t rb_stride(const ietidp_handle* h) { return kRb + 2 * (size_t)(h->opt.maxit_outer + 1); }

// small per-job launches (one job, engine stream)
#define LCHK(x)                                                                 \
    do {                                                                        \
        cudaError_t e_ = (x);                                                   \
        if (e_ != cudaSuccess) return fail(IETIDP_E_CUDA, cudaGetErrorString(e_)); \
    } while (0)

int primal(ietidp_handle* h, const double* g, cudaStream_t st, EngineJob& j) {
    LCHK(launch_primal_restrict(h->d_pd, h->nrows, h->crow_patch, h->crow_local, h->phi, g, h->rloc, st));
    LCHK(launch_coarse_solve(h->npi, h->nrows, h->crow_glob, h->gptr, h->glist, h->Linv, h->rloc, h->upi, h->uloc,
                             st));
    count(j, (h->nrows > 0) + (h->npi > 0));
    return IETIDP_OK;
}

void finish(EngineJob& j) {
    const ietidp_handle* h = j.h;
    auto t1 = std::chrono::steady_clock::now();
    ietidp_stats& S = j.S;
    S.outer_it = j.it;
    S.converged = j.conv && !(j.flags & IETI_FLAG_NOT_CONVERGED);
    S.kappa = lanczos_kappa(j.al, j.be);
    S.vcycles = j.vs[0];
    S.vcycle_dofs = j.vs[1];
    S.inner_its = j.vs[2];
    if (j.vs[4] > 0) {
        S.inner_it_avg = (double)j.vs[2] / (double)j.vs[4];
        S.inner_it_max = (int)j.vs[3];
    }
    S.basis_it_avg = h->basis_it_avg;
    S.basis_it_max = h->basis_it_max;
    S.t_setup_ms = h->t_setup_ms;
    S.t_solve_ms = std::chrono::duration<double, std::milli>(t1 - j.t0).count();
    if (j.rc == IETIDP_OK) {
        if (j.flags & IETI_FLAG_BREAKDOWN) {
            j.rc = IETIDP_E_BREAKDOWN;
            j.err = "CG breakdown in a local solve";
        } else if (!S.converged) {
            j.rc = IETIDP_E_NOT_CONVERGED;
            j.err = "solver did not converge";
        }
    }
    j.phase = EngineJob::DONE;
}

}  // namespace

// ---------------------------------------------------------------------------
// engine API (engine.h)
// ---------------------------------------------------------------------------
int ieti_engine_create(cudaStream_t st, ieti_engine** out) {
    auto* E = new ieti_engine();
    E->st = st;
    cudaError_t e = cudaEventCreateWithFlags(&E->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreate(&E->e0);
    if (e == cudaSuccess) e = cudaEventCreate(&E->e1);
    if (e == cudaSuccess) e = cudaEventCreate(&E->t0);
    if (e == cudaSuccess) e = cudaEventCreate(&E->t1);
    if (e == cudaSuccess) e = cudaMalloc((void**)&E->d_span, 2 * sizeof(unsigned long long));
    if (e != cudaSuccess) {
        delete E;
        return fail(IETIDP_E_CUDA, std::string("engine events: ") + cudaGetErrorString(e));
    }
    *out = E;
    return IETIDP_OK;
}

void ieti_engine_destroy(ieti_engine* E) {
    if (!E) return;
    cudaStreamSynchronize(E->st);
    clear_graphs(E);
    free_staging(E, E->stA);
    free_staging(E, E->stB);
    free_staging(E, E->stT);
    cudaStreamSynchronize(E->st);
    if (E->h_rb) cudaFreeHost(E->h_rb);
    if (E->d_span) cudaFree(E->d_span);
    for (auto s : E->side) cudaStreamDestroy(s);
    for (auto ev : E->join) cudaEventDestroy(ev);
    if (E->fork) cudaEventDestroy(E->fork);
    if (E->e0) cudaEventDestroy(E->e0);
    if (E->e1) cudaEventDestroy(E->e1);
    if (E->t0) cudaEventDestroy(E->t0);
    if (E->t1) cudaEventDestroy(E->t1);
    if (E->own_stream) cudaStreamDestroy(E->st);
    delete E;
}

cudaStream_t ieti_engine_stream(const ieti_engine* E) { return E->st; }

void ieti_engine_job_init(EngineJob& j, ietidp_handle* h, const double* f, double* u) {
    j = EngineJob{};
    j.h = h;
    j.f = f ? f : h->prob->f;
    j.u = u;
    j.t0 = std::chrono::steady_clock::now();
}

namespace {

// The small per-job launches of a tick stage (before and after its merged
// launch) are enqueued by these segment functions; the merged launches
// themselves run eagerly between them (timed with the engine's events).
//   segment 0: stage A inputs (B^T p, primal restriction / coarse solve, ...)
//   segment 1: stage A outputs (B u, outer CG step, read-back)
//   segment 2: stage B input (B_D^T r)
//   segment 3: stage B outputs (B_D w, next search direction)
bool in_A(const EngineJob* j) {
    return j->phase == EngineJob::INIT || j->phase == EngineJob::ITER || j->phase == EngineJob::RECOVER;
}
bool in_B(const EngineJob* j) { return j->phase == EngineJob::PRECF || j->phase == EngineJob::PREC; }

int segment(ieti_engine* E, int seg, std::vector<EngineJob*>& jobs, const std::vector<size_t>& rbo) {
    cudaStream_t st = E->st;
    for (size_t i = 0; i < jobs.size(); ++i) {
        EngineJob* j = jobs[i];
        ietidp_handle* h = j->h;
        if (seg == 0) {
            if (j->phase == EngineJob::INIT) {
                CU(cudaMemsetAsync(h->flags, 0, sizeof(int), st));
                CU(cudaMemsetAsync(h->vst, 0, sizeof(long long) * 8, st));
                CHK(primal(h, j->f, st, *j));
            } else if (j->phase == EngineJob::ITER) {
                LCHK(launch_bt(h->dual, h->p, h->gF, 0, st));
                count(*j, 1);
                CHK(primal(h, h->gF, st, *j));
            } else if (j->phase == EngineJob::RECOVER) {
                LCHK(launch_bt(h->dual, h->lam, h->tmp, 0, st));
                LCHK(launch_axpy_torn(h->prob->ntorn, j->f, -1.0, h->tmp, h->gR, st));
                count(*j, 2);
                CHK(primal(h, h->gR, st, *j));
            }
        } else if (seg == 1) {
            double* rb = E->h_rb + rbo[i];
            if (j->phase == EngineJob::INIT) {
                if (h->nlam > 0) {
                    LCHK(launch_b(h->dual, j->u, h->d, 0, st));
                    LCHK(launch_jump_scale(h->dual, j->u, h->scal, st));
                    LCHK(launch_outer_init(h->nlam, h->d, h->lam, h->r, h->state, st));
                    count(*j, 3);
                    CU(cudaMemcpyAsync(rb, h->state + 5, sizeof(double), cudaMemcpyDeviceToHost, st));
                    CU(cudaMemcpyAsync(rb + 1, h->scal, sizeof(double), cudaMemcpyDeviceToHost, st));
                }
                CU(cudaMemcpyAsync(rb + 2, h->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
                CU(cudaMemcpyAsync(rb + 8, h->vst, sizeof(long long) * 8, cudaMemcpyDeviceToHost, st));
            } else if (j->phase == EngineJob::ITER) {
                LCHK(launch_b(h->dual, h->uF, h->q, 0, st));
                LCHK(launch_outer_step1(h->nlam, h->p, h->q, h->lam, h->r, h->state, h->hist, -1, st));
                count(*j, 2);
                CU(cudaMemcpyAsync(rb, h->state + 4, sizeof(double), cudaMemcpyDeviceToHost, st));
            } else if (j->phase == EngineJob::RECOVER) {
                CU(cudaMemcpyAsync(rb + 2, h->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
                CU(cudaMemcpyAsync(rb + 8, h->vst, sizeof(long long) * 8, cudaMemcpyDeviceToHost, st));
                if (j->it > 0)
                    CU(cudaMemcpyAsync(rb + kRb, h->hist, sizeof(double) * 2 * j->it, cudaMemcpyDeviceToHost, st));
            }
        } else if (seg == 2) {
            if (!in_B(j)) continue;
            LCHK(launch_bt(h->dual, h->r, h->vS, 1, st));
            count(*j, 1);
        } else {
            if (!in_B(j)) continue;
            LCHK(launch_b(h->dual, h->wS, h->z, 1, st));
            if (j->phase == EngineJob::PRECF) {
                LCHK(launch_outer_first(h->nlam, h->r, h->z, h->p, h->state, st));
            } else {
                LCHK(launch_outer_step2(h->nlam, h->r, h->z, h->p, h->state, h->hist, -1, st));
            }
            count(*j, 2);
        }
    }
    return IETIDP_OK;
}

// ---------------------------------------------------------------------------
// CUDA graphs of the per-job launch segments: a segment whose launch sequence
// repeats (same jobs, same phases: every steady-state outer iteration) is
// captured on its second occurrence and replayed from then on as one graph
// launch.  IETIDP_GRAPHS=0 disables capture.
// ---------------------------------------------------------------------------
bool graphs_enabled() {
    const char* e = std::getenv("IETIDP_GRAPHS");
    return !(e && e[0] == '0');
}

std::vector<uintptr_t> segment_key(ieti_engine* E, int seg, const std::vector<EngineJob*>& jobs) {
    std::vector<uintptr_t> k;
    k.push_back((uintptr_t)seg);
    k.push_back((uintptr_t)E->h_rb);
    for (EngineJob* j : jobs) {
        k.push_back((uintptr_t)j->h);
        k.push_back((uintptr_t)j->h->serial);   // the address alone may be a recycled handle's
        k.push_back((uintptr_t)j->phase);
        k.push_back((uintptr_t)j->f);
        k.push_back((uintptr_t)j->u);
        k.push_back((uintptr_t)(j->phase == EngineJob::RECOVER ? j->it : 0));
        k.push_back((uintptr_t)j->fresh);
    }
    return k;
}

int staged_fn(ieti_engine* E, int seg, std::vector<EngineJob*>& jobs, const std::function<int()>& eager) {
    if (!graphs_enabled()) return eager();
    const auto key = segment_key(E, seg, jobs);
    auto it = E->graphs.find(key);
    if (it != E->graphs.end() && it->second->exec) {
        GraphEntry& G = *it->second;
        CU(cudaGraphLaunch(G.exec, E->st));
        for (size_t i = 0; i < jobs.size(); ++i) jobs[i]->S.launches += G.dl[i];
        ieti_host::g_kernel_launches += G.total;
        return IETIDP_OK;
    }
    // occurrence counts of keys not captured yet: a server whose job mix keeps
    // changing sees most keys once, so the table is bounded
    if (it == E->graphs.end() && E->seen.size() >= 4096) E->seen.clear();
    if (it != E->graphs.end() || ++E->seen[key] < 2) return eager();
    if (E->graphs.size() >= 256) clear_graphs(E);
    auto G = std::make_unique<GraphEntry>();
    std::vector<long long> l0(jobs.size());
    for (size_t i = 0; i < jobs.size(); ++i) l0[i] = jobs[i]->S.launches;
    const long long g0 = ieti_host::g_kernel_launches.load();
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(E->st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGetLastError();
        E->graphs[key] = std::move(G);   // not capturable: eager from now on
        return eager();
    }
    int rc = eager();
    cudaError_t e = cudaStreamEndCapture(E->st, &graph);
    if (rc == IETIDP_OK && e == cudaSuccess && graph) e = cudaGraphInstantiate(&G->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (rc != IETIDP_OK || e != cudaSuccess || !G->exec) {
        cudaGetLastError();
        if (G->exec) cudaGraphExecDestroy(G->exec);
        G->exec = nullptr;
        for (size_t i = 0; i < jobs.size(); ++i) jobs[i]->S.launches = l0[i];
        ieti_host::g_kernel_launches = g0;
        E->graphs[key] = std::move(G);
        return eager();
    }
    G->dl.resize(jobs.size());
    for (size_t i = 0; i < jobs.size(); ++i) G->dl[i] = jobs[i]->S.launches - l0[i];
    G->total = ieti_host::g_kernel_launches.load() - g0;
    CU(cudaGraphLaunch(G->exec, E->st));
    E->graphs[key] = std::move(G);
    return IETIDP_OK;
}

// the items of merged stage A (Neumann solves) or B (Dirichlet problems)
void stage_items(int stage, std::vector<EngineJob*>& jobs, std::vector<std::pair<ietidp_handle*, SolveArgs>>& items,
                 std::vector<size_t>& in) {
    for (size_t i = 0; i < jobs.size(); ++i) {
        EngineJob* j = jobs[i];
        ietidp_handle* h = j->h;
        if (stage == 0) {
            if (j->phase == EngineJob::INIT)
                items.emplace_back(h, ieti_solve_args(h, MODE_NEUMANN, j->f, j->u, h->opt.tol_inner,
                                                      h->opt.maxit_inner, h->vst));
            else if (j->phase == EngineJob::ITER)
                items.emplace_back(h, ieti_solve_args(h, MODE_NEUMANN, h->gF, h->uF, h->opt.tol_inner,
                                                      h->opt.maxit_inner, h->vst));
            else if (j->phase == EngineJob::RECOVER)
                items.emplace_back(h, ieti_solve_args(h, MODE_NEUMANN, h->gR, j->u, h->opt.tol_inner,
                                                      h->opt.maxit_inner, h->vst));
            else
                continue;
        } else {
            if (!in_B(j)) continue;
            items.emplace_back(h, ieti_solve_args(h, MODE_SCHUR, h->vS, h->wS, 0.0, 0, h->vst));
        }
        in.push_back(i);
    }
}

// Half a tick as one unit: the per-job launches before a merged stage, the
// merged launch of every job's local solves (one per kernel specialisation)
// and the per-job launches after it.  Its launch sequence repeats for the
// same jobs in the same phases (every steady-state outer iteration), so it is
// captured on its second occurrence and replayed from then on as ONE graph
// launch.  The graph owns a device copy of the merged launch's arguments and
// slot lists (the pinned staging buffers are rewritten by other stages).
// Stage A's duration comes from the kernels themselves: every CTA widens a
// [start, end] globaltimer span, which the graph resets before the launch and
// copies into the read-back area (at double offset `spanoff`) after it.
int half_tick(ieti_engine* E, int stage, std::vector<EngineJob*>& jobs, const std::vector<size_t>& rbo,
              size_t spanoff) {
    std::vector<std::pair<ietidp_handle*, SolveArgs>> items;
    std::vector<size_t> in;
    stage_items(stage, jobs, items, in);
    MergedPrep MP;
    long long ntune = 0;
    CHK(merged_prepare(E, items, MP, &ntune));   // autotuning (eager, before any capture)
    ieti_host::g_kernel_launches += ntune;
    const int segA = stage == 0 ? 0 : 2, segB = stage == 0 ? 1 : 3;
    cudaStream_t st = E->st;
    auto body = [&](const SolveArgs* da, const SlotDesc* ds) -> int {
        CHK(segment(E, segA, jobs, rbo));
        if (!MP.groups.empty()) {
            if (stage == 0) {
                CU(cudaMemsetAsync(E->d_span, 0xff, sizeof(unsigned long long), st));
                CU(cudaMemsetAsync(E->d_span + 1, 0, sizeof(unsigned long long), st));
            }
            long long nl = 0;
            CHK(merged_issue(E, MP, da, ds, stage == 0 ? E->d_span : nullptr, &nl));
            if (stage == 0)
                CU(cudaMemcpyAsync(E->h_rb + spanoff, E->d_span, 2 * sizeof(unsigned long long),
                                   cudaMemcpyDeviceToHost, st));
            ieti_host::g_kernel_launches += nl;
            for (size_t i : in) {
                jobs[i]->S.launches += nl;
                if (stage == 0) jobs[i]->S.neumann_launches += 1;
            }
        }
        return segment(E, segB, jobs, rbo);
    };
    Staging& S = stage == 0 ? E->stA : E->stB;
    auto eager = [&]() -> int {
        if (!MP.groups.empty()) CHK(merged_stage_copy(E, S, MP));
        return body(S.d_args, S.d_slots);
    };
    if (!graphs_enabled()) return eager();
    const auto key = segment_key(E, 10 + stage, jobs);
    auto it = E->graphs.find(key);
    if (it != E->graphs.end() && it->second->exec) {
        GraphEntry& G = *it->second;
        CU(cudaGraphLaunch(G.exec, st));
        for (size_t i = 0; i < jobs.size(); ++i) {
            jobs[i]->S.launches += G.dl[i];
            jobs[i]->S.neumann_launches += G.dn[i];
        }
        ieti_host::g_kernel_launches += G.total;
        return IETIDP_OK;
    }
    if (it == E->graphs.end() && E->seen.size() >= 4096) E->seen.clear();
    if (it != E->graphs.end() || ++E->seen[key] < 2) return eager();
    if (E->graphs.size() >= 256) clear_graphs(E);
    auto G = std::make_unique<GraphEntry>();
    if (!MP.groups.empty()) {
        // before the capture: the graph's own argument and slot buffers
        CU(cudaStreamSynchronize(st));
        CU(cudaMalloc(&G->d_args, sizeof(SolveArgs) * MP.args.size()));
        CU(cudaMalloc(&G->d_slots, sizeof(SlotDesc) * MP.slots.size()));
        CU(cudaMemcpy(G->d_args, MP.args.data(), sizeof(SolveArgs) * MP.args.size(), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(G->d_slots, MP.slots.data(), sizeof(SlotDesc) * MP.slots.size(), cudaMemcpyHostToDevice));
    }
    std::vector<long long> l0(jobs.size()), n0(jobs.size());
    for (size_t i = 0; i < jobs.size(); ++i) {
        l0[i] = jobs[i]->S.launches;
        n0[i] = jobs[i]->S.neumann_launches;
    }
    const long long g0 = ieti_host::g_kernel_launches.load();
    auto give_up = [&]() -> int {
        cudaGetLastError();
        if (G->exec) cudaGraphExecDestroy(G->exec);
        G->exec = nullptr;
        for (size_t i = 0; i < jobs.size(); ++i) {
            jobs[i]->S.launches = l0[i];
            jobs[i]->S.neumann_launches = n0[i];
        }
        ieti_host::g_kernel_launches = g0;
        E->graphs[key] = std::move(G);   // not capturable: eager from now on (the buffers stay owned)
        return eager();
    };
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) return give_up();
    int rc = body((const SolveArgs*)G->d_args, (const SlotDesc*)G->d_slots);
    cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (rc == IETIDP_OK && ce == cudaSuccess && graph) ce = cudaGraphInstantiate(&G->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (rc != IETIDP_OK || ce != cudaSuccess || !G->exec) return give_up();
    G->dl.resize(jobs.size());
    G->dn.resize(jobs.size());
    for (size_t i = 0; i < jobs.size(); ++i) {
        G->dl[i] = jobs[i]->S.launches - l0[i];
        G->dn[i] = jobs[i]->S.neumann_launches - n0[i];
    }
    G->total = ieti_host::g_kernel_launches.load() - g0;
    CU(cudaGraphLaunch(G->exec, st));
    E->graphs[key] = std::move(G);
    return IETIDP_OK;
}

}  // namespace

int ieti_engine_staged(ieti_engine* E, int seg, std::vector<EngineJob*>& jobs, const std::function<int()>& eager) {
    return staged_fn(E, seg, jobs, eager);
}

int ieti_engine_tick(ieti_engine* E, std::vector<EngineJob*>& jobs) {
    cudaStream_t st = E->st;
    // read-back area
    size_t need = 0;
    std::vector<size_t> rbo(jobs.size());
    for (size_t i = 0; i < jobs.size(); ++i) {
        rbo[i] = need;
        need += rb_stride(jobs[i]->h);
    }
    const size_t spanoff = need;   // [start, end] of merged stage A (globaltimer ns)
    need += 2;
    if (need > E->cap_rb) {
        CU(cudaStreamSynchronize(st));
        if (E->h_rb) cudaFreeHost(E->h_rb);
        E->h_rb = nullptr;
        E->cap_rb = 0;
        CU(cudaMallocHost((void**)&E->h_rb, sizeof(double) * std::max(need, (size_t)256)));
        E->cap_rb = std::max(need, (size_t)256);
        clear_graphs(E);   // captured read-backs point at the old buffer
    }
    bool anyA = false;
    for (EngineJob* j : jobs) anyA = anyA || in_A(j);
    CHK(half_tick(E, 0, jobs, rbo, spanoff));
    CU(cudaStreamSynchronize(st));
    float msA = 0.f;
    if (anyA) {
        unsigned long long sp[2];
        std::memcpy(sp, E->h_rb + spanoff, sizeof(sp));
        if (sp[1] > sp[0]) msA = (float)((double)(sp[1] - sp[0]) * 1e-6);
    }
    for (EngineJob* j : jobs)
        if (j->phase == EngineJob::INIT || j->phase == EngineJob::ITER || j->phase == EngineJob::RECOVER)
            j->S.neumann_ms += msA;
    // ---- host decisions --------------------------------------------------------
    for (size_t i = 0; i < jobs.size(); ++i) {
        EngineJob* j = jobs[i];
        ietidp_handle* h = j->h;
        const double* rb = E->h_rb + rbo[i];
        if (j->phase == EngineJob::INIT || j->phase == EngineJob::RECOVER) {
            std::memcpy(&j->flags, rb + 2, sizeof(int));
            std::memcpy(j->vs, rb + 8, sizeof(long long) * 8);
        }
        if (j->phase == EngineJob::INIT) {
            if (h->nlam == 0) {
                finish(*j);
                continue;
            }
            j->dd = rb[0];
            const double sc2 = rb[1];
            if (!std::isfinite(j->dd)) {
                j->rc = IETIDP_E_NONFINITE;
                j->err = "non-finite dual right-hand side";
                finish(*j);
                continue;
            }
            j->S.d_norm = std::sqrt(j->dd);
            j->S.d_scale = std::sqrt(sc2);
            const double tol = h->opt.tol_outer;
            if (j->S.d_norm <= tol * j->S.d_scale) {
                // the jump of u0 vanishes to rounding: lambda = 0
                j->conv = true;
                finish(*j);
                continue;
            }
            j->conv = false;
            j->thr2 = tol * tol * j->dd;
            j->phase = EngineJob::PRECF;
        } else if (j->phase == EngineJob::ITER) {
            const double rr = rb[0];
            if (!std::isfinite(rr)) {
                j->rc = IETIDP_E_NONFINITE;
                j->err = "non-finite dual residual";
                finish(*j);
                continue;
            }
            j->S.rel_res = std::sqrt(rr / j->dd);
            if (rr <= j->thr2) {
                j->conv = true;
                j->phase = EngineJob::RECOVER;
            } else if (j->it >= h->opt.maxit_outer) {
                j->phase = EngineJob::RECOVER;
            } else {
                j->phase = EngineJob::PREC;
            }
        } else if (j->phase == EngineJob::RECOVER) {
            for (int k = 0; k < j->it; ++k) {
                j->al.push_back(rb[kRb + 2 * k]);
                if (k < j->it - 1) j->be.push_back(rb[kRb + 2 * k + 1]);
            }
            finish(*j);
        }
    }
    CHK(half_tick(E, 1, jobs, rbo, spanoff));
    for (EngineJob* j : jobs) {
        if (j->phase == EngineJob::PRECF) {
            j->it = 1;
            j->phase = EngineJob::ITER;
        } else if (j->phase == EngineJob::PREC) {
            j->it += 1;
            j->phase = EngineJob::ITER;
        }
    }
    return IETIDP_OK;
}

int ieti_engine_merged(ieti_engine* E, int stage, std::vector<std::pair<ietidp_handle*, SolveArgs>>& items,
                       long long* nlaunch, bool timed) {
    if (timed) CU(cudaEventRecord(E->e0, E->st));
    CHK(merged_launch(E, stage == 0 ? E->stA : E->stB, items, nlaunch));
    if (timed) CU(cudaEventRecord(E->e1, E->st));
    return IETIDP_OK;
}

int ieti_engine_readback(ieti_engine* E, size_t n, double** out) {
    if (n > E->cap_rb) {
        CU(cudaStreamSynchronize(E->st));
        if (E->h_rb) cudaFreeHost(E->h_rb);
        E->h_rb = nullptr;
        E->cap_rb = 0;
        const size_t cap = std::max(n, (size_t)256);
        CU(cudaMallocHost((void**)&E->h_rb, sizeof(double) * cap));
        E->cap_rb = cap;
    }
    *out = E->h_rb;
    return IETIDP_OK;
}

float ieti_engine_timed_ms(ieti_engine* E) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, E->e0, E->e1) != cudaSuccess) {
        cudaGetLastError();
        return 0.f;
    }
    return ms;
}

int ieti_engine_run(ieti_engine* E, std::vector<EngineJob*>& jobs) {
    for (;;) {
        bool any = false;
        for (EngineJob* j : jobs) any = any || j->phase != EngineJob::DONE;
        if (!any) return IETIDP_OK;
        std::vector<EngineJob*> live;
        for (EngineJob* j : jobs)
            if (j->phase != EngineJob::DONE) live.push_back(j);
        CHK(ieti_engine_tick(E, live));
    }
}

extern "C" int ietidp_autotune_table(int* out, int max_entries) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    int n = 0;
    for (const auto& kv : g_tune) {
        if (out && n < max_entries) {
            int* o = out + 12 * n;
            o[0] = kv.first.dim;
            o[1] = kv.first.p0;
            o[2] = kv.first.p1;
            o[3] = kv.first.p2;
            o[4] = kv.first.kind;
            o[5] = kv.first.mixed;
            o[6] = kv.first.waves;
            o[7] = kv.second.threads;
            o[8] = (int)kv.second.smem;
            o[9] = kv.second.ctas_per_sm;
            o[10] = kv.first.kind == 1 || kv.second.xg;
            o[11] = std::max(1, kv.second.csize);
        }
        ++n;
    }
    return n;
}

// ---------------------------------------------------------------------------
// public solve entry points
// ---------------------------------------------------------------------------
namespace {

// the handle's engine works on a non-blocking stream of its own (the
// caller's stream may be the legacy default stream, which cannot be
// captured into a graph); run_jobs joins it with the handles' streams
int engine_of(ietidp_handle* h, ieti_engine** E) {
    if (!h->engine) {
        cudaStream_t s;
        CU(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        int rc = ieti_engine_create(s, &h->engine);
        if (rc != IETIDP_OK) {
            cudaStreamDestroy(s);
            return rc;
        }
        h->engine->own_stream = true;
    }
    *E = h->engine;
    return IETIDP_OK;
}

// run jobs on the engine of hs[0]; the other handles' streams are joined
// before and after, so work the caller queued on them stays ordered
int run_jobs(ietidp_handle* const* hs, int n, std::vector<EngineJob>& jobs, bool host,
             const double* const* f_host, double* const* u_host) {
    ieti_engine* E = nullptr;
    CHK(engine_of(hs[0], &E));
    cudaStream_t st = E->st;
    std::vector<cudaEvent_t> evs;
    auto cleanup = [&]() {
        for (auto ev : evs) cudaEventDestroy(ev);
    };
    // the engine's stream waits for work queued on every handle's stream
    for (int i = 0; i < n; ++i) {
        if (hs[i]->st == st) continue;
        bool dup = false;
        for (int k = 0; k < i; ++k) dup = dup || hs[k]->st == hs[i]->st;
        if (dup) continue;
        cudaEvent_t ev;
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) {
            evs.push_back(ev);
            e = cudaEventRecord(ev, hs[i]->st);
        }
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
        if (e != cudaSuccess) {
            cleanup();
            return fail(IETIDP_E_CUDA, std::string("stream join: ") + cudaGetErrorString(e));
        }
    }
    if (host)
        for (int i = 0; i < n; ++i)
            if (f_host && f_host[i]) {
                int rc = IETIDP_OK;
                cudaError_t e = cudaMemcpyAsync(hs[i]->fH, f_host[i], sizeof(double) * hs[i]->prob->ntorn,
                                                cudaMemcpyHostToDevice, st);
                if (e != cudaSuccess) rc = fail(IETIDP_E_CUDA, std::string("H2D: ") + cudaGetErrorString(e));
                if (rc != IETIDP_OK) {
                    cleanup();
                    return rc;
                }
            }
    std::vector<EngineJob*> ptr;
    for (auto& j : jobs) ptr.push_back(&j);
    const int method = hs[0]->opt.method;
    int rc = IETIDP_OK;
    for (int i = 1; i < n; ++i)
        if (hs[i]->opt.method != method) rc = fail(IETIDP_E_INVALID_ARG, "a batch mixes outer methods");
    if (rc == IETIDP_OK)
        rc = method == IETIDP_METHOD_SADDLE ? ieti_saddle_run(E, ptr) : ieti_engine_run(E, ptr);
    if (rc == IETIDP_OK && host) {
        for (int i = 0; i < n; ++i) {
            if (jobs[i].rc != IETIDP_OK && jobs[i].rc != IETIDP_E_NOT_CONVERGED) continue;
            cudaError_t e = cudaMemcpyAsync(u_host[i], hs[i]->uH, sizeof(double) * hs[i]->prob->ntorn,
                                            cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) {
                rc = fail(IETIDP_E_CUDA, std::string("D2H: ") + cudaGetErrorString(e));
                break;
            }
        }
        if (rc == IETIDP_OK) {
            cudaError_t e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rc = fail(IETIDP_E_CUDA, cudaGetErrorString(e));
        }
    }
    // later work on the handles' streams waits for the batch
    if (!evs.empty()) {
        cudaEvent_t done = evs[0];
        cudaEventRecord(done, st);
        for (int i = 0; i < n; ++i)
            if (hs[i]->st != st) cudaStreamWaitEvent(hs[i]->st, done, 0);
    }
    cleanup();
    return rc;
}

int check_batch(ietidp_handle* const* hs, int n, double* const* u) {
    if (!hs || n < 1 || !u) return fail(IETIDP_E_INVALID_ARG, "null argument");
    for (int i = 0; i < n; ++i) {
        if (!hs[i] || !u[i]) return fail(IETIDP_E_INVALID_ARG, "null handle or output in batch");
        for (int k = 0; k < i; ++k)
            if (hs[k] == hs[i]) return fail(IETIDP_E_INVALID_ARG, "a handle appears twice in one batch");
        if (hs[i]->device != hs[0]->device) return fail(IETIDP_E_INVALID_ARG, "batch spans several devices");
    }
    return IETIDP_OK;
}

int report(std::vector<EngineJob>& jobs, ietidp_stats* stats) {
    int first = IETIDP_OK;
    std::string err;
    for (size_t i = 0; i < jobs.size(); ++i) {
        if (stats) stats[i] = jobs[i].S;
        if (first == IETIDP_OK && jobs[i].rc != IETIDP_OK) {
            first = jobs[i].rc;
            err = jobs.size() > 1 ? "job " + std::to_string(i) + ": " + jobs[i].err : jobs[i].err;
        }
    }
    if (first != IETIDP_OK) return fail(first, err);
    return IETIDP_OK;
}

}  // namespace

extern "C" int ietidp_solve(ietidp_handle* h, const double* f, double* u_out, ietidp_stats* stats) {
    if (!h || !u_out) return fail(IETIDP_E_INVALID_ARG, "null argument");
    std::vector<EngineJob> jobs(1);
    ieti_engine_job_init(jobs[0], h, f, u_out);
    CHK(run_jobs(&h, 1, jobs, false, nullptr, nullptr));
    return report(jobs, stats);
}

extern "C" int ietidp_solve_host(ietidp_handle* h, const double* f_host, double* u_host, ietidp_stats* stats) {
    if (!h || !u_host) return fail(IETIDP_E_INVALID_ARG, "null argument");
    std::vector<EngineJob> jobs(1);
    ieti_engine_job_init(jobs[0], h, f_host ? h->fH : nullptr, h->uH);
    CHK(run_jobs(&h, 1, jobs, true, &f_host, &u_host));
    return report(jobs, stats);
}

extern "C" int ietidp_solve_batch(ietidp_handle* const* hs, int n, const double* const* f, double* const* u,
                                  ietidp_stats* stats) {
    CHK(check_batch(hs, n, u));
    std::vector<EngineJob> jobs(n);
    for (int i = 0; i < n; ++i) ieti_engine_job_init(jobs[i], hs[i], f ? f[i] : nullptr, u[i]);
    CHK(run_jobs(hs, n, jobs, false, nullptr, nullptr));
    return report(jobs, stats);
}

extern "C" int ietidp_solve_batch_host(ietidp_handle* const* hs, int n, const double* const* f_host,
                                       double* const* u_host, ietidp_stats* stats) {
    CHK(check_batch(hs, n, u_host));
    std::vector<EngineJob> jobs(n);
    for (int i = 0; i < n; ++i)
        ieti_engine_job_init(jobs[i], hs[i], (f_host && f_host[i]) ? hs[i]->fH : nullptr, hs[i]->uH);
    CHK(run_jobs(hs, n, jobs, true, f_host, u_host));
    return report(jobs, stats);
}

// V-cycles on the Neumann hierarchies of every patch of several handles in
// one merged launch per kernel specialisation (the batched form of
// ietidp_vcycles, timed on the engine's stream)
extern "C" int ietidp_vcycles_batch(ietidp_handle* const* hs, int n, const double* const* b, double* const* x,
                                    int ncycles, float* ms_out) {
    CHK(check_batch(hs, n, x));
    if (!b || ncycles < 0) return fail(IETIDP_E_INVALID_ARG, "bad argument");
    for (int i = 0; i < n; ++i)
        if (!b[i]) return fail(IETIDP_E_INVALID_ARG, "null input in batch");
    ieti_engine* E = nullptr;
    CHK(engine_of(hs[0], &E));
    cudaStream_t st = E->st;
    std::vector<cudaEvent_t> evs;
    auto join = [&](cudaStream_t from, cudaStream_t to) -> int {
        cudaEvent_t ev;
        cudaError_t er = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (er == cudaSuccess) {
            evs.push_back(ev);
            er = cudaEventRecord(ev, from);
        }
        if (er == cudaSuccess) er = cudaStreamWaitEvent(to, ev, 0);
        return er == cudaSuccess ? IETIDP_OK : fail(IETIDP_E_CUDA, std::string("stream join: ") + cudaGetErrorString(er));
    };
    int rc = IETIDP_OK;
    for (int i = 0; i < n && rc == IETIDP_OK; ++i)
        if (hs[i]->st != st) rc = join(hs[i]->st, st);
    if (rc == IETIDP_OK) {
        std::vector<std::pair<ietidp_handle*, SolveArgs>> items;
        for (int i = 0; i < n; ++i) {
            SolveArgs a = ieti_solve_args(hs[i], MODE_VCYCLE, b[i], x[i], 0.0, 0, hs[i]->vst);
            a.ncycles = ncycles;
            items.emplace_back(hs[i], a);
        }
        long long nl = 0;
        rc = ieti_engine_merged(E, 0, items, &nl, true);
        ieti_host::g_kernel_launches += nl;
    }
    if (rc == IETIDP_OK) {
        cudaError_t er = cudaStreamSynchronize(st);
        if (er != cudaSuccess) rc = fail(IETIDP_E_CUDA, cudaGetErrorString(er));
        else if (ms_out) *ms_out = ieti_engine_timed_ms(E);
    }
    for (int i = 0; i < n && rc == IETIDP_OK; ++i)
        if (hs[i]->st != st) rc = join(st, hs[i]->st);
    for (auto ev : evs) cudaEventDestroy(ev);
    return rc;
}

