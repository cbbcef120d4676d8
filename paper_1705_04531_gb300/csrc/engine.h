// Batched solve engine (ietidp_engine.cu): lockstep dual PCG over several
// jobs, one job = one handle and one right-hand side.
#pragma once
#include <cuda_runtime.h>

#include <chrono>
#include <functional>
#include <string>
#include <vector>

#include "host_internal.h"

struct ieti_engine;

struct EngineJob {
    // INIT: u0 = K~^{-1} f next; PRECF / PREC: preconditioner (first / later
    // iteration) in this tick's stage B; ITER: F p next; RECOVER: recovery
    // solve next; DONE: result and stats final
    // (MG-MG-S: RESTART recomputes the residual from the iterate; mixed-
    // precision refinement)
    enum Phase { INIT, PRECF, ITER, PREC, RECOVER, DONE, RESTART };
    ietidp_handle* h = nullptr;
    const double* f = nullptr;   // torn right-hand side (device)
    double* u = nullptr;         // torn solution (device)
    int phase = INIT;
    int it = 0;                  // outer iterations done
    double dd = 0, thr2 = 0;     // ||d||^2 and the squared stopping threshold
    bool conv = true;
    int rc = IETIDP_OK;          // the job's own result code
    std::string err;
    ietidp_stats S{};
    std::chrono::steady_clock::time_point t0;
    int flags = 0;
    long long vs[8] = {};
    double rho0 = 0.0;           // MG-MG-S: first BPCG inner product
    double rho_cycle = 0.0;      // MG-MG-S: inner product at the last (re)start
    bool fresh = false;          // MG-MG-S: next step starts a new search direction
    int restarts = 0;
    std::vector<double> al, be;  // CG coefficients (Lanczos condition estimate)
};

int ieti_engine_create(cudaStream_t st, ieti_engine** out);
void ieti_engine_destroy(ieti_engine* E);
cudaStream_t ieti_engine_stream(const ieti_engine* E);
void ieti_engine_job_init(EngineJob& j, ietidp_handle* h, const double* f, double* u);
// one outer iteration of every job in `jobs` (none DONE); returns a CUDA-level
// failure of the whole tick, per-job failures go to EngineJob::rc
int ieti_engine_tick(ieti_engine* E, std::vector<EngineJob*>& jobs);
// ticks until every job is DONE
int ieti_engine_run(ieti_engine* E, std::vector<EngineJob*>& jobs);
// one merged local-solve launch (stage 0 or 1 staging buffers: at most one
// use of each per synchronisation interval); timed: bracket it with the
// engine's events (ieti_engine_timed_ms after the next synchronisation)
int ieti_engine_merged(ieti_engine* E, int stage, std::vector<std::pair<ietidp_handle*, SolveArgs>>& items,
                       long long* nlaunch, bool timed);
float ieti_engine_timed_ms(ieti_engine* E);
// pinned read-back buffer of at least n doubles (valid until the next call)
int ieti_engine_readback(ieti_engine* E, size_t n, double** out);
// runs `eager` (stream-ordered launches on the engine's stream, nothing read
// back to the host inside) as segment `seg` of a tick: captured as a CUDA
// graph on the second occurrence of the same (segment, jobs, phases) and
// replayed from then on; kernel launch counts are replayed with it
int ieti_engine_staged(ieti_engine* E, int seg, std::vector<EngineJob*>& jobs, const std::function<int()>& eager);
// MG-MG-S jobs (handles with method IETIDP_METHOD_SADDLE), lockstep BPCG:
// one iteration of every job (none DONE) / iterations until all are DONE
int ieti_saddle_tick(ieti_engine* E, std::vector<EngineJob*>& jobs);
int ieti_saddle_run(ieti_engine* E, std::vector<EngineJob*>& jobs);
