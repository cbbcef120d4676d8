// Batched solve engine (ietidp_engine.cu): lockstep dual PCG over several
// jobs, one job = one handle and one right-hand side.
#pragma once
#include <cuda_runtime.h>

#include <chrono>
#include <string>
#include <vector>

#include "host_internal.h"

struct ieti_engine;

struct EngineJob {
    // INIT: u0 = K~^{-1} f next; PRECF / PREC: preconditioner (first / later
    // iteration) in this tick's stage B; ITER: F p next; RECOVER: recovery
    // solve next; DONE: result and stats final
    enum Phase { INIT, PRECF, ITER, PREC, RECOVER, DONE };
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
