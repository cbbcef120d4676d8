// MG-MG-S (Sec. 3.3): Bramble-Pasciak CG on the saddle-point system of Eq. 2,
//   [K~ B~^T; B~ 0] (u, lambda) = (f~, 0),
// for several handles in lockstep.  u in V~ is stored as (Delta parts in
// ker C, primal coefficients); K~ is block diagonal in that basis (Eq. 6):
// S_PiPi on the primal block, P_E K P_E on the Delta block (P_E: Euclidean
// projector on ker C).  Preconditioners: Khat^{-1} = diag(S_PiPi^{-1} /
// theta, P V^c P^T / omega_k) with c V-cycles on the patch's Neumann
// hierarchy (Sec. 4: c = 3) and omega_k = theta (1 - rho_k^c), rho_k a power-
// iteration estimate (60 steps) of the V-cycle contraction (the scaling keeps
// K~ - Khat positive definite, which BPCG needs; the paper does not state
// it; a non-positive inner product halves every scaling and restarts);
// Shat^{-1} = M_sD^{-1}, the scaled Dirichlet preconditioner.
//
// One tick = one BPCG iteration of every job: the Khat^{-1} applications of
// all jobs run in one merged launch per kernel specialisation, then the
// Dirichlet preconditioners likewise, then one synchronisation reads every
// job's inner product <r, r>_H; a job stops when it has dropped by
// tol_outer^2 relative to the first one.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "engine.h"
#include "host_internal.h"
#include "saddle.cuh"

using namespace ieti_host;

struct ieti_saddle_bufs {
    long long nt = 0, nU = 0;
    int npi = 0, nlam = 0;
    double *xu, *rtu, *ru, *pu, *Kru, *KmKru, *Kpu, *KmKpu, *qtu, *qu, *ft;
    double *xl, *rtl, *rl, *pl, *Sr, *Sp, *Br, *Bp, *Bq, *ql, *tl;
    double* sc;        // [0] rho, [1] rho_old, [2] sigma, [3] rho0
    double* partial;   // dot product partial sums
    double* Spp;       // S_PiPi (row-major)
    double* omega;     // per patch Delta-block scaling
    double theta_pi;   // primal-block scaling
};

namespace {

#define SCU(x)                                                                   \
    do {                                                                         \
        cudaError_t e_ = (x);                                                    \
        if (e_ != cudaSuccess) return fail(IETIDP_E_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

int count_launch(EngineJob& j, long long k) {
    j.S.launches += k;
    g_kernel_launches += k;
    return IETIDP_OK;
}

// lazily allocated per handle: BPCG vectors, S_PiPi on the device and the
// block scalings omega_k (power iteration, one merged launch)
int ensure_bufs(ieti_engine* E, ietidp_handle* h, long long* nl) {
    if (h->saddle) return IETIDP_OK;
    auto* b = new ieti_saddle_bufs();
    b->nt = h->prob->ntorn;
    b->npi = h->npi;
    b->nlam = h->nlam;
    b->nU = b->nt + b->npi;
    const long long nU = b->nU, nl_ = std::max(1, b->nlam);
    double* base = nullptr;
    const long long total = 10 * nU + b->nt + 11 * nl_ + 8 + 256 + (long long)b->npi * b->npi + h->npatch;
    int rc = h->mem.alloc(&base, total);
    if (rc != IETIDP_OK) {
        delete b;
        return rc;
    }
    double* q = base;
    double** U[10] = {&b->xu, &b->rtu, &b->ru, &b->pu, &b->Kru, &b->KmKru, &b->Kpu, &b->KmKpu, &b->qtu, &b->qu};
    for (auto pp : U) {
        *pp = q;
        q += nU;
    }
    b->ft = q;
    q += b->nt;
    double** Lm[11] = {&b->xl, &b->rtl, &b->rl, &b->pl, &b->Sr, &b->Sp, &b->Br, &b->Bp, &b->Bq, &b->ql, &b->tl};
    for (auto pp : Lm) {
        *pp = q;
        q += nl_;
    }
    b->sc = q;
    q += 8;
    b->partial = q;
    q += 256;
    b->Spp = q;
    q += (long long)b->npi * b->npi;
    b->omega = q;
    h->saddle = b;
    // the allocation is ordered on the handle's stream; the engine's stream
    // may differ
    SCU(cudaMemsetAsync(base, 0, sizeof(double) * total, h->st));
    if (b->npi)
        SCU(cudaMemcpyAsync(b->Spp, h->spp_host.data(), sizeof(double) * b->npi * b->npi, cudaMemcpyHostToDevice,
                            h->st));
    SCU(cudaStreamSynchronize(h->st));
    // omega_k = theta (1 - rho_k^c)
    std::vector<std::pair<ietidp_handle*, SolveArgs>> items;
    b->theta_pi = h->opt.saddle_theta;
    SolveArgs a = ieti_solve_args(h, MODE_POWER, nullptr, nullptr, 0.0, 60, nullptr);
    a.ncycles = h->opt.saddle_vcycles;
    a.theta = h->opt.saddle_theta;
    a.omega = b->omega;
    items.emplace_back(h, a);
    CHK(ieti_engine_merged(E, 0, items, nl, false));
    SCU(cudaStreamSynchronize(ieti_engine_stream(E)));
    return IETIDP_OK;
}

SaddleLin lin(double* c_num, double* c_den, double sign) {
    SaddleLin L;
    std::memset(&L, 0, sizeof(L));
    L.c = SaddleCoef{c_num, c_den, sign};
    return L;
}

void add(SaddleLin& L, double* y, const double* x, long long n, int mode) {
    if (n <= 0) return;
    L.y[L.njobs] = y;
    L.x[L.njobs] = x;
    L.n[L.njobs] = n;
    L.mode[L.njobs] = mode;
    ++L.njobs;
}

// torn functional g (device, n_torn) -> V~ vector out: Delta part P_E g,
// primal part sum_k A^T Phi^T g (uses out's torn part as the copy of g)
int restrict_to_vtilde(ietidp_handle* h, ieti_saddle_bufs* b, const double* g, double* out, bool accumulate_pi,
                       cudaStream_t st, EngineJob& j) {
    SCU(launch_primal_restrict(h->d_pd, h->nrows, h->crow_patch, h->crow_local, h->phi, g, h->rloc, st));
    SCU(launch_primal_assemble(b->npi, h->gptr, h->glist, h->rloc, out + b->nt, accumulate_pi ? 1 : 0, st));
    if (g != out) SCU(cudaMemcpyAsync(out, g, sizeof(double) * b->nt, cudaMemcpyDeviceToDevice, st));
    SCU(launch_project_kerC(h->nrows, h->d_pd, h->crow_patch, h->crow_ptr, h->c_idx, h->c_w, out, st));
    return count_launch(j, 3);
}

// K~ r: Delta part P_E K w, primal part S_PiPi u_Pi
int apply_Ktilde(ietidp_handle* h, ieti_saddle_bufs* b, const double* in, double* out, cudaStream_t st,
                 EngineJob& j) {
    SCU(launch_apply_K(h->d_pd, h->npatch, h->K64, in, out, st));
    SCU(launch_project_kerC(h->nrows, h->d_pd, h->crow_patch, h->crow_ptr, h->c_idx, h->c_w, out, st));
    SCU(launch_sp_matvec(b->npi, b->Spp, in + b->nt, out + b->nt, 1.0, st));
    return count_launch(j, 3);
}

// lambda-part of B~ applied to a V~ vector: B (Phi A u_Pi + w)
int apply_Btilde(ietidp_handle* h, ieti_saddle_bufs* b, const double* in, double* outl, cudaStream_t st,
                 EngineJob& j) {
    SCU(launch_function(h->npatch, h->d_pd, h->crow_glob, h->phi, in + b->nt, in, b->ft, st));
    SCU(launch_b(h->dual, b->ft, outl, 0, st));
    return count_launch(j, 2);
}

void finish(EngineJob& j, const std::chrono::steady_clock::time_point& t1) {
    ietidp_stats& S = j.S;
    S.outer_it = j.it;
    S.converged = j.conv && !(j.flags & IETI_FLAG_NOT_CONVERGED);
    S.vcycles = j.vs[0];
    S.vcycle_dofs = j.vs[1];
    S.basis_it_avg = j.h->basis_it_avg;
    S.basis_it_max = j.h->basis_it_max;
    S.t_setup_ms = j.h->t_setup_ms;
    S.t_solve_ms = std::chrono::duration<double, std::milli>(t1 - j.t0).count();
    if (j.rc == IETIDP_OK) {
        if (j.flags & IETI_FLAG_BREAKDOWN) {
            j.rc = IETIDP_E_BREAKDOWN;
            j.err = "breakdown in a local solve";
        } else if (!S.converged) {
            j.rc = IETIDP_E_NOT_CONVERGED;
            j.err = "BPCG did not converge";
        }
    }
    j.phase = EngineJob::DONE;
}

}  // namespace

void ieti_saddle_free(ietidp_handle* h) {
    delete h->saddle;   // device memory belongs to the handle's pool
    h->saddle = nullptr;
}

int ieti_saddle_tick(ieti_engine* E, std::vector<EngineJob*>& jobs) {
    cudaStream_t st = ieti_engine_stream(E);
    long long nl = 0;
    for (EngineJob* j : jobs) {
        long long n0 = nl;
        CHK(ensure_bufs(E, j->h, &nl));
        count_launch(*j, nl - n0);
    }
    double* hrb = nullptr;
    CHK(ieti_engine_readback(E, jobs.size() * 16, &hrb));
    {
        // ---- stage A: K-hat^{-1} of every job ------------------------------
        std::vector<std::pair<ietidp_handle*, SolveArgs>> A, B;
        for (EngineJob* j : jobs) {
            ietidp_handle* h = j->h;
            ieti_saddle_bufs* b = h->saddle;
            const bool init = j->phase == EngineJob::INIT || j->phase == EngineJob::RESTART;
            SolveArgs a = ieti_solve_args(h, MODE_KHAT, init ? b->rtu : b->qtu, init ? b->ru : b->qu, 0.0, 0, h->vst);
            a.ncycles = h->opt.saddle_vcycles;
            a.omega = b->omega;
            A.emplace_back(h, a);
            B.emplace_back(h, ieti_solve_args(h, MODE_SCHUR, h->vS, h->wS, 0.0, 0, h->vst));
        }
        CHK(ieti_engine_staged(E, 10, jobs, [&]() -> int {
        for (EngineJob* j : jobs) {
            ietidp_handle* h = j->h;
            ieti_saddle_bufs* b = h->saddle;
            const long long nU = b->nU;
            if (j->phase == EngineJob::INIT || j->phase == EngineJob::RESTART) {
                if (j->phase == EngineJob::INIT) {
                    SCU(cudaMemsetAsync(h->flags, 0, sizeof(int), st));
                    SCU(cudaMemsetAsync(h->vst, 0, sizeof(long long) * 8, st));
                    SCU(cudaMemsetAsync(b->xu, 0, sizeof(double) * nU, st));
                    if (b->nlam) {
                        SCU(cudaMemsetAsync(b->xl, 0, sizeof(double) * b->nlam, st));
                        SCU(cudaMemsetAsync(b->rtl, 0, sizeof(double) * b->nlam, st));
                    }
                    // rt = f~
                    CHK(restrict_to_vtilde(h, b, j->f, b->rtu, false, st, *j));
                } else {
                    // rt = f~ - K~ x_u - B~^T x_l, rt_l = -B~ x_u, in FP64 from the
                    // iterate (the recursively updated residuals drift by the
                    // rounding of the FP32 V-cycles)
                    CHK(restrict_to_vtilde(h, b, j->f, b->rtu, false, st, *j));
                    CHK(apply_Ktilde(h, b, b->xu, b->Kru, st, *j));
                    SCU(cudaMemsetAsync(b->ft, 0, sizeof(double) * b->nt, st));
                    SCU(launch_bt(h->dual, b->xl, b->ft, 0, st));
                    count_launch(*j, 1);
                    CHK(restrict_to_vtilde(h, b, b->ft, b->qtu, false, st, *j));
                    SaddleLin La = lin(nullptr, nullptr, -1.0);
                    add(La, b->rtu, b->Kru, nU, 1);
                    SCU(launch_lin(La, st));
                    SaddleLin Lb = lin(nullptr, nullptr, -1.0);
                    add(Lb, b->rtu, b->qtu, nU, 1);
                    SCU(launch_lin(Lb, st));
                    CHK(apply_Btilde(h, b, b->xu, b->rtl, st, *j));
                    SaddleLin Lc = lin(nullptr, nullptr, 1.0);
                    add(Lc, b->rtl, nullptr, b->nlam, 3);
                    SCU(launch_lin(Lc, st));
                    count_launch(*j, 3);
                }
                // Khat^{-1} input: rt (primal restriction of its Delta part for P^T)
                SCU(launch_primal_restrict(h->d_pd, h->nrows, h->crow_patch, h->crow_local, h->phi, b->rtu, h->rloc,
                                           st));
                count_launch(*j, 1);
            } else {
                // search directions: p = r + beta p (copies on the first step)
                SaddleLin L = lin(b->sc + 0, b->sc + 1, 1.0);
                const int md = j->fresh ? 2 : 0;
                add(L, b->pu, b->ru, nU, md);
                add(L, b->Kpu, b->Kru, nU, md);
                add(L, b->KmKpu, b->KmKru, nU, md);
                add(L, b->pl, b->rl, b->nlam, md);
                add(L, b->Sp, b->Sr, b->nlam, md);
                add(L, b->Bp, b->Br, b->nlam, md);
                SCU(launch_lin(L, st));
                count_launch(*j, 1);
                // qt = K~ p + B~^T p_l (B^T writes the interface entries only)
                SCU(cudaMemsetAsync(b->ft, 0, sizeof(double) * b->nt, st));
                SCU(launch_bt(h->dual, b->pl, b->ft, 0, st));
                count_launch(*j, 1);
                CHK(restrict_to_vtilde(h, b, b->ft, b->qtu, false, st, *j));
                SaddleLin L2 = lin(nullptr, nullptr, 1.0);
                add(L2, b->qtu, b->Kpu, nU, 1);
                SCU(launch_lin(L2, st));
                SCU(launch_primal_restrict(h->d_pd, h->nrows, h->crow_patch, h->crow_local, h->phi, b->qtu, h->rloc,
                                           st));
                count_launch(*j, 2);
            }
        }
        return IETIDP_OK;
        }));
        long long n0 = nl;
        CHK(ieti_engine_merged(E, 0, A, &nl, true));
        g_kernel_launches += nl - n0;
        for (EngineJob* j : jobs) {
            j->S.launches += nl - n0;
            j->S.neumann_launches += 1;
        }
        // ---- between: primal block, B~ of the result, Dirichlet preconditioner input
        CHK(ieti_engine_staged(E, 11, jobs, [&]() -> int {
        for (EngineJob* j : jobs) {
            ietidp_handle* h = j->h;
            ieti_saddle_bufs* b = h->saddle;
            const bool init = j->phase == EngineJob::INIT || j->phase == EngineJob::RESTART;
            double* src = init ? b->rtu : b->qtu;
            double* dst = init ? b->ru : b->qu;
            double* Bd = init ? b->Br : b->Bq;
            SCU(launch_spp_solve(b->npi, h->Linv, src + b->nt, dst + b->nt, 1.0 / b->theta_pi, st));
            count_launch(*j, 1);
            CHK(apply_Btilde(h, b, dst, Bd, st, *j));
            // t = B q - qt_l   (qt_l = B p: Bp; on the first tick rt_l = 0)
            SaddleLin L = lin(nullptr, nullptr, -1.0);
            add(L, b->tl, Bd, b->nlam, 2);
            SCU(launch_lin(L, st));
            if (!init || j->phase == EngineJob::RESTART) {
                SaddleLin L2 = lin(nullptr, nullptr, -1.0);
                add(L2, b->tl, init ? b->rtl : b->Bp, b->nlam, 1);
                SCU(launch_lin(L2, st));
            }
            SCU(launch_bt(h->dual, b->tl, h->vS, 1, st));
            count_launch(*j, init ? 2 : 3);
        }
        return IETIDP_OK;
        }));
        n0 = nl;
        CHK(ieti_engine_merged(E, 1, B, &nl, false));
        g_kernel_launches += nl - n0;
        for (EngineJob* j : jobs) j->S.launches += nl - n0;
        // ---- after: updates, next residual products, <r, r>_H --------------------
        CHK(ieti_engine_staged(E, 12, jobs, [&]() -> int {
        for (size_t i = 0; i < jobs.size(); ++i) {
            EngineJob* j = jobs[i];
            ietidp_handle* h = j->h;
            ieti_saddle_bufs* b = h->saddle;
            const long long nU = b->nU;
            const bool init = j->phase == EngineJob::INIT || j->phase == EngineJob::RESTART;
            SCU(launch_b(h->dual, h->wS, init ? b->rl : b->ql, 1, st));
            count_launch(*j, 1);
            if (!init) {
                // sigma = <K~ - Khat) p, q> + <Shat p_l, q_l>
                SaddleDot D{};
                D.njobs = 2;
                D.a[0] = b->KmKpu;
                D.b[0] = b->qu;
                D.n[0] = nU;
                D.a[1] = b->Sp;
                D.b[1] = b->ql;
                D.n[1] = b->nlam;
                SCU(launch_dot(D, b->partial, b->sc + 2, nullptr, st));
                // alpha = rho / sigma
                SaddleLin Lp = lin(b->sc + 0, b->sc + 2, 1.0);
                add(Lp, b->xu, b->pu, nU, 1);
                add(Lp, b->xl, b->pl, b->nlam, 1);
                SCU(launch_lin(Lp, st));
                SaddleLin Lm = lin(b->sc + 0, b->sc + 2, -1.0);
                add(Lm, b->rtu, b->qtu, nU, 1);
                add(Lm, b->rtl, b->Bp, b->nlam, 1);
                add(Lm, b->ru, b->qu, nU, 1);
                add(Lm, b->rl, b->ql, b->nlam, 1);
                add(Lm, b->Br, b->Bq, b->nlam, 1);
                SCU(launch_lin(Lm, st));
                SCU(launch_copy_scalar(b->sc + 0, b->sc + 1, st));
                count_launch(*j, 6);
            }
            // K~ r and the two parts of the H inner product
            CHK(apply_Ktilde(h, b, b->ru, b->Kru, st, *j));
            SaddleLin L1 = lin(nullptr, nullptr, 1.0);
            add(L1, b->KmKru, b->Kru, nU, 2);
            add(L1, b->Sr, b->Br, b->nlam, 2);
            SCU(launch_lin(L1, st));
            SaddleLin L2 = lin(nullptr, nullptr, -1.0);
            add(L2, b->KmKru, b->rtu, nU, 1);
            add(L2, b->Sr, b->rtl, b->nlam, 1);
            SCU(launch_lin(L2, st));
            SaddleDot D{};
            D.njobs = 2;
            D.a[0] = b->KmKru;
            D.b[0] = b->ru;
            D.n[0] = nU;
            D.a[1] = b->Sr;
            D.b[1] = b->rl;
            D.n[1] = b->nlam;
            SCU(launch_dot(D, b->partial, b->sc + 0, j->phase == EngineJob::INIT ? b->sc + 3 : nullptr, st));
            SCU(cudaMemcpyAsync(hrb + 16 * i, b->sc, sizeof(double) * 4, cudaMemcpyDeviceToHost, st));
            SCU(cudaMemcpyAsync(hrb + 16 * i + 4, h->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
            SCU(cudaMemcpyAsync(hrb + 16 * i + 8, h->vst, sizeof(long long) * 8, cudaMemcpyDeviceToHost, st));
            count_launch(*j, 5);
        }
        return IETIDP_OK;
        }));
        SCU(cudaStreamSynchronize(st));
        const float msA = ieti_engine_timed_ms(E);
        auto t1 = std::chrono::steady_clock::now();
        for (size_t i = 0; i < jobs.size(); ++i) {
            EngineJob* j = jobs[i];
            ietidp_handle* h = j->h;
            ieti_saddle_bufs* b = h->saddle;
            const double* r = hrb + 16 * i;
            j->S.neumann_ms += msA;
            std::memcpy(&j->flags, r + 4, sizeof(int));
            std::memcpy(j->vs, r + 8, sizeof(long long) * 8);
            const double rho = r[0];
            const bool stepped = j->phase == EngineJob::ITER;
            if (j->phase == EngineJob::INIT) {
                j->rho0 = rho;
                j->it = 0;
            } else if (j->phase == EngineJob::RESTART) {
                j->restarts += 1;
            } else {
                j->it += 1;
            }
            if (!stepped) {
                j->rho_cycle = rho;
                j->phase = EngineJob::ITER;
            }
            j->fresh = !stepped;
            // mixed precision: restart once the residual has dropped by 1e-4
            // since the last (re)start, before the FP32 rounding of the
            // recursively updated residuals dominates it
            const double rtol = h->opt.precision == IETIDP_PREC_MIXED ? 1e-4 : 0.0;
            bool done = false;
            if (!std::isfinite(rho)) {
                j->rc = IETIDP_E_NONFINITE;
                j->err = "non-finite BPCG inner product";
                done = true;
            } else if (j->rho0 <= 0.0) {
                j->conv = j->rho0 == 0.0;
                if (!j->conv) {
                    j->rc = IETIDP_E_BREAKDOWN;
                    j->err = "BPCG inner product not positive";
                }
                done = true;
            } else {
                j->S.rel_res = std::sqrt(std::max(rho, 0.0) / j->rho0);
                const double tol = h->opt.tol_outer;
                if (rho >= 0.0 && rho <= tol * tol * j->rho0) {
                    j->conv = true;
                    done = true;
                } else if (j->it >= h->opt.maxit_outer) {
                    j->conv = false;
                    done = true;
                } else if (stepped && rho < 0.0 && j->restarts < 10) {
                    // the inner product is not definite: Khat is not below K~
                    // (contraction underestimated); halve every block scaling
                    // (kept by the handle) and restart from the iterate
                    b->theta_pi *= 0.5;
                    SaddleLin Lw = lin(nullptr, nullptr, -0.5);
                    add(Lw, b->omega, b->omega, h->npatch, 1);
                    SCU(launch_lin(Lw, st));
                    count_launch(*j, 1);
                    j->phase = EngineJob::RESTART;
                } else if (stepped && rho <= rtol * rtol * j->rho_cycle && j->restarts < 100) {
                    j->phase = EngineJob::RESTART;
                } else if (rho < 0.0) {
                    j->rc = IETIDP_E_BREAKDOWN;
                    j->err = "BPCG inner product not positive";
                    j->conv = false;
                    done = true;
                }
            }
            if (done) {
                // u = Phi A x_Pi + x_Delta
                SCU(launch_function(h->npatch, h->d_pd, h->crow_glob, h->phi, b->xu + b->nt, b->xu, j->u, st));
                count_launch(*j, 1);
                finish(*j, t1);
            }
        }
    }
    return IETIDP_OK;
}

int ieti_saddle_run(ieti_engine* E, std::vector<EngineJob*>& all) {
    for (;;) {
        std::vector<EngineJob*> jobs;
        for (EngineJob* j : all)
            if (j->phase != EngineJob::DONE) jobs.push_back(j);
        if (jobs.empty()) break;
        CHK(ieti_saddle_tick(E, jobs));
    }
    SCU(cudaStreamSynchronize(ieti_engine_stream(E)));
    return IETIDP_OK;
}
