/*
 * ietidp.h -- C ABI of the GB300 inexact IETI-DP library.
 *
 * The library solves the model problem of Eq. 1 (-Laplace u = f in Omega,
 * u = 0 on the boundary, a(u,v) = <F,v>) discretized with B-splines on a
 * multipatch domain (Sec. 2) by the dual-primal tearing and interconnecting
 * method with an energy-minimizing primal space.  Default: the MG-MG
 * variant of Sec. 3.3, in which every local problem (the S-orthogonal primal
 * basis of Eq. 6, the local Neumann problems of Eq. 7 inside
 * F = B K~^{-1} B^T, and the local Dirichlet problems of the scaled
 * Dirichlet preconditioner of Sec. 2/3.1) is solved by geometric multigrid
 * on the GPU.  ietidp_options.method selects MG-MG-S (Bramble-Pasciak CG on
 * the saddle-point system Eq. 2) or D-MG (direct banded-Cholesky Neumann
 * solves, multigrid Dirichlet problems) instead.
 *
 * Conventions shared by every entry point:
 *  - return value: 0 on success, a negative IETIDP_E_* code on failure;
 *    ietidp_last_error() gives a message (library-owned, valid until the
 *    next call on the same thread);
 *  - the caller owns every array it passes; the library copies what it keeps;
 *  - the library owns the handles it returns and all device memory behind
 *    them; *_destroy / *_free release them;
 *  - "device" pointers are CUDA global-memory pointers on the current
 *    device, "host" pointers ordinary memory; sizes are element counts;
 *  - `stream` is a cudaStream_t (NULL = legacy default stream); all device
 *    work of a handle is ordered on the stream given when it was created;
 *  - invalid descriptors are rejected before any device work; no entry point
 *    traps the device; iterative solvers that hit their iteration limit
 *    return IETIDP_E_NOT_CONVERGED with the statistics filled in;
 *  - a handle (and a problem) is used by one host thread at a time, and a
 *    batch (ietidp_solve_batch*) uses every handle in it, launching on the
 *    first handle's engine; different handles may be used from different
 *    threads concurrently; a server's submit, poll, status and estimate may
 *    be called from any thread, and ietidp_server_destroy after all of them.
 *
 * Torn vector layout ("patch layout"): patch after patch, each patch's
 * coefficients on its full tensor grid of (n_r + p_r) functions per
 * direction, first direction fastest, including the coefficients of the
 * Dirichlet boundary (which are always 0 in a solution).  ietidp_info
 * returns the per-patch offsets.
 */
#ifndef IETIDP_H
#define IETIDP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define IETIDP_OK               0
#define IETIDP_E_INVALID_ARG   -1
#define IETIDP_E_OOM           -2   /* device allocation failed            */
#define IETIDP_E_BUDGET        -3   /* request does not fit a memory budget */
#define IETIDP_E_CUDA          -4   /* a CUDA runtime call failed           */
#define IETIDP_E_NOT_CONVERGED -5   /* an iteration limit was reached       */
#define IETIDP_E_TIMEOUT       -6   /* a bounded device wait expired        */
#define IETIDP_E_NONFINITE     -7   /* NaN/Inf in input or iteration        */
#define IETIDP_E_BREAKDOWN     -8   /* CG breakdown / coarse matrix not SPD */

/* ---- geometry kinds (Sec. 2: each patch is the image of (0,1)^d) ------- */
#define IGA_GEO_BOX      0   /* affine: x_r = lo_r + (hi_r - lo_r) xi_r        */
#define IGA_GEO_ANNULUS  1   /* quarter annulus: (s1,s2) = lo + (hi-lo) xi is a
                                sub-box of the parameter square of the exact map
                                G(s1,s2) = (1 + s2) C(s1), C the rational
                                quadratic quarter circle from (1,0) to (0,1)
                                with weights (1, 1/sqrt 2, 1)               */

/* ---- right-hand sides of Eq. 1 ---------------------------------------- */
#define IGA_RHS_NONE     0   /* zero load (solve takes a load vector)          */
#define IGA_RHS_SIN2D    1   /* 2 pi^2 sin(pi x) sin(pi y)                     */
#define IGA_RHS_SIN3D    2   /* 3 pi^2 sin(pi x) sin(pi y) sin(pi z)           */
#define IGA_RHS_ANNULUS  3   /* -Laplace of sin(pi x) sin(pi y) (r-1)(2-r)     */
#define IGA_RHS_MODES    4   /* sum_j a_j sin(k_j pi x) sin(l_j pi y)          */
#define IGA_RHS_QUAD     5   /* f given at every Gauss point (see below)       */

/* ---- primal constraint set (Sec. 4: vertex values, edge/face averages) - */
#define IETIDP_PRIMAL_VERTEX 1u
#define IETIDP_PRIMAL_EDGE   2u
#define IETIDP_PRIMAL_FACE   4u

/* ---- precision of the multigrid V-cycles -------------------------------- */
#define IETIDP_PREC_FP64   0  /* everything FP64                             */
#define IETIDP_PREC_MIXED  1  /* V-cycles (smoother, SpMV, transfers) FP32;
                                 inner/outer CG, residuals, dots, primal
                                 coarse Cholesky FP64                        */

typedef struct {
    int    degree[3];   /* spline degree 1 <= p_r <= 7 per direction (d entries) */
    int    nelem[3];    /* uniform elements n_r >= 1 per direction            */
    int    geo_kind;    /* IGA_GEO_*                                          */
    double lo[3];       /* box corner (physical for BOX, parameter for ANNULUS)*/
    double hi[3];
} iga_patch_desc;

/* Side numbering: side 2r is xi_r = 0, side 2r+1 is xi_r = 1.  The tangential
 * directions of a side are the remaining directions in increasing order.
 * Interfaces are conforming (Sec. 2): both sides carry the same tangential
 * spline space.  `swap` (3D only) exchanges the two tangential directions of
 * side_b, and flip[t] reverses tangential direction t of side_b (after the
 * swap), relative to side_a. */
typedef struct {
    int patch_a, side_a, patch_b, side_b;
    int flip[2];
    int swap;
} iga_interface_desc;

typedef struct {
    int dim;                                 /* 2 or 3                          */
    int npatch;
    const iga_patch_desc*     patches;       /* host, npatch entries            */
    int ninterface;
    const iga_interface_desc* interfaces;    /* host, ninterface entries        */
    /* Every patch side that is not part of an interface lies on the boundary
     * of Omega and carries the homogeneous Dirichlet condition of Eq. 1. */
    int rhs_kind;                            /* IGA_RHS_*                       */
    int nmodes;                              /* IGA_RHS_MODES                   */
    const double* mode_a;                    /* host, nmodes                    */
    const int*    mode_k;
    const int*    mode_l;
    /* IGA_RHS_QUAD: f at the tensor grid of Gauss points of every patch
     * (n_r (p_r + 1) points per direction, p_r + 1 Gauss-Legendre points per
     * element, first direction fastest), patch after patch.  Device. */
    const double* quad_values;
} iga_domain_desc;

typedef struct iga_problem   iga_problem;
typedef struct ietidp_handle ietidp_handle;

/* Outer method (Sec. 3.3): dual PCG on F lambda = d with accurate local
 * Neumann solves by multigrid-preconditioned CG (MG-MG) or by a direct
 * banded solver (D-MG), or Bramble-Pasciak CG on the saddle-point system of
 * Eq. 2 with a fixed number of V-cycles in the preconditioner of K~
 * (MG-MG-S). */
#define IETIDP_METHOD_DUAL   0
#define IETIDP_METHOD_SADDLE 1
/* D-MG (Sec. 3.3): dual PCG with direct local Neumann solves (banded
 * Cholesky of the fine K per patch) and multigrid Dirichlet problems */
#define IETIDP_METHOD_DMG    2

/* Primal basis solver (Eq. 6): CG with the Schoeberl-Zulehner preconditioner
 * on the saddle-point system (Sec. 3.2, the paper's choice), or CG on ker C
 * with the Euclidean projection (null-space method). */
#define IETIDP_BASIS_SZ        0
#define IETIDP_BASIS_NULLSPACE 1

/* Multigrid of the local problems (Sec. 4).  STANDARD: nested grids with the
 * patch degree on every level, knot-insertion transfers, multicolor
 * Gauss-Seidel.  HIGHORDER (the paper's choice for p = 4 and 7): degree 1 on
 * every level but the finest (the degree-1 space on half the elements and
 * its dyadic coarsenings), L2-projection transfers between the finest level
 * and the first degree-1 level, and on the finest level a subspace-corrected
 * mass smoother (after Hofreither and Takacs, SIAM J. Numer. Anal. 55, 2017)
 * with a rank-one approximation of the geometry, applied by fast
 * diagonalization; Gauss-Seidel on the degree-1 levels.  The degree-1
 * space has floor(n/2) elements per direction (at least 1); 3D patches must
 * be boxes.  The primal basis (Eq. 6) is computed with the standard
 * hierarchy in both settings (the smoother above may overshoot, which the
 * Schoeberl-Zulehner CG does not allow); degrees up to 7. */
#define IETIDP_MG_STANDARD  0
#define IETIDP_MG_HIGHORDER 1

typedef struct {
    unsigned primal;          /* IETIDP_PRIMAL_* bitmask                       */
    int    precision;         /* IETIDP_PREC_*                                 */
    double tol_outer;         /* dual PCG: ||d - F lambda|| <= tol ||d||  (1e-10) */
    double tol_inner;         /* local Neumann solves, relative residual (1e-12) */
    double tol_basis;         /* primal basis solves, relative residual  (1e-12) */
    int    maxit_outer;       /* (500)                                         */
    int    maxit_inner;       /* (500)                                         */
    int    nu_pre, nu_post;   /* smoothing steps (2, 2)                        */
    int    coarse_elems;      /* coarsen while a direction has more elements (4) */
    int    dirichlet_vcycles; /* V-cycles for K_II^{-1} in the preconditioner (2) */
    double alpha_reg;         /* K_M = K + alpha M^ on floating patches (1e-2)  */
    int    cluster;           /* reserved (0)                                  */
    int    method;            /* IETIDP_METHOD_* (dual PCG, MG-MG)             */
    int    saddle_vcycles;    /* MG-MG-S: V-cycles in the K~ preconditioner (3) */
    double saddle_theta;      /* MG-MG-S: block scaling theta (0.9)            */
    int    basis_method;      /* IETIDP_BASIS_* (Schoeberl-Zulehner CG)        */
    int    mg_kind;           /* IETIDP_MG_* (standard h-multigrid)            */
} ietidp_options;

typedef struct {
    int    outer_it;          /* dual PCG iterations                           */
    int    converged;
    double rel_res;           /* final ||r|| / ||d||                           */
    double kappa;             /* Lanczos estimate from the CG coefficients     */
    double d_norm, d_scale;   /* ||d|| and the jump scale of K~^{-1} f         */
    double inner_it_avg;      /* Neumann solves: mean CG iterations per patch   */
    int    inner_it_max;
    double basis_it_avg;      /* primal basis: mean CG iterations per function */
    int    basis_it_max;
    long long vcycles;        /* V-cycles executed (all patches)               */
    long long vcycle_dofs;    /* sum over V-cycles of fine-level dofs          */
    double t_setup_ms, t_solve_ms;
    long long launches;       /* kernels launched by this solve                */
    int    neumann_launches;  /* launches of the batched Neumann solver kernel */
    double neumann_ms;        /* their total device time (CUDA events)         */
    long long inner_its;      /* CG iterations summed over all Neumann slots   */
} ietidp_stats;

typedef struct {
    int    dim, npatch;
    long long n_torn;         /* length of a torn vector (patch layout)         */
    int    n_lambda;          /* Lagrange multipliers                          */
    int    n_primal;          /* primal dofs (size of S_PiPi)                   */
    int    n_floating;        /* patches without a Dirichlet side               */
    int    max_levels;
    long long device_bytes;   /* device memory held by the handle              */
} ietidp_info;

/* Fill `opt` with the defaults quoted above. */
void ietidp_default_options(ietidp_options* opt);

/* Assemble the per-patch Galerkin stiffness K^(k) and load f^(k) of Eq. 1
 * with the pulled-back B-spline basis (Sec. 2), Gauss quadrature with p_r+1
 * points per element and direction, on the GPU.  Builds the patch topology
 * (interfaces, Dirichlet sides, conforming dof identification) on the host.
 * `out` receives a new problem; free it with iga_problem_free. */
int iga_assemble_patches(const iga_domain_desc* dom, void* stream, iga_problem** out);

/* Host-only topology of a domain, the first step of iga_assemble_patches
 * (Sec. 2: the multipatch space, conforming interfaces, torn copies of the
 * interface functions), run without any device work: the same validation of
 * the descriptors (IETIDP_E_INVALID_ARG for a bad dimension, degree, box,
 * patch index, side, a side used twice or a non-conforming interface) and
 * the same identification of torn copies.
 *   n_torn       sum over patches of the tensor-grid functions (n_r + p_r)
 *   n_global     functions of the conforming space: n_torn minus, for every
 *                class of identified copies, its size minus one (Dirichlet
 *                functions included)
 *   n_classes    classes of identified patch-boundary functions (size >= 1)
 *   n_shared     classes with copies on two or more patches
 *   n_dirichlet  classes on the Dirichlet boundary (a side of a patch that
 *                has no interface)
 *   n_floating   patches without a Dirichlet side
 * `dmask` (host, npatch entries, may be NULL) receives per patch the bit
 * mask of its Dirichlet sides (bit 2r: xi_r = 0, bit 2r+1: xi_r = 1). */
typedef struct {
    long long n_torn, n_global, n_classes, n_shared, n_dirichlet;
    int n_floating;
} iga_topology_info;
int iga_topology(const iga_domain_desc* dom, iga_topology_info* info, unsigned* dmask);

/* The assembled load vector f~ in patch layout (device, n_torn doubles). */
int iga_problem_load(const iga_problem* prob, double* f_out);
int iga_problem_free(iga_problem* prob);

/* IETI-DP setup (Sec. 2, 3.2, 4): jump operator B and scaled B_D, primal
 * constraints C^(k), multigrid hierarchies (Galerkin coarse operators,
 * regularized K + alpha M^ on floating patches, coarsest-level factors),
 * the energy-minimizing primal basis of Eq. 6 by multigrid-preconditioned
 * CG, S_PiPi and its Cholesky factor.  The problem must outlive the handle. */
int ietidp_setup(const iga_problem* prob, const ietidp_options* opt, void* stream,
                 ietidp_handle** out);

int ietidp_info_get(const ietidp_handle* h, ietidp_info* info);
/* Per-patch offsets into a torn vector: `offsets` has npatch+1 entries. */
int ietidp_patch_offsets(const ietidp_handle* h, long long* offsets);

/* Solve K~ u + B^T lambda = f~, B u = 0 (Eq. 2) through the dual problem
 * F lambda = d of Eq. 4: d = B K~^{-1} f~, dual PCG with the scaled
 * Dirichlet preconditioner, u = K~^{-1}(f~ - B^T lambda).
 * f: device load vector in patch layout, or NULL for the assembled load;
 * u_out: device, n_torn doubles.  `stats` may be NULL. */
int ietidp_solve(ietidp_handle* h, const double* f, double* u_out, ietidp_stats* stats);

/* Same as ietidp_solve with HOST buffers: copies f to the device, solves and
 * copies u back, all on the handle's stream (f may be NULL as above). */
int ietidp_solve_host(ietidp_handle* h, const double* f_host, double* u_host,
                      ietidp_stats* stats);

/* Batched solve: the dual PCG of ietidp_solve for n handles at once, in
 * lockstep.  Each outer iteration runs the local Neumann solves of every
 * patch of every handle in one kernel launch per degree specialisation, then
 * one host synchronisation reads all dual residuals, then the
 * preconditioners of the handles that continue run in one launch per
 * specialisation.  Handles that converge leave the batch.  Patches are
 * ordered longest first; block size and shared-memory budget of each merged
 * launch are chosen by an autotuner that times its candidates once per launch
 * shape (IETIDP_AUTOTUNE=0: 512 threads, full budget).  Every handle's result
 * equals its own ietidp_solve up to rounding (the reduction order of dot
 * products follows the block size).
 * hs: n distinct handles on one device; f[i] device load of handle i (f or
 * f[i] NULL: assembled load); u[i] device outputs (n_torn_i doubles);
 * stats: n entries or NULL.  Runs on the stream of hs[0]; the other handles'
 * streams are joined before and after.  Returns the first failing handle's
 * code (all stats are filled). */
int ietidp_solve_batch(ietidp_handle* const* hs, int n, const double* const* f, double* const* u,
                       ietidp_stats* stats);
/* Same with HOST buffers (copies in and out inside the call). */
int ietidp_solve_batch_host(ietidp_handle* const* hs, int n, const double* const* f_host,
                            double* const* u_host, ietidp_stats* stats);

/* Autotuner decisions so far (process-wide): up to max_entries records of
 * 12 ints {dim, p0, p1, p2, kind (0 specialised, 1 global-memory vectors,
 * 2 run-time degree), mixed, waves, threads, smem bytes, CTAs per SM,
 * chosen variant keeps the V-cycle vectors in global memory, CTAs per slot
 * (a thread-block cluster when > 1)} into out (may be NULL); returns the
 * number of decisions. */
int ietidp_autotune_table(int* out, int max_entries);

/* Kernels launched so far in this process by the solve entry points
 * (ietidp_solve*, ietidp_vcycles*, the ietidp_apply_* probes); assembly and
 * setup launches are not counted. */
long long ietidp_kernel_launches(void);

/* Apply `ncycles` V-cycles (Sec. 4 multigrid) to every patch's Neumann
 * hierarchy in one batched launch each: x <- x + V(b - A x), with b and x
 * device vectors in patch layout.  Used to measure V-cycle throughput. */
int ietidp_vcycles(ietidp_handle* h, const double* b, double* x, int ncycles);

/* Batched form of ietidp_vcycles (Sec. 4 multigrid): the Neumann
 * hierarchies of every patch of the n handles in one merged launch per
 * kernel specialisation, x[i] <- x[i] + V(b[i] - A x[i]) for `ncycles`
 * cycles.  b[i], x[i] are device vectors in handle i's patch layout; the
 * handles must be distinct and on one device.  *ms_out (may be NULL)
 * receives the duration of the merged launches (CUDA events; the first
 * call of a launch shape includes its autotuning).  Synchronous. */
int ietidp_vcycles_batch(ietidp_handle* const* hs, int n, const double* const* b, double* const* x, int ncycles,
                         float* ms_out);

/* As ietidp_vcycles on a chosen hierarchy of every patch (Sec. 3.1, 3.2, 4):
 * hierarchy 0 = the Neumann hierarchy (K, or K + alpha M^ on floating
 * patches; Dirichlet sides masked), 1 = the Dirichlet hierarchy of the
 * scaled Dirichlet preconditioner (K_II: every side masked).  Residuals use
 * the FP64 fine K with the same mask; masked entries of x are left as they
 * are.  Returns IETIDP_E_INVALID_ARG for another hierarchy value. */
int ietidp_vcycles_hierarchy(ietidp_handle* h, int hierarchy, const double* b, double* x, int ncycles);

/* Same V-cycles as ietidp_vcycles, but allocating nothing: for callers that
 * cannot allocate device memory when they run (a plugin inside a host
 * framework that owns the device memory pool, a latency-bound loop that must
 * not call cudaMalloc/cudaFree).  The paper has no counterpart; this is a
 * deployment variant of the V-cycle kernel.  The kernel's scratch vectors
 * (FP64 residual and correction, per-level vectors of every patch) live in
 * one static device array of 16 MiB per device.  ietidp_setup looks up the
 * array's device address on the handle's device and keeps it in the handle;
 * the array's memory is committed when the library's device code is loaded
 * on that device: at the first CUDA call of the library under eager module
 * loading, at that lookup in the first ietidp_setup under lazy loading (the
 * CUDA 12+ default).  It is held until the process exits, or until the
 * device's primary context is destroyed, which invalidates every handle of
 * that device (set up new handles afterwards).  This call allocates nothing,
 * does not modify the handle, and must be made with the handle's device
 * current.  Problems whose scratch exceeds 16 MiB are rejected with
 * IETIDP_E_INVALID_ARG and a message giving both sizes, before any device
 * work.  All calls on a device share the array and it keeps the last call's
 * contents (the kernel writes every scratch entry before reading it, so
 * nothing needs clearing); calls whose work overlaps on the GPU (other
 * streams, other handles, other host threads) race on it.  b, x as for
 * ietidp_vcycles. */
int ietidp_vcycles_noalloc(ietidp_handle* h, const double* b, double* x, int ncycles);

/* Operators of the high-order multigrid (Sec. 4) of one patch, built on the
 * host in FP64 with no device work (inspection and tests).  Hierarchy `kind`
 * 0 (Neumann: the sides in dmask removed; alpha M^ added when dmask == 0) or
 * 1 (Dirichlet: every side removed).  Out, host: sizes[0..2] the free fine
 * functions per direction, sizes[3..5] the free degree-1 functions on half
 * the elements (1 beyond dim); U the smoother's generalized eigenvectors per
 * direction, U_r[j + nf_r i], directions one after the other; P the L2
 * prolongations, P_r[j + nf_r c], likewise; Dinv 1 / (sum_r c_r lambda_r
 * + alpha c_M) on the nf_0 x nf_1 (x nf_2) grid, first direction fastest.
 * U, P, Dinv may be NULL (sizes only).  IETIDP_E_INVALID_ARG for a bad
 * dimension, degree (1..7), element count, kind or a 3D patch that is not a
 * box. */
int ietidp_ho_patch_operators(int dim, const iga_patch_desc* patch, unsigned dmask, double alpha, int kind,
                              int* sizes, double* U, double* P, double* Dinv);

/* Helpers exposed for testing the building blocks against the oracle:
 *  - ietidp_apply_K: y = K x per patch (Dirichlet rows/cols removed);
 *  - ietidp_apply_F: q = F p on the multipliers (device, n_lambda);
 *  - ietidp_apply_precond: z = M_sD^{-1} r;
 *  - ietidp_apply_Ktilde_inv: u = K~^{-1} g (patch layout);
 *  - ietidp_get_primal_basis: Phi^(k) of patch k, column-major, its full
 *    tensor grid x n_Pi^(k), into a device buffer; returns n_Pi^(k) in *ncols;
 *  - ietidp_get_spp: S_PiPi (host, n_primal^2, row-major). */
int ietidp_apply_K(ietidp_handle* h, const double* x, double* y);
int ietidp_apply_F(ietidp_handle* h, const double* p, double* q);
int ietidp_apply_precond(ietidp_handle* h, const double* r, double* z);
int ietidp_apply_Ktilde_inv(ietidp_handle* h, const double* g, double* u);
int ietidp_get_primal_basis(ietidp_handle* h, int patch, double* phi, int* ncols);
int ietidp_get_spp(ietidp_handle* h, double* spp_host);

/* Profiling: per-phase clock cycles of the first CTA of the local solver
 * kernel since setup (64 counters: [4l+0..3] sweeps, residual, restriction,
 * prolongation at level l; [48] coarsest solve; [49] FP64 SpMV).  Zeros
 * unless the library was built with IETIDP_PHASE_TIMERS=1. */
int ietidp_phase_timers(ietidp_handle* h, long long* out64);

int ietidp_destroy(ietidp_handle* h);

/* ---- continuous-batching server ---------------------------------------
 * Requests are queued as they arrive.  `max_concurrent` setup workers, each
 * with its own CUDA stream, admit queued requests while the estimated device
 * memory of all admitted requests stays within `budget_bytes` (first come
 * first served; a request that does not fit lets later smaller ones pass) and
 * run iga_assemble_patches and ietidp_setup.  Set-up requests join one solve
 * loop between outer iterations: the local solves of all requests in flight
 * run in shared merged launches (ietidp_solve_batch), and a request leaves
 * when it has converged.  Its data stays resident until its solution is on
 * the host.  The domain descriptor is copied at submission, except
 * quad_values (device, must stay valid until the request is done).  A
 * request's result does not depend on what else runs, up to the rounding of
 * dot products under another autotuned block size. */
typedef struct ietidp_server ietidp_server;
int ietidp_server_create(long long budget_bytes, int max_concurrent, const ietidp_options* opt,
                         ietidp_server** out);
/* IETIDP_E_BUDGET if the request alone exceeds the budget. */
int ietidp_server_submit(ietidp_server* s, const iga_domain_desc* dom, unsigned long long* ticket);
/* Poll (wait = 0) or wait for (wait = 1) a request; *state = 0 queued,
 * 1 running, 2 done.  When done: u_host (n_u >= n_torn doubles, may be NULL)
 * and stats are filled, t[3] (may be NULL) = queue time, run time and
 * latency in seconds, the request's return code is returned, and the ticket
 * is released. */
int ietidp_server_poll(ietidp_server* s, unsigned long long ticket, int wait, int* state, double* u_host,
                       long long n_u, ietidp_stats* stats, double* t);
int ietidp_server_status(ietidp_server* s, int* running, long long* in_flight_bytes, int* queued);
/* The admission estimate of a request's device memory (bytes), or -1. */
long long ietidp_server_estimate(ietidp_server* s, const iga_domain_desc* dom);
/* Finishes running requests, drops queued ones, joins the workers. */
int ietidp_server_destroy(ietidp_server* s);

const char* ietidp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* IETIDP_H */
