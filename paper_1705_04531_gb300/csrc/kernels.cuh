// Launch wrappers shared by the host orchestration and the kernel files.
#pragma once
#include "common.cuh"

// ---- setup data ------------------------------------------------------------
struct AsmTables {          // per (patch, direction) assembly tables
    int nq;                 // Gauss points along the direction (n*(p+1))
    long long qoff;         // offset into qx / qw (nq entries)
    long long boff;         // offset into B / D ((p+1) values per point)
};

struct SetupArgs {
    int npatch, dim;
    const PatchDesc* pd;         // device
    const double* geo;           // device, per patch: kind, lo[3], hi[3] (7 doubles)
    const AsmTables* at;         // device, npatch*3
    double* qx; double* qw; double* Bv; double* Dv;
    const long long* qpoff;      // device, per patch: offset of its Gauss points (npatch+1)
    double* Gm;                  // 6 doubles per Gauss point
    double* Fw;                  // 1 double per Gauss point
    int rhs_kind;
    const double* modes;         // nmodes*3 (a, k, l)
    int nmodes;
    const double* quad_values;   // IGA_RHS_QUAD
    const long long* rowoff;     // device, per patch: prefix of fine n (npatch+1)
    double* K64;                 // value pool
    double* f;                   // torn load vector
    double* tab; int* itab;      // 1D table pools
    int* flags;
};

cudaError_t launch_assembly(const SetupArgs& a, long long total_qp, long long total_rows,
                            int max_S, cudaStream_t st);

struct TableJob { int patch, level, r; };
cudaError_t launch_tables(const SetupArgs& a, const TableJob* jobs_dev, int njobs, int max_m,
                          cudaStream_t st);
cudaError_t launch_mass_tables(const SetupArgs& a, const TableJob* jobs_dev, int njobs, cudaStream_t st);

// Galerkin coarsening of all patches whose fine level minus `depth` exists.
cudaError_t launch_galerkin(const PatchDesc* pd, const int* patch_list, int npl,
                            int depth, int max_rows, int max_S, double* K64, const double* tab,
                            const int* itab, cudaStream_t st);

// Dense inverses of the coarsest operators: job = patch*2 + kind.
cudaError_t launch_coarse_inverse(const PatchDesc* pd, int npatch, const double* K64,
                                  const double* tab, double alpha, double* A0inv64,
                                  float* A0inv32, double* work, int max_n0, int* flags,
                                  cudaStream_t st);

// Constraint weights: entries of C rows (vertex = 1, edge/face = normalized
// integrals of the tangential basis functions).
cudaError_t launch_regularize(const PatchDesc* pd, int npatch, const double* K64, const double* tab, double alpha,
                              double* KM64, cudaStream_t st);
cudaError_t launch_cweights(const PatchDesc* pd, int nrows, const int* crow_ptr,
                            const int* crow_patch, const int* crow_tang, const int* c_idx,
                            double* c_w, cudaStream_t st);

cudaError_t launch_to_f32(const double* src, float* dst, long long n, cudaStream_t st);
// lo = src - hi rounded to FP32 (the low part of an FP32 pair hi + lo)
cudaError_t launch_lo_f32(const double* src, const float* hi, float* lo, long long n, cudaStream_t st);

// D-MG: band of the fine K (Dirichlet and pinned dofs as identity rows) and its
// Cholesky factor, one CTA per listed patch (direct_kernels.cu)
cudaError_t launch_band_factor(const PatchDesc* pd, const int* plist, int npl, int max_n, int max_bw,
                               const double* K64, double* band, int* flags, cudaStream_t st);
// SZ basis: Hhat^{-1} = (0.99 C W)^{-1} per patch (W = Khat^{-1} C^T, layout of phi)
cudaError_t launch_sz_hinv(const PatchDesc* pd, int npatch, const int* crow_ptr, const int* c_idx,
                           const double* c_w, const double* szW, double* szHinv, int* flags, cudaStream_t st);

// Dense SPD: Cholesky factor and inverse of the lower factor, one CTA.
cudaError_t launch_chol_linv(const double* A, int n, double* Linv, double* work, int* flags,
                             cudaStream_t st);

// ---- solve data --------------------------------------------------------------
// dynamic shared memory budget of the specialised local solver kernel
constexpr size_t kSolveSmemCap = 220 * 1024;

struct SlotDesc {
    int patch;
    int kind;            // 0: Neumann hierarchy, 1: Dirichlet hierarchy
    int row;             // basis mode: global C row
    int its;             // index of the slot's iteration count in SolveArgs::its
    int handle;          // batched launches: index of the slot's arguments in SolveArgs::batch
    int pad;
    long long cg;        // offset of the slot's FP64 vectors (5 n)
    long long lv;        // offset of the slot's level vectors (3 nlvec)
};

// MODE_POWER: V-cycle contraction estimate per patch (BPCG scaling);
// MODE_KHAT: Delta block of the BPCG preconditioner, P V^ncycles P^T / omega
// MODE_SZW / MODE_BASIS_SZ: primal basis by Schoeberl-Zulehner CG (W = Khat^{-1} C^T
// per constraint row, then one SZ-CG per constraint row)
enum SlotMode {
    MODE_NEUMANN = 0,
    MODE_BASIS = 1,
    MODE_SCHUR = 2,
    MODE_VCYCLE = 3,
    MODE_POWER = 4,
    MODE_KHAT = 5,
    MODE_SZW = 6,
    MODE_BASIS_SZ = 7,
    MODE_NEUMANN_DIRECT = 8,  // D-MG: Neumann solve by the banded Cholesky factor
    MODE_VCYCLE_DIR = 9       // V-cycles on the Dirichlet hierarchy (K_II, every side masked)
};

// High-order multigrid of one patch (Sec. 4, p >= 4), per hierarchy kind
// (0 Neumann, 1 Dirichlet) and direction: free fine functions (count, first
// index), free functions of the degree-1 space on half the elements, and the
// offsets in the pool of the fast-diagonalization eigenvectors U (nf x nf,
// U[j + nf i] = eigenvector i at function j), of the L2-projection
// prolongation P (nf x nc, P[j + nf c]) and of 1 / eigenvalue sums (tensor
// nf0 x nf1 x nf2, first direction fastest).
struct HoDesc {
    int nf[2][3], lof[2][3], nc[2][3], loc[2][3];
    long long u[2][3], pt[2][3], dinv[2];
};

struct SolveArgs {
    const PatchDesc* pd;
    const SlotDesc* slots;
    int nslots;
    int mode;
    int mixed;                 // V-cycles in FP32
    const double* K64;
    const float* K32;
    const float* K32lo;        // K - K32 in FP32 (mixed path: K = K32 + K32lo to 48 bits)
    const double* KM64;        // K + alpha M^ (floating patches), all levels
    const float* KM32;
    const double* tab;
    const float* tabf;
    const int* itab;
    const double* A0inv64;
    const float* A0inv32;
    const int* crow_ptr;       // C rows: entries [crow_ptr[j], crow_ptr[j+1])
    const int* c_idx;          // local function index
    const double* c_w;         // weight
    double* phi;               // primal basis pool
    double* cg;                // FP64 vector pool
    void* lv;                  // level vector pool (double or float)
    const double* in;          // torn input
    double* out;               // torn output
    const double* rpi_loc;     // per C row: Phi^T g
    const double* upi_loc;     // per C row: (A u_Pi)
    int* its;                  // per slot iterations
    int* flags;
    double tol;
    int maxit;
    int nu1, nu2;
    double alpha;
    int ncycles;               // Schur / K-hat: V-cycles; V-cycle mode: cycles
    double theta;              // power mode: omega_k = theta (1 - rho_k^ncycles)
    double* omega;             // per patch BPCG scaling (written by the power mode, read by K-hat)
    double* szW;               // SZ basis: W = Khat^{-1} C^T pool (layout of phi)
    const double* szHinv;      // SZ basis: Hhat^{-1} pool (PatchDesc::szhoff)
    const double* band;        // D-MG: banded Cholesky factors (PatchDesc::bandoff)
    long long* vstats;         // [0] V-cycles, [1] V-cycle fine dofs (atomically added)
    size_t smem_bytes;         // dynamic shared memory of the launch (specialised kernels)
    int* dbg;                  // self-check record (debug builds only)
    long long* phase;          // phase timers (profiling builds only)
    // batched launches (several handles in one grid): per-handle arguments,
    // indexed by SlotDesc::handle; slots, nslots and smem_bytes of the launch
    // itself stay those of this struct.  nullptr: a single handle.
    const SolveArgs* batch;
    // [start, end] of the launch in globaltimer nanoseconds (or null): thread
    // 0 of every CTA lowers the start at entry and raises the end at exit
    unsigned long long* tspan;
    // high-order multigrid (null: the standard hierarchy): per-patch
    // descriptors and pools (FP64 / FP32), and the degree-1 hierarchies of
    // the companion problem (patch descriptors and value, table and
    // coarsest-inverse pools)
    const HoDesc* ho;
    const double* ho64;
    const float* ho32;
    const PatchDesc* sub_pd;
    const double* sub_K64;
    const float* sub_K32;
    const double* sub_tab;
    const float* sub_tabf;
    const int* sub_itab;
    const double* sub_A0inv64;
    const float* sub_A0inv32;
    // kernel variant switches for measurements (IETIDP_KFLAGS, 0 = all on):
    // 4 FP64 operator reads its input from global memory, 16 no L2 prefetch
    // of streamed color blocks, 32 the mixed path's stiffness operator in
    // FP64 instead of FP32 pairs, 128 that operator with its input in
    // natural order instead of the color-major ghost-padded layout, 256 one
    // lane per row in every color step (no lane groups on coarse levels)
    int kflags;
    // launch shape (host side): CTAs per slot, as one thread-block cluster
    // (global-vector variant, solve-phase modes); 0 or 1 = one CTA per slot
    int csize;
};

// generic kernel (degrees known at run time only)
cudaError_t launch_solve(const SolveArgs& a, int threads, cudaStream_t st);
// D-MG: Neumann solves of the slots by the banded Cholesky factors (same
// input / output conventions as MODE_NEUMANN); a.smem_bytes: dynamic shared
// memory for the substitution vector (slots whose n doubles fit use it)
constexpr size_t kDirectSmemCap = 160 * 1024;
cudaError_t launch_direct_neumann(const SolveArgs& a, int max_bw, cudaStream_t st);
// kernel specialised for (dim, p0, p1, p2); cudaErrorNotSupported if none exists
bool solve_variant_exists(int dim, int p0, int p1, int p2, int mixed);
// xg: V-cycle vectors in global memory (patches whose vectors exceed the
// shared-memory budget)
cudaError_t launch_solve_variant(const SolveArgs& a, int dim, int p0, int p1, int p2, int threads,
                                 cudaStream_t st, bool xg);
// resident CTAs per SM of a specialised launch (0 if no such kernel)
int solve_variant_ctas_per_sm(int dim, int p0, int p1, int p2, int mixed, bool xg, int threads, size_t smem);
// shared memory a specialised launch would use for this patch (uncapped)
size_t solve_smem_need(const PatchDesc& P, int mixed, bool xg = false);
// shared memory below which the specialised kernel cannot run this patch
size_t solve_smem_min(const PatchDesc& P, int mixed);
// shared memory of the per-level color tables alone (global-memory-vector variant's minimum)
size_t solve_smem_tables(const PatchDesc& P);

// ---- dual / primal helpers ---------------------------------------------------
struct DualArgs {
    int nlam;
    const long long* la; const long long* lb;   // torn indices of the two copies
    const int* ma; const int* mb;               // multiplicities
    int nie;                                    // interface torn entries
    const long long* ie_idx; const int* ie_mult;
    const int* ie_ptr; const int* ie_lam; const signed char* ie_sgn;
};

cudaError_t launch_bt(const DualArgs& d, const double* lam, double* torn, int scaled, cudaStream_t st);
cudaError_t launch_b(const DualArgs& d, const double* torn, double* q, int scaled, cudaStream_t st);
cudaError_t launch_jump_scale(const DualArgs& d, const double* torn, double* out2, cudaStream_t st);

cudaError_t launch_primal_restrict(const PatchDesc* pd, int nrows, const int* crow_patch,
                                   const int* crow_local, const double* phi, const double* g,
                                   double* rpi_loc, cudaStream_t st);
cudaError_t launch_coarse_solve(int npi, int nrows, const int* crow_glob, const int* gptr,
                                const int* glist, const double* Linv, const double* rpi_loc,
                                double* upi, double* upi_loc, cudaStream_t st);
cudaError_t launch_spp_local(const PatchDesc* pd, int nrows, const int* crow_patch,
                             const int* crow_local, const double* phi, const double* K64,
                             double* work, long long work_stride, double* sloc,
                             const long long* sloc_off, cudaStream_t st);
cudaError_t launch_spp_assemble(int npatch, const PatchDesc* pd, const int* crow_glob,
                                const double* sloc, const long long* sloc_off, double* S,
                                int npi, cudaStream_t st);

// outer PCG (one CTA): state = [rz, pq, alpha, beta, rr, nd, ...]
cudaError_t launch_outer_init(int n, const double* d, double* lam, double* r, double* state,
                              cudaStream_t st);
cudaError_t launch_outer_first(int n, const double* r, const double* z, double* p, double* state,
                               cudaStream_t st);
cudaError_t launch_outer_step1(int n, const double* p, const double* q, double* lam, double* r,
                               double* state, double* hist, int it, cudaStream_t st);
cudaError_t launch_outer_step2(int n, const double* r, const double* z, double* p, double* state,
                               double* hist, int it, cudaStream_t st);
cudaError_t launch_axpy_torn(long long n, const double* a, double s, const double* b,
                             double* out, cudaStream_t st);
cudaError_t launch_apply_K(const PatchDesc* pd, int npatch, const double* K64, const double* x,
                           double* y, cudaStream_t st);
