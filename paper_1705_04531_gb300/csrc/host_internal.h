// Host-side data model shared by the files of the C ABI (setup, solve
// engine, server): device-memory owner, assembled problem, IETI-DP handle.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/ietidp.h"
#include "kernels.cuh"

namespace ieti_host {

// error text of the calling thread (ietidp_last_error)
extern thread_local std::string g_err;
// kernels launched by the library in this process (ietidp_kernel_launches)
extern std::atomic<long long> g_kernel_launches;

inline int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define CU(x)                                                                        \
    do {                                                                             \
        cudaError_t e_ = (x);                                                        \
        if (e_ != cudaSuccess)                                                       \
            return fail(e_ == cudaErrorMemoryAllocation ? IETIDP_E_OOM : IETIDP_E_CUDA, \
                        std::string(#x) + ": " + cudaGetErrorString(e_));            \
    } while (0)

#define CHK(x)                         \
    do {                               \
        int rc_ = (x);                 \
        if (rc_ != IETIDP_OK) return rc_; \
    } while (0)

// Device allocations of one owner, stream-ordered (cudaMallocAsync /
// cudaFreeAsync on the owner's stream), so that releasing one problem's memory
// never synchronizes work that other streams have in flight.
struct DevMem {
    cudaStream_t st = nullptr;
    std::vector<void*> ptrs;
    long long bytes = 0;
    template <class T>
    int alloc(T** p, long long n) {
        *p = nullptr;
        if (n <= 0) n = 1;
        void* q = nullptr;
        cudaError_t e = cudaMallocAsync(&q, sizeof(T) * (size_t)n, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(IETIDP_E_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
        }
        ptrs.push_back(q);
        bytes += (long long)sizeof(T) * n;
        *p = (T*)q;
        return IETIDP_OK;
    }
    template <class T>
    int upload(T** p, const std::vector<T>& v, cudaStream_t s) {
        CHK(alloc(p, (long long)v.size()));
        if (!v.empty()) CU(cudaMemcpyAsync(*p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s));
        return IETIDP_OK;
    }
    void release() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
        ptrs.clear();
        bytes = 0;
    }
};

}  // namespace ieti_host

struct iga_problem {
    int dim = 0, npatch = 0;
    std::vector<iga_patch_desc> patches;
    std::vector<iga_interface_desc> interfaces;   // as given (companion problems of the high-order multigrid)
    std::vector<int> m;          // npatch*3 functions per direction
    std::vector<int> dmask;
    std::vector<long long> toff; // npatch+1
    long long ntorn = 0;
    // conforming identification: class id per torn index (-1 = patch-interior)
    std::vector<long long> cls;      // per torn index: class id or -1
    std::vector<std::vector<long long>> classes;   // torn indices of each class (sorted)
    std::vector<char> cls_dir;       // class on the Dirichlet boundary
    cudaStream_t stream = nullptr;
    ieti_host::DevMem mem;
    double* K64 = nullptr;           // fine stiffness (per patch, color-major)
    std::vector<long long> koff;     // per patch offset in K64
    std::vector<int> Sp;             // per patch padded row length
    double* f = nullptr;             // load (torn)
};

struct SlotGroup {        // slots served by one kernel specialisation
    int dim, p0, p1, p2;
    bool generic = false;     // run-time-degree kernel (no specialisation)
    bool xg = false;          // specialised kernel with V-cycle vectors in global memory
    SlotDesc* d = nullptr;    // device copy of the slots
    std::vector<SlotDesc> hs; // host copy (batched launches merge these)
    int n = 0;
    int its_off = 0;
    size_t smem = 0;
};

constexpr size_t kSmemCap = kSolveSmemCap;   // dynamic shared memory per CTA

struct ietidp_handle {
    // unique for the life of the process (a freed handle's address can be
    // reused by the next one; captured launch graphs are keyed by this)
    unsigned long long serial = 0;
    const iga_problem* prob = nullptr;
    ietidp_options opt;
    cudaStream_t st = nullptr;
    ieti_host::DevMem mem;
    int npatch = 0, dim = 0;
    std::vector<PatchDesc> pd;
    PatchDesc* d_pd = nullptr;
    double* K64 = nullptr;
    float* K32 = nullptr;
    float* K32lo = nullptr;   // K - K32 rounded to FP32 (mixed path)
    double* KM64 = nullptr;   // K + alpha M^ on floating patches (same offsets as K64)
    float* KM32 = nullptr;
    double* tab = nullptr;
    float* tabf = nullptr;
    int* itab = nullptr;
    double* A0inv64 = nullptr;
    float* A0inv32 = nullptr;
    // high-order multigrid: per-patch descriptors and operator pools, and the
    // companion degree-1 problem whose standard hierarchies sit below the
    // finest level (set up as a handle of its own, destroyed with this one)
    std::vector<HoDesc> ho;
    HoDesc* d_ho = nullptr;
    double* ho64 = nullptr;
    float* ho32 = nullptr;
    iga_problem* ho_prob = nullptr;
    ietidp_handle* ho_sub = nullptr;
    // constraints
    int nrows = 0, npi = 0;
    int *crow_ptr = nullptr, *c_idx = nullptr, *crow_patch = nullptr, *crow_local = nullptr,
        *crow_glob = nullptr, *gptr = nullptr, *glist = nullptr;
    double* c_w = nullptr;
    double* phi = nullptr;
    double* szW = nullptr;        // SZ basis: Khat^{-1} C^T (layout of phi)
    double* szHinv = nullptr;     // SZ basis: Hhat^{-1} per patch
    double* band = nullptr;       // D-MG: banded Cholesky factors of the fine stiffness
    int max_bw = 0;               // D-MG: largest half band width of the patches
    size_t direct_smem = 0;       // D-MG: shared memory of the substitution vector (largest patch that fits)
    double* Linv = nullptr;
    std::vector<double> spp_host;
    double *rloc = nullptr, *upi = nullptr, *uloc = nullptr;
    // dual
    DualArgs dual{};
    int nlam = 0;
    // slots
    std::vector<SlotGroup> gpatch;       // one slot per patch (Neumann / Schur)
    std::vector<SlotGroup> gbasis;       // one slot per primal row
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    double* cg = nullptr;
    void* lv = nullptr;
    int* its = nullptr;
    int* flags = nullptr;
    int* dbg = nullptr;       // self-check record of debug builds (6 ints)
    long long* phase = nullptr;   // phase timers of profiling builds (64)
    long long* vst = nullptr;     // [0..4] Neumann-type stats, [8..12] basis stats
    // torn buffers
    double *gF = nullptr, *uF = nullptr, *vS = nullptr, *wS = nullptr, *gR = nullptr, *tmp = nullptr;
    double *fH = nullptr, *uH = nullptr;   // device staging of ietidp_solve_host
    // dual vectors
    double *lam = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *d = nullptr;
    double *state = nullptr, *hist = nullptr, *scal = nullptr;
    double* h_pinned = nullptr;
    double t_setup_ms = 0;
    long long launches = 0;         // kernels launched since the last reset
    std::vector<cudaEvent_t> ev;    // Neumann solver launch brackets (pairs)
    int nev_used = 0;
    double basis_it_avg = 0;
    int basis_it_max = 0;
    int n_floating = 0;
    int device = 0;                 // device current at setup
    long long cg_patch_elems = 0;   // FP64 scratch used by the per-patch slots
    long long lv_patch_elems = 0;   // level-vector scratch used by the per-patch slots
    void* noalloc_base = nullptr;   // device address of the static scratch of ietidp_vcycles_noalloc
    struct ieti_engine* engine = nullptr;   // solve engine on this handle's stream (created on first solve)
    struct ieti_saddle_bufs* saddle = nullptr;   // MG-MG-S vectors (created on first saddle solve)
};

// high-order multigrid operators of every patch (highorder_setup.cu)
int ieti_ho_build(const iga_problem* Pb, const std::vector<PatchDesc>& pd, double alpha, std::vector<HoDesc>& desc,
                  std::vector<double>& pool);

// release the host part of the MG-MG-S buffers (device memory is the handle's)
void ieti_saddle_free(ietidp_handle* h);

// kernel arguments of one handle for a local-solve launch (slots, nslots and
// smem_bytes are filled by the caller)
SolveArgs ieti_solve_args(const ietidp_handle* h, int mode, const double* in, double* out, double tol, int maxit,
                          long long* vst);
