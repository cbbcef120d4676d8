// Host side of the C ABI: descriptor validation, multipatch topology
// (interfaces, Dirichlet sides, conforming identification of interface
// functions, primal objects, multipliers) as integer tables, device memory,
// and the launch sequence of assembly, setup and the dual CG of Sec. 2-4.
// No floating-point arithmetic of the method runs here: every number the
// solver computes comes from a kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <tuple>
#include <vector>

#include "host_internal.h"
#include "engine.h"

// device address of the static scratch of ietidp_vcycles_noalloc on the
// current device (defined with the array at the end of this file)
static cudaError_t ieti_noalloc_address(void** p);

// small vectors of one SZ basis slot (sz_device.cuh: kSmall)
static constexpr long long ieti_sz_small() { return 64; }

namespace ieti_host {
thread_local std::string g_err;
std::atomic<long long> g_kernel_launches{0};
}  // namespace ieti_host
using namespace ieti_host;

namespace {

struct UF {
    std::vector<long long> par;
    explicit UF(long long n) : par(n) { std::iota(par.begin(), par.end(), 0LL); }
    long long find(long long x) {
        while (par[x] != x) {
            par[x] = par[par[x]];
            x = par[x];
        }
        return x;
    }
    void unite(long long a, long long b) {
        a = find(a);
        b = find(b);
        if (a != b) par[std::max(a, b)] = std::min(a, b);
    }
};

}  // namespace

// ---------------------------------------------------------------------------
extern "C" const char* ietidp_last_error(void) { return g_err.c_str(); }

extern "C" long long ietidp_kernel_launches(void) { return g_kernel_launches.load(); }

// set the calling thread's error text (used by the server to hand a worker's
// error to the thread that polls the request)
void ieti_set_error(const std::string& msg) { g_err = msg; }

extern "C" void ietidp_default_options(ietidp_options* o) {
    std::memset(o, 0, sizeof(*o));
    o->primal = IETIDP_PRIMAL_VERTEX;
    o->precision = IETIDP_PREC_FP64;
    o->tol_outer = 1e-10;
    o->tol_inner = 1e-12;
    o->tol_basis = 1e-12;
    o->maxit_outer = 500;
    o->maxit_inner = 500;
    o->nu_pre = 2;
    o->nu_post = 2;
    o->coarse_elems = 4;
    o->dirichlet_vcycles = 2;
    o->alpha_reg = 1e-2;
    o->cluster = 0;
    o->method = IETIDP_METHOD_DUAL;
    o->saddle_vcycles = 3;
    o->saddle_theta = 0.9;
    o->basis_method = IETIDP_BASIS_SZ;
    o->mg_kind = IETIDP_MG_STANDARD;
}

// ---------------------------------------------------------------------------
// topology
// ---------------------------------------------------------------------------
static int build_topology(const iga_domain_desc* D, iga_problem* P) {
    int d = D->dim, N = D->npatch;
    P->dim = d;
    P->npatch = N;
    P->patches.assign(D->patches, D->patches + N);
    P->m.assign(3 * N, 1);
    P->toff.assign(N + 1, 0);
    for (int k = 0; k < N; ++k) {
        const iga_patch_desc& pk = D->patches[k];
        long long n = 1;
        for (int r = 0; r < d; ++r) {
            if (pk.degree[r] < 1 || pk.degree[r] > IETI_MAXP - 1)
                return fail(IETIDP_E_INVALID_ARG, "degree out of range [1,7] on patch " + std::to_string(k));
            if (pk.nelem[r] < 1) return fail(IETIDP_E_INVALID_ARG, "nelem < 1 on patch " + std::to_string(k));
            P->m[3 * k + r] = pk.nelem[r] + pk.degree[r];
            n *= P->m[3 * k + r];
        }
        if (pk.geo_kind != IGA_GEO_BOX && pk.geo_kind != IGA_GEO_ANNULUS)
            return fail(IETIDP_E_INVALID_ARG, "unknown geometry kind");
        if (pk.geo_kind == IGA_GEO_ANNULUS && d != 2)
            return fail(IETIDP_E_INVALID_ARG, "annulus geometry is two-dimensional");
        for (int r = 0; r < d; ++r)
            if (!(pk.hi[r] > pk.lo[r]) || !std::isfinite(pk.lo[r]) || !std::isfinite(pk.hi[r]))
                return fail(IETIDP_E_INVALID_ARG, "degenerate patch box on patch " + std::to_string(k));
        if (n > (1LL << 30)) return fail(IETIDP_E_INVALID_ARG, "patch too large");
        P->toff[k + 1] = P->toff[k] + n;
    }
    P->ntorn = P->toff[N];
    std::vector<int> partner(N * 6, -1);
    UF uf(P->ntorn);
    auto lidx = [&](int k, int i0, int i1, int i2) -> long long {
        return P->toff[k] + i0 + (long long)P->m[3 * k] * (i1 + (long long)P->m[3 * k + 1] * i2);
    };
    for (int t = 0; t < D->ninterface; ++t) {
        const iga_interface_desc& I = D->interfaces[t];
        if (I.patch_a < 0 || I.patch_a >= N || I.patch_b < 0 || I.patch_b >= N || I.patch_a == I.patch_b)
            return fail(IETIDP_E_INVALID_ARG, "interface " + std::to_string(t) + ": bad patch index");
        if (I.side_a < 0 || I.side_a >= 2 * d || I.side_b < 0 || I.side_b >= 2 * d)
            return fail(IETIDP_E_INVALID_ARG, "interface " + std::to_string(t) + ": bad side");
        if (partner[I.patch_a * 6 + I.side_a] >= 0 || partner[I.patch_b * 6 + I.side_b] >= 0)
            return fail(IETIDP_E_INVALID_ARG, "interface " + std::to_string(t) + ": side used twice");
        partner[I.patch_a * 6 + I.side_a] = I.patch_b;
        partner[I.patch_b * 6 + I.side_b] = I.patch_a;
        int ka = I.patch_a, kb = I.patch_b;
        int ra = I.side_a / 2, rb = I.side_b / 2;
        int ta[2] = {-1, -1}, tb[2] = {-1, -1}, na = 0, nb = 0;
        for (int r = 0; r < d; ++r) {
            if (r != ra) ta[na++] = r;
            if (r != rb) tb[nb++] = r;
        }
        if (d == 3 && I.swap) std::swap(tb[0], tb[1]);
        for (int u = 0; u < d - 1; ++u) {
            const iga_patch_desc &A = D->patches[ka], &B = D->patches[kb];
            if (A.degree[ta[u]] != B.degree[tb[u]] || A.nelem[ta[u]] != B.nelem[tb[u]])
                return fail(IETIDP_E_INVALID_ARG,
                            "interface " + std::to_string(t) + " is not conforming (degree/elements differ)");
        }
        int ma[3] = {P->m[3 * ka], P->m[3 * ka + 1], P->m[3 * ka + 2]};
        int mb[3] = {P->m[3 * kb], P->m[3 * kb + 1], P->m[3 * kb + 2]};
        int u0n = ma[ta[0]], u1n = d == 3 ? ma[ta[1]] : 1;
        for (int u1 = 0; u1 < u1n; ++u1)
            for (int u0 = 0; u0 < u0n; ++u0) {
                int ia[3] = {0, 0, 0}, ib[3] = {0, 0, 0};
                ia[ra] = (I.side_a & 1) ? ma[ra] - 1 : 0;
                ia[ta[0]] = u0;
                if (d == 3) ia[ta[1]] = u1;
                ib[rb] = (I.side_b & 1) ? mb[rb] - 1 : 0;
                int v[2] = {u0, u1};
                for (int q = 0; q < d - 1; ++q) {
                    int val = v[q];
                    if (I.flip[q]) val = mb[tb[q]] - 1 - val;
                    ib[tb[q]] = val;
                }
                uf.unite(lidx(ka, ia[0], ia[1], ia[2]), lidx(kb, ib[0], ib[1], ib[2]));
            }
    }
    P->dmask.assign(N, 0);
    for (int k = 0; k < N; ++k)
        for (int s = 0; s < 2 * d; ++s)
            if (partner[k * 6 + s] < 0) P->dmask[k] |= 1 << s;
    // classes of identified boundary functions
    std::map<long long, int> root2cls;
    P->cls.assign(P->ntorn, -1);
    for (int k = 0; k < N; ++k) {
        int* mm = &P->m[3 * k];
        for (int i2 = 0; i2 < mm[2]; ++i2)
            for (int i1 = 0; i1 < mm[1]; ++i1)
                for (int i0 = 0; i0 < mm[0]; ++i0) {
                    if (!ieti_on_boundary(mm, d, i0, i1, i2)) continue;
                    long long g = lidx(k, i0, i1, i2);
                    long long rt = uf.find(g);
                    auto it = root2cls.find(rt);
                    int c;
                    if (it == root2cls.end()) {
                        c = (int)P->classes.size();
                        root2cls[rt] = c;
                        P->classes.emplace_back();
                        P->cls_dir.push_back(0);
                    } else {
                        c = it->second;
                    }
                    P->cls[g] = c;
                    P->classes[c].push_back(g);
                    if (ieti_masked(P->dmask[k], mm, i0, i1, i2)) P->cls_dir[c] = 1;
                }
    }
    for (auto& c : P->classes) std::sort(c.begin(), c.end());
    return IETIDP_OK;
}

static int patch_of(const iga_problem* P, long long g) {
    return (int)(std::upper_bound(P->toff.begin(), P->toff.end(), g) - P->toff.begin()) - 1;
}

static void local_coords(const iga_problem* P, int k, long long g, int* ii) {
    long long loc = g - P->toff[k];
    const int* mm = &P->m[3 * k];
    ii[0] = (int)(loc % mm[0]);
    ii[1] = (int)((loc / mm[0]) % mm[1]);
    ii[2] = (int)(loc / ((long long)mm[0] * mm[1]));
}

// ---------------------------------------------------------------------------
extern "C" int iga_topology(const iga_domain_desc* D, iga_topology_info* info, unsigned* dmask) {
    if (!D || !info) return fail(IETIDP_E_INVALID_ARG, "null argument");
    if (D->dim != 2 && D->dim != 3) return fail(IETIDP_E_INVALID_ARG, "dim must be 2 or 3");
    if (D->npatch < 1 || !D->patches) return fail(IETIDP_E_INVALID_ARG, "no patches");
    if (D->ninterface < 0 || (D->ninterface > 0 && !D->interfaces))
        return fail(IETIDP_E_INVALID_ARG, "bad interface list");
    iga_problem P;   // host part only: no device memory is allocated
    int rc = build_topology(D, &P);
    if (rc != IETIDP_OK) return rc;
    std::memset(info, 0, sizeof(*info));
    info->n_torn = P.ntorn;
    info->n_global = P.ntorn;
    info->n_classes = (long long)P.classes.size();
    for (size_t c = 0; c < P.classes.size(); ++c) {
        info->n_global -= (long long)P.classes[c].size() - 1;
        if (P.classes[c].size() >= 2) info->n_shared += 1;
        if (P.cls_dir[c]) info->n_dirichlet += 1;
    }
    for (int k = 0; k < P.npatch; ++k) {
        if (P.dmask[k] == 0) info->n_floating += 1;
        if (dmask) dmask[k] = (unsigned)P.dmask[k];
    }
    return IETIDP_OK;
}

extern "C" int iga_assemble_patches(const iga_domain_desc* D, void* stream, iga_problem** out) {
    if (!D || !out) return fail(IETIDP_E_INVALID_ARG, "null argument");
    *out = nullptr;
    if (D->dim != 2 && D->dim != 3) return fail(IETIDP_E_INVALID_ARG, "dim must be 2 or 3");
    if (D->npatch < 1 || !D->patches) return fail(IETIDP_E_INVALID_ARG, "no patches");
    if (D->ninterface < 0 || (D->ninterface > 0 && !D->interfaces))
        return fail(IETIDP_E_INVALID_ARG, "bad interface list");
    if (D->rhs_kind < IGA_RHS_NONE || D->rhs_kind > IGA_RHS_QUAD) return fail(IETIDP_E_INVALID_ARG, "bad rhs kind");
    if (D->rhs_kind == IGA_RHS_QUAD && !D->quad_values) return fail(IETIDP_E_INVALID_ARG, "quad values missing");
    if (D->rhs_kind == IGA_RHS_MODES && (D->nmodes < 0 || (D->nmodes > 0 && (!D->mode_a || !D->mode_k || !D->mode_l))))
        return fail(IETIDP_E_INVALID_ARG, "bad modes");
    if ((D->rhs_kind == IGA_RHS_SIN3D) != (D->dim == 3 && D->rhs_kind == IGA_RHS_SIN3D))
        return fail(IETIDP_E_INVALID_ARG, "sin3d needs dim 3");
    auto* P = new iga_problem();
    P->stream = (cudaStream_t)stream;
    P->mem.st = P->stream;
    if (D->ninterface > 0) P->interfaces.assign(D->interfaces, D->interfaces + D->ninterface);
    int rc = build_topology(D, P);
    if (rc != IETIDP_OK) {
        delete P;
        return rc;
    }
    cudaStream_t st = P->stream;
    int d = D->dim, N = D->npatch;
    // single-level descriptors for assembly
    std::vector<PatchDesc> pd(N);
    std::vector<AsmTables> at(3 * N);
    std::vector<long long> qpoff(N + 1, 0), rowoff(N + 1, 0);
    std::vector<double> geo(7 * N, 0.0);
    long long qoff = 0, boff = 0, koff = 0;
    int max_S = 1;
    P->koff.assign(N, 0);
    for (int k = 0; k < N; ++k) {
        const iga_patch_desc& pk = D->patches[k];
        PatchDesc& q = pd[k];
        std::memset(&q, 0, sizeof(q));
        q.dim = d;
        for (int r = 0; r < 3; ++r) {
            q.p[r] = r < d ? pk.degree[r] : 0;
            q.nelem[r] = r < d ? pk.nelem[r] : 1;
        }
        q.L = 1;
        q.dmask = P->dmask[k];
        q.floating = P->dmask[k] == 0;
        q.toff = P->toff[k];
        LevelDesc& L = q.lev[0];
        L.n = 1;
        L.S = 1;
        for (int r = 0; r < 3; ++r) {
            L.m[r] = P->m[3 * k + r];
            L.n *= L.m[r];
            L.S *= 2 * q.p[r] + 1;
        }
        L.Sp = ieti_sp(L.S);
        q.n = L.n;
        L.koff = koff;
        P->koff[k] = koff;
        koff += (long long)L.n * L.Sp;
        max_S = std::max(max_S, L.S);
        long long nqp = 1;
        for (int r = 0; r < 3; ++r) {
            AsmTables& t = at[3 * k + r];
            t.nq = r < d ? pk.nelem[r] * (pk.degree[r] + 1) : 1;
            t.qoff = qoff;
            t.boff = boff;
            qoff += t.nq;
            boff += (long long)t.nq * (q.p[r] + 1);
            nqp *= t.nq;
        }
        qpoff[k + 1] = qpoff[k] + nqp;
        rowoff[k + 1] = rowoff[k] + L.n;
        geo[7 * k] = pk.geo_kind;
        for (int r = 0; r < 3; ++r) {
            geo[7 * k + 1 + r] = pk.lo[r];
            geo[7 * k + 4 + r] = pk.hi[r];
        }
    }
    long long total_qp = qpoff[N];
    DevMem scratch;
    scratch.st = st;
    SetupArgs a{};
    a.npatch = N;
    a.dim = d;
    PatchDesc* d_pd;
    AsmTables* d_at;
    long long *d_qpoff, *d_rowoff;
    double *d_geo, *d_modes = nullptr;
    int* d_flags;
    std::vector<double> modes;
    if (D->rhs_kind == IGA_RHS_MODES)
        for (int j = 0; j < D->nmodes; ++j) {
            modes.push_back(D->mode_a[j]);
            modes.push_back(D->mode_k[j]);
            modes.push_back(D->mode_l[j]);
        }
#define CKS(x)                      \
    do {                            \
        int rc_ = (x);              \
        if (rc_ != IETIDP_OK) {     \
            scratch.release();      \
            P->mem.release();       \
            delete P;               \
            return rc_;             \
        }                           \
    } while (0)
    CKS(scratch.upload(&d_pd, pd, st));
    CKS(scratch.upload(&d_at, at, st));
    CKS(scratch.upload(&d_qpoff, qpoff, st));
    CKS(scratch.upload(&d_rowoff, rowoff, st));
    CKS(scratch.upload(&d_geo, geo, st));
    if (!modes.empty()) CKS(scratch.upload(&d_modes, modes, st));
    CKS(scratch.alloc(&a.qx, qoff));
    CKS(scratch.alloc(&a.qw, qoff));
    CKS(scratch.alloc(&a.Bv, boff));
    CKS(scratch.alloc(&a.Dv, boff));
    CKS(scratch.alloc(&a.Gm, 6 * total_qp));
    CKS(scratch.alloc(&a.Fw, total_qp));
    CKS(scratch.alloc(&d_flags, 1));
    CKS(P->mem.alloc(&P->K64, koff));
    CKS(P->mem.alloc(&P->f, P->ntorn));
    a.pd = d_pd;
    a.geo = d_geo;
    a.at = d_at;
    a.qpoff = d_qpoff;
    a.rowoff = d_rowoff;
    a.rhs_kind = D->rhs_kind;
    a.modes = d_modes;
    a.nmodes = (int)modes.size() / 3;
    a.quad_values = D->quad_values;
    a.K64 = P->K64;
    a.f = P->f;
    a.flags = d_flags;
    cudaError_t e = cudaMemsetAsync(d_flags, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_assembly(a, total_qp, rowoff[N], max_S, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    scratch.release();
    if (e != cudaSuccess) {
        P->mem.release();
        delete P;
        return fail(IETIDP_E_CUDA, std::string("assembly: ") + cudaGetErrorString(e));
    }
#undef CKS
    *out = P;
    return IETIDP_OK;
}

extern "C" int iga_problem_load(const iga_problem* P, double* f_out) {
    if (!P || !f_out) return fail(IETIDP_E_INVALID_ARG, "null argument");
    CU(cudaMemcpyAsync(f_out, P->f, sizeof(double) * P->ntorn, cudaMemcpyDeviceToDevice, P->stream));
    CU(cudaStreamSynchronize(P->stream));
    return IETIDP_OK;
}

extern "C" int iga_problem_free(iga_problem* P) {
    if (!P) return IETIDP_OK;
    P->mem.release();
    cudaStreamSynchronize(P->stream);
    delete P;
    return IETIDP_OK;
}

// ---------------------------------------------------------------------------
// setup
// ---------------------------------------------------------------------------
static std::vector<std::array<int, 3>> schedule(const int* nel, int d, int cmin) {
    std::vector<std::array<int, 3>> s;
    std::array<int, 3> cur = {nel[0], d > 1 ? nel[1] : 1, d > 2 ? nel[2] : 1};
    s.push_back(cur);
    while (true) {
        std::array<int, 3> nx = cur;
        for (int r = 0; r < d; ++r)
            if (cur[r] > cmin && cur[r] % 2 == 0) nx[r] = cur[r] / 2;
        if (nx == cur) break;
        s.push_back(nx);
        cur = nx;
    }
    std::reverse(s.begin(), s.end());
    return s;
}

static int launch_group(ietidp_handle* h, SolveArgs a, const SlotGroup& g, cudaStream_t st) {
    a.slots = g.d;
    a.nslots = g.n;
    a.its = h->its;
    a.smem_bytes = g.smem;
    cudaError_t e;
    if (a.mode == MODE_NEUMANN_DIRECT) {
        a.smem_bytes = h->direct_smem;
        e = launch_direct_neumann(a, h->max_bw, st);
    } else if (!g.generic) e = launch_solve_variant(a, g.dim, g.p0, g.p1, g.p2, 512, st, g.xg);
    else e = launch_solve(a, 512, st);
    h->launches += 1;
    g_kernel_launches += 1;
    if (e != cudaSuccess) return fail(IETIDP_E_CUDA, std::string("solve kernel: ") + cudaGetErrorString(e));
    return IETIDP_OK;
}

SolveArgs ieti_solve_args(const ietidp_handle* h, int mode, const double* in, double* out, double tol, int maxit,
                          long long* vst) {
    SolveArgs a{};
    a.pd = h->d_pd;
    a.mode = mode;
    a.mixed = h->opt.precision == IETIDP_PREC_MIXED;
    a.K64 = h->K64;
    a.K32 = h->K32;
    a.K32lo = h->K32lo;
    a.KM64 = h->KM64;
    a.KM32 = h->KM32;
    a.tab = h->tab;
    a.tabf = h->tabf;
    a.itab = h->itab;
    a.A0inv64 = h->A0inv64;
    a.A0inv32 = h->A0inv32;
    a.crow_ptr = h->crow_ptr;
    a.c_idx = h->c_idx;
    a.c_w = h->c_w;
    a.phi = h->phi;
    a.cg = h->cg;
    a.lv = h->lv;
    a.in = in;
    a.out = out;
    a.rpi_loc = h->rloc;
    a.upi_loc = h->uloc;
    a.its = h->its;
    a.flags = h->flags;
    a.tol = tol;
    a.maxit = maxit;
    a.nu1 = h->opt.nu_pre;
    a.nu2 = h->opt.nu_post;
    a.alpha = h->opt.alpha_reg;
    a.ncycles = h->opt.dirichlet_vcycles;
    a.vstats = vst;
    a.dbg = h->dbg;
    a.phase = h->phase;
    a.batch = nullptr;
    a.szW = h->szW;
    a.szHinv = h->szHinv;
    a.band = h->band;
    static const int kflags = [] {
        const char* e = std::getenv("IETIDP_KFLAGS");
        return e ? std::atoi(e) : 0;
    }();
    a.kflags = kflags;
    // the high-order multigrid serves the solve phase; the primal basis
    // (Eq. 6) is computed with the patch's standard hierarchy, whose
    // symmetric Gauss-Seidel V-cycle V satisfies V K <= 1 as the
    // Schoeberl-Zulehner CG requires (K^ = (0.99 V)^-1 > K); the
    // subspace-corrected mass smoother may overshoot (eigenvalues of V K up to
    // 1 + its contraction rate), which makes K^ - K indefinite
    const bool basis_mode = mode == MODE_BASIS || mode == MODE_SZW || mode == MODE_BASIS_SZ;
    if (h->d_ho && !basis_mode) {
        const ietidp_handle* s = h->ho_sub;
        a.ho = h->d_ho;
        a.ho64 = h->ho64;
        a.ho32 = h->ho32;
        a.sub_pd = s->d_pd;
        a.sub_K64 = s->K64;
        a.sub_K32 = s->K32;
        a.sub_tab = s->tab;
        a.sub_tabf = s->tabf;
        a.sub_itab = s->itab;
        a.sub_A0inv64 = s->A0inv64;
        a.sub_A0inv32 = s->A0inv32;
    }
    if (mode == MODE_NEUMANN && h->opt.method == IETIDP_METHOD_DMG) a.mode = MODE_NEUMANN_DIRECT;
    return a;
}

// launch the slot groups with prepared kernel arguments on the handle's
// stream (groups of different specialisations concurrently on side streams)
static int run_solve_args(ietidp_handle* h, const SolveArgs& a, const std::vector<SlotGroup>& groups) {
    bool timed = a.mode == MODE_NEUMANN && h->nev_used + 2 <= (int)h->ev.size();
    if (timed) cudaEventRecord(h->ev[h->nev_used], h->st);
    if (groups.size() == 1) {
        CHK(launch_group(h, a, groups[0], h->st));
    } else if (!groups.empty()) {
        // groups of different specialisations run concurrently on side streams
        CU(cudaEventRecord(h->fork, h->st));
        for (size_t i = 0; i < groups.size(); ++i) {
            cudaStream_t s = h->side[i % h->side.size()];
            CU(cudaStreamWaitEvent(s, h->fork, 0));
            CHK(launch_group(h, a, groups[i], s));
        }
        for (size_t i = 0; i < std::min(groups.size(), h->side.size()); ++i) {
            CU(cudaEventRecord(h->join[i], h->side[i]));
            CU(cudaStreamWaitEvent(h->st, h->join[i], 0));
        }
    }
    if (timed) {
        cudaEventRecord(h->ev[h->nev_used + 1], h->st);
        h->nev_used += 2;
    }
    return IETIDP_OK;
}

static int run_solve(ietidp_handle* h, int mode, const std::vector<SlotGroup>& groups, const double* in,
                     double* out, double tol, int maxit, long long* vst) {
    return run_solve_args(h, ieti_solve_args(h, mode, in, out, tol, maxit, vst), groups);
}

static int make_groups(ietidp_handle* h, const std::vector<SlotDesc>& slots, std::vector<SlotGroup>& out,
                       cudaStream_t st) {
    bool mixed = h->opt.precision == IETIDP_PREC_MIXED;
    // key: (dim, p0, p1, p2, kind) with kind 0 = specialised, vectors in
    // shared memory; 1 = specialised, vectors in global memory (they do not
    // fit the budget); 2 = run-time-degree kernel (no specialisation)
    std::map<std::tuple<int, int, int, int, int>, std::vector<SlotDesc>> by;
    // IETIDP_FORCE_GENERIC=1 routes every slot to the run-time-degree kernel
    // (used to test that kernel on sizes the specialised one also handles)
    const char* fg = std::getenv("IETIDP_FORCE_GENERIC");
    const bool force_generic = fg && fg[0] == '1';
    for (const SlotDesc& sd : slots) {
        const PatchDesc& P = h->pd[sd.patch];
        // the high-order V-cycle exists in the run-time-degree kernel only
        int gen = (force_generic || h->d_ho || !solve_variant_exists(P.dim, P.p[0], P.p[1], P.p[2], mixed))
                      ? 2
                      : (solve_smem_min(P, mixed) > kSmemCap ? 1 : 0);
        by[std::make_tuple(P.dim, P.p[0], P.p[1], P.p[2], gen)].push_back(sd);
    }
    int off = 0;
    for (auto& kv : by) {
        SlotGroup g;
        int gen;
        std::tie(g.dim, g.p0, g.p1, g.p2, gen) = kv.first;
        g.generic = gen == 2;
        g.xg = gen == 1;
        g.n = (int)kv.second.size();
        g.its_off = off;
        off += g.n;
        g.hs = kv.second;
        size_t need = 0;
        for (const SlotDesc& sd : kv.second) need = std::max(need, solve_smem_need(h->pd[sd.patch], mixed, g.xg));
        g.smem = std::min(need, kSmemCap);
        CHK(h->mem.upload(&g.d, kv.second, st));
        out.push_back(g);
    }
    return IETIDP_OK;
}

extern "C" int ietidp_setup(const iga_problem* P, const ietidp_options* opt_in, void* stream, ietidp_handle** out) {
    if (!P || !out) return fail(IETIDP_E_INVALID_ARG, "null argument");
    *out = nullptr;
    ietidp_options opt;
    if (opt_in) opt = *opt_in;
    else ietidp_default_options(&opt);
    if (opt.precision != IETIDP_PREC_FP64 && opt.precision != IETIDP_PREC_MIXED)
        return fail(IETIDP_E_INVALID_ARG, "bad precision");
    if (opt.nu_pre < 0 || opt.nu_post < 0 || opt.coarse_elems < 1 || opt.dirichlet_vcycles < 1 ||
        opt.maxit_inner < 1 || opt.maxit_outer < 0 || !(opt.tol_outer > 0) || !(opt.tol_inner > 0) ||
        !(opt.tol_basis > 0) || opt.alpha_reg < 0)
        return fail(IETIDP_E_INVALID_ARG, "bad options");
    if ((opt.method != IETIDP_METHOD_DUAL && opt.method != IETIDP_METHOD_SADDLE && opt.method != IETIDP_METHOD_DMG) ||
        opt.saddle_vcycles < 1 ||
        !(opt.saddle_theta > 0 && opt.saddle_theta < 1) ||
        (opt.basis_method != IETIDP_BASIS_SZ && opt.basis_method != IETIDP_BASIS_NULLSPACE) ||
        (opt.mg_kind != IETIDP_MG_STANDARD && opt.mg_kind != IETIDP_MG_HIGHORDER))
        return fail(IETIDP_E_INVALID_ARG, "bad method options");
    auto t0 = std::chrono::steady_clock::now();
    static std::atomic<unsigned long long> g_serial{0};
    auto* h = new ietidp_handle();
    h->serial = ++g_serial;
    h->prob = P;
    h->opt = opt;
    h->st = (cudaStream_t)stream;
    h->mem.st = h->st;
    int rc = IETIDP_OK;
    auto bail = [&](int code) {
        if (h->ho_sub) ietidp_destroy(h->ho_sub);
        if (h->ho_prob) iga_problem_free(h->ho_prob);
        h->mem.release();
        if (h->h_pinned) cudaFreeHost(h->h_pinned);
        delete h;
        return code;
    };
#define CKH(x)                         \
    do {                               \
        int rc_ = (x);                 \
        if (rc_ != IETIDP_OK) return bail(rc_); \
    } while (0)
#define CUH(x)                                                                       \
    do {                                                                             \
        cudaError_t e_ = (x);                                                        \
        if (e_ != cudaSuccess)                                                       \
            return bail(fail(e_ == cudaErrorMemoryAllocation ? IETIDP_E_OOM : IETIDP_E_CUDA, \
                             std::string(#x) + ": " + cudaGetErrorString(e_)));      \
    } while (0)
    cudaStream_t st = h->st;
    int d = P->dim, N = P->npatch;
    h->npatch = N;
    h->dim = d;
    CUH(cudaGetDevice(&h->device));
    // address of the no-allocation V-cycle scratch on this device: looking it
    // up here (where allocating is allowed) commits the array's memory under
    // lazy module loading, so that ietidp_vcycles_noalloc never does
    CUH(ieti_noalloc_address(&h->noalloc_base));
    // ---- high-order multigrid: the companion degree-1 problem --------------
    // Sec. 4: below the finest level the hierarchy continues with splines of
    // degree 1 on half the elements of every direction (same geometry map and
    // patch layout, so the interfaces stay conforming); its standard
    // hierarchies (both side masks) are those of a handle of its own
    if (opt.mg_kind == IETIDP_MG_HIGHORDER) {
        std::vector<iga_patch_desc> p1(P->patches);
        for (auto& q : p1)
            for (int r = 0; r < P->dim; ++r) {
                q.degree[r] = 1;
                q.nelem[r] = std::max(1, q.nelem[r] / 2);
            }
        iga_domain_desc D1{};
        D1.dim = P->dim;
        D1.npatch = P->npatch;
        D1.patches = p1.data();
        D1.ninterface = (int)P->interfaces.size();
        D1.interfaces = P->interfaces.empty() ? nullptr : P->interfaces.data();
        D1.rhs_kind = IGA_RHS_NONE;
        CKH(iga_assemble_patches(&D1, stream, &h->ho_prob));
        ietidp_options o1 = opt;
        o1.mg_kind = IETIDP_MG_STANDARD;
        o1.method = IETIDP_METHOD_DUAL;
        CKH(ietidp_setup(h->ho_prob, &o1, stream, &h->ho_sub));
    }
    // ---- primal objects and constraint rows -------------------------------
    // object kind of a class: number of directions in which its first copy
    // lies on the patch boundary
    int ncls = (int)P->classes.size();
    std::vector<int> ctype(ncls, 0);
    std::map<std::tuple<int, int, int, int>, int> objkey;   // (type, patch, sideinfo, root) -> object
    std::vector<int> cls_obj(ncls, -1);
    std::vector<int> obj_type;
    std::vector<std::vector<int>> obj_classes;
    for (int c = 0; c < ncls; ++c) {
        const auto& cp = P->classes[c];
        if (P->cls_dir[c] || cp.size() < 2) continue;
        int k0 = patch_of(P, cp[0]);
        int ii[3];
        local_coords(P, k0, cp[0], ii);
        int t = 0;
        for (int r = 0; r < d; ++r)
            if (ii[r] == 0 || ii[r] == P->m[3 * k0 + r] - 1) ++t;
        ctype[c] = t;
        // entity key: minimum over copies of (patch, sides the copy lies on)
        std::tuple<int, int, int, int> key(t, 1 << 30, 0, 0);
        if (t == d) {
            key = std::make_tuple(t, -1, 0, c);   // vertex: each class is its own object
        } else {
            for (long long g : cp) {
                int k = patch_of(P, g);
                int jj[3];
                local_coords(P, k, g, jj);
                int sides = 0;
                for (int r = 0; r < d; ++r) {
                    if (jj[r] == 0) sides |= 1 << (2 * r);
                    if (jj[r] == P->m[3 * k + r] - 1) sides |= 1 << (2 * r + 1);
                }
                auto cand = std::make_tuple(t, k, sides, 0);
                if (cand < key) key = cand;
            }
        }
        auto it = objkey.find(key);
        int o;
        if (it == objkey.end()) {
            o = (int)obj_type.size();
            objkey[key] = o;
            obj_type.push_back(t);
            obj_classes.emplace_back();
        } else {
            o = it->second;
        }
        cls_obj[c] = o;
        obj_classes[o].push_back(c);
    }
    auto kind_of = [&](int t) -> unsigned {
        if (t == d) return IETIDP_PRIMAL_VERTEX;
        if (d == 2) return IETIDP_PRIMAL_EDGE;
        return t == 2 ? IETIDP_PRIMAL_EDGE : IETIDP_PRIMAL_FACE;
    };
    std::vector<int> obj_primal(obj_type.size(), -1);
    int npi = 0;
    for (size_t o = 0; o < obj_type.size(); ++o)
        if (opt.primal & kind_of(obj_type[o])) obj_primal[o] = npi++;
    h->npi = npi;
    // rows per patch: (patch, object) -> entries
    std::vector<std::map<int, std::vector<int>>> rows(N);   // patch -> primal index -> local idx list
    std::vector<std::map<int, int>> rowtang(N);
    for (size_t o = 0; o < obj_type.size(); ++o) {
        if (obj_primal[o] < 0) continue;
        for (int c : obj_classes[o])
            for (long long g : P->classes[c]) {
                int k = patch_of(P, g);
                int jj[3];
                local_coords(P, k, g, jj);
                int tang = 0;
                for (int r = 0; r < d; ++r)
                    if (!(jj[r] == 0 || jj[r] == P->m[3 * k + r] - 1)) tang |= 1 << r;
                rows[k][obj_primal[o]].push_back((int)(g - P->toff[k]));
                rowtang[k][obj_primal[o]] = tang;
            }
    }
    std::vector<int> crow_ptr(1, 0), c_idx, crow_patch, crow_local, crow_glob, crow_tang;
    std::vector<int> npi_k(N, 0), crow0(N, 0);
    for (int k = 0; k < N; ++k) {
        crow0[k] = (int)crow_patch.size();
        int lr = 0;
        for (auto& kv : rows[k]) {
            std::vector<int> ent = kv.second;
            std::sort(ent.begin(), ent.end());
            c_idx.insert(c_idx.end(), ent.begin(), ent.end());
            crow_ptr.push_back((int)c_idx.size());
            crow_patch.push_back(k);
            crow_local.push_back(lr++);
            crow_glob.push_back(kv.first);
            crow_tang.push_back(rowtang[k][kv.first]);
        }
        npi_k[k] = lr;
        if (lr > 64) return bail(fail(IETIDP_E_INVALID_ARG, "more than 64 primal constraints on one patch"));
        if (P->dmask[k] == 0 && lr == 0)
            return bail(fail(IETIDP_E_INVALID_ARG,
                             "patch " + std::to_string(k) + " has no Dirichlet side and no primal constraint"));
    }
    h->nrows = (int)crow_patch.size();
    std::vector<int> gptr(npi + 1, 0), glist;
    {
        std::vector<std::vector<int>> bylist(npi);
        for (int j = 0; j < h->nrows; ++j) bylist[crow_glob[j]].push_back(j);
        for (int J = 0; J < npi; ++J) {
            glist.insert(glist.end(), bylist[J].begin(), bylist[J].end());
            gptr[J + 1] = (int)glist.size();
        }
    }
    // ---- multipliers ---------------------------------------------------------
    bool vertex_primal = opt.primal & IETIDP_PRIMAL_VERTEX;
    std::vector<long long> la, lb;
    std::vector<int> ma, mb;
    std::map<long long, std::vector<std::pair<int, int>>> ie;   // torn idx -> (lam, sign)
    std::map<long long, int> ie_mult;
    for (int c = 0; c < ncls; ++c) {
        const auto& cp = P->classes[c];
        if (P->cls_dir[c] || cp.size() < 2) continue;
        if (vertex_primal && ctype[c] == d) continue;
        int mu = (int)cp.size();
        for (size_t i = 0; i < cp.size(); ++i)
            for (size_t j = i + 1; j < cp.size(); ++j) {
                int l = (int)la.size();
                la.push_back(cp[i]);
                lb.push_back(cp[j]);
                ma.push_back(mu);
                mb.push_back(mu);
                ie[cp[i]].push_back({l, 1});
                ie[cp[j]].push_back({l, -1});
                ie_mult[cp[i]] = mu;
                ie_mult[cp[j]] = mu;
            }
    }
    h->nlam = (int)la.size();
    std::vector<long long> ie_idx;
    std::vector<int> ie_m, ie_ptr(1, 0), ie_lam;
    std::vector<signed char> ie_sgn;
    for (auto& kv : ie) {
        ie_idx.push_back(kv.first);
        ie_m.push_back(ie_mult[kv.first]);
        for (auto& ls : kv.second) {
            ie_lam.push_back(ls.first);
            ie_sgn.push_back((signed char)ls.second);
        }
        ie_ptr.push_back((int)ie_lam.size());
    }
    // ---- levels and descriptors ----------------------------------------------
    h->pd.resize(N);
    long long koff = 0, toff_tab = 0, itoff = 0, a0off = 0, phioff = 0, szhoff = 0, bandoff = 0;
    int max_n0 = 1, max_S = 1, max_rows_lev = 1, max_L = 1;
    std::vector<TableJob> tjobs, mjobs;
    long long cg_need = 0, lv_need = 0;
    for (int k = 0; k < N; ++k) {
        const iga_patch_desc& pk = P->patches[k];
        PatchDesc& q = h->pd[k];
        std::memset(&q, 0, sizeof(q));
        q.dim = d;
        for (int r = 0; r < 3; ++r) {
            q.p[r] = r < d ? pk.degree[r] : 0;
            q.nelem[r] = r < d ? pk.nelem[r] : 1;
        }
        auto sch = schedule(q.nelem, d, opt.coarse_elems);
        if ((int)sch.size() > IETI_MAXLEV) return bail(fail(IETIDP_E_INVALID_ARG, "too many levels"));
        q.L = (int)sch.size();
        max_L = std::max(max_L, q.L);
        q.dmask = P->dmask[k];
        q.floating = q.dmask == 0;
        if (q.floating) h->n_floating++;
        q.toff = P->toff[k];
        int voff = 0, xoff = 0, boff = 0;
        for (int l = 0; l < q.L; ++l) {
            LevelDesc& L = q.lev[l];
            L.n = 1;
            L.S = 1;
            for (int r = 0; r < 3; ++r) {
                L.m[r] = r < d ? sch[l][r] + q.p[r] : 1;
                L.n *= L.m[r];
                L.S *= 2 * q.p[r] + 1;
                L.refined[r] = (l > 0 && r < d && sch[l][r] != sch[l - 1][r]) ? 1 : 0;
            }
            L.Sp = ieti_sp(L.S);
            koff = (koff + 3) & ~3LL;
            L.koff = koff;
            koff += (long long)L.n * L.Sp;
            L.voff = voff;
            voff += L.n;
            for (int r = 0; r < 3; ++r) L.xk[r] = (r < d) ? ieti_xk(L.m[r], q.p[r]) : 1;
            L.blk = L.xk[0] * L.xk[1] * L.xk[2];
            L.nx = l >= 1 ? ieti_cm_size(L.m, q.p, d) : L.n;
            L.xoff = xoff;
            xoff += (L.nx + 3) & ~3;
            L.boff = boff;
            boff += (L.n + 3) & ~3;
            max_S = std::max(max_S, L.S);
            max_rows_lev = std::max(max_rows_lev, L.n);
            for (int r = 0; r < d; ++r) {
                int W = q.p[r] + 2;
                if (l > 0) {
                    int mc = q.lev[l - 1].m[r];
                    L.rs[r] = (int)itoff;
                    itoff += mc;
                    L.ps[r] = (int)itoff;
                    itoff += L.m[r];
                    L.rw[r] = (int)toff_tab;
                    toff_tab += (long long)mc * W;
                    L.pw[r] = (int)toff_tab;
                    toff_tab += (long long)L.m[r] * W;
                    tjobs.push_back({k, l, r});
                }
                L.mw[r] = (int)toff_tab;
                toff_tab += (long long)L.m[r] * (2 * q.p[r] + 1);
                mjobs.push_back({k, l, r});
            }
        }
        q.n = q.lev[q.L - 1].n;
        q.nlvec = voff;
        q.nlx = xoff;
        q.nlb = boff;
        int n0 = q.lev[0].n;
        max_n0 = std::max(max_n0, n0);
        q.a0off[0] = a0off;
        a0off += (long long)n0 * n0;
        q.a0off[1] = a0off;
        a0off += (long long)n0 * n0;
        q.npi = npi_k[k];
        q.crow0 = crow0[k];
        q.phioff = phioff;
        phioff += (long long)q.n * q.npi;
        q.szhoff = szhoff;
        szhoff += (long long)q.npi * q.npi;
        q.bw = q.p[0] + q.lev[q.L - 1].m[0] * (q.p[1] + q.lev[q.L - 1].m[1] * q.p[2]);
        q.pin = -1;
        q.bandoff = 0;
        if (opt.method == IETIDP_METHOD_DMG) {
            const int* mm = q.lev[q.L - 1].m;
            if (q.floating) q.pin = mm[0] / 2 + mm[0] * (mm[1] / 2 + mm[1] * (mm[2] / 2));
            q.bandoff = bandoff;
            bandoff += (long long)q.n * (q.bw + 1);
        }
        cg_need = std::max(cg_need, (long long)q.n);
        lv_need = std::max(lv_need, (long long)q.nlvec);
        if (toff_tab > (1LL << 31) - 1 || itoff > (1LL << 31) - 1) return bail(fail(IETIDP_E_INVALID_ARG, "tables too large"));
    }
    bool mixed = opt.precision == IETIDP_PREC_MIXED;
    // ---- device memory -------------------------------------------------------
    CKH(h->mem.upload(&h->d_pd, h->pd, st));
    if (opt.mg_kind == IETIDP_MG_HIGHORDER) {
        std::vector<double> pool;
        CKH(ieti_ho_build(P, h->pd, opt.alpha_reg, h->ho, pool));
        std::vector<float> pool32(pool.begin(), pool.end());
        CKH(h->mem.upload(&h->d_ho, h->ho, st));
        CKH(h->mem.upload(&h->ho64, pool, st));
        CKH(h->mem.upload(&h->ho32, pool32, st));
    }
    // value pools: 16 elements of tail padding, since the local solver reads
    // color blocks widened to 16-byte boundaries (bulk prefetches)
    CKH(h->mem.alloc(&h->K64, koff + 16));
    if (mixed) CKH(h->mem.alloc(&h->K32, koff + 16));
    if (mixed) CKH(h->mem.alloc(&h->K32lo, koff + 16));
    if (h->n_floating > 0) {
        CKH(h->mem.alloc(&h->KM64, koff + 16));
        if (mixed) CKH(h->mem.alloc(&h->KM32, koff + 16));
    }
    CKH(h->mem.alloc(&h->tab, toff_tab));
    CKH(h->mem.alloc(&h->tabf, toff_tab));
    CKH(h->mem.alloc(&h->itab, itoff));
    CKH(h->mem.alloc(&h->A0inv64, a0off));
    CKH(h->mem.alloc(&h->A0inv32, a0off));
    CKH(h->mem.upload(&h->crow_ptr, crow_ptr, st));
    CKH(h->mem.upload(&h->c_idx, c_idx, st));
    CKH(h->mem.upload(&h->crow_patch, crow_patch, st));
    CKH(h->mem.upload(&h->crow_local, crow_local, st));
    CKH(h->mem.upload(&h->crow_glob, crow_glob, st));
    CKH(h->mem.upload(&h->gptr, gptr, st));
    CKH(h->mem.upload(&h->glist, glist, st));
    std::vector<int> crow_tang_v = crow_tang;
    int* d_tang;
    CKH(h->mem.upload(&d_tang, crow_tang_v, st));
    CKH(h->mem.alloc(&h->c_w, (long long)c_idx.size()));
    CKH(h->mem.alloc(&h->phi, phioff));
    if (opt.method == IETIDP_METHOD_DMG) CKH(h->mem.alloc(&h->band, bandoff));
    const bool sz = opt.basis_method == IETIDP_BASIS_SZ;
    if (sz) {
        CKH(h->mem.alloc(&h->szW, phioff));
        CKH(h->mem.alloc(&h->szHinv, szhoff));
    }
    CKH(h->mem.alloc(&h->Linv, (long long)npi * npi));
    CKH(h->mem.alloc(&h->rloc, h->nrows));
    CKH(h->mem.alloc(&h->upi, npi));
    CKH(h->mem.alloc(&h->uloc, h->nrows));
    CKH(h->mem.alloc(&h->flags, 1));
    CKH(h->mem.alloc(&h->dbg, 8));
    CKH(h->mem.alloc(&h->phase, 64));
    CUH(cudaMemsetAsync(h->phase, 0, sizeof(long long) * 64, st));
    CUH(cudaMemsetAsync(h->dbg, 0, sizeof(int) * 8, st));
    CKH(h->mem.alloc(&h->vst, 16));
    CUH(cudaMemsetAsync(h->flags, 0, sizeof(int), st));
    CUH(cudaMemsetAsync(h->vst, 0, sizeof(long long) * 16, st));
    // dual
    DualArgs& du = h->dual;
    du.nlam = h->nlam;
    du.nie = (int)ie_idx.size();
    {
        long long* p1;
        long long* p2;
        int *p3, *p4, *p5, *p6, *p7;
        long long* p8;
        signed char* p9;
        CKH(h->mem.upload(&p1, la, st));
        CKH(h->mem.upload(&p2, lb, st));
        CKH(h->mem.upload(&p3, ma, st));
        CKH(h->mem.upload(&p4, mb, st));
        CKH(h->mem.upload(&p8, ie_idx, st));
        CKH(h->mem.upload(&p5, ie_m, st));
        CKH(h->mem.upload(&p6, ie_ptr, st));
        CKH(h->mem.upload(&p7, ie_lam, st));
        CKH(h->mem.upload(&p9, ie_sgn, st));
        du.la = p1;
        du.lb = p2;
        du.ma = p3;
        du.mb = p4;
        du.ie_idx = p8;
        du.ie_mult = p5;
        du.ie_ptr = p6;
        du.ie_lam = p7;
        du.ie_sgn = p9;
    }
    // fine stiffness from the problem
    for (int k = 0; k < N; ++k) {
        const PatchDesc& q = h->pd[k];
        const LevelDesc& F = q.lev[q.L - 1];
        CUH(cudaMemcpyAsync(h->K64 + F.koff, P->K64 + P->koff[k], sizeof(double) * F.n * F.Sp,
                            cudaMemcpyDeviceToDevice, st));
    }
    // ---- multigrid tables, Galerkin hierarchy, coarsest inverses -----------
    {
        DevMem scratch;
        scratch.st = st;
        TableJob *d_tj = nullptr, *d_mj = nullptr;
        int* d_plist = nullptr;
        std::vector<int> plist(N);
        std::iota(plist.begin(), plist.end(), 0);
        int r1 = scratch.upload(&d_tj, tjobs, st);
        if (r1 == IETIDP_OK) r1 = scratch.upload(&d_mj, mjobs, st);
        if (r1 == IETIDP_OK) r1 = scratch.upload(&d_plist, plist, st);
        double* work = nullptr;
        if (r1 == IETIDP_OK) r1 = scratch.alloc(&work, (long long)N * 4 * max_n0 * max_n0);
        if (r1 != IETIDP_OK) {
            scratch.release();
            return bail(r1);
        }
        SetupArgs sa{};
        sa.npatch = N;
        sa.dim = d;
        sa.pd = h->d_pd;
        sa.tab = h->tab;
        sa.itab = h->itab;
        sa.flags = h->flags;
        cudaError_t e = launch_tables(sa, d_tj, (int)tjobs.size(), 0, st);
        if (e == cudaSuccess) e = launch_mass_tables(sa, d_mj, (int)mjobs.size(), st);
        for (int depth = 1; depth < max_L && e == cudaSuccess; ++depth)
            e = launch_galerkin(h->d_pd, d_plist, N, depth, max_rows_lev, max_S, h->K64, h->tab, h->itab, st);
        if (e == cudaSuccess)
            e = launch_coarse_inverse(h->d_pd, N, h->K64, h->tab, opt.alpha_reg, h->A0inv64, h->A0inv32, work,
                                      max_n0, h->flags, st);
        if (e == cudaSuccess && h->n_floating > 0)
            e = launch_regularize(h->d_pd, N, h->K64, h->tab, opt.alpha_reg, h->KM64, st);
        if (e == cudaSuccess && mixed) e = launch_to_f32(h->K64, h->K32, koff, st);
        if (e == cudaSuccess && mixed) e = launch_lo_f32(h->K64, h->K32, h->K32lo, koff, st);
        if (e == cudaSuccess && mixed && h->n_floating > 0) e = launch_to_f32(h->KM64, h->KM32, koff, st);
        if (e == cudaSuccess) e = launch_to_f32(h->tab, h->tabf, toff_tab, st);
        if (e == cudaSuccess)
            e = launch_cweights(h->d_pd, h->nrows, h->crow_ptr, h->crow_patch, d_tang, h->c_idx, h->c_w, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        scratch.release();
        if (e != cudaSuccess) return bail(fail(IETIDP_E_CUDA, std::string("hierarchy setup: ") + cudaGetErrorString(e)));
        int fl = 0;
        CUH(cudaMemcpy(&fl, h->flags, sizeof(int), cudaMemcpyDeviceToHost));
        if (fl & IETI_FLAG_TABLE) return bail(fail(IETIDP_E_INVALID_ARG, "transfer table construction failed"));
        if (fl & IETI_FLAG_NOT_SPD) return bail(fail(IETIDP_E_BREAKDOWN, "coarsest multigrid matrix not SPD"));
    }
    // ---- slots and vectors -------------------------------------------------
    int nslot_basis = h->nrows;
    int nslots_max = std::max(N, nslot_basis);
    long long cg_total = 0, lv_total = 0;
    std::vector<SlotDesc> sp(N), sb(nslot_basis);
    // basis slots: one per constraint row (sized by its patch); patch slots reuse the front
    {
        // slot s serves basis row s (if s < nrows) and patch s (if s < N)
        std::vector<long long> cgo(nslots_max), lvo(nslots_max);
        // high-order multigrid: x | b | r of the patch's levels, then those of
        // the degree-1 hierarchy, then two work tensors of the fine free grid
        auto lvneed = [&](const PatchDesc& q) {
            long long need = std::max<long long>(3LL * q.nlvec, (long long)q.nlx + q.nlb + q.n + 4);
            if (h->ho_sub) {
                const int k = (int)(&q - h->pd.data());
                need = std::max(need, 3LL * q.nlvec + 3LL * h->ho_sub->pd[k].nlvec + 2LL * q.n);
            }
            return need;
        };
        for (int s = 0; s < nslots_max; ++s) {
            long long n = 0, nl = 0;
            if (s < nslot_basis) {
                n = std::max<long long>(n, h->pd[crow_patch[s]].n);
                nl = std::max<long long>(nl, lvneed(h->pd[crow_patch[s]]));
            }
            if (s < N) {
                n = std::max<long long>(n, h->pd[s].n);
                nl = std::max<long long>(nl, lvneed(h->pd[s]));
            }
            nl = (nl + 3) & ~3LL;
            cgo[s] = cg_total;
            lvo[s] = lv_total;
            // Neumann / Schur / null-space basis slots: 5 n; SZ basis slots:
            // 8 n + 8 x 64 (sz_device.cuh)
            cg_total += (sz && s < nslot_basis) ? 8 * n + 8 * ieti_sz_small() : 5 * n;
            lv_total += nl;
        }
        for (int k = 0; k < N; ++k) sp[k] = SlotDesc{k, 0, 0, k, 0, 0, cgo[k], lvo[k]};
        h->cg_patch_elems = N < nslots_max ? cgo[N] : cg_total;
        h->lv_patch_elems = N < nslots_max ? lvo[N] : lv_total;
        for (int s = 0; s < nslot_basis; ++s) sb[s] = SlotDesc{crow_patch[s], 0, s, s, 0, 0, cgo[s], lvo[s]};
    }
    CKH(h->mem.alloc(&h->cg, cg_total));
    if (mixed) {
        float* lvf;
        CKH(h->mem.alloc(&lvf, lv_total));
        h->lv = lvf;
    } else {
        double* lvd;
        CKH(h->mem.alloc(&lvd, lv_total));
        h->lv = lvd;
    }
    CKH(h->mem.alloc(&h->its, nslots_max));
    CKH(make_groups(h, sp, h->gpatch, st));
    CKH(make_groups(h, sb, h->gbasis, st));
    {
        size_t ng = std::max(h->gpatch.size(), h->gbasis.size());
        if (ng > 1) {
            size_t ns = std::min<size_t>(ng, 8);
            h->side.resize(ns);
            h->join.resize(ns);
            for (size_t i = 0; i < ns; ++i) {
                CUH(cudaStreamCreateWithFlags(&h->side[i], cudaStreamNonBlocking));
                CUH(cudaEventCreateWithFlags(&h->join[i], cudaEventDisableTiming));
            }
            CUH(cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming));
        }
    }
    // ---- D-MG: banded Cholesky factors of the fine stiffness ---------------
    if (opt.method == IETIDP_METHOD_DMG) {
        std::vector<int> plist(N);
        int max_n = 0;
        // IETIDP_DIRECT_SMEM=0 keeps every substitution vector in global
        // memory (the path of patches above the shared-memory cap; for its tests)
        const char* ds = std::getenv("IETIDP_DIRECT_SMEM");
        const bool dsmem = !(ds && ds[0] == '0');
        for (int k = 0; k < N; ++k) {
            plist[k] = k;
            max_n = std::max(max_n, h->pd[k].n);
            h->max_bw = std::max(h->max_bw, h->pd[k].bw);
            const size_t zb = sizeof(double) * (size_t)h->pd[k].n;
            if (dsmem && zb <= kDirectSmemCap) h->direct_smem = std::max(h->direct_smem, zb);
            // the band factorization costs n bw^2 per patch: kept for patches
            // where that stays moderate (2D patches; large 3D patches are
            // what the paper's direct variants could not hold either)
            const double cost = (double)h->pd[k].n * h->pd[k].bw * h->pd[k].bw;
            if (cost > 2e10)
                return bail(fail(IETIDP_E_INVALID_ARG, "D-MG: banded factorization of patch " + std::to_string(k) +
                                                           " too large (n = " + std::to_string(h->pd[k].n) +
                                                           ", band " + std::to_string(h->pd[k].bw) + ")"));
        }
        int* d_plist;
        CKH(h->mem.upload(&d_plist, plist, st));
        CUH(cudaMemsetAsync(h->band, 0, sizeof(double) * bandoff, st));
        CUH(cudaMemsetAsync(h->flags, 0, sizeof(int), st));
        CUH(launch_band_factor(h->d_pd, d_plist, N, max_n, h->max_bw, h->K64, h->band, h->flags, st));
        int fl = 0;
        CUH(cudaMemcpyAsync(&fl, h->flags, sizeof(int), cudaMemcpyDeviceToHost, st));
        CUH(cudaStreamSynchronize(st));
        if (fl & IETI_FLAG_NOT_SPD) return bail(fail(IETIDP_E_BREAKDOWN, "banded Cholesky: stiffness not SPD"));
    }
    // ---- primal basis (Eq. 6) ---------------------------------------------
    // with the high-order multigrid the basis uses the standard hierarchy
    // (see ieti_solve_args), whose V-cycle weakens with the degree: more
    // iterations allowed there
    const int basis_maxit = h->d_ho ? 8 * opt.maxit_inner : opt.maxit_inner;
    if (nslot_basis > 0) {
        if (sz) {
            // W = Khat^{-1} C^T per constraint row, Hhat^{-1} per patch, then SZ-CG
            CHK(run_solve(h, MODE_SZW, h->gbasis, nullptr, nullptr, 0.0, 0, h->vst + 8));
            cudaError_t e = launch_sz_hinv(h->d_pd, N, h->crow_ptr, h->c_idx, h->c_w, h->szW, h->szHinv, h->flags, st);
            if (e != cudaSuccess) return bail(fail(IETIDP_E_CUDA, std::string("SZ set-up: ") + cudaGetErrorString(e)));
            CHK(run_solve(h, MODE_BASIS_SZ, h->gbasis, nullptr, nullptr, opt.tol_basis, basis_maxit, h->vst + 8));
        } else {
            CHK(run_solve(h, MODE_BASIS, h->gbasis, nullptr, nullptr, opt.tol_basis, basis_maxit, h->vst + 8));
        }
        CUH(cudaStreamSynchronize(st));
        std::vector<int> its(nslot_basis);
        CUH(cudaMemcpyAsync(its.data(), h->its, sizeof(int) * nslot_basis, cudaMemcpyDeviceToHost, st));
        CUH(cudaStreamSynchronize(st));
        long long s = 0;
        for (int v : its) {
            s += v;
            h->basis_it_max = std::max(h->basis_it_max, v);
        }
        h->basis_it_avg = (double)s / nslot_basis;
        int fl = 0;
        CUH(cudaMemcpy(&fl, h->flags, sizeof(int), cudaMemcpyDeviceToHost));
        {
            int dbg[8];
            CUH(cudaMemcpy(dbg, h->dbg, sizeof(dbg), cudaMemcpyDeviceToHost));
            if (dbg[0] != 0)
                return bail(fail(IETIDP_E_CUDA, "self-check: " + std::to_string(dbg[0]) + " bad accesses, first at site " +
                                                    std::to_string(dbg[1]) + " index " + std::to_string(dbg[2]) +
                                                    " limit " + std::to_string(dbg[3]) + " block " +
                                                    std::to_string(dbg[4]) + " thread " + std::to_string(dbg[5])));
        }
        if (fl & IETI_FLAG_BREAKDOWN) return bail(fail(IETIDP_E_BREAKDOWN, "CG breakdown in the primal basis"));
        if (fl & IETI_FLAG_NOT_CONVERGED)
            return bail(fail(IETIDP_E_NOT_CONVERGED, "primal basis solves did not converge"));
    }
    // ---- S_PiPi and its Cholesky factor -----------------------------------
    if (npi > 0) {
        DevMem scratch;
        scratch.st = st;
        double *work, *sloc, *S, *cw;
        long long *d_soff;
        std::vector<long long> soff(N + 1, 0);
        for (int k = 0; k < N; ++k) soff[k + 1] = soff[k] + (long long)npi_k[k] * npi_k[k];
        int r1 = scratch.alloc(&work, (long long)h->nrows * cg_need);
        if (r1 == IETIDP_OK) r1 = scratch.alloc(&sloc, soff[N]);
        if (r1 == IETIDP_OK) r1 = scratch.alloc(&S, (long long)npi * npi);
        if (r1 == IETIDP_OK) r1 = scratch.alloc(&cw, (long long)npi * npi);
        if (r1 == IETIDP_OK) r1 = scratch.upload(&d_soff, soff, st);
        if (r1 != IETIDP_OK) {
            scratch.release();
            return bail(r1);
        }
        cudaError_t e = launch_spp_local(h->d_pd, h->nrows, h->crow_patch, h->crow_local, h->phi, h->K64, work,
                                         cg_need, sloc, d_soff, st);
        if (e == cudaSuccess) e = launch_spp_assemble(N, h->d_pd, h->crow_glob, sloc, d_soff, S, npi, st);
        h->spp_host.assign((size_t)npi * npi, 0.0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->spp_host.data(), S, sizeof(double) * npi * npi, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = launch_chol_linv(S, npi, h->Linv, cw, h->flags, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        scratch.release();
        if (e != cudaSuccess) return bail(fail(IETIDP_E_CUDA, std::string("coarse setup: ") + cudaGetErrorString(e)));
        int fl = 0;
        CUH(cudaMemcpy(&fl, h->flags, sizeof(int), cudaMemcpyDeviceToHost));
        if (fl & IETI_FLAG_NOT_SPD) return bail(fail(IETIDP_E_BREAKDOWN, "S_PiPi is not SPD"));
    }
    // ---- solve-time buffers --------------------------------------------------
    long long nt = P->ntorn;
    CKH(h->mem.alloc(&h->gF, nt));
    CKH(h->mem.alloc(&h->uF, nt));
    CKH(h->mem.alloc(&h->vS, nt));
    CKH(h->mem.alloc(&h->wS, nt));
    CKH(h->mem.alloc(&h->gR, nt));
    CKH(h->mem.alloc(&h->tmp, nt));
    CKH(h->mem.alloc(&h->fH, nt));
    CKH(h->mem.alloc(&h->uH, nt));
    CUH(cudaMemsetAsync(h->gF, 0, sizeof(double) * nt, st));
    CUH(cudaMemsetAsync(h->vS, 0, sizeof(double) * nt, st));
    CUH(cudaMemsetAsync(h->tmp, 0, sizeof(double) * nt, st));
    long long nl = std::max(1, h->nlam);
    CKH(h->mem.alloc(&h->lam, nl));
    CKH(h->mem.alloc(&h->r, nl));
    CKH(h->mem.alloc(&h->z, nl));
    CKH(h->mem.alloc(&h->p, nl));
    CKH(h->mem.alloc(&h->q, nl));
    CKH(h->mem.alloc(&h->d, nl));
    CKH(h->mem.alloc(&h->state, 16));
    CKH(h->mem.alloc(&h->hist, 2 * (opt.maxit_outer + 2)));
    CKH(h->mem.alloc(&h->scal, 4));
    CUH(cudaMallocHost(&h->h_pinned, sizeof(double) * 16));
    h->ev.resize(2 * (2 * opt.maxit_outer + 8));
    for (auto& ev : h->ev) CUH(cudaEventCreate(&ev));
    CUH(cudaStreamSynchronize(st));
    auto t1 = std::chrono::steady_clock::now();
    h->t_setup_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
#undef CKH
#undef CUH
    *out = h;
    return rc;
}

// ---------------------------------------------------------------------------
// solve
// ---------------------------------------------------------------------------
static int ktilde_inv(ietidp_handle* h, const double* g, double* u) {
    cudaStream_t st = h->st;
    h->launches += (h->nrows > 0) + (h->npi > 0);
    g_kernel_launches += (h->nrows > 0) + (h->npi > 0);
    cudaError_t e = launch_primal_restrict(h->d_pd, h->nrows, h->crow_patch, h->crow_local, h->phi, g, h->rloc, st);
    if (e == cudaSuccess)
        e = launch_coarse_solve(h->npi, h->nrows, h->crow_glob, h->gptr, h->glist, h->Linv, h->rloc, h->upi, h->uloc, st);
    if (e != cudaSuccess) return fail(IETIDP_E_CUDA, std::string("primal: ") + cudaGetErrorString(e));
    return run_solve(h, MODE_NEUMANN, h->gpatch, g, u, h->opt.tol_inner, h->opt.maxit_inner, h->vst);
}

static int apply_F(ietidp_handle* h, const double* pv, double* qv) {
    h->launches += 2;
    g_kernel_launches += 2;
    cudaError_t e = launch_bt(h->dual, pv, h->gF, 0, h->st);
    if (e != cudaSuccess) return fail(IETIDP_E_CUDA, cudaGetErrorString(e));
    CHK(ktilde_inv(h, h->gF, h->uF));
    e = launch_b(h->dual, h->uF, qv, 0, h->st);
    if (e != cudaSuccess) return fail(IETIDP_E_CUDA, cudaGetErrorString(e));
    return IETIDP_OK;
}

static int apply_M(ietidp_handle* h, const double* rv, double* zv) {
    h->launches += 2;
    g_kernel_launches += 2;
    cudaError_t e = launch_bt(h->dual, rv, h->vS, 1, h->st);
    if (e != cudaSuccess) return fail(IETIDP_E_CUDA, cudaGetErrorString(e));
    CHK(run_solve(h, MODE_SCHUR, h->gpatch, h->vS, h->wS, 0.0, 0, h->vst));
    e = launch_b(h->dual, h->wS, zv, 1, h->st);
    if (e != cudaSuccess) return fail(IETIDP_E_CUDA, cudaGetErrorString(e));
    return IETIDP_OK;
}

extern "C" int ietidp_info_get(const ietidp_handle* h, ietidp_info* info) {
    if (!h || !info) return fail(IETIDP_E_INVALID_ARG, "null argument");
    std::memset(info, 0, sizeof(*info));
    info->dim = h->dim;
    info->npatch = h->npatch;
    info->n_torn = h->prob->ntorn;
    info->n_lambda = h->nlam;
    info->n_primal = h->npi;
    info->n_floating = h->n_floating;
    int ml = 0;
    for (auto& q : h->pd) ml = std::max(ml, q.L);
    info->max_levels = ml;
    info->device_bytes = h->mem.bytes;
    return IETIDP_OK;
}

extern "C" int ietidp_patch_offsets(const ietidp_handle* h, long long* off) {
    if (!h || !off) return fail(IETIDP_E_INVALID_ARG, "null argument");
    for (int k = 0; k <= h->npatch; ++k) off[k] = h->prob->toff[k];
    return IETIDP_OK;
}

// Per-phase clock cycles of CTA 0 of the local solver kernel, accumulated
// since the handle was created (non-zero only in builds compiled with
// IETIDP_PHASE_TIMERS=1).
extern "C" int ietidp_phase_timers(ietidp_handle* h, long long* out64) {
    if (!h || !out64) return fail(IETIDP_E_INVALID_ARG, "null argument");
    CU(cudaStreamSynchronize(h->st));
    CU(cudaMemcpy(out64, h->phase, sizeof(long long) * 64, cudaMemcpyDeviceToHost));
    return IETIDP_OK;
}

extern "C" int ietidp_vcycles(ietidp_handle* h, const double* b, double* x, int ncycles) {
    if (!h || !b || !x || ncycles < 0) return fail(IETIDP_E_INVALID_ARG, "bad argument");
    SolveArgs a = ieti_solve_args(h, MODE_VCYCLE, b, x, 0.0, 0, h->vst);
    a.ncycles = ncycles;
    return run_solve_args(h, a, h->gpatch);
}

extern "C" int ietidp_vcycles_hierarchy(ietidp_handle* h, int hierarchy, const double* b, double* x, int ncycles) {
    if (!h || !b || !x || ncycles < 0 || hierarchy < 0 || hierarchy > 1)
        return fail(IETIDP_E_INVALID_ARG, "bad argument");
    SolveArgs a = ieti_solve_args(h, hierarchy == 0 ? MODE_VCYCLE : MODE_VCYCLE_DIR, b, x, 0.0, 0, h->vst);
    a.ncycles = ncycles;
    return run_solve_args(h, a, h->gpatch);
}

extern "C" int ietidp_apply_K(ietidp_handle* h, const double* x, double* y) {
    if (!h || !x || !y) return fail(IETIDP_E_INVALID_ARG, "null argument");
    cudaError_t e = launch_apply_K(h->d_pd, h->npatch, h->K64, x, y, h->st);
    if (e != cudaSuccess) return fail(IETIDP_E_CUDA, cudaGetErrorString(e));
    CU(cudaStreamSynchronize(h->st));
    return IETIDP_OK;
}

extern "C" int ietidp_apply_F(ietidp_handle* h, const double* p, double* q) {
    if (!h || !p || !q) return fail(IETIDP_E_INVALID_ARG, "null argument");
    CHK(apply_F(h, p, q));
    CU(cudaStreamSynchronize(h->st));
    return IETIDP_OK;
}

extern "C" int ietidp_apply_precond(ietidp_handle* h, const double* r, double* z) {
    if (!h || !r || !z) return fail(IETIDP_E_INVALID_ARG, "null argument");
    CHK(apply_M(h, r, z));
    CU(cudaStreamSynchronize(h->st));
    return IETIDP_OK;
}

extern "C" int ietidp_apply_Ktilde_inv(ietidp_handle* h, const double* g, double* u) {
    if (!h || !g || !u) return fail(IETIDP_E_INVALID_ARG, "null argument");
    CHK(ktilde_inv(h, g, u));
    CU(cudaStreamSynchronize(h->st));
    return IETIDP_OK;
}

extern "C" int ietidp_get_primal_basis(ietidp_handle* h, int patch, double* phi, int* ncols) {
    if (!h || patch < 0 || patch >= h->npatch) return fail(IETIDP_E_INVALID_ARG, "bad patch");
    const PatchDesc& q = h->pd[patch];
    if (ncols) *ncols = q.npi;
    if (phi && q.npi)
        CU(cudaMemcpy(phi, h->phi + q.phioff, sizeof(double) * q.n * q.npi, cudaMemcpyDeviceToDevice));
    return IETIDP_OK;
}

extern "C" int ietidp_get_spp(ietidp_handle* h, double* spp) {
    if (!h || !spp) return fail(IETIDP_E_INVALID_ARG, "null argument");
    std::copy(h->spp_host.begin(), h->spp_host.end(), spp);
    return IETIDP_OK;
}

extern "C" int ietidp_destroy(ietidp_handle* h) {
    if (!h) return IETIDP_OK;
    cudaStreamSynchronize(h->st);
    ieti_engine_destroy(h->engine);
    h->engine = nullptr;
    ieti_saddle_free(h);
    h->mem.release();
    cudaStreamSynchronize(h->st);
    if (h->h_pinned) cudaFreeHost(h->h_pinned);
    for (auto& ev : h->ev) cudaEventDestroy(ev);
    for (auto& sd : h->side) cudaStreamDestroy(sd);
    for (auto& ev : h->join) cudaEventDestroy(ev);
    if (h->fork) cudaEventDestroy(h->fork);
    if (h->ho_sub) ietidp_destroy(h->ho_sub);
    if (h->ho_prob) iga_problem_free(h->ho_prob);
    delete h;
    return IETIDP_OK;
}

// ---------------------------------------------------------------------------
// V-cycles without any device allocation.
//
// Some callers cannot allocate device memory at the point where they want to
// run the smoother: a plugin running inside a host framework that owns the
// device memory pool and forbids allocations outside it, or a latency-bound
// loop that must not hit cudaMalloc/cudaFree (they may synchronize the device
// and take unbounded time).  For them the scratch vectors of the V-cycle
// kernel (the FP64 residual/correction vectors and the per-level vectors of
// every patch) live in one file-scope device array of fixed size instead of
// the handle's own buffers.  Host code cannot use the array's name as a
// device address, so ietidp_setup looks the address up with
// cudaGetSymbolAddress on the handle's device (with that device current) and
// keeps it in the handle; under lazy module loading that lookup is also the
// moment the array's memory is committed.  The call itself only reads the
// kept address.  Every call on a device shares the same array.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kNoAllocScratchBytes = 16u << 20;   // 16 MiB per device, held until exit
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
}  // namespace

static cudaError_t ieti_noalloc_address(void** p) {
    *p = nullptr;
    return cudaGetSymbolAddress(p, g_noalloc_scratch);
}

extern "C" int ietidp_vcycles_noalloc(ietidp_handle* h, const double* b, double* x, int ncycles) {
    if (!h || !b || !x || ncycles < 0) return fail(IETIDP_E_INVALID_ARG, "bad argument");
    int dev = -1;
    CU(cudaGetDevice(&dev));
    if (dev != h->device) return fail(IETIDP_E_INVALID_ARG, "the handle's device must be the current device");
    if (!h->noalloc_base) return fail(IETIDP_E_INVALID_ARG, "no static scratch address for this handle");
    const size_t tsz = h->opt.precision == IETIDP_PREC_MIXED ? sizeof(float) : sizeof(double);
    const size_t cg_bytes = ((size_t)h->cg_patch_elems * sizeof(double) + 255) & ~(size_t)255;
    const size_t need = cg_bytes + (size_t)h->lv_patch_elems * tsz;
    if (need > kNoAllocScratchBytes)
        return fail(IETIDP_E_INVALID_ARG, "problem needs " + std::to_string(need) +
                                              " bytes of V-cycle scratch; the static limit is " +
                                              std::to_string(kNoAllocScratchBytes) + " bytes");
    // the regular V-cycle launch with its scratch pointers redirected in a
    // local copy of the kernel arguments (the handle is not modified)
    SolveArgs a = ieti_solve_args(h, MODE_VCYCLE, b, x, 0.0, 0, h->vst);
    a.cg = (double*)h->noalloc_base;
    a.lv = (unsigned char*)h->noalloc_base + cg_bytes;
    a.ncycles = ncycles;
    return run_solve_args(h, a, h->gpatch);
}
