// Batched local solver of inexact IETI-DP, specialised at compile time for
// the patch dimension and spline degrees (stencil (2p_1+1)...(2p_d+1), Gauss-
// Seidel colors (p_1+1)...(p_d+1)), so that every stencil loop is unrolled and
// a row's loads are issued back to back.
//
// One CTA owns one local problem ("slot") for a whole launch.  Shared memory
// holds, as far as the launch's budget allows: the patch descriptor, the
// V-cycle vectors of every level, the coarsest-level inverse and the
// matrices of the coarse levels (loaded once per launch, then reused by every
// V-cycle of the CG).  The fine-level matrix streams from L2/HBM in
// color-major order (unit-stride per stencil diagonal).
//
// Modes (Sec. 3): Neumann solve inside F and K~^{-1} (CG on K, V-cycle on K
// or K + alpha M^, right-hand side P^T g, result P z + Phi u_Pi), primal basis
// (Eq. 6 by the null-space method, or by Schoeberl-Zulehner CG: sz_device.cuh),
// scaled-Dirichlet Schur application (two V-cycles on K_II), the MG-MG-S
// blocks (contraction estimate, K-hat), and a plain V-cycle iteration for
// benchmarking.
#pragma once
#include <math.h>
#include <cooperative_groups.h>
#include "kernels.cuh"
#include "sz_device.cuh"

namespace ieti_t {

constexpr int kMaxRows = 64;

// Optional self-check (compiled with -DIETI_DEBUG_BOUNDS): an index outside
// its buffer is recorded in dbg[] (count, site, index, limit, block, thread)
// and the access is skipped.
#ifdef IETI_DEBUG_BOUNDS
__device__ int* g_ieti_dbg;
__device__ __forceinline__ bool ieti_ok(long long idx, long long lim, int site) {
    if (idx >= 0 && idx < lim) return true;
    if (g_ieti_dbg && atomicAdd(&g_ieti_dbg[0], 1) == 0) {
        g_ieti_dbg[1] = site;
        g_ieti_dbg[2] = (int)idx;
        g_ieti_dbg[3] = (int)lim;
        g_ieti_dbg[4] = blockIdx.x;
        g_ieti_dbg[5] = threadIdx.x;
    }
    return false;
}
#define IETI_OK(idx, lim, site) ieti_ok((long long)(idx), (long long)(lim), (site))
#else
#define IETI_OK(idx, lim, site) true
#endif

// Optional phase timers (compiled with -DIETI_PHASE_TIMERS): thread 0 of CTA 0
// adds the clock cycles of each barrier-delimited phase to phase[]:
// [4*l + 0..3] = sweeps, residual, restriction, prolongation at level l,
// [48] coarsest solve, [49] FP64 SpMV, [50] V-cycle conversions.
#ifdef IETI_PHASE_TIMERS
#define IETI_T0() long long _t0 = (threadIdx.x == 0 && blockIdx.x == 0) ? clock64() : 0
#define IETI_T1(k) do { if (threadIdx.x == 0 && blockIdx.x == 0 && phase) phase[k] += clock64() - _t0; } while (0)
#else
#define IETI_T0() do {} while (0)
#define IETI_T1(k) do {} while (0)
#endif

struct Red {
    double v[32][4];
};

template <int K>
__device__ __forceinline__ void cta_sum(double* val, Red& sh) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) val[k] += __shfl_xor_sync(0xffffffffu, val[k], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) sh.v[w][k] = val[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int i = 0; i < nw; ++i) s += sh.v[i][k];
        val[k] = s;
    }
}

// The CTAs that share one slot: a thread-block cluster of `size` CTAs (1
// outside cluster launches).  Loops over a slot's rows and vector entries
// run over the group's threads; group barriers are cluster barriers (release
// / acquire: writes to global memory before the barrier are seen by every
// CTA of the cluster after it).  Shared-memory copies (descriptor, tables,
// staged matrices) stay per CTA.
// CL = false (the shared-vector variant, never launched as clusters): one
// CTA, resolved at compile time.
template <bool CL>
struct GrpT {
    int rank, size;
    __device__ __forceinline__ int tid() const {
        return CL ? rank * (int)blockDim.x + (int)threadIdx.x : (int)threadIdx.x;
    }
    __device__ __forceinline__ int nt() const { return CL ? size * (int)blockDim.x : (int)blockDim.x; }
    __device__ __forceinline__ bool many() const { return CL && size > 1; }
    __device__ __forceinline__ void sync() const {
        if (many())
            cooperative_groups::this_cluster().sync();
        else
            __syncthreads();
    }
};

template <bool CL>
__device__ __forceinline__ GrpT<CL> make_grp() {
    GrpT<CL> g{0, 1};
    if (CL) {
        g.rank = (int)cooperative_groups::this_cluster().block_rank();
        g.size = (int)cooperative_groups::this_cluster().num_blocks();
    }
    return g;
}

// sums over the group: each CTA's total by cta_sum, then the CTAs' totals in
// rank order (every CTA adds the same numbers in the same order, so all of
// them take the same branches on the result)
template <int K, bool CL>
__device__ __forceinline__ void grp_sum(double* val, Red& sh, double* tot, const GrpT<CL>& g) {
    cta_sum<K>(val, sh);
    if (!g.many()) return;
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) tot[k] = val[k];
    g.sync();
    auto cl = cooperative_groups::this_cluster();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int r = 0; r < g.size; ++r) s += *cl.map_shared_rank(tot + k, r);
        val[k] = s;
    }
    g.sync();
}

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

constexpr int sp_of(int S) { return (((S + 3) & ~3) / 4) % 2 == 0 ? ((S + 3) & ~3) + 4 : ((S + 3) & ~3); }

// per level (l >= 1) and color: storage offset and counts of the color's rows,
// base and strides of its ghost-padded block in the color-major x
struct CTab {
    int off, k0, k1, k2, xb, xk0, xk1;
};

// shared-memory plan of one slot for a dynamic budget B (same on host and device)
struct Plan {
    bool vec;       // x, b, r in shared memory
    bool a0;        // coarsest inverse in shared memory
    int ls;         // matrices of levels 1..ls in shared memory (0: none; the
                    // coarsest level is solved by its dense inverse)
    size_t tab_off, vec_off, a0_off, mat_off, used;
};

__host__ __device__ inline size_t ctab_bytes(const PatchDesc& P) {
    return align16((size_t)P.L * ieti_ncolors(P.p) * sizeof(CTab));
}
__host__ __device__ inline size_t vec_elems(const PatchDesc& P) {
    return (size_t)P.nlx + P.nlb + P.lev[P.L - 1].n;
}

__host__ __device__ inline Plan make_plan(const PatchDesc& P, size_t tsize, size_t B, bool want_vec) {
    Plan pl;
    size_t used = 0;
    pl.tab_off = 0;
    used += ctab_bytes(P);
    pl.vec_off = used;
    size_t vb = align16(vec_elems(P) * tsize);
    pl.vec = want_vec && used + vb <= B;   // vectors in shared memory (host checks they fit)
    if (pl.vec) used += vb;
    size_t ab = align16((size_t)P.lev[0].n * P.lev[0].n * tsize);
    pl.a0 = used + ab <= B;
    pl.a0_off = used;
    if (pl.a0) used += ab;
    pl.mat_off = used;
    pl.ls = 0;
    // levels 1..l are staged as one copy of their contiguous span in the
    // value pool (including the alignment gaps between levels); the fine
    // level too when everything fits
    for (int l = 1; l < P.L; ++l) {
        size_t span = (size_t)(P.lev[l].koff + (long long)P.lev[l].n * P.lev[l].S - P.lev[1].koff) * tsize;
        if (pl.mat_off + span > B) break;
        used = pl.mat_off + span;
        pl.ls = l;
    }
    pl.used = used;
    return pl;
}

// shared memory the specialised kernel cannot do without (tables + vectors)
inline size_t smem_min(const PatchDesc& P, size_t tsize) { return ctab_bytes(P) + align16(vec_elems(P) * tsize); }

// full shared-memory need of one slot (host side sizing); vectors included
// unless they live in global memory (xg)
inline size_t smem_need(const PatchDesc& P, size_t tsize, bool xg = false) {
    size_t b = ctab_bytes(P) + (xg ? 0 : align16(vec_elems(P) * tsize)) +
               align16((size_t)P.lev[0].n * P.lev[0].n * tsize);
    if (P.L > 1) {
        const LevelDesc& Lt = P.lev[P.L - 1];
        b += (size_t)(Lt.koff + (long long)Lt.n * Lt.S - P.lev[1].koff) * tsize;
    }
    return b;
}

template <typename T>
struct V4;
template <>
struct V4<float> {
    using type = float4;
};
template <>
struct V4<double> {
    using type = double2;   // two 16-byte loads per 4 values
};

template <typename T>
__device__ __forceinline__ void load4(const T* p, T* w);
template <>
__device__ __forceinline__ void load4<float>(const float* p, float* w) {
    float4 v = *reinterpret_cast<const float4*>(p);
    w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
}
template <>
__device__ __forceinline__ void load4<double>(const double* p, double* w) {
    double2 a = reinterpret_cast<const double2*>(p)[0];
    double2 b = reinterpret_cast<const double2*>(p)[1];
    w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
}

// dynamic shared memory of the specialised kernel; arrays resident there are
// addressed from this symbol so that the compiler emits shared-memory loads
extern __shared__ __align__(16) unsigned char ieti_dyn[];

template <typename T>
__device__ __forceinline__ T* shm(int elem_off) {
    return reinterpret_cast<T*>(ieti_dyn) + elem_off;
}

// bulk prefetch of [src, src + bytes) into L2 (sm_90+; nothing to wait for);
// src and bytes 16-byte aligned
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

template <typename T, int D, int P0, int P1, int P2, bool XG>
struct VC {
    static constexpr int W0 = 2 * P0 + 1, W1 = 2 * P1 + 1, W2 = 2 * P2 + 1;
    static constexpr int S = W0 * W1 * W2;
    static constexpr int C0 = P0 + 1, C1 = P1 + 1, C2 = P2 + 1, NC = C0 * C1 * C2;
    static constexpr int R0 = P0 + 2, R1 = P1 + 2, R2 = D == 3 ? P2 + 2 : 1;

    const PatchDesc* P;   // shared copy
    int mask;
    const T* Kg;          // global value pool (K or K + alpha M^)
    int ks_off;           // staged matrices of levels 1..ls (element offset in dynamic shared memory)
    int ls;
    long long kbase;
    const T* tab;
    const int* itab;
    int a0_off;           // coarsest inverse in shared memory (element offset), or -1
    const T* A0g;
    int x_off, b_off, r_off;   // vectors: element offsets in shared memory, or in gvec when XG
    T* gvec;              // the slot's level vectors in global memory (XG)

    __device__ __forceinline__ T* vp(int off) const {
        if constexpr (XG) return gvec + off;
        else return shm<T>(off);
    }
    const CTab* ct;       // [l * NC + c]
    long long* phase;     // phase timers (profiling builds)
    int kflags;           // SolveArgs::kflags
    GrpT<XG> g;           // the CTAs sharing the slot (a cluster, or this CTA)

    // one row of color (c0,c1,c2) at level l.  X: the row's own entry in x;
    // the neighbour at stencil offset (o0,o1,o2) lies e0(o0)+e1(o1)+e2(o2)
    // entries away (uniform color blocks): with d_r = floor((c_r+o_r)/C_r),
    // e_r = (o_r - C_r d_r) * stride_r * blk + d_r * xstride_r.
    template <bool VSH>
    __device__ __forceinline__ T row(const T* __restrict__ vg, int vs_off, int cnt, int q, const T* X, int c0,
                                     int c1, int c2, int blk, int xk0, int xk01, T* d) const {
        int e0[W0], e1[W1], e2[W2];
#pragma unroll
        for (int o = -P0; o <= P0; ++o) {
            const int dd = (c0 + o + C0) / C0 - 1;
            e0[o + P0] = (o - C0 * dd) * blk + dd;
        }
#pragma unroll
        for (int o = -P1; o <= P1; ++o) {
            const int dd = (c1 + o + C1) / C1 - 1;
            e1[o + P1] = (o - C1 * dd) * C0 * blk + dd * xk0;
        }
#pragma unroll
        for (int o = -P2; o <= P2; ++o) {
            const int dd = (c2 + o + C2) / C2 - 1;
            e2[o + P2] = D == 3 ? (o - C2 * dd) * C0 * C1 * blk + dd * xk01 : 0;
        }
        T acc[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
        for (int o = 0; o < S; ++o) {
            const int o0 = o % W0, o1 = (o / W0) % W1, o2 = o / (W0 * W1);
            const T a = VSH ? shm<T>(vs_off)[q + o * cnt] : __ldg(vg + q + (long long)o * cnt);
            acc[o & 3] += a * X[e0[o0] + e1[o1] + e2[o2]];
        }
        constexpr int oc = P0 + W0 * (P1 + W1 * P2);
        *d = VSH ? shm<T>(vs_off)[q + oc * cnt] : __ldg(vg + q + (long long)oc * cnt);
        return (acc[0] + acc[1]) + (acc[2] + acc[3]);
    }

    // G lanes per row (coarse levels: a color has at most blockDim / G rows;
    // used with G = 8, measured faster there than one lane per row, while
    // G = 2 and 4 on the 32-element level were slower):
    // lane `sub` of a row's group takes the stencil terms sub, sub + G, ...,
    // the group sums by shuffles and its first lane updates the row, so that a
    // row's dependent chain is about S / G terms long and G times as many
    // warps issue.  Warps whose rows all lie beyond the color skip; lanes past
    // the last row repeat it (valid addresses) and store nothing.
    template <bool VSH, int WHAT, int G>
    __device__ __noinline__ void split_pass(const LevelDesc& L, const CTab& t, int c0, int c1, int c2, int cnt,
                                               const T* __restrict__ vg, int vs, T* xl, const T* bl) const {
        const int tid = g.tid();
        if ((tid & ~31) / G >= cnt) return;
        const int blk = L.blk, xk0 = L.xk[0], xk01 = L.xk[0] * L.xk[1];
        const int sub = tid & (G - 1);
        const int qr = tid / G;
        const bool act = qr < cnt;
        const int q = act ? qr : cnt - 1;
        const int t0 = q % t.k0, tr = q / t.k0;
        const int t1 = tr % t.k1, t2 = tr / t.k1;
        const int i0 = c0 + C0 * t0, i1 = c1 + C1 * t1, i2 = c2 + C2 * t2;
        const bool msk = ieti_masked(mask, L.m, i0, i1, i2);
        const int own = (t0 + 1) + xk0 * (t1 + 1) + (D == 3 ? xk01 * (t2 + 1) : 0);
        const T* X = xl + own;
        auto term = [&](int o) {
            const int o0 = o % W0 - P0, o1 = (o / W0) % W1 - P1, o2 = o / (W0 * W1) - P2;
            const int d0 = (c0 + o0 + C0) / C0 - 1, d1 = (c1 + o1 + C1) / C1 - 1;
            int e = (o0 - C0 * d0) * blk + d0 + (o1 - C1 * d1) * C0 * blk + d1 * xk0;
            if (D == 3) {
                const int d2 = (c2 + o2 + C2) / C2 - 1;
                e += (o2 - C2 * d2) * C0 * C1 * blk + d2 * xk01;
            }
            const T a = VSH ? shm<T>(vs)[q + o * cnt] : __ldg(vg + q + (long long)o * cnt);
            return a * X[e];
        };
        constexpr int K = S / G;
        T acc0 = T(0), acc1 = T(0);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (k & 1) acc1 += term(sub + k * G);
            else acc0 += term(sub + k * G);
        }
        if (S % G != 0 && sub + K * G < S) acc0 += term(sub + K * G);
        T acc = acc0 + acc1;
#pragma unroll
        for (int w = G / 2; w > 0; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
        if (sub == 0 && act) {
            constexpr int oc = P0 + W0 * (P1 + W1 * P2);
            if (WHAT == 0) {
                if (!msk) {
                    const T dg = VSH ? shm<T>(vs)[q + oc * cnt] : __ldg(vg + q + (long long)oc * cnt);
                    xl[own] += (bl[q] - acc) / dg;
                }
            } else {
                vp(r_off)[i0 + L.m[0] * (i1 + L.m[1] * i2)] = msk ? T(0) : bl[q] - acc;
            }
        }
    }

    // sweep (WHAT = 0) or residual (WHAT = 1) over the rows of color c
    template <bool VSH, int WHAT>
    __device__ void color_pass(int l, int c) const {
        const int c0 = c % C0, c1 = (c / C0) % C1, c2 = c / (C0 * C1);
        const LevelDesc& L = P->lev[l];
        const CTab t = ct[l * NC + c];
        const int m0 = L.m[0], m1 = L.m[1];
        const int blk = L.blk, xk0 = L.xk[0], xk01 = L.xk[0] * L.xk[1];
        const int cnt = t.k0 * t.k1 * t.k2;
        const long long vrel = (long long)t.off * S;
        const T* vg = Kg + L.koff + vrel;
        const int vs = ks_off + (int)(L.koff - kbase + vrel);
        T* xl = vp(x_off + L.xoff + c * blk);
        const T* bl = vp(b_off + L.boff + t.off);
        const int nt = g.nt();
        if (!(kflags & 256) && cnt > 0 && 8 * cnt <= nt) {
            split_pass<VSH, WHAT, 8>(L, t, c0, c1, c2, cnt, vg, vs, xl, bl);
            if (WHAT == 0) g.sync();
            return;
        }
        for (int q = g.tid(); q < cnt; q += nt) {
            const int t0 = q % t.k0, tr = q / t.k0;
            const int t1 = tr % t.k1, t2 = tr / t.k1;
            const int i0 = c0 + C0 * t0, i1 = c1 + C1 * t1, i2 = c2 + C2 * t2;
            const bool msk = ieti_masked(mask, L.m, i0, i1, i2);
            const int own = (t0 + 1) + xk0 * (t1 + 1) + (D == 3 ? xk01 * (t2 + 1) : 0);
            if (WHAT == 0) {
                if (msk) continue;
                T dg;
                const T ax = row<VSH>(vg, vs, cnt, q, xl + own, c0, c1, c2, blk, xk0, xk01, &dg);
                xl[own] += (bl[q] - ax) / dg;
            } else {
                const int i = i0 + m0 * (i1 + m1 * i2);
                T rv = T(0);
                if (!msk) {
                    T dg;
                    rv = bl[q] - row<VSH>(vg, vs, cnt, q, xl + own, c0, c1, c2, blk, xk0, xk01, &dg);
                }
                vp(r_off)[i] = rv;
            }
        }
        if (WHAT == 0) g.sync();
    }

    // A level streamed from L2/HBM: its color blocks are moved into L2 by
    // bulk prefetches (one instruction of thread 0 per block, no registers or
    // shared memory held) one and two color steps before the step that reads
    // them, so the step's loads wait for L2 instead of HBM.  The copied range
    // is the block widened to 16-byte boundaries (the value pools carry 16
    // elements of tail padding).
    __device__ __forceinline__ void prefetch_block(int l, int c) const {
        if (kflags & 16) return;
        constexpr long long A = 16 / sizeof(T);
        const CTab t = ct[l * NC + c];
        const long long s0 = P->lev[l].koff + (long long)t.off * S;
        const long long len = (long long)t.k0 * t.k1 * t.k2 * S;
        const long long a = s0 & ~(A - 1), e = (s0 + len + A - 1) & ~(A - 1);
        bulk_prefetch_l2(Kg + a, (unsigned)((e - a) * (long long)sizeof(T)));
    }

    __device__ void sweep(int l, bool forward) const {
        if (l <= ls) {
            for (int cc = 0; cc < NC; ++cc) color_pass<true, 0>(l, forward ? cc : NC - 1 - cc);
        } else {
            // the color after the sweep's last one is the first of the next
            // sweep (or, after forward sweeps, of the residual)
            auto col = [&](int k) { return forward ? k % NC : NC - 1 - k % NC; };
            if (g.tid() == 0) {
                prefetch_block(l, col(0));
                prefetch_block(l, col(1));
            }
            for (int cc = 0; cc < NC; ++cc) {
                if (g.tid() == 0) prefetch_block(l, col(cc + 2));
                color_pass<false, 0>(l, col(cc));
            }
        }
    }

    __device__ void residual(int l) const {
        if (l <= ls) {
            for (int c = 0; c < NC; ++c) color_pass<true, 1>(l, c);
        } else {
            for (int c = 0; c < NC; ++c) {
                if (g.tid() == 0) prefetch_block(l, (c + 2) % NC);
                color_pass<false, 1>(l, c);
            }
        }
        g.sync();
    }

    // color-major position of natural (i0,i1,i2) at level l >= 1
    __device__ __forceinline__ int cm_pos(const LevelDesc& L, int i0, int i1, int i2) const {
        const int c = (i0 % C0) + C0 * ((i1 % C1) + C1 * (i2 % C2));
        return c * L.blk + (i0 / C0 + 1) + L.xk[0] * ((i1 / C1 + 1) + (D == 3 ? L.xk[1] * (i2 / C2 + 1) : 0));
    }

    // b_{l-1} = P^T r_l (r natural), x_{l-1} = 0
    __device__ void restrict_to(int l) const {
        const LevelDesc& F = P->lev[l];
        const LevelDesc& Cl = P->lev[l - 1];
        T* bc = vp(b_off + Cl.boff);
        T* xc = vp(x_off + Cl.xoff);
        const T* rs = vp(r_off);
        const int nxc = l - 1 >= 1 ? Cl.nx : Cl.n;
        for (int t = g.tid(); t < nxc; t += g.nt()) xc[t] = T(0);
        const int pp[3] = {P0, P1, P2};
        for (int I = g.tid(); I < Cl.n; I += g.nt()) {
            const int I0 = I % Cl.m[0], Ir = I / Cl.m[0];
            const int I1 = Ir % Cl.m[1], I2 = Ir / Cl.m[1];
            const int dst = l - 1 >= 1 ? ieti_store_pos(Cl.m, pp, I0, I1, I2) : I;
            if (ieti_masked(mask, Cl.m, I0, I1, I2)) {
                bc[dst] = T(0);
                continue;
            }
            const int a0 = itab[F.rs[0] + I0], a1 = itab[F.rs[1] + I1];
            const int a2 = D == 3 ? itab[F.rs[2] + I2] : 0;
            const T* w0 = tab + F.rw[0] + I0 * R0;
            const T* w1 = tab + F.rw[1] + I1 * R1;
            const T* w2 = D == 3 ? tab + F.rw[2] + I2 * R2 : nullptr;
            T acc = 0;
#pragma unroll
            for (int u2 = 0; u2 < R2; ++u2) {
                const int f2 = a2 + u2;
                const T ww2 = D == 3 ? w2[u2] : T(1);
                const bool ok2 = f2 < F.m[2];
#pragma unroll
                for (int u1 = 0; u1 < R1; ++u1) {
                    const int f1 = a1 + u1;
                    const bool ok1 = ok2 && f1 < F.m[1];
                    const T ww1 = w1[u1] * ww2;
                    const int rb = F.m[0] * ((ok1 ? f1 : 0) + F.m[1] * (ok1 ? f2 : 0));
                    T s = 0;
#pragma unroll
                    for (int u0 = 0; u0 < R0; ++u0) {
                        const int f0 = a0 + u0;
                        const bool ok = ok1 && f0 < F.m[0];
                        s += w0[u0] * (ok ? rs[rb + f0] : T(0));
                    }
                    acc += ww1 * s;
                }
            }
            bc[dst] = acc;
        }
        g.sync();
    }

    // x_l += P x_{l-1}
    __device__ void prolong_add(int l) const {
        const LevelDesc& F = P->lev[l];
        const LevelDesc& Cl = P->lev[l - 1];
        const T* xc = vp(x_off + Cl.xoff);
        T* x = vp(x_off + F.xoff);
        const bool cnat = l - 1 == 0;
        for (int i = g.tid(); i < F.n; i += g.nt()) {
            const int i0 = i % F.m[0], ir = i / F.m[0];
            const int i1 = ir % F.m[1], i2 = ir / F.m[1];
            if (ieti_masked(mask, F.m, i0, i1, i2)) continue;
            const int a0 = itab[F.ps[0] + i0], a1 = itab[F.ps[1] + i1];
            const int a2 = D == 3 ? itab[F.ps[2] + i2] : 0;
            const T* w0 = tab + F.pw[0] + i0 * R0;
            const T* w1 = tab + F.pw[1] + i1 * R1;
            const T* w2 = D == 3 ? tab + F.pw[2] + i2 * R2 : nullptr;
            // the coarse position (natural or color-major) is a sum of one
            // term per direction: f0(q0) + f1(q1) + f2(q2)
            int f0[R0], f1[R1], f2[R2];
#pragma unroll
            for (int u = 0; u < R0; ++u) {
                const int q = a0 + u;
                f0[u] = cnat ? q : (q % C0) * Cl.blk + q / C0 + 1;
            }
#pragma unroll
            for (int u = 0; u < R1; ++u) {
                const int q = a1 + u;
                f1[u] = cnat ? Cl.m[0] * q : (q % C1) * C0 * Cl.blk + Cl.xk[0] * (q / C1 + 1);
            }
#pragma unroll
            for (int u = 0; u < R2; ++u) {
                const int q = a2 + u;
                f2[u] = D != 3 ? 0
                               : (cnat ? Cl.m[0] * Cl.m[1] * q
                                       : (q % C2) * C0 * C1 * Cl.blk + Cl.xk[0] * Cl.xk[1] * (q / C2 + 1));
            }
            T acc = 0;
#pragma unroll
            for (int u2 = 0; u2 < R2; ++u2) {
                const int q2 = a2 + u2;
                const T ww2 = D == 3 ? w2[u2] : T(1);
                if (q2 >= Cl.m[2]) continue;
#pragma unroll
                for (int u1 = 0; u1 < R1; ++u1) {
                    const int q1 = a1 + u1;
                    if (q1 >= Cl.m[1]) continue;
                    const T ww1 = w1[u1] * ww2;
                    const int f12 = f1[u1] + f2[u2];
                    T s = 0;
#pragma unroll
                    for (int u0 = 0; u0 < R0; ++u0) {
                        const int q0 = a0 + u0;
                        if (q0 >= Cl.m[0]) continue;
                        s += w0[u0] * xc[f0[u0] + f12];
                    }
                    acc += ww1 * s;
                }
            }
            x[cm_pos(F, i0, i1, i2)] += acc;
        }
        g.sync();
    }

    __device__ void coarsest() const {
        const int n = P->lev[0].n;
        const T* b = vp(b_off + P->lev[0].boff);
        T* x = vp(x_off + P->lev[0].xoff);
        for (int i = g.tid(); i < n; i += g.nt()) {
            T acc0 = 0, acc1 = 0;
            int j = 0;
            if (a0_off >= 0) {
                const T* A = shm<T>(a0_off);
                for (; j + 1 < n; j += 2) {
                    acc0 += A[j * n + i] * b[j];
                    acc1 += A[(j + 1) * n + i] * b[j + 1];
                }
                if (j < n) acc0 += A[j * n + i] * b[j];
            } else {
                for (; j + 1 < n; j += 2) {
                    acc0 += A0g[(long long)j * n + i] * b[j];
                    acc1 += A0g[(long long)(j + 1) * n + i] * b[j + 1];
                }
                if (j < n) acc0 += A0g[(long long)j * n + i] * b[j];
            }
            x[i] = acc0 + acc1;
        }
        g.sync();
    }

    // x_fine = V(b_fine): b_fine (storage order, or natural for a 1-level
    // hierarchy) set by the caller
    __device__ __noinline__ void run(int nu1, int nu2) const {
        const int L = P->L;
        if (L == 1) {
            coarsest();
            return;
        }
        {
            T* x = vp(x_off + P->lev[L - 1].xoff);
            const int nx = P->lev[L - 1].nx;
            for (int i = g.tid(); i < nx; i += g.nt()) x[i] = T(0);
            g.sync();
        }
        for (int l = L - 1; l >= 1; --l) {
            {
                IETI_T0();
                for (int s = 0; s < nu1; ++s) sweep(l, true);
                IETI_T1(4 * l + 0);
            }
            {
                IETI_T0();
                residual(l);
                IETI_T1(4 * l + 1);
            }
            {
                IETI_T0();
                restrict_to(l);
                IETI_T1(4 * l + 2);
            }
        }
        {
            IETI_T0();
            coarsest();
            IETI_T1(48);
        }
        for (int l = 1; l <= L - 1; ++l) {
            {
                IETI_T0();
                prolong_add(l);
                IETI_T1(4 * l + 3);
            }
            {
                IETI_T0();
                for (int s = 0; s < nu2; ++s) sweep(l, false);
                IETI_T1(4 * l + 0);
            }
        }
    }

    // fill the color tables of every level
    __device__ void build_tables(CTab* tabs) const {
        const int pp[3] = {P0, P1, P2};
        for (int e = threadIdx.x; e < P->L * NC; e += blockDim.x) {
            const int l = e / NC, c = e % NC;
            const LevelDesc& L = P->lev[l];
            const int c0 = c % C0, c1 = (c / C0) % C1, c2 = c / (C0 * C1);
            CTab t;
            t.off = ieti_color_off(L.m, pp, c0, c1, c2);
            t.k0 = ieti_cnt(L.m[0], P0, c0);
            t.k1 = ieti_cnt(L.m[1], P1, c1);
            t.k2 = ieti_cnt(L.m[2], P2, c2);
            t.xk0 = L.xk[0];
            t.xk1 = L.xk[1];
            t.xb = c * L.blk;
            tabs[e] = t;
        }
    }
};

// y = K x (FP64, fine level), rows masked by `rowmask` set to 0; with `sub`,
// y = sub + scale K x; `only` = 1 keeps interface rows (boundary rows not on
// the Dirichlet boundary) and zeroes the others.  Rows are visited color by
// color so that each stencil diagonal is read with unit stride.  With
// xs_off >= 0, x is first copied to dynamic shared memory at that element
// offset (doubles; a free region of at least n doubles), so that a row's
// neighbour reads are shared-memory loads and its registers hold only the
// streamed matrix values.
template <int D, int P0, int P1, int P2, bool CL = false>
__device__ __noinline__ void spmv64(const PatchDesc& P, const double* __restrict__ K64, const double* x, double* y,
                                    int rowmask, const double* sub, double scale, int only,
                                    long long* phase = nullptr, int xs_off = -1, GrpT<CL> g = GrpT<CL>{0, 1}) {
    constexpr int W0 = 2 * P0 + 1, W1 = 2 * P1 + 1, W2 = 2 * P2 + 1, S = W0 * W1 * W2;
    constexpr int C0 = P0 + 1, C1 = P1 + 1, C2 = P2 + 1, NC = C0 * C1 * C2;
    const LevelDesc& F = P.lev[P.L - 1];
    const int m0 = F.m[0], m1 = F.m[1], m2 = F.m[2];
    IETI_T0();
    if (xs_off >= 0) {
        double* xs = shm<double>(xs_off);
        for (int i = threadIdx.x; i < F.n; i += blockDim.x) xs[i] = x[i];
        __syncthreads();
    }
    // all rows at once (no dependency between colors): row s of the storage
    // order belongs to the color whose range [off, off + cnt) contains it
    int kk0[C0], kk1[C1], kk2[C2];
#pragma unroll
    for (int c = 0; c < C0; ++c) kk0[c] = ieti_cnt(m0, P0, c);
#pragma unroll
    for (int c = 0; c < C1; ++c) kk1[c] = ieti_cnt(m1, P1, c);
#pragma unroll
    for (int c = 0; c < C2; ++c) kk2[c] = ieti_cnt(m2, P2, c);
    for (int s = g.tid(); s < F.n; s += g.nt()) {
        int off = 0, c = 0, cnt = 0;
#pragma unroll 1
        for (c = 0; c < NC; ++c) {
            cnt = kk0[c % C0] * kk1[(c / C0) % C1] * kk2[c / (C0 * C1)];
            if (s < off + cnt) break;
            off += cnt;
        }
        const int c0 = c % C0, c1 = (c / C0) % C1, c2 = c / (C0 * C1);
        const int k0 = kk0[c0], k1 = kk1[c1];
        const int q = s - off;
        const int t0 = q % k0, tr = q / k0;
        const int t1 = tr % k1, t2 = tr / k1;
        const int i0 = c0 + C0 * t0, i1 = c1 + C1 * t1, i2 = c2 + C2 * t2;
        const int i = i0 + m0 * (i1 + m1 * i2);
        bool take = !ieti_masked(rowmask, F.m, i0, i1, i2);
        if (only == 1) take = take && ieti_on_boundary(F.m, D, i0, i1, i2) && !ieti_masked(P.dmask, F.m, i0, i1, i2);
        double v = 0.0;
        if (take) {
            double acc[4] = {0.0, 0.0, 0.0, 0.0};
            const double* vq = K64 + F.koff + (long long)off * S + q;
#pragma unroll
            for (int o = 0; o < S; ++o) {
                const int o0 = o % W0 - P0, o1 = (o / W0) % W1 - P1, o2 = o / (W0 * W1) - P2;
                const bool ok = (unsigned)(i0 + o0) < (unsigned)m0 && (unsigned)(i1 + o1) < (unsigned)m1 &&
                                (unsigned)(i2 + o2) < (unsigned)m2;
                const int xi = ok ? i + o0 + m0 * (o1 + m1 * o2) : i;
                const double xv = xs_off >= 0 ? shm<double>(xs_off)[xi] : x[xi];
                acc[o & 3] += __ldg(vq + (long long)o * cnt) * xv;
            }
            v = scale * ((acc[0] + acc[1]) + (acc[2] + acc[3]));
        }
        if (sub) v = sub[i] + v;
        y[i] = v;
    }
    g.sync();
    IETI_T1(49);
}

// The same operator on the mixed path, on the FP32 pipes: K = Khi + Klo
// (Khi the FP32 rounding of K, Klo the FP32 rounding of the rest: 48
// significant bits together) and x = xhi + xlo staged in shared memory as
// FP32 pairs.  Each product Khi xhi is split exactly into its rounded value
// and rounding error by an FMA, the cross terms Khi xlo + Klo xhi are formed
// in FP32 (Klo xlo, 2^-48 relative, is dropped), and the row sum is carried as
// an unevaluated pair (s, c) with error-free two-sums: the FP64 row sum to
// about 2^-47 of the sum of the terms' magnitudes, for twelve FP32 operations
// per term instead of one FP64 FMA (GB300 runs FP64 at a small fraction of
// its FP32 rate).  xs_off: element offset (8-byte pairs) of the staging area.
__device__ __forceinline__ void df_add(float& s, float& c, float p, float e) {
    const float t = s + p;
    const float bb = t - s;
    const float err = (s - (t - bb)) + (p - bb);
    s = t;
    c += err + e;
}

template <int D, int P0, int P1, int P2>
__device__ __noinline__ void spmv_df(const PatchDesc& P, const float* __restrict__ Khi, const float* __restrict__ Klo,
                                     const double* x, double* y, int rowmask, const double* sub, double scale,
                                     int only, long long* phase, int xs_off) {
    constexpr int W0 = 2 * P0 + 1, W1 = 2 * P1 + 1, W2 = 2 * P2 + 1, S = W0 * W1 * W2;
    constexpr int C0 = P0 + 1, C1 = P1 + 1, C2 = P2 + 1, NC = C0 * C1 * C2;
    const LevelDesc& F = P.lev[P.L - 1];
    const int m0 = F.m[0], m1 = F.m[1], m2 = F.m[2];
    IETI_T0();
    float2* xs = reinterpret_cast<float2*>(shm<double>(xs_off));
    for (int i = threadIdx.x; i < F.n; i += blockDim.x) {
        const double v = x[i];
        const float hi = (float)v;
        xs[i] = make_float2(hi, (float)(v - (double)hi));
    }
    __syncthreads();
    int kk0[C0], kk1[C1], kk2[C2];
#pragma unroll
    for (int c = 0; c < C0; ++c) kk0[c] = ieti_cnt(m0, P0, c);
#pragma unroll
    for (int c = 0; c < C1; ++c) kk1[c] = ieti_cnt(m1, P1, c);
#pragma unroll
    for (int c = 0; c < C2; ++c) kk2[c] = ieti_cnt(m2, P2, c);
    for (int s = threadIdx.x; s < F.n; s += blockDim.x) {
        int off = 0, c = 0, cnt = 0;
#pragma unroll 1
        for (c = 0; c < NC; ++c) {
            cnt = kk0[c % C0] * kk1[(c / C0) % C1] * kk2[c / (C0 * C1)];
            if (s < off + cnt) break;
            off += cnt;
        }
        const int c0 = c % C0, c1 = (c / C0) % C1, c2 = c / (C0 * C1);
        const int k0 = kk0[c0], k1 = kk1[c1];
        const int q = s - off;
        const int t0 = q % k0, tr = q / k0;
        const int t1 = tr % k1, t2 = tr / k1;
        const int i0 = c0 + C0 * t0, i1 = c1 + C1 * t1, i2 = c2 + C2 * t2;
        const int i = i0 + m0 * (i1 + m1 * i2);
        bool take = !ieti_masked(rowmask, F.m, i0, i1, i2);
        if (only == 1) take = take && ieti_on_boundary(F.m, D, i0, i1, i2) && !ieti_masked(P.dmask, F.m, i0, i1, i2);
        double v = 0.0;
        if (take) {
            float sh[2] = {0.f, 0.f}, sc[2] = {0.f, 0.f};
            const long long base = F.koff + (long long)off * S + q;
#pragma unroll
            for (int o = 0; o < S; ++o) {
                const int o0 = o % W0 - P0, o1 = (o / W0) % W1 - P1, o2 = o / (W0 * W1) - P2;
                const bool ok = (unsigned)(i0 + o0) < (unsigned)m0 && (unsigned)(i1 + o1) < (unsigned)m1 &&
                                (unsigned)(i2 + o2) < (unsigned)m2;
                const int xi = ok ? i + o0 + m0 * (o1 + m1 * o2) : i;
                const float2 xv = xs[xi];
                const float ah = __ldg(Khi + base + (long long)o * cnt);
                const float al = __ldg(Klo + base + (long long)o * cnt);
                const float pr = ah * xv.x;
                const float pe = fmaf(ah, xv.x, -pr);
                const float cr = fmaf(ah, xv.y, al * xv.x);
                df_add(sh[o & 1], sc[o & 1], pr, pe + cr);
            }
            df_add(sh[0], sc[0], sh[1], sc[1]);
            v = scale * ((double)sh[0] + (double)sc[0]);
        }
        if (sub) v = sub[i] + v;
        y[i] = v;
    }
    __syncthreads();
    IETI_T1(49);
}

// The same operator with its input staged in the color-major, ghost-padded
// layout of the V-cycle vectors (color block c at c * blk, row (t0, t1, t2)
// of the block at (t0+1) + xk0 (t1+1) + xk0 xk1 (t2+1), zeros in the ghost
// layer): a warp's rows of one color read consecutive pairs (no bank
// conflicts) and every neighbour lies at a fixed offset per color (no bounds
// tests).  Rows are visited in storage order, each thread advancing its color
// as its row index passes the color's end; thread 0 moves the color blocks two
// colors ahead into L2 (bulk prefetch) as it enters each color.  `ct`: the
// fine level's color table; needs NC * blk pairs of staging space.
template <int D, int P0, int P1, int P2>
__device__ __noinline__ void spmv_df_cm(const PatchDesc& P, const CTab* __restrict__ ct, const float* __restrict__ Khi,
                                        const float* __restrict__ Klo, const double* x, double* y, int rowmask,
                                        const double* sub, double scale, int only, long long* phase, int xs_off,
                                        bool prefetch) {
    constexpr int W0 = 2 * P0 + 1, W1 = 2 * P1 + 1, W2 = 2 * P2 + 1, S = W0 * W1 * W2;
    constexpr int C0 = P0 + 1, C1 = P1 + 1, C2 = P2 + 1, NC = C0 * C1 * C2;
    const LevelDesc& F = P.lev[P.L - 1];
    const int m0 = F.m[0], m1 = F.m[1], m2 = F.m[2];
    const int blk = F.blk, xk0 = F.xk[0], xk1 = F.xk[1], xk01 = xk0 * xk1;
    IETI_T0();
    float2* xs = reinterpret_cast<float2*>(shm<double>(xs_off));
    for (int e = threadIdx.x; e < NC * blk; e += blockDim.x) {
        const int c = e / blk, w = e - c * blk;
        const int c0 = c % C0, c1 = (c / C0) % C1, c2 = c / (C0 * C1);
        const int t0 = w % xk0 - 1, t1 = (w / xk0) % xk1 - 1, t2 = D == 3 ? w / xk01 - 1 : 0;
        const int i0 = c0 + C0 * t0, i1 = c1 + C1 * t1, i2 = c2 + C2 * t2;
        const bool in = t0 >= 0 && i0 < m0 && t1 >= 0 && i1 < m1 && (D < 3 || (t2 >= 0 && i2 < m2));
        const double v = in ? x[i0 + m0 * (i1 + m1 * i2)] : 0.0;
        const float hi = (float)v;
        xs[e] = make_float2(hi, (float)(v - (double)hi));
    }
    constexpr long long A = 4;   // 16 bytes of FP32
    auto prefetch_color = [&](int c) {
        if (!prefetch || c >= NC) return;
        const CTab t = ct[c];
        const long long s0 = F.koff + (long long)t.off * S;
        const long long len = (long long)t.k0 * t.k1 * t.k2 * S;
        const long long lo = s0 & ~(A - 1), hi = (s0 + len + A - 1) & ~(A - 1);
        bulk_prefetch_l2(Khi + lo, (unsigned)((hi - lo) * 4));
        bulk_prefetch_l2(Klo + lo, (unsigned)((hi - lo) * 4));
    };
    if (threadIdx.x == 0) {
        prefetch_color(0);
        prefetch_color(1);
    }
    __syncthreads();
    int c = -1, off = 0, cnt = 0, end = 0;
    for (int s = threadIdx.x; s < F.n; s += blockDim.x) {
        while (s >= end) {
            ++c;
            const CTab t = ct[c];
            off = t.off;
            cnt = t.k0 * t.k1 * t.k2;
            end = off + cnt;
            if (threadIdx.x == 0) prefetch_color(c + 2);
        }
        const CTab t = ct[c];
        const int c0 = c % C0, c1 = (c / C0) % C1, c2 = c / (C0 * C1);
        const int q = s - off;
        const int t0 = q % t.k0, tr = q / t.k0;
        const int t1 = tr % t.k1, t2 = tr / t.k1;
        const int i0 = c0 + C0 * t0, i1 = c1 + C1 * t1, i2 = c2 + C2 * t2;
        const int i = i0 + m0 * (i1 + m1 * i2);
        bool take = !ieti_masked(rowmask, F.m, i0, i1, i2);
        if (only == 1) take = take && ieti_on_boundary(F.m, D, i0, i1, i2) && !ieti_masked(P.dmask, F.m, i0, i1, i2);
        double v = 0.0;
        if (take) {
            int e0[W0], e1[W1], e2[W2];
#pragma unroll
            for (int o = -P0; o <= P0; ++o) {
                const int dd = (c0 + o + C0) / C0 - 1;
                e0[o + P0] = (o - C0 * dd) * blk + dd;
            }
#pragma unroll
            for (int o = -P1; o <= P1; ++o) {
                const int dd = (c1 + o + C1) / C1 - 1;
                e1[o + P1] = (o - C1 * dd) * C0 * blk + dd * xk0;
            }
#pragma unroll
            for (int o = -P2; o <= P2; ++o) {
                const int dd = (c2 + o + C2) / C2 - 1;
                e2[o + P2] = D == 3 ? (o - C2 * dd) * C0 * C1 * blk + dd * xk01 : 0;
            }
            const float2* X = xs + c * blk + (t0 + 1) + xk0 * (t1 + 1) + (D == 3 ? xk01 * (t2 + 1) : 0);
            float sh[2] = {0.f, 0.f}, sc[2] = {0.f, 0.f};
            const long long base = F.koff + (long long)off * S + q;
#pragma unroll
            for (int o = 0; o < S; ++o) {
                const int o0 = o % W0, o1 = (o / W0) % W1, o2 = o / (W0 * W1);
                const float2 xv = X[e0[o0] + e1[o1] + e2[o2]];
                const float ah = __ldg(Khi + base + (long long)o * cnt);
                const float al = __ldg(Klo + base + (long long)o * cnt);
                const float pr = ah * xv.x;
                const float pe = fmaf(ah, xv.x, -pr);
                const float cr = fmaf(ah, xv.y, al * xv.x);
                df_add(sh[o & 1], sc[o & 1], pr, pe + cr);
            }
            df_add(sh[0], sc[0], sh[1], sc[1]);
            v = scale * ((double)sh[0] + (double)sc[0]);
        }
        if (sub) v = sub[i] + v;
        y[i] = v;
    }
    __syncthreads();
    IETI_T1(49);
}

template <typename T, int D, int P0, int P1, int P2, bool XG>
__device__ void vcycle_apply(const VC<T, D, P0, P1, P2, XG>& vc, const double* rin, double* zout, int nu1, int nu2) {
    const int L = vc.P->L;
    const LevelDesc& F = vc.P->lev[L - 1];
    const int n = F.n;
    T* b = vc.vp(vc.b_off + F.boff);
    const int pp[3] = {P0, P1, P2};
    const GrpT<XG> g = vc.g;
    for (int i = g.tid(); i < n; i += g.nt()) {
        const int i0 = i % F.m[0], ir = i / F.m[0];
        const int i1 = ir % F.m[1], i2 = ir / F.m[1];
        b[L > 1 ? ieti_store_pos(F.m, pp, i0, i1, i2) : i] = (T)rin[i];
    }
    g.sync();
    vc.run(nu1, nu2);
    const T* x = vc.vp(vc.x_off + F.xoff);
    for (int i = g.tid(); i < n; i += g.nt()) {
        const int i0 = i % F.m[0], ir = i / F.m[0];
        const int i1 = ir % F.m[1], i2 = ir / F.m[1];
        zout[i] = (double)x[L > 1 ? vc.cm_pos(F, i0, i1, i2) : i];
    }
    g.sync();
}

__device__ inline void project_kerC(const SolveArgs& a, const PatchDesc& P, double* v, double* coef) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = w; j < P.npi; j += nw) {
        const int row = P.crow0 + j;
        double d = 0.0, nn = 0.0;
        for (int e = a.crow_ptr[row] + lane; e < a.crow_ptr[row + 1]; e += 32) {
            const double ww = a.c_w[e];
            d += ww * v[a.c_idx[e]];
            nn += ww * ww;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            d += __shfl_xor_sync(0xffffffffu, d, o);
            nn += __shfl_xor_sync(0xffffffffu, nn, o);
        }
        if (lane == 0) coef[j] = d / nn;
    }
    __syncthreads();
    for (int j = w; j < P.npi; j += nw) {
        const int row = P.crow0 + j;
        const double cj = coef[j];
        for (int e = a.crow_ptr[row] + lane; e < a.crow_ptr[row + 1]; e += 32) v[a.c_idx[e]] -= a.c_w[e] * cj;
    }
    __syncthreads();
}

// v <- v - mean(v) over the n entries (the slot's group of CTAs)
template <bool CL>
__device__ inline void remove_mean(double* v, int n, Red& red, double* tot, const GrpT<CL>& g) {
    double s[1] = {0.0};
    for (int i = g.tid(); i < n; i += g.nt()) s[0] += v[i];
    grp_sum<1>(s, red, tot, g);
    const double mean = s[0] / n;
    for (int i = g.tid(); i < n; i += g.nt()) v[i] -= mean;
    g.sync();
}

__device__ inline void apply_C(const SolveArgs& a, const PatchDesc& P, const double* v, double* coef) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = w; j < P.npi; j += nw) {
        const int row = P.crow0 + j;
        double d = 0.0;
        for (int e = a.crow_ptr[row] + lane; e < a.crow_ptr[row + 1]; e += 32) d += a.c_w[e] * v[a.c_idx[e]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) coef[j] = d;
    }
    __syncthreads();
}

template <typename T, int D, int P0, int P1, int P2, bool XG>
__global__ void __launch_bounds__(512) k_solve_t(SolveArgs a0) {
    const IetiLaunchSpan span_(a0.tspan);
    __shared__ Red red;
    __shared__ double coef[kMaxRows];
    __shared__ double gtot[4];
    __shared__ PatchDesc sP;
    __shared__ SolveArgs sa;
    unsigned char* dyn = ieti_dyn;
    // a cluster launch serves one slot per cluster (its CTAs split the rows;
    // used for the modes of the solve phase on global-vector slots only)
    const GrpT<XG> grp = make_grp<XG>();
    const SlotDesc sd = a0.slots[blockIdx.x / grp.size];
    if (threadIdx.x == 0) {
        sa = a0.batch ? a0.batch[sd.handle] : a0;
        sa.slots = a0.slots;
        sa.nslots = a0.nslots;
        sa.smem_bytes = a0.smem_bytes;
    }
    __syncthreads();
    const SolveArgs& a = sa;
    if (grp.size > 1 && (!XG || !(a.mode == MODE_NEUMANN || a.mode == MODE_SCHUR || a.mode == MODE_VCYCLE ||
                                   a.mode == MODE_VCYCLE_DIR))) {
        // not a cluster mode (every CTA of the cluster returns here)
        if (grp.tid() == 0) atomicOr(a.flags, IETI_FLAG_BREAKDOWN);
        return;
    }
#ifdef IETI_DEBUG_BOUNDS
    if (threadIdx.x == 0) g_ieti_dbg = a.dbg;
    __syncthreads();
#endif
    {
        const int* src = (const int*)(a.pd + sd.patch);
        int* dst = (int*)&sP;
        for (int t = threadIdx.x; t < (int)(sizeof(PatchDesc) / sizeof(int)); t += blockDim.x) dst[t] = src[t];
    }
    __syncthreads();
    const PatchDesc& P = sP;
    const LevelDesc& F = P.lev[P.L - 1];
    const int n = F.n;
    double* x = a.cg + sd.cg;
    double* r = x + n;
    double* z = r + n;
    double* p = z + n;
    double* q = p + n;
    const int allsides = D == 2 ? 0xF : 0x3F;
    const int kind = (a.mode == MODE_SCHUR || a.mode == MODE_VCYCLE_DIR) ? 1 : 0;
    const T* A0g = (a.mixed ? (const T*)(const void*)a.A0inv32 : (const T*)(const void*)a.A0inv64) + P.a0off[kind];

    const Plan pl = make_plan(P, sizeof(T), a.smem_bytes, !XG);
    // the V-cycle vectors are dead between V-cycles (at least 12 n bytes in
    // the mixed path): the FP64 operator stages its input vector there
    const int xs_off = (!XG && pl.vec && !(a.kflags & 4)) ? (int)(pl.vec_off / sizeof(double)) : -1;
    const bool reg = kind == 0 && P.floating;
    const T* Kv = a.mixed ? (const T*)(const void*)(reg ? a.KM32 : a.K32)
                          : (const T*)(const void*)(reg ? a.KM64 : a.K64);
    __shared__ VC<T, D, P0, P1, P2, XG> vc_s;
    VC<T, D, P0, P1, P2, XG>& vc = vc_s;
    if (threadIdx.x == 0) {
        vc.P = &P;
        vc.mask = kind == 0 ? P.dmask : allsides;
        vc.Kg = Kv;
        vc.tab = a.mixed ? (const T*)(const void*)a.tabf : (const T*)(const void*)a.tab;
        vc.itab = a.itab;
        vc.x_off = XG ? 0 : (int)(pl.vec_off / sizeof(T));
        vc.gvec = (T*)a.lv + sd.lv;
        vc.b_off = vc.x_off + P.nlx;
        vc.r_off = vc.b_off + P.nlb;
        vc.kbase = P.L > 1 ? P.lev[1].koff : 0;
        vc.kflags = a.kflags;
        vc.ls = pl.ls;
        vc.ks_off = (int)(pl.mat_off / sizeof(T));
        vc.a0_off = pl.a0 ? (int)(pl.a0_off / sizeof(T)) : -1;
        vc.A0g = A0g;
        vc.ct = (const CTab*)(dyn + pl.tab_off);
        vc.phase = a.phase;
        vc.g = grp;
    }
    __syncthreads();
    vc.build_tables((CTab*)(dyn + pl.tab_off));
    if (pl.a0) {
        T* dst = (T*)(dyn + pl.a0_off);
        const int nn = P.lev[0].n * P.lev[0].n;
        for (int t = threadIdx.x; t < nn; t += blockDim.x) dst[t] = A0g[t];
    }
    if (pl.ls >= 1) {
        T* dst = (T*)(dyn + pl.mat_off);
        const long long cnt = P.lev[pl.ls].koff + (long long)P.lev[pl.ls].n * P.lev[pl.ls].S - P.lev[1].koff;
        const T* src = Kv + P.lev[1].koff;
        for (long long t = threadIdx.x; t < cnt; t += blockDim.x) dst[t] = src[t];
    }
    __syncthreads();
    long long vcount = 0;

    // the stiffness operator of the solve phase (CG, Schur complement,
    // V-cycle residuals): on the mixed path in FP32-pair arithmetic, else FP64
    const bool df = sizeof(T) == 4 && xs_off >= 0 && a.K32lo && !(a.kflags & 32);
    // the color-major staging takes NC blk pairs; the vector area holds at
    // least nlx + nlb + n FP32 values
    const bool dfcm = df && !(a.kflags & 128) &&
                      (size_t)ieti_ncolors(P.p) * F.blk * 8 <= (size_t)vec_elems(P) * sizeof(T);
    auto opK = [&](const double* in, double* out, int rmask, const double* sb, double sc, int only, long long* ph) {
        if (dfcm)
            spmv_df_cm<D, P0, P1, P2>(P, vc.ct + (P.L - 1) * ieti_ncolors(P.p), a.K32, a.K32lo, in, out, rmask, sb,
                                      sc, only, ph, xs_off, !(a.kflags & 16));
        else if (df)
            spmv_df<D, P0, P1, P2>(P, a.K32, a.K32lo, in, out, rmask, sb, sc, only, ph, xs_off);
        else
            spmv64<D, P0, P1, P2, XG>(P, a.K64, in, out, rmask, sb, sc, only, ph, xs_off, grp);
    };
    if (a.mode == MODE_SCHUR) {
        const double* v = a.in + P.toff;
        opK(v, r, allsides, nullptr, -1.0, 0, nullptr);
        for (int c = 0; c < a.ncycles; ++c) {
            if (c == 0) {
                vcycle_apply(vc, r, x, a.nu1, a.nu2);
            } else {
                opK(x, q, allsides, r, -1.0, 0, nullptr);
                vcycle_apply(vc, q, z, a.nu1, a.nu2);
                for (int i = grp.tid(); i < n; i += grp.nt()) x[i] += z[i];
                grp.sync();
            }
            ++vcount;
        }
        for (int i = grp.tid(); i < n; i += grp.nt()) p[i] = v[i] + x[i];
        grp.sync();
        opK(p, a.out + P.toff, 0, nullptr, 1.0, 1, nullptr);
        if (grp.tid() == 0 && a.vstats) {
            atomicAdd((unsigned long long*)&a.vstats[0], (unsigned long long)vcount);
            atomicAdd((unsigned long long*)&a.vstats[1], (unsigned long long)(vcount * n));
        }
        return;
    }

    if (a.mode == MODE_VCYCLE || a.mode == MODE_VCYCLE_DIR) {
        const double* bb = a.in + P.toff;
        double* xx = a.out + P.toff;
        const int rmask = kind == 0 ? P.dmask : allsides;
        for (int c = 0; c < a.ncycles; ++c) {
            opK(xx, r, rmask, bb, -1.0, 0, a.phase);
            for (int i = grp.tid(); i < n; i += grp.nt()) {
                const int i0 = i % F.m[0], ir = i / F.m[0];
                const int i1 = ir % F.m[1], i2 = ir / F.m[1];
                if (ieti_masked(rmask, F.m, i0, i1, i2)) r[i] = 0.0;
            }
            grp.sync();
            vcycle_apply(vc, r, z, a.nu1, a.nu2);
            for (int i = grp.tid(); i < n; i += grp.nt()) xx[i] += z[i];
            grp.sync();
            ++vcount;
        }
        if (grp.tid() == 0 && a.vstats) {
            atomicAdd((unsigned long long*)&a.vstats[0], (unsigned long long)vcount);
            atomicAdd((unsigned long long*)&a.vstats[1], (unsigned long long)(vcount * n));
        }
        return;
    }

    if (a.mode == MODE_POWER || a.mode == MODE_KHAT) {
        // operator of the Neumann hierarchy's fine level: K, or K + alpha M^
        // on floating patches
        const double* A64 = P.floating ? a.KM64 : a.K64;
        if (a.mode == MODE_POWER) {
            // energy-norm contraction of one V-cycle (I - V A) by power
            // iteration; start x_j = ((37 j) mod 101)/101 - 1/2 with j the rank
            // of the dof among the patch's free dofs
            const int lo0 = P.dmask & 1, lo1 = (P.dmask >> 2) & 1, lo2 = (P.dmask >> 4) & 1;
            const int nf0 = F.m[0] - lo0 - ((P.dmask >> 1) & 1);
            const int nf1 = F.m[1] - lo1 - ((P.dmask >> 3) & 1);
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int i0 = i % F.m[0], ir = i / F.m[0];
                const int i1 = ir % F.m[1], i2 = ir / F.m[1];
                if (ieti_masked(P.dmask, F.m, i0, i1, i2)) {
                    x[i] = 0.0;
                } else {
                    const long long j = (i0 - lo0) + (long long)nf0 * ((i1 - lo1) + (long long)nf1 * (i2 - (D == 3 ? lo2 : 0)));
                    x[i] = (double)((37 * j) % 101) / 101.0 - 0.5;
                }
            }
            __syncthreads();
            double rho = 0.0;
            for (int it = 0; it < a.maxit; ++it) {
                spmv64<D, P0, P1, P2>(P, A64, x, r, P.dmask, nullptr, 1.0, 0, nullptr, xs_off);
                vcycle_apply(vc, r, z, a.nu1, a.nu2);
                ++vcount;
                for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = x[i] - z[i];
                __syncthreads();
                spmv64<D, P0, P1, P2>(P, A64, p, q, P.dmask, nullptr, 1.0, 0, nullptr, xs_off);
                double s3[3] = {0.0, 0.0, 0.0};
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    s3[0] += x[i] * r[i];
                    s3[1] += p[i] * q[i];
                    s3[2] += p[i] * p[i];
                }
                cta_sum<3>(s3, red);
                rho = s3[0] > 0.0 ? sqrt(fmax(s3[1], 0.0) / s3[0]) : 0.0;
                const double inv = s3[2] > 0.0 ? 1.0 / sqrt(s3[2]) : 0.0;
                for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = p[i] * inv;
                __syncthreads();
            }
            if (threadIdx.x == 0) a.omega[sd.patch] = a.theta * (1.0 - pow(rho, (double)a.ncycles));
        } else {
            // w = P V^c P^T g / omega_k (c = ncycles V-cycles from zero, FP64
            // residuals); rpi_loc holds Phi^T g per constraint row
            const double* g = a.in + P.toff;
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int i0 = i % F.m[0], ir = i / F.m[0];
                const int i1 = ir % F.m[1], i2 = ir / F.m[1];
                r[i] = ieti_masked(P.dmask, F.m, i0, i1, i2) ? 0.0 : g[i];
            }
            __syncthreads();
            {
                const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
                for (int j = w; j < P.npi; j += nw) {
                    const int row = P.crow0 + j;
                    const double cj = a.rpi_loc[row];
                    for (int e = a.crow_ptr[row] + lane; e < a.crow_ptr[row + 1]; e += 32)
                        r[a.c_idx[e]] -= a.c_w[e] * cj;
                }
            }
            __syncthreads();
            for (int c = 0; c < a.ncycles; ++c) {
                if (c == 0) {
                    vcycle_apply(vc, r, x, a.nu1, a.nu2);
                } else {
                    spmv64<D, P0, P1, P2>(P, A64, x, q, P.dmask, r, -1.0, 0, nullptr, xs_off);
                    vcycle_apply(vc, q, z, a.nu1, a.nu2);
                    for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] += z[i];
                    __syncthreads();
                }
                ++vcount;
            }
            apply_C(a, P, x, coef);
            const double sc = 1.0 / a.omega[sd.patch];
            double* out = a.out + P.toff;
            const double* ph = a.phi + P.phioff;
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                double u = x[i];
                for (int j = 0; j < P.npi; ++j) u -= coef[j] * ph[(long long)j * n + i];
                out[i] = sc * u;
            }
        }
        if (threadIdx.x == 0 && a.vstats) {
            atomicAdd((unsigned long long*)&a.vstats[0], (unsigned long long)vcount);
            atomicAdd((unsigned long long*)&a.vstats[1], (unsigned long long)(vcount * n));
        }
        return;
    }

    if (a.mode == MODE_SZW || a.mode == MODE_BASIS_SZ) {
        auto vcyc = [&](const double* in, double* out) {
            vcycle_apply(vc, in, out, a.nu1, a.nu2);
            ++vcount;
        };
        auto spk = [&](const double* in, double* out) {
            spmv64<D, P0, P1, P2>(P, a.K64, in, out, P.dmask, nullptr, 1.0, 0, nullptr, xs_off);
        };
        double* base = a.cg + sd.cg;
        int it = 0;
        bool conv = true;
        if (a.mode == MODE_SZW) ieti_sz::szw_slot(a, P, sd, base, vcyc);
        else it = ieti_sz::sz_basis_slot(a, P, sd, base, &red.v[0][0], coef, vcyc, spk, &conv);
        if (threadIdx.x == 0) {
            if (a.mode == MODE_BASIS_SZ) {
                a.its[sd.its] = it;
                if (!conv) atomicOr(a.flags, IETI_FLAG_NOT_CONVERGED);
            }
            if (a.vstats) {
                atomicAdd((unsigned long long*)&a.vstats[0], (unsigned long long)vcount);
                atomicAdd((unsigned long long*)&a.vstats[1], (unsigned long long)(vcount * n));
            }
        }
        return;
    }

    const bool basis = a.mode == MODE_BASIS;
    double* phicol = nullptr;
    if (basis) {
        const int lr = sd.row - P.crow0;
        phicol = a.phi + P.phioff + (long long)lr * n;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            z[i] = 0.0;
            x[i] = 0.0;
        }
        __syncthreads();
        for (int e = a.crow_ptr[sd.row] + threadIdx.x; e < a.crow_ptr[sd.row + 1]; e += blockDim.x)
            if (IETI_OK(a.c_idx[e], n, 14)) z[a.c_idx[e]] = 1.0;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) phicol[i] = z[i];
        spmv64<D, P0, P1, P2>(P, a.K64, z, r, P.dmask, nullptr, -1.0, 0, nullptr, xs_off);
        project_kerC(a, P, r, coef);
    } else {
        const double* g = a.in + P.toff;
        for (int i = grp.tid(); i < n; i += grp.nt()) {
            const int i0 = i % F.m[0], ir = i / F.m[0];
            const int i1 = ir % F.m[1], i2 = ir / F.m[1];
            r[i] = ieti_masked(P.dmask, F.m, i0, i1, i2) ? 0.0 : g[i];
            x[i] = 0.0;
        }
        grp.sync();
        // b = P^T g = g - C^T (Phi^T g)
        {
            const int lane = threadIdx.x & 31, w = grp.tid() >> 5, nw = grp.nt() >> 5;
            for (int j = w; j < P.npi; j += nw) {
                const int row = P.crow0 + j;
                const double cj = a.rpi_loc[row];
                for (int e = a.crow_ptr[row] + lane; e < a.crow_ptr[row + 1]; e += 32) r[a.c_idx[e]] -= a.c_w[e] * cj;
            }
        }
        grp.sync();
        if (P.floating) remove_mean(r, n, red, gtot, grp);
    }
    double nb2;
    {
        double s[1] = {0.0};
        for (int i = grp.tid(); i < n; i += grp.nt()) s[0] += r[i] * r[i];
        grp_sum<1>(s, red, gtot, grp);
        nb2 = s[0];
    }
    int it = 0;
    bool conv = nb2 == 0.0;
    const double tol2 = a.tol * a.tol * nb2;
    // floating patches (Neumann mode): keep the preconditioned residual
    // orthogonal to the constants, the kernel of K
    const bool proj1 = !basis && P.floating;
    if (!conv) {
        vcycle_apply(vc, r, z, a.nu1, a.nu2);
        ++vcount;
        if (basis) project_kerC(a, P, z, coef);
        if (proj1) remove_mean(z, n, red, gtot, grp);
        double rz;
        {
            double s[1] = {0.0};
            for (int i = grp.tid(); i < n; i += grp.nt()) {
                p[i] = z[i];
                s[0] += r[i] * z[i];
            }
            grp_sum<1>(s, red, gtot, grp);
            rz = s[0];
        }
        for (it = 1; it <= a.maxit; ++it) {
            double s[1] = {0.0};
            if (basis)
                spmv64<D, P0, P1, P2>(P, a.K64, p, q, P.dmask, nullptr, 1.0, 0, a.phase, xs_off);
            else
                opK(p, q, P.dmask, nullptr, 1.0, 0, a.phase);
            if (basis) project_kerC(a, P, q, coef);
            for (int i = grp.tid(); i < n; i += grp.nt()) s[0] += p[i] * q[i];
            grp_sum<1>(s, red, gtot, grp);
            const double pq = s[0];
            if (!(pq > 0.0) || !isfinite(pq)) {
                if (grp.tid() == 0) atomicOr(a.flags, IETI_FLAG_BREAKDOWN);
                break;
            }
            const double alpha = rz / pq;
            double s2[1] = {0.0};
            for (int i = grp.tid(); i < n; i += grp.nt()) {
                x[i] += alpha * p[i];
                const double ri = r[i] - alpha * q[i];
                r[i] = ri;
                s2[0] += ri * ri;
            }
            grp_sum<1>(s2, red, gtot, grp);
            if (s2[0] <= tol2) {
                conv = true;
                break;
            }
            vcycle_apply(vc, r, z, a.nu1, a.nu2);
            ++vcount;
            if (basis) project_kerC(a, P, z, coef);
            if (proj1) remove_mean(z, n, red, gtot, grp);
            double s3[2] = {0.0, 0.0};
            for (int i = grp.tid(); i < n; i += grp.nt()) {
                s3[0] += r[i] * z[i];
                s3[1] += q[i] * z[i];
            }
            grp_sum<2>(s3, red, gtot, grp);
            const double beta = a.mixed ? -alpha * s3[1] / rz : s3[0] / rz;
            rz = s3[0];
            for (int i = grp.tid(); i < n; i += grp.nt()) p[i] = z[i] + beta * p[i];
            grp.sync();
        }
        if (!conv && it > a.maxit) it = a.maxit;
    }
    if (grp.tid() == 0) {
        a.its[sd.its] = it;
        if (!conv) atomicOr(a.flags, IETI_FLAG_NOT_CONVERGED);
        if (a.vstats) {
            atomicAdd((unsigned long long*)&a.vstats[0], (unsigned long long)vcount);
            atomicAdd((unsigned long long*)&a.vstats[1], (unsigned long long)(vcount * n));
            atomicAdd((unsigned long long*)&a.vstats[2], (unsigned long long)it);
            atomicMax((unsigned long long*)&a.vstats[3], (unsigned long long)it);
            if (nb2 > 0.0) atomicAdd((unsigned long long*)&a.vstats[4], 1ULL);
        }
    }
    if (basis) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) phicol[i] += x[i];
        return;
    }
    // every CTA of the group forms the coefficients (x is complete after the
    // group barrier that ended the CG) in its own shared memory
    apply_C(a, P, x, coef);
    for (int j = threadIdx.x; j < P.npi; j += blockDim.x) coef[j] -= a.upi_loc[P.crow0 + j];
    __syncthreads();
    double* out = a.out + P.toff;
    const double* ph = a.phi + P.phioff;
    for (int i = grp.tid(); i < n; i += grp.nt()) {
        double u = x[i];
        for (int j = 0; j < P.npi; ++j) u -= coef[j] * ph[(long long)j * n + i];
        out[i] = u;
    }
}

// occ != nullptr: report the resident CTAs per SM of a launch with `threads`
// threads and a.smem_bytes dynamic shared memory instead of launching
template <typename T, int D, int P0, int P1, int P2, bool XG>
cudaError_t launch_t(const SolveArgs& a, int threads, cudaStream_t st, int* occ) {
    auto kern = k_solve_t<T, D, P0, P1, P2, XG>;
    // the attribute is an upper bound shared by all host threads: always set
    // the fixed cap (a smaller value set by one thread could otherwise race
    // with a larger launch from another)
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSolveSmemCap);
    if (e != cudaSuccess) return e;
    if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, kern, threads, a.smem_bytes);
    if (a.nslots == 0) return cudaSuccess;
    if (a.csize > 1) {
        // one cluster of csize CTAs per slot (a shape whose cluster does not
        // fit on the GPU is refused by the launch: an error, nothing runs)
        if (!XG || a.csize > 8) return cudaErrorInvalidConfiguration;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)a.csize;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)(a.nslots * a.csize));
        cfg.blockDim = dim3((unsigned)threads);
        cfg.dynamicSmemBytes = a.smem_bytes;
        cfg.stream = st;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, kern, a);
    }
    kern<<<a.nslots, threads, a.smem_bytes, st>>>(a);
    return cudaGetLastError();
}

}  // namespace ieti_t
