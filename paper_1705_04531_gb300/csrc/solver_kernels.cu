// Local solver kernels of inexact IETI-DP (Sec. 3): one CTA owns one local
// problem ("slot": a patch and a right-hand side) for the whole solve, so a
// single launch runs a complete multigrid-preconditioned CG, or a complete
// scaled-Dirichlet Schur application, for every patch of every problem in
// the batch.  Colors of the multicolor Gauss-Seidel smoother, levels of the
// V-cycle and CG iterations are separated by CTA barriers only.
//
// Precision: the CG (vectors, residuals, dot products, the FP64 stiffness
// SpMV) is always FP64; the V-cycle (smoother, residual, transfers, coarsest
// solve) runs in T = double or T = float.
#include <math.h>
#include "kernels.cuh"
#include "sz_device.cuh"

namespace {

constexpr int kMaxRows = 64;   // primal rows per patch handled by one CTA

struct Red {
    double v[32][4];
};

// sum of up to 4 values over the CTA; every thread gets the totals
template <int K>
__device__ __forceinline__ void cta_sum(double* val, Red& sh) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
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

template <typename T>
struct Tabs {
    const T* tab;
    const int* itab;
};

// (A x)_i for one row: banded stiffness of a level plus, when alpha != 0,
// alpha times the Kronecker parameter mass.  Returns the diagonal in *diag.
// vals: the color block of the row's color (offset-major), cnt its rows,
// s the row's number q inside the color.  Each line of the stencil (fixed
// o1, o2) is read into registers first, WM entries at most (WM >= 2 p0 + 1,
// entries past the line's end predicated off), so that its loads are in
// flight together, and summed into four partial sums.
template <int WM, typename V, typename X, typename A>
__device__ __forceinline__ A row_apply_w(const V* __restrict__ vals, int cnt, int s, const X* x,
                                         const int* m, const int* p, int i0, int i1, int i2,
                                         const V* mt0, const V* mt1, const V* mt2, A alpha, A* diag) {
    int lo0 = max(-p[0], -i0), hi0 = min(p[0], m[0] - 1 - i0);
    int lo1 = max(-p[1], -i1), hi1 = min(p[1], m[1] - 1 - i1);
    int lo2 = max(-p[2], -i2), hi2 = min(p[2], m[2] - 1 - i2);
    int w0 = 2 * p[0] + 1, w1 = 2 * p[1] + 1;
    A acc[4] = {A(0), A(0), A(0), A(0)};
    for (int o2 = lo2; o2 <= hi2; ++o2)
        for (int o1 = lo1; o1 <= hi1; ++o1) {
            int ob = ((o2 + p[2]) * w1 + (o1 + p[1])) * w0 + p[0];
            int xb = i0 + m[0] * ((i1 + o1) + m[1] * (i2 + o2));
            A m12 = 0;
            if (alpha != A(0)) {
                m12 = (A)mt1[i1 * w1 + o1 + p[1]];
                if (mt2) m12 *= (A)mt2[i2 * (2 * p[2] + 1) + o2 + p[2]];
            }
            A vv[WM], xv[WM];
#pragma unroll
            for (int k = 0; k < WM; ++k) {
                const int o0 = lo0 + k;
                const bool ok = o0 <= hi0;
                vv[k] = ok ? (A)vals[(long long)(ob + o0) * cnt + s] : A(0);
                xv[k] = ok ? (A)x[xb + o0] : A(0);
            }
            if (alpha != A(0)) {
#pragma unroll
                for (int k = 0; k < WM; ++k) {
                    const int o0 = lo0 + k;
                    if (o0 <= hi0) vv[k] += alpha * (A)mt0[i0 * w0 + o0 + p[0]] * m12;
                }
            }
#pragma unroll
            for (int k = 0; k < WM; ++k) acc[k & 3] += vv[k] * xv[k];
        }
    if (diag) {
        int oc = ((p[2]) * w1 + p[1]) * w0 + p[0];
        A d = (A)vals[(long long)oc * cnt + s];
        if (alpha != A(0)) {
            A mm = (A)mt0[i0 * w0 + p[0]] * (A)mt1[i1 * w1 + p[1]];
            if (mt2) mm *= (A)mt2[i2 * (2 * p[2] + 1) + p[2]];
            d += alpha * mm;
        }
        *diag = d;
    }
    return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

template <typename V, typename X, typename A>
__device__ __forceinline__ A row_apply(const V* __restrict__ vals, int cnt, int s, const X* x,
                                       const int* m, const int* p, int i0, int i1, int i2,
                                       const V* mt0, const V* mt1, const V* mt2, A alpha, A* diag) {
    if (p[0] <= 1)
        return row_apply_w<3, V, X, A>(vals, cnt, s, x, m, p, i0, i1, i2, mt0, mt1, mt2, alpha, diag);
    if (p[0] <= 3)
        return row_apply_w<7, V, X, A>(vals, cnt, s, x, m, p, i0, i1, i2, mt0, mt1, mt2, alpha, diag);
    return row_apply_w<2 * (IETI_MAXP - 1) + 1, V, X, A>(vals, cnt, s, x, m, p, i0, i1, i2, mt0, mt1, mt2, alpha,
                                                         diag);
}

// Optional phase counters (built with -DIETI_PHASE_TIMERS): thread 0 of CTA 0
// adds clock cycles per phase to phase[]: [52] fine residuals of the
// high-order V-cycle, [53] its smoother, [54] restriction, [55] degree-1
// V-cycle, [56] prolongation, [57] the CG's fine operator (V-cycle mode:
// the residual), [58] V-cycle input / output conversions.
#ifdef IETI_PHASE_TIMERS
#define HO_DECL() long long _h0 = 0
#define HO_T0() do { if (threadIdx.x == 0 && blockIdx.x == 0) _h0 = clock64(); } while (0)
#define HO_T1(ph, k) do { if (threadIdx.x == 0 && blockIdx.x == 0 && (ph)) (ph)[k] += clock64() - _h0; } while (0)
#else
#define HO_DECL() do {} while (0)
#define HO_T0() do {} while (0)
#define HO_T1(ph, k) do {} while (0)
#endif

template <typename T>
struct VCycle {
    const PatchDesc* P;
    int mask;         // side mask of the hierarchy
    T alpha;          // regularization (0 unless Neumann hierarchy of a floating patch)
    const T* K;       // value pool in T
    const T* tab;     // 1D tables in T
    const int* itab;
    const T* A0inv;   // coarsest inverse
    T* lvec;          // this slot's level vectors: x | b | r, each nlvec
    int nlvec;
    // high-order multigrid (Sec. 4, p >= 4): null for the standard V-cycle;
    // else the patch's descriptor, the hierarchy kind, the operator pool, the
    // degree-1 hierarchy below the finest level and two work tensors of the
    // fine free grid
    const HoDesc* ho = nullptr;
    int hkind = 0;
    const T* hpool = nullptr;
    const VCycle<T>* coarse = nullptr;
    T* t1 = nullptr;
    T* t2 = nullptr;
    long long* phase = nullptr;   // phase counters (profiling builds)

    __device__ T* X(int l) const { return lvec + P->lev[l].voff; }
    __device__ T* B(int l) const { return lvec + nlvec + P->lev[l].voff; }
    __device__ T* R(int l) const { return lvec + 2 * nlvec + P->lev[l].voff; }

    __device__ void mass_tabs(const LevelDesc& L, const T** m0, const T** m1, const T** m2) const {
        *m0 = tab + L.mw[0];
        *m1 = tab + L.mw[1];
        *m2 = P->dim == 3 ? tab + L.mw[2] : nullptr;
    }

    // one Gauss-Seidel sweep over all colors (forward or backward)
    __device__ void sweep(int l, bool forward) const {
        const LevelDesc& L = P->lev[l];
        const int* p = P->p;
        int nc0 = p[0] + 1, nc1 = p[1] + 1, nc = ieti_ncolors(p);
        const T* vals = K + L.koff;
        T* x = X(l);
        const T* b = B(l);
        const T *m0, *m1, *m2;
        mass_tabs(L, &m0, &m1, &m2);
        for (int cc = 0; cc < nc; ++cc) {
            int c = forward ? cc : nc - 1 - cc;
            int c0 = c % nc0, c1 = (c / nc0) % nc1, c2 = c / (nc0 * nc1);
            int k0 = ieti_cnt(L.m[0], p[0], c0), k1 = ieti_cnt(L.m[1], p[1], c1),
                k2 = ieti_cnt(L.m[2], p[2], c2);
            int off = ieti_color_off(L.m, p, c0, c1, c2);
            int cnt = k0 * k1 * k2;
            for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
                int t0 = t % k0, t1 = (t / k0) % k1, t2 = t / (k0 * k1);
                int i0 = c0 + nc0 * t0, i1 = c1 + nc1 * t1, i2 = c2 + (p[2] + 1) * t2;
                if (ieti_masked(mask, L.m, i0, i1, i2)) continue;
                T d;
                T ax = row_apply<T, T, T>(vals + (long long)off * L.S, cnt, t, x, L.m, p, i0, i1, i2, m0, m1, m2, alpha, &d);
                int i = i0 + L.m[0] * (i1 + L.m[1] * i2);
                x[i] += (b[i] - ax) / d;
            }
            __syncthreads();
        }
    }

    // r = b - A x on level l (masked rows 0)
    __device__ void residual(int l) const {
        const LevelDesc& L = P->lev[l];
        const int* p = P->p;
        int nc0 = p[0] + 1, nc1 = p[1] + 1, nc = ieti_ncolors(p);
        const T* vals = K + L.koff;
        const T* x = X(l);
        const T* b = B(l);
        T* r = R(l);
        const T *m0, *m1, *m2;
        mass_tabs(L, &m0, &m1, &m2);
        for (int c = 0; c < nc; ++c) {
            int c0 = c % nc0, c1 = (c / nc0) % nc1, c2 = c / (nc0 * nc1);
            int k0 = ieti_cnt(L.m[0], p[0], c0), k1 = ieti_cnt(L.m[1], p[1], c1),
                k2 = ieti_cnt(L.m[2], p[2], c2);
            int off = ieti_color_off(L.m, p, c0, c1, c2);
            int cnt = k0 * k1 * k2;
            for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
                int t0 = t % k0, t1 = (t / k0) % k1, t2 = t / (k0 * k1);
                int i0 = c0 + nc0 * t0, i1 = c1 + nc1 * t1, i2 = c2 + (p[2] + 1) * t2;
                int i = i0 + L.m[0] * (i1 + L.m[1] * i2);
                if (ieti_masked(mask, L.m, i0, i1, i2)) {
                    r[i] = 0;
                    continue;
                }
                T ax = row_apply<T, T, T>(vals + (long long)off * L.S, cnt, t, x, L.m, p, i0, i1, i2, m0, m1, m2, alpha,
                                          (T*)nullptr);
                r[i] = b[i] - ax;
            }
        }
        __syncthreads();
    }

    // b_{l-1} = P^T r_l, x_{l-1} = 0
    __device__ void restrict_to(int l) const {
        const LevelDesc& F = P->lev[l];
        const LevelDesc& C = P->lev[l - 1];
        const T* r = R(l);
        T* bc = B(l - 1);
        T* xc = X(l - 1);
        int W0 = P->p[0] + 2, W1 = P->p[1] + 2, W2 = P->dim == 3 ? P->p[2] + 2 : 1;
        for (int I = threadIdx.x; I < C.n; I += blockDim.x) {
            int I0 = I % C.m[0], I1 = (I / C.m[0]) % C.m[1], I2 = I / (C.m[0] * C.m[1]);
            xc[I] = 0;
            if (ieti_masked(mask, C.m, I0, I1, I2)) {
                bc[I] = 0;
                continue;
            }
            int a0 = itab[F.rs[0] + I0], a1 = itab[F.rs[1] + I1], a2 = P->dim == 3 ? itab[F.rs[2] + I2] : 0;
            const T* w0 = tab + F.rw[0] + I0 * W0;
            const T* w1 = tab + F.rw[1] + I1 * W1;
            const T* w2 = P->dim == 3 ? tab + F.rw[2] + I2 * W2 : nullptr;
            T acc = 0;
            for (int u2 = 0; u2 < W2; ++u2) {
                int f2 = a2 + u2;
                if (f2 >= F.m[2]) break;
                T ww2 = w2 ? w2[u2] : T(1);
                if (ww2 == T(0)) continue;
                for (int u1 = 0; u1 < W1; ++u1) {
                    int f1 = a1 + u1;
                    if (f1 >= F.m[1]) break;
                    T ww1 = w1[u1] * ww2;
                    if (ww1 == T(0)) continue;
                    const T* rr = r + F.m[0] * (f1 + F.m[1] * f2);
                    T s = 0;
                    for (int u0 = 0; u0 < W0; ++u0) {
                        int f0 = a0 + u0;
                        if (f0 >= F.m[0]) break;
                        s += w0[u0] * rr[f0];
                    }
                    acc += ww1 * s;
                }
            }
            bc[I] = acc;
        }
        __syncthreads();
    }

    // x_l += P x_{l-1}
    __device__ void prolong_add(int l) const {
        const LevelDesc& F = P->lev[l];
        const LevelDesc& C = P->lev[l - 1];
        const T* xc = X(l - 1);
        T* x = X(l);
        int W0 = P->p[0] + 2, W1 = P->p[1] + 2, W2 = P->dim == 3 ? P->p[2] + 2 : 1;
        for (int i = threadIdx.x; i < F.n; i += blockDim.x) {
            int i0 = i % F.m[0], i1 = (i / F.m[0]) % F.m[1], i2 = i / (F.m[0] * F.m[1]);
            if (ieti_masked(mask, F.m, i0, i1, i2)) continue;
            int a0 = itab[F.ps[0] + i0], a1 = itab[F.ps[1] + i1], a2 = P->dim == 3 ? itab[F.ps[2] + i2] : 0;
            const T* w0 = tab + F.pw[0] + i0 * W0;
            const T* w1 = tab + F.pw[1] + i1 * W1;
            const T* w2 = P->dim == 3 ? tab + F.pw[2] + i2 * W2 : nullptr;
            T acc = 0;
            for (int u2 = 0; u2 < W2; ++u2) {
                int c2 = a2 + u2;
                if (c2 >= C.m[2]) break;
                T ww2 = w2 ? w2[u2] : T(1);
                if (ww2 == T(0)) continue;
                for (int u1 = 0; u1 < W1; ++u1) {
                    int c1 = a1 + u1;
                    if (c1 >= C.m[1]) break;
                    T ww1 = w1[u1] * ww2;
                    if (ww1 == T(0)) continue;
                    const T* xx = xc + C.m[0] * (c1 + C.m[1] * c2);
                    T s = 0;
                    for (int u0 = 0; u0 < W0; ++u0) {
                        int cc0 = a0 + u0;
                        if (cc0 >= C.m[0]) break;
                        s += w0[u0] * xx[cc0];
                    }
                    acc += ww1 * s;
                }
            }
            x[i] += acc;
        }
        __syncthreads();
    }

    __device__ void coarsest() const {
        const LevelDesc& L = P->lev[0];
        int n = L.n;
        const T* b = B(0);
        T* x = X(0);
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            T acc = 0;
            for (int j = 0; j < n; ++j) acc += A0inv[(long long)j * n + i] * b[j];
            x[i] = acc;
        }
        __syncthreads();
    }

    // x_fine = V(b_fine), with b already in B(L-1)
    __device__ void run(int nu1, int nu2) const {
        int L = P->L;
        if (L == 1) {
            coarsest();
            return;
        }
        {
            T* x = X(L - 1);
            for (int i = threadIdx.x; i < P->lev[L - 1].n; i += blockDim.x) x[i] = 0;
            __syncthreads();
        }
        for (int l = L - 1; l >= 1; --l) {
            for (int s = 0; s < nu1; ++s) sweep(l, true);
            residual(l);
            restrict_to(l);   // also zeroes x_{l-1}
        }
        coarsest();
        for (int l = 1; l <= L - 1; ++l) {
            prolong_add(l);
            for (int s = 0; s < nu2; ++s) sweep(l, false);
        }
    }
};

// FP64 SpMV of the fine stiffness for one row: natural index i
__device__ __forceinline__ double k64_row(const PatchDesc& P, const double* K64, const double* x, int i) {
    const LevelDesc& L = P.lev[P.L - 1];
    int i0 = i % L.m[0], i1 = (i / L.m[0]) % L.m[1], i2 = i / (L.m[0] * L.m[1]);
    int c0 = i0 % (P.p[0] + 1), c1 = i1 % (P.p[1] + 1), c2 = i2 % (P.p[2] + 1);
    int k0 = ieti_cnt(L.m[0], P.p[0], c0), k1 = ieti_cnt(L.m[1], P.p[1], c1), k2 = ieti_cnt(L.m[2], P.p[2], c2);
    int q = i0 / (P.p[0] + 1) + k0 * (i1 / (P.p[1] + 1) + k1 * (i2 / (P.p[2] + 1)));
    return row_apply<double, double, double>(K64 + L.koff + (long long)ieti_color_off(L.m, P.p, c0, c1, c2) * L.S,
                                             k0 * k1 * k2, q, x, L.m, P.p, i0, i1, i2, nullptr, nullptr,
                                             nullptr, 0.0, (double*)nullptr);
}

struct Slot {
    const PatchDesc* P;
    int n;
    double *x, *r, *z, *p, *q;
};

// out = in x_r W along direction r of a tensor with extents din (first
// direction fastest): out[.., a, ..] = sum_b W(a, b) in[.., b, ..] with
// W(a, b) = W[b + ldW a] (trans) or W[a + ldW b]; direction r gets extent nout
template <typename T>
__device__ void mode_prod(const T* in, T* out, const int* din, int r, int nout, const T* W, int ldW, bool trans) {
    int dout[3] = {din[0], din[1], din[2]};
    dout[r] = nout;
    const int total = dout[0] * dout[1] * dout[2];
    const int sin = r == 0 ? 1 : (r == 1 ? din[0] : din[0] * din[1]);
    const int nin = din[r];
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int i0 = idx % dout[0], rem = idx / dout[0], i1 = rem % dout[1], i2 = rem / dout[1];
        const int a = r == 0 ? i0 : (r == 1 ? i1 : i2);
        const T* line = in + (r == 0 ? 0 : i0) + din[0] * ((r == 1 ? 0 : i1) + din[1] * (r == 2 ? 0 : i2));
        T acc = 0;
        if (trans)
            for (int b = 0; b < nin; ++b) acc += W[b + (long long)ldW * a] * line[(long long)b * sin];
        else
            for (int b = 0; b < nin; ++b) acc += W[a + (long long)ldW * b] * line[(long long)b * sin];
        out[idx] = acc;
    }
    __syncthreads();
}

// the free sub-grid (first index lo_r, extent n_r per direction) of a full
// natural grid with extents m: gather into a tensor / add a tensor back
template <typename T>
__device__ void free_gather(const T* full, const int* m, const int* lo, const int* n, T* t) {
    const int total = n[0] * n[1] * n[2];
    for (int j = threadIdx.x; j < total; j += blockDim.x) {
        const int j0 = j % n[0], rem = j / n[0], j1 = rem % n[1], j2 = rem / n[1];
        t[j] = full[(j0 + lo[0]) + m[0] * ((j1 + lo[1]) + m[1] * (j2 + lo[2]))];
    }
    __syncthreads();
}
template <typename T>
__device__ void free_add(T* full, const int* m, const int* lo, const int* n, const T* t) {
    const int total = n[0] * n[1] * n[2];
    for (int j = threadIdx.x; j < total; j += blockDim.x) {
        const int j0 = j % n[0], rem = j / n[0], j1 = rem % n[1], j2 = rem / n[1];
        full[(j0 + lo[0]) + m[0] * ((j1 + lo[1]) + m[1] * (j2 + lo[2]))] += t[j];
    }
    __syncthreads();
}

// x_fine += L^-1 r_fine: fast diagonalization of the Kronecker-sum smoother
// of the finest level (U^T along every direction, scaling, U back)
template <typename T>
__device__ void ho_smooth(const VCycle<T>& vc) {
    const HoDesc& H = *vc.ho;
    const int kd = vc.hkind, d = vc.P->dim;
    const LevelDesc& F = vc.P->lev[vc.P->L - 1];
    int dims[3] = {H.nf[kd][0], H.nf[kd][1], H.nf[kd][2]};
    free_gather(vc.R(vc.P->L - 1), F.m, H.lof[kd], dims, vc.t1);
    T* cur = vc.t1;
    T* oth = vc.t2;
    for (int r = 0; r < d; ++r) {
        mode_prod(cur, oth, dims, r, dims[r], vc.hpool + H.u[kd][r], dims[r], true);
        T* t = cur;
        cur = oth;
        oth = t;
    }
    const T* Dinv = vc.hpool + H.dinv[kd];
    for (int j = threadIdx.x; j < dims[0] * dims[1] * dims[2]; j += blockDim.x) cur[j] *= Dinv[j];
    __syncthreads();
    for (int r = 0; r < d; ++r) {
        mode_prod(cur, oth, dims, r, dims[r], vc.hpool + H.u[kd][r], dims[r], false);
        T* t = cur;
        cur = oth;
        oth = t;
    }
    free_add(vc.X(vc.P->L - 1), F.m, H.lof[kd], dims, cur);
}

// high-order V-cycle: smoothing on the finest level, L2-projection transfer
// to the degree-1 hierarchy and its standard V-cycle, back, smoothing
template <typename T>
__device__ void ho_run(const VCycle<T>& vc, int nu1, int nu2) {
    HO_DECL();
    const HoDesc& H = *vc.ho;
    const int kd = vc.hkind, d = vc.P->dim, L = vc.P->L;
    const LevelDesc& F = vc.P->lev[L - 1];
    T* x = vc.X(L - 1);
    for (int i = threadIdx.x; i < F.n; i += blockDim.x) x[i] = 0;
    __syncthreads();
    for (int s = 0; s < nu1; ++s) {
        {
            HO_T0();
            vc.residual(L - 1);
            HO_T1(vc.phase, 52);
        }
        HO_T0();
        ho_smooth(vc);
        HO_T1(vc.phase, 53);
    }
    {
        HO_T0();
        vc.residual(L - 1);
        HO_T1(vc.phase, 52);
    }
    HO_T0();
    // restriction P^T r into the right-hand side of the degree-1 hierarchy
    const VCycle<T>& cv = *vc.coarse;
    const int Lc = cv.P->L;
    const LevelDesc& Cf = cv.P->lev[Lc - 1];
    int dims[3] = {H.nf[kd][0], H.nf[kd][1], H.nf[kd][2]};
    free_gather(vc.R(L - 1), F.m, H.lof[kd], dims, vc.t1);
    T* cur = vc.t1;
    T* oth = vc.t2;
    for (int r = 0; r < d; ++r) {
        mode_prod(cur, oth, dims, r, H.nc[kd][r], vc.hpool + H.pt[kd][r], H.nf[kd][r], true);
        dims[r] = H.nc[kd][r];
        T* t = cur;
        cur = oth;
        oth = t;
    }
    T* bc = cv.B(Lc - 1);
    for (int i = threadIdx.x; i < Cf.n; i += blockDim.x) bc[i] = 0;
    __syncthreads();
    free_add(bc, Cf.m, H.loc[kd], dims, cur);
    HO_T1(vc.phase, 54);
    {
        HO_T0();
        cv.run(2, 2);
        HO_T1(vc.phase, 55);
    }
    HO_T0();
    // prolongation P x_c
    free_gather(cv.X(Lc - 1), Cf.m, H.loc[kd], dims, vc.t1);
    cur = vc.t1;
    oth = vc.t2;
    for (int r = 0; r < d; ++r) {
        mode_prod(cur, oth, dims, r, H.nf[kd][r], vc.hpool + H.pt[kd][r], H.nf[kd][r], false);
        dims[r] = H.nf[kd][r];
        T* t = cur;
        cur = oth;
        oth = t;
    }
    free_add(x, F.m, H.lof[kd], dims, cur);
    HO_T1(vc.phase, 56);
    for (int s = 0; s < nu2; ++s) {
        {
            HO_T0();
            vc.residual(L - 1);
            HO_T1(vc.phase, 52);
        }
        HO_T0();
        ho_smooth(vc);
        HO_T1(vc.phase, 53);
    }
}

// one call per application (not inlined at the nine call sites of the kernel:
// a V-cycle is long enough that the call costs nothing, and inlining both
// hierarchies' V-cycles at every site multiplies the compile time)
template <typename T>
__device__ __noinline__ void vcycle_apply(const VCycle<T>& vc, const double* rin, double* zout, int nu1, int nu2) {
    HO_DECL();
    int L = vc.P->L;
    int n = vc.P->lev[L - 1].n;
    T* b = vc.B(L - 1);
    {
        HO_T0();
        for (int i = threadIdx.x; i < n; i += blockDim.x) b[i] = (T)rin[i];
        __syncthreads();
        HO_T1(vc.phase, 58);
    }
    if (vc.ho)
        ho_run(vc, nu1, nu2);
    else
        vc.run(nu1, nu2);
    const T* x = vc.X(L - 1);
    HO_T0();
    for (int i = threadIdx.x; i < n; i += blockDim.x) zout[i] = (double)x[i];
    __syncthreads();
    HO_T1(vc.phase, 58);
}

// Euclidean projection on ker C for the rows of this patch (rows have
// disjoint supports)
__device__ void project_kerC(const SolveArgs& a, const PatchDesc& P, double* v, double* coef) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = w; j < P.npi; j += nw) {
        int row = P.crow0 + j;
        double d = 0.0, nn = 0.0;
        for (int e = a.crow_ptr[row] + lane; e < a.crow_ptr[row + 1]; e += 32) {
            double ww = a.c_w[e];
            d += ww * v[a.c_idx[e]];
            nn += ww * ww;
        }
        for (int o = 16; o > 0; o >>= 1) {
            d += __shfl_xor_sync(0xffffffffu, d, o);
            nn += __shfl_xor_sync(0xffffffffu, nn, o);
        }
        if (lane == 0) coef[j] = d / nn;
    }
    __syncthreads();
    int e0 = a.crow_ptr[P.crow0], e1 = a.crow_ptr[P.crow0 + P.npi];
    for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        // row of entry e: rows are contiguous, find by scanning (npi small)
        int j = 0;
        while (a.crow_ptr[P.crow0 + j + 1] <= e) ++j;
        v[a.c_idx[e]] -= a.c_w[e] * coef[j];
    }
    __syncthreads();
}

// v <- v - mean(v) over the n entries (one CTA)
__device__ void remove_mean(double* v, int n, Red& red) {
    double s[1] = {0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) s[0] += v[i];
    cta_sum<1>(s, red);
    const double mean = s[0] / n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] -= mean;
    __syncthreads();
}

// C rows of this patch applied to v: coef[j] = c_j . v
__device__ void apply_C(const SolveArgs& a, const PatchDesc& P, const double* v, double* coef) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = w; j < P.npi; j += nw) {
        int row = P.crow0 + j;
        double d = 0.0;
        for (int e = a.crow_ptr[row] + lane; e < a.crow_ptr[row + 1]; e += 32) d += a.c_w[e] * v[a.c_idx[e]];
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) coef[j] = d;
    }
    __syncthreads();
}

template <typename T>
__global__ void __launch_bounds__(512) k_solve(SolveArgs a0) {
    const IetiLaunchSpan span_(a0.tspan);
    __shared__ Red red;
    __shared__ double coef[kMaxRows];
    __shared__ SolveArgs sa;
    const SlotDesc sd = a0.slots[blockIdx.x];
    if (threadIdx.x == 0) {
        sa = a0.batch ? a0.batch[sd.handle] : a0;
        sa.slots = a0.slots;
        sa.nslots = a0.nslots;
        sa.smem_bytes = a0.smem_bytes;
    }
    __syncthreads();
    const SolveArgs& a = sa;
    const PatchDesc& P = a.pd[sd.patch];
    const LevelDesc& F = P.lev[P.L - 1];
    const int n = F.n;
    double* x = a.cg + sd.cg;
    double* r = x + n;
    double* z = r + n;
    double* p = z + n;
    double* q = p + n;
    const int allsides = P.dim == 2 ? 0xF : 0x3F;
    const int kind = (a.mode == MODE_SCHUR || a.mode == MODE_VCYCLE_DIR) ? 1 : 0;

    VCycle<T> vc;
    vc.P = &P;
    vc.mask = kind == 0 ? P.dmask : allsides;
    // floating patches (Neumann hierarchy): the values of K + alpha M^ built
    // at set-up, so that the rows carry no mass terms
    const bool floatN = kind == 0 && P.floating;
    const T* KMv = a.mixed ? (const T*)(const void*)a.KM32 : (const T*)(const void*)a.KM64;
    const bool reg = floatN && KMv != nullptr;
    vc.alpha = (floatN && !reg) ? (T)a.alpha : T(0);
    vc.K = reg ? KMv : (a.mixed ? (const T*)(const void*)a.K32 : (const T*)(const void*)a.K64);
    vc.tab = a.mixed ? (const T*)(const void*)a.tabf : (const T*)(const void*)a.tab;
    vc.itab = a.itab;
    vc.A0inv = (a.mixed ? (const T*)(const void*)a.A0inv32 : (const T*)(const void*)a.A0inv64) + P.a0off[kind];
    vc.lvec = (T*)a.lv + sd.lv;
    vc.nlvec = P.nlvec;
    vc.phase = a.phase;
    // high-order multigrid: the degree-1 hierarchy of the companion problem
    // (same patch index) and the work tensors follow the slot's x | b | r
    VCycle<T> vco;
    if (a.ho) {
        const PatchDesc& Q = a.sub_pd[sd.patch];
        vco.P = &Q;
        vco.mask = vc.mask;
        vco.alpha = floatN ? (T)a.alpha : T(0);
        vco.K = a.mixed ? (const T*)(const void*)a.sub_K32 : (const T*)(const void*)a.sub_K64;
        vco.tab = a.mixed ? (const T*)(const void*)a.sub_tabf : (const T*)(const void*)a.sub_tab;
        vco.itab = a.sub_itab;
        vco.A0inv = (a.mixed ? (const T*)(const void*)a.sub_A0inv32 : (const T*)(const void*)a.sub_A0inv64) +
                    Q.a0off[kind];
        vco.lvec = vc.lvec + 3 * (long long)P.nlvec;
        vco.nlvec = Q.nlvec;
        vc.ho = a.ho + sd.patch;
        vc.hkind = kind;
        vc.hpool = a.mixed ? (const T*)(const void*)a.ho32 : (const T*)(const void*)a.ho64;
        vc.coarse = &vco;
        vc.t1 = vco.lvec + 3 * (long long)Q.nlvec;
        vc.t2 = vc.t1 + n;
    }
    long long vcount = 0;

    if (a.mode == MODE_SCHUR) {
        const double* v = a.in + P.toff;
        // r = -K v on interior rows
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            int i0 = i % F.m[0], i1 = (i / F.m[0]) % F.m[1], i2 = i / (F.m[0] * F.m[1]);
            r[i] = ieti_masked(allsides, F.m, i0, i1, i2) ? 0.0 : -k64_row(P, a.K64, v, i);
        }
        __syncthreads();
        for (int c = 0; c < a.ncycles; ++c) {
            if (c == 0) {
                vcycle_apply(vc, r, x, a.nu1, a.nu2);
            } else {
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    int i0 = i % F.m[0], i1 = (i / F.m[0]) % F.m[1], i2 = i / (F.m[0] * F.m[1]);
                    q[i] = ieti_masked(allsides, F.m, i0, i1, i2) ? 0.0 : r[i] - k64_row(P, a.K64, x, i);
                }
                __syncthreads();
                vcycle_apply(vc, q, z, a.nu1, a.nu2);
                for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] += z[i];
                __syncthreads();
            }
            ++vcount;
        }
        for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = v[i] + x[i];
        __syncthreads();
        double* out = a.out + P.toff;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            int i0 = i % F.m[0], i1 = (i / F.m[0]) % F.m[1], i2 = i / (F.m[0] * F.m[1]);
            bool gam = ieti_on_boundary(F.m, P.dim, i0, i1, i2) && !ieti_masked(P.dmask, F.m, i0, i1, i2);
            out[i] = gam ? k64_row(P, a.K64, p, i) : 0.0;
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
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                int i0 = i % F.m[0], i1 = (i / F.m[0]) % F.m[1], i2 = i / (F.m[0] * F.m[1]);
                out[i] = ieti_masked(P.dmask, F.m, i0, i1, i2) ? 0.0 : k64_row(P, a.K64, in, i);
            }
            __syncthreads();
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

    if (a.mode == MODE_POWER || a.mode == MODE_KHAT) {
        // fine operator of the Neumann hierarchy: K, or K + alpha M^ on
        // floating patches (same layout as K)
        const double* A64 = P.floating ? a.KM64 : a.K64;
        if (a.mode == MODE_POWER) {
            // energy-norm contraction of one V-cycle by power iteration from
            // x_j = ((37 j) mod 101)/101 - 1/2, j the rank among the free dofs
            const int lo0 = P.dmask & 1, lo1 = (P.dmask >> 2) & 1, lo2 = (P.dmask >> 4) & 1;
            const int nf0 = F.m[0] - lo0 - ((P.dmask >> 1) & 1);
            const int nf1 = F.m[1] - lo1 - ((P.dmask >> 3) & 1);
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                int i0 = i % F.m[0], i1 = (i / F.m[0]) % F.m[1], i2 = i / (F.m[0] * F.m[1]);
                if (ieti_masked(P.dmask, F.m, i0, i1, i2)) {
                    x[i] = 0.0;
                } else {
                    const long long j = (i0 - lo0) + (long long)nf0 * ((i1 - lo1) + (long long)nf1 * (i2 - (P.dim == 3 ? lo2 : 0)));
                    x[i] = (double)((37 * j) % 101) / 101.0 - 0.5;
                }
            }
            __syncthreads();
            double rho = 0.0;
            for (int it = 0; it < a.maxit; ++it) {
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    int i0 = i % F.m[0], i1 = (i / F.m[0]) % F.m[1], i2 = i / (F.m[0] * F.m[1]);
                    r[i] = ieti_masked(P.dmask, F.m, i0, i1, i2) ? 0.0 : k64_row(P, A64, x, i);
                }
                __syncthreads();
                vcycle_apply(vc, r, z, a.nu1, a.nu2);
                ++vcount;
                for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = x[i] - z[i];
                __syncthreads();
                double s3[3] = {0.0, 0.0, 0.0};
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    int i0 = i % F.m[0], i1 = (i / F.m[0]) % F.m[1], i2 = i / (F.m[0] * F.m[1]);
                    const double ap = ieti_masked(P.dmask, F.m, i0, i1, i2) ? 0.0 : k64_row(P, A64, p, i);
                    s3[0] += x[i] * r[i];
                    s3[1] += p[i] * ap;
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
            // w = P V^c P^T g / omega_k; rpi_loc holds Phi^T g per constraint row
            const double* g = a.in + P.toff;
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                int i0 = i % F.m[0], i1 = (i / F.m[0]) % F.m[1], i2 = i / (F.m[0] * F.m[1]);
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
                    for (int i = threadIdx.x; i < n; i += blockDim.x) {
                        int i0 = i % F.m[0], i1 = (i / F.m[0]) % F.m[1], i2 = i / (F.m[0] * F.m[1]);
                        q[i] = ieti_masked(P.dmask, F.m, i0, i1, i2) ? 0.0 : r[i] - k64_row(P, A64, x, i);
                    }
                    __syncthreads();
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

    if (a.mode == MODE_VCYCLE || a.mode == MODE_VCYCLE_DIR) {
        HO_DECL();
        const double* bb = a.in + P.toff;
        double* xx = a.out + P.toff;
        const int rmask = kind == 0 ? P.dmask : allsides;
        for (int c = 0; c < a.ncycles; ++c) {
            HO_T0();
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                int i0 = i % F.m[0], i1 = (i / F.m[0]) % F.m[1], i2 = i / (F.m[0] * F.m[1]);
                r[i] = ieti_masked(rmask, F.m, i0, i1, i2) ? 0.0 : bb[i] - k64_row(P, a.K64, xx, i);
            }
            __syncthreads();
            HO_T1(a.phase, 57);
            vcycle_apply(vc, r, z, a.nu1, a.nu2);
            for (int i = threadIdx.x; i < n; i += blockDim.x) xx[i] += z[i];
            __syncthreads();
            ++vcount;
        }
        if (threadIdx.x == 0 && a.vstats) {
            atomicAdd((unsigned long long*)&a.vstats[0], (unsigned long long)vcount);
            atomicAdd((unsigned long long*)&a.vstats[1], (unsigned long long)(vcount * n));
        }
        return;
    }

    const bool basis = a.mode == MODE_BASIS;
    double* phicol = nullptr;
    // ---- right-hand side -------------------------------------------------
    if (basis) {
        int lr = sd.row - P.crow0;
        phicol = a.phi + P.phioff + (long long)lr * n;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            z[i] = 0.0;
            x[i] = 0.0;
        }
        __syncthreads();
        for (int e = a.crow_ptr[sd.row] + threadIdx.x; e < a.crow_ptr[sd.row + 1]; e += blockDim.x)
            z[a.c_idx[e]] = 1.0;   // psi_j: indicator of the constraint's support
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            phicol[i] = z[i];
            int i0 = i % F.m[0], i1 = (i / F.m[0]) % F.m[1], i2 = i / (F.m[0] * F.m[1]);
            r[i] = ieti_masked(P.dmask, F.m, i0, i1, i2) ? 0.0 : -k64_row(P, a.K64, z, i);
        }
        __syncthreads();
        project_kerC(a, P, r, coef);
    } else {
        const double* g = a.in + P.toff;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            int i0 = i % F.m[0], i1 = (i / F.m[0]) % F.m[1], i2 = i / (F.m[0] * F.m[1]);
            r[i] = ieti_masked(P.dmask, F.m, i0, i1, i2) ? 0.0 : g[i];
            x[i] = 0.0;
        }
        __syncthreads();
        // b = P^T g = g - C^T (Phi^T g)
        int e0 = a.crow_ptr[P.crow0], e1 = a.crow_ptr[P.crow0 + P.npi];
        for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
            int j = 0;
            while (a.crow_ptr[P.crow0 + j + 1] <= e) ++j;
            r[a.c_idx[e]] -= a.c_w[e] * a.rpi_loc[P.crow0 + j];
        }
        __syncthreads();
        if (P.floating) {
            double s[1] = {0.0};
            for (int i = threadIdx.x; i < n; i += blockDim.x) s[0] += r[i];
            cta_sum<1>(s, red);
            double mean = s[0] / n;
            for (int i = threadIdx.x; i < n; i += blockDim.x) r[i] -= mean;
            __syncthreads();
        }
    }
    // ---- PCG ---------------------------------------------------------------
    double nb2;
    {
        double s[1] = {0.0};
        for (int i = threadIdx.x; i < n; i += blockDim.x) s[0] += r[i] * r[i];
        cta_sum<1>(s, red);
        nb2 = s[0];
    }
    int it = 0;
    bool conv = nb2 == 0.0;
    double tol2 = a.tol * a.tol * nb2;
    const bool proj1 = !basis && P.floating;   // keep z orthogonal to the constants
    if (!conv) {
        vcycle_apply(vc, r, z, a.nu1, a.nu2);
        ++vcount;
        if (basis) project_kerC(a, P, z, coef);
        if (proj1) remove_mean(z, n, red);
        double rz;
        {
            double s[1] = {0.0};
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                p[i] = z[i];
                s[0] += r[i] * z[i];
            }
            cta_sum<1>(s, red);
            rz = s[0];
        }
        for (it = 1; it <= a.maxit; ++it) {
            {
                double s[1] = {0.0};
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    int i0 = i % F.m[0], i1 = (i / F.m[0]) % F.m[1], i2 = i / (F.m[0] * F.m[1]);
                    double v = ieti_masked(P.dmask, F.m, i0, i1, i2) ? 0.0 : k64_row(P, a.K64, p, i);
                    q[i] = v;
                }
                __syncthreads();
                if (basis) project_kerC(a, P, q, coef);
                for (int i = threadIdx.x; i < n; i += blockDim.x) s[0] += p[i] * q[i];
                cta_sum<1>(s, red);
                double pq = s[0];
                if (!(pq > 0.0) || !isfinite(pq)) {
                    if (threadIdx.x == 0) atomicOr(a.flags, IETI_FLAG_BREAKDOWN);
                    break;
                }
                double alpha = rz / pq;
                double s2[1] = {0.0};
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    x[i] += alpha * p[i];
                    double ri = r[i] - alpha * q[i];
                    r[i] = ri;
                    s2[0] += ri * ri;
                }
                cta_sum<1>(s2, red);
                if (s2[0] <= tol2) {
                    conv = true;
                    break;
                }
                vcycle_apply(vc, r, z, a.nu1, a.nu2);
                ++vcount;
                if (basis) project_kerC(a, P, z, coef);
                if (proj1) remove_mean(z, n, red);
                double s3[2] = {0.0, 0.0};
                for (int i = threadIdx.x; i < n; i += blockDim.x) {
                    s3[0] += r[i] * z[i];
                    s3[1] += q[i] * z[i];
                }
                cta_sum<2>(s3, red);
                double beta;
                if (a.mixed) beta = -alpha * s3[1] / rz;   // flexible (Polak-Ribiere)
                else beta = s3[0] / rz;
                rz = s3[0];
                for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = z[i] + beta * p[i];
                __syncthreads();
            }
        }
        if (!conv && it > a.maxit) it = a.maxit;
    }
    if (threadIdx.x == 0) {
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
    // ---- epilogue ----------------------------------------------------------
    if (basis) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) phicol[i] += x[i];
        return;
    }
    // u = x - Phi (C x - u_Pi)
    apply_C(a, P, x, coef);
    for (int j = threadIdx.x; j < P.npi; j += blockDim.x) coef[j] -= a.upi_loc[P.crow0 + j];
    __syncthreads();
    double* out = a.out + P.toff;
    const double* ph = a.phi + P.phioff;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double u = x[i];
        for (int j = 0; j < P.npi; ++j) u -= coef[j] * ph[(long long)j * n + i];
        out[i] = u;
    }
}

}  // namespace

cudaError_t launch_solve(const SolveArgs& a, int threads, cudaStream_t st) {
    if (a.nslots == 0) return cudaSuccess;
    if (a.mixed) k_solve<float><<<a.nslots, threads, 0, st>>>(a);
    else k_solve<double><<<a.nslots, threads, 0, st>>>(a);
    return cudaGetLastError();
}
