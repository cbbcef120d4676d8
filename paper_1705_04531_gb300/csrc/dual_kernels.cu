// Dual-space and primal-space kernels of IETI-DP (Sec. 2):
//  - the jump operator B, its transpose, and the multiplicity-scaled B_D;
//  - the primal restriction r_Pi = sum_k A^(k)T Phi^(k)T g^(k), the direct
//    coarse solve with S_PiPi (Cholesky factor inverse, Sec. 3.3), and the
//    assembly of S_PiPi = sum_k A^T Phi^T K Phi A;
//  - the scalar steps of the outer CG on F lambda = d (one CTA, FP64).
#include <math.h>
#include "kernels.cuh"

namespace {

template <int K>
__device__ __forceinline__ void cta_sum(double* val, double (*sh)[4]) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k)
        for (int o = 16; o > 0; o >>= 1) val[k] += __shfl_xor_sync(0xffffffffu, val[k], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) sh[w][k] = val[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double s = 0.0;
        for (int i = 0; i < nw; ++i) s += sh[i][k];
        val[k] = s;
    }
    __syncthreads();
}

__global__ void k_bt(DualArgs d, const double* lam, double* torn, int scaled) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d.nie; e += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int t = d.ie_ptr[e]; t < d.ie_ptr[e + 1]; ++t) s += d.ie_sgn[t] * lam[d.ie_lam[t]];
        if (scaled) s /= d.ie_mult[e];
        torn[d.ie_idx[e]] = s;
    }
}

__global__ void k_b(DualArgs d, const double* torn, double* q, int scaled) {
    for (int l = blockIdx.x * blockDim.x + threadIdx.x; l < d.nlam; l += gridDim.x * blockDim.x) {
        double a = torn[d.la[l]], b = torn[d.lb[l]];
        if (scaled) {
            a /= d.ma[l];
            b /= d.mb[l];
        }
        q[l] = a - b;
    }
}

__global__ void k_jump_scale(DualArgs d, const double* torn, double* out) {
    __shared__ double sh[32][4];
    double s[1] = {0.0};
    for (int l = threadIdx.x; l < d.nlam; l += blockDim.x) {
        double a = torn[d.la[l]], b = torn[d.lb[l]];
        s[0] += a * a + b * b;
    }
    cta_sum<1>(s, sh);
    if (threadIdx.x == 0) out[0] = s[0];
}

// r_loc[j] = Phi_j . g over the patch (one CTA per primal row)
__global__ void k_primal_restrict(const PatchDesc* pd, const int* crow_patch, const int* crow_local,
                                  const double* phi, const double* g, double* rloc) {
    __shared__ double sh[32][4];
    int j = blockIdx.x;
    const PatchDesc& P = pd[crow_patch[j]];
    int n = P.n;
    const double* ph = phi + P.phioff + (long long)crow_local[j] * n;
    const double* gg = g + P.toff;
    double s[1] = {0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) s[0] += ph[i] * gg[i];
    cta_sum<1>(s, sh);
    if (threadIdx.x == 0) rloc[j] = s[0];
}

// u_Pi = S^{-1} r_Pi with S = L L^T: y = Linv r, u = Linv^T y.  One CTA.
__global__ void k_coarse_solve(int npi, int nrows, const int* crow_glob, const int* gptr, const int* glist,
                               const double* Linv, const double* rloc, double* upi, double* uloc) {
    extern __shared__ double sm[];
    double* rp = sm;
    double* y = sm + npi;
    for (int J = threadIdx.x; J < npi; J += blockDim.x) {
        double s = 0.0;
        for (int t = gptr[J]; t < gptr[J + 1]; ++t) s += rloc[glist[t]];
        rp[J] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npi; i += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k <= i; ++k) s += Linv[(long long)i * npi + k] * rp[k];
        y[i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < npi; i += blockDim.x) {
        double s = 0.0;
        for (int k = i; k < npi; ++k) s += Linv[(long long)k * npi + i] * y[k];
        upi[i] = s;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nrows; j += blockDim.x) uloc[j] = upi[crow_glob[j]];
}

__device__ __forceinline__ double k64_apply_row(const PatchDesc& P, const double* K64, const double* x, int i) {
    const LevelDesc& L = P.lev[P.L - 1];
    int i0 = i % L.m[0], i1 = (i / L.m[0]) % L.m[1], i2 = i / (L.m[0] * L.m[1]);
    if (ieti_masked(P.dmask, L.m, i0, i1, i2)) return 0.0;
    const double* vals = K64 + L.koff;
    int lo0 = max(-P.p[0], -i0), hi0 = min(P.p[0], L.m[0] - 1 - i0);
    int lo1 = max(-P.p[1], -i1), hi1 = min(P.p[1], L.m[1] - 1 - i1);
    int lo2 = max(-P.p[2], -i2), hi2 = min(P.p[2], L.m[2] - 1 - i2);
    int w0 = 2 * P.p[0] + 1, w1 = 2 * P.p[1] + 1;
    double acc = 0.0;
    for (int o2 = lo2; o2 <= hi2; ++o2)
        for (int o1 = lo1; o1 <= hi1; ++o1) {
            int ob = ((o2 + P.p[2]) * w1 + (o1 + P.p[1])) * w0 + P.p[0];
            int xb = i0 + L.m[0] * ((i1 + o1) + L.m[1] * (i2 + o2));
            for (int o0 = lo0; o0 <= hi0; ++o0)
                acc += vals[ieti_val_pos(L.m, P.p, L.S, i0, i1, i2, ob + o0)] * x[xb + o0];
        }
    return acc;
}

// S_loc(i, j) = phi_i^T K phi_j for the rows of one patch: one CTA per row j
__global__ void k_spp_local(const PatchDesc* pd, const int* crow_patch, const int* crow_local,
                            const double* phi, const double* K64, double* work, long long wstride,
                            double* sloc, const long long* sloc_off) {
    __shared__ double sh[32][4];
    int j = blockIdx.x;
    int k = crow_patch[j];
    const PatchDesc& P = pd[k];
    int n = P.n, lj = crow_local[j];
    const double* ph = phi + P.phioff;
    double* y = work + (long long)blockIdx.x * wstride;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        // Phi is 0 on masked functions; mask the columns too (masked columns
        // of x are zero)
        y[i] = k64_apply_row(P, K64, ph + (long long)lj * n, i);
    }
    __syncthreads();
    for (int li = 0; li < P.npi; ++li) {
        double s[1] = {0.0};
        for (int i = threadIdx.x; i < n; i += blockDim.x) s[0] += ph[(long long)li * n + i] * y[i];
        cta_sum<1>(s, sh);
        if (threadIdx.x == 0) sloc[sloc_off[k] + (long long)li * P.npi + lj] = s[0];
    }
}

// S_PiPi = sum_k A^T S_loc A, patches in order (deterministic)
__global__ void k_spp_assemble(int npatch, const PatchDesc* pd, const int* crow_glob, const double* sloc,
                               const long long* sloc_off, double* S, int npi) {
    for (long long t = threadIdx.x; t < (long long)npi * npi; t += blockDim.x) S[t] = 0.0;
    __syncthreads();
    for (int k = 0; k < npatch; ++k) {
        const PatchDesc& P = pd[k];
        int m = P.npi;
        for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
            int a = t / m, b = t % m;
            int A = crow_glob[P.crow0 + a], B = crow_glob[P.crow0 + b];
            // entries (a,b) of one patch map to distinct (A,B): no conflict
            S[(long long)A * npi + B] += sloc[sloc_off[k] + t];
        }
        __syncthreads();
    }
}

// outer CG state: [0] rz, [1] pq, [2] alpha, [3] beta, [4] rr, [5] dd
__global__ void k_outer_init(int n, const double* d, double* lam, double* r, double* st) {
    __shared__ double sh[32][4];
    double s[1] = {0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        lam[i] = 0.0;
        r[i] = d[i];
        s[0] += d[i] * d[i];
    }
    cta_sum<1>(s, sh);
    if (threadIdx.x == 0) {
        st[5] = s[0];
        st[4] = s[0];
        st[6] = 0.0;   // completed steps (history index of the next one)
    }
}

__global__ void k_outer_first(int n, const double* r, const double* z, double* p, double* st) {
    __shared__ double sh[32][4];
    double s[1] = {0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        p[i] = z[i];
        s[0] += r[i] * z[i];
    }
    cta_sum<1>(s, sh);
    if (threadIdx.x == 0) st[0] = s[0];
}

__global__ void k_outer_step1(int n, const double* p, const double* q, double* lam, double* r, double* st,
                              double* hist, int it) {
    __shared__ double sh[32][4];
    double s[1] = {0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) s[0] += p[i] * q[i];
    cta_sum<1>(s, sh);
    double alpha = st[0] / s[0];
    double s2[1] = {0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        lam[i] += alpha * p[i];
        double ri = r[i] - alpha * q[i];
        r[i] = ri;
        s2[0] += ri * ri;
    }
    cta_sum<1>(s2, sh);
    if (threadIdx.x == 0) {
        // it < 0: the step counter kept in st[6] (replayable launches)
        const int k = it >= 0 ? it : (int)st[6];
        st[1] = s[0];
        st[2] = alpha;
        st[4] = s2[0];
        st[6] = (double)(k + 1);
        hist[2 * k] = alpha;
    }
}

__global__ void k_outer_step2(int n, const double* r, const double* z, double* p, double* st, double* hist,
                              int it) {
    __shared__ double sh[32][4];
    double s[1] = {0.0};
    for (int i = threadIdx.x; i < n; i += blockDim.x) s[0] += r[i] * z[i];
    cta_sum<1>(s, sh);
    double beta = s[0] / st[0];
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = z[i] + beta * p[i];
    __syncthreads();
    if (threadIdx.x == 0) {
        const int k = it >= 0 ? it : (int)st[6] - 1;
        st[0] = s[0];
        st[3] = beta;
        hist[2 * k + 1] = beta;
    }
}

__global__ void k_axpy(long long n, const double* a, double s, const double* b, double* out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = a[i] + s * b[i];
}

// y = K x per patch (fine level, Dirichlet rows zero).  Rows are visited in
// storage order (color by color), so that each stencil diagonal is read with
// unit stride from the color-blocked value array.
__global__ void k_apply_K(const PatchDesc* pd, const double* K64, const double* x, double* y) {
    __shared__ int coff[(IETI_MAXP + 1) * (IETI_MAXP + 1) * (IETI_MAXP + 1) + 1];
    const PatchDesc& P = pd[blockIdx.y];
    const LevelDesc& L = P.lev[P.L - 1];
    const int C0 = P.p[0] + 1, C1 = P.p[1] + 1, C2 = P.p[2] + 1, NC = C0 * C1 * C2;
    const int W0 = 2 * P.p[0] + 1, W1 = 2 * P.p[1] + 1;
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int c = 0; c < NC; ++c) {
            coff[c] = acc;
            acc += ieti_cnt(L.m[0], P.p[0], c % C0) * ieti_cnt(L.m[1], P.p[1], (c / C0) % C1) *
                   ieti_cnt(L.m[2], P.p[2], c / (C0 * C1));
        }
        coff[NC] = acc;
    }
    __syncthreads();
    const double* vals = K64 + L.koff;
    const double* xp = x + P.toff;
    double* yp = y + P.toff;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < L.n; s += gridDim.x * blockDim.x) {
        int lo = 0, hi = NC - 1;   // color: last c with coff[c] <= s
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (coff[mid] <= s) lo = mid;
            else hi = mid - 1;
        }
        const int c = lo, c0 = c % C0, c1 = (c / C0) % C1, c2 = c / (C0 * C1);
        const int k0 = ieti_cnt(L.m[0], P.p[0], c0), k1 = ieti_cnt(L.m[1], P.p[1], c1);
        const int cnt = coff[c + 1] - coff[c];
        const int q = s - coff[c];
        const int t0 = q % k0, tr = q / k0, t1 = tr % k1, t2 = tr / k1;
        const int i0 = c0 + C0 * t0, i1 = c1 + C1 * t1, i2 = c2 + C2 * t2;
        const int i = i0 + L.m[0] * (i1 + L.m[1] * i2);
        if (ieti_masked(P.dmask, L.m, i0, i1, i2)) {
            yp[i] = 0.0;
            continue;
        }
        const double* v = vals + (long long)coff[c] * L.S + q;
        double acc = 0.0;
        int o = 0;
        for (int o2 = -P.p[2]; o2 <= P.p[2]; ++o2) {
            const bool ok2 = (unsigned)(i2 + o2) < (unsigned)L.m[2];
            for (int o1 = -P.p[1]; o1 <= P.p[1]; ++o1) {
                const bool ok1 = ok2 && (unsigned)(i1 + o1) < (unsigned)L.m[1];
                const int xb = i0 + L.m[0] * ((i1 + o1) + L.m[1] * (i2 + o2));
                for (int o0 = -P.p[0]; o0 <= P.p[0]; ++o0, ++o) {
                    if (ok1 && (unsigned)(i0 + o0) < (unsigned)L.m[0]) acc += v[(long long)o * cnt] * xp[xb + o0];
                }
            }
        }
        (void)W0;
        (void)W1;
        yp[i] = acc;
    }
}

int grid_for(long long n, int threads, int cap = 152 * 16) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

}  // namespace

cudaError_t launch_bt(const DualArgs& d, const double* lam, double* torn, int scaled, cudaStream_t st) {
    if (d.nie == 0) return cudaSuccess;
    k_bt<<<grid_for(d.nie, 256), 256, 0, st>>>(d, lam, torn, scaled);
    return cudaGetLastError();
}

cudaError_t launch_b(const DualArgs& d, const double* torn, double* q, int scaled, cudaStream_t st) {
    if (d.nlam == 0) return cudaSuccess;
    k_b<<<grid_for(d.nlam, 256), 256, 0, st>>>(d, torn, q, scaled);
    return cudaGetLastError();
}

cudaError_t launch_jump_scale(const DualArgs& d, const double* torn, double* out, cudaStream_t st) {
    k_jump_scale<<<1, 1024, 0, st>>>(d, torn, out);
    return cudaGetLastError();
}

cudaError_t launch_primal_restrict(const PatchDesc* pd, int nrows, const int* crow_patch, const int* crow_local,
                                   const double* phi, const double* g, double* rloc, cudaStream_t st) {
    if (nrows == 0) return cudaSuccess;
    k_primal_restrict<<<nrows, 256, 0, st>>>(pd, crow_patch, crow_local, phi, g, rloc);
    return cudaGetLastError();
}

cudaError_t launch_coarse_solve(int npi, int nrows, const int* crow_glob, const int* gptr, const int* glist,
                                const double* Linv, const double* rloc, double* upi, double* uloc,
                                cudaStream_t st) {
    if (npi == 0) return cudaSuccess;
    size_t sm = sizeof(double) * 2 * npi;
    k_coarse_solve<<<1, 512, sm, st>>>(npi, nrows, crow_glob, gptr, glist, Linv, rloc, upi, uloc);
    return cudaGetLastError();
}

cudaError_t launch_spp_local(const PatchDesc* pd, int nrows, const int* crow_patch, const int* crow_local,
                             const double* phi, const double* K64, double* work, long long wstride, double* sloc,
                             const long long* sloc_off, cudaStream_t st) {
    if (nrows == 0) return cudaSuccess;
    k_spp_local<<<nrows, 256, 0, st>>>(pd, crow_patch, crow_local, phi, K64, work, wstride, sloc, sloc_off);
    return cudaGetLastError();
}

cudaError_t launch_spp_assemble(int npatch, const PatchDesc* pd, const int* crow_glob, const double* sloc,
                                const long long* sloc_off, double* S, int npi, cudaStream_t st) {
    if (npi == 0) return cudaSuccess;
    k_spp_assemble<<<1, 512, 0, st>>>(npatch, pd, crow_glob, sloc, sloc_off, S, npi);
    return cudaGetLastError();
}

cudaError_t launch_outer_init(int n, const double* d, double* lam, double* r, double* state, cudaStream_t st) {
    k_outer_init<<<1, 1024, 0, st>>>(n, d, lam, r, state);
    return cudaGetLastError();
}
cudaError_t launch_outer_first(int n, const double* r, const double* z, double* p, double* state,
                               cudaStream_t st) {
    k_outer_first<<<1, 1024, 0, st>>>(n, r, z, p, state);
    return cudaGetLastError();
}
cudaError_t launch_outer_step1(int n, const double* p, const double* q, double* lam, double* r, double* state,
                               double* hist, int it, cudaStream_t st) {
    k_outer_step1<<<1, 1024, 0, st>>>(n, p, q, lam, r, state, hist, it);
    return cudaGetLastError();
}
cudaError_t launch_outer_step2(int n, const double* r, const double* z, double* p, double* state, double* hist,
                               int it, cudaStream_t st) {
    k_outer_step2<<<1, 1024, 0, st>>>(n, r, z, p, state, hist, it);
    return cudaGetLastError();
}
cudaError_t launch_axpy_torn(long long n, const double* a, double s, const double* b, double* out,
                             cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_axpy<<<grid_for(n, 256), 256, 0, st>>>(n, a, s, b, out);
    return cudaGetLastError();
}
cudaError_t launch_apply_K(const PatchDesc* pd, int npatch, const double* K64, const double* x, double* y,
                           cudaStream_t st) {
    k_apply_K<<<dim3(32, npatch), 256, 0, st>>>(pd, K64, x, y);
    return cudaGetLastError();
}
