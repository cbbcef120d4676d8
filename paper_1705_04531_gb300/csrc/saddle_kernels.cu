// Vector kernels of the MG-MG-S variant: Bramble-Pasciak CG on the saddle-
// point system of Eq. 2 (K~ u + B~^T lambda = f~, B~ u = 0).
//
// A vector of V~ is stored as one FP64 array of n_torn + n_Pi entries: the
// Delta parts w^(k) in ker C^(k) (patch layout, full tensor grids) followed
// by the global primal coefficients u_Pi; the function it represents is
// u^(k) = Phi^(k) A^(k) u_Pi + w^(k).  The scalars of the iteration stay on
// the device; coefficients are read there as ratios of device scalars.
#include <cuda_runtime.h>

#include "saddle.cuh"

namespace {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// y = scale * S x, S dense row-major n x n (one warp per row)
__global__ void k_sp_matvec(int n, const double* S, const double* x, double* y, double scale) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n) return;
    double s = 0.0;
    for (int k = lane; k < n; k += 32) s += S[(long long)row * n + k] * x[k];
    s = warp_sum(s);
    if (lane == 0) y[row] = scale * s;
}

// y = scale * S^{-1} x with S = L L^T given by Linv = L^{-1} (row-major): one CTA
__global__ void k_spp_solve(int n, const double* Linv, const double* x, double* y, double scale) {
    extern __shared__ double sm[];
    double* xs = sm;
    double* t = sm + n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] = x[i];
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double s = 0.0;
        for (int k = 0; k <= i; ++k) s += Linv[(long long)i * n + k] * xs[k];
        t[i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double s = 0.0;
        for (int k = i; k < n; ++k) s += Linv[(long long)k * n + i] * t[k];
        y[i] = scale * s;
    }
}

// out[J] (+)= sum of the per-row restrictions rloc over the rows of global
// primal dof J
__global__ void k_primal_assemble(int npi, const int* gptr, const int* glist, const double* rloc, double* out,
                                  int accumulate) {
    for (int J = blockIdx.x * blockDim.x + threadIdx.x; J < npi; J += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int t = gptr[J]; t < gptr[J + 1]; ++t) s += rloc[glist[t]];
        out[J] = accumulate ? out[J] + s : s;
    }
}

// Euclidean projection on ker C^(k): y <- y - sum_j (c_j.y / c_j.c_j) c_j,
// one warp per constraint row (rows of one patch have disjoint supports)
__global__ void k_project_kerC(int nrows, const PatchDesc* pd, const int* crow_patch, const int* crow_ptr,
                               const int* c_idx, const double* c_w, double* y) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= nrows) return;
    double* v = y + pd[crow_patch[row]].toff;
    double d = 0.0, nn = 0.0;
    for (int e = crow_ptr[row] + lane; e < crow_ptr[row + 1]; e += 32) {
        const double w = c_w[e];
        d += w * v[c_idx[e]];
        nn += w * w;
    }
    d = warp_sum(d);
    nn = warp_sum(nn);
    const double c = nn > 0.0 ? d / nn : 0.0;
    for (int e = crow_ptr[row] + lane; e < crow_ptr[row + 1]; e += 32) v[c_idx[e]] -= c_w[e] * c;
}

// out^(k) = w^(k) + sum_j Phi^(k)_j u_Pi[A^(k)(j)]; blockIdx.y = patch
__global__ void k_function(const PatchDesc* pd, const int* crow_glob, const double* phi, const double* uP,
                           const double* w, double* out) {
    const PatchDesc& P = pd[blockIdx.y];
    const int n = P.n;
    const double* ph = phi + P.phioff;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s = w[P.toff + i];
        for (int j = 0; j < P.npi; ++j) s += ph[(long long)j * n + i] * uP[crow_glob[P.crow0 + j]];
        out[P.toff + i] = s;
    }
}

__device__ __forceinline__ double coef_of(const SaddleCoef& c) {
    double v = c.num ? *c.num : 1.0;
    if (c.den) v = *c.den != 0.0 ? v / *c.den : 0.0;
    return c.sign * v;
}

// several updates with one coefficient c: mode 0 y = x + c y, mode 1 y += c x,
// mode 2 y = x (copy), mode 3 y = x - y
__global__ void k_lin(SaddleLin L) {
    const double c = coef_of(L.c);
    long long total = 0;
    for (int k = 0; k < L.njobs; ++k) total += L.n[k];
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        long long i = t;
        int k = 0;
        while (i >= L.n[k]) {
            i -= L.n[k];
            ++k;
        }
        double* y = L.y[k];
        const double x = L.x[k] ? L.x[k][i] : 0.0;
        switch (L.mode[k]) {
            case 0: y[i] = x + c * y[i]; break;
            case 1: y[i] += c * x; break;
            case 2: y[i] = x; break;
            default: y[i] = x - y[i]; break;
        }
    }
}

// sum_k a_k . b_k: per-CTA partial sums (fixed grid, deterministic order)
constexpr int kDotGrid = 256;
__global__ void k_dot_partial(SaddleDot D, double* partial) {
    __shared__ double sh[32];
    long long total = 0;
    for (int k = 0; k < D.njobs; ++k) total += D.n[k];
    double s = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        long long i = t;
        int k = 0;
        while (i >= D.n[k]) {
            i -= D.n[k];
            ++k;
        }
        s += D.a[k][i] * D.b[k][i];
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) partial[blockIdx.x] = v;
    }
}

__global__ void k_dot_final(const double* partial, int n, double* out, double* copy_to) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += partial[i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        v = warp_sum(v);
        if (threadIdx.x == 0) {
            *out = v;
            if (copy_to) *copy_to = v;
        }
    }
}

__global__ void k_copy_scalar(const double* src, double* dst) { *dst = *src; }

}  // namespace

cudaError_t launch_sp_matvec(int n, const double* S, const double* x, double* y, double scale, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_sp_matvec<<<(n + 7) / 8, 256, 0, st>>>(n, S, x, y, scale);
    return cudaGetLastError();
}

cudaError_t launch_spp_solve(int n, const double* Linv, const double* x, double* y, double scale, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_spp_solve<<<1, 512, sizeof(double) * 2 * n, st>>>(n, Linv, x, y, scale);
    return cudaGetLastError();
}

cudaError_t launch_primal_assemble(int npi, const int* gptr, const int* glist, const double* rloc, double* out,
                                   int accumulate, cudaStream_t st) {
    if (npi == 0) return cudaSuccess;
    k_primal_assemble<<<(npi + 255) / 256, 256, 0, st>>>(npi, gptr, glist, rloc, out, accumulate);
    return cudaGetLastError();
}

cudaError_t launch_project_kerC(int nrows, const PatchDesc* pd, const int* crow_patch, const int* crow_ptr,
                                const int* c_idx, const double* c_w, double* y, cudaStream_t st) {
    if (nrows == 0) return cudaSuccess;
    k_project_kerC<<<(nrows + 7) / 8, 256, 0, st>>>(nrows, pd, crow_patch, crow_ptr, c_idx, c_w, y);
    return cudaGetLastError();
}

cudaError_t launch_function(int npatch, const PatchDesc* pd, const int* crow_glob, const double* phi,
                            const double* uP, const double* w, double* out, cudaStream_t st) {
    k_function<<<dim3(32, npatch), 256, 0, st>>>(pd, crow_glob, phi, uP, w, out);
    return cudaGetLastError();
}

cudaError_t launch_lin(const SaddleLin& L, cudaStream_t st) {
    if (L.njobs == 0) return cudaSuccess;
    k_lin<<<1216, 256, 0, st>>>(L);
    return cudaGetLastError();
}

cudaError_t launch_dot(const SaddleDot& D, double* partial, double* out, double* copy_to, cudaStream_t st) {
    k_dot_partial<<<kDotGrid, 256, 0, st>>>(D, partial);
    k_dot_final<<<1, 256, 0, st>>>(partial, kDotGrid, out, copy_to);
    return cudaGetLastError();
}

cudaError_t launch_copy_scalar(const double* src, double* dst, cudaStream_t st) {
    k_copy_scalar<<<1, 1, 0, st>>>(src, dst);
    return cudaGetLastError();
}
