// Primal basis by Schoeberl-Zulehner preconditioned CG (Sec. 3.2), device
// side, shared by the specialised and the run-time-degree local solver
// kernels (one CTA per primal row j of a patch).
//
// Eq. 6:  [K C^T; C 0] (phi_j, mu_j) = (0, e_j).  Preconditioner blocks:
// Khat^{-1} = 0.99 V (one V-cycle on K, or K + alpha M^ on floating patches),
// Hhat = 0.99 H with H = C Khat^{-1} C^T; W = Khat^{-1} C^T and Hhat^{-1} are
// precomputed per patch (modes SZW and the per-patch inverse kernel).  CG runs
// in the inner product of D = P - [K C^T; C 0], positive definite when
// Khat > K and Hhat < C Khat^{-1} C^T; <r, r>_D = r.rt - r.(A r) with rt the
// unpreconditioned residual.  One V-cycle and one K product per step.  The
// iteration restarts from the FP64 residual after every 1e-4 of reduction
// (the recursions drift by the rounding of the preconditioner).
#pragma once
#include "kernels.cuh"

namespace ieti_sz {

constexpr double kKhatScale = 0.99;
constexpr int kSmall = 64;   // max constraint rows of one patch (small vectors)

// sum over the CTA of two partial values (sh: 64 doubles of shared memory)
__device__ inline void sum2(double& a, double& b, double* sh) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) {
        sh[w] = a;
        sh[32 + w] = b;
    }
    __syncthreads();
    a = 0.0;
    b = 0.0;
    for (int i = 0; i < nw; ++i) {
        a += sh[i];
        b += sh[32 + i];
    }
    __syncthreads();
}

// out[c] = (C v)_c for the rows of the patch (out: shared or global)
__device__ inline void apply_C(const SolveArgs& a, const PatchDesc& P, const double* v, double* out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = w; j < P.npi; j += nw) {
        const int row = P.crow0 + j;
        double d = 0.0;
        for (int e = a.crow_ptr[row] + lane; e < a.crow_ptr[row + 1]; e += 32) d += a.c_w[e] * v[a.c_idx[e]];
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) out[j] = d;
    }
    __syncthreads();
}

// SZW mode: W_j = 0.99 V(c_j), the preconditioner applied to constraint row j
template <class VCyc>
__device__ void szw_slot(const SolveArgs& a, const PatchDesc& P, const SlotDesc& sd, double* base, VCyc vcyc) {
    const int n = P.lev[P.L - 1].n;
    double* cj = base;
    double* w = base + n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) cj[i] = 0.0;
    __syncthreads();
    for (int e = a.crow_ptr[sd.row] + threadIdx.x; e < a.crow_ptr[sd.row + 1]; e += blockDim.x)
        cj[a.c_idx[e]] = a.c_w[e];
    __syncthreads();
    vcyc(cj, w);
    double* Wj = a.szW + P.phioff + (long long)(sd.row - P.crow0) * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) Wj[i] = kKhatScale * w[i];
}

// SZ-CG for phi_j; returns the iteration count, *conv whether it converged.
// base: 8 n + 8 kSmall doubles of the slot; red: 64 doubles of shared memory;
// coef: kSmall doubles of shared memory.
template <class VCyc, class SpmvK>
__device__ int sz_basis_slot(const SolveArgs& a, const PatchDesc& P, const SlotDesc& sd, double* base, double* red,
                             double* coef, VCyc vcyc, SpmvK spmvK, bool* conv) {
    const int n = P.lev[P.L - 1].n;
    const int npi = P.npi;
    const int jrow = sd.row - P.crow0;
    double* x1 = base;
    double* rt1 = base + n;
    double* r1 = base + 2 * (long long)n;
    double* p1 = base + 3 * (long long)n;
    double* Ap1 = base + 4 * (long long)n;
    double* Ar1 = base + 5 * (long long)n;
    double* q1 = base + 6 * (long long)n;
    double* t1 = base + 7 * (long long)n;
    double* sm = base + 8 * (long long)n;
    double* x2 = sm;
    double* rt2 = sm + kSmall;
    double* r2 = sm + 2 * kSmall;
    double* p2 = sm + 3 * kSmall;
    double* Ap2 = sm + 4 * kSmall;
    double* Ar2 = sm + 5 * kSmall;
    double* q2 = sm + 6 * kSmall;
    double* t2 = sm + 7 * kSmall;
    const double* Wp = a.szW + P.phioff;
    const double* Hi = a.szHinv + P.szhoff;

    // z = P^{-1} y (z1 may alias nothing of y); y1 == nullptr means y1 = 0
    auto precond = [&](const double* y1, const double* y2, double* z1, double* z2) {
        if (y1) {
            vcyc(y1, t1);
            for (int i = threadIdx.x; i < n; i += blockDim.x) t1[i] *= kKhatScale;
            __syncthreads();
            apply_C(a, P, t1, coef);
        } else {
            for (int i = threadIdx.x; i < n; i += blockDim.x) t1[i] = 0.0;
            for (int c = threadIdx.x; c < npi; c += blockDim.x) coef[c] = 0.0;
            __syncthreads();
        }
        for (int c = threadIdx.x; c < npi; c += blockDim.x) t2[c] = coef[c] - y2[c];
        __syncthreads();
        for (int c = threadIdx.x; c < npi; c += blockDim.x) {
            double s = 0.0;
            for (int k = 0; k < npi; ++k) s += Hi[c * npi + k] * t2[k];
            z2[c] = s;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            double s = t1[i];
            for (int c = 0; c < npi; ++c) s -= Wp[(long long)c * n + i] * z2[c];
            z1[i] = s;
        }
        __syncthreads();
    };
    // (o1, o2) = [K C^T; C 0] (y1, y2)
    auto saddle = [&](const double* y1, const double* y2, double* o1, double* o2) {
        spmvK(y1, o1);
        {
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
            for (int c = w; c < npi; c += nw) {
                const int row = P.crow0 + c;
                const double yc = y2[c];
                for (int e = a.crow_ptr[row] + lane; e < a.crow_ptr[row + 1]; e += 32) o1[a.c_idx[e]] += a.c_w[e] * yc;
            }
        }
        __syncthreads();
        apply_C(a, P, y1, o2);
    };
    // u1.v1 + u2.v2 and s1.w1 + s2.w2 in one reduction
    auto dots = [&](const double* u1, const double* v1, const double* u2, const double* v2, const double* s1,
                    const double* w1, const double* s2, const double* w2, double& d0, double& d1) {
        double a0 = 0.0, b0 = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            a0 += u1[i] * v1[i];
            b0 += s1[i] * w1[i];
        }
        for (int c = threadIdx.x; c < npi; c += blockDim.x) {
            a0 += u2[c] * v2[c];
            b0 += s2[c] * w2[c];
        }
        sum2(a0, b0, red);
        d0 = a0;
        d1 = b0;
    };

    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        x1[i] = 0.0;
        rt1[i] = 0.0;
    }
    for (int c = threadIdx.x; c < kSmall; c += blockDim.x) {
        x2[c] = 0.0;
        rt2[c] = c == jrow ? 1.0 : 0.0;
    }
    __syncthreads();
    precond(nullptr, rt2, r1, r2);
    saddle(r1, r2, Ar1, Ar2);
    double rr, rAr;
    dots(r1, rt1, r2, rt2, r1, Ar1, r2, Ar2, rr, rAr);
    double rho = rr - rAr;
    const double rho0 = rho;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        p1[i] = r1[i];
        Ap1[i] = Ar1[i];
    }
    for (int c = threadIdx.x; c < npi; c += blockDim.x) {
        p2[c] = r2[c];
        Ap2[c] = Ar2[c];
    }
    __syncthreads();
    *conv = !(rho0 > 0.0);
    int it = 0;
    const double tol2 = a.tol * a.tol;
    // the recursively updated residuals drift by the rounding of the
    // preconditioner (FP32 V-cycles, and the cancellation in
    // r.rt - r.(A r) in FP64 at tol_basis = 1e-12), so the iteration restarts
    // from the FP64 residual b - A x after every 1e-4 of reduction
    double rho_cycle = rho0;
    int restarts = 0;
    while (!*conv && it < a.maxit) {
        ++it;
        precond(Ap1, Ap2, q1, q2);
        double pAp, qAp;
        dots(p1, Ap1, p2, Ap2, q1, Ap1, q2, Ap2, pAp, qAp);
        const double sigma = pAp - qAp;
        if (!(sigma > 0.0) || !isfinite(sigma)) {
            if (threadIdx.x == 0) atomicOr(a.flags, IETI_FLAG_BREAKDOWN);
            break;
        }
        const double alpha = rho / sigma;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            x1[i] += alpha * p1[i];
            rt1[i] -= alpha * Ap1[i];
            r1[i] -= alpha * q1[i];
        }
        for (int c = threadIdx.x; c < npi; c += blockDim.x) {
            x2[c] += alpha * p2[c];
            rt2[c] -= alpha * Ap2[c];
            r2[c] -= alpha * q2[c];
        }
        __syncthreads();
        saddle(q1, q2, t1, t2);   // A q (t1/t2 free until the next precond)
        for (int i = threadIdx.x; i < n; i += blockDim.x) Ar1[i] -= alpha * t1[i];
        for (int c = threadIdx.x; c < npi; c += blockDim.x) Ar2[c] -= alpha * t2[c];
        __syncthreads();
        dots(r1, rt1, r2, rt2, r1, Ar1, r2, Ar2, rr, rAr);
        double rho_new = rr - rAr;
        if (rho_new >= 0.0 && rho_new <= tol2 * rho0) {
            *conv = true;
            break;
        }
        if ((rho_new <= 1e-8 * rho_cycle || rho_new < 0.0) && restarts < 20) {
            ++restarts;
            saddle(x1, x2, t1, t2);
            for (int i = threadIdx.x; i < n; i += blockDim.x) rt1[i] = -t1[i];
            for (int c = threadIdx.x; c < npi; c += blockDim.x) rt2[c] = (c == jrow ? 1.0 : 0.0) - t2[c];
            __syncthreads();
            precond(rt1, rt2, r1, r2);
            saddle(r1, r2, Ar1, Ar2);
            dots(r1, rt1, r2, rt2, r1, Ar1, r2, Ar2, rr, rAr);
            rho = rr - rAr;
            rho_cycle = rho;
            if (rho <= tol2 * rho0) {
                *conv = true;
                break;
            }
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                p1[i] = r1[i];
                Ap1[i] = Ar1[i];
            }
            for (int c = threadIdx.x; c < npi; c += blockDim.x) {
                p2[c] = r2[c];
                Ap2[c] = Ar2[c];
            }
            __syncthreads();
            continue;
        }
        const double beta = rho_new / rho;
        rho = rho_new;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            p1[i] = r1[i] + beta * p1[i];
            Ap1[i] = Ar1[i] + beta * Ap1[i];
        }
        for (int c = threadIdx.x; c < npi; c += blockDim.x) {
            p2[c] = r2[c] + beta * p2[c];
            Ap2[c] = Ar2[c] + beta * Ap2[c];
        }
        __syncthreads();
    }
    double* phicol = a.phi + P.phioff + (long long)jrow * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) phicol[i] = x1[i];
    __syncthreads();
    return it;
}

}  // namespace ieti_sz
