// D-MG (Sec. 3.3): direct local Neumann solves by banded Cholesky.
//
// Per patch, the fine-level stiffness K in the natural (lexicographic) order
// of its full tensor grid is a band matrix of half-width
// bw = p0 + m0 (p1 + m1 p2).  Rows and columns of functions on the Dirichlet
// boundary become identity rows (their entries of every vector stay 0).  On a
// patch without Dirichlet side K is singular (constants); one interior dof is
// pinned (identity row and column): for a right-hand side orthogonal to the
// constants -- P^T g is -- the pinned system gives one solution of K z = P^T g,
// and the energy projection P removes the constant in which the solutions
// differ (Sec. 3.2: w = P z).  The band is stored by columns, lower part:
// band[bandoff + j (bw+1) + (i - j)] = L(i, j) for j < i <= j + bw, and the
// reciprocal 1 / L(j, j) in place of the diagonal (the solves multiply).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace {

// natural index of the pinned dof of a floating patch (-1: none)
__device__ __forceinline__ bool pinned_or_masked(const PatchDesc& P, int i) {
    const LevelDesc& L = P.lev[P.L - 1];
    const int i0 = i % L.m[0], i1 = (i / L.m[0]) % L.m[1], i2 = i / (L.m[0] * L.m[1]);
    return i == P.pin || ieti_masked(P.dmask, L.m, i0, i1, i2);
}

// band of K (lower part) from the color-blocked values; one CTA row-block per
// (rows, patch)
__global__ void k_band_assemble(const PatchDesc* pd, const int* plist, const double* K64, double* band) {
    const PatchDesc& P = pd[plist[blockIdx.y]];
    const LevelDesc& L = P.lev[P.L - 1];
    const int bw = P.bw;
    double* B = band + P.bandoff;
    const int W0 = 2 * P.p[0] + 1, W1 = 2 * P.p[1] + 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += gridDim.x * blockDim.x) {
        const int i0 = i % L.m[0], i1 = (i / L.m[0]) % L.m[1], i2 = i / (L.m[0] * L.m[1]);
        const bool fixed = pinned_or_masked(P, i);
        for (int o2 = -P.p[2]; o2 <= P.p[2]; ++o2)
            for (int o1 = -P.p[1]; o1 <= P.p[1]; ++o1)
                for (int o0 = -P.p[0]; o0 <= P.p[0]; ++o0) {
                    const int d = o0 + L.m[0] * (o1 + L.m[1] * o2);
                    if (d > 0) continue;   // lower part: column j = i + d <= i
                    const int j0 = i0 + o0, j1 = i1 + o1, j2 = i2 + o2;
                    if (j0 < 0 || j0 >= L.m[0] || j1 < 0 || j1 >= L.m[1] || j2 < 0 || j2 >= L.m[2]) continue;
                    const int j = i + d;
                    double v;
                    if (d == 0) {
                        v = fixed ? 1.0 : K64[L.koff + ieti_val_pos(L.m, P.p, L.S, i0, i1, i2,
                                                                        (o0 + P.p[0]) + W0 * ((o1 + P.p[1]) + W1 * (o2 + P.p[2])))];
                    } else {
                        v = (fixed || pinned_or_masked(P, j))
                                ? 0.0
                                : K64[L.koff + ieti_val_pos(L.m, P.p, L.S, i0, i1, i2,
                                                            (o0 + P.p[0]) + W0 * ((o1 + P.p[1]) + W1 * (o2 + P.p[2])))];
                    }
                    B[(long long)j * (bw + 1) + (i - j)] = v;
                }
    }
}

// right-looking band Cholesky by panels of kPanel columns, one thread-block
// cluster per patch.  Every CTA of the cluster loads the panel (its columns'
// band entries, already updated by every earlier panel) and factors it in
// shared memory -- the same arithmetic on the same data, so the copies agree
// bit for bit; each CTA writes back its share of the panel (reciprocal
// diagonal) and applies the panel to its share of the trailing window as a
// rank-kPanel update: every entry A(r, c') with c' past the panel and
// r <= last panel column + bw loses sum_c L(r, c) L(c', c) over the panel
// columns c.  One warp per trailing column (round-robin over the cluster's
// warps), lanes over its rows (coalesced), four rows per lane in flight.
// Two cluster barriers per panel: after the loads (the panel is written back
// below) and after the updates (the next panel reads them).  A non-positive
// pivot sets the flag and continues with pivot 1, so that every CTA passes
// every barrier.
constexpr int kPanel = 8;

__global__ void __launch_bounds__(256) k_band_cholesky(const PatchDesc* pd, const int* plist, double* band,
                                                       int* flags) {
    extern __shared__ double pan[];           // [kPanel][bw + 1]
    __shared__ int bad;
    cg::cluster_group cl = cg::this_cluster();
    const int crank = (int)cl.block_rank(), csize = (int)cl.num_blocks();
    const PatchDesc& P = pd[plist[blockIdx.x / csize]];
    const int n = P.n, bw = P.bw;
    const long long cs = bw + 1;
    double* B = band + P.bandoff;
    if (threadIdx.x == 0) bad = 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int gwarp = crank * nwarp + warp, gnwarp = csize * nwarp;
    for (int j0 = 0; j0 < n; j0 += kPanel) {
        const int nb = min(kPanel, n - j0);
        const int ne = nb * (bw + 1);
        for (int e = threadIdx.x; e < ne; e += blockDim.x) pan[e] = B[(long long)j0 * cs + e];
        __threadfence();
        cl.sync();
        // factor the panel in shared memory
        for (int c = 0; c < nb; ++c) {
            double* pc = pan + c * cs;
            if (threadIdx.x == 0) {
                const double a = pc[0];
                if (!(a > 0.0)) bad = 1;
                pc[0] = a > 0.0 ? sqrt(a) : 1.0;
            }
            __syncthreads();
            const int w = min(bw, n - 1 - (j0 + c));
            const double inv = 1.0 / pc[0];
            for (int o = 1 + threadIdx.x; o <= w; o += blockDim.x) pc[o] *= inv;
            __syncthreads();
            // later panel columns c2: A(j0+c2+o2, j0+c2) -= L(j0+c2+o2, j0+c) L(j0+c2, j0+c)
            for (int c2 = c + 1; c2 < nb; ++c2) {
                const int d = c2 - c;
                if (d > w) break;
                const double l2 = pc[d];
                double* p2 = pan + c2 * cs;
                for (int o2 = threadIdx.x; o2 <= w - d; o2 += blockDim.x) p2[o2] -= pc[d + o2] * l2;
            }
            __syncthreads();
        }
        // this CTA's share of the panel back to the band
        const int per = (ne + csize - 1) / csize;
        const int e1 = min(ne, (crank + 1) * per);
        for (int e = crank * per + threadIdx.x; e < e1; e += blockDim.x) {
            const int c = e / (bw + 1), o = e - c * (bw + 1);
            B[(long long)j0 * cs + e] = o == 0 ? 1.0 / pan[e] : pan[e];
        }
        // rank-nb update of this CTA's share of the trailing window
        const int rmax = min(n - 1, j0 + nb - 1 + bw);
        for (int cp = j0 + nb + gwarp; cp <= rmax; cp += gnwarp) {
            double lc[kPanel];
#pragma unroll
            for (int c = 0; c < kPanel; ++c) {
                const int o = cp - (j0 + c);
                lc[c] = (c < nb && o <= bw) ? pan[c * cs + o] : 0.0;
            }
            double* col = B + (long long)cp * cs - cp;   // col[r] = A(r, cp)
            for (int r0 = cp + lane; r0 <= rmax; r0 += 128) {
                double v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = r0 + 32 * u;
                    v[u] = r <= rmax ? col[r] : 0.0;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int r = r0 + 32 * u;
                    if (r > rmax) break;
                    double acc = 0.0;
#pragma unroll
                    for (int c = 0; c < kPanel; ++c) {
                        const int o = r - (j0 + c);
                        if (c < nb && o <= bw) acc += pan[c * cs + o] * lc[c];
                    }
                    col[r] = v[u] - acc;
                }
            }
        }
        __threadfence();
        cl.sync();
    }
    if (threadIdx.x == 0 && crank == 0 && bad) atomicOr(flags, IETI_FLAG_NOT_SPD);
}

// (L L^T)^{-1} v in place, one CTA (v in shared or global memory).  Each
// step needs one column (forward) or one row (backward) of the factor.
__device__ void band_solve_loop(const double* B, int n, int bw, double* v) {
    __shared__ double s;
    const long long cs = bw + 1;
    for (int j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            s = v[j] * B[(long long)j * cs];
            v[j] = s;
        }
        __syncthreads();
        const int w = min(bw, n - 1 - j);
        for (int t = 1 + threadIdx.x; t <= w; t += blockDim.x) v[j + t] -= B[(long long)j * cs + t] * s;
        __syncthreads();
    }
    for (int j = n - 1; j >= 0; --j) {
        if (threadIdx.x == 0) {
            s = v[j] * B[(long long)j * cs];
            v[j] = s;
        }
        __syncthreads();
        const int w = min(bw, j);
        for (int t = 1 + threadIdx.x; t <= w; t += blockDim.x) v[j - t] -= B[(long long)(j - t) * cs + t] * s;
        __syncthreads();
    }
}

// Blocked sweeps (bw < blockDim): pivots in blocks of four.  Per block one
// CTA barrier: every thread k applies the block's four pivots to its row
// (forward: row 4b+4+k, the column entries L(r, 4b+i); backward: row 4b-1-k,
// the row entries L(4b+i, r), four consecutive doubles of column r), and
// thread 0 -- after a warp barrier, since threads 0..3 of its warp own the
// next block's rows -- solves the next block's 4x4 triangle and publishes
// its pivots in the other half of a double buffer.  The factor entries of
// the block four ahead (and, for thread 0, the triangle and reciprocal
// diagonal of the block two ahead) are loaded into register rings, so their
// latency overlaps the blocks before.
struct Tri4 {
    double l[6];   // L(1,0), L(2,0), L(3,0), L(2,1), L(3,1), L(3,2) of the block
    double d[4];   // 1 / L(i,i)
};

__device__ void band_solve(const double* B, int n, int bw, double* v) {
    if (n <= 0) return;
    if (bw >= (int)blockDim.x) {              // more band offsets than threads
        band_solve_loop(B, n, bw, v);
        return;
    }
    __shared__ double piv[2][4];
    const int k = threadIdx.x;
    const bool lead = threadIdx.x == 0, warp0 = threadIdx.x < 32;
    const long long cs = bw + 1;
    const int nblk = (n + 3) / 4;
    auto fE = [&](int b, int i) -> double {   // L(4b+4+k, 4b+i)
        const int c = 4 * b + i, r = c + 4 + k - i;
        return (b >= 0 && b < nblk && c < n && r < n && 4 + k - i <= bw) ? B[(long long)c * cs + (4 + k - i)] : 0.0;
    };
    auto gE = [&](int b, int i) -> double {   // L(4b+i, 4b-1-k)
        const int c = 4 * b - 1 - k, r = 4 * b + i;
        return (b >= 0 && c >= 0 && r < n && i + 1 + k <= bw) ? B[(long long)c * cs + (i + 1 + k)] : 0.0;
    };
    auto load_tri = [&](int b, Tri4& T) {
        const int j0 = 4 * b;
        const bool ok = lead && b >= 0 && b < nblk;
        auto e = [&](int i, int i2) -> double {   // L(j0+i, j0+i2)
            return (ok && j0 + i < n && i - i2 <= bw) ? B[(long long)(j0 + i2) * cs + (i - i2)] : 0.0;
        };
        T.l[0] = e(1, 0);
        T.l[1] = e(2, 0);
        T.l[2] = e(3, 0);
        T.l[3] = e(2, 1);
        T.l[4] = e(3, 1);
        T.l[5] = e(3, 2);
#pragma unroll
        for (int i = 0; i < 4; ++i) T.d[i] = (ok && j0 + i < n) ? B[(long long)(j0 + i) * cs] : 0.0;
    };
    auto fwd_tri = [&](int b, const Tri4& T, double* pv) {   // thread 0
        const int j0 = 4 * b, m = min(4, n - j0);
        const double x0 = v[j0] * T.d[0];
        const double x1 = m > 1 ? (v[j0 + 1] - T.l[0] * x0) * T.d[1] : 0.0;
        const double x2 = m > 2 ? (v[j0 + 2] - T.l[1] * x0 - T.l[3] * x1) * T.d[2] : 0.0;
        const double x3 = m > 3 ? (v[j0 + 3] - T.l[2] * x0 - T.l[4] * x1 - T.l[5] * x2) * T.d[3] : 0.0;
        const double x[4] = {x0, x1, x2, x3};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (i < m) v[j0 + i] = x[i];
            pv[i] = x[i];
        }
    };
    auto bwd_tri = [&](int b, const Tri4& T, double* pv) {   // thread 0
        const int j0 = 4 * b, m = min(4, n - j0);
        const double x3 = m > 3 ? v[j0 + 3] * T.d[3] : 0.0;
        const double x2 = m > 2 ? (v[j0 + 2] - T.l[5] * x3) * T.d[2] : 0.0;
        const double x1 = m > 1 ? (v[j0 + 1] - T.l[3] * x2 - T.l[4] * x3) * T.d[1] : 0.0;
        const double x0 = (v[j0] - T.l[0] * x1 - T.l[1] * x2 - T.l[2] * x3) * T.d[0];
        const double x[4] = {x0, x1, x2, x3};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (i < m) v[j0 + i] = x[i];
            pv[i] = x[i];
        }
    };
    double e[4][4];
    Tri4 T[2];
    // ---- L y = v --------------------------------------------------------------
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int i = 0; i < 4; ++i) e[u][i] = fE(u, i);
    }
    load_tri(0, T[0]);
    load_tri(1, T[1]);
    if (lead) fwd_tri(0, T[0], piv[0]);
    load_tri(2, T[0]);
    __syncthreads();
    for (int b0 = 0; b0 < nblk; b0 += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int b = b0 + u;
            if (b >= nblk) break;
            const double* s = piv[u & 1];
            const double acc = e[u][0] * s[0] + e[u][1] * s[1] + e[u][2] * s[2] + e[u][3] * s[3];
            const int r = 4 * b + 4 + k;
            if (r < n && acc != 0.0) v[r] -= acc;
#pragma unroll
            for (int i = 0; i < 4; ++i) e[u][i] = fE(b + 4, i);
            if (warp0) {
                __syncwarp();
                const int un = (u + 1) & 1;
                if (lead && b + 1 < nblk) fwd_tri(b + 1, T[un], piv[un]);
                load_tri(b + 3, T[un]);
            }
            __syncthreads();
        }
    }
    // ---- L^T x = y (blocks from the last) ---------------------------------------
    const int bl = nblk - 1;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
        for (int i = 0; i < 4; ++i) e[u][i] = gE(bl - u, i);
    }
    load_tri(bl, T[0]);
    load_tri(bl - 1, T[1]);
    if (lead) bwd_tri(bl, T[0], piv[0]);
    load_tri(bl - 2, T[0]);
    __syncthreads();
    for (int q0 = 0; q0 < nblk; q0 += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int b = bl - (q0 + u);
            if (b < 0) break;
            const double* s = piv[u & 1];
            const double acc = e[u][0] * s[0] + e[u][1] * s[1] + e[u][2] * s[2] + e[u][3] * s[3];
            const int r = 4 * b - 1 - k;
            if (r >= 0 && acc != 0.0) v[r] -= acc;
#pragma unroll
            for (int i = 0; i < 4; ++i) e[u][i] = gE(b - 4, i);
            if (warp0) {
                __syncwarp();
                const int un = (u + 1) & 1;
                if (lead && b - 1 >= 0) bwd_tri(b - 1, T[un], piv[un]);
                load_tri(b - 3, T[un]);
            }
            __syncthreads();
        }
    }
}

struct Red2 {
    double v[32];
};

__device__ double cta_sum1(double x, Red2& sh) {
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh.v[w] = x;
    __syncthreads();
    double s = 0.0;
    for (int i = 0; i < nw; ++i) s += sh.v[i];
    __syncthreads();
    return s;
}

// Neumann solve of one slot (patch): u = P z + Phi u_Pi with K z = P^T g
// solved directly (same input and output conventions as the multigrid
// Neumann mode of the local solver)
__global__ void __launch_bounds__(512) k_direct_neumann(SolveArgs a0) {
    const IetiLaunchSpan span_(a0.tspan);
    extern __shared__ double zsh[];
    __shared__ SolveArgs sa;
    __shared__ double coef[64];
    __shared__ Red2 red;
    const SlotDesc sd = a0.slots[blockIdx.x];
    if (threadIdx.x == 0) {
        sa = a0.batch ? a0.batch[sd.handle] : a0;
        sa.slots = a0.slots;
        sa.nslots = a0.nslots;
    }
    __syncthreads();
    const SolveArgs& a = sa;
    const PatchDesc& P = a.pd[sd.patch];
    const LevelDesc& F = P.lev[P.L - 1];
    const int n = F.n;
    // the substitution's vector in shared memory when it fits the launch's
    // dynamic budget (every step reads and updates it), else in global memory
    double* z = (size_t)n * sizeof(double) <= a0.smem_bytes ? zsh : a.cg + sd.cg;
    const double* g = a.in + P.toff;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int i0 = i % F.m[0], ir = i / F.m[0];
        const int i1 = ir % F.m[1], i2 = ir / F.m[1];
        z[i] = ieti_masked(P.dmask, F.m, i0, i1, i2) ? 0.0 : g[i];
    }
    __syncthreads();
    // b = P^T g = g - C^T (Phi^T g)
    {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int j = w; j < P.npi; j += nw) {
            const int row = P.crow0 + j;
            const double cj = a.rpi_loc[row];
            for (int e = a.crow_ptr[row] + lane; e < a.crow_ptr[row + 1]; e += 32) z[a.c_idx[e]] -= a.c_w[e] * cj;
        }
    }
    __syncthreads();
    if (P.floating) {
        // exact orthogonality to the constants (the kernel of K), then pin
        double s = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) s += z[i];
        s = cta_sum1(s, red);
        const double mean = s / n;
        for (int i = threadIdx.x; i < n; i += blockDim.x) z[i] -= mean;
        __syncthreads();
        if (threadIdx.x == 0 && P.pin >= 0) z[P.pin] = 0.0;
        __syncthreads();
    }
    band_solve(a.band + P.bandoff, n, P.bw, z);
    // u = z - Phi (C z - A u_Pi)
    {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
        for (int j = w; j < P.npi; j += nw) {
            const int row = P.crow0 + j;
            double d = 0.0;
            for (int e = a.crow_ptr[row] + lane; e < a.crow_ptr[row + 1]; e += 32) d += a.c_w[e] * z[a.c_idx[e]];
            for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            if (lane == 0) coef[j] = d - a.upi_loc[row];
        }
    }
    __syncthreads();
    double* out = a.out + P.toff;
    const double* ph = a.phi + P.phioff;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double u = z[i];
        for (int j = 0; j < P.npi; ++j) u -= coef[j] * ph[(long long)j * n + i];
        out[i] = u;
    }
}

}  // namespace

cudaError_t launch_band_factor(const PatchDesc* pd, const int* plist, int npl, int max_n, int max_bw,
                               const double* K64, double* band, int* flags, cudaStream_t st) {
    if (npl == 0) return cudaSuccess;
    k_band_assemble<<<dim3((max_n + 255) / 256, npl), 256, 0, st>>>(pd, plist, K64, band);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t sm = sizeof(double) * (size_t)kPanel * (size_t)(max_bw + 1);
    if (sm > 48 * 1024) {
        e = cudaFuncSetAttribute(k_band_cholesky, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    // CTAs per patch: enough warps that each takes a few trailing columns
    // per panel (bw / 48: 4 for the annulus' 204, 8 for bands of 396 and up)
    const int csize = std::max(1, std::min(8, max_bw / 48));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(npl * csize));
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, k_band_cholesky, pd, plist, band, flags);
    if (e != cudaSuccess && csize > 1) {
        // clusters that cannot be co-scheduled (launch-configuration error,
        // not sticky): one CTA per patch, the same arithmetic
        cudaGetLastError();
        cfg.gridDim = dim3((unsigned)npl);
        attr[0].val.clusterDim.x = 1;
        e = cudaLaunchKernelEx(&cfg, k_band_cholesky, pd, plist, band, flags);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_direct_neumann(const SolveArgs& a, int max_bw, cudaStream_t st) {
    if (a.nslots == 0) return cudaSuccess;
    // one thread per band row past a pivot block (bw + 1 threads, rounded to
    // warps; at most 512: wider bands take the strided sweep)
    const int threads = std::min(512, std::max(64, ((max_bw + 32) / 32) * 32));
    cudaError_t e = cudaFuncSetAttribute(k_direct_neumann, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kDirectSmemCap);
    if (e != cudaSuccess) return e;
    SolveArgs b = a;
    b.smem_bytes = std::min(a.smem_bytes, kDirectSmemCap);
    k_direct_neumann<<<a.nslots, threads, b.smem_bytes, st>>>(b);
    return cudaGetLastError();
}
