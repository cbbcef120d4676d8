// Setup kernels: B-spline tables, Gauss quadrature, Galerkin assembly of the
// stiffness and load of Eq. 1 (Sec. 2), multigrid transfer tables (canonical
// embedding of nested spline spaces, Sec. 4), Galerkin coarse operators,
// parameter-domain mass bands (K + alpha M^, Sec. 3.2), coarsest-level
// inverses, constraint weights, and a one-CTA dense Cholesky.
//
// All floating-point setup work runs here on the GPU; the host only supplies
// integer topology and offsets.
#include <math.h>
#include "kernels.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846;

// open uniform knot vector on [0,1] with n elements, degree p
__device__ __forceinline__ double knot(int i, int n, int p) {
    int k = i - p;
    k = k < 0 ? 0 : (k > n ? n : k);
    return (double)k / (double)n;
}

// q-th (ascending) Gauss-Legendre node and weight on [-1,1], nq points:
// Newton iteration on the three-term Legendre recurrence.
__device__ void gauss_node(int nq, int q, double* x, double* w) {
    int k = nq - 1 - q;
    double z = cos(kPi * (k + 0.75) / (nq + 0.5));
    double p1 = 1.0, p2 = 0.0, pp = 1.0;
    for (int it = 0; it < 100; ++it) {
        p1 = 1.0; p2 = 0.0;
        for (int j = 1; j <= nq; ++j) {
            double p3 = p2;
            p2 = p1;
            p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
        }
        pp = nq * (z * p1 - p2) / (z * z - 1.0);
        double dz = p1 / pp;
        z -= dz;
        if (fabs(dz) < 1e-16) break;
    }
    p1 = 1.0; p2 = 0.0;
    for (int j = 1; j <= nq; ++j) {
        double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
    }
    pp = nq * (z * p1 - p2) / (z * z - 1.0);
    *x = z;
    *w = 2.0 / ((1.0 - z * z) * pp * pp);
}

// Values and first derivatives of the p+1 B-splines that are nonzero on the
// knot span mu (t_mu <= x < t_mu+1): triangular Cox-de Boor scheme.
__device__ void basis_local(double x, int mu, int n, int p, double* N, double* dN) {
    double left[IETI_MAXP + 1], right[IETI_MAXP + 1], Q[IETI_MAXP + 1];
    N[0] = 1.0;
    Q[0] = 1.0;
    for (int j = 1; j <= p; ++j) {
        if (j == p)
            for (int k = 0; k < p; ++k) Q[k] = N[k];
        left[j] = x - knot(mu + 1 - j, n, p);
        right[j] = knot(mu + j, n, p) - x;
        double saved = 0.0;
        for (int r = 0; r < j; ++r) {
            double tmp = N[r] / (right[r + 1] + left[j - r]);
            N[r] = saved + right[r + 1] * tmp;
            saved = left[j - r] * tmp;
        }
        N[j] = saved;
    }
    for (int k = 0; k <= p; ++k) {
        int i = mu - p + k;
        double a = 0.0, b = 0.0;
        if (k >= 1) {
            double den = knot(i + p, n, p) - knot(i, n, p);
            if (den > 0) a = Q[k - 1] / den;
        }
        if (k <= p - 1) {
            double den = knot(i + p + 1, n, p) - knot(i + 1, n, p);
            if (den > 0) b = Q[k] / den;
        }
        dN[k] = p * (a - b);
    }
}

__device__ int find_patch(const long long* off, int np, long long g) {
    int lo = 0, hi = np - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// rational quadratic quarter circle C(t) and C'(t)
__device__ void circle(double t, double* cx, double* cy, double* dcx, double* dcy) {
    const double w1 = 0.70710678118654752440;
    double b0 = (1 - t) * (1 - t), b1 = 2 * t * (1 - t), b2 = t * t;
    double d0 = -2 * (1 - t), d1 = 2 - 4 * t, d2 = 2 * t;
    double W = b0 + w1 * b1 + b2, dW = d0 + w1 * d1 + d2;
    double Nx = b0 + w1 * b1, Ny = w1 * b1 + b2;
    double dNx = d0 + w1 * d1, dNy = w1 * d1 + d2;
    *cx = Nx / W;
    *cy = Ny / W;
    *dcx = (dNx * W - Nx * dW) / (W * W);
    *dcy = (dNy * W - Ny * dW) / (W * W);
}

// ---------------------------------------------------------------------------
__global__ void k_asm_tables(SetupArgs a) {
    int k = blockIdx.y / 3, r = blockIdx.y % 3;
    const PatchDesc& P = a.pd[k];
    if (r >= P.dim) return;
    AsmTables t = a.at[k * 3 + r];
    int p = P.p[r], n = P.nelem[r], nq = p + 1;
    for (int pt = blockIdx.x * blockDim.x + threadIdx.x; pt < t.nq; pt += gridDim.x * blockDim.x) {
        int e = pt / nq, q = pt % nq;
        double g, w;
        gauss_node(nq, q, &g, &w);
        double x = (e + 0.5 * (g + 1.0)) / n;
        a.qx[t.qoff + pt] = x;
        a.qw[t.qoff + pt] = 0.5 * w / n;
        double N[IETI_MAXP + 1], dN[IETI_MAXP + 1];
        basis_local(x, p + e, n, p, N, dN);
        for (int j = 0; j <= p; ++j) {
            a.Bv[t.boff + (long long)pt * (p + 1) + j] = N[j];
            a.Dv[t.boff + (long long)pt * (p + 1) + j] = dN[j];
        }
    }
}

__global__ void k_geometry(SetupArgs a, long long total) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
         g += (long long)gridDim.x * blockDim.x) {
        int k = find_patch(a.qpoff, a.npatch, g);
        const PatchDesc& P = a.pd[k];
        long long loc = g - a.qpoff[k];
        int d = P.dim;
        int qi[3] = {0, 0, 0};
        double xi[3] = {0, 0, 0}, w = 1.0;
        long long rem = loc;
        for (int r = 0; r < d; ++r) {
            AsmTables t = a.at[k * 3 + r];
            qi[r] = (int)(rem % t.nq);
            rem /= t.nq;
            xi[r] = a.qx[t.qoff + qi[r]];
            w *= a.qw[t.qoff + qi[r]];
        }
        const double* geo = a.geo + 7 * k;
        int kind = (int)geo[0];
        double X[3] = {0, 0, 0}, J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        if (kind == 0) {
            for (int r = 0; r < d; ++r) {
                double h = geo[4 + r] - geo[1 + r];
                X[r] = geo[1 + r] + h * xi[r];
                J[r][r] = h;
            }
        } else {
            double h0 = geo[4] - geo[1], h1 = geo[5] - geo[2];
            double s1 = geo[1] + h0 * xi[0], s2 = geo[2] + h1 * xi[1];
            double cx, cy, dcx, dcy;
            circle(s1, &cx, &cy, &dcx, &dcy);
            double rad = 1.0 + s2;
            X[0] = rad * cx;
            X[1] = rad * cy;
            J[0][0] = rad * dcx * h0;
            J[1][0] = rad * dcy * h0;
            J[0][1] = cx * h1;
            J[1][1] = cy * h1;
        }
        double det, inv[3][3];
        if (d == 2) {
            det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            inv[0][0] = J[1][1] / det;
            inv[0][1] = -J[0][1] / det;
            inv[1][0] = -J[1][0] / det;
            inv[1][1] = J[0][0] / det;
        } else {
            det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                  J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                  J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
            inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
            inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
            inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
            inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
            inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
            inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
            inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
            inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
            inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
        }
        double wd = w * fabs(det);
        double G[6] = {0, 0, 0, 0, 0, 0};
        // G_ab = w |det J| sum_c inv[a][c] inv[b][c]; packed upper triangle
        int idx = 0;
        for (int aa = 0; aa < d; ++aa)
            for (int bb = aa; bb < d; ++bb) {
                double s = 0.0;
                for (int c = 0; c < d; ++c) s += inv[aa][c] * inv[bb][c];
                G[idx++] = wd * s;
            }
        for (int t = 0; t < 6; ++t) a.Gm[g * 6 + t] = G[t];
        double f = 0.0;
        switch (a.rhs_kind) {
            case 1: f = 2 * kPi * kPi * sin(kPi * X[0]) * sin(kPi * X[1]); break;
            case 2: f = 3 * kPi * kPi * sin(kPi * X[0]) * sin(kPi * X[1]) * sin(kPi * X[2]); break;
            case 3: {
                double x = X[0], y = X[1], r = sqrt(x * x + y * y);
                double s = sin(kPi * x) * sin(kPi * y);
                double gg = (r - 1) * (2 - r), gp = 3 - 2 * r;
                f = 2 * kPi * kPi * s * gg -
                    2 * kPi * (gp / r) * (x * cos(kPi * x) * sin(kPi * y) + y * sin(kPi * x) * cos(kPi * y)) -
                    s * (3 / r - 4);
                break;
            }
            case 4:
                for (int j = 0; j < a.nmodes; ++j)
                    f += a.modes[3 * j] * sin(a.modes[3 * j + 1] * kPi * X[0]) * sin(a.modes[3 * j + 2] * kPi * X[1]);
                break;
            case 5: f = a.quad_values[g]; break;
            default: f = 0.0;
        }
        a.Fw[g] = wd * f;
    }
}

// gradient of tensor basis function with local (element) indices loc at the
// element point (e, q): reads the per-direction tables
struct PtTab {
    const double* B[3];
    const double* D[3];
};

__global__ void k_stiffness(SetupArgs a, long long total_rows) {
    int o = blockIdx.y;
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total_rows;
         g += (long long)gridDim.x * blockDim.x) {
        int k = find_patch(a.rowoff, a.npatch, g);
        const PatchDesc& P = a.pd[k];
        const LevelDesc& F = P.lev[P.L - 1];
        if (o >= F.S) continue;
        int i = (int)(g - a.rowoff[k]);
        int d = P.dim;
        int ii[3] = {i % F.m[0], (i / F.m[0]) % F.m[1], i / (F.m[0] * F.m[1])};
        int oo[3], jj[3], rem = o;
        for (int r = 0; r < 3; ++r) {
            int w = 2 * P.p[r] + 1;
            oo[r] = rem % w - P.p[r];
            rem /= w;
            jj[r] = ii[r] + oo[r];
        }
        bool inside = true;
        for (int r = 0; r < 3; ++r) inside &= (jj[r] >= 0 && jj[r] < F.m[r]);
        double acc = 0.0;
        if (inside) {
            int elo[3] = {0, 0, 0}, ehi[3] = {0, 0, 0}, nq[3] = {1, 1, 1};
            const double *Bt[3], *Dt[3];
            for (int r = 0; r < d; ++r) {
                int lo = max(ii[r], jj[r]) - P.p[r], hi = min(ii[r], jj[r]);
                elo[r] = max(lo, 0);
                ehi[r] = min(hi, P.nelem[r] - 1);
                nq[r] = P.p[r] + 1;
                AsmTables t = a.at[k * 3 + r];
                Bt[r] = a.Bv + t.boff;
                Dt[r] = a.Dv + t.boff;
            }
            long long qbase = a.qpoff[k];
            int nqd[3] = {a.at[k * 3 + 0].nq, d > 1 ? a.at[k * 3 + 1].nq : 1, d > 2 ? a.at[k * 3 + 2].nq : 1};
            for (int e2 = elo[2]; e2 <= ehi[2]; ++e2)
                for (int e1 = elo[1]; e1 <= ehi[1]; ++e1)
                    for (int e0 = elo[0]; e0 <= ehi[0]; ++e0)
                        for (int q2 = 0; q2 < nq[2]; ++q2)
                            for (int q1 = 0; q1 < nq[1]; ++q1)
                                for (int q0 = 0; q0 < nq[0]; ++q0) {
                                    int e[3] = {e0, e1, e2}, q[3] = {q0, q1, q2};
                                    double bi[3], di[3], bj[3], dj[3];
                                    int pt[3];
                                    for (int r = 0; r < 3; ++r) {
                                        if (r < d) {
                                            pt[r] = e[r] * nq[r] + q[r];
                                            int pr = P.p[r] + 1;
                                            bi[r] = Bt[r][(long long)pt[r] * pr + ii[r] - e[r]];
                                            di[r] = Dt[r][(long long)pt[r] * pr + ii[r] - e[r]];
                                            bj[r] = Bt[r][(long long)pt[r] * pr + jj[r] - e[r]];
                                            dj[r] = Dt[r][(long long)pt[r] * pr + jj[r] - e[r]];
                                        } else {
                                            pt[r] = 0;
                                            bi[r] = bj[r] = 1.0;
                                            di[r] = dj[r] = 0.0;
                                        }
                                    }
                                    long long qf = qbase + pt[0] + (long long)nqd[0] * (pt[1] + (long long)nqd[1] * pt[2]);
                                    const double* G = a.Gm + qf * 6;
                                    double gi[3] = {di[0] * bi[1] * bi[2], bi[0] * di[1] * bi[2], bi[0] * bi[1] * di[2]};
                                    double gj[3] = {dj[0] * bj[1] * bj[2], bj[0] * dj[1] * bj[2], bj[0] * bj[1] * dj[2]};
                                    if (d == 2) {
                                        acc += G[0] * gi[0] * gj[0] + G[1] * (gi[0] * gj[1] + gi[1] * gj[0]) +
                                               G[2] * gi[1] * gj[1];
                                    } else {
                                        acc += G[0] * gi[0] * gj[0] + G[3] * gi[1] * gj[1] + G[5] * gi[2] * gj[2] +
                                               G[1] * (gi[0] * gj[1] + gi[1] * gj[0]) +
                                               G[2] * (gi[0] * gj[2] + gi[2] * gj[0]) +
                                               G[4] * (gi[1] * gj[2] + gi[2] * gj[1]);
                                    }
                                }
        }
        a.K64[F.koff + ieti_val_pos(F.m, P.p, F.S, ii[0], ii[1], ii[2], o)] = acc;
    }
}

__global__ void k_load(SetupArgs a, long long total_rows) {
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total_rows;
         g += (long long)gridDim.x * blockDim.x) {
        int k = find_patch(a.rowoff, a.npatch, g);
        const PatchDesc& P = a.pd[k];
        const LevelDesc& F = P.lev[P.L - 1];
        int i = (int)(g - a.rowoff[k]);
        int d = P.dim;
        int ii[3] = {i % F.m[0], (i / F.m[0]) % F.m[1], i / (F.m[0] * F.m[1])};
        int elo[3] = {0, 0, 0}, ehi[3] = {0, 0, 0}, nq[3] = {1, 1, 1}, nqd[3] = {1, 1, 1};
        const double* Bt[3] = {nullptr, nullptr, nullptr};
        for (int r = 0; r < d; ++r) {
            elo[r] = max(ii[r] - P.p[r], 0);
            ehi[r] = min(ii[r], P.nelem[r] - 1);
            nq[r] = P.p[r] + 1;
            AsmTables t = a.at[k * 3 + r];
            Bt[r] = a.Bv + t.boff;
            nqd[r] = t.nq;
        }
        double acc = 0.0;
        long long qbase = a.qpoff[k];
        for (int e2 = elo[2]; e2 <= ehi[2]; ++e2)
            for (int e1 = elo[1]; e1 <= ehi[1]; ++e1)
                for (int e0 = elo[0]; e0 <= ehi[0]; ++e0)
                    for (int q2 = 0; q2 < nq[2]; ++q2)
                        for (int q1 = 0; q1 < nq[1]; ++q1)
                            for (int q0 = 0; q0 < nq[0]; ++q0) {
                                int e[3] = {e0, e1, e2}, q[3] = {q0, q1, q2}, pt[3] = {0, 0, 0};
                                double v = 1.0;
                                for (int r = 0; r < d; ++r) {
                                    pt[r] = e[r] * nq[r] + q[r];
                                    v *= Bt[r][(long long)pt[r] * (P.p[r] + 1) + ii[r] - e[r]];
                                }
                                long long qf = qbase + pt[0] + (long long)nqd[0] * (pt[1] + (long long)nqd[1] * pt[2]);
                                acc += a.Fw[qf] * v;
                            }
        a.f[P.toff + i] = acc;
    }
}

// ---- multigrid transfer tables --------------------------------------------
// Row form of the prolongation (fine i -> coarse start + weights), by the
// discrete B-spline recursion (Oslo algorithm) for one dyadic refinement:
//   alpha_{j,0}(i) = [t_j <= tau_i < t_{j+1}],
//   alpha_{j,k}(i) = (tau_{i+k}-t_j)/(t_{j+k}-t_j) alpha_{j,k-1}(i)
//                  + (t_{j+k+1}-tau_{i+k})/(t_{j+k+1}-t_{j+1}) alpha_{j+1,k-1}(i).
__global__ void k_prolong_rows(SetupArgs a, const TableJob* jobs) {
    TableJob jb = jobs[blockIdx.y];
    const PatchDesc& P = a.pd[jb.patch];
    const LevelDesc& Lf = P.lev[jb.level];
    const LevelDesc& Lc = P.lev[jb.level - 1];
    int r = jb.r, p = P.p[r], W = p + 2;
    int mf = Lf.m[r], mc = Lc.m[r];
    int nf = mf - p, nc = mc - p;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < mf; i += gridDim.x * blockDim.x) {
        double* w = a.tab + Lf.pw[r] + (long long)i * W;
        int* st = a.itab + Lf.ps[r] + i;
        for (int t = 0; t < W; ++t) w[t] = 0.0;
        if (!Lf.refined[r]) {
            *st = i;
            w[0] = 1.0;
            continue;
        }
        int mu = p + max(0, i - p) / 2;   // coarse span holding tau_i
        if (mu > p + nc - 1) mu = p + nc - 1;
        double al[IETI_MAXP + 2];
        // al[j - (mu - k)] holds alpha_{j,k}(i) for j = mu-k .. mu
        al[0] = 1.0;
        for (int k = 1; k <= p; ++k) {
            double nw[IETI_MAXP + 2];
            for (int jj = 0; jj <= k; ++jj) {
                int j = mu - k + jj;
                double v = 0.0;
                double tik = knot(i + k, nf, p);
                // alpha_{j,k-1}: index j-(mu-(k-1)) = jj-1
                if (jj - 1 >= 0) {
                    double den = knot(j + k, nc, p) - knot(j, nc, p);
                    if (den > 0) v += (tik - knot(j, nc, p)) / den * al[jj - 1];
                }
                // alpha_{j+1,k-1}: index jj
                if (jj <= k - 1) {
                    double den = knot(j + k + 1, nc, p) - knot(j + 1, nc, p);
                    if (den > 0) v += (knot(j + k + 1, nc, p) - tik) / den * al[jj];
                }
                nw[jj] = v;
            }
            for (int jj = 0; jj <= k; ++jj) al[jj] = nw[jj];
        }
        int start = mu - p;
        if (start < 0 || start + p > mc - 1) atomicOr(a.flags, IETI_FLAG_TABLE);
        *st = start;
        for (int t = 0; t <= p; ++t) w[t] = al[t];
    }
}

// Column form (restriction): for coarse J the contiguous fine rows with
// nonzero P(i, J).
__global__ void k_restrict_cols(SetupArgs a, const TableJob* jobs) {
    TableJob jb = jobs[blockIdx.y];
    const PatchDesc& P = a.pd[jb.patch];
    const LevelDesc& Lf = P.lev[jb.level];
    const LevelDesc& Lc = P.lev[jb.level - 1];
    int r = jb.r, p = P.p[r], W = p + 2;
    int mf = Lf.m[r], mc = Lc.m[r];
    for (int J = blockIdx.x * blockDim.x + threadIdx.x; J < mc; J += gridDim.x * blockDim.x) {
        int first = -1, last = -1;
        for (int i = 0; i < mf; ++i) {
            int s = a.itab[Lf.ps[r] + i];
            int t = J - s;
            if (t >= 0 && t < W && a.tab[Lf.pw[r] + (long long)i * W + t] != 0.0) {
                if (first < 0) first = i;
                last = i;
            }
        }
        double* w = a.tab + Lf.rw[r] + (long long)J * W;
        for (int t = 0; t < W; ++t) w[t] = 0.0;
        if (first < 0 || last - first + 1 > W) {
            atomicOr(a.flags, IETI_FLAG_TABLE);
            a.itab[Lf.rs[r] + J] = 0;
            continue;
        }
        a.itab[Lf.rs[r] + J] = first;
        for (int i = first; i <= last; ++i) {
            int s = a.itab[Lf.ps[r] + i];
            w[i - first] = a.tab[Lf.pw[r] + (long long)i * W + (J - s)];
        }
    }
}

// 1D parameter-domain mass band M(i, i+o) of one level, Gauss quadrature
__global__ void k_mass1d(SetupArgs a, const TableJob* jobs) {
    TableJob jb = jobs[blockIdx.y];
    const PatchDesc& P = a.pd[jb.patch];
    const LevelDesc& L = P.lev[jb.level];
    int r = jb.r, p = P.p[r], B = 2 * p + 1;
    int m = L.m[r], n = m - p;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m * B; t += gridDim.x * blockDim.x) {
        int i = t / B, o = t % B - p, j = i + o;
        double acc = 0.0;
        if (j >= 0 && j < m) {
            int lo = max(max(i, j) - p, 0), hi = min(min(i, j), n - 1);
            for (int e = lo; e <= hi; ++e)
                for (int q = 0; q <= p; ++q) {
                    double g, w;
                    gauss_node(p + 1, q, &g, &w);
                    double x = (e + 0.5 * (g + 1.0)) / n;
                    double N[IETI_MAXP + 1], dN[IETI_MAXP + 1];
                    basis_local(x, p + e, n, p, N, dN);
                    acc += 0.5 * w / n * N[i - e] * N[j - e];
                }
        }
        a.tab[L.mw[r] + t] = acc;
    }
}

// Galerkin coarse operator K_c = P^T K_f P (banded, full tensor grid)
__global__ void k_galerkin(const PatchDesc* pd, const int* plist, int depth, double* K64,
                           const double* tab, const int* itab) {
    const PatchDesc& P = pd[plist[blockIdx.z]];
    int lf = P.L - depth, lc = lf - 1;
    if (lc < 0) return;
    const LevelDesc& F = P.lev[lf];
    const LevelDesc& C = P.lev[lc];
    int O = blockIdx.y;
    if (O >= C.S) return;
    int oo[3], rem = O;
    for (int r = 0; r < 3; ++r) {
        int w = 2 * P.p[r] + 1;
        oo[r] = rem % w - P.p[r];
        rem /= w;
    }
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < C.n; I += gridDim.x * blockDim.x) {
        int Ii[3] = {I % C.m[0], (I / C.m[0]) % C.m[1], I / (C.m[0] * C.m[1])};
        int Jj[3];
        bool inside = true;
        for (int r = 0; r < 3; ++r) {
            Jj[r] = Ii[r] + oo[r];
            inside &= (Jj[r] >= 0 && Jj[r] < C.m[r]);
        }
        double acc = 0.0;
        if (inside) {
            int W[3], ai0[3], bi0[3];
            const double *wa[3], *wb[3];
            for (int r = 0; r < 3; ++r) {
                if (r < P.dim) {
                    W[r] = P.p[r] + 2;
                    ai0[r] = itab[F.rs[r] + Ii[r]];
                    bi0[r] = itab[F.rs[r] + Jj[r]];
                    wa[r] = tab + F.rw[r] + (long long)Ii[r] * W[r];
                    wb[r] = tab + F.rw[r] + (long long)Jj[r] * W[r];
                } else {
                    W[r] = 1;
                    ai0[r] = bi0[r] = 0;
                    wa[r] = wb[r] = nullptr;
                }
            }
            for (int t2 = 0; t2 < W[2]; ++t2)
                for (int t1 = 0; t1 < W[1]; ++t1)
                    for (int t0 = 0; t0 < W[0]; ++t0) {
                        int a[3] = {ai0[0] + t0, ai0[1] + t1, ai0[2] + t2};
                        double pa = 1.0;
                        bool ok = true;
                        int tt[3] = {t0, t1, t2};
                        for (int r = 0; r < P.dim; ++r) {
                            ok &= a[r] < F.m[r];
                            if (ok) pa *= wa[r][tt[r]];
                        }
                        if (!ok || pa == 0.0) continue;
                        for (int u2 = 0; u2 < W[2]; ++u2)
                            for (int u1 = 0; u1 < W[1]; ++u1)
                                for (int u0 = 0; u0 < W[0]; ++u0) {
                                    int b[3] = {bi0[0] + u0, bi0[1] + u1, bi0[2] + u2};
                                    int uu[3] = {u0, u1, u2};
                                    double pb = 1.0;
                                    int of = 0, mul = 1;
                                    bool ok2 = true;
                                    for (int r = 0; r < 3; ++r) {
                                        int dlt = b[r] - a[r];
                                        if (r < P.dim) {
                                            ok2 &= b[r] < F.m[r] && dlt >= -P.p[r] && dlt <= P.p[r];
                                            if (ok2) pb *= wb[r][uu[r]];
                                        }
                                        of += (dlt + P.p[r]) * mul;
                                        mul *= 2 * P.p[r] + 1;
                                    }
                                    if (!ok2 || pb == 0.0) continue;
                                    acc += pa * pb * K64[F.koff + ieti_val_pos(F.m, P.p, F.S, a[0], a[1], a[2], of)];
                                }
                    }
        }
        K64[C.koff + ieti_val_pos(C.m, P.p, C.S, Ii[0], Ii[1], Ii[2], O)] = acc;
    }
}

// one-CTA dense Cholesky (lower, in place, row-major A n x n), then the
// inverse of the factor into Linv (row-major, lower)
__device__ void cta_cholesky_linv(double* A, int n, double* Linv, int* flags) {
    for (int k = 0; k < n; ++k) {
        __syncthreads();
        if (threadIdx.x == 0) {
            double dkk = A[(long long)k * n + k];
            if (!(dkk > 0.0)) {
                atomicOr(flags, IETI_FLAG_NOT_SPD);
                dkk = 1.0;
            }
            A[(long long)k * n + k] = sqrt(dkk);
        }
        __syncthreads();
        double piv = A[(long long)k * n + k];
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[(long long)i * n + k] /= piv;
        __syncthreads();
        int nt = n - k - 1;
        long long pairs = (long long)nt * nt;
        for (long long t = threadIdx.x; t < pairs; t += blockDim.x) {
            int i = k + 1 + (int)(t / nt), j = k + 1 + (int)(t % nt);
            if (j <= i) A[(long long)i * n + j] -= A[(long long)i * n + k] * A[(long long)j * n + k];
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        for (int i = 0; i < j; ++i) Linv[(long long)i * n + j] = 0.0;
        Linv[(long long)j * n + j] = 1.0 / A[(long long)j * n + j];
        for (int i = j + 1; i < n; ++i) {
            double s = 0.0;
            for (int kk = j; kk < i; ++kk) s += A[(long long)i * n + kk] * Linv[(long long)kk * n + j];
            Linv[(long long)i * n + j] = -s / A[(long long)i * n + i];
        }
    }
    __syncthreads();
}

__global__ void k_chol_linv(double* A, int n, double* Linv, int* flags) {
    cta_cholesky_linv(A, n, Linv, flags);
}

__global__ void k_coarse_inverse(const PatchDesc* pd, const double* K64, const double* tab,
                                 double alpha, double* A0inv64, float* A0inv32, double* work,
                                 int max_n0, int* flags) {
    int job = blockIdx.x;
    int k = job >> 1, kind = job & 1;
    const PatchDesc& P = pd[k];
    const LevelDesc& L = P.lev[0];
    int n = L.n;
    double* A = work + (long long)job * 2 * max_n0 * max_n0;
    double* Li = A + (long long)max_n0 * max_n0;
    int mask = kind == 0 ? P.dmask : (P.dim == 2 ? 0xF : 0x3F);
    double al = (kind == 0 && P.floating) ? alpha : 0.0;
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
        int i = (int)(t / n), j = (int)(t % n);
        int ii[3] = {i % L.m[0], (i / L.m[0]) % L.m[1], i / (L.m[0] * L.m[1])};
        int jj[3] = {j % L.m[0], (j / L.m[0]) % L.m[1], j / (L.m[0] * L.m[1])};
        double v = 0.0;
        bool mi = ieti_masked(mask, L.m, ii[0], ii[1], ii[2]);
        bool mj = ieti_masked(mask, L.m, jj[0], jj[1], jj[2]);
        if (mi || mj) {
            v = (i == j) ? 1.0 : 0.0;
        } else {
            bool band = true;
            int of = 0, mul = 1;
            double mprod = 1.0;
            for (int r = 0; r < 3; ++r) {
                int dl = jj[r] - ii[r];
                band &= dl >= -P.p[r] && dl <= P.p[r];
                of += (dl + P.p[r]) * mul;
                mul *= 2 * P.p[r] + 1;
                if (band && r < P.dim) mprod *= tab[L.mw[r] + ii[r] * (2 * P.p[r] + 1) + dl + P.p[r]];
            }
            if (band) {
                v = K64[L.koff + ieti_val_pos(L.m, P.p, L.S, ii[0], ii[1], ii[2], of)] + al * mprod;
            }
        }
        A[t] = v;
    }
    cta_cholesky_linv(A, n, Li, flags);
    // A^{-1} = Linv^T Linv (symmetric)
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
        int i = (int)(t / n), j = (int)(t % n);
        double s = 0.0;
        for (int kk = max(i, j); kk < n; ++kk) s += Li[(long long)kk * n + i] * Li[(long long)kk * n + j];
        A0inv64[P.a0off[kind] + t] = s;
        A0inv32[P.a0off[kind] + t] = (float)s;
    }
}

// KM = K + alpha M^ on every level of the floating patches (M^ the Kronecker
// product of the 1D parameter mass bands of that level); other patches untouched
__global__ void k_regularize(const PatchDesc* pd, const double* K64, const double* tab, double alpha, double* KM64) {
    const PatchDesc& P = pd[blockIdx.y];
    if (!P.floating) return;
    for (int l = 0; l < P.L; ++l) {
        const LevelDesc& L = P.lev[l];
        long long total = (long long)L.n * L.S;
        for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
             t += (long long)gridDim.x * blockDim.x) {
            int i = (int)(t / L.S), o = (int)(t % L.S);
            int ii[3] = {i % L.m[0], (i / L.m[0]) % L.m[1], i / (L.m[0] * L.m[1])};
            long long pos = L.koff + ieti_val_pos(L.m, P.p, L.S, ii[0], ii[1], ii[2], o);
            int rem = o;
            double mm = 1.0;
            for (int r = 0; r < 3; ++r) {
                int w = 2 * P.p[r] + 1;
                int orr = rem % w;
                rem /= w;
                if (r < P.dim) mm *= tab[L.mw[r] + ii[r] * w + orr];
            }
            KM64[pos] = K64[pos] + alpha * mm;
        }
    }
}

__global__ void k_cweights(const PatchDesc* pd, const int* crow_ptr, const int* crow_patch,
                           const int* crow_tang, const int* c_idx, double* c_w) {
    int j = blockIdx.x;
    const PatchDesc& P = pd[crow_patch[j]];
    const LevelDesc& F = P.lev[P.L - 1];
    int b = crow_ptr[j], e = crow_ptr[j + 1];
    int tang = crow_tang[j];
    __shared__ double red[256];
    double part = 0.0;
    for (int t = b + threadIdx.x; t < e; t += blockDim.x) {
        int i = c_idx[t];
        int ii[3] = {i % F.m[0], (i / F.m[0]) % F.m[1], i / (F.m[0] * F.m[1])};
        double w = 1.0;
        for (int r = 0; r < P.dim; ++r)
            if (tang >> r & 1) {
                int p = P.p[r], n = P.nelem[r];
                w *= (knot(ii[r] + p + 1, n, p) - knot(ii[r], n, p)) / (p + 1);
            }
        c_w[t] = w;
        part += w;
    }
    red[threadIdx.x] = part;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    double tot = red[0];
    for (int t = b + threadIdx.x; t < e; t += blockDim.x) c_w[t] /= tot;
}

__global__ void k_to_f32(const double* s, float* d, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        d[i] = (float)s[i];
}

// lo = s - hi in FP32 (hi = FP32 rounding of s): hi + lo carries 48 bits of s
__global__ void k_lo_f32(const double* s, const float* hi, float* lo, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        lo[i] = (float)(s[i] - (double)hi[i]);
}

int grid_for(long long n, int threads, int cap = 152 * 32) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

}  // namespace

cudaError_t launch_assembly(const SetupArgs& a, long long total_qp, long long total_rows, int max_S,
                            cudaStream_t st) {
    k_asm_tables<<<dim3(64, a.npatch * 3), 128, 0, st>>>(a);
    IETI_CUDA_CHECK(cudaGetLastError());
    k_geometry<<<grid_for(total_qp, 256), 256, 0, st>>>(a, total_qp);
    IETI_CUDA_CHECK(cudaGetLastError());
    k_stiffness<<<dim3(grid_for(total_rows, 128, 4096), max_S), 128, 0, st>>>(a, total_rows);
    IETI_CUDA_CHECK(cudaGetLastError());
    k_load<<<grid_for(total_rows, 128), 128, 0, st>>>(a, total_rows);
    return cudaGetLastError();
}

cudaError_t launch_tables(const SetupArgs& a, const TableJob* jobs, int njobs, int max_m,
                          cudaStream_t st) {
    if (njobs == 0) return cudaSuccess;
    (void)max_m;
    k_prolong_rows<<<dim3(4, njobs), 128, 0, st>>>(a, jobs);
    IETI_CUDA_CHECK(cudaGetLastError());
    k_restrict_cols<<<dim3(4, njobs), 128, 0, st>>>(a, jobs);
    return cudaGetLastError();
}

cudaError_t launch_mass_tables(const SetupArgs& a, const TableJob* jobs, int njobs, cudaStream_t st) {
    if (njobs == 0) return cudaSuccess;
    k_mass1d<<<dim3(8, njobs), 128, 0, st>>>(a, jobs);
    return cudaGetLastError();
}

cudaError_t launch_galerkin(const PatchDesc* pd, const int* plist, int npl, int depth, int max_rows,
                            int max_S, double* K64, const double* tab, const int* itab, cudaStream_t st) {
    if (npl == 0) return cudaSuccess;
    dim3 g(grid_for(max_rows, 128, 1024), max_S, npl);
    k_galerkin<<<g, 128, 0, st>>>(pd, plist, depth, K64, tab, itab);
    return cudaGetLastError();
}

cudaError_t launch_coarse_inverse(const PatchDesc* pd, int npatch, const double* K64, const double* tab,
                                  double alpha, double* A0inv64, float* A0inv32, double* work, int max_n0,
                                  int* flags, cudaStream_t st) {
    k_coarse_inverse<<<npatch * 2, 256, 0, st>>>(pd, K64, tab, alpha, A0inv64, A0inv32, work, max_n0, flags);
    return cudaGetLastError();
}

cudaError_t launch_regularize(const PatchDesc* pd, int npatch, const double* K64, const double* tab, double alpha,
                              double* KM64, cudaStream_t st) {
    k_regularize<<<dim3(64, npatch), 256, 0, st>>>(pd, K64, tab, alpha, KM64);
    return cudaGetLastError();
}

cudaError_t launch_cweights(const PatchDesc* pd, int nrows, const int* crow_ptr, const int* crow_patch,
                            const int* crow_tang, const int* c_idx, double* c_w, cudaStream_t st) {
    if (nrows == 0) return cudaSuccess;
    k_cweights<<<nrows, 256, 0, st>>>(pd, crow_ptr, crow_patch, crow_tang, c_idx, c_w);
    return cudaGetLastError();
}

cudaError_t launch_to_f32(const double* s, float* d, long long n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_to_f32<<<grid_for(n, 256), 256, 0, st>>>(s, d, n);
    return cudaGetLastError();
}

cudaError_t launch_lo_f32(const double* s, const float* hi, float* lo, long long n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    k_lo_f32<<<grid_for(n, 256), 256, 0, st>>>(s, hi, lo, n);
    return cudaGetLastError();
}

cudaError_t launch_chol_linv(const double* A, int n, double* Linv, double* work, int* flags,
                             cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    IETI_CUDA_CHECK(cudaMemcpyAsync(work, A, sizeof(double) * n * n, cudaMemcpyDeviceToDevice, st));
    k_chol_linv<<<1, 512, 0, st>>>(work, n, Linv, flags);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// SZ basis: Hhat^{-1} = (0.99 H)^{-1}, H = C W with W = Khat^{-1} C^T (Sec. 3.2),
// one CTA per patch; Gauss-Jordan on the symmetrised SPD matrix (n_Pi^(k) <=
// 64) in dynamic shared memory (2 npi^2 doubles)
// ---------------------------------------------------------------------------
__global__ void k_sz_hinv(const PatchDesc* pd, const int* crow_ptr, const int* c_idx, const double* c_w,
                          const double* szW, double* szHinv, int* flags) {
    extern __shared__ double shm_sz[];
    const PatchDesc& P = pd[blockIdx.x];
    const int npi = P.npi, n = P.n;
    if (npi == 0) return;
    double* A = shm_sz;
    double* B = shm_sz + npi * npi;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const double* W = szW + P.phioff;
    for (int pr = w; pr < npi * npi; pr += nw) {
        const int i = pr / npi, j = pr % npi;
        const int row = P.crow0 + i;
        double d = 0.0;
        for (int e = crow_ptr[row] + lane; e < crow_ptr[row + 1]; e += 32) d += c_w[e] * W[(long long)j * n + c_idx[e]];
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) A[pr] = d;
    }
    __syncthreads();
    for (int pr = threadIdx.x; pr < npi * npi; pr += blockDim.x) {
        const int i = pr / npi, j = pr % npi;
        B[pr] = 0.99 * 0.5 * (A[pr] + A[j * npi + i]);
    }
    __syncthreads();
    for (int pr = threadIdx.x; pr < npi * npi; pr += blockDim.x) {
        A[pr] = B[pr];
        B[pr] = (pr / npi == pr % npi) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < npi; ++k) {
        const double piv = A[k * npi + k];
        if (!(piv > 0.0)) {
            if (threadIdx.x == 0) atomicOr(flags, IETI_FLAG_NOT_SPD);
            return;
        }
        __syncthreads();
        for (int c = threadIdx.x; c < npi; c += blockDim.x) {
            A[k * npi + c] /= piv;
            B[k * npi + c] /= piv;
        }
        __syncthreads();
        for (int pr = threadIdx.x; pr < npi * npi; pr += blockDim.x) {
            const int i = pr / npi, c = pr % npi;
            if (i == k) continue;
            const double f = A[i * npi + k];
            // column k of A is read by every row update: take it before it changes
            A[i * npi + c] -= (c == k ? 0.0 : f * A[k * npi + c]);
            B[i * npi + c] -= f * B[k * npi + c];
        }
        __syncthreads();
        for (int i = threadIdx.x; i < npi; i += blockDim.x)
            if (i != k) A[i * npi + k] = 0.0;
        __syncthreads();
    }
    double* out = szHinv + P.szhoff;
    for (int pr = threadIdx.x; pr < npi * npi; pr += blockDim.x) out[pr] = B[pr];
}

cudaError_t launch_sz_hinv(const PatchDesc* pd, int npatch, const int* crow_ptr, const int* c_idx,
                           const double* c_w, const double* szW, double* szHinv, int* flags, cudaStream_t st) {
    if (npatch == 0) return cudaSuccess;
    const size_t sm = sizeof(double) * 2 * 64 * 64;
    cudaError_t e = cudaFuncSetAttribute(k_sz_hinv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_sz_hinv<<<npatch, 256, sm, st>>>(pd, crow_ptr, c_idx, c_w, szW, szHinv, flags);
    return cudaGetLastError();
}
