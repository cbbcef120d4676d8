// Set-up of the high-order multigrid (Sec. 4, the setting of p >= 4): the
// finest level keeps the patch space; below it the degree-1 spaces on the
// dyadic grids from n/2 elements down (their hierarchy is the standard one of
// a companion problem with degree 1 and half the elements on every patch,
// set up as a handle of its own); between the finest level and the first
// degree-1 level the L2 projection in the parameter domain; on the finest
// level a subspace-corrected mass smoother (after Hofreither and Takacs,
// SIAM J. Numer. Anal. 55, 2017) with a rank-one approximation of the
// geometry, applied by fast diagonalization.
//
// Per patch and hierarchy kind (Neumann: Dirichlet sides masked; Dirichlet:
// every side masked) and per direction r this file computes, in FP64 on the
// host (1D problems of n_r + p_r unknowns):
//  * the free functions of direction r (first/last removed on masked ends);
//  * S~_r: the splines whose derivatives of the orders the end leaves free
//    (odd orders < p at an unmasked end, even orders 2..p-1 at a masked end)
//    vanish, and its mass-orthogonal complement S_G;
//  * Khat_r = sigma h^-2 M on S~_r plus the stiffness on S_G (no coupling),
//    with the 1D mass and stiffness weighted by the cross approximation of
//    the pulled-back coefficient |det J| J^-1 J^-T through the patch centre;
//  * the generalized eigenvectors U_r (U^T M U = I) and eigenvalues of
//    (Khat_r, M_r), and 1 / (sum_r c_r lambda_r + alpha c_M) on the tensor grid;
//  * the 1D L2-projection prolongation P_r = M_r^-1 M_{fc,r} from the free
//    degree-1 functions on n_r / 2 elements.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "host_internal.h"

using ieti_host::fail;

namespace {

constexpr double kSigma = 12.0;

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on the Legendre
// recurrence)
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) p1 = z, p0 = 1.0;
            double dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        double dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// open uniform knots of n elements, degree p
std::vector<double> knots(int n, int p) {
    std::vector<double> t;
    for (int i = 0; i <= p; ++i) t.push_back(0.0);
    for (int i = 1; i < n; ++i) t.push_back((double)i / n);
    for (int i = 0; i <= p; ++i) t.push_back(1.0);
    return t;
}

// values and first derivatives of all n + p basis functions at x (Cox-de Boor)
void basis_all(int n, int p, double x, std::vector<double>& N, std::vector<double>& dN) {
    const std::vector<double> t = knots(n, p);
    const int m = n + p, nk = (int)t.size();
    std::vector<double> cur(nk - 1, 0.0);
    int last = 0;
    for (int i = 0; i < nk - 1; ++i)
        if (t[i] < t[i + 1]) last = i;
    for (int i = 0; i < nk - 1; ++i)
        if (t[i] < t[i + 1] && ((x >= t[i] && x < t[i + 1]) || (i == last && x == t[i + 1]))) cur[i] = 1.0;
    std::vector<double> prev;
    for (int q = 1; q <= p; ++q) {
        prev = cur;
        cur.assign(nk - 1 - q, 0.0);
        for (int i = 0; i < nk - 1 - q; ++i) {
            double d1 = t[i + q] - t[i], d2 = t[i + q + 1] - t[i + 1];
            if (d1 > 0) cur[i] += (x - t[i]) / d1 * prev[i];
            if (d2 > 0) cur[i] += (t[i + q + 1] - x) / d2 * prev[i + 1];
        }
    }
    N.assign(cur.begin(), cur.begin() + m);
    dN.assign(m, 0.0);
    if (p > 0)
        for (int i = 0; i < m; ++i) {
            double d1 = t[i + p] - t[i], d2 = t[i + p + 1] - t[i + 1];
            if (d1 > 0) dN[i] += p / d1 * prev[i];
            if (d2 > 0) dN[i] -= p / d2 * prev[i + 1];
        }
}

// ---- small dense linear algebra (row-major n x n) --------------------------
bool cholesky(std::vector<double>& A, int n) {   // lower factor in place
    for (int j = 0; j < n; ++j) {
        double s = A[j * n + j];
        for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0.0)) return false;
        s = std::sqrt(s);
        A[j * n + j] = s;
        for (int i = j + 1; i < n; ++i) {
            double v = A[i * n + j];
            for (int k = 0; k < j; ++k) v -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = v / s;
        }
        for (int k = j + 1; k < n; ++k) A[j * n + k] = 0.0;
    }
    return true;
}
// B <- L^-1 B (B: n x c row-major)
void lsolve(const std::vector<double>& L, int n, std::vector<double>& B, int c) {
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < c; ++j) {
            double v = B[i * c + j];
            for (int k = 0; k < i; ++k) v -= L[i * n + k] * B[k * c + j];
            B[i * c + j] = v / L[i * n + i];
        }
}
// B <- L^-T B
void ltsolve(const std::vector<double>& L, int n, std::vector<double>& B, int c) {
    for (int i = n - 1; i >= 0; --i)
        for (int j = 0; j < c; ++j) {
            double v = B[i * c + j];
            for (int k = i + 1; k < n; ++k) v -= L[k * n + i] * B[k * c + j];
            B[i * c + j] = v / L[i * n + i];
        }
}
// symmetric eigen-decomposition by cyclic Jacobi rotations: A = V diag(e) V^T
void jacobi_eigen(std::vector<double> A, int n, std::vector<double>& e, std::vector<double>& V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                tot += A[i * n + j] * A[i * n + j];
                if (i != j) off += A[i * n + j] * A[i * n + j];
            }
        if (off <= 1e-30 * tot) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                const double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {
                    const double akp = A[k * n + p], akq = A[k * n + q];
                    A[k * n + p] = c * akp - s * akq;
                    A[k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = A[p * n + k], aqk = A[q * n + k];
                    A[p * n + k] = c * apk - s * aqk;
                    A[q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[k * n + p], vkq = V[k * n + q];
                    V[k * n + p] = c * vkp - s * vkq;
                    V[k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    e.resize(n);
    for (int i = 0; i < n; ++i) e[i] = A[i * n + i];
}

// orthonormal basis of the null space of C (q x m, q < m) by Householder QR
// of C^T: the last m - q columns of Q (m x (m - q), row-major)
std::vector<double> null_space(const std::vector<double>& C, int q, int m) {
    std::vector<double> Q((size_t)m * m, 0.0);
    for (int i = 0; i < m; ++i) Q[i * m + i] = 1.0;
    std::vector<double> R((size_t)m * q);   // C^T
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < m; ++j) R[j * q + i] = C[i * m + j];
    for (int k = 0; k < q; ++k) {
        double nrm = 0.0;
        for (int i = k; i < m; ++i) nrm += R[i * q + k] * R[i * q + k];
        nrm = std::sqrt(nrm);
        if (nrm == 0.0) continue;
        std::vector<double> v(m, 0.0);
        const double alpha = R[k * q + k] > 0 ? -nrm : nrm;
        for (int i = k; i < m; ++i) v[i] = R[i * q + k];
        v[k] -= alpha;
        double vv = 0.0;
        for (int i = k; i < m; ++i) vv += v[i] * v[i];
        if (vv == 0.0) continue;
        for (int j = 0; j < q; ++j) {
            double s = 0.0;
            for (int i = k; i < m; ++i) s += v[i] * R[i * q + j];
            s *= 2.0 / vv;
            for (int i = k; i < m; ++i) R[i * q + j] -= s * v[i];
        }
        for (int j = 0; j < m; ++j) {   // Q <- Q H
            double s = 0.0;
            for (int i = k; i < m; ++i) s += Q[j * m + i] * v[i];
            s *= 2.0 / vv;
            for (int i = k; i < m; ++i) Q[j * m + i] -= s * v[i];
        }
    }
    std::vector<double> Z((size_t)m * (m - q));
    for (int i = 0; i < m; ++i)
        for (int j = q; j < m; ++j) Z[i * (m - q) + (j - q)] = Q[i * m + j];
    return Z;
}

// derivatives of orders 1..p-1 of all basis functions at the end x = 0
// (end 0) or x = 1 (end 1): on the end element each function is a polynomial
// of degree p; its values at p + 1 points give its monomial coefficients
std::vector<std::vector<double>> end_derivs(int n, int p, int end) {
    const double a = end == 0 ? 0.0 : 1.0 - 1.0 / n, b = a + 1.0 / n;
    const int m = n + p;
    std::vector<double> V((size_t)(p + 1) * (p + 1)), vals((size_t)(p + 1) * m);
    for (int i = 0; i <= p; ++i) {
        const double tt = 0.5 - 0.5 * std::cos(M_PI * (i + 0.5) / (p + 1));
        std::vector<double> N, dN;
        basis_all(n, p, a + (b - a) * tt, N, dN);
        for (int j = 0; j <= p; ++j) V[i * (p + 1) + j] = std::pow(tt, j);
        for (int f = 0; f < m; ++f) vals[i * m + f] = N[f];
    }
    // solve V coef = vals by Gaussian elimination with partial pivoting
    const int np = p + 1;
    for (int c = 0; c < np; ++c) {
        int piv = c;
        for (int r = c + 1; r < np; ++r)
            if (std::fabs(V[r * np + c]) > std::fabs(V[piv * np + c])) piv = r;
        if (piv != c) {
            for (int j = 0; j < np; ++j) std::swap(V[c * np + j], V[piv * np + j]);
            for (int f = 0; f < m; ++f) std::swap(vals[c * m + f], vals[piv * m + f]);
        }
        for (int r = c + 1; r < np; ++r) {
            const double l = V[r * np + c] / V[c * np + c];
            for (int j = c; j < np; ++j) V[r * np + j] -= l * V[c * np + j];
            for (int f = 0; f < m; ++f) vals[r * m + f] -= l * vals[c * m + f];
        }
    }
    for (int c = np - 1; c >= 0; --c) {
        for (int f = 0; f < m; ++f) {
            double v = vals[c * m + f];
            for (int j = c + 1; j < np; ++j) v -= V[c * np + j] * vals[j * m + f];
            vals[c * m + f] = v / V[c * np + c];
        }
    }
    const double t0 = end == 0 ? 0.0 : 1.0;
    std::vector<std::vector<double>> out(p + 1, std::vector<double>(m, 0.0));
    for (int k = 1; k < p; ++k)
        for (int f = 0; f < m; ++f) {
            double d = 0.0;
            for (int j = k; j <= p; ++j) {
                double fac = 1.0;
                for (int i = j - k + 1; i <= j; ++i) fac *= i;
                d += vals[j * m + f] * fac * std::pow(t0, j - k);
            }
            out[k][f] = d / std::pow(b - a, k);
        }
    return out;
}

// diagonal of |det J| J^-1 J^-T of a patch at parameter xi
void coeff_diag(const iga_patch_desc& g, int d, const double* xi, double* A) {
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    if (g.geo_kind == IGA_GEO_BOX) {
        for (int r = 0; r < d; ++r) J[r][r] = g.hi[r] - g.lo[r];
    } else {
        const double w1 = 0.70710678118654752440;
        const double h0 = g.hi[0] - g.lo[0], h1 = g.hi[1] - g.lo[1];
        const double t = g.lo[0] + h0 * xi[0], s2 = g.lo[1] + h1 * xi[1];
        const double b0 = (1 - t) * (1 - t), b1 = 2 * t * (1 - t), b2 = t * t;
        const double d0 = -2 * (1 - t), d1 = 2 - 4 * t, d2 = 2 * t;
        const double W = b0 + w1 * b1 + b2, dW = d0 + w1 * d1 + d2;
        const double Nx = b0 + w1 * b1, Ny = w1 * b1 + b2, dNx = d0 + w1 * d1, dNy = w1 * d1 + d2;
        const double cx = Nx / W, cy = Ny / W;
        const double dcx = (dNx * W - Nx * dW) / (W * W), dcy = (dNy * W - Ny * dW) / (W * W);
        const double rad = 1.0 + s2;
        J[0][0] = rad * dcx * h0;
        J[1][0] = rad * dcy * h0;
        J[0][1] = cx * h1;
        J[1][1] = cy * h1;
    }
    if (d == 2) {
        const double det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        const double i00 = J[1][1] / det, i01 = -J[0][1] / det, i10 = -J[1][0] / det, i11 = J[0][0] / det;
        A[0] = std::fabs(det) * (i00 * i00 + i01 * i01);
        A[1] = std::fabs(det) * (i10 * i10 + i11 * i11);
    } else {   // boxes only in 3D
        const double det = J[0][0] * J[1][1] * J[2][2];
        for (int r = 0; r < 3; ++r) A[r] = std::fabs(det) / (J[r][r] * J[r][r]);
    }
}

struct Dir1D {
    std::vector<double> U;     // nf x nf, U[j + nf i] = eigenvector i at function j
    std::vector<double> lam;
    std::vector<double> P;     // nf x nc, P[j + nf c]
    int nf = 0, lof = 0, nc = 0, loc = 0;
    double c = 1.0;
};

}  // namespace

// HoDesc / pools for every patch; returns IETIDP_OK or an error code
int ieti_ho_build(const iga_problem* Pb, const std::vector<PatchDesc>& pd, double alpha,
                  std::vector<HoDesc>& desc, std::vector<double>& pool) {
    const int d = Pb->dim, N = Pb->npatch;
    desc.assign(N, HoDesc{});
    pool.clear();
    for (int k = 0; k < N; ++k) {
        const iga_patch_desc& g = Pb->patches[k];
        if (d == 3 && g.geo_kind != IGA_GEO_BOX) return fail(IETIDP_E_INVALID_ARG, "high-order multigrid: 3D patches must be boxes");
        HoDesc& H = desc[k];
        // rank-one cross approximation of the coefficient's diagonal through
        // the centre: om[r][s](x) = A_rr(centre with xi_s = x) / A_rr(centre)^((d-1)/d)
        double ctr[3] = {0.5, 0.5, 0.5}, Ac[3];
        coeff_diag(g, d, ctr, Ac);
        std::vector<std::vector<double>> gx(d), gw(d);
        for (int s = 0; s < d; ++s) {
            const int n = g.nelem[s], p = g.degree[s];
            std::vector<double> z, w;
            gauss_legendre(p + 1, z, w);
            for (int e = 0; e < n; ++e)
                for (int q = 0; q <= p; ++q) {
                    gx[s].push_back((e + 0.5 * (z[q] + 1.0)) / n);
                    gw[s].push_back(0.5 * w[q] / n);
                }
        }
        auto om = [&](int r, int s, double x) {
            double xi[3] = {0.5, 0.5, 0.5}, A[3];
            xi[s] = x;
            coeff_diag(g, d, xi, A);
            return A[r] / std::pow(Ac[r], (double)(d - 1) / d);
        };
        auto massw = [&](int s, double x) {
            double v = 1.0;
            for (int r = 0; r < d; ++r)
                if (r != s) v *= om(r, s, x);
            return std::pow(v, 1.0 / (d - 1));
        };
        for (int kind = 0; kind < 2; ++kind) {
            const int mask = kind == 0 ? Pb->dmask[k] : (d == 2 ? 0xF : 0x3F);
            const double al = (kind == 0 && Pb->dmask[k] == 0) ? alpha : 0.0;
            Dir1D D1[3];
            double cM = 1.0;
            for (int r = 0; r < d; ++r) {
                const int n = g.nelem[r], p = g.degree[r], m = n + p;
                const bool lo = mask >> (2 * r) & 1, hi = mask >> (2 * r + 1) & 1;
                Dir1D& D = D1[r];
                D.lof = lo ? 1 : 0;
                D.nf = m - (lo ? 1 : 0) - (hi ? 1 : 0);
                // weighted 1D mass (common direction weight) and stiffness (own weight)
                std::vector<double> M((size_t)m * m, 0.0), K((size_t)m * m, 0.0);
                double wm = 0.0, wsum = 0.0;
                for (size_t q = 0; q < gx[r].size(); ++q) {
                    std::vector<double> Nv, dNv;
                    basis_all(n, p, gx[r][q], Nv, dNv);
                    const double mw = massw(r, gx[r][q]) * gw[r][q], kw = om(r, r, gx[r][q]) * gw[r][q];
                    wm += massw(r, gx[r][q]);
                    wsum += 1.0;
                    for (int i = 0; i < m; ++i)
                        for (int j = 0; j < m; ++j) {
                            M[i * m + j] += mw * Nv[i] * Nv[j];
                            K[i * m + j] += kw * dNv[i] * dNv[j];
                        }
                }
                cM /= wm / wsum;   // arithmetic mean over the Gauss points
                // c_r: mean over the other directions of prod om(r,s)/massw(s)
                D.c = 1.0;
                for (int s = 0; s < d; ++s) {
                    if (s == r) continue;
                    double acc = 0.0;
                    for (size_t q = 0; q < gx[s].size(); ++q) acc += om(r, s, gx[s][q]) / massw(s, gx[s][q]);
                    D.c *= acc / gx[s].size();
                }
                const int nf = D.nf;
                std::vector<double> Mf((size_t)nf * nf), Kf((size_t)nf * nf);
                for (int i = 0; i < nf; ++i)
                    for (int j = 0; j < nf; ++j) {
                        Mf[i * nf + j] = M[(i + D.lof) * m + (j + D.lof)];
                        Kf[i * nf + j] = K[(i + D.lof) * m + (j + D.lof)];
                    }
                // constraints of S~ over the free functions
                std::vector<double> C;
                int q = 0;
                for (int end = 0; end < 2; ++end) {
                    const bool dir = end == 0 ? lo : hi;
                    auto der = end_derivs(n, p, end);
                    for (int kk = 1; kk < p; ++kk)
                        if ((kk % 2 == 0) == dir) {
                            for (int j = 0; j < nf; ++j) C.push_back(der[kk][j + D.lof]);
                            ++q;
                        }
                }
                // M-orthogonal projector onto S~ = ker C: Pt = Z (Z^T M Z)^-1 Z^T M
                std::vector<double> Pt((size_t)nf * nf, 0.0);
                if (q == 0) {
                    for (int i = 0; i < nf; ++i) Pt[i * nf + i] = 1.0;
                } else {
                    const int nz = nf - q;
                    std::vector<double> Z = null_space(C, q, nf);   // nf x nz
                    std::vector<double> MZ((size_t)nf * nz, 0.0), ZMZ((size_t)nz * nz, 0.0);
                    for (int i = 0; i < nf; ++i)
                        for (int j = 0; j < nz; ++j) {
                            double s = 0.0;
                            for (int l = 0; l < nf; ++l) s += Mf[i * nf + l] * Z[l * nz + j];
                            MZ[i * nz + j] = s;
                        }
                    for (int i = 0; i < nz; ++i)
                        for (int j = 0; j < nz; ++j) {
                            double s = 0.0;
                            for (int l = 0; l < nf; ++l) s += Z[l * nz + i] * MZ[l * nz + j];
                            ZMZ[i * nz + j] = s;
                        }
                    if (!cholesky(ZMZ, nz)) return fail(IETIDP_E_BREAKDOWN, "high-order multigrid: subspace mass not SPD");
                    // Y = (Z^T M Z)^-1 (M Z)^T  (nz x nf)
                    std::vector<double> Y((size_t)nz * nf);
                    for (int i = 0; i < nz; ++i)
                        for (int j = 0; j < nf; ++j) Y[i * nf + j] = MZ[j * nz + i];
                    lsolve(ZMZ, nz, Y, nf);
                    ltsolve(ZMZ, nz, Y, nf);
                    for (int i = 0; i < nf; ++i)
                        for (int j = 0; j < nf; ++j) {
                            double s = 0.0;
                            for (int l = 0; l < nz; ++l) s += Z[i * nz + l] * Y[l * nf + j];
                            Pt[i * nf + j] = s;
                        }
                }
                // Khat = sigma h^-2 Pt^T M Pt + Pg^T K Pg, Pg = I - Pt
                std::vector<double> Pg(Pt);
                for (int i = 0; i < nf * nf; ++i) Pg[i] = -Pg[i];
                for (int i = 0; i < nf; ++i) Pg[i * nf + i] += 1.0;
                auto sandwich = [&](const std::vector<double>& X, const std::vector<double>& A) {
                    std::vector<double> AX((size_t)nf * nf, 0.0), out((size_t)nf * nf, 0.0);
                    for (int i = 0; i < nf; ++i)
                        for (int j = 0; j < nf; ++j) {
                            double s = 0.0;
                            for (int l = 0; l < nf; ++l) s += A[i * nf + l] * X[l * nf + j];
                            AX[i * nf + j] = s;
                        }
                    for (int i = 0; i < nf; ++i)
                        for (int j = 0; j < nf; ++j) {
                            double s = 0.0;
                            for (int l = 0; l < nf; ++l) s += X[l * nf + i] * AX[l * nf + j];
                            out[i * nf + j] = s;
                        }
                    return out;
                };
                const double hsc = kSigma * (double)n * n;
                std::vector<double> Kh = sandwich(Pt, Mf), KG = sandwich(Pg, Kf);
                for (int i = 0; i < nf * nf; ++i) Kh[i] = hsc * Kh[i] + KG[i];
                // generalized eigen-decomposition of (Kh, Mf): Mf = L L^T,
                // L^-1 Kh L^-T = V diag V^T, U = L^-T V
                std::vector<double> L(Mf);
                if (!cholesky(L, nf)) return fail(IETIDP_E_BREAKDOWN, "high-order multigrid: 1D mass not SPD");
                std::vector<double> T(Kh);
                lsolve(L, nf, T, nf);                 // L^-1 Kh
                std::vector<double> Tt((size_t)nf * nf);
                for (int i = 0; i < nf; ++i)
                    for (int j = 0; j < nf; ++j) Tt[i * nf + j] = T[j * nf + i];
                lsolve(L, nf, Tt, nf);                // L^-1 (L^-1 Kh)^T = L^-1 Kh L^-T
                for (int i = 0; i < nf; ++i)
                    for (int j = 0; j < i; ++j) {
                        const double v = 0.5 * (Tt[i * nf + j] + Tt[j * nf + i]);
                        Tt[i * nf + j] = Tt[j * nf + i] = v;
                    }
                std::vector<double> V;
                jacobi_eigen(Tt, nf, D.lam, V);
                ltsolve(L, nf, V, nf);                // U = L^-T V (row j = function, column i = eigenvector)
                D.U.assign((size_t)nf * nf, 0.0);
                for (int j = 0; j < nf; ++j)
                    for (int i = 0; i < nf; ++i) D.U[j + (size_t)nf * i] = V[j * nf + i];
                // L2-projection prolongation from degree 1 on n/2 elements
                const int nc_el = std::max(1, n / 2), mc = nc_el + 1;
                D.loc = lo ? 1 : 0;
                D.nc = mc - (lo ? 1 : 0) - (hi ? 1 : 0);
                std::vector<double> z, w;
                gauss_legendre(std::max(p, 1) + 1, z, w);
                std::vector<double> Mfull((size_t)m * m, 0.0), Mfc((size_t)m * mc, 0.0);
                for (int e = 0; e < n; ++e)
                    for (size_t qq = 0; qq < z.size(); ++qq) {
                        const double x = (e + 0.5 * (z[qq] + 1.0)) / n, ww = 0.5 * w[qq] / n;
                        std::vector<double> Nf, dNf, Nc, dNc;
                        basis_all(n, p, x, Nf, dNf);
                        basis_all(nc_el, 1, x, Nc, dNc);
                        for (int i = 0; i < m; ++i) {
                            for (int j = 0; j < m; ++j) Mfull[i * m + j] += ww * Nf[i] * Nf[j];
                            for (int j = 0; j < mc; ++j) Mfc[i * mc + j] += ww * Nf[i] * Nc[j];
                        }
                    }
                std::vector<double> Lm((size_t)nf * nf), B((size_t)nf * D.nc);
                for (int i = 0; i < nf; ++i) {
                    for (int j = 0; j < nf; ++j) Lm[i * nf + j] = Mfull[(i + D.lof) * m + (j + D.lof)];
                    for (int j = 0; j < D.nc; ++j) B[i * D.nc + j] = Mfc[(i + D.lof) * mc + (j + D.loc)];
                }
                if (!cholesky(Lm, nf)) return fail(IETIDP_E_BREAKDOWN, "high-order multigrid: mass not SPD");
                lsolve(Lm, nf, B, D.nc);
                ltsolve(Lm, nf, B, D.nc);
                D.P.assign((size_t)nf * D.nc, 0.0);
                for (int j = 0; j < nf; ++j)
                    for (int c = 0; c < D.nc; ++c) D.P[j + (size_t)nf * c] = B[j * D.nc + c];
            }
            // descriptor and pool entries
            for (int r = 0; r < 3; ++r) {
                H.nf[kind][r] = r < d ? D1[r].nf : 1;
                H.lof[kind][r] = r < d ? D1[r].lof : 0;
                H.nc[kind][r] = r < d ? D1[r].nc : 1;
                H.loc[kind][r] = r < d ? D1[r].loc : 0;
            }
            for (int r = 0; r < d; ++r) {
                H.u[kind][r] = (long long)pool.size();
                pool.insert(pool.end(), D1[r].U.begin(), D1[r].U.end());
                H.pt[kind][r] = (long long)pool.size();
                pool.insert(pool.end(), D1[r].P.begin(), D1[r].P.end());
            }
            H.dinv[kind] = (long long)pool.size();
            const int n0 = H.nf[kind][0], n1 = H.nf[kind][1], n2 = H.nf[kind][2];
            for (int i2 = 0; i2 < n2; ++i2)
                for (int i1 = 0; i1 < n1; ++i1)
                    for (int i0 = 0; i0 < n0; ++i0) {
                        double s = D1[0].c * D1[0].lam[i0] + D1[1].c * D1[1].lam[i1];
                        if (d == 3) s += D1[2].c * D1[2].lam[i2];
                        if (al != 0.0) s += al * cM;
                        pool.push_back(1.0 / s);
                    }
            while (pool.size() % 4) pool.push_back(0.0);
        }
    }
    return IETIDP_OK;
}

// one patch's operators on the host, for inspection and tests (no device work)
extern "C" int ietidp_ho_patch_operators(int dim, const iga_patch_desc* patch, unsigned dmask, double alpha,
                                         int kind, int* sizes, double* U, double* P, double* Dinv) {
    if (!patch || !sizes || (dim != 2 && dim != 3) || (kind != 0 && kind != 1) || alpha < 0)
        return fail(IETIDP_E_INVALID_ARG, "bad argument");
    for (int r = 0; r < dim; ++r)
        if (patch->degree[r] < 1 || patch->degree[r] > IETI_MAXP - 1 || patch->nelem[r] < 1)
            return fail(IETIDP_E_INVALID_ARG, "bad degree or element count");
    iga_problem Pb;
    Pb.dim = dim;
    Pb.npatch = 1;
    Pb.patches.assign(1, *patch);
    Pb.dmask.assign(1, (int)dmask);
    std::vector<PatchDesc> pd(1);
    std::memset(pd.data(), 0, sizeof(PatchDesc));
    std::vector<HoDesc> desc;
    std::vector<double> pool;
    const int rc = ieti_ho_build(&Pb, pd, alpha, desc, pool);
    if (rc != IETIDP_OK) return rc;
    const HoDesc& H = desc[0];
    long long nu = 0, np = 0, nd = 1;
    for (int r = 0; r < 3; ++r) {
        sizes[r] = H.nf[kind][r];
        sizes[3 + r] = H.nc[kind][r];
        nd *= H.nf[kind][r];
    }
    for (int r = 0; r < dim; ++r) {
        const long long nf = H.nf[kind][r], nc = H.nc[kind][r];
        if (U) std::copy(pool.begin() + H.u[kind][r], pool.begin() + H.u[kind][r] + nf * nf, U + nu);
        if (P) std::copy(pool.begin() + H.pt[kind][r], pool.begin() + H.pt[kind][r] + nf * nc, P + np);
        nu += nf * nf;
        np += nf * nc;
    }
    if (Dinv) std::copy(pool.begin() + H.dinv[kind], pool.begin() + H.dinv[kind] + nd, Dinv);
    return IETIDP_OK;
}
