"""High-order multigrid for one patch (Sec. 4, the setting with p >= 4).

ORACLE (test infrastructure only).  Plain FP64 numpy/scipy.

Sec. 4 describes the multigrid used for the higher degrees only in words:
degree 1 on every grid level but the finest, L2 projections as transfers
between the finest space and the degree-1 space below it (the spaces are not
nested), and on the finest level a variant of the subspace-corrected mass
smoother of Hofreither and Takacs (Robust multigrid for isogeometric
analysis based on stable splittings of spline spaces, SIAM J. Numer. Anal.
55, 2017) that includes a rank-one approximation of the geometry; standard
Gauss-Seidel on the other levels.  Readings (the paper gives no more):

* levels: the finest level is the patch space (degree p, n elements per
  direction); below it the degree-1 spaces on the usual dyadic grids, the
  first of them on n/2 elements; the degree-1 levels form the Galerkin
  hierarchy of the degree-1 stiffness re-assembled on n/2 elements with the
  patch geometry (same quadrature rule as the fine level), down to 4
  elements, smoothed by the multicolor Gauss-Seidel of oracle.multigrid
  (2^d colors) and solved densely on the coarsest level;
* transfers between the finest and the first degree-1 level: prolongation
  P = (x)_r M_r^{-1} M_{fc,r}, the L2 projection in the parameter domain onto
  the finest space (M_r the 1D mass of the finest space, M_{fc,r} the mixed
  mass of finest and coarse basis), restriction P^T; Dirichlet sides are
  removed from both spaces before the projection;
* smoother on the finest level: x <- x + L^{-1} (b - A x), nu steps before
  and after the coarse correction, with L a Kronecker sum of 1D operators,
      L = sum_r c_r Khat_r (x) (x)_{s != r} M_s  (+ alpha c_M (x)_s M_s),
  inverted by fast diagonalization (generalized eigenvectors of the 1D
  pencils (Khat_r, M_r)).  Per direction the space splits M-orthogonally
  into the splines whose derivatives of the orders the boundary leaves free
  (odd orders below p at a Neumann end, even orders 2..p-1 at a Dirichlet
  end) vanish at both ends, S~, and its complement S_G of dimension at most
  p; Khat_r is sigma h^-2 M_r on S~ (the robust inverse inequality of that
  subspace bounds |u|_1^2 by 12 h^-2 ||u||^2) and the stiffness itself on
  S_G, with no coupling between the two;
* rank-one geometry: the pulled-back coefficient of Eq. 1, A(xi) = |det J|
  J^-1 J^-T, is replaced by its diagonal, each entry A_rr by the cross
  approximation prod_s omega_rs(xi_s) through the patch centre; direction
  r's stiffness is weighted by omega_rr, the mass of direction s by the
  geometric mean omega_s of omega_rs over r != s, and c_r is the mean of
  prod_{s != r} omega_rs / omega_s (1 in 2D); on floating patches the
  regularising parameter mass alpha M^ enters with c_M = 1 / prod_s
  mean(omega_s);
* sigma = 12, nu = 2 (pins below; the V-cycle contraction was measured for
  sigma in {6, 12, 24}).

Pins (tests/test_oracle_highorder.py): the splines of S~ have vanishing end
derivatives of the stated orders (by finite differences of the spline) and
satisfy the robust inverse inequality |u|_1^2 <= 12 h^-2 ||u||^2 for p = 2..7
while the full space does not; Khat equals sigma h^-2 M on S~, the
stiffness on the complement, with no coupling; the transfer maps the
degree-1 coefficients of a linear function to its degree-p coefficients
(Greville values); the cross approximation reproduces A_rr on the lines
through the patch centre and is exact for affine maps; the V-cycle is
symmetric and contracts at a rate bounded independently of p (2..7) and h
on the unit square and on the annulus, on floating and Dirichlet patches;
IETI-DP with these V-cycles equals the global direct solve.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import assembly, geometry, splines
from .multigrid import Hierarchy, MGOperator

SIGMA = 12.0
NU = 2


def _poly_derivs_at(knots, p, end, orders):
    """Derivatives of the given orders of every basis function at x = 0 (end
    0) or x = 1 (end 1): each function is a polynomial of degree p on the end
    element, fitted exactly from p + 1 values there and differentiated."""
    a, b = (knots[p], knots[p + 1]) if end == 0 else (knots[-p - 2], knots[-p - 1])
    xs = a + (b - a) * (0.5 - 0.5 * np.cos(np.pi * (np.arange(p + 1) + 0.5) / (p + 1)))
    vals = splines.basis_funs(knots, p, xs)                     # (p+1, m)
    t = (xs - a) / (b - a)
    V = np.vander(t, p + 1, increasing=True)                    # polynomial in t
    coef = np.linalg.solve(V, vals)                             # (p+1, m)
    x0 = 0.0 if end == 0 else 1.0
    out = []
    for k in orders:
        d = np.zeros(vals.shape[1])
        for j in range(k, p + 1):
            fac = np.prod(np.arange(j - k + 1, j + 1))
            d += coef[j] * fac * x0 ** (j - k)
        out.append(d / (b - a) ** k)
    return np.array(out).reshape(len(orders), -1)


def split_1d(n, p, lo_dir, hi_dir):
    """Constraint rows whose kernel is S~ for one direction: derivative
    functionals at both ends, over the free functions (Dirichlet ends'
    first/last function removed).  Returns (C, free index list)."""
    knots = splines.open_uniform_knots(n, p)
    m = n + p
    free = np.arange(m)
    if lo_dir:
        free = free[1:]
    if hi_dir:
        free = free[:-1]
    rows = []
    for end, dirichlet in ((0, lo_dir), (1, hi_dir)):
        orders = [k for k in range(1, p) if (k % 2 == 0) == dirichlet]
        if orders:
            D = _poly_derivs_at(knots, p, end, orders)
            rows.extend(D[:, free])
    C = np.array(rows) if rows else np.zeros((0, len(free)))
    return C, free


def weighted_1d(n, p, weight):
    """1D mass and stiffness of S_{p,n}(0,1) with a weight function, by the
    Gauss rule of the assembly (p+1 points per element)."""
    x, w = splines.gauss_points(n, p + 1)
    B, D = splines.basis_funs(splines.open_uniform_knots(n, p), p, x, deriv=True)
    om = weight(x)
    return B.T @ ((w * om)[:, None] * B), D.T @ ((w * om)[:, None] * D)


def khat_1d(n, p, free, C, Mw, Kw, sigma):
    """Modified 1D stiffness on the free functions: sigma h^-2 M on S~ = ker C,
    the stiffness on the M-orthogonal complement, no coupling."""
    M = Mw[np.ix_(free, free)]
    K = Kw[np.ix_(free, free)]
    if C.shape[0] == 0:
        Pt = np.eye(len(free))
    else:
        Z = sla.null_space(C)
        Pt = Z @ np.linalg.solve(Z.T @ M @ Z, Z.T @ M)         # M-orthogonal projector onto S~
    Pg = np.eye(len(free)) - Pt
    h = 1.0 / n
    return sigma / h ** 2 * (Pt.T @ M @ Pt) + Pg.T @ K @ Pg, M


def rank_one_weights(dom, k, npts=None):
    """Cross approximation of the diagonal of A(xi) = |det J| J^-1 J^-T through
    the patch centre: omega[r][s] is a callable of xi_s with
    A_rr(xi) ~ prod_s omega[r][s](xi_s)."""
    d = dom.dim
    centre = np.full(d, 0.5)

    def arr(xi):
        _, J = geometry.patch_map(dom, k, xi)
        Ji = np.linalg.inv(J)
        A = np.einsum("qac,qbc->qab", Ji, Ji) * np.abs(np.linalg.det(J))[:, None, None]
        return A

    a_c = np.diag(arr(centre[None, :])[0])
    om = []
    for r in range(d):
        row = []
        for s in range(d):
            def f(x, r=r, s=s):
                xi = np.tile(centre, (len(x), 1))
                xi[:, s] = x
                return arr(xi)[:, r, r] / a_c[r] ** ((d - 1) / d)
            row.append(f)
        om.append(row)
    return om


class HighOrderMG:
    """V-cycle preconditioner for (K + alpha M^) of patch k restricted to the
    unmasked dofs, with the hierarchy and smoother described above."""

    def __init__(self, dom, k, K_fine, side_mask, alpha=0.0, sigma=SIGMA, nu=NU, cmin=4):
        d = dom.dim
        self.d = d
        self.nu = nu
        self.deg = dom.patch_degree(k)
        self.nel = dom.patch_nelem(k)
        self.alpha = alpha
        from .multigrid import free_mask
        m = tuple(n + p for n, p in zip(self.nel, self.deg))
        self.free = np.nonzero(free_mask(m, side_mask))[0]
        A = sp.csr_matrix(K_fine)
        if alpha:
            A = A + alpha * assembly._kron_all([sp.csr_matrix(splines.mass_1d(n, p))
                                                for n, p in zip(self.nel, self.deg)])
        self.Af = sp.csr_matrix(A[self.free][:, self.free])
        self.A = [self.Af]          # finest operator last, as in multigrid.MGOperator
        # ---- smoother: 1D pencils per direction
        om = rank_one_weights(dom, k)
        self.U, self.lam, self.c = [], [], []
        mass_w = []
        for s in range(d):
            others = [r for r in range(d) if r != s]
            mass_w.append(lambda x, s=s, others=others:
                          np.prod([om[r][s](x) for r in others], axis=0) ** (1.0 / len(others)))
        xs = [splines.gauss_points(self.nel[s], self.deg[s] + 1)[0] for s in range(d)]
        cm = 1.0
        for r in range(d):
            lo, hi = bool(side_mask >> (2 * r) & 1), bool(side_mask >> (2 * r + 1) & 1)
            C, fr = split_1d(self.nel[r], self.deg[r], lo, hi)
            Mw, _ = weighted_1d(self.nel[r], self.deg[r], mass_w[r])
            _, Kw = weighted_1d(self.nel[r], self.deg[r], om[r][r])
            Kh, M = khat_1d(self.nel[r], self.deg[r], fr, C, Mw, Kw, sigma)
            lam, U = sla.eigh(Kh, M)
            self.U.append(U)
            self.lam.append(lam)
            cr = 1.0
            for s in range(d):
                if s != r:
                    cr *= np.mean(om[r][s](xs[s]) / mass_w[s](xs[s]))
            self.c.append(cr)
            cm /= np.mean(mass_w[r](xs[r]))
        self.cM = cm
        self.nfree = [len(u) for u in self.U]
        D = np.zeros(self.nfree[::-1])
        for r in range(d):
            shape = [1] * d
            shape[d - 1 - r] = self.nfree[r]
            D = D + self.c[r] * self.lam[r].reshape(shape)
        if alpha:
            D = D + alpha * self.cM
        self.Dinv = 1.0 / D
        # ---- degree-1 levels below
        dom1 = _degree_one_domain(dom, k)
        K1, _, _ = assembly.assemble_patch(dom1, k, with_rhs=False)
        nel1 = dom1.patch_nelem(k)
        self.coarse = MGOperator(Hierarchy(K1, nel1, (1,) * d, cmin), side_mask, alpha)
        # ---- L2-projection transfer finest <- first degree-1 level
        mats = []
        for r in range(d):
            lo, hi = bool(side_mask >> (2 * r) & 1), bool(side_mask >> (2 * r + 1) & 1)
            mats.append(sp.csr_matrix(l2_transfer_1d(self.nel[r], self.deg[r], nel1[r], lo, hi)))
        self.P = assembly._kron_all(mats)

    def smooth_inv(self, r):
        """L^{-1} r by fast diagonalization."""
        d = self.d
        R = r.reshape(self.nfree[::-1])
        for a in range(d):
            R = np.moveaxis(np.tensordot(self.U[a].T, R, axes=([1], [d - 1 - a])), 0, d - 1 - a)
        R = R * self.Dinv
        for a in range(d):
            R = np.moveaxis(np.tensordot(self.U[a], R, axes=([1], [d - 1 - a])), 0, d - 1 - a)
        return R.reshape(-1)

    def vcycle(self, b):
        x = np.zeros_like(b)
        for _ in range(self.nu):
            x += self.smooth_inv(b - self.Af @ x)
        r = b - self.Af @ x
        x += self.P @ self.coarse.vcycle(self.P.T @ r)
        for _ in range(self.nu):
            x += self.smooth_inv(b - self.Af @ x)
        return x


def _degree_one_domain(dom, k):
    """A copy of the domain whose patch k has degree 1 and half the elements
    per direction (same geometry map and patch grid)."""
    import copy
    d1 = copy.deepcopy(dom)
    c = dom.patch_coords(k)
    for r in range(dom.dim):
        d1.degree[r][c[r]] = 1
        d1.nelem[r][c[r]] = max(1, dom.nelem[r][c[r]] // 2)
    return d1


def l2_transfer_1d(n_f, p_f, n_c, lo_dir, hi_dir, p_c=1):
    """Prolongation from S_{p_c, n_c} to S_{p_f, n_f} by the L2 projection on
    (0,1), over the free functions of both spaces: M_f^-1 M_fc."""
    x, w = splines.gauss_points(n_f, max(p_f, p_c) + 1)
    Bf = splines.basis_funs(splines.open_uniform_knots(n_f, p_f), p_f, x)
    Bc = splines.basis_funs(splines.open_uniform_knots(n_c, p_c), p_c, x)
    Mf = Bf.T @ (w[:, None] * Bf)
    Mfc = Bf.T @ (w[:, None] * Bc)
    ff = np.arange(Bf.shape[1])
    fc = np.arange(Bc.shape[1])
    if lo_dir:
        ff, fc = ff[1:], fc[1:]
    if hi_dir:
        ff, fc = ff[:-1], fc[:-1]
    return np.linalg.solve(Mf[np.ix_(ff, ff)], Mfc[np.ix_(ff, fc)])
