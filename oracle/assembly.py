"""Galerkin matrices of one patch (Eq. 1 discretized with the pulled-back
B-spline basis of Sec. 2; parameter-domain mass of Sec. 3.2).

ORACLE (test infrastructure only).  Plain FP64 numpy/scipy.sparse.

Local dofs and Gauss points are both ordered on their tensor grids with the
first direction fastest.  Quadrature: p_r + 1 Gauss-Legendre points per
element and direction (the paper does not state its rule; with it the
identity-map matrices are exact).

    K_ij = sum_q w_q |det J_q| (J_q^{-T} grad N_i) . (J_q^{-T} grad N_j)
    f_i  = sum_q w_q |det J_q| f(G(xi_q)) N_i(xi_q)
    M^_ij = int_(0,1)^d N_i N_j  (no geometry)

Pins (tests/test_oracle_assembly.py): the 1D p=1 stiffness equals the
textbook [-1 2 -1]/h; K 1 = 0; the entries of M^ sum to 1; K and M^ are
symmetric; on the unit square the stiffness equals M1 x K2 + K1 x M2 built
from 1D matrices; Galerkin coarsening P^T K P equals re-assembly on the
coarse knots.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import geometry, splines


def _kron_all(mats):
    """kron(mats[d-1], ..., mats[0]): first direction fastest."""
    out = mats[0]
    for M in mats[1:]:
        out = sp.kron(M, out, format="csr")
    return sp.csr_matrix(out)


def patch_tables(dom, k):
    """Per direction: Gauss points, weights, basis values and derivatives."""
    deg = dom.patch_degree(k)
    nel = dom.patch_nelem(k)
    tabs = []
    for r in range(dom.dim):
        x, w = splines.gauss_points(nel[r], deg[r] + 1)
        B, D = splines.basis_funs(splines.open_uniform_knots(nel[r], deg[r]), deg[r], x, deriv=True)
        tabs.append((x, w, sp.csr_matrix(B), sp.csr_matrix(D)))
    return tabs


def quad_grid(dom, k, tabs):
    """Tensor grid of Gauss points (x fastest): parameters, weights."""
    d = dom.dim
    mesh = np.meshgrid(*[t[0] for t in tabs], indexing="ij")
    # meshgrid 'ij' makes the first axis slowest; reverse to x-fastest order
    xi = np.stack([m.transpose(tuple(range(d))[::-1]).ravel() for m in mesh], axis=1)
    wm = np.meshgrid(*[t[1] for t in tabs], indexing="ij")
    w = np.ones_like(wm[0])
    for m in wm:
        w = w * m
    w = w.transpose(tuple(range(d))[::-1]).ravel()
    return xi, w


def assemble_patch(dom, k, with_rhs=True):
    """Stiffness K (sparse), load f and parameter mass M^ of patch k on its
    full tensor grid of dofs (no boundary conditions applied)."""
    d = dom.dim
    tabs = patch_tables(dom, k)
    xi, w = quad_grid(dom, k, tabs)
    X, J = geometry.patch_map(dom, k, xi)
    detJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    # G^{ab} = w |det J| sum_c Jinv[a,c] Jinv[b,c]
    G = np.einsum("qac,qbc->qab", Jinv, Jinv) * (w * np.abs(detJ))[:, None, None]
    B = [t[2] for t in tabs]
    D = [t[3] for t in tabs]
    Phi = _kron_all(B)
    dPhi = []
    for a in range(d):
        mats = [D[r] if r == a else B[r] for r in range(d)]
        dPhi.append(_kron_all(mats))
    ndof = Phi.shape[1]
    K = sp.csr_matrix((ndof, ndof))
    for a in range(d):
        for b in range(d):
            g = G[:, a, b]
            if not np.any(g):
                continue
            K = K + dPhi[a].T @ sp.diags(g) @ dPhi[b]
    K = sp.csr_matrix(K)
    Mhat = _kron_all([sp.csr_matrix(splines.mass_1d(n, p))
                      for n, p in zip(dom.patch_nelem(k), dom.patch_degree(k))])
    f = None
    if with_rhs:
        if dom.rhs["kind"] == "quad":
            fq = np.asarray(dom.rhs["values"][k], dtype=np.float64)
        else:
            fq = geometry.rhs_values(dom, X)
        f = Phi.T @ (w * np.abs(detJ) * fq)
    return K, f, Mhat


def l2_error(dom, k, u_local, nq_extra=2):
    """||u_h - u||_{L2(patch k)}^2 with a finer Gauss rule (p+1+nq_extra)."""
    d = dom.dim
    deg = dom.patch_degree(k)
    nel = dom.patch_nelem(k)
    tabs = []
    for r in range(d):
        x, w = splines.gauss_points(nel[r], deg[r] + 1 + nq_extra)
        Bv = splines.basis_funs(splines.open_uniform_knots(nel[r], deg[r]), deg[r], x)
        tabs.append((x, w, sp.csr_matrix(Bv), None))
    xi, w = quad_grid(dom, k, tabs)
    X, J = geometry.patch_map(dom, k, xi)
    Phi = _kron_all([t[2] for t in tabs])
    uh = Phi @ u_local
    ue = geometry.exact_solution(dom, X)
    return float(np.sum(w * np.abs(np.linalg.det(J)) * (uh - ue) ** 2))


def row_stiffness_load(dom, k, i):
    """Row i of patch k's stiffness and the load entry f_i, computed alone:
    Gauss quadrature over the elements in the support of N_i only (same rule
    as ``assemble_patch``).  Returns (column indices, values, f_i).  Used to
    check single rows of a full-size solution one by one."""
    d = dom.dim
    deg = dom.patch_degree(k)
    nel = dom.patch_nelem(k)
    m = [n + p for n, p in zip(nel, deg)]
    ii = []
    rem = i
    for r in range(d):
        ii.append(rem % m[r])
        rem //= m[r]
    # per direction: elements of the support, their Gauss points, 1D tables
    per = []
    for r in range(d):
        e_lo, e_hi = max(ii[r] - deg[r], 0), min(ii[r], nel[r] - 1)
        g, w = np.polynomial.legendre.leggauss(deg[r] + 1)
        xs, ws = [], []
        for e in range(e_lo, e_hi + 1):
            xs.append((e + 0.5 * (g + 1.0)) / nel[r])
            ws.append(0.5 * w / nel[r])
        x = np.concatenate(xs)
        wq = np.concatenate(ws)
        B, D = splines.basis_funs(splines.open_uniform_knots(nel[r], deg[r]), deg[r], x, deriv=True)
        # global quadrature index (for Gauss-point right-hand sides)
        qidx = np.concatenate([e * (deg[r] + 1) + np.arange(deg[r] + 1) for e in range(e_lo, e_hi + 1)])
        per.append((x, wq, B, D, qidx))
    mesh = np.meshgrid(*[p_[0] for p_ in per], indexing="ij")
    xi = np.stack([mm.ravel() for mm in mesh], axis=1)
    wm = np.meshgrid(*[p_[1] for p_ in per], indexing="ij")
    w = np.ones(xi.shape[0])
    for mm in wm:
        w = w * mm.ravel()
    X, J = geometry.patch_map(dom, k, xi)
    detJ = np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    G = np.einsum("qac,qbc->qab", Jinv, Jinv) * (w * np.abs(detJ))[:, None, None]
    # values/gradients of all functions of the patch at these points (tensor)
    nq = [len(p_[0]) for p_ in per]
    idx = np.stack(np.meshgrid(*[np.arange(n) for n in nq], indexing="ij"), axis=-1).reshape(-1, d)
    vals = np.ones((xi.shape[0], int(np.prod(m))))
    grads = [np.ones_like(vals) for _ in range(d)]
    for r in range(d):
        Br = per[r][2][idx[:, r]]          # (q, m_r)
        Dr = per[r][3][idx[:, r]]
        # broadcast to the tensor grid of functions (first direction fastest)
        full_B = np.ones((xi.shape[0],) + tuple(m[::-1]))
        ax = d - r
        bshape = [xi.shape[0]] + [1] * d
        bshape[ax] = m[r]
        vals = vals * np.broadcast_to(Br.reshape(bshape), full_B.shape).reshape(xi.shape[0], -1)
        for a in range(d):
            src = Dr if a == r else Br
            grads[a] = grads[a] * np.broadcast_to(src.reshape(bshape), full_B.shape).reshape(xi.shape[0], -1)
    gi = np.stack([g_[:, i] for g_ in grads], axis=1)          # (q, d)
    row = np.zeros(int(np.prod(m)))
    for a in range(d):
        for b in range(d):
            row += (G[:, a, b] * gi[:, a]) @ grads[b]
    if dom.rhs["kind"] == "quad":
        qs = dom.quad_shape(k)
        flat = np.zeros(xi.shape[0], dtype=np.int64)
        stride = 1
        for r in range(d):
            flat += per[r][4][idx[:, r]] * stride
            stride *= qs[r]
        fq = np.asarray(dom.rhs["values"][k])[flat]
    else:
        fq = geometry.rhs_values(dom, X)
    f_i = float(np.sum(w * np.abs(detJ) * fq * vals[:, i]))
    cols = np.nonzero(row)[0]
    return cols, row[cols], f_i
