"""Multipatch numbering and the conforming global Galerkin solve (Sec. 2).

ORACLE (test infrastructure only).  Plain FP64 numpy/scipy.

The result IETI-DP computes is, by construction (tearing plus Lagrange
multipliers enforcing continuity, Eq. 2), the conforming Galerkin solution of
Eq. 1 in the multipatch spline space with homogeneous Dirichlet data.  This
module writes that definition out: one global dof per conforming basis
function, K = sum_k R_k^T K^(k) R_k, Dirichlet dofs removed, and a sparse
direct solve (scipy ``spsolve``).

Conforming numbering of a patch grid: along direction r, patch column c has
m_c = n_c + p_c functions; neighbouring columns share their interpolatory
end functions, so column c starts at global index O_c = sum_{c'<c} (m_c' - 1).

Interface objects: a global dof whose r-th global index equals some O_c
(c = 1..P_r-1) lies on an interface in direction r.  Counting those
directions: d of them = vertex; in 3D, 2 = edge and 1 = face; in 2D, 1 = edge.

Parity: this module is the definition-level oracle; it is pinned by the
manufactured-solution L2 convergence rate (order p+1) and by reducing, for a
1x1 grid, to the single-patch Galerkin solve.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import assembly, splines


class Multipatch:
    def __init__(self, dom):
        self.dom = dom
        d = dom.dim
        self.d = d
        self.m = []       # m[r][c]
        self.off = []     # off[r][c]
        self.Mg = []
        self.bps = []     # interior breakpoints per direction (global 1D index)
        for r in range(d):
            m = [dom.nelem[r][c] + dom.degree[r][c] for c in range(dom.grid[r])]
            off = np.concatenate([[0], np.cumsum(np.asarray(m) - 1)[:-1]]).astype(int)
            self.m.append(m)
            self.off.append(off)
            self.Mg.append(int(sum(m) - (len(m) - 1)))
            self.bps.append(set(int(o) for o in off[1:]))
        self.nglob = int(np.prod(self.Mg))
        # local -> global map per patch
        self.l2g = []
        for k in range(dom.npatch):
            c = dom.patch_coords(k)
            axes = [self.off[r][c[r]] + np.arange(self.m[r][c[r]]) for r in range(d)]
            self.l2g.append(self._flat(axes))
        gi = self.global_index_grid()
        bnd = np.zeros(self.nglob, dtype=bool)
        for r in range(d):
            bnd |= (gi[r] == 0) | (gi[r] == self.Mg[r] - 1)
        self.dirichlet = bnd
        self.free = np.nonzero(~bnd)[0]

    def _flat(self, axes):
        """Flat global indices (first direction fastest) of a tensor box."""
        idx = np.zeros(1, dtype=np.int64)
        stride = 1
        out = None
        for r, ax in enumerate(axes):
            if out is None:
                out = ax.astype(np.int64)
            else:
                out = (out[None, :] + stride * ax.astype(np.int64)[:, None]).ravel()
            stride *= self.Mg[r]
        return out

    def global_index_grid(self):
        """Per direction, the global 1D index of every global dof."""
        gi = []
        idx = np.arange(self.nglob)
        for r in range(self.d):
            gi.append(idx % self.Mg[r])
            idx = idx // self.Mg[r]
        return gi

    # ------------------------------------------------------------------
    def assemble(self):
        """Per-patch K^(k), f^(k), M^(k) (cached)."""
        if not hasattr(self, "K"):
            self.K, self.f, self.M = [], [], []
            for k in range(self.dom.npatch):
                K, f, M = assembly.assemble_patch(self.dom, k)
                self.K.append(K)
                self.f.append(f)
                self.M.append(M)
        return self.K, self.f, self.M

    def global_system(self):
        K, f, _ = self.assemble()
        rows, cols, vals = [], [], []
        fg = np.zeros(self.nglob)
        for k in range(self.dom.npatch):
            Kc = K[k].tocoo()
            g = self.l2g[k]
            rows.append(g[Kc.row])
            cols.append(g[Kc.col])
            vals.append(Kc.data)
            np.add.at(fg, g, f[k])
        Kg = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                           shape=(self.nglob, self.nglob))
        return Kg, fg

    def solve_global(self):
        """Conforming Galerkin solution (global coefficients, 0 on Dirichlet).

        Sparse direct solve of the SPD system: LU without pivoting (none is
        needed for SPD matrices) in a minimum-degree ordering of K + K^T,
        which keeps the fill of million-dof 2D systems to minutes."""
        Kg, fg = self.global_system()
        fr = self.free
        u = np.zeros(self.nglob)
        A = sp.csc_matrix(Kg[fr][:, fr])
        if A.shape[0] == 0:
            return u
        lu = spla.splu(A, permc_spec="MMD_AT_PLUS_A", diag_pivot_thresh=0.0,
                       options={"SymmetricMode": True})
        u[fr] = lu.solve(fg[fr])
        return u

    def to_patches(self, u):
        return [u[g] for g in self.l2g]

    def l2_error(self, u):
        s = 0.0
        for k in range(self.dom.npatch):
            s += assembly.l2_error(self.dom, k, u[self.l2g[k]])
        return np.sqrt(s)

    # ------------------------------------------------------------------
    def interface_type(self):
        """Per global dof: number of directions in which it is on an
        interface, plus the boolean per direction."""
        gi = self.global_index_grid()
        onbp = np.zeros((self.d, self.nglob), dtype=bool)
        for r in range(self.d):
            bp = np.array(sorted(self.bps[r]), dtype=np.int64)
            onbp[r] = np.isin(gi[r], bp)
        return onbp.sum(axis=0), onbp

    def copies(self, g):
        """All (patch, local index) pairs that hold global dof g."""
        coord = []
        gg = g
        for r in range(self.d):
            coord.append(gg % self.Mg[r])
            gg //= self.Mg[r]
        per_dir = []
        for r in range(self.d):
            opts = []
            for c in range(self.dom.grid[r]):
                a = coord[r] - self.off[r][c]
                if 0 <= a < self.m[r][c]:
                    opts.append((c, a))
            per_dir.append(opts)
        out = []
        for combo in itertools.product(*per_dir):
            k = 0
            stride = 1
            loc = 0
            lstride = 1
            for r, (c, a) in enumerate(combo):
                k += stride * c
                stride *= self.dom.grid[r]
                loc += lstride * a
                lstride *= self.m[r][c]
            out.append((k, loc))
        out.sort()
        return out

    def cell_of(self, r, G):
        """Patch column along r containing global 1D index G strictly inside."""
        for c in range(self.dom.grid[r]):
            if self.off[r][c] < G < self.off[r][c] + self.m[r][c] - 1:
                return c
        return None
