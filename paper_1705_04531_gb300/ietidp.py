"""Thin Python binding of the C ABI in ``include/ietidp.h`` (ctypes).

Argument marshalling only: every arithmetic step of assembly, setup and
solve runs in the CUDA kernels of ``libietidp.so``.  PyTorch supplies device
memory (tensors passed by pointer) and the CUDA stream.  If the library has
not been built, importing this module raises: there is no fallback path.

The functions keep the C names (``iga_assemble_patches``, ``ietidp_setup``,
``ietidp_solve`` ...); ``Problem`` and ``Solver`` wrap the handles.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libietidp.so")
if not os.path.exists(_LIBPATH):
    raise ImportError(f"{_LIBPATH} is missing: run paper_1705_04531_gb300.build.build() "
                      "(the library has no CPU fallback)")
_lib = C.CDLL(_LIBPATH)

# ---- constants (mirroring the header) --------------------------------------
IETIDP_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "BUDGET", -4: "CUDA", -5: "NOT_CONVERGED",
          -6: "TIMEOUT", -7: "NONFINITE", -8: "BREAKDOWN"}
IGA_GEO_BOX, IGA_GEO_ANNULUS = 0, 1
RHS = {"none": 0, "sin2d": 1, "sin3d": 2, "annulus": 3, "modes": 4, "quad": 5}
PRIMAL = {"vertex": 1, "edge": 2, "face": 4}
PREC_FP64, PREC_MIXED = 0, 1
METHOD = {"dual": 0, "saddle": 1, "dmg": 2}
BASIS = {"sz": 0, "nullspace": 1}


class iga_patch_desc(C.Structure):
    _fields_ = [("degree", C.c_int * 3), ("nelem", C.c_int * 3), ("geo_kind", C.c_int),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3)]


class iga_interface_desc(C.Structure):
    _fields_ = [("patch_a", C.c_int), ("side_a", C.c_int), ("patch_b", C.c_int), ("side_b", C.c_int),
                ("flip", C.c_int * 2), ("swap", C.c_int)]


class iga_domain_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("npatch", C.c_int), ("patches", C.POINTER(iga_patch_desc)),
                ("ninterface", C.c_int), ("interfaces", C.POINTER(iga_interface_desc)),
                ("rhs_kind", C.c_int), ("nmodes", C.c_int), ("mode_a", C.POINTER(C.c_double)),
                ("mode_k", C.POINTER(C.c_int)), ("mode_l", C.POINTER(C.c_int)),
                ("quad_values", C.c_void_p)]


class iga_topology_info(C.Structure):
    _fields_ = [("n_torn", C.c_longlong), ("n_global", C.c_longlong), ("n_classes", C.c_longlong),
                ("n_shared", C.c_longlong), ("n_dirichlet", C.c_longlong), ("n_floating", C.c_int)]


class ietidp_options(C.Structure):
    _fields_ = [("primal", C.c_uint), ("precision", C.c_int), ("tol_outer", C.c_double),
                ("tol_inner", C.c_double), ("tol_basis", C.c_double), ("maxit_outer", C.c_int),
                ("maxit_inner", C.c_int), ("nu_pre", C.c_int), ("nu_post", C.c_int),
                ("coarse_elems", C.c_int), ("dirichlet_vcycles", C.c_int), ("alpha_reg", C.c_double),
                ("cluster", C.c_int), ("method", C.c_int), ("saddle_vcycles", C.c_int),
                ("saddle_theta", C.c_double), ("basis_method", C.c_int), ("mg_kind", C.c_int)]


class ietidp_stats(C.Structure):
    _fields_ = [("outer_it", C.c_int), ("converged", C.c_int), ("rel_res", C.c_double),
                ("kappa", C.c_double), ("d_norm", C.c_double), ("d_scale", C.c_double),
                ("inner_it_avg", C.c_double), ("inner_it_max", C.c_int),
                ("basis_it_avg", C.c_double), ("basis_it_max", C.c_int),
                ("vcycles", C.c_longlong), ("vcycle_dofs", C.c_longlong),
                ("t_setup_ms", C.c_double), ("t_solve_ms", C.c_double),
                ("launches", C.c_longlong), ("neumann_launches", C.c_int), ("neumann_ms", C.c_double),
                ("inner_its", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ietidp_info(C.Structure):
    _fields_ = [("dim", C.c_int), ("npatch", C.c_int), ("n_torn", C.c_longlong), ("n_lambda", C.c_int),
                ("n_primal", C.c_int), ("n_floating", C.c_int), ("max_levels", C.c_int),
                ("device_bytes", C.c_longlong)]


_vp = C.c_void_p
_SIGS = {
    "ietidp_default_options": (None, [C.POINTER(ietidp_options)]),
    "iga_topology": (C.c_int, [C.POINTER(iga_domain_desc), C.POINTER(iga_topology_info), C.POINTER(C.c_uint)]),
    "iga_assemble_patches": (C.c_int, [C.POINTER(iga_domain_desc), _vp, C.POINTER(_vp)]),
    "iga_problem_load": (C.c_int, [_vp, _vp]),
    "iga_problem_free": (C.c_int, [_vp]),
    "ietidp_setup": (C.c_int, [_vp, C.POINTER(ietidp_options), _vp, C.POINTER(_vp)]),
    "ietidp_info_get": (C.c_int, [_vp, C.POINTER(ietidp_info)]),
    "ietidp_patch_offsets": (C.c_int, [_vp, C.POINTER(C.c_longlong)]),
    "ietidp_solve": (C.c_int, [_vp, _vp, _vp, C.POINTER(ietidp_stats)]),
    "ietidp_solve_host": (C.c_int, [_vp, _vp, _vp, C.POINTER(ietidp_stats)]),
    "ietidp_solve_batch": (C.c_int, [_vp, C.c_int, _vp, _vp, C.POINTER(ietidp_stats)]),
    "ietidp_solve_batch_host": (C.c_int, [_vp, C.c_int, _vp, _vp, C.POINTER(ietidp_stats)]),
    "ietidp_autotune_table": (C.c_int, [_vp, C.c_int]),
    "ietidp_kernel_launches": (C.c_longlong, []),
    "ietidp_vcycles": (C.c_int, [_vp, _vp, _vp, C.c_int]),
    "ietidp_vcycles_hierarchy": (C.c_int, [_vp, C.c_int, _vp, _vp, C.c_int]),
    "ietidp_vcycles_batch": (C.c_int, [C.POINTER(_vp), C.c_int, C.POINTER(_vp), C.POINTER(_vp), C.c_int,
                                       C.POINTER(C.c_float)]),
    "ietidp_vcycles_noalloc": (C.c_int, [_vp, _vp, _vp, C.c_int]),
    "ietidp_apply_K": (C.c_int, [_vp, _vp, _vp]),
    "ietidp_apply_F": (C.c_int, [_vp, _vp, _vp]),
    "ietidp_apply_precond": (C.c_int, [_vp, _vp, _vp]),
    "ietidp_apply_Ktilde_inv": (C.c_int, [_vp, _vp, _vp]),
    "ietidp_get_primal_basis": (C.c_int, [_vp, C.c_int, _vp, C.POINTER(C.c_int)]),
    "ietidp_get_spp": (C.c_int, [_vp, _vp]),
    "ietidp_phase_timers": (C.c_int, [_vp, _vp]),
    "ietidp_destroy": (C.c_int, [_vp]),
    "ietidp_last_error": (C.c_char_p, []),
    "ietidp_server_create": (C.c_int, [C.c_longlong, C.c_int, C.POINTER(ietidp_options), C.POINTER(_vp)]),
    "ietidp_server_submit": (C.c_int, [_vp, C.POINTER(iga_domain_desc), C.POINTER(C.c_ulonglong)]),
    "ietidp_server_poll": (C.c_int, [_vp, C.c_ulonglong, C.c_int, C.POINTER(C.c_int), _vp, C.c_longlong,
                                     C.POINTER(ietidp_stats), _vp]),
    "ietidp_server_status": (C.c_int, [_vp, C.POINTER(C.c_int), C.POINTER(C.c_longlong), C.POINTER(C.c_int)]),
    "ietidp_server_estimate": (C.c_longlong, [_vp, C.POINTER(iga_domain_desc)]),
    "ietidp_server_destroy": (C.c_int, [_vp]),
    "ietidp_ho_patch_operators": (C.c_int, [C.c_int, C.POINTER(iga_patch_desc), C.c_uint, C.c_double, C.c_int,
                                            C.POINTER(C.c_int), _vp, _vp, _vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS.keys())


class IetidpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _check(rc):
    if rc != IETIDP_OK:
        raise IetidpError(rc, _lib.ietidp_last_error().decode())
    return rc


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ---- domain marshalling ------------------------------------------------------
def domain_desc(dom: W.Domain):
    """C descriptors of a patch-grid domain: patches, interfaces between grid
    neighbours (no flips), right-hand side.  Returns (desc, keepalive)."""
    import torch
    d, N = dom.dim, dom.npatch
    pats = (iga_patch_desc * N)()
    for k in range(N):
        c = dom.patch_coords(k)
        pd, ne = dom.patch_degree(k), dom.patch_nelem(k)
        for r in range(3):
            pats[k].degree[r] = pd[r] if r < d else 0
            pats[k].nelem[r] = ne[r] if r < d else 1
            pats[k].lo[r] = c[r] / dom.grid[r] if r < d else 0.0
            pats[k].hi[r] = (c[r] + 1) / dom.grid[r] if r < d else 1.0
        pats[k].geo_kind = IGA_GEO_ANNULUS if dom.geometry == W.ANNULUS else IGA_GEO_BOX
    ifs = []
    for k in range(N):
        c = dom.patch_coords(k)
        stride = 1
        for r in range(d):
            if c[r] + 1 < dom.grid[r]:
                ifs.append((k, 2 * r + 1, k + stride, 2 * r))
            stride *= dom.grid[r]
    itf = (iga_interface_desc * max(1, len(ifs)))()
    for t, (a, sa, b, sb) in enumerate(ifs):
        itf[t].patch_a, itf[t].side_a, itf[t].patch_b, itf[t].side_b = a, sa, b, sb
    desc = iga_domain_desc()
    desc.dim, desc.npatch = d, N
    desc.patches = pats
    desc.ninterface = len(ifs)
    desc.interfaces = itf
    kind = dom.rhs["kind"]
    desc.rhs_kind = RHS[kind]
    keep = [pats, itf]
    if kind == "modes":
        n = len(dom.rhs["a"])
        a = (C.c_double * n)(*dom.rhs["a"])
        kk = (C.c_int * n)(*dom.rhs["k"])
        ll = (C.c_int * n)(*dom.rhs["l"])
        desc.nmodes, desc.mode_a, desc.mode_k, desc.mode_l = n, a, kk, ll
        keep += [a, kk, ll]
    if kind == "quad":
        vals = np.concatenate([np.asarray(v, dtype=np.float64) for v in dom.rhs["values"]])
        t = torch.from_numpy(vals).to("cuda")
        desc.quad_values = t.data_ptr()
        keep.append(t)
    return desc, keep


def primal_mask(primal):
    m = 0
    for p in primal:
        m |= PRIMAL[p]
    return m


def default_options(**kw) -> ietidp_options:
    o = ietidp_options()
    _lib.ietidp_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "primal" and not isinstance(v, int):
            v = primal_mask(v)
        if k == "precision" and isinstance(v, str):
            v = PREC_MIXED if v == "mixed" else PREC_FP64
        if k == "method" and isinstance(v, str):
            v = METHOD[v]
        if k == "basis_method" and isinstance(v, str):
            v = BASIS[v]
        if k == "mg_kind" and isinstance(v, str):
            v = {"standard": 0, "highorder": 1}[v]
        setattr(o, k, v)
    return o


# ---- C-named entry points ----------------------------------------------------
def iga_topology(desc):
    """Host-only topology of a domain descriptor (``domain_desc(dom)[0]`` or a
    hand-made ``iga_domain_desc``): (counts as a dict, Dirichlet side masks)."""
    info = iga_topology_info()
    dm = (C.c_uint * max(1, desc.npatch))()
    _check(_lib.iga_topology(C.byref(desc), C.byref(info), dm))
    out = {f: getattr(info, f) for f, _ in iga_topology_info._fields_}
    return out, [int(dm[k]) for k in range(desc.npatch)]


def ho_patch_operators(dom: W.Domain, k: int, kind: int, alpha: float = 1e-2):
    """High-order multigrid operators of patch k (host, FP64, no device work):
    (U_r list, P_r list, Dinv) with U_r[j, i] = eigenvector i at function j,
    P_r[j, c], Dinv on the free grid (first direction fastest)."""
    desc, keep = domain_desc(dom)
    _, dmask = iga_topology(desc)
    d = dom.dim
    sz = (C.c_int * 6)()
    pat = desc.patches[k]
    _check(_lib.ietidp_ho_patch_operators(d, C.byref(pat), dmask[k], alpha, kind, sz, None, None, None))
    nf, nc = list(sz[:3]), list(sz[3:])
    U = np.zeros(sum(nf[r] * nf[r] for r in range(d)))
    P = np.zeros(sum(nf[r] * nc[r] for r in range(d)))
    Dinv = np.zeros(int(np.prod(nf)))
    _check(_lib.ietidp_ho_patch_operators(d, C.byref(pat), dmask[k], alpha, kind, sz,
                                          U.ctypes.data_as(C.c_void_p), P.ctypes.data_as(C.c_void_p),
                                          Dinv.ctypes.data_as(C.c_void_p)))
    Us, Ps, ou, op = [], [], 0, 0
    for r in range(d):
        Us.append(U[ou:ou + nf[r] * nf[r]].reshape(nf[r], nf[r]).T.copy())   # [j, i]
        Ps.append(P[op:op + nf[r] * nc[r]].reshape(nc[r], nf[r]).T.copy())   # [j, c]
        ou += nf[r] * nf[r]
        op += nf[r] * nc[r]
    return Us, Ps, Dinv


def iga_assemble_patches(dom: W.Domain, stream=None):
    desc, keep = domain_desc(dom)
    h = C.c_void_p()
    _check(_lib.iga_assemble_patches(C.byref(desc), _stream_ptr(stream), C.byref(h)))
    return h


def ietidp_setup(problem, options: ietidp_options, stream=None):
    h = C.c_void_p()
    _check(_lib.ietidp_setup(problem, C.byref(options), _stream_ptr(stream), C.byref(h)))
    return h


def ietidp_solve(handle, f, u_out):
    st = ietidp_stats()
    rc = _lib.ietidp_solve(handle, _ptr(f), _ptr(u_out), C.byref(st))
    _check(rc)
    return st.as_dict()


def ietidp_solve_host(handle, f_host, u_host):
    st = ietidp_stats()
    fp = None if f_host is None else f_host.ctypes.data_as(C.c_void_p)
    _check(_lib.ietidp_solve_host(handle, fp, u_host.ctypes.data_as(C.c_void_p), C.byref(st)))
    return st.as_dict()


def ietidp_solve_batch(handles, fs, us):
    """Lockstep solve of several handles (device vectors; fs entries may be
    None for the assembled load).  Returns one stats dict per handle."""
    n = len(handles)
    hs = (C.c_void_p * n)(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    fp = (C.c_void_p * n)(*[None if f is None else f.data_ptr() for f in fs])
    up = (C.c_void_p * n)(*[u.data_ptr() for u in us])
    st = (ietidp_stats * n)()
    _check(_lib.ietidp_solve_batch(hs, n, fp, up, st))
    return [s.as_dict() for s in st]


def ietidp_solve_batch_host(handles, fs, us):
    """Same as ietidp_solve_batch with host numpy arrays (fs entries may be None)."""
    n = len(handles)
    hs = (C.c_void_p * n)(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    fp = (C.c_void_p * n)(*[None if f is None else f.ctypes.data for f in fs])
    up = (C.c_void_p * n)(*[u.ctypes.data for u in us])
    st = (ietidp_stats * n)()
    _check(_lib.ietidp_solve_batch_host(hs, n, fp, up, st))
    return [s.as_dict() for s in st]


def kernel_launches():
    """Kernels the library's solve entry points launched in this process."""
    return int(_lib.ietidp_kernel_launches())


def autotune_table():
    """Autotuner decisions: list of dicts (shape key and chosen configuration)."""
    n = _lib.ietidp_autotune_table(None, 0)
    buf = (C.c_int * (12 * max(n, 1)))()
    n = _lib.ietidp_autotune_table(buf, n)
    keys = ("dim", "p0", "p1", "p2", "kind", "mixed", "waves", "threads", "smem", "ctas_per_sm", "global_vectors",
            "cluster")
    return [dict(zip(keys, buf[12 * i:12 * i + 12])) for i in range(n)]


class Problem:
    """An assembled multipatch problem (device resident)."""

    def __init__(self, dom: W.Domain, stream=None):
        self.dom = dom
        self.h = iga_assemble_patches(dom, stream)

    def load(self):
        import torch
        n = int(sum(self.dom.patch_ndof(k) for k in range(self.dom.npatch)))
        f = torch.empty(n, dtype=torch.float64, device="cuda")
        _check(_lib.iga_problem_load(self.h, _ptr(f)))
        return f

    def close(self):
        if self.h:
            _lib.iga_problem_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """IETI-DP handle: setup on construction, ``solve`` per right-hand side."""

    def __init__(self, problem: Problem, stream=None, **opts):
        self.problem = problem
        if "primal" not in opts:
            opts["primal"] = problem.dom.primal
        self.options = default_options(**opts)
        self.h = ietidp_setup(problem.h, self.options, stream)
        self.info = ietidp_info()
        _check(_lib.ietidp_info_get(self.h, C.byref(self.info)))
        off = (C.c_longlong * (self.info.npatch + 1))()
        _check(_lib.ietidp_patch_offsets(self.h, off))
        self.offsets = np.array(off[:], dtype=np.int64)

    @property
    def n_torn(self):
        return int(self.info.n_torn)

    def solve(self, f=None, u=None):
        import torch
        if u is None:
            u = torch.empty(self.n_torn, dtype=torch.float64, device="cuda")
        st = ietidp_solve(self.h, f, u)
        return u, st

    def solve_host(self, f_host=None, u_host=None):
        if u_host is None:
            u_host = np.empty(self.n_torn)
        st = ietidp_solve_host(self.h, f_host, u_host)
        return u_host, st

    @staticmethod
    def solve_batch(solvers, fs=None, us=None):
        """Solve every solver's problem in one lockstep batch (device tensors)."""
        import torch
        if fs is None:
            fs = [None] * len(solvers)
        if us is None:
            us = [torch.empty(s.n_torn, dtype=torch.float64, device="cuda") for s in solvers]
        st = ietidp_solve_batch([s.h for s in solvers], fs, us)
        return us, st

    @staticmethod
    def solve_batch_host(solvers, fs=None, us=None):
        """Batched solve with host numpy buffers."""
        if fs is None:
            fs = [None] * len(solvers)
        if us is None:
            us = [np.empty(s.n_torn) for s in solvers]
        st = ietidp_solve_batch_host([s.h for s in solvers], fs, us)
        return us, st

    def vcycles(self, b, x, ncycles):
        _check(_lib.ietidp_vcycles(self.h, _ptr(b), _ptr(x), int(ncycles)))

    @staticmethod
    def vcycles_batch(solvers, bs, xs, ncycles):
        """V-cycles over the Neumann hierarchies of every patch of several
        solvers in merged launches; returns their duration in ms."""
        n = len(solvers)
        hv = (_vp * n)(*[s.h for s in solvers])
        bv = (_vp * n)(*[C.c_void_p(t.data_ptr()) for t in bs])
        xv = (_vp * n)(*[C.c_void_p(t.data_ptr()) for t in xs])
        ms = C.c_float(0.0)
        _check(_lib.ietidp_vcycles_batch(hv, n, bv, xv, int(ncycles), C.byref(ms)))
        return float(ms.value)

    def vcycles_hierarchy(self, hierarchy, b, x, ncycles):
        """V-cycles on the Neumann (0) or Dirichlet (1) hierarchy of every patch."""
        _check(_lib.ietidp_vcycles_hierarchy(self.h, int(hierarchy), _ptr(b), _ptr(x), int(ncycles)))

    def vcycles_noalloc(self, b, x, ncycles):
        """V-cycles whose scratch is the library's static device array (no
        allocation; see ietidp_vcycles_noalloc in the header)."""
        _check(_lib.ietidp_vcycles_noalloc(self.h, _ptr(b), _ptr(x), int(ncycles)))

    def phase_timers(self):
        out = np.zeros(64, dtype=np.int64)
        _check(_lib.ietidp_phase_timers(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def apply_K(self, x, y):
        _check(_lib.ietidp_apply_K(self.h, _ptr(x), _ptr(y)))

    def apply_F(self, p, q):
        _check(_lib.ietidp_apply_F(self.h, _ptr(p), _ptr(q)))

    def apply_precond(self, r, z):
        _check(_lib.ietidp_apply_precond(self.h, _ptr(r), _ptr(z)))

    def apply_Ktilde_inv(self, g, u):
        _check(_lib.ietidp_apply_Ktilde_inv(self.h, _ptr(g), _ptr(u)))

    def primal_basis(self, k):
        import torch
        nc = C.c_int()
        _check(_lib.ietidp_get_primal_basis(self.h, k, None, C.byref(nc)))
        n = int(self.offsets[k + 1] - self.offsets[k])
        out = torch.empty(max(1, nc.value * n), dtype=torch.float64, device="cuda")
        _check(_lib.ietidp_get_primal_basis(self.h, k, _ptr(out), C.byref(nc)))
        return out[: nc.value * n].reshape(nc.value, n)

    def spp(self):
        npi = int(self.info.n_primal)
        out = np.zeros(npi * npi)
        if npi:
            _check(_lib.ietidp_get_spp(self.h, out.ctypes.data_as(C.c_void_p)))
        return out.reshape(npi, npi)

    def split(self, u):
        """Torn vector -> list of per-patch numpy arrays."""
        a = u.detach().cpu().numpy() if hasattr(u, "detach") else np.asarray(u)
        return [a[self.offsets[k]:self.offsets[k + 1]] for k in range(len(self.offsets) - 1)]

    def close(self):
        if self.h:
            _lib.ietidp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server (ietidp_server_* in the C ABI).

    ``submit`` returns a ticket; ``poll``/``wait`` return (state, u, stats,
    times) -- u per patch layout on the host once the request is done."""

    def __init__(self, budget_bytes, max_concurrent=4, **opts):
        self.options = default_options(**opts)
        self.h = C.c_void_p()
        _check(_lib.ietidp_server_create(int(budget_bytes), int(max_concurrent), C.byref(self.options),
                                         C.byref(self.h)))
        self._keep = {}

    def estimate(self, dom):
        desc, keep = domain_desc(dom)
        return int(_lib.ietidp_server_estimate(self.h, C.byref(desc)))

    def submit(self, dom):
        desc, keep = domain_desc(dom)
        t = C.c_ulonglong()
        _check(_lib.ietidp_server_submit(self.h, C.byref(desc), C.byref(t)))
        n = int(sum(dom.patch_ndof(k) for k in range(dom.npatch)))
        self._keep[t.value] = (keep, n)
        return t.value

    def poll(self, ticket, wait=False):
        keep, n = self._keep[ticket]
        state = C.c_int()
        u = np.zeros(n)
        st = ietidp_stats()
        tm = np.zeros(3)
        rc = _lib.ietidp_server_poll(self.h, C.c_ulonglong(ticket), int(wait), C.byref(state),
                                     u.ctypes.data_as(C.c_void_p), n, C.byref(st),
                                     tm.ctypes.data_as(C.c_void_p))
        if state.value != 2:
            _check(rc)
            return state.value, None, None, None
        del self._keep[ticket]
        _check(rc)
        return 2, u, st.as_dict(), {"queue_s": tm[0], "run_s": tm[1], "latency_s": tm[2]}

    def wait(self, ticket):
        return self.poll(ticket, wait=True)

    def status(self):
        r, b, q = C.c_int(), C.c_longlong(), C.c_int()
        _check(_lib.ietidp_server_status(self.h, C.byref(r), C.byref(b), C.byref(q)))
        return {"running": r.value, "in_flight_bytes": b.value, "queued": q.value}

    def close(self):
        if self.h:
            _lib.ietidp_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
