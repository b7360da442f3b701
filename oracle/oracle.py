"""ctypes wrapper of the CPU oracle (pair_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
bench.py's CPU-baseline leg.  The product package never imports this module.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sysconfig
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pair_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OR_OK = 0


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-Wall", "-Wno-unused-result", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.check_call(cmd)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class or_params(C.Structure):
    _fields_ = [("distance", C.c_int), ("theta", C.c_double), ("eps_R", C.c_double),
                ("phi_R", C.c_double), ("phi_A", C.c_double), ("max_levels", C.c_int),
                ("max_coarse", C.c_int), ("coarse_sweeps", C.c_int), ("seed", C.c_uint64),
                ("f_sweeps", C.c_int), ("nair", C.c_int)]


class or_si_params(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iters", C.c_int), ("inner_tol", C.c_double),
                ("inner_maxit", C.c_int), ("use_sweep", C.c_int), ("g_inflow", C.c_double),
                ("inner_cycles", C.c_int), ("q_ang", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.or_air_setup.restype = C.c_void_p
        _lib.or_air_setup.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.POINTER(or_params), C.POINTER(C.c_int)]
        for name in ("or_hier_nlev", "or_hier_free", "or_hier_level_sizes", "or_hier_level_export",
                     "or_vcycle", "or_air_solve"):
            getattr(_lib, name).argtypes = None
        _lib.or_hier_free.argtypes = [C.c_void_p]
        _lib.or_hier_nlev.argtypes = [C.c_void_p]
        _lib.or_vcycle.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        _lib.or_air_solve.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int,
                                      C.POINTER(C.c_int), C.c_void_p]
        _lib.or_hier_level_sizes.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        _lib.or_hier_level_export.argtypes = [C.c_void_p, C.c_int] + [C.c_void_p] * 10
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def default_params(**kw) -> or_params:
    p = or_params()
    lib().or_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------------------
# Assembly
# ---------------------------------------------------------------------------

def hex_assemble(n: int, omega, sigma_t, scaled: bool = True):
    """CSR (rowptr, col, val) of the scaled operator A = D^{-1} L (scaled=True)
    or of L itself, for one direction omega on the n^3 hex mesh."""
    om = _f64(omega)
    st = _f64(sigma_t)
    nnz = lib().or_hex_nnz(C.c_int(n), _p(om), C.c_int(int(scaled)))
    if nnz < 0:
        raise RuntimeError(f"or_hex_nnz failed: {nnz}")
    N = 8 * n ** 3
    rowptr = np.zeros(N + 1, np.int32)
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz, np.float64)
    rc = lib().or_hex_assemble(C.c_int(n), _p(om), _p(st), C.c_int(int(scaled)), _p(rowptr), _p(col), _p(val))
    if rc != OR_OK:
        raise RuntimeError(f"or_hex_assemble failed: {rc}")
    return rowptr, col, val


def hex_rhs(n: int, omega, sigma_t, src, ginflow=None, scaled: bool = True):
    """b = M src + boundary inflow term (optionally scaled by D^{-1})."""
    N = 8 * n ** 3
    b = np.zeros(N)
    g = None if ginflow is None else _f64(ginflow)
    rc = lib().or_hex_rhs(C.c_int(n), _p(_f64(omega)), _p(_f64(sigma_t)), _p(_f64(src)), _p(g),
                          C.c_int(int(scaled)), _p(b))
    if rc != OR_OK:
        raise RuntimeError(f"or_hex_rhs failed: {rc}")
    return b


def sweep(rowptr, col, val, b, nb: int = 8):
    """Exact block forward substitution of the scaled system in upwind order."""
    N = len(rowptr) - 1
    x = np.zeros(N)
    order = np.zeros(N // nb, np.int32)
    rc = lib().or_sweep(C.c_int(N), C.c_int(nb), _p(_i32(rowptr)), _p(_i32(col)), _p(_f64(val)),
                        _p(_f64(b)), _p(x), _p(order))
    if rc != OR_OK:
        raise RuntimeError(f"or_sweep failed: {rc}")
    return x, order


# ---------------------------------------------------------------------------
# AIR
# ---------------------------------------------------------------------------

@dataclass
class Level:
    n: int
    nnz: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    dinv: np.ndarray
    coarsest: bool
    cf: np.ndarray | None = None
    pmap: np.ndarray | None = None
    cpts: np.ndarray | None = None
    zrowptr: np.ndarray | None = None
    zcol: np.ndarray | None = None
    zval: np.ndarray | None = None
    pmis_rounds: int = 0
    n_singular: int = 0


class Hierarchy:
    """Oracle AIR hierarchy built on a CSR matrix (sorted columns)."""

    def __init__(self, rowptr, col, val, params: or_params | None = None):
        self.params = params or default_params()
        self._rowptr, self._col, self._val = _i32(rowptr), _i32(col), _f64(val)
        st = C.c_int(0)
        self._h = lib().or_air_setup(C.c_int(len(rowptr) - 1), _p(self._rowptr), _p(self._col),
                                     _p(self._val), C.byref(self.params), C.byref(st))
        if st.value != OR_OK:
            self.free()
            raise RuntimeError(f"or_air_setup failed: {st.value}")
        self.n = len(rowptr) - 1

    def free(self):
        if getattr(self, "_h", None):
            lib().or_hier_free(C.c_void_p(self._h))
            self._h = None

    def __del__(self):
        self.free()

    @property
    def nlev(self) -> int:
        return lib().or_hier_nlev(C.c_void_p(self._h))

    def level(self, l: int) -> Level:
        s = np.zeros(7, np.int32)
        lib().or_hier_level_sizes(C.c_void_p(self._h), C.c_int(l), _p(s))
        n, nnz, nc, nnzZ, coarsest, rounds, nsing = (int(v) for v in s)
        rowptr = np.zeros(n + 1, np.int32)
        col = np.zeros(nnz, np.int32)
        val = np.zeros(nnz)
        dinv = np.zeros(n)
        if coarsest:
            lib().or_hier_level_export(C.c_void_p(self._h), C.c_int(l), _p(rowptr), _p(col), _p(val), _p(dinv),
                                       None, None, None, None, None, None)
            return Level(n, nnz, rowptr, col, val, dinv, True)
        cf = np.zeros(n, np.int8)
        pmap = np.zeros(n, np.int32)
        cpts = np.zeros(nc, np.int32)
        zr = np.zeros(nc + 1, np.int32)
        zc = np.zeros(nnzZ, np.int32)
        zv = np.zeros(nnzZ)
        lib().or_hier_level_export(C.c_void_p(self._h), C.c_int(l), _p(rowptr), _p(col), _p(val), _p(dinv),
                                   _p(cf), _p(pmap), _p(cpts), _p(zr), _p(zc), _p(zv))
        return Level(n, nnz, rowptr, col, val, dinv, False, cf, pmap, cpts, zr, zc, zv, rounds, nsing)

    def levels(self):
        return [self.level(l) for l in range(self.nlev)]

    def vcycle(self, b, x):
        b = _f64(b)
        x = _f64(x).copy()
        lib().or_vcycle(C.c_void_p(self._h), _p(b), _p(x))
        return x

    def solve(self, b, x0=None, tol: float = 1e-10, maxit: int = 200):
        b = _f64(b)
        x = np.zeros(self.n) if x0 is None else _f64(x0).copy()
        it = C.c_int(0)
        hist = np.zeros(maxit + 1)
        rc = lib().or_air_solve(C.c_void_p(self._h), _p(b), _p(x), C.c_double(tol), C.c_int(maxit),
                                C.byref(it), _p(hist))
        return x, hist[: it.value + 1], rc


# ---------------------------------------------------------------------------
# Source iteration
# ---------------------------------------------------------------------------

def si_hex(prob, tol=1e-8, max_iters=500, inner_tol=1e-10, inner_maxit=200, use_sweep=False,
           g_inflow=0.0, params: or_params | None = None, phi0=None, inner_cycles=0, q_ang=None):
    """Source iteration on a HexProblem; returns (phi, psi[M,N], info dict).
    inner_cycles > 0: each direction solved by exactly that many V-cycles from zero;
    q_ang: optional (M, N) nodal angular source added to each direction's source."""
    n, M, N = prob.n, prob.M, prob.N
    qa = None if q_ang is None else _f64(q_ang).reshape(M * N)
    sp = or_si_params(tol, max_iters, inner_tol, inner_maxit, int(use_sweep), g_inflow, int(inner_cycles),
                      qa.ctypes.data if qa is not None else None)
    prm = params or default_params()
    phi = np.zeros(N) if phi0 is None else _f64(phi0).copy()
    psi = np.zeros((M, N))
    info = np.zeros(4)
    rc = lib().or_si_hex(C.c_int(n), C.c_int(M), _p(_f64(prob.omega)), _p(_f64(prob.w)),
                         _p(_f64(prob.sigma_t)), _p(_f64(prob.sigma_s)), _p(_f64(prob.q)),
                         C.byref(sp), C.byref(prm), _p(phi), _p(psi), _p(info))
    return phi, psi, {"rc": rc, "si_iters": int(info[0]), "si_change": info[1],
                      "inner_iters": int(info[2]), "max_inner_resid": info[3]}


def csr_transpose(rowptr, col, val):
    N = len(rowptr) - 1
    tr = np.zeros(N + 1, np.int32)
    tc = np.zeros(len(col), np.int32)
    tv = np.zeros(len(col))
    rc = lib().or_csr_transpose(C.c_int(N), _p(_i32(rowptr)), _p(_i32(col)), _p(_f64(val)), _p(tr), _p(tc), _p(tv))
    if rc != OR_OK:
        raise RuntimeError(f"or_csr_transpose failed: {rc}")
    return tr, tc, tv


def si_adjoint_hex(prob, psi, g, tol=1e-8, max_iters=500, inner_tol=1e-10, inner_maxit=200, use_sweep=False,
                   params: or_params | None = None):
    """Adjoint SI and gradients of J = g^T phi w.r.t. sigma_t, sigma_s, q per element.
    Returns (dJ/dsigma_t, dJ/dsigma_s, dJ/dq, phi_adjoint, info)."""
    n, M, N, E = prob.n, prob.M, prob.N, prob.E
    sp = or_si_params(tol, max_iters, inner_tol, inner_maxit, int(use_sweep), 0.0)
    prm = params or default_params()
    dst, dss, dq = np.zeros(E), np.zeros(E), np.zeros(E)
    phis = np.zeros(N)
    info = np.zeros(2)
    rc = lib().or_si_adjoint_hex(C.c_int(n), C.c_int(M), _p(_f64(prob.omega)), _p(_f64(prob.w)),
                                 _p(_f64(prob.sigma_t)), _p(_f64(prob.sigma_s)), _p(_f64(prob.q)),
                                 _p(_f64(np.ascontiguousarray(psi).reshape(-1))), _p(_f64(g)), C.byref(sp),
                                 C.byref(prm), _p(dst), _p(dss), _p(dq), _p(phis), _p(info))
    return dst, dss, dq, phis, {"rc": rc, "iters": int(info[0]), "change": info[1]}


def si_adjoint_tet(prob, psi, g, tol=1e-8, max_iters=500, inner_tol=1e-10, inner_maxit=200, use_sweep=False,
                   params: or_params | None = None):
    """si_adjoint_hex on a TetProblem's mesh (P1, 4 DOFs per tet)."""
    M, N, E = prob.M, prob.N, prob.E
    sp = or_si_params(tol, max_iters, inner_tol, inner_maxit, int(use_sweep), 0.0)
    prm = params or default_params()
    dst, dss, dq = np.zeros(E), np.zeros(E), np.zeros(E)
    phis = np.zeros(N)
    info = np.zeros(2)
    rc = lib().or_si_adjoint_tet(*_tet_args(prob), C.c_int(M), _p(_f64(prob.omega)), _p(_f64(prob.w)),
                                 _p(_f64(prob.sigma_t)), _p(_f64(prob.sigma_s)), _p(_f64(prob.q)),
                                 _p(_f64(np.ascontiguousarray(psi).reshape(-1))), _p(_f64(g)), C.byref(sp),
                                 C.byref(prm), _p(dst), _p(dss), _p(dq), _p(phis), _p(info))
    return dst, dss, dq, phis, {"rc": rc, "iters": int(info[0]), "change": info[1]}


def detector_weights(prob, mask):
    """g with J = g^T phi = integral of phi_h over the elements in mask: g_K = M_K 1."""
    if hasattr(prob, "tets"):
        # P1 mass matrix of a tetrahedron K: |K| (1 + delta_ab) / 20, row sums |K| / 4
        g = np.zeros(prob.N)
        for e in np.nonzero(mask)[0]:
            x = prob.verts[prob.tets[e]]
            vol = abs(np.linalg.det(np.stack([x[1] - x[0], x[2] - x[0], x[3] - x[0]]))) / 6.0
            g[4 * e: 4 * e + 4] = vol / 4.0
        return g
    h = 1.0 / prob.n
    # row sums of the Q1 mass matrix: h^3 / 8 for every node
    g = np.zeros(prob.N)
    for e in np.nonzero(mask)[0]:
        g[8 * e: 8 * e + 8] = h ** 3 / 8.0
    return g


# ---------------------------------------------------------------------------
# Tetrahedra
# ---------------------------------------------------------------------------

def _tet_args(prob):
    return (C.c_int(prob.E), _p(_f64(prob.verts)), _p(_i32(prob.tets)), _p(_i32(prob.nbr)))


def tet_assemble(prob, omega, sigma_t=None, scaled: bool = True):
    """CSR of A = D^{-1} L (or L) for one direction on a TetProblem's mesh."""
    st = _f64(prob.sigma_t if sigma_t is None else sigma_t)
    om = _f64(omega)
    nnz = lib().or_tet_nnz(*_tet_args(prob), _p(om), C.c_int(int(scaled)))
    if nnz < 0:
        raise RuntimeError(f"or_tet_nnz failed: {nnz}")
    rowptr = np.zeros(prob.N + 1, np.int32)
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz)
    rc = lib().or_tet_assemble(*_tet_args(prob), _p(om), _p(st), C.c_int(int(scaled)), _p(rowptr), _p(col), _p(val))
    if rc != OR_OK:
        raise RuntimeError(f"or_tet_assemble failed: {rc}")
    return rowptr, col, val


def tet_rhs(prob, omega, src, ginflow=None, scaled: bool = True, sigma_t=None):
    b = np.zeros(prob.N)
    st = _f64(prob.sigma_t if sigma_t is None else sigma_t)
    g = None if ginflow is None else _f64(ginflow)
    rc = lib().or_tet_rhs(*_tet_args(prob), _p(_f64(omega)), _p(st), _p(_f64(src)), _p(g), C.c_int(int(scaled)),
                          _p(b))
    if rc != OR_OK:
        raise RuntimeError(f"or_tet_rhs failed: {rc}")
    return b


def sweep_scc(rowptr, col, val, b, nb):
    """Exact block solve by strongly connected components; returns (x, number of cycles)."""
    N = len(rowptr) - 1
    x = np.zeros(N)
    ncyc = C.c_int(0)
    rc = lib().or_sweep_scc(C.c_int(N), C.c_int(nb), _p(_i32(rowptr)), _p(_i32(col)), _p(_f64(val)), _p(_f64(b)),
                            _p(x), None, C.byref(ncyc))
    if rc != OR_OK:
        raise RuntimeError(f"or_sweep_scc failed: {rc}")
    return x, ncyc.value


def si_tet(prob, tol=1e-8, max_iters=500, inner_tol=1e-10, inner_maxit=200, use_sweep=False, g_inflow=0.0,
           params: or_params | None = None):
    M, N = prob.M, prob.N
    sp = or_si_params(tol, max_iters, inner_tol, inner_maxit, int(use_sweep), g_inflow)
    prm = params or default_params()
    phi = np.zeros(N)
    psi = np.zeros((M, N))
    info = np.zeros(4)
    rc = lib().or_si_tet(*_tet_args(prob), C.c_int(M), _p(_f64(prob.omega)), _p(_f64(prob.w)),
                         _p(_f64(prob.sigma_t)), _p(_f64(prob.sigma_s)), _p(_f64(prob.q)), C.byref(sp), C.byref(prm),
                         _p(phi), _p(psi), _p(info))
    return phi, psi, {"rc": rc, "si_iters": int(info[0]), "si_change": info[1], "inner_iters": int(info[2]),
                      "max_inner_resid": info[3]}
