"""Python binding of libpair (ctypes).  Argument marshalling only: every step
runs in the library's CUDA kernels.  PyTorch supplies device memory and the
current CUDA stream.  The binding fails loudly if the library is missing."""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libpair.so")

PAIR_OK = 0
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_SINGULAR", -4: "ERR_NOT_CONVERGED",
          -6: "ERR_NAN", -8: "ERR_CUDA",
          -9: "ERR_UNSUPPORTED", -10: "ERR_DEVICE", -11: "ERR_COMM"}


class PairError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class air_params(C.Structure):
    _fields_ = [("distance", C.c_int), ("theta", C.c_double), ("eps_R", C.c_double), ("phi_R", C.c_double),
                ("phi_A", C.c_double), ("max_levels", C.c_int), ("max_coarse", C.c_int),
                ("coarse_sweeps", C.c_int), ("seed", C.c_uint64), ("precision", C.c_int),
                ("f_sweeps", C.c_int), ("nair", C.c_int)]


class pair_csr(C.Structure):
    _fields_ = [("n", C.c_int), ("nnz", C.c_int), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p)]


class pair_level_info(C.Structure):
    _fields_ = [("n", C.c_int), ("nnz", C.c_int), ("nc", C.c_int), ("nnz_R", C.c_int), ("coarsest", C.c_int),
                ("pmis_rounds", C.c_int), ("n_singular", C.c_int)]


class air_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("rel_resid", C.c_double), ("rho", C.c_double)]


PAIR_MESH_HEX, PAIR_MESH_TET = 0, 1


class pair_mesh(C.Structure):
    _fields_ = [("kind", C.c_int), ("n", C.c_int), ("ntet", C.c_int), ("verts", C.c_void_p), ("tets", C.c_void_p),
                ("nbr", C.c_void_p)]


def hex_mesh(n: int) -> pair_mesh:
    return pair_mesh(PAIR_MESH_HEX, n, 0, None, None, None)


class TetMesh:
    """Device copy of a tetrahedral mesh (vertex coordinates, tets, face neighbours)."""

    def __init__(self, verts, tets, nbr, device="cuda"):
        self.verts = torch.as_tensor(np.ascontiguousarray(verts, np.float64), device=device).contiguous()
        self.tets = torch.as_tensor(np.ascontiguousarray(tets, np.int32), device=device).contiguous()
        self.nbr = torch.as_tensor(np.ascontiguousarray(nbr, np.int32), device=device).contiguous()
        self.ntet = self.tets.shape[0]
        self.struct = pair_mesh(PAIR_MESH_TET, 0, self.ntet, self.verts.data_ptr(), self.tets.data_ptr(),
                                self.nbr.data_ptr())

    @property
    def E(self) -> int:
        return self.ntet

    @property
    def N(self) -> int:
        return 4 * self.ntet


def _mesh_struct(mesh):
    if isinstance(mesh, TetMesh):
        return mesh.struct, mesh.ntet, 4 * mesh.ntet
    n = int(mesh)
    return hex_mesh(n), n ** 3, 8 * n ** 3


class pair_quad(C.Structure):
    _fields_ = [("M", C.c_int), ("omega", C.c_void_p), ("w", C.c_void_p)]


# pair_reduce_fn: int (*)(double *v, long long n, void *ctx)
REDUCE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_longlong, C.c_void_p)


class si_params(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iters", C.c_int), ("inner_tol", C.c_double), ("inner_maxit", C.c_int),
                ("batch", C.c_int), ("mem_budget_gb", C.c_double), ("g_inflow", C.c_double),
                ("use_graphs", C.c_int), ("fixed_iters", C.c_int), ("solver", C.c_int),
                ("inner_cycles", C.c_int), ("q_ang", C.c_void_p), ("phi_reduce", REDUCE_FN),
                ("reduce_ctx", C.c_void_p), ("concurrent", C.c_int),
                ("timing", C.c_int)]


class si_info(C.Structure):
    _fields_ = [("si_iters", C.c_int), ("si_change", C.c_double), ("vcycles", C.c_int),
                ("max_inner_resid", C.c_double), ("batches", C.c_int), ("rebuilt", C.c_int),
                ("t_setup_ms", C.c_double), ("t_solve_ms", C.c_double), ("levels_max", C.c_int),
                ("op_complexity", C.c_double), ("t_res0_ms", C.c_double), ("n_res0", C.c_int),
                ("gb_res0", C.c_double), ("t_relax0_ms", C.c_double), ("n_relax0", C.c_int),
                ("gb_relax0", C.c_double), ("t_setup_phase_ms", C.c_double * 4), ("t_relaxc_ms", C.c_double),
                ("n_relaxc", C.c_int), ("gb_relaxc", C.c_double), ("t_res32_ms", C.c_double),
                ("n_res32", C.c_int), ("gb_res32", C.c_double), ("outer_residuals", C.c_int),
                ("t_relaxc_level_ms", C.c_double * 8), ("timed_iters", C.c_int),
                ("t_xfer_ms", C.c_double), ("n_xfer", C.c_int), ("gb_xfer", C.c_double)]


_lib = None


def lib():
    """Loads libpair.so (built by build.py / __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpair.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i, d = C.c_void_p, C.c_int, C.c_double
        sig = {
            "air_params_default": (None, [C.POINTER(air_params)]),
            "si_params_default": (None, [C.POINTER(si_params)]),
            "pair_last_error": (C.c_char_p, []),
            "pair_kernel_launches": (C.c_longlong, []),
            "pair_residual_norm_noalloc": (i, [C.POINTER(pair_csr), vp, vp, vp, vp, vp]),
            "pair_csr_transpose": (i, [C.POINTER(pair_csr), vp, vp, vp, vp]),
            "pair_sweep": (i, [C.POINTER(pair_csr), i, vp, vp, vp, C.POINTER(i), C.POINTER(i)]),
            "si_adjoint": (i, [C.POINTER(pair_mesh), C.POINTER(pair_quad), vp, vp, vp, vp, vp, C.POINTER(air_params),
                               C.POINTER(si_params), vp, vp, vp, vp, vp, C.POINTER(si_info)]),
            "air_setup": (i, [C.POINTER(pair_csr), i, C.POINTER(air_params), vp, C.POINTER(vp)]),
            "air_vcycle": (i, [vp, vp, vp, vp]),
            "air_solve": (i, [vp, vp, vp, d, i, vp, C.POINTER(air_solve_info)]),
            "air_hier_nlevels": (i, [vp, i, C.POINTER(i)]),
            "air_level_info": (i, [vp, i, i, C.POINTER(pair_level_info)]),
            "air_level_export": (i, [vp, i, i] + [vp] * 9),
            "air_free": (None, [vp]),
            "dg_hex_nnz": (i, [C.POINTER(pair_mesh), vp, C.POINTER(i)]),
            "dg_assemble_hex": (i, [C.POINTER(pair_mesh), vp, vp, vp, vp, vp, vp]),
            "dg_assemble_tet": (i, [C.POINTER(pair_mesh), vp, vp, vp, vp, vp, i, C.POINTER(i), vp]),
            "si_solve": (i, [C.POINTER(pair_mesh), C.POINTER(pair_quad), vp, vp, vp, C.POINTER(air_params),
                             C.POINTER(si_params), vp, vp, vp, C.POINTER(si_info)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def kernel_source_sha(name: str = "cycle.cu") -> str:
    """Short hash of a kernel source file (ties stored profiler counters to the code they measured)."""
    import hashlib
    with open(os.path.join(_HERE, "csrc", name), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def kernel_launches() -> int:
    return lib().pair_kernel_launches()


def _check(st: int):
    if st != PAIR_OK:
        raise PairError(st, lib().pair_last_error().decode())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t: torch.Tensor):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return C.c_void_p(t.data_ptr())


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def default_air_params(**kw) -> air_params:
    p = air_params()
    lib().air_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def default_si_params(**kw) -> si_params:
    p = si_params()
    lib().si_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------------------
# AIR on user matrices
# ---------------------------------------------------------------------------

@dataclass
class LevelData:
    n: int
    nnz: int
    nc: int
    nnz_R: int
    coarsest: bool
    pmis_rounds: int
    n_singular: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    cf: np.ndarray | None
    pmap: np.ndarray | None
    cpts: np.ndarray | None
    zrowptr: np.ndarray | None
    zcol: np.ndarray | None
    zval: np.ndarray | None


class Hierarchy:
    """AIR hierarchies of a batch of CSR matrices (device tensors).  Vectors
    passed to vcycle/solve are the concatenation over the batch."""

    def __init__(self, mats, params: air_params | None = None):
        self.params = params or default_air_params()
        self._keep = []
        descs = (pair_csr * len(mats))()
        for k, (rowptr, col, val) in enumerate(mats):
            rowptr = rowptr.to(torch.int32).contiguous()
            col = col.to(torch.int32).contiguous()
            val = val.to(torch.float64).contiguous()
            self._keep += [rowptr, col, val]
            descs[k] = pair_csr(rowptr.numel() - 1, col.numel(), rowptr.data_ptr(), col.data_ptr(), val.data_ptr())
        self.sizes = [descs[k].n for k in range(len(mats))]
        self.count = len(mats)
        h = C.c_void_p()
        _check(lib().air_setup(descs, len(mats), C.byref(self.params), _stream(), C.byref(h)))
        self._h = h
        self._keep = []

    def free(self):
        if getattr(self, "_h", None):
            lib().air_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def nlevels(self, mat: int = 0) -> int:
        v = C.c_int()
        _check(lib().air_hier_nlevels(self._h, mat, C.byref(v)))
        return v.value

    def level(self, mat: int, l: int) -> LevelData:
        inf = pair_level_info()
        _check(lib().air_level_info(self._h, mat, l, C.byref(inf)))
        n, nnz, nc, nz = inf.n, inf.nnz, inf.nc, inf.nnz_R
        rowptr = np.zeros(n + 1, np.int32)
        col = np.zeros(nnz, np.int32)
        val = np.zeros(nnz)
        if inf.coarsest:
            _check(lib().air_level_export(self._h, mat, l, _np_ptr(rowptr), _np_ptr(col), _np_ptr(val),
                                          None, None, None, None, None, None))
            return LevelData(n, nnz, 0, 0, True, inf.pmis_rounds, inf.n_singular, rowptr, col, val,
                             None, None, None, None, None, None)
        cf = np.zeros(n, np.int8)
        pmap = np.zeros(n, np.int32)
        cpts = np.zeros(nc, np.int32)
        zr = np.zeros(nc + 1, np.int32)
        zc = np.zeros(nz, np.int32)
        zv = np.zeros(nz)
        _check(lib().air_level_export(self._h, mat, l, _np_ptr(rowptr), _np_ptr(col), _np_ptr(val), _np_ptr(cf),
                                      _np_ptr(pmap), _np_ptr(cpts), _np_ptr(zr), _np_ptr(zc), _np_ptr(zv)))
        return LevelData(n, nnz, nc, nz, False, inf.pmis_rounds, inf.n_singular, rowptr, col, val, cf, pmap, cpts,
                         zr, zc, zv)

    def vcycle(self, b: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
        _check(lib().air_vcycle(self._h, _dptr(b), _dptr(x), _stream()))
        return x

    def solve(self, b: torch.Tensor, x: torch.Tensor | None = None, tol: float = 1e-8, maxit: int = 100,
              raise_on_fail: bool = True):
        if x is None:
            x = torch.zeros_like(b)
        info = air_solve_info()
        st = lib().air_solve(self._h, _dptr(b), _dptr(x), tol, maxit, _stream(), C.byref(info))
        if raise_on_fail or st not in (PAIR_OK, -4):
            _check(st)
        return x, {"iters": info.iters, "rel_resid": info.rel_resid, "rho": info.rho, "status": st}


def residual_norm_noalloc(rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, b: torch.Tensor,
                          x: torch.Tensor, r: torch.Tensor | None = None, rnorm: torch.Tensor | None = None):
    """r = b - A x and ||r||_2 through the allocation-free entry point (the
    library allocates nothing; r and rnorm are allocated here by PyTorch unless
    given).  Returns (r, rnorm) as device tensors."""
    if r is None:
        r = torch.empty_like(b)
    if rnorm is None:
        rnorm = torch.empty(1, dtype=torch.float64, device=b.device)
    desc = pair_csr(rowptr.numel() - 1, col.numel(), rowptr.data_ptr(), col.data_ptr(), val.data_ptr())
    _check(lib().pair_residual_norm_noalloc(C.byref(desc), _dptr(b), _dptr(x), _dptr(r), _dptr(rnorm), _stream()))
    return r, rnorm


# ---------------------------------------------------------------------------
# DG transport
# ---------------------------------------------------------------------------

def dg_hex_nnz(n: int, omega) -> int:
    om = np.ascontiguousarray(omega, dtype=np.float64)
    v = C.c_int()
    _check(lib().dg_hex_nnz(C.byref(hex_mesh(n)), _np_ptr(om), C.byref(v)))
    return v.value


def dg_assemble_hex(n: int, omega, sigma_t: torch.Tensor):
    """Block-scaled upwind DG operator of one direction, device CSR tensors."""
    om = np.ascontiguousarray(omega, dtype=np.float64)
    nnz = dg_hex_nnz(n, om)
    dev = sigma_t.device
    N = 8 * n ** 3
    rowptr = torch.empty(N + 1, dtype=torch.int32, device=dev)
    col = torch.empty(nnz, dtype=torch.int32, device=dev)
    val = torch.empty(nnz, dtype=torch.float64, device=dev)
    st = sigma_t.to(torch.float64).contiguous()
    _check(lib().dg_assemble_hex(C.byref(hex_mesh(n)), _np_ptr(om), _dptr(st), _dptr(rowptr), _dptr(col),
                                 _dptr(val), _stream()))
    return rowptr, col, val


def dg_assemble_tet(mesh: "TetMesh", omega, sigma_t: torch.Tensor):
    """Block-scaled upwind P1 DG operator of one direction on a tetrahedral mesh."""
    om = np.ascontiguousarray(omega, dtype=np.float64)
    st = sigma_t.to(torch.float64).contiguous()
    rowptr = torch.empty(mesh.N + 1, dtype=torch.int32, device=st.device)
    nnz = C.c_int()
    _check(lib().dg_assemble_tet(C.byref(mesh.struct), _np_ptr(om), _dptr(st), _dptr(rowptr), None, None, 0,
                                 C.byref(nnz), _stream()))
    col = torch.empty(nnz.value, dtype=torch.int32, device=st.device)
    val = torch.empty(nnz.value, dtype=torch.float64, device=st.device)
    _check(lib().dg_assemble_tet(C.byref(mesh.struct), _np_ptr(om), _dptr(st), _dptr(rowptr), _dptr(col), _dptr(val),
                                 nnz.value, C.byref(nnz), _stream()))
    return rowptr, col, val


class _CudaView:
    """Zero-copy view of library-owned device memory (CUDA array interface)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (ptr, False), "version": 3,
                                         "strides": None}


class ReduceCallback:
    """The ctypes function for si_params.phi_reduce around fn(v): v is the library's
    array (N partial scalar-flux values, then one status value) as a float64 tensor
    view, on `device` ("cuda", or "cpu" for host memory), and fn must sum it over
    the processes in place, e.g. torch.distributed.all_reduce(v).  An exception in
    fn makes the library return PAIR_ERR_COMM; it is kept in .error."""

    def __init__(self, fn, device="cuda"):
        self.fn = fn
        self.device = torch.device(device)
        self.error = None
        self.cfunc = REDUCE_FN(self._call)

    def _call(self, ptr, n, ctx):
        try:
            if self.device.type == "cuda":
                v = torch.as_tensor(_CudaView(ptr, n), device=self.device)
            else:
                v = torch.from_numpy(np.ctypeslib.as_array((C.c_double * n).from_address(ptr)))
            self.fn(v)
            if self.device.type == "cuda":
                torch.cuda.synchronize(self.device)
            return 0
        except Exception as e:   # reported to the library as a status, re-raised by si_solve
            self.error = e
            return 1


def si_solve(n, omega, w, sigma_t, sigma_s, q, air: air_params | None = None, si: si_params | None = None,
             phi0=None, want_psi: bool = False, device="cuda", q_ang=None, phi_reduce=None):
    """Source iteration on the n^3 hex mesh (n an int) or on a TetMesh.  Cross
    sections may be CPU or CUDA tensors (CPU inputs are copied to the device and
    phi is returned on the device).  q_ang: optional (M, N) angular source density
    added per direction.  phi_reduce: optional fn(v) summing the partial scalar
    flux of this direction subset over the processes in place (see
    ReduceCallback).  Returns (phi, psi or None, info dict)."""
    air = air or default_air_params()
    si = si or default_si_params()
    qa_dev = None
    if q_ang is not None:
        qa_dev = torch.as_tensor(q_ang, dtype=torch.float64).to(device).contiguous()
        si = si_params.from_buffer_copy(si)
        si.q_ang = qa_dev.data_ptr()
    red = None
    if phi_reduce is not None:
        red = phi_reduce if isinstance(phi_reduce, ReduceCallback) else ReduceCallback(phi_reduce, device)
        si = si_params.from_buffer_copy(si)
        si.phi_reduce = red.cfunc
    om = np.ascontiguousarray(omega, dtype=np.float64)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    M = om.shape[0]
    mstruct, _, N = _mesh_struct(n)

    def dev_t(t):
        t = torch.as_tensor(t, dtype=torch.float64)
        return t.to(device, non_blocking=True).contiguous()

    st, ss, qq = dev_t(sigma_t), dev_t(sigma_s), dev_t(q)
    phi = torch.zeros(N, dtype=torch.float64, device=device) if phi0 is None else dev_t(phi0).clone()
    psi = torch.empty((M, N), dtype=torch.float64, device=device) if want_psi else None
    info = si_info()
    quad = pair_quad(M, om.ctypes.data, ww.ctypes.data)
    rc = lib().si_solve(C.byref(mstruct), C.byref(quad), _dptr(st), _dptr(ss), _dptr(qq), C.byref(air),
                        C.byref(si), _dptr(phi), _dptr(psi) if psi is not None else None, _stream(), C.byref(info))
    if red is not None and red.error is not None and rc == -11:
        raise PairError(rc, lib().pair_last_error().decode()) from red.error
    _check(rc)
    out = {f: getattr(info, f) for f, _ in si_info._fields_}
    out["t_setup_phase_ms"] = list(info.t_setup_phase_ms)
    return phi, psi, out


def _host_ptr(a, name):
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        if a.is_cuda or not a.is_contiguous() or a.dtype != torch.float64:
            raise ValueError(f"{name}: a contiguous float64 CPU tensor is required")
        return C.c_void_p(a.data_ptr())
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise ValueError(f"{name}: a contiguous float64 numpy array is required")
    return C.c_void_p(a.ctypes.data)


def si_solve_host(n, omega, w, sigma_t, sigma_s, q, phi, psi=None, air: air_params | None = None,
                  si: si_params | None = None, phi_reduce=None):
    """si_solve on HOST arrays (float64 numpy arrays or CPU tensors; pinned tensors
    make the copies asynchronous): the library copies sigma_t, sigma_s, q and the
    initial phi to the device on the current stream, solves, and writes phi (and
    psi, (M, N), if given) back in place.  Returns the info dict."""
    air = air or default_air_params()
    si = si or default_si_params()
    red = None
    if phi_reduce is not None:
        red = phi_reduce if isinstance(phi_reduce, ReduceCallback) else ReduceCallback(phi_reduce)
        si = si_params.from_buffer_copy(si)
        si.phi_reduce = red.cfunc
    om = np.ascontiguousarray(omega, dtype=np.float64)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    mstruct, _, _ = _mesh_struct(n)
    info = si_info()
    quad = pair_quad(om.shape[0], om.ctypes.data, ww.ctypes.data)
    rc = lib().si_solve(C.byref(mstruct), C.byref(quad), _host_ptr(sigma_t, "sigma_t"), _host_ptr(sigma_s, "sigma_s"),
                        _host_ptr(q, "q"), C.byref(air), C.byref(si), _host_ptr(phi, "phi"), _host_ptr(psi, "psi"),
                        _stream(), C.byref(info))
    if red is not None and red.error is not None and rc == -11:
        raise PairError(rc, lib().pair_last_error().decode()) from red.error
    _check(rc)
    return {f: getattr(info, f) if not isinstance(getattr(info, f), C.Array) else list(getattr(info, f))
            for f, _ in si_info._fields_}


def si_solve_problem(prob, mesh=None, **kw):
    """si_solve on an inputs.HexProblem or inputs.TetProblem (mesh: a TetMesh to reuse)."""
    if hasattr(prob, "tets"):
        mesh = mesh or TetMesh(prob.verts, prob.tets, prob.nbr)
        return si_solve(mesh, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q, **kw)
    return si_solve(prob.n, prob.omega, prob.w, prob.sigma_t, prob.sigma_s, prob.q, **kw)


def csr_transpose(rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor):
    """Transpose of a device CSR matrix (columns ascending in every row)."""
    n = rowptr.numel() - 1
    trp = torch.empty_like(rowptr)
    tc = torch.empty_like(col)
    tv = torch.empty_like(val)
    desc = pair_csr(n, col.numel(), rowptr.data_ptr(), col.data_ptr(), val.data_ptr())
    _check(lib().pair_csr_transpose(C.byref(desc), _dptr(trp), _dptr(tc), _dptr(tv), _stream()))
    return trp, tc, tv


def sweep(rowptr: torch.Tensor, col: torch.Tensor, val: torch.Tensor, b: torch.Tensor, nb: int):
    """Exact solve of one block-scaled upwind operator (device CSR, nb DOFs per
    element) by the level-scheduled GPU sweep.  Returns (x, cyclic components, levels)."""
    n = rowptr.numel() - 1
    b = b.to(torch.float64).contiguous()
    x = torch.empty_like(b)
    nc, nl = C.c_int(), C.c_int()
    desc = pair_csr(n, col.numel(), rowptr.data_ptr(), col.data_ptr(), val.data_ptr())
    _check(lib().pair_sweep(C.byref(desc), nb, _dptr(b), _dptr(x), _stream(), C.byref(nc), C.byref(nl)))
    return x, nc.value, nl.value


def si_adjoint(n, omega, w, sigma_t, sigma_s, q, psi: torch.Tensor, g: torch.Tensor,
               air: air_params | None = None, si: si_params | None = None, device="cuda"):
    """Gradients of J = g^T phi w.r.t. sigma_t, sigma_s and q per element, by
    adjoint source iteration on the transposed direction operators, on the n^3
    hex mesh (n an int) or on a TetMesh.
    psi: converged forward angular fluxes (M, N) on the device.
    Returns (dJ/dsigma_t, dJ/dsigma_s, dJ/dq, adjoint scalar flux, info)."""
    air = air or default_air_params()
    si = si or default_si_params()
    om = np.ascontiguousarray(omega, dtype=np.float64)
    ww = np.ascontiguousarray(w, dtype=np.float64)
    M = om.shape[0]
    mstruct, E, N = _mesh_struct(n)

    def dev_t(t):
        return torch.as_tensor(t, dtype=torch.float64).to(device).contiguous()

    st, ss, qq, gg = dev_t(sigma_t), dev_t(sigma_s), dev_t(q), dev_t(g)
    psi = dev_t(psi).reshape(M, N)
    dst = torch.empty(E, dtype=torch.float64, device=device)
    dss = torch.empty_like(dst)
    dq = torch.empty_like(dst)
    phis = torch.empty(N, dtype=torch.float64, device=device)
    info = si_info()
    quad = pair_quad(M, om.ctypes.data, ww.ctypes.data)
    _check(lib().si_adjoint(C.byref(mstruct), C.byref(quad), _dptr(st), _dptr(ss), _dptr(qq), _dptr(psi),
                            _dptr(gg), C.byref(air), C.byref(si), _dptr(dst), _dptr(dss), _dptr(dq), _dptr(phis),
                            _stream(), C.byref(info)))
    return dst, dss, dq, phis, {f: getattr(info, f) for f, _ in si_info._fields_ if f != "t_setup_phase_ms"}


class SIFunction(torch.autograd.Function):
    """phi = SI(sigma_t, sigma_s, q) on the n^3 hex mesh (or a TetMesh) with a fixed quadrature;
    backward runs the adjoint source iteration (si_adjoint) with g = dL/dphi."""

    @staticmethod
    def forward(ctx, sigma_t, sigma_s, q, n, omega, w, air=None, si=None):
        phi, psi, _ = si_solve(n, omega, w, sigma_t.detach(), sigma_s.detach(), q.detach(), air=air, si=si,
                               want_psi=True, device=sigma_t.device)
        ctx.save_for_backward(sigma_t, sigma_s, q, psi)
        ctx.cfg = (n, omega, w, air, si)
        return phi

    @staticmethod
    def backward(ctx, grad_phi):
        sigma_t, sigma_s, q, psi = ctx.saved_tensors
        n, omega, w, air, si = ctx.cfg
        dst, dss, dq, _, _ = si_adjoint(n, omega, w, sigma_t.detach(), sigma_s.detach(), q.detach(), psi,
                                        grad_phi.detach().contiguous(), air=air, si=si, device=sigma_t.device)
        return dst, dss, dq, None, None, None, None, None
