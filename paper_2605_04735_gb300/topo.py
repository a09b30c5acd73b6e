"""Python binding of libtopo.so (ctypes): argument marshalling only.

Every step of the solve, compliance and sensitivity runs in the library's
CUDA kernels.  Device memory and streams may come from PyTorch: pass CUDA
tensors and they are handed over by pointer (no copy); numpy arrays are
passed as host pointers and copied by the library.  There is no CPU
fallback: if the library is missing this module raises on import use.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtopo.so")

OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_NO_DENSITY, ERR_NOT_SOLVED, ERR_NOT_CONVERGED, \
    ERR_NAN, ERR_TIMEOUT = 0, -1, -2, -3, -4, -5, -6, -7, -8
BC_CANTILEVER, BC_MBB, BC_ROLLER_BOX, BC_CORNERS, BC_MBB_STRIP, BC_NONE = 0, 1, 2, 3, 4, 5
LOAD_EDGE_XL_BOTTOM, LOAD_EDGE_X0_TOP, LOAD_FACE_XL_TRACTION = 0, 1, 2
LOAD_DISC_XL, LOAD_HALFDISC_X0_TOP = 3, 4
PREC_FP64, PREC_FP32, PREC_DWORD = 0, 1, 2
RESIDUAL_DWORD, RESIDUAL_FP64 = 0, 1
PRECOND_JACOBI, PRECOND_GMG = 0, 1
OPERATOR_MODAL, OPERATOR_GATHER, OPERATOR_MODAL_SINGLE, OPERATOR_MODAL_PAIR = 0, 1, 2, 3
OPERATOR_TENSOR = 4
OPERATOR_MODAL_CLUSTER = 5


class Params(C.Structure):
    _fields_ = [("E0", C.c_double), ("Emin", C.c_double), ("nu", C.c_double),
                ("penal", C.c_double), ("h", C.c_double), ("load", C.c_double)]


class SolveOpts(C.Structure):
    _fields_ = [("precision", C.c_int), ("precond", C.c_int), ("rtol", C.c_double),
                ("inner_rtol", C.c_double), ("max_iter", C.c_int), ("max_outer", C.c_int),
                ("warm_start", C.c_int), ("gmg_levels", C.c_int), ("smooth_degree", C.c_int),
                ("check_every", C.c_int), ("residual", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("outer", C.c_int), ("status", C.c_int), ("detail", C.c_int),
                ("rel_residual", C.c_double), ("seconds", C.c_double)]


class SimpOpts(C.Structure):
    _fields_ = [("volfrac", C.c_double), ("filter_radius", C.c_double), ("move", C.c_double),
                ("eta", C.c_double), ("rho_min", C.c_double)]


class SimpInfo(C.Structure):
    _fields_ = [("compliance", C.c_double), ("volume", C.c_double), ("change", C.c_double),
                ("lambda_", C.c_double)]


class JobResult(C.Structure):
    _fields_ = [("job", C.c_int), ("design", C.c_int), ("status", C.c_int), ("detail", C.c_int),
                ("iters", C.c_int),
                ("outer", C.c_int), ("rel_residual", C.c_double), ("compliance", C.c_double),
                ("submit_s", C.c_double), ("start_s", C.c_double), ("finish_s", C.c_double)]


class TopoError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


_lib = None


def lib():
    """Load libtopo.so (built by __graft_entry__.build()); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libtopo.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        vp, i, sz, d = C.c_void_p, C.c_int, C.c_size_t, C.c_double
        sig = {
            "topo_default_params": (None, [C.POINTER(Params)]),
            "topo_default_opts": (None, [C.POINTER(SolveOpts)]),
            "topo_create_mesh": (i, [i, i, i, i, i, C.POINTER(Params), vp, C.POINTER(vp)]),
            "topo_create_batch": (i, [i, i, i, i, i, C.POINTER(Params), vp, i, i, i,
                                      C.POINTER(vp)]),
            "topo_set_density": (i, [vp, vp, sz, i]),
            "topo_solve": (i, [vp, C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
            "topo_solve_many": (i, [C.POINTER(vp), i, C.POINTER(SolveOpts), C.POINTER(SolveInfo)]),
            "topo_compliance": (i, [vp, C.POINTER(d)]),
            "topo_compliance_energy": (i, [vp, C.POINTER(d)]),
            "topo_sensitivity": (i, [vp, vp, sz, i]),
            "topo_get_displacement": (i, [vp, vp, sz, i]),
            "topo_set_displacement": (i, [vp, vp, sz, i]),
            "topo_apply": (i, [vp, i, vp, vp, sz, i]),
            "topo_apply_internal": (i, [vp, i, i]),
            "topo_mesh_info": (i, [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                   C.POINTER(C.c_longlong)]),
            "topo_footprint_bytes": (C.c_longlong, [i, i, i, C.POINTER(SolveOpts)]),
            "topo_set_stream": (i, [vp, vp]),
            "topo_set_levelset": (i, [vp, vp, sz, i, d, d, C.POINTER(d)]),
            "topo_element_energy": (i, [vp, vp, sz, i]),
            "topo_get_levelset": (i, [vp, vp, sz, i]),
            "topo_shape_rhs": (i, [vp, vp, vp, sz, i]),
            "topo_hilbertian_solve": (i, [vp, d, vp, vp, sz, i, d, i, C.POINTER(i)]),
            "topo_hj_evolve": (i, [vp, vp, sz, i, d, i, C.POINTER(d)]),
            "topo_reinit": (i, [vp, d, d, i, C.POINTER(i)]),
            "topo_nodal_density": (i, [vp, vp, sz, i]),
            "topo_levelset_from_density": (i, [vp, d, C.POINTER(C.c_longlong)]),
            "topo_extract_levelset_surface": (i, [vp, C.POINTER(C.c_longlong)]),
            "topo_get_surface": (i, [vp, vp, sz, i, C.POINTER(C.c_longlong)]),
            "topo_set_operator": (i, [vp, i]),
            "topo_profile_enable": (i, [vp, i]),
            "topo_profile_read": (i, [vp, C.POINTER(d), C.POINTER(C.c_longlong),
                                      C.POINTER(C.c_longlong), i]),
            "topo_debug_inject_timeout": (i, [vp, i]),
            "topo_set_throughput_mode": (i, [vp, i]),
            "topo_jacobi_inverse": (i, [vp, vp, sz, i]),
            "topo_profile_read_smoother": (i, [vp, C.POINTER(d), C.POINTER(C.c_longlong),
                                               C.POINTER(d), i]),
            "topo_sensitivity_noalloc": (i, [i, i, i, C.POINTER(Params), vp, vp, vp, vp, vp]),
            "topo_set_density_many": (i, [vp, i, vp, sz, i]),
            "topo_compliance_many": (i, [vp, i, vp]),
            "topo_sensitivity_many": (i, [vp, i, vp, sz, i]),
            "topo_server_create": (i, [C.c_longlong, i, C.POINTER(Params), C.POINTER(SolveOpts), vp,
                                       C.POINTER(vp)]),
            "topo_server_open": (i, [vp, i, i, i, i, i, C.POINTER(i)]),
            "topo_server_submit": (i, [vp, i, vp, sz, C.POINTER(i)]),
            "topo_server_poll": (i, [vp, i, C.POINTER(JobResult), i, C.POINTER(i)]),
            "topo_server_sensitivity": (i, [vp, i, vp, sz, i]),
            "topo_server_displacement": (i, [vp, i, vp, sz, i]),
            "topo_server_close": (i, [vp, i]),
            "topo_server_stats": (i, [vp, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong),
                                      C.POINTER(i), C.POINTER(i)]),
            "topo_server_free": (None, [vp]),
            "topo_default_simp_opts": (None, [C.POINTER(SimpOpts)]),
            "topo_simp_update": (i, [vp, C.POINTER(SimpOpts), C.POINTER(SimpInfo)]),
            "topo_filter": (i, [vp, d, vp, vp, sz, i]),
            "topo_get_density": (i, [vp, vp, sz, i]),
            "topo_free": (None, [vp]),
            "topo_status_string": (C.c_char_p, [i]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def status_string(st: int) -> str:
    return lib().topo_status_string(int(st)).decode()


def _check(st: int, what: str):
    if st != OK:
        raise TopoError(st, what)


def default_params(**kw) -> Params:
    p = Params()
    lib().topo_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def default_opts(**kw) -> SolveOpts:
    o = SolveOpts()
    lib().topo_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def default_simp_opts(**kw) -> SimpOpts:
    o = SimpOpts()
    lib().topo_default_simp_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def footprint_bytes(nx, ny, nz, opts: SolveOpts | None = None) -> int:
    return int(lib().topo_footprint_bytes(nx, ny, nz, C.byref(opts) if opts else None))


def sensitivity_noalloc(nx, ny, nz, u, rho, dc, c, params: Params | None = None, stream=None):
    """topo_sensitivity_noalloc on CUDA tensors (u: float64 DOFs, rho: float32
    elements, dc: float64 elements, c: one float64); enqueued, not synchronised.

    The C entry point receives raw pointers and cannot see how long they are,
    so the sizes are checked here, before anything is launched: u must hold
    3 (nx+1)(ny+1)(nz+1) values, rho and dc nx ny nz, c at least one
    (ValueError otherwise)."""
    pu, nu_, du = _ptr(u, np.float64)
    pr, nr, dr = _ptr(rho, np.float32)
    pd, nd, dd = _ptr(dc, np.float64)
    pc, nc, dcc = _ptr(c, np.float64)
    n_elem = int(nx) * int(ny) * int(nz)
    n_dof = 3 * (int(nx) + 1) * (int(ny) + 1) * (int(nz) + 1)
    if min(nx, ny, nz) < 1:
        raise ValueError("grid sizes must be positive")
    if nu_ != n_dof or nr != n_elem or nd != n_elem or nc < 1:
        raise ValueError(f"sizes do not match the {nx}x{ny}x{nz} grid: u {nu_} (want {n_dof}), "
                         f"rho {nr} and dc {nd} (want {n_elem}), c {nc} (want >= 1)")
    if not (du and dr and dd and dcc):
        raise TypeError("topo_sensitivity_noalloc takes device arrays only")
    s = None if stream is None else C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    _check(lib().topo_sensitivity_noalloc(nx, ny, nz, C.byref(params) if params else None,
                                          pu, pr, pd, pc, s), "topo_sensitivity_noalloc")


def _ptr(a, dtype):
    """(pointer, count, on_device) of a numpy array or a CUDA torch tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a C-contiguous {np.dtype(dtype).name} array")
        return a.ctypes.data, a.size, 0
    # torch tensor (duck-typed so numpy users need no torch)
    if not a.is_contiguous():
        raise TypeError("expected a contiguous tensor")
    want = {np.float32: "torch.float32", np.float64: "torch.float64"}[dtype]
    if str(a.dtype) != want:
        raise TypeError(f"expected {want}, got {a.dtype}")
    return a.data_ptr(), a.numel(), 1 if a.is_cuda else 0


def solve_many(meshes, opts: SolveOpts | None = None, check: bool = True):
    """Solve several meshes concurrently (one host thread, one stream each)."""
    n = len(meshes)
    arr = (C.c_void_p * n)(*[m._h for m in meshes])
    infos = (SolveInfo * n)()
    st = lib().topo_solve_many(arr, n, C.byref(opts) if opts else None, infos)
    if check:
        _check(st, "topo_solve_many")
    return list(infos)


def _handles(meshes):
    return (C.c_void_p * len(meshes))(*[m._h for m in meshes])


def set_density_many(meshes, rho):
    """Densities of n meshes of one grid at once (topo_set_density_many):
    rho is an (n, n_elem) float32 array or CUDA tensor, row b for meshes[b]."""
    n = len(meshes)
    p, cnt, dev = _ptr(rho, np.float32)
    if n == 0 or cnt % n:
        raise ValueError("rho must hold n_elem values per mesh")
    _check(lib().topo_set_density_many(_handles(meshes), n, p, cnt // n, dev),
           "topo_set_density_many")


def compliance_many(meshes) -> np.ndarray:
    """f^T u of each solved mesh (topo_compliance_many)."""
    n = len(meshes)
    c = np.empty(n, np.float64)
    _check(lib().topo_compliance_many(_handles(meshes), n, c.ctypes.data), "topo_compliance_many")
    return c


def sensitivity_many(meshes, out=None):
    """Element sensitivities of n solved meshes of one grid
    (topo_sensitivity_many) into `out`, an (n, n_elem) float64 array or CUDA
    tensor (default: a new numpy array)."""
    n = len(meshes)
    if out is None:
        out = np.empty((n, meshes[0].n_elem), np.float64)
    p, cnt, dev = _ptr(out, np.float64)
    if n == 0 or cnt % n:
        raise ValueError("out must hold n_elem values per mesh")
    _check(lib().topo_sensitivity_many(_handles(meshes), n, p, cnt // n, dev),
           "topo_sensitivity_many")
    return out


def _stream_arg(stream):
    if stream is None:
        return None
    return C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)


def create_batch(n, nx, ny, nz, bc=None, load=None, params: "Params | None" = None,
                 stream=None, opts: "SolveOpts | None" = None):
    """n meshes of one grid that solve_many runs as one batch (topo_create_batch);
    `opts` fixes the multigrid settings (default: default_opts())."""
    bc = BC_CANTILEVER if bc is None else bc
    load = LOAD_EDGE_XL_BOTTOM if load is None else load
    o = opts or default_opts()
    hs = (C.c_void_p * n)()
    _check(lib().topo_create_batch(nx, ny, nz, bc, load, C.byref(params) if params else None,
                                   _stream_arg(stream), n, o.gmg_levels, o.smooth_degree, hs),
           "topo_create_batch")
    return [Mesh(nx, ny, nz, bc, load, _handle=C.c_void_p(h)) for h in hs]


class Mesh:
    """One structured hex8 design domain held on the current CUDA device."""

    def __init__(self, nx, ny, nz, bc=BC_CANTILEVER, load=LOAD_EDGE_XL_BOTTOM,
                 params: Params | None = None, stream=None, _handle=None):
        if _handle is not None:
            h = _handle
        else:
            h = C.c_void_p()
            _check(lib().topo_create_mesh(nx, ny, nz, bc, load,
                                          C.byref(params) if params else None,
                                          _stream_arg(stream), C.byref(h)), "topo_create_mesh")
        self._h = h
        self.nx, self.ny, self.nz, self.bc, self.load = nx, ny, nz, bc, load
        self.n_elem = nx * ny * nz
        self.n_nodes = (nx + 1) * (ny + 1) * (nz + 1)
        self.n_dof = 3 * self.n_nodes

    def close(self):
        if getattr(self, "_h", None):
            lib().topo_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_density(self, rho):
        p, n, dev = _ptr(rho, np.float32)
        _check(lib().topo_set_density(self._h, p, n, dev), "topo_set_density")

    def solve(self, opts: SolveOpts | None = None, check: bool = True) -> SolveInfo:
        info = SolveInfo()
        st = lib().topo_solve(self._h, C.byref(opts) if opts else None, C.byref(info))
        if check:
            _check(st, "topo_solve")
        return info

    def compliance(self) -> float:
        c = C.c_double()
        _check(lib().topo_compliance(self._h, C.byref(c)), "topo_compliance")
        return c.value

    def compliance_energy(self) -> float:
        c = C.c_double()
        _check(lib().topo_compliance_energy(self._h, C.byref(c)), "topo_compliance_energy")
        return c.value

    def sensitivity(self, out=None):
        if out is None:
            out = np.empty(self.n_elem, dtype=np.float64)
        p, n, dev = _ptr(out, np.float64)
        _check(lib().topo_sensitivity(self._h, p, n, dev), "topo_sensitivity")
        return out

    def displacement(self, out=None):
        if out is None:
            out = np.empty(self.n_dof, dtype=np.float64)
        p, n, dev = _ptr(out, np.float64)
        _check(lib().topo_get_displacement(self._h, p, n, dev), "topo_get_displacement")
        return out

    def set_displacement(self, u):
        p, n, dev = _ptr(u, np.float64)
        _check(lib().topo_set_displacement(self._h, p, n, dev), "topo_set_displacement")

    def apply(self, x, precision=PREC_FP64, out=None):
        if out is None:
            out = np.empty(self.n_dof, dtype=np.float64)
        px, n, dev = _ptr(x, np.float64)
        py, n2, dev2 = _ptr(out, np.float64)
        if dev != dev2:
            raise TypeError("x and out must both be host or both be device arrays")
        _check(lib().topo_apply(self._h, precision, px, py, n, dev), "topo_apply")
        return out

    def set_levelset(self, phi=None, eta=1.0, eps0=1e-3) -> float:
        """Ersatz material from the nodal level set phi (Eqs. (7)-(9)), or from
        the mesh's current level set if phi is None; returns the material
        volume V(phi) of Eq. (10)."""
        if phi is None:
            p, n, dev = None, self.n_nodes, 0
        else:
            p, n, dev = _ptr(phi, np.float64)
        vol = C.c_double()
        _check(lib().topo_set_levelset(self._h, p, n, dev, eta, eps0, C.byref(vol)),
               "topo_set_levelset")
        return vol.value

    def levelset(self, out=None):
        if out is None:
            out = np.empty(self.n_nodes, np.float64)
        p, n, dev = _ptr(out, np.float64)
        _check(lib().topo_get_levelset(self._h, p, n, dev), "topo_get_levelset")
        return out

    def shape_rhs(self):
        """(bJ, bV): nodal right-hand sides of Eqs. (14), (15) for the last solve."""
        bJ = np.empty(self.n_nodes, np.float64)
        bV = np.empty(self.n_nodes, np.float64)
        _check(lib().topo_shape_rhs(self._h, bJ.ctypes.data, bV.ctypes.data, self.n_nodes, 0),
               "topo_shape_rhs")
        return bJ, bV

    def hilbertian_solve(self, b, ell, rtol=1e-10, max_iter=2000, out=None):
        """v with A_H v = b, v = 0 on the loaded nodes (Eqs. (19), (20)); returns (v, iters)."""
        if out is None:
            out = np.empty(self.n_nodes, np.float64)
        pb, n, dev = _ptr(b, np.float64)
        pv, n2, dev2 = _ptr(out, np.float64)
        if n != n2 or dev != dev2:
            raise TypeError("b and out must be alike")
        it = C.c_int()
        _check(lib().topo_hilbertian_solve(self._h, ell, pb, pv, n, dev, rtol, max_iter,
                                           C.byref(it)), "topo_hilbertian_solve")
        return out, it.value

    def hj_evolve(self, v, gamma=0.5, steps=1) -> float:
        """Evolve the mesh's level set under speed v (Eqs. (21), (22)); returns dt."""
        p, n, dev = _ptr(v, np.float64)
        dt = C.c_double()
        _check(lib().topo_hj_evolve(self._h, p, n, dev, gamma, steps, C.byref(dt)),
               "topo_hj_evolve")
        return dt.value

    def nodal_density(self, out=None):
        """Nodal densities of the current element densities (Eqs. (25)-(27))."""
        if out is None:
            out = np.empty(self.n_nodes, np.float64)
        p, n, dev = _ptr(out, np.float64)
        _check(lib().topo_nodal_density(self._h, p, n, dev), "topo_nodal_density")
        return out

    def levelset_from_density(self, rho_t=0.5) -> int:
        """SIMP -> level set: nodal densities, iso-surface, signed distance
        (Eqs. (25)-(30)) into the mesh's level set; returns the triangle count."""
        n = C.c_longlong()
        _check(lib().topo_levelset_from_density(self._h, rho_t, C.byref(n)),
               "topo_levelset_from_density")
        return n.value

    def extract_levelset_surface(self) -> int:
        n = C.c_longlong()
        _check(lib().topo_extract_levelset_surface(self._h, C.byref(n)),
               "topo_extract_levelset_surface")
        return n.value

    def surface(self):
        """The last extracted triangle soup, (n, 3, 3) float64."""
        n = C.c_longlong()
        lib().topo_get_surface(self._h, None, 0, 0, C.byref(n))
        out = np.empty((n.value, 3, 3), np.float64)
        _check(lib().topo_get_surface(self._h, out.ctypes.data if n.value else None, n.value, 0,
                                      C.byref(n)), "topo_get_surface")
        return out

    def reinit(self, gamma=0.5, tol=1e-4, max_steps=500) -> int:
        """Reinitialise the mesh's level set (Eqs. (23), (24)); returns the steps taken."""
        st = C.c_int()
        _check(lib().topo_reinit(self._h, gamma, tol, max_steps, C.byref(st)), "topo_reinit")
        return st.value

    def element_energy(self, out=None):
        """w_e = u_e^T k^0 u_e (unit E) of the last solve."""
        if out is None:
            out = np.empty(self.n_elem, np.float64)
        p, n, dev = _ptr(out, np.float64)
        _check(lib().topo_element_energy(self._h, p, n, dev), "topo_element_energy")
        return out

    def apply_internal(self, precision=PREC_FP32, reps=1):
        _check(lib().topo_apply_internal(self._h, precision, reps), "topo_apply_internal")

    def simp_update(self, opts: SimpOpts | None = None) -> SimpInfo:
        info = SimpInfo()
        _check(lib().topo_simp_update(self._h, C.byref(opts) if opts else None, C.byref(info)),
               "topo_simp_update")
        return info

    def filter(self, dc, radius=2.0, out=None):
        if out is None:
            out = np.empty(self.n_elem, np.float64)
        p, n, dev = _ptr(dc, np.float64)
        q, n2, dev2 = _ptr(out, np.float64)
        _check(lib().topo_filter(self._h, radius, p, q, n, dev), "topo_filter")
        return out

    def density(self, out=None):
        if out is None:
            out = np.empty(self.n_elem, np.float32)
        p, n, dev = _ptr(out, np.float32)
        _check(lib().topo_get_density(self._h, p, n, dev), "topo_get_density")
        return out

    def set_operator(self, kind):
        """OPERATOR_MODAL (default, automatic FP32 kernel form), OPERATOR_GATHER,
        OPERATOR_MODAL_SINGLE, OPERATOR_MODAL_PAIR, OPERATOR_TENSOR or
        OPERATOR_MODAL_CLUSTER for all later calls."""
        _check(lib().topo_set_operator(self._h, kind), "topo_set_operator")

    def set_stream(self, stream):
        """Order subsequent calls against `stream` (int handle or torch.cuda.Stream)."""
        s = C.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
        _check(lib().topo_set_stream(self._h, s), "topo_set_stream")

    def info(self):
        a, b, c = C.c_longlong(), C.c_longlong(), C.c_longlong()
        _check(lib().topo_mesh_info(self._h, C.byref(a), C.byref(b), C.byref(c)), "topo_mesh_info")
        return {"n_nodes": a.value, "n_free_dof": b.value, "device_bytes": c.value}

    def profile(self, enable=True):
        _check(lib().topo_profile_enable(self._h, int(enable)), "topo_profile_enable")

    def profile_read(self, reset=True):
        """(summed ms of the timed operator launches, their count, all kernel launches)."""
        ms, n, a = C.c_double(), C.c_longlong(), C.c_longlong()
        _check(lib().topo_profile_read(self._h, C.byref(ms), C.byref(n), C.byref(a), int(reset)),
               "topo_profile_read")
        return ms.value, n.value, a.value

    def jacobi_inverse(self, out=None):
        """1 / diag(K) in FP64, DOF order (topo_jacobi_inverse)."""
        if out is None:
            out = np.empty(self.n_dof, dtype=np.float64)
        p, n, dev = _ptr(out, np.float64)
        _check(lib().topo_jacobi_inverse(self._h, p, n, dev), "topo_jacobi_inverse")
        return out

    def set_throughput_mode(self, enable: bool = True):
        """The multigrid's throughput form (topo_set_throughput_mode), as the
        solve server uses for its designs."""
        _check(lib().topo_set_throughput_mode(self._h, int(bool(enable))),
               "topo_set_throughput_mode")

    def debug_inject_timeout(self, count: int = 1):
        """Arm (1) or disarm (0) the test hook of topo_debug_inject_timeout."""
        _check(lib().topo_debug_inject_timeout(self._h, int(count)), "topo_debug_inject_timeout")

    def profile_read_smoother(self, reset=True):
        """(summed ms of the timed finest-level Chebyshev steps, design-launches,
        their algorithmic bytes)."""
        ms, n, b = C.c_double(), C.c_longlong(), C.c_double()
        _check(lib().topo_profile_read_smoother(self._h, C.byref(ms), C.byref(n), C.byref(b),
                                                int(reset)), "topo_profile_read_smoother")
        return ms.value, n.value, b.value


class Server:
    """Continuous-batching solve server (see topo_server_* in include/topo.h)."""

    def __init__(self, mem_budget_bytes: int, max_active: int = 64, params: Params | None = None,
                 opts: SolveOpts | None = None, stream=None):
        h = C.c_void_p()
        st = None if stream is None else C.c_void_p(stream if isinstance(stream, int)
                                                     else stream.cuda_stream)
        _check(lib().topo_server_create(int(mem_budget_bytes), int(max_active),
                                        C.byref(params) if params else None,
                                        C.byref(opts) if opts else None, st, C.byref(h)),
               "topo_server_create")
        self._h = h
        self._dims = {}

    def close(self):
        if getattr(self, "_h", None):
            lib().topo_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def open(self, nx, ny, nz, bc, load) -> int:
        d = C.c_int()
        _check(lib().topo_server_open(self._h, nx, ny, nz, bc, load, C.byref(d)), "topo_server_open")
        self._dims[d.value] = (nx, ny, nz)
        return d.value

    def submit(self, design: int, rho: np.ndarray) -> int:
        p, n, dev = _ptr(rho, np.float32)
        if dev:
            raise TypeError("topo_server_submit takes host densities")
        j = C.c_int()
        _check(lib().topo_server_submit(self._h, design, p, n, C.byref(j)), "topo_server_submit")
        return j.value

    def poll(self, wait: bool = False, max_out: int = 256):
        out = (JobResult * max_out)()
        n = C.c_int()
        _check(lib().topo_server_poll(self._h, int(wait), out, max_out, C.byref(n)),
               "topo_server_poll")
        return [out[k] for k in range(n.value)]

    def sensitivity(self, design: int, out=None):
        nx, ny, nz = self._dims[design]
        if out is None:
            out = np.empty(nx * ny * nz, np.float64)
        p, n, dev = _ptr(out, np.float64)
        _check(lib().topo_server_sensitivity(self._h, design, p, n, dev), "topo_server_sensitivity")
        return out

    def displacement(self, design: int, out=None):
        nx, ny, nz = self._dims[design]
        if out is None:
            out = np.empty(3 * (nx + 1) * (ny + 1) * (nz + 1), np.float64)
        p, n, dev = _ptr(out, np.float64)
        _check(lib().topo_server_displacement(self._h, design, p, n, dev),
               "topo_server_displacement")
        return out

    def retire(self, design: int):
        _check(lib().topo_server_close(self._h, design), "topo_server_close")

    def stats(self):
        a, b, c, d = C.c_longlong(), C.c_longlong(), C.c_int(), C.c_int()
        _check(lib().topo_server_stats(self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)),
               "topo_server_stats")
        return {"bytes_in_use": a.value, "peak_bytes": b.value, "active": c.value,
                "waiting": d.value}


def simp_optimize(mesh: "Mesh", rho0, simp_opts: SimpOpts | None = None,
                  solve_opts: SolveOpts | None = None, max_iter: int = 100, tol: float = 0.01,
                  callback=None):
    """SIMP loop on the device: solve (warm-started), then filter + OC update,
    until max |Delta rho| <= tol (Sec. 4.1's stopping rule) or max_iter.
    Returns the per-iteration (compliance, volume, change) history."""
    mesh.set_density(rho0)
    hist = []
    for it in range(max_iter):
        so = solve_opts or default_opts()
        so.warm_start = 1 if it else 0
        mesh.solve(so)
        info = mesh.simp_update(simp_opts)
        hist.append((info.compliance, info.volume, info.change))
        if callback:
            callback(it, info)
        if info.change <= tol:
            break
    return hist
