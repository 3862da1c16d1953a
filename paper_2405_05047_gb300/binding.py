"""ctypes binding of ``include/mg.h``.

The functions named like the C entry points (``mg_setup``, ``mg_solve``, ...)
take the same arguments, with torch tensors accepted wherever the C function
takes a device pointer and numpy arrays wherever it takes a host pointer.
``Context`` / ``Hierarchy`` wrap them for convenience.  Device memory of the
hierarchy comes from PyTorch's caching allocator through the ``mg_allocator``
callbacks, and every call runs on the CUDA stream the context was created
with (PyTorch's current stream by default).
"""
from __future__ import annotations

import ctypes as C
import os
import sys
import weakref

import numpy as np

MG_OK, MG_PENDING = 0, 1
MG_ERR_INVALID, MG_ERR_OOM, MG_ERR_ADMISSION = -1, -2, -3
MG_ERR_NOT_CONVERGED, MG_ERR_BREAKDOWN, MG_ERR_NAN, MG_ERR_TIMEOUT, MG_ERR_CUDA = -4, -5, -6, -7, -8
# solve outcomes that still come with valid statistics (and x)
SOLVE_OUTCOMES = (MG_OK, MG_ERR_NOT_CONVERGED, MG_ERR_BREAKDOWN, MG_ERR_NAN)
MG_FP64, MG_MIXED_FP32, MG_MIXED_BF16 = 0, 1, 2
MG_ERR_CANCELLED = -9
MG_SMOOTHER_JACOBI, MG_SMOOTHER_VANKA = 0, 1
MG_POISSON, MG_TRANSPORT, MG_ELASTICITY, MG_OSEEN = 0, 1, 2, 3
MG_KRYLOV_AUTO, MG_CG, MG_BICGSTAB, MG_GMRES, MG_MGITER = 0, 1, 2, 3, 4
MG_OP_MATVEC, MG_OP_SMOOTH, MG_OP_RESTRICT, MG_OP_PROLONG_ADD, MG_OP_COARSE = 0, 1, 2, 3, 4
MG_TIME_VCYCLE, MG_TIME_VCYCLE_GRAPH = 5, 6

_HERE = os.path.dirname(os.path.abspath(__file__))


def lib_path() -> str:
    return os.path.join(_HERE, "libmg_gb300.so")


class MGError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"mg error {code}: {msg}")
        self.code = code


class MgMesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("origin", C.c_double * 3), ("extent", C.c_double * 3),
                ("macro", C.c_int * 3), ("n_leaves", C.c_int64),
                ("leaf_level", C.POINTER(C.c_int32)), ("leaf_anchor", C.POINTER(C.c_int32)),
                ("axis", C.c_void_p * 3)]


class MgProblem(C.Structure):
    _fields_ = [("kind", C.c_int), ("eps", C.c_double), ("beta", C.c_double * 3), ("mu", C.c_double),
                ("lambda_", C.c_double), ("supg_delta0", C.c_double), ("dirichlet_mask", C.c_uint32 * 3),
                ("nu", C.c_double), ("dt", C.c_double), ("lps_alpha0", C.c_double), ("conv", C.c_void_p),
                ("mass", C.c_double), ("pin_origin", C.c_int)]


class MgOpts(C.Structure):
    _fields_ = [("nu1", C.c_int), ("nu2", C.c_int), ("omega", C.c_double), ("min_level", C.c_int),
                ("max_levels", C.c_int), ("krylov", C.c_int), ("restart", C.c_int), ("store_fp64", C.c_int),
                ("store_fp32", C.c_int), ("launch_mode", C.c_int),
                ("tail_rows", C.c_int), ("store_bf16", C.c_int), ("autotune", C.c_int),
                ("inner_rtol", C.c_double), ("sell_sigma", C.c_int), ("col16", C.c_int),
                ("row_lanes", C.c_int), ("smoother", C.c_int), ("vanka_rows", C.c_int),
                ("vanka_omega", C.c_double), ("stage_x", C.c_int)]


class MgInfo(C.Structure):
    _fields_ = [("dim", C.c_int), ("nc", C.c_int), ("levels", C.c_int), ("n_nodes", C.c_int64),
                ("n_dofs", C.c_int64), ("n_free", C.c_int64), ("level_nodes", C.c_int64 * 32),
                ("level_nnzb", C.c_int64 * 32), ("level_rows_nnzb", C.c_int64 * 32),
                ("bytes_device", C.c_size_t), ("n_hanging", C.c_int64), ("omega", C.c_double),
                ("bytes_workspace", C.c_size_t), ("tail_levels", C.c_int), ("tail_cluster", C.c_int),
                ("vcycle_ms", C.c_double), ("col16_slices", C.c_int64), ("col32_slices", C.c_int64),
                ("level_col16", C.c_int * 32), ("level_omega", C.c_double * 32),
                ("level_block_values", C.c_int * 32), ("level_smoother", C.c_int * 32),
                ("level_vanka_nnzb", C.c_int64 * 32),
                ("level_sigma", C.c_int64 * 32),
                ("level_lanes", C.c_int * 32)]


class MgStats(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("vcycles", C.c_int), ("precision", C.c_int),
                ("rel_res", C.c_double), ("solve_ms", C.c_double), ("setup_ms", C.c_double),
                ("launches", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MgProfEntry(C.Structure):
    _fields_ = [("kernel", C.c_char * 128), ("level", C.c_int), ("launches", C.c_int64), ("ms", C.c_double)]


_MALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class MgNsParams(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("graded", C.c_int), ("re", C.c_double),
                ("dt", C.c_double), ("lid", C.c_double), ("prec", C.c_int), ("krylov", C.c_int),
                ("rtol", C.c_double), ("max_it", C.c_int), ("nu", C.c_int), ("smoother", C.c_int)]


class MgNsStats(C.Structure):
    _fields_ = [("steps", C.c_int), ("status", C.c_int), ("iters", C.c_int64), ("iters_max", C.c_int),
                ("rel_res_max", C.c_double), ("ms_momentum", C.c_double), ("ms_pres_rhs", C.c_double),
                ("ms_pres_solve", C.c_double), ("ms_pres_up", C.c_double), ("ms_total", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MgAllocator(C.Structure):
    _fields_ = [("malloc_fn", _MALLOC), ("free_fn", _FREE), ("user", C.c_void_p)]


_lib = None

# the C ABI: name -> (restype, argtypes)
_SIGS = {
    "mg_strerror": (C.c_char_p, [C.c_int]),
    "mg_last_error": (C.c_char_p, []),
    "mg_default_opts": (None, [C.POINTER(MgOpts)]),
    "mg_init": (C.c_int, [C.c_int, C.c_size_t, C.POINTER(MgAllocator), C.c_void_p, C.POINTER(C.c_void_p)]),
    "mg_destroy": (C.c_int, [C.c_void_p]),
    "mg_setup": (C.c_int, [C.c_void_p, C.POINTER(MgMesh), C.POINTER(MgProblem), C.POINTER(MgOpts),
                           C.POINTER(C.c_void_p)]),
    "mg_hier_info": (C.c_int, [C.c_void_p, C.POINTER(MgInfo)]),
    "mg_node_coords": (C.c_int, [C.c_void_p, C.c_void_p]),
    "mg_free": (C.c_int, [C.c_void_p]),
    "mg_assemble_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mg_mesh_nodes": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "mg_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_int,
                           C.POINTER(MgStats)]),
    "mg_solve_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_int,
                                C.POINTER(MgStats)]),
    "mg_solve_profiled": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_int,
                                    C.POINTER(MgStats), C.POINTER(MgProfEntry), C.c_int, C.POINTER(C.c_int)]),
    "mg_vcycle": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "mg_apply": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "mg_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_int,
                            C.POINTER(C.c_uint64)]),
    "mg_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(MgStats)]),
    "mg_cancel": (C.c_int, [C.c_void_p, C.c_uint64]),
    "mg_launch_count": (C.c_int64, [C.c_void_p]),
    "mg_time_op": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double)]),
    "mg_serve_config": (C.c_int, [C.c_void_p, C.c_int]),
    "mg_serve_reserve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "mg_tune": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int]),
    "mg_restrict_static": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "mg_time_steps": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int,
                                C.c_int, C.POINTER(MgStats)]),
    "mg_solve_batch": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                 C.POINTER(C.c_void_p), C.c_double, C.c_int, C.c_int, C.POINTER(MgStats)]),
    "mg_batch_fits": (C.c_int, [C.c_void_p, C.c_int]),
    "mg_update_problem": (C.c_int, [C.c_void_p, C.POINTER(MgProblem)]),
    "mg_serve_batching": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "mg_ns_default_params": (None, [C.POINTER(MgNsParams)]),
    "mg_ns_setup": (C.c_int, [C.c_void_p, C.POINTER(MgNsParams), C.POINTER(C.c_void_p)]),
    "mg_ns_sizes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "mg_ns_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "mg_ns_steps": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(MgNsStats)]),
    "mg_ns_pressure_hierarchy": (C.c_void_p, [C.c_void_p]),
    "mg_ns_free": (C.c_int, [C.c_void_p]),
    "mg_time_steps2": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                 C.c_double, C.c_int, C.c_int, C.POINTER(MgStats)]),
}


def load_library(path: str | None = None):
    """Load the in-tree CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or lib_path()
    if not os.path.exists(path):
        raise MGError(-8, f"{path} not built: run paper_2405_05047_gb300/build.py (needs nvcc)")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name, None)
        if fn is None:
            continue
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc, allow=(MG_OK,)):
    if rc not in allow:
        lib = load_library()
        raise MGError(rc, f"{lib.mg_strerror(rc).decode()}: {lib.mg_last_error().decode()}")
    return rc


def _ptr(t):
    """Device pointer of a torch tensor (must be contiguous) or an int."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    assert t.is_contiguous(), "vectors must be contiguous"
    return t.data_ptr()


def _host_ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- allocator
class _TorchAllocator:
    """mg_allocator backed by torch.cuda.caching_allocator_alloc."""

    def __init__(self, device, stream):
        import torch
        self._torch = torch
        self.device = device
        self.stream = stream

        def _m(size, user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(size), self.device, self.stream))
            except Exception:
                return None

        def _f(ptr, user):
            torch.cuda.caching_allocator_delete(int(ptr))

        self.cm = _MALLOC(_m)
        self.cf = _FREE(_f)
        self.struct = MgAllocator(self.cm, self.cf, None)


# ---------------------------------------------------------------- C entry points
def mg_init(device=0, hbm_budget_bytes=0, allocator="torch", stream=None):
    """Returns (ctx_handle, keepalive).  stream: a torch.cuda.Stream or None
    for PyTorch's current stream."""
    import torch
    lib = load_library()
    if not torch.cuda.is_available():
        raise MGError(-8, "no CUDA device: the GB300 library has no CPU path")
    torch.cuda.set_device(device)
    st = stream if stream is not None else torch.cuda.current_stream(device)
    keep = None
    alloc_p = None
    if allocator == "torch":
        keep = _TorchAllocator(device, st)
        alloc_p = C.byref(keep.struct)
    out = C.c_void_p()
    _check(lib.mg_init(device, hbm_budget_bytes, alloc_p, C.c_void_p(st.cuda_stream), C.byref(out)))
    return out, (keep, st)


def mg_destroy(ctx):
    return _check(load_library().mg_destroy(ctx))


def make_mesh(leafmesh):
    lev = np.ascontiguousarray(leafmesh.level, dtype=np.int32)
    anc = np.ascontiguousarray(leafmesh.anchor, dtype=np.int32)
    m = MgMesh()
    m.dim = leafmesh.dim
    for d in range(leafmesh.dim):
        m.origin[d] = leafmesh.origin[d]
        m.extent[d] = leafmesh.extent[d]
        m.macro[d] = leafmesh.macro[d]
    m.n_leaves = lev.shape[0]
    m.leaf_level = lev.ctypes.data_as(C.POINTER(C.c_int32))
    m.leaf_anchor = anc.ctypes.data_as(C.POINTER(C.c_int32))
    keep = [lev, anc]
    axis = getattr(leafmesh, "axis", None)
    if axis is not None:
        for d in range(leafmesh.dim):
            a = np.ascontiguousarray(axis[d], dtype=np.float64)
            keep.append(a)
            m.axis[d] = a.ctypes.data
    return m, tuple(keep)


def make_problem(kind=MG_POISSON, eps=1.0, beta=(0.0, 0.0, 0.0), mu=1.0, lam=1.0, supg_delta0=0.5,
                 dirichlet=(0xFF,), nu=1e-3, dt=0.01, lps_alpha0=0.5, conv=None, mass=0.0, pin_origin=0):
    """conv (OSEEN): nodal convection field at the finest nodes, (n_nodes, dim).
    mass (POISSON, TRANSPORT): coefficient s of s (u, v); 1/dt for a
    backward-Euler step."""
    p = MgProblem()
    p.mass = mass
    p.pin_origin = int(pin_origin)
    p.kind = kind
    p.eps = eps
    for d in range(3):
        p.beta[d] = beta[d] if d < len(beta) else 0.0
    p.mu = mu
    p.lambda_ = lam
    p.supg_delta0 = supg_delta0
    p.nu = nu
    p.dt = dt
    p.lps_alpha0 = lps_alpha0
    if conv is not None:
        arr = np.ascontiguousarray(conv, dtype=np.float64)
        p._conv = arr                 # kept alive with the struct
        p.conv = arr.ctypes.data
    nc = 3 if kind in (MG_ELASTICITY, MG_OSEEN) else 1
    masks = tuple(dirichlet) * (nc if len(dirichlet) == 1 else 1)
    for c in range(3):
        p.dirichlet_mask[c] = masks[c] if c < len(masks) else 0
    return p


def make_opts(**kw):
    o = MgOpts()
    load_library().mg_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def mg_setup(ctx, leafmesh, problem: MgProblem, opts: MgOpts | None = None):
    lib = load_library()
    m, keep = make_mesh(leafmesh)
    out = C.c_void_p()
    _check(lib.mg_setup(ctx, C.byref(m), C.byref(problem), C.byref(opts) if opts is not None else None,
                        C.byref(out)))
    return out


def mg_mesh_nodes(leafmesh):
    """Physical coordinates (n_nodes, dim) of the finest nodes, external order."""
    lib = load_library()
    m, keep = make_mesh(leafmesh)
    n = C.c_int64()
    _check(lib.mg_mesh_nodes(C.byref(m), C.byref(n), None))
    xyz = np.empty((n.value, leafmesh.dim), dtype=np.float64)
    _check(lib.mg_mesh_nodes(C.byref(m), C.byref(n), xyz.ctypes.data))
    return xyz


def mg_hier_info(h) -> MgInfo:
    info = MgInfo()
    _check(load_library().mg_hier_info(h, C.byref(info)))
    return info


def mg_node_coords(h, n_nodes, dim):
    xyz = np.zeros((n_nodes, dim), dtype=np.float64)
    _check(load_library().mg_node_coords(h, _host_ptr(xyz)))
    return xyz


def mg_free(h):
    return _check(load_library().mg_free(h))


def mg_assemble_rhs(h, f, b, g=None):
    return _check(load_library().mg_assemble_rhs(h, _ptr(f), _ptr(g) if g is not None else None, _ptr(b)))


def mg_solve(h, b, x, rtol, max_it, prec=MG_FP64):
    st = MgStats()
    rc = load_library().mg_solve(h, _ptr(b), _ptr(x), rtol, max_it, prec, C.byref(st))
    _check(rc, allow=SOLVE_OUTCOMES)
    return st


def mg_solve_batch(ctx, hs, bs, xs, rtol, max_it, prec=MG_MIXED_FP32):
    """Batched solve of len(hs) problems in one launch; bs / xs: device
    tensors (n_dofs doubles each).  Returns (status, [MgStats per problem])."""
    k = len(hs)
    if not (len(bs) == k and len(xs) == k):
        raise ValueError("hs, bs and xs must have the same length")
    H = (C.c_void_p * max(k, 1))(*[h for h in hs])
    Bp = (C.c_void_p * max(k, 1))(*[_ptr(b) for b in bs])
    Xp = (C.c_void_p * max(k, 1))(*[_ptr(x) for x in xs])
    st = (MgStats * max(k, 1))()
    rc = load_library().mg_solve_batch(ctx, k, H, Bp, Xp, rtol, max_it, prec, st)
    _check(rc, allow=SOLVE_OUTCOMES)
    return rc, [st[i] for i in range(k)]


def mg_batch_fits(h, prec=MG_MIXED_FP32) -> bool:
    rc = load_library().mg_batch_fits(h, prec)
    if rc < 0:
        _check(rc)
    return rc == 1


def mg_solve_profiled(h, b, x, rtol, max_it, prec=MG_FP64, cap=256):
    """mg_solve with per-kernel event timing: (stats, [{kernel, level,
    launches, ms}, ...] sorted by ms, largest first)."""
    st = MgStats()
    ents = (MgProfEntry * cap)()
    n = C.c_int(0)
    rc = load_library().mg_solve_profiled(h, _ptr(b), _ptr(x), rtol, max_it, prec, C.byref(st), ents, cap,
                                          C.byref(n))
    _check(rc, allow=SOLVE_OUTCOMES)
    out = [{"kernel": e.kernel.decode(), "level": e.level, "launches": e.launches, "ms": e.ms}
           for e in ents[:min(n.value, cap)]]
    return st, out


def mg_solve_host(h, b: np.ndarray, x: np.ndarray, rtol, max_it, prec=MG_FP64):
    st = MgStats()
    rc = load_library().mg_solve_host(h, _host_ptr(b), _host_ptr(x), rtol, max_it, prec, C.byref(st))
    _check(rc, allow=SOLVE_OUTCOMES)
    return st


def mg_time_steps(h, theta, f, g, n_steps, rtol, max_it, prec=MG_FP64):
    """Backward-Euler steps in place on theta; f, g: (n_steps, n_dofs) device
    arrays or None.  Returns (status, [MgStats per step])."""
    sts = (MgStats * max(n_steps, 1))()
    rc = load_library().mg_time_steps(h, _ptr(theta), _ptr(f) if f is not None else None,
                                      _ptr(g) if g is not None else None, n_steps, rtol, max_it, prec, sts)
    _check(rc, allow=SOLVE_OUTCOMES)
    return rc, list(sts)[:n_steps]


def mg_time_steps2(h, u, v, f, g, n_steps, dt, rtol, max_it, prec=MG_FP64):
    """Backward-Euler steps of d_t^2 u + A u = f in place on (u, v); f, g:
    (n_steps, n_dofs) device arrays or None.  Returns (status, [MgStats])."""
    sts = (MgStats * max(n_steps, 1))()
    rc = load_library().mg_time_steps2(h, _ptr(u), _ptr(v), _ptr(f) if f is not None else None,
                                       _ptr(g) if g is not None else None, n_steps, dt, rtol, max_it, prec, sts)
    _check(rc, allow=SOLVE_OUTCOMES)
    return rc, list(sts)[:n_steps]


def mg_vcycle(h, r, z, prec=MG_FP64):
    return _check(load_library().mg_vcycle(h, _ptr(r), _ptr(z), prec))


def mg_apply(h, level, op, x, x2, out, prec=MG_FP64):
    return _check(load_library().mg_apply(h, level, op, _ptr(x), _ptr(x2), _ptr(out), prec))


def mg_submit(ctx, h, b, x, rtol, max_it, prec=MG_MIXED_FP32):
    t = C.c_uint64()
    _check(load_library().mg_submit(ctx, h, _ptr(b), _ptr(x), rtol, max_it, prec, C.byref(t)))
    return t.value


def mg_poll(ctx, ticket):
    st = MgStats()
    rc = load_library().mg_poll(ctx, ticket, C.byref(st))
    return rc, st


def mg_cancel(ctx, ticket):
    return load_library().mg_cancel(ctx, ticket)


def mg_restrict_static(h, level, x, b, d, prec=MG_FP64):
    """d = R_l (b - A_l x) without any device allocation (static scratch)."""
    return _check(load_library().mg_restrict_static(h, level, _ptr(x), _ptr(b), _ptr(d), prec))


def mg_serve_config(ctx, max_slots):
    return _check(load_library().mg_serve_config(ctx, max_slots))


# ---------------------------------------------------------------- wrappers
class Context:
    def __init__(self, device=0, hbm_budget_bytes=0, allocator="torch", stream=None):
        self.handle, self._keep = mg_init(device, hbm_budget_bytes, allocator, stream)
        self.device = device
        self._hiers = weakref.WeakSet()

    @property
    def stream(self):
        return self._keep[1]

    def submit(self, hier, b, x, rtol=1e-8, max_it=200, prec=MG_MIXED_FP32):
        return mg_submit(self.handle, hier.handle, b, x, rtol, max_it, prec)

    def poll(self, ticket):
        return mg_poll(self.handle, ticket)

    def cancel(self, ticket):
        return mg_cancel(self.handle, ticket)

    def serve_config(self, max_slots):
        return mg_serve_config(self.handle, max_slots)

    def serve_batching(self, max_batch, min_batch=2):
        return _check(load_library().mg_serve_batching(self.handle, max_batch, min_batch))

    def serve_reserve(self, hier, slots, prec=MG_MIXED_FP32):
        return _check(load_library().mg_serve_reserve(self.handle, hier.handle, slots, prec))

    def solve_batch(self, hiers, bs, xs, rtol=1e-8, max_it=200, prec=MG_MIXED_FP32):
        """mg_solve_batch over Hierarchy objects: (status, [MgStats])."""
        return mg_solve_batch(self.handle, [h.handle for h in hiers], bs, xs, rtol, max_it, prec)

    def close(self):
        """Free every hierarchy of this context, then the context."""
        if self.handle:
            for h in list(self._hiers):
                h.free()
            mg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class Hierarchy:
    """A resident multigrid hierarchy for one mesh and problem."""

    def __init__(self, ctx: Context, leafmesh, problem: MgProblem, opts: MgOpts | None = None):
        self.ctx = ctx
        if not ctx.handle:
            raise MGError(-1, "context is closed")
        self.handle = mg_setup(ctx.handle, leafmesh, problem, opts)
        ctx._hiers.add(self)
        self.info = mg_hier_info(self.handle)
        self.nc = self.info.nc
        self.n_nodes = self.info.n_nodes
        self.n_dofs = self.info.n_dofs
        self.levels = self.info.levels

    def coords(self):
        return mg_node_coords(self.handle, self.n_nodes, self.info.dim)

    def level_nodes(self):
        return [self.info.level_nodes[l] for l in range(self.levels)]

    def assemble_rhs(self, f, b, g=None):
        return mg_assemble_rhs(self.handle, f, b, g)

    def solve(self, b, x, rtol=1e-10, max_it=200, prec=MG_FP64):
        return mg_solve(self.handle, b, x, rtol, max_it, prec)

    def time_steps(self, theta, f, g, n_steps, rtol=1e-10, max_it=200, prec=MG_FP64):
        return mg_time_steps(self.handle, theta, f, g, n_steps, rtol, max_it, prec)

    def update_problem(self, problem):
        """mg_update_problem: new coefficients, same mesh and structure."""
        _check(load_library().mg_update_problem(self.handle, C.byref(problem)))
        self.info = mg_hier_info(self.handle)

    def batch_fits(self, prec=MG_MIXED_FP32):
        return mg_batch_fits(self.handle, prec)

    def time_steps2(self, u, v, f, g, n_steps, dt, rtol=1e-10, max_it=200, prec=MG_FP64):
        return mg_time_steps2(self.handle, u, v, f, g, n_steps, dt, rtol, max_it, prec)

    def solve_profiled(self, b, x, rtol=1e-10, max_it=200, prec=MG_FP64):
        return mg_solve_profiled(self.handle, b, x, rtol, max_it, prec)

    def solve_host(self, b, x, rtol=1e-10, max_it=200, prec=MG_FP64):
        return mg_solve_host(self.handle, b, x, rtol, max_it, prec)

    def vcycle(self, r, z, prec=MG_FP64):
        return mg_vcycle(self.handle, r, z, prec)

    def apply(self, level, op, x, x2, out, prec=MG_FP64):
        return mg_apply(self.handle, level, op, x, x2, out, prec)

    def time_op(self, level, op, prec=MG_FP64, reps=20):
        ms = C.c_double()
        _check(load_library().mg_time_op(self.handle, level, op, prec, reps, C.byref(ms)))
        return ms.value

    def tune(self, prec=MG_MIXED_FP32, tail_rows=-1, cluster=1):
        _check(load_library().mg_tune(self.handle, prec, tail_rows, cluster))
        self.info = mg_hier_info(self.handle)

    def launch_count(self):
        return int(load_library().mg_launch_count(self.handle))

    def free(self):
        if self.handle:
            mg_free(self.handle)
            self.handle = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.free()
        except Exception:
            pass


class NavierStokes:
    """The driven cavity's explicit pressure correction (mg_ns_*): velocity
    (n_v x 3) and pressure (n_p) state on the device."""

    def __init__(self, ctx, **params):
        import torch
        lib = load_library()
        p = MgNsParams()
        lib.mg_ns_default_params(C.byref(p))
        for k, v in params.items():
            setattr(p, k, v)
        self.params = p
        h = C.c_void_p()
        _check(lib.mg_ns_setup(ctx.handle, C.byref(p), C.byref(h)))
        self.handle = h
        nv, npr = (C.c_int * 3)(), (C.c_int * 3)()
        _check(lib.mg_ns_sizes(h, nv, npr))
        self.n_vel = tuple(nv)
        self.n_pres = tuple(npr)
        self.nv = int(np.prod(self.n_vel))
        self.np = int(np.prod(self.n_pres))
        self._torch = torch

    def pressure_info(self):
        return mg_hier_info(load_library().mg_ns_pressure_hierarchy(self.handle))

    def set_state(self, u=None, p=None, q=None):
        _check(load_library().mg_ns_state(self.handle, _ptr(u), _ptr(p), _ptr(q), 0))

    def get_state(self):
        t = self._torch
        u = t.empty((self.nv, 3), device="cuda", dtype=t.float64)
        p = t.empty(self.np, device="cuda", dtype=t.float64)
        q = t.empty(self.np, device="cuda", dtype=t.float64)
        _check(load_library().mg_ns_state(self.handle, _ptr(u), _ptr(p), _ptr(q), 1))
        return u, p, q

    def steps(self, n):
        st = MgNsStats()
        rc = load_library().mg_ns_steps(self.handle, n, C.byref(st))
        _check(rc, allow=SOLVE_OUTCOMES)
        return st

    def free(self):
        if self.handle:
            load_library().mg_ns_free(self.handle)
            self.handle = None
