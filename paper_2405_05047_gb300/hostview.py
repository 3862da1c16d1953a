"""Host-only view of the hierarchy the library builds (``include/mg_debug.h``).

Returns the library's own level matrices as scipy CSR matrices for
inspection and for CPU-side tests; nothing here is on the solve path.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import scipy.sparse as sp

from . import binding as B

_SIGS = {
    "mg_host_build": (C.c_int, [C.POINTER(B.MgMesh), C.POINTER(B.MgProblem), C.POINTER(B.MgOpts),
                                C.POINTER(C.c_void_p)]),
    "mg_host_levels": (C.c_int, [C.c_void_p]),
    "mg_host_level": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                C.POINTER(C.c_int), C.POINTER(C.c_int64), C.POINTER(C.POINTER(C.c_int64)),
                                C.POINTER(C.POINTER(C.c_int64)), C.POINTER(C.POINTER(C.c_double))]),
    "mg_host_nodes": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.POINTER(C.c_uint8)), C.POINTER(C.c_int64)]),
    "mg_host_coarse_inverse": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.POINTER(C.c_double))]),
    "mg_host_omega": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "mg_host_free": (C.c_int, [C.c_void_p]),
}

A, P, R, LOAD, SMOOTHER, HMAT, LIFT = 0, 1, 2, 3, 4, 5, 6


def _lib():
    lib = B.load_library()
    for n, (res, args) in _SIGS.items():
        f = getattr(lib, n)
        f.restype, f.argtypes = res, args
    return lib


class HostHierarchy:
    def __init__(self, leafmesh, problem, opts=None):
        self.lib = _lib()
        m, self._keep = B.make_mesh(leafmesh)
        out = C.c_void_p()
        rc = self.lib.mg_host_build(C.byref(m), C.byref(problem), C.byref(opts) if opts is not None else None,
                                    C.byref(out))
        if rc != 0:
            raise B.MGError(rc, B.load_library().mg_last_error().decode())
        self.h = out
        self.levels = self.lib.mg_host_levels(self.h)

    def matrix(self, level, which):
        n, m, nb, nnz = C.c_int64(), C.c_int64(), C.c_int(), C.c_int64()
        ptr, col, val = C.POINTER(C.c_int64)(), C.POINTER(C.c_int64)(), C.POINTER(C.c_double)()
        rc = self.lib.mg_host_level(self.h, level, which, C.byref(n), C.byref(m), C.byref(nb), C.byref(nnz),
                                    C.byref(ptr), C.byref(col), C.byref(val))
        if rc != 0:
            raise B.MGError(rc)
        n, m, nc, nnz = n.value, m.value, nb.value, nnz.value
        if n == 0:                      # a matrix the level does not have
            return sp.csr_matrix((0, 0))
        p = np.ctypeslib.as_array(ptr, shape=(n + 1,)).copy()
        c = np.ctypeslib.as_array(col, shape=(max(nnz, 1),))[:nnz].copy()
        v = np.ctypeslib.as_array(val, shape=(max(nnz * nc * nc, 1),))[:nnz * nc * nc].copy()
        if nc == 1:
            return sp.csr_matrix((v, c, p), shape=(n, m))
        return sp.bsr_matrix((v.reshape(nnz, nc, nc), c, p), shape=(n * nc, m * nc)).tocsr()

    def fixmask(self, level):
        fm, n = C.POINTER(C.c_uint8)(), C.c_int64()
        self.lib.mg_host_nodes(self.h, level, C.byref(fm), C.byref(n))
        return np.ctypeslib.as_array(fm, shape=(n.value,)).copy()

    def omega(self, level):
        w = C.c_double()
        self.lib.mg_host_omega(self.h, level, C.byref(w))
        return w.value

    def coarse_inverse(self):
        n, inv = C.c_int64(), C.POINTER(C.c_double)()
        self.lib.mg_host_coarse_inverse(self.h, C.byref(n), C.byref(inv))
        return np.ctypeslib.as_array(inv, shape=(n.value * n.value,)).copy().reshape(n.value, n.value)

    def __del__(self):
        try:
            self.lib.mg_host_free(self.h)
        except Exception:
            pass
