"""Python binding of the GB300 p-multigrid spectral element Laplace solver.

Argument marshalling only: every function forwards to the C ABI of
``libsem_gb300.so`` (declared in ``include/sem.h``) with the same name.  Device
buffers are passed as CUDA tensors (or raw device pointers), streams as
``torch.cuda.Stream`` (or raw ``cudaStream_t`` integers).  Importing this
module fails loudly when the CUDA library has not been built: there is no CPU
fallback of any kind.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, byref, c_byte, c_char_p, c_double, c_int, c_longlong, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsem_gb300.so")
SEM_MAX_LEVELS = 8

SEM_OK, SEM_NOT_CONVERGED = 0, 1
SEM_EINVAL, SEM_ECUDA, SEM_ENOMEM, SEM_NAN, SEM_BREAKDOWN, SEM_TIMEOUT = -1, -2, -3, -4, -5, -6
OUTER = {"pcg": 0, "fgmres": 1, "pdc": 2}
PRECISION = {"fp64": 0, "mixed_fp32": 1, "mixed_tf32": 2}
SMOOTHER = {"chebyshev": 0, "learned": 1, "asm": 2}

EXPORTS = ("sem_default_options", "sem_mesh_nodes2d", "sem_setup", "sem_teardown", "sem_query",
           "sem_dirichlet_nodes", "sem_node_coords", "sem_element_map", "sem_lambda_max", "sem_diagonal",
           "sem_apply", "sem_apply32", "sem_update_eta", "sem_fnpf_rhs", "sem_fnpf_step", "pmg_vcycle", "laplace_solve", "laplace_solve_host", "sem_last_error",
           "sem_cg_csr_noalloc", "sem_mlp_get_weights", "sem_mlp_set_weights", "sem_mlp_forward",
           "sem_mlp_gradient", "sem_mlp_adam", "sem_learned_sweep", "sem_learned_train", "laplace_solve_batch", "sem_tile_shapes", "sem_tc_kernel", "sem_elem_matrices", "sem_fp64_rate",
           "sem_asm_subdomains", "sem_asm_apply", "sem_asm_apply32")


class SemMesh(Structure):
    _fields_ = [("dim", c_int), ("nvert", c_int), ("vxy", POINTER(c_double)), ("ntri", c_int),
                ("tri", POINTER(c_int)), ("nlayers", c_int), ("depth", c_double),
                ("eta", POINTER(c_double)), ("face_bc", POINTER(c_byte)), ("col_layers", POINTER(c_int)),
                ("z_iface", POINTER(c_double)), ("edge_arc", POINTER(c_double))]


class SemOptions(Structure):
    _fields_ = [("outer", c_int), ("precision", c_int), ("nu1", c_int), ("nu2", c_int), ("k_cheb", c_int),
                ("cheb_lo", c_double), ("cheb_hi", c_double), ("lanczos_steps", c_int), ("nlevels", c_int),
                ("level_p", c_int * SEM_MAX_LEVELS), ("rtol", c_double), ("atol", c_double), ("imax", c_int),
                ("gmres_m", c_int), ("coarse_rtol", c_double), ("coarse_imax", c_int), ("profile", c_int),
                ("inner_imax", c_int), ("inner_rtol", c_double), ("debug_barrier_extra", c_int),
                ("smoother", c_int), ("mlp_hidden", c_int), ("mlp_seed", ctypes.c_ulonglong), ("batch", c_int),
                ("autotune", c_int), ("learned_tau", c_double), ("surface_ops", c_int), ("batch_mode", c_int),
                ("asm_overlap", c_int), ("level_pz", c_int * SEM_MAX_LEVELS), ("deterministic", c_int),
                ("elem_matrices", c_int), ("coarse_bj", c_int), ("fused_small", c_int)]


class SemStats(Structure):
    _fields_ = [("status", c_int), ("iters", c_int), ("fnorm", c_double), ("res0", c_double),
                ("res_final", c_double), ("q_mean", c_double), ("fine_applies", c_longlong),
                ("vcycles", c_longlong), ("coarse_iters_max", c_int), ("ms", c_double),
                ("apply_ms", c_double), ("apply_launches", c_longlong), ("kernel_launches", c_longlong),
                ("inner_iters", c_longlong), ("learned_accepts", c_longlong), ("learned_fallbacks", c_longlong),
                ("graph_iterations", c_longlong), ("apply32_ms", c_double), ("apply32_launches", c_longlong),
                ("apply_tc_ms", c_double), ("apply_tc_launches", c_longlong), ("asm_ms", c_double),
                ("asm_launches", c_longlong), ("lift_ms", c_double), ("lift_launches", c_longlong)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class SemError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"status {status}: {msg}")
        self.status = status


_lib = None


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2009_00705_gb300.build.build() "
                          "(the solver has no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    L.sem_default_options.argtypes = [POINTER(SemOptions), c_int]
    L.sem_default_options.restype = None
    L.sem_mesh_nodes2d.argtypes = [POINTER(SemMesh), c_int, POINTER(c_longlong), POINTER(c_double)]
    L.sem_setup.argtypes = [POINTER(SemMesh), c_int, POINTER(SemOptions), POINTER(c_void_p)]
    L.sem_teardown.argtypes = [c_void_p]
    L.sem_teardown.restype = None
    L.sem_query.argtypes = [c_void_p, c_int, POINTER(c_longlong), POINTER(c_longlong), POINTER(c_longlong),
                            POINTER(c_int)]
    L.sem_dirichlet_nodes.argtypes = [c_void_p, c_int, POINTER(c_longlong)]
    L.sem_node_coords.argtypes = [c_void_p, c_int, POINTER(c_double)]
    L.sem_element_map.argtypes = [c_void_p, c_int, POINTER(c_int)]
    L.sem_lambda_max.argtypes = [c_void_p, POINTER(c_double)]
    L.sem_diagonal.argtypes = [c_void_p, c_int, POINTER(c_double)]
    L.sem_tile_shapes.argtypes = [c_void_p, c_int, POINTER(c_int), POINTER(c_int)]
    L.sem_tile_shapes.restype = c_int
    L.sem_tc_kernel.argtypes = [c_void_p, c_int, POINTER(c_int)]
    L.sem_tc_kernel.restype = c_int
    L.sem_elem_matrices.argtypes = [c_void_p, c_int, POINTER(c_int)]
    L.sem_elem_matrices.restype = c_int
    L.sem_fp64_rate.argtypes = [POINTER(c_double)]
    L.sem_fp64_rate.restype = c_int
    L.sem_apply.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_void_p]
    L.sem_apply32.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_int, c_void_p]
    L.sem_update_eta.argtypes = [c_void_p, POINTER(c_double), c_int]
    L.sem_asm_subdomains.argtypes = [c_void_p, c_int, POINTER(c_longlong), POINTER(c_int)]
    L.sem_asm_apply.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_int, c_void_p]
    L.sem_asm_apply32.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_int, c_void_p]
    L.sem_fnpf_rhs.argtypes = [c_void_p, c_void_p, c_void_p, c_double, c_int, c_int, c_double, c_void_p, c_void_p,
                               c_void_p]
    L.sem_fnpf_step.argtypes = [c_void_p, c_void_p, c_void_p, c_double, c_double, c_int, c_int, c_double,
                                POINTER(SemStats), c_void_p]
    L.pmg_vcycle.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    L.laplace_solve.argtypes = [c_void_p, c_void_p, c_void_p, c_double, c_void_p, POINTER(SemStats), c_void_p]
    L.laplace_solve_host.argtypes = [c_void_p, c_void_p, c_void_p, c_double, c_void_p, POINTER(SemStats),
                                     c_void_p]
    L.sem_last_error.restype = c_char_p
    L.sem_cg_csr_noalloc.argtypes = [c_longlong, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                     c_double, c_int, POINTER(c_int), c_void_p]
    L.sem_cg_csr_noalloc.restype = c_int
    fp = POINTER(ctypes.c_float)
    L.sem_mlp_get_weights.argtypes = [c_void_p, fp, fp, fp, fp]
    L.sem_mlp_set_weights.argtypes = [c_void_p, fp, fp, fp, fp]
    L.sem_mlp_forward.argtypes = [c_void_p, c_int, c_void_p, c_void_p, c_void_p]
    L.sem_mlp_gradient.argtypes = [c_void_p, c_int, c_void_p, c_void_p, POINTER(c_double), fp, fp, fp, fp, c_void_p]
    L.sem_learned_train.argtypes = [c_void_p, c_int, c_int, c_double, ctypes.c_ulonglong, POINTER(c_double),
                                    POINTER(c_double), c_void_p]
    L.sem_mlp_adam.argtypes = [c_void_p, fp, fp, fp, fp, c_double, c_int, c_void_p]
    L.sem_learned_sweep.argtypes = [c_void_p, c_void_p, c_void_p, POINTER(c_int), POINTER(c_double), c_void_p]
    L.laplace_solve_batch.argtypes = [POINTER(c_void_p), c_int, POINTER(c_void_p), c_double, POINTER(c_void_p),
                                      POINTER(SemStats), c_void_p]
    for name in ("sem_mlp_get_weights", "sem_mlp_set_weights", "sem_mlp_forward", "sem_mlp_gradient",
                 "sem_mlp_adam", "sem_learned_sweep", "sem_learned_train", "laplace_solve_batch"):
        getattr(L, name).restype = c_int
    for name in ("sem_mesh_nodes2d", "sem_setup", "sem_query", "sem_dirichlet_nodes", "sem_node_coords",
                 "sem_element_map", "sem_lambda_max", "sem_diagonal", "sem_apply", "sem_apply32", "sem_update_eta", "sem_fnpf_rhs", "sem_fnpf_step", "pmg_vcycle",
                 "laplace_solve", "laplace_solve_host"):
        getattr(L, name).restype = c_int
    _lib = L
    return L


def _check(status: int, allow=(SEM_OK,)) -> int:
    if status not in allow:
        raise SemError(status, lib().sem_last_error().decode())
    return status


def _ptr(t) -> int:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(s) -> int | None:
    if s is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _dptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(POINTER(ctype))


class _MeshArgs:
    """Keeps the numpy arrays of a SemMesh alive while the library reads them."""

    def __init__(self, mesh, eta_nodal=None):
        self.vxy = np.ascontiguousarray(mesh.vxy, dtype=np.float64)
        self.tri = np.ascontiguousarray(mesh.tri, dtype=np.int32)
        self.fb = np.ascontiguousarray(mesh.face_bc, dtype=np.int8)
        self.eta = None if eta_nodal is None else np.ascontiguousarray(eta_nodal, dtype=np.float64)

        def opt(name, dtype):
            v = getattr(mesh, name, None)
            return None if v is None else np.ascontiguousarray(v, dtype=dtype)

        self.col = opt("col_layers", np.int32)
        self.zif = opt("z_iface", np.float64)
        self.arc = opt("edge_arc", np.float64)
        self.s = SemMesh(int(mesh.dim), int(self.vxy.shape[0]), _dptr(self.vxy, c_double), int(self.tri.shape[0]),
                         _dptr(self.tri, c_int), int(getattr(mesh, "nlayers", 0) or 0),
                         float(getattr(mesh, "depth", 1.0)),
                         _dptr(self.eta, c_double) if self.eta is not None else None, _dptr(self.fb, c_byte),
                         _dptr(self.col, c_int) if self.col is not None else None,
                         _dptr(self.zif, c_double) if self.zif is not None else None,
                         _dptr(self.arc, c_double) if self.arc is not None else None)


# ---------------------------------------------------------------- C ABI, same names
def sem_default_options(P: int, **overrides) -> SemOptions:
    o = SemOptions()
    lib().sem_default_options(byref(o), int(P))
    for k, v in overrides.items():
        if k == "levels":
            # orders p, or (p, pz) pairs for anisotropic prism levels (semi-coarsening)
            o.nlevels = len(v)
            for i, p in enumerate(v):
                p, pz = (p if isinstance(p, (tuple, list)) else (p, 0))
                o.level_p[i] = int(p)
                o.level_pz[i] = int(pz)
        elif k == "outer":
            o.outer = OUTER[v] if isinstance(v, str) else int(v)
        elif k == "precision":
            o.precision = PRECISION[v] if isinstance(v, str) else int(v)
        elif k == "smoother":
            o.smoother = SMOOTHER[v] if isinstance(v, str) else int(v)
        elif k in dict(SemOptions._fields_):
            setattr(o, k, v)
        else:
            raise TypeError(f"unknown solver option {k!r}")
    return o


def sem_mesh_nodes2d(mesh, p: int) -> np.ndarray:
    m = _MeshArgs(mesh)
    n = c_longlong(0)
    _check(lib().sem_mesh_nodes2d(byref(m.s), int(p), byref(n), None))
    xy = np.zeros((n.value, 2))
    _check(lib().sem_mesh_nodes2d(byref(m.s), int(p), byref(n), _dptr(xy, c_double)))
    return xy


def sem_setup(mesh, P: int, opts: SemOptions | None = None, eta_nodal=None) -> int:
    m = _MeshArgs(mesh, eta_nodal)
    h = c_void_p()
    _check(lib().sem_setup(byref(m.s), int(P), byref(opts) if opts is not None else None, byref(h)))
    return h.value


def sem_teardown(h: int) -> None:
    lib().sem_teardown(h)


def sem_query(h: int, level: int = 0) -> dict:
    N, nd, ne, npe = c_longlong(), c_longlong(), c_longlong(), c_int()
    _check(lib().sem_query(h, level, byref(N), byref(nd), byref(ne), byref(npe)))
    return {"ndof": N.value, "ndirichlet": nd.value, "nelem": ne.value, "np": npe.value}


def sem_dirichlet_nodes(h: int, level: int = 0) -> np.ndarray:
    q = sem_query(h, level)
    out = np.zeros(q["ndirichlet"], dtype=np.int64)
    _check(lib().sem_dirichlet_nodes(h, level, _dptr(out, c_longlong)))
    return out


def sem_node_coords(h: int, level: int = 0, dim: int = 3) -> np.ndarray:
    q = sem_query(h, level)
    out = np.zeros((q["ndof"], dim))
    _check(lib().sem_node_coords(h, level, _dptr(out, c_double)))
    return out


def sem_element_map(h: int, level: int = 0) -> np.ndarray:
    q = sem_query(h, level)
    out = np.zeros((q["nelem"], q["np"]), dtype=np.int32)
    _check(lib().sem_element_map(h, level, _dptr(out, c_int)))
    return out


def sem_lambda_max(h: int, nlevels: int) -> np.ndarray:
    out = np.zeros(nlevels)
    _check(lib().sem_lambda_max(h, _dptr(out, c_double)))
    return out


def sem_diagonal(h: int, level: int = 0) -> np.ndarray:
    q = sem_query(h, level)
    out = np.zeros(q["ndof"])
    _check(lib().sem_diagonal(h, level, _dptr(out, c_double)))
    return out


def sem_fp64_rate() -> float:
    """Measured FP64 FMA rate of the current device (TFLOP/s)."""
    r = c_double(0.0)
    _check(lib().sem_fp64_rate(byref(r)))
    return r.value


def sem_tc_kernel(h: int, level: int = 0) -> int:
    """The Chebyshev sweeps' operator at a level under MIXED_TF32: 0 FP32 apply, 1 warp-level
    MMA kernel, 2 tcgen05 kernel."""
    k = c_int(0)
    _check(lib().sem_tc_kernel(h, level, byref(k)))
    return k.value


def sem_tile_shapes(h: int, level: int = 0):
    """(elements per CTA pass of the FP64 prism apply, of the FP32 one) at a level."""
    a, b = c_int(0), c_int(0)
    _check(lib().sem_tile_shapes(h, level, byref(a), byref(b)))
    return a.value, b.value


def sem_apply(h: int, level: int, x, y, stream=None) -> None:
    _check(lib().sem_apply(h, level, _ptr(x), _ptr(y), _stream(stream)))


def sem_asm_subdomains(h: int, level: int = 0) -> list:
    """Free global node ids of every element's Schwarz subdomain on `level` (ascending)."""
    ne = sem_query(h, level)["nelem"]
    ptr = np.zeros(ne + 1, dtype=np.int64)
    _check(lib().sem_asm_subdomains(h, level, ptr.ctypes.data_as(POINTER(c_longlong)), None))
    nodes = np.zeros(max(int(ptr[-1]), 1), dtype=np.int32)
    _check(lib().sem_asm_subdomains(h, level, None, nodes.ctypes.data_as(POINTER(c_int))))
    return [nodes[ptr[k]:ptr[k + 1]].astype(np.int64) for k in range(ne)]


def sem_asm_apply(h: int, level: int, r, z, adjoint: bool = False, stream=None) -> None:
    """z = S^{-1} r (or S^{-T} r) with the handle's Schwarz blocks (FP64 handles, double buffers)."""
    _check(lib().sem_asm_apply(h, level, _ptr(r), _ptr(z), int(bool(adjoint)), _stream(stream)))


def sem_asm_apply32(h: int, level: int, r, z, adjoint: bool = False, stream=None) -> None:
    """The same with float buffers on a mixed-precision handle."""
    _check(lib().sem_asm_apply32(h, level, _ptr(r), _ptr(z), int(bool(adjoint)), _stream(stream)))


ETA_STRATEGY = {"finest": 0, "linear_coarse": 1, "all": 2}


def sem_update_eta(h: int, eta_nodal, strategy="all") -> None:
    """New surface elevation at the order-P 2D nodes; strategy 'finest', 'linear_coarse' or 'all'."""
    e = np.ascontiguousarray(eta_nodal, dtype=np.float64)
    st = ETA_STRATEGY[strategy] if isinstance(strategy, str) else int(strategy)
    _check(lib().sem_update_eta(h, e.ctypes.data_as(POINTER(c_double)), st))


def sem_fnpf_rhs(h: int, eta, phis, deta, dphis, g=9.81, linear=False, strategy="all", tol=1e-10, stream=None):
    """Right-hand sides of the free-surface conditions at the surface nodes (device arrays)."""
    st = ETA_STRATEGY[strategy] if isinstance(strategy, str) else int(strategy)
    _check(lib().sem_fnpf_rhs(h, _ptr(eta), _ptr(phis), float(g), int(bool(linear)), st, float(tol), _ptr(deta),
                              _ptr(dphis), _stream(stream)))


def sem_fnpf_step(h: int, eta, phis, dt, g=9.81, linear=False, strategy="all", tol=1e-10, stream=None) -> dict:
    """One ERK4 step of (eta, phis) in place (device arrays); returns the summed solve stats."""
    st = ETA_STRATEGY[strategy] if isinstance(strategy, str) else int(strategy)
    out = SemStats()
    _check(lib().sem_fnpf_step(h, _ptr(eta), _ptr(phis), float(dt), float(g), int(bool(linear)), st, float(tol),
                               byref(out), _stream(stream)))
    return out.as_dict()


def sem_apply32(h: int, level: int, x, y, tensor_cores: int = 0, stream=None) -> None:
    """FP32 operator apply (x, y float32 device buffers); tensor_cores 1 (or True) selects the TF32
    warp-MMA kernel the V-cycle uses, 2 the tcgen05 kernel (order 6 only)."""
    _check(lib().sem_apply32(h, level, _ptr(x), _ptr(y), int(tensor_cores), _stream(stream)))


def pmg_vcycle(h: int, r, z, stream=None) -> None:
    _check(lib().pmg_vcycle(h, _ptr(r), _ptr(z), _stream(stream)))


def laplace_solve(h: int, rhs, dirichlet_eta, tol: float, phi, stream=None, allow_not_converged=False) -> dict:
    st = SemStats()
    allow = (SEM_OK, SEM_NOT_CONVERGED) if allow_not_converged else (SEM_OK,)
    _check(lib().laplace_solve(h, _ptr(rhs), _ptr(dirichlet_eta), float(tol), _ptr(phi), byref(st),
                               _stream(stream)), allow)
    return st.as_dict()


def laplace_solve_host(h: int, rhs, dirichlet_eta: np.ndarray, tol: float, phi: np.ndarray, stream=None) -> dict:
    """Host-buffer variant: dirichlet_eta / rhs / phi are host arrays (pinned memory recommended)."""
    st = SemStats()

    def hp(a):
        if a is None:
            return None
        return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
    _check(lib().laplace_solve_host(h, hp(rhs), hp(dirichlet_eta), float(tol), hp(phi), byref(st),
                                    _stream(stream)))
    return st.as_dict()


def sem_cg_csr_noalloc(n: int, rowptr, col, vals, dinv, b, x, rtol: float, imax: int, stream=None,
                       allow_not_converged=False) -> int:
    """Jacobi-PCG on a caller-supplied CSR matrix that allocates nothing (device buffers
    in, device buffer out; scratch in the library's static device array).  Returns the
    iteration count."""
    it = c_int(0)
    allow = (SEM_OK, SEM_NOT_CONVERGED) if allow_not_converged else (SEM_OK,)
    _check(lib().sem_cg_csr_noalloc(int(n), _ptr(rowptr), _ptr(col), _ptr(vals), _ptr(dinv), _ptr(b), _ptr(x),
                                    float(rtol), int(imax), byref(it), _stream(stream)), allow)
    return it.value


def _mlp_shapes(h: int, hidden: int):
    npe = sem_query(h, 0)["np"]
    return {"W1": (hidden, npe), "b1": (hidden,), "W2": (npe, hidden), "b2": (npe,)}


def sem_mlp_get_weights(h: int, hidden: int) -> dict:
    out = {k: np.zeros(v, dtype=np.float32) for k, v in _mlp_shapes(h, hidden).items()}
    fp = POINTER(ctypes.c_float)
    _check(lib().sem_mlp_get_weights(h, *(out[k].ctypes.data_as(fp) for k in ("W1", "b1", "W2", "b2"))))
    return out


def sem_mlp_set_weights(h: int, W1, b1, W2, b2) -> None:
    arrs = [np.ascontiguousarray(a, dtype=np.float32) for a in (W1, b1, W2, b2)]
    fp = POINTER(ctypes.c_float)
    _check(lib().sem_mlp_set_weights(h, *(a.ctypes.data_as(fp) for a in arrs)))


def sem_mlp_forward(h: int, B: int, X, Y, stream=None) -> None:
    _check(lib().sem_mlp_forward(h, int(B), _ptr(X), _ptr(Y), _stream(stream)))


def sem_mlp_gradient(h: int, hidden: int, B: int, X, T, stream=None):
    """(loss, dict of gradients shaped like the weights)."""
    g = {k: np.zeros(v, dtype=np.float32) for k, v in _mlp_shapes(h, hidden).items()}
    loss = c_double(0.0)
    fp = POINTER(ctypes.c_float)
    _check(lib().sem_mlp_gradient(h, int(B), _ptr(X), _ptr(T), byref(loss),
                                  *(g[k].ctypes.data_as(fp) for k in ("W1", "b1", "W2", "b2")), _stream(stream)))
    return loss.value, g


def sem_mlp_adam(h: int, grads: dict, lr: float, reset: bool = False, stream=None) -> None:
    """One Adam step of the network's master weights with the given gradients (host arrays
    shaped like the weights: keys W1, b1, W2, b2)."""
    fp = POINTER(ctypes.c_float)
    g = {k: np.ascontiguousarray(grads[k], dtype=np.float32) for k in ("W1", "b1", "W2", "b2")}
    _check(lib().sem_mlp_adam(h, *(g[k].ctypes.data_as(fp) for k in ("W1", "b1", "W2", "b2")), float(lr),
                              1 if reset else 0, _stream(stream)))


def sem_learned_sweep(h: int, f, u, stream=None):
    """One learned sweep on the finest level (FP32 device vectors; u updated in place).
    Returns (accepted, alpha)."""
    acc, alpha = c_int(0), c_double(0.0)
    _check(lib().sem_learned_sweep(h, _ptr(f), _ptr(u), byref(acc), byref(alpha), _stream(stream)))
    return bool(acc.value), alpha.value


def sem_learned_train(h: int, snapshots: int, steps: int, lr: float = 1e-3, seed: int = 1, stream=None):
    """(loss of the first step, loss of the last step)."""
    l0, l1 = c_double(0.0), c_double(0.0)
    _check(lib().sem_learned_train(h, int(snapshots), int(steps), float(lr), ctypes.c_ulonglong(seed), byref(l0),
                                   byref(l1), _stream(stream)))
    return l0.value, l1.value


def laplace_solve_batch(handles, etas, tol: float, phis, stream=None, allow_not_converged=False):
    """Lockstep batched solve of several tanks (handles set up with batch=1, inner_imax=0);
    returns the list of per-tank stats."""
    n = len(handles)
    hs = (c_void_p * n)(*[int(h) for h in handles])
    es = (c_void_p * n)(*[_ptr(e) for e in etas])
    ps = (c_void_p * n)(*[_ptr(p) for p in phis])
    st = (SemStats * n)()
    allow = (SEM_OK, SEM_NOT_CONVERGED) if allow_not_converged else (SEM_OK,)
    _check(lib().laplace_solve_batch(hs, n, es, float(tol), ps, st, _stream(stream)), allow)
    return [st[i].as_dict() for i in range(n)]


def sem_last_error() -> str:
    return lib().sem_last_error().decode()


# ---------------------------------------------------------------- convenience wrapper
class Solver:
    """Owns one sem_handle.  ``mesh`` is any object with dim, vxy, tri, nlayers,
    depth and face_bc (e.g. workloads.Mesh); ``eta_nodal`` is eta at the order-P
    2D nodes (see sem_mesh_nodes2d), or None for a flat surface."""

    def __init__(self, mesh, P: int, eta_nodal=None, **opts):
        self.P = P
        self.dim = int(mesh.dim)
        self.opts = sem_default_options(P, **opts)
        self.nlevels = self.opts.nlevels
        self.h = sem_setup(mesh, P, self.opts, eta_nodal)

    def close(self):
        if self.h:
            sem_teardown(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query(self, level=0):
        return sem_query(self.h, level)

    def dirichlet_nodes(self, level=0):
        return sem_dirichlet_nodes(self.h, level)

    def coords(self, level=0):
        return sem_node_coords(self.h, level, self.dim)

    def element_map(self, level=0):
        return sem_element_map(self.h, level)

    def lambdas(self):
        return sem_lambda_max(self.h, self.nlevels)

    def diagonal(self, level=0):
        return sem_diagonal(self.h, level)

    def tile_shapes(self, level=0):
        return sem_tile_shapes(self.h, level)

    def tc_kernel(self, level=0):
        return sem_tc_kernel(self.h, level)

    def elem_matrices(self, level=0):
        """Form of the level's FP64 applies: 0 sum-factorised, 1 FP64 element matrices,
        2 double-FP32 element matrices."""
        kind = c_int(0)
        _check(lib().sem_elem_matrices(self.h, level, byref(kind)))
        return kind.value

    def apply(self, level, x, y, stream=None):
        sem_apply(self.h, level, x, y, stream)

    def update_eta(self, eta_nodal, strategy="all"):
        sem_update_eta(self.h, eta_nodal, strategy)

    def fnpf_rhs(self, eta, phis, deta, dphis, **kw):
        sem_fnpf_rhs(self.h, eta, phis, deta, dphis, **kw)

    def fnpf_step(self, eta, phis, dt, **kw):
        return sem_fnpf_step(self.h, eta, phis, dt, **kw)

    def apply32(self, level, x, y, tensor_cores=False, stream=None):
        sem_apply32(self.h, level, x, y, tensor_cores, stream)

    # additive Schwarz smoother (smoother="asm")
    def asm_subdomains(self, level=0):
        return sem_asm_subdomains(self.h, level)

    def asm_apply(self, level, r, z, adjoint=False, stream=None):
        sem_asm_apply(self.h, level, r, z, adjoint, stream)

    def asm_apply32(self, level, r, z, adjoint=False, stream=None):
        sem_asm_apply32(self.h, level, r, z, adjoint, stream)

    def vcycle(self, r, z, stream=None):
        pmg_vcycle(self.h, r, z, stream)

    def solve(self, dirichlet_eta, phi, tol=0.0, rhs=None, stream=None, allow_not_converged=False):
        return laplace_solve(self.h, rhs, dirichlet_eta, tol, phi, stream, allow_not_converged)

    def solve_host(self, dirichlet_eta, phi, tol=0.0, rhs=None, stream=None):
        return laplace_solve_host(self.h, rhs, dirichlet_eta, tol, phi, stream)

    # correction network of the learned smoothing sweep (smoother="learned")
    def mlp_weights(self):
        return sem_mlp_get_weights(self.h, self.opts.mlp_hidden)

    def set_mlp_weights(self, W1, b1, W2, b2):
        sem_mlp_set_weights(self.h, W1, b1, W2, b2)

    def mlp_gradient(self, B, X, T, stream=None):
        return sem_mlp_gradient(self.h, self.opts.mlp_hidden, B, X, T, stream)

    def mlp_forward(self, B, X, Y, stream=None):
        sem_mlp_forward(self.h, B, X, Y, stream)

    def adam_step(self, grads, lr, reset=False, stream=None):
        sem_mlp_adam(self.h, grads, lr, reset, stream)

    def learned_sweep(self, f, u, stream=None):
        return sem_learned_sweep(self.h, f, u, stream)

    def train(self, snapshots, steps, lr=1e-3, seed=1, stream=None):
        return sem_learned_train(self.h, snapshots, steps, lr, seed, stream)
