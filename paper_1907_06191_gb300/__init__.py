"""Python binding of libdgsigma (include/dgsigma.h): GB300-native DG
diffusion in the extracellular space around axons and the displacement
covariance Sigma (Cervantes et al., arXiv 1907.06191).

The functions here carry the C names and only marshal arguments (numpy
arrays, ctypes structs); every step of the method runs in the library's
CUDA kernels.  There is no fallback: if the library has not been built the
import raises.  ``DGSolver`` is a small convenience wrapper over the same
calls.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

__all__ = [
    "DG_OK", "DG_EINVAL", "DG_ENOMEM", "DG_ECUDA", "DG_EUNSTABLE", "DG_ENONFINITE",
    "DG_ETIMEOUT", "DG_ESTATE", "DG_FP64", "DG_FP32", "DG_WALL_REMOVED",
    "DG_WALL_PAPER", "DG_BC_ABSORBING", "DG_BC_PERIODIC", "DG_ROUND_NEAREST",
    "DG_ROUND_STOCHASTIC", "DG_ELEMENT_SQUARE", "DG_ELEMENT_TRIANGLE", "DgError", "dg_config",
    "dg_info", "lib", "library_path", "DGSolver", "EXPORTS",
]

DG_OK, DG_EINVAL, DG_ENOMEM, DG_ECUDA = 0, 1, 2, 3
DG_EUNSTABLE, DG_ENONFINITE, DG_ETIMEOUT, DG_ESTATE = 4, 5, 6, 7
DG_FP64, DG_FP32 = 0, 1
DG_WALL_REMOVED, DG_WALL_PAPER = 0, 1
DG_BC_ABSORBING, DG_BC_PERIODIC = 0, 1
DG_ROUND_NEAREST, DG_ROUND_STOCHASTIC = 0, 1
DG_ELEMENT_SQUARE, DG_ELEMENT_TRIANGLE = 0, 1


class dg_config(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("precision", ctypes.c_int),
                ("D", ctypes.c_double), ("sigma0", ctypes.c_double),
                ("eta", ctypes.c_double), ("cfl_safety", ctypes.c_double),
                ("wall_mode", ctypes.c_int), ("boundary", ctypes.c_int),
                ("power_iters", ctypes.c_int), ("device", ctypes.c_int),
                ("rounding", ctypes.c_int), ("element", ctypes.c_int)]


class dg_info(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("n_nodes", ctypes.c_int),
                ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("n_active", ctypes.c_longlong), ("dof_per_source", ctypes.c_longlong),
                ("m", ctypes.c_int), ("precision", ctypes.c_int),
                ("h", ctypes.c_double), ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("t", ctypes.c_double), ("steps", ctypes.c_longlong),
                ("state_bytes", ctypes.c_size_t), ("halo_max", ctypes.c_int),
                ("n_geometries", ctypes.c_int), ("n_elements_padded", ctypes.c_longlong)]


_P = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_I, _D, _SZ = ctypes.c_int, ctypes.c_double, ctypes.c_size_t

# name -> (restype, argtypes); the exported C ABI
EXPORTS = {
    "dg_config_default": (None, [ctypes.POINTER(dg_config)]),
    "dg_create": (_I, [ctypes.POINTER(dg_config), ctypes.POINTER(_P)]),
    "dg_destroy": (None, [_P]),
    "dg_strerror": (ctypes.c_char_p, [_I]),
    "dg_last_error": (ctypes.c_char_p, [_P]),
    "dg_set_stream": (_I, [_P, _P]),
    "dg_set_geometry_mask": (_I, [_P, _P, _I, _I, _D, _D, _D]),
    "dg_set_geometry_disks": (_I, [_P, _DP, _DP, _DP, _I, _D, _I, _I]),
    "dg_set_geometry_batch": (_I, [_P, _I, _P, _DP, _DP, _DP, _DP, _P, _P]),
    "dg_get_mask": (_I, [_P, _P]),
    "dg_get_info": (_I, [_P, ctypes.POINTER(dg_info)]),
    "dg_set_sources": (_I, [_P, _DP, _I]),
    "dg_query_dt": (_I, [_P, _DP, _DP]),
    "dg_step": (_I, [_P, _I, _D]),
    "dg_propagate_to": (_I, [_P, _D]),
    "dg_moments": (_I, [_P, _DP]),
    "dg_covariance": (_I, [_P, _DP, _DP, _DP]),
    "dg_covariance_batch": (_I, [_P, _DP, _DP, _DP]),
    "dg_ls_residual": (_I, [_P, _DP]),
    "dg_mixture_covariance": (_I, [_P, _DP, _DP, _I, _DP, _DP]),
    "dg_apply_operator": (_I, [_P]),
    "dg_get_nodes": (_I, [_P, _DP]),
    "dg_set_nodes": (_I, [_P, _DP]),
    "dg_get_elements": (_I, [_P, _P, _I, _DP]),
    "dg_get_elements_batch": (_I, [_P, _P, _I, _DP]),
    "dg_state_size": (_I, [_P, ctypes.POINTER(_SZ)]),
    "dg_get_state": (_I, [_P, _P, _SZ]),
    "dg_set_state": (_I, [_P, _P, _SZ]),
    "dg_state_bytes": (_I, [_P, _I, ctypes.POINTER(_SZ)]),
    "dg_bind_state": (_I, [_P, _P, _SZ]),
    "dg_moments_dense_static": (_I, [_P, _I, _I, _I, _I, _I, _D, _D, _D, _P, _P, _P]),
    "dg_rasterize_disks": (_I, [_DP, _DP, _DP, _I, _D, _I, _P]),
    "dg_basis_tables": (_I, [_I, _I, _DP, _DP, _DP, _DP]),
    "dg_set_growing_window": (_I, [_P, _D]),
    "dg_debug_fail_alloc": (_I, [_I]),
    "dg_set_launch": (_I, [_P, _I]),
    "dg_get_launch": (_I, [_P, ctypes.POINTER(_I)]),
    "dg_set_contraction": (_I, [_P, _I]),
    "dg_get_contraction": (_I, [_P, ctypes.POINTER(_I)]),
    "dg_set_triangle_fusion": (_I, [_P, _I]),
    "dg_get_triangle_fusion": (_I, [_P, ctypes.POINTER(_I)]),
    "dg_debug_copies": (_I, [_P, _I, ctypes.POINTER(ctypes.c_ulonglong)]),
    "dg_triangle_tables": (_I, [_I, _DP, _DP, _DP, _DP, _DP]),
    # learned surrogate (include/dgsurrogate.h)
    "sg_create": (_I, [_I, ctypes.c_ulonglong, _I, ctypes.POINTER(_P)]),
    "sg_destroy": (None, [_P]),
    "sg_last_error": (ctypes.c_char_p, [_P]),
    "sg_param_count": (_I, [_P, ctypes.POINTER(_SZ)]),
    "sg_get_params": (_I, [_P, _P]),
    "sg_set_params": (_I, [_P, _P]),
    "sg_predict": (_I, [_P, _P, _P, _I, _P]),
    "sg_gradients": (_I, [_P, _P, _P, _P, _I, _P, _P]),
    "sg_train_step": (_I, [_P, _P, _P, _P, _I, ctypes.c_float, _P]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """The loaded library; raises if it was not built (no fallback)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(
                f"libdgsigma is not built ({path} missing); run "
                "paper_1907_06191_gb300._build.build() or __graft_entry__.build()")
        L = ctypes.CDLL(path)
        for name, (res, args) in EXPORTS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class DgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def default_config(**kw) -> dg_config:
    cfg = dg_config()
    lib().dg_config_default(ctypes.byref(cfg))
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise TypeError(f"unknown config field {k}")
        setattr(cfg, k, v)
    return cfg


class DGSolver:
    """One library context: geometry, start points, RK3 stepping, moments and
    Sigma.  Methods map one to one onto the C calls."""

    def __init__(self, **cfg):
        self._L = lib()
        self.cfg = default_config(**cfg)
        h = _P()
        rc = self._L.dg_create(ctypes.byref(self.cfg), ctypes.byref(h))
        if rc != DG_OK:
            raise DgError(rc, f"dg_create: {self._L.dg_strerror(rc).decode()}")
        self.ctx = h
        self._bound = None

    def _ck(self, rc: int, what: str):
        if rc != DG_OK:
            msg = self._L.dg_last_error(self.ctx).decode()
            raise DgError(rc, f"{what}: {self._L.dg_strerror(rc).decode()}: {msg}")

    def close(self):
        if getattr(self, "ctx", None):
            self._L.dg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # geometry
    def set_geometry_mask(self, active, h: float, x0: float = 0.0, y0: float = 0.0):
        a = np.ascontiguousarray(active, dtype=np.uint8)
        ny, nx = a.shape
        self._ck(self._L.dg_set_geometry_mask(self.ctx, a.ctypes.data, nx, ny, h, x0, y0),
                 "dg_set_geometry_mask")

    def set_geometry_disks(self, cx, cy, r, L: float, n_cell: int, tiles: int):
        cx, cy, r = _f64(cx), _f64(cy), _f64(r)
        self._ck(self._L.dg_set_geometry_disks(self.ctx, _dp(cx), _dp(cy), _dp(r), int(r.size),
                                               L, n_cell, tiles), "dg_set_geometry_disks")

    def set_geometry_batch(self, disks_list, L, n_cell, tiles):
        """disks_list: G tuples (cx, cy, r); L, n_cell, tiles: G values each."""
        G = len(disks_list)
        nd = np.array([len(np.atleast_1d(d[2])) for d in disks_list], dtype=np.int32)
        cat = [np.concatenate([_f64(np.atleast_1d(d[k])) for d in disks_list]) if nd.sum() else
               np.zeros(1) for k in range(3)]
        Lh = _f64(L)
        nc = np.ascontiguousarray(n_cell, dtype=np.int32)
        tl = np.ascontiguousarray(tiles, dtype=np.int32)
        self._ck(self._L.dg_set_geometry_batch(self.ctx, G, nd.ctypes.data, _dp(cat[0]), _dp(cat[1]),
                                               _dp(cat[2]), _dp(Lh), nc.ctypes.data, tl.ctypes.data),
                 "dg_set_geometry_batch")

    def covariance_batch(self):
        inf = self.info()
        G = inf.n_geometries
        s3, mu, mass = np.zeros((G, 3)), np.zeros((G, 2)), np.zeros((G, inf.m))
        self._ck(self._L.dg_covariance_batch(self.ctx, _dp(s3), _dp(mu), _dp(mass)),
                 "dg_covariance_batch")
        return s3, mu, mass

    def ls_residual(self) -> np.ndarray:
        """Least-squares residual of the Gaussian fit, one value per geometry."""
        out = np.zeros(self.info().n_geometries)
        self._ck(self._L.dg_ls_residual(self.ctx, _dp(out)), "dg_ls_residual")
        return out

    def get_elements_batch(self, idx) -> np.ndarray:
        """Node values [k, n, n] of elements idx = [(geometry, source, ex, ey), ...]."""
        idx = np.ascontiguousarray(idx, dtype=np.int32).reshape(-1, 4)
        out = np.zeros((idx.shape[0],) + self.node_shape())
        self._ck(self._L.dg_get_elements_batch(self.ctx, idx.ctypes.data, idx.shape[0], _dp(out)),
                 "dg_get_elements_batch")
        return out

    def info(self) -> dg_info:
        inf = dg_info()
        self._ck(self._L.dg_get_info(self.ctx, ctypes.byref(inf)), "dg_get_info")
        return inf

    def get_mask(self) -> np.ndarray:
        inf = self.info()
        out = np.zeros((inf.ny, inf.nx), dtype=np.uint8)
        self._ck(self._L.dg_get_mask(self.ctx, out.ctypes.data), "dg_get_mask")
        return out

    # sources and time stepping
    def set_sources(self, xy):
        """Start points [m, 2], or [G, m, 2] for a batch of G geometries."""
        G = self.info().n_geometries
        xy = _f64(xy).reshape(-1, 2)
        if xy.shape[0] % G:
            raise ValueError(f"{xy.shape[0]} start points do not split over {G} geometries")
        self._ck(self._L.dg_set_sources(self.ctx, _dp(xy), xy.shape[0] // G), "dg_set_sources")

    def query_dt(self):
        dt, rho = ctypes.c_double(), ctypes.c_double()
        self._ck(self._L.dg_query_dt(self.ctx, ctypes.byref(dt), ctypes.byref(rho)), "dg_query_dt")
        return dt.value, rho.value

    def debug_copies(self, mode: int) -> int:
        """Set the stage kernel's copy mode (0 tensor copies, 1 cp.async, 2
        test hook: waits that run out); returns the tensor copies made since
        the last call."""
        n = ctypes.c_ulonglong(0)
        self._ck(self._L.dg_debug_copies(self.ctx, int(mode), ctypes.byref(n)), "dg_debug_copies")
        return n.value

    def set_growing_window(self, r_factor: float):
        """Advance only elements within r_factor sqrt(sigma0^2 + 2 D t) of the
        start-point box (0 turns it off)."""
        self._ck(self._L.dg_set_growing_window(self.ctx, float(r_factor)), "dg_set_growing_window")

    def set_launch(self, blocks_per_sm: int):
        """Stage-kernel launch shape: -1 tuned, 0 one block per chunk, k
        persistent blocks per SM."""
        self._ck(self._L.dg_set_launch(self.ctx, int(blocks_per_sm)), "dg_set_launch")

    def get_launch(self) -> int:
        k = ctypes.c_int()
        self._ck(self._L.dg_get_launch(self.ctx, ctypes.byref(k)), "dg_get_launch")
        return k.value

    def set_contraction(self, mode: int):
        """FP32 p = 5 element contractions: -1 tuned, 0 CUDA cores, 1 tensor
        cores."""
        self._ck(self._L.dg_set_contraction(self.ctx, int(mode)), "dg_set_contraction")

    def get_contraction(self) -> int:
        k = ctypes.c_int()
        self._ck(self._L.dg_get_contraction(self.ctx, ctypes.byref(k)), "dg_get_contraction")
        return k.value

    def set_triangle_fusion(self, fused: int):
        """Pixel triangles: 1 one launch per stage (FP32, p = 2, 3), 0 two."""
        self._ck(self._L.dg_set_triangle_fusion(self.ctx, int(fused)), "dg_set_triangle_fusion")

    def get_triangle_fusion(self) -> int:
        k = ctypes.c_int()
        self._ck(self._L.dg_get_triangle_fusion(self.ctx, ctypes.byref(k)), "dg_get_triangle_fusion")
        return k.value

    def step(self, nsteps: int, dt: float):
        self._ck(self._L.dg_step(self.ctx, int(nsteps), float(dt)), "dg_step")

    def propagate_to(self, delta: float):
        self._ck(self._L.dg_propagate_to(self.ctx, float(delta)), "dg_propagate_to")

    def moments(self) -> np.ndarray:
        inf = self.info()
        out = np.zeros((inf.n_geometries * inf.m, 6))
        self._ck(self._L.dg_moments(self.ctx, _dp(out)), "dg_moments")
        return out

    def covariance(self):
        s3, mu, mass = np.zeros(3), np.zeros(2), np.zeros(self.info().m)
        self._ck(self._L.dg_covariance(self.ctx, _dp(s3), _dp(mu), _dp(mass)), "dg_covariance")
        return s3, mu, mass

    def mixture_covariance(self, mom, mom0):
        """Sigma and mu of externally supplied raw moments [m, 6] (t and 0)."""
        mom, mom0 = _f64(mom).reshape(-1, 6), _f64(mom0).reshape(-1, 6)
        s3, mu = np.zeros(3), np.zeros(2)
        self._ck(self._L.dg_mixture_covariance(self.ctx, _dp(mom), _dp(mom0), mom.shape[0],
                                               _dp(s3), _dp(mu)), "dg_mixture_covariance")
        return s3, mu

    def apply_operator(self):
        self._ck(self._L.dg_apply_operator(self.ctx), "dg_apply_operator")

    def node_shape(self):
        """Nodes of one element: (p+1, p+1) for squares (j, i), (2, N) for the
        two triangles of a pixel."""
        inf = self.info()
        if self.cfg.element == DG_ELEMENT_TRIANGLE:
            return (2, inf.n_nodes // 2)
        return (inf.p + 1, inf.p + 1)

    def get_nodes(self) -> np.ndarray:
        inf = self.info()
        out = np.zeros((inf.m, inf.ny, inf.nx) + self.node_shape())
        self._ck(self._L.dg_get_nodes(self.ctx, _dp(out)), "dg_get_nodes")
        return out

    def set_nodes(self, u):
        inf = self.info()
        u = _f64(u).reshape((inf.m, inf.ny, inf.nx) + self.node_shape())
        self._ck(self._L.dg_set_nodes(self.ctx, _dp(u)), "dg_set_nodes")

    def get_elements(self, idx) -> np.ndarray:
        """Node values [k, n, n] of elements idx = [(source, ex, ey), ...]."""
        idx = np.ascontiguousarray(idx, dtype=np.int32).reshape(-1, 3)
        out = np.zeros((idx.shape[0],) + self.node_shape())
        self._ck(self._L.dg_get_elements(self.ctx, idx.ctypes.data, idx.shape[0], _dp(out)),
                 "dg_get_elements")
        return out

    # checkpoint
    def get_state(self) -> bytes:
        sz = ctypes.c_size_t()
        self._ck(self._L.dg_state_size(self.ctx, ctypes.byref(sz)), "dg_state_size")
        buf = ctypes.create_string_buffer(sz.value)
        self._ck(self._L.dg_get_state(self.ctx, buf, sz.value), "dg_get_state")
        return buf.raw

    def set_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._ck(self._L.dg_set_state(self.ctx, buf, len(blob)), "dg_set_state")

    # device memory and streams from torch
    def state_bytes(self, m: int) -> int:
        sz = ctypes.c_size_t()
        self._ck(self._L.dg_state_bytes(self.ctx, int(m), ctypes.byref(sz)), "dg_state_bytes")
        return sz.value

    def bind_state(self, tensor):
        """Use a CUDA tensor's memory (uint8, >= state_bytes(m)) for the state."""
        if tensor is None:
            self._ck(self._L.dg_bind_state(self.ctx, None, 0), "dg_bind_state")
            self._bound = None
            return
        nbytes = tensor.numel() * tensor.element_size()
        self._ck(self._L.dg_bind_state(self.ctx, ctypes.c_void_p(tensor.data_ptr()), nbytes),
                 "dg_bind_state")
        self._bound = tensor

    def set_stream(self, stream_ptr: int | None):
        self._ck(self._L.dg_set_stream(self.ctx, ctypes.c_void_p(stream_ptr) if stream_ptr else None),
                 "dg_set_stream")


def rasterize_disks(cx, cy, r, L: float, npix: int = 128) -> np.ndarray:
    """Occupancy raster [npix, npix] (1 inside a disk) of a periodic cell."""
    cx, cy, r = _f64(cx), _f64(cy), _f64(r)
    out = np.zeros((npix, npix), dtype=np.uint8)
    rc = lib().dg_rasterize_disks(_dp(cx), _dp(cy), _dp(r), int(r.size), float(L), int(npix),
                                  out.ctypes.data)
    if rc != DG_OK:
        raise DgError(rc, f"dg_rasterize_disks: {lib().dg_strerror(rc).decode()}")
    return out


def basis_tables(p: int, precision: int = DG_FP64):
    """(xi, w, D, D2) of order p as the kernels of that precision use them."""
    n = p + 1
    xi, w = np.zeros(n), np.zeros(n)
    D, D2 = np.zeros((n, n)), np.zeros((n, n))
    rc = lib().dg_basis_tables(int(p), int(precision), _dp(xi), _dp(w), _dp(D), _dp(D2))
    if rc != DG_OK:
        raise DgError(rc, f"dg_basis_tables: {lib().dg_strerror(rc).decode()}")
    return xi, w, D, D2


def triangle_tables(p: int):
    """(r, s, G, Lf, mono) of the triangle elements as the kernels use them."""
    n = (p + 1) * (p + 2) // 2
    r, s_, G = np.zeros(n), np.zeros(n), np.zeros((2, 2, n, n))
    Lf, mono = np.zeros((2, 3, n, p + 1)), np.zeros((6, n))
    rc = lib().dg_triangle_tables(int(p), _dp(r), _dp(s_), _dp(G), _dp(Lf), _dp(mono))
    if rc != DG_OK:
        raise DgError(rc, f"dg_triangle_tables: {lib().dg_strerror(rc).decode()}")
    return r, s_, G, Lf, mono


class Surrogate:
    """The learned covariance surrogate (include/dgsurrogate.h).  Batches are
    CUDA tensors: occ uint8 [B, 128, 128], cond float32 [B, 2], target
    float32 [B, 3]."""

    def __init__(self, max_batch: int = 4096, seed: int = 1, device: int = 0):
        self._L = lib()
        h = _P()
        rc = self._L.sg_create(int(max_batch), int(seed), int(device), ctypes.byref(h))
        if rc != DG_OK:
            raise DgError(rc, "sg_create")
        self.net = h
        self.max_batch = max_batch

    def _ck(self, rc, what):
        if rc != DG_OK:
            raise DgError(rc, f"{what}: {self._L.sg_last_error(self.net).decode()}")

    def close(self):
        if getattr(self, "net", None):
            self._L.sg_destroy(self.net)
            self.net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def param_count(self) -> int:
        n = ctypes.c_size_t()
        self._ck(self._L.sg_param_count(self.net, ctypes.byref(n)), "sg_param_count")
        return n.value

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.param_count(), dtype=np.float32)
        self._ck(self._L.sg_get_params(self.net, out.ctypes.data), "sg_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._ck(self._L.sg_set_params(self.net, p.ctypes.data), "sg_set_params")

    @staticmethod
    def _ptr(t):
        return ctypes.c_void_p(t.data_ptr())

    def predict(self, occ, cond, out):
        B = occ.shape[0]
        self._ck(self._L.sg_predict(self.net, self._ptr(occ), self._ptr(cond), B, self._ptr(out)),
                 "sg_predict")

    def gradients(self, occ, cond, target):
        loss = np.zeros(1, dtype=np.float32)
        g = np.zeros(self.param_count(), dtype=np.float32)
        self._ck(self._L.sg_gradients(self.net, self._ptr(occ), self._ptr(cond), self._ptr(target),
                                      occ.shape[0], loss.ctypes.data, g.ctypes.data), "sg_gradients")
        return float(loss[0]), g

    def train_step(self, occ, cond, target, lr: float) -> float:
        loss = np.zeros(1, dtype=np.float32)
        self._ck(self._L.sg_train_step(self.net, self._ptr(occ), self._ptr(cond), self._ptr(target),
                                       occ.shape[0], float(lr), loss.ctypes.data), "sg_train_step")
        return float(loss[0])
