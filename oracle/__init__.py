"""ctypes access to the FP64 CPU oracle (``tsdf_oracle.cpp``).

Test infrastructure only: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it. Nothing on the product path may import it.
It does not import the CUDA package either; the only thing the two sides share is
the seeded input generator, which holds none of the method's arithmetic.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional, Sequence as Seq

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsdf_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libtsdf_oracle.so")
CFLAGS = ["-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
          "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle (g++, IEEE double, no FP contraction) into _build/."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", *CFLAGS, _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile a modified copy of the oracle source (used by tests that plant a
    mistake in the oracle and check that a pin catches it)."""
    src = out_path + ".cpp"
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.check_call(["g++", *CFLAGS, src, "-o", out_path])
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


class _Params(ctypes.Structure):
    _fields_ = [("voxel_size", ctypes.c_float), ("truncation", ctypes.c_float),
                ("origin", ctypes.c_double * 3), ("grid_dim", ctypes.c_int32),
                ("block_capacity", ctypes.c_int64), ("process_variance", ctypes.c_float),
                ("depth_min", ctypes.c_float), ("depth_max", ctypes.c_float),
                ("raycast_near", ctypes.c_float), ("raycast_far", ctypes.c_float),
                ("sigma_coeff", ctypes.c_float), ("alloc_half_samples", ctypes.c_int32),
                ("amb_px", ctypes.c_double), ("amb_trunc", ctypes.c_double),
                ("store_values", ctypes.c_int32), ("update_rule", ctypes.c_int32),
                ("update_weight", ctypes.c_float), ("weight_max", ctypes.c_float),
                ("refine_steps", ctypes.c_int32)]


class _Intr(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float), ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def _load(path: Optional[str] = None) -> ctypes.CDLL:
    lib = ctypes.CDLL(path or build())
    sig = {
        "ov_create": (_P, [ctypes.POINTER(_Params)]),
        "ov_destroy": (None, [_P]),
        "ov_num_blocks": (ctypes.c_int64, [_P]),
        "ov_alloc_half_samples": (ctypes.c_int32, [ctypes.POINTER(_Params)]),
        "ov_frame_blocks": (ctypes.c_int64, [ctypes.POINTER(_Params), _F, ctypes.POINTER(_Intr), _D, _U32, ctypes.c_int64]),
        "ov_allocate": (None, [_P, _F, ctypes.POINTER(_Intr), _D, ctypes.c_int32, _I64, _I32]),
        "ov_integrate": (None, [_P, _F, _F, ctypes.POINTER(_Intr), _D]),
        "ov_export": (None, [_P, _I32, _D, _D, _U8]),
        "ov_raycast": (None, [_P, ctypes.POINTER(_Intr), _D, ctypes.c_int64, _I32, _D, _D, _D, _I32]),
        "ov_replay_voxels": (None, [ctypes.POINTER(_Params), ctypes.c_int32, ctypes.POINTER(_F), ctypes.POINTER(_F),
                                    ctypes.POINTER(_Intr), _D, ctypes.c_int64, _I32, _I32, _D, _D, _U8]),
        "ov_dense_create": (_P, [ctypes.POINTER(_Params)]),
        "ov_dense_integrate": (None, [_P, _F, _F, ctypes.POINTER(_Intr), _D]),
        "ov_dense_read": (None, [_P, ctypes.c_int64, _I32, _D, _D, _U8]),
        "ov_dense_coverage": (None, [_P, _P, _I64, _I64]),
        "ov_num_threads": (ctypes.c_int32, []),
        "ov_field": (None, [_P, ctypes.c_int64, _D, _D]),
        "ov_mlp_param_count": (ctypes.c_int32, []),
        "ov_mlp_features": (None, [_F, ctypes.POINTER(_Intr), ctypes.POINTER(_Params), ctypes.c_int64, _I32, _D, _U8]),
        "ov_mlp_forward": (None, [_D, ctypes.c_int64, _D, _D]),
        "ov_mlp_loss_grad": (None, [_D, ctypes.c_int64, _D, _D, _D, _D]),
        "ov_mlp_variance_map": (None, [_D, _F, ctypes.POINTER(_Intr), ctypes.POINTER(_Params), _F]),
        "ov_count_outside": (ctypes.c_int64, [_P, _I32, _I32]),
        "ov_evict": (ctypes.c_int64, [_P, _I32, _I32, _I32, _D, _D]),
        "ov_shift": (ctypes.c_int64, [_P, _I32, _I32, _D, _D]),
        "ov_import": (ctypes.c_int32, [_P, ctypes.c_int64, _I32, _D, _D, ctypes.c_int32]),
        "ov_origin": (None, [_P, _D]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib_cache: dict = {}


def lib(path: Optional[str] = None) -> ctypes.CDLL:
    key = path or "default"
    if key not in _lib_cache:
        _lib_cache[key] = _load(path)
    return _lib_cache[key]


def _ptr(a: Optional[np.ndarray], t):
    return None if a is None else a.ctypes.data_as(t)


def make_params(vol, amb_px: float = 1e-3, amb_trunc: float = 1e-5, store_values: bool = True,
                alloc_half_samples: int = 0, process_variance: Optional[float] = None) -> _Params:
    """Oracle settings from a ``synth.VolumeParams``-like object."""
    p = _Params()
    p.voxel_size = vol.voxel_size
    p.truncation = vol.truncation
    p.origin = (ctypes.c_double * 3)(*[float(o) for o in vol.origin])
    p.grid_dim = int(vol.grid_dim)
    p.block_capacity = int(vol.block_capacity)
    p.process_variance = vol.process_variance if process_variance is None else process_variance
    p.depth_min, p.depth_max = vol.depth_min, vol.depth_max
    p.raycast_near, p.raycast_far = vol.raycast_near, vol.raycast_far
    p.sigma_coeff = vol.sigma_coeff
    p.alloc_half_samples = int(alloc_half_samples)
    p.amb_px, p.amb_trunc = float(amb_px), float(amb_trunc)
    p.store_values = int(bool(store_values))
    p.update_rule = int(getattr(vol, "update_rule", 0))
    p.update_weight = float(getattr(vol, "update_weight", 0.1))
    p.weight_max = float(getattr(vol, "weight_max", 1.0))
    p.refine_steps = int(getattr(vol, "refine_steps", 0))
    return p


def make_intr(intr) -> _Intr:
    return _Intr(intr.fx, intr.fy, intr.cx, intr.cy, int(intr.width), int(intr.height))


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Export:
    coords: np.ndarray       # (n, 3) int32 block coordinates, ascending key order
    alloc_frame: np.ndarray  # (n,) int32
    T: np.ndarray            # (n, 512) float64, NaN = chi
    P: np.ndarray            # (n, 512) float64
    amb: np.ndarray          # (n, 512) bool


class OracleVolume:
    """Sparse FP64 TSDF volume: allocation, Alg. 3 integration, raycast."""

    def __init__(self, vol, intr, lib_path: Optional[str] = None, **kw):
        self.lib = lib(lib_path)
        self.vol = vol
        self.params = make_params(vol, **kw)
        self.intr = make_intr(intr)
        self.h = self.lib.ov_create(ctypes.byref(self.params))
        if not self.h:
            raise ValueError("oracle: invalid volume parameters")
        self.frame = 0

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.ov_destroy(self.h)
            self.h = None

    @property
    def half_samples(self) -> int:
        return int(self.lib.ov_alloc_half_samples(ctypes.byref(self.params)))

    def frame_blocks(self, depth, pose) -> np.ndarray:
        d, T = _f32(depth), _f64(pose)
        n = self.lib.ov_frame_blocks(ctypes.byref(self.params), _ptr(d, _F), ctypes.byref(self.intr),
                                     _ptr(T, _D), None, 0)
        out = np.empty(n, np.uint32)
        self.lib.ov_frame_blocks(ctypes.byref(self.params), _ptr(d, _F), ctypes.byref(self.intr),
                                 _ptr(T, _D), _ptr(out, _U32), n)
        return out

    def allocate(self, depth, pose, frame: Optional[int] = None):
        d, T = _f32(depth), _f64(pose)
        n_new, over = ctypes.c_int64(0), ctypes.c_int32(0)
        fr = self.frame if frame is None else frame
        self.lib.ov_allocate(self.h, _ptr(d, _F), ctypes.byref(self.intr), _ptr(T, _D), fr,
                             ctypes.byref(n_new), ctypes.byref(over))
        return int(n_new.value), bool(over.value)

    def integrate(self, depth, pose, var=None):
        d, T = _f32(depth), _f64(pose)
        v = None if var is None else _f32(var)
        self.lib.ov_integrate(self.h, _ptr(d, _F), _ptr(v, _F), ctypes.byref(self.intr), _ptr(T, _D))

    def fuse(self, depth, pose, var=None):
        """Allocate then integrate one frame (the per-frame fusion step)."""
        n_new, over = self.allocate(depth, pose)
        self.integrate(depth, pose, var)
        self.frame += 1
        return n_new, over

    @property
    def n_blocks(self) -> int:
        return int(self.lib.ov_num_blocks(self.h))

    def export(self, values: bool = True) -> Export:
        n = self.n_blocks
        cf = np.empty((n, 4), np.int32)
        if values and self.params.store_values:
            T = np.empty((n, 512)); P = np.empty((n, 512)); amb = np.empty((n, 512), np.uint8)
            self.lib.ov_export(self.h, _ptr(cf, _I32), _ptr(T, _D), _ptr(P, _D), _ptr(amb, _U8))
        else:
            T = P = amb = np.empty((n, 0))
            self.lib.ov_export(self.h, _ptr(cf, _I32), None, None, None)
        return Export(cf[:, :3].copy(), cf[:, 3].copy(), T, P, amb.astype(bool))

    def raycast(self, pose, uv: Optional[np.ndarray] = None, intr=None):
        """Raycast listed pixels (n, 2) int (u, v), or the full image."""
        it = self.intr if intr is None else make_intr(intr)
        if uv is None:
            vv, uu = np.meshgrid(np.arange(it.height), np.arange(it.width), indexing="ij")
            uv = np.stack([uu.ravel(), vv.ravel()], -1)
        uv = np.ascontiguousarray(uv, np.int32)
        n = uv.shape[0]
        depth = np.empty(n); vert = np.empty((n, 3)); nrm = np.empty((n, 3)); flags = np.empty(n, np.int32)
        T = _f64(pose)
        self.lib.ov_raycast(self.h, ctypes.byref(it), _ptr(T, _D), n, _ptr(uv, _I32), _ptr(depth, _D),
                            _ptr(vert, _D), _ptr(nrm, _D), _ptr(flags, _I32))
        return depth, vert, nrm, flags


    # Eviction and volume shift (section "Discussion"): see ov_evict / ov_shift.
    def _take(self, n, call) -> Export:
        cf = np.empty((n, 4), np.int32)
        T = np.empty((n, 512)); P = np.empty((n, 512))
        m = call(_ptr(cf, _I32), _ptr(T, _D), _ptr(P, _D))
        assert m == n
        return Export(cf[:, :3].copy(), cf[:, 3].copy(), T, P, np.zeros((n, 512), bool))

    def evict(self, lo, hi) -> Export:
        """Remove and return (ascending key order) every block outside the box [lo, hi)."""
        a = np.ascontiguousarray(lo, np.int32); b = np.ascontiguousarray(hi, np.int32)
        n = int(self.lib.ov_count_outside(self.h, _ptr(a, _I32), _ptr(b, _I32)))
        return self._take(n, lambda cf, T, P: self.lib.ov_evict(self.h, _ptr(a, _I32), _ptr(b, _I32), cf, T, P))

    def shift(self, d) -> Export:
        """Move the grid by d blocks; return the blocks that left it."""
        dd = np.ascontiguousarray(d, np.int32)
        nb = int(self.params.grid_dim) // 8
        lo = dd.copy(); hi = dd + nb
        n = int(self.lib.ov_count_outside(self.h, _ptr(lo, _I32), _ptr(hi, _I32)))
        out = self._take(n, lambda cf, T, P: self.lib.ov_shift(self.h, _ptr(dd, _I32), cf, T, P))
        o = np.empty(3)
        self.lib.ov_origin(self.h, _ptr(o, _D))
        self.params.origin = (ctypes.c_double * 3)(*o)
        return out

    @property
    def origin(self) -> np.ndarray:
        o = np.empty(3)
        self.lib.ov_origin(self.h, _ptr(o, _D))
        return o

    def import_blocks(self, coords, T, P, frame: Optional[int] = None):
        """Add blocks (coords (n, 3), T and P (n, 512), NaN T = chi) at the
        current frame; raises ValueError when the oracle refuses them."""
        coords = np.asarray(coords, np.int32)
        n = coords.shape[0]
        cf = np.zeros((n, 4), np.int32)
        cf[:, :3] = coords[:, :3]
        T = np.ascontiguousarray(T, np.float64).reshape(n, 512)
        P = np.ascontiguousarray(P, np.float64).reshape(n, 512)
        fr = self.frame if frame is None else frame
        if self.lib.ov_import(self.h, n, _ptr(cf, _I32), _ptr(T, _D), _ptr(P, _D), fr) != 0:
            raise ValueError("oracle: import refused")

    def field(self, points: np.ndarray) -> np.ndarray:
        """Trilinear field at world points (n, 3); NaN where undefined."""
        pts = np.ascontiguousarray(points, np.float64).reshape(-1, 3)
        out = np.empty(pts.shape[0])
        self.lib.ov_field(self.h, pts.shape[0], _ptr(pts, _D), _ptr(out, _D))
        return out


def replay_voxels(vol, intr, depths: Seq[np.ndarray], poses: np.ndarray, voxels: np.ndarray,
                  alloc_frame: np.ndarray, vars_: Optional[Seq[np.ndarray]] = None,
                  lib_path: Optional[str] = None, **kw):
    """Per-voxel Alg. 3 replay over a sequence (sampled full-size parity): each
    listed voxel takes every frame from its block's allocation frame on."""
    L = lib(lib_path)
    p = make_params(vol, **kw)
    it = make_intr(intr)
    ds = [_f32(d) for d in depths]
    darr = (_F * len(ds))(*[_ptr(d, _F) for d in ds])
    varr = None
    if vars_ is not None:
        vs = [_f32(v) for v in vars_]
        varr = (_F * len(vs))(*[_ptr(v, _F) for v in vs])
    P_ = _f64(poses).reshape(-1, 16)
    vox = np.ascontiguousarray(voxels, np.int32)
    af = np.ascontiguousarray(alloc_frame, np.int32)
    n = vox.shape[0]
    T = np.empty(n); P = np.empty(n); amb = np.empty(n, np.uint8)
    L.ov_replay_voxels(ctypes.byref(p), len(ds), darr, varr, ctypes.byref(it), _ptr(P_, _D), n,
                       _ptr(vox, _I32), _ptr(af, _I32), _ptr(T, _D), _ptr(P, _D), _ptr(amb, _U8))
    return T, P, amb.astype(bool)


class DenseOracle:
    """Dense brute force: Alg. 3 on every voxel of a G^3 grid (no allocation)."""

    def __init__(self, vol, intr, **kw):
        self.lib = lib()
        self.params = make_params(vol, **kw)
        self.intr = make_intr(intr)
        self.h = self.lib.ov_dense_create(ctypes.byref(self.params))

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.ov_destroy(self.h)
            self.h = None

    def integrate(self, depth, pose, var=None):
        d, T = _f32(depth), _f64(pose)
        v = None if var is None else _f32(var)
        self.lib.ov_dense_integrate(self.h, _ptr(d, _F), _ptr(v, _F), ctypes.byref(self.intr), _ptr(T, _D))

    def read(self, voxels: np.ndarray):
        vox = np.ascontiguousarray(voxels, np.int32)
        n = vox.shape[0]
        T = np.empty(n); P = np.empty(n); amb = np.empty(n, np.uint8)
        self.lib.ov_dense_read(self.h, n, _ptr(vox, _I32), _ptr(T, _D), _ptr(P, _D), _ptr(amb, _U8))
        return T, P, amb.astype(bool)

    def coverage(self, sparse: OracleVolume):
        nv, nm = ctypes.c_int64(0), ctypes.c_int64(0)
        self.lib.ov_dense_coverage(self.h, sparse.h, ctypes.byref(nv), ctypes.byref(nm))
        return int(nv.value), int(nm.value)


class Mlp:
    """FP64 learned-variance network (27-32-32-1, ReLU) of the oracle."""

    def __init__(self, weights: np.ndarray, lib_path: Optional[str] = None):
        self.lib = lib(lib_path)
        self.n_params = int(self.lib.ov_mlp_param_count())
        self.w = np.ascontiguousarray(weights, np.float64).ravel()
        assert self.w.size == self.n_params

    def features(self, depth, intr, vol, uv):
        uv = np.ascontiguousarray(uv, np.int32).reshape(-1, 2)
        n = uv.shape[0]
        f = np.empty((n, 27)); valid = np.empty(n, np.uint8)
        p = make_params(vol)
        self.lib.ov_mlp_features(_ptr(_f32(depth), _F), ctypes.byref(make_intr(intr)), ctypes.byref(p), n,
                                 _ptr(uv, _I32), _ptr(f, _D), _ptr(valid, _U8))
        return f, valid.astype(bool)

    def forward(self, feats):
        x = _f64(feats).reshape(-1, 27)
        out = np.empty(x.shape[0])
        self.lib.ov_mlp_forward(_ptr(self.w, _D), x.shape[0], _ptr(x, _D), _ptr(out, _D))
        return out

    def loss_grad(self, feats, s):
        x = _f64(feats).reshape(-1, 27)
        s = _f64(s)
        g = np.empty(self.n_params); loss = np.empty(1)
        self.lib.ov_mlp_loss_grad(_ptr(self.w, _D), x.shape[0], _ptr(x, _D), _ptr(s, _D), _ptr(g, _D), _ptr(loss, _D))
        return float(loss[0]), g

    def variance_map(self, depth, intr, vol):
        d = _f32(depth)
        out = np.empty(d.shape, np.float32)
        p = make_params(vol)
        self.lib.ov_mlp_variance_map(_ptr(self.w, _D), _ptr(d, _F), ctypes.byref(make_intr(intr)), ctypes.byref(p),
                                     _ptr(out, _F))
        return out


def num_threads() -> int:
    return int(lib().ov_num_threads())


def voxel_coords(export: Export) -> np.ndarray:
    """(n*512, 3) voxel indices matching the flattened T/P of an export."""
    l = np.arange(512)
    local = np.stack([l & 7, (l >> 3) & 7, l >> 6], -1)
    return (export.coords[:, None, :].astype(np.int64) * 8 + local[None]).reshape(-1, 3)
