"""Thin ctypes binding of libtsdf.so (include/tsdf.h) for torch CUDA tensors.

Argument marshalling only: every step of allocation, integration and raycasting
runs in the library's CUDA kernels. There is no CPU fallback: if the library is
missing or no CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtsdf.so")
# the same library built with TSDF_DEBUG: device-side index checks that report
# TSDF_ERR_BOUNDS (python -m paper_1311_7194_b300.build --debug)
DEBUG_LIB_PATH = os.path.join(_HERE, "libtsdf_debug.so")

OK, ERR_INVALID_ARG, ERR_CAPACITY, ERR_HASH_FULL, ERR_CUDA, ERR_NOT_READY, ERR_OUT_OF_MEMORY, ERR_BOUNDS = range(8)
STORAGE_F32, STORAGE_F16, STORAGE_SNORM16 = 0, 1, 2
UPDATE_KALMAN, UPDATE_AVERAGE, UPDATE_WEIGHTED = 0, 1, 2      # tsdf_update_rule

# Every function the header declares (checked against include/tsdf.h by the tests).
EXPORTED = ["tsdf_config_default", "tsdf_status_string", "tsdf_debug_build", "tsdf_debug_check_slot", "tsdf_create", "tsdf_create_ex", "tsdf_destroy",
            "tsdf_reset", "tsdf_allocate", "tsdf_integrate", "tsdf_integrate_batch", "tsdf_raycast",
            "tsdf_raycast_noalloc", "tsdf_raycast_trace", "tsdf_icp_params_default", "tsdf_icp", "tsdf_icp_sums",
            "tsdf_icp_solve", "tsdf_mesh", "tsdf_mesh_case", "tsdf_graph_create", "tsdf_graph_launch", "tsdf_graph_launch_host", "tsdf_graph_instantiations",
            "tsdf_graph_set_events", "tsdf_graph_destroy", "tsdf_get_launch_config", "tsdf_set_launch_config",
            "tsdf_autotune", "tsdf_mlp_param_count", "tsdf_set_variance_mlp", "tsdf_mlp_variance",
            "tsdf_mlp_features", "tsdf_mlp_harvest", "tsdf_mlp_forward", "tsdf_mlp_loss_grad", "tsdf_mlp_adam",
            "tsdf_quadratic_variance",
            "tsdf_get_status", "tsdf_get_stats", "tsdf_export", "tsdf_get_config", "tsdf_evict", "tsdf_shift",
            "tsdf_import"]


class TsdfError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_string(status)} (status {status})")


class Config(ctypes.Structure):
    _fields_ = [("voxel_size", ctypes.c_float), ("truncation", ctypes.c_float),
                ("origin", ctypes.c_double * 3), ("grid_dim", ctypes.c_int32),
                ("block_capacity", ctypes.c_int64), ("process_variance", ctypes.c_float),
                ("depth_min", ctypes.c_float), ("depth_max", ctypes.c_float),
                ("raycast_near", ctypes.c_float), ("raycast_far", ctypes.c_float),
                ("sigma_coeff", ctypes.c_float), ("storage", ctypes.c_int32),
                ("alloc_half_samples", ctypes.c_int32), ("update_rule", ctypes.c_int32),
                ("update_weight", ctypes.c_float), ("weight_max", ctypes.c_float),
                ("refine_steps", ctypes.c_int32)]


class Intrinsics(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_float), ("fy", ctypes.c_float), ("cx", ctypes.c_float),
                ("cy", ctypes.c_float), ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class LaunchConfig(ctypes.Structure):
    _fields_ = [("integrate_voxels_per_thread", ctypes.c_int32), ("integrate_ctas_per_sm", ctypes.c_int32),
                ("raycast_tile_w", ctypes.c_int32), ("raycast_tile_h", ctypes.c_int32),
                ("raycast_persistent", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class Stats(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_int64), ("new_blocks", ctypes.c_int64),
                ("visible_blocks", ctypes.c_int64), ("voxel_updates", ctypes.c_int64),
                ("raycast_blocks", ctypes.c_int64), ("rays_hit", ctypes.c_int64),
                ("frames", ctypes.c_int64), ("voxel_updates_total", ctypes.c_int64),
                ("visible_blocks_total", ctypes.c_int64), ("rays_hit_total", ctypes.c_int64),
                ("raycast_blocks_total", ctypes.c_int64), ("voxels_touched_total", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class IcpParams(ctypes.Structure):
    _fields_ = [("dist_max", ctypes.c_float), ("normal_cos_min", ctypes.c_float), ("eig_threshold", ctypes.c_float),
                ("iterations", ctypes.c_int32)]


class IcpResult(ctypes.Structure):
    _fields_ = [("matches", ctypes.c_int64), ("rms", ctypes.c_double), ("rank", ctypes.c_int32),
                ("iterations", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {"matches": int(self.matches), "rms": float(self.rms), "rank": int(self.rank),
                "iterations": int(self.iterations)}


class RaycastCounts(ctypes.Structure):
    _fields_ = [("samples", ctypes.c_int64), ("table_lookups", ctypes.c_int64), ("t_sectors", ctypes.c_int64),
                ("table_sectors", ctypes.c_int64), ("rays", ctypes.c_int64), ("rays_hit", ctypes.c_int64),
                ("march_samples", ctypes.c_int64), ("skips", ctypes.c_int64), ("rescans", ctypes.c_int64),
                ("rescan_samples", ctypes.c_int64), ("refine_samples", ctypes.c_int64),
                ("normal_samples", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_lib: Optional[ctypes.CDLL] = None
_P = ctypes.c_void_p
_PD = ctypes.POINTER(ctypes.c_double)


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Load libtsdf.so (built by ``python -m paper_1311_7194_b300.build``)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libtsdf.so not found at {p}: build it with "
                          "`python -m paper_1311_7194_b300.build` (needs nvcc)")
    lib = ctypes.CDLL(p)
    sig = {
        "tsdf_config_default": (None, [ctypes.POINTER(Config)]),
        "tsdf_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "tsdf_create": (ctypes.c_int, [ctypes.c_float, ctypes.c_float, ctypes.c_int64, ctypes.POINTER(_P)]),
        "tsdf_create_ex": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(_P)]),
        "tsdf_destroy": (None, [_P]),
        "tsdf_reset": (ctypes.c_int, [_P, _P]),
        "tsdf_allocate": (ctypes.c_int, [_P, _P, ctypes.POINTER(Intrinsics), _PD, _P]),
        "tsdf_integrate": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(Intrinsics), _PD, _P]),
        "tsdf_integrate_batch": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(_P), ctypes.POINTER(_P),
                                                ctypes.POINTER(Intrinsics), _PD, _P]),
        "tsdf_raycast": (ctypes.c_int, [_P, ctypes.POINTER(Intrinsics), _PD, _P, _P, _P, _P]),
        "tsdf_raycast_noalloc": (ctypes.c_int, [_P, ctypes.POINTER(Intrinsics), _PD, _P, _P, _P, _P]),
        "tsdf_raycast_trace": (ctypes.c_int, [_P, ctypes.POINTER(Intrinsics), _PD, ctypes.POINTER(RaycastCounts),
                                              _P]),
        "tsdf_mesh": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64), _P]),
        "tsdf_mesh_case": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                          ctypes.POINTER(ctypes.c_int8)]),
        "tsdf_icp_params_default": (None, [ctypes.POINTER(IcpParams)]),
        "tsdf_icp": (ctypes.c_int, [_P, _P, ctypes.POINTER(Intrinsics), _P, _P, _PD, ctypes.POINTER(IcpParams), _PD,
                                    ctypes.POINTER(IcpResult), _P]),
        "tsdf_icp_sums": (ctypes.c_int, [_P, _P, ctypes.POINTER(Intrinsics), _P, _P, _PD, ctypes.POINTER(IcpParams),
                                         _PD, _PD, ctypes.POINTER(ctypes.c_float), _P]),
        "tsdf_icp_solve": (ctypes.c_int, [_PD, ctypes.POINTER(ctypes.c_float), ctypes.c_float, _PD, _PD,
                                          ctypes.POINTER(ctypes.c_int32)]),
        "tsdf_graph_create": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(Intrinsics), ctypes.POINTER(_P)]),
        "tsdf_graph_launch": (ctypes.c_int, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _PD, _P, _P, _P, _P]),
        "tsdf_graph_launch_host": (ctypes.c_int, [_P, ctypes.POINTER(_P), _PD, _P, _P, _P, _P]),
        "tsdf_graph_instantiations": (ctypes.c_int64, [_P]),
        "tsdf_graph_set_events": (ctypes.c_int, [_P, ctypes.POINTER(_P)]),
        "tsdf_get_launch_config": (ctypes.c_int, [_P, ctypes.POINTER(LaunchConfig)]),
        "tsdf_mlp_param_count": (ctypes.c_int32, []),
        "tsdf_set_variance_mlp": (ctypes.c_int, [_P, _P, ctypes.c_int64]),
        "tsdf_mlp_variance": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(Intrinsics), _P, _P]),
        "tsdf_mlp_features": (ctypes.c_int, [_P, _P, ctypes.POINTER(Intrinsics), ctypes.c_int64, _P, _P, _P, _P]),
        "tsdf_mlp_harvest": (ctypes.c_int, [_P, _P, _P, ctypes.POINTER(Intrinsics), ctypes.c_int64, _P, _P, _P, _P]),
        "tsdf_mlp_forward": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P]),
        "tsdf_mlp_loss_grad": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P, _P, _P, _P]),
        "tsdf_mlp_adam": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                         ctypes.c_float, ctypes.c_float, ctypes.c_int32, _P]),
        "tsdf_set_launch_config": (ctypes.c_int, [_P, ctypes.POINTER(LaunchConfig)]),
        "tsdf_autotune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(_P), ctypes.POINTER(Intrinsics), _PD,
                                         ctypes.c_char_p, ctypes.POINTER(LaunchConfig), ctypes.POINTER(ctypes.c_int32)]),
        "tsdf_graph_destroy": (None, [_P]),
        "tsdf_quadratic_variance": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_float, _P, _P]),
        "tsdf_get_status": (ctypes.c_int, [_P]),
        "tsdf_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(Stats)]),
        "tsdf_export": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
        "tsdf_get_config": (ctypes.c_int, [_P, ctypes.POINTER(Config)]),
        "tsdf_evict": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.c_int64, _P, _P, _P, ctypes.POINTER(ctypes.c_int64), _P]),
        "tsdf_shift": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int32), ctypes.c_int64, _P, _P, _P,
                                      ctypes.POINTER(ctypes.c_int64), _P]),
        "tsdf_import": (ctypes.c_int, [_P, ctypes.c_int64, _P, _P, _P, _P]),
        "tsdf_debug_build": (ctypes.c_int, []),
        "tsdf_debug_check_slot": (ctypes.c_int, [_P, ctypes.c_int64, _P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def status_string(status: int) -> str:
    try:
        return load().tsdf_status_string(int(status)).decode()
    except ImportError:
        return f"status {status}"


def _check(status: int, what: str):
    if status != OK:
        raise TsdfError(status, what)


def default_config() -> Config:
    c = Config()
    load().tsdf_config_default(ctypes.byref(c))
    return c


def config_from(vol, **overrides) -> Config:
    """Config from a ``synth.VolumeParams``-like object (fields of the same names)."""
    c = default_config()
    c.voxel_size = vol.voxel_size
    c.truncation = vol.truncation
    c.origin = (ctypes.c_double * 3)(*[float(o) for o in vol.origin])
    c.grid_dim = int(vol.grid_dim)
    c.block_capacity = int(vol.block_capacity)
    c.process_variance = getattr(vol, "process_variance", 0.0)
    c.depth_min, c.depth_max = vol.depth_min, vol.depth_max
    c.raycast_near, c.raycast_far = vol.raycast_near, vol.raycast_far
    c.sigma_coeff = vol.sigma_coeff
    c.update_rule = int(getattr(vol, "update_rule", UPDATE_KALMAN))
    c.update_weight = float(getattr(vol, "update_weight", c.update_weight))
    c.weight_max = float(getattr(vol, "weight_max", c.weight_max))
    c.refine_steps = int(getattr(vol, "refine_steps", 0))
    for k, v in overrides.items():
        setattr(c, k, v)
    return c


def mesh_case(pattern: int):
    """tsdf_mesh_case (host only): the triangles (edge-number triples) of a
    corner pattern."""
    n = ctypes.c_int32()
    e = (ctypes.c_int8 * 24)()
    _check(load().tsdf_mesh_case(int(pattern), ctypes.byref(n), e), "tsdf_mesh_case")
    return [tuple(e[3 * k:3 * k + 3]) for k in range(n.value)]


def icp_params(**kw) -> IcpParams:
    """tsdf_icp_params with the library defaults, fields overridden by ``kw``."""
    p = IcpParams()
    load().tsdf_icp_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def icp_solve(sums, box, theta: float = 0.005):
    """tsdf_icp_solve (host only): (r, t, rank) from Eq. 4 sums and the box."""
    s = (ctypes.c_double * 29)(*[float(x) for x in np.asarray(sums, np.float64).ravel()])
    b = (ctypes.c_float * 6)(*[float(x) for x in np.asarray(box, np.float32).ravel()])
    r = (ctypes.c_double * 3)()
    t = (ctypes.c_double * 3)()
    k = ctypes.c_int32()
    _check(load().tsdf_icp_solve(s, b, float(theta), r, t, ctypes.byref(k)), "tsdf_icp_solve")
    return np.array(r[:]), np.array(t[:]), int(k.value)


def intrinsics(intr) -> Intrinsics:
    return Intrinsics(intr.fx, intr.fy, intr.cx, intr.cy, int(intr.width), int(intr.height))


def _pose(pose) -> ctypes.Array:
    a = np.ascontiguousarray(np.asarray(pose, dtype=np.float64).reshape(16))
    return (ctypes.c_double * 16)(*a.tolist())


def _dev_ptr(t, n: int, what: str) -> int:
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA torch tensor")
    if t.dtype != torch.float32 or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{what} must be a contiguous float32 tensor of {n} elements")
    return t.data_ptr()


def _host_ptr(a, n: int, what: str) -> int:
    import torch
    if isinstance(a, torch.Tensor):
        if a.is_cuda or a.dtype != torch.float32 or not a.is_contiguous() or a.numel() != n:
            raise ValueError(f"{what} must be a contiguous float32 CPU tensor of {n} elements")
        return a.data_ptr()
    if not isinstance(a, np.ndarray) or a.dtype != np.float32 or not a.flags.c_contiguous or a.size != n:
        raise ValueError(f"{what} must be a contiguous float32 array of {n} elements")
    return a.ctypes.data


def _stream(stream) -> int:
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return s.cuda_stream


@dataclass
class Export:
    coords: np.ndarray       # (n, 3) int32 block coordinates, pool order
    alloc_frame: np.ndarray  # (n,) int32
    T: np.ndarray            # (n, 512) float32, NaN = chi
    P: np.ndarray            # (n, 512) float32

    def sorted(self, nb: int) -> "Export":
        key = self.coords[:, 0].astype(np.int64) + nb * (self.coords[:, 1] + nb * self.coords[:, 2].astype(np.int64))
        o = np.argsort(key, kind="stable")
        return Export(self.coords[o], self.alloc_frame[o], self.T[o], self.P[o])


@dataclass
class Evicted:
    """Blocks removed by Volume.evict / Volume.shift, in pool order: block
    coordinates (n, 3) before the call, allocation frames (n,), T (n, 512)
    float32 (NaN = chi) and P (n, 512)."""
    coords: np.ndarray
    frames: np.ndarray
    T: np.ndarray
    P: np.ndarray


class Volume:
    """A sparse TSDF volume on the current CUDA device (tsdf_create_ex)."""

    def __init__(self, config: Config, lib: Optional[ctypes.CDLL] = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libtsdf needs a CUDA device")
        self.lib = lib or load()
        self.config = config
        h = _P()
        _check(self.lib.tsdf_create_ex(ctypes.byref(config), ctypes.byref(h)), "tsdf_create_ex")
        self.h = h

    @classmethod
    def from_params(cls, vol, lib: Optional[ctypes.CDLL] = None, **overrides) -> "Volume":
        return cls(config_from(vol, **overrides), lib)

    def close(self):
        if getattr(self, "h", None):
            self.lib.tsdf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def nb(self) -> int:
        return int(self.config.grid_dim) // 8

    def reset(self, stream=None):
        _check(self.lib.tsdf_reset(self.h, _stream(stream)), "tsdf_reset")

    def allocate(self, depth, intr, pose, stream=None):
        K = intrinsics(intr)
        _check(self.lib.tsdf_allocate(self.h, _dev_ptr(depth, K.width * K.height, "depth"), ctypes.byref(K),
                                      _pose(pose), _stream(stream)), "tsdf_allocate")

    def integrate(self, depth, intr, pose, variance=None, stream=None):
        K = intrinsics(intr)
        n = K.width * K.height
        _check(self.lib.tsdf_integrate(self.h, _dev_ptr(depth, n, "depth"), _dev_ptr(variance, n, "variance"),
                                       ctypes.byref(K), _pose(pose), _stream(stream)), "tsdf_integrate")

    def integrate_batch(self, depths, intr, poses, variances=None, stream=None):
        """tsdf_integrate_batch: allocate and fuse K <= 8 frames in one pass
        (bitwise equal to K sequential allocate + integrate calls)."""
        K = intrinsics(intr)
        n = K.width * K.height
        k = len(depths)
        dptr = (_P * k)(*[_dev_ptr(d, n, "depth") for d in depths])
        vptr = None if variances is None else (_P * k)(*[_dev_ptr(v, n, "variance") for v in variances])
        poses = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(k, 16))
        _check(self.lib.tsdf_integrate_batch(self.h, k, dptr, vptr, ctypes.byref(K),
                                             poses.ctypes.data_as(_PD), _stream(stream)), "tsdf_integrate_batch")

    def fuse(self, depth, intr, pose, variance=None, stream=None):
        """Allocate then integrate one frame."""
        self.allocate(depth, intr, pose, stream)
        self.integrate(depth, intr, pose, variance, stream)

    def raycast(self, intr, pose, out=None, stream=None):
        """Returns (depth (H,W), normal (H,W,3), vertex (H,W,3)) CUDA tensors."""
        import torch
        K = intrinsics(intr)
        H, W = K.height, K.width
        if out is None:
            dev = torch.device("cuda", torch.cuda.current_device())
            out = (torch.empty((H, W), dtype=torch.float32, device=dev),
                   torch.empty((H, W, 3), dtype=torch.float32, device=dev),
                   torch.empty((H, W, 3), dtype=torch.float32, device=dev))
        d, n, v = out
        _check(self.lib.tsdf_raycast(self.h, ctypes.byref(K), _pose(pose), _dev_ptr(d, H * W, "depth_out"),
                                     _dev_ptr(n, 3 * H * W, "normal_out"), _dev_ptr(v, 3 * H * W, "vertex_out"),
                                     _stream(stream)), "tsdf_raycast")
        return out

    def raycast_noalloc(self, intr, pose, out, stream=None):
        """tsdf_raycast_noalloc: the raycast into caller-owned ``out`` maps
        (depth (H,W), normal (H,W,3), vertex (H,W,3)) with no device allocation,
        for callers that must not allocate during the call (images up to
        1280 x 1024 pixels; concurrent calls on one device race)."""
        K = intrinsics(intr)
        H, W = K.height, K.width
        d, n, v = out
        _check(self.lib.tsdf_raycast_noalloc(self.h, ctypes.byref(K), _pose(pose), _dev_ptr(d, H * W, "depth_out"),
                                             _dev_ptr(n, 3 * H * W, "normal_out"),
                                             _dev_ptr(v, 3 * H * W, "vertex_out"), _stream(stream)),
               "tsdf_raycast_noalloc")
        return out

    def raycast_trace(self, intr, pose, stream=None) -> dict:
        """tsdf_raycast_trace: traversal counts of the raycast at ``pose``
        (samples, table lookups, distinct 32-byte sectors of T and of the block
        table read, rays, hits). Synchronous."""
        K = intrinsics(intr)
        c = RaycastCounts()
        _check(self.lib.tsdf_raycast_trace(self.h, ctypes.byref(K), _pose(pose), ctypes.byref(c), _stream(stream)),
               "tsdf_raycast_trace")
        return c.as_dict()

    def mesh(self, stream=None):
        """tsdf_mesh: the marching-cubes surface as an (n, 3, 3) float32 device
        tensor of world-space triangles."""
        import torch
        n = ctypes.c_int64(0)
        _check(self.lib.tsdf_mesh(self.h, None, 0, ctypes.byref(n), _stream(stream)), "tsdf_mesh")
        out = torch.empty((max(int(n.value), 1), 3, 3), dtype=torch.float32,
                          device=torch.device("cuda", torch.cuda.current_device()))
        if n.value:
            _check(self.lib.tsdf_mesh(self.h, ctypes.c_void_p(out.data_ptr()), int(n.value), ctypes.byref(n),
                                      _stream(stream)), "tsdf_mesh")
        return out[:int(n.value)]

    def icp(self, depth, intr, model_vertex, model_normal, model_pose, pose0, params=None, stream=None):
        """tsdf_icp: refine ``pose0`` (4x4 camera -> world) by registering the
        frame ``depth`` (H, W) to the model maps (H, W, 3 world vertex / normal,
        from a raycast at ``model_pose``). Returns (pose, statistics)."""
        K = intrinsics(intr)
        n = K.width * K.height
        prm = icp_params(**(params or {}))
        pose = _pose(pose0)
        res = IcpResult()
        _check(self.lib.tsdf_icp(self.h, _dev_ptr(depth, n, "depth"), ctypes.byref(K),
                                 _dev_ptr(model_vertex, 3 * n, "model_vertex"),
                                 _dev_ptr(model_normal, 3 * n, "model_normal"), _pose(model_pose), ctypes.byref(prm),
                                 pose, ctypes.byref(res), _stream(stream)), "tsdf_icp")
        return np.array(pose[:], np.float64).reshape(4, 4), res.as_dict()

    def icp_sums(self, depth, intr, model_vertex, model_normal, model_pose, pose, params=None, stream=None):
        """tsdf_icp_sums: the 29 plain Eq. 4 sums and the matched box of one
        matching pass at ``pose``."""
        K = intrinsics(intr)
        n = K.width * K.height
        prm = icp_params(**(params or {}))
        sums = (ctypes.c_double * 29)()
        box = (ctypes.c_float * 6)()
        _check(self.lib.tsdf_icp_sums(self.h, _dev_ptr(depth, n, "depth"), ctypes.byref(K),
                                      _dev_ptr(model_vertex, 3 * n, "model_vertex"),
                                      _dev_ptr(model_normal, 3 * n, "model_normal"), _pose(model_pose),
                                      ctypes.byref(prm), _pose(pose), sums, box, _stream(stream)), "tsdf_icp_sums")
        return np.array(sums[:]), np.array(box[:], np.float32)

    def launch_config(self) -> dict:
        c = LaunchConfig()
        _check(self.lib.tsdf_get_launch_config(self.h, ctypes.byref(c)), "tsdf_get_launch_config")
        return c.as_dict()

    def set_launch_config(self, **kw):
        c = LaunchConfig()
        _check(self.lib.tsdf_get_launch_config(self.h, ctypes.byref(c)), "tsdf_get_launch_config")
        names = {f for f, _ in LaunchConfig._fields_}
        for k, v in kw.items():
            if k not in names:
                raise TypeError(f"set_launch_config: unknown field {k!r} (fields: {sorted(names)})")
            setattr(c, k, int(v))
        _check(self.lib.tsdf_set_launch_config(self.h, ctypes.byref(c)), "tsdf_set_launch_config")

    def autotune(self, depths, intr, poses, cache_path: Optional[str] = None):
        """tsdf_autotune: returns (chosen launch shape, loaded_from_cache). Empties the volume."""
        K = intrinsics(intr)
        n = K.width * K.height
        k = len(depths)
        dptr = (_P * k)(*[_dev_ptr(d, n, "depth") for d in depths])
        poses = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(k, 16))
        out = LaunchConfig()
        hit = ctypes.c_int32(0)
        _check(self.lib.tsdf_autotune(self.h, k, dptr, ctypes.byref(K), poses.ctypes.data_as(_PD),
                                      None if cache_path is None else cache_path.encode(), ctypes.byref(out),
                                      ctypes.byref(hit)), "tsdf_autotune")
        return out.as_dict(), bool(hit.value)

    def set_variance_mlp(self, bf16_weights):
        """Install a learned-variance network (numpy uint16 bfloat16 bits, 1985)
        or remove it (None)."""
        if bf16_weights is None:
            _check(self.lib.tsdf_set_variance_mlp(self.h, None, 0), "tsdf_set_variance_mlp")
            return
        w = np.ascontiguousarray(bf16_weights, np.uint16)
        _check(self.lib.tsdf_set_variance_mlp(self.h, w.ctypes.data_as(_P), w.size), "tsdf_set_variance_mlp")

    def status(self) -> int:
        return int(self.lib.tsdf_get_status(self.h))

    def check(self):
        _check(self.status(), "tsdf_get_status")

    def stats(self) -> dict:
        s = Stats()
        _check(self.lib.tsdf_get_stats(self.h, ctypes.byref(s)), "tsdf_get_stats")
        return s.as_dict()

    def export(self, values: bool = True) -> Export:
        n = ctypes.c_int64(0)
        _check(self.lib.tsdf_export(self.h, None, None, None, 0, ctypes.byref(n)), "tsdf_export")
        m = int(n.value)
        cf = np.empty((m, 4), np.int32)
        T = np.empty((m, 512), np.float32) if values else np.empty((m, 0), np.float32)
        P = np.empty((m, 512), np.float32) if values else np.empty((m, 0), np.float32)
        _check(self.lib.tsdf_export(self.h, cf.ctypes.data_as(_P), T.ctypes.data_as(_P) if values else None,
                                    P.ctypes.data_as(_P) if values else None, m, ctypes.byref(n)), "tsdf_export")
        return Export(cf[:, :3].copy(), cf[:, 3].copy(), T, P)

    def get_config(self) -> Config:
        """tsdf_get_config: the volume's configuration now (the origin moves with shift)."""
        c = Config()
        _check(self.lib.tsdf_get_config(self.h, ctypes.byref(c)), "tsdf_get_config")
        return c

    @property
    def origin(self) -> tuple:
        return tuple(float(x) for x in self.get_config().origin)

    def _evicted(self, call, what: str) -> Evicted:
        n = ctypes.c_int64(0)
        st = call(0, None, None, None, ctypes.byref(n))
        if st == OK:
            m = 0
        elif st == ERR_CAPACITY:
            m = int(n.value)
        else:
            _check(st, what)
        cf = np.empty((m, 4), np.int32)
        T = np.empty((m, 512), np.float32)
        P = np.empty((m, 512), np.float32)
        if m:
            _check(call(m, cf.ctypes.data_as(_P), T.ctypes.data_as(_P), P.ctypes.data_as(_P), ctypes.byref(n)), what)
        return Evicted(cf[:, :3].copy(), cf[:, 3].copy(), T, P)

    def evict(self, lo, hi, stream=None) -> Evicted:
        """tsdf_evict: remove and return every block outside the block box [lo, hi)."""
        a = (ctypes.c_int32 * 3)(*[int(x) for x in lo])
        b = (ctypes.c_int32 * 3)(*[int(x) for x in hi])
        return self._evicted(lambda m, cf, T, P, n: self.lib.tsdf_evict(self.h, a, b, m, cf, T, P, n,
                                                                         _stream(stream)), "tsdf_evict")

    def shift(self, d, stream=None) -> Evicted:
        """tsdf_shift: move the grid by d blocks (origin += 8 s d); returns the
        blocks that left it."""
        dd = (ctypes.c_int32 * 3)(*[int(x) for x in d])
        out = self._evicted(lambda m, cf, T, P, n: self.lib.tsdf_shift(self.h, dd, m, cf, T, P, n, _stream(stream)),
                            "tsdf_shift")
        self.config = self.get_config()
        return out

    def import_blocks(self, coords, T, P, stream=None):
        """tsdf_import: add blocks (coords (n, 3) or (n, 4), T and P (n, 512))."""
        coords = np.asarray(coords, np.int32)
        n = coords.shape[0]
        cf = np.zeros((n, 4), np.int32)
        cf[:, :3] = coords[:, :3]
        T = np.ascontiguousarray(T, np.float32).reshape(n, 512)
        P = np.ascontiguousarray(P, np.float32).reshape(n, 512)
        _check(self.lib.tsdf_import(self.h, n, cf.ctypes.data_as(_P), T.ctypes.data_as(_P), P.ctypes.data_as(_P),
                                    _stream(stream)), "tsdf_import")


class Graph:
    """tsdf_graph_*: one fusion step (K frames, then a raycast at the last pose)
    recorded as a CUDA graph and replayed per step."""

    def __init__(self, volume: "Volume", intr, K: int = 1):
        self.volume = volume
        self.lib = volume.lib
        self.K = int(K)
        self.intr = intrinsics(intr)
        h = _P()
        _check(self.lib.tsdf_graph_create(volume.h, self.K, ctypes.byref(self.intr), ctypes.byref(h)),
               "tsdf_graph_create")
        self.h = h

    def launch(self, depths, poses, out, variances=None, stream=None):
        n = self.intr.width * self.intr.height
        dptr = (_P * self.K)(*[_dev_ptr(d, n, "depth") for d in depths])
        vptr = None if variances is None else (_P * self.K)(*[_dev_ptr(v, n, "variance") for v in variances])
        poses = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(self.K, 16))
        d, nm, vm = out
        _check(self.lib.tsdf_graph_launch(self.h, dptr, vptr, poses.ctypes.data_as(_PD), _dev_ptr(d, n, "depth_out"),
                                          _dev_ptr(nm, 3 * n, "normal_out"), _dev_ptr(vm, 3 * n, "vertex_out"),
                                          _stream(stream)), "tsdf_graph_launch")
        return out

    def launch_host(self, depths, poses, out, stream=None):
        """The same step from K host depth maps (torch CPU tensors, pinned for an
        overlapped copy, or numpy arrays; float32, contiguous). The library
        copies them on its own stream; keep them unchanged until the step's
        work on ``stream`` has completed."""
        n = self.intr.width * self.intr.height
        hptr = (_P * self.K)(*[_host_ptr(d, n, "depth") for d in depths])
        poses = np.ascontiguousarray(np.asarray(poses, dtype=np.float64).reshape(self.K, 16))
        d, nm, vm = out
        _check(self.lib.tsdf_graph_launch_host(self.h, hptr, poses.ctypes.data_as(_PD), _dev_ptr(d, n, "depth_out"),
                                               _dev_ptr(nm, 3 * n, "normal_out"), _dev_ptr(vm, 3 * n, "vertex_out"),
                                               _stream(stream)), "tsdf_graph_launch_host")
        return out

    def set_events(self, events):
        """Four torch.cuda.Event (timing) recorded at the stage boundaries of the
        next launches, or None."""
        if events is None:
            _check(self.lib.tsdf_graph_set_events(self.h, None), "tsdf_graph_set_events")
            return
        for e in events:
            if e.cuda_event == 0:
                e.record()          # make torch create the event
        arr = (_P * 4)(*[e.cuda_event for e in events])
        _check(self.lib.tsdf_graph_set_events(self.h, arr), "tsdf_graph_set_events")

    @property
    def instantiations(self) -> int:
        return int(self.lib.tsdf_graph_instantiations(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.tsdf_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def quadratic_variance(depth, sigma_coeff: float, out=None, stream=None):
    import torch
    n = depth.numel()
    if out is None:
        out = torch.empty_like(depth)
    _check(load().tsdf_quadratic_variance(_dev_ptr(depth, n, "depth"), n, float(sigma_coeff),
                                          _dev_ptr(out, n, "var_out"), _stream(stream)), "tsdf_quadratic_variance")
    return out
