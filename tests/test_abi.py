"""The C-ABI library builds, loads and exports every symbol include/tsdf.h
declares; host-side argument checks answer without touching a GPU."""
import ctypes
import math
import os
import re

import pytest

from paper_1311_7194_b300 import build as pkg_build
from paper_1311_7194_b300 import tsdf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tsdf.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(tsdf_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return tsdf.load()


def test_header_lists_the_entry_points():
    fns = header_functions()
    for name in ["tsdf_create", "tsdf_allocate", "tsdf_integrate", "tsdf_raycast", "tsdf_destroy"]:
        assert name in fns
    assert sorted(tsdf.EXPORTED) == fns


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(tsdf.LIB_PATH)
    for name in header_functions():
        assert hasattr(raw, name), f"{name} declared in tsdf.h but not exported"


def test_config_defaults(lib):
    c = tsdf.default_config()
    assert math.isclose(c.voxel_size, 1.5e-3, rel_tol=1e-6)
    assert math.isclose(c.truncation, 7.5e-3, rel_tol=1e-6)
    assert c.grid_dim == 2048 and c.block_capacity == 1 << 20
    assert c.storage == tsdf.STORAGE_F32 and c.alloc_half_samples == 0
    assert c.update_rule == tsdf.UPDATE_KALMAN
    assert math.isclose(c.update_weight, 0.1, rel_tol=1e-6) and c.weight_max == 1.0
    assert c.refine_steps == 0
    assert math.isclose(c.origin[0], -1024 * 1.5e-3, rel_tol=1e-6)


def test_status_strings(lib):
    for s in range(8):
        assert lib.tsdf_status_string(s).decode() != "unknown status"
    assert lib.tsdf_status_string(99).decode() == "unknown status"


def test_release_library_is_not_a_debug_build(lib):
    """The release library compiles the device index checks out; its
    tsdf_debug_check_slot launches nothing."""
    assert lib.tsdf_debug_build() == 0
    assert lib.tsdf_debug_check_slot(None, 0, None) == tsdf.ERR_INVALID_ARG


@pytest.mark.parametrize("field,value", [
    ("voxel_size", 0.0), ("voxel_size", float("nan")), ("truncation", -1.0),
    ("grid_dim", 100), ("grid_dim", 0), ("grid_dim", 8 * 1700), ("block_capacity", 0),
    ("block_capacity", 1 << 40), ("process_variance", -1.0), ("sigma_coeff", float("inf")),
    ("depth_max", 0.05), ("raycast_near", 0.0), ("raycast_far", 0.01), ("storage", 7),
    ("alloc_half_samples", -1), ("refine_steps", -1), ("refine_steps", 9)])
def test_create_rejects_bad_config(lib, field, value):
    c = tsdf.default_config()
    setattr(c, field, value)
    h = ctypes.c_void_p()
    assert lib.tsdf_create_ex(ctypes.byref(c), ctypes.byref(h)) == tsdf.ERR_INVALID_ARG
    assert not h.value


@pytest.mark.parametrize("rule,weight,wmax", [
    (3, 0.1, 1.0), (-1, 0.1, 1.0), (tsdf.UPDATE_AVERAGE, 0.0, 1.0), (tsdf.UPDATE_AVERAGE, 1.5, 1.0),
    (tsdf.UPDATE_AVERAGE, float("nan"), 1.0), (tsdf.UPDATE_WEIGHTED, -1.0, 1.0),
    (tsdf.UPDATE_WEIGHTED, 2.0, 1.0), (tsdf.UPDATE_WEIGHTED, 0.5, float("inf"))])
def test_create_rejects_bad_update_rules(lib, rule, weight, wmax):
    """Alg. 1 needs 0 < w <= 1, Alg. 2 needs w > 0 and a finite W_max >= w
    (checked on the host, before any device memory is touched)."""
    c = tsdf.default_config()
    c.update_rule, c.update_weight, c.weight_max = rule, weight, wmax
    h = ctypes.c_void_p()
    assert lib.tsdf_create_ex(ctypes.byref(c), ctypes.byref(h)) == tsdf.ERR_INVALID_ARG
    assert not h.value


def test_null_arguments_are_rejected(lib):
    K = tsdf.Intrinsics(100.0, 100.0, 31.5, 23.5, 64, 48)
    pose = (ctypes.c_double * 16)(*[1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1])
    assert lib.tsdf_create_ex(None, None) == tsdf.ERR_INVALID_ARG
    assert lib.tsdf_create(1e-3, 5e-3, 16, None) == tsdf.ERR_INVALID_ARG
    assert lib.tsdf_allocate(None, None, ctypes.byref(K), pose, None) == tsdf.ERR_INVALID_ARG
    assert lib.tsdf_integrate(None, None, None, ctypes.byref(K), pose, None) == tsdf.ERR_INVALID_ARG
    assert lib.tsdf_raycast(None, ctypes.byref(K), pose, None, None, None, None) == tsdf.ERR_INVALID_ARG
    assert lib.tsdf_reset(None, None) == tsdf.ERR_INVALID_ARG
    assert lib.tsdf_get_status(None) == tsdf.ERR_INVALID_ARG
    assert lib.tsdf_get_stats(None, None) == tsdf.ERR_INVALID_ARG
    n = ctypes.c_int64()
    assert lib.tsdf_export(None, None, None, None, 0, ctypes.byref(n)) == tsdf.ERR_INVALID_ARG
    assert lib.tsdf_quadratic_variance(None, -1, 1e-3, None, None) == tsdf.ERR_INVALID_ARG
    assert lib.tsdf_raycast_trace(None, ctypes.byref(K), pose, None, None) == tsdf.ERR_INVALID_ARG
    c3 = (ctypes.c_int32 * 3)(0, 0, 0)
    assert lib.tsdf_get_config(None, None) == tsdf.ERR_INVALID_ARG
    assert lib.tsdf_evict(None, c3, c3, 0, None, None, None, ctypes.byref(n), None) == tsdf.ERR_INVALID_ARG
    assert lib.tsdf_shift(None, c3, 0, None, None, None, ctypes.byref(n), None) == tsdf.ERR_INVALID_ARG
    assert lib.tsdf_import(None, 1, None, None, None, None) == tsdf.ERR_INVALID_ARG
    assert lib.tsdf_graph_launch_host(None, None, pose, None, None, None, None) == tsdf.ERR_INVALID_ARG
    lib.tsdf_destroy(None)


def test_bad_pose_and_intrinsics_are_rejected_before_any_device_work(lib):
    fake = ctypes.c_void_p(0x1000)      # never dereferenced: checks come first
    good = tsdf.Intrinsics(100.0, 100.0, 31.5, 23.5, 64, 48)
    eye = [1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1]
    bad_pose = (ctypes.c_double * 16)(*(eye[:3] + [float("nan")] + eye[4:]))
    assert lib.tsdf_allocate(fake, fake, ctypes.byref(good), bad_pose, None) == tsdf.ERR_INVALID_ARG
    for K in [tsdf.Intrinsics(0.0, 100.0, 31.5, 23.5, 64, 48), tsdf.Intrinsics(100.0, 100.0, 31.5, 23.5, 0, 48),
              tsdf.Intrinsics(100.0, float("inf"), 31.5, 23.5, 64, 48),
              tsdf.Intrinsics(100.0, 100.0, 31.5, 23.5, 1 << 16, 1 << 16)]:
        pose = (ctypes.c_double * 16)(*eye)
        assert lib.tsdf_integrate(fake, fake, None, ctypes.byref(K), pose, None) == tsdf.ERR_INVALID_ARG
        assert lib.tsdf_raycast(fake, ctypes.byref(K), pose, None, None, None, None) == tsdf.ERR_INVALID_ARG


def test_binding_refuses_cpu_tensors(lib):
    import torch
    with pytest.raises((TypeError, RuntimeError)):
        tsdf._dev_ptr(torch.zeros(4), 4, "depth")


def test_host_map_argument_checks():
    """The binding's host-map marshalling (tsdf_graph_launch_host): contiguous
    float32 host arrays of the image size pass as their own address; anything
    else is refused before the library is called."""
    import numpy as np
    import torch
    a = np.zeros((4, 6), np.float32)
    assert tsdf._host_ptr(a, 24, "depth") == a.ctypes.data
    t = torch.zeros((4, 6), dtype=torch.float32)
    assert tsdf._host_ptr(t, 24, "depth") == t.data_ptr()
    for bad in (np.zeros((4, 6), np.float64), np.zeros((4, 7), np.float32), np.zeros((6, 4), np.float32).T,
                torch.zeros((4, 6), dtype=torch.float64), [0.0] * 24):
        with pytest.raises(ValueError):
            tsdf._host_ptr(bad, 24, "depth")
