"""The TSDF_DEBUG build (libtsdf_debug.so): device-side index checks that stand
in for a memory checker on tiny configurations.

A failed check skips the access and sets a sticky error (TSDF_ERR_BOUNDS);
nothing traps. The tests run the sphere sequence through allocation,
integration (single and K-batched), raycast and marching cubes under the
checks, require that no check fires and that every result equals the release
library's bit for bit, and provoke the error only from the host: a pool slot
outside the pool asked for through tsdf_debug_check_slot, which the check
catches before any access.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1311_7194_b300 import build, synth, tsdf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def libs():
    build.build()
    build.build(debug=True)
    torch.cuda.set_device(0)
    release = tsdf.load()
    debug = tsdf.load(tsdf.DEBUG_LIB_PATH)
    assert debug.tsdf_debug_build() == 1 and release.tsdf_debug_build() == 0
    return release, debug


def _run(lib, seq, batched=False):
    vol = tsdf.Volume.from_params(seq.volume, lib=lib)
    d = [torch.from_numpy(x).cuda() for x in seq.depth]
    if batched:
        for k in range(0, seq.n_frames, 4):
            vol.integrate_batch(d[k:k + 4], seq.intr, seq.poses[k:k + 4])
    else:
        for k in range(seq.n_frames):
            vol.fuse(d[k], seq.intr, seq.poses[k])
    maps = vol.raycast(seq.intr, seq.poses[-1])
    tris = vol.mesh()
    torch.cuda.synchronize()
    status = vol.status()
    e = vol.export()
    out = (e.coords, e.alloc_frame, e.T, e.P, *(m.cpu().numpy() for m in maps), tris.cpu().numpy())
    vol.close()
    return status, out


def _equal(a, b):
    for x, y in zip(a, b):
        assert np.array_equal(np.nan_to_num(np.asarray(x), nan=-7.0), np.nan_to_num(np.asarray(y), nan=-7.0))


@pytest.mark.parametrize("batched", [False, True], ids=["sequential", "batched"])
def test_checks_pass_and_results_are_unchanged(libs, batched):
    release, debug = libs
    seq = synth.sphere_sequence(n_frames=8)
    st_r, out_r = _run(release, seq, batched)
    st_d, out_d = _run(debug, seq, batched)
    assert st_r == tsdf.OK and st_d == tsdf.OK, (st_r, st_d)
    _equal(out_r, out_d)


def test_a_slot_outside_the_pool_is_reported_not_read(libs):
    release, debug = libs
    seq = synth.sphere_sequence(n_frames=2)
    vol = tsdf.Volume.from_params(seq.volume, lib=debug)
    vol.fuse(torch.from_numpy(seq.depth[0]).cuda(), seq.intr, seq.poses[0])
    cap = int(vol.config.block_capacity)
    assert debug.tsdf_debug_check_slot(vol.h, 0, None) == tsdf.OK
    assert vol.status() == tsdf.OK
    assert debug.tsdf_debug_check_slot(vol.h, cap + 5, None) == tsdf.OK
    assert vol.status() == tsdf.ERR_BOUNDS
    assert debug.tsdf_debug_check_slot(vol.h, -1, None) == tsdf.OK
    assert vol.status() == tsdf.ERR_BOUNDS        # sticky
    vol.close()
    # the release library launches nothing for the same request
    vr = tsdf.Volume.from_params(seq.volume, lib=release)
    assert release.tsdf_debug_check_slot(vr.h, cap + 5, None) == tsdf.ERR_NOT_READY
    assert vr.status() == tsdf.OK
    vr.close()


def test_a_pool_too_small_is_a_capacity_error_not_an_index_error(libs):
    """Allocation into a 64-block pool drops the highest-key new blocks
    (TSDF_ERR_CAPACITY); no index check fires on the way, and the fused volume
    equals the release library's."""
    release, debug = libs
    seq = synth.sphere_sequence(n_frames=3)
    res = []
    for lib in (release, debug):
        vol = tsdf.Volume.from_params(seq.volume, lib=lib, block_capacity=64)
        for k in range(seq.n_frames):
            vol.fuse(torch.from_numpy(seq.depth[k]).cuda(), seq.intr, seq.poses[k])
        vol.raycast(seq.intr, seq.poses[-1])
        torch.cuda.synchronize()
        res.append((vol.status(), vol.export()))
        vol.close()
    assert res[0][0] == tsdf.ERR_CAPACITY and res[1][0] == tsdf.ERR_CAPACITY
    _equal((res[0][1].coords, res[0][1].T, res[0][1].P), (res[1][1].coords, res[1][1].T, res[1][1].P))
