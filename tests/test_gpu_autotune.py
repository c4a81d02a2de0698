"""Launch shapes change speed only: every integrate / raycast shape gives the
same volume and maps bit for bit; the autotuner picks a valid shape and caches
it."""
import os

import numpy as np
import pytest
import torch

from paper_1311_7194_b300 import synth, tsdf

pytestmark = pytest.mark.gpu

SHAPES = [dict(integrate_voxels_per_thread=8, integrate_ctas_per_sm=4, raycast_tile_w=8, raycast_tile_h=8),
          dict(integrate_voxels_per_thread=4, integrate_ctas_per_sm=24, raycast_tile_w=32, raycast_tile_h=4),
          dict(integrate_voxels_per_thread=8, integrate_ctas_per_sm=16, raycast_tile_w=16, raycast_tile_h=16),
          dict(integrate_voxels_per_thread=4, integrate_ctas_per_sm=1, raycast_tile_w=8, raycast_tile_h=16),
          dict(raycast_persistent=1), dict(raycast_persistent=1, integrate_voxels_per_thread=8)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1311_7194_b300 import build
    build.build()
    torch.cuda.set_device(0)


def _run(seq, storage=tsdf.STORAGE_F32, **shape):
    vol = tsdf.Volume.from_params(seq.volume, storage=storage)
    if shape:
        vol.set_launch_config(**shape)
    for k in range(seq.n_frames):
        vol.fuse(torch.from_numpy(seq.depth[k]).cuda(), seq.intr, seq.poses[k])
    maps = [t.cpu().numpy() for t in vol.raycast(seq.intr, seq.poses[-1])]
    return vol.export(), maps


@pytest.mark.parametrize("storage", [tsdf.STORAGE_F32, tsdf.STORAGE_SNORM16], ids=["f32", "snorm16"])
def test_launch_shapes_do_not_change_results(storage):
    seq = synth.room_sequence(n_frames=6, width=157, height=117, grid_dim=512, voxel_size=6e-3,
                              block_capacity=1 << 16)
    ref_e, ref_m = _run(seq, storage)
    for shape in SHAPES:
        e, m = _run(seq, storage, **shape)
        assert np.array_equal(ref_e.coords, e.coords)
        chi = np.isnan(ref_e.T)
        assert np.array_equal(chi, np.isnan(e.T))
        assert np.array_equal(ref_e.T[~chi], e.T[~chi]) and np.array_equal(ref_e.P[~chi], e.P[~chi])
        for a, b in zip(ref_m, m):
            assert np.array_equal(np.isnan(a), np.isnan(b))
            assert np.array_equal(a[~np.isnan(a)], b[~np.isnan(b)])


def test_bad_launch_shapes_are_rejected():
    seq = synth.sphere_sequence(n_frames=1)
    vol = tsdf.Volume.from_params(seq.volume)
    for bad in [dict(integrate_voxels_per_thread=2), dict(integrate_ctas_per_sm=0),
                dict(integrate_ctas_per_sm=33), dict(raycast_tile_w=7), dict(raycast_persistent=2)]:
        with pytest.raises(tsdf.TsdfError):
            vol.set_launch_config(**bad)
    with pytest.raises(TypeError):
        vol.set_launch_config(integrate_vpt=8)   # not a field name: rejected, not ignored
    assert vol.launch_config() == dict(integrate_voxels_per_thread=4, integrate_ctas_per_sm=12,
                                       raycast_tile_w=16, raycast_tile_h=8, raycast_persistent=0)


def test_autotune_picks_a_valid_shape_and_caches_it(tmp_path):
    seq = synth.sphere_sequence(n_frames=6)
    d = [torch.from_numpy(x).cuda() for x in seq.depth]
    cache = str(tmp_path / "tune.jsonl")
    vol = tsdf.Volume.from_params(seq.volume)
    shape, hit = vol.autotune(d, seq.intr, seq.poses, cache)
    assert not hit and os.path.exists(cache)
    assert shape["integrate_voxels_per_thread"] in (4, 8) and 1 <= shape["integrate_ctas_per_sm"] <= 32
    assert (shape["raycast_tile_w"], shape["raycast_tile_h"]) in [(16, 8), (8, 8), (32, 4), (8, 16), (16, 16)]
    assert vol.stats()["n_blocks"] == 0          # the tuner leaves the volume empty
    vol2 = tsdf.Volume.from_params(seq.volume)
    shape2, hit2 = vol2.autotune(d, seq.intr, seq.poses, cache)
    assert hit2 and shape2 == shape and vol2.launch_config() == shape


def test_persistent_raycast_with_a_pool_beyond_32_bit_voxel_indices():
    """Pools of more than 2^23 blocks (2^32 voxels) take the persistent kernel
    with 64-bit voxel indexing; it must agree with the per-pixel kernel."""
    seq = synth.room_sequence(n_frames=4, width=157, height=117, grid_dim=512, voxel_size=6e-3,
                              block_capacity=(1 << 23) + 8)
    vol = tsdf.Volume.from_params(seq.volume, storage=tsdf.STORAGE_F16)    # 3 KB per block: 25 GB
    for k in range(seq.n_frames):
        vol.fuse(torch.from_numpy(seq.depth[k]).cuda(), seq.intr, seq.poses[k])
    maps = {}
    for persistent in (0, 1):
        vol.set_launch_config(raycast_persistent=persistent)
        maps[persistent] = [t.cpu().numpy() for t in vol.raycast(seq.intr, seq.poses[-1])]
    for a, b in zip(maps[0], maps[1]):
        assert np.array_equal(np.isnan(a), np.isnan(b)) and np.array_equal(a[~np.isnan(a)], b[~np.isnan(b)])
    assert (maps[1][0] > 0).sum() > 5000
    vol.close()
