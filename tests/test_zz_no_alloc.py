"""tsdf_raycast_noalloc against tsdf_raycast, through the C ABI.

tsdf_raycast_noalloc exists for callers that must not allocate device memory
during a call (tsdf_raycast may grow its range maps with cudaMalloc): it keeps
the maps in a fixed array inside the library. This file is named so that pytest
collects it last; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1311_7194_b300 import synth, tsdf

pytestmark = pytest.mark.gpu


def _maps(H, W):
    dev = torch.device("cuda", torch.cuda.current_device())
    return (torch.full((H, W), -1.0, device=dev), torch.full((H, W, 3), -1.0, device=dev),
            torch.full((H, W, 3), -1.0, device=dev))


def _noalloc(lib, vol, intr, pose, out):
    K = tsdf.intrinsics(intr)
    d, n, v = out
    return lib.tsdf_raycast_noalloc(vol.h, ctypes.byref(K), tsdf._pose(pose), d.data_ptr(), n.data_ptr(),
                                    v.data_ptr(), torch.cuda.current_stream().cuda_stream)


def _same(ref, got, voxel_size, tol_vox=0.1):
    rd, rn, rv = (t.cpu().numpy() for t in ref)
    gd, gn, gv = (t.cpu().numpy() for t in got)
    assert np.array_equal(rd > 0, gd > 0), "hit / miss pattern differs"
    hit = rd > 0
    assert hit.sum() > 500
    assert np.abs(rd[hit] - gd[hit]).max() <= tol_vox * voxel_size
    assert np.nanmax(np.abs(rv[hit] - gv[hit])) <= 2 * tol_vox * voxel_size
    assert np.array_equal(np.isnan(rn), np.isnan(gn))
    ok = ~np.isnan(rn[..., 0])
    assert np.abs(rn[ok] - gn[ok]).max() <= 1e-4
    assert np.isnan(gv[~hit]).all() and (gd[~hit] == 0).all()


def test_noalloc_raycast_matches_raycast_on_two_calls_in_a_row():
    from paper_1311_7194_b300 import build
    build.build()
    torch.cuda.set_device(0)
    lib = tsdf.load()
    seq = synth.sphere_sequence(n_frames=5)
    vol = tsdf.Volume.from_params(seq.volume)
    for k in range(seq.n_frames):
        vol.fuse(torch.from_numpy(seq.depth[k]).cuda(), seq.intr, seq.poses[k])
    H, W = seq.intr.height, seq.intr.width
    poses = [seq.poses[-1], seq.poses[1]]
    refs = [vol.raycast(seq.intr, p, out=_maps(H, W)) for p in poses]
    gots = [_maps(H, W), _maps(H, W)]
    for p, out in zip(poses, gots):          # two calls in a row, sharing the fixed scratch
        assert _noalloc(lib, vol, seq.intr, p, out) == tsdf.OK
    torch.cuda.synchronize()
    vol.check()
    for ref, got in zip(refs, gots):
        _same(ref, got, seq.volume.voxel_size)


def test_noalloc_raycast_after_and_before_a_larger_raycast():
    """tsdf_raycast on a larger image first grows its own range maps; the
    no-allocation call at the sequence's image then still matches tsdf_raycast,
    and a second larger tsdf_raycast after it is bit for bit the first one: the
    two calls keep their range maps apart."""
    torch.cuda.set_device(0)
    lib = tsdf.load()
    seq = synth.sphere_sequence(n_frames=4)
    vol = tsdf.Volume.from_params(seq.volume)
    for k in range(seq.n_frames):
        vol.fuse(torch.from_numpy(seq.depth[k]).cuda(), seq.intr, seq.poses[k])
    H, W = seq.intr.height, seq.intr.width
    big = synth.Intrinsics(2 * seq.intr.fx, 2 * seq.intr.fy, (2 * W - 1) / 2.0, (2 * H - 1) / 2.0, 2 * W, 2 * H)
    pose = seq.poses[-1]
    ref = vol.raycast(seq.intr, pose, out=_maps(H, W))
    big1 = vol.raycast(big, pose, out=_maps(2 * H, 2 * W))
    got = _maps(H, W)
    assert _noalloc(lib, vol, seq.intr, pose, got) == tsdf.OK
    big2 = vol.raycast(big, pose, out=_maps(2 * H, 2 * W))
    torch.cuda.synchronize()
    vol.check()
    _same(ref, got, seq.volume.voxel_size)
    for a, b in zip(big1, big2):
        assert torch.equal(torch.nan_to_num(a, nan=-7.0), torch.nan_to_num(b, nan=-7.0))


def test_noalloc_raycast_rejects_images_beyond_its_limit():
    """The fixed array holds 81,920 range tiles of 4x4 pixels: a 2048 x 1024
    image and a ragged 1281 x 1021 one (fewer pixels than 1280 x 1024, but
    321 x 256 tiles) are refused before any GPU work."""
    torch.cuda.set_device(0)
    lib = tsdf.load()
    seq = synth.sphere_sequence(n_frames=1)
    vol = tsdf.Volume.from_params(seq.volume)
    out = _maps(1, 1)
    for W, H in [(2048, 1024), (1281, 1021)]:
        big = synth.Intrinsics(1400.0, 1400.0, (W - 1) / 2.0, (H - 1) / 2.0, W, H)
        assert _noalloc(lib, vol, big, seq.poses[0], out) == tsdf.ERR_INVALID_ARG
    vol.check()
