"""K-frame batched integration (tsdf_integrate_batch) against K sequential
allocate + integrate calls: block sets, allocation frames, T and P must be equal
bit for bit (the same per-voxel operations in the same order)."""
import json

import numpy as np
import pytest
import torch

import oracle
from oracle import compare
from paper_1311_7194_b300 import synth, tsdf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1311_7194_b300 import build
    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _sequential(seq, vars_=None, **over):
    vol = tsdf.Volume.from_params(seq.volume, **over)
    for k in range(seq.n_frames):
        vol.fuse(_cuda(seq.depth[k]), seq.intr, seq.poses[k], None if vars_ is None else _cuda(vars_[k]))
    return vol


def _batched(seq, splits, vars_=None, **over):
    vol = tsdf.Volume.from_params(seq.volume, **over)
    k = 0
    for K in splits:
        d = [_cuda(seq.depth[k + j]) for j in range(K)]
        v = None if vars_ is None else [_cuda(vars_[k + j]) for j in range(K)]
        vol.integrate_batch(d, seq.intr, seq.poses[k:k + K], v)
        k += K
    assert k == seq.n_frames
    return vol


def _assert_same(a, b):
    ea, eb = a.export(), b.export()
    assert np.array_equal(ea.coords, eb.coords)
    assert np.array_equal(ea.alloc_frame, eb.alloc_frame)
    ta, tb = ea.T.view(np.uint32), eb.T.view(np.uint32)
    chi = np.isnan(ea.T)
    assert np.array_equal(chi, np.isnan(eb.T))
    assert np.array_equal(ta[~chi], tb[~chi]), "T differs"
    assert np.array_equal(ea.P.view(np.uint32)[~chi], eb.P.view(np.uint32)[~chi]), "P differs"
    sa, sb = a.stats(), b.stats()
    assert sa["frames"] == sb["frames"] and sa["voxel_updates_total"] == sb["voxel_updates_total"]
    # voxels touched (a: one frame per call, b: K frames per call): every update
    # of a one-frame call touches its voxel once; a K-frame call touches each
    # voxel it updates once, however many of its frames update it (at most 8)
    assert sa["voxels_touched_total"] == sa["voxel_updates_total"]
    assert sb["voxel_updates_total"] / 8 <= sb["voxels_touched_total"] <= sb["voxel_updates_total"]
    return ea


@pytest.mark.parametrize("splits", [[4, 4, 2], [8, 2], [1] * 10, [3, 7]])
def test_batch_equals_sequential_sphere(splits):
    seq = synth.sphere_sequence(n_frames=10)
    _assert_same(_sequential(seq), _batched(seq, splits))


def test_batch_equals_sequential_room_ragged():
    seq = synth.room_sequence(n_frames=16, width=157, height=117, grid_dim=512, voxel_size=6e-3,
                              block_capacity=1 << 16)
    _assert_same(_sequential(seq), _batched(seq, [8, 8]))


def test_batch_with_variance_maps_and_process_variance():
    seq = synth.sphere_sequence(n_frames=8)
    rng = np.random.default_rng(7)
    vars_ = [rng.uniform(0.5e-7, 4e-7, seq.depth[0].shape).astype(np.float32) for _ in range(8)]
    a = _sequential(seq, vars_, process_variance=3e-8)
    b = _batched(seq, [5, 3], vars_, process_variance=3e-8)
    _assert_same(a, b)


def test_batch_matches_oracle():
    seq = synth.sphere_sequence(n_frames=8)
    vol = _batched(seq, [8])
    ov = oracle.OracleVolume(seq.volume, seq.intr, amb_px=5e-4)
    for k in range(seq.n_frames):
        ov.fuse(seq.depth[k], seq.poses[k])
    nb = seq.volume.grid_dim // 8
    ge, oe = vol.export(), ov.export()
    r = compare.compare_blocks(ge.coords, ge.alloc_frame, oe.coords, oe.alloc_frame, nb)
    assert r["keys_equal"] and r["frames_equal"], r
    _, _, gT, gP = compare.sort_by_key(ge.coords, ge.alloc_frame, ge.T, ge.P, nb)
    v = compare.compare_values(gT, gP, oe.T, oe.P, oe.amb, seq.volume.truncation)
    assert v["ok"], json.dumps(v)


def test_batch_rejects_bad_arguments():
    seq = synth.sphere_sequence(n_frames=1)
    vol = tsdf.Volume.from_params(seq.volume)
    d = _cuda(seq.depth[0])
    for bad in ([], [d] * 9):
        poses = np.stack([seq.poses[0]] * len(bad)) if bad else np.zeros((0, 4, 4))
        with pytest.raises(tsdf.TsdfError) as ei:
            vol.integrate_batch(bad, seq.intr, poses)
        assert ei.value.status == tsdf.ERR_INVALID_ARG
