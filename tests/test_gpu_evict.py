"""Block eviction, import and volume shift on the GPU (tsdf_evict, tsdf_import,
tsdf_shift; section "Discussion") against the oracle.

Bars: the evicted block set equals the oracle's; evicted and kept data move bit
for bit (compared with the export taken before); an evict + import round trip
restores the volume and its raycast bit for bit; after a shift the origin
equals the oracle's exactly, and fusing and raycasting further frames meet the
parity bars of test_gpu_parity.
"""
import ctypes
import json

import numpy as np
import pytest
import torch

import oracle
from oracle import compare
from paper_1311_7194_b300 import synth, tsdf

pytestmark = pytest.mark.gpu

AMB_PX = 5e-4
STORAGES = [tsdf.STORAGE_F32, tsdf.STORAGE_F16, tsdf.STORAGE_SNORM16]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1311_7194_b300 import build
    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _fuse(vol, ov, seq, frames):
    for k in frames:
        vol.fuse(_cuda(seq.depth[k]), seq.intr, seq.poses[k])
        if ov is not None:
            ov.fuse(seq.depth[k], seq.poses[k])


def _keys(coords, nb):
    c = np.asarray(coords, np.int64)
    return c[:, 0] + nb * (c[:, 1] + nb * c[:, 2])


def _by_key(coords, frames, T, P, nb):
    o = np.argsort(_keys(coords, nb), kind="stable")
    return _keys(coords, nb)[o], np.asarray(frames)[o], T[o], P[o]


def _bits(a):
    """float32 bit patterns, every NaN (chi) mapped to one pattern: the host
    export and the device decode of a 16-bit chi may give different NaNs."""
    b = np.ascontiguousarray(a, np.float32).view(np.uint32).copy()
    b[np.isnan(np.asarray(a, np.float32))] = 0x7fc00000
    return b


def _check_values(vol, ov, seq):
    nb = seq.volume.grid_dim // 8
    ge, oe = vol.export(), ov.export()
    r = compare.compare_blocks(ge.coords, ge.alloc_frame, oe.coords, oe.alloc_frame, nb)
    assert r["keys_equal"] and r["frames_equal"], r
    _, _, gT, gP = compare.sort_by_key(ge.coords, ge.alloc_frame, ge.T, ge.P, nb)
    v = compare.compare_values(gT, gP, oe.T, oe.P, oe.amb, seq.volume.truncation)
    assert v["ok"], json.dumps(v)
    return v


def _check_raycast(vol, ov, seq, pose, min_compared=100):
    gd, gn, gv = (t.cpu().numpy() for t in vol.raycast(seq.intr, pose))
    od, ovx, onr, ofl = ov.raycast(pose)
    r = compare.compare_raycast(gd, gn, gv, od, ovx, onr, ofl, seq.intr, pose, seq.volume.voxel_size,
                                seq.volume.truncation, field_fn=ov.field)
    assert r["ok"], json.dumps(r)
    assert r["compared"] >= min_compared, json.dumps(r)
    return r


@pytest.mark.parametrize("storage", STORAGES, ids=["f32", "f16", "snorm16"])
def test_evict_and_import_move_data_bit_exactly(storage):
    seq = synth.sphere_sequence(n_frames=6)
    nb = seq.volume.grid_dim // 8
    vol = tsdf.Volume.from_params(seq.volume, storage=storage)
    ov = oracle.OracleVolume(seq.volume, seq.intr, amb_px=AMB_PX, store_values=False)
    _fuse(vol, ov, seq, range(6))
    pose = seq.poses[-1]
    maps0 = [t.cpu().numpy() for t in vol.raycast(seq.intr, pose)]
    before = vol.export()
    lo, hi = [5, 10, 8], [20, 30, 16]
    ev = vol.evict(lo, hi)
    oev = ov.evict(lo, hi)
    # the same blocks as the oracle's eviction, and exactly those outside the box
    assert len(ev.coords) > 100
    assert np.array_equal(np.sort(_keys(ev.coords, nb)), np.sort(_keys(oev.coords, nb)))
    out = np.any((before.coords < lo) | (before.coords >= hi), axis=1)
    kb, fb, Tb, Pb = _by_key(before.coords, before.alloc_frame, before.T, before.P, nb)
    ke, fe, Te, Pe = _by_key(ev.coords, ev.frames, ev.T, ev.P, nb)
    sel = np.isin(kb, ke)
    assert sel.sum() == out.sum()
    assert np.array_equal(fb[sel], fe)
    assert np.array_equal(_bits(Tb[sel]), _bits(Te)) and np.array_equal(_bits(Pb[sel]), _bits(Pe))
    # the kept blocks keep their data bit for bit (whatever slot they now hold)
    after = vol.export()
    ka, fa, Ta, Pa = _by_key(after.coords, after.alloc_frame, after.T, after.P, nb)
    assert np.array_equal(ka, kb[~sel]) and np.array_equal(fa, fb[~sel])
    assert np.array_equal(_bits(Ta), _bits(Tb[~sel])) and np.array_equal(_bits(Pa), _bits(Pb[~sel]))
    assert vol.stats()["n_blocks"] == len(before.coords) - len(ev.coords)
    # back again: the volume and its raycast, bit for bit
    vol.import_blocks(ev.coords, ev.T, ev.P)
    ov.import_blocks(oev.coords, oev.T, oev.P)
    back = vol.export()
    k1, f1, T1, P1 = _by_key(back.coords, back.alloc_frame, back.T, back.P, nb)
    assert np.array_equal(k1, kb)
    assert np.array_equal(_bits(T1), _bits(Tb)) and np.array_equal(_bits(P1), _bits(Pb))
    assert np.array_equal(f1[~sel], fb[~sel]) and np.all(f1[sel] == 6)
    maps1 = [t.cpu().numpy() for t in vol.raycast(seq.intr, pose)]
    for a, b in zip(maps0, maps1):
        assert np.array_equal(_bits(a), _bits(b))
    oe = ov.export(values=False)
    r = compare.compare_blocks(back.coords, back.alloc_frame, oe.coords, oe.alloc_frame, nb)
    assert r["keys_equal"] and r["frames_equal"], r
    vol.check()


def test_evict_then_fuse_and_raycast_match_the_oracle():
    """Compaction of a larger pool (freed slots refilled from its end), then more
    frames fused and raycast: parity with the oracle, which evicted the same box."""
    seq = synth.room_sequence(n_frames=8, width=157, height=117, grid_dim=512, voxel_size=6e-3,
                              block_capacity=1 << 16)
    vol = tsdf.Volume.from_params(seq.volume)
    ov = oracle.OracleVolume(seq.volume, seq.intr, amb_px=AMB_PX)
    _fuse(vol, ov, seq, range(4))
    nb = seq.volume.grid_dim // 8
    c = vol.export(values=False).coords
    lo = np.percentile(c, 25, axis=0).astype(int)
    hi = (np.percentile(c, 90, axis=0) + 1).astype(int)
    ev, oev = vol.evict(lo, hi), ov.evict(lo, hi)
    assert 0.2 * len(c) < len(ev.coords) < 0.9 * len(c)
    assert np.array_equal(np.sort(_keys(ev.coords, nb)), np.sort(_keys(oev.coords, nb)))
    _fuse(vol, ov, seq, range(4, 8))
    vol.check()
    v = _check_values(vol, ov, seq)
    assert v["compared"] > 100000
    _check_raycast(vol, ov, seq, seq.poses[-1])


def test_shift_then_fuse_and_raycast_match_the_oracle():
    seq = synth.sphere_sequence(n_frames=10)
    vol = tsdf.Volume.from_params(seq.volume)
    ov = oracle.OracleVolume(seq.volume, seq.intr, amb_px=AMB_PX)
    _fuse(vol, ov, seq, range(5))
    nb = seq.volume.grid_dim // 8
    d = [4, -2, 3]
    ev, oev = vol.shift(d), ov.shift(d)
    assert len(ev.coords) > 0
    assert np.array_equal(np.sort(_keys(ev.coords, nb)), np.sort(_keys(oev.coords, nb)))
    # the same double-precision origin on both sides
    assert vol.origin == tuple(float(x) for x in ov.origin)
    assert np.allclose(vol.origin, np.asarray(seq.volume.origin) + 8 * np.asarray(d) * float(np.float32(seq.volume.voxel_size)),
                       rtol=0, atol=1e-12)
    e = vol.export(values=False)
    assert np.all((e.coords >= 0) & (e.coords < nb))
    _check_values(vol, ov, seq)
    _fuse(vol, ov, seq, range(5, 10))
    vol.check()
    v = _check_values(vol, ov, seq)
    assert v["compared"] > 100000
    _check_raycast(vol, ov, seq, seq.poses[-1])


def test_eviction_and_import_errors_change_nothing():
    seq = synth.sphere_sequence(n_frames=3)
    vol = tsdf.Volume.from_params(seq.volume)
    _fuse(vol, None, seq, range(3))
    lib = vol.lib
    before = vol.export()
    lo = (ctypes.c_int32 * 3)(5, 10, 8)
    hi = (ctypes.c_int32 * 3)(20, 30, 16)
    n = ctypes.c_int64(0)
    buf = np.empty((1, 4), np.int32)
    assert lib.tsdf_evict(vol.h, lo, hi, 1, buf.ctypes.data_as(ctypes.c_void_p), None, None, ctypes.byref(n),
                          None) == tsdf.ERR_CAPACITY
    assert n.value > 1
    bad = (ctypes.c_int32 * 3)(21, 10, 8)         # lo > hi on x
    assert lib.tsdf_evict(vol.h, bad, hi, 10, None, None, None, ctypes.byref(n), None) == tsdf.ERR_INVALID_ARG
    big = (ctypes.c_int32 * 3)(1 << 24, 0, 0)
    assert lib.tsdf_shift(vol.h, big, 10, None, None, None, ctypes.byref(n), None) == tsdf.ERR_INVALID_ARG
    with pytest.raises(tsdf.TsdfError):           # an allocated block
        vol.import_blocks(before.coords[:1], before.T[:1], before.P[:1])
    with pytest.raises(tsdf.TsdfError):           # outside the grid
        vol.import_blocks(np.array([[-1, 0, 0]]), before.T[:1], before.P[:1])
    after = vol.export()
    assert np.array_equal(after.coords, before.coords)
    assert np.array_equal(_bits(after.T), _bits(before.T))
    # a pool that cannot take the blocks back
    small = tsdf.Volume.from_params(seq.volume, block_capacity=len(before.coords) + 1)
    _fuse(small, None, seq, range(3))
    ev = small.evict([5, 10, 8], [20, 30, 16])
    assert len(ev.coords) > 2
    _fuse(small, None, seq, range(3))                # the freed slots fill up again
    free = small.config.block_capacity - small.stats()["n_blocks"]
    assert free < len(ev.coords)
    with pytest.raises(tsdf.TsdfError) as err:
        small.import_blocks(ev.coords, ev.T, ev.P)
    assert err.value.status == tsdf.ERR_CAPACITY
    vol.check()
