"""16-bit distance storage (FP16, snorm16; P stays float32).

Only how T is held between launches changes, so block sets, chi patterns and P
equal the float32 volume's exactly (P never depends on T), and T differs by at
most one rounding half-step per update: each Alg. 3 update is a contraction
(T' = (1-K) T + K T_k), so an earlier storage error never grows. Bound per
update: snorm16 delta/32767/2, FP16 2^-11 delta (half an ulp of |T| <= delta).
The errors against the FP64 oracle are reported."""
import json

import numpy as np
import pytest
import torch

import oracle
from oracle import compare
from paper_1311_7194_b300 import synth, tsdf

pytestmark = pytest.mark.gpu

HALF_STEP = {tsdf.STORAGE_SNORM16: 0.5 / 32767 * 1.001, tsdf.STORAGE_F16: 2.0 ** -11}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1311_7194_b300 import build
    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _fuse(seq, storage, batch=None):
    vol = tsdf.Volume.from_params(seq.volume, storage=storage)
    d = [torch.from_numpy(x).cuda() for x in seq.depth]
    if batch:
        for k in range(0, seq.n_frames, batch):
            vol.integrate_batch(d[k:k + batch], seq.intr, seq.poses[k:k + batch])
    else:
        for k in range(seq.n_frames):
            vol.fuse(d[k], seq.intr, seq.poses[k])
    vol.check()
    return vol


def _sequences():
    return [synth.sphere_sequence(n_frames=10),
            synth.room_sequence(n_frames=10, width=160, height=120, grid_dim=512, voxel_size=6e-3,
                                block_capacity=1 << 16)]


@pytest.mark.parametrize("storage", [tsdf.STORAGE_F16, tsdf.STORAGE_SNORM16], ids=["f16", "snorm16"])
@pytest.mark.parametrize("batch", [None, 5], ids=["sequential", "batched"])
def test_16bit_storage_against_float32_and_oracle(storage, batch):
    for seq in _sequences():
        n = seq.n_frames
        delta = seq.volume.truncation
        bound = n * HALF_STEP[storage] * delta
        ref = _fuse(seq, tsdf.STORAGE_F32).export()
        got = _fuse(seq, storage, batch).export()
        assert np.array_equal(ref.coords, got.coords) and np.array_equal(ref.alloc_frame, got.alloc_frame)
        chi = np.isnan(ref.T)
        assert np.array_equal(chi, np.isnan(got.T))
        assert np.array_equal(ref.P[~chi], got.P[~chi]), "P must not depend on the storage of T"
        err32 = np.abs(got.T[~chi].astype(np.float64) - ref.T[~chi])
        assert err32.max() <= bound, (err32.max() / delta, bound / delta)
        # against the FP64 oracle
        ov = oracle.OracleVolume(seq.volume, seq.intr, amb_px=5e-4)
        for k in range(n):
            ov.fuse(seq.depth[k], seq.poses[k])
        oe = ov.export()
        nb = seq.volume.grid_dim // 8
        _, _, gT, gP = compare.sort_by_key(got.coords, got.alloc_frame, got.T, got.P, nb)
        v = compare.compare_values(gT, gP, oe.T, oe.P, oe.amb, delta, tol_T=bound / delta + 1e-5)
        assert v["ok"], json.dumps(v)
        ok = ~np.isnan(oe.T) & ~oe.amb
        e = np.abs(gT.astype(np.float64) - oe.T)[ok] / delta
        print(f"{seq.name} storage={storage} batch={batch}: |T - oracle|/delta max {e.max():.3e} "
              f"rms {np.sqrt((e ** 2).mean()):.3e} (bound {bound / delta:.3e})")


@pytest.mark.parametrize("storage", [tsdf.STORAGE_F16, tsdf.STORAGE_SNORM16], ids=["f16", "snorm16"])
def test_16bit_storage_raycast_parity(storage):
    seq = synth.sphere_sequence(n_frames=10)
    vol = _fuse(seq, storage)
    ov = oracle.OracleVolume(seq.volume, seq.intr, amb_px=5e-4)
    for k in range(seq.n_frames):
        ov.fuse(seq.depth[k], seq.poses[k])
    pose = seq.poses[-1]
    gd, gn, gv = (t.cpu().numpy() for t in vol.raycast(seq.intr, pose))
    od, ovx, onr, ofl = ov.raycast(pose)
    r = compare.compare_raycast(gd, gn, gv, od, ovx, onr, ofl, seq.intr, pose, seq.volume.voxel_size,
                                seq.volume.truncation, field_fn=ov.field, tol_field=0.1)
    assert r["ok"], json.dumps(r)
    assert r["compared"] > 1500
