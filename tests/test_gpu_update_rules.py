"""The paper's other update rules as integrate variants: Alg. 1 (running
average with a fixed weight) and Alg. 2 (weighted average bounded by W_max)
against the FP64 oracle, K-batched equal to sequential, and a re-run of the
paper's comparison of the rules on measurements whose variance keeps growing
(section "Integration of Measurements", after Alg. 3): the Kalman filter, told
each frame's variance, keeps the estimate close to the truth where the fixed
weights of Alg. 1 and Alg. 2 let the noisier data in."""
import json

import numpy as np
import pytest
import torch

import oracle
from oracle import compare
from paper_1311_7194_b300 import synth, tsdf

pytestmark = pytest.mark.gpu

RULES = {"average": dict(update_rule=tsdf.UPDATE_AVERAGE, update_weight=0.25, weight_max=1.0),
         "weighted": dict(update_rule=tsdf.UPDATE_WEIGHTED, update_weight=0.5, weight_max=2.5)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1311_7194_b300 import build
    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.mark.parametrize("rule", list(RULES))
def test_update_rule_matches_oracle(rule):
    seq = synth.with_volume(synth.room_sequence(n_frames=10, width=157, height=117, grid_dim=512, voxel_size=6e-3,
                                                block_capacity=1 << 16), **RULES[rule])
    vol = tsdf.Volume.from_params(seq.volume)
    ov = oracle.OracleVolume(seq.volume, seq.intr, amb_px=5e-4)
    for k in range(seq.n_frames):
        vol.fuse(_cuda(seq.depth[k]), seq.intr, seq.poses[k])
        ov.fuse(seq.depth[k], seq.poses[k])
    nb = seq.volume.grid_dim // 8
    ge, oe = vol.export(), ov.export()
    r = compare.compare_blocks(ge.coords, ge.alloc_frame, oe.coords, oe.alloc_frame, nb)
    assert r["keys_equal"] and r["frames_equal"], r
    _, _, gT, gP = compare.sort_by_key(ge.coords, ge.alloc_frame, ge.T, ge.P, nb)
    if RULES[rule]["update_rule"] == tsdf.UPDATE_AVERAGE:      # Alg. 1 keeps no second quantity
        gP, oP = np.ones_like(gP), np.ones_like(oe.P)
    else:
        oP = oe.P
        w, wmax = RULES[rule]["update_weight"], RULES[rule]["weight_max"]
        ok = ~np.isnan(gT)
        assert (gP[ok] >= w).all() and (gP[ok] <= wmax).all()
        assert (gP[ok] == wmax).mean() > 0.05           # the bound is reached
    v = compare.compare_values(gT, gP, oe.T, oP, oe.amb, seq.volume.truncation)
    assert v["ok"], json.dumps(v)
    assert v["compared"] > 100000, json.dumps(v)


@pytest.mark.parametrize("rule", list(RULES))
def test_update_rule_batched_equals_sequential(rule):
    seq = synth.with_volume(synth.sphere_sequence(n_frames=10), **RULES[rule])
    a = tsdf.Volume.from_params(seq.volume)
    for k in range(seq.n_frames):
        a.fuse(_cuda(seq.depth[k]), seq.intr, seq.poses[k])
    b = tsdf.Volume.from_params(seq.volume)
    for k0, K in ((0, 6), (6, 4)):
        b.integrate_batch([_cuda(seq.depth[k0 + j]) for j in range(K)], seq.intr, seq.poses[k0:k0 + K])
    ea, eb = a.export(), b.export()
    assert np.array_equal(ea.coords, eb.coords)
    chi = np.isnan(ea.T)
    assert np.array_equal(chi, np.isnan(eb.T))
    assert np.array_equal(ea.T.view(np.uint32)[~chi], eb.T.view(np.uint32)[~chi])
    assert np.array_equal(ea.P.view(np.uint32)[~chi], eb.P.view(np.uint32)[~chi])


def _plane_errors(seq, sig, at, **rule):
    """RMS error of T against the true distance (plane depth - voxel z) over the
    voxels within 2 voxels of the plane, after each frame listed in ``at``."""
    vol = tsdf.Volume.from_params(seq.volume, **rule)
    rms = []
    for k in range(seq.n_frames):
        var = _cuda(np.full(seq.depth[k].shape, sig[k] ** 2, np.float32))
        vol.fuse(_cuda(seq.depth[k]), seq.intr, seq.poses[k], var)
        if k not in at:
            continue
        e = vol.export()
        s = seq.volume.voxel_size
        z = seq.volume.origin[2] + (e.coords[:, 2:3] * 8 + (np.arange(512) >> 6)[None, :]) * s
        x = seq.volume.origin[0] + (e.coords[:, 0:1] * 8 + (np.arange(512) & 7)[None, :]) * s
        y = seq.volume.origin[1] + (e.coords[:, 1:2] * 8 + ((np.arange(512) >> 3) & 7)[None, :]) * s
        near = (np.abs(0.8 - z) <= 2 * s) & (np.abs(x / z) < 0.3) & (np.abs(y / z) < 0.2)
        truth = 0.8 - z
        d = (e.T - truth)[near & ~np.isnan(e.T)]
        rms.append(float(np.sqrt((d.astype(np.float64) ** 2).mean())))
    return np.array(rms)


def test_kalman_resists_data_of_growing_variance():
    """Static camera, plane at 0.8 m, deviation rising from 1 mm to 5 mm over 60
    frames (Kinect-like at 1-2 m). The three rules are tuned to the same steady
    smoothing at the first deviation: gain 0.1 (Kalman: Q = p/90; Alg. 1: w =
    0.1; Alg. 2: w = 1, W_max = 9)."""
    n = 60
    sig = synth.noise_ramp(n, 1e-3, 5e-3)
    seq = synth.plane_sequence(distance=0.8, n_frames=n, width=96, height=72, f=90.0, voxel_size=2e-3,
                               grid_dim=512, noise_sigma=1e-3, noise_sigma_end=5e-3, seed=31)
    seq = synth.with_volume(seq, truncation=0.02)
    p0 = float(sig[0] ** 2)
    at = set(range(20, 25)) | set(range(n - 10, n))
    kal = _plane_errors(seq, sig, at, process_variance=p0 / 90)
    avg = _plane_errors(seq, sig, at, update_rule=tsdf.UPDATE_AVERAGE, update_weight=0.1)
    wgt = _plane_errors(seq, sig, at, update_rule=tsdf.UPDATE_WEIGHTED, update_weight=1.0, weight_max=9.0)
    early, late = slice(0, 5), slice(5, 15)
    print(f"RMS error (mm), frames 20-24 / last 10: Kalman {1e3 * kal[early].mean():.3f} / "
          f"{1e3 * kal[late].mean():.3f}, Alg. 1 {1e3 * avg[early].mean():.3f} / {1e3 * avg[late].mean():.3f}, "
          f"Alg. 2 {1e3 * wgt[early].mean():.3f} / {1e3 * wgt[late].mean():.3f}")
    # similar smoothing while the data are good (deviation ~1.3-1.4 mm)
    assert abs(kal[early].mean() / avg[early].mean() - 1.0) < 0.5
    # once the data degrade the fixed weights let them in
    assert kal[late].mean() < 0.7 * avg[late].mean()
    assert kal[late].mean() < 0.7 * wgt[late].mean()
