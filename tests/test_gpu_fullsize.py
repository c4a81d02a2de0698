"""Full-size parity of the two other benchmark workloads, in the launch
configurations the benchmark times, on outputs the oracle computes one by one.

- High-resolution small object: 1280x1024, 4096^3 grid of 0.15 mm voxels, one
  CUDA graph per frame, T stored as float32, FP16 or snorm16. Sampled voxels
  against the oracle's per-voxel replay (Alg. 3 from each block's allocation
  frame on), and the float32 raycast maps at sampled pixels against the
  oracle's march over its own fused field.
- Batched + graphed: 640x480, 3000^3 grid of 1 mm voxels, K = 8 frames per
  graph launch (the per-voxel frame loop of the batched integrate). Sampled
  voxels against the replay, and the last batch's raycast maps at sampled
  pixels against the oracle's march.
Both sequences are shortened (the oracle fuses every allocated block of every
frame in FP64): 10 frames of the capsules' arc, the first 16 frames of the
batched workload's 1000-frame trajectory; images and grids keep their full
sizes.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import compare
from paper_1311_7194_b300 import synth, tsdf

pytestmark = pytest.mark.gpu

AMB_PX = 5e-4
HALF_STEP = {tsdf.STORAGE_SNORM16: 0.5 / 32767 * 1.001, tsdf.STORAGE_F16: 2.0 ** -11}
# the shape the autotuner picks for each workload on a B300 (results do not depend on it)
CAPSULE_SHAPE = dict(integrate_voxels_per_thread=8, integrate_ctas_per_sm=16, raycast_persistent=1)
BATCHED_SHAPE = dict(integrate_voxels_per_thread=4, integrate_ctas_per_sm=16, raycast_persistent=1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1311_7194_b300 import build
    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _capsules(n=10):
    return synth.capsule_sequence(n_frames=n, device="cuda", block_capacity=1 << 20)


def _batched(n=16):
    # the first n frames of the benchmark's 1000-frame trajectory
    return synth.room_sequence(seed=1, n_frames=n, trajectory_frames=1000, device="cuda", grid_dim=3000,
                               voxel_size=1e-3, block_capacity=1 << 21, origin=(0.0, -0.036, 0.0))


def _sampled_voxels(seq, n, seed):
    """n voxels drawn from the blocks the oracle allocates over the sequence,
    with their FP64 T and P replayed from their blocks' allocation frames."""
    ov = oracle.OracleVolume(seq.volume, seq.intr, store_values=False)
    for k in range(seq.n_frames):
        ov.allocate(seq.depth[k], seq.poses[k], k)
    oe = ov.export(values=False)
    rng = np.random.default_rng(seed)
    pick = rng.choice(oe.coords.shape[0], size=min(n, oe.coords.shape[0]), replace=False)
    local = rng.integers(0, 512, size=pick.size)
    vox = oe.coords[pick] * 8 + np.stack([local & 7, (local >> 3) & 7, local >> 6], -1)
    T, P, amb = oracle.replay_voxels(seq.volume, seq.intr, list(seq.depth), seq.poses, vox,
                                     oe.alloc_frame[pick], amb_px=AMB_PX)
    return oe, oe.coords[pick], local, T, P, amb


def _gpu_values(vol, coords, local, nb):
    ge = vol.export()
    keys = compare.block_keys(ge.coords, nb)
    order = np.argsort(keys)
    want = compare.block_keys(coords, nb)
    at = np.searchsorted(keys[order], want)
    assert np.all(at < keys.size) and np.array_equal(keys[order][at], want), "a sampled block is not allocated"
    slot = order[at]
    return ge, ge.T[slot, local].astype(np.float64), ge.P[slot, local].astype(np.float64)


def _raycast_parity(seq, ov, pose, maps, n, seed, min_both):
    """The bars of the room's full-size raycast test at n sampled pixels: the
    hit / miss pattern away from silhouettes and multiple crossings, depth
    within 0.1 voxel, vertex within 0.2 voxel, normals within 5 degrees; a hit
    among several crossings must be a zero of the oracle's field, not nearer
    than the oracle's first crossing."""
    gd, gn, gv = (t.cpu().numpy() for t in maps)
    H, W = seq.intr.height, seq.intr.width
    s, delta = seq.volume.voxel_size, seq.volume.truncation
    rng = np.random.default_rng(seed)
    # half of the pixels uniform over the image, half among the GPU's hits (a
    # small object leaves most of the image empty)
    seen = np.argwhere(gd[2:H - 2, 2:W - 2] > 0) + 2
    hits = seen[rng.choice(seen.shape[0], size=min(n // 2, seen.shape[0]), replace=False)]
    cv = np.concatenate([rng.integers(2, H - 2, n - n // 2), hits[:, 0]])
    cu = np.concatenate([rng.integers(2, W - 2, n - n // 2), hits[:, 1]])
    n = cu.size
    dy, dx = np.meshgrid(np.arange(-2, 3), np.arange(-2, 3), indexing="ij")
    pu, pv = cu[:, None, None] + dx, cv[:, None, None] + dy
    od, ovx, onr, ofl = ov.raycast(pose, uv=np.stack([pu.ravel(), pv.ravel()], -1))
    od, ovx, onr, ofl = od.reshape(n, 5, 5), ovx.reshape(n, 5, 5, 3), onr.reshape(n, 5, 5, 3), ofl.reshape(n, 5, 5)
    dirs = compare.ray_dirs(seq.intr, pose)
    sil = np.array([compare.silhouette(od[i], (ofl[i] & 1) > 0, onr[i], ofl[i], dirs[pv[i], pu[i]], delta)[2, 2]
                    for i in range(n)])
    o_hit, multi = (ofl[:, 2, 2] & 1) > 0, (ofl[:, 2, 2] & 8) > 0
    o_d, o_v, o_n = od[:, 2, 2], ovx[:, 2, 2], onr[:, 2, 2]
    g_d, g_v, g_n = gd[cv, cu], gv[cv, cu], gn[cv, cu]
    g_hit = g_d > 0
    clear = ~sil & ~multi
    assert not np.any(clear & (g_hit != o_hit)), "hit / miss differs away from silhouettes"
    both = clear & g_hit & o_hit
    assert both.sum() >= min_both, int(both.sum())
    dz = np.abs(g_d[both] - o_d[both]) / s
    dv = np.linalg.norm(g_v[both] - o_v[both], axis=-1) / s
    cosang = np.clip((g_n[both] * o_n[both]).sum(-1), -1.0, 1.0)
    assert dz.max() <= 0.1, float(dz.max())
    assert dv.max() <= 0.2, float(dv.max())
    assert np.degrees(np.arccos(cosang)).max() <= 5.0
    amb = ~sil & multi & g_hit
    if amb.any():
        dc = np.stack([(cu[amb] - seq.intr.cx) / seq.intr.fx, (cv[amb] - seq.intr.cy) / seq.intr.fy,
                       np.ones(int(amb.sum()))], -1)
        P = np.asarray(pose)
        pts = P[:3, 3] + (g_d[amb][:, None] * dc) @ P[:3, :3].T
        f = ov.field(pts) / s
        assert np.all(np.abs(f) <= 0.02), float(np.nanmax(np.abs(f)))
        assert np.all(~o_hit[amb] | (g_d[amb] >= o_d[amb] - 0.1 * s))


@pytest.mark.parametrize("storage", [tsdf.STORAGE_F32, tsdf.STORAGE_F16, tsdf.STORAGE_SNORM16],
                         ids=["f32", "f16", "snorm16"])
def test_capsules_fullsize_sampled_voxels(storage):
    from paper_1311_7194_b300.pipeline import FusionPipeline
    seq = _capsules()
    vol = tsdf.Volume.from_params(seq.volume, storage=storage)
    vol.set_launch_config(**CAPSULE_SHAPE)
    pipe = FusionPipeline(vol, seq.intr, graph=True)
    for k in range(seq.n_frames):
        pipe.step(torch.from_numpy(seq.depth[k]).cuda(), seq.poses[k])
    vol.check()
    oe, coords, local, T, P, amb = _sampled_voxels(seq, 4000, seed=21)
    nb = seq.volume.grid_dim // 8
    ge, gT, gP = _gpu_values(vol, coords, local, nb)
    assert ge.coords.shape[0] == oe.coords.shape[0], "block counts differ"
    delta = seq.volume.truncation
    tol = 1e-5 if storage == tsdf.STORAGE_F32 else seq.n_frames * HALF_STEP[storage] + 1e-5
    v = compare.compare_values(gT[:, None], gP[:, None], T[:, None], P[:, None], amb[:, None], delta, tol_T=tol)
    assert v["ok"], v
    assert v["compared"] > 300, v
    pipe.graph.close()
    vol.close()


def test_capsules_fullsize_sampled_raycast():
    from paper_1311_7194_b300.pipeline import FusionPipeline
    seq = _capsules()
    vol = tsdf.Volume.from_params(seq.volume)
    vol.set_launch_config(**CAPSULE_SHAPE)
    pipe = FusionPipeline(vol, seq.intr, graph=True)
    ov = oracle.OracleVolume(seq.volume, seq.intr, amb_px=AMB_PX)
    for k in range(seq.n_frames):
        pipe.step(torch.from_numpy(seq.depth[k]).cuda(), seq.poses[k])
        ov.fuse(seq.depth[k], seq.poses[k])
    vol.check()
    _raycast_parity(seq, ov, seq.poses[-1], pipe.maps, n=1200, seed=23, min_both=300)
    pipe.graph.close()
    vol.close()


def test_batched_fullsize_sampled_voxels_and_raycast():
    K = 8
    seq = _batched()
    H, W = seq.intr.height, seq.intr.width
    vol = tsdf.Volume.from_params(seq.volume)
    vol.set_launch_config(**BATCHED_SHAPE)
    g = tsdf.Graph(vol, seq.intr, K)
    dev = torch.device("cuda", 0)
    maps = (torch.empty((H, W), device=dev), torch.empty((H, W, 3), device=dev), torch.empty((H, W, 3), device=dev))
    d = [torch.from_numpy(x).cuda() for x in seq.depth]
    for k in range(0, seq.n_frames, K):
        g.launch(d[k:k + K], seq.poses[k:k + K], maps)
    torch.cuda.synchronize()
    vol.check()
    oe, coords, local, T, P, amb = _sampled_voxels(seq, 4000, seed=25)
    nb = seq.volume.grid_dim // 8
    ge, gT, gP = _gpu_values(vol, coords, local, nb)
    assert ge.coords.shape[0] == oe.coords.shape[0], "block counts differ"
    v = compare.compare_values(gT[:, None], gP[:, None], T[:, None], P[:, None], amb[:, None],
                               seq.volume.truncation)
    assert v["ok"], v
    assert v["compared"] > 300, v
    # the last launch's raycast, at the batch's last pose
    ov = oracle.OracleVolume(seq.volume, seq.intr, amb_px=AMB_PX)
    for k in range(seq.n_frames):
        ov.fuse(seq.depth[k], seq.poses[k])
    _raycast_parity(seq, ov, seq.poses[-1], maps, n=1200, seed=27, min_both=300)
    g.close()
    vol.close()
