"""Registration on the GPU (tsdf_icp, section "Registration") against the FP64
registration oracle: the Eq. 4 sums of one matching pass, the refined pose
of a known motion, and frame-to-model tracking of the noisy room sequence
through the library's own raycast maps."""
import numpy as np
import pytest
import torch

import pins
from oracle import icp as oicp
from paper_1311_7194_b300 import synth, tsdf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1311_7194_b300 import build
    build.build()
    torch.cuda.set_device(0)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _angle(Ra, Rb):
    return float(np.arccos(np.clip((np.trace(Ra @ Rb.T) - 1) / 2, -1, 1)))


def _case(W=320, H=240):
    intr, depth, model_pose, true_pose, mv, mn = pins._room_icp_case(W, H)
    seq = synth.room_sequence(n_frames=1, width=W, height=H, grid_dim=512, voxel_size=6e-3, block_capacity=1 << 12)
    vol = tsdf.Volume.from_params(seq.volume)
    return vol, intr, depth, model_pose, true_pose, mv, mn


def test_icp_sums_match_oracle():
    vol, intr, depth, model_pose, true_pose, mv, mn = _case()
    sums, box = vol.icp_sums(_cuda(depth), intr, _cuda(mv), _cuda(mn), model_pose, model_pose)
    p, q, n = oicp.match(depth, intr, model_pose, mv, mn, model_pose, oicp.IcpParams())
    A, g, rss, N = oicp.unscaled_sums(p, q, n)
    iu = np.triu_indices(6)
    ref = np.concatenate([A[iu], g, [rss, N]])
    # a few pairs at the rounding edge of a float32 decision may go either way
    assert abs(sums[28] - N) <= 1e-3 * N, (sums[28], N)
    scale = np.abs(ref).max(axis=None)
    big = np.abs(ref) > 1e-3 * scale
    assert np.abs(sums[big] / ref[big] - 1).max() < 5e-3, np.abs(sums[big] / ref[big] - 1).max()
    lo = np.minimum(p.min(0), q.min(0))
    hi = np.maximum(p.max(0), q.max(0))
    assert np.abs(box[:3] - lo).max() < 1e-4 and np.abs(box[3:] - hi).max() < 1e-4


def test_icp_recovers_a_known_motion():
    vol, intr, depth, model_pose, true_pose, mv, mn = _case()
    pose, res = vol.icp(_cuda(depth), intr, _cuda(mv), _cuda(mn), model_pose, model_pose, {"iterations": 12})
    opose, oinfo = oicp.icp(depth, intr, model_pose, mv, mn, model_pose, oicp.IcpParams(iterations=12))
    assert res["rank"] == 6 and res["matches"] > 40000, res
    assert np.linalg.norm(pose[:3, 3] - true_pose[:3, 3]) < 2e-4
    assert _angle(pose[:3, :3], true_pose[:3, :3]) < 2e-4
    # the same fixed point as the FP64 oracle
    assert np.linalg.norm(pose[:3, 3] - opose[:3, 3]) < 2e-5
    assert _angle(pose[:3, :3], opose[:3, :3]) < 2e-5
    assert abs(res["rms"] - oinfo["rms"]) < 0.05 * oinfo["rms"] + 1e-6


def test_icp_rejects_bad_arguments():
    vol, intr, depth, model_pose, _, mv, mn = _case(64, 48)
    for bad in ({"iterations": 0}, {"dist_max": -1.0}, {"normal_cos_min": 2.0}, {"eig_threshold": -0.1}):
        with pytest.raises(tsdf.TsdfError):
            vol.icp(_cuda(depth), intr, _cuda(mv), _cuda(mn), model_pose, model_pose, bad)


def test_icp_tracks_the_room_sequence():
    """Frame-to-model tracking: for each frame, raycast the model at the last
    estimated pose, register the frame (noisy, 2 % edge dropout) starting from
    that pose, and fuse it at the registered pose. Drift against the true
    trajectory stays within a few millimetres over 40 frames of a camera moving
    about 8 mm and 0.4 degrees per frame."""
    seq = synth.room_sequence(n_frames=40, width=320, height=240, grid_dim=1024, voxel_size=3e-3,
                              block_capacity=1 << 18, trajectory_frames=1200, device="cuda")
    vol = tsdf.Volume.from_params(seq.volume)
    d = torch.from_numpy(seq.depth).cuda()
    est = [seq.poses[0].copy()]
    vol.fuse(d[0], seq.intr, est[0])
    errs, angs = [], []
    for k in range(1, seq.n_frames):
        _, nrm, vtx = vol.raycast(seq.intr, est[-1])
        pose, res = vol.icp(d[k], seq.intr, vtx, nrm, est[-1], est[-1], {"iterations": 8})
        assert res["matches"] > 10000, (k, res)
        est.append(pose)
        vol.fuse(d[k], seq.intr, pose)
        errs.append(np.linalg.norm(pose[:3, 3] - seq.poses[k][:3, 3]))
        angs.append(_angle(pose[:3, :3], seq.poses[k][:3, :3]))
    step = np.median([np.linalg.norm(seq.poses[k][:3, 3] - seq.poses[k - 1][:3, 3]) for k in range(1, 40)])
    print(f"median true step {1e3 * step:.1f} mm; tracking error max {1e3 * max(errs):.2f} mm, "
          f"final {1e3 * errs[-1]:.2f} mm, max angle {np.rad2deg(max(angs)):.3f} deg")
    assert step > 5e-3                      # the camera really moves
    assert max(errs) < 0.01 and np.rad2deg(max(angs)) < 0.5
