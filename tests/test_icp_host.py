"""The host half of tsdf_icp (tsdf_icp_solve: unit-cube restatement built from
the plain Eq. 4 sums, Jacobi eigen-decomposition, the Eq. 8 test and the motion
recovery), run on the CPU, against the registration oracle, which forms the
scaled system point by point and decomposes it with numpy."""
import numpy as np
import pytest

import pins
from oracle import icp as oicp
from paper_1311_7194_b300 import synth, tsdf


def _sums(p, q, n):
    A, g, rss, N = oicp.unscaled_sums(p, q, n)
    iu = np.triu_indices(6)
    box = np.concatenate([np.minimum(p.min(0), q.min(0)), np.maximum(p.max(0), q.max(0))]).astype(np.float32)
    return np.concatenate([A[iu], g, [rss, N]]), box


def _oracle_motion(p, q, n, box, theta):
    # the oracle's scaled system, with the box rounded to float as the library receives it
    lo, hi = box[:3].astype(np.float64), box[3:].astype(np.float64)
    m, S = 0.5 * (lo + hi), np.maximum(hi - lo, 1e-9)
    c_hat = (np.cross(p, n) - np.cross(m[None, :], n)) / S[None, :]
    J = np.concatenate([c_hat, n], 1)
    r = ((p - q) * n).sum(1)
    x, rank = oicp.solve(J.T @ J, -(J.T @ r), p.shape[0], theta)
    rr = x[:3] / S
    return rr, x[3:] - np.cross(rr, m), rank


@pytest.mark.parametrize("case", ["room", "plane", "room_theta0"])
def test_host_solve_matches_oracle(case):
    tsdf.load()
    if case == "plane":
        scene = synth.Scene(ground_plane=True)
        intr = synth.Intrinsics.centred(105.0, 160, 120)
        pose = synth.look_at((0.2, 1.2, -0.4), (0.0, 0.0, 0.6))
        _, mv, mn = synth.render_maps(scene, intr, pose)
        depth = synth.render_depth(scene, intr, pins._small_motion(pose, 0.5, (1, 0, 0), (0, 0.004, 0))).numpy()
        mv, mn = mv.numpy(), mn.numpy()
    else:
        intr, depth, pose, _, mv, mn = pins._room_icp_case()
    depth = np.where(np.isfinite(depth), depth, 0).astype(np.float32)
    theta = 0.0 if case == "room_theta0" else 0.005
    p, q, n = oicp.match(depth, intr, pose, mv, mn, pose, oicp.IcpParams())
    sums, box = _sums(p, q, n)
    r, t, rank = tsdf.icp_solve(sums, box, theta)
    ro, to, ranko = _oracle_motion(p, q, n, box, theta)
    assert rank == ranko == (3 if case == "plane" else 6)
    scale = max(np.abs(ro).max(), np.abs(to).max())
    assert scale > 1e-4
    assert np.allclose(r, ro, rtol=0, atol=1e-8 * scale + 1e-15), (r, ro)
    assert np.allclose(t, to, rtol=0, atol=1e-8 * scale + 1e-15), (t, to)


def test_host_solve_rejects_bad_arguments():
    tsdf.load()
    with pytest.raises(tsdf.TsdfError):
        tsdf.icp_solve(np.zeros(29), np.zeros(6), -1.0)
