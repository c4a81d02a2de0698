"""CPU oracle for the point-to-plane registration step (section "Registration",
Eqs. 2-8). TEST INFRASTRUCTURE ONLY: plain FP64 numpy, written from the paper,
sharing nothing with the CUDA library; only the tests, the package's smoke check
and the benchmark's CPU legs use it.

What it follows:
  * Chen-Medioni point-to-plane ICP with projective matching and rejection by
    distance and by normal deviation (section "Registration", first paragraph).
  * Eq. 2: minimise sum(((R p_i + t - q_i) . n_i)^2); Eq. 3: small-angle R with
    r = (alpha, beta, gamma); Eq. 4: the 6x6 normal equations with c_i = p_i x n_i.
  * Eqs. 5-7: the problem restated in the box of the points shrunk to the unit
    cube: p^ = S^-1 (p - m), c^ = S^-1 (c - m x n).
  * Eq. 8: the solution kept only along eigenvectors of the scaled matrix whose
    eigenvalue per pair exceeds theta.

Readings (where the paper is silent or at odds with itself):
  * Points: the frame's pixel u with depth D back-projects to X = D K^-1 (u, 1)
    in its camera and to p = R X + t in the world with the current pose
    estimate; p is matched to the model pixel nearest to its projection into the
    model camera (floor(x + 1/2) per axis), whose vertex is q and normal n.
  * Measurements: a frame depth outside [depth_min, depth_max] (the volume's
    sensor range) is no measurement, as for integration.
  * Frame normals: the cross product of the central differences of the
    back-projected neighbours, (X(u+1) - X(u-1)) x (X(v+1) - X(v-1)), normalised
    and turned to face the camera; a pixel with an invalid 4-neighbour has none.
  * Rejection: the pair is dropped when |p - q| > dist_max or when the frame's
    world normal and n have a dot product below cos_min.
  * Scaling: m is the centre and S the diagonal of the side lengths of the
    axis-aligned box of all matched p and q. Substituting c = S c^ + m x n into
    the residual (p - q).n + r.c + t.n gives (p - q).n + (S r).c^ + (t + r x m).n,
    so the scaled unknowns are r^ = S r and t^ = t + r x m, and the solution is
    recovered as r = S^-1 r^, t = t^ - r x m. (The printed recovery,
    r = S r^ and t = t^ + r x m, does not follow from the printed substitution.)
  * Eq. 8 with a singular matrix: x^' = sum over kept eigenpairs of
    v_i (v_i . b^) / lambda_i, which equals the printed projection of the solution
    whenever the matrix is invertible.
  * Pose update: p -> exp([r]x) p + t, applied on the left of the current pose
    (the small-angle matrix of Eq. 3 is the first-order form of exp([r]x)).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np


@dataclass
class IcpParams:
    dist_max: float = 0.05
    cos_min: float = 0.8
    theta: float = 0.005
    iterations: int = 10
    depth_min: float = 0.1      # a depth outside [depth_min, depth_max] is no measurement,
    depth_max: float = 4.0      # as for integration


def _backproject(depth, intr, prm: IcpParams):
    H, W = depth.shape
    v, u = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    d = depth.astype(np.float64)
    X = np.stack([(u - intr.cx) / intr.fx * d, (v - intr.cy) / intr.fy * d, d], -1)
    with np.errstate(invalid="ignore"):
        ok = np.isfinite(d) & (d > 0) & (d >= prm.depth_min) & (d <= prm.depth_max)
    return X, ok


def frame_normals(depth, intr, prm: IcpParams):
    """Camera-frame unit normals of a depth map (H, W, 3) and their validity."""
    X, ok = _backproject(depth, intr, prm)
    H, W = depth.shape
    n = np.full((H, W, 3), np.nan)
    val = np.zeros((H, W), bool)
    dx = X[1:-1, 2:] - X[1:-1, :-2]
    dy = X[2:, 1:-1] - X[:-2, 1:-1]
    c = np.cross(dx, dy)
    good = ok[1:-1, 2:] & ok[1:-1, :-2] & ok[2:, 1:-1] & ok[:-2, 1:-1] & ok[1:-1, 1:-1]
    norm = np.linalg.norm(c, axis=-1)
    good &= norm > 0
    c = c / np.where(norm > 0, norm, 1.0)[..., None]
    flip = (c * X[1:-1, 1:-1]).sum(-1) > 0
    c = np.where(flip[..., None], -c, c)
    n[1:-1, 1:-1] = np.where(good[..., None], c, np.nan)
    val[1:-1, 1:-1] = good
    return n, val


def match(depth, intr, pose, model_vertex, model_normal, model_pose, prm: IcpParams):
    """Matched pairs (p, q, n) in world coordinates (each (N, 3))."""
    X, ok = _backproject(depth, intr, prm)
    nf, okn = frame_normals(depth, intr, prm)
    R, t = pose[:3, :3], pose[:3, 3]
    p = X @ R.T + t
    ns = nf @ R.T
    Rm, tm = model_pose[:3, :3], model_pose[:3, 3]
    xm = (p - tm) @ Rm                       # R_m^T (p - t_m), row vectors
    H, W = depth.shape
    with np.errstate(invalid="ignore", divide="ignore"):
        um = np.floor(intr.fx * xm[..., 0] / xm[..., 2] + intr.cx + 0.5)
        vm = np.floor(intr.fy * xm[..., 1] / xm[..., 2] + intr.cy + 0.5)
    sel = ok & okn & (xm[..., 2] > 0) & (um >= 0) & (um < W) & (vm >= 0) & (vm < H)
    ui = np.where(sel, um, 0).astype(np.int64)
    vi = np.where(sel, vm, 0).astype(np.int64)
    q = model_vertex[vi, ui].astype(np.float64)
    n = model_normal[vi, ui].astype(np.float64)
    sel &= np.isfinite(q).all(-1) & np.isfinite(n).all(-1)
    with np.errstate(invalid="ignore"):
        sel &= np.linalg.norm(p - q, axis=-1) <= prm.dist_max
        sel &= (ns * n).sum(-1) >= prm.cos_min
    return p[sel], q[sel], n[sel]


def unscaled_sums(p, q, n):
    """Eq. 4 sums: A = sum J J^T, g = sum J r with J = (p x n, n), r = (p - q).n;
    also sum r^2 and the count."""
    c = np.cross(p, n)
    J = np.concatenate([c, n], 1)
    r = ((p - q) * n).sum(1)
    return J.T @ J, J.T @ r, float((r * r).sum()), int(p.shape[0])


def box(p, q):
    pts = np.concatenate([p, q], 0)
    lo, hi = pts.min(0), pts.max(0)
    return 0.5 * (lo + hi), np.maximum(hi - lo, 1e-9)


def scaled_system(p, q, n):
    """Eqs. 5-7: C = sum J^ J^T with J^ = (c^, n), c^ = S^-1 (c - m x n), and
    b^ = -sum J^ ((p - q).n); also m and the diagonal of S."""
    m, S = box(p, q)
    c_hat = (np.cross(p, n) - np.cross(m[None, :], n)) / S[None, :]
    J = np.concatenate([c_hat, n], 1)
    r = ((p - q) * n).sum(1)
    return J.T @ J, -(J.T @ r), m, S


def solve(C, b, N, theta):
    """Eq. 8: the solution restricted to eigen-directions with lambda / N > theta."""
    lam, V = np.linalg.eigh(C)
    keep = lam / max(N, 1) > theta
    x = V[:, keep] @ ((V[:, keep].T @ b) / lam[keep])
    return x, int(keep.sum())


def rotation(r):
    """exp([r]x) by Rodrigues' formula."""
    a = float(np.linalg.norm(r))
    if a < 1e-300:
        return np.eye(3)
    k = r / a
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + np.sin(a) * K + (1 - np.cos(a)) * (K @ K)


def step(depth, intr, pose, model_vertex, model_normal, model_pose, prm: IcpParams):
    """One ICP iteration: returns (new pose, info)."""
    p, q, n = match(depth, intr, pose, model_vertex, model_normal, model_pose, prm)
    N = p.shape[0]
    if N < 6:
        return pose.copy(), {"matches": N, "rank": 0, "rms": float("nan")}
    C, b, m, S = scaled_system(p, q, n)
    x, rank = solve(C, b, N, prm.theta)
    r = x[:3] / S
    t = x[3:] - np.cross(r, m)
    inc = np.eye(4)
    inc[:3, :3] = rotation(r)
    inc[:3, 3] = t
    rr = ((p - q) * n).sum(1)
    return inc @ pose, {"matches": N, "rank": rank, "rms": float(np.sqrt((rr * rr).mean())), "r": r, "t": t}


def icp(depth, intr, pose0, model_vertex, model_normal, model_pose, prm: Optional[IcpParams] = None):
    """prm.iterations ICP iterations from pose0; returns (pose, info of the last)."""
    prm = prm or IcpParams()
    pose = np.asarray(pose0, np.float64).copy()
    info = {}
    for _ in range(prm.iterations):
        pose, info = step(depth, intr, pose, model_vertex, model_normal, model_pose, prm)
    return pose, info
