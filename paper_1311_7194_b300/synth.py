"""Seeded synthetic depth-map sequences: the inputs that both the CUDA path and the
CPU oracle are fed.

The paper's captured scans (Artec Spider / Eva hand and mannequin scans, the ASUS
Xtion test scene) are not available, so analytic scenes stand in for them: depth
maps are produced by exact ray casting of spheres, oriented boxes, capsules and a
ground plane, then perturbed with a noise model whose deviation grows
quadratically with depth (the sensor model described in the Introduction and in
the Kalman section, Alg. 3), plus edge-pixel dropout.

This module holds none of the fusion method's arithmetic (no TSDF, no
allocation, no Kalman update, no raycast of a voxel field): it only draws scenes,
trajectories and noisy depth maps. Every random number comes from a NumPy
``default_rng`` seeded per scene and per frame, so a sequence is reproducible
from its name, seed and sizes. Ray casting runs in float64 on the requested torch
device; the same arrays are then handed to both implementations under test.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np
import torch


# ----------------------------------------------------------------------------
# camera, volume and scene descriptions
# ----------------------------------------------------------------------------

@dataclass(frozen=True)
class Intrinsics:
    """Pinhole camera, OpenCV axes (x right, y down, z forward).

    A pixel (u, v) has its centre at integer coordinates; unstated principal
    points use cx = (W-1)/2, cy = (H-1)/2."""
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    @staticmethod
    def centred(f: float, width: int, height: int) -> "Intrinsics":
        return Intrinsics(float(f), float(f), (width - 1) / 2.0, (height - 1) / 2.0,
                          int(width), int(height))


@dataclass(frozen=True)
class VolumeParams:
    """Sparse TSDF volume settings (section "Volumetric Scene Representation").

    ``grid_dim`` voxels per axis, voxel i sampled at origin + i * voxel_size,
    blocks of 8^3 voxels, ``block_capacity`` blocks in the pool."""
    voxel_size: float
    truncation: float
    origin: tuple
    grid_dim: int
    block_capacity: int
    depth_min: float
    depth_max: float
    raycast_near: float
    raycast_far: float
    sigma_coeff: float          # sensor deviation sigma = sigma_coeff * z^2
    process_variance: float = 0.0
    update_rule: int = 0        # 0 Alg. 3 (Kalman), 1 Alg. 1 (running average), 2 Alg. 2 (weighted)
    update_weight: float = 0.1  # w_k of Alg. 1 / Alg. 2
    weight_max: float = 1.0     # W_max of Alg. 2
    refine_steps: int = 0       # Gauss-Newton steps refining T_k in the depth map (0 = off)


@dataclass
class Scene:
    spheres: np.ndarray = field(default_factory=lambda: np.zeros((0, 4)))    # cx cy cz r
    boxes: np.ndarray = field(default_factory=lambda: np.zeros((0, 7)))      # cx cy cz hx hy hz yaw
    capsules: np.ndarray = field(default_factory=lambda: np.zeros((0, 7)))   # ax ay az bx by bz r
    ground_plane: bool = False                                                 # plane y = 0, +y outside
    plane_z: Optional[float] = None    # world plane z = plane_z facing -z (camera tests)


@dataclass
class Sequence:
    """A posed depth-map sequence plus the volume it is fused into."""
    name: str
    seed: int
    intr: Intrinsics
    volume: VolumeParams
    scene: Scene
    poses: np.ndarray            # (F, 4, 4) float64, camera -> world
    depth: np.ndarray            # (F, H, W) float32, 0 = no measurement
    clean_depth: Optional[np.ndarray] = None   # (F, H, W) float64 noise-free, inf = no hit

    @property
    def n_frames(self) -> int:
        return int(self.poses.shape[0])


# ----------------------------------------------------------------------------
# poses and trajectories
# ----------------------------------------------------------------------------

def look_at(eye, target, up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """Camera -> world pose of a camera at ``eye`` looking at ``target``.

    OpenCV camera axes: z forward, y down, x = y cross z (right)."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, np.asarray(up, np.float64))
    nx = np.linalg.norm(x)
    if nx < 1e-6:
        x = np.cross(z, np.array([0.0, 0.0, 1.0]))
        nx = np.linalg.norm(x)
    x /= nx
    y = np.cross(z, x)
    T = np.eye(4)
    T[:3, 0], T[:3, 1], T[:3, 2], T[:3, 3] = x, y, z, eye
    return T


def catmull_rom_closed(points: np.ndarray, n: int) -> np.ndarray:
    """n samples, uniform in parameter, of the closed uniform Catmull-Rom spline
    through ``points`` (m, 3)."""
    m = points.shape[0]
    out = np.empty((n, 3))
    for i in range(n):
        s = i * m / n
        k = int(math.floor(s))
        t = s - k
        p0, p1, p2, p3 = (points[(k + j - 1) % m] for j in range(4))
        t2, t3 = t * t, t * t * t
        out[i] = 0.5 * ((2 * p1) + (-p0 + p2) * t + (2 * p0 - 5 * p1 + 4 * p2 - p3) * t2
                        + (-p0 + 3 * p1 - 3 * p2 + p3) * t3)
    return out


# ----------------------------------------------------------------------------
# analytic ray casting (float64, torch, any device)
# ----------------------------------------------------------------------------

def _pixel_rays(intr: Intrinsics, pose: np.ndarray, device) -> tuple:
    T = torch.as_tensor(pose, dtype=torch.float64, device=device)
    v, u = torch.meshgrid(torch.arange(intr.height, dtype=torch.float64, device=device),
                          torch.arange(intr.width, dtype=torch.float64, device=device),
                          indexing="ij")
    dc = torch.stack([(u - intr.cx) / intr.fx, (v - intr.cy) / intr.fy, torch.ones_like(u)], -1)
    dw = dc @ T[:3, :3].T          # (H, W, 3), camera z component of dc is 1
    o = T[:3, 3]
    return o, dw


def _hit_sphere(o, d, c, r):
    oc = o - c
    A = (d * d).sum(-1)
    B = (d * oc).sum(-1)           # half of the linear coefficient
    C = (oc * oc).sum() - r * r
    disc = B * B - A * C
    sq = torch.sqrt(torch.clamp(disc, min=0.0))
    t0 = (-B - sq) / A
    t1 = (-B + sq) / A
    t = torch.where(t0 > 0, t0, t1)
    return torch.where((disc >= 0) & (t > 0), t, torch.full_like(t, math.inf))


def _hit_box(o, d, box):
    cx, cy, cz, hx, hy, hz, yaw = (float(b) for b in box)
    cyaw, syaw = math.cos(yaw), math.sin(yaw)
    # world -> box local: rotate by -yaw around y after translating
    ox, oy, oz = (o[0] - cx), (o[1] - cy), (o[2] - cz)
    lox = cyaw * ox - syaw * oz
    loz = syaw * ox + cyaw * oz
    ldx = cyaw * d[..., 0] - syaw * d[..., 2]
    ldz = syaw * d[..., 0] + cyaw * d[..., 2]
    ldy = d[..., 1]
    tn = torch.full_like(ldx, -math.inf)
    tf = torch.full_like(ldx, math.inf)
    for lo, ld, h in ((lox, ldx, hx), (oy, ldy, hy), (loz, ldz, hz)):
        inv = 1.0 / ld                       # +-inf for axis-parallel rays is fine
        ta = (-h - lo) * inv
        tb = (h - lo) * inv
        ta, tb = torch.minimum(ta, tb), torch.maximum(ta, tb)
        ta = torch.nan_to_num(ta, nan=-math.inf)
        tb = torch.nan_to_num(tb, nan=math.inf)
        tn = torch.maximum(tn, ta)
        tf = torch.minimum(tf, tb)
    t = torch.where(tn > 0, tn, tf)
    return torch.where((tn <= tf) & (t > 0), t, torch.full_like(t, math.inf))


def _hit_capsule(o, d, cap):
    a = torch.as_tensor(cap[:3], dtype=torch.float64, device=d.device)
    b = torch.as_tensor(cap[3:6], dtype=torch.float64, device=d.device)
    r = float(cap[6])
    ba = b - a
    oa = o - a
    baba = float((ba * ba).sum())
    bard = (d * ba).sum(-1)
    baoa = float((ba * oa).sum())
    rdoa = (d * oa).sum(-1)
    oaoa = float((oa * oa).sum())
    dd = (d * d).sum(-1)
    A = baba * dd - bard * bard
    B = baba * rdoa - baoa * bard
    C = baba * oaoa - baoa * baoa - r * r * baba
    h = B * B - A * C
    sq = torch.sqrt(torch.clamp(h, min=0.0))
    t_cyl = (-B - sq) / A
    y = baoa + t_cyl * bard
    cyl_ok = (h >= 0) & (A.abs() > 1e-300) & (y > 0) & (y < baba) & (t_cyl > 0)
    t = torch.where(cyl_ok, t_cyl, torch.full_like(t_cyl, math.inf))
    t = torch.minimum(t, _hit_sphere(o, d, a, r))
    t = torch.minimum(t, _hit_sphere(o, d, b, r))
    return t


def render_depth(scene: Scene, intr: Intrinsics, pose: np.ndarray, device="cpu") -> torch.Tensor:
    """Exact camera-z depth of the nearest scene surface per pixel (inf = no hit)."""
    o, d = _pixel_rays(intr, pose, device)
    best = torch.full(d.shape[:2], math.inf, dtype=torch.float64, device=device)
    for s in scene.spheres:
        c = torch.as_tensor(s[:3], dtype=torch.float64, device=device)
        best = torch.minimum(best, _hit_sphere(o, d, c, float(s[3])))
    for b in scene.boxes:
        best = torch.minimum(best, _hit_box(o, d, b))
    for cp in scene.capsules:
        best = torch.minimum(best, _hit_capsule(o, d, cp))
    if scene.ground_plane:
        t = -o[1] / d[..., 1]
        best = torch.minimum(best, torch.where((d[..., 1] < 0) & (t > 0), t,
                                               torch.full_like(t, math.inf)))
    if scene.plane_z is not None:
        t = (scene.plane_z - o[2]) / d[..., 2]
        best = torch.minimum(best, torch.where(t > 0, t, torch.full_like(t, math.inf)))
    return best


def render_maps(scene: Scene, intr: Intrinsics, pose: np.ndarray, device="cpu"):
    """Exact model maps of the scene seen from ``pose``: camera-z depth (H, W),
    world vertex and world unit normal (H, W, 3), NaN where the ray misses. The
    normal is the gradient of the analytic signed distance (central differences
    of 1e-6 m), turned to face the camera: the maps a perfect raycast of the
    scene would return."""
    z = render_depth(scene, intr, pose, device)
    o, d = _pixel_rays(intr, pose, device)
    hit = torch.isfinite(z)
    vert = o + z[..., None] * d
    eps = 1e-6
    g = torch.zeros_like(vert)
    for a in range(3):
        e = torch.zeros(3, dtype=torch.float64, device=device)
        e[a] = eps
        g[..., a] = (scene_sdf(scene, vert + e) - scene_sdf(scene, vert - e)) / (2 * eps)
    n = g / g.norm(dim=-1, keepdim=True)
    n = torch.where(((n * d).sum(-1, keepdim=True) > 0), -n, n)
    nan = torch.full_like(vert, math.nan)
    vert = torch.where(hit[..., None], vert, nan)
    n = torch.where(hit[..., None] & torch.isfinite(n), n, nan)
    return z, vert, n


def scene_sdf(scene: Scene, p: torch.Tensor) -> torch.Tensor:
    """Analytic signed distance of the scene union at world points p (..., 3);
    positive outside. Used as ground truth when measuring surface error."""
    p = p.to(torch.float64)
    best = torch.full(p.shape[:-1], math.inf, dtype=torch.float64, device=p.device)
    for s in scene.spheres:
        c = torch.as_tensor(s[:3], dtype=torch.float64, device=p.device)
        best = torch.minimum(best, (p - c).norm(dim=-1) - float(s[3]))
    for b in scene.boxes:
        cx, cy, cz, hx, hy, hz, yaw = (float(v) for v in b)
        x, y, z = p[..., 0] - cx, p[..., 1] - cy, p[..., 2] - cz
        lx = math.cos(yaw) * x - math.sin(yaw) * z
        lz = math.sin(yaw) * x + math.cos(yaw) * z
        q = torch.stack([lx.abs() - hx, y.abs() - hy, lz.abs() - hz], -1)
        outside = q.clamp(min=0).norm(dim=-1)
        inside = q.max(dim=-1).values.clamp(max=0)
        best = torch.minimum(best, outside + inside)
    for cp in scene.capsules:
        a = torch.as_tensor(cp[:3], dtype=torch.float64, device=p.device)
        b = torch.as_tensor(cp[3:6], dtype=torch.float64, device=p.device)
        pa, ba = p - a, b - a
        h = ((pa * ba).sum(-1) / (ba * ba).sum()).clamp(0, 1)
        best = torch.minimum(best, (pa - h[..., None] * ba).norm(dim=-1) - float(cp[6]))
    if scene.ground_plane:
        best = torch.minimum(best, p[..., 1])
    if scene.plane_z is not None:
        best = torch.minimum(best, scene.plane_z - p[..., 2])
    return best


# ----------------------------------------------------------------------------
# sensor model
# ----------------------------------------------------------------------------

def _edge_band(clean: np.ndarray, jump: float, radius: int = 2) -> np.ndarray:
    """Pixels within ``radius`` px (Chebyshev) of a 4-neighbour depth jump > ``jump``
    (a neighbour with no surface counts as a jump)."""
    z = np.where(np.isfinite(clean), clean, 1e30)
    j = np.zeros(z.shape, bool)
    dx = np.abs(np.diff(z, axis=1)) > jump
    dy = np.abs(np.diff(z, axis=0)) > jump
    j[:, :-1] |= dx
    j[:, 1:] |= dx
    j[:-1, :] |= dy
    j[1:, :] |= dy
    out = np.zeros_like(j)
    H, W = j.shape
    for oy in range(-radius, radius + 1):
        for ox in range(-radius, radius + 1):
            ys, yd = (slice(max(0, -oy), H - max(0, oy)), slice(max(0, oy), H - max(0, -oy)))
            xs, xd = (slice(max(0, -ox), W - max(0, ox)), slice(max(0, ox), W - max(0, -ox)))
            out[yd, xd] |= j[ys, xs]
    return out


def incidence_cos(clean: np.ndarray, intr: Intrinsics) -> np.ndarray:
    """|cos| between each pixel's ray and the surface normal of the exact depth
    map (central differences of back-projected points; 1 where undefined)."""
    H, W = clean.shape
    v, u = np.meshgrid(np.arange(H, dtype=np.float64), np.arange(W, dtype=np.float64), indexing="ij")
    z = np.where(np.isfinite(clean), clean, np.nan)
    P = np.stack([z * (u - intr.cx) / intr.fx, z * (v - intr.cy) / intr.fy, z], -1)
    a = np.full_like(P, np.nan)
    b = np.full_like(P, np.nan)
    a[:, 1:-1] = P[:, 2:] - P[:, :-2]
    b[1:-1, :] = P[2:, :] - P[:-2, :]
    n = np.cross(a, b)
    with np.errstate(invalid="ignore", divide="ignore"):
        c = np.abs((n * P).sum(-1)) / (np.linalg.norm(n, axis=-1) * np.linalg.norm(P, axis=-1))
    return np.where(np.isfinite(c), c, 1.0)


def sense(clean: np.ndarray, vol: VolumeParams, rng: np.random.Generator,
          noise: bool = True, dropout_frac: float = 0.0, jump: float = 0.0, intr: Optional[Intrinsics] = None,
          edge_gain: float = 0.0, angle_gain: float = 0.0) -> np.ndarray:
    """Noisy float32 depth from exact depth: z + N(0, sigma^2), out-of-range -> 0,
    and ``dropout_frac`` of the valid pixels dropped from the edge band.

    sigma = a z^2 (the quadratic sensor), multiplied by (1 + edge_gain) inside the
    edge band and by (1 + angle_gain (1 - |cos|)) with the incidence cosine, when
    those gains are set (a sensor that is also poorer near edges and at grazing
    angles)."""
    z = clean.copy()
    finite = np.isfinite(z)
    if noise:
        n = rng.standard_normal(z.shape)
        zf = np.where(finite, z, 0.0)
        sigma = vol.sigma_coeff * zf * zf
        if edge_gain:
            sigma = sigma * np.where(_edge_band(clean, jump), 1.0 + edge_gain, 1.0)
        if angle_gain and intr is not None:
            sigma = sigma * (1.0 + angle_gain * (1.0 - incidence_cos(clean, intr)))
        z = np.where(finite, zf + sigma * n, z)
    ok = np.isfinite(z) & (z >= vol.depth_min) & (z <= vol.depth_max)
    out = np.where(ok, z, 0.0).astype(np.float32)
    if dropout_frac > 0:
        band = np.flatnonzero((_edge_band(clean, jump) & ok).ravel())
        n_drop = min(band.size, int(round(dropout_frac * ok.sum())))
        if n_drop > 0:
            out.ravel()[rng.choice(band, size=n_drop, replace=False)] = 0.0
    return out


def _render_all(scene, intr, poses, vol, seed, device, noise, dropout_frac, keep_clean, edge_gain=0.0,
                angle_gain=0.0):
    F = poses.shape[0]
    depth = np.empty((F, intr.height, intr.width), np.float32)
    clean_all = np.empty((F, intr.height, intr.width)) if keep_clean else None
    for f in range(F):
        clean = render_depth(scene, intr, poses[f], device).cpu().numpy()
        rng = np.random.default_rng([seed, f, 7])
        depth[f] = sense(clean, vol, rng, noise=noise, dropout_frac=dropout_frac,
                         jump=2.0 * vol.truncation, intr=intr, edge_gain=edge_gain, angle_gain=angle_gain)
        if keep_clean:
            clean_all[f] = clean
    return depth, clean_all


# ----------------------------------------------------------------------------
# the workloads
# ----------------------------------------------------------------------------

def sphere_sequence(seed: int = 0, n_frames: int = 10, width: int = 160, height: int = 120,
                    f: float = 140.0, noise: bool = True, grid_dim: int = 256,
                    voxel_size: float = 1e-3, device="cpu", keep_clean: bool = False) -> Sequence:
    """Analytic sphere r = 0.1 m, camera on a 30 degree arc of radius 0.5 m around
    its centre (raised 10 degrees above its equator), 160x120, fx = fy = 140, sigma = 1.5e-3 z^2, 256^3 grid of 1 mm voxels,
    truncation 5 voxels, pool of 8192 blocks."""
    rng = np.random.default_rng(seed)
    centre = np.zeros(3)
    scene = Scene(spheres=np.array([[0.0, 0.0, 0.0, 0.1]]))
    th0 = rng.uniform(0, 2 * math.pi)
    ths = th0 + np.linspace(0.0, math.radians(30.0), n_frames)
    el = math.radians(10.0)     # arc raised 10 degrees so no pose is a symmetric matrix
    poses = np.stack([look_at(centre + 0.5 * np.array([math.cos(el) * math.cos(t), math.sin(el),
                                                        math.cos(el) * math.sin(t)]), centre)
                      for t in ths])
    half = grid_dim // 2
    vol = VolumeParams(voxel_size=voxel_size, truncation=5 * voxel_size,
                       origin=tuple(float(c - half * voxel_size) for c in centre),
                       grid_dim=grid_dim, block_capacity=8192, depth_min=0.05,
                       depth_max=1.0, raycast_near=0.05, raycast_far=1.0, sigma_coeff=1.5e-3)
    intr = Intrinsics.centred(f, width, height)
    depth, clean = _render_all(scene, intr, poses, vol, seed, device, noise, 0.0, keep_clean)
    return Sequence("sphere", seed, intr, vol, scene, poses, depth, clean)


def room_scene(seed: int) -> Scene:
    """Ground plane y = 0 plus 50 seeded primitives (spheres and yawed boxes, half and
    half, sizes U(0.05, 0.5) m) resting on it inside the 3 m cube."""
    rng = np.random.default_rng([seed, 1000])
    spheres, boxes = [], []
    for i in range(50):
        x, z = rng.uniform(0.25, 2.75, size=2)
        if i % 2 == 0:
            r = 0.5 * rng.uniform(0.05, 0.5)
            spheres.append([x, r, z, r])
        else:
            hx, hy, hz = 0.5 * rng.uniform(0.05, 0.5, size=3)
            boxes.append([x, hy, z, hx, hy, hz, rng.uniform(0, math.pi)])
    return Scene(spheres=np.array(spheres), boxes=np.array(boxes), ground_plane=True)


def room_trajectory(seed: int, n_frames: int) -> np.ndarray:
    """Camera poses on a closed Catmull-Rom spline through 8 seeded control points at
    1-2 m height, looking at targets interpolated through 8 seeded points near the floor."""
    rng = np.random.default_rng([seed, 2000])
    ctrl = np.column_stack([rng.uniform(0.5, 2.5, 8), rng.uniform(1.0, 2.0, 8), rng.uniform(0.5, 2.5, 8)])
    tgt = np.column_stack([rng.uniform(0.75, 2.25, 8), rng.uniform(0.0, 0.5, 8), rng.uniform(0.75, 2.25, 8)])
    eyes = catmull_rom_closed(ctrl, n_frames)
    targets = catmull_rom_closed(tgt, n_frames)
    return np.stack([look_at(e, t) for e, t in zip(eyes, targets)])


def room_sequence(seed: int = 1, n_frames: int = 300, width: int = 640, height: int = 480,
                  f: float = 525.0, grid_dim: int = 2048, voxel_size: float = 1.5e-3,
                  block_capacity: int = 1 << 20, noise: bool = True, dropout: float = 0.02,
                  device="cpu", keep_clean: bool = False, origin=None, edge_gain: float = 0.0,
                  angle_gain: float = 0.0, sigma_coeff: float = 1.5e-3,
                  trajectory_frames: Optional[int] = None) -> Sequence:
    """Room-scale workload: ground plane + 50 primitives in a 3 m cube, 640x480,
    fx = fy = 525, 300 frames on a seeded spline, sigma = 1.5e-3 z^2, 2 % edge
    dropout, depth range [0.3, 4] m, 2048^3 grid of 1.5 mm voxels (truncation
    5 voxels), pool of 2^20 blocks. Smaller sizes give the reduced parity cases.
    ``edge_gain`` / ``angle_gain`` select a sensor that is also noisier near depth
    edges and at grazing incidence (the learned-variance workload).
    ``trajectory_frames`` > n_frames spreads the closed spline over that many
    frames and renders the first n_frames (a slower camera)."""
    scene = room_scene(seed)
    poses = room_trajectory(seed, max(n_frames, trajectory_frames or n_frames))[:n_frames]
    if origin is None:
        origin = (-0.036, -0.036, -0.036)
    vol = VolumeParams(voxel_size=voxel_size, truncation=5 * voxel_size, origin=tuple(origin),
                       grid_dim=grid_dim, block_capacity=block_capacity, depth_min=0.3,
                       depth_max=4.0, raycast_near=0.3, raycast_far=4.0, sigma_coeff=sigma_coeff)
    intr = Intrinsics(f * width / 640.0, f * width / 640.0, (width - 1) / 2.0, (height - 1) / 2.0,
                      width, height)
    depth, clean = _render_all(scene, intr, poses, vol, seed, device, noise, dropout, keep_clean, edge_gain,
                               angle_gain)
    return Sequence("room", seed, intr, vol, scene, poses, depth, clean)


def capsule_sequence(seed: int = 2, n_frames: int = 200, width: int = 1280, height: int = 1024,
                     f: float = 1400.0, grid_dim: int = 4096, voxel_size: float = 1.5e-4,
                     block_capacity: int = 1 << 21, noise: bool = True, device="cpu",
                     keep_clean: bool = False) -> Sequence:
    """High-resolution small object: union of 20 seeded capsules (radius 5-12 mm,
    length 20-60 mm) inside a 12 cm ball seen from 0.3 m, 1280x1024, fx = fy = 1400,
    sigma = 2e-4 z^2, 4096^3 grid of 0.15 mm voxels."""
    rng = np.random.default_rng([seed, 3000])
    caps = []
    for _ in range(20):
        c = rng.standard_normal(3)
        c *= 0.06 * rng.uniform() ** (1 / 3) / np.linalg.norm(c)
        a = rng.standard_normal(3)
        a /= np.linalg.norm(a)
        L = rng.uniform(0.02, 0.06)
        caps.append([*(c - 0.5 * L * a), *(c + 0.5 * L * a), rng.uniform(0.005, 0.012)])
    scene = Scene(capsules=np.array(caps))
    th0 = rng.uniform(0, 2 * math.pi)
    poses = []
    for i in range(n_frames):
        t = i / max(1, n_frames - 1)
        th = th0 + math.radians(90.0) * t
        ph = math.radians(20.0) * math.sin(2 * math.pi * t)
        eye = 0.3 * np.array([math.cos(ph) * math.cos(th), math.sin(ph), math.cos(ph) * math.sin(th)])
        poses.append(look_at(eye, np.zeros(3)))
    poses = np.stack(poses)
    half = grid_dim // 2
    vol = VolumeParams(voxel_size=voxel_size, truncation=5 * voxel_size,
                       origin=(-half * voxel_size,) * 3, grid_dim=grid_dim,
                       block_capacity=block_capacity, depth_min=0.1, depth_max=0.6,
                       raycast_near=0.1, raycast_far=0.6, sigma_coeff=2e-4)
    intr = Intrinsics(f * width / 1280.0, f * width / 1280.0, (width - 1) / 2.0, (height - 1) / 2.0,
                      width, height)
    depth, clean = _render_all(scene, intr, poses, vol, seed, device, noise, 0.0, keep_clean)
    return Sequence("capsules", seed, intr, vol, scene, poses, depth, clean)


def noise_ramp(n_frames: int, sigma0: float, sigma1: Optional[float]) -> np.ndarray:
    """Per-frame deviations rising linearly from sigma0 (first frame) to sigma1
    (last frame); constant sigma0 when sigma1 is None."""
    if sigma1 is None or n_frames < 2:
        return np.full(n_frames, float(sigma0))
    return sigma0 + (sigma1 - sigma0) * np.arange(n_frames) / (n_frames - 1)


def plane_sequence(distance: float = 0.5, n_frames: int = 4, width: int = 64, height: int = 48,
                   f: float = 60.0, voxel_size: float = 2e-3, grid_dim: int = 256,
                   noise_sigma: float = 0.0, seed: int = 5, static: bool = True,
                   offset=(0.0, 0.0, 0.0), noise_sigma_end: Optional[float] = None) -> Sequence:
    """Fronto-parallel plane z = ``distance`` in front of a camera at the world origin
    looking down +z. With ``static`` every frame has the identity pose; otherwise the
    camera slides sideways. Per-pixel Gaussian noise of deviation ``noise_sigma``,
    or rising linearly to ``noise_sigma_end`` over the frames (``noise_ramp``)."""
    scene = Scene(plane_z=distance)
    poses = []
    for i in range(n_frames):
        T = np.eye(4)
        T[:3, 3] = np.asarray(offset, np.float64)
        if not static:
            T[0, 3] += 0.01 * i
        poses.append(T)
    poses = np.stack(poses)
    vol = VolumeParams(voxel_size=voxel_size, truncation=5 * voxel_size,
                       origin=(-0.5 * grid_dim * voxel_size, -0.5 * grid_dim * voxel_size, 0.0),
                       grid_dim=grid_dim, block_capacity=8192, depth_min=0.01, depth_max=10.0,
                       raycast_near=0.01, raycast_far=10.0, sigma_coeff=0.0)
    intr = Intrinsics.centred(f, width, height)
    depth = np.empty((n_frames, height, width), np.float32)
    sig = noise_ramp(n_frames, noise_sigma, noise_sigma_end)
    for i in range(n_frames):
        clean = render_depth(scene, intr, poses[i]).numpy()
        rng = np.random.default_rng([seed, i])
        z = clean + (sig[i] * rng.standard_normal(clean.shape) if sig[i] > 0 else 0.0)
        depth[i] = np.where(np.isfinite(z) & (z > 0), z, 0.0).astype(np.float32)
    return Sequence("plane", seed, intr, vol, scene, poses, depth, None)


def with_volume(seq: Sequence, **kw) -> Sequence:
    """Copy of ``seq`` with some volume settings replaced."""
    return replace(seq, volume=replace(seq.volume, **kw))
