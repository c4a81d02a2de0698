"""Comparison of the CUDA library's outputs with the oracle's (test infrastructure).

Works on plain numpy arrays; imports neither the CUDA package nor torch.

Tolerances (from the arithmetic; see the parity tests):
  * block sets and allocation frames: bit-exact;
  * T: |T_gpu - T_oracle| <= 1e-5 delta and identical chi patterns, on voxels the
    oracle does not flag as ambiguous (a pixel-rounding or truncation decision
    within float32 rounding distance of its boundary in some frame);
  * P: relative 1e-5 on the same voxels;
  * raycast: away from silhouettes, the same hit / miss decision and depth within
    0.1 voxel; vertex within 0.1 voxel along the ray; normals within a few
    degrees.
"""
from __future__ import annotations

import numpy as np


def block_keys(coords: np.ndarray, nb: int) -> np.ndarray:
    c = coords.astype(np.int64)
    return c[:, 0] + nb * (c[:, 1] + nb * c[:, 2])


def sort_by_key(coords, alloc_frame, T, P, nb):
    o = np.argsort(block_keys(coords, nb), kind="stable")
    return coords[o], alloc_frame[o], T[o], P[o]


def compare_blocks(g_coords, g_frames, o_coords, o_frames, nb) -> dict:
    gk, ok_ = block_keys(g_coords, nb), block_keys(o_coords, nb)
    go, oo = np.argsort(gk), np.argsort(ok_)
    gk, ok_ = gk[go], ok_[oo]
    res = {"n_gpu": int(gk.size), "n_oracle": int(ok_.size)}
    res["missing"] = int(np.setdiff1d(ok_, gk).size)
    res["extra"] = int(np.setdiff1d(gk, ok_).size)
    res["keys_equal"] = bool(gk.size == ok_.size and np.array_equal(gk, ok_))
    res["frames_equal"] = bool(res["keys_equal"] and np.array_equal(g_frames[go], o_frames[oo]))
    return res


def compare_values(gT, gP, oT, oP, amb, delta, tol_T=1e-5, tol_P=1e-5) -> dict:
    """gT, gP: float32 (n, 512) sorted like the oracle's; oT, oP: float64; amb: bool."""
    gT = gT.astype(np.float64).ravel()
    gP = gP.astype(np.float64).ravel()
    oT, oP, amb = oT.ravel(), oP.ravel(), amb.ravel()
    clear = ~amb
    g_chi, o_chi = np.isnan(gT), np.isnan(oT)
    chi_mismatch = int((clear & (g_chi != o_chi)).sum())
    both = clear & ~g_chi & ~o_chi
    dT = np.abs(gT[both] - oT[both])
    rP = np.abs(gP[both] / oP[both] - 1.0)
    return {
        "voxels": int(oT.size),
        "valid": int((~o_chi).sum()),
        "compared": int(both.sum()),
        "ambiguous": int(amb.sum()),
        "ambiguous_valid_frac": float((amb & ~o_chi).sum() / max(1, (~o_chi).sum())),
        "chi_mismatch": chi_mismatch,
        "max_dT_over_delta": float(dT.max() / delta) if dT.size else 0.0,
        "q999_dT_over_delta": float(np.quantile(dT, 0.999) / delta) if dT.size else 0.0,
        "max_rel_dP": float(rP.max()) if rP.size else 0.0,
        "ok": bool(chi_mismatch == 0 and (dT.size == 0 or dT.max() <= tol_T * delta)
                   and (rP.size == 0 or rP.max() <= tol_P)),
    }


def ray_dirs(intr, pose) -> np.ndarray:
    """Unit world ray directions (H, W, 3)."""
    v, u = np.meshgrid(np.arange(intr.height, dtype=np.float64), np.arange(intr.width, dtype=np.float64),
                       indexing="ij")
    dc = np.stack([(u - intr.cx) / intr.fx, (v - intr.cy) / intr.fy, np.ones_like(u)], -1)
    d = dc @ np.asarray(pose)[:3, :3].T
    return d / np.linalg.norm(d, axis=-1, keepdims=True)


def silhouette(o_depth, o_hit, o_normal, o_flags, dirs, delta, radius=2) -> np.ndarray:
    """Pixels near a silhouette of the oracle's raycast: a miss or a depth jump
    > 2 delta within ``radius`` px, a grazing ray (|n . ray| < 0.1), or an oracle
    bisection / gradient that met an undefined sample."""
    H, W = o_depth.shape
    z = np.where(o_hit, o_depth, np.nan)
    bad = np.zeros((H, W), bool)
    for dy in range(-radius, radius + 1):
        for dx in range(-radius, radius + 1):
            ys = slice(max(0, dy), H + min(0, dy))
            yd = slice(max(0, -dy), H + min(0, -dy))
            xs = slice(max(0, dx), W + min(0, dx))
            xd = slice(max(0, -dx), W + min(0, -dx))
            with np.errstate(invalid="ignore"):
                bad[yd, xd] |= np.isnan(z[ys, xs]) | (np.abs(z[ys, xs] - z[yd, xd]) > 2 * delta)
    # neighbours outside the image count as misses
    edge = np.ones((H, W), bool)
    edge[radius:H - radius, radius:W - radius] = False
    bad |= edge
    with np.errstate(invalid="ignore"):
        graze = np.abs((o_normal * dirs).sum(-1)) < 0.1
    bad |= o_hit & (graze | ~np.isfinite(o_normal[..., 0]))
    bad |= (o_flags & 2) > 0
    return bad & _dilate(o_hit, radius)


def _dilate(m, r):
    H, W = m.shape
    out = m.copy()
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            ys = slice(max(0, dy), H + min(0, dy))
            yd = slice(max(0, -dy), H + min(0, -dy))
            xs = slice(max(0, dx), W + min(0, dx))
            xd = slice(max(0, -dx), W + min(0, -dx))
            out[yd, xd] |= m[ys, xs]
    return out


def ray_points(intr, pose, depth) -> np.ndarray:
    """World points at camera depth ``depth`` (H, W) along every pixel's ray."""
    v, u = np.meshgrid(np.arange(intr.height, dtype=np.float64), np.arange(intr.width, dtype=np.float64),
                       indexing="ij")
    dc = np.stack([(u - intr.cx) / intr.fx, (v - intr.cy) / intr.fy, np.ones_like(u)], -1)
    pose = np.asarray(pose)
    return pose[:3, 3] + (depth[..., None] * dc) @ pose[:3, :3].T


def compare_raycast(g_depth, g_normal, g_vertex, o_depth, o_vertex, o_normal, o_flags, intr, pose,
                    voxel_size, delta, field_fn=None, tol_vox=0.1, tol_deg=5.0, tol_field=0.02) -> dict:
    """Raycast parity away from silhouettes.

    Where the oracle's first crossing is unique within one coarse step (flag 8
    clear), the GPU must agree on hit / miss, depth (tol_vox voxels), vertex and
    normal. Where it is not unique, several crossings are correct results of a
    march that samples every delta/2: the GPU may miss, and a GPU hit must be a
    true zero of the oracle's field (|f| <= tol_field voxels, evaluated with
    ``field_fn`` on world points) no nearer than the oracle's first crossing."""
    H, W = intr.height, intr.width
    o_depth = o_depth.reshape(H, W)
    o_vertex = o_vertex.reshape(H, W, 3)
    o_normal = o_normal.reshape(H, W, 3)
    o_flags = o_flags.reshape(H, W)
    o_hit = (o_flags & 1) > 0
    multi = (o_flags & 8) > 0
    g_hit = g_depth > 0
    dirs = ray_dirs(intr, pose)
    sil = silhouette(o_depth, o_hit, o_normal, o_flags, dirs, delta)
    clear = ~sil & ~multi
    hit_mismatch = int((clear & (g_hit != o_hit)).sum())
    both = clear & g_hit & o_hit
    dz = np.abs(g_depth[both] - o_depth[both]) / voxel_size
    dv = np.linalg.norm(g_vertex[both] - o_vertex[both], axis=-1) / voxel_size
    gn, on = g_normal[both], o_normal[both]
    okn = np.isfinite(gn[:, 0]) & np.isfinite(on[:, 0])
    ang = np.degrees(np.arccos(np.clip((gn[okn] * on[okn]).sum(-1), -1, 1)))
    res = {
        "pixels": H * W, "oracle_hits": int(o_hit.sum()), "gpu_hits": int(g_hit.sum()),
        "silhouette": int(sil.sum()), "compared": int(both.sum()), "hit_mismatch": hit_mismatch,
        "max_dz_vox": float(dz.max()) if dz.size else 0.0,
        "p99_dz_vox": float(np.percentile(dz, 99)) if dz.size else 0.0,
        "n_dz_over_tol": int((dz > tol_vox).sum()),
        "max_dvertex_vox": float(dv.max()) if dv.size else 0.0,
        "max_normal_deg": float(ang.max()) if ang.size else 0.0,
        "normal_undefined_mismatch": int((~okn).sum()),
    }
    ok = (hit_mismatch == 0 and res["max_dz_vox"] <= tol_vox and res["max_dvertex_vox"] <= tol_vox * 2.0
          and res["max_normal_deg"] <= tol_deg)
    amb = ~sil & multi & g_hit
    res["multi_crossing"] = int((~sil & multi).sum())
    res["multi_checked"] = int(amb.sum())
    if amb.any():
        if field_fn is None:
            ok = False
        else:
            pts = ray_points(intr, pose, np.where(amb, g_depth, 0.0))[amb]
            f = field_fn(pts) / voxel_size
            not_before = ~o_hit[amb] | (g_depth[amb] >= o_depth[amb] - tol_vox * voxel_size)
            bad = ~(np.abs(f) <= tol_field) | ~not_before
            res["multi_invalid"] = int(bad.sum())
            res["multi_max_field_vox"] = float(np.nanmax(np.abs(f))) if f.size else 0.0
            ok = ok and not bad.any()
    res["ok"] = bool(ok)
    return res
