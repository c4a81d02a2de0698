"""Pins for the CPU oracle: checks against facts fixed by the paper and by
mathematics, independent of the oracle's own code.

Each ``pin_*`` function raises AssertionError when the oracle (optionally a
variant library at ``lib_path``) disagrees with the fact it pins. They are run by
``test_oracle_pins.py`` on the real oracle and by ``test_oracle_mutations.py`` on
copies of the oracle with planted mistakes, which each must break at least one pin.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

import oracle
from paper_1311_7194_b300 import synth


# ----------------------------------------------------------------------------
# fixtures built from plain geometry
# ----------------------------------------------------------------------------

def _plane_volume(s=2e-3, G=64, z_centre=0.5, Q=0.0, sigma=0.0, cap=4096):
    return synth.VolumeParams(voxel_size=s, truncation=5 * s,
                              origin=(-G / 2 * s, -G / 2 * s, z_centre - G / 2 * s), grid_dim=G,
                              block_capacity=cap, depth_min=0.05, depth_max=5.0,
                              raycast_near=0.05, raycast_far=5.0, sigma_coeff=sigma,
                              process_variance=Q)


def _voxel_world(vol, coords):
    """World positions of voxel indices (n, 3) (voxel i sits at origin + i s)."""
    s = float(np.float32(vol.voxel_size))
    return np.asarray(vol.origin)[None, :] + coords.astype(np.float64) * s


def _fuse(ov, depths, poses, vars_=None):
    for k in range(len(depths)):
        ov.fuse(depths[k], poses[k], None if vars_ is None else vars_[k])


def _const_frames(n, seed, H=24, W=32, equal_var=False, d0=0.5, spread=2e-3):
    rng = np.random.default_rng(seed)
    D = (d0 + rng.uniform(-spread, spread, n)).astype(np.float32)
    p = (np.full(n, 1e-6) if equal_var else rng.uniform(0.5e-6, 2e-6, n)).astype(np.float32)
    depths = [np.full((H, W), D[k], np.float32) for k in range(n)]
    vars_ = [np.full((H, W), p[k], np.float32) for k in range(n)]
    return D.astype(np.float64), p.astype(np.float64), depths, vars_


# ----------------------------------------------------------------------------
# Alg. 3 and Eq. 9 closed forms
# ----------------------------------------------------------------------------

def _rule_volume(rule, w, wmax):
    from dataclasses import replace
    return replace(_plane_volume(), update_rule=rule, update_weight=w, weight_max=wmax)


def _rule_run(rule, w, wmax, n, seed, lib_path):
    """Static camera, fronto-parallel plane at depth D_k in frame k: every voxel's
    T_k = D_k - z exactly. Returns (T_k matrix, export, valid-in-all mask,
    valid-in-some mask)."""
    vol = _rule_volume(rule, w, wmax)
    intr = synth.Intrinsics.centred(30.0, 32, 24)
    D, p, depths, vars_ = _const_frames(n, seed=seed, spread=4e-3)
    ov = oracle.OracleVolume(vol, intr, lib_path=lib_path)
    _fuse(ov, depths, [np.eye(4)] * n, vars_)
    e = ov.export()
    xyz = _voxel_world(vol, oracle.voxel_coords(e))
    Tk = D[None, :] - xyz[:, 2:3]
    delta = vol.truncation
    valid = np.abs(Tk) < delta * (1 - 1e-6)
    clear = (valid | (np.abs(Tk) > delta * (1 + 1e-6))).all(1) & np.repeat(e.alloc_frame == 0, 512)
    return Tk, e, valid, clear


def pin_alg1_running_average(lib_path=None):
    """Alg. 1 with a fixed weight w is an exponential moving average: unrolling
    T_n = (1 - w) T_{n-1} + w T_k(n) from T_1 = T_k(1) gives
    T_N = (1 - w)^(N-1) T_k(1) + sum_{n=2..N} w (1 - w)^(N-n) T_k(n), over the
    frames in which the voxel is inside the band (the first of them sets T)."""
    w, n = 0.375, 8            # weights exactly representable in float32, as the library holds them
    Tk, e, valid, clear = _rule_run(1, w, 1.0, n, 21, lib_path)
    T = e.T.ravel()
    checked = 0
    for m in (valid.all(1) & clear, valid.any(1) & ~valid.all(1) & clear):
        rows = np.nonzero(m)[0]
        exp = np.empty(rows.size)
        for i, r in enumerate(rows):
            seq = Tk[r][valid[r]]
            N = seq.size
            coef = np.array([(1 - w) ** (N - 1)] + [w * (1 - w) ** (N - k) for k in range(2, N + 1)])
            exp[i] = (coef * seq).sum()
        assert np.allclose(T[rows], exp, rtol=0, atol=1e-12), np.abs(T[rows] - exp).max()
        checked += rows.size
    assert checked > 5000, checked
    none = (~valid).all(1) & clear
    assert none.sum() > 1000 and np.isnan(T[none]).all()


def pin_alg2_weighted_average(lib_path=None):
    """Alg. 2 with a constant weight w: while W + w stays under W_max the result
    is the plain mean of the measurements and W = (count) w; once W is held at
    W_max the update becomes T <- a T + (1 - a) T_k with a = W_max / (W_max + w).
    With W_max = 2.5 w the first three measurements are averaged, and every later
    one enters with the geometric weight (1 - a) a^(N-n)."""
    w, n = 0.25, 8             # w and W_max exactly representable in float32
    Tk, e, valid, clear = _rule_run(2, w, 1e6, n, 22, lib_path)        # W_max never reached
    m = valid.all(1) & clear
    assert m.sum() > 5000
    assert np.allclose(e.T.ravel()[m], Tk[m].mean(1), rtol=0, atol=1e-12)
    assert np.allclose(e.P.ravel()[m], n * w, rtol=1e-12, atol=0)
    part = valid.any(1) & ~valid.all(1) & clear
    assert part.sum() > 1000
    cnt = valid[part].sum(1)
    assert np.allclose(e.T.ravel()[part], (Tk[part] * valid[part]).sum(1) / cnt, rtol=0, atol=1e-12)
    assert np.allclose(e.P.ravel()[part], cnt * w, rtol=1e-12, atol=0)
    Tk, e, valid, clear = _rule_run(2, w, 2.5 * w, n, 23, lib_path)    # W_max reached at the third
    m = valid.all(1) & clear
    a = 2.5 / 3.5
    exp = a ** (n - 3) * Tk[m][:, :3].mean(1) + sum((1 - a) * a ** (n - k) * Tk[m][:, k - 1] for k in range(4, n + 1))
    assert np.allclose(e.T.ravel()[m], exp, rtol=0, atol=1e-12), np.abs(e.T.ravel()[m] - exp).max()
    assert np.allclose(e.P.ravel()[m], 2.5 * w, rtol=1e-12, atol=0)


def pin_kalman_closed_form(lib_path=None):
    """With Q = 0, Alg. 3 fed measurements T_k of variances p_k ends at the
    inverse-variance weighted mean: T = sum(T_k/p_k)/sum(1/p_k), P = 1/sum(1/p_k)
    (induction on the update). A static camera sees a fronto-parallel plane at a
    different depth D_k each frame, so every voxel's T_k = D_k - z exactly."""
    vol = _plane_volume()
    intr = synth.Intrinsics.centred(30.0, 32, 24)
    n = 9
    D, p, depths, vars_ = _const_frames(n, seed=11)
    ov = oracle.OracleVolume(vol, intr, lib_path=lib_path)
    _fuse(ov, depths, [np.eye(4)] * n, vars_)
    e = ov.export()
    xyz = _voxel_world(vol, oracle.voxel_coords(e))
    Tk = D[None, :] - xyz[:, 2:3]                           # (voxels, frames)
    delta = vol.truncation
    all_valid = (np.abs(Tk) < delta * (1 - 1e-6)).all(1)
    none_valid = (np.abs(Tk) > delta * (1 + 1e-6)).all(1)
    first0 = np.repeat(e.alloc_frame == 0, 512)
    T, P = e.T.ravel(), e.P.ravel()
    m = all_valid & first0
    assert m.sum() > 5000, m.sum()
    w = 1.0 / p
    T_exp = (Tk[m] * w).sum(1) / w.sum()
    P_exp = 1.0 / w.sum()
    assert np.allclose(T[m], T_exp, rtol=0, atol=1e-12), np.abs(T[m] - T_exp).max()
    assert np.allclose(P[m], P_exp, rtol=1e-12, atol=0), np.abs(P[m] / P_exp - 1).max()
    assert none_valid.sum() > 1000
    assert np.isnan(T[none_valid]).all(), "voxels never within delta must stay chi"
    # voxels inside the truncation band in some frames only: the weighted mean runs
    # over exactly the frames whose |T_k| <= delta
    valid = np.abs(Tk) < delta * (1 - 1e-6)
    clear = ((np.abs(Tk) < delta * (1 - 1e-6)) | (np.abs(Tk) > delta * (1 + 1e-6))).all(1)
    part = valid.any(1) & ~valid.all(1) & clear & first0
    assert part.sum() > 1000, part.sum()
    wv = np.where(valid[part], w[None, :], 0.0)
    assert np.allclose(T[part], (Tk[part] * wv).sum(1) / wv.sum(1), rtol=0, atol=1e-12)
    assert np.allclose(P[part], 1.0 / wv.sum(1), rtol=1e-12, atol=0)


def pin_eq9_mean(lib_path=None):
    """Eq. 9: N measurements of equal variance sigma^2 give their arithmetic mean
    with variance sigma^2 / N."""
    vol = _plane_volume()
    intr = synth.Intrinsics.centred(30.0, 32, 24)
    n = 7
    D, p, depths, vars_ = _const_frames(n, seed=12, equal_var=True)
    ov = oracle.OracleVolume(vol, intr, lib_path=lib_path)
    _fuse(ov, depths, [np.eye(4)] * n, vars_)
    e = ov.export()
    xyz = _voxel_world(vol, oracle.voxel_coords(e))
    Tk = D[None, :] - xyz[:, 2:3]
    m = (np.abs(Tk) < vol.truncation * (1 - 1e-6)).all(1) & np.repeat(e.alloc_frame == 0, 512)
    assert m.sum() > 5000
    assert np.allclose(e.T.ravel()[m], Tk[m].mean(1), rtol=0, atol=1e-12)
    assert np.allclose(e.P.ravel()[m], p[0] / n, rtol=1e-12, atol=0)


def pin_process_variance_steady_state(lib_path=None):
    """With process variance Q > 0 and a constant measurement variance p, the
    posterior variance of Alg. 3 converges to the fixed point of
    P = (P+Q) p / (P+Q+p), i.e. P = (-Q + sqrt(Q^2 + 4 Q p)) / 2."""
    Q, pv = 2e-7, 1e-6
    vol = _plane_volume(Q=Q)
    intr = synth.Intrinsics.centred(30.0, 32, 24)
    n = 80
    depths = [np.full((24, 32), 0.5, np.float32)] * n
    vars_ = [np.full((24, 32), pv, np.float32)] * n
    ov = oracle.OracleVolume(vol, intr, lib_path=lib_path)
    _fuse(ov, depths, [np.eye(4)] * n, vars_)
    e = ov.export()
    xyz = _voxel_world(vol, oracle.voxel_coords(e))
    Tk = 0.5 - xyz[:, 2]
    m = (np.abs(Tk) < vol.truncation * (1 - 1e-6)) & np.repeat(e.alloc_frame == 0, 512)
    assert m.sum() > 5000
    p32 = float(np.float32(pv))
    Q32 = float(np.float32(Q))
    P_inf = (-Q32 + math.sqrt(Q32 * Q32 + 4 * Q32 * p32)) / 2
    assert np.allclose(e.P.ravel()[m], P_inf, rtol=1e-9, atol=0), np.abs(e.P.ravel()[m] / P_inf - 1).max()
    assert np.allclose(e.T.ravel()[m], Tk[m], rtol=0, atol=1e-13)


def pin_first_measurement_and_quadratic_variance(lib_path=None):
    """One frame into an empty volume: T = T_k and P = p_k (first branch of
    Alg. 3), with the default variance p_k = (a D^2)^2 of a sensor whose deviation
    grows quadratically with depth (Introduction; Alg. 3 text); voxels with
    |T_k| > delta hold chi (Eq. 1)."""
    a = 1.5e-3
    vol = _plane_volume(sigma=a)
    intr = synth.Intrinsics.centred(30.0, 32, 24)
    D = np.float32(0.5031)
    ov = oracle.OracleVolume(vol, intr, lib_path=lib_path)
    ov.fuse(np.full((24, 32), D, np.float32), np.eye(4), None)
    e = ov.export()
    z = _voxel_world(vol, oracle.voxel_coords(e))[:, 2]
    Tk = float(D) - z
    T, P = e.T.ravel(), e.P.ravel()
    valid = np.abs(Tk) < vol.truncation * (1 - 1e-6)
    invalid = np.abs(Tk) > vol.truncation * (1 + 1e-6)
    assert np.allclose(T[valid], Tk[valid], rtol=0, atol=1e-15)
    p_exp = (float(np.float32(a)) * float(D) ** 2) ** 2
    assert np.allclose(P[valid], p_exp, rtol=1e-14, atol=0)
    assert np.isnan(T[invalid]).all()


# ----------------------------------------------------------------------------
# projective measurement T_k (Fusion, last paragraph)
# ----------------------------------------------------------------------------

def pin_projection_nearest_pixel(lib_path=None):
    """A voxel reads the pixel nearest to its projection: the depth map encodes
    each pixel's index, so T + z_c recovers which pixel a voxel used; that pixel's
    centre must lie within half a pixel of the voxel's projection, computed here
    with the inverse pose from numpy.linalg.inv."""
    rng = np.random.default_rng(21)
    W, H, f = 40, 30, 36.0
    intr = synth.Intrinsics(f, f * 1.1, 19.3, 14.8, W, H)
    ang = rng.uniform(-0.3, 0.3, 3)
    cx_, sx_ = math.cos(ang[0]), math.sin(ang[0])
    cy_, sy_ = math.cos(ang[1]), math.sin(ang[1])
    cz_, sz_ = math.cos(ang[2]), math.sin(ang[2])
    Rx = np.array([[1, 0, 0], [0, cx_, -sx_], [0, sx_, cx_]])
    Ry = np.array([[cy_, 0, sy_], [0, 1, 0], [-sy_, 0, cy_]])
    Rz = np.array([[cz_, -sz_, 0], [sz_, cz_, 0], [0, 0, 1]])
    pose = np.eye(4)
    pose[:3, :3] = Rz @ Ry @ Rx
    pose[:3, 3] = rng.uniform(-0.2, 0.2, 3)
    centre = pose[:3, :3] @ np.array([0.0, 0.0, 1.0]) + pose[:3, 3]
    s, G = 2e-3, 64
    vol = synth.VolumeParams(voxel_size=s, truncation=5 * s, origin=tuple(centre - G / 2 * s),
                             grid_dim=G, block_capacity=4096, depth_min=0.05, depth_max=5.0,
                             raycast_near=0.05, raycast_far=5.0, sigma_coeff=1e-3)
    idx = np.arange(W * H).reshape(H, W)
    depth = (1.0 + 1e-5 * idx).astype(np.float32)
    ov = oracle.OracleVolume(vol, intr, lib_path=lib_path, amb_px=1e-9)
    ov.fuse(depth, pose)
    e = ov.export()
    vox = oracle.voxel_coords(e)
    T = e.T.ravel()
    ok = ~np.isnan(T)
    assert ok.sum() > 2000, ok.sum()
    Xw = _voxel_world(vol, vox[ok])
    inv = np.linalg.inv(pose)
    Xc = Xw @ inv[:3, :3].T + inv[:3, 3]
    Dread = T[ok] + Xc[:, 2]
    k = np.rint((Dread - 1.0) / 1e-5).astype(np.int64)
    u_read, v_read = k % W, k // W
    assert np.abs(Dread - depth.ravel()[k]).max() < 1e-9
    uf = intr.fx * Xc[:, 0] / Xc[:, 2] + intr.cx
    vf = intr.fy * Xc[:, 1] / Xc[:, 2] + intr.cy
    assert np.abs(uf - u_read).max() <= 0.5 + 1e-9, np.abs(uf - u_read).max()
    assert np.abs(vf - v_read).max() <= 0.5 + 1e-9, np.abs(vf - v_read).max()
    # every voxel whose projection falls inside the image and whose read depth is
    # within delta must have been updated (no valid measurement is skipped)
    Xw_all = _voxel_world(vol, vox)
    Xc_all = Xw_all @ inv[:3, :3].T + inv[:3, 3]
    ua = np.floor(intr.fx * Xc_all[:, 0] / Xc_all[:, 2] + intr.cx + 0.5)
    va = np.floor(intr.fy * Xc_all[:, 1] / Xc_all[:, 2] + intr.cy + 0.5)
    inside = (ua >= 0) & (ua < W) & (va >= 0) & (va < H) & (Xc_all[:, 2] > 0)
    kk = np.where(inside, va * W + ua, 0).astype(np.int64)
    Tk = depth.ravel()[kk].astype(np.float64) - Xc_all[:, 2]
    want = inside & (np.abs(Tk) < vol.truncation * (1 - 1e-6)) & ~e.amb.ravel()
    assert (ok | ~want).all(), "a voxel with a valid measurement was left chi"


# ----------------------------------------------------------------------------
# allocation (section "Updating Sparse Structure")
# ----------------------------------------------------------------------------

def pin_alloc_exact_rational(lib_path=None):
    """The allocated blocks are the blocks holding the surface samples: each valid
    pixel's ray sampled at D + m delta / J, m = -J..J. Here every sample is placed
    with exact rational arithmetic (fractions) from the same inputs; a block
    decision may differ from single precision only for samples within 1e-2 voxel
    of a block or grid boundary."""
    rng = np.random.default_rng(31)
    W, H = 9, 7
    intr = synth.Intrinsics(7.0, 7.5, 4.2, 2.9, W, H)
    s, G = 4e-3, 64
    vol = synth.VolumeParams(voxel_size=s, truncation=5 * s, origin=(-0.13, -0.12, 0.2), grid_dim=G,
                             block_capacity=100000, depth_min=0.05, depth_max=5.0,
                             raycast_near=0.05, raycast_far=5.0, sigma_coeff=1e-3)
    pose = synth.look_at(rng.uniform(-0.05, 0.05, 3), np.array([0.0, 0.0, 0.33]), up=(0.1, 1.0, 0.05))
    depth = rng.uniform(0.25, 0.45, (H, W)).astype(np.float32)
    depth[0, 0] = 0.0
    depth[1, 2] = np.nan
    ov = oracle.OracleVolume(vol, intr, lib_path=lib_path)
    keys = set(int(k) for k in ov.frame_blocks(depth, pose))
    J = ov.half_samples
    assert J == 10, J
    nb = G // 8
    sF, dF = Fraction(float(np.float32(s))), Fraction(float(np.float32(5 * s)))
    org = [Fraction(o) for o in vol.origin]
    R = [[Fraction(float(pose[r, c])) for c in range(3)] for r in range(3)]
    t = [Fraction(float(pose[r, 3])) for r in range(3)]
    sure, maybe = set(), set()
    eps = Fraction(1, 100)
    for j in range(H):
        for i in range(W):
            d = float(depth[j, i])
            if not (d > 0 and math.isfinite(d)):
                continue
            xn = (i - Fraction(float(np.float32(intr.cx)))) / Fraction(float(np.float32(intr.fx)))
            yn = (j - Fraction(float(np.float32(intr.cy)))) / Fraction(float(np.float32(intr.fy)))
            for m in range(-J, J + 1):
                z = Fraction(d) + m * dF / J
                pc = (xn * z, yn * z, z)
                q = [(sum(R[r][c] * pc[c] for c in range(3)) + t[r] - org[r]) / sF for r in range(3)]
                cands = []
                edge = False
                for r in range(3):
                    fl = math.floor(q[r])
                    opts = {fl}
                    if q[r] - fl < eps:
                        opts.add(fl - 1)
                    if fl + 1 - q[r] < eps:
                        opts.add(fl + 1)
                    cands.append(opts)
                    blocks = {o // 8 for o in opts if 0 <= o < G}
                    if len(blocks) != 1 or len({o for o in opts}) != len([o for o in opts if 0 <= o < G]):
                        edge = True
                blist = {(a // 8, b // 8, c // 8) for a in cands[0] for b in cands[1] for c in cands[2]
                         if 0 <= a < G and 0 <= b < G and 0 <= c < G}
                kl = {bx + nb * (by + nb * bz) for bx, by, bz in blist}
                if not edge and len(kl) == 1:
                    sure |= kl
                maybe |= kl
    assert len(sure) > 20, len(sure)
    assert sure <= keys, sorted(sure - keys)[:10]
    assert keys <= maybe, sorted(keys - maybe)[:10]


def pin_alloc_capacity_and_order(lib_path=None):
    """A pool with room for only part of a frame's blocks keeps the lowest keys
    (ascending key order), flags the overflow, and a repeated frame adds nothing."""
    rng = np.random.default_rng(41)
    intr = synth.Intrinsics.centred(30.0, 32, 24)
    vol = _plane_volume(cap=100000)
    depth = (0.5 + rng.uniform(-0.01, 0.01, (24, 32))).astype(np.float32)
    full = oracle.OracleVolume(vol, intr, lib_path=lib_path)
    keys = full.frame_blocks(depth, np.eye(4))
    n_new, over = full.allocate(depth, np.eye(4), 0)
    assert n_new == len(keys) and not over
    assert full.allocate(depth, np.eye(4), 1) == (0, False)
    cap = len(keys) // 3
    small = oracle.OracleVolume(synth.VolumeParams(**{**vol.__dict__, "block_capacity": cap}), intr,
                                lib_path=lib_path)
    n_new, over = small.allocate(depth, np.eye(4), 0)
    assert n_new == cap and over
    e = small.export(values=False)
    nb = vol.grid_dim // 8
    got = e.coords[:, 0] + nb * (e.coords[:, 1] + nb * e.coords[:, 2])
    assert np.array_equal(np.sort(got), np.sort(keys)[:cap])


def pin_dense_equals_sparse(lib_path=None):
    """Dense brute force (Alg. 3 on every voxel of the grid) and the sparse volume
    agree on every voxel of every block allocated at the first frame, and the
    blocks the sampling misses hold almost no valid voxels."""
    seq = synth.sphere_sequence(n_frames=4, noise=True, grid_dim=128, voxel_size=2e-3)
    ov = oracle.OracleVolume(seq.volume, seq.intr, lib_path=lib_path)
    dn = oracle.DenseOracle(seq.volume, seq.intr)
    if lib_path is not None:
        dn.lib = oracle.lib(lib_path)
        dn.h = dn.lib.ov_dense_create(oracle.ctypes.byref(dn.params))
    for k in range(seq.n_frames):
        ov.fuse(seq.depth[k], seq.poses[k])
        dn.integrate(seq.depth[k], seq.poses[k])
    e = ov.export()
    vox = oracle.voxel_coords(e)
    Td, Pd, _ = dn.read(vox)
    m = np.repeat(e.alloc_frame == 0, 512)
    Ts, Ps = e.T.ravel(), e.P.ravel()
    assert np.array_equal(np.isnan(Ts[m]), np.isnan(Td[m]))
    ok = m & ~np.isnan(Ts)
    assert ok.sum() > 10000
    assert np.array_equal(Ts[ok], Td[ok]) and np.array_equal(Ps[ok], Pd[ok])
    n_valid, n_missed = dn.coverage(ov)
    assert n_valid > 10000 and n_missed / n_valid < 0.02, (n_valid, n_missed)


# ----------------------------------------------------------------------------
# raycast (section "Scene Rendering")
# ----------------------------------------------------------------------------

def pin_plane_raycast_exact(lib_path=None):
    """A fronto-parallel plane seen by cameras with identity rotation gives
    T = d0 - z at every voxel, an affine field that trilinear interpolation
    reproduces exactly: the raycast depth equals d0 - t_z, the vertex lies on the
    plane and the normal is (0, 0, -1)."""
    d0 = 0.5
    vol = _plane_volume(sigma=1e-3)
    intr = synth.Intrinsics.centred(30.0, 32, 24)
    poses = []
    for k in range(3):
        T = np.eye(4)
        T[:3, 3] = [0.004 * k, -0.003 * k, 0.002 * k]
        poses.append(T)
    ov = oracle.OracleVolume(vol, intr, lib_path=lib_path)
    for T in poses:
        ov.fuse(np.full((24, 32), d0 - T[2, 3], np.float32), T)
    Tq = np.eye(4)
    Tq[:3, 3] = [0.001, 0.002, 0.01]
    depth, vert, nrm, flags = ov.raycast(Tq)
    hit = (flags & 1) > 0
    assert hit.sum() > 40, hit.sum()
    # frame k measured the plane at world z = D_k + t_z with variance (a D_k^2)^2;
    # the fused zero level is their inverse-variance weighted mean (Alg. 3, Q = 0)
    Dk = np.array([float(np.float32(d0 - T[2, 3])) for T in poses])
    planes = Dk + np.array([T[2, 3] for T in poses])
    w = 1.0 / (float(np.float32(1e-3)) * Dk ** 2) ** 2
    plane = float((planes * w).sum() / w.sum())
    assert np.allclose(depth[hit], plane - Tq[2, 3], atol=1e-9, rtol=0), np.abs(depth[hit] - (plane - Tq[2, 3])).max()
    assert np.allclose(vert[hit, 2], plane, atol=1e-9)
    ok = (flags & 4) == 0
    assert (hit & ok).sum() > 20
    assert np.allclose(nrm[hit & ok], [0.0, 0.0, -1.0], atol=1e-9)
    assert np.isnan(vert[~hit]).all() and (depth[~hit] == 0).all()


def pin_sphere_raycast_analytic(lib_path=None):
    """Fusing noise-free views of a sphere and raycasting gives the analytic
    ray-sphere depth up to the error of the projective distance (the measured
    depth is constant over a pixel's footprint): within 0.5 voxel where the
    surface faces the camera (cos > 0.9) and 1.5 voxel at cos > 0.5."""
    seq = synth.sphere_sequence(noise=False, keep_clean=True)
    ov = oracle.OracleVolume(seq.volume, seq.intr, lib_path=lib_path)
    _fuse(ov, seq.depth, seq.poses)
    pose = seq.poses[-1]
    d, v, n, fl = ov.raycast(pose)
    H, W = seq.intr.height, seq.intr.width
    d = d.reshape(H, W)
    hit = (fl & 1).reshape(H, W) > 0
    gt = seq.clean_depth[-1]
    o, dw = synth._pixel_rays(seq.intr, pose, "cpu")
    dw = dw.numpy()
    with np.errstate(invalid="ignore"):
        P = o.numpy() + gt[..., None] * dw
        nrm = P / np.linalg.norm(P, axis=-1, keepdims=True)
        cosv = np.abs((nrm * dw).sum(-1)) / np.linalg.norm(dw, axis=-1)
    s = seq.volume.voxel_size
    assert abs(int(hit.sum()) - int(np.isfinite(gt).sum())) < 0.03 * np.isfinite(gt).sum()
    err = np.abs(d - gt) / s
    m9 = hit & np.isfinite(gt) & (cosv > 0.9)
    m5 = hit & np.isfinite(gt) & (cosv > 0.5)
    assert m9.sum() > 300 and m5.sum() > 1500
    assert err[m9].max() < 0.5 and err[m9].mean() < 0.1, (err[m9].max(), err[m9].mean())
    assert err[m5].max() < 1.5, err[m5].max()
    nn = n.reshape(H, W, 3)
    good = m9 & np.isfinite(nn[..., 0])
    ang = np.degrees(np.arccos(np.clip((nn[good] * nrm[good]).sum(-1), -1.0, 1.0)))
    # the per-pixel staircase of the projective distance tilts the gradient by a
    # few degrees; a wrong sign or axis would be off by tens of degrees
    assert np.median(ang) < 6.0 and ang.max() < 15.0, (np.median(ang), ang.max())


# ----------------------------------------------------------------------------
# learned variance network (an addition to the paper; see the oracle)
# ----------------------------------------------------------------------------

def _bf16(x):
    """Round float64 values to bfloat16 (nearest even) and widen back."""
    f = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((f + 0x7FFF + ((f >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _random_mlp(rng, lib_path=None):
    n = int(oracle.lib(lib_path).ov_mlp_param_count())
    w = _bf16(rng.normal(0.0, 0.3, n))
    return oracle.Mlp(w, lib_path)


def pin_mlp_gradient_finite_differences(lib_path=None):
    """The backward pass equals central finite differences of the summed loss
    (out + s exp(-out)) / 2 for every bias and a sample of weights."""
    rng = np.random.default_rng(61)
    net = _random_mlp(rng, lib_path)
    x = rng.uniform(-1, 1, (40, 27))
    x[:, 25] = rng.uniform(0.1, 1.0, 40)
    x[:, 26] = rng.uniform(0, 1, 40)
    s = rng.uniform(0.1, 4.0, 40)
    loss, g = net.loss_grad(x, s)
    idx = np.concatenate([rng.choice(net.n_params, 150, replace=False), np.arange(864, 896),
                          np.arange(1920, 1985)])
    h = 1e-6
    for i in idx:
        wp, wm = net.w.copy(), net.w.copy()
        wp[i] += h
        wm[i] -= h
        lp, _ = oracle.Mlp(wp, lib_path).loss_grad(x, s)
        lm, _ = oracle.Mlp(wm, lib_path).loss_grad(x, s)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    out = net.forward(x)
    assert abs(loss - 0.5 * (out + s * np.exp(-out)).sum()) < 1e-9 * abs(loss)


def pin_mlp_closed_forms(lib_path=None):
    """A network with only b3 = c outputs c everywhere; one path through the
    depth input (W1[0][25] = W2[0][0] = W3[0] = 1) outputs D/4, and the same
    path with a negative first weight is cut by ReLU to 0."""
    n = int(oracle.lib(lib_path).ov_mlp_param_count())
    rng = np.random.default_rng(62)
    x = rng.uniform(-1, 1, (25, 27))
    x[:, 25] = rng.uniform(0.1, 1.0, 25)
    w = np.zeros(n)
    w[-1] = 0.37
    assert np.allclose(oracle.Mlp(w, lib_path).forward(x), 0.37, atol=0, rtol=1e-15)
    w = np.zeros(n)
    w[0 * 27 + 25] = 1.0                       # W1[0][25]
    w[864 + 32 + 0] = 1.0                      # W2[0][0]
    w[864 + 32 + 1024 + 32 + 0] = 1.0          # W3[0]
    assert np.allclose(oracle.Mlp(w, lib_path).forward(x), x[:, 25], atol=1e-15)
    w[0 * 27 + 25] = -1.0
    assert np.allclose(oracle.Mlp(w, lib_path).forward(x), 0.0, atol=1e-15)


def pin_mlp_features_on_planes(lib_path=None):
    """A fronto-parallel plane gives a zero patch, D/4, and the incidence cosine
    of the viewing ray 1/|(xn, yn, 1)|; a plane tilted by theta about the camera
    x axis gives |n . ray| with n = (0, -sin theta, cos theta); pixels outside
    the image or with no measurement read +1."""
    W, H, f = 24, 18, 20.0
    intr = synth.Intrinsics.centred(f, W, H)
    vol = _plane_volume()
    net = oracle.Mlp(np.zeros(int(oracle.lib(lib_path).ov_mlp_param_count())), lib_path)
    d0 = 0.8
    depth = np.full((H, W), d0, np.float32)
    uv = np.array([[12, 9], [3, 4], [20, 15], [0, 0]])
    feat, valid = net.features(depth, intr, vol, uv)
    assert valid.all()
    assert np.allclose(feat[:3, :25], 0.0)
    assert np.allclose(feat[:, 25], float(np.float32(d0)) / 4)
    xn = (uv[:3, 0] - intr.cx) / intr.fx
    yn = (uv[:3, 1] - intr.cy) / intr.fy
    assert np.allclose(feat[:3, 26], 1.0 / np.sqrt(1 + xn ** 2 + yn ** 2), atol=1e-6)
    corner = feat[3, :25].reshape(5, 5)
    assert (corner[:2, :] == 1).all() and (corner[:, :2] == 1).all() and feat[3, 26] == 0.0
    th = 0.5
    v, u = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    ynp = (v - intr.cy) / intr.fy
    # plane through (0, 0, d0) with normal (0, -sin th, cos th): z = d0 / (cos th - sin th yn) * cos th
    depth_t = (d0 * np.cos(th) / (np.cos(th) - np.sin(th) * ynp)).astype(np.float32)
    feat, valid = net.features(depth_t, intr, vol, uv[:3])
    nrm = np.array([0.0, -np.sin(th), np.cos(th)])
    xn, yn = (uv[:3, 0] - intr.cx) / intr.fx, (uv[:3, 1] - intr.cy) / intr.fy
    ray = np.stack([xn, yn, np.ones(3)], -1)
    want = np.abs(ray @ nrm) / np.linalg.norm(ray, axis=-1)
    assert np.allclose(feat[:, 26], want, atol=2e-4), (feat[:, 26], want)
    dd = depth_t[:, :].astype(np.float64)
    k = 0
    exp_patch = np.array([np.clip((dd[uv[k, 1] + dy, uv[k, 0] + dx] - dd[uv[k, 1], uv[k, 0]]) / vol.truncation, -1, 1)
                          for dy in range(-2, 3) for dx in range(-2, 3)])
    assert np.allclose(feat[0, :25], exp_patch, atol=2e-6)
    bad = depth.copy()
    bad[9, 12] = np.nan
    _, valid = net.features(bad, intr, vol, uv[:1])
    assert not valid[0]


def pin_mlp_variance_fallback(lib_path=None):
    """Variance = p_quad exp(out): the zero network gives the quadratic model,
    b3 = 0.5 scales it by e^0.5, outputs inside [-ln 4, ln 64] scale it by
    e^out, and an output outside that range falls back to it."""
    W, H = 16, 12
    intr = synth.Intrinsics.centred(14.0, W, H)
    vol = _plane_volume(sigma=1.5e-3)
    depth = np.random.default_rng(63).uniform(0.45, 0.55, (H, W)).astype(np.float32)
    depth[3, 4] = 0.0
    n = int(oracle.lib(lib_path).ov_mlp_param_count())
    pq = ((np.float64(np.float32(1.5e-3)) * depth.astype(np.float64) ** 2) ** 2)
    for b3, scale in ((0.0, 1.0), (0.5, np.exp(0.5)), (2.0, np.exp(2.0)), (4.0, np.exp(4.0)), (-1.0, np.exp(-1.0)),
                      (4.3, 1.0), (-1.5, 1.0)):
        w = np.zeros(n)
        w[-1] = b3
        var = oracle.Mlp(w, lib_path).variance_map(depth, intr, vol).astype(np.float64)
        ok = depth > 0
        assert np.allclose(var[ok], (pq * scale)[ok], rtol=1e-6), b3
        assert var[3, 4] == 0.0


# ----------------------------------------------------------------------------
# point-to-plane registration (section "Registration", Eqs. 2-8)
# ----------------------------------------------------------------------------

def _small_motion(pose, rot_deg, axis, trans):
    from oracle import icp as oicp
    a = np.asarray(axis, np.float64)
    inc = np.eye(4)
    inc[:3, :3] = oicp.rotation(np.deg2rad(rot_deg) * a / np.linalg.norm(a))
    inc[:3, 3] = trans
    return inc @ pose


def _room_icp_case(W=160, H=120):
    seq = synth.room_sequence(n_frames=2, width=W, height=H, device="cpu")
    model_pose = seq.poses[0]
    true_pose = _small_motion(model_pose, 1.0, (0.3, 1.0, 0.2), (0.012, -0.008, 0.015))
    _, mv, mn = synth.render_maps(seq.scene, seq.intr, model_pose)
    depth = synth.render_depth(seq.scene, seq.intr, true_pose).numpy()
    depth = np.where(np.isfinite(depth), depth, 0.0).astype(np.float32)
    return seq.intr, depth, model_pose, true_pose, mv.numpy(), mn.numpy()


def pin_icp_recovers_a_known_motion(lib_path=None):
    """Noise-free frame rendered at a pose 1 degree and 2 cm from the model's:
    ICP started at the model pose returns the frame's true pose (the whole chain:
    projective matching, Eq. 4 sums, the unit-cube restatement, Eq. 8 and the
    pose update). Exact maps of the analytic room stand in for the raycast."""
    from oracle import icp as oicp
    intr, depth, model_pose, true_pose, mv, mn = _room_icp_case()
    pose, info = oicp.icp(depth, intr, model_pose, mv, mn, model_pose, oicp.IcpParams(iterations=12))
    assert info["matches"] > 10000 and info["rank"] == 6, info
    dt = np.linalg.norm(pose[:3, 3] - true_pose[:3, 3])
    ang = np.arccos(np.clip((np.trace(pose[:3, :3] @ true_pose[:3, :3].T) - 1) / 2, -1, 1))
    # projective matching pairs each frame point with the model point on the
    # nearest pixel's ray, which leaves a bias far below a pixel's footprint
    assert dt < 2e-4 and ang < 2e-4, (dt, ang)
    start = np.linalg.norm(model_pose[:3, 3] - true_pose[:3, 3])
    assert start > 0.015


def pin_icp_scaled_equals_unscaled(lib_path=None):
    """With no eigen-direction dropped (theta = 0), the unit-cube restatement
    (Eqs. 5-7) and its recovery give the same motion as solving Eq. 4 directly."""
    from oracle import icp as oicp
    intr, depth, model_pose, true_pose, mv, mn = _room_icp_case()
    p, q, n = oicp.match(depth, intr, model_pose, mv, mn, model_pose, oicp.IcpParams())
    A, g, _, N = oicp.unscaled_sums(p, q, n)
    x = np.linalg.solve(A, -g)
    C, b, m, S = oicp.scaled_system(p, q, n)
    xh, rank = oicp.solve(C, b, N, 0.0)
    assert rank == 6
    r = xh[:3] / S
    t = xh[3:] - np.cross(r, m)
    assert np.allclose(r, x[:3], rtol=1e-7, atol=1e-12) and np.allclose(t, x[3:], rtol=1e-7, atol=1e-12)
    assert np.abs(x).max() > 1e-3     # a real motion, not a trivial zero


def pin_icp_plane_keeps_unobservable_motion_out(lib_path=None):
    """A single plane constrains only the motion along its normal and the tilts:
    Eq. 8 keeps three eigen-directions and a frame moved within the plane (3 cm
    along it, 2 degrees about its normal) leaves the pose where it started."""
    from oracle import icp as oicp
    scene = synth.Scene(ground_plane=True)
    intr = synth.Intrinsics.centred(105.0, 160, 120)
    model_pose = synth.look_at((0.2, 1.2, -0.4), (0.0, 0.0, 0.6))
    moved = np.eye(4)
    moved[:3, :3] = oicp.rotation(np.deg2rad(2.0) * np.array([0.0, 1.0, 0.0]))
    moved[:3, 3] = (0.03, 0.0, 0.01)
    true_pose = moved @ model_pose
    _, mv, mn = synth.render_maps(scene, intr, model_pose)
    depth = synth.render_depth(scene, intr, true_pose).numpy()
    depth = np.where(np.isfinite(depth), depth, 0.0).astype(np.float32)
    pose, info = oicp.step(depth, intr, model_pose, mv.numpy(), mn.numpy(), model_pose, oicp.IcpParams())
    assert info["matches"] > 5000 and info["rank"] == 3, info
    assert np.abs(pose - model_pose).max() < 1e-6       # float32 depth leaves ~1e-8 m of residual


# ----------------------------------------------------------------------------
# T_k refined by gradient steps in the depth map (section "Integration of
# Measurements", last paragraph)
# ----------------------------------------------------------------------------

def _refined_single_frame(depth, intr, steps, lib_path, s=2e-3, G=128, z_centre=0.6):
    from dataclasses import replace
    vol = replace(_plane_volume(s=s, G=G, z_centre=z_centre, sigma=1e-3, cap=1 << 14), refine_steps=steps)
    ov = oracle.OracleVolume(vol, intr, lib_path=lib_path)
    ov.fuse(depth, np.eye(4))
    e = ov.export()
    xyz = _voxel_world(vol, oracle.voxel_coords(e))
    T = e.T.ravel()
    ok = ~np.isnan(T) & ~e.amb.ravel()
    return vol, xyz[ok], T[ok]


def pin_refined_tk_plane_distances(lib_path=None):
    """Gauss-Newton steps move to the foot of the perpendicular: for a
    fronto-parallel plane the refined T_k is the z-difference itself; for a plane
    tilted by 35 degrees it is the signed perpendicular distance
    d0 cos(theta) - n.X, smaller than the z-difference by cos(theta)."""
    W, H, f = 96, 72, 90.0
    intr = synth.Intrinsics.centred(f, W, H)
    d0 = 0.6
    flat = np.full((H, W), d0, np.float32)
    vol, X, T = _refined_single_frame(flat, intr, 3, lib_path)
    assert T.size > 5000
    assert np.abs(T - (float(np.float32(d0)) - X[:, 2])).max() < 1e-9
    th = np.deg2rad(35.0)
    v, u = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    yn = (v - intr.cy) / intr.fx
    tilt = (d0 * np.cos(th) / (np.cos(th) - np.sin(th) * yn)).astype(np.float32)
    vol, X, T = _refined_single_frame(tilt, intr, 3, lib_path)
    n = np.array([0.0, -np.sin(th), np.cos(th)])
    exact = d0 * np.cos(th) - X @ n
    zdiff_scale = np.abs(exact).max() / np.cos(th)
    assert T.size > 5000 and zdiff_scale > 0.5 * vol.truncation
    err = np.abs(T - exact)
    assert np.percentile(err, 99) < 1e-3 * vol.truncation and err.max() < 1e-2 * vol.truncation, err.max()


def pin_refined_tk_sphere_distance(lib_path=None):
    """Near a sphere the refined T_k approaches the Euclidean distance |X - c| - r
    (up to the bilinear interpolation of the depth map), which the plain
    z-difference overestimates away from the centre of the view."""
    W, H, f = 96, 72, 90.0
    intr = synth.Intrinsics.centred(f, W, H)
    c, r = np.array([0.01, -0.02, 0.6]), 0.12
    scene = synth.Scene(spheres=np.array([[c[0], c[1], c[2], r]]))
    depth = synth.render_depth(scene, intr, np.eye(4)).numpy()
    depth = np.where(np.isfinite(depth), depth, 0.0).astype(np.float32)
    vol, X, T = _refined_single_frame(depth, intr, 3, lib_path, z_centre=0.55)
    _, X0, T0 = _refined_single_frame(depth, intr, 0, lib_path, z_centre=0.55)
    # voxels whose viewing ray passes within 0.7 r of the centre: there
    # neighbouring pixels differ by less than delta, so the steps apply (nearer
    # the silhouette the depth map has edges and T_k stays the z-difference); and
    # beyond 0.45 r, where the surface is oblique enough for the z-difference to
    # overestimate the distance
    def ring(P):
        ray = P / np.linalg.norm(P, axis=1, keepdims=True)
        miss = np.linalg.norm(np.cross(ray, c[None, :]), axis=1)      # distance of the ray from c
        return (miss > 0.45 * r) & (miss < 0.7 * r)
    exact = np.linalg.norm(X - c, axis=1) - r
    m = ring(X)
    assert m.sum() > 2000
    err = np.abs(T - exact)[m]
    assert np.percentile(err, 99) < 0.02 * vol.truncation, np.percentile(err, 99)
    m0 = ring(X0)
    err0 = np.abs(T0 - (np.linalg.norm(X0 - c, axis=1) - r))[m0]
    assert np.median(err0) > 10 * np.median(err), (np.median(err0), np.median(err))


# ----------------------------------------------------------------------------
# marching-cubes surface (section "Scene Rendering", the polygonising renderer)
# ----------------------------------------------------------------------------

def _edge_use(tris):
    """Directed mesh edges (vertex keys rounded to 1e-9) and their counts."""
    from collections import Counter
    key = lambda p: tuple(np.round(p, 9))
    d = Counter()
    for t in tris:
        for a, b in ((0, 1), (1, 2), (2, 0)):
            d[(key(t[a]), key(t[b]))] += 1
    return d


def pin_mesh_sphere_closed_and_outward(lib_path=None):
    """The exact signed distance of a sphere sampled on a lattice gives a closed,
    consistently oriented surface: every directed edge appears once and its
    reverse once, V - E + F = 2, vertices lie on the sphere within the linear
    interpolation error, and every triangle's normal points outward."""
    from oracle import mesh as omesh
    s, n, r = 1.0, 24, 7.3
    c = np.array([11.2, 12.1, 11.7])
    g = np.indices((n, n, n)).transpose(1, 2, 3, 0).astype(np.float64)
    T = np.linalg.norm(g - c, axis=-1) - r
    tris = omesh.mesh(T, (0.0, 0.0, 0.0), s)
    assert tris.shape[0] > 500
    use = _edge_use(tris)
    assert all(v == 1 for v in use.values())
    assert all(use.get((b, a), 0) == 1 for (a, b) in use)
    V = len({p for e in use for p in e})
    E = len(use) // 2
    assert V - E + tris.shape[0] == 2
    d = np.abs(np.linalg.norm(tris - c, axis=-1) - r)
    assert d.max() < 0.05 * s, d.max()
    nrm = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    assert (np.einsum("ij,ij->i", nrm, tris.mean(1) - c) > 0).all()


def pin_mesh_every_case_closed(lib_path=None):
    """Each of the 256 corner sign patterns, embedded in a lattice with a
    one-voxel margin of positive values, gives a closed oriented surface (all
    directed edges paired), and every crossed edge lies on exactly one loop."""
    from oracle import mesh as omesh
    for case in range(1, 255):
        T = np.ones((4, 4, 4))
        for cidx in range(8):
            if case >> cidx & 1:
                T[1 + (cidx & 1), 1 + ((cidx >> 1) & 1), 1 + ((cidx >> 2) & 1)] = -1.0
        tris = omesh.mesh(T, (0.0, 0.0, 0.0), 1.0)
        use = _edge_use(tris)
        assert all(v == 1 and use.get((b, a), 0) == 1 for (a, b), v in use.items()), case
    for case in range(256):
        # every crossed edge of the cell is on exactly one loop
        ins = tuple(bool(case >> k & 1) for k in range(8))
        crossed = sorted(k for k, (a, b) in enumerate(omesh.EDGES) if ins[a] != ins[b])
        assert sorted(e for l in omesh.case_polygons(ins) for e in l) == crossed, case


# ----------------------------------------------------------------------------
# eviction and volume shift (section "Discussion")
# ----------------------------------------------------------------------------

def _fused(seq, n, lib_path=None):
    ov = oracle.OracleVolume(seq.volume, seq.intr, lib_path=lib_path, amb_px=5e-4)
    for k in range(n):
        ov.fuse(seq.depth[k], seq.poses[k])
    return ov


def _by_key(e, nb):
    key = e.coords[:, 0].astype(np.int64) + nb * (e.coords[:, 1] + nb * e.coords[:, 2].astype(np.int64))
    o = np.argsort(key)
    return key[o], e.T[o], e.P[o], e.alloc_frame[o]


def _same_values(a, b):
    return np.array_equal(np.isnan(a), np.isnan(b)) and np.array_equal(np.nan_to_num(a), np.nan_to_num(b))


def pin_evict_takes_the_blocks_outside_the_box_and_import_restores(lib_path=None):
    """Eviction is bookkeeping: the evicted blocks are exactly those a brute-force
    test of the exported coordinates puts outside the box, with their exported
    values; the kept ones are untouched; importing the evicted ones restores
    the volume (section "Discussion")."""
    sphere = synth.sphere_sequence(n_frames=4)
    ov = _fused(sphere, 4, lib_path)
    nb = sphere.volume.grid_dim // 8
    before = ov.export()
    lo, hi = np.array([5, 10, 8]), np.array([20, 30, 16])
    out = np.any((before.coords < lo) | (before.coords >= hi), axis=1)
    assert 0 < out.sum() < len(out)
    ev = ov.evict(lo, hi)
    # the evicted set, by brute force over the exported coordinates
    k_ev, T_ev, P_ev, f_ev = _by_key(ev, nb)
    sel = oracle.Export(before.coords[out], before.alloc_frame[out], before.T[out], before.P[out], before.amb[out])
    k_ref, T_ref, P_ref, f_ref = _by_key(sel, nb)
    assert np.array_equal(k_ev, k_ref) and np.array_equal(f_ev, f_ref)
    assert _same_values(T_ev, T_ref) and _same_values(P_ev, P_ref)
    # the kept ones, untouched
    after = ov.export()
    assert len(after.coords) == int((~out).sum())
    assert not np.any((after.coords < lo) | (after.coords >= hi))
    keep = oracle.Export(before.coords[~out], before.alloc_frame[~out], before.T[~out], before.P[~out],
                         before.amb[~out])
    ka, Ta, Pa, _ = _by_key(after, nb)
    kk, Tk, Pk, _ = _by_key(keep, nb)
    assert np.array_equal(ka, kk) and _same_values(Ta, Tk) and _same_values(Pa, Pk)
    # and back: the whole volume again (imported blocks count as allocated now)
    ov.import_blocks(ev.coords, ev.T, ev.P)
    k1, T1, P1, f1 = _by_key(ov.export(), nb)
    k0, T0, P0, f0 = _by_key(before, nb)
    assert np.array_equal(k1, k0) and _same_values(T1, T0) and _same_values(P1, P0)
    moved = np.isin(k0, k_ev)
    assert np.array_equal(f1[~moved], f0[~moved]) and np.all(f1[moved] == ov.frame)


def _refused(fn) -> bool:
    try:
        fn()
    except ValueError:
        return True
    return False


def pin_import_refuses_duplicates_and_allocated_blocks(lib_path=None):
    """A block is allocated once: importing an allocated block, a block twice or
    one outside the grid is refused and changes nothing."""
    sphere = synth.sphere_sequence(n_frames=2)
    ov = _fused(sphere, 2, lib_path)
    e = ov.export()
    n = ov.n_blocks
    assert _refused(lambda: ov.import_blocks(e.coords[:1], e.T[:1], e.P[:1]))          # already allocated
    ev = ov.evict([0, 0, 0], [16, 32, 32])
    assert len(ev.coords) > 1
    twice = np.concatenate([ev.coords[:1], ev.coords[:1]])
    assert _refused(lambda: ov.import_blocks(twice, np.concatenate([ev.T[:1]] * 2), np.concatenate([ev.P[:1]] * 2)))
    assert _refused(lambda: ov.import_blocks(np.array([[-1, 0, 0]]), ev.T[:1], ev.P[:1]))   # outside the grid
    assert ov.n_blocks == n - len(ev.coords)


def pin_shift_and_its_inverse_restore_the_volume(lib_path=None):
    """A shift by d moves the origin by 8 s d and evicts the blocks leaving the
    grid; shifting back and importing them restores the volume."""
    sphere = synth.sphere_sequence(n_frames=3)
    ov = _fused(sphere, 3, lib_path)
    nb = sphere.volume.grid_dim // 8
    before = ov.export()
    o0 = ov.origin.copy()
    d = np.array([4, -3, 2])                      # blocks at x < 4 and z < 2 leave the grid
    ev = ov.shift(d)
    assert len(ev.coords) > 0
    assert np.allclose(ov.origin, o0 + 8 * d * float(np.float32(sphere.volume.voxel_size)), rtol=0, atol=1e-15)
    mid = ov.export()
    assert np.all((mid.coords >= 0) & (mid.coords < nb))
    ev_back = ov.shift(-d)
    assert len(ev_back.coords) == 0               # nothing leaves on the way back
    ov.import_blocks(ev.coords, ev.T, ev.P)
    k1, T1, P1, _ = _by_key(ov.export(), nb)
    k0, T0, P0, _ = _by_key(before, nb)
    assert np.array_equal(k1, k0) and _same_values(T1, T0) and _same_values(P1, P0)
    assert np.allclose(ov.origin, o0, rtol=0, atol=1e-15)


def pin_fusing_into_a_shifted_volume_matches_the_unshifted_one(lib_path=None):
    """Voxel i' = i - 8d of the shifted grid is voxel i of the original: after a
    shift by d, fusing the remaining frames gives the same T and P at the same
    world positions (block coordinates moved by -d)."""
    sphere = synth.sphere_sequence(n_frames=4)
    nb = sphere.volume.grid_dim // 8
    ref = _fused(sphere, 4, lib_path)
    ov = _fused(sphere, 2, lib_path)
    d = np.array([1, -2, 1])                      # keeps every block of the sphere inside the grid
    assert len(ov.shift(d).coords) == 0
    for k in range(2, 4):
        ov.fuse(sphere.depth[k], sphere.poses[k])
    a, b = ref.export(), ov.export()
    b_world = oracle.Export(b.coords + d, b.alloc_frame, b.T, b.P, b.amb)
    ka, Ta, Pa, _ = _by_key(a, nb)
    kb, Tb, Pb, _ = _by_key(b_world, nb)
    assert np.array_equal(ka, kb)
    amb = _by_key(oracle.Export(a.coords, a.alloc_frame, a.amb.astype(float), a.amb.astype(float), a.amb), nb)[1] > 0
    amb |= _by_key(oracle.Export(b_world.coords, b.alloc_frame, b.amb.astype(float), b.amb.astype(float), b.amb),
                  nb)[1] > 0
    ok = ~amb
    assert np.array_equal(np.isnan(Ta)[ok], np.isnan(Tb)[ok])
    both = ok & ~np.isnan(Ta) & ~np.isnan(Tb)
    delta = float(sphere.volume.truncation)
    assert both.sum() > 50000
    assert np.max(np.abs(Ta[both] - Tb[both])) < 1e-9 * delta
    assert np.max(np.abs(Pa[both] - Pb[both]) / Pa[both]) < 1e-9


# ----------------------------------------------------------------------------
# per-voxel replay (the sampled full-size parity checker) and the raycast's
# crossing-uniqueness flag
# ----------------------------------------------------------------------------

def pin_replay_closed_form(lib_path=None):
    """The per-voxel replay of a sequence applies Alg. 3 to the frames from the
    voxel's allocation frame on. With Q = 0 and a static camera seeing a
    fronto-parallel plane at depth D_k in frame k (T_k = D_k - z exactly), the
    result is the inverse-variance weighted mean over exactly those frames
    f >= a whose |T_k| <= delta: T = sum(T_k/p_k)/sum(1/p_k), P = 1/sum(1/p_k).
    Allocation frames are drawn at random per voxel (including before the first
    frame and after the last), so a replay that starts a frame early or late,
    or ignores the allocation frame, disagrees with the closed form."""
    vol = _plane_volume()
    intr = synth.Intrinsics.centred(30.0, 32, 24)
    n = 9
    D, p, depths, vars_ = _const_frames(n, seed=21, spread=4e-3)
    rng = np.random.default_rng(22)
    G = vol.grid_dim
    s = float(np.float32(vol.voxel_size))
    # voxels whose camera depth lies within 1.5 delta of the plane's depths
    iz_lo = int((0.5 - 1.5 * vol.truncation - vol.origin[2]) / s)
    iz_hi = int((0.5 + 1.5 * vol.truncation - vol.origin[2]) / s)
    m = 6000
    vox = np.stack([rng.integers(0, G, m), rng.integers(0, G, m), rng.integers(iz_lo, iz_hi + 1, m)], -1)
    alloc = rng.integers(-1, n + 1, m).astype(np.int32)
    T, P, amb = oracle.replay_voxels(vol, intr, depths, np.stack([np.eye(4)] * n), vox, alloc, vars_,
                                     lib_path=lib_path)
    Tk = D[None, :] - _voxel_world(vol, vox)[:, 2:3]          # (voxels, frames)
    delta = vol.truncation
    frames = np.arange(n)[None, :] >= alloc[:, None]
    valid = (np.abs(Tk) < delta * (1 - 1e-6)) & frames
    clear = ((np.abs(Tk) < delta * (1 - 1e-6)) | (np.abs(Tk) > delta * (1 + 1e-6))).all(1)
    w = np.where(valid, 1.0 / p[None, :], 0.0)
    some = valid.any(1) & clear
    late = some & (alloc > 0) & (alloc < n)
    assert some.sum() > 2000 and late.sum() > 1500, (some.sum(), late.sum())
    assert not amb[clear].any()
    T_exp = (Tk[some] * w[some]).sum(1) / w[some].sum(1)
    assert np.allclose(T[some], T_exp, rtol=0, atol=1e-12), np.abs(T[some] - T_exp).max()
    assert np.allclose(P[some], 1.0 / w[some].sum(1), rtol=1e-12, atol=0)
    none = ~valid.any(1) & clear
    assert none.sum() > 200 and np.isnan(T[none]).all() and np.isnan(P[none]).all()


def pin_replay_equals_integrate(lib_path=None):
    """Replaying every voxel of every allocated block from its block's
    allocation frame reproduces the sparse volume that allocation plus Alg. 3
    integration built frame by frame, bit for bit (the same measurement and
    update in the same order per voxel), including blocks that joined the pool
    mid-sequence. The full-size voxel parity rests on this equivalence."""
    seq = synth.sphere_sequence(n_frames=6)
    ov = oracle.OracleVolume(seq.volume, seq.intr, lib_path=lib_path)
    _fuse(ov, seq.depth, seq.poses)
    e = ov.export()
    assert (e.alloc_frame > 0).sum() > 50, (e.alloc_frame > 0).sum()
    vox = oracle.voxel_coords(e)
    T, P, amb = oracle.replay_voxels(seq.volume, seq.intr, list(seq.depth), seq.poses, vox,
                                     np.repeat(e.alloc_frame, 512), lib_path=lib_path)
    Te, Pe = e.T.ravel(), e.P.ravel()
    assert np.array_equal(T, Te, equal_nan=True)
    assert np.array_equal(P, Pe, equal_nan=True)
    assert np.array_equal(amb, e.amb.ravel())
    assert (~np.isnan(Te)).sum() > 100000


def _slab_volume(thick, lib_path=None, cut=None):
    """Blocks holding the lattice samples of an analytic field of the world z
    alone, imported straight into an oracle volume: a single plane at z_front
    (T = z_front - z, positive on the camera side) when thick is None, else a
    slab from z_front to z_back = z_front + thick * delta
    (T = max(z_front - z, z - z_back)); chi where |T| > delta, and behind
    z_front + cut * delta when cut is given. z_front lies a
    quarter voxel past a lattice plane. Along z the trilinear field is the
    linear interpolation of those samples, whose zero crossings are exactly
    z_front and z_back (both ends of each crossing's lattice interval lie on
    the same face's branch). Returns (volume, z_front)."""
    vol = _plane_volume(G=64, z_centre=0.5)
    intr = synth.Intrinsics.centred(30.0, 32, 24)
    s = float(np.float32(vol.voxel_size))
    delta = float(np.float32(vol.truncation))
    o = vol.origin[2]
    z_front = o + (round((0.5 - o) / s) + 0.25) * s
    nb = vol.grid_dim // 8
    bz, by, bx = np.meshgrid(np.arange(nb), np.arange(nb), np.arange(nb), indexing="ij")
    coords = np.stack([bx.ravel(), by.ravel(), bz.ravel()], -1)
    l = np.arange(512)
    z = o + (coords[:, 2:3] * 8 + (l >> 6)[None, :]) * s
    T = z_front - z if thick is None else np.maximum(z_front - z, z - (z_front + thick * delta))
    T = np.where(np.abs(T) <= delta, T, np.nan)
    if cut is not None:
        T = np.where(z <= z_front + cut * delta, T, np.nan)
    keep = ~np.isnan(T).all(1)
    ov = oracle.OracleVolume(vol, intr, lib_path=lib_path)
    ov.import_blocks(coords[keep], T[keep], np.ones_like(T[keep]))
    return ov, z_front


def pin_crossing_uniqueness(lib_path=None):
    """The raycast flags a hit (flag 8) when the field along its ray changes
    sign more than once, or is undefined, within a coarse step (delta/2) of the
    crossing: a march that samples every delta/2 could then return another zero
    crossing. Analytic fields fix the answer:
      * a single plane has one crossing on every ray: no hit is flagged;
      * a slab 0.3 delta thick puts a second crossing 0.3 delta behind the
        first: every hit is flagged;
      * a slab 0.8 delta thick puts it beyond delta/2: no hit is flagged;
      * a plane whose field is chi from 0.2 delta behind it on has undefined
        samples within delta/2 of the crossing: every hit is flagged.
    In each case the hit depth is the front face."""
    pose = np.eye(4)
    pose[:3, 3] = [0.001, -0.002, 0.0]
    for thick, cut, flagged in [(None, None, False), (0.3, None, True), (0.8, None, False), (None, 0.2, True)]:
        ov, z_front = _slab_volume(thick, lib_path, cut)
        depth, _, _, flags = ov.raycast(pose)
        hit = (flags & 1) > 0
        assert hit.sum() > 30, hit.sum()
        assert np.allclose(depth[hit], z_front, rtol=0, atol=1e-9), np.abs(depth[hit] - z_front).max()
        f8 = (flags[hit] & 8) > 0
        assert f8.all() if flagged else not f8.any(), (thick, f8.mean())


ALL_PINS = [pin_kalman_closed_form, pin_eq9_mean, pin_process_variance_steady_state,
            pin_alg1_running_average, pin_alg2_weighted_average,
            pin_first_measurement_and_quadratic_variance, pin_projection_nearest_pixel,
            pin_alloc_exact_rational, pin_alloc_capacity_and_order, pin_dense_equals_sparse,
            pin_plane_raycast_exact, pin_sphere_raycast_analytic, pin_mlp_gradient_finite_differences,
            pin_mlp_closed_forms, pin_mlp_features_on_planes, pin_mlp_variance_fallback,
            pin_refined_tk_plane_distances, pin_refined_tk_sphere_distance,
            pin_evict_takes_the_blocks_outside_the_box_and_import_restores,
            pin_import_refuses_duplicates_and_allocated_blocks, pin_shift_and_its_inverse_restore_the_volume,
            pin_fusing_into_a_shifted_volume_matches_the_unshifted_one, pin_replay_closed_form,
            pin_replay_equals_integrate, pin_crossing_uniqueness]

# the registration oracle is numpy code (oracle/icp.py); its own mutation test
# plants mistakes in copies of that module
ICP_PINS = [pin_icp_recovers_a_known_motion, pin_icp_scaled_equals_unscaled,
            pin_icp_plane_keeps_unobservable_motion_out]
MESH_PINS = [pin_mesh_sphere_closed_and_outward, pin_mesh_every_case_closed]


def run_all(lib_path=None, stop_at_first: bool = False) -> list:
    """Names of the pins that fail for the library at ``lib_path`` (only the
    first one with ``stop_at_first``)."""
    failed = []
    for pin in ALL_PINS:
        try:
            pin(lib_path)
        except AssertionError:
            failed.append(pin.__name__)
            if stop_at_first:
                break
    return failed
