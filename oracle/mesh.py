"""CPU oracle for the marching-cubes surface of the TSDF (section "Scene
Rendering": the paper's alternative renderer polygonises the non-empty blocks
by marching cubes). TEST INFRASTRUCTURE ONLY: plain FP64 numpy / Python,
written from the published method, sharing nothing with the CUDA library.

Readings (the paper names the method and gives no table):
  * A cell is the cube of 8 lattice voxels i + {0,1}^3; it is polygonised only
    when all 8 are defined (allocated, not chi), the rule the raycast uses for a
    defined sample. A corner is inside when T < 0 (Eq. 1: negative inside).
  * The surface crosses an edge whose corners differ in inside-ness, at the
    linear zero of T along it.
  * On each face of the cell the crossings pair up into segments; a face with
    four crossings (two inside corners diagonal to each other) pairs each
    inside corner's two edges, so the inside corners stay apart. A face decision
    depends only on that face, so two cells sharing it agree and the surface is
    closed.
  * Each segment is directed so that the inside corner it cuts off lies on the
    side that makes the polygon's normal point from inside to outside (towards
    growing T); the directed segments chain into loops, each loop starts at its
    smallest edge number and is split into the fan (v0, v_k, v_k+1).
  * Edge numbering: corners c = x + 2y + 4z; edges 0-3 run along x from corners
    0, 2, 4, 6; edges 4-7 along y from corners 0, 1, 4, 5; edges 8-11 along z
    from corners 0, 1, 2, 3.
"""
from __future__ import annotations

import itertools

import numpy as np

CORNER = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], np.float64)


def _edges():
    out = []
    for axis, step in ((0, 1), (1, 2), (2, 4)):
        starts = [c for c in range(8) if not (c & step)]
        out += [(c, c + step) for c in starts]
    return out


EDGES = _edges()           # 12 (corner a, corner b) pairs, a < b
EDGE_OF = {frozenset(e): k for k, e in enumerate(EDGES)}


def _faces():
    """Six faces: (outward normal, corners in cyclic order)."""
    faces = []
    for axis in range(3):
        for side in (0, 1):
            cs = [c for c in range(8) if CORNER[c, axis] == side]
            centre = CORNER[cs].mean(0)
            # cyclic order by angle around the face centre in the face plane
            u, v = [a for a in range(3) if a != axis]
            cs.sort(key=lambda c: np.arctan2(CORNER[c, v] - centre[v], CORNER[c, u] - centre[u]))
            n = np.zeros(3)
            n[axis] = 1.0 if side else -1.0
            faces.append((n, cs))
    return faces


FACES = _faces()


def case_polygons(inside):
    """Loops of edge numbers for one cell, given its 8 inside flags."""
    segs = {}
    for n, cs in FACES:
        k = len(cs)
        crossed = [EDGE_OF[frozenset((cs[i], cs[(i + 1) % k]))] for i in range(k)
                   if inside[cs[i]] != inside[cs[(i + 1) % k]]]
        if not crossed:
            continue
        if len(crossed) == 2:
            ins = [c for c in cs if inside[c]]
            pairs = [(crossed[0], crossed[1], ins[0])]
        else:
            pairs = []
            for i, c in enumerate(cs):
                if inside[c]:
                    prev_e = EDGE_OF[frozenset((cs[i - 1], c))]
                    next_e = EDGE_OF[frozenset((c, cs[(i + 1) % k]))]
                    pairs.append((prev_e, next_e, c))
        for e1, e2, corner in pairs:
            A = CORNER[list(EDGES[e1])].mean(0)
            B = CORNER[list(EDGES[e2])].mean(0)
            I = CORNER[corner]
            if np.dot(np.cross(B - A, I - A), n) > 0:
                e1, e2 = e2, e1
            segs[e1] = e2
    loops = []
    left = dict(segs)
    while left:
        start = min(left)
        loop = [start]
        nxt = left.pop(start)
        while nxt != start:
            loop.append(nxt)
            nxt = left.pop(nxt)
        loops.append(loop)
    return loops


def case_triangles(inside):
    """Triangles (edge-number triples) of one cell."""
    tris = []
    for loop in case_polygons(inside):
        i0 = loop.index(min(loop))
        loop = loop[i0:] + loop[:i0]
        for k in range(1, len(loop) - 1):
            tris.append((loop[0], loop[k], loop[k + 1]))
    return tris


def mesh(T: np.ndarray, origin, voxel_size):
    """Triangles (n, 3, 3) in world coordinates of a lattice field T (nx, ny, nz)
    with NaN where undefined: voxel i sits at origin + i * voxel_size."""
    T = np.asarray(T, np.float64)
    nx, ny, nz = T.shape
    out = []
    cache = {}
    s = float(voxel_size)
    org = np.asarray(origin, np.float64)
    for i, j, k in itertools.product(range(nx - 1), range(ny - 1), range(nz - 1)):
        vals = T[i:i + 2, j:j + 2, k:k + 2]
        if np.isnan(vals).any():
            continue
        v8 = np.array([vals[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)])
        inside = tuple(bool(x < 0) for x in v8)
        if all(inside) or not any(inside):
            continue
        tris = cache.get(inside)
        if tris is None:
            tris = cache[inside] = case_triangles(inside)
        base = np.array([i, j, k], np.float64)
        for tri in tris:
            pts = []
            for e in tri:
                a, b = EDGES[e]
                t = v8[a] / (v8[a] - v8[b])
                pts.append(org + (base + CORNER[a] + t * (CORNER[b] - CORNER[a])) * s)
            out.append(pts)
    return np.array(out, np.float64).reshape(-1, 3, 3)


def mesh_from_export(coords, T_blocks, grid_dim, origin, voxel_size):
    """Marching cubes over an exported sparse volume (block coordinates (n, 3),
    T (n, 512), NaN = chi): the blocks are scattered into a dense lattice
    covering their bounding box (unallocated = undefined)."""
    coords = np.asarray(coords, np.int64)
    lo = coords.min(0)
    hi = coords.max(0) + 1
    shape = tuple(int(x) for x in (hi - lo) * 8)
    dense = np.full(shape, np.nan)
    for b, c in enumerate(coords):
        blk = np.asarray(T_blocks[b], np.float64).reshape(8, 8, 8)     # [z][y][x]
        o = (c - lo) * 8
        dense[o[0]:o[0] + 8, o[1]:o[1] + 8, o[2]:o[2] + 8] = blk.transpose(2, 1, 0)
    org = np.asarray(origin, np.float64) + lo * 8 * float(voxel_size)
    return mesh(dense, org, voxel_size)
