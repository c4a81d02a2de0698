"""The library's marching-cubes case table (tsdf_mesh_case, built on the host
from the published construction) against the marching-cubes oracle, which
builds each pattern's polygons independently: the same triangles, edge by
edge, for all 256 corner patterns (CPU only)."""
from oracle import mesh as omesh
from paper_1311_7194_b300 import tsdf


def test_case_table_equals_oracle_for_every_pattern():
    tsdf.load()
    worst = 0
    for pattern in range(256):
        inside = tuple(bool(pattern >> c & 1) for c in range(8))
        assert tsdf.mesh_case(pattern) == omesh.case_triangles(inside), pattern
        worst = max(worst, len(omesh.case_triangles(inside)))
    assert worst <= 8
