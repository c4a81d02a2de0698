"""tsdf_raycast_trace: the traced raycast takes the same rays and crossings as
tsdf_raycast, leaves the volume untouched, and its counts are consistent."""
import numpy as np
import pytest
import torch

from paper_1311_7194_b300 import synth, tsdf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1311_7194_b300 import build
    build.build()
    torch.cuda.set_device(0)


@pytest.mark.parametrize("storage", [tsdf.STORAGE_F32, tsdf.STORAGE_F16], ids=["f32", "f16"])
def test_trace_counts_are_consistent(storage):
    seq = synth.room_sequence(n_frames=6, width=157, height=117, grid_dim=512, voxel_size=6e-3,
                              block_capacity=1 << 16)
    vol = tsdf.Volume.from_params(seq.volume, storage=storage)
    for k in range(seq.n_frames):
        vol.fuse(torch.from_numpy(seq.depth[k]).cuda(), seq.intr, seq.poses[k])
    pose = seq.poses[-1]
    before = [t.cpu().numpy() for t in vol.raycast(seq.intr, pose)]
    hits = vol.stats()["rays_hit"]
    c = vol.raycast_trace(seq.intr, pose)
    after = [t.cpu().numpy() for t in vol.raycast(seq.intr, pose)]
    for a, b in zip(before, after):                   # tracing changed nothing
        assert np.array_equal(np.isnan(a), np.isnan(b)) and np.array_equal(a[~np.isnan(a)], b[~np.isnan(b)])
    W, H = seq.intr.width, seq.intr.height
    assert c["rays"] == W * H
    assert c["rays_hit"] == hits > 1000
    # every hit takes six normal samples after its march; every sample inside the
    # grid reads at least one table entry; sectors are bounded by what was read
    assert c["samples"] >= 6 * c["rays_hit"] + c["rays_hit"]
    assert c["table_lookups"] >= c["rays_hit"]
    bytes_T = 4 if storage == tsdf.STORAGE_F32 else 2
    n_blocks = vol.stats()["n_blocks"]
    assert 0 < c["t_sectors"] <= n_blocks * 512 * bytes_T // 32
    assert c["t_sectors"] <= 8 * c["samples"]
    assert 0 < c["table_sectors"] <= c["table_lookups"]
    assert c["table_sectors"] <= (512 // 8) ** 3 // 8
    # the phase counts add up to the samples taken
    assert c["samples"] == c["march_samples"] + c["rescan_samples"] + c["refine_samples"] + c["normal_samples"]
    assert c["normal_samples"] <= 6 * c["rays_hit"]
    assert c["rescan_samples"] <= 16 * c["rescans"]
    assert c["refine_samples"] <= 10 * c["rays_hit"]
    assert c["march_samples"] >= c["rays_hit"] and c["skips"] <= c["march_samples"]
