"""The CUDA-graph step driver (tsdf_graph_*) against direct calls: the same
fused volume and raycast maps bit for bit, one graph instantiation for the whole
sequence (later steps update it in place)."""
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


def _maps(H, W):
    return (torch.empty((H, W), device="cuda"), torch.empty((H, W, 3), device="cuda"),
            torch.empty((H, W, 3), device="cuda"))


def _same_maps(a, b):
    for x, y in zip(a, b):
        x, y = x.cpu().numpy(), y.cpu().numpy()
        assert np.array_equal(np.isnan(x), np.isnan(y))
        m = ~np.isnan(x)
        assert np.array_equal(x[m], y[m])


def _same_volume(a, b):
    ea, eb = a.export(), b.export()
    assert np.array_equal(ea.coords, eb.coords) and np.array_equal(ea.alloc_frame, eb.alloc_frame)
    chi = np.isnan(ea.T)
    assert np.array_equal(chi, np.isnan(eb.T))
    assert np.array_equal(ea.T[~chi], eb.T[~chi]) and np.array_equal(ea.P[~chi], eb.P[~chi])


@pytest.mark.parametrize("K", [1, 4])
def test_graph_steps_equal_direct_calls(K):
    seq = synth.sphere_sequence(n_frames=8)
    H, W = seq.intr.height, seq.intr.width
    d = [torch.from_numpy(x).cuda() for x in seq.depth]
    direct = tsdf.Volume.from_params(seq.volume)
    graphed = tsdf.Volume.from_params(seq.volume)
    g = tsdf.Graph(graphed, seq.intr, K)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    g.set_events(ev)
    for k0 in range(0, seq.n_frames, K):
        if K == 1:
            direct.fuse(d[k0], seq.intr, seq.poses[k0])
        else:
            direct.integrate_batch(d[k0:k0 + K], seq.intr, seq.poses[k0:k0 + K])
        ref = direct.raycast(seq.intr, seq.poses[k0 + K - 1], out=_maps(H, W))
        got = g.launch(d[k0:k0 + K], seq.poses[k0:k0 + K], _maps(H, W))
        torch.cuda.synchronize()
        _same_maps(ref, got)
        assert ev[0].elapsed_time(ev[3]) > 0.0
    assert g.instantiations == 1
    graphed.check()
    _same_volume(direct, graphed)
    assert graphed.stats()["frames"] == seq.n_frames
    g.close()


def test_graph_rejects_bad_arguments():
    seq = synth.sphere_sequence(n_frames=1)
    vol = tsdf.Volume.from_params(seq.volume)
    for K in (0, 9):
        with pytest.raises(tsdf.TsdfError):
            tsdf.Graph(vol, seq.intr, K)


@pytest.mark.parametrize("K,pinned", [(1, True), (1, False), (4, True)], ids=["K1-pinned", "K1-pageable", "K4-pinned"])
def test_host_input_steps_equal_device_input_steps(K, pinned):
    """tsdf_graph_launch_host: the library's copy (private stream, two staging
    sets used alternately) gives the same volume and maps bit for bit as steps
    fed from device maps; steps are enqueued back to back, so a staging set is
    reused while earlier steps may still run."""
    seq = synth.sphere_sequence(n_frames=12)
    H, W = seq.intr.height, seq.intr.width
    d = [torch.from_numpy(x).cuda() for x in seq.depth]
    host = torch.from_numpy(seq.depth)
    host = host.pin_memory() if pinned else seq.depth
    dev_vol = tsdf.Volume.from_params(seq.volume)
    host_vol = tsdf.Volume.from_params(seq.volume)
    gd, gh = tsdf.Graph(dev_vol, seq.intr, K), tsdf.Graph(host_vol, seq.intr, K)
    ref_maps, got_maps = [], []
    for k0 in range(0, seq.n_frames, K):
        ref_maps.append(gd.launch(d[k0:k0 + K], seq.poses[k0:k0 + K], _maps(H, W)))
        got_maps.append(gh.launch_host([host[k] for k in range(k0, k0 + K)], seq.poses[k0:k0 + K], _maps(H, W)))
    torch.cuda.synchronize()
    for a, b in zip(ref_maps, got_maps):
        _same_maps(a, b)
    assert gh.instantiations == 1
    host_vol.check()
    _same_volume(dev_vol, host_vol)
    assert host_vol.stats()["frames"] == seq.n_frames
    gd.close()
    gh.close()


def test_host_input_rejects_bad_arguments():
    seq = synth.sphere_sequence(n_frames=1)
    vol = tsdf.Volume.from_params(seq.volume)
    g = tsdf.Graph(vol, seq.intr, 1)
    H, W = seq.intr.height, seq.intr.width
    with pytest.raises(ValueError):            # wrong size
        g.launch_host([np.zeros((H, W + 1), np.float32)], [seq.poses[0]], _maps(H, W))
    with pytest.raises(ValueError):            # a device tensor where a host map belongs
        g.launch_host([torch.zeros((H, W), device="cuda")], [seq.poses[0]], _maps(H, W))
    bad = np.array(seq.poses[0], dtype=np.float64).copy()
    bad[0, 3] = np.nan
    with pytest.raises(tsdf.TsdfError):
        g.launch_host([seq.depth[0]], [bad], _maps(H, W))
    assert vol.stats()["frames"] == 0
    g.close()
