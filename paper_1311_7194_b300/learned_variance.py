"""Training and use of the learned measurement-variance network.

Residual harvesting, the network's forward and backward passes and the Adam
updates run in libtsdf's kernels (tsdf_mlp_*); this module only orders the
calls, draws minibatch indices and keeps the buffers (torch tensors).

Training data: for each frame k of a training sequence, the model fused from
frames 0..k-1 (quadratic variances) is raycast at pose k; the residual between
the measured depth and that prediction, at pixels where both exist and the
residual lies within 4 truncation distances (wider than the band, so that the
heavy errors of poor pixels are seen), is a sample of the measurement error the
variance should describe. The network minimises the Gaussian negative
log-likelihood (out + s exp(-out)) / 2, s = r^2 / p_quad, i.e. it learns
log(E[r^2] / p_quad) as a function of the pixel's neighbourhood.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Iterable, List, Optional

import numpy as np
import torch

from . import tsdf

N_PARAMS = 1985
LOG4 = float(np.log(4.0))
LOG64 = float(np.log(64.0))     # the network's output is used within [-LOG4, LOG64]


def _p(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def bf16_bits(w: np.ndarray) -> np.ndarray:
    """float32 -> bfloat16 bits (round to nearest even)."""
    f = np.ascontiguousarray(w, np.float32).view(np.uint32).astype(np.uint64)
    return (((f + 0x7FFF + ((f >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint16)


def bf16_values(bits: np.ndarray) -> np.ndarray:
    return (np.asarray(bits, np.uint16).astype(np.uint32) << 16).view(np.float32)


def init_weights(seed: int = 0) -> np.ndarray:
    """He-initialised float32 weights with a zero output layer (the untrained
    network reproduces the quadratic model exactly)."""
    rng = np.random.default_rng(seed)
    w = np.zeros(N_PARAMS, np.float32)
    w[:864] = rng.normal(0, np.sqrt(2.0 / 27), 864)
    w[896:896 + 1024] = rng.normal(0, np.sqrt(2.0 / 32), 1024)
    return w


@dataclass
class Dataset:
    feats: torch.Tensor     # (N, 27) float32, device
    s: torch.Tensor         # (N,) float32, device: r^2 / p_quad

    @property
    def n(self) -> int:
        return int(self.s.numel())


def harvest(sequences: Iterable, max_n: int = 2_000_000, frame_stride: int = 1) -> Dataset:
    """Residual samples from posed sequences (see the module docstring)."""
    lib = tsdf.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    feats = torch.empty((max_n, 27), dtype=torch.float32, device=dev)
    s = torch.empty(max_n, dtype=torch.float32, device=dev)
    count = torch.zeros(1, dtype=torch.int32, device=dev)
    for seq in sequences:
        vol = tsdf.Volume.from_params(seq.volume)
        H, W = seq.intr.height, seq.intr.width
        pred = (torch.empty((H, W), device=dev), torch.empty((H, W, 3), device=dev), torch.empty((H, W, 3), device=dev))
        K = tsdf.intrinsics(seq.intr)
        depth = torch.from_numpy(seq.depth).to(dev)
        for k in range(seq.n_frames):
            if k > 0 and k % frame_stride == 0:
                vol.raycast(seq.intr, seq.poses[k], out=pred)
                tsdf._check(lib.tsdf_mlp_harvest(vol.h, _p(depth[k]), _p(pred[0]), ctypes.byref(K), max_n, _p(feats),
                                                 _p(s), _p(count), _stream()), "tsdf_mlp_harvest")
            vol.fuse(depth[k], seq.intr, seq.poses[k])
        vol.check()
        vol.close()
    n = min(int(count.item()), max_n)
    return Dataset(feats[:n].clone(), s[:n].clone())


def train(data: Dataset, steps: int = 2000, batch: int = 4096, lr: float = 2e-3, seed: int = 0,
          w0: Optional[np.ndarray] = None, log_every: int = 100):
    """Adam on the NLL; returns (bfloat16 weight bits, [(step, mean loss)])."""
    lib = tsdf.load()
    dev = data.s.device
    w32 = torch.from_numpy(init_weights(seed) if w0 is None else np.asarray(w0, np.float32)).to(dev)
    wq = torch.from_numpy(bf16_bits(w32.cpu().numpy()).view(np.int16)).to(dev)
    m = torch.zeros(N_PARAMS, device=dev)
    v = torch.zeros(N_PARAMS, device=dev)
    grad = torch.zeros(N_PARAMS, device=dev)
    loss = torch.zeros(1, device=dev)
    rng = np.random.default_rng(seed + 1)
    B = min(batch, data.n)
    idx_all = torch.from_numpy(rng.integers(0, data.n, size=(steps, B), dtype=np.int32)).to(dev)
    history = []
    acc_loss, acc_n = 0.0, 0
    for t in range(1, steps + 1):
        tsdf._check(lib.tsdf_mlp_loss_grad(_p(wq), B, _p(idx_all[t - 1]), _p(data.feats), _p(data.s), _p(grad),
                                           _p(loss), _stream()), "tsdf_mlp_loss_grad")
        tsdf._check(lib.tsdf_mlp_adam(_p(w32), _p(wq), _p(m), _p(v), _p(grad), lr, 0.9, 0.999, 1e-8, 1.0 / B, t,
                                      _stream()), "tsdf_mlp_adam")
        if t % log_every == 0 or t == steps:
            acc_loss = float(loss.item())
            history.append((t, acc_loss / (B * (t - acc_n))))
            loss.zero_()
            acc_n = t
    return wq.cpu().numpy().view(np.uint16).copy(), history


def mean_loss(wq_bits: np.ndarray, data: Dataset) -> float:
    """Mean NLL (out + s exp(-out)) / 2 of a network over a dataset (GPU)."""
    lib = tsdf.load()
    dev = data.s.device
    wq = torch.from_numpy(np.asarray(wq_bits, np.uint16).view(np.int16)).to(dev)
    grad = torch.zeros(N_PARAMS, device=dev)
    loss = torch.zeros(1, device=dev)
    tsdf._check(lib.tsdf_mlp_loss_grad(_p(wq), data.n, None, _p(data.feats), _p(data.s), _p(grad), _p(loss),
                                       _stream()), "tsdf_mlp_loss_grad")
    return float(loss.item()) / data.n


def surface_errors(vol: tsdf.Volume, seq, poses: List[np.ndarray], scene) -> np.ndarray:
    """The scene's analytic signed distance at the raycast vertices of ``poses``
    (metres): how far the fused surface lies from the true one, per hit."""
    from . import synth
    errs = []
    for pose in poses:
        _, _, vert = vol.raycast(seq.intr, pose)
        v = vert.reshape(-1, 3)
        v = v[torch.isfinite(v[:, 0])]
        errs.append(synth.scene_sdf(scene, v.double()).cpu().numpy())
    return np.concatenate(errs)


def surface_error(vol: tsdf.Volume, seq, poses: List[np.ndarray], scene) -> dict:
    """Mean absolute and RMS surface error (metres) at the raycast vertices."""
    e = surface_errors(vol, seq, poses, scene)
    return {"mae": float(np.mean(np.abs(e))), "rms": float(np.sqrt(np.mean(e ** 2))), "hits": int(e.size)}
