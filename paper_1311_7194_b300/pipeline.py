"""Per-frame live fusion loop over the C ABI (section "Pipeline Overview": scene
rendering, registration, fusion per acquired depth map; registration is outside
this library, so each frame is fused at its given pose and the fused model is
raycast at that pose for the next frame's alignment).

``FusionPipeline.step`` enqueues allocate -> integrate -> raycast for one depth
map already on the device; ``step_host`` starts from a host depth map: with a
graph, the library copies it (tsdf_graph_launch_host: a private copy stream and
two staging sets, so the copy overlaps the previous step); without one, it is
copied into one of two device staging buffers on the step's stream. Nothing
here synchronises: results are read by the caller when needed.
"""
from __future__ import annotations

from typing import Optional

import torch

from . import tsdf


class FusionPipeline:
    """``graph=True`` runs each step as one CUDA graph launch (tsdf_graph_*):
    the same results, without per-kernel launch gaps."""

    def __init__(self, volume: tsdf.Volume, intr, device: Optional[torch.device] = None, graph: bool = False):
        self.volume = volume
        self.intr = intr
        self.graph = tsdf.Graph(volume, intr, 1) if graph else None
        dev = device or torch.device("cuda", torch.cuda.current_device())
        H, W = intr.height, intr.width
        self.depth_map = torch.empty((H, W), dtype=torch.float32, device=dev)
        self.normal_map = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
        self.vertex_map = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
        self._staging = [torch.empty((H, W), dtype=torch.float32, device=dev) for _ in range(2)]
        self._k = 0

    @property
    def maps(self):
        return self.depth_map, self.normal_map, self.vertex_map

    def step(self, depth: torch.Tensor, pose, variance: Optional[torch.Tensor] = None, stream=None):
        """Fuse one device depth map at ``pose`` and raycast the model at ``pose``."""
        if self.graph is not None:
            self.graph.launch([depth], [pose], self.maps, None if variance is None else [variance], stream)
            return
        self.volume.allocate(depth, self.intr, pose, stream)
        self.volume.integrate(depth, self.intr, pose, variance, stream)
        self.volume.raycast(self.intr, pose, out=self.maps, stream=stream)

    def step_host(self, depth_host: torch.Tensor, pose, stream=None):
        """``step`` from a (pinned) host depth map; keep it unchanged until the
        step's work on the stream has completed."""
        if self.graph is not None:
            self.graph.launch_host([depth_host], [pose], self.maps, stream)
            return
        buf = self._staging[self._k & 1]
        self._k += 1
        s = torch.cuda.current_stream() if stream is None else stream
        with torch.cuda.stream(s):
            buf.copy_(depth_host, non_blocking=True)
        self.step(buf, pose, stream=s)
