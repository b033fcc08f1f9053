"""Camera-pose tracking (Sec. IV, Table 1): per frame, a coarse-to-fine search over camera
poses around the previous estimate. Each stage renders every hypothesised camera's view of
the whole scene (b3d_render_camera_batch), scores the images (b3d_score_depth_batch),
normalises and draws (b3d_lse_resample); the best drawn cell centres the next stage, and
the frame's estimate is the best drawn cell of all stages (each grid contains its centre,
but a stage's draws need not include it). Argument marshalling and the
choice of the best drawn cell only; every render, score, normalisation and draw runs in the
library.
"""
from __future__ import annotations

import numpy as np

from . import b3d


class CameraTracker:
    """Scene meshes at their world poses; tracks the camera_from_world pose."""

    def __init__(self, cam, meshes, world_poses, closed, device=0):
        import torch
        self.torch = torch
        self.ctx = b3d.Context(device)
        self.cam = cam
        self.ids = [self.ctx.load_mesh(m, closed=c) for m, c in zip(meshes, closed)]
        self.world = np.array(world_poses, np.float32).reshape(-1, 4, 4)
        self.dev = torch.device("cuda", device)
        self._bufs = {}

    def close(self):
        self.ctx.close()

    def _buf(self, n):
        t = self.torch
        if n not in self._bufs:
            H, W = self.cam.height, self.cam.width
            self._bufs[n] = (t.empty((n, 4, 4), dtype=t.float32, device=self.dev),
                             t.empty((n, H, W), dtype=t.float32, device=self.dev),
                             t.empty(n, dtype=t.float32, device=self.dev))
        return self._bufs[n]

    def frame(self, depth, prev, stages, lik, m, seed):
        """One frame: observed depth [H, W] (host), the search centre prev [4, 4] (host; the
        previous estimate, or a prediction from it). lik: one likelihood for every stage, or
        a list with one per stage (coarse stages may score with a wider inlier radius).
        Returns the new estimate [4, 4] (host) and its score."""
        t = self.torch
        ctx = self.ctx
        obs = t.as_tensor(np.ascontiguousarray(depth, np.float32), device=self.dev)
        b3d.b3d_set_scene(ctx.h, b3d.intrinsics(self.cam), self.ids, self.world, obs, ctx.stream)
        centre = np.asarray(prev, np.float32)
        liks = [b3d.lik_params(**(lik[k] if isinstance(lik, (list, tuple)) else lik)) for k in range(len(stages))]
        idx = t.empty(m, dtype=t.int32, device=self.dev)
        logz = t.empty(1, dtype=t.float32, device=self.dev)
        logq = t.empty(m, dtype=t.float32, device=self.dev)
        best_pose, best_ll = centre, -np.inf
        for k, st in enumerate(stages):
            n = st.n_per_axis ** 3 * st.n_rot
            poses, depth_buf, ll = self._buf(n)
            b3d.b3d_expand_hypotheses(ctx.h, centre, np.eye(3, dtype=np.float32), b3d.stage_params(st), poses, ctx.stream)
            b3d.b3d_render_camera_batch(ctx.h, n, poses, depth_buf, None, ctx.stream)
            b3d.b3d_score_depth_batch(ctx.h, -1, n, depth_buf, None, liks[k], ll, ctx.stream)
            b3d.b3d_lse_resample(ctx.h, n, ll, m, seed, k, logz, idx, logq, ctx.stream)
            drawn = idx.long()
            best = drawn[t.argmax(ll[drawn])]
            centre = poses[best].cpu().numpy()
            v = float(ll[best])
            if k == len(stages) - 1 or (v > best_ll and liks[k].radius == liks[-1].radius):
                # the best drawn cell among the stages scored like the last one
                if v > best_ll or k == len(stages) - 1 and liks[k].radius != liks[max(k - 1, 0)].radius:
                    best_pose, best_ll = centre, v
        return best_pose, best_ll


def predict(prev2, prev1):
    """Constant-velocity prediction of the next camera pose from the last two estimates
    (right-multiplied motion: prev1 (prev2^-1 prev1))."""
    a = np.asarray(prev2, np.float64)
    b = np.asarray(prev1, np.float64)
    return (b @ (np.linalg.inv(a) @ b)).astype(np.float32)
