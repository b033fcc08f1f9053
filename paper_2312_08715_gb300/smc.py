"""SMC over the number of objects (Sec. III-B, Eq. 2 and 3) on the device.

Each of the M particles is a scene hypothesis with its own library context. At step k every
particle proposes object k's pose with its own single-sample coarse-to-fine search (one
batched launch over all particles, path density as log q), re-scores its scene at the
proposed pose (one batched launch) and updates its log weight:

    W = LL_1(x) - log q(x_1),    W += LL_k(x_1..k) - LL_{k-1}(x_1..k-1) - log q(x_k),

uniform priors being constants that cancel between particles. When the effective sample
size falls below ``ess_frac * M`` the particles are resampled in proportion to their weights
(the library's log-sum-exp + resampling, draws of stage k) and every weight becomes their
mean. The weight arithmetic is a few elementwise operations on M device scalars; every
render, score, normalisation and draw runs in the library's kernels.

Seeds: particle j draws its step-k proposal with ``seed + 1000 k + j``.
"""
from __future__ import annotations

import math

import numpy as np

from . import b3d


class SceneSMC:
    """Particles over a scene whose objects 0 .. n_fixed-1 are known and whose next objects
    are placed one per step. meshes: synth.Mesh list (fixed first, then those to place);
    poses: [n, 4, 4] host, the fixed objects' poses (the others are overwritten)."""

    def __init__(self, cam, meshes, poses, closed, n_fixed, m, device=0):
        import torch
        self.torch = torch
        self.cam, self.n_fixed, self.m = cam, int(n_fixed), int(m)
        self.n_obj = len(meshes)
        self.host_poses = np.array(poses, np.float32).reshape(self.n_obj, 4, 4)
        self.ctxs = [b3d.Context(device) for _ in range(self.m)]
        self.ids = [[c.load_mesh(mesh, closed=cl) for mesh, cl in zip(meshes, closed)] for c in self.ctxs]
        self.owner = b3d.Context(device)
        self.dev = torch.device("cuda", device)

    def close(self):
        for c in self.ctxs + [self.owner]:
            c.close()

    def set_tuning(self, **t):
        b3d.b3d_set_tuning(self.owner.h, **t)

    def run(self, obs_depth, centres, G, lik: dict, stages, seed, ess_frac=0.5):
        """Place len(centres) objects. Returns poses [M, K, 4, 4] (device), log weights [M]
        (device), the log evidence estimate, and per step the ESS and whether it resampled."""
        t = self.torch
        M, K, f = self.m, len(centres), self.n_fixed
        obs = t.as_tensor(np.ascontiguousarray(obs_depth, np.float32), device=self.dev)
        P = t.zeros((M, K, 4, 4), dtype=t.float32, device=self.dev)
        logw = t.zeros(M, dtype=t.float64, device=self.dev)
        ll_prev = t.zeros(M, dtype=t.float64, device=self.dev)
        part = t.empty((M, 1, 4, 4), dtype=t.float32, device=self.dev)
        pw = t.empty((M, 1), dtype=t.float32, device=self.dev)
        pq = t.empty((M, 1), dtype=t.float32, device=self.dev)
        ll = t.empty((M, 1), dtype=t.float32, device=self.dev)
        lk = b3d.lik_params(**lik)
        stream = self.owner.stream
        info = []
        for k in range(K):
            slot = f + k
            for j, c in enumerate(self.ctxs):
                b3d.b3d_set_scene(c.h, b3d.intrinsics(self.cam), self.ids[j][:slot + 1], self.host_poses[:slot + 1],
                                  obs, stream)
                for i in range(k):
                    b3d.b3d_set_object_pose_dev(c.h, f + i, P[j, i], stream)
            items = [b3d.c2f_item(c.h, slot, centres[k], b3d.schedule(stages, 1, seed + 1000 * k + j, G, True),
                                  part[j], pw[j], pq[j]) for j, c in enumerate(self.ctxs)]
            b3d.b3d_enumerate_multi(self.owner.h, items, lk, stream)
            P[:, k] = part[:, 0]
            for j, c in enumerate(self.ctxs):
                b3d.b3d_set_object_pose_dev(c.h, slot, P[j, k], stream)
            b3d.b3d_score_multi(self.owner.h, [(c.h, slot, 1, P[j, k], ll[j]) for j, c in enumerate(self.ctxs)], lk,
                                stream)
            llk = ll[:, 0].double()
            logw += llk - ll_prev - pq[:, 0].double()
            ll_prev = llk
            z = t.logsumexp(logw, 0)
            ess = float(t.exp(2 * z - t.logsumexp(2 * logw, 0)))
            resampled = ess < ess_frac * M
            if resampled:
                idx = t.empty(M, dtype=t.int32, device=self.dev)
                lz = t.empty(1, dtype=t.float32, device=self.dev)
                lq = t.empty(M, dtype=t.float32, device=self.dev)
                lw32 = logw.float().contiguous()
                b3d.b3d_lse_resample(self.owner.h, M, lw32, M, seed, k, lz, idx, lq, stream)
                P = P[idx.long()].contiguous()
                ll_prev = ll_prev[idx.long()]
                logw = t.full_like(logw, float(z) - math.log(M))
            info.append(dict(ess=ess, resampled=bool(resampled)))
        z = t.logsumexp(logw, 0)
        return P, logw, float(z) - math.log(M), info
