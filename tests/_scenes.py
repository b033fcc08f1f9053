"""Scene set-up shared by the GPU tests: one seeded workload fed identically to the CUDA
library (through the C ABI) and to the CPU oracle."""
import numpy as np

from paper_2312_08715_gb300 import synth


def closed_flags(scene):
    """Voxel objects and boxes are closed solids; the table quad is not."""
    return [m.faces.shape[0] > 2 for m in scene.meshes]


def observed(orc, wl, clean=False):
    depth, _ = orc.render(wl.scene)
    return depth.astype(np.float32) if clean else synth.corrupt_depth(depth, wl.scene.camera.far, wl.draws)


def gpu_context(scene, obs, device=0, budget=0):
    from paper_2312_08715_gb300 import b3d
    ctx = b3d.Context(device, budget)
    ids = [ctx.load_mesh(m, closed=c) for m, c in zip(scene.meshes, closed_flags(scene))]
    ctx.set_scene(scene.camera, ids, scene.poses, obs)
    return ctx


def jitter_poses(rng, pose, n, trans=0.02, rot_deg=10.0):
    out = [np.asarray(pose, np.float64)]
    for _ in range(n - 1):
        P = np.array(pose, np.float64)
        ax = rng.normal(size=3)
        ax /= np.linalg.norm(ax)
        ang = np.radians(rng.uniform(-rot_deg, rot_deg))
        K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
        R = np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K
        P[:3, :3] = R @ P[:3, :3]
        P[:3, 3] += rng.uniform(-trans, trans, size=3)
        out.append(P)
    return np.stack(out).astype(np.float32)


def ll_tolerance(ref):
    """|LL_gpu - LL_oracle| <= 1e-4 * sum_i |l_i| + the oracle's ambiguity bound."""
    return 1e-4 * ref["scale"] + ref["bound"]
