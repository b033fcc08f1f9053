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


def check_ll(got, ref, what, tight_frac=0.9):
    """Every hypothesis within 1e-4 * scale + the oracle's FP32-decision bound, and most
    of them within 1e-4 * scale alone (the bound is not what makes them pass)."""
    tol = ll_tolerance(ref)
    err = np.abs(np.asarray(got, np.float64) - ref["ll"])
    bad = np.nonzero(err > tol)[0]
    assert bad.size == 0, f"{what}: {bad.size} hypotheses outside tolerance, e.g. {bad[:5]} err {err[bad[:5]]} tol {tol[bad[:5]]}"
    tight = err <= 1e-4 * ref["scale"]
    print(f"{what}: n={err.size} max|dLL|={err.max():.3g} median={np.median(err):.3g} "
          f"tight={tight.mean():.3f} flagged={np.mean(ref['bound'] > 0):.3f}")
    assert tight.mean() >= tight_frac, f"{what}: only {tight.mean():.2f} of hypotheses within 1e-4 * scale"
    return err


def check_grad(dpose, dsigma, dpout, ref, gbound, what):
    """Per hypothesis, each gradient (the se(3) pose gradient by its norm, dLL/dsigma,
    dLL/dp_out) within 1e-3 relative of the FP64 oracle plus the oracle's bound on what FP32
    visibility decisions can move it (oracle.score_grad_bound: the exact change of switching
    each flagged pixel to each of its alternatives, summed); and every hypothesis whose bound
    is zero within 1e-3 alone. Returns the fraction of hypotheses within 1e-3 alone."""
    rows = np.linalg.norm
    parts = (("pose", dpose, ref["dpose"], rows(gbound[:, :6], axis=1), lambda a: rows(a, axis=1)),
             ("sigma", dsigma, ref["dsigma"], gbound[:, 6], np.abs),
             ("p_out", dpout, ref["dpout"], gbound[:, 7], np.abs))
    tight_all = np.ones(len(ref["ll"]), bool)
    for name, g, r, b, norm in parts:
        err = norm(np.asarray(g, np.float64) - r)
        scale = norm(r)
        bad = np.nonzero(err > 1e-3 * scale + b)[0]
        assert bad.size == 0, f"{what} {name}: hypotheses {bad} rel err {(err / scale)[bad]} bound {(b / scale)[bad]}"
        tight = err <= 1e-3 * scale
        loose = np.nonzero(~tight & (b == 0))[0]
        assert loose.size == 0, f"{what} {name}: unbounded hypotheses {loose} rel err {(err / scale)[loose]}"
        print(f"{what} {name}: max rel {np.max(err / scale):.2e} median {np.median(err / scale):.2e} "
              f"within 1e-3 alone {tight.mean():.3f} bounded {np.mean(b > 0):.3f}")
        tight_all &= tight
    return float(tight_all.mean())


def se3_exp_fp64(xi):
    """Exp of twists xi [n, 6] = (v, w) as 4x4 matrices in FP64: the matrix exponential of
    [[W, v], [0, 0]] with W = [w]x (scipy's expm)."""
    from scipy.linalg import expm
    xi = np.asarray(xi, np.float64).reshape(-1, 6)
    out = np.empty((xi.shape[0], 4, 4))
    for i, (v0, v1, v2, w0, w1, w2) in enumerate(xi):
        A = np.array([[0, -w2, w1, v0], [w2, 0, -w0, v1], [-w1, w0, 0, v2], [0, 0, 0, 0]])
        out[i] = expm(A)
    return out
