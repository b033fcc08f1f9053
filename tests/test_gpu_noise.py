"""Hierarchical noise: every hypothesis scored under a grid of noise settings in one fused
pass (rendered once), and the likelihood with the noise marginalised over the grid, against
the FP64 oracle scoring each setting separately."""
import numpy as np
import pytest

from _scenes import gpu_context, jitter_poses, observed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRIDS = [(0, [0.0025, 0.005, 0.01], [0.001, 0.01, 0.1], 1),
         (1, [0.002, 0.003, 0.006], [0.01, 0.1], 2),
         (0, [0.005], [0.01], 1)]


@pytest.mark.parametrize("scene_name", ["single_object", "tabletop"])
@pytest.mark.parametrize("kind,radii,pouts,w", GRIDS)
def test_noise_grid_matches_oracle(orc, request, scene_name, kind, radii, pouts, w):
    from paper_2312_08715_gb300 import b3d
    wl = request.getfixturevalue(scene_name)
    sc = wl.scene
    obs = observed(orc, wl)
    poses = jitter_poses(np.random.default_rng(13), wl.hidden, 60, trans=0.01, rot_deg=5)
    G = len(radii) * len(pouts)
    logw = np.log(np.linspace(1, 2, G) / np.linspace(1, 2, G).sum())
    ref = orc.score_noise(sc, wl.slot, poses, kind, radii, pouts, w, obs, log_weight=logw)
    ctx = gpu_context(sc, obs)
    grid = b3d.noise_grid(kind, radii, pouts, half_window=w, log_weight=logw)
    ll, marg = ctx.score_noise(wl.slot, poses, grid)
    ctx.sync()
    ll, marg = ll.cpu().numpy().astype(np.float64), marg.cpu().numpy().astype(np.float64)
    # every setting: within 1e-4 * scale + the oracle's FP32-decision bound, and at least 90%
    # within 1e-4 * scale alone (the parity bar of the single-setting score)
    err = np.abs(ll - ref["ll"])
    tol = 1e-4 * ref["scale"] + ref["bound"]
    assert (err <= tol).all(), (err.max(), np.argwhere(err > tol)[:5])
    assert (err <= 1e-4 * ref["scale"]).mean() >= 0.9
    # log-sum-exp moves by at most the largest change of its terms (plus FP32 rounding of it)
    assert (np.abs(marg - ref["marginal"]) <= tol.max(axis=1) + 1e-6 * np.abs(ref["marginal"])).all()
    # one setting of the grid scored alone agrees with the single-setting kernel
    plain = ctx.score(wl.slot, poses, dict(kind=kind, radius=radii[0], p_outlier=pouts[0], half_window=w))
    np.testing.assert_allclose(ll[:, 0], plain.cpu().numpy(), rtol=2e-6)
    ctx.close()
