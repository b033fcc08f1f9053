"""Pins of the FP64 CPU oracle to things other than itself: hand-derived images and closed
forms, special cases that reduce to a library routine, invariants, brute force on tiny
inputs and central finite differences. CPU only."""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, linalg
from scipy.spatial.transform import Rotation

from paper_2312_08715_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden_grid(name):
    rows = [ln.split() for ln in open(os.path.join(GOLD, name)) if ln.strip() and not ln.startswith("#")]
    return np.array(rows, dtype=np.float64)


def _closed(name):
    return json.load(open(os.path.join(GOLD, "closed_forms.json")))[name]


def _one_object_scene(mesh, pose, cam):
    return synth.Scene(cam, [mesh], np.asarray(pose, np.float32)[None].copy())


# ---------------------------------------------------------------------------------------
# Depth renderer
# ---------------------------------------------------------------------------------------

def test_cube_faceon_matches_hand_derived_image(orc):
    cam = synth.Camera(8, 8, 8.0, 8.0, 4.0, 4.0, 0.01, 2.0)
    mesh = synth.voxel_mesh([[0, 0, 0]], 0.2, origin=(-0.1, -0.1, -0.1))
    scene = _one_object_scene(mesh, synth.rigid(np.eye(3), [0, 0, 0.6]), cam)
    depth, tid = orc.render(scene)
    want = _golden_grid("cube_faceon_8x8.txt")
    # inputs are float32 (0.6 and -0.1 round by < 3e-8), the derivation is exact
    np.testing.assert_allclose(depth, want, rtol=0, atol=1e-7)
    assert ((tid >= 0) == (want < 2.0)).all()
    # covered pixels carry the -z face (triangles 8, 9 of the voxel), which faces the camera
    assert set(np.unique(tid[tid >= 0])) <= {8, 9}


def test_side_face_depth_is_ray_plane_intersection(orc):
    """Off-axis cube: pixels that see its -x side face have depth x_face / slope exactly."""
    cam = synth.Camera(128, 16, 64.0, 64.0, 64.0, 8.0, 0.01, 2.0)
    p = 0.1
    mesh = synth.voxel_mesh([[0, 0, 0]], p, origin=(-p / 2, -p / 2, -p / 2))
    tx, tz = 0.2, 0.6
    scene = _one_object_scene(mesh, synth.rigid(np.eye(3), [tx, 0, tz]), cam)
    depth, tid = orc.render(scene)
    f32 = lambda x: float(np.float32(x))
    # exact geometry of the float32 inputs: faces at f32(-p/2) + f32(t), f32(p/2) + f32(t)
    x_face = f32(-p / 2) + f32(tx)
    zf, zb = f32(-p / 2) + f32(tz), f32(p / 2) + f32(tz)
    half = f32(p / 2)
    n_side = 0
    for v in range(16):
        for u in range(128):
            su = (u + 0.5 - 64) / 64.0
            sv = (v + 0.5 - 8) / 64.0
            # the front face (z = zf) is hit iff the ray meets it inside the square
            if abs(su * zf - f32(tx)) <= half and abs(sv * zf) <= half:
                assert depth[v, u] == pytest.approx(zf, abs=1e-12)
                continue
            if su > 0:
                z = x_face / su
                if zf <= z <= zb and abs(sv * z) <= half:
                    n_side += 1
                    assert depth[v, u] == pytest.approx(z, rel=1e-12)
                    assert tid[v, u] in (0, 1)  # -x face triangles
                    continue
            assert tid[v, u] == -1 and depth[v, u] == 2.0
    assert n_side > 0


def test_pose_convention_rotation_and_translation(orc):
    """A small voxel at object x = +5 cm under a +90 deg rotation about z must land at
    camera y = +5 cm (below the centre row): catches a transposed rotation or a wrong
    translation slot."""
    cam = synth.Camera(64, 64, 64.0, 64.0, 32.0, 32.0, 0.01, 2.0)
    p = 0.01
    mesh = synth.voxel_mesh([[0, 0, 0]], p, origin=(0.05 - p / 2, -p / 2, -p / 2))
    Rz = Rotation.from_euler("z", 90, degrees=True).as_matrix()
    scene = _one_object_scene(mesh, synth.rigid(Rz, [0, 0, 0.5]), cam)
    depth, tid = orc.render(scene)
    vs, us = np.nonzero(tid >= 0)
    assert len(us) > 0
    # (0, 0.05, 0.5) projects to u = 32, v = 32 + 64 * 0.1 = 38.4
    assert us.mean() + 0.5 == pytest.approx(32.0, abs=0.6)
    assert vs.mean() + 0.5 == pytest.approx(38.4, abs=0.6)


def test_near_far_and_ties(orc):
    cam = synth.Camera(8, 8, 8.0, 8.0, 4.0, 4.0, 0.4, 2.0)
    mesh = synth.voxel_mesh([[0, 0, 0]], 0.2, origin=(-0.1, -0.1, -0.1))
    # front face at 0.35 < near: triangles with a vertex in front of near are dropped;
    # the back face's triangles (all vertices at z = 0.55) remain and are seen from inside.
    scene = _one_object_scene(mesh, synth.rigid(np.eye(3), [0, 0, 0.45]), cam)
    depth, tid = orc.render(scene)
    assert set(np.unique(tid[tid >= 0])) <= {10, 11}  # +z face triangles
    assert np.allclose(depth[tid >= 0], 0.55)
    # beyond far: nothing rendered
    scene = _one_object_scene(mesh, synth.rigid(np.eye(3), [0, 0, 2.5]), cam)
    depth, tid = orc.render(scene)
    assert (tid == -1).all() and (depth == 2.0).all()
    # two coincident objects: equal depths go to the smaller global triangle id
    scene = synth.Scene(cam, [mesh, mesh], np.stack([synth.rigid(np.eye(3), [0, 0, 0.8])] * 2).astype(np.float32))
    depth, tid = orc.render(scene)
    assert tid[tid >= 0].max() < 12


def test_object_order_is_irrelevant(orc, tabletop):
    sc = tabletop.scene
    d0, t0 = orc.render(sc)
    perm = [3, 0, 4, 1, 6, 2, 5]
    sc2 = synth.Scene(sc.camera, [sc.meshes[k] for k in perm], sc.poses[perm].copy())
    d1, t1 = orc.render(sc2)
    np.testing.assert_array_equal(d0, d1)
    # map permuted global ids back to the original numbering
    f0 = np.cumsum([0] + [m.n_faces for m in sc.meshes])
    f1 = np.cumsum([0] + [sc.meshes[k].n_faces for k in perm])
    back = np.full(t1.shape, -1)
    for new, old in enumerate(perm):
        sel = (t1 >= f1[new]) & (t1 < f1[new + 1])
        back[sel] = t1[sel] - f1[new] + f0[old]
    np.testing.assert_array_equal(back, t0)


# ---------------------------------------------------------------------------------------
# Likelihood
# ---------------------------------------------------------------------------------------

def test_frustum_volume_closed_form_and_quadrature(orc, single_object):
    cam = single_object.scene.camera
    g = _closed("frustum_volume_64x48_f60_near0.01_far2")
    V = orc.frustum_volume(cam)
    assert V == pytest.approx(g["value"], rel=g["rtol"])
    area = lambda z: (cam.width * z / cam.fx) * (cam.height * z / cam.fy)
    q, _ = integrate.quad(area, cam.near, cam.far)
    assert V == pytest.approx(q, rel=1e-12)


def test_self_score_closed_form(orc, single_object):
    sc = single_object.scene
    depth, tid = orc.render(sc)
    ell, cnt, _, _ = orc.pixel_loglik(sc.camera, single_object.lik, depth, tid, depth)
    assert (cnt == 1).all()
    g = _closed("self_score_64x48_r5mm_pout0.01_w1")
    assert ell.sum() == pytest.approx(g["value"], rel=g["rtol"])
    # the same through the per-hypothesis path
    res = orc.score(sc, 0, sc.poses[0][None], single_object.lik, depth, flags=False)
    assert res["ll"][0] == pytest.approx(g["value"], rel=g["rtol"])


def test_self_score_gaussian_limit(orc, single_object):
    """sigma = 1 mm << ray spacing (>= 6.9 mm): every S_i is one Gaussian peak."""
    sc = single_object.scene
    depth, tid = orc.render(sc)
    lk = dict(kind=1, radius=0.001, p_outlier=0.01, half_window=1)
    ell, _, ss, _ = orc.pixel_loglik(sc.camera, lk, depth, tid, depth)
    peak = (2 * math.pi * 0.001 ** 2) ** -1.5
    np.testing.assert_allclose(ss, peak, rtol=1e-9)
    V = 64 * 48 / 3600 * (8 - 1e-6) / 3
    assert ell.sum() == pytest.approx(3072 * math.log(0.01 / V + 0.99 * peak / 9), rel=1e-9)


@pytest.mark.parametrize("w", [1, 2])
def test_plane_counts_and_borders(orc, w):
    """Rendered = observed = the plane z = 1 seen by a 6x5 camera with f = 60: neighbour
    points are 1/60 m apart along rows and columns and sqrt(2)/60 diagonally. With
    r = 2 cm a pixel counts itself and its 4-neighbours inside the image."""
    cam = synth.Camera(6, 5, 60.0, 60.0, 3.0, 2.5, 0.01, 2.0)
    plane = np.ones((5, 6))
    lk = dict(kind=0, radius=0.02, p_outlier=0.25, half_window=w)
    ell, cnt, _, _ = orc.pixel_loglik(cam, lk, plane, np.zeros((5, 6), np.int32), plane)
    want = np.full((5, 6), 5)
    want[0, :] -= 1; want[-1, :] -= 1; want[:, 0] -= 1; want[:, -1] -= 1
    np.testing.assert_array_equal(cnt, want)
    V = 6 * 5 / 3600 * (8 - 1e-6) / 3
    K = (2 * w + 1) ** 2
    ball = 4 / 3 * math.pi * 0.02 ** 3
    np.testing.assert_allclose(ell, np.log(0.25 / V + 0.75 * want / (K * ball)), rtol=1e-12)
    # invalid observations are not scored; a 1/|y|-style normaliser is one flag away
    obs = plane.copy(); obs[2, 3] = 0.0; obs[1, 1] = np.nan
    ell2, _, _, _ = orc.pixel_loglik(cam, dict(lk, norm=30.0), plane, None, obs)
    assert np.isnan(ell2[2, 3]) and np.isnan(ell2[1, 1])
    sel = np.isfinite(ell2)
    np.testing.assert_allclose(ell2[sel], np.log(0.25 / V + 0.75 * want[sel] / (30.0 * ball)), rtol=1e-12)


def test_miss_mode_b_excludes_misses(orc):
    cam = synth.Camera(6, 5, 60.0, 60.0, 3.0, 2.5, 0.01, 2.0)
    far = np.full((5, 6), 2.0)
    tid = np.full((5, 6), -1, np.int32)
    lk = dict(kind=0, radius=0.02, p_outlier=0.25, half_window=1)
    _, cnt_a, _, _ = orc.pixel_loglik(cam, lk, far, tid, far)
    _, cnt_b, _, _ = orc.pixel_loglik(cam, dict(lk, miss_mode=1), far, tid, far)
    assert (cnt_a >= 1).all() and (cnt_b == 0).all()


def test_brute_force_argmax_tiny_grid(orc, single_object):
    """Noise-free observation of the hidden pose; a 3x3x3 grid (1 cm) around it. The hidden
    pose scores the self-score closed form and wins; every other cell scores less."""
    wl = single_object
    sc = wl.scene
    depth, _ = orc.render(sc)
    poses = orc.expand(wl.hidden, np.eye(3), 3, 0.01, np.eye(3)[None])
    res = orc.score(sc, 0, poses, wl.lik, depth, flags=False)
    assert int(np.argmax(res["ll"])) == 13
    assert res["ll"][13] == pytest.approx(_closed("self_score_64x48_r5mm_pout0.01_w1")["value"], rel=1e-7)
    assert (np.delete(res["ll"], 13) < res["ll"][13] - 100).all()


def test_hypothesis_order_invariance(orc, single_object):
    wl = single_object
    poses = orc.expand(wl.hidden, np.eye(3), 4, 0.01, np.eye(3)[None])
    obs = synth.corrupt_depth(orc.render(wl.scene)[0], 2.0, wl.draws)
    rng = np.random.default_rng(5)
    perm = rng.permutation(len(poses))
    a = orc.score(wl.scene, 0, poses, wl.lik, obs, flags=False)["ll"]
    b = orc.score(wl.scene, 0, poses[perm], wl.lik, obs, flags=False)["ll"]
    np.testing.assert_array_equal(a[perm], b)


# ---------------------------------------------------------------------------------------
# Log-sum-exp, Philox, resampling
# ---------------------------------------------------------------------------------------

def test_lse_against_long_double_and_special_cases(orc):
    rng = np.random.default_rng(1)
    ll = rng.normal(-5000, 40, size=10007)
    Z, logp = orc.lse(ll)
    m = np.max(ll)
    zl = np.longdouble(m) + np.log(np.sum(np.exp(ll.astype(np.longdouble) - np.longdouble(m))))
    assert Z == pytest.approx(float(zl), abs=1e-9)
    assert np.exp(logp).sum() == pytest.approx(1.0, abs=1e-12)
    Z2, _ = orc.lse(ll + 123.0)
    assert Z2 == pytest.approx(Z + 123.0, abs=1e-9)
    Zu, logpu = orc.lse(np.full(777, 3.5))
    np.testing.assert_allclose(logpu, -math.log(777), atol=1e-12)
    assert Zu == pytest.approx(3.5 + math.log(777))


def test_philox_matches_numpy(orc):
    """numpy's Philox is Philox4x64-10; it increments the counter before each block."""
    rng = np.random.default_rng(2)
    for _ in range(20):
        key = [int(x) for x in rng.integers(0, 2 ** 63, size=2, dtype=np.int64)]
        ctr = [int(x) for x in rng.integers(0, 2 ** 63, size=4, dtype=np.int64)]
        ref = np.random.Philox(key=key, counter=ctr).random_raw(4)
        nxt = list(ctr)
        nxt[0] += 1
        np.testing.assert_array_equal(orc.philox(nxt, key), ref)
    assert orc.uniform24(0xFFFFFFFFFFFFFFFF) == pytest.approx(1 - 2 ** -24)
    assert orc.uniform24(0) == 0.0


def test_resample_inverse_cdf_matches_searchsorted(orc):
    rng = np.random.default_rng(3)
    ll = rng.normal(0, 2, size=513)
    idx, logq, margin = orc.resample(ll, 300, seed=77, stage=2)
    w = np.exp(ll - ll.max())
    cdf = np.cumsum(w)
    for m in range(300):
        x = orc.philox([m, 2, 0, 0], [77, 0])[0]
        u = orc.uniform24(x)
        assert idx[m] == np.searchsorted(cdf, u * cdf[-1], side="right")
    Z, logp = orc.lse(ll)
    np.testing.assert_allclose(logq, logp[idx], atol=1e-12)
    assert (margin >= 0).all()


def test_resample_degenerate_and_chi2(orc):
    ll = np.full(50, -1e4)
    ll[17] = 0.0
    idx, _, _ = orc.resample(ll, 200, seed=1, stage=0)
    assert (idx == 17).all()
    p = np.array([0.1, 0.2, 0.3, 0.15, 0.25])
    idx, _, _ = orc.resample(np.log(p), 40000, seed=9, stage=1)
    counts = np.bincount(idx, minlength=5)
    from scipy.stats import chisquare
    assert chisquare(counts, 40000 * p).pvalue > 1e-4


# ---------------------------------------------------------------------------------------
# Coarse-to-fine grids
# ---------------------------------------------------------------------------------------

def test_fibonacci_rotations_are_minimal_arcs(orc):
    n = 200
    R = orc.rotation_set(0, n)
    phi = (1 + 5 ** 0.5) / 2
    for k in range(n):
        z = 1 - (2 * k + 1) / n
        rho = math.sqrt(1 - z * z)
        d = np.array([rho * math.cos(2 * math.pi * k / phi), rho * math.sin(2 * math.pi * k / phi), z])
        np.testing.assert_allclose(R[k] @ np.array([0, 0, 1.0]), d, atol=1e-12)
        ref, _ = Rotation.align_vectors([d], [[0, 0, 1.0]])
        np.testing.assert_allclose(R[k], ref.as_matrix(), atol=1e-9)


def test_perturbation_rotations(orc):
    """Kind 1 is a low-discrepancy set uniform in the ball of rotation vectors of radius
    rot_max, the identity first. Pinned by what such a set must satisfy: rotations within
    the radius, the moments of the uniform ball (P(|r| <= R/2) = 1/8, E|r| = 3R/4,
    E[r r^T] = R^2/5 I, E[r] = 0), and a covering radius within twice the radius of the
    ball's volume per point (the earlier set, whose angle and axis azimuth came from one
    golden-ratio sequence, left holes of 0.49 R at 2,048 members)."""
    assert np.array_equal(orc.rotation_set(1, 1, 0.2)[0], np.eye(3))
    for n, tmax in ((2048, math.radians(1.0)), (200, math.radians(10)), (4096, 0.3)):
        R = orc.rotation_set(1, n, tmax)
        assert np.array_equal(R[0], np.eye(3))
        np.testing.assert_allclose(np.einsum("nij,nkj->nik", R, R), np.broadcast_to(np.eye(3), R.shape), atol=1e-12)
        np.testing.assert_allclose(np.linalg.det(R), 1.0, atol=1e-12)
        rv = Rotation.from_matrix(R[1:]).as_rotvec()
        r = np.linalg.norm(rv, axis=1)
        assert r.max() <= tmax * (1 + 1e-9) and r.min() > 0
        tol = 3.0 / math.sqrt(n)  # a few standard errors of a random set; a uniform low-discrepancy set does better
        assert abs(np.mean(r <= tmax / 2) - 1 / 8) < tol
        assert abs(r.mean() / tmax - 0.75) < tol
        assert np.abs(rv.mean(axis=0)).max() / tmax < tol
        np.testing.assert_allclose(rv.T @ rv / len(rv) / (tmax ** 2 / 5), np.eye(3), atol=2 * tol)
        # coverage: seeded targets uniform in the ball of 0.9 R
        rng = np.random.default_rng(n)
        u = rng.normal(size=(300, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        targets = Rotation.from_rotvec(u * (0.9 * tmax * rng.random(300)[:, None] ** (1 / 3)))
        members = Rotation.from_matrix(R)
        nearest = max(np.linalg.norm((members.inv() * targets[i]).as_rotvec(), axis=1).min() for i in range(300))
        assert nearest < 2.0 * tmax * (4 * math.pi / (3 * n)) ** (1 / 3), nearest / tmax


def test_expand_grid_layout(orc):
    rng = np.random.default_rng(4)
    Rc = synth.random_rotation(rng)
    centre = synth.rigid(Rc, [0.1, -0.2, 0.7])
    G = synth.random_rotation(rng)
    rot = orc.rotation_set(1, 3, 0.2)
    P = orc.expand(centre, G, 10, 0.01, rot)
    assert P.shape == (3000, 4, 4)
    for h in [0, 555, 1555, 2999, 1234]:
        ir, rest = divmod(h, 1000)
        ix, rest = divmod(rest, 100)
        iy, iz = divmod(rest, 10)
        off = (np.array([ix, iy, iz]) - 5) * 0.01
        np.testing.assert_allclose(P[h][:3, :3], Rc @ rot[ir], atol=1e-12)
        np.testing.assert_allclose(P[h][:3, 3], centre[:3, 3] + G @ off, atol=1e-12)
    # odd n is centred
    P = orc.expand(centre, G, 9, 0.02, np.eye(3)[None])
    np.testing.assert_allclose(P[(4 * 9 + 4) * 9 + 4], centre, atol=1e-12)


def test_enumerate_c2f_recovers_hidden_pose(orc, single_object):
    """Noise-free observation; a 2-stage schedule whose grids contain the hidden pose."""
    wl = single_object
    sc = wl.scene
    depth, _ = orc.render(sc)
    centre = wl.hidden.astype(np.float64).copy()
    centre[:3, 3] += [0.02, -0.01, 0.03]
    stages = [synth.StageSpec(7, 0.01, 1, 1, 0.0), synth.StageSpec(5, 0.0025, 1, 1, 0.0)]
    out = orc.enumerate_c2f(sc, 0, centre, np.eye(3), wl.lik, depth, stages, m=16, seed=3)
    np.testing.assert_allclose(out["centres"][1][:3, 3], wl.hidden[:3, 3], atol=1e-6)
    # the particles jitter uniformly inside the final cell around the hidden pose
    assert (np.abs(out["particles"][:, :3, 3] - wl.hidden[:3, 3]) <= 0.0025 / 2 + 1e-7).all()
    # logq: categorical log-prob of the cell minus the log cell volume
    np.testing.assert_allclose(out["logq"], out["logw"] - out["z"][-1] - 3 * math.log(0.0025), atol=1e-9)


def test_path_density_matches_path_frequencies(orc, single_object):
    """With one particle per proposal (Sec. III-B: sample a cell in proportion to its score,
    recurse into it, then a uniform point in the last cell) the reported path density
    exp(logq) * step_T^3 is the probability of the sampled path of cells: over 2,000 seeds
    the frequencies of the paths of a 2-stage, 2^3-cell schedule match it (chi-square), and
    with one stage it reduces to the last-stage density."""
    from scipy import stats
    wl = single_object
    sc = wl.scene
    obs = synth.corrupt_depth(orc.render(sc)[0], 2.0, wl.draws)
    lk = dict(kind=1, radius=0.01, p_outlier=0.01, half_window=1)
    centre = wl.hidden.astype(np.float64)
    stages = [synth.StageSpec(2, 0.0002, 1, 1, 0.0), synth.StageSpec(2, 0.0001, 1, 1, 0.0)]
    n = 2000
    count, prob = {}, {}
    for seed in range(n):
        o = orc.enumerate_c2f(sc, 0, centre, np.eye(3), lk, obs, stages, 1, seed, path_density=True)
        key = tuple(o["idx"][:, 0])
        count[key] = count.get(key, 0) + 1
        prob[key] = math.exp(o["logq"][0] + 3 * math.log(stages[-1].step))
    keys = sorted(count)
    assert len(keys) >= 10  # a spread-out proposal, so the test has power
    p = np.array([prob[k] for k in keys])
    assert p.sum() <= 1 + 1e-9 and p.sum() > 0.99  # the unseen paths are rare
    c = np.array([count[k] for k in keys], dtype=np.float64)
    e = n * p
    keep = e >= 5
    chi2 = float(((c[keep] - e[keep]) ** 2 / e[keep]).sum())
    assert stats.chi2.sf(chi2, int(keep.sum()) - 1) > 1e-3, (chi2, keep.sum())
    one = orc.enumerate_c2f(sc, 0, centre, np.eye(3), lk, obs, stages[:1], 4, 5, path_density=True)
    last = orc.enumerate_c2f(sc, 0, centre, np.eye(3), lk, obs, stages[:1], 4, 5)
    np.testing.assert_array_equal(one["logq"], last["logq"])


# ---------------------------------------------------------------------------------------
# Gradient of the Gaussian-window log-likelihood
# ---------------------------------------------------------------------------------------

def _hat(xi):
    v, w = xi[:3], xi[3:]
    M = np.zeros((4, 4))
    M[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    M[:3, 3] = v
    return M


def _fixed_vis_ll(orc, sc, slot, pose, tid, lk, obs):
    d = orc.render_fixed(sc, slot, pose, tid)
    ell, _, _, _ = orc.pixel_loglik(sc.camera, lk, d, tid, obs)
    return np.nansum(ell)


def test_gradient_matches_fixed_visibility_central_differences(orc, single_object):
    wl = single_object
    sc = wl.scene
    lk = dict(kind=1, radius=0.003, p_outlier=0.01, half_window=2)
    obs = synth.corrupt_depth(orc.render(sc)[0], 2.0, wl.draws)
    pose = wl.hidden.astype(np.float64).copy()
    pose[:3, 3] += [0.004, -0.003, 0.005]
    g = orc.score_grad(sc, 0, pose[None], lk, obs)
    _, tid = orc.render(sc, slot=0, slot_pose=pose)
    # FP64 allows a small step; at 1e-4 the O(h^2) term of this sharply curved (sigma = 3 mm)
    # likelihood is still ~1e-2 relative.
    h = 1e-6
    fd = np.zeros(6)
    for k in range(6):
        e = np.zeros(6); e[k] = h
        lp = _fixed_vis_ll(orc, sc, 0, linalg.expm(_hat(e)) @ pose, tid, lk, obs)
        lm = _fixed_vis_ll(orc, sc, 0, linalg.expm(_hat(-e)) @ pose, tid, lk, obs)
        fd[k] = (lp - lm) / (2 * h)
    scale = np.abs(fd).max()
    np.testing.assert_allclose(g["dpose"][0], fd, rtol=1e-5, atol=1e-5 * scale)
    # sigma and p_out: the rendered image does not depend on them
    base = dict(lk)
    for key, out in (("radius", "dsigma"), ("p_outlier", "dpout")):
        hs = 1e-7 if key == "radius" else 1e-6
        lp = orc.score(sc, 0, pose[None], dict(base, **{key: base[key] + hs}), obs, flags=False)["ll"][0]
        lm = orc.score(sc, 0, pose[None], dict(base, **{key: base[key] - hs}), obs, flags=False)["ll"][0]
        assert g[out][0] == pytest.approx((lp - lm) / (2 * hs), rel=1e-5)
    assert g["ll"][0] == pytest.approx(orc.score(sc, 0, pose[None], lk, obs, flags=False)["ll"][0], rel=1e-12)


def test_gradient_of_translation_along_view_axis(orc):
    """A fronto-parallel face: moving the object by dz along the optical axis moves every
    rendered point's depth by dz, so dz_j/dv = (0, 0, 1) exactly; with observed = rendered
    + 1 mm in depth the pose gradient's x, y parts cancel by symmetry."""
    cam = synth.Camera(8, 8, 8.0, 8.0, 4.0, 4.0, 0.01, 2.0)
    mesh = synth.voxel_mesh([[0, 0, 0]], 0.2, origin=(-0.1, -0.1, -0.1))
    pose = synth.rigid(np.eye(3), [0, 0, 0.6])
    scene = _one_object_scene(mesh, pose, cam)
    depth, tid = orc.render(scene)
    obs = np.where(tid >= 0, depth + 0.001, depth)
    lk = dict(kind=1, radius=0.003, p_outlier=0.01, half_window=1)
    g = orc.score_grad(scene, 0, pose[None], lk, obs)["dpose"][0]
    assert g[2] > 0  # moving back toward the observation raises the likelihood
    assert abs(g[0]) < 1e-9 * abs(g[2]) and abs(g[1]) < 1e-9 * abs(g[2])


# ---------------------------------------------------------------------------------------
# SMC over the number of objects (Eq. 2 and 3)
# ---------------------------------------------------------------------------------------

def _two_object_scene(orc):
    """Two blobs far apart on a 96x72 image (disjoint footprints), camera 0.6 m above."""
    rng = np.random.default_rng(77)
    cells = [np.argwhere(rng.random((6, 6, 4)) < 0.7) for _ in range(2)]
    meshes = [synth.voxel_mesh(c, 0.01, origin=(-0.03, -0.03, -0.02)) for c in cells]
    cam = synth.Camera(96, 72, 90.0, 90.0, 48.0, 36.0, 0.01, 2.0)
    poses = np.stack([synth.rigid(np.eye(3), [-0.12, 0.0, 0.6]), synth.rigid(np.eye(3), [0.12, 0.02, 0.6])])
    sc = synth.Scene(cam, meshes, poses.astype(np.float32))
    obs = orc.render(sc)[0].astype(np.float32)
    return sc, obs


def test_smc_weights_of_a_near_exact_proposal(orc):
    """Importance sampling with a proposal proportional to the target gives every particle
    the same weight, the target's normaliser: with one stage of 1-micron cells, W_1 is
    log Z + 3 log step (Eq. 2), and the step-2 increment of Eq. 3 is
    log Z' + 3 log step - LL_1(x_1) for a second object whose footprint is disjoint."""
    sc, obs = _two_object_scene(orc)
    lk = dict(kind=1, radius=0.004, p_outlier=0.01, half_window=1)
    stages = [synth.StageSpec(3, 1e-6, 1, 1, 0.0)]
    # centres off the render's pixel-aligned true poses, so no pixel centre sits within a
    # micron's reach of an edge (the likelihood is then smooth across a cell)
    centres = [sc.poses[0].astype(np.float64), sc.poses[1].astype(np.float64)]
    centres[0][:3, 3] += [0.00123, -0.00071, 0.00037]
    centres[1][:3, 3] += [-0.00052, 0.00091, -0.00043]
    out = orc.smc_parse(sc, 0, centres, np.eye(3), lk, obs, stages, m=3, seed=5, ess_frac=0.0)
    for j in range(3):
        one = synth.Scene(sc.camera, sc.meshes[:1], sc.poses[:1].copy())
        e1 = orc.enumerate_c2f(one, 0, centres[0], np.eye(3), lk, obs, stages, 1, 5 + j, path_density=True)
        w1 = e1["z"][-1] + 3 * math.log(1e-6)
        two = synth.Scene(sc.camera, sc.meshes, np.stack([e1["particles"][0], sc.poses[1]]).astype(np.float64))
        e2 = orc.enumerate_c2f(two, 1, centres[1], np.eye(3), lk, obs, stages, 1, 5 + 1000 + j, path_density=True)
        one.poses[0] = e1["particles"][0]
        ll1 = orc.score(one, 0, e1["particles"][:1], lk, obs, flags=False)["ll"][0]
        w2 = w1 + e2["z"][-1] + 3 * math.log(1e-6) - ll1
        assert out["logw"][j] == pytest.approx(w2, abs=0.05), (j, out["logw"][j], w2)
    # with a single step, resampling keeps the mean weight: the evidence does not change
    a = orc.smc_parse(sc, 0, centres[:1], np.eye(3), lk, obs, stages, m=4, seed=9, ess_frac=0.0)
    b = orc.smc_parse(sc, 0, centres[:1], np.eye(3), lk, obs, stages, m=4, seed=9, ess_frac=2.0)
    assert b["idx"][0] is not None and a["idx"][0] is None
    assert a["log_evidence"] == pytest.approx(b["log_evidence"], abs=1e-9)
    np.testing.assert_allclose(b["logw"], b["log_evidence"], atol=1e-9)


# ---------------------------------------------------------------------------------------
# Hierarchical noise: scoring over a grid of noise settings
# ---------------------------------------------------------------------------------------

def test_noise_grid_marginal_special_cases(orc, single_object):
    """One setting: the marginal is its log-likelihood plus its log weight. Identical
    settings: plus the log of their total mass. Any grid: between the best weighted term and
    that plus log G; independent of the order of the settings."""
    wl = single_object
    sc = wl.scene
    obs = synth.corrupt_depth(orc.render(sc)[0], 2.0, wl.draws)
    poses = np.stack([wl.hidden, wl.hidden @ synth.rigid(np.eye(3), [0.004, 0, 0])]).astype(np.float64)
    one = orc.score_noise(sc, 0, poses, 0, [0.005], [0.01], 1, obs, log_weight=[-0.7])
    ref = orc.score(sc, 0, poses, dict(kind=0, radius=0.005, p_outlier=0.01, half_window=1), obs, flags=False)["ll"]
    np.testing.assert_array_equal(one["ll"][:, 0], ref)
    np.testing.assert_allclose(one["marginal"], ref - 0.7, rtol=0, atol=1e-9)
    same = orc.score_noise(sc, 0, poses, 0, [0.005, 0.005], [0.01, 0.01], 1, obs, log_weight=[0.1, -0.3, 0.2, 0.0])
    np.testing.assert_allclose(same["marginal"], ref + np.log(np.exp([0.1, -0.3, 0.2, 0.0]).sum()), rtol=0, atol=1e-9)
    r, p = [0.0025, 0.005, 0.01], [0.001, 0.01, 0.1]
    w = np.log(np.arange(1, 10) / 45.0)
    g = orc.score_noise(sc, 0, poses, 1, r, p, 1, obs, log_weight=w)
    best = (g["ll"] + w).max(axis=1)
    assert (g["marginal"] >= best).all() and (g["marginal"] <= best + math.log(9)).all()
    perm = [2, 0, 1]
    w2 = w.reshape(3, 3)[perm].ravel()
    g2 = orc.score_noise(sc, 0, poses, 1, [r[k] for k in perm], p, 1, obs, log_weight=w2)
    np.testing.assert_allclose(g2["marginal"], g["marginal"], rtol=0, atol=1e-8)
