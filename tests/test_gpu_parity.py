"""GPU parity: the CUDA path, called through the C ABI, against the FP64 CPU oracle on
identical seeded inputs. Tolerances (from the FP32 arithmetic of the kernels):
  - triangle-id maps identical except at pixels the oracle flags as edge/depth ties
    (coverage within 1e-4 px of an edge, depths within 1e-5 relative), and at no more than
    1e-4 of all pixels;
  - depth within 1e-5 relative where the triangle ids agree;
  - log-likelihood within 1e-4 * sum_i |l_i| plus the oracle's bound on what FP32-resolution
    decisions (flagged pixels, inlier-ball borderline pairs) can change;
  - the argmax hypothesis identical unless the oracle's top-two gap is inside that tolerance.
"""
import math

import numpy as np
import pytest

from paper_2312_08715_gb300 import synth
from _scenes import check_grad, check_ll, gpu_context, jitter_poses, ll_tolerance, observed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


def _check_render(orc, scene, slot, poses, depth, tid, max_frac=1e-4):
    """Ids identical except at pixels the oracle flags as edge or depth ties (bit 0), and at
    no more than max_frac of all pixels; depths within 1e-5 relative where the ids agree,
    except where the oracle flags the depth as ill-conditioned (bit 2: the ray meets the
    plane so obliquely that the FP32 resolution of the vertices moves it by more)."""
    n_mis = n_px = n_cond = 0
    for k, P in enumerate(poses):
        od, ot, of = orc.render(scene, slot=slot, slot_pose=P, edge_tol=1e-4, z_tol=1e-5, want_flags=True)
        mis = ot != tid[k]
        assert not (mis & ((of & 1) == 0)).any(), f"pose {k}: {int((mis & ((of & 1) == 0)).sum())} unflagged id mismatches"
        agree = ~mis & ((of & 4) == 0)  # where the ids agree and the depth is well conditioned
        rel = np.abs(depth[k][agree] - od[agree]) / od[agree]
        assert rel.max() <= 1e-5, f"pose {k}: depth rel err {rel.max()}"
        n_cond += int(((of & 4) != 0).sum())
        n_mis += int(mis.sum())
        n_px += mis.size
    print(f"render ids: {n_mis} of {n_px} pixels differ (all flagged); {n_cond} ill-conditioned depths")
    assert n_mis <= max(1, max_frac * n_px), f"{n_mis} of {n_px} pixels differ"
    return n_mis


_check_ll = check_ll


def _check_argmax(got, ref):
    o = ref["ll"]
    top = np.argsort(o)[::-1]
    gap = o[top[0]] - o[top[1]] if o.size > 1 else np.inf
    if gap > ll_tolerance(ref)[top[0]] * 2:
        assert int(np.argmax(got)) == int(top[0])


# ---------------------------------------------------------------------------------------
# rendering
# ---------------------------------------------------------------------------------------

def test_render_single_object(orc, single_object):
    wl = single_object
    sc = wl.scene
    poses = jitter_poses(np.random.default_rng(11), wl.hidden, 32)
    ctx = gpu_context(sc, observed(orc, wl))
    d, t = ctx.render(0, poses)
    ctx.sync()
    _check_render(orc, sc, 0, poses, _np(d), _np(t))


def test_render_tabletop_composite(orc, tabletop):
    wl = tabletop
    sc = wl.scene
    poses = jitter_poses(np.random.default_rng(12), wl.hidden, 6, trans=0.05, rot_deg=30)
    ctx = gpu_context(sc, observed(orc, wl))
    d, t = ctx.render(wl.slot, poses)
    ctx.sync()
    _check_render(orc, sc, wl.slot, poses, _np(d), _np(t))
    # every other object is present in the composite
    ids = _np(t)[0]
    f_off = np.cumsum([0] + [m.n_faces for m in sc.meshes])
    for o in range(len(sc.meshes)):
        if o != wl.slot:
            assert ((ids >= f_off[o]) & (ids < f_off[o + 1])).any() or o == 1


def test_render_large_footprint_and_ragged_image(orc):
    """An object close to the camera covers several screen tiles; a ragged 37x29 image. Ids
    identical except at flagged pixels, and at no more than 1e-4 of the pixels (16 poses:
    307,200 and 17,168 pixels, so 30 and 1)."""
    rng = np.random.default_rng(13)
    cells = np.array(np.unravel_index(rng.permutation(512)[:300], (8, 8, 8))).T
    mesh = synth.voxel_mesh(cells, 0.02, origin=(-0.08, -0.08, -0.08))
    for cam, z in [(synth.Camera(160, 120, 150.0, 150.0, 80.0, 60.0, 0.01, 2.0), 0.22),
                   (synth.Camera(37, 29, 30.0, 31.0, 17.3, 15.1, 0.01, 2.0), 0.35)]:
        R = synth.random_rotation(rng)
        pose = synth.rigid(R, [0.01, -0.02, z]).astype(np.float32)
        sc = synth.Scene(cam, [mesh], pose[None].copy())
        obs = orc.render(sc)[0].astype(np.float32)
        ctx = gpu_context(sc, obs)
        poses = jitter_poses(rng, pose, 16, trans=0.01, rot_deg=5)
        d, t = ctx.render(0, poses)
        ctx.sync()
        _check_render(orc, sc, 0, poses, _np(d), _np(t), max_frac=1e-4)
        lik = dict(kind=0, radius=0.005, p_outlier=0.01, half_window=2)
        ll = _np(ctx.score(0, poses, lik))
        ll2 = _np(ctx.score_depth(d, lik, t, slot=0))  # 37 x 29: no 16-byte vector access
        ctx.sync()
        ref = orc.score(sc, 0, poses, lik, obs)
        _check_ll(ll, ref, "large footprint")
        _check_ll(ll2, ref, "large footprint, materialised")


@pytest.mark.parametrize("nt,hi", [(64, 0), (128, 1), (256, 0)])
def test_widest_tile_with_the_largest_window(orc, nt, hi):
    """tile_w 256 with the largest half window (7): the kernel narrows the tile so the tile and
    its halo fit its shared-memory region; an object covering most of a 160x120 image."""
    from paper_2312_08715_gb300 import b3d
    rng = np.random.default_rng(14)
    cells = np.array(np.unravel_index(rng.permutation(512)[:300], (8, 8, 8))).T
    mesh = synth.voxel_mesh(cells, 0.02, origin=(-0.08, -0.08, -0.08))
    cam = synth.Camera(160, 120, 150.0, 150.0, 80.0, 60.0, 0.01, 2.0)
    pose = synth.rigid(synth.random_rotation(rng), [0.01, -0.02, 0.22]).astype(np.float32)
    sc = synth.Scene(cam, [mesh], pose[None].copy())
    obs = synth.corrupt_depth(orc.render(sc)[0], cam.far, synth.noise_draws(rng, 120, 160))
    ctx = gpu_context(sc, obs)
    b3d.b3d_set_tuning(ctx.h, tile_w=256, cta_threads=nt, ctas_per_sm=0, high_occupancy=hi, batch_chunk=4)
    poses = jitter_poses(rng, pose, 6, trans=0.01, rot_deg=5)
    lik = dict(kind=1, radius=0.004, p_outlier=0.01, half_window=7)
    ll = _np(ctx.score(0, poses, lik))
    ctx.sync()
    _check_ll(ll, orc.score(sc, 0, poses, lik, obs), f"tile 256, w 7, {nt} threads")
    ctx.close()


def test_near_plane_and_out_of_view(orc, single_object):
    wl = single_object
    sc = wl.scene
    obs = observed(orc, wl)
    P = [wl.hidden.copy() for _ in range(4)]
    P[1][:3, 3] = [0.0, 0.0, 0.03]    # straddles the near plane (0.01 m)
    P[2][:3, 3] = [5.0, 0.0, 0.5]     # far outside the view
    P[3][:3, 3] = [0.0, 0.0, -0.5]    # behind the camera
    poses = np.stack(P).astype(np.float32)
    ctx = gpu_context(sc, obs)
    d, t = ctx.render(0, poses)
    ll = ctx.score(0, poses, wl.lik)
    ctx.sync()
    # vertices 3 cm from the camera project thousands of pixels off-screen, where FP32 edge
    # functions resolve ~1e-4 px: every mismatch must still be a flagged pixel, but more of
    # the (few) pixels are allowed to flip than in the workloads' geometry
    _check_render(orc, sc, 0, poses, _np(d), _np(t), max_frac=5e-3)
    ref = orc.score(sc, 0, poses, wl.lik, obs)
    _check_ll(_np(ll), ref, "near/out of view")


# ---------------------------------------------------------------------------------------
# scoring
# ---------------------------------------------------------------------------------------

def test_score_single_object_full_grid(orc, single_object):
    """1,000 hypotheses: 10^3 translation grid (1 cm) around the hidden pose."""
    wl = single_object
    sc = wl.scene
    obs = observed(orc, wl)
    poses = orc.expand(wl.hidden, np.eye(3), 10, 0.01, np.eye(3)[None]).astype(np.float32)
    ref = orc.score(sc, 0, poses, wl.lik, obs)
    ctx = gpu_context(sc, obs)
    ll = _np(ctx.score(0, poses, wl.lik))
    ctx.sync()
    _check_ll(ll, ref, "plain 64x48")
    _check_argmax(ll, ref)
    assert int(np.argmax(ll)) == 555
    # permuting the hypotheses permutes the scores bit for bit
    perm = np.random.default_rng(1).permutation(1000)
    ll2 = _np(ctx.score(0, poses[perm], wl.lik))
    ctx.sync()
    np.testing.assert_array_equal(ll[perm], ll2)


def test_every_launch_shape_matches_oracle(orc, single_object):
    """The autotuner's candidate launch shapes change only how the work is tiled."""
    from paper_2312_08715_gb300 import b3d
    wl = single_object
    sc = wl.scene
    obs = observed(orc, wl)
    poses = orc.expand(wl.hidden, np.eye(3), 6, 0.01, orc.rotation_set(1, 3, 0.1)).astype(np.float32)
    ref = orc.score(sc, 0, poses, wl.lik, obs)
    ctx = gpu_context(sc, obs)
    outs = []
    for tw, nt, cps, hi in [(8, 128, 0, 0), (32, 256, 2, 0), (64, 256, 0, 1), (256, 128, 1, 1), (48, 64, 0, 0),
                            (96, 32, 0, 1), (8, 32, 3, 0), (40, 64, 0, 1)]:
        b3d.b3d_set_tuning(ctx.h, tw, nt, cps, hi)
        outs.append(_np(ctx.score(0, poses, wl.lik)))
        ctx.sync()
        _check_ll(outs[-1], ref, f"tuning {tw}/{nt}/{cps}/{hi}")
    for o in outs[1:]:
        np.testing.assert_allclose(o, outs[0], rtol=2e-6, atol=1e-3)
    st = b3d.stage_params(synth.StageSpec(7, 0.01, 1, 4, 0.1))
    best = b3d.b3d_autotune(ctx.h, 0, wl.hidden, np.eye(3), st, b3d.lik_params(**wl.lik))
    assert best["cta_threads"] in (32, 64, 128, 256) and 8 <= best["tile_w"] <= 256
    assert b3d.b3d_get_tuning(ctx.h) == best
    _check_ll(_np(ctx.score(0, poses, wl.lik)), ref, "autotuned")
    ctx.close()


def test_work_counters_do_not_depend_on_the_tuned_shape(orc, single_object):
    """Work counting is compiled into one launch shape; a counting launch uses it whatever
    shape is tuned, so the counts (and the roofline built on them) never come out empty."""
    from paper_2312_08715_gb300 import b3d
    wl = single_object
    sc = wl.scene
    obs = observed(orc, wl)
    poses = orc.expand(wl.hidden, np.eye(3), 5, 0.01, orc.rotation_set(1, 3, 0.1)).astype(np.float32)
    ctx = gpu_context(sc, obs)
    counts = []
    for nt, hi in [(128, 0), (128, 1), (256, 0), (32, 1)]:
        b3d.b3d_set_tuning(ctx.h, 64, nt, 0, hi)
        b3d.b3d_set_instrumentation(ctx.h, b3d.B3D_INSTR_WORK)
        b3d.b3d_work_counters(ctx.h)  # reads and clears
        ll = _np(ctx.score(0, poses, wl.lik))
        ctx.sync()
        counts.append(np.asarray(b3d.b3d_work_counters(ctx.h)))
        b3d.b3d_set_instrumentation(ctx.h, 0)
        _check_ll(ll, orc.score(sc, 0, poses, wl.lik, obs), f"counting with {nt}/{hi} tuned")
    assert counts[0][0] == len(poses) and (counts[0] > 0).all(), counts[0]
    for c in counts[1:]:
        assert np.array_equal(c, counts[0]), (c, counts[0])
    ctx.close()


@pytest.mark.parametrize("w,miss_mode", [(2, 0), (1, 1)])
def test_score_smooth_and_miss_modes(orc, single_object, w, miss_mode):
    wl = single_object
    sc = wl.scene
    obs = observed(orc, wl)
    poses = orc.expand(wl.hidden, np.eye(3), 5, 0.004, orc.rotation_set(1, 4, 0.1)).astype(np.float32)
    for lik in (dict(kind=1, radius=0.003, p_outlier=0.01, half_window=w, miss_mode=miss_mode),
                dict(kind=0, radius=0.005, p_outlier=0.05, half_window=w, miss_mode=miss_mode)):
        ref = orc.score(sc, 0, poses, lik, obs)
        ctx = gpu_context(sc, obs)
        ll = _np(ctx.score(0, poses, lik))
        ctx.sync()
        _check_ll(ll, ref, f"lik {lik}")
        _check_argmax(ll, ref)


def test_two_pass_matches_fused(orc, single_object):
    """Render to HBM then score the materialised images == the fused path == the oracle."""
    wl = single_object
    sc = wl.scene
    obs = observed(orc, wl)
    poses = orc.expand(wl.hidden, np.eye(3), 4, 0.01, np.eye(3)[None]).astype(np.float32)
    ref = orc.score(sc, 0, poses, wl.lik, obs)
    ctx = gpu_context(sc, obs)
    d, t = ctx.render(0, poses)
    ll2 = _np(ctx.score_depth(d, wl.lik, t))
    ll2s = _np(ctx.score_depth(d, wl.lik, t, slot=0))
    ll1 = _np(ctx.score(0, poses, wl.lik))
    lk_b = dict(wl.lik, miss_mode=1)
    ll3 = _np(ctx.score_depth(d, lk_b, t, slot=0))
    ctx.sync()
    _check_ll(ll1, ref, "fused")
    _check_ll(ll2, ref, "two-pass")
    _check_ll(ll2s, ref, "two-pass against the slot's background")
    _check_ll(ll3, orc.score(sc, 0, poses, lk_b, obs), "two-pass miss_mode 1")


def test_two_pass_tabletop_composite(orc, tabletop):
    """The materialised form on the five-object tabletop: render (background fill, then the
    object over its screen box) and score (the box where each image differs from the scene,
    scored against the background terms) == the oracle, in both miss modes, with and without
    the id output."""
    wl = tabletop
    sc = wl.scene
    obs = observed(orc, wl)
    poses = jitter_poses(np.random.default_rng(21), wl.hidden, 12, trans=0.03, rot_deg=20)
    ctx = gpu_context(sc, obs)
    d, t = ctx.render(wl.slot, poses)
    d_only, _ = ctx.render(wl.slot, poses, want_tid=False)
    for lk in (wl.lik, dict(wl.lik, miss_mode=1), dict(kind=1, radius=0.004, p_outlier=0.02, half_window=2)):
        ref = orc.score(sc, wl.slot, poses, lk, obs)
        for slot in (-1, wl.slot, 0):
            ll = _np(ctx.score_depth(d, lk, t, slot=slot))
            ctx.sync()
            _check_ll(ll, ref, f"two-pass tabletop {lk}, reference without slot {slot}")
    ctx.sync()
    _check_render(orc, sc, wl.slot, poses[:4], _np(d[:4]), _np(t[:4]))
    _check_depth(orc, sc, wl.slot, poses[:4], _np(d_only[:4]))
    ctx.close()


def _check_depth(orc, scene, slot, poses, depth, max_frac=1e-4):
    """Depth-only renders (the rectangle rasteriser): within 1e-5 relative of the oracle
    except at pixels it flags as edge or depth ties (bit 0) or ill-conditioned depths
    (bit 2), and those at most max_frac of all."""
    n_bad = n_px = 0
    for k, P in enumerate(poses):
        od, _, of = orc.render(scene, slot=slot, slot_pose=P, edge_tol=1e-4, z_tol=1e-5, want_flags=True)
        bad = np.abs(depth[k] - od) > 1e-5 * od
        assert not (bad & ((of & 5) == 0)).any(), f"pose {k}: {int((bad & ((of & 5) == 0)).sum())} unflagged depth mismatches"
        n_bad += int(bad.sum())
        n_px += bad.size
    assert n_bad <= max(1, max_frac * n_px), f"{n_bad} of {n_px} pixels differ"


def _oracle_image_ll(orc, cam, lk, depth, tid, obs):
    out = []
    for k in range(depth.shape[0]):
        ell, _, _, _ = orc.pixel_loglik(cam, lk, depth[k].astype(np.float64), None if tid is None else tid[k], obs)
        out.append(ell.sum())
    return np.array(out)


@pytest.mark.parametrize("offset", [0, 1])
def test_score_depth_of_arbitrary_images(orc, tabletop, offset):
    """Images that are not renders of the scene: the observation itself, renders with noisy
    patches, images of one constant depth and of misses only, then the same with random id
    images in miss mode 1. offset 1 shifts the buffers by one element (no 16-byte vector
    access). Smooth likelihood (no FP32 inlier-ball decisions), against the oracle's
    per-pixel terms summed in FP64."""
    from paper_2312_08715_gb300 import b3d
    wl = tabletop
    sc = wl.scene
    cam = sc.camera
    obs = observed(orc, wl)
    rng = np.random.default_rng(22)
    poses = jitter_poses(rng, wl.hidden, 4, trans=0.02, rot_deg=10)
    ctx = gpu_context(sc, obs)
    d, _ = ctx.render(wl.slot, poses)
    imgs = [obs.astype(np.float32)]
    for k in range(4):
        im = _np(d[k]).copy()
        y, x = rng.integers(0, cam.height - 8), rng.integers(0, cam.width - 8)
        im[y:y + 8, x:x + 8] += rng.normal(0, 0.01, size=(8, 8)).astype(np.float32)
        imgs.append(im)
    imgs.append(np.full((cam.height, cam.width), 0.9, np.float32))
    imgs.append(np.full((cam.height, cam.width), cam.far, np.float32))
    imgs = np.stack(imgs)
    n, H, W = imgs.shape
    buf = torch.zeros(n * H * W + offset, dtype=torch.float32, device="cuda")
    view = buf[offset:].view(n, H, W)
    view.copy_(torch.as_tensor(imgs))
    lk = dict(kind=1, radius=0.004, p_outlier=0.02, half_window=2)
    ll = torch.empty(n, dtype=torch.float32, device="cuda")
    b3d.b3d_score_depth_batch(ctx.h, -1, n, view, None, b3d.lik_params(**lk), ll, ctx.stream)
    got = _np(ll).astype(np.float64)
    ctx.sync()
    ref = _oracle_image_ll(orc, cam, lk, imgs, None, obs)
    scale = np.array([np.abs(orc.pixel_loglik(cam, lk, im.astype(np.float64), None, obs)[0]).sum() for im in imgs])
    assert (np.abs(got - ref) <= 1e-4 * scale).all(), (got - ref, scale)
    # miss mode 1: ids mark a random third of the pixels as carrying no point
    ids = np.where(rng.random((n, H, W)) < 1 / 3, -1, 0).astype(np.int32)
    tbuf = torch.zeros(n * H * W + offset, dtype=torch.int32, device="cuda")
    tview = tbuf[offset:].view(n, H, W)
    tview.copy_(torch.as_tensor(ids))
    lk1 = dict(lk, miss_mode=1)
    b3d.b3d_score_depth_batch(ctx.h, wl.slot, n, view, tview, b3d.lik_params(**lk1), ll, ctx.stream)
    got1 = _np(ll).astype(np.float64)
    ctx.sync()
    ref1 = _oracle_image_ll(orc, cam, lk1, imgs, ids, obs)
    scale1 = np.array([np.abs(orc.pixel_loglik(cam, lk1, im.astype(np.float64), i, obs)[0]).sum()
                       for im, i in zip(imgs, ids)])
    assert (np.abs(got1 - ref1) <= 1e-4 * scale1).all(), (got1 - ref1, scale1)
    ctx.close()


@pytest.mark.parametrize("offset", [0, 1])
def test_render_fill_paths(orc, single_object, offset):
    """The background fill with 16-byte vector stores (aligned outputs) and with scalar
    stores (outputs one element off a 16-byte boundary) write identical images, with ids
    (triangle rasteriser) and depth only (rectangle rasteriser, checked against the
    oracle)."""
    from paper_2312_08715_gb300 import b3d
    wl = single_object
    sc = wl.scene
    ctx = gpu_context(sc, observed(orc, wl))
    poses = torch.as_tensor(jitter_poses(np.random.default_rng(23), wl.hidden, 8), device="cuda")
    d0, t0 = ctx.render(0, poses)
    H, W = sc.camera.height, sc.camera.width
    db = torch.zeros(8 * H * W + offset, dtype=torch.float32, device="cuda")
    tb = torch.zeros(8 * H * W + offset, dtype=torch.int32, device="cuda")
    b3d.b3d_render_batch(ctx.h, 0, 8, poses.reshape(8, 16), db[offset:], tb[offset:], ctx.stream)
    d1, _ = ctx.render(0, poses, want_tid=False)
    db2 = torch.zeros(8 * H * W + offset, dtype=torch.float32, device="cuda")
    b3d.b3d_render_batch(ctx.h, 0, 8, poses.reshape(8, 16), db2[offset:], None, ctx.stream)
    ctx.sync()
    assert torch.equal(db[offset:].view(8, H, W), d0) and torch.equal(tb[offset:].view(8, H, W), t0)
    assert torch.equal(db2[offset:].view(8, H, W), d1)
    _check_depth(orc, sc, 0, _np(poses), _np(d1))
    ctx.close()


@pytest.mark.parametrize("kind,n_rot,rot_max", [(1, 1, 0.2), (1, 7, 0.05), (1, 200, math.radians(10)),
                                                (1, 2048, math.radians(1)), (1, 4097, math.radians(2)), (0, 200, 0.0)])
def test_rotation_sets_match_oracle(orc, single_object, kind, n_rot, rot_max):
    """The library's rotation sets (computed on the device) against the oracle's, member by
    member, through the grid expansion of a rotated, offset centre."""
    wl = single_object
    ctx = gpu_context(wl.scene, observed(orc, wl))
    st = synth.StageSpec(3, 0.004, kind, n_rot, rot_max)
    got = _np(ctx.expand(wl.centre, wl.grid_frame, st))
    ctx.sync()
    want = orc.expand(wl.centre, wl.grid_frame, 3, 0.004, orc.rotation_set(kind, n_rot, rot_max))
    np.testing.assert_allclose(got, want, atol=2e-6)
    if kind == 1:  # member 0 is the identity: the centre's own rotation is in every set
        np.testing.assert_allclose(got[13], wl.centre, atol=2e-6)


def test_tabletop_first_stage_full_size_sampled(orc, tabletop):
    """Full first-stage grid (9^3 x 200 = 145,800 hypotheses) in one launch, 40 sampled
    hypotheses checked against the oracle one by one; the grid poses against the oracle's."""
    wl = tabletop
    sc = wl.scene
    obs = observed(orc, wl)
    st = wl.stages[0]
    ctx = gpu_context(sc, obs)
    poses_gpu = ctx.expand(wl.centre, wl.grid_frame, st)
    ll = ctx.score(wl.slot, poses_gpu, wl.lik)
    ctx.sync()
    ll = _np(ll)
    assert ll.shape == (145800,) and np.isfinite(ll).all()
    rot = orc.rotation_set(st.rot_kind, st.n_rot, st.rot_max)
    P_orc = orc.expand(wl.centre, wl.grid_frame, st.n_per_axis, st.step, rot)
    np.testing.assert_allclose(_np(poses_gpu), P_orc, atol=2e-6)
    rng = np.random.default_rng(7)
    sample = np.concatenate([rng.choice(145800, 39, replace=False), [int(np.argmax(ll))]])
    ref = orc.score(sc, wl.slot, P_orc[sample], wl.lik, obs)
    _check_ll(ll[sample], ref, "tabletop stage 1 sample")


# ---------------------------------------------------------------------------------------
# log-sum-exp + resampling
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 7, 2048, 2049, 145800, 1_000_003])
def test_lse_resample(orc, n):
    rng = np.random.default_rng(n)
    ll = synth.random_ll(rng, n)
    m = 100
    from paper_2312_08715_gb300 import b3d
    ctx = b3d.Context(0)
    t = torch.as_tensor(ll, device="cuda")
    for stage in (0, 3):
        logz, idx, logq = ctx.lse_resample(t, m, seed=1234, stage=stage)
        ctx.sync()
        Z, _ = orc.lse(ll.astype(np.float64))
        assert abs(float(_np(logz)[0]) - Z) <= 1e-5 * max(1.0, abs(Z)) + 1e-4
        oi, oq, om = orc.resample(ll.astype(np.float64), m, 1234, stage)
        gi = _np(idx)
        solid = om > 1e-5
        np.testing.assert_array_equal(gi[solid], oi[solid])
        assert (gi >= 0).all() and (gi < n).all()
        np.testing.assert_allclose(_np(logq)[solid], oq[solid], atol=1e-4 * max(1.0, abs(Z)))
    ctx.close()


def test_lse_resample_degenerate(orc):
    from paper_2312_08715_gb300 import b3d
    ctx = b3d.Context(0)
    ll = np.full(5000, -1e4, np.float32)
    ll[4321] = 0.0
    logz, idx, logq = ctx.lse_resample(torch.as_tensor(ll, device="cuda"), 64, seed=5, stage=1)
    ctx.sync()
    assert (_np(idx) == 4321).all()
    assert abs(float(_np(logz)[0])) < 1e-6
    ll = np.full(3000, 2.5, np.float32)
    logz, idx, _ = ctx.lse_resample(torch.as_tensor(ll, device="cuda"), 1000, seed=6, stage=0)
    ctx.sync()
    assert float(_np(logz)[0]) == pytest.approx(2.5 + math.log(3000), abs=1e-4)
    oi, _, om = orc.resample(ll.astype(np.float64), 1000, 6, 0)
    np.testing.assert_array_equal(_np(idx)[om > 1e-5], oi[om > 1e-5])
    ctx.close()


@pytest.mark.parametrize("n,n_shards", [(145800, 3), (2049, 2), (7, 3)])
def test_lse_resample_shards_match_the_unsplit_call(orc, n, n_shards):
    """A categorical split into contiguous shards, as over ranks (the exchange of a sharded
    C2F stage): each shard's log normaliser, then each shard's draws by
    b3d_lse_resample_shard with its share of the probability, one shard after another on
    this GPU. Combined by maximum, every draw has one owner and the draws are the unsplit
    call's and the oracle's, except draws whose CDF margin is below 1e-5."""
    from paper_2312_08715_gb300 import b3d, multigpu
    ctx = b3d.Context(0)
    ll = synth.random_ll(np.random.default_rng(n + 1), n)
    t = torch.as_tensor(ll, device="cuda")
    m, seed, stage = 100, 77, 2
    spans = [multigpu.shard_range(n, r, n_shards) for r in range(n_shards)]
    logz_all = [float(ctx.lse_resample(t[b:e], 0, seed, stage)[0].item()) for b, e in spans]
    idx = np.full(m, -1, np.int64)
    logq = np.full(m, -np.inf)
    owners = np.zeros(m, np.int64)
    for r, (b, e) in enumerate(spans):
        Z, before, mass = multigpu.shard_masses(logz_all, r)
        zl, i, q = ctx.lse_resample_shard(t[b:e], m, seed, stage, before, mass, Z, b)
        ctx.sync()
        assert float(_np(zl)[0]) == pytest.approx(logz_all[r], abs=0)
        i, q = _np(i).astype(np.int64), _np(q).astype(np.float64)
        owners += i >= 0
        assert ((i == -1) | ((i >= b) & (i < e))).all()
        idx, logq = np.maximum(idx, i), np.maximum(logq, q)
    assert (owners == 1).all()
    _, gi, gq = ctx.lse_resample(t, m, seed, stage)
    ctx.sync()
    oi, oq, om = orc.resample(ll.astype(np.float64), m, seed, stage)
    solid = om > 1e-5
    np.testing.assert_array_equal(idx[solid], oi[solid])
    np.testing.assert_array_equal(idx[solid], _np(gi)[solid])
    Z, _ = orc.lse(ll.astype(np.float64))
    np.testing.assert_allclose(logq[solid], oq[solid], atol=1e-4 * max(1.0, abs(Z)))
    ctx.close()


# ---------------------------------------------------------------------------------------
# coarse-to-fine enumeration
# ---------------------------------------------------------------------------------------

def test_enumerate_c2f_matches_oracle(orc, single_object):
    wl = single_object
    sc = wl.scene
    obs = observed(orc, wl)
    centre = wl.hidden.astype(np.float64).copy()
    centre[:3, 3] += [0.012, -0.007, 0.02]
    stages = [synth.StageSpec(7, 0.01, 1, 3, math.radians(3)), synth.StageSpec(5, 0.003, 1, 2, math.radians(1))]
    M = 16
    ref = orc.enumerate_c2f(sc, 0, centre, np.eye(3), wl.lik, obs, stages, M, seed=9)
    ctx = gpu_context(sc, obs)
    parts, logw, logq = ctx.enumerate_c2f(0, centre.astype(np.float32), stages, wl.lik, M, 9, np.eye(3))
    ctx.sync()
    np.testing.assert_allclose(_np(parts), ref["particles"], atol=2e-6)
    scale = np.abs(ref["logw"]).max()
    np.testing.assert_allclose(_np(logw), ref["logw"], atol=1e-4 * scale * 4)
    np.testing.assert_allclose(_np(logq), ref["logq"], atol=1e-4 * scale * 4)


def test_enumerate_path_density_matches_oracle(orc, single_object):
    """One particle per proposal and the density of its whole path of cells (Sec. III-B),
    single-scene and batched (8 proposals in one launch), against the oracle."""
    from paper_2312_08715_gb300 import b3d
    wl = single_object
    sc = wl.scene
    obs = observed(orc, wl)
    centre = wl.hidden.astype(np.float64).copy()
    centre[:3, 3] += [0.006, -0.004, 0.009]
    stages = [synth.StageSpec(5, 0.008, 1, 3, math.radians(3)), synth.StageSpec(5, 0.002, 1, 2, math.radians(1)),
              synth.StageSpec(3, 0.0007, 1, 1, 0.0)]
    ctx = gpu_context(sc, obs)
    owner = b3d.Context(0)
    items, outs, refs = [], [], []
    for k in range(8):
        ref = orc.enumerate_c2f(sc, 0, centre, np.eye(3), wl.lik, obs, stages, 1, 40 + k, path_density=True)
        refs.append(ref)
        o = (torch.empty((1, 4, 4), device="cuda"), torch.empty(1, device="cuda"), torch.empty(1, device="cuda"))
        outs.append(o)
        items.append(b3d.c2f_item(ctx.h, 0, centre.astype(np.float32), b3d.schedule(stages, 1, 40 + k, np.eye(3), True),
                                  *o))
    b3d.b3d_enumerate_multi(owner.h, items, b3d.lik_params(**wl.lik), owner.stream)
    single = ctx.enumerate_c2f(0, centre.astype(np.float32), stages, wl.lik, 1, 40, np.eye(3), path_density=True)
    owner.sync()
    ctx.sync()
    for k, (ref, o) in enumerate(zip(refs, outs)):
        scale = abs(ref["logw"][0])
        np.testing.assert_allclose(_np(o[0])[0], ref["particles"][0], atol=2e-6)
        assert abs(float(_np(o[1])[0]) - ref["logw"][0]) <= 4e-4 * scale
        # the path sums T score differences, each good to the score tolerance
        assert abs(float(_np(o[2])[0]) - ref["logq"][0]) <= len(stages) * 4e-4 * scale, (k, _np(o[2]), ref["logq"])
    for got, o in zip(single, outs[0]):
        np.testing.assert_array_equal(_np(got), _np(o))
    ctx.close()
    owner.close()


def test_enumerate_c2f_tabletop_tracks_hidden_pose(orc, tabletop):
    """Three stages of 145,800 hypotheses around a tracking prior (<= 2 cm, <= 5 deg off)
    end within a few millimetres of the hidden pose (a sanity check of the whole path)."""
    wl = tabletop
    sc = wl.scene
    obs = observed(orc, wl)
    ctx = gpu_context(sc, obs)
    parts, logw, logq = ctx.enumerate_c2f(wl.slot, wl.centre, wl.stages, wl.lik, 100, 3, wl.grid_frame)
    ctx.sync()
    p = _np(parts)
    best = p[int(np.argmax(_np(logw)))]
    assert np.linalg.norm(best[:3, 3] - wl.hidden[:3, 3]) < 0.006
    assert np.isfinite(_np(logq)).all()


# ---------------------------------------------------------------------------------------
# gradient
# ---------------------------------------------------------------------------------------

def test_score_grad_matches_oracle(orc, single_object):
    """Every hypothesis: within 1e-3 relative of the oracle's gradient plus its bound on what
    FP32 visibility decisions at flagged pixels can move it; at least 6 of the 8 within 1e-3
    alone (so the bound cannot be what makes the test pass)."""
    wl = single_object
    sc = wl.scene
    obs = observed(orc, wl)
    lik = dict(kind=1, radius=0.003, p_outlier=0.01, half_window=2)
    poses = jitter_poses(np.random.default_rng(21), wl.hidden, 8, trans=0.006, rot_deg=4)
    ref = orc.score_grad(sc, 0, poses, lik, obs)
    ctx = gpu_context(sc, obs)
    ll, dpose, ds, dp = (_np(x) for x in ctx.score_grad(0, poses, lik))
    ctx.sync()
    sref = orc.score(sc, 0, poses, lik, obs)
    _check_ll(ll, sref, "score_grad forward")
    gb = orc.score_grad_bound(sc, 0, poses, lik, obs)["gbound"]
    frac = check_grad(dpose, ds, dp, ref, gb, "single object")
    assert frac >= 6 / 8, frac


# ---------------------------------------------------------------------------------------
# argument errors and the HBM budget
# ---------------------------------------------------------------------------------------

def test_errors_and_budget(orc, single_object):
    from paper_2312_08715_gb300 import b3d
    wl = single_object
    sc = wl.scene
    ctx = gpu_context(sc, observed(orc, wl))
    P = torch.as_tensor(wl.hidden[None], device="cuda")
    out = torch.empty(1, device="cuda")
    with pytest.raises(b3d.B3DError) as e:
        b3d.b3d_score_batch(ctx.h, 0, 1, P, b3d.lik_params(half_window=9), out)
    assert e.value.status == b3d.B3D_EINVAL
    with pytest.raises(b3d.B3DError) as e:
        b3d.b3d_score_batch(ctx.h, 3, 1, P, b3d.lik_params(), out)
    assert e.value.status == b3d.B3D_ENOTFOUND
    with pytest.raises(b3d.B3DError) as e:
        b3d.b3d_score_batch(ctx.h, 0, -1, P, b3d.lik_params(), out)
    assert e.value.status == b3d.B3D_EINVAL
    b3d.b3d_score_batch(ctx.h, 0, 0, P, b3d.lik_params(), out)  # n = 0 is a no-op
    H, W = sc.camera.height, sc.camera.width
    img = torch.zeros((1, H, W), device="cuda")
    for slot, status in ((1, b3d.B3D_ENOTFOUND), (-2, b3d.B3D_ENOTFOUND)):
        with pytest.raises(b3d.B3DError) as e:
            b3d.b3d_score_depth_batch(ctx.h, slot, 1, img, None, b3d.lik_params(), out)
        assert e.value.status == status
    with pytest.raises(b3d.B3DError) as e:  # miss mode 1 needs the id images
        b3d.b3d_score_depth_batch(ctx.h, 0, 1, img, None, b3d.lik_params(miss_mode=1), out)
    assert e.value.status == b3d.B3D_EINVAL
    b3d.b3d_score_depth_batch(ctx.h, 0, 0, img, None, b3d.lik_params(), out)  # n = 0 is a no-op
    ctx.sync()
    small = b3d.Context(0, hbm_budget_bytes=64 * 1024)
    with pytest.raises(b3d.B3DError) as e:
        small.load_mesh(sc.meshes[0])
    assert e.value.status == b3d.B3D_EBUDGET
    small.close()
    ctx.close()
