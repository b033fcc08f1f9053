"""Edge cases of the newer entry points: empty batches, invalid grids and schedules, a
camera that sees nothing, a frame with no valid pixel, a session with no fixed object."""
import math

import numpy as np
import pytest

from paper_2312_08715_gb300 import synth
from _scenes import gpu_context, observed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noise_grid_arguments(orc, single_object):
    from paper_2312_08715_gb300 import b3d
    wl = single_object
    ctx = gpu_context(wl.scene, observed(orc, wl))
    P = torch.as_tensor(wl.hidden[None], device="cuda")
    ll = torch.empty((1, 1), device="cuda")
    m = torch.empty(1, device="cuda")
    b3d.b3d_score_noise_batch(ctx.h, 0, 0, P, b3d.noise_grid(0, [0.005], [0.01]), ll, m)  # empty: no-op
    for bad in (b3d.noise_grid(0, [0.005], [0.01], half_window=3), b3d.noise_grid(2, [0.005], [0.01]),
                b3d.noise_grid(0, [0.005], [1.0]), b3d.noise_grid(0, [-0.001], [0.01])):
        with pytest.raises(b3d.B3DError) as e:
            b3d.b3d_score_noise_batch(ctx.h, 0, 1, P, bad, ll, m)
        assert e.value.status == b3d.B3D_EINVAL
    g = b3d.noise_grid(0, [0.005], [0.01])
    g.n_radius = 5
    with pytest.raises(b3d.B3DError):
        b3d.b3d_score_noise_batch(ctx.h, 0, 1, P, g, ll, m)
    # loglik may be NULL: the marginal alone
    b3d.b3d_score_noise_batch(ctx.h, 0, 1, P, b3d.noise_grid(0, [0.005, 0.01], [0.01]), None, m)
    ctx.sync()
    assert np.isfinite(m.cpu().numpy()).all()
    ctx.close()


def test_path_density_argument_and_single_stage(orc, single_object):
    from paper_2312_08715_gb300 import b3d
    wl = single_object
    ctx = gpu_context(wl.scene, observed(orc, wl))
    st = [synth.StageSpec(3, 0.01, 1, 2, math.radians(2))]
    sch = b3d.schedule(st, 4, 1, np.eye(3), True)
    sch.path_density = 2
    out = (torch.empty((4, 4, 4), device="cuda"), torch.empty(4, device="cuda"), torch.empty(4, device="cuda"))
    with pytest.raises(b3d.B3DError) as e:
        b3d.b3d_enumerate_c2f(ctx.h, 0, wl.hidden, sch, b3d.lik_params(**wl.lik), *out)
    assert e.value.status == b3d.B3D_EINVAL
    # one stage: the path density is the last-stage density
    a = [x.cpu().numpy().copy() for x in ctx.enumerate_c2f(0, wl.hidden, st, wl.lik, 4, 1, np.eye(3), path_density=True)]
    b = [x.cpu().numpy().copy() for x in ctx.enumerate_c2f(0, wl.hidden, st, wl.lik, 4, 1, np.eye(3))]
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    ctx.close()


def test_camera_that_sees_nothing_and_empty_batch():
    from paper_2312_08715_gb300 import b3d
    v = synth.camera_video(0, 24, n_frames=1)
    ctx = b3d.Context(0)
    ids = [ctx.load_mesh(m, closed=i < len(v.scene.meshes) - 1) for i, m in enumerate(v.scene.meshes)]
    ctx.set_scene(v.scene.camera, ids, v.scene.poses, np.zeros((24, 24), np.float32))
    away = v.cam_from_world[0].astype(np.float64).copy()
    away[:3, 3] += [0.0, 0.0, -5.0]  # the whole scene behind the camera
    d, t = ctx.render_camera(away[None].astype(np.float32))
    ctx.sync()
    assert (d.cpu().numpy() == v.scene.camera.far).all() and (t.cpu().numpy() == -1).all()
    b3d.b3d_render_camera_batch(ctx.h, 0, None, None)  # empty: no-op, even with NULL buffers
    with pytest.raises(b3d.B3DError):
        b3d.b3d_render_camera_batch(ctx.h, 1, None, d)
    ctx.close()


def test_server_frame_without_valid_pixels_and_all_objects_tracked():
    from paper_2312_08715_gb300 import b3d
    st = synth.tracking_stream(0, n_objects=2, width=48, height=36, f=45.0, n_frames=2, vox_lo=300, vox_hi=800,
                               seed_base=9100)
    sch = b3d.schedule([synth.tracking_stage(3, 0.01, 4, 5.0)], 4, 0, np.eye(3))
    srv = b3d.Server(b3d.server_config(b3d.lik_params(kind=0, radius=0.005, p_outlier=0.01, half_window=1), sch,
                                       max_batch_items=8, device_timeout_ms=30000))
    meshes = [(m.verts, m.faces) for m in st.scene.meshes[:2]]
    sid = srv.open_session(st.scene.camera, meshes, st.truth[0][:2], 2, st.seed, closed=True,
                           grid_frame=st.grid_frame)  # no fixed object: both tracked
    bad = np.full((36, 48), np.nan, np.float32)
    bad[0, :5] = -1.0
    r = srv.wait(srv.submit(sid, bad), 30000)
    assert r["status"] == 0 and r["n_track"] == 2 and np.isfinite(r["poses"]).all()
    with pytest.raises(b3d.B3DError) as e:
        srv.open_session(st.scene.camera, meshes, st.truth[0][:2], 3, st.seed)  # n_track > n_obj
    assert e.value.status == b3d.B3D_EINVAL
    srv.close()
