"""Batched form: many scenes of uneven image size, mesh and hypothesis count in one
persistent launch (work queue over scene and hypothesis chunks) and a batched
coarse-to-fine enumeration, captured into a CUDA graph. Results must equal the
single-scene calls bit for bit (same kernel body, same launch shape) and, on a sample,
the oracle within the parity tolerance."""
import math

import numpy as np
import pytest

from paper_2312_08715_gb300 import synth
from _scenes import check_ll, gpu_context, jitter_poses, ll_tolerance, observed

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _np(t):
    return t.detach().cpu().numpy()


def _scenes(orc):
    """Four scenes: 64x48 single object, tabletops at 80x60, 160x120 and 124x93."""
    out = []
    wl = synth.single_object_workload(1)
    out.append((wl, observed(orc, wl), 0))
    for trial, (W, H) in enumerate([(80, 60), (160, 120), (124, 93)]):
        wl = synth.tabletop_workload(10 + trial, n_objects=2 + trial, width=W, height=H, f=0.9375 * W)
        out.append((wl, observed(orc, wl), wl.slot))
    return out


def test_score_multi_equals_single_scene_calls(orc):
    from paper_2312_08715_gb300 import b3d
    scenes = _scenes(orc)
    rng = np.random.default_rng(31)
    counts = [1000, 37, 2500, 129]
    ctxs, poses, singles = [], [], []
    for (wl, obs, slot), n in zip(scenes, counts):
        ctx = gpu_context(wl.scene, obs)
        b3d.b3d_set_tuning(ctx.h, 64, 128, 0, 1, 4)
        P = torch.as_tensor(jitter_poses(rng, wl.hidden, n, trans=0.02, rot_deg=8), device="cuda")
        singles.append(_np(ctx.score(slot, P, wl.lik)))
        ctxs.append(ctx)
        poses.append(P)
    owner = b3d.Context(0)
    for chunk in (1, 4, 64):
        b3d.b3d_set_tuning(owner.h, 64, 128, 0, 1, chunk)
        outs = [torch.full((n,), float("nan"), device="cuda") for n in counts]
        items = [(c.h, sc[2], n, p, o) for c, sc, n, p, o in zip(ctxs, scenes, counts, poses, outs)]
        b3d.b3d_score_multi(owner.h, items, b3d.lik_params(**scenes[0][0].lik), owner.stream)
        owner.sync()
        for k in range(len(scenes)):
            np.testing.assert_array_equal(_np(outs[k]), singles[k])
    # one scene against the oracle on a sample
    wl, obs, slot = scenes[2]
    sel = np.arange(0, 2500, 97)
    ref = orc.score(wl.scene, slot, _np(poses[2])[sel], wl.lik, obs)
    err = np.abs(singles[2][sel].astype(np.float64) - ref["ll"])
    assert (err <= ll_tolerance(ref)).all()
    for c in ctxs + [owner]:
        c.close()


def _stages():
    return [synth.StageSpec(5, 0.01, 1, 4, math.radians(6)), synth.StageSpec(5, 0.003, 1, 3, math.radians(2))]


def test_enumerate_multi_equals_single_and_replays_as_graph(orc):
    from paper_2312_08715_gb300 import b3d
    scenes = _scenes(orc)
    M = [16, 8, 32, 5]
    ctxs, items, outs, singles = [], [], [], []
    for k, ((wl, obs, slot), m) in enumerate(zip(scenes, M)):
        ctx = gpu_context(wl.scene, obs)
        b3d.b3d_set_tuning(ctx.h, 64, 128, 0, 1, 4)
        centre = wl.hidden.astype(np.float64).copy()
        centre[:3, 3] += [0.01, -0.008, 0.012]
        G = wl.grid_frame
        singles.append([_np(x).copy() for x in ctx.enumerate_c2f(slot, centre.astype(np.float32), _stages(), wl.lik,
                                                                 m, 100 + k, G)])
        ctx.sync()
        o = (torch.empty((m, 4, 4), device="cuda"), torch.empty(m, device="cuda"), torch.empty(m, device="cuda"))
        outs.append(o)
        sch = b3d.schedule(_stages(), m, 100 + k, G)
        items.append(b3d.c2f_item(ctx.h, slot, centre.astype(np.float32), sch, *o))
        ctxs.append(ctx)
    owner = b3d.Context(0)
    b3d.b3d_set_tuning(owner.h, 64, 128, 0, 1, 4)
    lik = b3d.lik_params(**scenes[0][0].lik)
    b3d.b3d_enumerate_multi(owner.h, items, lik, owner.stream)  # sizes the scratch
    owner.sync()
    for k in range(len(scenes)):
        for got, want in zip(outs[k], singles[k]):
            np.testing.assert_array_equal(_np(got), want)
    # capture the whole batched schedule into a CUDA graph and replay it
    for o in outs:
        for t in o:
            t.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            b3d.b3d_enumerate_multi(owner.h, items, lik, side)
    for rep in range(2):
        for o in outs:
            for t in o:
                t.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for k in range(len(scenes)):
            for got, want in zip(outs[k], singles[k]):
                np.testing.assert_array_equal(_np(got), want)
    owner.sync()
    for c in ctxs + [owner]:
        c.close()


def test_enumerate_c2f_captures_as_graph(orc, single_object):
    from paper_2312_08715_gb300 import b3d
    wl = single_object
    ctx = gpu_context(wl.scene, observed(orc, wl))
    centre = wl.hidden.copy()
    out = (torch.empty((8, 4, 4), device="cuda"), torch.empty(8, device="cuda"), torch.empty(8, device="cuda"))
    eager = [_np(x).copy() for x in ctx.enumerate_c2f(0, centre, _stages(), wl.lik, 8, 5, np.eye(3), out=out)]
    ctx.sync()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            b3d.b3d_enumerate_c2f(ctx.h, 0, centre, b3d.schedule(_stages(), 8, 5, np.eye(3)), b3d.lik_params(**wl.lik),
                                  *out, side)
    for t in out:
        t.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    for got, want in zip(out, eager):
        np.testing.assert_array_equal(_np(got), want)
    ctx.close()


def test_largest_batched_scene_matches_oracle(orc):
    """The largest scene the batched workload draws: 8 objects of 16k-20k voxels (5 mm, about
    1.8 million triangles) at 320x240 (fx = 300), in one batched launch with a small scene,
    its first-stage grid (5^3 translations of 2 cm x 40 perturbations of 10 deg) scored in
    full and checked against the oracle on 40 sampled hypotheses and the GPU's argmax."""
    from paper_2312_08715_gb300 import b3d
    big = synth.tabletop_workload(3, n_objects=8, width=320, height=240, f=300.0, vox_lo=16000, vox_hi=20000,
                                  seed_base=2500)
    assert len(big.scene.meshes) == 10 and big.scene.camera.width == 320
    small = synth.single_object_workload(2)
    obs_b, obs_s = observed(orc, big), observed(orc, small)
    cb, cs = gpu_context(big.scene, obs_b), gpu_context(small.scene, obs_s)
    R = orc.rotation_set(1, 40, math.radians(10.0))
    P = orc.expand(big.centre, big.grid_frame, 5, 0.02, R)
    Pb = torch.as_tensor(P.astype(np.float32), device="cuda")
    Ps = torch.as_tensor(jitter_poses(np.random.default_rng(3), small.hidden, 300), device="cuda")
    ob = torch.full((len(P),), float("nan"), device="cuda")
    os_ = torch.full((300,), float("nan"), device="cuda")
    owner = b3d.Context(0)
    b3d.b3d_score_multi(owner.h, [(cs.h, 0, 300, Ps, os_), (cb.h, big.slot, len(P), Pb, ob)],
                        b3d.lik_params(**big.lik), owner.stream)
    owner.sync()
    ll = _np(ob)
    assert np.isfinite(ll).all() and np.isfinite(_np(os_)).all()
    np.testing.assert_array_equal(_np(cs.score(0, Ps, small.lik)), _np(os_))
    top = int(np.argmax(ll))
    sel = np.unique(np.concatenate([np.random.default_rng(8).choice(len(P), 40, replace=False), [top]]))
    ref = orc.score(big.scene, big.slot, P[sel], big.lik, obs_b)
    check_ll(ll[sel], ref, "8 objects, 320x240")
    best = int(np.argmax(ref["ll"]))
    if sel[best] != top:
        assert ref["ll"][best] - ref["ll"][sel == top][0] <= 2 * ll_tolerance(ref)[best]
    for c in (cb, cs, owner):
        c.close()


def test_autotune_multi_keeps_a_candidate_shape_and_bit_identical_results(orc):
    """The batched autotuner times b3d_enumerate_multi on the items themselves and keeps one
    of its candidate shapes (the owner's, or 128/256-thread CTAs with 64/128-pixel tiles) and
    batch chunks (1-32); the batched results under the kept tuning equal the single-scene
    calls under the same tuning, bit for bit."""
    from paper_2312_08715_gb300 import b3d
    scenes = _scenes(orc)
    M = [16, 8, 32, 5]
    ctxs, items, outs, centres = [], [], [], []
    for k, ((wl, obs, slot), m) in enumerate(zip(scenes, M)):
        ctx = gpu_context(wl.scene, obs)
        centre = wl.hidden.astype(np.float64).copy()
        centre[:3, 3] += [0.01, -0.008, 0.012]
        o = (torch.empty((m, 4, 4), device="cuda"), torch.empty(m, device="cuda"), torch.empty(m, device="cuda"))
        outs.append(o)
        items.append(b3d.c2f_item(ctx.h, slot, centre.astype(np.float32), b3d.schedule(_stages(), m, 200 + k, wl.grid_frame),
                                  *o))
        ctxs.append(ctx)
        centres.append(centre.astype(np.float32))
    owner = b3d.Context(0)
    b3d.b3d_set_tuning(owner.h, 96, 64, 0, 0, 4)
    lik = b3d.lik_params(**scenes[0][0].lik)
    t = b3d.b3d_autotune_multi(owner.h, items, lik, owner.stream)
    owner.sync()
    shapes = [(96, 64)] + [(tw, nt) for nt in (128, 256) for tw in (64, 128)]
    assert (t["tile_w"], t["cta_threads"]) in shapes, t
    assert t["batch_chunk"] in (1, 2, 4, 8, 16, 32), t
    assert b3d.b3d_get_tuning(owner.h) == t
    b3d.b3d_enumerate_multi(owner.h, items, lik, owner.stream)
    owner.sync()
    for k, ((wl, obs, slot), m) in enumerate(zip(scenes, M)):
        b3d.b3d_set_tuning(ctxs[k].h, **t)
        single = [_np(x).copy() for x in ctxs[k].enumerate_c2f(slot, centres[k], _stages(), wl.lik, m, 200 + k,
                                                               wl.grid_frame)]
        ctxs[k].sync()
        for got, want in zip(outs[k], single):
            np.testing.assert_array_equal(_np(got), want)
    for c in ctxs + [owner]:
        c.close()
