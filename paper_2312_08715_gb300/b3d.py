"""Python binding of libb3d: the C ABI of include/b3d.h, name for name, over ctypes.

Argument marshalling only: every step of the path runs in the library's kernels. Device
buffers are passed as integer addresses (for torch tensors, ``t.data_ptr()``) and streams as
integer ``cudaStream_t`` handles (``torch.cuda.current_stream().cuda_stream``); host arrays
are numpy arrays. The module refuses to load without the compiled library: there is no
fallback path.

On top of the raw functions, ``Context`` is a thin convenience wrapper used by the tests
and the benchmark (still marshalling only), and ``ScoreSmooth`` is the
``torch.autograd.Function`` over ``b3d_score_grad``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

B3D_OK = 0
B3D_EINVAL = -1
B3D_ENOMEM = -2
B3D_EBUDGET = -3
B3D_ECUDA = -4
B3D_ETIMEOUT = -5
B3D_ENOTFOUND = -6
B3D_EDEVICE = -7
B3D_EBUSY = -8
B3D_ECLOSED = -9
B3D_MAX_STAGES = 8
B3D_MAX_HALF_WINDOW = 7
B3D_MAX_NOISE_R = 4
B3D_MAX_NOISE_P = 4
B3D_MESH_CLOSED = 1
B3D_NOALLOC_MAX_SCORES = 2147483647
B3D_INSTR_TIMING = 1
B3D_INSTR_WORK = 2
B3D_K_SCORE, B3D_K_RENDER, B3D_K_SCORE_DEPTH, B3D_K_RESAMPLE, B3D_K_SELECT, B3D_K_GRAD, B3D_K_SCENE = range(7)
B3D_K_COUNT = 7

_STATUS = {0: "B3D_OK", -1: "B3D_EINVAL", -2: "B3D_ENOMEM", -3: "B3D_EBUDGET", -4: "B3D_ECUDA",
           -5: "B3D_ETIMEOUT", -6: "B3D_ENOTFOUND", -7: "B3D_EDEVICE", -8: "B3D_EBUSY", -9: "B3D_ECLOSED"}


class b3d_intrinsics(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("near_z", C.c_float), ("far_z", C.c_float)]


class b3d_lik_params(C.Structure):
    _fields_ = [("kind", C.c_int32), ("radius", C.c_float), ("p_outlier", C.c_float), ("half_window", C.c_int32),
                ("volume", C.c_float), ("norm", C.c_float), ("miss_mode", C.c_int32)]


class b3d_stage(C.Structure):
    _fields_ = [("n_per_axis", C.c_int32), ("step", C.c_float), ("rot_kind", C.c_int32), ("n_rot", C.c_int32),
                ("rot_max", C.c_float)]


class b3d_tuning(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("cta_threads", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("high_occupancy", C.c_int32), ("batch_chunk", C.c_int32)]


class b3d_c2f_schedule(C.Structure):
    _fields_ = [("n_stages", C.c_int32), ("stage", b3d_stage * B3D_MAX_STAGES), ("n_particles", C.c_int32),
                ("seed", C.c_uint64), ("grid_frame", C.c_float * 9), ("path_density", C.c_int32)]


class b3d_noise_grid(C.Structure):
    _fields_ = [("kind", C.c_int32), ("half_window", C.c_int32), ("n_radius", C.c_int32), ("n_pout", C.c_int32),
                ("radius", C.c_float * 4), ("p_outlier", C.c_float * 4), ("log_weight", C.c_float * 16),
                ("volume", C.c_float), ("norm", C.c_float), ("miss_mode", C.c_int32)]


class b3d_score_item(C.Structure):
    _fields_ = [("scene", C.c_void_p), ("obj_slot", C.c_int32), ("n_hyp", C.c_int64), ("poses_dev", C.c_void_p),
                ("loglik_dev", C.c_void_p)]


class b3d_c2f_item(C.Structure):
    _fields_ = [("scene", C.c_void_p), ("obj_slot", C.c_int32), ("centre_pose", C.c_float * 16),
                ("centre_dev", C.c_void_p), ("schedule", b3d_c2f_schedule), ("particles_dev", C.c_void_p),
                ("logw_dev", C.c_void_p), ("logq_dev", C.c_void_p), ("map_dev", C.c_void_p)]


class b3d_server_config(C.Structure):
    _fields_ = [("max_sessions", C.c_int32), ("max_batch_items", C.c_int32), ("max_batch_frames", C.c_int32),
                ("max_inflight", C.c_int32),
                ("queue_depth", C.c_int32), ("device_timeout_ms", C.c_int32), ("batch_linger_us", C.c_int32),
                ("lik", b3d_lik_params),
                ("schedule", b3d_c2f_schedule), ("tuning", b3d_tuning)]


class b3d_session_desc(C.Structure):
    _fields_ = [("intr", b3d_intrinsics), ("n_obj", C.c_int32), ("n_track", C.c_int32), ("verts", C.c_void_p),
                ("n_v", C.c_void_p), ("faces", C.c_void_p), ("n_f", C.c_void_p), ("mesh_flags", C.c_void_p),
                ("poses", C.c_void_p), ("seed", C.c_uint64), ("grid_frame", C.c_float * 9)]


class b3d_frame_result(C.Structure):
    _fields_ = [("ticket", C.c_int64), ("session", C.c_int32), ("status", C.c_int32), ("frame_index", C.c_int64),
                ("latency_ms", C.c_double), ("queue_ms", C.c_double), ("batch_frames", C.c_int32),
                ("n_track", C.c_int32)]


class b3d_server_stats(C.Structure):
    _fields_ = [("frames_done", C.c_int64), ("frames_failed", C.c_int64), ("batches", C.c_int64),
                ("hypotheses", C.c_int64), ("sessions", C.c_int32), ("max_batch_frames_seen", C.c_int32),
                ("hbm_budget", C.c_uint64), ("hbm_reserved", C.c_uint64), ("hbm_used", C.c_uint64)]


_P = C.c_void_p
_SIGNATURES = {
    "b3d_create": (C.c_int32, [C.POINTER(C.c_void_p), C.c_int32, C.c_uint64]),
    "b3d_destroy": (C.c_int32, [_P]),
    "b3d_last_error": (C.c_char_p, [_P]),
    "b3d_launch_count": (C.c_int64, [_P]),
    "b3d_load_mesh": (C.c_int32, [_P, _P, C.c_int64, _P, C.c_int64, C.c_int32, C.POINTER(C.c_int32)]),
    "b3d_set_scene": (C.c_int32, [_P, C.POINTER(b3d_intrinsics), C.c_int32, _P, _P, _P, _P]),
    "b3d_set_observation": (C.c_int32, [_P, _P, _P]),
    "b3d_set_object_pose_dev": (C.c_int32, [_P, C.c_int32, _P, _P]),
    "b3d_render_batch": (C.c_int32, [_P, C.c_int32, C.c_int64, _P, _P, _P, _P]),
    "b3d_score_batch": (C.c_int32, [_P, C.c_int32, C.c_int64, _P, C.POINTER(b3d_lik_params), _P, _P]),
    "b3d_score_depth_batch": (C.c_int32, [_P, C.c_int32, C.c_int64, _P, _P, C.POINTER(b3d_lik_params), _P, _P]),
    "b3d_score_noise_batch": (C.c_int32, [_P, C.c_int32, C.c_int64, _P, C.POINTER(b3d_noise_grid), _P, _P, _P]),
    "b3d_render_camera_batch": (C.c_int32, [_P, C.c_int64, _P, _P, _P, _P]),
    "b3d_expand_hypotheses": (C.c_int32, [_P, _P, _P, C.POINTER(b3d_stage), _P, _P]),
    "b3d_lse_resample": (C.c_int32, [_P, C.c_int64, _P, C.c_int32, C.c_uint64, C.c_int32, _P, _P, _P, _P]),
    "b3d_enumerate_c2f": (C.c_int32, [_P, C.c_int32, _P, C.POINTER(b3d_c2f_schedule), C.POINTER(b3d_lik_params),
                                      _P, _P, _P, _P]),
    "b3d_score_multi": (C.c_int32, [_P, C.c_int32, C.POINTER(b3d_score_item), C.POINTER(b3d_lik_params), _P]),
    "b3d_enumerate_multi": (C.c_int32, [_P, C.c_int32, C.POINTER(b3d_c2f_item), C.POINTER(b3d_lik_params), _P]),
    "b3d_autotune_multi": (C.c_int32, [_P, C.c_int32, C.POINTER(b3d_c2f_item), C.POINTER(b3d_lik_params),
                                       C.POINTER(b3d_tuning), _P]),
    "b3d_score_grad": (C.c_int32, [_P, C.c_int32, C.c_int64, _P, C.POINTER(b3d_lik_params), _P, _P, _P, _P, _P]),
    "b3d_refine_smooth": (C.c_int32, [_P, C.c_int32, C.c_int64, _P, C.POINTER(b3d_lik_params), C.c_int32, C.c_float,
                                      C.c_float, C.c_float, C.c_float, _P, _P]),
    "b3d_lse_resample_noalloc": (C.c_int32, [C.c_int64, _P, C.c_int32, C.c_uint64, C.c_int32, _P, _P, _P, _P]),
    "b3d_se3_compose": (C.c_int32, [_P, C.c_int64, _P, _P, _P, _P]),
    "b3d_lse_resample_shard": (C.c_int32, [_P, C.c_int64, _P, C.c_int32, C.c_uint64, C.c_int32, C.c_double, C.c_double,
                                           C.c_double, C.c_int64, _P, _P, _P, _P]),
    "b3d_get_tuning": (C.c_int32, [_P, C.POINTER(b3d_tuning)]),
    "b3d_set_tuning": (C.c_int32, [_P, C.POINTER(b3d_tuning)]),
    "b3d_autotune": (C.c_int32, [_P, C.c_int32, _P, _P, C.POINTER(b3d_stage), C.POINTER(b3d_lik_params),
                                 C.POINTER(b3d_tuning), _P]),
    "b3d_set_instrumentation": (C.c_int32, [_P, C.c_int32]),
    "b3d_kernel_time": (C.c_int32, [_P, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "b3d_work_counters": (C.c_int32, [_P, _P]),
    "b3d_sync": (C.c_int32, [_P, _P]),
    "b3d_server_create": (C.c_int32, [C.POINTER(C.c_void_p), C.c_int32, C.c_uint64, C.POINTER(b3d_server_config)]),
    "b3d_server_destroy": (C.c_int32, [_P]),
    "b3d_server_last_error": (C.c_char_p, []),
    "b3d_session_open": (C.c_int32, [_P, C.POINTER(b3d_session_desc), C.c_int32, C.POINTER(C.c_int32)]),
    "b3d_session_close": (C.c_int32, [_P, C.c_int32]),
    "b3d_frame_submit": (C.c_int32, [_P, C.c_int32, _P, C.c_int32, C.POINTER(C.c_int64)]),
    "b3d_frame_wait": (C.c_int32, [_P, C.c_int64, C.c_int32, C.POINTER(b3d_frame_result), _P, C.c_int32]),
    "b3d_frame_next": (C.c_int32, [_P, C.c_int32, C.POINTER(b3d_frame_result), _P, C.c_int32]),
    "b3d_server_pause": (C.c_int32, [_P, C.c_int32]),
    "b3d_server_get_stats": (C.c_int32, [_P, C.POINTER(b3d_server_stats)]),
    "b3d_session_export": (C.c_int32, [_P, C.c_int32, _P, _P, _P, C.POINTER(C.c_int64)]),
    "b3d_session_import": (C.c_int32, [_P, C.c_int32, _P, _P, _P, C.c_int64]),
    "b3d_frame_seed": (C.c_uint64, [C.c_uint64, C.c_int64, C.c_int32]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libb3d.so (building it in-tree first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libb3d is not built ({_build.LIB} missing); run paper_2312_08715_gb300.build.build()")
    lib = C.CDLL(_build.LIB)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class B3DError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


def _addr(x):
    """Address of a device/host buffer: torch tensor, numpy array, int or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ------------------------------------------------------------------------------------------
# the C ABI, name for name
# ------------------------------------------------------------------------------------------

def b3d_create(device: int = 0, hbm_budget_bytes: int = 0):
    lib = load()
    out = C.c_void_p()
    st = lib.b3d_create(C.byref(out), device, hbm_budget_bytes)
    if st != B3D_OK:
        raise B3DError(st, lib.b3d_last_error(None).decode())
    return out.value


def b3d_destroy(ctx):
    return load().b3d_destroy(ctx)


def b3d_last_error(ctx) -> str:
    return load().b3d_last_error(ctx).decode()


def b3d_launch_count(ctx) -> int:
    return int(load().b3d_launch_count(ctx))


def _check(ctx, st):
    if st != B3D_OK:
        raise B3DError(st, b3d_last_error(ctx))
    return st


def b3d_load_mesh(ctx, verts, faces, flags=B3D_MESH_CLOSED) -> int:
    v = np.ascontiguousarray(verts, dtype=np.float32).reshape(-1, 3)
    f = np.ascontiguousarray(faces, dtype=np.int32).reshape(-1, 3)
    mid = C.c_int32(-1)
    _check(ctx, load().b3d_load_mesh(ctx, v.ctypes.data, v.shape[0], f.ctypes.data, f.shape[0], flags, C.byref(mid)))
    return int(mid.value)


def intrinsics(cam) -> b3d_intrinsics:
    return b3d_intrinsics(int(cam.width), int(cam.height), float(cam.fx), float(cam.fy), float(cam.cx),
                          float(cam.cy), float(cam.near), float(cam.far))


def lik_params(kind=0, radius=0.005, p_outlier=0.01, half_window=1, volume=0.0, norm=0.0, miss_mode=0):
    return b3d_lik_params(int(kind), float(radius), float(p_outlier), int(half_window), float(volume), float(norm),
                          int(miss_mode))


def stage_params(s) -> b3d_stage:
    return b3d_stage(int(s.n_per_axis), float(s.step), int(s.rot_kind), int(s.n_rot), float(s.rot_max))


def schedule(stages, n_particles, seed, grid_frame, path_density=False) -> b3d_c2f_schedule:
    sch = b3d_c2f_schedule()
    sch.path_density = 1 if path_density else 0
    sch.n_stages = len(stages)
    for k, s in enumerate(stages):
        sch.stage[k] = stage_params(s)
    sch.n_particles = int(n_particles)
    sch.seed = int(seed)
    g = np.asarray(grid_frame, dtype=np.float32).reshape(9)
    for k in range(9):
        sch.grid_frame[k] = float(g[k])
    return sch


def b3d_set_scene(ctx, intr: b3d_intrinsics, mesh_ids, poses, obs_depth_dev, stream=None):
    ids = np.ascontiguousarray(mesh_ids, dtype=np.int32)
    P = np.ascontiguousarray(poses, dtype=np.float32).reshape(-1, 16)
    return _check(ctx, load().b3d_set_scene(ctx, C.byref(intr), ids.size, ids.ctypes.data, P.ctypes.data,
                                            _addr(obs_depth_dev), _stream(stream)))


def b3d_set_observation(ctx, obs_depth_dev, stream=None):
    return _check(ctx, load().b3d_set_observation(ctx, _addr(obs_depth_dev), _stream(stream)))


def b3d_set_object_pose_dev(ctx, obj, pose_dev, stream=None):
    return _check(ctx, load().b3d_set_object_pose_dev(ctx, obj, _addr(pose_dev), _stream(stream)))


def b3d_render_batch(ctx, obj_slot, n_hyp, poses_dev, depth_dev, triid_dev=None, stream=None):
    return _check(ctx, load().b3d_render_batch(ctx, obj_slot, n_hyp, _addr(poses_dev), _addr(depth_dev),
                                               _addr(triid_dev), _stream(stream)))


def b3d_score_batch(ctx, obj_slot, n_hyp, poses_dev, lik: b3d_lik_params, loglik_dev, stream=None):
    return _check(ctx, load().b3d_score_batch(ctx, obj_slot, n_hyp, _addr(poses_dev), C.byref(lik),
                                              _addr(loglik_dev), _stream(stream)))


def b3d_score_depth_batch(ctx, obj_slot, n_hyp, depth_dev, triid_dev, lik: b3d_lik_params, loglik_dev, stream=None):
    return _check(ctx, load().b3d_score_depth_batch(ctx, obj_slot, n_hyp, _addr(depth_dev), _addr(triid_dev), C.byref(lik),
                                                    _addr(loglik_dev), _stream(stream)))


def b3d_render_camera_batch(ctx, n_hyp, poses_dev, depth_dev, triid_dev=None, stream=None):
    return _check(ctx, load().b3d_render_camera_batch(ctx, n_hyp, _addr(poses_dev), _addr(depth_dev), _addr(triid_dev),
                                                      _stream(stream)))


def noise_grid(kind, radii, p_outliers, half_window=1, log_weight=None, volume=0.0, norm=0.0,
               miss_mode=0) -> b3d_noise_grid:
    """Grid of len(radii) x len(p_outliers) settings; log_weight [n_r * n_p] (default 0)."""
    g = b3d_noise_grid()
    g.kind, g.half_window = int(kind), int(half_window)
    g.n_radius, g.n_pout = len(radii), len(p_outliers)
    for i, r in enumerate(radii):
        g.radius[i] = float(r)
    for j, p in enumerate(p_outliers):
        g.p_outlier[j] = float(p)
    lw = np.zeros(len(radii) * len(p_outliers)) if log_weight is None else np.asarray(log_weight, np.float64).ravel()
    for k, v in enumerate(lw):
        g.log_weight[k] = float(v)
    g.volume, g.norm, g.miss_mode = float(volume), float(norm), int(miss_mode)
    return g


def b3d_score_noise_batch(ctx, obj_slot, n_hyp, poses_dev, grid: b3d_noise_grid, loglik_dev, marginal_dev,
                          stream=None):
    return _check(ctx, load().b3d_score_noise_batch(ctx, obj_slot, n_hyp, _addr(poses_dev), C.byref(grid),
                                                    _addr(loglik_dev), _addr(marginal_dev), _stream(stream)))


def b3d_expand_hypotheses(ctx, centre_pose, grid_frame, stage: b3d_stage, poses_dev, stream=None):
    c = np.ascontiguousarray(centre_pose, dtype=np.float32).reshape(16)
    g = np.ascontiguousarray(grid_frame, dtype=np.float32).reshape(9)
    return _check(ctx, load().b3d_expand_hypotheses(ctx, c.ctypes.data, g.ctypes.data, C.byref(stage),
                                                    _addr(poses_dev), _stream(stream)))


def b3d_lse_resample(ctx, n, loglik_dev, m, seed, stage, logz_dev, idx_dev, logq_dev, stream=None):
    return _check(ctx, load().b3d_lse_resample(ctx, n, _addr(loglik_dev), m, seed, stage, _addr(logz_dev),
                                               _addr(idx_dev), _addr(logq_dev), _stream(stream)))


def b3d_lse_resample_shard(ctx, n, loglik_dev, m, seed, stage, mass_before, mass, logz_global, index_base, logz_dev,
                           idx_dev, logq_dev, stream=None):
    return _check(ctx, load().b3d_lse_resample_shard(ctx, n, _addr(loglik_dev), m, seed, stage, float(mass_before),
                                                     float(mass), float(logz_global), int(index_base), _addr(logz_dev),
                                                     _addr(idx_dev), _addr(logq_dev), _stream(stream)))


def b3d_lse_resample_noalloc(n, loglik_dev, m, seed, stage, logz_dev, idx_dev, logq_dev, stream=None):
    """Context-free, allocation-free log-sum-exp + resampling (scratch is a fixed array in
    the library; calls that overlap on the GPU race). Raises B3DError on a non-zero status."""
    st = load().b3d_lse_resample_noalloc(n, _addr(loglik_dev), m, seed, stage, _addr(logz_dev), _addr(idx_dev),
                                         _addr(logq_dev), _stream(stream))
    if st != B3D_OK:
        raise B3DError(st, "b3d_lse_resample_noalloc failed (no context: status only)")
    return st


def b3d_enumerate_c2f(ctx, obj_slot, centre_pose, sch: b3d_c2f_schedule, lik: b3d_lik_params, particles_dev,
                      logw_dev, logq_dev, stream=None):
    c = np.ascontiguousarray(centre_pose, dtype=np.float32).reshape(16)
    return _check(ctx, load().b3d_enumerate_c2f(ctx, obj_slot, c.ctypes.data, C.byref(sch), C.byref(lik),
                                                _addr(particles_dev), _addr(logw_dev), _addr(logq_dev),
                                                _stream(stream)))


def b3d_score_grad(ctx, obj_slot, n_hyp, poses_dev, lik: b3d_lik_params, loglik_dev, dpose_dev=None,
                   dsigma_dev=None, dpout_dev=None, stream=None):
    return _check(ctx, load().b3d_score_grad(ctx, obj_slot, n_hyp, _addr(poses_dev), C.byref(lik), _addr(loglik_dev),
                                             _addr(dpose_dev), _addr(dsigma_dev), _addr(dpout_dev),
                                             _stream(stream)))


def b3d_refine_smooth(ctx, obj_slot, n_hyp, poses_dev, lik: b3d_lik_params, n_steps, lr, beta1=0.9, beta2=0.999,
                      eps=1e-8, loglik_dev=None, stream=None):
    return _check(ctx, load().b3d_refine_smooth(ctx, obj_slot, n_hyp, _addr(poses_dev), C.byref(lik), n_steps, lr,
                                                beta1, beta2, eps, _addr(loglik_dev), _stream(stream)))


def b3d_get_tuning(ctx) -> dict:
    t = b3d_tuning()
    _check(ctx, load().b3d_get_tuning(ctx, C.byref(t)))
    return dict(tile_w=t.tile_w, cta_threads=t.cta_threads, ctas_per_sm=t.ctas_per_sm, high_occupancy=t.high_occupancy,
                batch_chunk=t.batch_chunk)


def b3d_set_tuning(ctx, tile_w=64, cta_threads=256, ctas_per_sm=0, high_occupancy=0, batch_chunk=4):
    return _check(ctx, load().b3d_set_tuning(ctx, C.byref(b3d_tuning(tile_w, cta_threads, ctas_per_sm,
                                                                       high_occupancy, batch_chunk))))


def b3d_autotune(ctx, obj_slot, centre_pose, grid_frame, stage: b3d_stage, lik: b3d_lik_params, stream=None) -> dict:
    c = np.ascontiguousarray(centre_pose, dtype=np.float32).reshape(16)
    g = np.ascontiguousarray(grid_frame, dtype=np.float32).reshape(9)
    t = b3d_tuning()
    _check(ctx, load().b3d_autotune(ctx, obj_slot, c.ctypes.data, g.ctypes.data, C.byref(stage), C.byref(lik),
                                    C.byref(t), _stream(stream)))
    return dict(tile_w=t.tile_w, cta_threads=t.cta_threads, ctas_per_sm=t.ctas_per_sm, high_occupancy=t.high_occupancy,
                batch_chunk=t.batch_chunk)


def b3d_score_multi(owner, items, lik: b3d_lik_params, stream=None):
    """items: sequence of (scene ctx handle, obj_slot, n_hyp, poses_dev, loglik_dev)."""
    arr = (b3d_score_item * len(items))(*[b3d_score_item(sc, slot, n, _addr(p), _addr(o)) for sc, slot, n, p, o in items])
    return _check(owner, load().b3d_score_multi(owner, len(items), arr, C.byref(lik), _stream(stream)))


def c2f_item(scene, obj_slot, centre_pose, sch: b3d_c2f_schedule, particles_dev, logw_dev, logq_dev,
             centre_dev=None, map_dev=None) -> b3d_c2f_item:
    it = b3d_c2f_item()
    it.scene = scene
    it.obj_slot = int(obj_slot)
    c = np.asarray(centre_pose if centre_pose is not None else np.eye(4), dtype=np.float32).reshape(16)
    for k in range(16):
        it.centre_pose[k] = float(c[k])
    it.centre_dev = _addr(centre_dev)
    it.schedule = sch
    it.particles_dev = _addr(particles_dev)
    it.logw_dev = _addr(logw_dev)
    it.logq_dev = _addr(logq_dev)
    it.map_dev = _addr(map_dev)
    return it


def b3d_enumerate_multi(owner, items, lik: b3d_lik_params, stream=None):
    """items: sequence of b3d_c2f_item (see c2f_item)."""
    arr = (b3d_c2f_item * len(items))(*items)
    return _check(owner, load().b3d_enumerate_multi(owner, len(items), arr, C.byref(lik), _stream(stream)))


def b3d_autotune_multi(owner, items, lik: b3d_lik_params, stream=None) -> dict:
    """items: sequence of b3d_c2f_item; returns the tuning kept in the owner."""
    arr = (b3d_c2f_item * len(items))(*items)
    t = b3d_tuning()
    _check(owner, load().b3d_autotune_multi(owner, len(items), arr, C.byref(lik), C.byref(t), _stream(stream)))
    return dict(tile_w=t.tile_w, cta_threads=t.cta_threads, ctas_per_sm=t.ctas_per_sm, high_occupancy=t.high_occupancy,
                batch_chunk=t.batch_chunk)


def b3d_set_instrumentation(ctx, flags):
    return _check(ctx, load().b3d_set_instrumentation(ctx, flags))


def b3d_kernel_time(ctx, kernel_class):
    ms, n = C.c_double(0), C.c_int64(0)
    _check(ctx, load().b3d_kernel_time(ctx, kernel_class, C.byref(ms), C.byref(n)))
    return float(ms.value), int(n.value)


def b3d_work_counters(ctx):
    out = np.zeros(8, np.int64)
    _check(ctx, load().b3d_work_counters(ctx, out.ctypes.data))
    return out


def b3d_sync(ctx, stream=None):
    return _check(ctx, load().b3d_sync(ctx, _stream(stream)))


# ------------------------------------------------------------------------------------------
# thin convenience layer (torch tensors for device memory and streams)
# ------------------------------------------------------------------------------------------

# ------------------------------------------------------------------------------------------
# serving: the tracking server
# ------------------------------------------------------------------------------------------

def _scheck(st):
    if st != B3D_OK:
        raise B3DError(st, load().b3d_server_last_error().decode())
    return st


def server_config(lik: b3d_lik_params, sch: b3d_c2f_schedule, max_sessions=32, max_batch_items=256, max_inflight=2,
                  queue_depth=4, device_timeout_ms=0, tuning=None, max_batch_frames=0,
                  batch_linger_us=0) -> b3d_server_config:
    c = b3d_server_config()
    c.max_sessions = int(max_sessions)
    c.max_batch_items = int(max_batch_items)
    c.max_batch_frames = int(max_batch_frames)
    c.max_inflight = int(max_inflight)
    c.queue_depth = int(queue_depth)
    c.device_timeout_ms = int(device_timeout_ms)
    c.batch_linger_us = int(batch_linger_us)
    c.lik = lik
    c.schedule = sch
    if tuning is not None:
        c.tuning = b3d_tuning(int(tuning["tile_w"]), int(tuning["cta_threads"]), int(tuning["ctas_per_sm"]),
                              int(tuning["high_occupancy"]), int(tuning["batch_chunk"]))
    return c


def b3d_frame_seed(seed, frame, obj) -> int:
    return int(load().b3d_frame_seed(int(seed), int(frame), int(obj)))


def b3d_server_last_error() -> str:
    return load().b3d_server_last_error().decode()


def b3d_server_create(device: int, hbm_budget_bytes: int, cfg: b3d_server_config):
    out = C.c_void_p()
    _scheck(load().b3d_server_create(C.byref(out), int(device), int(hbm_budget_bytes), C.byref(cfg)))
    return out.value


def b3d_server_destroy(srv):
    return _scheck(load().b3d_server_destroy(srv))


def b3d_session_open(srv, desc: b3d_session_desc, timeout_ms=0) -> int:
    sid = C.c_int32(-1)
    _scheck(load().b3d_session_open(srv, C.byref(desc), int(timeout_ms), C.byref(sid)))
    return int(sid.value)


def b3d_session_close(srv, sid):
    return _scheck(load().b3d_session_close(srv, int(sid)))


def b3d_frame_submit(srv, sid, depth, timeout_ms=0) -> int:
    D = np.ascontiguousarray(depth, dtype=np.float32)
    t = C.c_int64(0)
    _scheck(load().b3d_frame_submit(srv, int(sid), D.ctypes.data, int(timeout_ms), C.byref(t)))
    return int(t.value)


def b3d_frame_wait(srv, ticket, timeout_ms, res: b3d_frame_result, poses):
    P = poses
    return _scheck(load().b3d_frame_wait(srv, int(ticket), int(timeout_ms), C.byref(res), _addr(P),
                                         0 if P is None else int(P.size)))


def b3d_frame_next(srv, timeout_ms, res: b3d_frame_result, poses):
    P = poses
    return _scheck(load().b3d_frame_next(srv, int(timeout_ms), C.byref(res), _addr(P), 0 if P is None else int(P.size)))


def b3d_server_pause(srv, paused):
    return _scheck(load().b3d_server_pause(srv, 1 if paused else 0))


def b3d_server_get_stats(srv) -> dict:
    s = b3d_server_stats()
    _scheck(load().b3d_server_get_stats(srv, C.byref(s)))
    return {k: getattr(s, k) for k, _ in b3d_server_stats._fields_}


def b3d_session_export(srv, sid, poses, particles, logw) -> int:
    nxt = C.c_int64(0)
    _scheck(load().b3d_session_export(srv, int(sid), _addr(poses), _addr(particles), _addr(logw), C.byref(nxt)))
    return int(nxt.value)


def b3d_session_import(srv, sid, poses, particles, logw, next_frame):
    return _scheck(load().b3d_session_import(srv, int(sid), _addr(poses), _addr(particles), _addr(logw),
                                             int(next_frame)))


class Server:
    """Convenience wrapper over the b3d_server_* / b3d_session_* / b3d_frame_* functions
    (marshalling only)."""

    def __init__(self, cfg: b3d_server_config, device: int = 0, hbm_budget_bytes: int = 0):
        self.h = b3d_server_create(device, hbm_budget_bytes, cfg)
        self.cfg = cfg
        self._n_track = {}

    def close(self):
        if self.h:
            b3d_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def open_session(self, cam, meshes, poses, n_track, seed, closed=True, grid_frame=None, timeout_ms=0) -> int:
        """meshes: list of (verts [n,3], faces [m,3]); poses [n_obj, 4, 4] (tracked first);
        closed: one flag for all meshes or one per mesh."""
        vs = [np.ascontiguousarray(v, dtype=np.float32).reshape(-1, 3) for v, _ in meshes]
        fs = [np.ascontiguousarray(f, dtype=np.int32).reshape(-1, 3) for _, f in meshes]
        n = len(meshes)
        vp = (C.c_void_p * n)(*[v.ctypes.data for v in vs])
        fp = (C.c_void_p * n)(*[f.ctypes.data for f in fs])
        nv = np.array([v.shape[0] for v in vs], dtype=np.int64)
        nf = np.array([f.shape[0] for f in fs], dtype=np.int64)
        cl = [closed] * n if isinstance(closed, bool) else list(closed)
        fl = np.array([B3D_MESH_CLOSED if c else 0 for c in cl], dtype=np.int32)
        P = np.ascontiguousarray(poses, dtype=np.float32).reshape(n, 16)
        d = b3d_session_desc()
        d.intr = intrinsics(cam)
        d.n_obj = n
        d.n_track = int(n_track)
        d.verts = C.cast(vp, C.c_void_p)
        d.n_v = nv.ctypes.data
        d.faces = C.cast(fp, C.c_void_p)
        d.n_f = nf.ctypes.data
        d.mesh_flags = fl.ctypes.data
        d.poses = P.ctypes.data
        d.seed = int(seed)
        if grid_frame is not None:
            g = np.asarray(grid_frame, dtype=np.float32).reshape(9)
            for k in range(9):
                d.grid_frame[k] = float(g[k])
        sid = b3d_session_open(self.h, d, timeout_ms)
        self._n_track[sid] = int(n_track)
        return sid

    def close_session(self, sid):
        b3d_session_close(self.h, sid)

    def submit(self, sid, depth, timeout_ms=0) -> int:
        return b3d_frame_submit(self.h, sid, depth, timeout_ms)

    def _result(self, res, P):
        r = {k: getattr(res, k) for k, _ in b3d_frame_result._fields_}
        r["poses"] = P[:res.n_track].copy()
        return r

    def wait(self, ticket, timeout_ms=10000) -> dict:
        res = b3d_frame_result()
        P = np.zeros((self.cfg.max_batch_items, 4, 4), dtype=np.float32)
        b3d_frame_wait(self.h, ticket, timeout_ms, res, P)
        return self._result(res, P)

    def next(self, timeout_ms=10000) -> dict:
        res = b3d_frame_result()
        P = np.zeros((self.cfg.max_batch_items, 4, 4), dtype=np.float32)
        b3d_frame_next(self.h, timeout_ms, res, P)
        return self._result(res, P)

    def pause(self, paused=True):
        b3d_server_pause(self.h, paused)

    def stats(self) -> dict:
        return b3d_server_get_stats(self.h)

    def export_session(self, sid):
        nt, M = self._n_track[int(sid)], self.cfg.schedule.n_particles
        poses = np.zeros((nt, 4, 4), np.float32)
        part = np.zeros((nt, M, 4, 4), np.float32)
        logw = np.zeros((nt, M), np.float32)
        nxt = b3d_session_export(self.h, sid, poses, part, logw)
        return {"poses": poses, "particles": part, "logw": logw, "next_frame": nxt}

    def import_session(self, sid, state):
        P = np.ascontiguousarray(state["poses"], dtype=np.float32)
        part = np.ascontiguousarray(state["particles"], dtype=np.float32)
        lw = np.ascontiguousarray(state["logw"], dtype=np.float32)
        b3d_session_import(self.h, sid, P, part, lw, state["next_frame"])


class Context:
    """Owns a b3d context; methods allocate outputs with torch and call the C ABI."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.h = b3d_create(device, hbm_budget_bytes)
        self.cam = None
        self.n_obj = 0

    def close(self):
        if self.h:
            b3d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def stream(self):
        return self.torch.cuda.current_stream(self.device)

    def launches(self) -> int:
        return b3d_launch_count(self.h)

    def load_mesh(self, mesh, closed=True) -> int:
        return b3d_load_mesh(self.h, mesh.verts, mesh.faces, B3D_MESH_CLOSED if closed else 0)

    def set_scene(self, cam, mesh_ids, poses, obs_depth):
        obs = self._dev(obs_depth, self.torch.float32)
        b3d_set_scene(self.h, intrinsics(cam), mesh_ids, poses, obs, self.stream)
        self.cam = cam
        self.n_obj = len(mesh_ids)
        self._obs = obs  # keep alive until the stream has consumed it

    def set_observation(self, obs_depth):
        obs = self._dev(obs_depth, self.torch.float32)
        b3d_set_observation(self.h, obs, self.stream)
        self._obs = obs

    def _dev(self, x, dtype):
        t = self.torch
        if isinstance(x, t.Tensor):
            return x.to(device=self.device, dtype=dtype).contiguous()
        return t.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=self.device)

    def render(self, slot, poses, want_tid=True):
        P = self._dev(poses, self.torch.float32).reshape(-1, 16)
        n = P.shape[0]
        H, W = self.cam.height, self.cam.width
        depth = self.torch.empty((n, H, W), dtype=self.torch.float32, device=self.device)
        tid = self.torch.empty((n, H, W), dtype=self.torch.int32, device=self.device) if want_tid else None
        b3d_render_batch(self.h, slot, n, P, depth, tid, self.stream)
        return depth, tid

    def score(self, slot, poses, lik: dict, out=None):
        P = self._dev(poses, self.torch.float32).reshape(-1, 16)
        n = P.shape[0]
        ll = out if out is not None else self.torch.empty(n, dtype=self.torch.float32, device=self.device)
        b3d_score_batch(self.h, slot, n, P, lik_params(**lik), ll, self.stream)
        return ll

    def render_camera(self, poses, want_tid=True, out=None):
        """Camera hypotheses poses [n, 4, 4] (camera_from_world); the scene poses are world poses."""
        t = self.torch
        P = self._dev(poses, t.float32).reshape(-1, 16)
        n = P.shape[0]
        H, W = self.cam.height, self.cam.width
        if out is None:
            depth = t.empty((n, H, W), dtype=t.float32, device=self.device)
            tid = t.empty((n, H, W), dtype=t.int32, device=self.device) if want_tid else None
        else:
            depth, tid = out
        b3d_render_camera_batch(self.h, n, P, depth, tid, self.stream)
        return depth, tid

    def score_noise(self, slot, poses, grid: b3d_noise_grid):
        """Returns (loglik [n, n_r * n_p], marginal [n])."""
        t = self.torch
        P = self._dev(poses, t.float32).reshape(-1, 16)
        n = P.shape[0]
        ll = t.empty((n, grid.n_radius * grid.n_pout), dtype=t.float32, device=self.device)
        marg = t.empty(n, dtype=t.float32, device=self.device)
        b3d_score_noise_batch(self.h, slot, n, P, grid, ll, marg, self.stream)
        return ll, marg

    def score_depth(self, depth, lik: dict, tid=None, slot=-1):
        """Sum of l_i of each image; slot: the object the images re-pose (-1: none), which
        only narrows the region compared against the scene."""
        n = depth.shape[0]
        ll = self.torch.empty(n, dtype=self.torch.float32, device=self.device)
        b3d_score_depth_batch(self.h, slot, n, depth, tid, lik_params(**lik), ll, self.stream)
        return ll

    def expand(self, centre, grid_frame, stage):
        n = stage.n_per_axis ** 3 * stage.n_rot
        poses = self.torch.empty((n, 4, 4), dtype=self.torch.float32, device=self.device)
        b3d_expand_hypotheses(self.h, centre, grid_frame, stage_params(stage), poses, self.stream)
        return poses

    def lse_resample(self, ll, m, seed, stage):
        t = self.torch
        logz = t.empty(1, dtype=t.float32, device=self.device)
        idx = t.empty(max(m, 1), dtype=t.int32, device=self.device)
        logq = t.empty(max(m, 1), dtype=t.float32, device=self.device)
        b3d_lse_resample(self.h, ll.numel(), ll, m, seed, stage, logz, idx, logq, self.stream)
        return logz, idx[:m], logq[:m]

    def lse_resample_shard(self, ll, m, seed, stage, mass_before, mass, logz_global, index_base):
        """This rank's draws of a categorical split over ranks (idx -1 where another rank owns
        the draw), and its shard's own log normaliser."""
        t = self.torch
        logz = t.empty(1, dtype=t.float32, device=self.device)
        idx = t.empty(max(m, 1), dtype=t.int32, device=self.device)
        logq = t.empty(max(m, 1), dtype=t.float32, device=self.device)
        b3d_lse_resample_shard(self.h, ll.numel(), ll, m, seed, stage, mass_before, mass, logz_global, index_base, logz,
                               idx, logq, self.stream)
        return logz, idx[:m], logq[:m]

    def enumerate_c2f(self, slot, centre, stages, lik: dict, n_particles, seed, grid_frame, out=None,
                      path_density=False):
        t = self.torch
        if out is None:
            out = (t.empty((n_particles, 4, 4), dtype=t.float32, device=self.device),
                   t.empty(n_particles, dtype=t.float32, device=self.device),
                   t.empty(n_particles, dtype=t.float32, device=self.device))
        particles, logw, logq = out
        b3d_enumerate_c2f(self.h, slot, centre, schedule(stages, n_particles, seed, grid_frame, path_density),
                          lik_params(**lik),
                          particles, logw, logq, self.stream)
        return particles, logw, logq

    def score_grad(self, slot, poses, lik: dict):
        t = self.torch
        P = self._dev(poses, t.float32).reshape(-1, 16)
        n = P.shape[0]
        ll = t.empty(n, dtype=t.float32, device=self.device)
        dpose = t.empty((n, 6), dtype=t.float32, device=self.device)
        ds = t.empty(n, dtype=t.float32, device=self.device)
        dp = t.empty(n, dtype=t.float32, device=self.device)
        b3d_score_grad(self.h, slot, n, P, lik_params(**lik), ll, dpose, ds, dp, self.stream)
        return ll, dpose, ds, dp

    def se3_compose(self, xi, poses, out=None):
        """Exp(xi^) T for twists xi [n, 6] (v, w) and poses [n, 4, 4] (a new tensor, or out)."""
        t = self.torch
        x = self._dev(xi, t.float32).reshape(-1, 6)
        P = self._dev(poses, t.float32).reshape(-1, 16)
        if out is None:
            out = t.empty((P.shape[0], 4, 4), dtype=t.float32, device=self.device)
        b3d_se3_compose(self.h, P.shape[0], x, P, out, self.stream)
        return out

    def refine(self, slot, poses, lik: dict, n_steps, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        """Adam refinement of poses [n, 4, 4] under the smooth likelihood, all on the device;
        returns the refined poses (a new tensor) and the log-likelihood the last step scored."""
        t = self.torch
        P = self._dev(poses, t.float32).reshape(-1, 16).clone()
        ll = t.empty(P.shape[0], dtype=t.float32, device=self.device)
        b3d_refine_smooth(self.h, slot, P.shape[0], P, lik_params(**lik), n_steps, lr, beta1, beta2, eps, ll,
                          self.stream)
        return P.reshape(-1, 4, 4), ll

    def set_object_pose_dev(self, obj, pose_dev):
        b3d_set_object_pose_dev(self.h, obj, pose_dev, self.stream)

    def sync(self):
        b3d_sync(self.h, self.stream)


def b3d_se3_compose(ctx, n, xi_dev, poses_dev, out_dev, stream=None):
    return _check(ctx, load().b3d_se3_compose(ctx, n, _addr(xi_dev), _addr(poses_dev), _addr(out_dev), _stream(stream)))


def make_score_smooth():
    """Build the autograd.Function over b3d_score_grad (imports torch lazily)."""
    import torch

    class ScoreSmooth(torch.autograd.Function):
        """loglik = score of poses Exp(xi^) T0 under the smooth likelihood with noise
        (sigma, p_out); gradients w.r.t. xi (exact at xi = 0: re-base T0 after each step),
        sigma and p_out from the library's backward kernel. sigma and p_out may be plain
        floats (no gradient; the only form that can be captured in a CUDA graph, since a
        device scalar would be read back to the host) or scalar tensors."""

        @staticmethod
        def forward(fctx, xi, sigma, p_out, b3d_ctx, slot, T0, half_window):
            poses = b3d_ctx.se3_compose(xi.detach(), T0)
            lik = dict(kind=1, radius=float(sigma), p_outlier=float(p_out), half_window=int(half_window))
            ll, dpose, ds, dp = b3d_ctx.score_grad(slot, poses, lik)
            fctx.save_for_backward(dpose, ds, dp)
            return ll

        @staticmethod
        def backward(fctx, g):
            dpose, ds, dp = fctx.saved_tensors
            need = fctx.needs_input_grad
            gs = (g * ds).sum().reshape(()) if need[1] else None
            gp = (g * dp).sum().reshape(()) if need[2] else None
            return (g[:, None] * dpose if need[0] else None, gs, gp, None, None, None, None)

    return ScoreSmooth
