"""Python wrapper of the FP64 CPU oracle (``b3d_oracle.c``).

TEST INFRASTRUCTURE. Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this module. The product library never imports it, and it
shares no code with the CUDA path: it takes plain numpy arrays (float64) and the seeded
inputs of ``paper_2312_08715_gb300.synth``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import types

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "b3d_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liborc.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available). Returns the library path."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("near_z", C.c_double), ("far_z", C.c_double)]


class _Lik(C.Structure):
    _fields_ = [("kind", C.c_int32), ("radius", C.c_double), ("p_outlier", C.c_double),
                ("half_window", C.c_int32), ("volume", C.c_double), ("norm", C.c_double),
                ("miss_mode", C.c_int32)]


class _Scene(C.Structure):
    _fields_ = [("n_obj", C.c_int32), ("v_off", C.c_void_p), ("f_off", C.c_void_p),
                ("verts", C.c_void_p), ("faces", C.c_void_p), ("poses", C.c_void_p)]


class _Stage(C.Structure):
    _fields_ = [("n_per_axis", C.c_int32), ("step", C.c_double), ("rot_kind", C.c_int32),
                ("n_rot", C.c_int32), ("rot_max", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _lib.orc_frustum_volume.restype = C.c_double
        _lib.orc_uniform24.restype = C.c_double
        _lib.orc_uniform24.argtypes = [C.c_uint64]
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def camera(cam) -> _Camera:
    return _Camera(int(cam.width), int(cam.height), float(cam.fx), float(cam.fy), float(cam.cx),
                   float(cam.cy), float(cam.near), float(cam.far))


def lik(kind=0, radius=0.005, p_outlier=0.01, half_window=1, volume=0.0, norm=0.0, miss_mode=0) -> _Lik:
    return _Lik(int(kind), float(radius), float(p_outlier), int(half_window), float(volume), float(norm),
                int(miss_mode))


class SceneArrays:
    """Flattened scene for the oracle: keeps the numpy buffers alive with the struct."""

    def __init__(self, scene, poses=None):
        meshes = scene.meshes
        self.cam = camera(scene.camera)
        self.v_off = np.cumsum([0] + [m.verts.shape[0] for m in meshes]).astype(np.int64)
        self.f_off = np.cumsum([0] + [m.faces.shape[0] for m in meshes]).astype(np.int64)
        self.verts = _f64(np.concatenate([m.verts for m in meshes]))
        self.faces = np.ascontiguousarray(np.concatenate([m.faces for m in meshes]), dtype=np.int32)
        self.poses = _f64((scene.poses if poses is None else poses).reshape(-1, 16))
        self.st = _Scene(len(meshes), _p(self.v_off), _p(self.f_off), _p(self.verts), _p(self.faces),
                         _p(self.poses))
        self.H, self.W = int(scene.camera.height), int(scene.camera.width)


def frustum_volume(cam) -> float:
    return float(lib().orc_frustum_volume(C.byref(camera(cam))))


def render(scene, slot=-1, slot_pose=None, edge_tol=0.0, z_tol=0.0, want_flags=False, arrays=None):
    sa = arrays or SceneArrays(scene)
    depth = np.empty((sa.H, sa.W), np.float64)
    triid = np.empty((sa.H, sa.W), np.int32)
    flags = np.empty((sa.H, sa.W), np.uint8) if want_flags else None
    sp = _f64(slot_pose).reshape(16) if slot_pose is not None else None
    rc = lib().orc_render(C.byref(sa.cam), C.byref(sa.st), C.c_int32(slot), _p(sp), C.c_double(edge_tol),
                          C.c_double(z_tol), _p(depth), _p(triid), _p(flags))
    assert rc == 0, rc
    return (depth, triid, flags) if want_flags else (depth, triid)


def render_fixed(scene, slot, slot_pose, triid, arrays=None):
    sa = arrays or SceneArrays(scene)
    depth = np.empty((sa.H, sa.W), np.float64)
    tid = np.ascontiguousarray(triid, dtype=np.int32)
    rc = lib().orc_render_fixed(C.byref(sa.cam), C.byref(sa.st), C.c_int32(slot), _p(_f64(slot_pose).reshape(16)),
                                _p(tid), _p(depth))
    assert rc == 0, rc
    return depth


def pixel_loglik(cam, lk: dict, depth_ren, triid_ren, depth_obs, border_tol=0.0):
    c = camera(cam)
    H, W = int(cam.height), int(cam.width)
    ell = np.empty((H, W), np.float64)
    cnt = np.empty((H, W), np.int32)
    ss = np.empty((H, W), np.float64)
    nb = C.c_int64(0)
    dr = _f64(depth_ren)
    tr = np.ascontiguousarray(triid_ren, dtype=np.int32) if triid_ren is not None else None
    do = _f64(depth_obs)
    rc = lib().orc_pixel_loglik(C.byref(c), C.byref(lik(**lk)), _p(dr), _p(tr), _p(do), C.c_double(border_tol),
                                _p(ell), _p(cnt), _p(ss), C.byref(nb))
    assert rc == 0, rc
    return ell, cnt, ss, int(nb.value)


def score(scene, slot, poses, lk: dict, depth_obs, edge_tol=1e-4, z_tol=1e-5, border_tol=1e-3, n_threads=0,
          flags=True, arrays=None):
    """Per-hypothesis ll, with (when flags) scale, ambiguity bound, #flagged px, #borderline."""
    sa = arrays or SceneArrays(scene)
    P = _f64(poses).reshape(-1, 16)
    n = P.shape[0]
    ll = np.empty(n, np.float64)
    out = dict(ll=ll)
    scale = bound = nf = nb = None
    if flags:
        scale, bound = np.empty(n), np.empty(n)
        nf, nb = np.empty(n, np.int32), np.empty(n, np.int32)
        out.update(scale=scale, bound=bound, n_flag=nf, n_border=nb)
    rc = lib().orc_score(C.byref(sa.cam), C.byref(sa.st), C.c_int32(slot), C.c_int64(n), _p(P), C.byref(lik(**lk)),
                         _p(_f64(depth_obs)), C.c_double(edge_tol), C.c_double(z_tol), C.c_double(border_tol),
                         _p(ll), _p(scale), _p(bound), _p(nf), _p(nb), C.c_int32(n_threads))
    assert rc == 0, rc
    return out


def lse(ll):
    ll = _f64(ll)
    z = C.c_double(0)
    logp = np.empty_like(ll)
    rc = lib().orc_lse(C.c_int64(ll.size), _p(ll), C.byref(z), _p(logp))
    assert rc == 0, rc
    return float(z.value), logp


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.empty(4, np.uint64)
    lib().orc_philox4x64(_p(c), _p(k), _p(out))
    return out


def uniform24(x) -> float:
    return float(lib().orc_uniform24(C.c_uint64(int(x))))


def resample(ll, m, seed, stage):
    ll = _f64(ll)
    idx = np.empty(m, np.int32)
    logq = np.empty(m, np.float64)
    margin = np.empty(m, np.float64)
    rc = lib().orc_resample(C.c_int64(ll.size), _p(ll), C.c_int32(m), C.c_uint64(seed), C.c_int32(stage),
                            _p(idx), _p(logq), _p(margin))
    assert rc == 0, rc
    return idx, logq, margin


def rotation_set(kind, n, rot_max=0.0):
    R = np.empty((n, 3, 3), np.float64)
    rc = lib().orc_rotation_set(C.c_int32(kind), C.c_int32(n), C.c_double(rot_max), _p(R))
    assert rc == 0, rc
    return R


def expand(centre, G, n, step, rotset):
    rotset = _f64(rotset).reshape(-1, 9)
    nh = n ** 3 * rotset.shape[0]
    poses = np.empty((nh, 4, 4), np.float64)
    rc = lib().orc_expand(_p(_f64(centre).reshape(16)), _p(_f64(G).reshape(9)), C.c_int32(n), C.c_double(step),
                          _p(rotset), C.c_int32(rotset.shape[0]), _p(poses))
    assert rc == 0, rc
    return poses


def enumerate_c2f(scene, slot, centre, G, lk: dict, depth_obs, stages, m, seed, n_threads=0, arrays=None,
                  path_density=False):
    sa = arrays or SceneArrays(scene)
    T = len(stages)
    st = (_Stage * T)(*[_Stage(s.n_per_axis, s.step, s.rot_kind, s.n_rot, s.rot_max) for s in stages])
    particles = np.empty((m, 4, 4))
    logw, logq = np.empty(m), np.empty(m)
    centres, zs = np.empty((T, 4, 4)), np.empty(T)
    idx = np.empty((T, m), np.int32)
    rc = lib().orc_enumerate_c2f(C.byref(sa.cam), C.byref(sa.st), C.c_int32(slot), _p(_f64(centre).reshape(16)),
                                 _p(_f64(G).reshape(9)), C.byref(lik(**lk)), _p(_f64(depth_obs)), C.c_int32(T), st,
                                 C.c_int32(m), C.c_uint64(seed), C.c_int32(1 if path_density else 0), _p(particles),
                                 _p(logw), _p(logq), _p(centres),
                                 _p(zs), _p(idx), C.c_int32(n_threads))
    assert rc == 0, rc
    return dict(particles=particles, logw=logw, logq=logq, centres=centres, z=zs, idx=idx)


def score_grad(scene, slot, poses, lk: dict, depth_obs, n_threads=0, arrays=None):
    sa = arrays or SceneArrays(scene)
    P = _f64(poses).reshape(-1, 16)
    n = P.shape[0]
    ll, dpose, ds, dp = np.empty(n), np.empty((n, 6)), np.empty(n), np.empty(n)
    rc = lib().orc_score_grad(C.byref(sa.cam), C.byref(sa.st), C.c_int32(slot), C.c_int64(n), _p(P),
                              C.byref(lik(**lk)), _p(_f64(depth_obs)), _p(ll), _p(dpose), _p(ds), _p(dp),
                              C.c_int32(n_threads))
    assert rc == 0, rc
    return dict(ll=ll, dpose=dpose, dsigma=ds, dpout=dp)


def score_grad_bound(scene, slot, poses, lk: dict, depth_obs, edge_tol=1e-4, z_tol=1e-5, n_threads=0, arrays=None):
    """Per hypothesis, the bound [n, 8] on how far FP32 visibility decisions can move
    (dLL/dxi [6], dLL/dsigma, dLL/dp_out) of score_grad, and the number of flagged pixels."""
    sa = arrays or SceneArrays(scene)
    P = _f64(poses).reshape(-1, 16)
    n = P.shape[0]
    gb = np.empty((n, 8))
    nf = np.empty(n, np.int32)
    rc = lib().orc_score_grad_bound(C.byref(sa.cam), C.byref(sa.st), C.c_int32(slot), C.c_int64(n), _p(P),
                                    C.byref(lik(**lk)), _p(_f64(depth_obs)), C.c_double(edge_tol), C.c_double(z_tol),
                                    _p(gb), _p(nf), C.c_int32(n_threads))
    assert rc == 0, rc
    return dict(gbound=gb, n_flag=nf)


def max_threads() -> int:
    return int(lib().orc_max_threads())


def smc_parse(scene, n_fixed, centres, G, lk: dict, depth_obs, stages, m, seed, ess_frac=0.5, n_threads=0):
    """SMC over the number of objects (Sec. III-B, Eq. 2 and 3), each particle proposing the
    next object's pose with its own single-sample coarse-to-fine search.

    Objects 0 .. n_fixed-1 of ``scene`` are known and fixed; objects n_fixed .. are placed one
    per step, in order, around ``centres[k]``. The step-k target p_k is the likelihood of the
    scene holding the fixed objects and the first k+1 placed objects at the particle's poses
    (uniform priors: constants that cancel between particles). Particle j draws its step-k
    proposal with seed ``seed + 1000 k + j``; its log density log q is the path density.
    Log weights: W = LL_1(x) - log q(x_1), then W += LL_k - LL_{k-1} - log q(x_k). When the
    effective sample size falls below ess_frac * m, the particles are resampled in proportion
    to their weights (draws of stage k with ``seed``) and every weight becomes their mean.
    Returns the particles' poses [m, K, 4, 4], log weights, the log evidence estimate
    (log-mean weight) and, per step, the ESS before resampling and the resampled indices.
    """
    K = len(centres)
    meshes = scene.meshes[:n_fixed + K]
    poses = np.tile(_f64(scene.poses[:n_fixed + K])[None], (m, 1, 1, 1))
    logw = np.zeros(m)
    ll_prev = np.zeros(m)
    ess_all, idx_all = [], []
    for k in range(K):
        slot = n_fixed + k
        sub_meshes = meshes[:slot + 1]
        for j in range(m):
            sub = types.SimpleNamespace(camera=scene.camera, meshes=sub_meshes, poses=poses[j, :slot + 1].copy())
            arrays = SceneArrays(sub)
            out = enumerate_c2f(sub, slot, centres[k], G, lk, depth_obs, stages, 1, seed + 1000 * k + j,
                                n_threads=n_threads, arrays=arrays, path_density=True)
            x = out["particles"][0]
            poses[j, slot] = x
            sub.poses[slot] = x
            ll = score(sub, slot, x[None], lk, depth_obs, flags=False, n_threads=n_threads,
                       arrays=SceneArrays(sub))["ll"][0]
            logw[j] += ll - ll_prev[j] - out["logq"][0]
            ll_prev[j] = ll
        z, _ = lse(logw)
        z2, _ = lse(2 * logw)
        ess = math.exp(2 * z - z2)
        ess_all.append(ess)
        if ess < ess_frac * m:
            idx, _, _ = resample(logw, m, seed, k)
            poses, ll_prev = poses[idx].copy(), ll_prev[idx].copy()
            logw = np.full(m, z - math.log(m))
            idx_all.append(idx)
        else:
            idx_all.append(None)
    z, _ = lse(logw)
    return dict(poses=poses[:, n_fixed:], logw=logw, log_evidence=z - math.log(m), ess=ess_all, idx=idx_all)


def score_noise(scene, slot, poses, kind, radii, p_outliers, half_window, depth_obs, log_weight=None, n_threads=0):
    """Hierarchical noise (Alg. 1): the log-likelihood of each hypothesis under
    every setting (radii[i], p_outliers[j]) at g = i * len(p_outliers) + j, and the marginal
    log sum_g exp(ll_g + log_weight_g), the noise integrated out over the grid with the
    settings' prior masses. Returns ll [n, G], marginal [n], and per setting the flags' scale
    and ambiguity bound [n, G]."""
    nr, npo = len(radii), len(p_outliers)
    lw = np.zeros(nr * npo) if log_weight is None else _f64(log_weight).ravel()
    P = _f64(poses).reshape(-1, 16)
    ll = np.empty((P.shape[0], nr * npo))
    scale, bound = np.empty_like(ll), np.empty_like(ll)
    arrays = SceneArrays(scene)
    for i, r in enumerate(radii):
        for j, p in enumerate(p_outliers):
            out = score(scene, slot, P, dict(kind=kind, radius=float(r), p_outlier=float(p), half_window=half_window),
                        depth_obs, n_threads=n_threads, arrays=arrays)
            g = i * npo + j
            ll[:, g], scale[:, g], bound[:, g] = out["ll"], out["scale"], out["bound"]
    a = ll + lw[None, :]
    m = a.max(axis=1)
    marginal = m + np.log(np.exp(a - m[:, None]).sum(axis=1))
    return dict(ll=ll, marginal=marginal, scale=scale, bound=bound)
