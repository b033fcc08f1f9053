"""Seeded synthetic inputs for the Bayes3D render-and-score path.

The paper's objects (YCB meshes, robot captures) are not available, so every input here
is synthetic and seeded: voxel meshes (the paper's object representation: voxels placed
on the points of a fused cloud, Sec. III and the pipeline figure), tabletop scenes
(scene graph of Alg. 1: objects resting on a table with a planar offset and a yaw),
cameras looking at the table origin with up = +z (camera pose prior, Sec. III-A (ii)),
and the random draws that corrupt an observed depth image (Gaussian depth noise and
uniform outliers).

This module holds none of the method's arithmetic: no projection, rasterisation,
likelihood, normalisation or resampling. It is shared by the tests, the benchmark and
the smoke check, and it feeds the CUDA path and the CPU oracle identically.

Seed convention: workload c, trial k uses ``numpy.random.default_rng(1000 * c + k)``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Corners of a unit voxel, index a + 2b + 4c for offsets (a, b, c) in {0,1}^3.
_CORNERS = np.array([[a, b, c] for c in (0, 1) for b in (0, 1) for a in (0, 1)], dtype=np.int64)

# The six faces of a voxel as corner quads, counter-clockwise seen from outside, so the
# right-hand normal of each triangle (c0,c1,c2), (c0,c2,c3) points out of the voxel.
_FACE_QUADS = {
    "-x": ((0, 0, 0), (0, 0, 1), (0, 1, 1), (0, 1, 0)),
    "+x": ((1, 0, 0), (1, 1, 0), (1, 1, 1), (1, 0, 1)),
    "-y": ((0, 0, 0), (1, 0, 0), (1, 0, 1), (0, 0, 1)),
    "+y": ((0, 1, 0), (0, 1, 1), (1, 1, 1), (1, 1, 0)),
    "-z": ((0, 0, 0), (0, 1, 0), (1, 1, 0), (1, 0, 0)),
    "+z": ((0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)),
}


def _corner_index(abc):
    a, b, c = abc
    return a + 2 * b + 4 * c


_VOXEL_TRIS = []
for _quad in _FACE_QUADS.values():
    q = [_corner_index(x) for x in _quad]
    _VOXEL_TRIS.append((q[0], q[1], q[2]))
    _VOXEL_TRIS.append((q[0], q[2], q[3]))
_VOXEL_TRIS = np.array(_VOXEL_TRIS, dtype=np.int64)  # [12, 3]


@dataclasses.dataclass
class Mesh:
    verts: np.ndarray  # [V, 3] float32, object frame, metres
    faces: np.ndarray  # [F, 3] int32, vertex indices

    @property
    def n_faces(self) -> int:
        return int(self.faces.shape[0])


@dataclasses.dataclass
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    near: float
    far: float


@dataclasses.dataclass
class Scene:
    """A flat scene: object k is ``meshes[k]`` at ``poses[k]`` (4x4 cam_from_obj, float32)."""
    camera: Camera
    meshes: list
    poses: np.ndarray  # [n_obj, 4, 4] float32


def voxel_mesh(ijk: np.ndarray, pitch: float, origin) -> Mesh:
    """Voxel mesh: 8 vertices and 12 outward triangles per occupied lattice cell.

    ``ijk`` [n,3] integer lattice cells; a corner at integer lattice point L has object
    coordinates ``origin + pitch * L``, evaluated in float64 from the integer, so corners
    shared by neighbouring voxels are bitwise identical in float32.
    """
    ijk = np.asarray(ijk, dtype=np.int64).reshape(-1, 3)
    n = ijk.shape[0]
    lattice = ijk[:, None, :] + _CORNERS[None, :, :]  # [n, 8, 3]
    verts = (np.asarray(origin, dtype=np.float64)[None, None, :]
             + pitch * lattice.astype(np.float64)).reshape(-1, 3).astype(np.float32)
    faces = (_VOXEL_TRIS[None, :, :] + 8 * np.arange(n, dtype=np.int64)[:, None, None]).reshape(-1, 3)
    return Mesh(verts=verts, faces=faces.astype(np.int32))


def box_mesh(size, centre=(0.0, 0.0, 0.0)) -> Mesh:
    """One cuboid of 12 outward triangles (the occluder)."""
    sx, sy, sz = (float(s) for s in size)
    lo = np.asarray(centre, dtype=np.float64) - 0.5 * np.array([sx, sy, sz])
    verts = (lo[None, :] + _CORNERS.astype(np.float64) * np.array([sx, sy, sz])[None, :]).astype(np.float32)
    return Mesh(verts=verts, faces=_VOXEL_TRIS.astype(np.int32).copy())


def table_mesh(size=1.0, divisions=1) -> Mesh:
    """Table top: a square of side ``size`` at z = 0 facing +z, split into divisions^2
    squares of two triangles each."""
    h = 0.5 * size
    g = np.linspace(-h, h, divisions + 1)
    X, Y = np.meshgrid(g, g, indexing="xy")
    verts = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], 1).astype(np.float32)
    faces = []
    for r in range(divisions):
        for c in range(divisions):
            v0 = r * (divisions + 1) + c
            v1, v2, v3 = v0 + 1, v0 + divisions + 2, v0 + divisions + 1
            faces += [[v0, v1, v2], [v0, v2, v3]]
    return Mesh(verts=verts, faces=np.array(faces, dtype=np.int32))


def random_rotation(rng) -> np.ndarray:
    """Uniform rotation (Shoemake's quaternion from three uniforms), float64 3x3."""
    u1, u2, u3 = rng.random(3)
    a, b = math.sqrt(1.0 - u1), math.sqrt(u1)
    x, y = a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2)
    z, w = b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def yaw(theta: float) -> np.ndarray:
    c, s = math.cos(theta), math.sin(theta)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rigid(R, t) -> np.ndarray:
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def look_at_origin(distance: float, elevation: float, azimuth: float) -> np.ndarray:
    """cam_from_world for a camera at the given distance/elevation/azimuth that looks at
    the world origin with world +z as up (OpenCV axes: x right, y down, z forward)."""
    eye = distance * np.array([math.cos(elevation) * math.cos(azimuth),
                               math.cos(elevation) * math.sin(azimuth),
                               math.sin(elevation)])
    zc = -eye / np.linalg.norm(eye)
    xc = np.cross(zc, np.array([0.0, 0.0, 1.0]))
    xc /= np.linalg.norm(xc)
    yc = np.cross(zc, xc)
    R = np.stack([xc, yc, zc])
    return rigid(R, -R @ eye)


@dataclasses.dataclass
class NoiseDraws:
    """Random draws that turn a clean depth render into an observation."""
    noise: np.ndarray        # [H, W] N(0, sigma) depth noise (metres)
    outlier: np.ndarray      # [H, W] bool, pixel replaced by an outlier
    outlier_depth: np.ndarray  # [H, W] uniform outlier depth


def noise_draws(rng, height, width, sigma=0.002, p_outlier=0.1, lo=0.01, hi=2.0) -> NoiseDraws:
    return NoiseDraws(noise=rng.normal(0.0, sigma, size=(height, width)),
                      outlier=rng.random((height, width)) < p_outlier,
                      outlier_depth=rng.uniform(lo, hi, size=(height, width)))


def corrupt_depth(clean: np.ndarray, far: float, draws: NoiseDraws) -> np.ndarray:
    """Observed depth: noise on surface pixels (depth < far), background left at far,
    then outlier pixels replaced by their uniform depth. Float32 [H, W]."""
    clean = np.asarray(clean, dtype=np.float64)
    obs = np.where(clean < far, clean + draws.noise, clean)
    obs = np.where(draws.outlier, draws.outlier_depth, obs)
    return obs.astype(np.float32)


# ---------------------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------------------

@dataclasses.dataclass
class StageSpec:
    n_per_axis: int
    step: float
    rot_kind: int   # 0 Fibonacci-sphere set, 1 perturbation set
    n_rot: int
    rot_max: float  # radians (radius of the perturbation set's ball of rotation vectors)


@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    slot: int                 # object whose pose is hypothesised
    hidden: np.ndarray        # [4,4] float32 true cam_from_obj of the slot object
    centre: np.ndarray        # [4,4] float32 grid centre
    grid_frame: np.ndarray    # [3,3] float32 rotation of the translation grid (cam_from_grid)
    stages: list
    lik: dict
    draws: NoiseDraws
    n_particles: int = 100
    seed: int = 0
    extra: dict = dataclasses.field(default_factory=dict)


def single_object_workload(trial: int = 0) -> Workload:
    """Single voxel object, 64x48 camera, 10^3 translation grid (1 cm) around the hidden
    pose with the rotation fixed, inlier-ball likelihood r = 5 mm, p_out = 0.01, 3x3 window."""
    rng = np.random.default_rng(1000 * 0 + trial)
    cells = np.array(np.unravel_index(rng.permutation(1000)[:500], (10, 10, 10))).T
    mesh = voxel_mesh(cells, 0.01, origin=(-0.05, -0.05, -0.05))
    cam = Camera(64, 48, 60.0, 60.0, 32.0, 24.0, 0.01, 2.0)
    R = random_rotation(rng)
    hidden = rigid(R, [0.0, 0.0, 0.5]).astype(np.float32)
    draws = noise_draws(rng, cam.height, cam.width)
    scene = Scene(cam, [mesh], hidden[None].copy())
    return Workload(name="single-object 64x48, 500 voxels, 1000 hyps", scene=scene, slot=0,
                    hidden=hidden, centre=hidden.copy(), grid_frame=np.eye(3, dtype=np.float32),
                    stages=[StageSpec(10, 0.01, 1, 1, 0.0)],
                    lik=dict(kind=0, radius=0.005, p_outlier=0.01, half_window=1),
                    draws=draws, n_particles=100, seed=trial)


def _blob_cells(rng, pitch, lo=2000, hi=8000):
    """Union of 1-3 random ellipsoids voxelised at ``pitch``; retried until the voxel
    count lies in [lo, hi]. Returns integer cells with the lowest layer at k = 0."""
    # ellipsoid size scaled to the requested count (1 for the default 2,000-8,000 voxels of
    # 5 mm, whose 2.5-7.5 cm semi-axes suit it)
    scale = ((lo + hi) / 2.0 / 5000.0) ** (1.0 / 3.0) * (pitch / 0.005)
    for _ in range(1000):
        n_ell = int(rng.integers(1, 4))
        ells = []
        for _e in range(n_ell):
            axes = rng.uniform(0.025, 0.075, size=3) * scale
            centre = np.concatenate([rng.uniform(-0.03, 0.03, size=2) * scale, [axes[2]]])
            ells.append((centre, axes))
        ext = max(float(np.max(np.abs(c) + a)) for c, a in ells) + pitch
        n = int(math.ceil(ext / pitch))
        g = np.arange(-n, n)
        I, J, K = np.meshgrid(g, g, np.arange(0, 2 * n), indexing="ij")
        centres = np.stack([(I + 0.5) * pitch, (J + 0.5) * pitch, (K + 0.5) * pitch], -1)
        occ = np.zeros(I.shape, dtype=bool)
        for c, a in ells:
            occ |= (((centres - c) / a) ** 2).sum(-1) <= 1.0
        cnt = int(occ.sum())
        if lo <= cnt <= hi:
            cells = np.argwhere(occ)
            cells[:, 0] -= n
            cells[:, 1] -= n
            cells[:, 2] -= cells[:, 2].min()
            return cells
    raise RuntimeError("could not draw a blob in the voxel-count range")


def tabletop_workload(trial: int = 0, n_objects: int = 5, width=160, height=120, f=150.0,
                      vox_lo=2000, vox_hi=8000, seed_base=1000) -> Workload:
    """Tabletop scene: a 1 m table quad at z = 0, one box occluder and ``n_objects``
    voxel blobs (5 mm pitch) resting on the table with random yaw and no overlap. Camera
    0.8 m from the origin, 45 degrees above the table, looking at the origin (up = +z).
    Three coarse-to-fine stages of 9^3 translations x 200 rotations in the table frame."""
    rng = np.random.default_rng(seed_base + trial)
    pitch = 0.005
    cam = Camera(width, height, f, f, width / 2.0, height / 2.0, 0.01, 2.0)
    cam_from_world = look_at_origin(0.8, math.radians(45.0), rng.uniform(0, 2 * math.pi))

    meshes, world_poses, radii = [table_mesh(1.0)], [np.eye(4)], [0.0]
    occ_size = (0.04, 0.20, 0.15)
    occ_mesh = box_mesh(occ_size, centre=(0.0, 0.0, occ_size[2] / 2))
    placed = []  # (xy, radius)
    objects = []
    for _ in range(n_objects):
        cells = _blob_cells(rng, pitch, vox_lo, vox_hi)
        objects.append(voxel_mesh(cells, pitch, origin=(0.0, 0.0, 0.0)))

    half = [0.3 + 0.03 * max(0, n_objects - 5)]

    def place(radius):
        # rejection sampling in a square that widens when it gets crowded
        for _ in range(20):
            for _ in range(2000):
                xy = rng.uniform(-half[0], half[0], size=2)
                if all(np.linalg.norm(xy - p) > radius + r for p, r in placed):
                    placed.append((xy, radius))
                    return xy
            half[0] *= 1.2
        raise RuntimeError("placement failed")

    occ_r = 0.5 * math.hypot(occ_size[0], occ_size[1])
    xy = place(occ_r)
    meshes.append(occ_mesh)
    world_poses.append(rigid(yaw(rng.uniform(0, 2 * math.pi)), [xy[0], xy[1], 0.0]))
    for m in objects:
        r = float(np.max(np.linalg.norm(m.verts[:, :2].astype(np.float64), axis=1)))
        xy = place(r)
        meshes.append(m)
        world_poses.append(rigid(yaw(rng.uniform(0, 2 * math.pi)), [xy[0], xy[1], 0.0]))
    poses = np.stack([cam_from_world @ P for P in world_poses]).astype(np.float32)
    scene = Scene(cam, meshes, poses)

    slot = 2  # first voxel object (0 = table, 1 = occluder)
    # Tracking prior for the slot object: the true table pose moved by <= 2 cm and <= 5 deg.
    dxy = rng.uniform(-0.02, 0.02, size=2)
    dth = math.radians(rng.uniform(-5.0, 5.0))
    Wp = world_poses[slot]
    prior_world = rigid(yaw(dth) @ Wp[:3, :3], Wp[:3, 3] + np.array([dxy[0], dxy[1], 0.0]))
    centre = (cam_from_world @ prior_world).astype(np.float32)
    # Tracking priors for every object (used by the multi-object parse).
    priors = []
    for k in range(len(meshes)):
        dxy_k = rng.uniform(-0.02, 0.02, size=2)
        dth_k = math.radians(rng.uniform(-5.0, 5.0))
        Wk = world_poses[k]
        pk = rigid(yaw(dth_k) @ Wk[:3, :3], Wk[:3, 3] + np.array([dxy_k[0], dxy_k[1], 0.0]))
        priors.append((cam_from_world @ pk).astype(np.float32))
    draws = noise_draws(rng, cam.height, cam.width)
    stages = [StageSpec(9, 0.02, 0, 200, 0.0),
              StageSpec(9, 0.005, 1, 200, math.radians(10.0)),
              StageSpec(9, 0.001, 1, 200, math.radians(2.0))]
    return Workload(name=f"tabletop {n_objects}-object {width}x{height}, 3 stages x 9^3 x 200",
                    scene=scene, slot=slot, hidden=poses[slot].copy(), centre=centre,
                    grid_frame=cam_from_world[:3, :3].astype(np.float32), stages=stages,
                    lik=dict(kind=0, radius=0.005, p_outlier=0.01, half_window=1),
                    draws=draws, n_particles=100, seed=trial,
                    extra=dict(cam_from_world=cam_from_world, priors=np.stack(priors),
                               object_slots=list(range(2, 2 + n_objects))))


def random_ll(rng, n: int, spread: float = 30.0) -> np.ndarray:
    """Synthetic log-likelihood vector shaped like a C2F stage: a broad floor with a few
    sharp peaks (float32)."""
    ll = -spread * rng.random(n) * 10.0
    k = max(1, n // 1000)
    peaks = rng.integers(0, n, size=k)
    ll[peaks] = rng.uniform(-spread, 0.0, size=k)
    return ll.astype(np.float32)


def batched_workloads(n_scenes: int = 64, seed_base: int = 2000, pitch: float = 0.005):
    """Independent tabletop scenes for the batched form, each drawn log-uniform: 1-8
    objects, 500-20,000 voxels per object, image width 80-320 (4:3, fx = 0.9375 W),
    1,000-50,000 hypotheses per coarse-to-fine stage (two stages: a 5^3 translation grid of
    2 cm then 5 mm, times a perturbation set sized to the count)."""
    out = []
    for k in range(n_scenes):
        rng = np.random.default_rng(seed_base + k)
        n_obj = int(rng.integers(1, 9))
        W = int(round(float(np.exp(rng.uniform(np.log(80), np.log(320)))) / 4.0)) * 4
        H = W * 3 // 4
        v = float(np.exp(rng.uniform(np.log(500), np.log(20000))))
        n_hyp = float(np.exp(rng.uniform(np.log(1000), np.log(50000))))
        n_rot = max(1, int(round(n_hyp / 125.0)))
        wl = tabletop_workload(trial=k, n_objects=n_obj, width=W, height=H, f=0.9375 * W,
                               vox_lo=int(0.8 * v), vox_hi=int(1.25 * v), seed_base=seed_base + 100000)
        wl.stages = [StageSpec(5, 0.02, 1, n_rot, math.radians(10.0)),
                     StageSpec(5, 0.005, 1, n_rot, math.radians(3.0))]
        wl.name = f"batched scene {k}: {n_obj} objects, {W}x{H}, ~{int(v)} voxels, {125 * n_rot} hypotheses/stage"
        out.append(wl)
    return out


@dataclasses.dataclass
class TrackingStream:
    """One session of the tracking loop: a tabletop scene whose first ``n_track`` objects
    move on smooth random trajectories while the camera and the table stay fixed."""
    name: str
    scene: Scene              # meshes (tracked objects first, then the table) at their frame-0 poses
    n_track: int
    truth: np.ndarray         # [F, n_obj, 4, 4] float32 true cam_from_obj of every object per frame
    grid_frame: np.ndarray    # [3, 3] float32 cam_from_table (axes of the translation grid)
    seed: int                 # the session's seed (random draws of the enumeration)
    noise_seed: int

    @property
    def n_frames(self) -> int:
        return int(self.truth.shape[0])

    def draws(self, frame: int) -> NoiseDraws:
        rng = np.random.default_rng([self.noise_seed, int(frame)])
        return noise_draws(rng, self.scene.camera.height, self.scene.camera.width)

    def scene_at(self, frame: int) -> Scene:
        return Scene(self.scene.camera, self.scene.meshes, self.truth[frame].copy())


def tracking_stream(k: int, n_objects: int, width=320, height=240, f=300.0, n_frames=40, vox_lo=2000,
                    vox_hi=8000, seed_base=4000, max_step=0.012, max_turn_deg=4.0) -> TrackingStream:
    """Session ``k`` of the serving workload: ``n_objects`` voxel blobs (5 mm pitch) on a 1 m
    table, camera 0.8 m away and 45 degrees above the table looking at its centre. Each
    object follows x(t) = x0 + a (sin(w t + p) - sin p) per table axis and the same form in
    yaw, with a w <= max_step per axis and per frame (so <= sqrt(2) max_step of translation)
    and yaw amplitude x rate <= max_turn_deg per frame."""
    rng = np.random.default_rng(seed_base + k)
    pitch = 0.005
    cam = Camera(width, height, f, f, width / 2.0, height / 2.0, 0.01, 2.0)
    cam_from_world = look_at_origin(0.8, math.radians(45.0), rng.uniform(0, 2 * math.pi))
    objects = [voxel_mesh(_blob_cells(rng, pitch, vox_lo, vox_hi), pitch, origin=(0.0, 0.0, 0.0))
               for _ in range(n_objects)]
    placed = []
    half = 0.12 + 0.03 * n_objects
    starts = []
    for m in objects:
        r = float(np.max(np.linalg.norm(m.verts[:, :2].astype(np.float64), axis=1)))
        for _ in range(20):
            ok = False
            for _ in range(2000):
                xy = rng.uniform(-half, half, size=2)
                if all(np.linalg.norm(xy - p) > r + q for p, q in placed):
                    ok = True
                    break
            if ok:
                break
            half *= 1.2
        else:
            raise RuntimeError("placement failed")
        placed.append((xy, r))
        starts.append(xy)
    t = np.arange(n_frames, dtype=np.float64)
    truth = np.zeros((n_frames, n_objects + 1, 4, 4), dtype=np.float64)
    for o, xy in enumerate(starts):
        a = rng.uniform(0.02, 0.06, size=2)
        w = rng.uniform(0.5, 1.0, size=2) * max_step / a
        p = rng.uniform(0, 2 * math.pi, size=2)
        b = math.radians(rng.uniform(5.0, 20.0))
        wb = rng.uniform(0.5, 1.0) * math.radians(max_turn_deg) / b
        pb = rng.uniform(0, 2 * math.pi)
        th0 = rng.uniform(0, 2 * math.pi)
        for i, ti in enumerate(t):
            x = xy[0] + a[0] * (math.sin(w[0] * ti + p[0]) - math.sin(p[0]))
            y = xy[1] + a[1] * (math.sin(w[1] * ti + p[1]) - math.sin(p[1]))
            th = th0 + b * (math.sin(wb * ti + pb) - math.sin(pb))
            truth[i, o] = cam_from_world @ rigid(yaw(th), [x, y, 0.0])
    truth[:, n_objects] = cam_from_world  # the table
    meshes = objects + [table_mesh(1.0)]
    scene = Scene(cam, meshes, truth[0].astype(np.float32))
    return TrackingStream(name=f"tracking session {k}: {n_objects} objects, {width}x{height}, {n_frames} frames",
                          scene=scene, n_track=n_objects, truth=truth.astype(np.float32),
                          grid_frame=cam_from_world[:3, :3].astype(np.float32), seed=seed_base + k,
                          noise_seed=seed_base + 7919 * (k + 1))


def tracking_stage(n_per_axis=5, step=0.01, n_rot=50, rot_max_deg=5.0) -> StageSpec:
    """The per-frame enumeration of the tracking loop: a translation grid of n_per_axis^3
    cells around the previous estimate times n_rot rotation perturbations."""
    return StageSpec(n_per_axis, step, 1, n_rot, math.radians(rot_max_deg))


@dataclasses.dataclass
class CameraVideo:
    """Camera-pose tracking video (the setting of Table 1): one object resting on a table at
    the world origin, the camera panning around it; frame 0's pose is given."""
    name: str
    scene: Scene              # meshes (object, table) at their WORLD poses
    cam_from_world: np.ndarray  # [F, 4, 4] float32 true camera poses
    seed: int

    @property
    def n_frames(self) -> int:
        return int(self.cam_from_world.shape[0])

    def draws(self, frame: int) -> NoiseDraws:
        rng = np.random.default_rng([self.seed, int(frame)])
        return noise_draws(rng, self.scene.camera.height, self.scene.camera.width)

    def camera_scene(self, frame: int) -> Scene:
        """The scene as seen by the camera of ``frame`` (object poses cam_from_obj)."""
        H = self.cam_from_world[frame].astype(np.float64)
        poses = np.stack([H @ P for P in self.scene.poses.astype(np.float64)]).astype(np.float32)
        return Scene(self.scene.camera, self.scene.meshes, poses)


def camera_video(k: int, size: int, n_frames=120, vox_lo=8000, vox_hi=16000, seed_base=5000) -> CameraVideo:
    """Video ``k`` at ``size`` x ``size`` pixels (fx = fy = size): a voxel blob (5 mm pitch)
    with a random yaw at the origin of a 1 m table (20 x 20 squares), and two boxes placed
    around it (a blob on a bare plane would leave the camera's orbit angle unobservable);
    the camera looks at the origin from 0.6 m and 35 degrees up, its azimuth sweeping
    0.5 degrees a frame with a slow oscillation of elevation (+-3 degrees) and distance
    (+-3 cm)."""
    rng = np.random.default_rng(seed_base + k)
    obj = voxel_mesh(_blob_cells(rng, 0.005, vox_lo, vox_hi), 0.005, origin=(0.0, 0.0, 0.0))
    boxes = [box_mesh((0.04, 0.12, 0.08), centre=(0.0, 0.0, 0.04)), box_mesh((0.10, 0.03, 0.05), centre=(0.0, 0.0, 0.025))]
    cam = Camera(size, size, float(size), float(size), size / 2.0, size / 2.0, 0.01, 2.0)
    world = [rigid(yaw(rng.uniform(0, 2 * math.pi)), [0.0, 0.0, 0.0])]
    for b, (x, y) in zip(boxes, [(0.16, 0.05), (-0.1, -0.15)]):
        world.append(rigid(yaw(rng.uniform(0, 2 * math.pi)), [x, y, 0.0]))
    world.append(np.eye(4))
    world = np.stack(world)
    az0, ph = rng.uniform(0, 2 * math.pi), rng.uniform(0, 2 * math.pi)
    frames = []
    for f in range(n_frames):
        az = az0 + math.radians(0.5) * f
        el = math.radians(35.0 + 3.0 * math.sin(0.05 * f + ph))
        dist = 0.6 + 0.03 * math.sin(0.031 * f + 2 * ph)
        frames.append(look_at_origin(dist, el, az))
    scene = Scene(cam, [obj] + boxes + [table_mesh(1.0, 20)], world.astype(np.float32))
    return CameraVideo(name=f"camera video {k}: {size}x{size}, {n_frames} frames", scene=scene,
                       cam_from_world=np.stack(frames).astype(np.float32), seed=seed_base + 31 * k)


def camera_stages():
    """Per-frame coarse-to-fine search around the previous camera pose, rotations and
    translations in turn: 2,048 rotations about the world origin (+-1 degree), then a 3^3
    translation grid in camera axes (3 mm); again at +-0.3 degree / 1 mm and +-0.1 degree /
    0.4 mm. A joint 6-D grid of the same size leaves too coarse a rotation spacing for this
    sharply peaked likelihood (a 0.1 degree or 1 mm error costs ~300 nats at 64x64)."""
    return [StageSpec(1, 0.001, 1, 2048, math.radians(1.0)), StageSpec(3, 0.003, 1, 1, 0.0),
            StageSpec(1, 0.001, 1, 2048, math.radians(0.3)), StageSpec(3, 0.001, 1, 1, 0.0),
            StageSpec(1, 0.001, 1, 2048, math.radians(0.1)), StageSpec(3, 0.0004, 1, 1, 0.0)]
