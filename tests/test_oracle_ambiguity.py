"""Pins of the oracle's ambiguity machinery: the render flags (which pixels FP32 may assign
to another triangle or depth) and the per-hypothesis bound (how far FP32-resolution
decisions may move a log-likelihood). These two decide which GPU/oracle differences the
parity tests accept, so each is checked here on hand-built scenes whose answer the
geometry fixes. CPU only.

Geometry used throughout: an 8x8 camera with fx = fy = 8, cx = cy = 4, so the centre of
pixel (u, v) sees the direction ((u - 3.5)/8, (v - 3.5)/8, 1); at depth 1 a world x of
(u - 3.5)/8 lands exactly on the centres of column u, and one pixel is 1/8 m wide. Every
coordinate below is a dyadic rational (exact in float32 and float64) unless stated.

Flag semantics under test (edge_tol = 1e-4 px, z_tol = 1e-5 relative):
  bit 0: the triangle id could change (a coverage within edge_tol of an edge, or two
         depths within z_tol of each other);
  bit 1: additionally the depth could change by more than z_tol.
Bound semantics (Eq. 1 with the window of Sec. III-B): every bit-1 pixel adds one point's
largest effect on l_i (the jump l(1) - l(0) for the ball) for every valid observed pixel
whose window holds it; every observed pixel with k borderline pairs adds the largest change
of l_i when k of its window pairs flip. A pair is borderline when |d^2 - r^2| <= 1e-3 r^2,
or when its rendered pixel is a bit-0 tie whose alternative depth can carry d across r.
"""
import math

import numpy as np
import pytest

from paper_2312_08715_gb300 import synth

EDGE_TOL, Z_TOL, BORDER = 1e-4, 1e-5, 1e-3
CAM8 = synth.Camera(8, 8, 8.0, 8.0, 4.0, 4.0, 0.01, 2.0)


def _square(x0, x1, y0, y1, z):
    """Two triangles (A, B, C), (A, C, D) of the rectangle A=(x0,y0) B=(x1,y0) C=(x1,y1)
    D=(x0,y1) in the plane z (object frame = camera frame)."""
    v = np.array([[x0, y0, z], [x1, y0, z], [x1, y1, z], [x0, y1, z]], np.float32)
    return synth.Mesh(verts=v, faces=np.array([[0, 1, 2], [0, 2, 3]], np.int32))


def _scene(meshes, cam=CAM8):
    return synth.Scene(cam, list(meshes), np.stack([np.eye(4, dtype=np.float32)] * len(meshes)))


def _render(orc, scene):
    return orc.render(scene, edge_tol=EDGE_TOL, z_tol=Z_TOL, want_flags=True)


def _ell(n, r, p, K, V):
    """Eq. 1 with the inlier ball (the plain path): l = log(p/V + (1 - p) n / (K (4/3) pi r^3))."""
    return math.log(p / V + (1 - p) * n / (K * 4.0 / 3.0 * math.pi * r ** 3))


def _volume(cam):
    return cam.width * cam.height / (cam.fx * cam.fy) * (cam.far ** 3 - cam.near ** 3) / 3.0


# ---------------------------------------------------------------------------------------
# render flags
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("shift_px,covered_from,flag_col2", [
    (0.0, 2, 3),               # edge exactly through the centres of column 2: covered (>= 0), flagged
    (+0.5 * EDGE_TOL, 3, 3),   # just outside by half the tolerance: not covered, still flagged
    (-0.5 * EDGE_TOL, 2, 3),   # just inside by half the tolerance: covered, flagged
    (+2.0 * EDGE_TOL, 3, 0),   # outside by twice the tolerance: neither
    (-2.0 * EDGE_TOL, 2, 0),   # inside by twice the tolerance: covered, not flagged
])
def test_edge_through_pixel_centres(orc, shift_px, covered_from, flag_col2):
    """Square x in [-0.1875 + shift/8, 0.25], y in [-0.25, 0.25] at z = 1. Its left edge
    lies on the centres of column 2 (shifted by shift_px pixels); its other edges are half
    a pixel from the nearest centres and its diagonal stays >= 0.047 px from every centre
    (the centres satisfy 8u - 7v = 5.5 nowhere). So rows 2..5 are covered from column
    `covered_from` to 5, the id/depth of column 2 (rows 2..5) is ambiguous exactly when
    |shift| < edge_tol, and then both bits are set: the alternative is the far background
    (depth 2 against 1). No other pixel is flagged."""
    sq = _square(-0.1875 + shift_px / 8.0, 0.25, -0.25, 0.25, 1.0)
    depth, tid, flags = _render(orc, _scene([sq]))
    want_cov = np.zeros((8, 8), bool)
    want_cov[2:6, covered_from:6] = True
    np.testing.assert_array_equal(tid >= 0, want_cov)
    np.testing.assert_array_equal(depth, np.where(want_cov, 1.0, 2.0))
    want = np.zeros((8, 8), np.uint8)
    want[2:6, 2] = flag_col2
    np.testing.assert_array_equal(flags, want)


def test_shared_edge_of_coplanar_triangles_sets_bit0_only(orc):
    """Square [-0.25, 0.25]^2 at z = 1 spans screen [2, 6]^2: its diagonal from (2, 2) to
    (6, 6) passes through the centres (k + 1/2, k + 1/2), k = 2..5, where both triangles
    cover with margin 0 at the same depth. The id there is a tie (bit 0); the depth is not
    (bit 1 clear). Every other covered centre is >= 1/sqrt(2) px from the diagonal and 1/2
    px from the border."""
    depth, tid, flags = _render(orc, _scene([_square(-0.25, 0.25, -0.25, 0.25, 1.0)]))
    want = np.zeros((8, 8), np.uint8)
    for k in range(2, 6):
        want[k, k] = 1
    np.testing.assert_array_equal(flags, want)
    assert (tid[2:6, 2:6] >= 0).all() and (depth[2:6, 2:6] == 1.0).all()


@pytest.mark.parametrize("z2,tie", [(1.0, True), (1.0 + 0.5 * Z_TOL, True), (1.0 + 2.0 * Z_TOL, False)])
def test_depth_ties_between_objects(orc, z2, tie):
    """Two copies of the square of the previous test, at z = 1 and z = z2 (float32: 1 + 5e-6
    rounds to 1 + 42 * 2^-23 and 1 + 2e-5 to 1 + 168 * 2^-23, relative gaps 5.0e-6 and
    2.0e-5). Within z_tol every covered pixel's id is a tie (bit 0) whose depth moves by at
    most z_tol (bit 1 clear); beyond it only the diagonal's own tie remains. The nearer
    (or, at equal depth, the smaller id: object 0) wins."""
    a = _square(-0.25, 0.25, -0.25, 0.25, 1.0)
    b = _square(-0.25, 0.25, -0.25, 0.25, z2)
    depth, tid, flags = _render(orc, _scene([a, b]))
    want = np.zeros((8, 8), np.uint8)
    if tie:
        want[2:6, 2:6] = 1
    else:
        for k in range(2, 6):
            want[k, k] = 1
    np.testing.assert_array_equal(flags, want)
    assert (tid[2:6, 2:6] <= 1).all() and (tid[2:6, 2:6] >= 0).all()  # object 0's triangles
    assert (depth[2:6, 2:6] == 1.0).all()


# ---------------------------------------------------------------------------------------
# the log-likelihood bound
# ---------------------------------------------------------------------------------------

LIK = dict(kind=0, radius=0.005, p_outlier=0.01, half_window=1)


def _jump(cam, lk):
    V = _volume(cam)
    K = (2 * lk["half_window"] + 1) ** 2
    return _ell(1, lk["radius"], lk["p_outlier"], K, V) - _ell(0, lk["radius"], lk["p_outlier"], K, V)


def _score(orc, scene, obs, lk=LIK):
    return orc.score(scene, 0, scene.poses[0][None], lk, obs, edge_tol=EDGE_TOL, z_tol=Z_TOL, border_tol=BORDER)


@pytest.mark.parametrize("x0,n_win", [(-0.1875, 9), (-0.4375, 6)])
def test_bound_counts_observations_seeing_a_flagged_pixel(orc, x0, n_win):
    """The square with its left edge on the centres of column 2 (x0 = -0.1875) or column 0
    (x0 = -0.4375, the image border; its diagonal stays >= 0.037 px from every centre):
    rows 2..5 of that column are bit-1 pixels (4 of them). The observation is a wall at
    1.5 m, 0.5 m from every rendered point, so no pair is borderline. Each bit-1 pixel adds
    one jump per valid observed pixel in its 3x3 window: 9 inside the image, 6 at the
    border (window slots outside the image are not observations). An invalid observation
    (depth 0) at row 3 in the next column lies in the windows of rows 2, 3 and 4 only."""
    col = 2 if x0 == -0.1875 else 0
    sc = _scene([_square(x0, 0.25, -0.25, 0.25, 1.0)])
    obs = np.full((8, 8), 1.5)
    r = _score(orc, sc, obs)
    assert r["n_flag"][0] == 4 and r["n_border"][0] == 0
    assert r["bound"][0] == pytest.approx(4 * n_win * _jump(CAM8, LIK), rel=1e-12)
    obs[3, col + 1] = 0.0
    r = _score(orc, sc, obs)
    assert r["bound"][0] == pytest.approx((4 * n_win - 3) * _jump(CAM8, LIK), rel=1e-12)


def test_bound_of_one_borderline_pair(orc):
    """The plane z = 1 over the whole image (a square of side 2 m; its diagonal u = v passes
    through centres, so those pixels carry bit 0 only and must add nothing). Neighbouring
    rendered points are 1/8 m apart, far outside r = 5 mm, so every observed pixel on the
    plane has exactly one inlier: itself, at distance 0 (not borderline). The observation
    at row 2, column 5 is pushed back along its ray so that its own pair lies at
    d = r (1 - 2e-4): inside the ball, |d^2 - r^2| = 4e-4 r^2 <= 1e-3 r^2. Its count n = 1
    can step to 0 or 2 when that one pair flips, so the bound is max(l(2) - l(1),
    l(1) - l(0)) = l(1) - l(0) (l is concave in n), and nothing else adds."""
    sc = _scene([_square(-1.0, 1.0, -1.0, 1.0, 1.0)])
    _, _, flags = _render(orc, sc)
    assert (flags[np.arange(8), np.arange(8)] == 1).all() and flags.sum() == 8
    obs = np.ones((8, 8))
    ray = np.array([(5.5 - 4) / 8, (2.5 - 4) / 8, 1.0])
    obs[2, 5] = 1.0 + LIK["radius"] * (1 - 2e-4) / np.linalg.norm(ray)
    r = _score(orc, sc, obs)
    assert r["n_border"][0] == 1 and r["n_flag"][0] == 0
    assert r["bound"][0] == pytest.approx(_jump(CAM8, LIK), rel=1e-12)
    # the same pair 2e-3 r^2 from the boundary is not borderline
    obs[2, 5] = 1.0 + LIK["radius"] * (1 - 1e-3) / np.linalg.norm(ray)
    r = _score(orc, sc, obs)
    assert r["n_border"][0] == 0 and r["bound"][0] == 0.0


@pytest.mark.parametrize("w", [1, 2])
def test_bound_of_borderline_neighbours_on_a_plane(orc, w):
    """A 6x5 camera with f = 60 sees the plane z = 1 (observed = rendered, exactly):
    row and column neighbours are 1/60 m apart, diagonal ones sqrt(2)/60, and pixels two
    apart 2/60. With r = (1/60)(1 + 2e-4) every pair of 4-neighbours is inside the ball and
    borderline (|d^2 - r^2| = 4.0e-4 r^2), every other pair is far from the boundary. So an
    observed pixel with k in-image 4-neighbours has n = k + 1 inliers and k borderline pairs,
    and adds max(l(min(n + k, K)) - l(n), l(n) - l(max(n - k, 0))). The borderline pairs
    number 2 x (5 x 5 + 4 x 6) = 98: each of the 49 adjacencies counted from both ends."""
    cam = synth.Camera(6, 5, 60.0, 60.0, 3.0, 2.5, 0.01, 2.0)
    sc = _scene([_square(-1.0, 1.0, -1.0, 1.0, 1.0)], cam)
    lk = dict(kind=0, radius=(1 / 60) * (1 + 2e-4), p_outlier=0.25, half_window=w)
    obs = np.ones((5, 6))
    _, _, flags = _render(orc, sc)
    assert not flags.any()  # the diagonal u - v = 1/2 misses every centre by 1/(2 sqrt 2) px
    r = _score(orc, sc, obs, lk)
    V, K = _volume(cam), (2 * w + 1) ** 2
    ell = lambda n: _ell(n, lk["radius"], lk["p_outlier"], K, V)
    want = 0.0
    for y in range(5):
        for x in range(6):
            k = (x > 0) + (x < 5) + (y > 0) + (y < 4)
            n = k + 1
            want += max(ell(min(n + k, K)) - ell(n), ell(n) - ell(max(n - k, 0)))
    assert r["n_border"][0] == 98
    assert r["bound"][0] == pytest.approx(want, rel=1e-12)
    assert r["n_flag"][0] == 0


def _tie_scene(gap):
    """The plane z = 1 over the whole image, and a copy of it at z = 1 + gap (object 1)."""
    return _scene([_square(-1.0, 1.0, -1.0, 1.0, 1.0), _square(-1.0, 1.0, -1.0, 1.0, 1.0 + gap)])


@pytest.mark.parametrize("gap,counted", [(0.5 * Z_TOL, True), (2.0 * Z_TOL, False)])
def test_bound_of_a_pair_behind_a_depth_tie(orc, gap, counted):
    """Two planes at z = 1 and z = 1 + gap. With gap = 5e-6 (within z_tol) every pixel is an
    id tie whose depth FP32 may take from either plane: bit 0, not bit 1. The observation at
    row 2, column 5 lies d = r + 4 um from plane 1's point on its ray: outside the ball and,
    at |d^2 - r^2| = 1.6e-3 r^2, outside the 1e-3 band; but plane 2's point is 5e-6 |r_j|
    (5.2 um) further along the ray, which puts the pair inside. So the pair can flip: its
    pixel (n = 0, one pair) adds max(l(1) - l(0), 0) = one jump. With gap = 2e-5 there is
    no tie and the bound is 0. (The diagonal's coplanar tie cannot move a depth.)"""
    sc = _tie_scene(gap)
    _, _, flags = _render(orc, sc)
    assert (flags == (1 if counted else 0) | np.eye(8, dtype=np.uint8)).all()
    obs = np.ones((8, 8))
    ray = np.array([(5.5 - 4) / 8, (2.5 - 4) / 8, 1.0])
    obs[2, 5] = 1.0 + (LIK["radius"] + 4e-6) / np.linalg.norm(ray)
    r = _score(orc, sc, obs)
    assert r["n_border"][0] == 0 and r["n_flag"][0] == 0
    assert r["bound"][0] == (pytest.approx(_jump(CAM8, LIK), rel=1e-12) if counted else 0.0)


def test_smooth_bound_of_depth_ties(orc):
    """The same tie (gap 5e-6, float32: m = 42 * 2^-23) under the Gaussian kernel, s = 5 mm,
    observed = the plane: every S_i is one peak g = (2 pi s^2)^(-3/2) (neighbours 1/8 m
    apart add exp(-312)). Each tie pixel j may slide along its ray to the other plane, by
    delta_j = m |r_j|, which changes one Gaussian term of each of the 9 (or fewer, at the
    border) observed pixels seeing it by at most g e^(-1/2) delta_j / s, so each such (i, j)
    adds log(a + b (g + dN)) - log(a + b (g - dN)), a = p/V, b = (1 - p)/9. Without the
    tie the bound is 0: the diagonal's tie is between coplanar triangles (m = 0)."""
    lk = dict(kind=1, radius=0.005, p_outlier=0.01, half_window=1)
    obs = np.ones((8, 8))
    assert _score(orc, _tie_scene(2.0 * Z_TOL), obs, lk)["bound"][0] == 0.0
    r = _score(orc, _tie_scene(0.5 * Z_TOL), obs, lk)
    m = float(np.float32(1.0 + 0.5 * Z_TOL)) - 1.0
    assert m == 42 * 2.0 ** -23
    g = (2 * math.pi * 0.005 ** 2) ** -1.5
    a, b = 0.01 / _volume(CAM8), 0.99 / 9
    want = 0.0
    for y in range(8):
        for x in range(8):
            dN = g * math.exp(-0.5) / 0.005 * m * math.sqrt(((x - 3.5) / 8) ** 2 + ((y - 3.5) / 8) ** 2 + 1)
            n_obs = (min(x + 1, 7) - max(x - 1, 0) + 1) * (min(y + 1, 7) - max(y - 1, 0) + 1)
            want += n_obs * (math.log(a + b * (g + dN)) - math.log(a + b * (g - dN)))
    assert r["bound"][0] == pytest.approx(want, rel=1e-9)


# ---------------------------------------------------------------------------------------
# the gradient bound
# ---------------------------------------------------------------------------------------

SMOOTH = dict(kind=1, radius=0.005, p_outlier=0.01, half_window=1)


def _grad(orc, scene, obs):
    g = orc.score_grad(scene, 0, scene.poses[0][None], SMOOTH, obs)
    return np.concatenate([g["dpose"][0], g["dsigma"], g["dpout"]])


def _gbound(orc, scene, obs):
    r = orc.score_grad_bound(scene, 0, scene.poses[0][None], SMOOTH, obs, edge_tol=EDGE_TOL, z_tol=Z_TOL)
    return r["gbound"][0], int(r["n_flag"][0])


def test_gradient_bound_is_zero_without_flags(orc):
    """Rectangle x in [-0.25, 0.25], y in [-0.25, 0.125] at z = 1 (screen [2, 6] x [2, 5]):
    every edge half a pixel from the centres, the diagonal (4v - 3u = 2 through the corners)
    >= 0.1 px from every centre. No pixel is flagged, so nothing can move the gradient."""
    sc = _scene([_square(-0.25, 0.25, -0.25, 0.125, 1.0)])
    assert not _render(orc, sc)[2].any()
    gb, nf = _gbound(orc, sc, np.full((8, 8), 1.002))
    assert nf == 0 and (gb == 0).all()


@pytest.mark.parametrize("shift_px", [0.0, 0.5 * EDGE_TOL])
def test_gradient_bound_of_one_edge_pixel_is_its_switch(orc, shift_px):
    """A one-row rectangle x in [-0.1875 + shift/8, 0.25], y in [-0.125, 0] at z = 1 covers
    row 3, columns 2..5 (column 2 only when shift = 0, on its edge). Pixel (3, 2) is the
    only flagged pixel, its one alternative the other assignment (background or the
    rectangle). The two renders differ at that pixel alone (the plane and every other
    pixel's depth, ray and normal are the same), so the gradient of the FP64 definition
    (orc_score_grad, pinned by central differences) changes by exactly the switch the bound
    adds: gbound = |grad(shift = 0) - grad(shift = tol/2)|, component by component, seen
    from either side. The observation is a wall 2 mm behind the plane."""
    obs = np.full((8, 8), 1.002)
    sc = _scene([_square(-0.1875 + shift_px / 8.0, 0.25, -0.125, 0.0, 1.0)])
    sc_in = _scene([_square(-0.1875, 0.25, -0.125, 0.0, 1.0)])
    sc_out = _scene([_square(-0.1875 + 0.5 * EDGE_TOL / 8.0, 0.25, -0.125, 0.0, 1.0)])
    assert (_render(orc, sc_in)[1][3, 2] >= 0) and (_render(orc, sc_out)[1][3, 2] < 0)
    gb, nf = _gbound(orc, sc, obs)
    want = np.abs(_grad(orc, sc_in, obs) - _grad(orc, sc_out, obs))
    assert nf == 1
    assert want[2] > 0 and want[6] > 0 and want[7] > 0  # (x, y and z-rotation terms vanish face-on)
    np.testing.assert_allclose(gb, want, rtol=1e-9, atol=1e-12 * want.max())


def _roof(right_first):
    """A crease: plane z = 1 + (x_e - x)/2 for x in [-0.25, x_e] and plane z = 1 for x in
    [x_e, 0.25], x_e = -0.0625 (on the centres of column 3), y in [-0.125, 0] (row 3). Both
    planes give depth 1 on the crease, with different normals."""
    xe = -0.0625
    zl = 1.0 + 0.5 * (xe + 0.25)
    left = [[-0.25, -0.125, zl], [xe, -0.125, 1.0], [xe, 0.0, 1.0], [-0.25, 0.0, zl]]
    right = [[xe, -0.125, 1.0], [0.25, -0.125, 1.0], [0.25, 0.0, 1.0], [xe, 0.0, 1.0]]
    v = np.array(right + left if right_first else left + right, np.float32)
    f = np.array([[0, 1, 2], [0, 2, 3], [4, 5, 6], [4, 6, 7]], np.int32)
    return _scene([synth.Mesh(verts=v, faces=f)])


def test_gradient_bound_of_a_crease_pixel_is_its_switch(orc):
    """On the crease pixel (3, 3) both planes reach depth 1 exactly: an id tie between two
    triangles of the slot object with different planes, so the pixel's dz/dxi depends on
    which wins (bit 0; the depth does not move). Listing the right plane's triangles first
    hands the tie to the other plane (equal depths go to the smaller id) and changes
    nothing else, so the gradient difference of the two listings is exactly the switch."""
    obs = np.full((8, 8), 1.002)
    a, b = _roof(False), _roof(True)
    ta, tb = _render(orc, a)[1], _render(orc, b)[1]
    # the first-listed plane wins in each: the left plane in a, the right plane in b
    assert 0 <= ta[3, 3] < 2 and 0 <= tb[3, 3] < 2
    fa = _render(orc, a)[2]
    assert fa[3, 3] == 1 and fa.sum() == 1
    gb, nf = _gbound(orc, a, obs)
    want = np.abs(_grad(orc, a, obs) - _grad(orc, b, obs))
    assert nf == 1
    np.testing.assert_allclose(gb, want, rtol=1e-9, atol=1e-12 * np.abs(_grad(orc, a, obs)).max())
    assert want[:6].max() > 0 and want[6:].max() == 0  # the depth stays: sigma and p_out do not move


@pytest.mark.parametrize("D,cy,flagged", [(0.012, 4.4, True), (0.096, 3.7, False)])
def test_ill_conditioned_depth_is_flagged(orc, D, cy, flagged):
    """A horizontal strip y = D (x in [-1, 1], z in [0.5, 1.5]; largest vertex coordinate
    V = 1.5) seen by pixel row 4 only: its ray (y/z = (4.5 - cy)/8, 0.0125 or 0.1) meets the
    strip at z = 0.96, the rows above and below miss it, and no edge or diagonal comes
    within 0.17 px of a centre. On a plane at distance D from the camera centre,
    |n . r| z = D, so moving the plane by the FP32 resolution of its vertices, 2^-22 V,
    moves the depth by the relative amount 2^-22 V / D: 3.0e-5 for D = 1.2 cm (above
    z_tol = 1e-5: bit 2, the depth is ill-conditioned) and 3.7e-6 for D = 9.6 cm (below)."""
    cam = synth.Camera(8, 8, 8.0, 8.0, 4.0, cy, 0.01, 2.0)
    v = np.array([[-1, D, 0.5], [1, D, 0.5], [1, D, 1.5], [-1, D, 1.5]], np.float32)
    sc = _scene([synth.Mesh(verts=v, faces=np.array([[0, 1, 2], [0, 2, 3]], np.int32))], cam)
    depth, tid, flags = _render(orc, sc)
    assert (tid[4] >= 0).all() and (tid[np.arange(8) != 4] < 0).all()
    np.testing.assert_allclose(depth[4], float(np.float32(D)) / ((4.5 - cy) / 8.0), rtol=1e-12)
    want = np.zeros((8, 8), np.uint8)
    want[4] = 4 if flagged else 0
    assert 2.0 ** -22 * 1.5 / float(np.float32(D)) > Z_TOL if flagged else 2.0 ** -22 * 1.5 / float(np.float32(D)) < Z_TOL
    np.testing.assert_array_equal(flags, want)


def test_bound_of_a_pair_seen_through_an_ill_conditioned_depth(orc):
    """The strip at D = 1.2 cm of the previous test (depth resolution 2^-22 V / |n.r| along
    each ray of row 4, about 2.9e-5 m) with an observation 8 um beyond the inlier ball of the
    rendered point in its own pixel (row 4, column 2): outside the 1e-3 band, inside the
    depth resolution, so the pair can flip: one count step (n = 0, one pair: l(1) - l(0))."""
    cam = synth.Camera(8, 8, 8.0, 8.0, 4.0, 4.4, 0.01, 2.0)
    D = 0.012
    v = np.array([[-1, D, 0.5], [1, D, 0.5], [1, D, 1.5], [-1, D, 1.5]], np.float32)
    sc = _scene([synth.Mesh(verts=v, faces=np.array([[0, 1, 2], [0, 2, 3]], np.int32))], cam)
    depth, _, flags = _render(orc, sc)
    ray = np.array([(2.5 - 4) / 8, (4.5 - 4.4) / 8, 1.0])
    obs = np.full((8, 8), -1.0)  # nothing else observed
    obs[4, 2] = depth[4, 2] + (LIK["radius"] + 8e-6) / np.linalg.norm(ray)
    r = orc.score(sc, 0, sc.poses[0][None], LIK, obs, edge_tol=EDGE_TOL, z_tol=Z_TOL, border_tol=BORDER)
    V = orc.frustum_volume(cam)
    K = 9
    assert r["n_border"][0] == 0 and r["n_flag"][0] == 0
    assert r["bound"][0] == pytest.approx(_ell(1, 0.005, 0.01, K, V) - _ell(0, 0.005, 0.01, K, V), rel=1e-12)
