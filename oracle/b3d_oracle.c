/*
 * b3d_oracle.c - plain FP64 CPU oracle for the Bayes3D render-and-score path
 * (Gothoskar et al., "Bayes3D: fast learning and inference in structured generative
 * models of 3D objects and scenes", arXiv 2312.08715).
 *
 * TEST INFRASTRUCTURE. Only the tests, the package smoke check and the benchmark's CPU
 * baseline leg load this library. It shares no code, header, table or constant with the
 * CUDA library; the CUDA path never links or calls it.
 *
 * Every function is the plain definition, written for a reader to check against the
 * paper by eye: no blocking, no culling, no incremental tricks. Where the paper is silent
 * the reading used is stated at the function. FP64 throughout.
 *
 * Conventions
 *   - Poses are row-major 4x4 cam_from_obj: p_cam = R p_obj + t, R = P[0..2,0..2],
 *     t = (P[3], P[7], P[11]). OpenCV camera axes: x right, y down, z forward.
 *   - Pixel (u, v) is column u, row v; its ray passes through the pixel centre:
 *     r(u,v) = ((u + 1/2 - cx)/fx, (v + 1/2 - cy)/fy, 1). Depth is camera z.
 *   - A scene is a list of objects; object o owns faces f_off[o]..f_off[o+1]-1 and
 *     vertices v_off[o]..v_off[o+1]-1 (face indices are local to the object). The global
 *     triangle id of face f of object o is f_off[o] + f.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int32_t width, height;
    double fx, fy, cx, cy, near_z, far_z;
} orc_camera;

typedef struct {
    int32_t kind;        /* 0: inlier ball of radius r; 1: isotropic 3D Gaussian, sd sigma */
    double radius;       /* r (kind 0) or sigma (kind 1), metres */
    double p_outlier;
    int32_t half_window; /* w: window (2w+1)^2 pixels */
    double volume;       /* V of Eq. 1; <= 0 selects the camera frustum volume */
    double norm;         /* normaliser replacing 1/|y| of Eq. 1; <= 0 selects (2w+1)^2 */
    int32_t miss_mode;   /* 0: a pixel with no triangle renders at far; 1: it has no point */
} orc_lik;

typedef struct {
    int32_t n_obj;
    const int64_t *v_off;  /* [n_obj + 1] */
    const int64_t *f_off;  /* [n_obj + 1] */
    const double *verts;   /* [v_off[n_obj], 3] object frame */
    const int32_t *faces;  /* [f_off[n_obj], 3] object-local vertex indices */
    const double *poses;   /* [n_obj, 16] cam_from_obj */
} orc_scene;

typedef struct {
    int32_t n_per_axis;
    double step;
    int32_t rot_kind;    /* 0 Fibonacci-sphere set, 1 perturbation set */
    int32_t n_rot;
    double rot_max;
} orc_stage;

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------------------ */
/* Camera geometry                                                                        */
/* ------------------------------------------------------------------------------------ */

static void pixel_ray(const orc_camera *cam, int u, int v, double r[3]) {
    r[0] = ((double)u + 0.5 - cam->cx) / cam->fx;
    r[1] = ((double)v + 0.5 - cam->cy) / cam->fy;
    r[2] = 1.0;
}

/* V of Eq. 1, the volume of the scene the camera sees. Reading: the camera frustum between the
 * near and far planes. A slice at depth z spans (W z / fx) x (H z / fy), so
 * V = (W H / (fx fy)) * (far^3 - near^3) / 3. */
double orc_frustum_volume(const orc_camera *cam) {
    double a = (double)cam->width * (double)cam->height / (cam->fx * cam->fy);
    return a * (cam->far_z * cam->far_z * cam->far_z - cam->near_z * cam->near_z * cam->near_z) / 3.0;
}

static void apply_pose(const double *P, const double *p, double out[3]) {
    for (int i = 0; i < 3; ++i)
        out[i] = P[4 * i + 0] * p[0] + P[4 * i + 1] * p[1] + P[4 * i + 2] * p[2] + P[4 * i + 3];
}

static void cross3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ------------------------------------------------------------------------------------ */
/* Depth renderer (Alg. 1, DepthRenderer; the depth buffer of Sec. III-A (iii))           */
/* ------------------------------------------------------------------------------------ */
/*
 * Standard z-buffer over every triangle of every scene object.
 * Readings:
 *   - coverage: the pixel centre is inside the screen-space triangle or on its boundary
 *     (all three edge functions, oriented by the sign of the triangle's signed area, are
 *     >= 0). Triangles with zero screen area cover nothing.
 *   - depth: camera z of the intersection of the pixel-centre ray with the triangle's
 *     plane, z = (n . a) / (n . r).
 *   - a triangle with any vertex at z < near is dropped; a fragment with z > far is dropped.
 *   - the nearest fragment wins; equal depths go to the smaller global triangle id.
 *   - a pixel with no fragment has depth = far and triangle id -1.
 *
 * Ambiguity flags (optional, flags != NULL), used to make FP32-vs-FP64 parity well posed:
 *   bit 0: the triangle id at this pixel could change under a perturbation of the edge
 *          tests by edge_tol_px pixels or of depths by z_tol_rel (relative);
 *   bit 1: additionally, the depth at this pixel could change by more than z_tol_rel;
 *   bit 2: the depth is ill-conditioned: moving the winning triangle's plane by the FP32
 *          resolution of its camera-frame vertices (2 ulps of their largest coordinate,
 *          2^-22 max|v|) moves the depth along the pixel ray by more than z_tol_rel
 *          (the ray meets the plane at a grazing angle: dz = 2^-22 max|v| / |n.r|, n the
 *          unit normal, r the pixel ray with r_z = 1).
 * These are computed by a second pass over the triangles; they do not alter the image.
 */
typedef struct {
    double a[3], b[3], c[3];     /* camera-frame vertices */
    double su[3], sv[3];         /* screen coordinates */
    double area;                 /* signed screen area x2 */
    double n[3];                 /* (b - a) x (c - a) */
} tri_cam;

static int setup_tri(const orc_camera *cam, const double *P, const double *verts, const int32_t *f, tri_cam *t) {
    apply_pose(P, verts + 3 * (int64_t)f[0], t->a);
    apply_pose(P, verts + 3 * (int64_t)f[1], t->b);
    apply_pose(P, verts + 3 * (int64_t)f[2], t->c);
    const double *p[3] = {t->a, t->b, t->c};
    for (int k = 0; k < 3; ++k) {
        if (!(p[k][2] >= cam->near_z)) return 0;
        t->su[k] = cam->fx * p[k][0] / p[k][2] + cam->cx;
        t->sv[k] = cam->fy * p[k][1] / p[k][2] + cam->cy;
    }
    t->area = (t->su[1] - t->su[0]) * (t->sv[2] - t->sv[0]) - (t->sv[1] - t->sv[0]) * (t->su[2] - t->su[0]);
    if (t->area == 0.0) return 0;
    double e1[3] = {t->b[0] - t->a[0], t->b[1] - t->a[1], t->b[2] - t->a[2]};
    double e2[3] = {t->c[0] - t->a[0], t->c[1] - t->a[1], t->c[2] - t->a[2]};
    cross3(e1, e2, t->n);
    return 1;
}

/* Smallest signed distance (pixels) from the pixel centre to the three edges, positive
 * inside. Covered iff >= 0. */
static double coverage_margin(const tri_cam *t, double pu, double pv) {
    double s = t->area > 0 ? 1.0 : -1.0;
    double m = INFINITY;
    for (int k = 0; k < 3; ++k) {
        int k1 = (k + 1) % 3;
        double du = t->su[k1] - t->su[k], dv = t->sv[k1] - t->sv[k];
        double e = du * (pv - t->sv[k]) - dv * (pu - t->su[k]);
        double d = s * e / sqrt(du * du + dv * dv);
        if (d < m) m = d;
    }
    return m;
}

static double plane_depth(const tri_cam *t, const double r[3]) {
    double nr = dot3(t->n, r);
    if (nr == 0.0) return INFINITY;
    return dot3(t->n, t->a) / nr;
}

static const double *object_pose(const orc_scene *sc, int o, int32_t slot, const double *slot_pose) {
    if (o == slot && slot_pose) return slot_pose;
    return sc->poses + 16 * (int64_t)o;
}

/* Camera-frame vertices of the triangle with global id g. */
static void tri_vertices_cam(const orc_scene *sc, int32_t slot, const double *slot_pose, int32_t g, double A[3],
                             double B[3], double C[3]) {
    int o = 0;
    while (o + 1 < sc->n_obj && g >= sc->f_off[o + 1]) ++o;
    const double *Po = object_pose(sc, o, slot, slot_pose);
    const double *verts = sc->verts + 3 * sc->v_off[o];
    const int32_t *f = sc->faces + 3 * (int64_t)g;
    apply_pose(Po, verts + 3 * (int64_t)f[0], A);
    apply_pose(Po, verts + 3 * (int64_t)f[1], B);
    apply_pose(Po, verts + 3 * (int64_t)f[2], C);
}

/* Depth change along the ray r (r_z = 1) of pixel (x, y) when the plane of triangle g moves by
 * the FP32 resolution of its camera-frame vertices: 2^-22 max|v| / |n.r|, n the unit normal. */
static double depth_resolution(const orc_camera *cam, const orc_scene *sc, int32_t slot, const double *slot_pose,
                               int32_t g, int x, int y) {
    double A[3], B[3], C[3], e1[3], e2[3], n[3], r[3];
    tri_vertices_cam(sc, slot, slot_pose, g, A, B, C);
    double vmax = 0;
    for (int k = 0; k < 3; ++k) vmax = fmax(vmax, fmax(fabs(A[k]), fmax(fabs(B[k]), fabs(C[k]))));
    for (int k = 0; k < 3; ++k) { e1[k] = B[k] - A[k]; e2[k] = C[k] - A[k]; }
    cross3(e1, e2, n);
    pixel_ray(cam, x, y, r);
    const double nr = fabs(dot3(n, r)) / sqrt(dot3(n, n));
    return nr > 0 ? ldexp(vmax, -22) / nr : INFINITY;
}

static void pixel_range(double lo, double hi, double tol, int n, int *a, int *b) {
    double fa = ceil(lo - 0.5 - tol), fb = floor(hi - 0.5 + tol);
    if (fa < 0) fa = 0;
    if (fb > n - 1) fb = n - 1;
    if (!(fa <= fb)) { *a = 1; *b = 0; return; }
    *a = (int)fa;
    *b = (int)fb;
}

/* zmove (optional, with flags): per pixel, the largest |depth change| among the alternatives
 * that set its flags (0 where none). */
static int render_core(const orc_camera *cam, const orc_scene *sc, int32_t slot, const double *slot_pose,
                       double edge_tol_px, double z_tol_rel, double *depth, int32_t *triid, uint8_t *flags,
                       double *zmove) {
    if (!cam || !sc || !depth || !triid || cam->width <= 0 || cam->height <= 0) return ORC_EINVAL;
    const int W = cam->width, H = cam->height;
    const int64_t P = (int64_t)W * H;
    double *best_z = malloc(sizeof(double) * P), *second_z = malloc(sizeof(double) * P);
    double *best_m = malloc(sizeof(double) * P);
    if (!best_z || !second_z || !best_m) { free(best_z); free(second_z); free(best_m); return ORC_ENOMEM; }
    for (int64_t i = 0; i < P; ++i) { best_z[i] = INFINITY; second_z[i] = INFINITY; best_m[i] = 0; triid[i] = -1; }
    const double tol = flags ? edge_tol_px : 0.0;

    for (int pass = 0; pass < (flags ? 2 : 1); ++pass) {
        if (pass == 1)
            for (int64_t i = 0; i < P; ++i) {
                flags[i] = 0;
                if (zmove) zmove[i] = 0.0;
            }
        for (int o = 0; o < sc->n_obj; ++o) {
            const double *Po = object_pose(sc, o, slot, slot_pose);
            const double *verts = sc->verts + 3 * sc->v_off[o];
            for (int64_t f = sc->f_off[o]; f < sc->f_off[o + 1]; ++f) {
                tri_cam t;
                if (!setup_tri(cam, Po, verts, sc->faces + 3 * f, &t)) continue;
                double umin = fmin(t.su[0], fmin(t.su[1], t.su[2])), umax = fmax(t.su[0], fmax(t.su[1], t.su[2]));
                double vmin = fmin(t.sv[0], fmin(t.sv[1], t.sv[2])), vmax = fmax(t.sv[0], fmax(t.sv[1], t.sv[2]));
                int x0, x1, y0, y1;
                pixel_range(umin, umax, tol, W, &x0, &x1);
                pixel_range(vmin, vmax, tol, H, &y0, &y1);
                const int32_t gid = (int32_t)f;
                for (int y = y0; y <= y1; ++y)
                    for (int x = x0; x <= x1; ++x) {
                        double r[3];
                        pixel_ray(cam, x, y, r);
                        double m = coverage_margin(&t, x + 0.5, y + 0.5);
                        double z = plane_depth(&t, r);
                        if (!(z <= cam->far_z)) continue;
                        const int64_t i = (int64_t)y * W + x;
                        if (pass == 0) {
                            if (m < 0) continue;
                            if (z < best_z[i] || (z == best_z[i] && gid < triid[i])) {
                                second_z[i] = best_z[i];
                                best_z[i] = z;
                                triid[i] = gid;
                                best_m[i] = m;
                            } else if (z < second_z[i]) {
                                second_z[i] = z;
                            }
                        } else {
                            /* a triangle other than the winner whose coverage is marginal and
                             * that is not behind the winner could take the pixel */
                            if (gid == triid[i] || fabs(m) >= tol) continue;
                            double zb = triid[i] >= 0 ? best_z[i] : cam->far_z;
                            if (z <= zb * (1.0 + z_tol_rel)) {
                                flags[i] |= 1;
                                if (fabs(z - zb) > z_tol_rel * zb) flags[i] |= 2;
                                if (zmove) zmove[i] = fmax(zmove[i], fabs(z - zb));
                            }
                        }
                    }
            }
        }
    }
    for (int64_t i = 0; i < P; ++i) {
        if (triid[i] >= 0) {
            depth[i] = best_z[i];
            if (flags) {
                /* the winner's depth itself is fixed only to the FP32 resolution of its plane */
                const double dz = depth_resolution(cam, sc, slot, slot_pose, triid[i], (int)(i % W), (int)(i / W));
                if (dz > z_tol_rel * best_z[i]) {
                    flags[i] |= 4;
                    if (zmove) zmove[i] = fmax(zmove[i], dz);
                }
                /* the winner itself barely covers the pixel: the next candidate takes over */
                if (best_m[i] < tol) {
                    double alt = isinf(second_z[i]) ? cam->far_z : second_z[i];
                    flags[i] |= 1;
                    if (fabs(alt - best_z[i]) > z_tol_rel * best_z[i]) flags[i] |= 2;
                    if (zmove) zmove[i] = fmax(zmove[i], fabs(alt - best_z[i]));
                }
                /* near-equal depths: the id decided by the depth test could swap */
                if (second_z[i] - best_z[i] <= z_tol_rel * best_z[i]) {
                    flags[i] |= 1;
                    if (zmove) zmove[i] = fmax(zmove[i], second_z[i] - best_z[i]);
                }
            }
        } else {
            depth[i] = cam->far_z;
        }
    }
    free(best_z); free(second_z); free(best_m);
    return ORC_OK;
}

int orc_render(const orc_camera *cam, const orc_scene *sc, int32_t slot, const double *slot_pose,
               double edge_tol_px, double z_tol_rel, double *depth, int32_t *triid, uint8_t *flags) {
    return render_core(cam, sc, slot, slot_pose, edge_tol_px, z_tol_rel, depth, triid, flags, NULL);
}

/* Depth with visibility held fixed: pixel i keeps triangle triid[i] (rendered with the
 * scene's poses except slot at slot_pose); its depth is the intersection of the pixel ray
 * with that triangle's plane, whether or not the centre is still inside the triangle.
 * Used to check the fixed-visibility gradient by central differences. */
int orc_render_fixed(const orc_camera *cam, const orc_scene *sc, int32_t slot, const double *slot_pose,
                     const int32_t *triid, double *depth) {
    if (!cam || !sc || !triid || !depth) return ORC_EINVAL;
    const int W = cam->width, H = cam->height;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const int64_t i = (int64_t)y * W + x;
            int32_t g = triid[i];
            if (g < 0) { depth[i] = cam->far_z; continue; }
            int o = 0;
            while (o + 1 < sc->n_obj && g >= sc->f_off[o + 1]) ++o;
            const double *Po = object_pose(sc, o, slot, slot_pose);
            const double *verts = sc->verts + 3 * sc->v_off[o];
            const int32_t *f = sc->faces + 3 * (int64_t)g;
            double a[3], b[3], c[3], e1[3], e2[3], n[3], r[3];
            apply_pose(Po, verts + 3 * (int64_t)f[0], a);
            apply_pose(Po, verts + 3 * (int64_t)f[1], b);
            apply_pose(Po, verts + 3 * (int64_t)f[2], c);
            for (int k = 0; k < 3; ++k) { e1[k] = b[k] - a[k]; e2[k] = c[k] - a[k]; }
            cross3(e1, e2, n);
            pixel_ray(cam, x, y, r);
            depth[i] = dot3(n, a) / dot3(n, r);
        }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Windowed robust likelihood (Eq. 1 with the window truncation of Sec. III-B)            */
/* ------------------------------------------------------------------------------------ */
/*
 * For every observed pixel i with finite depth > 0, with observed point
 * qt_i = depth_obs[i] * r_i and rendered points q_j = depth_ren[j] * r_j over the
 * (2w+1)^2 pixels j around i that lie inside the image:
 *   kind 0:  n_i = #{ j : |qt_i - q_j|^2 <= r^2 },
 *            l_i = log( p_out / V + (1 - p_out) * n_i / (K * (4/3) pi r^3) )
 *   kind 1:  S_i = sum_j (2 pi s^2)^(-3/2) exp(-|qt_i - q_j|^2 / (2 s^2)),
 *            l_i = log( p_out / V + (1 - p_out) * S_i / K )
 * Readings: the inlier kernel of Eq. 1 is the uniform density of a ball of radius r
 * (kind 0) or an isotropic Gaussian with per-coordinate standard deviation s (kind 1);
 * the normaliser 1/|y| becomes 1/K with K = (2w+1)^2 (window slots outside the image count
 * in K and contribute nothing); the prefactor sigma/sigma_max of Eq. 1 is left out (a
 * constant for fixed noise parameters); rendered pixels without a triangle sit at the far
 * plane (miss_mode 0) or carry no point (miss_mode 1). Pixels not scored get NaN.
 *
 * Outputs (each optional): ell[H*W], count[H*W] (kind 0 n_i), ssum[H*W] (kind 1 S_i).
 * *n_border counts window pairs with |d^2 - r^2| <= border_tol * r^2 (kind 0).
 */
static void lik_constants(const orc_camera *cam, const orc_lik *lk, double *V, double *K) {
    int w = lk->half_window;
    *V = lk->volume > 0 ? lk->volume : orc_frustum_volume(cam);
    *K = lk->norm > 0 ? lk->norm : (double)((2 * w + 1) * (2 * w + 1));
}

int orc_pixel_loglik(const orc_camera *cam, const orc_lik *lk, const double *depth_ren, const int32_t *triid_ren,
                     const double *depth_obs, double border_tol, double *ell, int32_t *count, double *ssum,
                     int64_t *n_border) {
    if (!cam || !lk || !depth_ren || !depth_obs || lk->half_window < 0 || !(lk->radius > 0)) return ORC_EINVAL;
    if (lk->miss_mode == 1 && !triid_ren) return ORC_EINVAL;
    const int W = cam->width, H = cam->height, w = lk->half_window;
    double V, K;
    lik_constants(cam, lk, &V, &K);
    const double r = lk->radius, r2 = r * r;
    const double ball = 4.0 / 3.0 * ORC_PI * r * r * r;
    const double gnorm = pow(2.0 * ORC_PI * r2, -1.5);
    int64_t nb = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const int64_t i = (int64_t)y * W + x;
            double d_obs = depth_obs[i];
            if (!(d_obs > 0) || !isfinite(d_obs)) {
                if (ell) ell[i] = NAN;
                if (count) count[i] = 0;
                if (ssum) ssum[i] = 0;
                continue;
            }
            double ri[3], qt[3];
            pixel_ray(cam, x, y, ri);
            for (int k = 0; k < 3; ++k) qt[k] = d_obs * ri[k];
            int n = 0;
            double S = 0.0;
            for (int dy = -w; dy <= w; ++dy)
                for (int dx = -w; dx <= w; ++dx) {
                    int xj = x + dx, yj = y + dy;
                    if (xj < 0 || xj >= W || yj < 0 || yj >= H) continue;
                    const int64_t j = (int64_t)yj * W + xj;
                    if (lk->miss_mode == 1 && triid_ren[j] < 0) continue;
                    double rj[3], q[3];
                    pixel_ray(cam, xj, yj, rj);
                    for (int k = 0; k < 3; ++k) q[k] = depth_ren[j] * rj[k];
                    double d2 = (qt[0] - q[0]) * (qt[0] - q[0]) + (qt[1] - q[1]) * (qt[1] - q[1]) +
                                (qt[2] - q[2]) * (qt[2] - q[2]);
                    if (lk->kind == 0) {
                        if (d2 <= r2) ++n;
                        if (fabs(d2 - r2) <= border_tol * r2) ++nb;
                    } else {
                        S += gnorm * exp(-d2 / (2.0 * r2));
                    }
                }
            double li = lk->kind == 0 ? log(lk->p_outlier / V + (1.0 - lk->p_outlier) * n / (K * ball))
                                      : log(lk->p_outlier / V + (1.0 - lk->p_outlier) * S / K);
            if (ell) ell[i] = li;
            if (count) count[i] = n;
            if (ssum) ssum[i] = S;
        }
    if (n_border) *n_border = nb;
    return ORC_OK;
}

/* l_i as a function of the inlier count n (kind 0). */
static double ell_of_count(const orc_camera *cam, const orc_lik *lk, int n) {
    double V, K;
    lik_constants(cam, lk, &V, &K);
    const double r = lk->radius, ball = 4.0 / 3.0 * ORC_PI * r * r * r;
    return log(lk->p_outlier / V + (1.0 - lk->p_outlier) * n / (K * ball));
}

/* Largest change of one observed pixel's l_i that moving ONE rendered point of its window
 * can cause: a count step 0 <-> 1 (kind 0, the largest step since l is concave in n) or
 * one Gaussian term between 0 and its peak (kind 1). */
static double pixel_jump(const orc_camera *cam, const orc_lik *lk) {
    double V, K;
    lik_constants(cam, lk, &V, &K);
    const double r = lk->radius;
    double top = lk->kind == 0 ? (1.0 - lk->p_outlier) / (K * (4.0 / 3.0 * ORC_PI * r * r * r))
                               : (1.0 - lk->p_outlier) * pow(2.0 * ORC_PI * r * r, -1.5) / K;
    return log(lk->p_outlier / V + top) - log(lk->p_outlier / V);
}

/* Largest change of l_i when k of its window pairs may each flip in or out of the ball,
 * from the current count n (kind 0). */
static double count_flip_bound(const orc_camera *cam, const orc_lik *lk, int n, int k) {
    const int w = lk->half_window, slots = (2 * w + 1) * (2 * w + 1);
    int hi = n + k > slots ? slots : n + k, lo = n - k < 0 ? 0 : n - k;
    double l = ell_of_count(cam, lk, n);
    return fmax(ell_of_count(cam, lk, hi) - l, l - ell_of_count(cam, lk, lo));
}

/* ------------------------------------------------------------------------------------ */
/* Per-hypothesis log-likelihood: render the scene with object `slot` at each pose, then */
/* sum l_i over the scored pixels (the product over i of Eq. 1, in logs).                */
/* ------------------------------------------------------------------------------------ */
/*
 * Outputs per hypothesis h (each optional except ll):
 *   ll[h]     = sum_i l_i
 *   scale[h]  = sum_i |l_i|                (the tolerance scale)
 *   bound[h]  = largest |change of ll| that FP32-resolution decisions could cause:
 *               - every depth-ambiguous rendered pixel j (flag bit 1) may move anywhere:
 *                 one point's jump for each valid observed pixel whose window contains it;
 *               - a rendered pixel j whose id is a tie but whose depth stays within
 *                 z_tol_rel (bit 0 without bit 1) may move along its ray to the depth of
 *                 an alternative: by up to delta_j = m_j |r_j|, m_j the largest depth
 *                 change among the alternatives that set its flag (0 for coplanar ones);
 *                 so may a pixel whose depth is ill-conditioned (bit 2), by its depth
 *                 resolution;
 *               - kind 0: the change of l_i when its borderline pairs flip, a pair (i, j)
 *                 being borderline when |d^2 - r^2| <= border_tol r^2 or, for such a tie
 *                 pixel j, when |d - r| <= delta_j;
 *               - kind 1: for each tie pixel j and valid observed i in its window, the
 *                 change of l_i when S_i moves by the Gaussian's steepest slope
 *                 (2 pi s^2)^(-3/2) e^(-1/2) / s times delta_j.
 *   n_flag[h] = number of depth-ambiguous rendered pixels; n_border[h] = pairs within the
 *               border_tol band.
 */
int orc_score(const orc_camera *cam, const orc_scene *sc, int32_t slot, int64_t n_hyp, const double *poses,
              const orc_lik *lk, const double *depth_obs, double edge_tol_px, double z_tol_rel, double border_tol,
              double *ll, double *scale, double *bound, int32_t *n_flag, int32_t *n_border, int32_t n_threads) {
    if (!cam || !sc || !lk || !depth_obs || !ll || n_hyp < 0 || (n_hyp > 0 && !poses)) return ORC_EINVAL;
    if (slot < 0 || slot >= sc->n_obj) return ORC_EINVAL;
    const int W = cam->width, H = cam->height, w = lk->half_window;
    const int64_t P = (int64_t)W * H;
    const int want_flags = (bound || n_flag || n_border) ? 1 : 0;
    const double jump = pixel_jump(cam, lk);
    int err = ORC_OK;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
    for (int64_t h = 0; h < n_hyp; ++h) {
        double *depth = malloc(sizeof(double) * P), *ell = malloc(sizeof(double) * P);
        int32_t *tid = malloc(sizeof(int32_t) * P), *cnt = malloc(sizeof(int32_t) * P);
        uint8_t *fl = want_flags ? malloc(P) : NULL;
        double *ss = want_flags && lk->kind == 1 ? malloc(sizeof(double) * P) : NULL;
        double *zmv = want_flags ? malloc(sizeof(double) * P) : NULL;
        if (!depth || !ell || !tid || !cnt || (want_flags && (!fl || !zmv)) || (want_flags && lk->kind == 1 && !ss)) {
            err = ORC_ENOMEM;
        } else {
            render_core(cam, sc, slot, poses + 16 * h, edge_tol_px, z_tol_rel, depth, tid, fl, zmv);
            int64_t nb = 0;
            orc_pixel_loglik(cam, lk, depth, tid, depth_obs, border_tol, ell, cnt, ss, &nb);
            double s = 0, a = 0, bd = 0;
            int32_t nf = 0;
            for (int64_t i = 0; i < P; ++i) {
                if (isnan(ell[i])) continue;
                s += ell[i];
                a += fabs(ell[i]);
            }
            if (want_flags) {
                for (int y = 0; y < H; ++y)
                    for (int x = 0; x < W; ++x) {
                        if (!(fl[(int64_t)y * W + x] & 2)) continue;
                        ++nf;
                        for (int dy = -w; dy <= w; ++dy)
                            for (int dx = -w; dx <= w; ++dx) {
                                int xi = x + dx, yi = y + dy;
                                if (xi < 0 || xi >= W || yi < 0 || yi >= H) continue;
                                if (!isnan(ell[(int64_t)yi * W + xi])) bd += jump;
                            }
                    }
                /* pixels whose depth may move by a bounded amount zmv: id ties within z_tol (bit 0
                 * without bit 1) and ill-conditioned depths (bit 2) */
                int n_tie = 0;
                for (int64_t j = 0; j < P; ++j)
                    if (!(fl[j] & 2) && zmv[j] > 0 && !(lk->miss_mode == 1 && tid[j] < 0)) ++n_tie;
                if (lk->kind == 1 && n_tie > 0) {
                    double V, K;
                    lik_constants(cam, lk, &V, &K);
                    const double s_ = lk->radius, pa = lk->p_outlier / V, pb = (1.0 - lk->p_outlier) / K;
                    const double slope = pow(2.0 * ORC_PI * s_ * s_, -1.5) * exp(-0.5) / s_;
                    for (int y = 0; y < H; ++y)
                        for (int x = 0; x < W; ++x) {
                            const int64_t j = (int64_t)y * W + x;
                            if ((fl[j] & 2) || !(zmv[j] > 0) || (lk->miss_mode == 1 && tid[j] < 0)) continue;
                            double rj[3];
                            pixel_ray(cam, x, y, rj);
                            const double dN = slope * zmv[j] * sqrt(dot3(rj, rj));
                            for (int dy = -w; dy <= w; ++dy)
                                for (int dx = -w; dx <= w; ++dx) {
                                    int xi = x + dx, yi = y + dy;
                                    if (xi < 0 || xi >= W || yi < 0 || yi >= H) continue;
                                    const int64_t i = (int64_t)yi * W + xi;
                                    if (isnan(ell[i])) continue;
                                    bd += log(pa + pb * (ss[i] + dN)) - log(pa + pb * fmax(ss[i] - dN, 0.0));
                                }
                        }
                }
                if (lk->kind == 0 && (nb > 0 || n_tie > 0)) {
                    /* recount borderline pairs per observed pixel to size their steps */
                    const double r2 = lk->radius * lk->radius;
                    for (int y = 0; y < H; ++y)
                        for (int x = 0; x < W; ++x) {
                            const int64_t i = (int64_t)y * W + x;
                            if (isnan(ell[i])) continue;
                            double ri[3];
                            pixel_ray(cam, x, y, ri);
                            int k_b = 0;
                            for (int dy = -w; dy <= w; ++dy)
                                for (int dx = -w; dx <= w; ++dx) {
                                    int xj = x + dx, yj = y + dy;
                                    if (xj < 0 || xj >= W || yj < 0 || yj >= H) continue;
                                    const int64_t j = (int64_t)yj * W + xj;
                                    if (lk->miss_mode == 1 && tid[j] < 0) continue;
                                    double rj[3];
                                    pixel_ray(cam, xj, yj, rj);
                                    double d2 = 0;
                                    for (int k = 0; k < 3; ++k) {
                                        double d = depth_obs[i] * ri[k] - depth[j] * rj[k];
                                        d2 += d * d;
                                    }
                                    const int tie = !(fl[j] & 2) && zmv[j] > 0;
                                    if (fabs(d2 - r2) <= border_tol * r2 ||
                                        (tie && fabs(sqrt(d2) - lk->radius) <= zmv[j] * sqrt(dot3(rj, rj))))
                                        ++k_b;
                                }
                            if (k_b > 0) bd += count_flip_bound(cam, lk, cnt[i], k_b);
                        }
                }
            }
            ll[h] = s;
            if (scale) scale[h] = a;
            if (bound) bound[h] = bd;
            if (n_flag) n_flag[h] = nf;
            if (n_border) n_border[h] = (int32_t)nb;
        }
        free(depth); free(ell); free(tid); free(cnt); free(fl); free(ss); free(zmv);
    }
    return err;
}

/* ------------------------------------------------------------------------------------ */
/* Log-sum-exp normalisation (the categorical over C2F cells, Sec. III-B)                 */
/* ------------------------------------------------------------------------------------ */
/* m = max ll; Z = m + log sum_h exp(ll_h - m); logp_h = ll_h - Z. Entries equal to -inf
 * get logp = -inf. Returns EINVAL for n <= 0 or if every entry is -inf or NaN. */
int orc_lse(int64_t n, const double *ll, double *z_out, double *logp) {
    if (n <= 0 || !ll || !z_out) return ORC_EINVAL;
    double m = -INFINITY;
    for (int64_t h = 0; h < n; ++h)
        if (ll[h] > m) m = ll[h];
    if (!isfinite(m)) return ORC_EINVAL;
    double s = 0;
    for (int64_t h = 0; h < n; ++h) s += exp(ll[h] - m);
    double Z = m + log(s);
    *z_out = Z;
    if (logp)
        for (int64_t h = 0; h < n; ++h) logp[h] = ll[h] - Z;
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Counter-based uniforms: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11)              */
/* ------------------------------------------------------------------------------------ */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
    __uint128_t p = (__uint128_t)a * (__uint128_t)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(0xD2E7470EE14C6C93ULL, x0, &hi0, &lo0);
        mulhilo64(0xCA5A826395121157ULL, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B97F4A7C15ULL;
        k1 += 0xBB67AE8584CAA73BULL;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* 24-bit uniform in [0, 1): exactly representable in FP32 and FP64 alike. */
double orc_uniform24(uint64_t x) { return (double)(x >> 40) * (1.0 / 16777216.0); }

/* Uniform number `lane` (0..3) of block (m, stage, stream) under seed. */
static double draw_uniform(uint64_t seed, int64_t m, int32_t stage, int32_t stream, int lane) {
    uint64_t ctr[4] = {(uint64_t)m, (uint64_t)(uint32_t)stage, (uint64_t)(uint32_t)stream, 0};
    uint64_t key[2] = {seed, 0};
    uint64_t out[4];
    orc_philox4x64(ctr, key, out);
    return orc_uniform24(out[lane]);
}

/* ------------------------------------------------------------------------------------ */
/* Categorical resampling by inverse CDF (sample the next region "with probability        */
/* proportional to its score", Sec. III-B)                                               */
/* ------------------------------------------------------------------------------------ */
/* Weights w_h = exp(ll_h - max ll), S = sum w_h, CDF_k = sum_{h<=k} w_h. Draw m uses
 * u_m = uniform24(philox(ctr = (m, stage, 0, 0), key = (seed, 0)).x0) and picks
 * idx_m = min{ k : CDF_k > u_m S }. logq_m = ll[idx_m] - Z. margin_m = distance of u_m S
 * to the nearer end of the chosen interval, divided by S (small = decision fragile). */
int orc_resample(int64_t n, const double *ll, int32_t m, uint64_t seed, int32_t stage, int32_t *idx,
                 double *logq, double *margin) {
    if (n <= 0 || m < 0 || !ll || (m > 0 && !idx)) return ORC_EINVAL;
    double Z;
    if (orc_lse(n, ll, &Z, NULL) != ORC_OK) return ORC_EINVAL;
    double mx = -INFINITY;
    for (int64_t h = 0; h < n; ++h)
        if (ll[h] > mx) mx = ll[h];
    double *cdf = malloc(sizeof(double) * n);
    if (!cdf) return ORC_ENOMEM;
    double s = 0;
    for (int64_t h = 0; h < n; ++h) { s += exp(ll[h] - mx); cdf[h] = s; }
    for (int32_t k = 0; k < m; ++k) {
        double t = draw_uniform(seed, k, stage, 0, 0) * s;
        int64_t lo = 0, hi = n - 1;
        while (lo < hi) { /* first index with cdf > t */
            int64_t mid = lo + (hi - lo) / 2;
            if (cdf[mid] > t) hi = mid; else lo = mid + 1;
        }
        idx[k] = (int32_t)lo;
        if (logq) logq[k] = ll[lo] - Z;
        if (margin) {
            double left = lo > 0 ? cdf[lo - 1] : 0.0;
            margin[k] = fmin(t - left, cdf[lo] - t) / s;
        }
    }
    free(cdf);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Coarse-to-fine hypothesis grids (the partitions Pi_t of Sec. III-B)                   */
/* ------------------------------------------------------------------------------------ */
static void rot_axis_angle(const double axis[3], double angle, double *R) {
    double n = sqrt(dot3(axis, axis));
    double k[3] = {axis[0] / n, axis[1] / n, axis[2] / n};
    double c = cos(angle), s = sin(angle), C = 1.0 - c;
    R[0] = c + k[0] * k[0] * C;        R[1] = k[0] * k[1] * C - k[2] * s; R[2] = k[0] * k[2] * C + k[1] * s;
    R[3] = k[1] * k[0] * C + k[2] * s; R[4] = c + k[1] * k[1] * C;        R[5] = k[1] * k[2] * C - k[0] * s;
    R[6] = k[2] * k[0] * C - k[1] * s; R[7] = k[2] * k[1] * C + k[0] * s; R[8] = c + k[2] * k[2] * C;
}

/* Weyl sequence frac(1/2 + k a) in exact 64-bit fixed point: A = round(2^64 a); the top 53
 * bits of 2^63 + k A (mod 2^64) give the value as a double in [0, 1). */
static double weyl_u(uint64_t A, int32_t k) {
    const uint64_t x = 0x8000000000000000ull + (uint64_t)k * A;
    return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

/* Rotation sets (reading; the paper gives no scheme):
 *   kind 0, Fibonacci sphere: d_k = (sqrt(1-z^2) cos(2 pi k / phi), sqrt(1-z^2) sin(2 pi k / phi), z),
 *           z = 1 - (2k+1)/n, phi the golden ratio; R_k is the minimal-arc rotation taking
 *           +z to d_k (pi about x for the antipode, identity for +z itself).
 *   kind 1, perturbation: a low-discrepancy set uniform in the ball of rotation vectors of
 *           radius rot_max. R_0 is the identity (the grid centre's own rotation); for k >= 1,
 *           R_k = Exp(rot_max cbrt(u0) d) with d = (sqrt(1-z^2) cos(2 pi u2),
 *           sqrt(1-z^2) sin(2 pi u2), z), z = 1 - 2 u1, where (u0, u1, u2) = frac(1/2 + k a)
 *           is the 3-D R-sequence (Roberts): a = (1/g, 1/g^2, 1/g^3), g the real root above 1
 *           of x^4 = x + 1. (u -> the ball is volume-preserving: radius cbrt(u0), direction
 *           uniform on the sphere.)
 * Output R[n, 9] row-major. */
#define ORC_R3_A1 0xd1b54a32d192ed04ull /* round(2^64 / g) */
#define ORC_R3_A2 0xabc98388fb8fac03ull /* round(2^64 / g^2) */
#define ORC_R3_A3 0x8cb92ba72f3d8dd7ull /* round(2^64 / g^3) */
int orc_rotation_set(int32_t kind, int32_t n, double rot_max, double *R) {
    if (n <= 0 || !R || (kind != 0 && kind != 1)) return ORC_EINVAL;
    const double phi = (1.0 + sqrt(5.0)) / 2.0;
    for (int k = 0; k < n; ++k) {
        double z = 1.0 - (2.0 * k + 1.0) / n;
        double rho = sqrt(fmax(0.0, 1.0 - z * z));
        double ang = 2.0 * ORC_PI * k / phi;
        double d[3] = {rho * cos(ang), rho * sin(ang), z};
        double *Rk = R + 9 * k;
        if (kind == 0) {
            double ez[3] = {0, 0, 1}, ax[3];
            cross3(ez, d, ax);
            double sn = sqrt(dot3(ax, ax));
            if (sn == 0.0) {
                if (z > 0) { double I[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}; memcpy(Rk, I, sizeof I); }
                else { double X[3] = {1, 0, 0}; rot_axis_angle(X, ORC_PI, Rk); }
            } else {
                rot_axis_angle(ax, atan2(sn, z), Rk);
            }
        } else {
            const double u0 = weyl_u(ORC_R3_A1, k), u1 = weyl_u(ORC_R3_A2, k), u2 = weyl_u(ORC_R3_A3, k);
            const double theta = rot_max * cbrt(u0);
            const double zz = 1.0 - 2.0 * u1, s = sqrt(fmax(0.0, 1.0 - zz * zz));
            double e[3] = {s * cos(2.0 * ORC_PI * u2), s * sin(2.0 * ORC_PI * u2), zz};
            if (k == 0 || theta == 0.0) { double I[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}; memcpy(Rk, I, sizeof I); }
            else rot_axis_angle(e, theta, Rk);
        }
    }
    return ORC_OK;
}

/* Grid offset of index i on an axis of n points with spacing step: odd n is centred
 * ((i - (n-1)/2) step); even n puts the centre at i = n/2 ((i - n/2) step). */
static double grid_offset(int i, int n, double step) {
    return (n % 2 ? (i - (n - 1) / 2) : (i - n / 2)) * step;
}

/* Hypothesis h = ((ir * n + ix) * n + iy) * n + iz of one stage:
 *   R_h = R_c R_ir        (rotation sets act in the object frame)
 *   t_h = t_c + G (o_ix, o_iy, o_iz)   (G: grid frame rotation, cam_from_grid)
 * Output poses[n^3 * n_rot, 16]. */
int orc_expand(const double *centre, const double *G, int32_t n, double step, const double *rotset,
               int32_t n_rot, double *poses) {
    if (!centre || !G || !rotset || !poses || n <= 0 || n_rot <= 0) return ORC_EINVAL;
    int64_t h = 0;
    for (int ir = 0; ir < n_rot; ++ir)
        for (int ix = 0; ix < n; ++ix)
            for (int iy = 0; iy < n; ++iy)
                for (int iz = 0; iz < n; ++iz, ++h) {
                    const double *Rk = rotset + 9 * ir;
                    double *P = poses + 16 * h;
                    double o[3] = {grid_offset(ix, n, step), grid_offset(iy, n, step), grid_offset(iz, n, step)};
                    for (int a = 0; a < 3; ++a) {
                        for (int b = 0; b < 3; ++b)
                            P[4 * a + b] = centre[4 * a + 0] * Rk[0 * 3 + b] + centre[4 * a + 1] * Rk[1 * 3 + b] +
                                           centre[4 * a + 2] * Rk[2 * 3 + b];
                        P[4 * a + 3] = centre[4 * a + 3] + G[3 * a + 0] * o[0] + G[3 * a + 1] * o[1] + G[3 * a + 2] * o[2];
                    }
                    P[12] = 0; P[13] = 0; P[14] = 0; P[15] = 1;
                }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------ */
/* Coarse-to-fine enumeration (Sec. III-B), one object                                    */
/* ------------------------------------------------------------------------------------ */
/*
 * For stage t = 0..T-1: expand the stage grid around centre_t, score every hypothesis
 * (scoring strategy: one point per cell, its centre, weight 1), draw M cells by
 * orc_resample(seed, stage t), and take as centre_{t+1} the drawn cell with the highest
 * ll (ties to the smaller hypothesis index). After the last stage each particle is its
 * drawn cell's pose with a uniform translation jitter inside the cell:
 * t += G ((u0 - 1/2) s, (u1 - 1/2) s, (u2 - 1/2) s), u from philox(ctr = (m, T, 1, 0)).
 *   logw_m = ll_T(idx_m)  (score of the drawn cell)
 *   logq_m = ll_T(idx_m) - Z_T - 3 log(s_T)  (categorical x uniform-in-cell density)
 * Optional diagnostics: centres[T,16], zs[T], idx_all[T, M].
 */
int orc_enumerate_c2f(const orc_camera *cam, const orc_scene *sc, int32_t slot, const double *centre0,
                      const double *G, const orc_lik *lk, const double *depth_obs, int32_t n_stages,
                      const orc_stage *stages, int32_t m, uint64_t seed, int32_t path_density, double *particles,
                      double *logw, double *logq, double *centres, double *zs, int32_t *idx_all, int32_t n_threads) {
    if (!cam || !sc || !centre0 || !G || !lk || !depth_obs || n_stages <= 0 || !stages || m <= 0 || !particles)
        return ORC_EINVAL;
    double centre[16];
    memcpy(centre, centre0, sizeof centre);
    double path = 0.0;  /* log probability of the cells that centred the later stages */
    int err = ORC_OK;
    int32_t *idx = malloc(sizeof(int32_t) * m);
    double *poses = NULL, *ll = NULL, *rot = NULL;
    for (int t = 0; t < n_stages && err == ORC_OK; ++t) {
        const orc_stage *st = &stages[t];
        int64_t nh = (int64_t)st->n_per_axis * st->n_per_axis * st->n_per_axis * st->n_rot;
        free(poses); free(ll); free(rot);
        poses = malloc(sizeof(double) * 16 * nh);
        ll = malloc(sizeof(double) * nh);
        rot = malloc(sizeof(double) * 9 * st->n_rot);
        if (!poses || !ll || !rot || !idx) { err = ORC_ENOMEM; break; }
        if (centres) memcpy(centres + 16 * t, centre, sizeof centre);
        if ((err = orc_rotation_set(st->rot_kind, st->n_rot, st->rot_max, rot)) != ORC_OK) break;
        if ((err = orc_expand(centre, G, st->n_per_axis, st->step, rot, st->n_rot, poses)) != ORC_OK) break;
        if ((err = orc_score(cam, sc, slot, nh, poses, lk, depth_obs, 0, 0, 0, ll, NULL, NULL, NULL, NULL,
                             n_threads)) != ORC_OK) break;
        double Z;
        orc_lse(nh, ll, &Z, NULL);
        if (zs) zs[t] = Z;
        if ((err = orc_resample(nh, ll, m, seed, t, idx, NULL, NULL)) != ORC_OK) break;
        if (idx_all) memcpy(idx_all + (int64_t)t * m, idx, sizeof(int32_t) * m);
        int32_t best = idx[0];
        for (int k = 1; k < m; ++k)
            if (ll[idx[k]] > ll[best] || (ll[idx[k]] == ll[best] && idx[k] < best)) best = idx[k];
        if (t + 1 < n_stages) {
            memcpy(centre, poses + 16 * (int64_t)best, sizeof centre);
            if (path_density) path += ll[best] - Z;
        } else {
            const double s = st->step;
            for (int k = 0; k < m; ++k) {
                double *out = particles + 16 * (int64_t)k;
                memcpy(out, poses + 16 * (int64_t)idx[k], sizeof(double) * 16);
                double u[3];
                for (int l = 0; l < 3; ++l) u[l] = (draw_uniform(seed, k, n_stages, 1, l) - 0.5) * s;
                for (int a = 0; a < 3; ++a) out[4 * a + 3] += G[3 * a + 0] * u[0] + G[3 * a + 1] * u[1] + G[3 * a + 2] * u[2];
                if (logw) logw[k] = ll[idx[k]];
                if (logq) logq[k] = ll[idx[k]] - Z - 3.0 * log(s) + path;
            }
        }
    }
    free(idx); free(poses); free(ll); free(rot);
    return err;
}

/* ------------------------------------------------------------------------------------ */
/* Gradient of the Gaussian-window log-likelihood (kind 1)                                */
/* ------------------------------------------------------------------------------------ */
/*
 * With a = p_out / V, b = (1 - p_out) / K, N_ij = (2 pi s^2)^(-3/2) exp(-d_ij^2 / (2 s^2)),
 * S_i = sum_j N_ij, p_i = a + b S_i, LL = sum_i log p_i:
 *   dLL/ds     = sum_i (b / p_i) sum_j N_ij (d_ij^2 / s^3 - 3 / s)
 *   dLL/dp_out = sum_i (1/V - S_i / K) / p_i
 *   dLL/dxi    = sum_j g_j dz_j/dxi,  g_j = sum_{i : j in win(i)} (b / p_i) N_ij (qt_i - q_j).r_j / s^2
 * Pose derivative (reading; the paper is silent): left perturbation in the camera frame,
 * T(xi) = Exp([v, w]^) T at xi = 0, visibility held fixed, and the rendered point sliding
 * along its pixel ray on the fixed triangle's plane (n . (z r - a) = 0):
 *   dz_j/dv = n / (n . r_j),   dz_j/dw = (q_j x n) / (n . r_j)
 * Only pixels whose triangle belongs to object `slot` move; misses and other objects don't.
 * Output dpose[n_hyp, 6] ordered (v, w).
 */
int orc_score_grad(const orc_camera *cam, const orc_scene *sc, int32_t slot, int64_t n_hyp, const double *poses,
                   const orc_lik *lk, const double *depth_obs, double *ll, double *dpose, double *dsigma,
                   double *dpout, int32_t n_threads) {
    if (!cam || !sc || !lk || lk->kind != 1 || !depth_obs || !ll || (n_hyp > 0 && !poses)) return ORC_EINVAL;
    if (slot < 0 || slot >= sc->n_obj || !(lk->radius > 0)) return ORC_EINVAL;
    const int W = cam->width, H = cam->height, w = lk->half_window;
    const int64_t P = (int64_t)W * H;
    double V, K;
    lik_constants(cam, lk, &V, &K);
    const double s = lk->radius, s2 = s * s;
    const double gnorm = pow(2.0 * ORC_PI * s2, -1.5);
    const double a = lk->p_outlier / V, b = (1.0 - lk->p_outlier) / K;
    int err = ORC_OK;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
    for (int64_t h = 0; h < n_hyp; ++h) {
        double *depth = malloc(sizeof(double) * P), *inv_p = malloc(sizeof(double) * P);
        int32_t *tid = malloc(sizeof(int32_t) * P);
        if (!depth || !inv_p || !tid) { err = ORC_ENOMEM; free(depth); free(inv_p); free(tid); continue; }
        const double *Ph = poses + 16 * h;
        orc_render(cam, sc, slot, Ph, 0, 0, depth, tid, NULL);
        double L = 0, gs = 0, gp = 0, gx[6] = {0, 0, 0, 0, 0, 0};
        /* pass 1: p_i, and the sigma / p_out terms */
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const int64_t i = (int64_t)y * W + x;
                inv_p[i] = 0;
                double d_obs = depth_obs[i];
                if (!(d_obs > 0) || !isfinite(d_obs)) continue;
                double ri[3];
                pixel_ray(cam, x, y, ri);
                double S = 0, dS = 0;
                for (int dy = -w; dy <= w; ++dy)
                    for (int dx = -w; dx <= w; ++dx) {
                        int xj = x + dx, yj = y + dy;
                        if (xj < 0 || xj >= W || yj < 0 || yj >= H) continue;
                        const int64_t j = (int64_t)yj * W + xj;
                        if (lk->miss_mode == 1 && tid[j] < 0) continue;
                        double rj[3], d2 = 0;
                        pixel_ray(cam, xj, yj, rj);
                        for (int k = 0; k < 3; ++k) {
                            double d = d_obs * ri[k] - depth[j] * rj[k];
                            d2 += d * d;
                        }
                        double N = gnorm * exp(-d2 / (2.0 * s2));
                        S += N;
                        dS += N * (d2 / (s2 * s) - 3.0 / s);
                    }
                double p = a + b * S;
                L += log(p);
                gs += b * dS / p;
                gp += (1.0 / V - S / K) / p;
                inv_p[i] = 1.0 / p;
            }
        /* pass 2: pose gradient through the slot object's rendered points */
        const int64_t f0 = sc->f_off[slot], f1 = sc->f_off[slot + 1];
        const double *verts = sc->verts + 3 * sc->v_off[slot];
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const int64_t j = (int64_t)y * W + x;
                if (tid[j] < f0 || tid[j] >= f1) continue;
                double rj[3], qj[3];
                pixel_ray(cam, x, y, rj);
                for (int k = 0; k < 3; ++k) qj[k] = depth[j] * rj[k];
                double g = 0;
                for (int dy = -w; dy <= w; ++dy)
                    for (int dx = -w; dx <= w; ++dx) {
                        int xi = x + dx, yi = y + dy;
                        if (xi < 0 || xi >= W || yi < 0 || yi >= H) continue;
                        const int64_t i = (int64_t)yi * W + xi;
                        if (inv_p[i] == 0) continue;
                        double ri[3], diff[3], d2 = 0;
                        pixel_ray(cam, xi, yi, ri);
                        for (int k = 0; k < 3; ++k) {
                            diff[k] = depth_obs[i] * ri[k] - qj[k];
                            d2 += diff[k] * diff[k];
                        }
                        double N = gnorm * exp(-d2 / (2.0 * s2));
                        g += b * inv_p[i] * N * dot3(diff, rj) / s2;
                    }
                const int32_t *f = sc->faces + 3 * (int64_t)tid[j];
                double A[3], B[3], C[3], e1[3], e2[3], n[3], qxn[3];
                apply_pose(Ph, verts + 3 * (int64_t)f[0], A);
                apply_pose(Ph, verts + 3 * (int64_t)f[1], B);
                apply_pose(Ph, verts + 3 * (int64_t)f[2], C);
                for (int k = 0; k < 3; ++k) { e1[k] = B[k] - A[k]; e2[k] = C[k] - A[k]; }
                cross3(e1, e2, n);
                double nr = dot3(n, rj);
                cross3(qj, n, qxn);
                for (int k = 0; k < 3; ++k) {
                    gx[k] += g * n[k] / nr;
                    gx[3 + k] += g * qxn[k] / nr;
                }
            }
        ll[h] = L;
        if (dpose) for (int k = 0; k < 6; ++k) dpose[6 * h + k] = gx[k];
        if (dsigma) dsigma[h] = gs;
        if (dpout) dpout[h] = gp;
        free(depth); free(inv_p); free(tid);
    }
    return err;
}

/* ------------------------------------------------------------------------------------ */
/* Bound on the gradient change FP32 visibility decisions can cause (kind 1)              */
/* ------------------------------------------------------------------------------------ */
/*
 * The gradient of orc_score_grad holds visibility fixed, so a rendered pixel j whose
 * assignment FP32 may decide differently (flagged by orc_render with edge_tol_px and
 * z_tol_rel) can give the FP32 path another gradient. The alternatives of a flagged pixel
 * are the ones that set its flag:
 *   - a triangle other than the winner whose coverage is within edge_tol_px of its boundary
 *     and whose depth is not behind the winner's by more than z_tol_rel;
 *   - a covering triangle whose depth is within z_tol_rel of the winner's;
 *   - when the winner's own coverage is within edge_tol_px: the nearest other covering
 *     triangle, else the background (a miss);
 *   - when the winner's depth is ill-conditioned (flag bit 2): the same triangle with its
 *     depth moved either way by its FP32 resolution.
 * For each alternative the exact change of (dLL/dxi [6], dLL/ds, dLL/dp_out) when j alone
 * switches to it (all other pixels held) is formed from the definitions of orc_score_grad:
 * the observed pixels i in win(j) get S_i' = S_i - N(qt_i - q_j) + N(qt_i - q_j'); the
 * slot object's rendered pixels k within 2w of j get g_k through the changed 1/p_i; j
 * itself gets g_j' dz_j'/dxi (dz/dxi from the alternative's plane; 0 when it is not the
 * slot object's). gbound[h, 0..7] is the sum over flagged pixels of the largest absolute
 * change, component by component, over their alternatives: a first-order bound (single
 * switches added, their interaction neglected). n_flag[h] counts the flagged pixels.
 */
#define ORC_MAX_ALT 8

typedef struct {
    int32_t t;     /* global triangle id, -1 for the background */
    double z;      /* its depth at the pixel */
    double n[3];   /* its camera-frame plane normal (slot object only) */
} orc_alt;

static void tri_normal_cam(const orc_scene *sc, int32_t slot, const double *slot_pose, int32_t g, double n[3]) {
    int o = 0;
    while (o + 1 < sc->n_obj && g >= sc->f_off[o + 1]) ++o;
    const double *Po = object_pose(sc, o, slot, slot_pose);
    const double *verts = sc->verts + 3 * sc->v_off[o];
    const int32_t *f = sc->faces + 3 * (int64_t)g;
    double A[3], B[3], C[3], e1[3], e2[3];
    apply_pose(Po, verts + 3 * (int64_t)f[0], A);
    apply_pose(Po, verts + 3 * (int64_t)f[1], B);
    apply_pose(Po, verts + 3 * (int64_t)f[2], C);
    for (int k = 0; k < 3; ++k) { e1[k] = B[k] - A[k]; e2[k] = C[k] - A[k]; }
    cross3(e1, e2, n);
}

static void add_alt(orc_alt *list, uint8_t *cnt, int32_t t, double z, const double n[3], int same_t_ok) {
    if (!same_t_ok)
        for (int k = 0; k < *cnt; ++k)
            if (list[k].t == t) return;
    if (*cnt >= ORC_MAX_ALT) return;
    orc_alt *a = &list[(*cnt)++];
    a->t = t;
    a->z = z;
    for (int k = 0; k < 3; ++k) a->n[k] = n ? n[k] : 0.0;
}

int orc_score_grad_bound(const orc_camera *cam, const orc_scene *sc, int32_t slot, int64_t n_hyp,
                         const double *poses, const orc_lik *lk, const double *depth_obs, double edge_tol_px,
                         double z_tol_rel, double *gbound, int32_t *n_flag, int32_t n_threads) {
    if (!cam || !sc || !lk || lk->kind != 1 || !depth_obs || !gbound || (n_hyp > 0 && !poses)) return ORC_EINVAL;
    if (slot < 0 || slot >= sc->n_obj || !(lk->radius > 0) || lk->half_window < 0 || lk->half_window > 4)
        return ORC_EINVAL;
    const int W = cam->width, H = cam->height, w = lk->half_window;
    const int64_t P = (int64_t)W * H;
    double V, K;
    lik_constants(cam, lk, &V, &K);
    const double s = lk->radius, s2 = s * s;
    const double gnorm = pow(2.0 * ORC_PI * s2, -1.5);
    const double a = lk->p_outlier / V, b = (1.0 - lk->p_outlier) / K;
    const int64_t f0 = sc->f_off[slot], f1 = sc->f_off[slot + 1];
    const double tol = edge_tol_px;
    int err = ORC_OK;
#ifdef _OPENMP
    if (n_threads <= 0) n_threads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
    for (int64_t h = 0; h < n_hyp; ++h) {
        const double *Ph = poses + 16 * h;
        double *depth = malloc(sizeof(double) * P), *S = malloc(sizeof(double) * P);
        double *dS = malloc(sizeof(double) * P), *pp = malloc(sizeof(double) * P);
        double *wm = malloc(sizeof(double) * P), *sec_z = malloc(sizeof(double) * P);
        double *J = malloc(sizeof(double) * 6 * P), *zmv = malloc(sizeof(double) * P);
        int32_t *tid = malloc(sizeof(int32_t) * P), *sec_t = malloc(sizeof(int32_t) * P);
        uint8_t *fl = malloc(P), *nalt = malloc(P);
        orc_alt *alts = malloc(sizeof(orc_alt) * ORC_MAX_ALT * P);
        if (!depth || !S || !dS || !pp || !wm || !sec_z || !J || !zmv || !tid || !sec_t || !fl || !nalt || !alts) {
            err = ORC_ENOMEM;
            goto done;
        }
        render_core(cam, sc, slot, Ph, edge_tol_px, z_tol_rel, depth, tid, fl, zmv);
        for (int64_t i = 0; i < P; ++i) { nalt[i] = 0; wm[i] = INFINITY; sec_z[i] = INFINITY; sec_t[i] = -1; }
        /* alternatives of the flagged pixels: one pass over every triangle's pixel box */
        for (int o = 0; o < sc->n_obj; ++o) {
            const double *Po = object_pose(sc, o, slot, Ph);
            const double *verts = sc->verts + 3 * sc->v_off[o];
            for (int64_t f = sc->f_off[o]; f < sc->f_off[o + 1]; ++f) {
                tri_cam t;
                if (!setup_tri(cam, Po, verts, sc->faces + 3 * f, &t)) continue;
                double umin = fmin(t.su[0], fmin(t.su[1], t.su[2])), umax = fmax(t.su[0], fmax(t.su[1], t.su[2]));
                double vmin = fmin(t.sv[0], fmin(t.sv[1], t.sv[2])), vmax = fmax(t.sv[0], fmax(t.sv[1], t.sv[2]));
                int x0, x1, y0, y1;
                pixel_range(umin, umax, tol, W, &x0, &x1);
                pixel_range(vmin, vmax, tol, H, &y0, &y1);
                for (int y = y0; y <= y1; ++y)
                    for (int x = x0; x <= x1; ++x) {
                        const int64_t i = (int64_t)y * W + x;
                        if (!fl[i]) continue;
                        double r[3];
                        pixel_ray(cam, x, y, r);
                        const double m = coverage_margin(&t, x + 0.5, y + 0.5);
                        const double z = plane_depth(&t, r);
                        if (!(z <= cam->far_z)) continue;
                        const int32_t g = (int32_t)f;
                        if (g == tid[i]) { wm[i] = m; continue; }
                        const double zb = tid[i] >= 0 ? depth[i] : cam->far_z;
                        if ((fabs(m) < tol && z <= zb * (1.0 + z_tol_rel)) || (m >= 0 && z - zb <= z_tol_rel * zb))
                            add_alt(alts + ORC_MAX_ALT * i, nalt + i, g, z, t.n, 0);
                        if (m >= 0 && (z < sec_z[i] || (z == sec_z[i] && g < sec_t[i]))) { sec_z[i] = z; sec_t[i] = g; }
                    }
            }
        }
        for (int64_t i = 0; i < P; ++i) {
            if (fl[i] & 4) {
                /* an ill-conditioned depth: the same triangle, its depth moved either way by its
                 * resolution */
                double n[3];
                tri_normal_cam(sc, slot, Ph, tid[i], n);
                add_alt(alts + ORC_MAX_ALT * i, nalt + i, tid[i], depth[i] + zmv[i], n, 1);
                add_alt(alts + ORC_MAX_ALT * i, nalt + i, tid[i], depth[i] - zmv[i], n, 1);
            }
            if (!fl[i] || tid[i] < 0 || !(wm[i] < tol)) continue;
            if (sec_t[i] >= 0) {
                double n[3];
                tri_normal_cam(sc, slot, Ph, sec_t[i], n);
                add_alt(alts + ORC_MAX_ALT * i, nalt + i, sec_t[i], sec_z[i], n, 0);
            } else {
                add_alt(alts + ORC_MAX_ALT * i, nalt + i, -1, cam->far_z, NULL, 0);
            }
        }
        /* observed side: S_i, dS_i/ds, p_i; rendered side: dz_k/dxi of the slot's pixels */
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const int64_t i = (int64_t)y * W + x;
                pp[i] = 0;
                const double d_obs = depth_obs[i];
                if (!(d_obs > 0) || !isfinite(d_obs)) continue;
                double ri[3];
                pixel_ray(cam, x, y, ri);
                double Si = 0, dSi = 0;
                for (int dy = -w; dy <= w; ++dy)
                    for (int dx = -w; dx <= w; ++dx) {
                        int xj = x + dx, yj = y + dy;
                        if (xj < 0 || xj >= W || yj < 0 || yj >= H) continue;
                        const int64_t j = (int64_t)yj * W + xj;
                        if (lk->miss_mode == 1 && tid[j] < 0) continue;
                        double rj[3], d2 = 0;
                        pixel_ray(cam, xj, yj, rj);
                        for (int k = 0; k < 3; ++k) { double d = d_obs * ri[k] - depth[j] * rj[k]; d2 += d * d; }
                        const double N = gnorm * exp(-d2 / (2.0 * s2));
                        Si += N;
                        dSi += N * (d2 / (s2 * s) - 3.0 / s);
                    }
                S[i] = Si; dS[i] = dSi; pp[i] = a + b * Si;
            }
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const int64_t k = (int64_t)y * W + x;
                for (int c = 0; c < 6; ++c) J[6 * k + c] = 0;
                if (tid[k] < f0 || tid[k] >= f1) continue;
                double n[3], r[3], q[3], qxn[3];
                tri_normal_cam(sc, slot, Ph, tid[k], n);
                pixel_ray(cam, x, y, r);
                for (int c = 0; c < 3; ++c) q[c] = depth[k] * r[c];
                cross3(q, n, qxn);
                const double nr = dot3(n, r);
                for (int c = 0; c < 3; ++c) { J[6 * k + c] = n[c] / nr; J[6 * k + 3 + c] = qxn[c] / nr; }
            }
        double gb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        int32_t nf = 0;
        double Sn[81], dSn[81], pn[81];  /* the window of j: (2w+1)^2 <= 81 for w <= 4 */
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                const int64_t j = (int64_t)y * W + x;
                if (!nalt[j]) continue;
                ++nf;
                double rj[3];
                pixel_ray(cam, x, y, rj);
                const int old_pt = !(lk->miss_mode == 1 && tid[j] < 0);
                const double z_old = depth[j];
                double worst[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                for (int q = 0; q < nalt[j]; ++q) {
                    const orc_alt *A = alts + ORC_MAX_ALT * j + q;
                    const int new_pt = !(lk->miss_mode == 1 && A->t < 0);
                    const double z_new = A->t >= 0 ? A->z : cam->far_z;
                    double dlt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                    /* observed pixels i in win(j): new S_i, dS_i, p_i; sigma and p_out terms */
                    for (int dy = -w; dy <= w; ++dy)
                        for (int dx = -w; dx <= w; ++dx) {
                            const int ii = (dy + w) * (2 * w + 1) + (dx + w);
                            int xi = x + dx, yi = y + dy;
                            pn[ii] = 0;
                            if (xi < 0 || xi >= W || yi < 0 || yi >= H) continue;
                            const int64_t i = (int64_t)yi * W + xi;
                            if (pp[i] == 0) continue;
                            double ri[3], d2o = 0, d2n = 0;
                            pixel_ray(cam, xi, yi, ri);
                            for (int c = 0; c < 3; ++c) {
                                double qt = depth_obs[i] * ri[c];
                                d2o += (qt - z_old * rj[c]) * (qt - z_old * rj[c]);
                                d2n += (qt - z_new * rj[c]) * (qt - z_new * rj[c]);
                            }
                            const double No = old_pt ? gnorm * exp(-d2o / (2.0 * s2)) : 0.0;
                            const double Nn = new_pt ? gnorm * exp(-d2n / (2.0 * s2)) : 0.0;
                            Sn[ii] = S[i] - No + Nn;
                            dSn[ii] = dS[i] - (old_pt ? No * (d2o / (s2 * s) - 3.0 / s) : 0.0) +
                                      (new_pt ? Nn * (d2n / (s2 * s) - 3.0 / s) : 0.0);
                            pn[ii] = a + b * Sn[ii];
                            dlt[6] += b * dSn[ii] / pn[ii] - b * dS[i] / pp[i];
                            dlt[7] += (1.0 / V - Sn[ii] / K) / pn[ii] - (1.0 / V - S[i] / K) / pp[i];
                        }
                    /* the slot's rendered pixels k within 2w of j: g_k through the changed p_i */
                    for (int ky = y - 2 * w; ky <= y + 2 * w; ++ky)
                        for (int kx = x - 2 * w; kx <= x + 2 * w; ++kx) {
                            if (kx < 0 || kx >= W || ky < 0 || ky >= H) continue;
                            const int64_t k = (int64_t)ky * W + kx;
                            const int is_j = k == j;
                            const int slot_old = tid[k] >= f0 && tid[k] < f1;
                            const int slot_new = is_j ? (A->t >= f0 && A->t < f1) : slot_old;
                            if (!slot_old && !slot_new) continue;
                            double rk[3];
                            pixel_ray(cam, kx, ky, rk);
                            double g_old = 0, g_new = 0;
                            for (int dy = -w; dy <= w; ++dy)
                                for (int dx = -w; dx <= w; ++dx) {
                                    int xi = kx + dx, yi = ky + dy;
                                    if (xi < 0 || xi >= W || yi < 0 || yi >= H) continue;
                                    const int64_t i = (int64_t)yi * W + xi;
                                    if (pp[i] == 0) continue;
                                    const int in_j = abs(xi - x) <= w && abs(yi - y) <= w;
                                    const double p_new = in_j ? pn[(yi - y + w) * (2 * w + 1) + (xi - x + w)] : pp[i];
                                    double ri[3];
                                    pixel_ray(cam, xi, yi, ri);
                                    for (int v = 0; v < 2; ++v) {
                                        if (v == 0 && !slot_old) continue;
                                        if (v == 1 && !slot_new) continue;
                                        const double zk = (is_j && v == 1) ? z_new : depth[k];
                                        double diff[3], d2 = 0;
                                        for (int c = 0; c < 3; ++c) {
                                            diff[c] = depth_obs[i] * ri[c] - zk * rk[c];
                                            d2 += diff[c] * diff[c];
                                        }
                                        const double t = gnorm * exp(-d2 / (2.0 * s2)) * dot3(diff, rk) / s2;
                                        if (v == 0) g_old += b * t / pp[i];
                                        else g_new += b * t / p_new;
                                    }
                                }
                            double Jn[6];
                            if (is_j && slot_new) {
                                double qn[3], qxn[3];
                                for (int c = 0; c < 3; ++c) qn[c] = z_new * rk[c];
                                cross3(qn, A->n, qxn);
                                const double nr = dot3(A->n, rk);
                                for (int c = 0; c < 3; ++c) { Jn[c] = A->n[c] / nr; Jn[3 + c] = qxn[c] / nr; }
                            } else {
                                for (int c = 0; c < 6; ++c) Jn[c] = J[6 * k + c];
                            }
                            for (int c = 0; c < 6; ++c)
                                dlt[c] += (slot_new ? g_new * Jn[c] : 0.0) - (slot_old ? g_old * J[6 * k + c] : 0.0);
                        }
                    for (int c = 0; c < 8; ++c) worst[c] = fmax(worst[c], fabs(dlt[c]));
                }
                for (int c = 0; c < 8; ++c) gb[c] += worst[c];
            }
        for (int c = 0; c < 8; ++c) gbound[8 * h + c] = gb[c];
        if (n_flag) n_flag[h] = nf;
    done:
        free(depth); free(S); free(dS); free(pp); free(wm); free(sec_z); free(J); free(zmv);
        free(tid); free(sec_t); free(fl); free(nalt); free(alts);
    }
    return err;
}

int orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
