// k_render.cu - rasterisation and windowed-likelihood kernels of libb3d.
//
// The render kernel draws one pose hypothesis per CTA iteration into a shared-memory
// z-buffer of packed (depth bits << 32 | triangle id) keys (64-bit atomicMin: the nearest
// fragment wins, equal depths go to the smaller id) and composites it with the fixed
// objects' background keys. The score kernel does the same with depth bits alone, then
// scores every observed pixel whose (2w+1)^2 window can see the object (the windowed Eq. 1
// likelihood of Sec. III-B). Pixels whose window cannot see the object keep their
// background term, precomputed once per scene, so a hypothesis costs work in proportion to
// its screen footprint:
//   LL_h = sum_i l_i(h) = LL_bg + sum_{i in footprint + w} (l_i(h) - l_i(bg)),
// an exact identity (the terms outside the dilated footprint are equal, bit for bit, since
// they are computed by the same device function from the same inputs).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "b3d_device.cuh"
#include "b3d_internal.h"

namespace b3d {

// ------------------------------------------------------------------------------------------
// score kernel
// ------------------------------------------------------------------------------------------
// One hypothesis per CTA iteration of a persistent grid:
//  1. pose; screen bounding box of the object; whether the near plane can cut it. For a
//     quad (voxel) mesh wholly beyond the near plane: the camera position o in the object
//     frame and, per face class (axis, outward sign), the contiguous range of quads whose
//     plane has o on its outer side (the faces turned towards the camera); the rest are
//     never loaded.
//  2. quad meshes: the camera-frame position of every lattice plane along each axis (the
//     rotation column times the plane coordinate, plus t on the x axis), so a corner is the
//     sum of three shared terms and every quad sharing a corner gets the same bits.
//  3. per screen tile: clear a 32-bit z-buffer of depth bits, rasterise with atomicMin (the
//     score depends only on the nearest depth, so no triangle id rides along), composite
//     with the fixed objects' depths, score the tile's observed pixels against their
//     background terms.
//  4. block reduction to one log-likelihood.
// STATS: count the work done (hypotheses, projected vertices/corners, primitives, pixel
// tests, fragments, composited pixels, scored pixels, window pairs) into S.stats.
// WT: the half window compiled in (1 or 2: sliding-window scoring), 0: runtime L.w.

// Screen corner of a camera-frame point; approximate reciprocal (the same bits for the same
// point in every quad that shares it).
__device__ __forceinline__ float4 screen_pt(float x, float y, float z, const Cam &c) {
    const float iz = __fdividef(1.0f, z);
    return make_float4(fmaf(c.fx, x * iz, c.cx), fmaf(c.fy, y * iz, c.cy), iz, z);
}

__device__ __forceinline__ float4 sum3(const float4 &X, const float4 &Y, const float4 &Z) {
    return make_float4((X.x + Y.x) + Z.x, (X.y + Y.y) + Z.y, (X.z + Y.z) + Z.z, 0.f);
}

// Quad raster with per-pixel coverage and depth (see raster_quad); the pixel loop is
// flattened (no division) and the plane uses one approximate reciprocal.
template <class Store>
__device__ __forceinline__ void raster_quad_fast(float4 C0, float4 C1, float4 C2, float4 C3, int rx0, int rx1, int ry0,
                                                 int ry1, float far_z, Store store, unsigned long long *tests) {
    const float area = edge_fn(C0.x, C0.y, C1.x, C1.y, C2.x, C2.y);
    if (!(area != 0.f)) return;
    const float umin = fminf(fminf(C0.x, C1.x), fminf(C2.x, C3.x)), umax = fmaxf(fmaxf(C0.x, C1.x), fmaxf(C2.x, C3.x));
    const float vmin = fminf(fminf(C0.y, C1.y), fminf(C2.y, C3.y)), vmax = fmaxf(fmaxf(C0.y, C1.y), fmaxf(C2.y, C3.y));
    const int x0 = (int)ceilf(fmaxf(umin - 0.5f, (float)rx0)), x1 = (int)floorf(fminf(umax - 0.5f, (float)rx1));
    const int y0 = (int)ceilf(fmaxf(vmin - 0.5f, (float)ry0)), y1 = (int)floorf(fminf(vmax - 0.5f, (float)ry1));
    if (x0 > x1 || y0 > y1) return;
    const int cnt = (x1 - x0 + 1) * (y1 - y0 + 1);
    if (tests) *tests += (unsigned long long)cnt;
    const float s = area > 0.f ? 1.f : -1.f;
    const float inv = __fdividef(1.0f, area);
    const float du1 = C1.x - C0.x, dv1 = C1.y - C0.y, du2 = C2.x - C0.x, dv2 = C2.y - C0.y;
    const float dz1 = C1.z - C0.z, dz2 = C2.z - C0.z;
    const float al = fmaf(dz1, dv2, -(dz2 * dv1)) * inv, be = fmaf(dz2, du1, -(dz1 * du2)) * inv;
    int x = x0, y = y0;
    for (int k = 0; k < cnt; ++k) {
        const float px = (float)x + 0.5f, py = (float)y + 0.5f;
        const bool in = s * edge_fn(C0.x, C0.y, C1.x, C1.y, px, py) >= 0.f && s * edge_fn(C1.x, C1.y, C2.x, C2.y, px, py) >= 0.f &&
                        s * edge_fn(C2.x, C2.y, C3.x, C3.y, px, py) >= 0.f && s * edge_fn(C3.x, C3.y, C0.x, C0.y, px, py) >= 0.f;
        if (in) {
            const float z = __fdividef(1.0f, fmaf(al, px - C0.x, fmaf(be, py - C0.y, C0.z)));
            if (z <= far_z) store(x, y, z);
        }
        if (++x > x1) { x = x0; ++y; }
    }
}

// Sum of l_i - l_i(bg) over pixel column x, rows [ya, yb], with the (2W+1)^2 window of
// rendered depths slid down the column in registers. Window slots outside the image (and
// pixels without a point) hold -1 and contribute nothing; the terms are formed in the same
// order and by the same expressions as pixel_ell, so unchanged pixels give 0 exactly.
template <int W>
__device__ __forceinline__ float score_column(const SceneView &S, const Lik &L, const float *lut, const Cam &c,
                                              const float *zd, int zx0, int zy0, int zw, int x, int ya, int yb,
                                              unsigned long long *n_px, unsigned long long *n_pairs) {
    constexpr int D = 2 * W + 1;
    float rx[D], ry[D], win[D][D];
    bool colok[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const int xj = x + d - W;
        colok[d] = xj >= 0 && xj < c.W;
        rx[d] = ((float)xj + 0.5f - c.cx) * c.inv_fx;
    }
    auto load_row = [&](int yj, float *row) {
        const bool rowok = yj >= 0 && yj < c.H;
#pragma unroll
        for (int d = 0; d < D; ++d) row[d] = (rowok && colok[d]) ? zd[(yj - zy0) * zw + (x + d - W - zx0)] : -1.f;
    };
#pragma unroll
    for (int r = 1; r < D; ++r) {
        load_row(ya - W + r - 1, win[r]);
        ry[r] = ((float)(ya - W + r - 1) + 0.5f - c.cy) * c.inv_fy;
    }
    float acc = 0.f;
    for (int y = ya; y <= yb; ++y) {
#pragma unroll
        for (int r = 0; r + 1 < D; ++r) {
            ry[r] = ry[r + 1];
#pragma unroll
            for (int d = 0; d < D; ++d) win[r][d] = win[r + 1][d];
        }
        load_row(y + W, win[D - 1]);
        ry[D - 1] = ((float)(y + W) + 0.5f - c.cy) * c.inv_fy;
        const int64_t gi = (int64_t)y * c.W + x;
        const float4 q = S.obs[gi];
        if (q.w == 0.f) continue;
        int n = 0;
        float Ssum = 0.f;
#pragma unroll
        for (int r = 0; r < D; ++r) {
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const float z = win[r][d];
                const float ex = fmaf(-z, rx[d], q.x), ey = fmaf(-z, ry[r], q.y), ez = q.z - z;
                const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                if (L.kind == 0) n += (z >= 0.f && d2 <= L.r2) ? 1 : 0;
                else if (z >= 0.f) Ssum += __expf(-d2 * L.inv2s2);
            }
        }
        const float l = L.kind == 0 ? lut[n] : __logf(fmaf(L.bg, Ssum, L.a));
        acc += l - S.ell_bg[gi];
        if (n_px) {
            ++*n_px;
            *n_pairs += (unsigned long long)((min(y + W, c.H - 1) - max(y - W, 0) + 1) *
                                             (min(x + W, c.W - 1) - max(x - W, 0) + 1));
        }
    }
    return acc;
}

template <class PS, bool STATS, int WT, int NT>
__global__ void __launch_bounds__(NT, NT <= 128 ? 2 * kScoreMinBlocks : kScoreMinBlocks)
    k_score(SceneView S, Lik L, PS P, int64_t n_hyp, float *out_ll) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned *zb = reinterpret_cast<unsigned *>(smem_raw);                       // [kRegionPx]
    float *zd = reinterpret_cast<float *>(smem_raw);                             // same memory, as depths
    float4 *lat = reinterpret_cast<float4 *>(smem_raw + kRegionPx * sizeof(unsigned));  // lattice planes
    __shared__ float s_lut[kMaxLut];
    __shared__ float s_pose[12];
    __shared__ int s_bb[4];
    __shared__ int s_flags;  // bit 0: on screen, bit 1: quad path, bit 2: whole object beyond near
    __shared__ int s_rng[13];  // class first quads [6], exclusive prefix of counts [6], total
    __shared__ float s_red[NT / 32];

    const Cam &c = S.cam;
    const MeshView &m = S.mesh;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < L.n_lut; i += nt) s_lut[i] = L.lut[i];
    const int w = WT > 0 ? WT : L.w;
    const int n_lat = m.nc[0] + m.nc[1] + m.nc[2];
    const int nc0 = m.nc[0], nc01 = m.nc[0] + m.nc[1];
    auto lat_off = [&](int a) { return a == 0 ? 0 : (a == 1 ? nc0 : nc01); };
    unsigned long long cnt[kNumStats] = {0, 0, 0, 0, 0, 0, 0, 0};

    for (int64_t h = blockIdx.x; h < n_hyp; h += gridDim.x) {
        __syncthreads();
        if (tid == 0) {
            if (STATS) ++cnt[0];
            pose12(P, h, s_pose);
            bool front = false;
            int f = object_bbox(m, s_pose, c, s_bb, &front) ? 1 : 0;
            if (front) f |= 4;
            if (f && front && m.n_quads > 0) {
                f |= 2;
                const float *R = s_pose, *t = s_pose + 9;
                float o[3];
                for (int a = 0; a < 3; ++a) o[a] = -fmaf(R[a], t[0], fmaf(R[3 + a], t[1], R[6 + a] * t[2]));
                int tot = 0;
                for (int cls = 0; cls < 6; ++cls) {
                    const int a = cls >> 1;
                    const float *cd = m.coords + lat_off(a);
                    const int n = m.nc[a];
                    int lo = 0, hi = n;  // first plane with coordinate >= o
                    while (lo < hi) { const int mid = (lo + hi) >> 1; if (cd[mid] < o[a]) lo = mid + 1; else hi = mid; }
                    const int below = lo;
                    hi = n;  // first plane with coordinate > o
                    while (lo < hi) { const int mid = (lo + hi) >> 1; if (cd[mid] <= o[a]) lo = mid + 1; else hi = mid; }
                    const int not_above = lo;
                    const int *off = m.class_off + cls * m.np1;
                    // +axis faces face the camera when their plane is below o; -axis when above
                    const int b = (cls & 1) ? off[0] : off[not_above];
                    const int e = (cls & 1) ? off[below] : off[n];
                    s_rng[cls] = b;
                    s_rng[6 + cls] = tot;
                    tot += e - b;
                }
                s_rng[12] = tot;
            }
            s_flags = f;
        }
        __syncthreads();
        const int flags = s_flags;
        if (!(flags & 1)) {
            if (tid == 0) out_ll[h] = (float)*S.ll_bg;
            continue;
        }
        const float *pose = s_pose;
        const bool quad = (flags & 2) != 0, front = (flags & 4) != 0;
        const int bx0 = s_bb[0], bx1 = s_bb[1], by0 = s_bb[2], by1 = s_bb[3];
        if (quad) {
            for (int k = tid; k < n_lat; k += nt) {
                const int a = k < nc0 ? 0 : (k < nc01 ? 1 : 2);
                const float v = m.coords[k];
                lat[k] = make_float4(fmaf(pose[a], v, a == 0 ? pose[9] : 0.f), fmaf(pose[3 + a], v, a == 0 ? pose[10] : 0.f),
                                     fmaf(pose[6 + a], v, a == 0 ? pose[11] : 0.f), 0.f);
            }
            if (STATS) cnt[1] += (unsigned long long)((n_lat - tid + nt - 1) / nt);
        }
        const int sx0 = max(bx0 - w, 0), sx1 = min(bx1 + w, c.W - 1);
        const int sy0 = max(by0 - w, 0), sy1 = min(by1 + w, c.H - 1);
        const int sw = sx1 - sx0 + 1;
        const int tw = min(sw, S.tile_w);
        const int th = max(1, kRegionPx / (tw + 2 * w) - 2 * w);
        float acc = 0.f;
        for (int ty0 = sy0; ty0 <= sy1; ty0 += th) {
            for (int tx0 = sx0; tx0 <= sx1; tx0 += tw) {
                const int tx1 = min(tx0 + tw - 1, sx1), ty1 = min(ty0 + th - 1, sy1);
                const int zx0 = max(tx0 - w, 0), zx1 = min(tx1 + w, c.W - 1);
                const int zy0 = max(ty0 - w, 0), zy1 = min(ty1 + w, c.H - 1);
                const int zw = zx1 - zx0 + 1, zh = zy1 - zy0 + 1, nz = zw * zh;
                const int rx0 = max(zx0, bx0), rx1 = min(zx1, bx1), ry0 = max(zy0, by0), ry1 = min(zy1, by1);
                const bool need = rx0 <= rx1 && ry0 <= ry1;
                for (int i = tid; i < nz; i += nt) zb[i] = 0xffffffffu;
                __syncthreads();
                if (need) {
                    auto store = [&](int x, int y, float z) {
                        if (STATS) ++cnt[4];
                        atomicMin(&zb[(y - zy0) * zw + (x - zx0)], __float_as_uint(z));
                    };
                    if (quad) {
                        const int total = s_rng[12];
                        for (int k = tid; k < total; k += nt) {
                            int cls = 0;
#pragma unroll
                            for (int j = 1; j < 6; ++j) cls += k >= s_rng[6 + j] ? 1 : 0;
                            const unsigned q = m.quads[s_rng[cls] + (k - s_rng[6 + cls])];
                            const int a = cls >> 1, p = (q >> 18) & 511, b0 = (q >> 9) & 511, c0 = q & 511;
                            const int ab = a == 2 ? 0 : a + 1, ac = a == 0 ? 2 : a - 1;
                            // the plane term is shared by all corners, the in-plane terms take two
                            // values each; corners are summed in x, y, z order
                            const float4 Tp = lat[lat_off(a) + p];
                            const float4 Tb0 = lat[lat_off(ab) + b0], Tb1 = lat[lat_off(ab) + b0 + 1];
                            const float4 Tc0 = lat[lat_off(ac) + c0], Tc1 = lat[lat_off(ac) + c0 + 1];
                            float4 W0, W1, W2, W3;  // camera-frame corners k0 (b0,c0) k1 (b1,c0) k2 (b1,c1) k3 (b0,c1)
                            if (a == 0) {
                                W0 = sum3(Tp, Tb0, Tc0); W1 = sum3(Tp, Tb1, Tc0); W2 = sum3(Tp, Tb1, Tc1); W3 = sum3(Tp, Tb0, Tc1);
                            } else if (a == 1) {
                                W0 = sum3(Tc0, Tp, Tb0); W1 = sum3(Tc0, Tp, Tb1); W2 = sum3(Tc1, Tp, Tb1); W3 = sum3(Tc1, Tp, Tb0);
                            } else {
                                W0 = sum3(Tb0, Tc0, Tp); W1 = sum3(Tb1, Tc0, Tp); W2 = sum3(Tb1, Tc1, Tp); W3 = sum3(Tb0, Tc1, Tp);
                            }
                            if (STATS) { cnt[1] += 4; ++cnt[2]; }
                            raster_quad_fast(screen_pt(W0.x, W0.y, W0.z, c), screen_pt(W1.x, W1.y, W1.z, c),
                                             screen_pt(W2.x, W2.y, W2.z, c), screen_pt(W3.x, W3.y, W3.z, c), rx0, rx1, ry0,
                                             ry1, c.far_z, store, STATS ? &cnt[3] : nullptr);
                        }
                    } else {
                        const int4 *tris = front ? m.tris_surf : m.tris_full;
                        const int n_t = front ? m.n_surf : m.n_full;
                        const int cull = front ? m.closed : 0;
                        for (int t = tid; t < n_t; t += nt) {
                            float4 A, B, C;
                            tri_screen(m, tris[t], pose, c, A, B, C);
                            if (STATS) { cnt[1] += 3; ++cnt[2]; }
                            raster_tri(A, B, C, cull, rx0, rx1, ry0, ry1, c.far_z, store, STATS ? &cnt[3] : nullptr);
                        }
                    }
                }
                __syncthreads();
                // composite with the fixed objects in place: depth bits -> rendered depth
                {
                    const int dq = nt / zw, dr = nt - dq * zw;
                    int y = tid / zw, x = tid - y * zw;
                    for (int i = tid; i < nz; i += nt) {
                        const unsigned bgb = (unsigned)(S.bg[(int64_t)(zy0 + y) * c.W + zx0 + x] >> 32);
                        const unsigned v = min(zb[i], bgb);
                        zd[i] = v == 0xffffffffu ? (L.miss_mode ? -1.f : c.far_z) : __uint_as_float(v);
                        x += dr;
                        y += dq;
                        if (x >= zw) { x -= zw; ++y; }
                    }
                }
                if (STATS) cnt[5] += (unsigned long long)((nz - tid + nt - 1) / nt);
                __syncthreads();
                const int tww = tx1 - tx0 + 1, thh = ty1 - ty0 + 1;
                if (WT > 0) {
                    // thread -> (column, run of rows)
                    const int nseg = max(1, nt / tww);
                    const int rps = (thh + nseg - 1) / nseg;
                    const int seg = tid / tww, col = tid - seg * tww;
                    if (seg < nseg) {
                        const int ya = ty0 + seg * rps, yb = min(ya + rps - 1, ty1);
                        if (ya <= yb)
                            acc += score_column<WT>(S, L, s_lut, c, zd, zx0, zy0, zw, tx0 + col, ya, yb,
                                                    STATS ? &cnt[6] : nullptr, STATS ? &cnt[7] : nullptr);
                    }
                } else {
                    const int n_tile = tww * thh;
                    const int dq = nt / tww, dr = nt - dq * tww;
                    int y = tid / tww, x = tid - y * tww;
                    for (int k = tid; k < n_tile; k += nt) {
                        const int gx = tx0 + x, gy = ty0 + y;
                        const int64_t gi = (int64_t)gy * c.W + gx;
                        const float4 q = S.obs[gi];
                        if (q.w != 0.f) {
                            if (STATS) {
                                ++cnt[6];
                                cnt[7] += (unsigned long long)((min(gy + w, c.H - 1) - max(gy - w, 0) + 1) *
                                                               (min(gx + w, c.W - 1) - max(gx - w, 0) + 1));
                            }
                            const float l = pixel_ell(L, s_lut, c, q, gx, gy,
                                                      [&](int xj, int yj) { return zd[(yj - zy0) * zw + (xj - zx0)]; });
                            acc += l - S.ell_bg[gi];
                        }
                        x += dr;
                        y += dq;
                        if (x >= tww) { x -= tww; ++y; }
                    }
                }
                __syncthreads();
            }
        }
        const float tot = block_sum(acc, s_red);
        if (tid == 0) out_ll[h] = (float)(*S.ll_bg + (double)tot);
    }
    if (STATS)
        for (int k = 0; k < kNumStats; ++k)
            if (cnt[k]) atomicAdd(&S.stats[k], cnt[k]);
}

// ------------------------------------------------------------------------------------------
// render kernel: depth and triangle id of every pixel (64-bit keys)
// ------------------------------------------------------------------------------------------
template <class PS>
__global__ void __launch_bounds__(kThreads) k_render(SceneView S, PS P, int64_t n_hyp, float *out_depth, int *out_tid) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long *zb = reinterpret_cast<unsigned long long *>(smem_raw);  // [kRegionPx]
    __shared__ float s_pose[12];
    __shared__ int s_bb[4];
    __shared__ int s_flags;
    const Cam &c = S.cam;
    const MeshView &m = S.mesh;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t npx = (int64_t)c.W * c.H;
    for (int64_t h = blockIdx.x; h < n_hyp; h += gridDim.x) {
        __syncthreads();
        if (tid == 0) {
            pose12(P, h, s_pose);
            bool front = false;
            s_flags = (object_bbox(m, s_pose, c, s_bb, &front) ? 1 : 0) | (front ? 4 : 0);
        }
        __syncthreads();
        const float *pose = s_pose;
        const bool has_bb = (s_flags & 1) != 0, front = (s_flags & 4) != 0;
        const int bx0 = s_bb[0], bx1 = s_bb[1], by0 = s_bb[2], by1 = s_bb[3];
        const int4 *tris = front ? m.tris_surf : m.tris_full;
        const int n_t = front ? m.n_surf : m.n_full;
        const int cull = front ? m.closed : 0;
        const int tw = min(c.W, kRegionPx);
        const int th = max(1, kRegionPx / tw);
        for (int ty0 = 0; ty0 < c.H; ty0 += th) {
            for (int tx0 = 0; tx0 < c.W; tx0 += tw) {
                const int tx1 = min(tx0 + tw - 1, c.W - 1), ty1 = min(ty0 + th - 1, c.H - 1);
                const int zw = tx1 - tx0 + 1, zh = ty1 - ty0 + 1;
                const int rx0 = max(tx0, bx0), rx1 = min(tx1, bx1), ry0 = max(ty0, by0), ry1 = min(ty1, by1);
                const bool need = has_bb && rx0 <= rx1 && ry0 <= ry1;
                if (need) {
                    for (int i = tid; i < zw * zh; i += nt) zb[i] = kEmptyKey;
                    __syncthreads();
                    for (int t = tid; t < n_t; t += nt) {
                        const int4 tr = tris[t];
                        float4 A, B, C;
                        tri_screen(m, tr, pose, c, A, B, C);
                        const unsigned gid = (unsigned)(S.tri_base + tr.w);
                        raster_tri(A, B, C, cull, rx0, rx1, ry0, ry1, c.far_z, [&](int x, int y, float z) {
                            atomicMin(&zb[(y - ty0) * zw + (x - tx0)], pack_key(z, gid));
                        });
                    }
                    __syncthreads();
                }
                for (int i = tid; i < zw * zh; i += nt) {
                    const int gx = tx0 + i % zw, gy = ty0 + i / zw;
                    const int64_t gi = (int64_t)gy * c.W + gx;
                    unsigned long long key = S.bg[gi];
                    if (need) key = min(key, zb[i]);
                    out_depth[h * npx + gi] = key_depth(key, 0, c.far_z);
                    if (out_tid) out_tid[h * npx + gi] = key == kEmptyKey ? -1 : (int)(unsigned)(key & 0xffffffffu);
                }
                __syncthreads();
            }
        }
    }
}

// ------------------------------------------------------------------------------------------
// scene set-up kernels
// ------------------------------------------------------------------------------------------

__global__ void k_obs_points(Cam c, const float *depth, float4 *obs) {
    const int64_t n = (int64_t)c.W * c.H;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = depth[i];
        const int x = (int)(i % c.W), y = (int)(i / c.W);
        if (d > 0.f && isfinite(d)) {
            const float rx = ((float)x + 0.5f - c.cx) * c.inv_fx, ry = ((float)y + 0.5f - c.cy) * c.inv_fy;
            obs[i] = make_float4(d * rx, d * ry, d, 1.f);
        } else {
            obs[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    }
}

__global__ void k_fill_u64(unsigned long long *p, int64_t n, unsigned long long v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

// Background render of one fixed object: one warp per triangle, lanes split its pixels.
// Closed meshes skip their back and internal faces unless the near plane cuts them.
__global__ void k_bg_raster(Cam c, MeshView m, const float *pose16, int tri_base, unsigned long long *bg) {
    __shared__ int s_front;
    float P[12];
    const float *p = pose16;
    P[0] = p[0]; P[1] = p[1]; P[2] = p[2]; P[3] = p[4]; P[4] = p[5]; P[5] = p[6];
    P[6] = p[8]; P[7] = p[9]; P[8] = p[10]; P[9] = p[3]; P[10] = p[7]; P[11] = p[11];
    if (threadIdx.x == 0) {
        int bb[4];
        bool front = false;
        object_bbox(m, P, c, bb, &front);
        s_front = front ? 1 : 0;
    }
    __syncthreads();
    const bool front = s_front != 0;
    const int4 *tris = front ? m.tris_surf : m.tris_full;
    const int n_t = front ? m.n_surf : m.n_full;
    const int cull = front ? m.closed : 0;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t t = warp; t < n_t; t += n_warps) {
        const int4 tr = tris[t];
        float4 A, B, C;
        tri_screen(m, tr, P, c, A, B, C);
        if (A.z < 0.f || B.z < 0.f || C.z < 0.f) continue;
        const float umin = fminf(A.x, fminf(B.x, C.x)), umax = fmaxf(A.x, fmaxf(B.x, C.x));
        const float vmin = fminf(A.y, fminf(B.y, C.y)), vmax = fmaxf(A.y, fmaxf(B.y, C.y));
        const int x0 = (int)ceilf(fmaxf(umin - 0.5f, 0.f)), x1 = (int)floorf(fminf(umax - 0.5f, (float)(c.W - 1)));
        const int y0 = (int)ceilf(fmaxf(vmin - 0.5f, 0.f)), y1 = (int)floorf(fminf(vmax - 0.5f, (float)(c.H - 1)));
        if (x0 > x1 || y0 > y1) continue;
        const int bw = x1 - x0 + 1;
        const int64_t nb = (int64_t)bw * (y1 - y0 + 1);
        const unsigned gid = (unsigned)(tri_base + tr.w);
        for (int64_t k = lane; k < nb; k += 32) {
            const int x = x0 + (int)(k % bw), y = y0 + (int)(k / bw);
            raster_tri(A, B, C, cull, x, x, y, y, c.far_z,
                       [&](int xx, int yy, float z) { atomicMin(&bg[(int64_t)yy * c.W + xx], pack_key(z, gid)); });
        }
    }
}

// Per-pixel background terms: l_i of the fixed objects alone and, when requested, the
// sigma / p_out derivatives of l_i (kind 1).
__global__ void k_bg_tables(SceneView S, Lik L, float *ell_bg, float *gs_bg, float *gp_bg) {
    __shared__ float s_lut[kMaxLut];
    for (int i = threadIdx.x; i < L.n_lut; i += blockDim.x) s_lut[i] = L.lut[i];
    __syncthreads();
    const Cam &c = S.cam;
    const int64_t n = (int64_t)c.W * c.H;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 q = S.obs[i];
        const int x = (int)(i % c.W), y = (int)(i / c.W);
        float l = 0.f, gs = 0.f, gp = 0.f;
        if (q.w != 0.f) {
            auto fetch = [&](int xj, int yj) { return key_depth(S.bg[(int64_t)yj * c.W + xj], L.miss_mode, c.far_z); };
            l = pixel_ell(L, s_lut, c, q, x, y, fetch);
            if (gs_bg) {
                float Si, dSi, bp;
                pixel_terms(L, c, q, x, y, fetch, Si, dSi);
                pixel_noise_grads(L, Si, dSi, gs, gp, bp);
            }
        }
        ell_bg[i] = l;
        if (gs_bg) { gs_bg[i] = gs; gp_bg[i] = gp; }
    }
}

// Sums of up to three arrays in double precision, fixed order (one block).
__global__ void k_sums(const float *a, const float *b, const float *c, int64_t n, double *out) {
    __shared__ double red[3][1024 / 32];
    double s[3] = {0, 0, 0};
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        s[0] += a[i];
        if (b) s[1] += b[i];
        if (c) s[2] += c[i];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < 3; ++k) {
        double v = s[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = 0;
        for (int k = 0; k < nw; ++k) v += red[threadIdx.x][k];
        out[threadIdx.x] = v;
    }
}

// ------------------------------------------------------------------------------------------
// two-pass scoring of materialised depth images [n, H, W]
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_score_depth(SceneView S, Lik L, const float *depth, const int *tid_in,
                                                          int64_t n_hyp, float *out_ll) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *zd = reinterpret_cast<float *>(smem_raw);
    __shared__ float s_lut[kMaxLut];
    __shared__ float s_red[kThreads / 32];
    const Cam &c = S.cam;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < L.n_lut; i += nt) s_lut[i] = L.lut[i];
    const int w = L.w;
    const int64_t npx = (int64_t)c.W * c.H;
    const int rows = max(1, (2 * kRegionPx) / c.W - 2 * w);  // 32 KB of float depths per tile
    for (int64_t h = blockIdx.x; h < n_hyp; h += gridDim.x) {
        const float *img = depth + h * npx;
        const int *tim = tid_in ? tid_in + h * npx : nullptr;
        float acc = 0.f;
        for (int ty0 = 0; ty0 < c.H; ty0 += rows) {
            const int ty1 = min(ty0 + rows - 1, c.H - 1);
            const int zy0 = max(ty0 - w, 0), zy1 = min(ty1 + w, c.H - 1);
            const int nz = (zy1 - zy0 + 1) * c.W;
            __syncthreads();
            for (int i = tid; i < nz; i += nt) {
                const int64_t gi = (int64_t)zy0 * c.W + i;
                float d = img[gi];
                if (L.miss_mode == 1 && tim[gi] < 0) d = -1.f;
                zd[i] = d;
            }
            __syncthreads();
            const int n_t = (ty1 - ty0 + 1) * c.W;
            for (int k = tid; k < n_t; k += nt) {
                const int x = k % c.W, y = ty0 + k / c.W;
                const float4 q = S.obs[(int64_t)y * c.W + x];
                if (q.w == 0.f) continue;
                acc += pixel_ell(L, s_lut, c, q, x, y, [&](int xj, int yj) { return zd[(yj - zy0) * c.W + xj]; });
            }
        }
        const float tot = block_sum(acc, s_red);
        if (tid == 0) out_ll[h] = tot;
        __syncthreads();
    }
}

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------

static int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

template <class K>
static int persistent_grid(K kernel, int smem, int64_t n, int grid) {
    if (grid > 0) return (int)std::min<int64_t>(grid, std::max<int64_t>(n, 1));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem);
    if (per_sm <= 0) per_sm = 1;
    return (int)std::min<int64_t>((int64_t)per_sm * sm_count(), std::max<int64_t>(n, 1));
}

template <class PS, int NT>
static int launch_score_nt(const SceneView &sv, const Lik &L, PS P, int64_t n, float *ll, int grid, cudaStream_t s) {
    const int n_lat = sv.mesh.nc[0] + sv.mesh.nc[1] + sv.mesh.nc[2];
    const int smem = kRegionPx * (int)sizeof(unsigned) + n_lat * (int)sizeof(float4);
    auto pick = [&](auto st) {
        constexpr bool ST = decltype(st)::value;
        return L.w == 1 ? k_score<PS, ST, 1, NT> : (L.w == 2 ? k_score<PS, ST, 2, NT> : k_score<PS, ST, 0, NT>);
    };
    auto kern = sv.stats ? pick(std::true_type{}) : pick(std::false_type{});
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    per_sm = std::max(per_sm, 1);
    // grid > 0: CTAs per SM requested by the tuning (capped by occupancy); 0: occupancy
    const int ctas = grid > 0 ? std::min(grid, per_sm) : per_sm;
    const int g = (int)std::min<int64_t>((int64_t)ctas * sm_count(), std::max<int64_t>(n, 1));
    kern<<<g, NT, smem, s>>>(sv, L, P, n, ll);
    return g;
}

// grid encodes the tuning: bits 0-7 CTAs per SM (0 = as many as fit), bit 8: 128-thread CTAs.
template <class PS>
static int launch_score(const SceneView &sv, const Lik &L, PS P, int64_t n, float *ll, int grid, cudaStream_t s) {
    if (n <= 0) return 0;
    if (grid & 256) return launch_score_nt<PS, 128>(sv, L, P, n, ll, grid & 255, s);
    return launch_score_nt<PS, 256>(sv, L, P, n, ll, grid & 255, s);
}

int launch_score_list(const SceneView &sv, const Lik &L, PoseList P, int64_t n, float *ll, int grid, cudaStream_t s) {
    return launch_score(sv, L, P, n, ll, grid, s);
}

int launch_score_grid(const SceneView &sv, const Lik &L, PoseGrid P, int64_t n, float *ll, int grid, cudaStream_t s) {
    return launch_score(sv, L, P, n, ll, grid, s);
}

int launch_render_list(const SceneView &sv, PoseList P, int64_t n, float *depth, int *tid, int grid, cudaStream_t s) {
    if (n <= 0) return 0;
    const int smem = kRegionPx * (int)sizeof(unsigned long long);
    auto kern = k_render<PoseList>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    const int g = persistent_grid(kern, smem, n, grid);
    kern<<<g, kThreads, smem, s>>>(sv, P, n, depth, tid);
    return g;
}

void launch_score_depth(const SceneView &sv, const Lik &L, const float *depth, const int *tid, int64_t n, float *ll,
                        int grid, cudaStream_t s) {
    if (n <= 0) return;
    const int smem = 2 * kRegionPx * (int)sizeof(float);
    const int g = persistent_grid(k_score_depth, smem, n, grid);
    k_score_depth<<<g, kThreads, smem, s>>>(sv, L, depth, tid, n, ll);
}

void launch_obs_points(const Cam &cam, const float *depth, float4 *obs, cudaStream_t s) {
    const int64_t n = (int64_t)cam.W * cam.H;
    k_obs_points<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(cam, depth, obs);
}

void launch_bg_clear(unsigned long long *bg, int64_t n, cudaStream_t s) {
    k_fill_u64<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(bg, n, kEmptyKey);
}

void launch_bg_raster(const Cam &cam, const MeshView &m, const float *pose16_dev, int tri_base,
                      unsigned long long *bg, cudaStream_t s) {
    if (m.n_full <= 0) return;
    const int warps_per_block = 8;
    const int blocks = (int)std::min<int64_t>((m.n_full + warps_per_block - 1) / warps_per_block, 8 * sm_count());
    k_bg_raster<<<blocks, 32 * warps_per_block, 0, s>>>(cam, m, pose16_dev, tri_base, bg);
}

void launch_bg_tables(const SceneView &sv, const Lik &L, float *ell_bg, float *gs_bg, float *gp_bg, cudaStream_t s) {
    const int64_t n = (int64_t)sv.cam.W * sv.cam.H;
    k_bg_tables<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(sv, L, ell_bg, gs_bg, gp_bg);
}

void launch_bg_sums(const float *a, const float *b, const float *c, int64_t n, double *out, cudaStream_t s) {
    k_sums<<<1, 1024, 0, s>>>(a, b, c, n, out);
}

}  // namespace b3d
