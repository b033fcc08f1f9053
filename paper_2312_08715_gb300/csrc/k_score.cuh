// k_score.cuh - the fused render + score kernel of libb3d and its launcher, a template
// instantiated per launch shape in the k_score_*.cu translation units (compiled in parallel).
//
// One hypothesis per CTA iteration of a persistent grid renders the object into a
// shared-memory z-buffer of depth bits, composites it with the fixed objects' depths and
// scores, against their background terms, the observed pixels whose window can see it:
//   LL_h = LL_bg + sum_{i in footprint + w} (l_i(h) - l_i(bg)),
// an exact identity (unchanged pixels are formed by the same expressions in the same order
// as the background table, so their terms cancel bit for bit).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>

#include "b3d_device.cuh"
#include "b3d_internal.h"

namespace b3d {

// launch shape that also gets a work-counting build (for the roofline accounting)
constexpr int kStatsNT = 128, kStatsMinB = 6;

inline int score_sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

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

// Packed pairs of FP32 values for the f32x2 arithmetic of sm_100 and later: each lane of a
// pair is rounded as the scalar operation rounds it, so the results are the scalar ones.
typedef unsigned long long f32x2_t;
__device__ __forceinline__ f32x2_t pk2(float a, float b) {
    f32x2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(f32x2_t v, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ f32x2_t fma2(f32x2_t a, f32x2_t b, f32x2_t c) {
    f32x2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f32x2_t sub2(f32x2_t a, f32x2_t b) {
    f32x2_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2_t mul2(f32x2_t a, f32x2_t b) {
    f32x2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
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
    const bool ball_skips_empty = L.r2 < 0.25f;
    const float r2b = __int_as_float(__float_as_int(L.r2) + 1) * 0x1p100f;  // (next float above r2) 2^100
    const float rxc = rx[W];  // the column's own ray
    // negated column rays packed for the f32x2 window terms (half window 1)
    const f32x2_t nrx01 = pk2(-rx[0], -rx[1]), nrx22 = pk2(-rx[D - 1], -rx[D - 1]);
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
        const float2 qe = S.qe[gi];  // observed depth (0: no point) and the background's term
        // the observed point, formed from its depth as the observation kernel forms it
        const float4 q = make_float4(__fmul_rn(qe.x, rxc), __fmul_rn(qe.x, ry[W]), qe.x, 1.f);
        int n = 0;
        float Ssum = 0.f;
        if (L.kind == 0 && ball_skips_empty) {
            // an empty slot holds z = -1, a point at least 1 m from q (q.z > 0): it can only
            // fail the inlier test, so the count needs no separate z >= 0 test
            // the count on the FMA pipe rather than the (half-rate) ALU pipe: (r2+ - d2) 2^100,
            // saturated to [0, 1], is 1 exactly when d2 <= r2 (r2+ the next float above r2, and
            // any nonzero difference times 2^100 is above 1) and 0 otherwise; the same n as the
            // comparison pixel_ell makes
            float nf = 0.f;
            if constexpr (W == 1) {
                // eight of the nine window elements as four packed pairs (columns 0-1 of each
                // row, and column 2 of rows 0-1), the last one scalar: per element the same
                // arithmetic as the scalar loop below; the 0/1 terms add up exactly in any order
                const f32x2_t qx2 = pk2(q.x, q.x), qy2 = pk2(q.y, q.y), qz2 = pk2(q.z, q.z);
                auto pair = [&](f32x2_t z2, f32x2_t nrx, f32x2_t nry) {
                    const f32x2_t ex = fma2(z2, nrx, qx2), ey = fma2(z2, nry, qy2), ez = sub2(qz2, z2);
                    float d2a, d2b;
                    upk2(fma2(ex, ex, fma2(ey, ey, mul2(ez, ez))), d2a, d2b);
                    nf += __saturatef(fmaf(-d2a, 0x1p100f, r2b));
                    nf += __saturatef(fmaf(-d2b, 0x1p100f, r2b));
                };
#pragma unroll
                for (int r = 0; r < D; ++r) pair(pk2(win[r][0], win[r][1]), nrx01, pk2(-ry[r], -ry[r]));
                pair(pk2(win[0][2], win[1][2]), nrx22, pk2(-ry[0], -ry[1]));
                const float z = win[2][2];
                const float exs = fmaf(-z, rx[2], q.x), eys = fmaf(-z, ry[2], q.y), ezs = q.z - z;
                nf += __saturatef(fmaf(-fmaf(exs, exs, fmaf(eys, eys, ezs * ezs)), 0x1p100f, r2b));
            } else {
#pragma unroll
                for (int r = 0; r < D; ++r) {
#pragma unroll
                    for (int d = 0; d < D; ++d) {
                        const float z = win[r][d];
                        const float ex = fmaf(-z, rx[d], q.x), ey = fmaf(-z, ry[r], q.y), ez = q.z - z;
                        nf += __saturatef(fmaf(-fmaf(ex, ex, fmaf(ey, ey, ez * ez)), 0x1p100f, r2b));
                    }
                }
            }
            n = (int)nf;
        } else {
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
        }
        const float l = L.kind == 0 ? lut[n] : __logf(fmaf(L.bg, Ssum, L.a));
        // a pixel without a point is skipped only now: a branch around the window loop costs
        // more than the loop (the lanes' pixels diverge)
        if (qe.x == 0.f) continue;
        acc += l - qe.y;
        if (n_px) {
            ++*n_px;
            *n_pairs += (unsigned long long)((min(y + W, c.H - 1) - max(y - W, 0) + 1) *
                                             (min(x + W, c.W - 1) - max(x - W, 0) + 1));
        }
    }
    return acc;
}

// z-buffer pixels per tile for a CTA of NT threads (measured: 3072 for 128 threads leaves room
// for one more resident CTA per SM than 4096 while still holding a tabletop footprint in one
// tile; 8192 for 256 threads, 3 CTAs per SM, holds most of a 320x240 footprint in one or two
// tiles: the serving images' hypotheses re-stage their rectangles for fewer tiles)
template <int NT>
constexpr int score_region() { return NT <= 64 ? 2048 : (NT == 128 ? 3072 : 8192); }
// pixels per thread whose background depths the composite loads together
#ifndef B3D_COMPOSITE_BATCH
#define B3D_COMPOSITE_BATCH 4
#endif
constexpr int kCompBatch = B3D_COMPOSITE_BATCH;
constexpr int kStageStride = 6;  // float4 per staged rectangle: four edges, plane, pixel box
// Layout of a warp's 32 staged records: component k of lane l's record at [k * 32 + l], so
// the lanes' stores and the owners' loads touch consecutive 16-byte words (rather than
// words 96 bytes apart, which shared four banks between lanes l and l + 4).
__device__ __forceinline__ int stage_slot(int l, int k) { return k * 32 + l; }
// Pixels a candidate of the cooperative rasteriser covers (a block of kCandX x kCandY): the
// owner lookup, record loads and index arithmetic are shared by the block's pixel tests.
#ifndef B3D_CAND_X
#define B3D_CAND_X 2
#endif
#ifndef B3D_CAND_Y
#define B3D_CAND_Y 1
#endif
constexpr int kCandX = B3D_CAND_X, kCandY = B3D_CAND_Y;

// A rectangle edge a->b staged for the pixel tests: its canonical origin (the
// lexicographically smaller endpoint, as edge_fn) and direction, with the quad's
// orientation sign folded into the direction. Relative to the canonical direction
// (from the smaller endpoint to the larger) the swap and the sign cancel:
// (sw ? -s : s) * (sw ? a - b : b - a) = s * (b - a) exactly, since negation is exact in
// round-to-nearest. So fmaf(E.z, py - E.y, -(E.w * (px - E.x))) equals s * edge_fn(a, b, p)
// bit for bit (up to the sign of a zero), and the test is e >= 0.
__device__ __forceinline__ float4 stage_edge(float ax, float ay, float bx, float by, float s) {
    const bool sw = (bx < ax) || (bx == ax && by < ay);
    return make_float4(sw ? bx : ax, sw ? by : ay, s * (bx - ax), s * (by - ay));
}

__device__ __forceinline__ bool staged_inside(const float4 &E, float px, float py) {
    return fmaf(E.z, py - E.y, -(E.w * (px - E.x))) >= 0.f;
}

// The mesh's lattice plane coordinates into the .w of the CTA's lattice table, once per
// mesh (before the barrier that precedes the first render_tiles): each hypothesis's lattice
// pass then reads them from shared memory rather than from a global load that misses L1.
__device__ __forceinline__ void lattice_coords(const MeshView &m, float4 *lat) {
    if (m.n_quads <= 0) return;
    const int n = m.nc[0] + m.nc[1] + m.nc[2];
    for (int k = threadIdx.x; k < n; k += blockDim.x) lat[k].w = m.coords[k];
}

// Per-CTA shared state of one hypothesis.
template <int NT>
struct ScoreShared {
    float pose[12];
    int bb[4];
    int fbb[4];   // bounding box of the tile's fragments
    int flags;    // bit 0: on screen, bit 1: rectangle path, bit 2: whole object beyond near
    int rng[13];  // class first rectangles [6], exclusive prefix of counts [6], total
    float red[NT / 32];
    int own[NT];  // per warp: the lane whose candidate run starts at each position of a window
};

// Renders the hypothesis whose pose thread 0 has put in sh.pose, tile by tile, into the
// shared-memory z-buffer and composites it with the fixed objects' depths (misses: far, or
// -1 with miss_mode 1); for each tile with fragments calls
// visit(zd, zx0, zy0, zw, qx0, qx1, qy0, qy1, tx0, tx1, ty0, ty1): the tile's depths zd
// (origin zx0, zy0, row pitch zw; the tile [tx0, tx1] x [ty0, ty1] plus w around it) and the
// pixels to score, those whose half-window w reaches a fragment. Returns false when the
// object is off screen (nothing visited). All threads of the CTA must call it.
// TAGS: the z-buffer holds 64-bit keys (depth bits, tag) in zb's memory (kRegionPx of them),
// the tag being the rectangle's face class or the triangle's global id; the composite writes
// the depths to zdt and the winning tags to tagt (-1 where the fixed objects are nearer).
template <bool STATS, int NT, bool TAGS = false, class Visit>
__device__ __forceinline__ bool render_tiles(const SceneView &S, int w, int miss_mode, ScoreShared<NT> &sh,
                                             float4 *s_stage, unsigned *zb, float4 *lat, unsigned long long *cnt,
                                             Visit &&visit, float *zdt = nullptr, int *tagt = nullptr) {
    constexpr int REG = TAGS ? kRegionPx : score_region<NT>();
    float *zd = TAGS ? zdt : reinterpret_cast<float *>(zb);  // 32-bit keys: the same memory, as depths
    unsigned long long *zb64 = reinterpret_cast<unsigned long long *>(zb);
    const Cam &c = S.cam;
    const MeshView &m = S.mesh;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
    const int n_lat = m.nc[0] + m.nc[1] + m.nc[2];
    const int nc0 = m.nc[0], nc01 = m.nc[0] + m.nc[1];
    auto lat_off = [&](int a) { return a == 0 ? 0 : (a == 1 ? nc0 : nc01); };
    if (wid == 0) {
        // warp 0: lane k < 8 projects corner k of the object's box (the arithmetic of
        // object_bbox, reduced with exact min / max), lane c < 6 finds face class c's range
        __syncwarp();
        const float *P = sh.pose;
        float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
        bool cfront = true;
        const bool has = m.n_full > 0;
        if (has && lane < 8) {
            const float ox = (lane & 1) ? m.hi[0] : m.lo[0], oy = (lane & 2) ? m.hi[1] : m.lo[1];
            const float oz = (lane & 4) ? m.hi[2] : m.lo[2];
            float x, y, z;
            xform(P, ox, oy, oz, x, y, z);
            if (!(z >= c.near_z)) {
                cfront = false;
            } else {
                umin = umax = fmaf(c.fx, x / z, c.cx);
                vmin = vmax = fmaf(c.fy, y / z, c.cy);
            }
        }
        const bool front = has && __all_sync(0xffffffffu, cfront);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            umin = fminf(umin, __shfl_xor_sync(0xffffffffu, umin, o));
            umax = fmaxf(umax, __shfl_xor_sync(0xffffffffu, umax, o));
            vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
            vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
        }
        int bb0 = 0, bb1 = c.W - 1, bb2 = 0, bb3 = c.H - 1;
        if (front) {
            const float lo_u = fmaxf(umin - 0.5f, -2.f), hi_u = fminf(umax - 0.5f, (float)c.W + 1.f);
            const float lo_v = fmaxf(vmin - 0.5f, -2.f), hi_v = fminf(vmax - 0.5f, (float)c.H + 1.f);
            bb0 = max((int)ceilf(lo_u) - 1, 0);
            bb1 = min((int)floorf(hi_u) + 1, c.W - 1);
            bb2 = max((int)ceilf(lo_v) - 1, 0);
            bb3 = min((int)floorf(hi_v) + 1, c.H - 1);
        }
        int f = has && bb0 <= bb1 && bb2 <= bb3 ? 1 : 0;
        if (front) f |= 4;
        if (f && front && m.n_quads > 0) {
            f |= 2;
            int cnt = 0, b = 0;
            if (lane < 6) {
                const int cls = lane, a = cls >> 1;
                const float *R = P, *t = P + 9;
                const float oa = -fmaf(R[a], t[0], fmaf(R[3 + a], t[1], R[6 + a] * t[2]));
                // the plane coordinates from the lattice table's .w (shared memory, set once
                // per mesh and rewritten unchanged by each lattice pass, after a barrier)
                const float4 *cd = lat + lat_off(a);
                const int n = m.nc[a];
                int lo = 0, hi = n;  // first plane with coordinate >= o
                while (lo < hi) { const int mid = (lo + hi) >> 1; if (cd[mid].w < oa) lo = mid + 1; else hi = mid; }
                const int below = lo;
                hi = n;  // first plane with coordinate > o
                while (lo < hi) { const int mid = (lo + hi) >> 1; if (cd[mid].w <= oa) lo = mid + 1; else hi = mid; }
                const int not_above = lo;
                const int *off = m.class_off + cls * m.np1;
                // +axis faces face the camera when their plane is below o; -axis when above
                b = (cls & 1) ? off[0] : off[not_above];
                const int e = (cls & 1) ? off[below] : off[n];
                cnt = e - b;
            }
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) {
                const int up = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += up;
            }
            if (lane < 6) {
                sh.rng[lane] = b;
                sh.rng[6 + lane] = incl - cnt;
            }
            if (lane == 5) sh.rng[12] = incl;
        }
        if (lane == 0) {
            sh.bb[0] = bb0; sh.bb[1] = bb1; sh.bb[2] = bb2; sh.bb[3] = bb3;
            sh.flags = f;
        }
    }
    __syncthreads();
    const int flags = sh.flags;
    if (!(flags & 1)) return false;
    const float *pose = sh.pose;
    const bool quad = (flags & 2) != 0, front = (flags & 4) != 0;
    const int bx0 = sh.bb[0], bx1 = sh.bb[1], by0 = sh.bb[2], by1 = sh.bb[3];
    if (quad) {
        for (int k = tid; k < n_lat; k += nt) {
            const int a = k < nc0 ? 0 : (k < nc01 ? 1 : 2);
            const float v = lat[k].w;  // the plane's coordinate (lattice_coords)
            lat[k] = make_float4(fmaf(pose[a], v, a == 0 ? pose[9] : 0.f), fmaf(pose[3 + a], v, a == 0 ? pose[10] : 0.f),
                                 fmaf(pose[6 + a], v, a == 0 ? pose[11] : 0.f), v);
        }
        if (STATS) cnt[1] += (unsigned long long)((n_lat - tid + nt - 1) / nt);
    }
    const int sx0 = max(bx0 - w, 0), sx1 = min(bx1 + w, c.W - 1);
    const int sy0 = max(by0 - w, 0), sy1 = min(by1 + w, c.H - 1);
    const int sw = sx1 - sx0 + 1;
    // the tile plus its halo must fit the region even one row high: (tw + 2w)(1 + 2w) <= REG
    const int tw = min(min(sw, S.tile_w), REG / (1 + 2 * w) - 2 * w);
    const int th = max(1, REG / (tw + 2 * w) - 2 * w);
    for (int ty0 = sy0; ty0 <= sy1; ty0 += th) {
        for (int tx0 = sx0; tx0 <= sx1; tx0 += tw) {
            const int tx1 = min(tx0 + tw - 1, sx1), ty1 = min(ty0 + th - 1, sy1);
            const int zx0 = max(tx0 - w, 0), zx1 = min(tx1 + w, c.W - 1);
            const int zy0 = max(ty0 - w, 0), zy1 = min(ty1 + w, c.H - 1);
            const int zw = zx1 - zx0 + 1, zh = zy1 - zy0 + 1, nz = zw * zh;
            const int rx0 = max(zx0, bx0), rx1 = min(zx1, bx1), ry0 = max(zy0, by0), ry1 = min(zy1, by1);
            const bool need = rx0 <= rx1 && ry0 <= ry1;
            for (int i = tid; i < nz; i += nt) {
                if constexpr (TAGS) zb64[i] = kEmptyKey;
                else zb[i] = 0xffffffffu;
            }
            if (tid == 0) { sh.fbb[0] = INT32_MAX; sh.fbb[1] = -1; sh.fbb[2] = INT32_MAX; sh.fbb[3] = -1; }
            __syncthreads();
            if (need) {
                // box of this lane's fragments (triangles) or candidate boxes (rectangles)
                int fx0 = INT32_MAX, fx1 = -1, fy0 = INT32_MAX, fy1 = -1;
                auto store = [&](int x, int y, float z) {
                    if (STATS) ++cnt[4];
                    atomicMin(&zb[(y - zy0) * zw + (x - zx0)], __float_as_uint(z));
                    fx0 = min(fx0, x); fx1 = max(fx1, x); fy0 = min(fy0, y); fy1 = max(fy1, y);
                };
                if (quad) {
                    // Each warp takes 32 rectangles at a time: every lane projects one and
                    // stages its screen corners, plane and pixel box; then the warp shares out
                    // the pixel-centre candidates of all 32 among its lanes.
                    // Candidate block (x, y) of a rectangle with edges E0-E3, plane Pl and pixel
                    // box ending at (xe, ye):
                    auto raster_block = [&](const float4 &E0, const float4 &E1, const float4 &E2, const float4 &E3,
                                            const float4 &Pl, int x, int y, int xe, int ye, bool valid, unsigned tag) {
#pragma unroll
                        for (int e = 0; e < kCandY; ++e) {
                            const float py = (float)(y + e) + 0.5f;
#pragma unroll
                            for (int d = 0; d < kCandX; ++d) {
                                const float px = (float)(x + d) + 0.5f;
                                // every test evaluated and one predicated store: branches on the
                                // tests cost more than the tests (the lanes' pixels diverge)
                                const bool in = valid & (x + d <= xe) & (kCandY == 1 || y + e <= ye) & staged_inside(E0, px, py) &
                                                staged_inside(E1, px, py) & staged_inside(E2, px, py) & staged_inside(E3, px, py);
                                const float z = __fdividef(1.0f, fmaf(Pl.x, px, fmaf(Pl.y, py, Pl.z)));
                                if (in & (z <= c.far_z)) {
                                    if (STATS) ++cnt[4];
                                    const int zi = (y + e - zy0) * zw + (x + d - zx0);
                                    if constexpr (TAGS) atomicMin(&zb64[zi], ((unsigned long long)__float_as_uint(z) << 32) | tag);
                                    else atomicMin(&zb[zi], __float_as_uint(z));
                                }
                            }
                        }
                    };
                    const int total = sh.rng[12];
                    float4 *stg = s_stage + (wid * 32) * kStageStride;
                    for (int base = wid * 32; base < total; base += nt) {
                        const int k = base + lane;
                        int cand = 0;
                        if (k < total) {
                            int cls = 0;
#pragma unroll
                            for (int j = 1; j < 6; ++j) cls += k >= sh.rng[6 + j] ? 1 : 0;
                            const uint2 q = m.quads[sh.rng[cls] + (k - sh.rng[6 + cls])];
                            const int a = cls >> 1, p = (q.x >> 18) & 511, b0 = (q.x >> 9) & 511, c0 = q.x & 511;
                            const int b1 = b0 + (int)((q.y >> 9) & 511), c1 = c0 + (int)(q.y & 511);
                            const int ab = a == 2 ? 0 : a + 1, ac = a == 0 ? 2 : a - 1;
                            // the plane term is shared by all corners, the in-plane terms take two
                            // values each; corners are summed in x, y, z order
                            const float4 Tp = lat[lat_off(a) + p];
                            const float4 Tb0 = lat[lat_off(ab) + b0], Tb1 = lat[lat_off(ab) + b1];
                            const float4 Tc0 = lat[lat_off(ac) + c0], Tc1 = lat[lat_off(ac) + c1];
                            float4 W0, W1, W2, W3;  // corners k0 (b0,c0) k1 (b1,c0) k2 (b1,c1) k3 (b0,c1)
                            if (a == 0) {
                                W0 = sum3(Tp, Tb0, Tc0); W1 = sum3(Tp, Tb1, Tc0); W2 = sum3(Tp, Tb1, Tc1); W3 = sum3(Tp, Tb0, Tc1);
                            } else if (a == 1) {
                                W0 = sum3(Tc0, Tp, Tb0); W1 = sum3(Tc0, Tp, Tb1); W2 = sum3(Tc1, Tp, Tb1); W3 = sum3(Tc1, Tp, Tb0);
                            } else {
                                W0 = sum3(Tb0, Tc0, Tp); W1 = sum3(Tb1, Tc0, Tp); W2 = sum3(Tb1, Tc1, Tp); W3 = sum3(Tb0, Tc1, Tp);
                            }
                            const float4 C0 = screen_pt(W0.x, W0.y, W0.z, c), C1 = screen_pt(W1.x, W1.y, W1.z, c);
                            const float4 C2 = screen_pt(W2.x, W2.y, W2.z, c), C3 = screen_pt(W3.x, W3.y, W3.z, c);
                            if (STATS) { cnt[1] += 4; ++cnt[2]; }
                            const float area = edge_fn(C0.x, C0.y, C1.x, C1.y, C2.x, C2.y);
                            if (area != 0.f) {
                                const float umin = fminf(fminf(C0.x, C1.x), fminf(C2.x, C3.x));
                                const float umax = fmaxf(fmaxf(C0.x, C1.x), fmaxf(C2.x, C3.x));
                                const float vmin = fminf(fminf(C0.y, C1.y), fminf(C2.y, C3.y));
                                const float vmax = fmaxf(fmaxf(C0.y, C1.y), fmaxf(C2.y, C3.y));
                                const int x0 = (int)ceilf(fmaxf(umin - 0.5f, (float)rx0));
                                const int x1 = (int)floorf(fminf(umax - 0.5f, (float)rx1));
                                const int y0 = (int)ceilf(fmaxf(vmin - 0.5f, (float)ry0));
                                const int y1 = (int)floorf(fminf(vmax - 0.5f, (float)ry1));
                                if (x0 <= x1 && y0 <= y1) {
                                    // candidates are blocks of kCandX x kCandY pixels
                                    const int bw2 = (x1 - x0 + kCandX) / kCandX;
                                    cand = bw2 * ((y1 - y0 + kCandY) / kCandY);
                                    // the fragment box as the union of the candidate boxes (a pixel in
                                    // it without a fragment in its window scores 0 exactly)
                                    fx0 = min(fx0, x0); fx1 = max(fx1, x1); fy0 = min(fy0, y0); fy1 = max(fy1, y1);
                                    if (STATS) cnt[3] += (unsigned long long)((x1 - x0 + 1) * (y1 - y0 + 1));
                                    const float inv = __fdividef(1.0f, area);
                                    const float du1 = C1.x - C0.x, dv1 = C1.y - C0.y, du2 = C2.x - C0.x, dv2 = C2.y - C0.y;
                                    const float dz1 = C1.z - C0.z, dz2 = C2.z - C0.z;
                                    const float al = fmaf(dz1, dv2, -(dz2 * dv1)) * inv;
                                    const float be = fmaf(dz2, du1, -(dz1 * du2)) * inv;
                                    const float sgn = area > 0.f ? 1.f : -1.f;
                                    const float4 E0 = stage_edge(C0.x, C0.y, C1.x, C1.y, sgn);
                                    const float4 E1 = stage_edge(C1.x, C1.y, C2.x, C2.y, sgn);
                                    const float4 E2 = stage_edge(C2.x, C2.y, C3.x, C3.y, sgn);
                                    const float4 E3 = stage_edge(C3.x, C3.y, C0.x, C0.y, sgn);
                                    // 1/z = al px + be py + K over the quad's plane
                                    const float K = fmaf(-al, C0.x, fmaf(-be, C0.y, C0.z));
                                    // the candidate's row is floor((k + 1/2) / candidates per row), exact
                                    // in float with an approximate reciprocal for the region's sizes (the
                                    // quotient is at least 1/(2 bw2) from an integer; the error is below
                                    // (k + 1/2) 2^-21 / bw2)
                                    const float4 Pl = make_float4(al, be, K, __fdividef(1.0f, (float)bw2));
                                    stg[stage_slot(lane, 0)] = E0;
                                    stg[stage_slot(lane, 1)] = E1;
                                    stg[stage_slot(lane, 2)] = E2;
                                    stg[stage_slot(lane, 3)] = E3;
                                    stg[stage_slot(lane, 4)] = Pl;
                                    // box extents below 2^16 and 2^13; TAGS: the class in the top bits
                                    const int ends = (x1 - x0) | ((y1 - y0) << 16) | (TAGS ? cls << 29 : 0);
                                    stg[stage_slot(lane, 5)] = make_float4(__int_as_float(x0), __int_as_float(y0), __int_as_float(bw2),
                                                         __int_as_float(ends));
                                }
                            }
                        }
                        int incl = cand;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const int up = __shfl_up_sync(0xffffffffu, incl, o);
                            if (lane >= o) incl += up;
                        }
                        const int n_cand = __shfl_sync(0xffffffffu, incl, 31);
                        const int excl = incl - cand;
                        int *own = sh.own + wid * 32;
                        int carry = 0;  // the lane whose run holds the window's first position
                        __syncwarp();
                        for (int r0 = 0; r0 < n_cand; r0 += 32) {
                            // runs [excl, incl) tile [0, n_cand) in lane order: the owner of
                            // position j is the lane whose run starts last at or before j
                            const bool starts = cand > 0 && excl >= r0 && excl < r0 + 32;
                            if (starts) own[excl - r0] = lane;
                            const unsigned pos = __reduce_or_sync(0xffffffffu, starts ? 1u << (excl - r0) : 0u);
                            __syncwarp();
                            const unsigned upto = pos & (0xffffffffu >> (31 - lane));
                            const int lo = upto ? own[31 - __clz(upto)] : carry;
                            carry = __shfl_sync(0xffffffffu, lo, 31);
                            const int j = r0 + lane;
                            const int kk = j - __shfl_sync(0xffffffffu, excl, lo);
                            __syncwarp();
                            {  // lanes past the last candidate run the tests with their stores masked
                                const float4 Pl = stg[stage_slot(lo, 4)], Bx = stg[stage_slot(lo, 5)];
                                const float4 E0 = stg[stage_slot(lo, 0)], E1 = stg[stage_slot(lo, 1)];
                                const float4 E2 = stg[stage_slot(lo, 2)], E3 = stg[stage_slot(lo, 3)];
                                const int bw2 = __float_as_int(Bx.z), ends = __float_as_int(Bx.w);
                                const int bx = __float_as_int(Bx.x), by = __float_as_int(Bx.y);
                                const int xe = bx + (ends & 0xffff), ye = by + (TAGS ? (ends >> 16) & 0x1fff : ends >> 16);
                                const int row = (int)(((float)kk + 0.5f) * Pl.w);
                                raster_block(E0, E1, E2, E3, Pl, bx + kCandX * (kk - row * bw2), by + kCandY * row, xe, ye,
                                             j < n_cand, (unsigned)ends >> 29);
                            }
                        }
                        __syncwarp();
                    }
                } else {
                    const int4 *tris = front ? m.tris_surf : m.tris_full;
                    const int n_t = front ? m.n_surf : m.n_full;
                    const int cull = front ? m.closed : 0;
                    for (int t = tid; t < n_t; t += nt) {
                        float4 A, B, C;
                        tri_screen(m, tris[t], pose, c, A, B, C);
                        if (STATS) { cnt[1] += 3; ++cnt[2]; }
                        if constexpr (TAGS) {
                            const unsigned long long gid = (unsigned)(S.tri_base + tris[t].w);
                            raster_tri(A, B, C, cull, rx0, rx1, ry0, ry1, c.far_z, [&](int x, int y, float z) {
                                atomicMin(&zb64[(y - zy0) * zw + (x - zx0)], ((unsigned long long)__float_as_uint(z) << 32) | gid);
                                fx0 = min(fx0, x); fx1 = max(fx1, x); fy0 = min(fy0, y); fy1 = max(fy1, y);
                            });
                        } else {
                            raster_tri(A, B, C, cull, rx0, rx1, ry0, ry1, c.far_z, store, STATS ? &cnt[3] : nullptr);
                        }
                    }
                }
                // the tile's fragment box: pixels outside it +- w keep their background terms
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    fx0 = min(fx0, __shfl_xor_sync(0xffffffffu, fx0, o));
                    fx1 = max(fx1, __shfl_xor_sync(0xffffffffu, fx1, o));
                    fy0 = min(fy0, __shfl_xor_sync(0xffffffffu, fy0, o));
                    fy1 = max(fy1, __shfl_xor_sync(0xffffffffu, fy1, o));
                }
                if (lane == 0 && fx1 >= 0) {
                    atomicMin(&sh.fbb[0], fx0); atomicMax(&sh.fbb[1], fx1);
                    atomicMin(&sh.fbb[2], fy0); atomicMax(&sh.fbb[3], fy1);
                }
            }
            __syncthreads();
            if (sh.fbb[1] < 0) {  // nothing of the object in this tile: every term is unchanged
                __syncthreads();
                continue;
            }
            // composite with the fixed objects in place (depth bits -> rendered depth) over
            // the fragment box + 2w, the depths the scored windows read
            const int cx0 = max(sh.fbb[0] - 2 * w, zx0), cx1 = min(sh.fbb[1] + 2 * w, zx1);
            const int cy0 = max(sh.fbb[2] - 2 * w, zy0), cy1 = min(sh.fbb[3] + 2 * w, zy1);
            {
                const int cw = cx1 - cx0 + 1, n_c = cw * (cy1 - cy0 + 1);
                const int dq = nt / cw, dr = nt - dq * cw;
                int y = tid / cw, x = tid - y * cw;
                // kCompBatch pixels per thread at a time: their background loads are issued
                // together, so their latencies overlap
                for (int i = tid; i < n_c; i += kCompBatch * nt) {
                    int zi[kCompBatch];
                    if constexpr (TAGS) {
                        unsigned long long bgk[kCompBatch];
#pragma unroll
                        for (int u = 0; u < kCompBatch; ++u) {
                            zi[u] = -1;
                            bgk[u] = 0ull;
                            if (i + u * nt < n_c) {
                                const int gx = cx0 + x, gy = cy0 + y;
                                zi[u] = (gy - zy0) * zw + (gx - zx0);
                                bgk[u] = S.bg[(int64_t)gy * c.W + gx];
                            }
                            x += dr;
                            y += dq;
                            if (x >= cw) { x -= cw; ++y; }
                        }
#pragma unroll
                        for (int u = 0; u < kCompBatch; ++u) {
                            if (zi[u] >= 0) {
                                const unsigned long long key = zb64[zi[u]];
                                const bool obj = key < bgk[u];
                                zd[zi[u]] = key_depth(obj ? key : bgk[u], miss_mode, c.far_z);
                                tagt[zi[u]] = obj ? (int)(unsigned)key : -1;
                            }
                        }
                        continue;
                    }
                    unsigned bgb[kCompBatch];
#pragma unroll
                    for (int u = 0; u < kCompBatch; ++u) {
                        zi[u] = -1;
                        bgb[u] = 0u;
                        if (i + u * nt < n_c) {
                            const int gx = cx0 + x, gy = cy0 + y;
                            zi[u] = (gy - zy0) * zw + (gx - zx0);
                            const int64_t gi = (int64_t)gy * c.W + gx;
                            bgb[u] = S.bgz ? S.bgz[gi] : (unsigned)(S.bg[gi] >> 32);
                        }
                        x += dr;
                        y += dq;
                        if (x >= cw) { x -= cw; ++y; }
                    }
#pragma unroll
                    for (int u = 0; u < kCompBatch; ++u) {
                        if (zi[u] >= 0) {
                            const unsigned v = min(zb[zi[u]], bgb[u]);
                            zd[zi[u]] = v == 0xffffffffu ? (miss_mode ? -1.f : c.far_z) : __uint_as_float(v);
                        }
                    }
                }
                if (STATS) cnt[5] += (unsigned long long)((n_c - tid + nt - 1) / nt);
            }
            __syncthreads();
            // score the tile's pixels within the fragment box + w
            const int qx0 = max(sh.fbb[0] - w, tx0), qx1 = min(sh.fbb[1] + w, tx1);
            const int qy0 = max(sh.fbb[2] - w, ty0), qy1 = min(sh.fbb[3] + w, ty1);
            visit(static_cast<const float *>(zd), zx0, zy0, zw, qx0, qx1, qy0, qy1, tx0, tx1, ty0, ty1);
            __syncthreads();
        }
    }
    return true;
}

// Scores the hypothesis whose pose thread 0 has put in sh.pose: returns, in thread 0, the
// sum of l_i - l_i(bg) over the pixels whose window can see the object (0 when it is off
// screen). All threads of the CTA must call it.
template <bool STATS, int WT, int NT>
__device__ __forceinline__ float score_body(const SceneView &S, const Lik &L, const float *s_lut, ScoreShared<NT> &sh,
                                            float4 *s_stage, unsigned *zb, float4 *lat, unsigned long long *cnt) {
    const Cam &c = S.cam;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int w = WT > 0 ? WT : L.w;
    float acc = 0.f;
    const bool drawn = render_tiles<STATS, NT>(
        S, w, L.miss_mode, sh, s_stage, zb, lat, cnt,
        [&](const float *zd, int zx0, int zy0, int zw, int qx0, int qx1, int qy0, int qy1, int, int, int, int) {
            const int tww = qx1 - qx0 + 1, thh = qy1 - qy0 + 1;
            if (WT > 0) {
                // thread -> (column, run of rows)
                const int nseg = max(1, nt / tww);
                const int rps = (thh + nseg - 1) / nseg;
                const int seg = tid / tww, col = tid - seg * tww;
                if (seg < nseg && col < tww) {
                    const int ya = qy0 + seg * rps, yb = min(ya + rps - 1, qy1);
                    if (ya <= yb)
                        acc += score_column<WT>(S, L, s_lut, c, zd, zx0, zy0, zw, qx0 + col, ya, yb,
                                                STATS ? &cnt[6] : nullptr, STATS ? &cnt[7] : nullptr);
                }
            } else {
                const int n_tile = tww * thh;
                const int dq = nt / tww, dr = nt - dq * tww;
                int y = tid / tww, x = tid - y * tww;
                for (int k = tid; k < n_tile; k += nt) {
                    const int gx = qx0 + x, gy = qy0 + y;
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
        });
    if (!drawn) return 0.f;
    return block_sum(acc, sh.red);
}

template <class PS, bool STATS, int WT, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_score(SceneView S, Lik L, PS P, int64_t n_hyp, float *out_ll) {
    constexpr int REG = score_region<NT>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned *zb = reinterpret_cast<unsigned *>(smem_raw);                        // [REG]
    float4 *lat = reinterpret_cast<float4 *>(smem_raw + REG * sizeof(unsigned));  // lattice planes
    __shared__ float s_lut[kMaxLut];
    __shared__ ScoreShared<NT> sh;
    __shared__ float4 s_stage[NT * kStageStride];  // per lane: a rectangle's corners, plane, pixel box
    const int tid = threadIdx.x;
    for (int i = tid; i < L.n_lut; i += blockDim.x) s_lut[i] = L.lut[i];
    lattice_coords(S.mesh, lat);
    unsigned long long cnt[kNumStats] = {0, 0, 0, 0, 0, 0, 0, 0};
    __shared__ long long s_next;
    // With a counter, CTAs take their next hypothesis from it as they finish one (so they all
    // finish together however uneven the hypotheses' costs); thread 0 asks for it at the start
    // of the current one and publishes it at the end.
    int64_t h = blockIdx.x;
    __syncthreads();
    while (h < n_hyp) {
        long long nxt = h + gridDim.x;
        if (tid == 0) {
            if (S.work) nxt = (long long)gridDim.x + (long long)atomicAdd(S.work, 1ull);
            if (STATS) ++cnt[0];
            pose12(P, h, sh.pose);
        }
        const float tot = score_body<STATS, WT, NT>(S, L, s_lut, sh, s_stage, zb, lat, cnt);
        if (tid == 0) {
            out_ll[h] = (float)(*S.ll_bg + (double)tot);
            s_next = nxt;
        }
        __syncthreads();  // the next write of s_next comes after score_body's barriers
        h = s_next;
    }
    if (STATS)
        for (int k = 0; k < kNumStats; ++k)
            if (cnt[k]) atomicAdd(&S.stats[k], cnt[k]);
}

// Batched form: the hypotheses of many scenes (uneven image sizes, meshes and counts) in one
// persistent launch. CTAs take chunks of hypotheses from a global counter (a work queue
// over scenes and hypothesis chunks); when a chunk starts a new scene the CTA stages that
// scene's descriptor in shared memory. Scores are bit-identical to the single-scene kernel.
template <int WT, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_score_multi(const BatchItem *items, int n_items, const int64_t *item_begin, int64_t total, int chunk,
                  unsigned long long *counter) {
    constexpr int REG = score_region<NT>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned *zb = reinterpret_cast<unsigned *>(smem_raw);
    float4 *lat = reinterpret_cast<float4 *>(smem_raw + REG * sizeof(unsigned));
    __shared__ __align__(16) BatchItem s_item;
    __shared__ ScoreShared<NT> sh;
    __shared__ float4 s_stage[NT * kStageStride];
    __shared__ long long s_work[2];
    const int tid = threadIdx.x;
    int cur = -1;
    for (;;) {
        __syncthreads();
        if (tid == 0) s_work[0] = (long long)atomicAdd(counter, 1ull) * chunk;
        __syncthreads();
        const int64_t b = s_work[0];
        if (b >= total) break;
        const int64_t e = min(b + (int64_t)chunk, total);
        for (int64_t g = b; g < e;) {
            __syncthreads();
            if (tid == 0) {  // the scene holding hypothesis g
                int lo = 0, hi = n_items - 1;
                while (lo < hi) { const int mid = (lo + hi + 1) >> 1; if (item_begin[mid] <= g) lo = mid; else hi = mid - 1; }
                s_work[1] = lo;
            }
            __syncthreads();
            const int it = (int)s_work[1];
            if (it != cur) {
                const float4 *src = reinterpret_cast<const float4 *>(items + it);
                float4 *dst = reinterpret_cast<float4 *>(&s_item);
                for (int k = tid; k < (int)(sizeof(BatchItem) / sizeof(float4)); k += blockDim.x) dst[k] = src[k];
                cur = it;
                __syncthreads();
                lattice_coords(s_item.S.mesh, lat);  // ordered before use by render_tiles' first barrier
            }
            const int64_t ib = item_begin[it], ie = min(item_begin[it + 1], e);
            for (; g < ie; ++g) {
                __syncthreads();
                if (tid == 0) {
                    if (s_item.pose_kind == 0) pose12(s_item.list, g - ib, sh.pose);
                    else pose12(s_item.grid, g - ib, sh.pose);
                }
                const float tot = score_body<false, WT, NT>(s_item.S, s_item.L, s_item.L.lut, sh, s_stage, zb, lat, nullptr);
                if (tid == 0) s_item.out_ll[g - ib] = (float)(*s_item.S.ll_bg + (double)tot);
            }
        }
    }
}

template <int NT, int MINB>
int launch_score_multi_nt(const BatchItem *items, int n_items, const int64_t *item_begin, int64_t total, int chunk,
                          unsigned long long *counter, int w, int max_lat, int grid, cudaStream_t s) {
    const int smem = score_region<NT>() * (int)sizeof(unsigned) + max_lat * (int)sizeof(float4);
    auto kern = w == 1 ? k_score_multi<1, NT, MINB> : (w == 2 ? k_score_multi<2, NT, MINB> : k_score_multi<0, NT, MINB>);
    const int per_sm = kernel_ctas_per_sm(kern, NT, smem);
    const int ctas = grid > 0 ? std::min(grid, per_sm) : per_sm;
    const int64_t n_chunks = (total + chunk - 1) / chunk;
    const int g = (int)std::min<int64_t>((int64_t)ctas * score_sm_count(), std::max<int64_t>(n_chunks, 1));
    kern<<<g, NT, smem, s>>>(items, n_items, item_begin, total, chunk, counter);
    return g;
}

template <class PS, int NT, int MINB>
int launch_score_nt(const SceneView &sv, const Lik &L, PS P, int64_t n, float *ll, int grid, cudaStream_t s) {
    const int n_lat = sv.mesh.nc[0] + sv.mesh.nc[1] + sv.mesh.nc[2];
    const int smem = score_region<NT>() * (int)sizeof(unsigned) + n_lat * (int)sizeof(float4);
    // work counting is compiled for one launch shape only (kStatsNT, kStatsMinB)
    constexpr bool ST = NT == kStatsNT && MINB == kStatsMinB;
    auto kern = L.w == 1 ? k_score<PS, false, 1, NT, MINB> : (L.w == 2 ? k_score<PS, false, 2, NT, MINB> : k_score<PS, false, 0, NT, MINB>);
    if constexpr (ST) {
        if (sv.stats) kern = L.w == 1 ? k_score<PS, true, 1, NT, MINB> : (L.w == 2 ? k_score<PS, true, 2, NT, MINB> : k_score<PS, true, 0, NT, MINB>);
    }
    const int per_sm = kernel_ctas_per_sm(kern, NT, smem);
    // grid > 0: CTAs per SM requested by the tuning (capped by occupancy); 0: occupancy
    const int ctas = grid > 0 ? std::min(grid, per_sm) : per_sm;
    const int g = (int)std::min<int64_t>((int64_t)ctas * score_sm_count(), std::max<int64_t>(n, 1));
    if (sv.work) cudaMemsetAsync(sv.work, 0, sizeof(unsigned long long), s);
    kern<<<g, NT, smem, s>>>(sv, L, P, n, ll);
    return g;
}

}  // namespace b3d
