// b3d_device.cuh - device helpers shared by the render/score and gradient kernels of
// libb3d. Everything here is inline so that every kernel evaluates the same expressions in
// the same order: a pixel whose inputs are unchanged gets bit-identical terms everywhere.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "b3d_internal.h"

namespace b3d {

// ------------------------------------------------------------------------------------------
// small helpers
// ------------------------------------------------------------------------------------------

__device__ __forceinline__ float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum over kThreads threads; result valid in thread 0. Uses red[kThreads/32].
__device__ __forceinline__ float block_sum(float v, float *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum(v);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    v = 0.f;
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.f;
        v = warp_sum(v);
    }
    return v;
}

__device__ __forceinline__ void pose12(const PoseList &P, int64_t h, float *o) {
    const float *p = P.p + 16 * h;
    o[0] = p[0]; o[1] = p[1]; o[2] = p[2];
    o[3] = p[4]; o[4] = p[5]; o[5] = p[6];
    o[6] = p[8]; o[7] = p[9]; o[8] = p[10];
    o[9] = p[3]; o[10] = p[7]; o[11] = p[11];
}

// Coarse-to-fine grid: h = ((ir * n + ix) * n + iy) * n + iz; R_h = R_c R_ir and
// t_h = t_c + G (o_ix, o_iy, o_iz), o_i = (i - c) step with c = (n-1)/2 (odd n) or n/2.
__device__ __forceinline__ void pose12(const PoseGrid &P, int64_t h, float *o) {
    const int n = P.n;
    const int64_t n2 = (int64_t)n * n, n3 = n2 * n;
    int ir, ix, iy, iz;
    if (h <= INT32_MAX && n3 <= INT32_MAX) {  // the same quotients in 32-bit arithmetic
        const unsigned hh = (unsigned)h, m2 = (unsigned)n2, m3 = (unsigned)n3, m1 = (unsigned)n;
        const unsigned qr = hh / m3;
        unsigned r = hh - qr * m3;
        const unsigned qx = r / m2;
        r -= qx * m2;
        const unsigned qy = r / m1;
        ir = (int)qr; ix = (int)qx; iy = (int)qy; iz = (int)(r - qy * m1);
    } else {
        ir = (int)(h / n3);
        int64_t rem = h - (int64_t)ir * n3;
        ix = (int)(rem / n2);
        rem -= (int64_t)ix * n2;
        iy = (int)(rem / n);
        iz = (int)(rem - (int64_t)iy * n);
    }
    const int c = (n & 1) ? (n - 1) / 2 : n / 2;
    const float ox = (float)(ix - c) * P.step, oy = (float)(iy - c) * P.step, oz = (float)(iz - c) * P.step;
    const float *C = P.centre;
    const float *Rk = P.rot + 9 * ir;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int b = 0; b < 3; ++b)
            o[3 * a + b] = fmaf(C[4 * a + 0], Rk[b], fmaf(C[4 * a + 1], Rk[3 + b], C[4 * a + 2] * Rk[6 + b]));
        o[9 + a] = C[4 * a + 3] + fmaf(P.G[3 * a + 0], ox, fmaf(P.G[3 * a + 1], oy, P.G[3 * a + 2] * oz));
    }
}

// Camera-frame point of an object-frame point under a 12-float pose.
__device__ __forceinline__ void xform(const float *P, float x, float y, float z, float &cx, float &cy, float &cz) {
    cx = fmaf(P[0], x, fmaf(P[1], y, fmaf(P[2], z, P[9])));
    cy = fmaf(P[3], x, fmaf(P[4], y, fmaf(P[5], z, P[10])));
    cz = fmaf(P[6], x, fmaf(P[7], y, fmaf(P[8], z, P[11])));
}

// Screen vertex (u, v, 1/z, z); 1/z = -1 marks a vertex in front of the near plane.
__device__ __forceinline__ float4 project(const float *P, float4 v, const Cam &c) {
    float x, y, z;
    xform(P, v.x, v.y, v.z, x, y, z);
    if (!(z >= c.near_z)) return make_float4(0.f, 0.f, -1.f, z);
    const float iz = 1.0f / z;
    return make_float4(fmaf(c.fx, x * iz, c.cx), fmaf(c.fy, y * iz, c.cy), iz, z);
}

// Edge function of the directed edge a->b at p, evaluated from the lexicographically
// smaller endpoint so that the two triangles sharing an edge get exactly opposite values
// (no pixel centre falls through a shared edge, none is claimed twice except at e = 0).
__device__ __forceinline__ float edge_fn(float ax, float ay, float bx, float by, float px, float py) {
    const bool sw = (bx < ax) || (bx == ax && by < ay);
    const float x0 = sw ? bx : ax, y0 = sw ? by : ay, x1 = sw ? ax : bx, y1 = sw ? ay : by;
    const float e = fmaf(x1 - x0, py - y0, -((y1 - y0) * (px - x0)));
    return sw ? -e : e;
}

__device__ __forceinline__ unsigned long long pack_key(float z, unsigned id) {
    return ((unsigned long long)__float_as_uint(z) << 32) | (unsigned long long)id;
}

__device__ __forceinline__ float key_depth(unsigned long long k, int miss_mode, float far_z) {
    return k == kEmptyKey ? (miss_mode ? -1.f : far_z) : __uint_as_float((unsigned)(k >> 32));
}

// Rasterise one triangle (screen vertices A, B, C as (u, v, 1/z, z)) over the pixel centres
// in [rx0, rx1] x [ry0, ry1], calling store(x, y, z) for each fragment. Coverage: all three
// edge functions, oriented by the sign of the signed area, are >= 0. Depth:
// perspective-correct, 1/z interpolated with screen barycentrics. With cull set, triangles
// whose screen area is not negative (turned away from the camera) are skipped.
// tests (optional) counts the pixel-centre coverage tests made.
template <class Store>
__device__ __forceinline__ void raster_tri(float4 A, float4 B, float4 C, int cull, int rx0, int rx1, int ry0, int ry1,
                                           float far_z, Store store, unsigned long long *tests = nullptr) {
    if (A.z < 0.f || B.z < 0.f || C.z < 0.f) return;
    const float area = edge_fn(A.x, A.y, B.x, B.y, C.x, C.y);
    if (cull ? !(area < 0.f) : !(area != 0.f)) return;
    const float umin = fminf(A.x, fminf(B.x, C.x)), umax = fmaxf(A.x, fmaxf(B.x, C.x));
    const float vmin = fminf(A.y, fminf(B.y, C.y)), vmax = fmaxf(A.y, fmaxf(B.y, C.y));
    const int x0 = (int)ceilf(fmaxf(umin - 0.5f, (float)rx0)), x1 = (int)floorf(fminf(umax - 0.5f, (float)rx1));
    const int y0 = (int)ceilf(fmaxf(vmin - 0.5f, (float)ry0)), y1 = (int)floorf(fminf(vmax - 0.5f, (float)ry1));
    if (x0 > x1 || y0 > y1) return;
    if (tests) *tests += (unsigned long long)((x1 - x0 + 1) * (y1 - y0 + 1));
    const float s = area > 0.f ? 1.f : -1.f;
    for (int y = y0; y <= y1; ++y) {
        const float py = (float)y + 0.5f;
        for (int x = x0; x <= x1; ++x) {
            const float px = (float)x + 0.5f;
            const float e0 = edge_fn(A.x, A.y, B.x, B.y, px, py);
            const float e1 = edge_fn(B.x, B.y, C.x, C.y, px, py);
            const float e2 = edge_fn(C.x, C.y, A.x, A.y, px, py);
            if (s * e0 < 0.f || s * e1 < 0.f || s * e2 < 0.f) continue;
            const float den = fmaf(e1, A.z, fmaf(e2, B.z, e0 * C.z));
            const float z = area / den;
            if (!(z <= far_z)) continue;
            store(x, y, z);
        }
    }
}

// Screen bounding box (pixel-centre index ranges, clipped, 1 px margin) of the object's
// bounding box under pose P; the whole image if a corner is in front of the near plane
// (*front = false then: the near plane may cut the object open). Returns false if it
// misses the image or the mesh is empty.
__device__ __forceinline__ bool object_bbox(const MeshView &m, const float *P, const Cam &c, int *bb,
                                            bool *front = nullptr) {
    if (front) *front = false;
    if (m.n_full <= 0) return false;
    float umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY;
    bool all_front = true;
    for (int k = 0; k < 8; ++k) {
        const float ox = (k & 1) ? m.hi[0] : m.lo[0], oy = (k & 2) ? m.hi[1] : m.lo[1], oz = (k & 4) ? m.hi[2] : m.lo[2];
        float x, y, z;
        xform(P, ox, oy, oz, x, y, z);
        if (!(z >= c.near_z)) { all_front = false; break; }
        const float u = fmaf(c.fx, x / z, c.cx), v = fmaf(c.fy, y / z, c.cy);
        umin = fminf(umin, u); umax = fmaxf(umax, u);
        vmin = fminf(vmin, v); vmax = fmaxf(vmax, v);
    }
    if (front) *front = all_front;
    if (!all_front) {
        bb[0] = 0; bb[1] = c.W - 1; bb[2] = 0; bb[3] = c.H - 1;
        return true;
    }
    const float lo_u = fmaxf(umin - 0.5f, -2.f), hi_u = fminf(umax - 0.5f, (float)c.W + 1.f);
    const float lo_v = fmaxf(vmin - 0.5f, -2.f), hi_v = fminf(vmax - 0.5f, (float)c.H + 1.f);
    bb[0] = max((int)ceilf(lo_u) - 1, 0);
    bb[1] = min((int)floorf(hi_u) + 1, c.W - 1);
    bb[2] = max((int)ceilf(lo_v) - 1, 0);
    bb[3] = min((int)floorf(hi_v) + 1, c.H - 1);
    return bb[0] <= bb[1] && bb[2] <= bb[3];
}

// Screen vertices of triangle tr (welded vertex indices) under pose P.
__device__ __forceinline__ void tri_screen(const MeshView &m, int4 tr, const float *P, const Cam &c, float4 &A, float4 &B,
                                           float4 &C) {
    A = project(P, m.verts[tr.x], c);
    B = project(P, m.verts[tr.y], c);
    C = project(P, m.verts[tr.z], c);
}

// l_i of observed point q at pixel (xi, yi): the (2w+1)^2 window over rendered depths given
// by fetch(x, y) (negative = no point). Kind 0 counts points inside the ball and looks the
// term up in lut; kind 1 sums Gaussian kernels. Explicit fma order: the same inputs give
// the same bits in every kernel that calls this.
template <class Fetch>
__device__ __forceinline__ float pixel_ell(const Lik &L, const float *lut, const Cam &c, float4 q, int xi, int yi,
                                           Fetch fetch) {
    int n = 0;
    float S = 0.f;
    for (int dy = -L.w; dy <= L.w; ++dy) {
        const int yj = yi + dy;
        if (yj < 0 || yj >= c.H) continue;
        const float ry = ((float)yj + 0.5f - c.cy) * c.inv_fy;
        for (int dx = -L.w; dx <= L.w; ++dx) {
            const int xj = xi + dx;
            if (xj < 0 || xj >= c.W) continue;
            const float z = fetch(xj, yj);
            if (z < 0.f) continue;
            const float rx = ((float)xj + 0.5f - c.cx) * c.inv_fx;
            const float ex = fmaf(-z, rx, q.x), ey = fmaf(-z, ry, q.y), ez = q.z - z;
            const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
            if (L.kind == 0) n += d2 <= L.r2 ? 1 : 0;
            else S += __expf(-d2 * L.inv2s2);
        }
    }
    return L.kind == 0 ? lut[n] : __logf(fmaf(L.bg, S, L.a));
}


// Kind-1 value and derivatives of pixel i in one pass over its window. With
// E_i = sum_j exp(-d_ij^2 / (2 s^2)) (accumulated exactly as pixel_ell does, so l equals
// pixel_ell's value bit for bit), S_i = (2 pi s^2)^(-3/2) E_i and p_i = a + b S_i:
//   l  = log p_i
//   gs = d l / d s     = b (2 pi s^2)^(-3/2) sum_j exp(..) (d_ij^2 / s^2 - 3) / (s p_i)
//   gp = d l / d p_out = (1 / V - S_i / K) / p_i
//   bp = b / p_i (the weight of pixel i in d LL / d z_j).
// The per-pixel results of pixel_ell_grads from its window sums E and D (also used by the
// gradient kernel's unrolled window loop, so both give the same bits).
__device__ __forceinline__ void grads_from_sums(const Lik &L, float E, float D, float &l, float &gs, float &gp,
                                                float &bp) {
    const float p = fmaf(L.bg, E, L.a);
    l = __logf(p);
    const float ip = 1.f / p;
    gs = L.bg * D / L.s * ip;
    gp = fmaf(-L.gnorm * E, L.inv_K, L.inv_V) * ip;
    bp = L.b * ip;
}

template <class Fetch>
__device__ __forceinline__ void pixel_ell_grads(const Lik &L, const Cam &c, float4 q, int xi, int yi, Fetch fetch,
                                                float &l, float &gs, float &gp, float &bp) {
    float E = 0.f, D = 0.f;
    for (int dy = -L.w; dy <= L.w; ++dy) {
        const int yj = yi + dy;
        if (yj < 0 || yj >= c.H) continue;
        const float ry = ((float)yj + 0.5f - c.cy) * c.inv_fy;
        for (int dx = -L.w; dx <= L.w; ++dx) {
            const int xj = xi + dx;
            if (xj < 0 || xj >= c.W) continue;
            const float z = fetch(xj, yj);
            if (z < 0.f) continue;
            const float rx = ((float)xj + 0.5f - c.cx) * c.inv_fx;
            const float ex = fmaf(-z, rx, q.x), ey = fmaf(-z, ry, q.y), ez = q.z - z;
            const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
            const float e = __expf(-d2 * L.inv2s2);
            E += e;
            D = fmaf(e, fmaf(d2, L.inv_s2, -3.f), D);
        }
    }
    grads_from_sums(L, E, D, l, gs, gp, bp);
}

}  // namespace b3d
