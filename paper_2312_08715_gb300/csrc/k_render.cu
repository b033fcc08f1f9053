// k_render.cu - scene set-up kernels of libb3d and the camera-hypothesis renderer, plus the
// launch dispatch of the fused score kernel (whose shapes live in k_score_*.cu).
//
// Set-up, once per scene (or per fixed object): the observed point cloud; the background
// z-buffer of the fixed objects, packed (depth bits << 32 | triangle id) keys built with
// 64-bit atomicMin (the nearest fragment wins, equal depths go to the smaller id); the
// per-pixel background terms l_i(bg) of the windowed Eq. 1 likelihood (Sec. III-B) and
// their FP64 sum, which let the score kernels work in proportion to a hypothesis's screen
// footprint:
//   LL_h = sum_i l_i(h) = LL_bg + sum_{i in footprint + w} (l_i(h) - l_i(bg)),
// an exact identity (the terms outside the dilated footprint are equal, bit for bit, since
// they are computed by the same device function from the same inputs).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "b3d_device.cuh"
#include "b3d_internal.h"
#include "k_score_shapes.h"

namespace b3d {

// Camera hypotheses: every scene object k at H_h P_k, H_h the hypothesised camera_from_world
// pose and P_k the object's world pose (the scene poses), rendered into the full image
// (nothing is fixed, so there is no background).
__global__ void __launch_bounds__(kThreads) k_render_camera(Cam c, const MeshView *meshes, const int *tri_base,
                                                            const float *world, int n_obj, PoseList P, int64_t n_hyp,
                                                            float *out_depth, int *out_tid) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long *zb = reinterpret_cast<unsigned long long *>(smem_raw);  // [kRegionPx]
    __shared__ float s_pose[12];
    __shared__ int s_bb[4];
    __shared__ int s_flags;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int64_t npx = (int64_t)c.W * c.H;
    const int tw = min(c.W, kRegionPx);
    const int th = max(1, kRegionPx / tw);
    for (int64_t h = blockIdx.x; h < n_hyp; h += gridDim.x) {
        for (int ty0 = 0; ty0 < c.H; ty0 += th) {
            for (int tx0 = 0; tx0 < c.W; tx0 += tw) {
                const int tx1 = min(tx0 + tw - 1, c.W - 1), ty1 = min(ty0 + th - 1, c.H - 1);
                const int zw = tx1 - tx0 + 1, zh = ty1 - ty0 + 1;
                __syncthreads();
                for (int i = tid; i < zw * zh; i += nt) zb[i] = kEmptyKey;
                for (int k = 0; k < n_obj; ++k) {
                    __syncthreads();
                    const MeshView &m = meshes[k];
                    if (tid == 0) {
                        // pose of object k in the hypothesised camera: H_h P_k (rotation rows,
                        // then translation), in the layout of pose12
                        float Hh[12];
                        pose12(P, h, Hh);
                        const float *W = world + 16 * k;
                        for (int r = 0; r < 3; ++r) {
                            for (int col = 0; col < 3; ++col)
                                s_pose[3 * r + col] = fmaf(Hh[3 * r], W[col], fmaf(Hh[3 * r + 1], W[4 + col], Hh[3 * r + 2] * W[8 + col]));
                            s_pose[9 + r] = fmaf(Hh[3 * r], W[3], fmaf(Hh[3 * r + 1], W[7], fmaf(Hh[3 * r + 2], W[11], Hh[9 + r])));
                        }
                        bool front = false;
                        s_flags = (object_bbox(m, s_pose, c, s_bb, &front) ? 1 : 0) | (front ? 4 : 0);
                    }
                    __syncthreads();
                    const bool front = (s_flags & 4) != 0;
                    const int rx0 = max(tx0, s_bb[0]), rx1 = min(tx1, s_bb[1]);
                    const int ry0 = max(ty0, s_bb[2]), ry1 = min(ty1, s_bb[3]);
                    if (!(s_flags & 1) || rx0 > rx1 || ry0 > ry1) continue;
                    const int4 *tris = front ? m.tris_surf : m.tris_full;
                    const int n_t = front ? m.n_surf : m.n_full;
                    const int cull = front ? m.closed : 0;
                    const int base = tri_base[k];
                    for (int t = tid; t < n_t; t += nt) {
                        const int4 tr = tris[t];
                        float4 A, B, C;
                        tri_screen(m, tr, s_pose, c, A, B, C);
                        const unsigned gid = (unsigned)(base + tr.w);
                        raster_tri(A, B, C, cull, rx0, rx1, ry0, ry1, c.far_z, [&](int x, int y, float z) {
                            atomicMin(&zb[(y - ty0) * zw + (x - tx0)], pack_key(z, gid));
                        });
                    }
                }
                __syncthreads();
                for (int i = tid; i < zw * zh; i += nt) {
                    const int gx = tx0 + i % zw, gy = ty0 + i / zw;
                    const int64_t gi = (int64_t)gy * c.W + gx;
                    const unsigned long long key = zb[i];
                    out_depth[h * npx + gi] = key_depth(key, 0, c.far_z);
                    if (out_tid) out_tid[h * npx + gi] = key == kEmptyKey ? -1 : (int)(unsigned)(key & 0xffffffffu);
                }
            }
        }
    }
}

// Depth only, for images whose whole z-buffer fits in shared memory: the nearest depth of
// every object at H_h P_k in 32-bit depth bits (the same nearest depth as the 64-bit keys),
// one pass over each object's triangles per hypothesis (the tiled kernel above sets every
// triangle up once per screen tile).
constexpr int kMaxCamObjects = 16;

template <int NT>
__global__ void __launch_bounds__(NT) k_render_camera_depth(Cam c, const MeshView *meshes, const float *world,
                                                            int n_obj, PoseList P, int64_t n_hyp, float *out_depth) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned *zb = reinterpret_cast<unsigned *>(smem_raw);  // [W H] depth bits
    __shared__ float s_pose[kMaxCamObjects][12];
    __shared__ int s_bb[kMaxCamObjects][4];
    __shared__ int s_flags[kMaxCamObjects];
    const int tid = threadIdx.x;
    const int npx = c.W * c.H;
    for (int64_t h = blockIdx.x; h < n_hyp; h += gridDim.x) {
        __syncthreads();
        for (int k = tid; k < n_obj; k += NT) {
            // pose of object k in the hypothesised camera, H_h P_k, in the layout of pose12
            float Hh[12];
            pose12(P, h, Hh);
            const float *W = world + 16 * k;
            for (int r = 0; r < 3; ++r) {
                for (int col = 0; col < 3; ++col)
                    s_pose[k][3 * r + col] = fmaf(Hh[3 * r], W[col], fmaf(Hh[3 * r + 1], W[4 + col], Hh[3 * r + 2] * W[8 + col]));
                s_pose[k][9 + r] = fmaf(Hh[3 * r], W[3], fmaf(Hh[3 * r + 1], W[7], fmaf(Hh[3 * r + 2], W[11], Hh[9 + r])));
            }
            bool front = false;
            s_flags[k] = (object_bbox(meshes[k], s_pose[k], c, s_bb[k], &front) ? 1 : 0) | (front ? 4 : 0);
        }
        for (int i = tid; i < npx; i += NT) zb[i] = 0xffffffffu;
        __syncthreads();
        for (int k = 0; k < n_obj; ++k) {
            if (!(s_flags[k] & 1)) continue;
            const MeshView &m = meshes[k];
            const bool front = (s_flags[k] & 4) != 0;
            const int4 *tris = front ? m.tris_surf : m.tris_full;
            const int n_t = front ? m.n_surf : m.n_full;
            const int cull = front ? m.closed : 0;
            const int rx0 = s_bb[k][0], rx1 = s_bb[k][1], ry0 = s_bb[k][2], ry1 = s_bb[k][3];
            for (int t = tid; t < n_t; t += NT) {
                float4 A, B, C;
                tri_screen(m, tris[t], s_pose[k], c, A, B, C);
                raster_tri(A, B, C, cull, rx0, rx1, ry0, ry1, c.far_z,
                           [&](int x, int y, float z) { atomicMin(&zb[y * c.W + x], __float_as_uint(z)); });
            }
        }
        __syncthreads();
        float *dst = out_depth + h * npx;
        for (int i = tid; i < npx; i += NT) {
            const unsigned v = zb[i];
            dst[i] = v == 0xffffffffu ? c.far_z : __uint_as_float(v);
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

__global__ void k_bg_depth(int64_t n, float far_z, const unsigned long long *bg, float *bgd) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = bg[i];
        bgd[i] = key_depth(k, 0, far_z);
        bgd[n + i] = key_depth(k, 1, far_z);
    }
}

struct BgSources {
    const unsigned long long *p[kMaxBgSources];
};

__global__ void k_bg_min(int64_t n, BgSources src, int n_src, unsigned long long *dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        unsigned long long v = kEmptyKey;
        for (int k = 0; k < n_src; ++k) v = min(v, src.p[k][i]);
        dst[i] = v;
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

// Background render of a fixed object with few triangles (a table, a box): one thread per
// pixel tests every triangle, so image-sized triangles spread over the whole grid. The same
// per-pixel raster_tri call as k_bg_raster, hence the same z-buffer.
constexpr int kSmallMesh = 32;
__global__ void k_bg_raster_px(Cam c, MeshView m, const float *pose16, int tri_base, unsigned long long *bg) {
    __shared__ int s_front;
    __shared__ float4 s_abc[3 * kSmallMesh];
    __shared__ unsigned s_gid[kSmallMesh];
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
    const int n_t = min(front ? m.n_surf : m.n_full, kSmallMesh);
    const int cull = front ? m.closed : 0;
    for (int t = threadIdx.x; t < n_t; t += blockDim.x) {
        const int4 tr = tris[t];
        tri_screen(m, tr, P, c, s_abc[3 * t], s_abc[3 * t + 1], s_abc[3 * t + 2]);
        s_gid[t] = (unsigned)(tri_base + tr.w);
    }
    __syncthreads();
    const int64_t n = (int64_t)c.W * c.H;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % c.W), y = (int)(i / c.W);
        for (int t = 0; t < n_t; ++t) {
            const unsigned gid = s_gid[t];
            raster_tri(s_abc[3 * t], s_abc[3 * t + 1], s_abc[3 * t + 2], cull, x, x, y, y, c.far_z,
                       [&](int xx, int yy, float z) { atomicMin(&bg[(int64_t)yy * c.W + xx], pack_key(z, gid)); });
        }
    }
}

// Per-pixel background terms: l_i of the fixed objects alone and, when requested, the
// sigma / p_out derivatives of l_i (kind 1).
// Also sums l_i (and the derivative terms) over the image in double precision, in a fixed
// order: each block reduces its pixels into part[3 block ..], and the block that finishes
// last (a ticket on *counter, which it resets) adds the block partials in block order.
// pixel_ell with the half window W compiled in and each window element's terms predicated
// instead of skipped (a skipped element adds nothing, so n and S, and the value, are
// pixel_ell's bit for bit).
template <int W, class Fetch>
__device__ __forceinline__ float pixel_ell_w(const Lik &L, const float *lut, const Cam &c, float4 q, int xi, int yi,
                                             Fetch fetch) {
    int n = 0;
    float S = 0.f;
#pragma unroll
    for (int dy = -W; dy <= W; ++dy) {
        const int yj = yi + dy;
        const bool rowok = yj >= 0 && yj < c.H;
        const float ry = ((float)yj + 0.5f - c.cy) * c.inv_fy;
#pragma unroll
        for (int dx = -W; dx <= W; ++dx) {
            const int xj = xi + dx;
            const float z = (rowok && xj >= 0 && xj < c.W) ? fetch(xj, yj) : -1.f;
            const float rx = ((float)xj + 0.5f - c.cx) * c.inv_fx;
            const float ex = fmaf(-z, rx, q.x), ey = fmaf(-z, ry, q.y), ez = q.z - z;
            const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
            if (L.kind == 0) n += (z >= 0.f && d2 <= L.r2) ? 1 : 0;
            else if (z >= 0.f) S += __expf(-d2 * L.inv2s2);
        }
    }
    return L.kind == 0 ? lut[n] : __logf(fmaf(L.bg, S, L.a));
}

__global__ void __launch_bounds__(256) k_bg_tables(SceneView S, Lik L, float *ell_bg, float *gs_bg, float *gp_bg,
                                                   float2 *qe, unsigned *bgz, double *part, unsigned *counter,
                                                   double *out) {
    __shared__ float s_lut[kMaxLut];
    __shared__ double s_red[3][256 / 32];
    __shared__ bool s_last;
    for (int i = threadIdx.x; i < L.n_lut; i += blockDim.x) s_lut[i] = L.lut[i];
    __syncthreads();
    const Cam &c = S.cam;
    const int64_t n = (int64_t)c.W * c.H;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 q = S.obs[i];
        const int y = (int)i / c.W, x = (int)i - y * c.W;  // an image has at most 2^26 pixels
        float l = 0.f, gs = 0.f, gp = 0.f;
        if (q.w != 0.f) {
            auto fetch = [&](int xj, int yj) { return key_depth(S.bg[(int64_t)yj * c.W + xj], L.miss_mode, c.far_z); };
            l = L.w == 1 ? pixel_ell_w<1>(L, s_lut, c, q, x, y, fetch)
                         : (L.w == 2 ? pixel_ell_w<2>(L, s_lut, c, q, x, y, fetch) : pixel_ell(L, s_lut, c, q, x, y, fetch));
            if (gs_bg) {
                float l1, bp;
                pixel_ell_grads(L, c, q, x, y, fetch, l1, gs, gp, bp);
            }
        }
        ell_bg[i] = l;
        // the score kernels' packed inputs: observed depth (0 where no point) with this term,
        // and the background's depth bits
        qe[i] = make_float2(q.w != 0.f ? q.z : 0.f, l);
        bgz[i] = (unsigned)(S.bg[i] >> 32);
        acc[0] += (double)l;
        if (gs_bg) {
            gs_bg[i] = gs;
            gp_bg[i] = gp;
            acc[1] += (double)gs;
            acc[2] += (double)gp;
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < 3; ++k) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_red[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = 0.0;
        for (int w = 0; w < nw; ++w) v += s_red[threadIdx.x][w];
        part[3 * blockIdx.x + threadIdx.x] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // thread t adds the partials of blocks t, t + 256, ... in order; then a fixed tree
    const volatile double *vp = part;
    for (int k = 0; k < 3; ++k) {
        double v = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) v += vp[3 * b + k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_red[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = 0.0;
        for (int w = 0; w < nw; ++w) v += s_red[threadIdx.x][w];
        out[threadIdx.x] = v;
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------

int kernel_ctas_per_sm_impl(const void *kernel, int threads, int smem) {
    static std::mutex mu;
    static std::map<std::tuple<const void *, int, int, int>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(kernel, threads, smem, dev);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    // Dynamic plus static shared memory above 48 KB needs the opt-in. The opt-in is a
    // per-kernel maximum that only ever rises here: every size a launch uses is queried
    // first, so it stays covered whatever other sizes are queried later.
    static std::map<std::pair<const void *, int>, int> opt_in;
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, kernel);
    int &cur = opt_in[std::make_pair(kernel, dev)];
    if (smem + (int)fa.sharedSizeBytes > 48 * 1024 && smem > cur) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        cur = smem;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
    per_sm = per_sm > 0 ? per_sm : 1;
    cache.emplace(key, per_sm);
    return per_sm;
}

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
    const int per_sm = kernel_ctas_per_sm(kernel, kThreads, smem);
    return (int)std::min<int64_t>((int64_t)per_sm * sm_count(), std::max<int64_t>(n, 1));
}

// grid encodes the tuning: bits 0-7 CTAs per SM (0 = as many as fit), bits 8-11 the launch
// shape (see kScoreShapes: CTA size and the CTAs per SM its registers are capped for).
template <class PS>
static int launch_score(const SceneView &sv, const Lik &L, PS P, int64_t n, float *ll, int grid, cudaStream_t s) {
    if (n <= 0) return 0;
    const int c = grid & 255;
    // work counting is compiled into one launch shape only (kStatsNT x kStatsMinB = 128 x 6,
    // checked where that shape is instantiated): use it whenever work is counted
    if (sv.stats) return launch_score_nt<PS, 128, 6>(sv, L, P, n, ll, c, s);
    switch ((grid >> 8) & 15) {
    case 1: return launch_score_nt<PS, 128, 6>(sv, L, P, n, ll, c, s);
    case 2: return launch_score_nt<PS, 64, 10>(sv, L, P, n, ll, c, s);
    case 3: return launch_score_nt<PS, 32, 16>(sv, L, P, n, ll, c, s);
    case 4: return launch_score_nt<PS, 256, 4>(sv, L, P, n, ll, c, s);
    case 5: return launch_score_nt<PS, 128, 8>(sv, L, P, n, ll, c, s);
    case 6: return launch_score_nt<PS, 64, 14>(sv, L, P, n, ll, c, s);
    case 7: return launch_score_nt<PS, 32, 24>(sv, L, P, n, ll, c, s);
    default: return launch_score_nt<PS, 256, 3>(sv, L, P, n, ll, c, s);
    }
}

int launch_score_multi(const BatchItem *items, int n_items, const int64_t *item_begin, int64_t total, int chunk,
                       unsigned long long *counter, int w, int max_lat, int grid, cudaStream_t s) {
    if (total <= 0) return 0;
    const int c = grid & 255;
    switch ((grid >> 8) & 15) {
    case 1: return launch_score_multi_nt<128, 6>(items, n_items, item_begin, total, chunk, counter, w, max_lat, c, s);
    case 2: return launch_score_multi_nt<64, 10>(items, n_items, item_begin, total, chunk, counter, w, max_lat, c, s);
    case 3: return launch_score_multi_nt<32, 16>(items, n_items, item_begin, total, chunk, counter, w, max_lat, c, s);
    case 4: return launch_score_multi_nt<256, 4>(items, n_items, item_begin, total, chunk, counter, w, max_lat, c, s);
    case 5: return launch_score_multi_nt<128, 8>(items, n_items, item_begin, total, chunk, counter, w, max_lat, c, s);
    case 6: return launch_score_multi_nt<64, 14>(items, n_items, item_begin, total, chunk, counter, w, max_lat, c, s);
    case 7: return launch_score_multi_nt<32, 24>(items, n_items, item_begin, total, chunk, counter, w, max_lat, c, s);
    default: return launch_score_multi_nt<256, 3>(items, n_items, item_begin, total, chunk, counter, w, max_lat, c, s);
    }
}

int launch_score_list(const SceneView &sv, const Lik &L, PoseList P, int64_t n, float *ll, int grid, cudaStream_t s) {
    return launch_score(sv, L, P, n, ll, grid, s);
}

int launch_score_grid(const SceneView &sv, const Lik &L, PoseGrid P, int64_t n, float *ll, int grid, cudaStream_t s) {
    return launch_score(sv, L, P, n, ll, grid, s);
}

int launch_render_camera(const Cam &cam, const MeshView *meshes, const int *tri_base, const float *world, int n_obj,
                         PoseList P, int64_t n, float *depth, int *tid, cudaStream_t s) {
    if (n <= 0) return 0;
    const int64_t npx = (int64_t)cam.W * cam.H;
    if (!tid && n_obj <= kMaxCamObjects && npx * (int64_t)sizeof(unsigned) <= 200 * 1024) {
        // depth only and the image's z-buffer fits in shared memory: one pass per hypothesis
        const int smem = (int)(npx * (int64_t)sizeof(unsigned));
        if (npx > 16384) {
            auto kern = k_render_camera_depth<1024>;
            const int per_sm = kernel_ctas_per_sm(kern, 1024, smem);
            const int g = (int)std::min<int64_t>((int64_t)per_sm * sm_count(), n);
            kern<<<g, 1024, smem, s>>>(cam, meshes, world, n_obj, P, n, depth);
            return g;
        }
        auto kern = k_render_camera_depth<256>;
        const int per_sm = kernel_ctas_per_sm(kern, 256, smem);
        const int g = (int)std::min<int64_t>((int64_t)per_sm * sm_count(), n);
        kern<<<g, 256, smem, s>>>(cam, meshes, world, n_obj, P, n, depth);
        return g;
    }
    const int smem = kRegionPx * (int)sizeof(unsigned long long);
    auto kern = k_render_camera;
    const int g = persistent_grid(kern, smem, n, 0);
    kern<<<g, kThreads, smem, s>>>(cam, meshes, tri_base, world, n_obj, P, n, depth, tid);
    return g;
}

void launch_obs_points(const Cam &cam, const float *depth, float4 *obs, cudaStream_t s) {
    const int64_t n = (int64_t)cam.W * cam.H;
    k_obs_points<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(cam, depth, obs);
}

void launch_bg_depth(int64_t n, float far_z, const unsigned long long *bg, float *bgd, cudaStream_t s) {
    k_bg_depth<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(n, far_z, bg, bgd);
}

void launch_bg_min(int64_t n, const unsigned long long *const *src, int n_src, unsigned long long *dst, cudaStream_t s) {
    BgSources b{};
    for (int k = 0; k < n_src && k < kMaxBgSources; ++k) b.p[k] = src[k];
    k_bg_min<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(n, b, std::min(n_src, kMaxBgSources), dst);
}

void launch_bg_clear(unsigned long long *bg, int64_t n, cudaStream_t s) {
    k_fill_u64<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(bg, n, kEmptyKey);
}

void launch_bg_raster(const Cam &cam, const MeshView &m, const float *pose16_dev, int tri_base,
                      unsigned long long *bg, cudaStream_t s) {
    if (m.n_full <= 0) return;
    if (m.n_full <= kSmallMesh) {
        const int64_t n = (int64_t)cam.W * cam.H;
        k_bg_raster_px<<<(int)std::min<int64_t>((n + 255) / 256, 8 * sm_count()), 256, 0, s>>>(cam, m, pose16_dev,
                                                                                              tri_base, bg);
        return;
    }
    const int warps_per_block = 8;
    const int blocks = (int)std::min<int64_t>((m.n_full + warps_per_block - 1) / warps_per_block, 8 * sm_count());
    k_bg_raster<<<blocks, 32 * warps_per_block, 0, s>>>(cam, m, pose16_dev, tri_base, bg);
}

int bg_table_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096)); }

void launch_bg_tables(const SceneView &sv, const Lik &L, float *ell_bg, float *gs_bg, float *gp_bg, float2 *qe,
                      unsigned *bgz, double *part, unsigned *counter, double *sums, cudaStream_t s) {
    const int64_t n = (int64_t)sv.cam.W * sv.cam.H;
    k_bg_tables<<<bg_table_blocks(n), 256, 0, s>>>(sv, L, ell_bg, gs_bg, gp_bg, qe, bgz, part, counter, sums);
}

}  // namespace b3d
