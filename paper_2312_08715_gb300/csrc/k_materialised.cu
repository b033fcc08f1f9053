// k_materialised.cu - the render-then-score form of libb3d: depth (and triangle-id) images
// of every hypothesis written to device memory, and the windowed likelihood of such images.
// Each direction is one pass over the images at close to memory bandwidth; the per-pixel
// work is confined to where an image differs from the scene's background, and the CTAs of a
// persistent grid overlap one hypothesis's streaming with another's raster or scoring.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "k_score.cuh"

namespace b3d {

// ------------------------------------------------------------------------------------------
// materialised render
// ------------------------------------------------------------------------------------------
// Depth only (k_render_fused), one hypothesis per CTA iteration: the background depths
// (misses at the far plane) are streamed into the whole image, then the object is drawn by
// the fused score kernel's renderer (merged voxel rectangles, cooperative raster, 32-bit
// depth bits) and each tile's composited depths overwrite its fragment box.
// With triangle ids (k_fill_bg, then k_render_obj): every pixel gets the background key's
// depth and id (a band of kBandPx background keys stays in shared memory while the CTA
// streams that band of many images), then the object's triangles over its screen box, with
// 64-bit atomicMin on packed (depth bits, triangle id) (the nearest fragment wins, equal
// depths go to the smaller id), overwrite the pixels where they are nearer.
constexpr int kBandPx = 4096;

inline int n_bands(int64_t npx) { return (int)((npx + kBandPx - 1) / kBandPx); }

// V = 4: 16-byte vector stores (the image size a multiple of 4 pixels and both outputs
// 16-byte aligned), else 1.
template <int V>
__global__ void __launch_bounds__(256) k_fill_bg(Cam c, const unsigned long long *bg, int64_t n_hyp, float *out_depth,
                                                 int *out_tid) {
    __shared__ __align__(16) float s_d[kBandPx];
    __shared__ __align__(16) int s_t[kBandPx];
    const int64_t npx = (int64_t)c.W * c.H, b0 = (int64_t)blockIdx.y * kBandPx;
    const int n = (int)min((int64_t)kBandPx, npx - b0);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long key = bg[b0 + i];
        s_d[i] = key_depth(key, 0, c.far_z);
        s_t[i] = key == kEmptyKey ? -1 : (int)(unsigned)(key & 0xffffffffu);
    }
    __syncthreads();
    for (int64_t h = blockIdx.x; h < n_hyp; h += gridDim.x) {
        float *dst = out_depth + h * npx + b0;
        int *tdst = out_tid ? out_tid + h * npx + b0 : nullptr;
        if (V == 4) {
            for (int k = threadIdx.x; k < n / 4; k += blockDim.x) {
                __stcs(reinterpret_cast<float4 *>(dst) + k, reinterpret_cast<const float4 *>(s_d)[k]);
                if (tdst) __stcs(reinterpret_cast<int4 *>(tdst) + k, reinterpret_cast<const int4 *>(s_t)[k]);
            }
        } else {
            for (int k = threadIdx.x; k < n; k += blockDim.x) {
                __stcs(dst + k, s_d[k]);
                if (tdst) __stcs(tdst + k, s_t[k]);
            }
        }
    }
}

template <class PS>
__global__ void __launch_bounds__(kThreads) k_render_obj(SceneView S, PS P, int64_t n_hyp, float *out_depth,
                                                         int *out_tid) {
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
        if (!(s_flags & 1)) continue;
        const float *pose = s_pose;
        const bool front = (s_flags & 4) != 0;
        const int bx0 = s_bb[0], bx1 = s_bb[1], by0 = s_bb[2], by1 = s_bb[3];
        const int4 *tris = front ? m.tris_surf : m.tris_full;
        const int n_t = front ? m.n_surf : m.n_full;
        const int cull = front ? m.closed : 0;
        const int tw = min(bx1 - bx0 + 1, kRegionPx);
        const int th = max(1, kRegionPx / tw);
        for (int ty0 = by0; ty0 <= by1; ty0 += th) {
            for (int tx0 = bx0; tx0 <= bx1; tx0 += tw) {
                const int tx1 = min(tx0 + tw - 1, bx1), ty1 = min(ty0 + th - 1, by1);
                const int zw = tx1 - tx0 + 1, nz = zw * (ty1 - ty0 + 1);
                for (int i = tid; i < nz; i += nt) zb[i] = kEmptyKey;
                __syncthreads();
                for (int t = tid; t < n_t; t += nt) {
                    const int4 tr = tris[t];
                    float4 A, B, C;
                    tri_screen(m, tr, pose, c, A, B, C);
                    const unsigned gid = (unsigned)(S.tri_base + tr.w);
                    raster_tri(A, B, C, cull, tx0, tx1, ty0, ty1, c.far_z, [&](int x, int y, float z) {
                        atomicMin(&zb[(y - ty0) * zw + (x - tx0)], pack_key(z, gid));
                    });
                }
                __syncthreads();
                const int dq = nt / zw, dr = nt - dq * zw;
                int y = tid / zw, x = tid - y * zw;
                for (int i = tid; i < nz; i += nt) {
                    const unsigned long long key = zb[i];
                    if (key != kEmptyKey) {
                        const int64_t gi = (int64_t)(ty0 + y) * c.W + (tx0 + x);
                        if (key < S.bg[gi]) {
                            out_depth[h * npx + gi] = key_depth(key, 0, c.far_z);
                            if (out_tid) out_tid[h * npx + gi] = (int)(unsigned)(key & 0xffffffffu);
                        }
                    }
                    x += dr;
                    y += dq;
                    if (x >= zw) { x -= zw; ++y; }
                }
                __syncthreads();  // the next tile clears the z-buffer this one was read from
            }
        }
    }
}

// V = 4: 16-byte vector accesses (the image size a multiple of 4 pixels and the buffers
// 16-byte aligned), else 1.
template <int NT, int MINB, int V>
__global__ void __launch_bounds__(NT, MINB) k_render_fused(SceneView S, PoseList P, int64_t n_hyp, float *out_depth) {
    constexpr int REG = score_region<NT>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned *zb = reinterpret_cast<unsigned *>(smem_raw);
    float4 *lat = reinterpret_cast<float4 *>(smem_raw + REG * sizeof(unsigned));
    __shared__ ScoreShared<NT> sh;
    __shared__ float4 s_stage[NT * kStageStride];
    const Cam &c = S.cam;
    const int tid = threadIdx.x;
    const int64_t npx = (int64_t)c.W * c.H;
    __shared__ long long s_next;
    lattice_coords(S.mesh, lat);  // ordered before use by the loop's first barrier
    int64_t h = blockIdx.x;  // then from the counter S.work when given
    while (h < n_hyp) {
        __syncthreads();
        long long nxt = h + gridDim.x;
        if (tid == 0) {
            if (S.work) nxt = (long long)gridDim.x + (long long)atomicAdd(S.work, 1ull);
            pose12(P, h, sh.pose);
        }
        float *dst = out_depth + h * npx;
        // the background first; render_tiles' barriers order these stores before the tiles'
        if (V == 4) {  // four loads in flight per thread
            const float4 *src = reinterpret_cast<const float4 *>(S.bgd);
            float4 *d4 = reinterpret_cast<float4 *>(dst);
            const int n4 = (int)(npx / 4);
            int k = tid;
            for (; k + 3 * NT < n4; k += 4 * NT) {
                const float4 a0 = __ldg(src + k), a1 = __ldg(src + k + NT), a2 = __ldg(src + k + 2 * NT),
                             a3 = __ldg(src + k + 3 * NT);
                __stcs(d4 + k, a0); __stcs(d4 + k + NT, a1); __stcs(d4 + k + 2 * NT, a2); __stcs(d4 + k + 3 * NT, a3);
            }
            for (; k < n4; k += NT) __stcs(d4 + k, __ldg(src + k));
        } else {
            for (int64_t k = tid; k < npx; k += NT) __stcs(dst + k, __ldg(S.bgd + k));
        }
        render_tiles<false, NT>(S, 0, 0, sh, s_stage, zb, lat, nullptr,
                                [&](const float *zd, int zx0, int zy0, int zw, int qx0, int qx1, int qy0, int qy1, int, int, int, int) {
                                    const int tww = qx1 - qx0 + 1, n = tww * (qy1 - qy0 + 1);
                                    const int dq = NT / tww, dr = NT - dq * tww;
                                    int y = tid / tww, x = tid - y * tww;
                                    for (int k = tid; k < n; k += NT) {
                                        const int gx = qx0 + x, gy = qy0 + y;
                                        dst[(int64_t)gy * c.W + gx] = zd[(gy - zy0) * zw + (gx - zx0)];
                                        x += dr;
                                        y += dq;
                                        if (x >= tww) { x -= tww; ++y; }
                                    }
                                });
        if (tid == 0) s_next = nxt;
        __syncthreads();
        h = s_next;
    }
}

// ------------------------------------------------------------------------------------------
// scoring of materialised depth images [n, H, W]
// ------------------------------------------------------------------------------------------
// The windowed likelihood of pixel i depends only on the depths in its window, so where an
// image's window holds the same bits as the background image (the scene's fixed objects,
// misses mapped as the likelihood maps them), l_i equals the background term exactly. One
// image per CTA iteration:
//  1. stream the image, comparing each depth's bits with the background's: the box of
//     pixels that differ;
//  2. score the pixels of box + w against their background terms (the depths of box + 2w,
//     read back through the cache, tile by tile in shared memory), with the sliding-window
//     column scorer of the fused kernel (WT = 1, 2) or pixel_ell (WT = 0):
//       LL_h = LL_bg + sum_{i in box + w} (l_i - l_i(bg)).
// MM = 1: miss mode 1 (pixels with id -1 carry no point).
__device__ __forceinline__ void box_note(int i, int W, int &x0, int &x1, int &y0, int &y1) {
    const int y = i / W, x = i - y * W;
    x0 = min(x0, x); x1 = max(x1, x); y0 = min(y0, y); y1 = max(y1, y);
}

template <int WT, int NT, int MINB, int V, int MM>
__global__ void __launch_bounds__(NT, MINB) k_score_fused(SceneView S, Lik L, const float *depth, const int *tid_in,
                                                          int64_t n_hyp, float *out_ll) {
    constexpr int REG = score_region<NT>();
    constexpr int U = 4;  // vector loads in flight per thread in the streaming pass
    __shared__ __align__(16) float zd[REG];  // depths of the tile + w
    __shared__ float s_lut[kMaxLut];
    __shared__ float s_red[NT / 32];
    __shared__ int s_box[NT / 32][4];
    const Cam &c = S.cam;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int i = tid; i < L.n_lut; i += NT) s_lut[i] = L.lut[i];
    const int w = WT > 0 ? WT : L.w;
    const int64_t npx = (int64_t)c.W * c.H;
    const float *bgd = S.bgd + (MM ? npx : 0);
    __shared__ long long s_next;
    int64_t h = blockIdx.x;  // then from the counter S.work when given
    while (h < n_hyp) {
        __syncthreads();
        long long nxt = h + gridDim.x;
        if (tid == 0 && S.work) nxt = (long long)gridDim.x + (long long)atomicAdd(S.work, 1ull);
        const float *img = depth + h * npx;
        const int *tim = MM ? tid_in + h * npx : nullptr;
        // 1. the box of pixels whose depth bits differ from the background's
        int x0 = INT32_MAX, x1 = -1, y0 = INT32_MAX, y1 = -1;
        if (V == 4) {
            const int64_t n4 = npx / 4;
            const float4 *src = reinterpret_cast<const float4 *>(img);
            const int4 *tsrc = reinterpret_cast<const int4 *>(tim);
            const float4 *gsrc = reinterpret_cast<const float4 *>(bgd);
            for (int64_t k0 = tid; k0 < n4; k0 += U * NT) {
                float4 d[U], g[U];
                int4 t[U];
#pragma unroll
                for (int j = 0; j < U; ++j) {
                    const int64_t k = k0 + j * NT;
                    const bool ok = k < n4;
                    d[j] = ok ? __ldg(src + k) : make_float4(0.f, 0.f, 0.f, 0.f);
                    g[j] = ok ? __ldg(gsrc + k) : make_float4(0.f, 0.f, 0.f, 0.f);
                    t[j] = (MM && ok) ? __ldg(tsrc + k) : make_int4(0, 0, 0, 0);
                }
#pragma unroll
                for (int j = 0; j < U; ++j) {
                    const int64_t k = k0 + j * NT;
                    const float e[4] = {t[j].x < 0 ? -1.f : d[j].x, t[j].y < 0 ? -1.f : d[j].y,
                                        t[j].z < 0 ? -1.f : d[j].z, t[j].w < 0 ? -1.f : d[j].w};
                    const float b[4] = {g[j].x, g[j].y, g[j].z, g[j].w};
#pragma unroll
                    for (int v = 0; v < 4; ++v)
                        if (__float_as_uint(e[v]) != __float_as_uint(b[v])) box_note((int)(4 * k + v), c.W, x0, x1, y0, y1);
                }
            }
        } else {
            for (int64_t k = tid; k < npx; k += NT) {
                float d = __ldg(img + k);
                if (MM && __ldg(tim + k) < 0) d = -1.f;
                if (__float_as_uint(d) != __float_as_uint(__ldg(bgd + k))) box_note((int)k, c.W, x0, x1, y0, y1);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x0 = min(x0, __shfl_xor_sync(0xffffffffu, x0, o));
            x1 = max(x1, __shfl_xor_sync(0xffffffffu, x1, o));
            y0 = min(y0, __shfl_xor_sync(0xffffffffu, y0, o));
            y1 = max(y1, __shfl_xor_sync(0xffffffffu, y1, o));
        }
        if (lane == 0) { s_box[wid][0] = x0; s_box[wid][1] = x1; s_box[wid][2] = y0; s_box[wid][3] = y1; }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < NT / 32; ++k) {
            x0 = min(x0, s_box[k][0]); x1 = max(x1, s_box[k][1]);
            y0 = min(y0, s_box[k][2]); y1 = max(y1, s_box[k][3]);
        }
        // 2. score box + w
        float acc = 0.f;
        if (x1 >= 0) {
            const int sx0 = max(x0 - w, 0), sx1 = min(x1 + w, c.W - 1);
            const int sy0 = max(y0 - w, 0), sy1 = min(y1 + w, c.H - 1);
            const int tw = min(min(sx1 - sx0 + 1, S.tile_w), REG / (1 + 2 * w) - 2 * w);
            const int th = max(1, REG / (tw + 2 * w) - 2 * w);
            for (int ty0 = sy0; ty0 <= sy1; ty0 += th) {
                for (int tx0 = sx0; tx0 <= sx1; tx0 += tw) {
                    const int tx1 = min(tx0 + tw - 1, sx1), ty1 = min(ty0 + th - 1, sy1);
                    const int zx0 = max(tx0 - w, 0), zx1 = min(tx1 + w, c.W - 1);
                    const int zy0 = max(ty0 - w, 0), zy1 = min(ty1 + w, c.H - 1);
                    const int zw = zx1 - zx0 + 1, nz = zw * (zy1 - zy0 + 1);
                    {
                        const int dq = NT / zw, dr = NT - dq * zw;
                        int y = tid / zw, x = tid - y * zw;
                        for (int i = tid; i < nz; i += NT) {
                            const int64_t gi = (int64_t)(zy0 + y) * c.W + (zx0 + x);
                            float d = img[gi];
                            if (MM && tim[gi] < 0) d = -1.f;
                            zd[i] = d;
                            x += dr;
                            y += dq;
                            if (x >= zw) { x -= zw; ++y; }
                        }
                    }
                    __syncthreads();
                    const int tww = tx1 - tx0 + 1, thh = ty1 - ty0 + 1;
                    if (WT > 0) {
                        // thread -> (column, run of rows)
                        const int nseg = max(1, NT / tww);
                        const int rps = (thh + nseg - 1) / nseg;
                        const int seg = tid / tww, col = tid - seg * tww;
                        if (seg < nseg && col < tww) {
                            const int ya = ty0 + seg * rps, yb = min(ya + rps - 1, ty1);
                            if (ya <= yb)
                                acc += score_column<WT>(S, L, s_lut, c, zd, zx0, zy0, zw, tx0 + col, ya, yb, nullptr,
                                                        nullptr);
                        }
                    } else {
                        const int n_t = tww * thh;
                        const int dq = NT / tww, dr = NT - dq * tww;
                        int y = tid / tww, x = tid - y * tww;
                        for (int k = tid; k < n_t; k += NT) {
                            const int gx = tx0 + x, gy = ty0 + y;
                            const int64_t gi = (int64_t)gy * c.W + gx;
                            const float4 q = S.obs[gi];
                            if (q.w != 0.f)
                                acc += pixel_ell(L, s_lut, c, q, gx, gy,
                                                 [&](int xj, int yj) { return zd[(yj - zy0) * zw + (xj - zx0)]; }) -
                                       S.ell_bg[gi];
                            x += dr;
                            y += dq;
                            if (x >= tww) { x -= tww; ++y; }
                        }
                    }
                    __syncthreads();
                }
            }
        }
        const float tot = block_sum(acc, s_red);
        if (tid == 0) {
            out_ll[h] = (float)(*S.ll_bg + (double)tot);
            s_next = nxt;
        }
        __syncthreads();
        h = s_next;
    }
}

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------
static bool aligned16p(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// persistent grid: as many CTAs as fit (or `grid` when > 0), at most one per item
template <class K>
static int persistent_grid(K kernel, int threads, int smem, int64_t n, int grid) {
    if (grid > 0) return (int)std::min<int64_t>(grid, std::max<int64_t>(n, 1));
    const int per_sm = kernel_ctas_per_sm(kernel, threads, smem);
    return (int)std::min<int64_t>((int64_t)per_sm * score_sm_count(), std::max<int64_t>(n, 1));
}

// Launch shape of the fused materialised kernels: 128-thread CTAs; register caps from
// launch-bound sweeps on the 160x120 tabletop stage (145,800 images): the renderer at 8
// CTAs per SM (64 registers; 3.64 against 3.77 ms at 6), the ball scorer at 10 (48
// registers, no spills; 2.32 against 2.59 ms at 6, 2.44 at 8, 2.53 at 12, where it spills).
constexpr int kMatNT = 128, kRenderMinB = 8;
template <int WT>
constexpr int score_fused_minb() { return WT == 1 ? 10 : 6; }

int launch_render_list(const SceneView &sv, PoseList P, int64_t n, float *depth, int *tid, int grid, cudaStream_t s) {
    if (n <= 0) return 0;
    const int64_t npx = (int64_t)sv.cam.W * sv.cam.H;
    if (tid) {
        const bool vec = npx % 4 == 0 && aligned16p(depth) && aligned16p(tid);
        auto fill = vec ? k_fill_bg<4> : k_fill_bg<1>;
        const int nb = n_bands(npx);
        const int per_sm = kernel_ctas_per_sm(fill, 256, 0);
        const int64_t x = std::max<int64_t>(1, ((int64_t)per_sm * score_sm_count() + nb - 1) / nb);
        fill<<<dim3((unsigned)std::min<int64_t>(x, n), (unsigned)nb), 256, 0, s>>>(sv.cam, sv.bg, n, depth, tid);
        const int smem = kRegionPx * (int)sizeof(unsigned long long);
        auto kern = k_render_obj<PoseList>;
        kern<<<persistent_grid(kern, kThreads, smem, n, grid), kThreads, smem, s>>>(sv, P, n, depth, tid);
        return 2;
    }
    const bool vec = npx % 4 == 0 && aligned16p(depth);
    const int n_lat = sv.mesh.nc[0] + sv.mesh.nc[1] + sv.mesh.nc[2];
    const int smem = score_region<kMatNT>() * (int)sizeof(unsigned) + n_lat * (int)sizeof(float4);
    auto kern = vec ? k_render_fused<kMatNT, kRenderMinB, 4> : k_render_fused<kMatNT, kRenderMinB, 1>;
    if (sv.work) cudaMemsetAsync(sv.work, 0, sizeof(unsigned long long), s);
    kern<<<persistent_grid(kern, kMatNT, smem, n, grid), kMatNT, smem, s>>>(sv, P, n, depth);
    return 1;
}

template <int WT>
static void launch_score_fused(const SceneView &sv, const Lik &L, const float *depth, const int *tid, int64_t n,
                               float *ll, int grid, cudaStream_t s) {
    const int64_t npx = (int64_t)sv.cam.W * sv.cam.H;
    const bool mm = L.miss_mode == 1;
    const bool vec = npx % 4 == 0 && aligned16p(depth) && (!mm || aligned16p(tid));
    constexpr int MB = score_fused_minb<WT>();
    auto kern = vec ? (mm ? k_score_fused<WT, kMatNT, MB, 4, 1> : k_score_fused<WT, kMatNT, MB, 4, 0>)
                    : (mm ? k_score_fused<WT, kMatNT, MB, 1, 1> : k_score_fused<WT, kMatNT, MB, 1, 0>);
    if (sv.work) cudaMemsetAsync(sv.work, 0, sizeof(unsigned long long), s);
    kern<<<persistent_grid(kern, kMatNT, 0, n, grid), kMatNT, 0, s>>>(sv, L, depth, tid, n, ll);
}

int launch_score_depth(const SceneView &sv, const Lik &L, const float *depth, const int *tid, int64_t n, float *ll,
                       int grid, cudaStream_t s) {
    if (n <= 0) return 0;
    if (L.w == 1) launch_score_fused<1>(sv, L, depth, tid, n, ll, grid, s);
    else if (L.w == 2) launch_score_fused<2>(sv, L, depth, tid, n, ll, grid, s);
    else launch_score_fused<0>(sv, L, depth, tid, n, ll, grid, s);
    return 1;
}

}  // namespace b3d
