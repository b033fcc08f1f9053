// k_score_noise.cu - scoring under a grid of noise settings (the hierarchical noise of
// Alg. 1): each hypothesis is rendered once (render_tiles of the fused kernel)
// and every scored pixel's window is evaluated under all n_radius x n_pout settings, with
// the per-setting background terms of the fixed objects subtracted as in the single-setting
// kernel (the same per-pixel routine builds the background tables, so unchanged pixels
// cancel bit for bit). A marginal over the grid (log-sum-exp with the settings' prior log
// weights) is formed per hypothesis.
#include <cuda_runtime.h>
#include <math.h>

#include "k_score.cuh"

namespace b3d {

// l_g for every setting g = 4 i + j (internal layout; i < nr radii, j < np outlier
// probabilities) of observed point q at pixel (xi, yi), the window's rendered depths given
// by fetch (negative: no point). The window is visited in pixel_ell's order and each pair's
// squared distance is formed by pixel_ell's expression; lut holds kNoiseLut entries per g.
// WT: the half window compiled in (1, 2; 0: runtime N.w). Every window element is
// evaluated and its terms predicated (a branch on a missing point costs more than the
// element: the lanes' pixels diverge); a predicated-off element adds nothing, so the sums
// are those of the element-skipping loop.
template <int WT, class Fetch>
__device__ __forceinline__ void noise_pixel_w(const NoiseLik &N, const float *lut, const Cam &c, float4 q, int xi, int yi,
                                              Fetch fetch, float *l) {
    const int w = WT > 0 ? WT : N.w;
    int n[kMaxNoiseR];
    float S[kMaxNoiseR];
#pragma unroll
    for (int i = 0; i < kMaxNoiseR; ++i) { n[i] = 0; S[i] = 0.f; }
#pragma unroll
    for (int dy = -w; dy <= w; ++dy) {
        const int yj = yi + dy;
        const bool rowok = yj >= 0 && yj < c.H;
        const float ry = ((float)yj + 0.5f - c.cy) * c.inv_fy;
#pragma unroll
        for (int dx = -w; dx <= w; ++dx) {
            const int xj = xi + dx;
            const float z = (rowok && xj >= 0 && xj < c.W) ? fetch(xj, yj) : -1.f;
            const bool valid = z >= 0.f;
            const float rx = ((float)xj + 0.5f - c.cx) * c.inv_fx;
            const float ex = fmaf(-z, rx, q.x), ey = fmaf(-z, ry, q.y), ez = q.z - z;
            const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
#pragma unroll
            for (int i = 0; i < kMaxNoiseR; ++i) {
                if (i >= N.nr) break;
                if (N.kind == 0) n[i] += (valid & (d2 <= N.r2[i])) ? 1 : 0;
                else if (valid) S[i] += __expf(-d2 * N.inv2s2[i]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < kMaxNoiseR; ++i)
#pragma unroll
        for (int j = 0; j < kMaxNoiseP; ++j) {
            const int g = i * kMaxNoiseP + j;
            l[g] = 0.f;
            if (i < N.nr && j < N.np)
                l[g] = N.kind == 0 ? lut[g * kNoiseLut + n[i]] : __logf(fmaf(N.bg[g], S[i], N.a[j]));
        }
}

// l_g for every setting g = 4 i + j (internal layout; i < nr radii, j < np outlier
// probabilities) of observed point q at pixel (xi, yi), the window's rendered depths given
// by fetch (negative: no point). The window is visited in pixel_ell's order and each pair's
// squared distance is formed by pixel_ell's expression; lut holds kNoiseLut entries per g.
template <class Fetch>
__device__ __forceinline__ void noise_pixel(const NoiseLik &N, const float *lut, const Cam &c, float4 q, int xi, int yi,
                                            Fetch fetch, float *l) {
    if (N.w == 1) noise_pixel_w<1>(N, lut, c, q, xi, yi, fetch, l);
    else if (N.w == 2) noise_pixel_w<2>(N, lut, c, q, xi, yi, fetch, l);
    else noise_pixel_w<0>(N, lut, c, q, xi, yi, fetch, l);
}

__device__ __forceinline__ void load_noise_lut(const NoiseLik &N, float *s_lut) {
    for (int k = threadIdx.x; k < kMaxNoise * kNoiseLut; k += blockDim.x) s_lut[k] = N.lut[k];
}

// Per-pixel background terms of every setting and their double-precision sums (fixed
// order: block partials, then the last block adds them in block order).
__global__ void __launch_bounds__(256) k_bg_noise_tables(SceneView S, NoiseLik N, float *nell, double *part,
                                                         unsigned *counter, double *sums) {
    __shared__ float s_lut[kMaxNoise * kNoiseLut];
    __shared__ double s_red[kMaxNoise][256 / 32];
    __shared__ bool s_last;
    load_noise_lut(N, s_lut);
    __syncthreads();
    const Cam &c = S.cam;
    const int64_t n = (int64_t)c.W * c.H;
    double acc[kMaxNoise];
#pragma unroll
    for (int g = 0; g < kMaxNoise; ++g) acc[g] = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 q = S.obs[i];
        const int x = (int)(i % c.W), y = (int)(i / c.W);
        float l[kMaxNoise];
#pragma unroll
        for (int g = 0; g < kMaxNoise; ++g) l[g] = 0.f;
        if (q.w != 0.f)
            noise_pixel(N, s_lut, c, q, x, y,
                        [&](int xj, int yj) { return key_depth(S.bg[(int64_t)yj * c.W + xj], N.miss_mode, c.far_z); }, l);
#pragma unroll
        for (int g = 0; g < kMaxNoise; ++g) {
            if ((g >> 2) < N.nr && (g & 3) < N.np) {
                nell[(int64_t)g * n + i] = l[g];
                acc[g] += (double)l[g];
            }
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int g = 0; g < kMaxNoise; ++g) {
        double v = acc[g];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_red[g][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < kMaxNoise) {
        double v = 0.0;
        for (int w = 0; w < nw; ++w) v += s_red[threadIdx.x][w];
        part[kMaxNoise * blockIdx.x + threadIdx.x] = v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x < kMaxNoise) {
        const volatile double *vp = part;
        double v = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) v += vp[kMaxNoise * b + threadIdx.x];
        sums[threadIdx.x] = v;
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// One hypothesis per CTA iteration: render, then the noise-grid terms of the scored pixels.
// out_ll [n_hyp, nr * np] (may be NULL) in the public layout g = i * np + j; out_marg
// [n_hyp] = log sum_g exp(ll_g + logw_g).
template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    k_score_noise(SceneView S, NoiseLik N, PoseList P, int64_t n_hyp, const float *nell, const double *nsums,
                  float *out_ll, float *out_marg) {
    constexpr int REG = score_region<NT>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned *zb = reinterpret_cast<unsigned *>(smem_raw);
    float4 *lat = reinterpret_cast<float4 *>(smem_raw + REG * sizeof(unsigned));
    __shared__ float s_lut[kMaxNoise * kNoiseLut];
    __shared__ ScoreShared<NT> sh;
    __shared__ float4 s_stage[NT * kStageStride];
    __shared__ float s_red[kMaxNoise][NT / 32];
    __shared__ double s_ll[kMaxNoise];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    load_noise_lut(N, s_lut);
    const Cam &c = S.cam;
    const int64_t npx = (int64_t)c.W * c.H;
    const int G = N.nr * N.np;
    __shared__ long long s_next;
    lattice_coords(S.mesh, lat);  // ordered before use by the loop's first barrier
    int64_t h = blockIdx.x;  // then from the counter S.work, as in the single-setting kernel
    while (h < n_hyp) {
        __syncthreads();
        long long nxt = h + gridDim.x;
        if (tid == 0) {
            if (S.work) nxt = (long long)gridDim.x + (long long)atomicAdd(S.work, 1ull);
            pose12(P, h, sh.pose);
        }
        float acc[kMaxNoise];
#pragma unroll
        for (int g = 0; g < kMaxNoise; ++g) acc[g] = 0.f;
        const int nt = blockDim.x;
        render_tiles<false, NT>(
            S, N.w, N.miss_mode, sh, s_stage, zb, lat, nullptr,
            [&](const float *zd, int zx0, int zy0, int zw, int qx0, int qx1, int qy0, int qy1, int, int, int, int) {
                const int tww = qx1 - qx0 + 1, thh = qy1 - qy0 + 1;
                const int n_tile = tww * thh;
                const int dq = nt / tww, dr = nt - dq * tww;
                int y = tid / tww, x = tid - y * tww;
                for (int k = tid; k < n_tile; k += nt) {
                    const int gx = qx0 + x, gy = qy0 + y;
                    const int64_t gi = (int64_t)gy * c.W + gx;
                    const float4 q = S.obs[gi];
                    if (q.w != 0.f) {
                        float l[kMaxNoise];
                        noise_pixel(N, s_lut, c, q, gx, gy,
                                    [&](int xj, int yj) { return zd[(yj - zy0) * zw + (xj - zx0)]; }, l);
#pragma unroll
                        for (int g = 0; g < kMaxNoise; ++g)
                            if ((g >> 2) < N.nr && (g & 3) < N.np) acc[g] += l[g] - nell[(int64_t)g * npx + gi];
                    }
                    x += dr;
                    y += dq;
                    if (x >= tww) { x -= tww; ++y; }
                }
            });
        // block sums of the per-setting deltas, then ll_g = LL_bg_g + delta_g
#pragma unroll
        for (int g = 0; g < kMaxNoise; ++g) {
            const float v = warp_sum(acc[g]);
            if (lane == 0) s_red[g][wid] = v;
        }
        __syncthreads();
        if (tid < kMaxNoise && (tid >> 2) < N.nr && (tid & 3) < N.np) {
            float v = 0.f;
            for (int w = 0; w < NT / 32; ++w) v += s_red[tid][w];
            const float ll = (float)(nsums[tid] + (double)v);
            s_ll[tid] = ll;
            if (out_ll) out_ll[h * G + (tid >> 2) * N.np + (tid & 3)] = ll;
        }
        __syncthreads();
        if (tid == 0) {
            double m = -INFINITY;
            for (int g = 0; g < kMaxNoise; ++g)
                if ((g >> 2) < N.nr && (g & 3) < N.np) m = fmax(m, s_ll[g] + (double)N.logw[g]);
            double sum = 0.0;
            for (int g = 0; g < kMaxNoise; ++g)
                if ((g >> 2) < N.nr && (g & 3) < N.np) sum += exp(s_ll[g] + (double)N.logw[g] - m);
            out_marg[h] = (float)(m + log(sum));
            s_next = nxt;
        }
        __syncthreads();
        h = s_next;
    }
}

int launch_bg_noise_tables(const SceneView &sv, const NoiseLik &N, float *nell, double *part, unsigned *counter,
                           double *sums, cudaStream_t s) {
    const int64_t n = (int64_t)sv.cam.W * sv.cam.H;
    const int blocks = bg_table_blocks(n);
    k_bg_noise_tables<<<blocks, 256, 0, s>>>(sv, N, nell, part, counter, sums);
    return blocks;
}

void launch_score_noise(const SceneView &sv, const NoiseLik &N, const float *poses, int64_t n_hyp, const float *nell,
                        const double *nsums, float *out_ll, float *out_marg, cudaStream_t s) {
    constexpr int NT = 128, MINB = 4;
    const int n_lat = sv.mesh.nc[0] + sv.mesh.nc[1] + sv.mesh.nc[2];
    const int smem = score_region<NT>() * (int)sizeof(unsigned) + n_lat * (int)sizeof(float4);
    auto kern = k_score_noise<NT, MINB>;
    const int per_sm = kernel_ctas_per_sm(kern, NT, smem);
    const int g = (int)std::min<int64_t>((int64_t)per_sm * score_sm_count(), std::max<int64_t>(n_hyp, 1));
    if (sv.work) cudaMemsetAsync(sv.work, 0, sizeof(unsigned long long), s);
    kern<<<g, NT, smem, s>>>(sv, N, PoseList{poses}, n_hyp, nell, nsums, out_ll, out_marg);
}

}  // namespace b3d
