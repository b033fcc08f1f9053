// k_c2f.cu - coarse-to-fine kernels of libb3d: rotation sets and grid expansion (the
// partitions Pi_t of Sec. III-B), fused log-sum-exp + categorical resampling (the next
// region is drawn with probability proportional to its score), and the per-stage
// centre selection / final uniform-in-cell jitter.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "b3d_device.cuh"
#include "b3d_internal.h"

namespace b3d {

// ------------------------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11): ten rounds of two 64x64->128 multiplies with a Weyl-sequence key schedule.
// ------------------------------------------------------------------------------------------
struct U64x4 {
    unsigned long long v[4];
};

__device__ __forceinline__ U64x4 philox4x64(unsigned long long c0, unsigned long long c1, unsigned long long c2,
                                            unsigned long long c3, unsigned long long k0, unsigned long long k1) {
    const unsigned long long M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const unsigned long long hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const unsigned long long n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    U64x4 o;
    o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
    return o;
}

// Top 24 bits as a uniform in [0, 1), exact in float.
__device__ __forceinline__ float uniform24(unsigned long long x) { return (float)(x >> 40) * (1.0f / 16777216.0f); }

// ------------------------------------------------------------------------------------------
// rotation sets (computed in double on the device, stored as float)
// ------------------------------------------------------------------------------------------
__device__ void axis_angle(double kx, double ky, double kz, double ang, float *R) {
    const double nrm = sqrt(kx * kx + ky * ky + kz * kz);
    kx /= nrm; ky /= nrm; kz /= nrm;
    const double c = cos(ang), s = sin(ang), C = 1.0 - c;
    R[0] = (float)(c + kx * kx * C);      R[1] = (float)(kx * ky * C - kz * s); R[2] = (float)(kx * kz * C + ky * s);
    R[3] = (float)(ky * kx * C + kz * s); R[4] = (float)(c + ky * ky * C);      R[5] = (float)(ky * kz * C - kx * s);
    R[6] = (float)(kz * kx * C - ky * s); R[7] = (float)(kz * ky * C + kx * s); R[8] = (float)(c + kz * kz * C);
}

// frac(1/2 + k a) with A = round(2^64 a): the top 53 bits of 2^63 + k A (mod 2^64), exact
__device__ __forceinline__ double weyl_u(unsigned long long A, int k) {
    const unsigned long long x = 0x8000000000000000ull + (unsigned long long)k * A;
    return (double)(x >> 11) * (1.0 / 9007199254740992.0);
}

__global__ void k_rotation_set(int kind, int n, double rot_max, float *out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double phi = (1.0 + sqrt(5.0)) / 2.0, pi = 3.14159265358979323846;
    const double z = 1.0 - (2.0 * k + 1.0) / n;
    const double rho = sqrt(fmax(0.0, 1.0 - z * z));
    const double ang = 2.0 * pi * k / phi;
    const double dx = rho * cos(ang), dy = rho * sin(ang), dz = z;
    float *R = out + 9 * k;
    const float I[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    if (kind == 0) {
        // minimal arc from +z to d: axis +z x d = (-dy, dx, 0), angle atan2(|axis|, dz)
        const double sn = sqrt(dx * dx + dy * dy);
        if (sn == 0.0) {
            if (dz > 0) for (int i = 0; i < 9; ++i) R[i] = I[i];
            else axis_angle(1.0, 0.0, 0.0, pi, R);
        } else {
            axis_angle(-dy, dx, 0.0, atan2(sn, dz), R);
        }
    } else {
        // low-discrepancy set uniform in the ball of rotation vectors of radius rot_max:
        // member 0 the identity, member k the 3-D R-sequence point frac(1/2 + k (1/g, 1/g^2,
        // 1/g^3)) (g^4 = g + 1) mapped volume-preservingly onto the ball (radius cbrt(u0),
        // z = 1 - 2 u1, azimuth 2 pi u2); the sequence in exact 64-bit fixed point
        const double u0 = weyl_u(0xd1b54a32d192ed04ull, k), u1 = weyl_u(0xabc98388fb8fac03ull, k);
        const double u2 = weyl_u(0x8cb92ba72f3d8dd7ull, k);
        const double theta = rot_max * cbrt(u0);
        const double ez = 1.0 - 2.0 * u1, es = sqrt(fmax(0.0, 1.0 - ez * ez));
        if (k == 0 || theta == 0.0) for (int i = 0; i < 9; ++i) R[i] = I[i];
        else axis_angle(es * cos(2.0 * pi * u2), es * sin(2.0 * pi * u2), ez, theta, R);
    }
}

// ------------------------------------------------------------------------------------------
// grid expansion to explicit poses, centre set-up
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void write_pose16(const float *o, float *P) {
    P[0] = o[0]; P[1] = o[1]; P[2] = o[2]; P[3] = o[9];
    P[4] = o[3]; P[5] = o[4]; P[6] = o[5]; P[7] = o[10];
    P[8] = o[6]; P[9] = o[7]; P[10] = o[8]; P[11] = o[11];
    P[12] = 0.f; P[13] = 0.f; P[14] = 0.f; P[15] = 1.f;
}

__global__ void k_expand(PoseGrid P, int64_t n, float *poses) {
    for (int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h < n; h += (int64_t)gridDim.x * blockDim.x) {
        float o[12];
        pose12(P, h, o);
        write_pose16(o, poses + 16 * h);
    }
}

struct F16 {
    float v[16];
};

__global__ void k_set16(float *dst, F16 src) {
    if (threadIdx.x < 16) dst[threadIdx.x] = src.v[threadIdx.x];
}

// ------------------------------------------------------------------------------------------
// fused log-sum-exp + categorical resampling
// ------------------------------------------------------------------------------------------
constexpr int kLseThreads = 256;
constexpr int kLseMaxBlocks = 1024;
constexpr int kLseMinChunk = 512;

__device__ __forceinline__ float lse_weight(float x, float m) {
    return (x == x && m > -INFINITY) ? __expf(x - m) : 0.f;  // NaN and -inf entries weigh 0
}

// Phase A (every block): chunk max m_b and s_b = sum exp(ll - m_b) -> part[b].
// Phase B (the last block to finish, by an atomic ticket; no block waits on another):
// global max M, S = sum_b s_b exp(m_b - M), chunk prefix sums, logZ = M + log S, then each
// draw k: t = u_k S, chunk by binary search on the chunk prefix, element by a warp scan of
// exp(ll - M) within the chunk (first inclusive prefix > t). The counter is reset for the
// next launch.
struct LseShared {
    float red[kLseThreads / 32];
    float w[kLseMaxBlocks];
    float pre[kLseMaxBlocks];  // exclusive prefix of w
    float cp[kLseThreads / 32][kLseMinChunk];         // per warp: inclusive prefix of one chunk,
    float cl[kLseThreads / 32][kLseMinChunk];         // its scores
    unsigned cm[kLseThreads / 32][kLseMinChunk / 32];  // and which of its weights are positive
    float M, S;
    bool last;
};

// Block bid of nb blocks working on one score vector (see k_lse_resample). With a shard
// (the vector is one rank's contiguous part of a categorical split over ranks), draw k
// belongs to this rank when its uniform u falls in [before, before + mass), the rank's share
// of the probability; its index within the vector is then the inverse CDF at
// (u - before) / mass, which is the global inverse CDF at u in exact arithmetic. Draws of
// other ranks get idx -1; logq uses the global normaliser; idx is offset by base.
__device__ __forceinline__ void lse_body(LseShared &sh, int bid, int nb, const float *ll, int64_t n, int chunk, int m,
                                         unsigned long long seed, int stage, float2 *part, unsigned *counter,
                                         float *logz, int *idx, float *logq, int *err,
                                         const LseShard *shard = nullptr) {
    float *s_red = sh.red, *s_w = sh.w, *s_pre = sh.pre;
    float &s_M = sh.M, &s_S = sh.S;
    bool &s_last = sh.last;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = kLseThreads / 32;
    const int64_t b0 = (int64_t)bid * chunk, b1 = std::min<int64_t>(n, b0 + chunk);

    // phase A
    float mx = -INFINITY;
    for (int64_t i = b0 + tid; i < b1; i += kLseThreads) mx = fmaxf(mx, ll[i]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) s_red[wid] = mx;
    __syncthreads();
    if (tid == 0) {
        float v = -INFINITY;
        for (int k = 0; k < nw; ++k) v = fmaxf(v, s_red[k]);
        s_M = v;
    }
    __syncthreads();
    const float mb = s_M;
    float sm = 0.f;
    for (int64_t i = b0 + tid; i < b1; i += kLseThreads) sm += lse_weight(ll[i], mb);
    for (int o = 16; o > 0; o >>= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
    __syncthreads();
    if (lane == 0) s_red[wid] = sm;
    __syncthreads();
    if (tid == 0) {
        float v = 0.f;
        for (int k = 0; k < nw; ++k) v += s_red[k];
        part[bid] = make_float2(mb, v);
        __threadfence();
        const unsigned ticket = atomicAdd(counter, 1u);
        s_last = ticket == (unsigned)nb - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();

    // phase B
    const int B = nb;
    float gm = -INFINITY;
    for (int b = tid; b < B; b += kLseThreads) gm = fmaxf(gm, __ldcg(&part[b].x));
    for (int o = 16; o > 0; o >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, o));
    if (lane == 0) s_red[wid] = gm;
    __syncthreads();
    if (tid == 0) {
        float v = -INFINITY;
        for (int k = 0; k < nw; ++k) v = fmaxf(v, s_red[k]);
        s_M = v;
    }
    __syncthreads();
    const float M = s_M;
    for (int b = tid; b < B; b += kLseThreads) {
        const float2 p = __ldcg(&part[b]);
        s_w[b] = (p.x > -INFINITY && M > -INFINITY) ? p.y * __expf(p.x - M) : 0.f;
    }
    __syncthreads();
    {
        // exclusive prefix of the chunk weights in a fixed order: every thread sums a run of
        // consecutive chunks, the run totals are scanned (warp scans, then the warps in
        // order), and each thread writes its run's prefixes
        const int R = (B + kLseThreads - 1) / kLseThreads;
        const int r0 = min(tid * R, B), r1 = min(r0 + R, B);
        float run = 0.f;
        for (int b = r0; b < r1; ++b) run += s_w[b];
        float inc = run;
        for (int o = 1; o < 32; o <<= 1) {
            const float up = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += up;
        }
        if (lane == 31) s_red[wid] = inc;
        __syncthreads();
        if (tid == 0) {
            float acc = 0.f;
            for (int k = 0; k < nw; ++k) {
                const float v = s_red[k];
                s_red[k] = acc;
                acc += v;
            }
            s_S = acc;
            *counter = 0u;
            *logz = (M > -INFINITY) ? M + __logf(acc) : -INFINITY;
            if (!(M > -INFINITY) && m > 0 && !shard) atomicOr(err, 4);
        }
        __syncthreads();
        float acc = s_red[wid] + (inc - run);
        for (int b = r0; b < r1; ++b) {
            s_pre[b] = acc;
            acc += s_w[b];
        }
    }
    __syncthreads();
    const float S = s_S;
    const float Z = shard ? shard->logz : ((M > -INFINITY) ? M + __logf(S) : -INFINITY);
    const long long ibase = shard ? shard->base : 0;
    int cached = -1;  // the chunk whose prefix this warp holds
    for (int k = wid; k < m; k += nw) {
        if (!(M > -INFINITY)) {
            if (lane == 0) { idx[k] = -1; logq[k] = -INFINITY; }
            continue;
        }
        const U64x4 r = philox4x64((unsigned long long)k, (unsigned long long)(unsigned)stage, 0ull, 0ull, seed, 0ull);
        float t;
        if (shard) {
            const double u = (double)(r.v[0] >> 40) * (1.0 / 16777216.0);  // the same 24-bit uniform, exact
            if (!(u >= shard->before && u < shard->before + shard->mass)) {
                if (lane == 0) { idx[k] = -1; logq[k] = -INFINITY; }
                continue;
            }
            t = (float)((u - shard->before) / shard->mass) * S;
        } else {
            t = uniform24(r.v[0]) * S;
        }
        // first chunk whose inclusive prefix exceeds t; if rounding leaves none, the last
        // chunk with weight
        int lo = 0, hi = B - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_pre[mid] + s_w[mid] > t) hi = mid; else lo = mid + 1;
        }
        int b = lo;
        if (!(s_pre[b] + s_w[b] > t)) {
            b = B - 1;
            while (b > 0 && s_w[b] == 0.f) --b;
        }
        const int64_t e0 = (int64_t)b * chunk, e1 = std::min<int64_t>(n, e0 + chunk);
        if (chunk <= kLseMinChunk) {
            // the chunk's inclusive prefix (the same groups of 32 and the same warp scans as
            // the streaming search below, so the same sums) and its positive weights, kept
            // per warp: further draws in the chunk only search shared memory
            float *cp = sh.cp[wid], *cl = sh.cl[wid];
            unsigned *cm = sh.cm[wid];
            const int len = (int)(e1 - e0);
            if (b != cached) {
                constexpr int G = kLseMinChunk / 32;
                float lv[G];  // every load of the chunk in flight before the scan
#pragma unroll
                for (int j = 0; j < G; ++j) {
                    const int i = 32 * j + lane;
                    lv[j] = i < len ? __ldcg(&ll[e0 + i]) : -INFINITY;
                }
                float c1 = s_pre[b];
#pragma unroll
                for (int j = 0; j < G; ++j) {
                    const int i = 32 * j + lane;
                    if (32 * j >= len) break;
                    const float wv = i < len ? lse_weight(lv[j], M) : 0.f;
                    float inc = wv;
                    for (int o = 1; o < 32; o <<= 1) {
                        const float up = __shfl_up_sync(0xffffffffu, inc, o);
                        if (lane >= o) inc += up;
                    }
                    if (i < len) {
                        cp[i] = c1 + inc;
                        cl[i] = lv[j];
                    }
                    const unsigned pos = __ballot_sync(0xffffffffu, i < len && wv > 0.f);
                    if (lane == 0) cm[j] = pos;
                    c1 += __shfl_sync(0xffffffffu, inc, 31);
                }
                cached = b;
                __syncwarp();
            }
            if (lane == 0) {
                // first element with a positive weight whose inclusive prefix exceeds t (the
                // prefix never decreases); if rounding leaves none, the last positive one
                int lo = 0, hi = len;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (cp[mid] > t) hi = mid; else lo = mid + 1;
                }
                int found = -1;
                for (int i = lo; i < len; ++i)
                    if ((cm[i >> 5] >> (i & 31)) & 1u) { found = i; break; }
                if (found < 0)
                    for (int i = len - 1; i >= 0; --i)
                        if ((cm[i >> 5] >> (i & 31)) & 1u) { found = i; break; }
                idx[k] = found >= 0 ? (int)(ibase + e0 + found) : -1;
                logq[k] = found >= 0 ? cl[found] - Z : -INFINITY;
            }
            __syncwarp();
            continue;
        }
        float c0 = s_pre[b];
        int64_t found = -1, last_pos = -1;
        // 128 elements per pass, four independent loads in flight per lane
        for (int64_t base = e0; base < e1 && found < 0; base += 128) {
            float wv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t i = base + 32 * u + lane;
                wv[u] = i < e1 ? lse_weight(__ldcg(&ll[i]), M) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t i = base + 32 * u + lane;
                float inc = wv[u];
                for (int o = 1; o < 32; o <<= 1) {
                    const float up = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += up;
                }
                const unsigned hit = __ballot_sync(0xffffffffu, i < e1 && wv[u] > 0.f && c0 + inc > t);
                const unsigned pos = __ballot_sync(0xffffffffu, i < e1 && wv[u] > 0.f);
                if (found < 0) {
                    if (pos) last_pos = base + 32 * u + 31 - __clz(pos);
                    if (hit) found = base + 32 * u + __ffs(hit) - 1;
                }
                c0 += __shfl_sync(0xffffffffu, inc, 31);
            }
        }
        if (found < 0) found = last_pos;
        if (lane == 0) {
            idx[k] = found >= 0 ? (int)(ibase + found) : -1;
            logq[k] = found >= 0 ? __ldcg(&ll[found]) - Z : -INFINITY;
        }
    }
}

__global__ void __launch_bounds__(kLseThreads) k_lse_resample(const float *ll, int64_t n, int chunk, int m,
                                                              unsigned long long seed, int stage, float2 *part,
                                                              unsigned *counter, float *logz, int *idx, float *logq,
                                                              int *err) {
    __shared__ LseShared sh;
    lse_body(sh, blockIdx.x, gridDim.x, ll, n, chunk, m, seed, stage, part, counter, logz, idx, logq, err);
}

// One rank's shard of a categorical split over ranks (see lse_body).
__global__ void __launch_bounds__(kLseThreads) k_lse_shard(const float *ll, int64_t n, int chunk, int m,
                                                           unsigned long long seed, int stage, LseShard shard,
                                                           float2 *part, unsigned *counter, float *logz, int *idx,
                                                           float *logq, int *err) {
    __shared__ LseShared sh;
    lse_body(sh, blockIdx.x, gridDim.x, ll, n, chunk, m, seed, stage, part, counter, logz, idx, logq, err, &shard);
}

// Batched: the blocks of every scene's score vector in one grid; block_begin[i] is the
// first block of item i.
__global__ void __launch_bounds__(kLseThreads) k_lse_multi(const LseItem *items, int n_items, const int *block_begin,
                                                           int *err) {
    __shared__ LseShared sh;
    __shared__ int s_it;
    if (threadIdx.x == 0) {
        int lo = 0, hi = n_items - 1;
        while (lo < hi) { const int mid = (lo + hi + 1) >> 1; if (block_begin[mid] <= (int)blockIdx.x) lo = mid; else hi = mid - 1; }
        s_it = lo;
    }
    __syncthreads();
    const LseItem it = items[s_it];
    lse_body(sh, (int)blockIdx.x - it.block_begin, it.n_blocks, it.ll, it.n, it.chunk, it.m, it.seed, it.stage, it.part,
             it.counter, it.logz, it.idx, it.logq, err);
}

int lse_blocks(int64_t n) {
    const int64_t b = (n + kLseMinChunk - 1) / kLseMinChunk;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, kLseMaxBlocks));
}

void launch_lse_resample(const float *ll, int64_t n, int m, uint64_t seed, int stage, float2 *part, unsigned *counter,
                         float *logz, int *idx, float *logq, int *err, cudaStream_t s) {
    const int B = lse_blocks(n);
    const int chunk = (int)((n + B - 1) / B);
    k_lse_resample<<<B, kLseThreads, 0, s>>>(ll, n, chunk, m, (unsigned long long)seed, stage, part, counter, logz, idx,
                                             logq, err);
}

void launch_lse_shard(const float *ll, int64_t n, int m, uint64_t seed, int stage, const LseShard &shard, float2 *part,
                      unsigned *counter, float *logz, int *idx, float *logq, int *err, cudaStream_t s) {
    const int B = lse_blocks(n);
    const int chunk = (int)((n + B - 1) / B);
    k_lse_shard<<<B, kLseThreads, 0, s>>>(ll, n, chunk, m, (unsigned long long)seed, stage, shard, part, counter, logz,
                                          idx, logq, err);
}

// ------------------------------------------------------------------------------------------
// centre selection / particles
// ------------------------------------------------------------------------------------------
// centre_next (not last; at the last stage only when non-NULL) = pose of the drawn cell with
// the highest score (ties to the smaller index). Last: particle k = pose of drawn cell idx_k
// with t += G ((u - 1/2) step), its score and proposal log density score - logZ - 3 log(step).
// path (with stage > 0 or not last): logq[0] carries, between stages, the sum of the log
// probabilities (score - logZ) of the cells that centred the later stages; the last stage
// adds it to every particle's log density.
__device__ __forceinline__ void select_body(float *s_v, int *s_i, const float *ll, const int *idx, int m,
                                            const PoseGrid &P, const float *logz, int last, int path, int stage,
                                            unsigned long long seed, int n_stages, float *centre_next,
                                            float *particles, float *logw, float *logq) {
    const int tid = threadIdx.x;
    if (!last || centre_next) {
        float bv = -INFINITY;
        int bi = INT32_MAX;
        for (int k = tid; k < m; k += blockDim.x) {
            const int i = idx[k];
            if (i < 0) continue;
            const float v = ll[i];
            if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
        }
        s_v[tid] = bv;
        s_i[tid] = bi;
        __syncthreads();
        for (int st = blockDim.x / 2; st > 0; st >>= 1) {
            if (tid < st) {
                const float v = s_v[tid + st];
                const int i = s_i[tid + st];
                if (v > s_v[tid] || (v == s_v[tid] && i < s_i[tid])) { s_v[tid] = v; s_i[tid] = i; }
            }
            __syncthreads();
        }
        if (tid == 0) {
            float o[12];
            const int best = s_i[0] == INT32_MAX ? 0 : s_i[0];
            pose12(P, best, o);
            write_pose16(o, centre_next);
            if (path && !last) {
                const float term = s_i[0] == INT32_MAX ? -INFINITY : ll[best] - *logz;
                logq[0] = stage == 0 ? term : logq[0] + term;
            }
        }
        if (!last) return;
    }
    const float Z = *logz;
    const float lstep = 3.f * logf(P.step);
    const float acc = path && stage > 0 ? logq[0] : 0.f;
    __syncthreads();
    for (int k = tid; k < m; k += blockDim.x) {
        const int i = idx[k];
        float o[12];
        pose12(P, i < 0 ? 0 : i, o);
        const U64x4 r = philox4x64((unsigned long long)k, (unsigned long long)(unsigned)n_stages, 1ull, 0ull, seed, 0ull);
        const float u0 = (uniform24(r.v[0]) - 0.5f) * P.step, u1 = (uniform24(r.v[1]) - 0.5f) * P.step,
                    u2 = (uniform24(r.v[2]) - 0.5f) * P.step;
        for (int a = 0; a < 3; ++a) o[9 + a] += fmaf(P.G[3 * a + 0], u0, fmaf(P.G[3 * a + 1], u1, P.G[3 * a + 2] * u2));
        write_pose16(o, particles + 16 * (int64_t)k);
        const float v = i < 0 ? -INFINITY : ll[i];
        logw[k] = v;
        logq[k] = v - Z - lstep + acc;
    }
}

__global__ void k_c2f_select(const float *ll, const int *idx, int m, PoseGrid P, const float *logz, int last, int path,
                             int stage, unsigned long long seed, int n_stages, float *centre_next, float *particles,
                             float *logw, float *logq) {
    __shared__ float s_v[256];
    __shared__ int s_i[256];
    select_body(s_v, s_i, ll, idx, m, P, logz, last, path, stage, seed, n_stages, centre_next, particles, logw, logq);
}

// Batched: one block per scene.
__global__ void k_select_multi(const SelectItem *items, int last, int stage) {
    __shared__ float s_v[256];
    __shared__ int s_i[256];
    const SelectItem &it = items[blockIdx.x];
    select_body(s_v, s_i, it.ll, it.idx, it.m, it.grid, it.logz, last, it.path, stage, it.seed, it.n_stages,
                it.centre_next, it.particles, it.logw, it.logq);
}

// ------------------------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------------------------
void launch_set16(float *dst, const float *src16, cudaStream_t s) {
    F16 v;
    for (int i = 0; i < 16; ++i) v.v[i] = src16[i];
    k_set16<<<1, 32, 0, s>>>(dst, v);
}

void launch_rotation_set(int kind, int n, double rot_max, float *out, cudaStream_t s) {
    k_rotation_set<<<(n + 127) / 128, 128, 0, s>>>(kind, n, rot_max, out);
}

void launch_expand(PoseGrid P, int64_t n, float *poses, cudaStream_t s) {
    if (n <= 0) return;
    k_expand<<<(int)std::min<int64_t>((n + 255) / 256, 65535), 256, 0, s>>>(P, n, poses);
}

void launch_c2f_select(const float *ll, const int *idx, int m, PoseGrid P, const float *logz, int last, int path,
                       int stage, uint64_t seed, int n_stages, float *centre_next, float *particles, float *logw,
                       float *logq, cudaStream_t s) {
    k_c2f_select<<<1, 256, 0, s>>>(ll, idx, m, P, logz, last, path, stage, (unsigned long long)seed, n_stages,
                                   centre_next, particles, logw, logq);
}

void launch_lse_multi(const LseItem *items, int n_items, int total_blocks, const int *block_begin, int *err,
                      cudaStream_t s) {
    if (n_items <= 0 || total_blocks <= 0) return;
    k_lse_multi<<<total_blocks, kLseThreads, 0, s>>>(items, n_items, block_begin, err);
}

void launch_select_multi(const SelectItem *items, int n_items, int last, int stage, cudaStream_t s) {
    if (n_items <= 0) return;
    k_select_multi<<<n_items, 256, 0, s>>>(items, last, stage);
}

__global__ void k_gather16(const float *const *pairs, int n) {
    const int i = blockIdx.x, k = threadIdx.x;
    if (i < n && k < 16) {
        const float *src = pairs[2 * i];
        float *dst = const_cast<float *>(pairs[2 * i + 1]);
        dst[k] = src[k];
    }
}

void launch_gather16(const float *const *pairs, int n, cudaStream_t s) {
    if (n > 0) k_gather16<<<n, 32, 0, s>>>(pairs, n);
}

void launch_copy16(const float *src, float *dst, cudaStream_t s) {
    cudaMemcpyAsync(dst, src, 16 * sizeof(float), cudaMemcpyDeviceToDevice, s);
}

}  // namespace b3d
