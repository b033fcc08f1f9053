// k_grad.cu - forward + backward of the smooth (Gaussian-window) likelihood.
//
// One CTA iteration per hypothesis recomputes the forward (render into a shared-memory
// z-buffer, composite with the fixed objects) and then, with visibility held fixed:
//   pass A, observed pixels i near the object: S_i, dS_i/ds, p_i = a + b S_i, giving the
//           deltas of l_i, dl_i/ds, dl_i/dp_out against the background tables and
//           b / p_i (kept in shared memory);
//   pass B, rendered pixels j of the object: g_j = dLL/dz_j
//           = sum_{i : j in win(i)} (b / p_i) N_ij (qt_i - q_j).r_j / s^2,
//           times dz_j/dxi = [n / (n.r_j), (q_j x n) / (n.r_j)] (left perturbation of the
//           pose in the camera frame; the point slides along its pixel ray on the plane of
//           its triangle, normal n), accumulated over j.
// The forward uses the same triangle sets as the renderer (surface set with back faces
// skipped when the whole object lies beyond the near plane, every triangle otherwise).
// Nothing per pixel is stored in global memory.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "b3d_device.cuh"
#include "b3d_internal.h"

namespace b3d {

constexpr int kGradSmem = kRegionPx * ((int)sizeof(unsigned long long) + 3 * (int)sizeof(float));
constexpr int kGradThreads = 512;  // threads per hypothesis: a launch of a few hundred hypotheses is one wave
constexpr int kGradMinBlocks = 2;

template <class PS, int NT>
__global__ void __launch_bounds__(NT, kGradMinBlocks)
    k_grad(SceneView S, Lik L, PS P, int64_t n_hyp, float *out_ll, float *out_dpose, float *out_ds, float *out_dp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long *zb = reinterpret_cast<unsigned long long *>(smem_raw);
    float *zd = reinterpret_cast<float *>(zb + kRegionPx);  // rendered depth per Z pixel
    int *tj = reinterpret_cast<int *>(zd + kRegionPx);      // original face of the object, or -1
    float *ip = reinterpret_cast<float *>(tj + kRegionPx);  // (b / p_i) (2 pi s^2)^(-3/2) / s^2
    __shared__ float s_pose[12];
    __shared__ float s_cof[9];  // cofactor matrix of the linear part: maps object normals to camera normals
    __shared__ int s_bb[5];
    __shared__ int s_front;
    __shared__ float s_red[9][NT / 32];

    const Cam &c = S.cam;
    const MeshView &m = S.mesh;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int w = L.w;
    const float wscale = L.gnorm * L.inv_s2;

    for (int64_t h = blockIdx.x; h < n_hyp; h += gridDim.x) {
        __syncthreads();
        if (tid == 0) {
            pose12(P, h, s_pose);
            bool front = false;
            s_bb[4] = object_bbox(m, s_pose, c, s_bb, &front) ? 1 : 0;
            s_front = front ? 1 : 0;
            // columns of the cofactor matrix: m1 x m2, m2 x m0, m0 x m1 (m_k the columns of
            // the linear part), so that (M a) x (M b) = cof(M) (a x b)
            const float *R = s_pose;
            const float m0[3] = {R[0], R[3], R[6]}, m1[3] = {R[1], R[4], R[7]}, m2[3] = {R[2], R[5], R[8]};
            const float *cols[3][2] = {{m1, m2}, {m2, m0}, {m0, m1}};
            for (int k = 0; k < 3; ++k) {
                const float *u = cols[k][0], *v = cols[k][1];
                s_cof[0 + k] = u[1] * v[2] - u[2] * v[1];
                s_cof[3 + k] = u[2] * v[0] - u[0] * v[2];
                s_cof[6 + k] = u[0] * v[1] - u[1] * v[0];
            }
        }
        __syncthreads();
        const float *pose = s_pose;
        const bool has_bb = s_bb[4] != 0, front = s_front != 0;
        const int bx0 = s_bb[0], bx1 = s_bb[1], by0 = s_bb[2], by1 = s_bb[3];
        const int4 *tris = front ? m.tris_surf : m.tris_full;
        const int n_t = front ? m.n_surf : m.n_full;
        const int cull = front ? m.closed : 0;
        float acc_l = 0.f, acc_s = 0.f, acc_p = 0.f, g6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (has_bb) {
            const int sx0 = max(bx0 - w, 0), sx1 = min(bx1 + w, c.W - 1);
            const int sy0 = max(by0 - w, 0), sy1 = min(by1 + w, c.H - 1);
            const int sw = sx1 - sx0 + 1;
            const int tw = min(sw, 48);
            const int th = max(1, kRegionPx / (tw + 4 * w) - 4 * w);
            for (int ty0 = sy0; ty0 <= sy1; ty0 += th) {
                for (int tx0 = sx0; tx0 <= sx1; tx0 += tw) {
                    const int tx1 = min(tx0 + tw - 1, sx1), ty1 = min(ty0 + th - 1, sy1);
                    // Z: depths needed by pass A over I = T + w, i.e. T + 2w
                    const int zx0 = max(tx0 - 2 * w, 0), zx1 = min(tx1 + 2 * w, c.W - 1);
                    const int zy0 = max(ty0 - 2 * w, 0), zy1 = min(ty1 + 2 * w, c.H - 1);
                    const int zw = zx1 - zx0 + 1, zh = zy1 - zy0 + 1;
                    const int ix0 = max(tx0 - w, 0), ix1 = min(tx1 + w, c.W - 1);
                    const int iy0 = max(ty0 - w, 0), iy1 = min(ty1 + w, c.H - 1);
                    const int iw = ix1 - ix0 + 1, ih = iy1 - iy0 + 1;
                    const int rx0 = max(zx0, bx0), rx1 = min(zx1, bx1), ry0 = max(zy0, by0), ry1 = min(zy1, by1);
                    const bool need = rx0 <= rx1 && ry0 <= ry1;
                    if (need) {
                        for (int i = tid; i < zw * zh; i += NT) zb[i] = kEmptyKey;
                        __syncthreads();
                        for (int t = tid; t < n_t; t += NT) {
                            const int4 tr = tris[t];
                            float4 A, B, C;
                            tri_screen(m, tr, pose, c, A, B, C);
                            const unsigned gid = (unsigned)(S.tri_base + tr.w);
                            raster_tri(A, B, C, cull, rx0, rx1, ry0, ry1, c.far_z, [&](int x, int y, float z) {
                                atomicMin(&zb[(y - zy0) * zw + (x - zx0)], pack_key(z, gid));
                            });
                        }
                        __syncthreads();
                    }
                    for (int i = tid; i < zw * zh; i += NT) {
                        const int gy = zy0 + i / zw, gx = zx0 + (i - (i / zw) * zw);
                        const unsigned long long kb = S.bg[(int64_t)gy * c.W + gx];
                        unsigned long long key = kb;
                        int t = -1;
                        if (need && zb[i] < kb) {
                            key = zb[i];
                            t = (int)(unsigned)(key & 0xffffffffu) - S.tri_base;
                        }
                        zd[i] = key_depth(key, L.miss_mode, c.far_z);
                        tj[i] = t;
                    }
                    __syncthreads();
                    auto fetch = [&](int xj, int yj) { return zd[(yj - zy0) * zw + (xj - zx0)]; };
                    // pass A over I (one window loop gives l_i and its derivatives); deltas
                    // accumulate over the tile T only
                    for (int k = tid; k < iw * ih; k += NT) {
                        const int y = iy0 + k / iw, x = ix0 + (k - (k / iw) * iw);
                        const int64_t gi = (int64_t)y * c.W + x;
                        const float4 q = S.obs[gi];
                        float bp = 0.f;
                        if (q.w != 0.f) {
                            float l, gs, gp;
                            pixel_ell_grads(L, c, q, x, y, fetch, l, gs, gp, bp);
                            if (x >= tx0 && x <= tx1 && y >= ty0 && y <= ty1) {
                                acc_l += l - S.ell_bg[gi];
                                acc_s += gs - S.gs_bg[gi];
                                acc_p += gp - S.gp_bg[gi];
                            }
                        }
                        ip[k] = bp * wscale;
                    }
                    __syncthreads();
                    // pass B over the object's rendered pixels in T
                    const int tww = tx1 - tx0 + 1;
                    for (int k = tid; k < tww * (ty1 - ty0 + 1); k += NT) {
                        const int y = ty0 + k / tww, x = tx0 + (k - (k / tww) * tww);
                        const int zi = (y - zy0) * zw + (x - zx0);
                        const int t = tj[zi];
                        if (t < 0) continue;
                        const float z = zd[zi];
                        const float rx = ((float)x + 0.5f - c.cx) * c.inv_fx, ry = ((float)y + 0.5f - c.cy) * c.inv_fy;
                        const float qx = z * rx, qy = z * ry, qz = z;
                        float g = 0.f;
                        for (int dy = -w; dy <= w; ++dy) {
                            const int yi = y + dy;
                            if (yi < 0 || yi >= c.H) continue;
                            for (int dx = -w; dx <= w; ++dx) {
                                const int xi = x + dx;
                                if (xi < 0 || xi >= c.W) continue;
                                const float bpi = ip[(yi - iy0) * iw + (xi - ix0)];
                                if (bpi == 0.f) continue;
                                const float4 qi = S.obs[(int64_t)yi * c.W + xi];
                                const float ex = qi.x - qx, ey = qi.y - qy, ez = qi.z - qz;
                                const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                                g = fmaf(bpi * __expf(-d2 * L.inv2s2), fmaf(ex, rx, fmaf(ey, ry, ez)), g);
                            }
                        }
                        // the face's normal: object-frame cross product mapped by the cofactor matrix
                        const int4 f = m.faces[t];
                        const float4 A = m.verts[f.x], B = m.verts[f.y], C = m.verts[f.z];
                        const float e1x = B.x - A.x, e1y = B.y - A.y, e1z = B.z - A.z;
                        const float e2x = C.x - A.x, e2y = C.y - A.y, e2z = C.z - A.z;
                        const float ox = e1y * e2z - e1z * e2y, oy = e1z * e2x - e1x * e2z, oz = e1x * e2y - e1y * e2x;
                        const float nx = fmaf(s_cof[0], ox, fmaf(s_cof[1], oy, s_cof[2] * oz));
                        const float ny = fmaf(s_cof[3], ox, fmaf(s_cof[4], oy, s_cof[5] * oz));
                        const float nz = fmaf(s_cof[6], ox, fmaf(s_cof[7], oy, s_cof[8] * oz));
                        const float nr = fmaf(nx, rx, fmaf(ny, ry, nz));
                        if (nr == 0.f) continue;
                        const float gn = g / nr;
                        g6[0] += gn * nx;
                        g6[1] += gn * ny;
                        g6[2] += gn * nz;
                        g6[3] += gn * (qy * nz - qz * ny);
                        g6[4] += gn * (qz * nx - qx * nz);
                        g6[5] += gn * (qx * ny - qy * nx);
                    }
                    __syncthreads();
                }
            }
        }
        // one reduction of the nine sums: warp trees, then warps in order
        const float vals[9] = {acc_l, acc_s, acc_p, g6[0], g6[1], g6[2], g6[3], g6[4], g6[5]};
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float v = warp_sum(vals[k]);
            if (lane == 0) s_red[k][wid] = v;
        }
        __syncthreads();
        if (tid < 9) {
            float tot = 0.f;
            for (int k = 0; k < NT / 32; ++k) tot += s_red[tid][k];
            if (tid == 0) out_ll[h] = (float)(S.sums_bg[0] + (double)tot);
            else if (tid == 1) { if (out_ds) out_ds[h] = (float)(S.sums_bg[1] + (double)tot); }
            else if (tid == 2) { if (out_dp) out_dp[h] = (float)(S.sums_bg[2] + (double)tot); }
            else if (out_dpose) out_dpose[6 * h + (tid - 3)] = tot;
        }
    }
}

// P <- Exp(xi^) P for one row-major 4x4 pose P (rows 0-2 read and written) and the twist
// xi = (v, w): Rodrigues for the rotation and the SE(3) V matrix for the translation, with
// series for sin(th)/th, (1 - cos th)/th^2 and (th - sin th)/th^3 below th = 0.1 (in float
// the closed forms lose most of their digits to cancellation at the angles a refinement
// step takes).
__device__ __forceinline__ void se3_left_compose(const float xi[6], float *P) {
    const float wx = xi[3], wy = xi[4], wz = xi[5];
    const float th2 = wx * wx + wy * wy + wz * wz, th = sqrtf(th2);
    float a, b, c;  // R = I + a W + b W^2, V = I + b W + c W^2 with W = [w]x (unnormalised)
    if (th < 0.1f) {  // series to th^4: the next terms are below 3e-10
        const float th4 = th2 * th2;
        a = 1.f - th2 / 6.f + th4 / 120.f;
        b = 0.5f - th2 / 24.f + th4 / 720.f;
        c = 1.f / 6.f - th2 / 120.f + th4 / 5040.f;
    } else {
        const float s = sinf(th), co = cosf(th);
        a = s / th;
        b = (1.f - co) / th2;
        c = (th - s) / (th2 * th);
    }
    const float W[9] = {0.f, -wz, wy, wz, 0.f, -wx, -wy, wx, 0.f};
    float W2[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int q = 0; q < 3; ++q)
            W2[3 * r + q] = W[3 * r] * W[q] + W[3 * r + 1] * W[3 + q] + W[3 * r + 2] * W[6 + q];
    float R[9], V[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float id = (k % 4 == 0) ? 1.f : 0.f;
        R[k] = id + a * W[k] + b * W2[k];
        V[k] = id + b * W[k] + c * W2[k];
    }
    float T[12];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        T[4 * r] = P[4 * r]; T[4 * r + 1] = P[4 * r + 1]; T[4 * r + 2] = P[4 * r + 2]; T[4 * r + 3] = P[4 * r + 3];
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float tv = V[3 * r] * xi[0] + V[3 * r + 1] * xi[1] + V[3 * r + 2] * xi[2];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            P[4 * r + q] = R[3 * r] * T[q] + R[3 * r + 1] * T[4 + q] + R[3 * r + 2] * T[8 + q] + (q == 3 ? tv : 0.f);
    }
}

// One Adam step per pose on the ascent direction of loglik (gradient g = -dpose of the loss
// -loglik; moments m, v [n, 6]; bc1 = 1 - beta1^t, bc2 = 1 - beta2^t), then the re-basing
// T <- Exp(xi^) T with xi = -lr mhat / (sqrt(vhat) + eps).
__global__ void k_adam_se3(int64_t n, const float *dpose, float *m, float *v, float *poses, float lr, float b1, float b2,
                           float eps, float bc1, float bc2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float xi[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float g = -dpose[6 * i + k];
            const float mk = fmaf(b1, m[6 * i + k], (1.f - b1) * g);
            const float vk = fmaf(b2, v[6 * i + k], (1.f - b2) * g * g);
            m[6 * i + k] = mk;
            v[6 * i + k] = vk;
            xi[k] = -lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
        }
        se3_left_compose(xi, poses + 16 * i);
    }
}

// out_i = Exp(xi_i^) in_i for n poses (out may be in): the left se(3) update of the
// gradient's parameterisation.
__global__ void k_se3_compose(int64_t n, const float *xi, const float *in, float *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float x[6], P[16];
#pragma unroll
        for (int k = 0; k < 6; ++k) x[k] = xi[6 * i + k];
#pragma unroll
        for (int k = 0; k < 16; ++k) P[k] = in[16 * i + k];
        se3_left_compose(x, P);
#pragma unroll
        for (int k = 0; k < 12; ++k) out[16 * i + k] = P[k];
        out[16 * i + 12] = 0.f;
        out[16 * i + 13] = 0.f;
        out[16 * i + 14] = 0.f;
        out[16 * i + 15] = 1.f;
    }
}

void launch_se3_compose(int64_t n, const float *xi, const float *in, float *out, cudaStream_t s) {
    if (n <= 0) return;
    const int blocks = (int)std::min<int64_t>((n + 127) / 128, 1024);
    k_se3_compose<<<blocks, 128, 0, s>>>(n, xi, in, out);
}

void launch_adam_se3(int64_t n, const float *dpose, float *m, float *v, float *poses, float lr, float b1, float b2,
                     float eps, float bc1, float bc2, cudaStream_t s) {
    if (n <= 0) return;
    const int blocks = (int)std::min<int64_t>((n + 127) / 128, 1024);
    k_adam_se3<<<blocks, 128, 0, s>>>(n, dpose, m, v, poses, lr, b1, b2, eps, bc1, bc2);
}

int launch_grad_list(const SceneView &sv, const Lik &L, PoseList P, int64_t n, float *ll, float *dpose, float *dsigma,
                     float *dpout, int grid, cudaStream_t s) {
    if (n <= 0) return 0;
    auto kern = k_grad<PoseList, kGradThreads>;
    const int per_sm = kernel_ctas_per_sm(kern, kGradThreads, kGradSmem);
    int g = grid;
    if (g <= 0) {
        static int sms = 0;
        if (!sms) {
            int dev = 0;
            cudaGetDevice(&dev);
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            sms = std::max(1, sms);
        }
        g = per_sm * sms;
    }
    g = (int)std::min<int64_t>(g, n);
    kern<<<g, kGradThreads, kGradSmem, s>>>(sv, L, P, n, ll, dpose, dsigma, dpout);
    return g;
}

}  // namespace b3d
