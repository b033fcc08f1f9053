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

template <class PS>
__global__ void __launch_bounds__(kThreads) k_grad(SceneView S, Lik L, PS P, int64_t n_hyp, float *out_ll,
                                                   float *out_dpose, float *out_ds, float *out_dp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long *zb = reinterpret_cast<unsigned long long *>(smem_raw);
    float *zd = reinterpret_cast<float *>(zb + kRegionPx);  // rendered depth per Z pixel
    int *tj = reinterpret_cast<int *>(zd + kRegionPx);      // original face of the object, or -1
    float *ip = reinterpret_cast<float *>(tj + kRegionPx);  // b / p_i
    __shared__ float s_lut[kMaxLut];
    __shared__ float s_pose[12];
    __shared__ int s_bb[5];
    __shared__ int s_front;
    __shared__ float s_red[kThreads / 32];

    const Cam &c = S.cam;
    const MeshView &m = S.mesh;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < L.n_lut; i += nt) s_lut[i] = L.lut[i];
    const int w = L.w;

    for (int64_t h = blockIdx.x; h < n_hyp; h += gridDim.x) {
        __syncthreads();
        if (tid == 0) {
            pose12(P, h, s_pose);
            bool front = false;
            s_bb[4] = object_bbox(m, s_pose, c, s_bb, &front) ? 1 : 0;
            s_front = front ? 1 : 0;
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
                        for (int i = tid; i < zw * zh; i += nt) zb[i] = kEmptyKey;
                        __syncthreads();
                        for (int t = tid; t < n_t; t += nt) {
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
                    for (int i = tid; i < zw * zh; i += nt) {
                        const int gx = zx0 + i % zw, gy = zy0 + i / zw;
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
                    // pass A over I; deltas accumulate over the tile T only
                    for (int k = tid; k < iw * ih; k += nt) {
                        const int x = ix0 + k % iw, y = iy0 + k / iw;
                        const int64_t gi = (int64_t)y * c.W + x;
                        const float4 q = S.obs[gi];
                        float bp = 0.f;
                        if (q.w != 0.f) {
                            float Si, dSi, gs, gp;
                            pixel_terms(L, c, q, x, y, fetch, Si, dSi);
                            pixel_noise_grads(L, Si, dSi, gs, gp, bp);
                            if (x >= tx0 && x <= tx1 && y >= ty0 && y <= ty1) {
                                acc_l += pixel_ell(L, s_lut, c, q, x, y, fetch) - S.ell_bg[gi];
                                acc_s += gs - S.gs_bg[gi];
                                acc_p += gp - S.gp_bg[gi];
                            }
                        }
                        ip[k] = bp;
                    }
                    __syncthreads();
                    // pass B over the object's rendered pixels in T
                    const int tww = tx1 - tx0 + 1;
                    for (int k = tid; k < tww * (ty1 - ty0 + 1); k += nt) {
                        const int x = tx0 + k % tww, y = ty0 + k / tww;
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
                                const float N = L.gnorm * __expf(-d2 * L.inv2s2);
                                g += bpi * N * fmaf(ex, rx, fmaf(ey, ry, ez)) * L.inv_s2;
                            }
                        }
                        // triangle normal in the camera frame
                        const int4 f = m.faces[t];
                        float ax, ay, az, bx, by, bz, cx_, cy_, cz_;
                        const float4 A = m.verts[f.x], B = m.verts[f.y], C = m.verts[f.z];
                        xform(pose, A.x, A.y, A.z, ax, ay, az);
                        xform(pose, B.x, B.y, B.z, bx, by, bz);
                        xform(pose, C.x, C.y, C.z, cx_, cy_, cz_);
                        const float e1x = bx - ax, e1y = by - ay, e1z = bz - az;
                        const float e2x = cx_ - ax, e2y = cy_ - ay, e2z = cz_ - az;
                        const float nx = e1y * e2z - e1z * e2y, ny = e1z * e2x - e1x * e2z, nz = e1x * e2y - e1y * e2x;
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
        float vals[9] = {acc_l, acc_s, acc_p, g6[0], g6[1], g6[2], g6[3], g6[4], g6[5]};
        for (int k = 0; k < 9; ++k) {
            const float tot = block_sum(vals[k], s_red);
            if (tid == 0) vals[k] = tot;
            __syncthreads();
        }
        if (tid == 0) {
            out_ll[h] = (float)(S.sums_bg[0] + (double)vals[0]);
            if (out_ds) out_ds[h] = (float)(S.sums_bg[1] + (double)vals[1]);
            if (out_dp) out_dp[h] = (float)(S.sums_bg[2] + (double)vals[2]);
            if (out_dpose)
                for (int k = 0; k < 6; ++k) out_dpose[6 * h + k] = vals[3 + k];
        }
    }
}

int launch_grad_list(const SceneView &sv, const Lik &L, PoseList P, int64_t n, float *ll, float *dpose, float *dsigma,
                     float *dpout, int grid, cudaStream_t s) {
    if (n <= 0) return 0;
    auto kern = k_grad<PoseList>;
    const int per_sm = kernel_ctas_per_sm(kern, kThreads, kGradSmem);
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
    kern<<<g, kThreads, kGradSmem, s>>>(sv, L, P, n, ll, dpose, dsigma, dpout);
    return g;
}

}  // namespace b3d
