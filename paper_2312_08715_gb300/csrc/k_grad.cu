// k_grad.cu - forward + backward of the smooth (Gaussian-window) likelihood.
//
// One CTA iteration per hypothesis recomputes the forward with the score kernel's tile
// renderer in its tagged mode (64-bit (depth, tag) keys: the rectangle's face class, or the
// triangle's id, of the nearest surface at each pixel; composite with the fixed objects) and
// then, with visibility held fixed, per tile:
//   pass A, observed pixels i near the object: S_i, dS_i/ds, p_i = a + b S_i, giving the
//           deltas of l_i, dl_i/ds, dl_i/dp_out against the background tables and
//           b / p_i (kept in shared memory);
//   pass B, rendered pixels j of the object: g_j = dLL/dz_j
//           = sum_{i : j in win(i)} (b / p_i) N_ij (qt_i - q_j).r_j / s^2,
//           times dz_j/dxi = [n / (n.r_j), (q_j x n) / (n.r_j)] (left perturbation of the
//           pose in the camera frame; the point slides along its pixel ray on the plane of
//           its face, normal n), accumulated over j.
// The renderer uses the score kernel's primitive sets (rectangles of a voxel mesh, with the
// face classes turned away from the camera skipped; triangles otherwise), so the forward is
// the score kernel's. Nothing per pixel is stored in global memory.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "b3d_device.cuh"
#include "b3d_internal.h"
#include "k_score.cuh"

namespace b3d {

constexpr int kGradThreads = 256;  // threads per hypothesis: a launch of a few hundred hypotheses is one wave
constexpr int kGradMinBlocks = 2;
// dynamic shared memory: 64-bit keys (after the composite: pass A's weights and observed
// depths), depths and tags of a kRegionPx tile, then the lattice planes
constexpr int kGradSmemFixed = kRegionPx * ((int)sizeof(unsigned long long) + 2 * (int)sizeof(float));

template <class PS, int NT, int WT>
__global__ void __launch_bounds__(NT, kGradMinBlocks)
    k_grad(SceneView S, Lik L, PS P, int64_t n_hyp, float *out_ll, float *out_dpose, float *out_ds, float *out_dp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned *zb = reinterpret_cast<unsigned *>(smem_raw);               // [kRegionPx] 64-bit keys
    // the keys' memory once the composite has read them: per pixel of I,
    // ((b / p_i) (2 pi s^2)^(-3/2) / s^2, observed depth)
    float2 *ipq = reinterpret_cast<float2 *>(smem_raw);
    float *zd = reinterpret_cast<float *>(smem_raw + kRegionPx * 8);     // depth per zone pixel
    int *tg = reinterpret_cast<int *>(zd + kRegionPx);                   // face class / triangle id, or -1
    float4 *lat = reinterpret_cast<float4 *>(tg + kRegionPx);            // lattice planes
    __shared__ ScoreShared<NT> sh;
    __shared__ float4 s_stage[NT * kStageStride];
    __shared__ float s_cof[9];  // cofactor matrix of the linear part: maps object normals to camera normals
    __shared__ float s_red[9][NT / 32];

    const Cam &c = S.cam;
    const MeshView &m = S.mesh;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int w = WT > 0 ? WT : L.w;
    const float wscale = L.gnorm * L.inv_s2;
    lattice_coords(m, lat);  // ordered before use by the loop's first barrier

    for (int64_t h = blockIdx.x; h < n_hyp; h += gridDim.x) {
        __syncthreads();
        if (tid == 0) {
            pose12(P, h, sh.pose);
            // columns of the cofactor matrix: m1 x m2, m2 x m0, m0 x m1 (m_k the columns of
            // the linear part), so that (M a) x (M b) = cof(M) (a x b)
            const float *R = sh.pose;
            const float m0[3] = {R[0], R[3], R[6]}, m1[3] = {R[1], R[4], R[7]}, m2[3] = {R[2], R[5], R[8]};
            const float *cols[3][2] = {{m1, m2}, {m2, m0}, {m0, m1}};
            for (int k = 0; k < 3; ++k) {
                const float *u = cols[k][0], *v = cols[k][1];
                s_cof[0 + k] = u[1] * v[2] - u[2] * v[1];
                s_cof[3 + k] = u[2] * v[0] - u[0] * v[2];
                s_cof[6 + k] = u[0] * v[1] - u[1] * v[0];
            }
        }
        float acc_l = 0.f, acc_s = 0.f, acc_p = 0.f, g6[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        // zone = tile + 2w: pass A over I = T + w reads the depths of T + 2w
        render_tiles<false, NT, true>(
            S, 2 * w, L.miss_mode, sh, s_stage, zb, lat, nullptr,
            [&](const float *zdt, int zx0, int zy0, int zw, int, int, int, int, int tx0, int tx1, int ty0, int ty1) {
                const bool quad = (sh.flags & 2) != 0;
                // I: pixels whose window reaches a fragment, and that pass B of this tile reads
                const int ix0 = max(max(sh.fbb[0], tx0) - w, 0), ix1 = min(min(sh.fbb[1], tx1) + w, c.W - 1);
                const int iy0 = max(max(sh.fbb[2], ty0) - w, 0), iy1 = min(min(sh.fbb[3], ty1) + w, c.H - 1);
                const int iw = ix1 - ix0 + 1, n_i = iw * (iy1 - iy0 + 1);
                // pass A: one pixel per thread and step; the window's terms in pixel_ell_grads' order
                {
                    const int dq = NT / iw, dr = NT - dq * iw;
                    int yy = tid / iw, xx = tid - yy * iw;
                    for (int k = tid; k < n_i; k += NT) {
                        const int x = ix0 + xx, y = iy0 + yy;
                        const int64_t gi = (int64_t)y * c.W + x;
                        const float4 q = S.obs[gi];
                        float bp = 0.f;
                        if (q.w != 0.f) {
                            float l, gs, gp;
                            if (WT > 0) {
                                float E = 0.f, D = 0.f;
                                // the window's columns in packed f32x2 pairs (each lane rounded as
                                // the scalar loop rounds it), the exponentials and the running sums
                                // per element in the scalar loop's order
                                const f32x2_t qx2 = pk2(q.x, q.x), qy2 = pk2(q.y, q.y), qz2 = pk2(q.z, q.z);
                                const f32x2_t nis2 = pk2(-L.inv2s2, -L.inv2s2), is2 = pk2(L.inv_s2, L.inv_s2);
                                const f32x2_t m3 = pk2(-3.f, -3.f);
                                float nrx[2 * WT + 1];
#pragma unroll
                                for (int dx = -WT; dx <= WT; ++dx) nrx[dx + WT] = -(((float)(x + dx) + 0.5f - c.cx) * c.inv_fx);
                                auto acc1 = [&](float z, float e, float t) {
                                    if (z >= 0.f) {  // predicated: a missing point adds nothing
                                        E += e;
                                        D = fmaf(e, t, D);
                                    }
                                };
#pragma unroll
                                for (int dy = -WT; dy <= WT; ++dy) {
                                    const int yj = y + dy;
                                    const bool rowok = yj >= 0 && yj < c.H;
                                    const float nry = -(((float)yj + 0.5f - c.cy) * c.inv_fy);
                                    float zr[2 * WT + 1];
#pragma unroll
                                    for (int dx = -WT; dx <= WT; ++dx) {
                                        const int xj = x + dx;
                                        zr[dx + WT] = (rowok && xj >= 0 && xj < c.W) ? zdt[(yj - zy0) * zw + (xj - zx0)] : -1.f;
                                    }
#pragma unroll
                                    for (int k = 0; k + 1 < 2 * WT + 1; k += 2) {
                                        const f32x2_t z2 = pk2(zr[k], zr[k + 1]);
                                        const f32x2_t ex = fma2(z2, pk2(nrx[k], nrx[k + 1]), qx2), ey = fma2(z2, pk2(nry, nry), qy2);
                                        const f32x2_t ez = sub2(qz2, z2);
                                        const f32x2_t d2 = fma2(ex, ex, fma2(ey, ey, mul2(ez, ez)));
                                        float ga, gb, ta, tb;
                                        upk2(mul2(d2, nis2), ga, gb);
                                        upk2(fma2(d2, is2, m3), ta, tb);
                                        acc1(zr[k], __expf(ga), ta);
                                        acc1(zr[k + 1], __expf(gb), tb);
                                    }
                                    {
                                        const float z = zr[2 * WT];
                                        const float ex = fmaf(z, nrx[2 * WT], q.x), ey = fmaf(z, nry, q.y), ez = q.z - z;
                                        const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                                        acc1(z, __expf(-d2 * L.inv2s2), fmaf(d2, L.inv_s2, -3.f));
                                    }
                                }
                                grads_from_sums(L, E, D, l, gs, gp, bp);
                            } else {  // runtime half window: pixel_ell_grads' own loop
                                pixel_ell_grads(L, c, q, x, y, [&](int xj, int yj) { return zdt[(yj - zy0) * zw + (xj - zx0)]; },
                                                l, gs, gp, bp);
                            }
                            if (x >= tx0 && x <= tx1 && y >= ty0 && y <= ty1) {
                                acc_l += l - S.ell_bg[gi];
                                acc_s += gs - S.gs_bg[gi];
                                acc_p += gp - S.gp_bg[gi];
                            }
                        }
                        ipq[k] = make_float2(bp * wscale, q.z);
                        xx += dr;
                        yy += dq;
                        if (xx >= iw) { xx -= iw; ++yy; }
                    }
                }
                __syncthreads();
                // pass B over the object's rendered pixels in T (within the fragment box)
                {
                    const int jx0 = max(sh.fbb[0], tx0), jx1 = min(sh.fbb[1], tx1);
                    const int jy0 = max(sh.fbb[2], ty0), jy1 = min(sh.fbb[3], ty1);
                    const int jw = jx1 - jx0 + 1, n_j = jx1 >= jx0 && jy1 >= jy0 ? jw * (jy1 - jy0 + 1) : 0;
                    const int dq = NT / max(jw, 1), dr = NT - dq * max(jw, 1);
                    int yy = tid / max(jw, 1), xx = tid - yy * max(jw, 1);
                    for (int k = tid; k < n_j; k += NT) {
                        const int x = jx0 + xx, y = jy0 + yy;
                        xx += dr;
                        yy += dq;
                        if (xx >= jw) { xx -= jw; ++yy; }
                        const int zi = (y - zy0) * zw + (x - zx0);
                        const int t = tg[zi];
                        if (t < 0) continue;
                        const float z = zdt[zi];
                        const float rx = ((float)x + 0.5f - c.cx) * c.inv_fx, ry = ((float)y + 0.5f - c.cy) * c.inv_fy;
                        const float qx = z * rx, qy = z * ry, qz = z;
                        float g = 0.f;
                        auto term = [&](int xi, int yi) {
                            // pixels outside I carry no weight (b / p_i = 0 adds nothing)
                            const bool ok = xi >= ix0 && xi <= ix1 && yi >= iy0 && yi <= iy1;
                            const float2 bq = ok ? ipq[(yi - iy0) * iw + (xi - ix0)] : make_float2(0.f, 0.f);
                            const float bpi = bq.x;
                            // the observed point from its depth, as the observation kernel forms it
                            const float rxi = ((float)xi + 0.5f - c.cx) * c.inv_fx, ryi = ((float)yi + 0.5f - c.cy) * c.inv_fy;
                            const float ex = __fmul_rn(bq.y, rxi) - qx, ey = __fmul_rn(bq.y, ryi) - qy, ez = bq.y - qz;
                            const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                            g = fmaf(bpi * __expf(-d2 * L.inv2s2), fmaf(ex, rx, fmaf(ey, ry, ez)), g);
                        };
                        if (WT > 0) {
#pragma unroll
                            for (int dy = -WT; dy <= WT; ++dy)
#pragma unroll
                                for (int dx = -WT; dx <= WT; ++dx) term(x + dx, y + dy);
                        } else {
                            for (int dy = -w; dy <= w; ++dy)
                                for (int dx = -w; dx <= w; ++dx) term(x + dx, y + dy);
                        }
                        // the face's normal in the camera frame: a rectangle's face class gives its
                        // axis (the cofactor matrix's column; the sign cancels in n / (n.r)); a
                        // triangle's object-frame cross product is mapped by the cofactor matrix
                        float nx, ny, nz;
                        if (quad) {
                            const int a = t >> 1;
                            nx = s_cof[a];
                            ny = s_cof[3 + a];
                            nz = s_cof[6 + a];
                        } else {
                            const int4 f = m.faces[t - S.tri_base];
                            const float4 A = m.verts[f.x], B = m.verts[f.y], C = m.verts[f.z];
                            const float e1x = B.x - A.x, e1y = B.y - A.y, e1z = B.z - A.z;
                            const float e2x = C.x - A.x, e2y = C.y - A.y, e2z = C.z - A.z;
                            const float ox = e1y * e2z - e1z * e2y, oy = e1z * e2x - e1x * e2z, oz = e1x * e2y - e1y * e2x;
                            nx = fmaf(s_cof[0], ox, fmaf(s_cof[1], oy, s_cof[2] * oz));
                            ny = fmaf(s_cof[3], ox, fmaf(s_cof[4], oy, s_cof[5] * oz));
                            nz = fmaf(s_cof[6], ox, fmaf(s_cof[7], oy, s_cof[8] * oz));
                        }
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
                }
            },
            zd, tg);
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
    auto kern = L.w == 2 ? k_grad<PoseList, kGradThreads, 2>
                         : (L.w == 1 ? k_grad<PoseList, kGradThreads, 1> : k_grad<PoseList, kGradThreads, 0>);
    const int n_lat = sv.mesh.nc[0] + sv.mesh.nc[1] + sv.mesh.nc[2];
    const int smem = kGradSmemFixed + n_lat * (int)sizeof(float4);
    const int per_sm = kernel_ctas_per_sm(kern, kGradThreads, smem);
    int g = grid;
    if (g <= 0) g = per_sm * score_sm_count();
    g = (int)std::min<int64_t>(g, n);
    // tiles as wide as the region allows (the score kernel's tuned width is not this kernel's)
    SceneView v = sv;
    v.tile_w = kRegionPx;
    v.work = nullptr;
    kern<<<g, kGradThreads, smem, s>>>(v, L, P, n, ll, dpose, dsigma, dpout);
    return g;
}

}  // namespace b3d
