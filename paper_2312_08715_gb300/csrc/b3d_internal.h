// b3d_internal.h - device-side data layout and kernel launchers of libb3d (not part of
// the public ABI; include/b3d.h is).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "b3d.h"

namespace b3d {

#ifndef B3D_THREADS
#define B3D_THREADS 256
#endif
#ifndef B3D_SCORE_MIN_BLOCKS
#define B3D_SCORE_MIN_BLOCKS 3
#endif
constexpr int kThreads = B3D_THREADS;  // threads per CTA of the render/score kernels
constexpr int kScoreMinBlocks = B3D_SCORE_MIN_BLOCKS;  // CTAs per SM the score kernel is built for
constexpr int kRegionPx = 4096;        // z-buffer pixels per screen tile in shared memory
constexpr int kWorkRing = 64;          // hypothesis counters per context (one per launch in flight)
constexpr int kMaxPlanes = 511;        // lattice planes per axis of a quad mesh
constexpr int kMaxHalfWindow = 7;
constexpr int kMaxLut = (2 * kMaxHalfWindow + 1) * (2 * kMaxHalfWindow + 1) + 1;
constexpr unsigned long long kEmptyKey = ~0ull;
constexpr int kNumStats = 8;  // work counters of the fused kernel (see k_fused)

struct Cam {
    int W, H;
    float fx, fy, cx, cy, near_z, far_z;
    float inv_fx, inv_fy;
};

// One object's render data.
//  - verts: welded vertices (bitwise-equal positions merged), object frame.
//  - tris_surf: the triangles that can be the nearest surface when the whole object lies
//    beyond the near plane: for a closed outward mesh, coincident internal face pairs are
//    removed (and back faces are skipped per hypothesis); otherwise all triangles.
//  - tris_full: every non-degenerate triangle, used when the near plane cuts the object
//    open (then internal and back faces can be visible).
//  - faces: the original faces on welded vertices (triangle id -> vertices).
//  - rectangles (optional, voxel meshes): every surface triangle pairs with another into a
//    unit square of the vertex lattice, and the coplanar squares of each lattice plane and
//    outward side are merged into rectangles of at most 3 x 3 squares; rectangles are grouped by face class
//    (axis, outward sign) and sorted by lattice plane, so the faces turned towards a camera
//    position are one contiguous range per class.
struct MeshView {
    const float4 *verts;
    const int4 *tris_surf;      // (v0, v1, v2, original face index)
    const int4 *tris_full;
    const int4 *faces;          // [n_faces] (v0, v1, v2, 0)
    int n_surf, n_full, n_faces;
    int closed;                 // back faces may be skipped (whole object beyond near)
    float lo[3], hi[3];         // object-frame bounding box of the vertices
    // voxel rectangles
    int n_quads;                // 0: no rectangle representation
    const uint2 *quads;         // .x: class(3) 0(2) plane(9) b0(9) c0(9); .y: b extent(9) c extent(9)
    const int *class_off;       // [6 * (np1)]: first rectangle of class c with plane >= p
    const float *coords;        // lattice plane coordinates, x planes then y then z
    int nc[3];                  // planes per axis
    int np1;                    // stride of class_off (max planes + 1)
};

// Windowed likelihood constants (Eq. 1 with the window of Sec. III-B).
struct Lik {
    int kind;        // 0 inlier ball, 1 Gaussian
    int w;           // half window
    int miss_mode;   // 0 miss = far-plane point, 1 miss = no point
    int n_lut;       // (2w+1)^2 + 1
    float r2;        // kind 0: r^2
    float inv2s2;    // kind 1: 1 / (2 s^2)
    float a;         // p_out / V
    float bg;        // kind 1: (1 - p_out) / K * (2 pi s^2)^(-3/2)
    float lut[kMaxLut];  // kind 0: l(n) = log(a + (1 - p_out) n / (K (4/3) pi r^3))
    // gradient constants (kind 1)
    float s;         // sigma
    float inv_s2;    // 1 / s^2
    float b;         // (1 - p_out) / K
    float inv_V;     // 1 / V
    float inv_K;     // 1 / K
    float gnorm;     // (2 pi s^2)^(-3/2)
};

// A grid of noise settings (hierarchical noise): nr radii (kind 0) or standard deviations
// (kind 1) times np outlier probabilities; setting g = 4 i + j internally (i < nr, j < np).
constexpr int kMaxNoiseR = 4, kMaxNoiseP = 4, kMaxNoise = kMaxNoiseR * kMaxNoiseP;
constexpr int kNoiseLut = 26;  // (2w+1)^2 + 1 for half windows up to 2
struct NoiseLik {
    int kind, w, miss_mode, nr, np;
    float r2[kMaxNoiseR];       // kind 0: r_i^2
    float inv2s2[kMaxNoiseR];   // kind 1: 1 / (2 s_i^2)
    float a[kMaxNoiseP];        // p_j / V
    float bg[kMaxNoise];        // kind 1: (1 - p_j) / K (2 pi s_i^2)^(-3/2)
    float logw[kMaxNoise];      // prior log weight of the setting
    float lut[kMaxNoise * kNoiseLut];  // kind 0: log(a_j + (1 - p_j) n / (K (4/3) pi r_i^3))
};

// The scene as the fused kernels see it, for one hypothesised object (the slot).
struct SceneView {
    Cam cam;
    const float4 *obs;                 // [H*W] observed points (x, y, z, 1) or (0,0,0,0) if not scored
    const unsigned long long *bg;      // [H*W] (depth bits << 32 | triangle id) of the fixed objects
    const float *bgd;                  // [2][H*W] their depth, misses at the far plane / -1 (miss modes 0, 1)
    const float *ell_bg;               // [H*W] l_i of the fixed objects alone (0 where not scored)
    // The fused score kernels' per-pixel inputs, packed (12 B a pixel instead of 28, so a
    // hypothesis's screen box stays in L1 across the CTAs of an SM); NULL until the
    // likelihood tables of this background are built:
    const float2 *qe;                  // [H*W] (observed depth or 0 where no point, ell_bg)
    const unsigned *bgz;               // [H*W] depth bits of the fixed objects (bg >> 32)
    const double *ll_bg;               // [1]   sum of ell_bg
    const float *gs_bg;                // [H*W] d l_i / d sigma, fixed objects alone (gradient only)
    const float *gp_bg;                // [H*W] d l_i / d p_out, fixed objects alone (gradient only)
    const double *sums_bg;             // [3]   sums of ell_bg, gs_bg, gp_bg (gradient only)
    MeshView mesh;                     // the slot object
    int tri_base;                      // global triangle id of the slot object's face 0
    int *err;                          // device error flag
    unsigned long long *stats;         // [kNumStats] work counters, or NULL (no counting)
    int tile_w;                        // widest screen tile of the score kernel (pixels)
    unsigned long long *work;          // hypothesis counter of a persistent kernel (zeroed by its launcher) or
                                       // NULL: CTA c takes hypotheses c, c + grid, ...
};

// Hypothesis poses as 12 floats: R row-major (9) then t (3).
struct PoseList {
    const float *p;  // [n, 16]
};

struct PoseGrid {
    const float *centre;  // device [16] cam_from_obj of the grid centre
    const float *rot;     // device [n_rot, 9]
    float G[9];           // cam_from_grid rotation
    int n;                // points per axis
    int n_rot;
    float step;
};

// One scene of a batched launch (device memory): its view, likelihood constants, the poses
// of its hypotheses (a list or a coarse-to-fine grid) and where its scores go. Its size is a
// multiple of 16 bytes: kernels copy descriptors of an array of them as float4.
struct __align__(16) BatchItem {
    SceneView S;
    Lik L;
    PoseList list;
    PoseGrid grid;
    int pose_kind;      // 0: list, 1: grid
    int n_hyp;
    float *out_ll;
};
static_assert(sizeof(BatchItem) % 16 == 0, "BatchItem must tile float4 copies");

// One rank's share of a categorical whose scores are split over ranks (contiguous shards):
// the probability mass of the ranks before it, its own mass (the last rank's runs to 1),
// the global log normaliser and the global index of its first score.
struct LseShard {
    double before, mass;
    float logz;
    long long base;
};

// One scene's segment of a batched log-sum-exp + resampling launch.
struct LseItem {
    const float *ll;
    int64_t n;
    int chunk, block_begin, n_blocks, m;
    unsigned long long seed;
    int stage;
    float2 *part;
    unsigned *counter;
    float *logz;
    int *idx;
    float *logq;
};

// One scene's centre selection / particles of a batched coarse-to-fine stage.
struct SelectItem {
    const float *ll;
    const int *idx;
    int m;
    PoseGrid grid;
    const float *logz;
    float *centre_next;
    float *particles, *logw, *logq;
    unsigned long long seed;
    int n_stages;
    int path;  // accumulate the path density in logq (see b3d_c2f_schedule)
};

// Dynamic shared memory opt-in and resident CTAs per SM of a kernel, set and queried once
// per kernel and size (no runtime calls afterwards, e.g. while a graph is captured).
int kernel_ctas_per_sm_impl(const void *kernel, int threads, int smem);  // cached by (kernel, threads, smem)

template <class K>
inline int kernel_ctas_per_sm(K kernel, int threads, int smem) {
    return kernel_ctas_per_sm_impl(reinterpret_cast<const void *>(kernel), threads, smem);
}

// ---- launchers (k_render.cu) -------------------------------------------------------------
void launch_obs_points(const Cam &cam, const float *depth, float4 *obs, cudaStream_t s);
void launch_bg_clear(unsigned long long *bg, int64_t n, cudaStream_t s);
// dst[i] = min over the n_src buffers src[k][i] (n_src <= kMaxBgSources), kEmptyKey if none
constexpr int kMaxBgSources = 16;
void launch_bg_min(int64_t n, const unsigned long long *const *src, int n_src, unsigned long long *dst, cudaStream_t s);
// bgd[m * W H + i] = depth of background key i under miss mode m (0: far plane, 1: -1)
void launch_bg_depth(int64_t n, float far_z, const unsigned long long *bg, float *bgd, cudaStream_t s);
void launch_bg_raster(const Cam &cam, const MeshView &m, const float *pose16_dev, int tri_base,
                      unsigned long long *bg, cudaStream_t s);
// Per-pixel background terms and their double-precision sums (sums[0..2]); part holds
// 3 x bg_table_blocks(W H) doubles, counter one zeroed word (left zeroed).
int bg_table_blocks(int64_t n);
void launch_bg_tables(const SceneView &sv, const Lik &L, float *ell_bg, float *gs_bg, float *gp_bg, float2 *qe,
                      unsigned *bgz, double *part, unsigned *counter, double *sums, cudaStream_t s);
int launch_score_list(const SceneView &sv, const Lik &L, PoseList P, int64_t n, float *ll, int grid, cudaStream_t s);
int launch_score_grid(const SceneView &sv, const Lik &L, PoseGrid P, int64_t n, float *ll, int grid, cudaStream_t s);
// ---- launchers (k_materialised.cu) -------------------------------------------------------
// Materialised render; returns the number of kernel launches.
int launch_render_list(const SceneView &sv, PoseList P, int64_t n, float *depth, int *tid, int grid, cudaStream_t s);
// Materialised images (sv: the scene's full background and its terms); returns the number of
// kernel launches.
int launch_score_depth(const SceneView &sv, const Lik &L, const float *depth, const int *tid, int64_t n, float *ll,
                       int grid, cudaStream_t s);
// Adam step + se(3) re-basing of n poses [n, 16] from their loglik gradients dpose [n, 6]
// (k_grad.cu); m, v [n, 6] moments; bc1, bc2 the bias corrections of this step.
void launch_se3_compose(int64_t n, const float *xi, const float *in, float *out, cudaStream_t s);
void launch_adam_se3(int64_t n, const float *dpose, float *m, float *v, float *poses, float lr, float b1, float b2,
                     float eps, float bc1, float bc2, cudaStream_t s);
int launch_grad_list(const SceneView &sv, const Lik &L, PoseList P, int64_t n, float *ll, float *dpose,
                     float *dsigma, float *dpout, int grid, cudaStream_t s);

// Batched score launch over items [0, n_items) of `items` (device), their hypotheses
// flattened in item order with item_begin[n_items + 1] (device) the offsets; CTAs take
// `chunk` hypotheses at a time from *counter (zeroed by the caller before the launch).
int launch_score_multi(const BatchItem *items, int n_items, const int64_t *item_begin, int64_t total, int chunk,
                       unsigned long long *counter, int w, int max_lat, int grid, cudaStream_t s);

// ---- launchers (k_c2f.cu) ----------------------------------------------------------------
void launch_lse_multi(const LseItem *items, int n_items, int total_blocks, const int *block_begin, int *err,
                      cudaStream_t s);
void launch_select_multi(const SelectItem *items, int n_items, int last, int stage, cudaStream_t s);
// dst[i][0..15] = src[i][0..15] for pairs (src, dst) in device memory
void launch_gather16(const float *const *pairs, int n, cudaStream_t s);
void launch_set16(float *dst, const float *src16_host_values, cudaStream_t s);
void launch_rotation_set(int kind, int n, double rot_max, float *out, cudaStream_t s);
void launch_expand(PoseGrid P, int64_t n, float *poses, cudaStream_t s);
int lse_blocks(int64_t n);
void launch_lse_resample(const float *ll, int64_t n, int m, uint64_t seed, int stage, float2 *part,
                         unsigned *counter, float *logz, int *idx, float *logq, int *err, cudaStream_t s);
void launch_lse_shard(const float *ll, int64_t n, int m, uint64_t seed, int stage, const LseShard &shard, float2 *part,
                      unsigned *counter, float *logz, int *idx, float *logq, int *err, cudaStream_t s);
void launch_c2f_select(const float *ll, const int *idx, int m, PoseGrid P, const float *logz, int last, int path,
                       int stage, uint64_t seed, int n_stages, float *centre_next, float *particles, float *logw,
                       float *logq, cudaStream_t s);
void launch_copy16(const float *src, float *dst, cudaStream_t s);

// Camera hypotheses (k_render.cu): every object k at H_h world[k], full image, no background.
int launch_render_camera(const Cam &cam, const MeshView *meshes, const int *tri_base, const float *world, int n_obj,
                         PoseList P, int64_t n, float *depth, int *tid, cudaStream_t s);

// Noise-grid scoring (k_score_noise.cu): per-setting background tables and sums (part holds
// kMaxNoise x blocks doubles, returns blocks), and the fused scoring launch.
int launch_bg_noise_tables(const SceneView &sv, const NoiseLik &N, float *nell, double *part, unsigned *counter,
                           double *sums, cudaStream_t s);
void launch_score_noise(const SceneView &sv, const NoiseLik &N, const float *poses, int64_t n_hyp, const float *nell,
                        const double *nsums, float *out_ll, float *out_marg, cudaStream_t s);

// Context hooks used by the tracking server (defined with the context in b3d_api.cu).
uint64_t ctx_used_bytes(b3d_ctx *ctx);
void ctx_set_budget(b3d_ctx *ctx, uint64_t budget);
b3d_status ctx_alloc_bytes(b3d_ctx *ctx, size_t bytes, void **out, const char *what);
float *ctx_scene_poses(b3d_ctx *ctx);  // device [n_obj, 16]
int *ctx_err_flag(b3d_ctx *ctx);       // device [1]
// Shared backgrounds of a context whose first n_slots objects are hypothesised in turn (a
// tracking session): one z-buffer per object (allocated by ctx_prepare_shared_bg, rendered
// when its pose changed), each slot's background the per-pixel minimum over the other
// objects' buffers (the same keys as rasterising them into one buffer). ctx_tracked_moved:
// the poses of objects [0, n_slots) changed on the device (the others kept theirs).
b3d_status ctx_prepare_shared_bg(b3d_ctx *ctx, cudaStream_t s);
b3d_status ctx_build_slot_bgs(b3d_ctx *ctx, int32_t n_slots, cudaStream_t s);
void ctx_tracked_moved(b3d_ctx *ctx, int32_t n_slots);
// Allocate and fill everything a batched enumeration of `slot` needs (background caches,
// likelihood tables, rotation sets), so later calls allocate nothing.
b3d_status ctx_prepare_slot(b3d_ctx *ctx, int32_t slot, const b3d_lik_params *lik, const b3d_c2f_schedule *sch,
                            cudaStream_t s);
b3d_status owner_reserve(b3d_ctx *owner, int64_t n_items, const b3d_c2f_schedule *sch);

}  // namespace b3d
