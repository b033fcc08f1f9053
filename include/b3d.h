/*
 * b3d.h - C ABI of libb3d, a GB300 (sm_103a) implementation of the render-and-score hot
 * path of Bayes3D's coarse-to-fine sequential Monte Carlo inference (Gothoskar et al.,
 * arXiv 2312.08715): many 6-DoF pose hypotheses of voxel-mesh objects are rasterised into
 * depth images, scored against an observed depth image under the paper's windowed
 * outlier-mixture likelihood (Eq. 1 with the window truncation of Sec. III-B), reduced to
 * one log-likelihood per hypothesis, normalised by log-sum-exp and resampled to seed the
 * next, finer pose grid (the coarse-to-fine proposal of Sec. III-B).
 *
 * Conventions shared by every entry point
 *   - Every call returns a b3d_status: B3D_OK (0) or a negative error. No exception or
 *     longjmp crosses the ABI. b3d_last_error() describes the last failure on a context.
 *   - Argument errors are detected on the host, before any work is queued. Device-side
 *     failures (a kernel's own bounds or timeout checks) set a flag in the context that
 *     b3d_sync() reports as B3D_EDEVICE.
 *   - Pointers named *_dev are caller-owned device memory on the context's device, 16-byte
 *     aligned, with the size each call states; the library neither frees nor retains them
 *     past the call (work queued on the stream reads/writes them asynchronously, so keep
 *     them alive until the stream reaches that point). Host pointers are read during the
 *     call only.
 *   - Meshes, the scene and all internal scratch are owned by the context and freed by
 *     b3d_destroy(). The context's device allocations count against hbm_budget_bytes.
 *   - All device work is asynchronous on the caller's stream (a cudaStream_t passed as
 *     b3d_stream; NULL is the legacy default stream). A context is not thread-safe: use
 *     one context per host thread, or serialise calls.
 *   - Poses are row-major 4x4 float32 cam_from_obj matrices (p_cam = R p_obj + t,
 *     t = (P[3], P[7], P[11]), bottom row 0 0 0 1). OpenCV camera axes: x right, y down,
 *     z forward. Pixel (u, v) is column u, row v; its ray passes through the pixel centre,
 *     ((u + 1/2 - cx)/fx, (v + 1/2 - cy)/fy, 1). Depth is camera z.
 *   - Images are row-major [H, W] float32; batches of images are [n, H, W].
 */
#ifndef B3D_H
#define B3D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t b3d_status;
#define B3D_OK 0
#define B3D_EINVAL (-1)    /* invalid argument (message in b3d_last_error) */
#define B3D_ENOMEM (-2)    /* a device or host allocation failed */
#define B3D_EBUDGET (-3)   /* the allocation would exceed the context's HBM budget */
#define B3D_ECUDA (-4)     /* a CUDA runtime call failed */
#define B3D_ETIMEOUT (-5)  /* a bounded wait expired */
#define B3D_ENOTFOUND (-6) /* unknown mesh id or object slot */
#define B3D_EDEVICE (-7)   /* a kernel raised the context's device error flag */
#define B3D_EBUSY (-8)     /* no free slot (server sessions, or a session's frame queue) */
#define B3D_ECLOSED (-9)   /* the session was closed (or the server stopped) before the frame ran */

#define B3D_MAX_STAGES 8
#define B3D_MAX_HALF_WINDOW 7

/* load_mesh flags */
#define B3D_MESH_CLOSED 1  /* closed, outward-oriented (counter-clockwise seen from outside)
                              solid, e.g. a voxel mesh: back faces and coincident internal
                              face pairs can never be the nearest surface, so the library
                              skips them (triangle ids reported stay the original ones) */

typedef struct b3d_ctx b3d_ctx;
typedef void *b3d_stream; /* cudaStream_t */

/* Pinhole camera: image size, focal lengths and principal point in pixels, near/far planes
 * in metres. A triangle with a vertex closer than near_z is not drawn; fragments beyond
 * far_z are dropped; a pixel without a fragment renders at far_z. */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy, near_z, far_z;
} b3d_intrinsics;

/* Likelihood of Eq. 1, truncated to a (2w+1)^2 pixel window (Sec. III-B):
 *   l_i = log( p_out / V + (1 - p_out) / K * sum_{j in win(i)} k(qt_i, q_j) )
 * over observed pixels i with finite depth > 0 (qt_i its point), rendered points q_j.
 *   kind 0 ("plain"): k = 1{|qt - q|^2 <= r^2} / ((4/3) pi r^3)   (inlier ball)
 *   kind 1 ("smooth"): k = (2 pi s^2)^(-3/2) exp(-|qt - q|^2 / (2 s^2))
 * radius is r (kind 0) or s (kind 1), metres. volume <= 0 selects V = the camera frustum
 * between near and far, (W H / (fx fy)) (far^3 - near^3) / 3; norm <= 0 selects
 * K = (2w+1)^2 (window slots outside the image count in K and contribute 0).
 * miss_mode 0: a rendered pixel without a triangle is a point on the far plane;
 * miss_mode 1: it carries no point. 0 <= half_window <= B3D_MAX_HALF_WINDOW,
 * 0 < p_outlier < 1, radius > 0. */
typedef struct {
    int32_t kind;
    float radius;
    float p_outlier;
    int32_t half_window;
    float volume;
    float norm;
    int32_t miss_mode;
} b3d_lik_params;

/* One coarse-to-fine stage (a partition Pi_t of Sec. III-B): an n^3 translation grid of
 * spacing step (odd n centred, even n with the centre at index n/2) times a rotation set
 * of n_rot rotations, hypothesis h = ((ir * n + ix) * n + iy) * n + iz with
 *   R_h = R_centre R_ir,  t_h = t_centre + G (o_ix, o_iy, o_iz).
 * rot_kind 0: Fibonacci-sphere set, R_k the minimal-arc rotation taking +z to
 *   d_k = (sqrt(1-z^2) cos(2 pi k / phi), sqrt(1-z^2) sin(2 pi k / phi), z),
 *   z = 1 - (2k+1)/n_rot, phi the golden ratio;
 * rot_kind 1: perturbation set, uniform in the ball of rotation vectors of radius rot_max:
 *   R_0 = I; for k >= 1, R_k = Exp(rot_max cbrt(u0) e), e = (sqrt(1-z^2) cos(2 pi u2),
 *   sqrt(1-z^2) sin(2 pi u2), z), z = 1 - 2 u1, (u0, u1, u2) = frac(1/2 + k (1/g, 1/g^2, 1/g^3))
 *   the 3-D R-sequence (g^4 = g + 1), evaluated in exact 64-bit fixed point. */
typedef struct {
    int32_t n_per_axis;
    float step;
    int32_t rot_kind;
    int32_t n_rot;
    float rot_max;
} b3d_stage;

/* A coarse-to-fine schedule: stages, particles drawn per stage, the seed of the
 * counter-based generator, and G, the rotation (row-major 3x3, cam_from_grid) whose
 * columns are the translation grid's axes in the camera frame. path_density selects what
 * logq reports: 0, the last stage's proposal density of each particle given that stage's
 * grid (log P_T(cell) - 3 log step_T); 1, the density of the whole coarse-to-fine path
 * (the sum over stages of the log probability of the cell that centred the next stage,
 * plus the last stage's term), which is the proposal density q of Sec. III-B when
 * n_particles = 1 (each particle its own proposal). */
typedef struct {
    int32_t n_stages;
    b3d_stage stage[B3D_MAX_STAGES];
    int32_t n_particles;
    uint64_t seed;
    float grid_frame[9];
    int32_t path_density;
} b3d_c2f_schedule;

/* Create a context on CUDA device `device`. Allocations made on its behalf may total at
 * most hbm_budget_bytes (0 = no limit). *out receives the context, or NULL on error. */
b3d_status b3d_create(b3d_ctx **out, int32_t device, uint64_t hbm_budget_bytes);

/* Free the context and everything it owns. Waits for the device to finish its work. */
b3d_status b3d_destroy(b3d_ctx *ctx);

/* Message of the last failed call on ctx (never NULL; "" after success). With ctx NULL,
 * the message of the last failed b3d_create on this thread. Valid until the next call. */
const char *b3d_last_error(b3d_ctx *ctx);

/* Number of kernels the library launched on this context so far (a running count). */
int64_t b3d_launch_count(b3d_ctx *ctx);

/* Load an object model (the paper's voxel object model, Sec. III: voxels placed on the
 * points of a fused cloud; here any triangle mesh). verts: host [n_v, 3] float32 object
 * frame; faces: host [n_f, 3] int32 vertex indices in [0, n_v). flags: B3D_MESH_CLOSED or 0.
 * Triangle ids reported by the renderer are face indices of this array (offset per scene
 * object, see b3d_set_scene). *mesh_id receives a context-local id. n_f >= 1. */
b3d_status b3d_load_mesh(b3d_ctx *ctx, const float *verts, int64_t n_v, const int32_t *faces, int64_t n_f,
                         int32_t flags, int32_t *mesh_id);

/* Set the scene (the scene graph of Alg. 1, flattened): n_obj objects, object k is mesh
 * mesh_ids[k] at host pose poses[16 k .. 16 k + 15]; camera intrinsics; and the observed
 * depth image obs_depth_dev [H, W] (copied to an observed point cloud on the device; the
 * caller's buffer is no longer needed once the stream has passed this call). Pixels with
 * depth <= 0 or not finite are not scored. The global triangle id of face f of object k is
 * f + (sum of the face counts of objects 0..k-1). */
b3d_status b3d_set_scene(b3d_ctx *ctx, const b3d_intrinsics *intr, int32_t n_obj, const int32_t *mesh_ids,
                         const float *poses, const float *obs_depth_dev, b3d_stream stream);

/* Replace the observed depth image of the current scene (same size). */
b3d_status b3d_set_observation(b3d_ctx *ctx, const float *obs_depth_dev, b3d_stream stream);

/* Set the pose of scene object `obj` from device memory pose_dev [16] (no host round
 * trip; used to fix an object at a pose found on the device). */
b3d_status b3d_set_object_pose_dev(b3d_ctx *ctx, int32_t obj, const float *pose_dev, b3d_stream stream);

/* Render n_hyp hypotheses (the depth renderer of Alg. 1, DepthRenderer): the scene with
 * object obj_slot at poses_dev [n_hyp, 16] and every other object at its scene pose.
 * Writes depth_dev [n_hyp, H, W] (far_z where nothing is drawn) and, unless NULL,
 * triid_dev [n_hyp, H, W] (global triangle id, -1 where nothing is drawn). Nearest
 * fragment wins; equal depths go to the smaller triangle id. */
b3d_status b3d_render_batch(b3d_ctx *ctx, int32_t obj_slot, int64_t n_hyp, const float *poses_dev, float *depth_dev,
                            int32_t *triid_dev, b3d_stream stream);

/* Render and score n_hyp hypotheses in one pass (render, Eq. 1 likelihood per observed
 * pixel, sum over pixels): loglik_dev [n_hyp] receives sum_i l_i for the scene with
 * object obj_slot at poses_dev [n_hyp, 16]. The rendered images never leave the chip. */
b3d_status b3d_score_batch(b3d_ctx *ctx, int32_t obj_slot, int64_t n_hyp, const float *poses_dev,
                           const b3d_lik_params *lik, float *loglik_dev, b3d_stream stream);

/* Score materialised depth images under the Eq. 1 likelihood: depth_dev [n_hyp, H, W] (e.g.
 * from b3d_render_batch) against the scene's observation; triid_dev [n_hyp, H, W] is needed only for
 * miss_mode 1 (pixels with id -1 carry no point), else may be NULL. loglik_dev [n_hyp]
 * receives sum_i l_i. The images may hold any depths. A pixel whose window holds exactly
 * the depths of a reference image takes the reference's term, computed once per scene and
 * likelihood (the same value, bit for bit), so the cost follows the region where an image
 * differs from the reference: the scene without object obj_slot (images of that object
 * re-posed, as b3d_render_batch writes them, differ only around it), or with every object
 * when obj_slot is -1. The choice changes the sums only by FP32 summation order. */
b3d_status b3d_score_depth_batch(b3d_ctx *ctx, int32_t obj_slot, int64_t n_hyp, const float *depth_dev,
                                 const int32_t *triid_dev, const b3d_lik_params *lik, float *loglik_dev,
                                 b3d_stream stream);

/* Expand one coarse-to-fine stage (the partition of the pose region into cells, Sec. III-B)
 * around centre_pose (host [16]) with grid frame G (host [9], row-major cam_from_grid):
 * poses_dev [n^3 * n_rot, 16] in hypothesis order (see b3d_stage). */
b3d_status b3d_expand_hypotheses(b3d_ctx *ctx, const float *centre_pose, const float *grid_frame,
                                 const b3d_stage *stage, float *poses_dev, b3d_stream stream);

/* Log-sum-exp normalisation and categorical resampling (Sec. III-B: the next region is
 * sampled with probability proportional to its score). For loglik_dev [n] (n >= 1):
 * logz_dev [1] = log sum_h exp(ll_h); for draw k < m, u_k = the top 24 bits of the first
 * word of Philox4x64-10 (Salmon et al., SC'11) at counter (k, stage, 0, 0) and key
 * (seed, 0), divided by 2^24; idx_dev[k] = min{ h : sum_{g<=h} exp(ll_g) > u_k sum_g exp(ll_g) }
 * and logq_dev[k] = ll[idx_k] - logz. m may be 0 (idx/logq then unused). */
b3d_status b3d_lse_resample(b3d_ctx *ctx, int64_t n, const float *loglik_dev, int32_t m, uint64_t seed,
                            int32_t stage, float *logz_dev, int32_t *idx_dev, float *logq_dev, b3d_stream stream);

/* One rank's part of b3d_lse_resample when the scores of one categorical (one C2F stage,
 * Sec. III-B) are split over ranks in contiguous shards, rank r holding scores
 * [index_base, index_base + n) of the whole vector. With logz_r the log normaliser of each
 * rank's shard (this call's logz_dev, or b3d_lse_resample with m = 0), log Z the
 * log-sum-exp of all logz_r, mass_before = sum over earlier ranks of exp(logz_r - log Z)
 * and mass = exp(logz_r - log Z) (the last rank passes 1 - mass_before, so that every
 * uniform has an owner): draw k (the uniform u_k of b3d_lse_resample, same seed, stage and
 * counter) belongs to this rank when mass_before <= u_k < mass_before + mass, and then
 * idx_dev[k] = index_base + min{ h : sum_{g<=h} exp(ll_g) > ((u_k - mass_before) / mass)
 * sum_g exp(ll_g) } over this shard, which in exact arithmetic is the index the unsplit
 * call draws; logq_dev[k] = ll[idx] - logz_global. Draws of other ranks get idx -1 and logq
 * -inf, so combining the ranks' outputs by maximum gives every draw. logz_dev [1] receives
 * this shard's own log normaliser. Errors: B3D_EINVAL for n outside [1, 2^31-1], m < 0,
 * NULL outputs, masses outside [0, 1] or index_base + n > 2^31. */
b3d_status b3d_lse_resample_shard(b3d_ctx *ctx, int64_t n, const float *loglik_dev, int32_t m, uint64_t seed,
                                  int32_t stage, double mass_before, double mass, double logz_global, int64_t index_base,
                                  float *logz_dev, int32_t *idx_dev, float *logq_dev, b3d_stream stream);

/* Log-sum-exp and resampling for callers that cannot allocate device memory. The paper has
 * no counterpart: this is a library service. It computes exactly what b3d_lse_resample
 * computes (same kernel, same definition of idx/logq/logz), without a context and without
 * allocating: the kernel's scratch (1024 partial sums and a completion counter, 8 KB) is a
 * fixed array inside the library that every GPU loading the library holds until the
 * process exits. Callers that cannot allocate include code under another framework's
 * allocator lock or hard memory cap (an allocation would deadlock or fail), loops that
 * cannot afford the implicit device synchronisation an allocation may bring, and
 * embeddings that forbid the library from allocating.
 *   - Works on the calling thread's current device. The first call on a device (and the
 *     first after the device's context was reset) looks up the array's device address,
 *     which may load the library's module there; make that first call before any stream
 *     capture begins.
 *   - Every call shares the one array and clears its counter on `stream` first; calls
 *     that overlap on the GPU (other streams, other threads) race: serialise them.
 *   - n must be in [1, B3D_NOALLOC_MAX_SCORES] (else B3D_EINVAL), m >= 0, outputs as in
 *     b3d_lse_resample. If every score is -inf (m > 0), every idx is -1, every logq -inf
 *     and logz -inf: that is how this call reports the case (there is no context, so no
 *     b3d_sync flag and no b3d_last_error text). Returns B3D_EINVAL or B3D_ECUDA on error. */
#define B3D_NOALLOC_MAX_SCORES 2147483647LL
b3d_status b3d_lse_resample_noalloc(int64_t n, const float *loglik_dev, int32_t m, uint64_t seed, int32_t stage,
                                    float *logz_dev, int32_t *idx_dev, float *logq_dev, b3d_stream stream);

/* Coarse-to-fine enumeration of object obj_slot's pose (Sec. III-B). Stage t expands
 * its grid around centre_t (centre_0 = centre_pose, host [16]), scores every hypothesis
 * with lik (scoring strategy: the cell centre, weight 1), draws n_particles cells by
 * b3d_lse_resample(seed, stage t), and takes as centre_{t+1} the drawn cell with the
 * highest score (ties to the smaller index). After the last stage, particle k is its
 * drawn cell's pose moved uniformly within the cell, t += G ((u0-1/2) s, (u1-1/2) s,
 * (u2-1/2) s) with (u0, u1, u2) the top-24-bit uniforms of words 0..2 of Philox at
 * counter (k, n_stages, 1, 0), key (seed, 0):
 *   particles_dev [M, 16], logw_dev [M] = the drawn cell's score,
 *   logq_dev [M] = score - logZ_last - 3 log(s_last)   (proposal density q).
 * Every step runs on the device; the call can be captured into a CUDA graph once it has
 * run once with the same sizes (scratch is sized on first use). */
b3d_status b3d_enumerate_c2f(b3d_ctx *ctx, int32_t obj_slot, const float *centre_pose,
                             const b3d_c2f_schedule *schedule, const b3d_lik_params *lik, float *particles_dev,
                             float *logw_dev, float *logq_dev, b3d_stream stream);

/* Batched form (the paper has one scene at a time; this is how many independent scenes
 * share one GPU): the hypotheses of every item, each item a scene held by its own context
 * (its current b3d_set_scene) on the owner's device, are rendered and scored in ONE
 * persistent launch whose CTAs take batch_chunk hypotheses at a time from a work queue over
 * (scene, hypothesis chunk). Items may differ in image size, meshes, object slot and
 * hypothesis count; the likelihood is shared (its frustum volume is each scene's own).
 * Scores equal those of b3d_score_batch on each scene alone. The owner's context supplies
 * the launch shape (b3d_tuning) and the scratch; scratch is sized on first use, after
 * which the call can be captured into a CUDA graph (it allocates nothing and only copies its
 * descriptors from pinned host memory). */
typedef struct {
    b3d_ctx *scene;          /* context holding the scene */
    int32_t obj_slot;
    int64_t n_hyp;
    const float *poses_dev;  /* [n_hyp, 16] */
    float *loglik_dev;       /* [n_hyp] */
} b3d_score_item;

b3d_status b3d_score_multi(b3d_ctx *owner, int32_t n_items, const b3d_score_item *items, const b3d_lik_params *lik,
                           b3d_stream stream);

/* Batched coarse-to-fine enumeration: every item runs b3d_enumerate_c2f on its own scene and
 * schedule (all schedules with the same number of stages); each stage is one batched score
 * launch, one batched log-sum-exp + resampling launch and one batched selection launch over
 * all items. Outputs per item as b3d_enumerate_c2f. An item's centre may be read from
 * device memory (centre_dev, copied before the first stage, so it may point into the
 * item's own particles_dev). Same graph-capture rule as b3d_score_multi. */
typedef struct {
    b3d_ctx *scene;
    int32_t obj_slot;
    float centre_pose[16];        /* host centre, used when centre_dev is NULL */
    const float *centre_dev;      /* device [16] centre (e.g. a previous particle), or NULL */
    b3d_c2f_schedule schedule;
    float *particles_dev;  /* [M, 16] */
    float *logw_dev;       /* [M] */
    float *logq_dev;       /* [M] */
    float *map_dev;        /* [16] or NULL: the highest-scoring cell drawn at the last stage */
} b3d_c2f_item;

b3d_status b3d_enumerate_multi(b3d_ctx *owner, int32_t n_items, const b3d_c2f_item *items, const b3d_lik_params *lik,
                               b3d_stream stream);

/* Forward and backward of the smooth (kind 1) likelihood, Eq. 1 with its Gaussian mixture
 * components (sigma and p_outlier the noise parameters of Alg. 1), for n_hyp poses: loglik_dev [n],
 * dpose_dev [n, 6] = d loglik / d xi at xi = 0 for the left perturbation
 * T(xi) = Exp([v, w]^) T in the camera frame, ordered (v, w), with visibility held fixed
 * and each rendered point sliding along its pixel ray on the plane of its face (the voxel
 * rectangle, or the triangle of a mesh without rectangles, the forward renders);
 * dsigma_dev [n] and dpout_dev [n] = d loglik / d s and d loglik / d p_outlier. Any of the
 * gradient outputs may be NULL. The forward is recomputed; nothing per pixel is stored. */
b3d_status b3d_score_grad(b3d_ctx *ctx, int32_t obj_slot, int64_t n_hyp, const float *poses_dev,
                          const b3d_lik_params *lik, float *loglik_dev, float *dpose_dev, float *dsigma_dev,
                          float *dpout_dev, b3d_stream stream);

/* Gradient pose refinement under the smooth (kind 1) likelihood, every step on the device:
 * n_steps Adam steps (learning rate lr, moments beta1, beta2, epsilon eps, as torch.optim.Adam
 * without weight decay) ascending loglik in the left se(3) perturbation of b3d_score_grad,
 * each step re-basing the pose (T <- Exp([v, w]^) T, so the perturbation restarts at 0 and
 * its gradient stays exact): one forward + backward launch and one update launch per step.
 * poses_dev [n, 16] (row-major 4x4) is updated in place; loglik_dev [n] (may be NULL)
 * receives the log-likelihood at the poses the last step scored (before its update). The
 * Adam moments live in context scratch and start at 0 on every call. n_steps >= 1,
 * lr > 0, 0 <= beta1, beta2 < 1, eps > 0. */
b3d_status b3d_refine_smooth(b3d_ctx *ctx, int32_t obj_slot, int64_t n_hyp, float *poses_dev,
                             const b3d_lik_params *lik, int32_t n_steps, float lr, float beta1, float beta2, float eps,
                             float *loglik_dev, b3d_stream stream);

/* The left se(3) update of the gradient's parameterisation (the convention of
 * b3d_score_grad): out_dev[i] = Exp([v_i, w_i]^) poses_dev[i] for n twists xi_dev [n, 6]
 * ordered (v, w) and row-major 4x4 poses [n, 16]; Exp by Rodrigues' formula and the SE(3) V
 * matrix, in FP32 with series forms below a rotation of 0.1 rad. out_dev may be poses_dev.
 * The same arithmetic re-bases the poses inside b3d_refine_smooth. n >= 0; B3D_EINVAL for
 * NULL buffers when n > 0. */
b3d_status b3d_se3_compose(b3d_ctx *ctx, int64_t n, const float *xi_dev, const float *poses_dev, float *out_dev,
                           b3d_stream stream);

/* Camera hypotheses (the camera-pose tracking of Sec. IV, Table 1): render n_hyp hypothesised
 * camera poses poses_dev [n_hyp, 16] (row-major camera_from_world) of the scene, every object
 * k at H_h P_k where P_k is its scene pose read as world_from_object. Writes depth_dev
 * [n_hyp, H, W] (far_z where nothing is drawn) and, unless NULL, triid_dev [n_hyp, H, W], as
 * b3d_render_batch; score them with b3d_score_depth_batch. */
b3d_status b3d_render_camera_batch(b3d_ctx *ctx, int64_t n_hyp, const float *poses_dev, float *depth_dev,
                                   int32_t *triid_dev, b3d_stream stream);

/* Hierarchical noise (Alg. 1: p_out ~ U(0,1), sigma ~ U(0, sigma_max), hypotheses scored
 * under several noise settings): a grid of n_radius inlier radii (kind 0)
 * or Gaussian standard deviations (kind 1) times n_pout outlier probabilities. Setting
 * g = i * n_pout + j is (radius[i], p_outlier[j]); log_weight[g] is the log of its prior mass
 * (quadrature weight; all 0 for equal weights). volume, norm, miss_mode as b3d_lik_params. */
#define B3D_MAX_NOISE_R 4
#define B3D_MAX_NOISE_P 4
typedef struct {
    int32_t kind;
    int32_t half_window; /* 0..2 */
    int32_t n_radius;    /* 1..B3D_MAX_NOISE_R */
    int32_t n_pout;      /* 1..B3D_MAX_NOISE_P */
    float radius[B3D_MAX_NOISE_R];
    float p_outlier[B3D_MAX_NOISE_P];
    float log_weight[B3D_MAX_NOISE_R * B3D_MAX_NOISE_P];
    float volume;
    float norm;
    int32_t miss_mode;
} b3d_noise_grid;

/* Score n_hyp hypotheses of object obj_slot (poses_dev [n_hyp, 16]) under every setting of
 * the noise grid in one fused pass (each hypothesis rendered once): loglik_dev
 * [n_hyp, n_radius * n_pout] (may be NULL) receives the log-likelihood under each setting,
 * marginal_dev [n_hyp] log sum_g exp(loglik_g + log_weight_g), the likelihood with the noise
 * marginalised over the grid. */
b3d_status b3d_score_noise_batch(b3d_ctx *ctx, int32_t obj_slot, int64_t n_hyp, const float *poses_dev,
                                 const b3d_noise_grid *grid, float *loglik_dev, float *marginal_dev,
                                 b3d_stream stream);

/* Launch shape of the fused render + score kernel (no counterpart in the paper: a property
 * of this implementation). tile_w: widest screen tile in pixels (8..256); cta_threads: 32,
 * 64, 128 or 256 (one hypothesis per CTA at a time); ctas_per_sm: CTAs resident per SM
 * (0 = as many as fit); high_occupancy: 1 selects the build whose registers are capped so
 * that more CTAs fit on an SM, 0 the regular one; batch_chunk (1..1024): see b3d_score_multi. */
typedef struct {
    int32_t tile_w;
    int32_t cta_threads;
    int32_t ctas_per_sm;
    int32_t high_occupancy;
    int32_t batch_chunk; /* batched form: hypotheses a CTA takes from the work queue at a time */
} b3d_tuning;

b3d_status b3d_get_tuning(b3d_ctx *ctx, b3d_tuning *out);
b3d_status b3d_set_tuning(b3d_ctx *ctx, const b3d_tuning *tuning);

/* Autotuner: times the score kernel on one coarse-to-fine stage of object obj_slot of the
 * current scene (grid around centre_pose, host [16]; grid_frame host [9]) for each
 * candidate launch shape (CTA size x tile width x CTAs per SM), keeps the fastest in the
 * context and returns it in *best (may be NULL). Synchronises the stream (not for use while
 * capturing a graph); run it once per workload shape, e.g. during warm-up. */
b3d_status b3d_autotune(b3d_ctx *ctx, int32_t obj_slot, const float *centre_pose, const float *grid_frame,
                        const b3d_stage *stage, const b3d_lik_params *lik, b3d_tuning *best, b3d_stream stream);

/* Autotuner for the batched form: times b3d_enumerate_multi on these items (owner, items and
 * lik as there) for the owner's current launch shape and for 128- or 256-thread CTAs with 64-
 * or 128-pixel tiles, then the fastest shape with 1 to 32 hypotheses per work-queue grab;
 * keeps the fastest tuning in the owner and returns it in *best (may be NULL). The items'
 * outputs hold the last timed run's results. Synchronises the stream (not for use while
 * capturing a graph). No counterpart in the paper: the launch shape is a property of this
 * implementation, and a mix of scenes of uneven size may want another shape than any one
 * scene (b3d_autotune times a single stage of one object). */
b3d_status b3d_autotune_multi(b3d_ctx *owner, int32_t n_items, const b3d_c2f_item *items, const b3d_lik_params *lik,
                              b3d_tuning *best, b3d_stream stream);

/* Instrumentation (off by default; used by the benchmark).
 * flags bit 0 (B3D_INSTR_TIMING): bracket every kernel launch of the library with CUDA
 *   events recorded on the launching stream; b3d_kernel_time() reports the device time.
 * flags bit 1 (B3D_INSTR_WORK): the render/score kernels count the work they do
 *   (b3d_work_counters); counting slows them, so never enable it for a timed run. */
#define B3D_INSTR_TIMING 1
#define B3D_INSTR_WORK 2
b3d_status b3d_set_instrumentation(b3d_ctx *ctx, int32_t flags);

/* Kernel classes for b3d_kernel_time. */
#define B3D_K_SCORE 0       /* fused render + score (b3d_score_batch, b3d_enumerate_c2f) */
#define B3D_K_RENDER 1      /* b3d_render_batch */
#define B3D_K_SCORE_DEPTH 2 /* b3d_score_depth_batch */
#define B3D_K_RESAMPLE 3    /* log-sum-exp + resampling */
#define B3D_K_SELECT 4      /* coarse-to-fine centre selection / particles */
#define B3D_K_GRAD 5        /* b3d_score_grad */
#define B3D_K_SCENE 6       /* scene set-up: observed points, background render and tables, grids */
#define B3D_K_COUNT 7

/* Device time (milliseconds) and number of launches of one kernel class recorded since the
 * previous call for that class (waits for the recorded events; then resets the class). */
b3d_status b3d_kernel_time(b3d_ctx *ctx, int32_t kernel_class, double *total_ms, int64_t *launches);

/* Work counted by the render/score kernels since the previous call (then cleared; waits
 * for the device): out[8] = hypotheses, vertices transformed, triangles processed,
 * pixel-centre coverage tests, fragments written, z-buffer pixels composited, observed
 * pixels scored, window pairs evaluated. */
b3d_status b3d_work_counters(b3d_ctx *ctx, int64_t *out);

/* Wait for the stream, then report (and clear) the context's device error flag. */
b3d_status b3d_sync(b3d_ctx *ctx, b3d_stream stream);

/* ==========================================================================================
 * Serving: a tracking server (the particle-filter tracking loop of Sec. IV, Table 1,
 * applied to object poses) that accepts depth frames from many concurrent sessions and
 * batches them continuously.
 *
 * Each session owns a scene (its meshes, camera, fixed objects) and, on the device, the
 * pose estimate and particles of each tracked object. A frame runs, for every tracked
 * object k, one coarse-to-fine enumeration (the server's schedule) centred on object k's
 * current estimate, scored against the new depth frame with every other object held at
 * its estimate from the previous frame; object k's new estimate is the highest-scoring
 * cell drawn at the last stage, and its particles are kept on the device. All tracked
 * objects of a frame are enumerated together, in one batched launch.
 *
 * Continuous batching: a worker thread issues a batch as soon as fewer than max_inflight
 * batches are on the device and any session has a queued frame. A batch takes the oldest
 * queued frame of every ready session (at most one frame per session, at most
 * max_batch_items tracked objects), so frames that arrive while others run join the next
 * batch rather than waiting for a fixed schedule. Frames of one session run in submission
 * order. Every result is independent of which other frames shared its batch: the kernels
 * compute each item on its own, with a launch shape fixed at server creation, and the
 * random draws of frame f, object k come from b3d_frame_seed(session seed, f, k).
 *
 * Admission: a session is admitted only if its device memory (measured after building
 * its meshes, scene and per-object buffers) fits in the server's HBM budget next to the
 * sessions already admitted and the batch scratch reserved at creation; otherwise
 * b3d_session_open returns B3D_EBUDGET (after waiting up to its timeout for a close).
 *
 * Thread safety: every b3d_server_* / b3d_session_* / b3d_frame_* call may be made from
 * any host thread. Closing a session or destroying the server frees device memory, which
 * waits for the device.
 * ========================================================================================== */
typedef struct b3d_server b3d_server;

typedef struct {
    int32_t max_sessions;     /* session slots, >= 1 */
    int32_t max_batch_items;  /* tracked objects per batched launch, >= 1 (batch scratch is
                                 reserved for this many at creation) */
    int32_t max_batch_frames; /* frames per batched launch (0: no limit; 1: no batching across
                                 sessions) */
    int32_t max_inflight;     /* batches on the device at once, 1..2 (2: the next batch is
                                 issued while one runs) */
    int32_t queue_depth;      /* frames a session may have submitted and not completed, 1..64 */
    int32_t device_timeout_ms; /* a batch not finished after this long fails the server
                                  (B3D_ETIMEOUT); 0 = 60000 */
    int32_t batch_linger_us;  /* while a batch runs, wait up to this long for more frames
                                 before issuing the next one (0: issue at once); the wait
                                 ends early once every session has a frame queued */
    b3d_lik_params lik;       /* likelihood of every session */
    b3d_c2f_schedule schedule; /* per object and frame; its seed is replaced by b3d_frame_seed */
    b3d_tuning tuning;        /* launch shape of the score kernel (tile_w 0: library default) */
} b3d_server_config;

/* One session's scene. Object k is the mesh verts[k] [n_v[k], 3] / faces[k] [n_f[k], 3]
 * (host, read during the call; mesh_flags[k] as b3d_load_mesh, or all 0 when NULL) at pose
 * poses[16 k ..]. Objects 0 .. n_track-1 are tracked: poses[] is their estimate before
 * frame 0. Objects n_track .. n_obj-1 (a table, walls) stay where poses[] puts them.
 * grid_frame (row-major cam_from_grid) orients this session's translation grids; all zero
 * takes the server schedule's. */
typedef struct {
    b3d_intrinsics intr;
    int32_t n_obj;
    int32_t n_track;  /* 1 .. n_obj */
    const float *const *verts;
    const int64_t *n_v;
    const int32_t *const *faces;
    const int64_t *n_f;
    const int32_t *mesh_flags;
    const float *poses;
    uint64_t seed;
    float grid_frame[9];
} b3d_session_desc;

/* Completion record of one frame. */
typedef struct {
    int64_t ticket;
    int32_t session;
    int32_t status;          /* B3D_OK, B3D_EDEVICE (a kernel flag), B3D_ECLOSED or B3D_ETIMEOUT */
    int64_t frame_index;     /* 0-based within the session */
    double latency_ms;       /* b3d_frame_submit entry -> result on the host */
    double queue_ms;         /* b3d_frame_submit entry -> issued to the device */
    int32_t batch_frames;    /* frames in the batch it ran in */
    int32_t n_track;         /* poses returned */
} b3d_frame_result;

typedef struct {
    int64_t frames_done;     /* completed with B3D_OK */
    int64_t frames_failed;   /* completed with another status */
    int64_t batches;
    int64_t hypotheses;      /* scored by completed batches */
    int32_t sessions;
    int32_t max_batch_frames_seen;
    uint64_t hbm_budget, hbm_reserved; /* bytes: budget; sessions + batch scratch admitted */
    uint64_t hbm_used;       /* bytes the server's contexts hold now */
} b3d_server_stats;

/* Create a server on `device` with at most hbm_budget_bytes of device memory (0: no
 * limit); starts its worker and completion threads. B3D_EBUDGET if the batch scratch
 * alone does not fit. */
b3d_status b3d_server_create(b3d_server **out, int32_t device, uint64_t hbm_budget_bytes,
                             const b3d_server_config *cfg);

/* Cancel queued frames (B3D_ECLOSED), wait for batches on the device (bounded by the
 * device timeout), stop the threads and free everything. */
b3d_status b3d_server_destroy(b3d_server *srv);

/* Message of the calling thread's last failed server call ("" after success). */
const char *b3d_server_last_error(void);

/* Build and admit a session. Waits up to timeout_ms (0: no wait) for a slot or budget to
 * free up; B3D_EBUSY (no slot) or B3D_EBUDGET (no memory) when it does not. */
b3d_status b3d_session_open(b3d_server *srv, const b3d_session_desc *desc, int32_t timeout_ms,
                            int32_t *session_id);

/* Cancel the session's queued frames (their results report B3D_ECLOSED), wait for its
 * frames on the device (B3D_ETIMEOUT after the device timeout) and free it. */
b3d_status b3d_session_close(b3d_server *srv, int32_t session_id);

/* Queue a depth frame (host [H, W] float32, copied during the call; pixels <= 0 or not
 * finite are not scored). Waits up to timeout_ms for a free queue entry (B3D_EBUSY when
 * none frees). *ticket identifies the frame. */
b3d_status b3d_frame_submit(b3d_server *srv, int32_t session_id, const float *depth, int32_t timeout_ms,
                            int64_t *ticket);

/* Wait up to timeout_ms for frame `ticket` (B3D_ETIMEOUT if not finished; B3D_ENOTFOUND if
 * unknown or already collected). On return the result is collected: *res is filled and,
 * when poses is non-NULL, poses [n_track, 16] (room for poses_capacity floats; B3D_EINVAL,
 * result kept, when too small) receives the new estimates. The call's status is B3D_OK
 * whenever a result was returned; the frame's own status is res->status. */
b3d_status b3d_frame_wait(b3d_server *srv, int64_t ticket, int32_t timeout_ms, b3d_frame_result *res,
                          float *poses, int32_t poses_capacity);

/* Like b3d_frame_wait for whichever uncollected frame finished first. */
b3d_status b3d_frame_next(b3d_server *srv, int32_t timeout_ms, b3d_frame_result *res, float *poses,
                          int32_t poses_capacity);

/* Stop (1) or resume (0) issuing new batches; batches on the device still finish. Frames
 * keep queueing while paused. */
b3d_status b3d_server_pause(b3d_server *srv, int32_t paused);

b3d_status b3d_server_get_stats(b3d_server *srv, b3d_server_stats *out);

/* Checkpoint of a session's tracking state: estimates [n_track, 16], particles
 * [n_track, M, 16] and their log scores [n_track, M] (M = schedule.n_particles; host
 * arrays; NULL skips one), and the index of the next frame. The session must be idle (no
 * queued or running frame): B3D_EBUSY otherwise. */
b3d_status b3d_session_export(b3d_server *srv, int32_t session_id, float *poses, float *particles, float *logw,
                              int64_t *next_frame);
/* Restore a checkpoint into an idle session of the same shape (the next frame continues
 * from it exactly as the exporting session would have). */
b3d_status b3d_session_import(b3d_server *srv, int32_t session_id, const float *poses, const float *particles,
                              const float *logw, int64_t next_frame);

/* Seed of the random draws of frame `frame` of object `obj` in a session seeded `seed`
 * (SplitMix64 finaliser over the three values; pure host function). */
uint64_t b3d_frame_seed(uint64_t seed, int64_t frame, int32_t obj);

#ifdef __cplusplus
}
#endif

#endif /* B3D_H */
