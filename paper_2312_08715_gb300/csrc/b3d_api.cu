// b3d_api.cu - host runtime behind the C ABI of include/b3d.h: the context (device
// allocations under an HBM budget, error reporting, launch counting), mesh preparation
// (vertex welding, culling of coincident internal faces of closed meshes, spatial chunking
// for shared-memory staging), scene state (observed point cloud, background z-buffer of
// the fixed objects and its likelihood tables, cached per object slot and likelihood), and
// the dispatch of every entry point onto the caller's stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "b3d.h"
#include "b3d_internal.h"

using namespace b3d;

namespace {

struct MeshRec {
    int64_t n_faces = 0;  // original face count (triangle ids are 0..n_faces-1)
    int32_t flags = 0;
    float4 *verts = nullptr;
    int4 *tris_surf = nullptr, *tris_full = nullptr, *faces = nullptr;
    int n_surf = 0, n_full = 0, n_verts = 0;
    float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    // voxel quads (n_quads == 0: none)
    uint2 *quads = nullptr;
    int *class_off = nullptr;
    float *coords = nullptr;
    int n_quads = 0, nc[3] = {0, 0, 0}, np1 = 0;
};

struct LikKey {
    int kind, w, miss_mode;
    float radius, p_out, volume, norm;
    bool operator==(const LikKey &o) const {
        return kind == o.kind && w == o.w && miss_mode == o.miss_mode && radius == o.radius && p_out == o.p_out &&
               volume == o.volume && norm == o.norm;
    }
};

thread_local std::string g_create_error;

// Background of one object slot: z-buffer of the other scene objects, the per-pixel terms
// of the fixed objects alone and their sums. Each slot keeps its own, so hypotheses of
// different objects of one scene can be scored in the same launch.
struct BgCache {
    unsigned long long *bg = nullptr;
    float *bgd = nullptr;  // [2][npx] background depth under miss modes 0 and 1
    float *ell = nullptr, *gs = nullptr, *gp = nullptr;
    float2 *qe = nullptr;     // score kernels' packed (observed depth, ell) per pixel
    unsigned *bgz = nullptr;  // and background depth bits, both written with ell
    double *sums = nullptr, *part = nullptr;  // sums [3]; per-block partials of the table kernel
    unsigned *counter = nullptr;               // its last-block ticket (zero between launches)
    int64_t cap = 0, gcap = 0;
    bool dirty = true, lik_valid = false, grad_valid = false, bgd_valid = false;
    LikKey key{};
    // noise-grid tables [kMaxNoise][H W], their sums [kMaxNoise], partials and ticket
    float *nell = nullptr;
    double *nsums = nullptr, *npart = nullptr;
    unsigned *ncounter = nullptr;
    int64_t ncap = 0;
    bool nvalid = false;
    b3d_noise_grid nkey{};
};

}  // namespace

struct b3d_ctx {
    int device = 0;
    uint64_t budget = 0, used = 0;
    std::string err;
    int64_t launches = 0;
    std::map<void *, size_t> allocs;
    std::vector<MeshRec> meshes;

    // scene
    bool has_scene = false;
    Cam cam{};
    std::vector<int32_t> obj_mesh;
    // per-object z-buffers for shared slot backgrounds (see ctx_prepare_shared_bg)
    std::vector<unsigned long long *> objz;
    std::vector<char> objz_ok;
    std::vector<int64_t> tri_base;
    float *d_poses = nullptr;
    int pose_cap = 0;
    float4 *d_obs = nullptr;
    int64_t px_cap = 0;
    // background caches: entry 0 holds every object, entry k + 1 every object but k
    std::vector<BgCache> bgc;

    int *d_err = nullptr;
    // camera-hypothesis render: the scene's mesh views and triangle bases on the device
    MeshView *d_views = nullptr;
    int *d_tri_base = nullptr;
    int views_cap = 0;
    bool views_dirty = true;
    std::vector<MeshView> h_views;
    std::vector<int> h_tri_base;

    // coarse-to-fine and resampling scratch
    float *d_ll = nullptr;
    int64_t ll_cap = 0;
    float *d_refine = nullptr;  // [n][6 + 6 + 6 + 1]: Adam moments m, v, gradients, scores
    int64_t refine_cap = 0;
    float2 *d_part = nullptr;
    unsigned *d_counter = nullptr;
    unsigned long long *d_work = nullptr;  // ring of kWorkRing hypothesis counters of the persistent kernels
    unsigned work_slot = 0;
    float *d_logz = nullptr;
    int *d_idx = nullptr;
    float *d_logq_tmp = nullptr;
    int idx_cap = 0;
    float *d_centre = nullptr;  // [3][16]: two ping-pong centres and one expand scratch
    std::map<std::tuple<int, int, float>, float *> rot_cache;

    // launch shape of the score kernel
    int tile_w = 64;
    int cta_threads = 256;
    int ctas_per_sm = 0;
    int high_occupancy = 0;
    int score_code() const {
        const int nt = cta_threads == 128 ? 1 : (cta_threads == 64 ? 2 : (cta_threads == 32 ? 3 : 0));
        return ((nt + (high_occupancy ? 4 : 0)) << 8) | (ctas_per_sm & 255);
    }

    // batched form (this context as owner): descriptors, scores and resampling scratch
    int batch_chunk = 4;
    unsigned char *d_batch = nullptr;
    size_t batch_cap = 0;
    unsigned char *h_batch[2] = {nullptr, nullptr};
    size_t h_batch_cap[2] = {0, 0};
    cudaEvent_t batch_ev[2] = {nullptr, nullptr};
    int batch_flip = 0;
    float *d_bll = nullptr;
    int64_t bll_cap = 0;
    float2 *d_bpart = nullptr;
    int64_t bpart_cap = 0;
    unsigned *d_bcnt = nullptr;
    int64_t bcnt_cap = 0;
    unsigned long long *d_bwork = nullptr;
    int64_t bwork_cap = 0;
    int *d_bidx = nullptr;
    float *d_blogq = nullptr;
    int64_t bidx_cap = 0;
    float *d_blogz = nullptr;
    int64_t blogz_cap = 0;

    // instrumentation
    int instr = 0;
    unsigned long long *d_stats = nullptr;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[B3D_K_COUNT];
    std::vector<cudaEvent_t> event_pool;
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

b3d_status fail(b3d_ctx *ctx, b3d_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return st;
}

b3d_status cuda_fail(b3d_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, B3D_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

b3d_status check_launch(b3d_ctx *ctx, const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, what);
    return B3D_OK;
}

cudaEvent_t take_event(b3d_ctx *ctx) {
    if (!ctx->event_pool.empty()) {
        cudaEvent_t e = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets the launches made during its lifetime with events on stream s (when timing).
struct Timed {
    b3d_ctx *ctx;
    int cls;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    Timed(b3d_ctx *c, int k, cudaStream_t st) : ctx(c), cls(k), s(st) {
        if (ctx->instr & B3D_INSTR_TIMING) {
            a = take_event(ctx);
            cudaEventRecord(a, s);
        }
    }
    ~Timed() {
        if (a) {
            cudaEvent_t b = take_event(ctx);
            cudaEventRecord(b, s);
            ctx->pending[cls].push_back({a, b});
        }
    }
};

template <class T>
b3d_status dalloc(b3d_ctx *ctx, T **p, size_t count, const char *what) {
    *p = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    if (ctx->budget && ctx->used + bytes > ctx->budget)
        return fail(ctx, B3D_EBUDGET, std::string(what) + ": allocation of " + std::to_string(bytes) +
                                          " bytes exceeds the HBM budget (" + std::to_string(ctx->used) + " of " +
                                          std::to_string(ctx->budget) + " used)");
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, B3D_ENOMEM, std::string(what) + ": cudaMalloc failed: " + cudaGetErrorString(e));
    }
    ctx->allocs[q] = bytes;
    ctx->used += bytes;
    *p = static_cast<T *>(q);
    return B3D_OK;
}

template <class T>
void dfree(b3d_ctx *ctx, T *&p) {
    if (!p) return;
    auto it = ctx->allocs.find((void *)p);
    if (it != ctx->allocs.end()) {
        ctx->used -= it->second;
        ctx->allocs.erase(it);
    }
    cudaFree((void *)p);
    p = nullptr;
}

bool finite_all(const float *p, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// Build the device-side likelihood constants from the public parameters.
b3d_status make_lik(b3d_ctx *ctx, const b3d_lik_params *lp, Lik *L) {
    if (!lp) return fail(ctx, B3D_EINVAL, "lik is NULL");
    if (lp->kind != 0 && lp->kind != 1) return fail(ctx, B3D_EINVAL, "lik.kind must be 0 (ball) or 1 (Gaussian)");
    if (!(lp->radius > 0.f) || !std::isfinite(lp->radius)) return fail(ctx, B3D_EINVAL, "lik.radius must be > 0");
    if (!(lp->p_outlier > 0.f && lp->p_outlier < 1.f)) return fail(ctx, B3D_EINVAL, "lik.p_outlier must be in (0,1)");
    if (lp->half_window < 0 || lp->half_window > B3D_MAX_HALF_WINDOW)
        return fail(ctx, B3D_EINVAL, "lik.half_window must be in [0, " + std::to_string(B3D_MAX_HALF_WINDOW) + "]");
    if (lp->miss_mode != 0 && lp->miss_mode != 1) return fail(ctx, B3D_EINVAL, "lik.miss_mode must be 0 or 1");
    if (!std::isfinite(lp->volume) || !std::isfinite(lp->norm)) return fail(ctx, B3D_EINVAL, "lik.volume/norm not finite");
    const Cam &c = ctx->cam;
    const int w = lp->half_window;
    const double V = lp->volume > 0 ? (double)lp->volume
                                    : (double)c.W * c.H / ((double)c.fx * c.fy) *
                                          ((double)c.far_z * c.far_z * c.far_z - (double)c.near_z * c.near_z * c.near_z) / 3.0;
    const double K = lp->norm > 0 ? (double)lp->norm : (double)((2 * w + 1) * (2 * w + 1));
    const double r = lp->radius, p = lp->p_outlier, pi = 3.14159265358979323846;
    memset(L, 0, sizeof(Lik));
    L->kind = lp->kind;
    L->w = w;
    L->miss_mode = lp->miss_mode;
    L->n_lut = (2 * w + 1) * (2 * w + 1) + 1;
    L->r2 = (float)(r * r);
    L->inv2s2 = (float)(1.0 / (2.0 * r * r));
    L->a = (float)(p / V);
    const double gnorm = pow(2.0 * pi * r * r, -1.5);
    L->bg = (float)((1.0 - p) / K * gnorm);
    const double ball = 4.0 / 3.0 * pi * r * r * r;
    for (int n = 0; n < L->n_lut; ++n) L->lut[n] = (float)log(p / V + (1.0 - p) * n / (K * ball));
    L->s = (float)r;
    L->inv_s2 = (float)(1.0 / (r * r));
    L->b = (float)((1.0 - p) / K);
    L->inv_V = (float)(1.0 / V);
    L->inv_K = (float)(1.0 / K);
    L->gnorm = (float)gnorm;
    return B3D_OK;
}

LikKey key_of(const b3d_lik_params *lp) {
    return LikKey{lp->kind, lp->half_window, lp->miss_mode, lp->radius, lp->p_outlier, lp->volume, lp->norm};
}

MeshView view_of(const MeshRec &m) {
    MeshView v{};
    v.verts = m.verts;
    v.tris_surf = m.tris_surf;
    v.tris_full = m.tris_full;
    v.faces = m.faces;
    v.n_surf = m.n_surf;
    v.n_full = m.n_full;
    v.n_faces = (int)m.n_faces;
    v.closed = (m.flags & B3D_MESH_CLOSED) ? 1 : 0;
    for (int k = 0; k < 3; ++k) { v.lo[k] = m.lo[k]; v.hi[k] = m.hi[k]; v.nc[k] = m.nc[k]; }
    v.n_quads = m.n_quads;
    v.quads = m.quads;
    v.class_off = m.class_off;
    v.coords = m.coords;
    v.np1 = m.np1;
    return v;
}

b3d_status check_slot(b3d_ctx *ctx, int32_t slot) {
    if (!ctx->has_scene) return fail(ctx, B3D_EINVAL, "no scene: call b3d_set_scene first");
    if (slot < 0 || slot >= (int32_t)ctx->obj_mesh.size())
        return fail(ctx, B3D_ENOTFOUND, "object slot " + std::to_string(slot) + " is not in the scene");
    return B3D_OK;
}

BgCache &bg_cache(b3d_ctx *ctx, int32_t slot) {
    const size_t k = (size_t)(slot + 1);
    if (ctx->bgc.size() <= k) ctx->bgc.resize(k + 1);
    return ctx->bgc[k];
}

// Mark the background of every slot whose z-buffer holds object `obj` (-1: all slots), and
// the object's own z-buffer of the shared backgrounds.
void bg_invalidate(b3d_ctx *ctx, int32_t obj) {
    for (size_t k = 0; k < ctx->bgc.size(); ++k)
        if (obj < 0 || (int32_t)k != obj + 1) ctx->bgc[k].dirty = true;
    for (size_t o = 0; o < ctx->objz_ok.size(); ++o)
        if (obj < 0 || (int32_t)o == obj) ctx->objz_ok[o] = 0;
}

void bg_invalidate_lik(b3d_ctx *ctx) {
    for (BgCache &c : ctx->bgc) c.lik_valid = c.grad_valid = c.nvalid = false;
}

// Background z-buffer of every scene object except `slot` (slot = -1: all objects).
b3d_status ensure_bg(b3d_ctx *ctx, int32_t slot, cudaStream_t s) {
    BgCache &c = bg_cache(ctx, slot);
    const int64_t npx = (int64_t)ctx->cam.W * ctx->cam.H;
    b3d_status st;
    if (c.cap < npx) {
        dfree(ctx, c.bg); dfree(ctx, c.bgd); dfree(ctx, c.ell); dfree(ctx, c.gs); dfree(ctx, c.gp);
        dfree(ctx, c.qe); dfree(ctx, c.bgz);
        c.cap = c.gcap = 0;
        if ((st = dalloc(ctx, &c.bg, (size_t)npx, "background z-buffer")) != B3D_OK) return st;
        if ((st = dalloc(ctx, &c.bgd, (size_t)2 * npx, "background depth")) != B3D_OK) return st;
        if ((st = dalloc(ctx, &c.ell, (size_t)npx, "background likelihood")) != B3D_OK) return st;
        if ((st = dalloc(ctx, &c.qe, (size_t)npx, "packed observation and background terms")) != B3D_OK) return st;
        if ((st = dalloc(ctx, &c.bgz, (size_t)npx, "background depth bits")) != B3D_OK) return st;
        if (!c.sums && (st = dalloc(ctx, &c.sums, 3, "background sums")) != B3D_OK) return st;
        dfree(ctx, c.part);
        if ((st = dalloc(ctx, &c.part, (size_t)3 * bg_table_blocks(npx), "background partial sums")) != B3D_OK) return st;
        if (!c.counter) {
            if ((st = dalloc(ctx, &c.counter, 1, "background sum ticket")) != B3D_OK) return st;
            cudaMemsetAsync(c.counter, 0, sizeof(unsigned), s);
        }
        c.cap = npx;
        c.dirty = true;
    }
    if (!c.dirty) return B3D_OK;
    Timed tm(ctx, B3D_K_SCENE, s);
    launch_bg_clear(c.bg, npx, s);
    ++ctx->launches;
    for (size_t o = 0; o < ctx->obj_mesh.size(); ++o) {
        if ((int32_t)o == slot) continue;
        const MeshRec &m = ctx->meshes[ctx->obj_mesh[o]];
        if (m.n_full <= 0) continue;
        launch_bg_raster(ctx->cam, view_of(m), ctx->d_poses + 16 * o, (int)ctx->tri_base[o], c.bg, s);
        ++ctx->launches;
    }
    c.dirty = false;
    c.lik_valid = c.grad_valid = c.nvalid = c.bgd_valid = false;
    return check_launch(ctx, "background render");
}

// The background's depth under both miss modes (after ensure_bg), for the materialised form.
b3d_status ensure_bg_depth(b3d_ctx *ctx, int32_t slot, cudaStream_t s) {
    BgCache &c = bg_cache(ctx, slot);
    if (c.bgd_valid) return B3D_OK;
    Timed tm(ctx, B3D_K_SCENE, s);
    launch_bg_depth((int64_t)ctx->cam.W * ctx->cam.H, ctx->cam.far_z, c.bg, c.bgd, s);
    ++ctx->launches;
    c.bgd_valid = true;
    return check_launch(ctx, "background depth");
}

SceneView scene_view(b3d_ctx *ctx, int32_t slot) {
    SceneView sv{};
    sv.cam = ctx->cam;
    sv.obs = ctx->d_obs;
    if ((size_t)(slot + 1) < ctx->bgc.size()) {
        const BgCache &c = ctx->bgc[(size_t)(slot + 1)];
        sv.bg = c.bg;
        sv.bgd = c.bgd;
        sv.ell_bg = c.ell;
        sv.qe = c.lik_valid ? c.qe : nullptr;
        sv.bgz = c.lik_valid ? c.bgz : nullptr;
        sv.ll_bg = c.sums;
        sv.gs_bg = c.gs;
        sv.gp_bg = c.gp;
        sv.sums_bg = c.sums;
    }
    if (slot >= 0) {
        sv.mesh = view_of(ctx->meshes[ctx->obj_mesh[slot]]);
        sv.tri_base = (int)ctx->tri_base[slot];
    }
    sv.err = ctx->d_err;
    sv.stats = (ctx->instr & B3D_INSTR_WORK) ? ctx->d_stats : nullptr;
    sv.tile_w = ctx->tile_w;
    return sv;
}

// A hypothesis counter for one persistent launch (its launcher zeroes it): a ring, so launches
// of this context on different streams use different counters unless kWorkRing are in flight.
unsigned long long *take_work(b3d_ctx *ctx) { return ctx->d_work + (ctx->work_slot++ % kWorkRing); }

// Per-pixel terms of the background of `slot` (after ensure_bg) for these likelihood
// parameters; with grad, also the sigma / p_out derivative tables.
b3d_status ensure_bg_lik(b3d_ctx *ctx, int32_t slot, const b3d_lik_params *lp, const Lik &L, bool grad,
                         cudaStream_t s) {
    BgCache &c = bg_cache(ctx, slot);
    const LikKey k = key_of(lp);
    const int64_t npx = (int64_t)ctx->cam.W * ctx->cam.H;
    b3d_status st;
    if (grad && c.gcap < npx) {
        dfree(ctx, c.gs); dfree(ctx, c.gp);
        c.gcap = 0;
        if ((st = dalloc(ctx, &c.gs, (size_t)npx, "background sigma gradient")) != B3D_OK) return st;
        if ((st = dalloc(ctx, &c.gp, (size_t)npx, "background p_out gradient")) != B3D_OK) return st;
        c.gcap = npx;
        c.grad_valid = false;
    }
    if (c.lik_valid && c.key == k && (!grad || c.grad_valid)) return B3D_OK;
    SceneView sv = scene_view(ctx, slot);
    Timed tm(ctx, B3D_K_SCENE, s);
    launch_bg_tables(sv, L, c.ell, grad ? c.gs : nullptr, grad ? c.gp : nullptr, c.qe, c.bgz, c.part, c.counter,
                     c.sums, s);
    ++ctx->launches;
    c.key = k;
    c.lik_valid = true;
    c.grad_valid = grad;
    return check_launch(ctx, "background likelihood tables");
}

// Device constants of a noise grid (the same formulas as make_lik, per setting).
b3d_status make_noise(b3d_ctx *ctx, const b3d_noise_grid *gr, NoiseLik *N) {
    if (!gr) return fail(ctx, B3D_EINVAL, "noise grid is NULL");
    if (gr->kind != 0 && gr->kind != 1) return fail(ctx, B3D_EINVAL, "grid.kind must be 0 or 1");
    if (gr->half_window < 0 || gr->half_window > 2) return fail(ctx, B3D_EINVAL, "grid.half_window must be in [0, 2]");
    if (gr->n_radius < 1 || gr->n_radius > B3D_MAX_NOISE_R || gr->n_pout < 1 || gr->n_pout > B3D_MAX_NOISE_P)
        return fail(ctx, B3D_EINVAL, "grid.n_radius and grid.n_pout must be in [1, 4]");
    if (gr->miss_mode != 0 && gr->miss_mode != 1) return fail(ctx, B3D_EINVAL, "grid.miss_mode must be 0 or 1");
    if (!std::isfinite(gr->volume) || !std::isfinite(gr->norm)) return fail(ctx, B3D_EINVAL, "grid.volume/norm not finite");
    for (int i = 0; i < gr->n_radius; ++i)
        if (!(gr->radius[i] > 0.f) || !std::isfinite(gr->radius[i])) return fail(ctx, B3D_EINVAL, "grid radii must be > 0");
    for (int j = 0; j < gr->n_pout; ++j)
        if (!(gr->p_outlier[j] > 0.f && gr->p_outlier[j] < 1.f)) return fail(ctx, B3D_EINVAL, "grid p_outlier must be in (0,1)");
    if (!finite_all(gr->log_weight, (int64_t)gr->n_radius * gr->n_pout)) return fail(ctx, B3D_EINVAL, "grid log weights not finite");
    const Cam &c = ctx->cam;
    const int w = gr->half_window;
    const double V = gr->volume > 0 ? (double)gr->volume
                                    : (double)c.W * c.H / ((double)c.fx * c.fy) *
                                          ((double)c.far_z * c.far_z * c.far_z - (double)c.near_z * c.near_z * c.near_z) / 3.0;
    const double K = gr->norm > 0 ? (double)gr->norm : (double)((2 * w + 1) * (2 * w + 1));
    const double pi = 3.14159265358979323846;
    const int n_lut = (2 * w + 1) * (2 * w + 1) + 1;
    memset(N, 0, sizeof(NoiseLik));
    N->kind = gr->kind;
    N->w = w;
    N->miss_mode = gr->miss_mode;
    N->nr = gr->n_radius;
    N->np = gr->n_pout;
    for (int j = 0; j < gr->n_pout; ++j) N->a[j] = (float)(gr->p_outlier[j] / V);
    for (int i = 0; i < gr->n_radius; ++i) {
        const double r = gr->radius[i];
        N->r2[i] = (float)(r * r);
        N->inv2s2[i] = (float)(1.0 / (2.0 * r * r));
        const double gnorm = pow(2.0 * pi * r * r, -1.5), ball = 4.0 / 3.0 * pi * r * r * r;
        for (int j = 0; j < gr->n_pout; ++j) {
            const double p = gr->p_outlier[j];
            const int g = i * kMaxNoiseP + j;
            N->bg[g] = (float)((1.0 - p) / K * gnorm);
            N->logw[g] = gr->log_weight[i * gr->n_pout + j];
            for (int n = 0; n < n_lut; ++n) N->lut[g * kNoiseLut + n] = (float)log(p / V + (1.0 - p) * n / (K * ball));
        }
    }
    return B3D_OK;
}

// Per-setting background tables of `slot` (after ensure_bg) for this noise grid.
b3d_status ensure_bg_noise(b3d_ctx *ctx, int32_t slot, const b3d_noise_grid *gr, const NoiseLik &N, cudaStream_t s) {
    BgCache &c = bg_cache(ctx, slot);
    const int64_t npx = (int64_t)ctx->cam.W * ctx->cam.H;
    b3d_status st;
    if (c.ncap < npx) {
        dfree(ctx, c.nell); dfree(ctx, c.npart);
        c.ncap = 0;
        if ((st = dalloc(ctx, &c.nell, (size_t)kMaxNoise * npx, "noise-grid background tables")) != B3D_OK) return st;
        if ((st = dalloc(ctx, &c.npart, (size_t)kMaxNoise * bg_table_blocks(npx), "noise-grid partial sums")) != B3D_OK)
            return st;
        if (!c.nsums && (st = dalloc(ctx, &c.nsums, kMaxNoise, "noise-grid background sums")) != B3D_OK) return st;
        if (!c.ncounter) {
            if ((st = dalloc(ctx, &c.ncounter, 1, "noise-grid sum ticket")) != B3D_OK) return st;
            cudaMemsetAsync(c.ncounter, 0, sizeof(unsigned), s);
        }
        c.ncap = npx;
        c.nvalid = false;
    }
    if (c.nvalid && memcmp(&c.nkey, gr, sizeof(b3d_noise_grid)) == 0) return B3D_OK;
    Timed tm(ctx, B3D_K_SCENE, s);
    launch_bg_noise_tables(scene_view(ctx, slot), N, c.nell, c.npart, c.ncounter, c.nsums, s);
    ++ctx->launches;
    c.nkey = *gr;
    c.nvalid = true;
    return check_launch(ctx, "noise-grid background tables");
}

b3d_status ensure_scratch(b3d_ctx *ctx, int64_t n_ll, int m) {
    b3d_status st;
    if (n_ll > ctx->ll_cap) {
        dfree(ctx, ctx->d_ll);
        if ((st = dalloc(ctx, &ctx->d_ll, (size_t)n_ll, "score buffer")) != B3D_OK) { ctx->ll_cap = 0; return st; }
        ctx->ll_cap = n_ll;
    }
    if (!ctx->d_part) {
        if ((st = dalloc(ctx, &ctx->d_part, 1024, "resampling partials")) != B3D_OK) return st;
        if ((st = dalloc(ctx, &ctx->d_counter, 1, "resampling counter")) != B3D_OK) return st;
        cudaMemset(ctx->d_counter, 0, sizeof(unsigned));
        if ((st = dalloc(ctx, &ctx->d_logz, B3D_MAX_STAGES, "log normalisers")) != B3D_OK) return st;
        if ((st = dalloc(ctx, &ctx->d_centre, 3 * 16, "grid centres")) != B3D_OK) return st;
    }
    if (m > ctx->idx_cap) {
        dfree(ctx, ctx->d_idx);
        dfree(ctx, ctx->d_logq_tmp);
        if ((st = dalloc(ctx, &ctx->d_idx, (size_t)m, "draw indices")) != B3D_OK) { ctx->idx_cap = 0; return st; }
        if ((st = dalloc(ctx, &ctx->d_logq_tmp, (size_t)m, "draw log-probabilities")) != B3D_OK) { ctx->idx_cap = 0; return st; }
        ctx->idx_cap = m;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "scratch set-up");
    return B3D_OK;
}

b3d_status rotation_table(b3d_ctx *ctx, const b3d_stage &st, float **out, cudaStream_t s) {
    const float rm = st.rot_kind == 0 ? 0.f : st.rot_max;
    auto key = std::make_tuple(st.rot_kind, st.n_rot, rm);
    auto it = ctx->rot_cache.find(key);
    if (it != ctx->rot_cache.end()) { *out = it->second; return B3D_OK; }
    float *p = nullptr;
    b3d_status r = dalloc(ctx, &p, (size_t)9 * st.n_rot, "rotation set");
    if (r != B3D_OK) return r;
    {
        Timed tm(ctx, B3D_K_SCENE, s);
        launch_rotation_set(st.rot_kind, st.n_rot, (double)rm, p, s);
    }
    ++ctx->launches;
    ctx->rot_cache[key] = p;
    *out = p;
    return check_launch(ctx, "rotation set");
}

b3d_status check_stage(b3d_ctx *ctx, const b3d_stage &st, int64_t *n_out) {
    if (st.n_per_axis < 1 || st.n_per_axis > 1024) return fail(ctx, B3D_EINVAL, "stage.n_per_axis must be in [1, 1024]");
    if (st.n_rot < 1) return fail(ctx, B3D_EINVAL, "stage.n_rot must be >= 1");
    if (st.rot_kind != 0 && st.rot_kind != 1) return fail(ctx, B3D_EINVAL, "stage.rot_kind must be 0 or 1");
    if (!(st.step > 0.f) || !std::isfinite(st.step)) return fail(ctx, B3D_EINVAL, "stage.step must be > 0");
    if (!std::isfinite(st.rot_max)) return fail(ctx, B3D_EINVAL, "stage.rot_max must be finite");
    const int64_t n = (int64_t)st.n_per_axis * st.n_per_axis * st.n_per_axis * st.n_rot;
    if (n > INT32_MAX) return fail(ctx, B3D_EINVAL, "stage has more than 2^31-1 hypotheses");
    *n_out = n;
    return B3D_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }


template <class T>
b3d_status grow(b3d_ctx *ctx, T *&p, int64_t &cap, int64_t need, const char *what, bool zero = false) {
    if (need <= cap && p) return B3D_OK;
    dfree(ctx, p);
    cap = 0;
    b3d_status st = dalloc(ctx, &p, (size_t)std::max<int64_t>(need, 1), what);
    if (st != B3D_OK) return st;
    if (zero) {
        cudaError_t e = cudaMemset(p, 0, sizeof(T) * (size_t)std::max<int64_t>(need, 1));
        if (e != cudaSuccess) return cuda_fail(ctx, e, what);
    }
    cap = need;
    return B3D_OK;
}

bool stream_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Pinned staging buffer for one batched call's descriptors (double-buffered: a buffer is
// rewritten only after the copy that last read it has run).
b3d_status batch_staging(b3d_ctx *ctx, size_t bytes, cudaStream_t s, unsigned char **host, int *slot) {
    const int b = ctx->batch_flip;
    if (ctx->batch_ev[b] && !stream_capturing(s)) cudaEventSynchronize(ctx->batch_ev[b]);
    if (ctx->h_batch_cap[b] < bytes) {
        // both buffers grow together, so a later call (possibly under graph capture) finds its
        // buffer allocated
        if (stream_capturing(s)) return fail(ctx, B3D_EINVAL, "batched call must run once with these sizes before capture");
        for (int k = 0; k < 2; ++k) {
            if (ctx->batch_ev[k]) cudaEventSynchronize(ctx->batch_ev[k]);
            if (ctx->h_batch[k]) cudaFreeHost(ctx->h_batch[k]);
            ctx->h_batch[k] = nullptr;
            ctx->h_batch_cap[k] = 0;
            cudaError_t e = cudaMallocHost((void **)&ctx->h_batch[k], bytes);
            if (e != cudaSuccess) { cudaGetLastError(); return fail(ctx, B3D_ENOMEM, "pinned staging allocation failed"); }
            ctx->h_batch_cap[k] = bytes;
        }
    }
    if (ctx->batch_cap < bytes) {
        dfree(ctx, ctx->d_batch);
        ctx->batch_cap = 0;
        b3d_status st = dalloc(ctx, &ctx->d_batch, bytes, "batch descriptors");
        if (st != B3D_OK) return st;
        ctx->batch_cap = bytes;
    }
    *host = ctx->h_batch[b];
    *slot = b;
    return B3D_OK;
}

b3d_status batch_upload(b3d_ctx *ctx, int slot, size_t bytes, cudaStream_t s) {
    cudaError_t e = cudaMemcpyAsync(ctx->d_batch, ctx->h_batch[slot], bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch descriptor upload");
    if (!stream_capturing(s)) {
        if (!ctx->batch_ev[slot]) cudaEventCreateWithFlags(&ctx->batch_ev[slot], cudaEventDisableTiming);
        cudaEventRecord(ctx->batch_ev[slot], s);
    }
    ctx->batch_flip ^= 1;
    return B3D_OK;
}

// Staging layout of b3d_enumerate_multi: centres | BatchItem[T][n] | LseItem[T][n] |
// SelectItem[T][n] | item_begin[T][n+1] | block_begin[T][n+1] | device-centre pairs[n].
struct MultiLayout {
    size_t o_cent, o_bi, o_li, o_si, o_ib, o_bb, o_gp, bytes;
};

MultiLayout multi_layout(int64_t n_items, int T) {
    MultiLayout l;
    l.o_cent = 0;
    l.o_bi = l.o_cent + align16(sizeof(float) * 32 * n_items);
    l.o_li = l.o_bi + align16(sizeof(BatchItem) * (size_t)T * n_items);
    l.o_si = l.o_li + align16(sizeof(LseItem) * (size_t)T * n_items);
    l.o_ib = l.o_si + align16(sizeof(SelectItem) * (size_t)T * n_items);
    l.o_bb = l.o_ib + align16(sizeof(int64_t) * (size_t)T * (n_items + 1));
    l.o_gp = l.o_bb + align16(sizeof(int) * (size_t)T * (n_items + 1));
    l.bytes = l.o_gp + align16(sizeof(float *) * 2 * (size_t)n_items);
    return l;
}

// Scores of one stage, resampling partials and counters, draws and normalisers of a
// batched enumeration (grown to the need, never shrunk).
b3d_status multi_scratch(b3d_ctx *owner, int64_t need_ll, int64_t need_part, int64_t n_items, int64_t sum_m, int T) {
    b3d_status st;
    if ((st = grow(owner, owner->d_bll, owner->bll_cap, need_ll, "batched scores")) != B3D_OK) return st;
    if ((st = grow(owner, owner->d_bpart, owner->bpart_cap, need_part, "batched partials")) != B3D_OK) return st;
    if ((st = grow(owner, owner->d_bcnt, owner->bcnt_cap, n_items, "batched counters", true)) != B3D_OK) return st;
    if ((st = grow(owner, owner->d_bwork, owner->bwork_cap, 8, "work counters")) != B3D_OK) return st;
    if (owner->bidx_cap < sum_m) {
        dfree(owner, owner->d_blogq);
        int64_t c2 = 0;
        if ((st = grow(owner, owner->d_bidx, owner->bidx_cap, sum_m, "batched draws")) != B3D_OK) return st;
        if ((st = grow(owner, owner->d_blogq, c2, sum_m, "batched draw log-probabilities")) != B3D_OK) return st;
    }
    return grow(owner, owner->d_blogz, owner->blogz_cap, n_items * T, "batched normalisers");
}

}  // namespace

// ==========================================================================================
// C ABI
// ==========================================================================================
extern "C" {

b3d_status b3d_create(b3d_ctx **out, int32_t device, uint64_t hbm_budget_bytes) {
    if (!out) { g_create_error = "out is NULL"; return B3D_EINVAL; }
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        g_create_error = "no CUDA device " + std::to_string(device) + " (" + std::to_string(n) + " visible" +
                         (e != cudaSuccess ? std::string(", ") + cudaGetErrorString(e) : std::string()) + ")";
        return B3D_EINVAL;
    }
    b3d_ctx *ctx = new (std::nothrow) b3d_ctx();
    if (!ctx) { g_create_error = "host allocation failed"; return B3D_ENOMEM; }
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    DeviceGuard g(device);
    b3d_status st = dalloc(ctx, &ctx->d_err, 1, "error flag");
    if (st == B3D_OK) st = dalloc(ctx, &ctx->d_work, kWorkRing, "work counters");
    if (st != B3D_OK) {
        g_create_error = ctx->err;
        if (ctx->d_err) cudaFree(ctx->d_err);
        delete ctx;
        return st;
    }
    cudaMemset(ctx->d_err, 0, sizeof(int));
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        g_create_error = std::string("device set-up: ") + cudaGetErrorString(e);
        cudaFree(ctx->d_err);
        delete ctx;
        return B3D_ECUDA;
    }
    g_create_error.clear();
    *out = ctx;
    return B3D_OK;
}

b3d_status b3d_destroy(b3d_ctx *ctx) {
    if (!ctx) return B3D_EINVAL;
    {
        DeviceGuard g(ctx->device);
        cudaDeviceSynchronize();
        for (auto &kv : ctx->allocs) cudaFree(kv.first);
        for (auto &v : ctx->pending)
            for (auto &ab : v) { cudaEventDestroy(ab.first); cudaEventDestroy(ab.second); }
        for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
        for (int k = 0; k < 2; ++k) {
            if (ctx->h_batch[k]) cudaFreeHost(ctx->h_batch[k]);
            if (ctx->batch_ev[k]) cudaEventDestroy(ctx->batch_ev[k]);
        }
    }
    delete ctx;
    return B3D_OK;
}

const char *b3d_last_error(b3d_ctx *ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

int64_t b3d_launch_count(b3d_ctx *ctx) { return ctx ? ctx->launches : 0; }

b3d_status b3d_load_mesh(b3d_ctx *ctx, const float *verts, int64_t n_v, const int32_t *faces, int64_t n_f, int32_t flags,
                         int32_t *mesh_id) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    if (!verts || !faces || !mesh_id) return fail(ctx, B3D_EINVAL, "verts, faces and mesh_id must be non-NULL");
    if (n_v < 1 || n_f < 1) return fail(ctx, B3D_EINVAL, "a mesh needs n_v >= 1 and n_f >= 1");
    if (n_f > (int64_t)1 << 30) return fail(ctx, B3D_EINVAL, "too many faces");
    if (flags & ~B3D_MESH_CLOSED) return fail(ctx, B3D_EINVAL, "unknown mesh flags");
    if (!finite_all(verts, 3 * n_v)) return fail(ctx, B3D_EINVAL, "vertex coordinates must be finite");
    for (int64_t i = 0; i < 3 * n_f; ++i)
        if (faces[i] < 0 || faces[i] >= n_v) return fail(ctx, B3D_EINVAL, "face " + std::to_string(i / 3) + " indexes a missing vertex");

    // 1. weld vertices with bitwise-equal coordinates (-0 == +0)
    struct K3 {
        uint32_t a, b, c;
        bool operator==(const K3 &o) const { return a == o.a && b == o.b && c == o.c; }
    };
    struct H3 {
        size_t operator()(const K3 &k) const {
            uint64_t h = k.a * 0x9E3779B97F4A7C15ULL;
            h ^= (uint64_t)k.b * 0xC2B2AE3D27D4EB4FULL + (h << 6) + (h >> 2);
            h ^= (uint64_t)k.c * 0x165667B19E3779F9ULL + (h << 6) + (h >> 2);
            return (size_t)h;
        }
    };
    auto bits = [](float x) {
        if (x == 0.f) x = 0.f;
        uint32_t u;
        memcpy(&u, &x, 4);
        return u;
    };
    std::unordered_map<K3, int32_t, H3> weld;
    weld.reserve((size_t)n_v * 2);
    std::vector<int32_t> remap((size_t)n_v);
    std::vector<float> wv;
    for (int64_t i = 0; i < n_v; ++i) {
        K3 k{bits(verts[3 * i]), bits(verts[3 * i + 1]), bits(verts[3 * i + 2])};
        auto it = weld.find(k);
        if (it == weld.end()) {
            const int32_t id = (int32_t)(wv.size() / 3);
            weld.emplace(k, id);
            wv.push_back(verts[3 * i]); wv.push_back(verts[3 * i + 1]); wv.push_back(verts[3 * i + 2]);
            remap[i] = id;
        } else {
            remap[i] = it->second;
        }
    }
    // 2. triangles on welded vertices; drop degenerate ones (they cover nothing)
    struct Tri { int32_t a, b, c, f; };
    std::vector<Tri> tris;
    tris.reserve((size_t)n_f);
    for (int64_t f = 0; f < n_f; ++f) {
        Tri t{remap[faces[3 * f]], remap[faces[3 * f + 1]], remap[faces[3 * f + 2]], (int32_t)f};
        if (t.a == t.b || t.b == t.c || t.a == t.c) continue;
        tris.push_back(t);
    }
    const std::vector<Tri> full = tris;
    // 3. closed meshes: coincident triangles of opposite orientation are internal faces
    if (flags & B3D_MESH_CLOSED) {
        struct KT {
            int32_t a, b, c;
            bool operator==(const KT &o) const { return a == o.a && b == o.b && c == o.c; }
        };
        struct HT {
            size_t operator()(const KT &k) const {
                return (size_t)((uint64_t)k.a * 0x9E3779B97F4A7C15ULL ^ (uint64_t)k.b * 0xC2B2AE3D27D4EB4FULL ^
                                (uint64_t)k.c * 0x165667B19E3779F9ULL);
            }
        };
        std::unordered_map<KT, std::vector<int32_t>, HT> groups;
        groups.reserve(tris.size() * 2);
        auto parity = [](const Tri &t) {  // +1 if (a,b,c) is an even permutation of its sorted order
            int v[3] = {t.a, t.b, t.c}, inv = 0;
            for (int i = 0; i < 3; ++i)
                for (int j = i + 1; j < 3; ++j) inv += v[i] > v[j];
            return (inv & 1) ? -1 : 1;
        };
        for (size_t i = 0; i < tris.size(); ++i) {
            int v[3] = {tris[i].a, tris[i].b, tris[i].c};
            std::sort(v, v + 3);
            groups[KT{v[0], v[1], v[2]}].push_back((int32_t)i);
        }
        std::vector<char> drop(tris.size(), 0);
        for (auto &kv : groups) {
            auto &g = kv.second;
            if (g.size() < 2) continue;
            std::vector<int32_t> pos, neg;
            for (int32_t i : g) (parity(tris[i]) > 0 ? pos : neg).push_back(i);
            const size_t k = std::min(pos.size(), neg.size());
            for (size_t j = 0; j < k; ++j) { drop[pos[j]] = 1; drop[neg[j]] = 1; }
        }
        std::vector<Tri> kept;
        kept.reserve(tris.size());
        for (size_t i = 0; i < tris.size(); ++i)
            if (!drop[i]) kept.push_back(tris[i]);
        tris.swap(kept);
    }
    // 4. spatial order (Morton code of the centroid): neighbouring threads get nearby
    //    triangles
    MeshRec rec;
    rec.n_faces = n_f;
    rec.flags = flags;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (const Tri &t : full)
        for (int32_t v : {t.a, t.b, t.c})
            for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], wv[3 * v + k]); hi[k] = std::max(hi[k], wv[3 * v + k]); }
    if (full.empty())
        for (int k = 0; k < 3; ++k) { lo[k] = 0; hi[k] = 0; }
    for (int k = 0; k < 3; ++k) { rec.lo[k] = lo[k]; rec.hi[k] = hi[k]; }
    auto spread = [](uint32_t x) {  // 10 bits -> every third bit
        x &= 0x3ff;
        x = (x | (x << 16)) & 0x30000ff;
        x = (x | (x << 8)) & 0x300f00f;
        x = (x | (x << 4)) & 0x30c30c3;
        x = (x | (x << 2)) & 0x9249249;
        return x;
    };
    auto morton = [&](const Tri &t) {
        uint32_t q[3];
        for (int k = 0; k < 3; ++k) {
            const float cen = (wv[3 * t.a + k] + wv[3 * t.b + k] + wv[3 * t.c + k]) / 3.f;
            const float ext = hi[k] - lo[k];
            q[k] = ext > 0 ? (uint32_t)std::min(1023.f, std::max(0.f, (cen - lo[k]) / ext * 1023.f)) : 0u;
        }
        return spread(q[0]) | (spread(q[1]) << 1) | (spread(q[2]) << 2);
    };
    auto sorted_int4 = [&](const std::vector<Tri> &v) {
        std::vector<std::pair<uint32_t, int32_t>> order(v.size());
        for (size_t i = 0; i < v.size(); ++i) order[i] = {morton(v[i]), (int32_t)i};
        std::sort(order.begin(), order.end());
        std::vector<int4> out;
        out.reserve(v.size());
        for (auto &o : order) out.push_back(make_int4(v[o.second].a, v[o.second].b, v[o.second].c, v[o.second].f));
        return out;
    };
    std::vector<int4> h_full = sorted_int4(full), h_surf = sorted_int4(tris);
    std::vector<float4> h_verts(wv.size() / 3);
    for (size_t i = 0; i < h_verts.size(); ++i) h_verts[i] = make_float4(wv[3 * i], wv[3 * i + 1], wv[3 * i + 2], 0.f);
    std::vector<int4> h_faces((size_t)n_f);
    for (int64_t f = 0; f < n_f; ++f)
        h_faces[f] = make_int4(remap[faces[3 * f]], remap[faces[3 * f + 1]], remap[faces[3 * f + 2]], 0);

    // 5. voxel rectangles: a closed mesh whose surface triangles pair up into unit squares of
    //    the vertex lattice (distinct coordinates per axis), each square axis-aligned; the
    //    squares of each plane are merged into rectangles of at most 4 x 4 squares
    std::vector<uint2> h_quads;
    std::vector<int> h_off;
    std::vector<float> h_coords;
    int nc[3] = {0, 0, 0}, np1 = 0;
    bool quads_ok = (flags & B3D_MESH_CLOSED) && !tris.empty();
    std::vector<float> axis_vals[3];
    std::vector<std::unordered_map<uint32_t, int>> axis_idx(3);
    if (quads_ok) {
        for (int a = 0; a < 3; ++a) {
            std::vector<float> &vals = axis_vals[a];
            for (const Tri &t : tris)
                for (int32_t v : {t.a, t.b, t.c}) vals.push_back(wv[3 * v + a]);
            std::sort(vals.begin(), vals.end());
            vals.erase(std::unique(vals.begin(), vals.end()), vals.end());
            if ((int)vals.size() > kMaxPlanes) quads_ok = false;
            for (size_t i = 0; i < vals.size(); ++i) axis_idx[a][bits(vals[i])] = (int)i;
            nc[a] = (int)vals.size();
        }
    }
    if (quads_ok) {
        struct QKey {
            uint32_t k;
            bool operator==(const QKey &o) const { return k == o.k; }
        };
        std::unordered_map<uint32_t, std::vector<std::pair<int, int>>> groups;  // key -> (tri, missing corner)
        for (size_t i = 0; i < tris.size() && quads_ok; ++i) {
            const Tri &t = tris[i];
            const int32_t vv[3] = {t.a, t.b, t.c};
            int axis = -1;
            for (int a = 0; a < 3 && axis < 0; ++a)
                if (bits(wv[3 * vv[0] + a]) == bits(wv[3 * vv[1] + a]) && bits(wv[3 * vv[0] + a]) == bits(wv[3 * vv[2] + a]))
                    axis = a;
            if (axis < 0) { quads_ok = false; break; }
            const int ab = (axis + 1) % 3, ac = (axis + 2) % 3;
            int ib[3], ic[3];
            for (int k = 0; k < 3; ++k) {
                ib[k] = axis_idx[ab][bits(wv[3 * vv[k] + ab])];
                ic[k] = axis_idx[ac][bits(wv[3 * vv[k] + ac])];
            }
            const int b0 = std::min({ib[0], ib[1], ib[2]}), b1 = std::max({ib[0], ib[1], ib[2]});
            const int c0 = std::min({ic[0], ic[1], ic[2]}), c1 = std::max({ic[0], ic[1], ic[2]});
            if (b1 != b0 + 1 || c1 != c0 + 1) { quads_ok = false; break; }
            // corners k0 (b0,c0) k1 (b1,c0) k2 (b1,c1) k3 (b0,c1); which one is missing
            bool has[4] = {false, false, false, false};
            for (int k = 0; k < 3; ++k) has[(ib[k] == b0 ? (ic[k] == c0 ? 0 : 3) : (ic[k] == c0 ? 1 : 2))] = true;
            int missing = -1, present = 0;
            for (int k = 0; k < 4; ++k) { if (!has[k]) missing = k; else ++present; }
            if (present != 3) { quads_ok = false; break; }
            // outward normal sign along the plane axis
            double e1[3], e2[3];
            for (int k = 0; k < 3; ++k) {
                e1[k] = (double)wv[3 * vv[1] + k] - wv[3 * vv[0] + k];
                e2[k] = (double)wv[3 * vv[2] + k] - wv[3 * vv[0] + k];
            }
            const double nrm = e1[ab] * e2[ac] - e1[ac] * e2[ab];
            const int cls = 2 * axis + (nrm > 0 ? 1 : 0);
            const int p = axis_idx[axis][bits(wv[3 * vv[0] + axis])];
            const uint32_t key = ((uint32_t)cls << 27) | ((uint32_t)p << 18) | ((uint32_t)b0 << 9) | (uint32_t)c0;
            groups[key].push_back({(int)i, missing});
        }
        if (quads_ok) {
            // every unit square must be exactly two triangles split along a diagonal
            std::map<std::pair<int, int>, std::vector<std::pair<int, int>>> planes;  // (class, plane) -> squares
            for (auto &kv : groups) {
                auto &g = kv.second;
                if (g.size() != 2 || (g[0].second + 2) % 4 != g[1].second) { quads_ok = false; break; }
                const int cls = (int)(kv.first >> 27), p = (int)((kv.first >> 18) & 511);
                planes[{cls, p}].push_back({(int)((kv.first >> 9) & 511), (int)(kv.first & 511)});
            }
            if (quads_ok) {
                // greedy merge of each plane's squares into rectangles (same plane and outward
                // side, so the union renders exactly as the squares do) of at most
                // kMaxRectExtent squares a side: a long strip seen at an angle has a screen box
                // many times its area, and the rasteriser tests every pixel of the box
                constexpr int kMaxRectExtent = 4;
                std::vector<uint2> rects;
                for (auto &pl : planes) {
                    const int cls = pl.first.first, p = pl.first.second;
                    int bmin = INT32_MAX, bmax = -1, cmin = INT32_MAX, cmax = -1;
                    for (auto &sq : pl.second) {
                        bmin = std::min(bmin, sq.first); bmax = std::max(bmax, sq.first);
                        cmin = std::min(cmin, sq.second); cmax = std::max(cmax, sq.second);
                    }
                    const int nb = bmax - bmin + 1, ncs = cmax - cmin + 1;
                    std::vector<char> occ((size_t)nb * ncs, 0);
                    for (auto &sq : pl.second) occ[(size_t)(sq.first - bmin) * ncs + (sq.second - cmin)] = 1;
                    for (int b = 0; b < nb; ++b)
                        for (int c = 0; c < ncs; ++c) {
                            if (!occ[(size_t)b * ncs + c]) continue;
                            int wc = 1;
                            while (c + wc < ncs && wc < kMaxRectExtent && occ[(size_t)b * ncs + c + wc]) ++wc;
                            int hb = 1;
                            for (;;) {
                                if (b + hb >= nb || hb >= kMaxRectExtent) break;
                                bool row = true;
                                for (int k = 0; k < wc && row; ++k) row = occ[(size_t)(b + hb) * ncs + c + k] != 0;
                                if (!row) break;
                                ++hb;
                            }
                            for (int bb = 0; bb < hb; ++bb)
                                for (int k = 0; k < wc; ++k) occ[(size_t)(b + bb) * ncs + c + k] = 0;
                            const uint32_t b0 = (uint32_t)(b + bmin), c0 = (uint32_t)(c + cmin);
                            rects.push_back(make_uint2(((uint32_t)cls << 29) | ((uint32_t)p << 18) | (b0 << 9) | c0,
                                                       ((uint32_t)hb << 9) | (uint32_t)wc));
                        }
                }
                // rectangles are already grouped by (class, plane) in ascending order
                np1 = std::max({nc[0], nc[1], nc[2]}) + 1;
                h_off.assign((size_t)6 * np1, 0);
                for (int cls = 0; cls < 6; ++cls) {
                    const int a = cls >> 1;
                    for (int p = 0; p < np1; ++p) {
                        const int pp = std::min(p, nc[a]);
                        // first rectangle with class > cls, or class == cls and plane >= pp
                        auto it = std::lower_bound(rects.begin(), rects.end(), 0, [&](const uint2 &q, int) {
                            const int qc = (int)(q.x >> 29), qp = (int)((q.x >> 18) & 511);
                            return qc < cls || (qc == cls && qp < pp);
                        });
                        h_off[(size_t)cls * np1 + p] = (int)(it - rects.begin());
                    }
                }
                h_quads = std::move(rects);
                for (int a = 0; a < 3; ++a) h_coords.insert(h_coords.end(), axis_vals[a].begin(), axis_vals[a].end());
            }
        }
    }
    if (!quads_ok) { h_quads.clear(); h_off.clear(); h_coords.clear(); nc[0] = nc[1] = nc[2] = 0; np1 = 0; }
    rec.n_surf = (int)h_surf.size();
    rec.n_full = (int)h_full.size();
    rec.n_verts = (int)h_verts.size();
    rec.n_quads = (int)h_quads.size();
    for (int k = 0; k < 3; ++k) rec.nc[k] = nc[k];
    rec.np1 = np1;

    DeviceGuard g(ctx->device);
    b3d_status st = B3D_OK;
    auto up = [&](auto **dst, const auto &vec, const char *what) {
        if (st != B3D_OK) return;
        if ((st = dalloc(ctx, dst, vec.size(), what)) != B3D_OK) return;
        if (!vec.empty()) {
            cudaError_t e = cudaMemcpy(*dst, vec.data(), vec.size() * sizeof(vec[0]), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) st = cuda_fail(ctx, e, what);
        }
    };
    up(&rec.verts, h_verts, "mesh vertices");
    up(&rec.tris_surf, h_surf, "mesh surface triangles");
    up(&rec.tris_full, h_full, "mesh triangles");
    up(&rec.faces, h_faces, "mesh faces");
    if (rec.n_quads > 0) {
        up(&rec.quads, h_quads, "mesh rectangles");
        up(&rec.class_off, h_off, "mesh quad classes");
        up(&rec.coords, h_coords, "mesh lattice");
    }
    if (st != B3D_OK) {
        dfree(ctx, rec.verts); dfree(ctx, rec.tris_surf); dfree(ctx, rec.tris_full); dfree(ctx, rec.faces);
        dfree(ctx, rec.quads); dfree(ctx, rec.class_off); dfree(ctx, rec.coords);
        return st;
    }
    ctx->meshes.push_back(rec);
    *mesh_id = (int32_t)ctx->meshes.size() - 1;
    return B3D_OK;
}

b3d_status b3d_set_scene(b3d_ctx *ctx, const b3d_intrinsics *intr, int32_t n_obj, const int32_t *mesh_ids,
                         const float *poses, const float *obs_depth_dev, b3d_stream stream) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    if (!intr || !obs_depth_dev) return fail(ctx, B3D_EINVAL, "intrinsics and obs_depth_dev must be non-NULL");
    if (n_obj < 1 || !mesh_ids || !poses) return fail(ctx, B3D_EINVAL, "a scene needs n_obj >= 1, mesh_ids and poses");
    if (intr->width < 1 || intr->height < 1 || (int64_t)intr->width * intr->height > ((int64_t)1 << 26))
        return fail(ctx, B3D_EINVAL, "image size must be >= 1x1 and at most 2^26 pixels");
    const float vals[6] = {intr->fx, intr->fy, intr->cx, intr->cy, intr->near_z, intr->far_z};
    if (!finite_all(vals, 6) || !(intr->fx > 0) || !(intr->fy > 0) || !(intr->near_z > 0) || !(intr->far_z > intr->near_z))
        return fail(ctx, B3D_EINVAL, "intrinsics need fx, fy > 0 and 0 < near_z < far_z, all finite");
    for (int32_t k = 0; k < n_obj; ++k)
        if (mesh_ids[k] < 0 || mesh_ids[k] >= (int32_t)ctx->meshes.size())
            return fail(ctx, B3D_ENOTFOUND, "scene object " + std::to_string(k) + " names an unknown mesh");
    if (!finite_all(poses, 16 * (int64_t)n_obj)) return fail(ctx, B3D_EINVAL, "poses must be finite");
    int64_t total_faces = 0;
    for (int32_t k = 0; k < n_obj; ++k) total_faces += ctx->meshes[mesh_ids[k]].n_faces;
    if (total_faces >= INT32_MAX) return fail(ctx, B3D_EINVAL, "scene has more than 2^31-1 triangles");
    if (!aligned16(obs_depth_dev) && ((uintptr_t)obs_depth_dev & 3u))
        return fail(ctx, B3D_EINVAL, "obs_depth_dev must be 4-byte aligned");

    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t npx = (int64_t)intr->width * intr->height;
    b3d_status st;
    for (unsigned long long *z : ctx->objz) dfree(ctx, z);  // shared backgrounds follow the new scene
    ctx->objz.clear();
    ctx->objz_ok.clear();
    if (npx > ctx->px_cap) {
        dfree(ctx, ctx->d_obs);
        ctx->px_cap = 0;
        if ((st = dalloc(ctx, &ctx->d_obs, (size_t)npx, "observed points")) != B3D_OK) return st;
        ctx->px_cap = npx;
    }
    // drop the background caches of slots the new scene does not have
    while (ctx->bgc.size() > (size_t)n_obj + 1) {
        BgCache &c = ctx->bgc.back();
        dfree(ctx, c.bg); dfree(ctx, c.bgd); dfree(ctx, c.ell); dfree(ctx, c.gs); dfree(ctx, c.gp); dfree(ctx, c.sums);
        dfree(ctx, c.qe); dfree(ctx, c.bgz); dfree(ctx, c.part); dfree(ctx, c.counter);
        dfree(ctx, c.nell); dfree(ctx, c.nsums); dfree(ctx, c.npart); dfree(ctx, c.ncounter);
        ctx->bgc.pop_back();
    }
    if (n_obj > ctx->pose_cap) {
        dfree(ctx, ctx->d_poses);
        ctx->pose_cap = 0;
        if ((st = dalloc(ctx, &ctx->d_poses, (size_t)16 * n_obj, "scene poses")) != B3D_OK) return st;
        ctx->pose_cap = n_obj;
    }
    cudaError_t e = cudaMemcpyAsync(ctx->d_poses, poses, sizeof(float) * 16 * n_obj, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "scene poses upload");
    Cam c{};
    c.W = intr->width; c.H = intr->height;
    c.fx = intr->fx; c.fy = intr->fy; c.cx = intr->cx; c.cy = intr->cy;
    c.near_z = intr->near_z; c.far_z = intr->far_z;
    c.inv_fx = 1.0f / intr->fx; c.inv_fy = 1.0f / intr->fy;
    ctx->cam = c;
    ctx->obj_mesh.assign(mesh_ids, mesh_ids + n_obj);
    ctx->tri_base.assign(n_obj, 0);
    for (int32_t k = 1; k < n_obj; ++k) ctx->tri_base[k] = ctx->tri_base[k - 1] + ctx->meshes[mesh_ids[k - 1]].n_faces;
    {
        Timed tm(ctx, B3D_K_SCENE, s);
        launch_obs_points(c, obs_depth_dev, ctx->d_obs, s);
    }
    ++ctx->launches;
    ctx->has_scene = true;
    ctx->views_dirty = true;
    bg_invalidate(ctx, -1);
    bg_invalidate_lik(ctx);
    return check_launch(ctx, "set_scene");
}

b3d_status b3d_set_observation(b3d_ctx *ctx, const float *obs_depth_dev, b3d_stream stream) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    if (!ctx->has_scene) return fail(ctx, B3D_EINVAL, "no scene: call b3d_set_scene first");
    if (!obs_depth_dev) return fail(ctx, B3D_EINVAL, "obs_depth_dev is NULL");
    DeviceGuard g(ctx->device);
    {
        Timed tm(ctx, B3D_K_SCENE, (cudaStream_t)stream);
        launch_obs_points(ctx->cam, obs_depth_dev, ctx->d_obs, (cudaStream_t)stream);
    }
    ++ctx->launches;
    bg_invalidate_lik(ctx);
    return check_launch(ctx, "set_observation");
}

b3d_status b3d_set_object_pose_dev(b3d_ctx *ctx, int32_t obj, const float *pose_dev, b3d_stream stream) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    b3d_status st = check_slot(ctx, obj);
    if (st != B3D_OK) return st;
    if (!pose_dev) return fail(ctx, B3D_EINVAL, "pose_dev is NULL");
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaMemcpyAsync(ctx->d_poses + 16 * obj, pose_dev, 16 * sizeof(float), cudaMemcpyDeviceToDevice,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set_object_pose_dev");
    bg_invalidate(ctx, obj);
    return B3D_OK;
}

b3d_status b3d_render_batch(b3d_ctx *ctx, int32_t obj_slot, int64_t n_hyp, const float *poses_dev, float *depth_dev,
                            int32_t *triid_dev, b3d_stream stream) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    b3d_status st = check_slot(ctx, obj_slot);
    if (st != B3D_OK) return st;
    if (n_hyp < 0) return fail(ctx, B3D_EINVAL, "n_hyp must be >= 0");
    if (n_hyp == 0) return B3D_OK;
    if (!poses_dev || !depth_dev) return fail(ctx, B3D_EINVAL, "poses_dev and depth_dev must be non-NULL");
    if (!aligned16(poses_dev)) return fail(ctx, B3D_EINVAL, "poses_dev must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_bg(ctx, obj_slot, s)) != B3D_OK) return st;
    if (!triid_dev && (st = ensure_bg_depth(ctx, obj_slot, s)) != B3D_OK) return st;
    {
        Timed tm(ctx, B3D_K_RENDER, s);
        SceneView sv = scene_view(ctx, obj_slot);
        sv.work = take_work(ctx);
        ctx->launches += launch_render_list(sv, PoseList{poses_dev}, n_hyp, depth_dev, triid_dev, 0, s);
    }
    return check_launch(ctx, "render_batch");
}

b3d_status b3d_score_batch(b3d_ctx *ctx, int32_t obj_slot, int64_t n_hyp, const float *poses_dev,
                           const b3d_lik_params *lik, float *loglik_dev, b3d_stream stream) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    b3d_status st = check_slot(ctx, obj_slot);
    if (st != B3D_OK) return st;
    Lik L;
    if ((st = make_lik(ctx, lik, &L)) != B3D_OK) return st;
    if (n_hyp < 0) return fail(ctx, B3D_EINVAL, "n_hyp must be >= 0");
    if (n_hyp == 0) return B3D_OK;
    if (!poses_dev || !loglik_dev) return fail(ctx, B3D_EINVAL, "poses_dev and loglik_dev must be non-NULL");
    if (!aligned16(poses_dev)) return fail(ctx, B3D_EINVAL, "poses_dev must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_bg(ctx, obj_slot, s)) != B3D_OK) return st;
    if ((st = ensure_bg_lik(ctx, obj_slot, lik, L, false, s)) != B3D_OK) return st;
    {
        Timed tm(ctx, B3D_K_SCORE, s);
        SceneView sv = scene_view(ctx, obj_slot);
        sv.work = take_work(ctx);
        launch_score_list(sv, L, PoseList{poses_dev}, n_hyp, loglik_dev, ctx->score_code(), s);
    }
    ++ctx->launches;
    return check_launch(ctx, "score_batch");
}

b3d_status b3d_render_camera_batch(b3d_ctx *ctx, int64_t n_hyp, const float *poses_dev, float *depth_dev,
                                   int32_t *triid_dev, b3d_stream stream) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    if (!ctx->has_scene) return fail(ctx, B3D_EINVAL, "no scene: call b3d_set_scene first");
    if (n_hyp < 0) return fail(ctx, B3D_EINVAL, "n_hyp must be >= 0");
    if (n_hyp == 0) return B3D_OK;
    if (!poses_dev || !depth_dev) return fail(ctx, B3D_EINVAL, "poses_dev and depth_dev must be non-NULL");
    if (!aligned16(poses_dev)) return fail(ctx, B3D_EINVAL, "poses_dev must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int n_obj = (int)ctx->obj_mesh.size();
    b3d_status st;
    if (ctx->views_dirty) {
        if (n_obj > ctx->views_cap) {
            dfree(ctx, ctx->d_views); dfree(ctx, ctx->d_tri_base);
            ctx->views_cap = 0;
            if ((st = dalloc(ctx, &ctx->d_views, (size_t)n_obj, "scene mesh views")) != B3D_OK) return st;
            if ((st = dalloc(ctx, &ctx->d_tri_base, (size_t)n_obj, "scene triangle bases")) != B3D_OK) return st;
            ctx->views_cap = n_obj;
        }
        ctx->h_views.resize(n_obj);
        ctx->h_tri_base.resize(n_obj);
        for (int k = 0; k < n_obj; ++k) {
            ctx->h_views[k] = view_of(ctx->meshes[ctx->obj_mesh[k]]);
            ctx->h_tri_base[k] = (int)ctx->tri_base[k];
        }
        cudaError_t e = cudaMemcpyAsync(ctx->d_views, ctx->h_views.data(), sizeof(MeshView) * n_obj,
                                        cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ctx->d_tri_base, ctx->h_tri_base.data(), sizeof(int) * n_obj, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "scene views upload");
        ctx->views_dirty = false;
    }
    {
        Timed tm(ctx, B3D_K_RENDER, s);
        launch_render_camera(ctx->cam, ctx->d_views, ctx->d_tri_base, ctx->d_poses, n_obj, PoseList{poses_dev}, n_hyp,
                             depth_dev, triid_dev, s);
    }
    ++ctx->launches;
    return check_launch(ctx, "render_camera_batch");
}

b3d_status b3d_score_noise_batch(b3d_ctx *ctx, int32_t obj_slot, int64_t n_hyp, const float *poses_dev,
                                 const b3d_noise_grid *grid, float *loglik_dev, float *marginal_dev,
                                 b3d_stream stream) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    b3d_status st = check_slot(ctx, obj_slot);
    if (st != B3D_OK) return st;
    NoiseLik N;
    if ((st = make_noise(ctx, grid, &N)) != B3D_OK) return st;
    if (n_hyp < 0) return fail(ctx, B3D_EINVAL, "n_hyp must be >= 0");
    if (n_hyp == 0) return B3D_OK;
    if (!poses_dev || !marginal_dev) return fail(ctx, B3D_EINVAL, "poses_dev and marginal_dev must be non-NULL");
    if (!aligned16(poses_dev)) return fail(ctx, B3D_EINVAL, "poses_dev must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_bg(ctx, obj_slot, s)) != B3D_OK) return st;
    if ((st = ensure_bg_noise(ctx, obj_slot, grid, N, s)) != B3D_OK) return st;
    const BgCache &c = bg_cache(ctx, obj_slot);
    {
        Timed tm(ctx, B3D_K_SCORE, s);
        SceneView sv = scene_view(ctx, obj_slot);
        sv.work = take_work(ctx);
        launch_score_noise(sv, N, poses_dev, n_hyp, c.nell, c.nsums, loglik_dev, marginal_dev, s);
    }
    ++ctx->launches;
    return check_launch(ctx, "score_noise_batch");
}

b3d_status b3d_score_depth_batch(b3d_ctx *ctx, int32_t obj_slot, int64_t n_hyp, const float *depth_dev,
                                 const int32_t *triid_dev, const b3d_lik_params *lik, float *loglik_dev,
                                 b3d_stream stream) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    if (!ctx->has_scene) return fail(ctx, B3D_EINVAL, "no scene: call b3d_set_scene first");
    if (obj_slot != -1) {
        b3d_status sst = check_slot(ctx, obj_slot);
        if (sst != B3D_OK) return sst;
    }
    Lik L;
    b3d_status st = make_lik(ctx, lik, &L);
    if (st != B3D_OK) return st;
    if (n_hyp < 0) return fail(ctx, B3D_EINVAL, "n_hyp must be >= 0");
    if (n_hyp == 0) return B3D_OK;
    if (!depth_dev || !loglik_dev) return fail(ctx, B3D_EINVAL, "depth_dev and loglik_dev must be non-NULL");
    if (lik->miss_mode == 1 && !triid_dev) return fail(ctx, B3D_EINVAL, "miss_mode 1 needs triid_dev");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_bg(ctx, obj_slot, s)) != B3D_OK) return st;
    if ((st = ensure_bg_depth(ctx, obj_slot, s)) != B3D_OK) return st;
    if ((st = ensure_bg_lik(ctx, obj_slot, lik, L, false, s)) != B3D_OK) return st;
    {
        Timed tm(ctx, B3D_K_SCORE_DEPTH, s);
        SceneView sv = scene_view(ctx, obj_slot);
        sv.work = take_work(ctx);
        ctx->launches += launch_score_depth(sv, L, depth_dev, triid_dev, n_hyp, loglik_dev, 0, s);
    }
    return check_launch(ctx, "score_depth_batch");
}

b3d_status b3d_expand_hypotheses(b3d_ctx *ctx, const float *centre_pose, const float *grid_frame,
                                 const b3d_stage *stage, float *poses_dev, b3d_stream stream) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    if (!centre_pose || !grid_frame || !stage || !poses_dev)
        return fail(ctx, B3D_EINVAL, "centre_pose, grid_frame, stage and poses_dev must be non-NULL");
    if (!finite_all(centre_pose, 16) || !finite_all(grid_frame, 9)) return fail(ctx, B3D_EINVAL, "non-finite pose or grid frame");
    int64_t n;
    b3d_status st = check_stage(ctx, *stage, &n);
    if (st != B3D_OK) return st;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_scratch(ctx, 0, 0)) != B3D_OK) return st;
    float *rot = nullptr;
    if ((st = rotation_table(ctx, *stage, &rot, s)) != B3D_OK) return st;
    float *centre = ctx->d_centre + 32;
    Timed tm(ctx, B3D_K_SCENE, s);
    launch_set16(centre, centre_pose, s);
    PoseGrid P{};
    P.centre = centre;
    P.rot = rot;
    for (int k = 0; k < 9; ++k) P.G[k] = grid_frame[k];
    P.n = stage->n_per_axis;
    P.n_rot = stage->n_rot;
    P.step = stage->step;
    launch_expand(P, n, poses_dev, s);
    ctx->launches += 2;
    return check_launch(ctx, "expand_hypotheses");
}

b3d_status b3d_lse_resample(b3d_ctx *ctx, int64_t n, const float *loglik_dev, int32_t m, uint64_t seed, int32_t stage,
                            float *logz_dev, int32_t *idx_dev, float *logq_dev, b3d_stream stream) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    if (n < 1 || n > INT32_MAX) return fail(ctx, B3D_EINVAL, "n must be in [1, 2^31-1]");
    if (m < 0) return fail(ctx, B3D_EINVAL, "m must be >= 0");
    if (!loglik_dev || !logz_dev) return fail(ctx, B3D_EINVAL, "loglik_dev and logz_dev must be non-NULL");
    if (m > 0 && (!idx_dev || !logq_dev)) return fail(ctx, B3D_EINVAL, "idx_dev and logq_dev must be non-NULL when m > 0");
    DeviceGuard g(ctx->device);
    b3d_status st = ensure_scratch(ctx, 0, 0);
    if (st != B3D_OK) return st;
    {
        Timed tm(ctx, B3D_K_RESAMPLE, (cudaStream_t)stream);
        launch_lse_resample(loglik_dev, n, m, seed, stage, ctx->d_part, ctx->d_counter, logz_dev, idx_dev, logq_dev,
                            ctx->d_err, (cudaStream_t)stream);
    }
    ++ctx->launches;
    return check_launch(ctx, "lse_resample");
}

b3d_status b3d_lse_resample_shard(b3d_ctx *ctx, int64_t n, const float *loglik_dev, int32_t m, uint64_t seed,
                                  int32_t stage, double mass_before, double mass, double logz_global, int64_t index_base,
                                  float *logz_dev, int32_t *idx_dev, float *logq_dev, b3d_stream stream) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    if (n < 1 || n > INT32_MAX) return fail(ctx, B3D_EINVAL, "n must be in [1, 2^31-1]");
    if (m < 0) return fail(ctx, B3D_EINVAL, "m must be >= 0");
    if (!loglik_dev || !logz_dev) return fail(ctx, B3D_EINVAL, "loglik_dev and logz_dev must be non-NULL");
    if (m > 0 && (!idx_dev || !logq_dev)) return fail(ctx, B3D_EINVAL, "idx_dev and logq_dev must be non-NULL when m > 0");
    if (!(mass_before >= 0.0 && mass_before <= 1.0) || !(mass >= 0.0 && mass_before + mass <= 1.0 + 1e-12))
        return fail(ctx, B3D_EINVAL, "need 0 <= mass_before, 0 <= mass and mass_before + mass <= 1");
    if (std::isnan(logz_global) || logz_global == INFINITY) return fail(ctx, B3D_EINVAL, "logz_global must be < +inf");
    if (index_base < 0 || index_base + n > (int64_t)INT32_MAX + 1)
        return fail(ctx, B3D_EINVAL, "index_base + n must be in [0, 2^31]");
    DeviceGuard g(ctx->device);
    b3d_status st = ensure_scratch(ctx, 0, 0);
    if (st != B3D_OK) return st;
    LseShard sh;
    sh.before = mass_before;
    sh.mass = mass;
    sh.logz = (float)logz_global;
    sh.base = (long long)index_base;
    {
        Timed tm(ctx, B3D_K_RESAMPLE, (cudaStream_t)stream);
        launch_lse_shard(loglik_dev, n, m, seed, stage, sh, ctx->d_part, ctx->d_counter, logz_dev, idx_dev, logq_dev,
                         ctx->d_err, (cudaStream_t)stream);
    }
    ++ctx->launches;
    return check_launch(ctx, "lse_resample_shard");
}

b3d_status b3d_enumerate_c2f(b3d_ctx *ctx, int32_t obj_slot, const float *centre_pose, const b3d_c2f_schedule *sch,
                             const b3d_lik_params *lik, float *particles_dev, float *logw_dev, float *logq_dev,
                             b3d_stream stream) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    b3d_status st = check_slot(ctx, obj_slot);
    if (st != B3D_OK) return st;
    Lik L;
    if ((st = make_lik(ctx, lik, &L)) != B3D_OK) return st;
    if (!centre_pose || !sch || !particles_dev || !logw_dev || !logq_dev)
        return fail(ctx, B3D_EINVAL, "centre_pose, schedule and the three outputs must be non-NULL");
    if (!finite_all(centre_pose, 16) || !finite_all(sch->grid_frame, 9)) return fail(ctx, B3D_EINVAL, "non-finite centre or grid frame");
    if (sch->n_stages < 1 || sch->n_stages > B3D_MAX_STAGES) return fail(ctx, B3D_EINVAL, "n_stages must be in [1, 8]");
    if (sch->path_density != 0 && sch->path_density != 1) return fail(ctx, B3D_EINVAL, "path_density must be 0 or 1");
    if (sch->n_particles < 1 || sch->n_particles > (1 << 20)) return fail(ctx, B3D_EINVAL, "n_particles must be in [1, 2^20]");
    int64_t n_max = 0, n_t[B3D_MAX_STAGES];
    for (int t = 0; t < sch->n_stages; ++t) {
        if ((st = check_stage(ctx, sch->stage[t], &n_t[t])) != B3D_OK) return st;
        n_max = std::max(n_max, n_t[t]);
    }
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_scratch(ctx, n_max, sch->n_particles)) != B3D_OK) return st;
    float *rot[B3D_MAX_STAGES];
    for (int t = 0; t < sch->n_stages; ++t)
        if ((st = rotation_table(ctx, sch->stage[t], &rot[t], s)) != B3D_OK) return st;
    if ((st = ensure_bg(ctx, obj_slot, s)) != B3D_OK) return st;
    if ((st = ensure_bg_lik(ctx, obj_slot, lik, L, false, s)) != B3D_OK) return st;
    SceneView sv = scene_view(ctx, obj_slot);
    sv.work = take_work(ctx);  // CTAs take hypotheses from a counter
    {
        Timed tm(ctx, B3D_K_SCENE, s);
        launch_set16(ctx->d_centre, centre_pose, s);
    }
    ++ctx->launches;
    for (int t = 0; t < sch->n_stages; ++t) {
        PoseGrid P{};
        P.centre = ctx->d_centre + 16 * (t & 1);
        P.rot = rot[t];
        for (int k = 0; k < 9; ++k) P.G[k] = sch->grid_frame[k];
        P.n = sch->stage[t].n_per_axis;
        P.n_rot = sch->stage[t].n_rot;
        P.step = sch->stage[t].step;
        {
            Timed tm(ctx, B3D_K_SCORE, s);
            launch_score_grid(sv, L, P, n_t[t], ctx->d_ll, ctx->score_code(), s);
        }
        {
            Timed tm(ctx, B3D_K_RESAMPLE, s);
            launch_lse_resample(ctx->d_ll, n_t[t], sch->n_particles, sch->seed, t, ctx->d_part, ctx->d_counter,
                                ctx->d_logz + t, ctx->d_idx, ctx->d_logq_tmp, ctx->d_err, s);
        }
        const int last = t == sch->n_stages - 1;
        {
            Timed tm(ctx, B3D_K_SELECT, s);
            launch_c2f_select(ctx->d_ll, ctx->d_idx, sch->n_particles, P, ctx->d_logz + t, last, sch->path_density, t,
                              sch->seed,
                              sch->n_stages, last ? nullptr : ctx->d_centre + 16 * ((t + 1) & 1), particles_dev, logw_dev,
                              logq_dev, s);
        }
        ctx->launches += 3;
    }
    return check_launch(ctx, "enumerate_c2f");
}

b3d_status b3d_score_multi(b3d_ctx *owner, int32_t n_items, const b3d_score_item *items, const b3d_lik_params *lik,
                           b3d_stream stream) {
    if (!owner) return B3D_EINVAL;
    owner->err.clear();
    if (n_items < 1 || !items) return fail(owner, B3D_EINVAL, "need n_items >= 1 and items");
    Lik L0;
    b3d_status st;
    std::vector<Lik> Ls((size_t)n_items);
    int64_t total = 0;
    int max_lat = 0;
    for (int32_t i = 0; i < n_items; ++i) {
        const b3d_score_item &it = items[i];
        if (!it.scene || it.scene->device != owner->device)
            return fail(owner, B3D_EINVAL, "item " + std::to_string(i) + ": scene context missing or on another device");
        if ((st = check_slot(it.scene, it.obj_slot)) != B3D_OK) return fail(owner, st, "item " + std::to_string(i) + ": " + it.scene->err);
        if ((st = make_lik(it.scene, lik, &Ls[i])) != B3D_OK) return fail(owner, st, it.scene->err);
        if (it.n_hyp < 0 || it.n_hyp > INT32_MAX) return fail(owner, B3D_EINVAL, "item n_hyp out of range");
        if (it.n_hyp > 0 && (!it.poses_dev || !it.loglik_dev || !aligned16(it.poses_dev)))
            return fail(owner, B3D_EINVAL, "item poses_dev (16-byte aligned) and loglik_dev must be non-NULL");
        total += it.n_hyp;
        const MeshRec &m = it.scene->meshes[it.scene->obj_mesh[it.obj_slot]];
        max_lat = std::max(max_lat, m.nc[0] + m.nc[1] + m.nc[2]);
    }
    (void)L0;
    if (total == 0) return B3D_OK;
    DeviceGuard g(owner->device);
    cudaStream_t s = (cudaStream_t)stream;
    for (int32_t i = 0; i < n_items; ++i) {
        if ((st = ensure_bg(items[i].scene, items[i].obj_slot, s)) != B3D_OK) return fail(owner, st, items[i].scene->err);
        if ((st = ensure_bg_lik(items[i].scene, items[i].obj_slot, lik, Ls[i], false, s)) != B3D_OK)
            return fail(owner, st, items[i].scene->err);
    }
    if ((st = grow(owner, owner->d_bwork, owner->bwork_cap, 8, "work counters")) != B3D_OK) return st;
    // heavier scenes first in the work queue (hypotheses x pixels)
    std::vector<int> order((size_t)n_items);
    for (int i = 0; i < n_items; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const double ca = (double)items[a].n_hyp * items[a].scene->cam.W * items[a].scene->cam.H;
        const double cb = (double)items[b].n_hyp * items[b].scene->cam.W * items[b].scene->cam.H;
        return ca > cb;
    });
    const size_t off_items = 0, off_begin = align16(sizeof(BatchItem) * n_items);
    const size_t bytes = off_begin + align16(sizeof(int64_t) * (n_items + 1));
    unsigned char *h = nullptr;
    int slot = 0;
    if ((st = batch_staging(owner, bytes, s, &h, &slot)) != B3D_OK) return st;
    BatchItem *bi = reinterpret_cast<BatchItem *>(h + off_items);
    int64_t *ib = reinterpret_cast<int64_t *>(h + off_begin);
    int64_t acc = 0;
    for (int k = 0; k < n_items; ++k) {
        const b3d_score_item &it = items[order[k]];
        BatchItem b;
        memset(&b, 0, sizeof b);
        b.S = scene_view(it.scene, it.obj_slot);
        b.S.tile_w = owner->tile_w;
        b.S.stats = nullptr;
        b.L = Ls[order[k]];
        b.list = PoseList{it.poses_dev};
        b.pose_kind = 0;
        b.n_hyp = (int)it.n_hyp;
        b.out_ll = it.loglik_dev;
        bi[k] = b;
        ib[k] = acc;
        acc += it.n_hyp;
    }
    ib[n_items] = acc;
    if ((st = batch_upload(owner, slot, bytes, s)) != B3D_OK) return st;
    {
        Timed tm(owner, B3D_K_SCORE, s);
        cudaMemsetAsync(owner->d_bwork, 0, sizeof(unsigned long long), s);
        launch_score_multi(reinterpret_cast<const BatchItem *>(owner->d_batch + off_items), n_items,
                           reinterpret_cast<const int64_t *>(owner->d_batch + off_begin), total, owner->batch_chunk,
                           owner->d_bwork, lik->half_window, max_lat, owner->score_code(), s);
    }
    ++owner->launches;
    return check_launch(owner, "score_multi");
}

b3d_status b3d_enumerate_multi(b3d_ctx *owner, int32_t n_items, const b3d_c2f_item *items, const b3d_lik_params *lik,
                               b3d_stream stream) {
    if (!owner) return B3D_EINVAL;
    owner->err.clear();
    if (n_items < 1 || !items) return fail(owner, B3D_EINVAL, "need n_items >= 1 and items");
    b3d_status st;
    const int T = items[0].schedule.n_stages;
    if (T < 1 || T > B3D_MAX_STAGES) return fail(owner, B3D_EINVAL, "n_stages must be in [1, 8]");
    std::vector<Lik> Ls((size_t)n_items);
    std::vector<int64_t> nh((size_t)n_items * T);
    int max_lat = 0;
    int64_t sum_m = 0;
    for (int32_t i = 0; i < n_items; ++i) {
        const b3d_c2f_item &it = items[i];
        const std::string tag = "item " + std::to_string(i) + ": ";
        if (!it.scene || it.scene->device != owner->device)
            return fail(owner, B3D_EINVAL, tag + "scene context missing or on another device");
        if ((st = check_slot(it.scene, it.obj_slot)) != B3D_OK) return fail(owner, st, tag + it.scene->err);
        if ((st = make_lik(it.scene, lik, &Ls[i])) != B3D_OK) return fail(owner, st, tag + it.scene->err);
        const b3d_c2f_schedule &sch = it.schedule;
        if (sch.n_stages != T) return fail(owner, B3D_EINVAL, tag + "every schedule needs the same number of stages");
        if (sch.n_particles < 1 || sch.n_particles > (1 << 20)) return fail(owner, B3D_EINVAL, tag + "n_particles out of range");
        if (sch.path_density != 0 && sch.path_density != 1) return fail(owner, B3D_EINVAL, tag + "path_density must be 0 or 1");
        if (!it.particles_dev || !it.logw_dev || !it.logq_dev) return fail(owner, B3D_EINVAL, tag + "outputs must be non-NULL");
        if ((!it.centre_dev && !finite_all(it.centre_pose, 16)) || !finite_all(sch.grid_frame, 9))
            return fail(owner, B3D_EINVAL, tag + "non-finite centre or grid frame");
        for (int t = 0; t < T; ++t)
            if ((st = check_stage(owner, sch.stage[t], &nh[(size_t)i * T + t])) != B3D_OK) return st;
        const MeshRec &m = it.scene->meshes[it.scene->obj_mesh[it.obj_slot]];
        max_lat = std::max(max_lat, m.nc[0] + m.nc[1] + m.nc[2]);
        sum_m += sch.n_particles;
    }
    DeviceGuard g(owner->device);
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<float *> rot((size_t)n_items * T);
    for (int32_t i = 0; i < n_items; ++i) {
        b3d_ctx *sc = items[i].scene;
        if ((st = ensure_bg(sc, items[i].obj_slot, s)) != B3D_OK) return fail(owner, st, sc->err);
        if ((st = ensure_bg_lik(sc, items[i].obj_slot, lik, Ls[i], false, s)) != B3D_OK) return fail(owner, st, sc->err);
        for (int t = 0; t < T; ++t)
            if ((st = rotation_table(sc, items[i].schedule.stage[t], &rot[(size_t)i * T + t], s)) != B3D_OK)
                return fail(owner, st, sc->err);
    }
    // scratch: scores of one stage, resampling partials and counters, draws, normalisers
    int64_t need_ll = 0, need_part = 0;
    for (int t = 0; t < T; ++t) {
        int64_t a = 0, b = 0;
        for (int32_t i = 0; i < n_items; ++i) { a += nh[(size_t)i * T + t]; b += lse_blocks(nh[(size_t)i * T + t]); }
        need_ll = std::max(need_ll, a);
        need_part = std::max(need_part, b);
    }
    if ((st = multi_scratch(owner, need_ll, need_part, n_items, sum_m, T)) != B3D_OK) return st;
    // heavier scenes first in the work queue (first-stage hypotheses x pixels)
    std::vector<int> order((size_t)n_items);
    for (int i = 0; i < n_items; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        const double ca = (double)nh[(size_t)a * T] * items[a].scene->cam.W * items[a].scene->cam.H;
        const double cb = (double)nh[(size_t)b * T] * items[b].scene->cam.W * items[b].scene->cam.H;
        return ca > cb;
    });
    const MultiLayout lay = multi_layout(n_items, T);
    const size_t o_cent = lay.o_cent, o_bi = lay.o_bi, o_li = lay.o_li, o_si = lay.o_si, o_ib = lay.o_ib,
                 o_bb = lay.o_bb, o_gp = lay.o_gp, bytes = lay.bytes;
    unsigned char *h = nullptr;
    int slot = 0;
    if ((st = batch_staging(owner, bytes, s, &h, &slot)) != B3D_OK) return st;
    unsigned char *d = owner->d_batch;
    float *hc = reinterpret_cast<float *>(h + o_cent);
    float *dc = reinterpret_cast<float *>(d + o_cent);
    std::vector<int64_t> midx((size_t)n_items);
    int64_t macc = 0;
    const float **gp = reinterpret_cast<const float **>(h + o_gp);
    int n_gather = 0;
    for (int k = 0; k < n_items; ++k) {
        const int i = order[k];
        memcpy(hc + 32 * k, items[i].centre_pose, 16 * sizeof(float));
        if (items[i].centre_dev) {  // device centre: copied into the slot after the upload
            gp[2 * n_gather] = items[i].centre_dev;
            gp[2 * n_gather + 1] = dc + 32 * k;
            ++n_gather;
        }
        midx[k] = macc;
        macc += items[i].schedule.n_particles;
    }
    std::vector<int64_t> totals(T);
    std::vector<int> blocks(T);
    for (int t = 0; t < T; ++t) {
        BatchItem *bi = reinterpret_cast<BatchItem *>(h + o_bi) + (size_t)t * n_items;
        LseItem *li = reinterpret_cast<LseItem *>(h + o_li) + (size_t)t * n_items;
        SelectItem *si = reinterpret_cast<SelectItem *>(h + o_si) + (size_t)t * n_items;
        int64_t *ib = reinterpret_cast<int64_t *>(h + o_ib) + (size_t)t * (n_items + 1);
        int *bb = reinterpret_cast<int *>(h + o_bb) + (size_t)t * (n_items + 1);
        int64_t acc = 0;
        int bacc = 0;
        int64_t pacc = 0;
        for (int k = 0; k < n_items; ++k) {
            const int i = order[k];
            const b3d_c2f_item &it = items[i];
            const b3d_stage &stg = it.schedule.stage[t];
            const int64_t n = nh[(size_t)i * T + t];
            PoseGrid P{};
            P.centre = dc + 32 * k + 16 * (t & 1);
            P.rot = rot[(size_t)i * T + t];
            for (int q = 0; q < 9; ++q) P.G[q] = it.schedule.grid_frame[q];
            P.n = stg.n_per_axis;
            P.n_rot = stg.n_rot;
            P.step = stg.step;
            BatchItem b;
            memset(&b, 0, sizeof b);
            b.S = scene_view(it.scene, it.obj_slot);
            b.S.tile_w = owner->tile_w;
            b.S.stats = nullptr;
            b.L = Ls[i];
            b.grid = P;
            b.pose_kind = 1;
            b.n_hyp = (int)n;
            b.out_ll = owner->d_bll + acc;
            bi[k] = b;
            ib[k] = acc;
            const int nb = lse_blocks(n);
            LseItem l;
            memset(&l, 0, sizeof l);
            l.ll = owner->d_bll + acc;
            l.n = n;
            l.n_blocks = nb;
            l.chunk = (int)((n + nb - 1) / nb);
            l.block_begin = bacc;
            l.m = it.schedule.n_particles;
            l.seed = (unsigned long long)it.schedule.seed;
            l.stage = t;
            l.part = owner->d_bpart + pacc;
            l.counter = owner->d_bcnt + k;
            l.logz = owner->d_blogz + (size_t)k * T + t;
            l.idx = owner->d_bidx + midx[k];
            l.logq = owner->d_blogq + midx[k];
            li[k] = l;
            bb[k] = bacc;
            SelectItem sv;
            memset(&sv, 0, sizeof sv);
            sv.ll = l.ll;
            sv.idx = l.idx;
            sv.m = l.m;
            sv.grid = P;
            sv.logz = l.logz;
            sv.centre_next = t == T - 1 ? it.map_dev : dc + 32 * k + 16 * ((t + 1) & 1);
            sv.particles = it.particles_dev;
            sv.logw = it.logw_dev;
            sv.logq = it.logq_dev;
            sv.seed = l.seed;
            sv.n_stages = T;
            sv.path = it.schedule.path_density;
            si[k] = sv;
            acc += n;
            bacc += nb;
            pacc += nb;
        }
        ib[n_items] = acc;
        bb[n_items] = bacc;
        totals[t] = acc;
        blocks[t] = bacc;
    }
    if ((st = batch_upload(owner, slot, bytes, s)) != B3D_OK) return st;
    if (n_gather > 0) {
        launch_gather16(reinterpret_cast<const float *const *>(d + o_gp), n_gather, s);
        ++owner->launches;
    }
    cudaMemsetAsync(owner->d_bwork, 0, sizeof(unsigned long long) * 8, s);
    for (int t = 0; t < T; ++t) {
        {
            Timed tm(owner, B3D_K_SCORE, s);
            launch_score_multi(reinterpret_cast<const BatchItem *>(d + o_bi) + (size_t)t * n_items, n_items,
                               reinterpret_cast<const int64_t *>(d + o_ib) + (size_t)t * (n_items + 1), totals[t],
                               owner->batch_chunk, owner->d_bwork + t, lik->half_window, max_lat, owner->score_code(), s);
        }
        {
            Timed tm(owner, B3D_K_RESAMPLE, s);
            launch_lse_multi(reinterpret_cast<const LseItem *>(d + o_li) + (size_t)t * n_items, n_items, blocks[t],
                             reinterpret_cast<const int *>(d + o_bb) + (size_t)t * (n_items + 1), owner->d_err, s);
        }
        {
            Timed tm(owner, B3D_K_SELECT, s);
            launch_select_multi(reinterpret_cast<const SelectItem *>(d + o_si) + (size_t)t * n_items, n_items,
                                t == T - 1, t, s);
        }
        owner->launches += 3;
    }
    return check_launch(owner, "enumerate_multi");
}

b3d_status b3d_score_grad(b3d_ctx *ctx, int32_t obj_slot, int64_t n_hyp, const float *poses_dev,
                          const b3d_lik_params *lik, float *loglik_dev, float *dpose_dev, float *dsigma_dev,
                          float *dpout_dev, b3d_stream stream) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    b3d_status st = check_slot(ctx, obj_slot);
    if (st != B3D_OK) return st;
    Lik L;
    if ((st = make_lik(ctx, lik, &L)) != B3D_OK) return st;
    if (lik->kind != 1) return fail(ctx, B3D_EINVAL, "score_grad needs the smooth likelihood (kind 1)");
    if (n_hyp < 0) return fail(ctx, B3D_EINVAL, "n_hyp must be >= 0");
    if (n_hyp == 0) return B3D_OK;
    if (!poses_dev || !loglik_dev) return fail(ctx, B3D_EINVAL, "poses_dev and loglik_dev must be non-NULL");
    if (!aligned16(poses_dev)) return fail(ctx, B3D_EINVAL, "poses_dev must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_bg(ctx, obj_slot, s)) != B3D_OK) return st;
    if ((st = ensure_bg_lik(ctx, obj_slot, lik, L, true, s)) != B3D_OK) return st;
    {
        Timed tm(ctx, B3D_K_GRAD, s);
        launch_grad_list(scene_view(ctx, obj_slot), L, PoseList{poses_dev}, n_hyp, loglik_dev, dpose_dev, dsigma_dev,
                         dpout_dev, 0, s);
    }
    ++ctx->launches;
    return check_launch(ctx, "score_grad");
}

b3d_status b3d_refine_smooth(b3d_ctx *ctx, int32_t obj_slot, int64_t n_hyp, float *poses_dev,
                             const b3d_lik_params *lik, int32_t n_steps, float lr, float beta1, float beta2, float eps,
                             float *loglik_dev, b3d_stream stream) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    b3d_status st = check_slot(ctx, obj_slot);
    if (st != B3D_OK) return st;
    Lik L;
    if ((st = make_lik(ctx, lik, &L)) != B3D_OK) return st;
    if (lik->kind != 1) return fail(ctx, B3D_EINVAL, "refine_smooth needs the smooth likelihood (kind 1)");
    if (n_hyp < 0) return fail(ctx, B3D_EINVAL, "n_hyp must be >= 0");
    if (n_steps < 1) return fail(ctx, B3D_EINVAL, "n_steps must be >= 1");
    if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f) ||
        !std::isfinite(lr) || !std::isfinite(eps))
        return fail(ctx, B3D_EINVAL, "need lr > 0, 0 <= beta1, beta2 < 1, eps > 0 (finite)");
    if (n_hyp == 0) return B3D_OK;
    if (!poses_dev) return fail(ctx, B3D_EINVAL, "poses_dev must be non-NULL");
    if (!aligned16(poses_dev)) return fail(ctx, B3D_EINVAL, "poses_dev must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (n_hyp > ctx->refine_cap) {
        dfree(ctx, ctx->d_refine);
        ctx->refine_cap = 0;
        if ((st = dalloc(ctx, &ctx->d_refine, (size_t)19 * n_hyp, "refinement state")) != B3D_OK) return st;
        ctx->refine_cap = n_hyp;
    }
    float *m = ctx->d_refine, *v = m + 6 * n_hyp, *dpose = v + 6 * n_hyp, *ll = dpose + 6 * n_hyp;
    cudaMemsetAsync(m, 0, sizeof(float) * 12 * (size_t)n_hyp, s);
    if ((st = ensure_bg(ctx, obj_slot, s)) != B3D_OK) return st;
    if ((st = ensure_bg_lik(ctx, obj_slot, lik, L, true, s)) != B3D_OK) return st;
    const SceneView sv = scene_view(ctx, obj_slot);
    double p1 = 1.0, p2 = 1.0;
    for (int t = 1; t <= n_steps; ++t) {
        {
            Timed tm(ctx, B3D_K_GRAD, s);
            launch_grad_list(sv, L, PoseList{poses_dev}, n_hyp, t == n_steps && loglik_dev ? loglik_dev : ll, dpose,
                             nullptr, nullptr, 0, s);
        }
        p1 *= beta1;
        p2 *= beta2;
        launch_adam_se3(n_hyp, dpose, m, v, poses_dev, lr, beta1, beta2, eps, (float)(1.0 - p1), (float)(1.0 - p2), s);
        ctx->launches += 2;
    }
    return check_launch(ctx, "refine_smooth");
}

b3d_status b3d_se3_compose(b3d_ctx *ctx, int64_t n, const float *xi_dev, const float *poses_dev, float *out_dev,
                           b3d_stream stream) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    if (n < 0) return fail(ctx, B3D_EINVAL, "n must be >= 0");
    if (n == 0) return B3D_OK;
    if (!xi_dev || !poses_dev || !out_dev) return fail(ctx, B3D_EINVAL, "xi_dev, poses_dev and out_dev must be non-NULL");
    DeviceGuard g(ctx->device);
    launch_se3_compose(n, xi_dev, poses_dev, out_dev, (cudaStream_t)stream);
    ++ctx->launches;
    return check_launch(ctx, "se3_compose");
}

b3d_status b3d_get_tuning(b3d_ctx *ctx, b3d_tuning *out) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    if (!out) return fail(ctx, B3D_EINVAL, "out is NULL");
    out->tile_w = ctx->tile_w;
    out->cta_threads = ctx->cta_threads;
    out->ctas_per_sm = ctx->ctas_per_sm;
    out->high_occupancy = ctx->high_occupancy;
    out->batch_chunk = ctx->batch_chunk;
    return B3D_OK;
}

b3d_status b3d_set_tuning(b3d_ctx *ctx, const b3d_tuning *t) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    if (!t) return fail(ctx, B3D_EINVAL, "tuning is NULL");
    if (t->tile_w < 8 || t->tile_w > 256) return fail(ctx, B3D_EINVAL, "tile_w must be in [8, 256]");
    if (t->cta_threads != 32 && t->cta_threads != 64 && t->cta_threads != 128 && t->cta_threads != 256)
        return fail(ctx, B3D_EINVAL, "cta_threads must be 32, 64, 128 or 256");
    if (t->ctas_per_sm < 0 || t->ctas_per_sm > 32) return fail(ctx, B3D_EINVAL, "ctas_per_sm must be in [0, 32]");
    if (t->high_occupancy != 0 && t->high_occupancy != 1) return fail(ctx, B3D_EINVAL, "high_occupancy must be 0 or 1");
    if (t->batch_chunk < 1 || t->batch_chunk > 1024) return fail(ctx, B3D_EINVAL, "batch_chunk must be in [1, 1024]");
    ctx->batch_chunk = t->batch_chunk;
    ctx->tile_w = t->tile_w;
    ctx->cta_threads = t->cta_threads;
    ctx->ctas_per_sm = t->ctas_per_sm;
    ctx->high_occupancy = t->high_occupancy;
    return B3D_OK;
}

b3d_status b3d_autotune(b3d_ctx *ctx, int32_t obj_slot, const float *centre_pose, const float *grid_frame,
                        const b3d_stage *stage, const b3d_lik_params *lik, b3d_tuning *best, b3d_stream stream) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    b3d_status st = check_slot(ctx, obj_slot);
    if (st != B3D_OK) return st;
    Lik L;
    if ((st = make_lik(ctx, lik, &L)) != B3D_OK) return st;
    if (!centre_pose || !grid_frame || !stage) return fail(ctx, B3D_EINVAL, "centre_pose, grid_frame and stage must be non-NULL");
    int64_t n;
    if ((st = check_stage(ctx, *stage, &n)) != B3D_OK) return st;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_scratch(ctx, n, 1)) != B3D_OK) return st;
    float *rot = nullptr;
    if ((st = rotation_table(ctx, *stage, &rot, s)) != B3D_OK) return st;
    if ((st = ensure_bg(ctx, obj_slot, s)) != B3D_OK) return st;
    if ((st = ensure_bg_lik(ctx, obj_slot, lik, L, false, s)) != B3D_OK) return st;
    float *centre = ctx->d_centre + 32;
    launch_set16(centre, centre_pose, s);
    PoseGrid P{};
    P.centre = centre;
    P.rot = rot;
    for (int k = 0; k < 9; ++k) P.G[k] = grid_frame[k];
    P.n = stage->n_per_axis;
    P.n_rot = stage->n_rot;
    P.step = stage->step;
    cudaEvent_t e0 = take_event(ctx), e1 = take_event(ctx);
    const b3d_tuning saved{ctx->tile_w, ctx->cta_threads, ctx->ctas_per_sm, ctx->high_occupancy, ctx->batch_chunk};
    b3d_tuning win = saved;
    float win_ms = INFINITY;
    for (int hi : {0, 1})
        for (int nt : {256, 128, 64, 32})
            for (int tw : {32, 64, 96, 128}) {
                const int cps = 0;
                ctx->tile_w = tw;
                ctx->cta_threads = nt;
                ctx->ctas_per_sm = cps;
                ctx->high_occupancy = hi;
                SceneView sv = scene_view(ctx, obj_slot);
                sv.work = take_work(ctx);  // as enumerate_c2f launches it
                launch_score_grid(sv, L, P, n, ctx->d_ll, ctx->score_code(), s);  // warm
                cudaEventRecord(e0, s);
                launch_score_grid(sv, L, P, n, ctx->d_ll, ctx->score_code(), s);
                cudaEventRecord(e1, s);
                ctx->launches += 2;
                cudaError_t e = cudaEventSynchronize(e1);
                if (e != cudaSuccess) {
                    ctx->tile_w = saved.tile_w; ctx->cta_threads = saved.cta_threads; ctx->ctas_per_sm = saved.ctas_per_sm;
                    ctx->high_occupancy = saved.high_occupancy;
                    return cuda_fail(ctx, e, "autotune");
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < win_ms) { win_ms = ms; win = b3d_tuning{tw, nt, cps, hi, ctx->batch_chunk}; }
            }
    ctx->event_pool.push_back(e0);
    ctx->event_pool.push_back(e1);
    ctx->tile_w = win.tile_w;
    ctx->cta_threads = win.cta_threads;
    ctx->ctas_per_sm = win.ctas_per_sm;
    ctx->high_occupancy = win.high_occupancy;
    if (best) *best = win;
    return check_launch(ctx, "autotune");
}

b3d_status b3d_autotune_multi(b3d_ctx *owner, int32_t n_items, const b3d_c2f_item *items, const b3d_lik_params *lik,
                              b3d_tuning *best, b3d_stream stream) {
    if (!owner) return B3D_EINVAL;
    owner->err.clear();
    if (n_items < 1 || !items || !lik) return fail(owner, B3D_EINVAL, "need n_items >= 1, items and lik");
    DeviceGuard g(owner->device);
    cudaStream_t s = (cudaStream_t)stream;
    const b3d_tuning saved{owner->tile_w, owner->cta_threads, owner->ctas_per_sm, owner->high_occupancy, owner->batch_chunk};
    auto apply = [&](const b3d_tuning &t) {
        owner->tile_w = t.tile_w; owner->cta_threads = t.cta_threads; owner->ctas_per_sm = t.ctas_per_sm;
        owner->high_occupancy = t.high_occupancy; owner->batch_chunk = t.batch_chunk;
    };
    // one untimed pass with the current tuning: sizes the scratch and builds every item's tables
    b3d_status st = b3d_enumerate_multi(owner, n_items, items, lik, stream);
    if (st != B3D_OK) return st;
    cudaEvent_t e0 = take_event(owner), e1 = take_event(owner);
    auto timed = [&](const b3d_tuning &t, float *ms) -> b3d_status {
        apply(t);
        b3d_status r = b3d_enumerate_multi(owner, n_items, items, lik, stream);  // warm
        if (r == B3D_OK) {
            cudaEventRecord(e0, s);
            r = b3d_enumerate_multi(owner, n_items, items, lik, stream);
            cudaEventRecord(e1, s);
        }
        if (r != B3D_OK) return r;
        cudaError_t e = cudaEventSynchronize(e1);
        if (e != cudaSuccess) return cuda_fail(owner, e, "autotune_multi");
        cudaEventElapsedTime(ms, e0, e1);
        return B3D_OK;
    };
    // launch shapes: the current one and 128- or 256-thread CTAs with 64- or 128-pixel tiles
    std::vector<b3d_tuning> shapes{saved};
    for (int nt : {128, 256})
        for (int tw : {64, 128}) shapes.push_back(b3d_tuning{tw, nt, 0, 0, saved.batch_chunk});
    b3d_tuning win = saved;
    float win_ms = INFINITY;
    for (const b3d_tuning &t : shapes) {
        float ms = 0.f;
        if ((st = timed(t, &ms)) != B3D_OK) break;
        if (ms < win_ms) { win_ms = ms; win = t; }
    }
    // then hypotheses per work-queue grab
    for (int chunk : {1, 2, 4, 8, 16, 32}) {
        if (st != B3D_OK) break;
        b3d_tuning t = win;
        t.batch_chunk = chunk;
        float ms = 0.f;
        if ((st = timed(t, &ms)) != B3D_OK) break;
        if (ms < win_ms) { win_ms = ms; win = t; }
    }
    owner->event_pool.push_back(e0);
    owner->event_pool.push_back(e1);
    if (st != B3D_OK) {
        apply(saved);
        return st;
    }
    apply(win);
    if (best) *best = win;
    return B3D_OK;
}

b3d_status b3d_set_instrumentation(b3d_ctx *ctx, int32_t flags) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    if (flags & ~(B3D_INSTR_TIMING | B3D_INSTR_WORK)) return fail(ctx, B3D_EINVAL, "unknown instrumentation flags");
    DeviceGuard g(ctx->device);
    if ((flags & B3D_INSTR_WORK) && !ctx->d_stats) {
        b3d_status st = dalloc(ctx, &ctx->d_stats, kNumStats, "work counters");
        if (st != B3D_OK) return st;
        cudaError_t e = cudaMemset(ctx->d_stats, 0, kNumStats * sizeof(unsigned long long));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "work counters");
    }
    ctx->instr = flags;
    return B3D_OK;
}

b3d_status b3d_kernel_time(b3d_ctx *ctx, int32_t kernel_class, double *total_ms, int64_t *launches) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    if (kernel_class < 0 || kernel_class >= B3D_K_COUNT || !total_ms || !launches)
        return fail(ctx, B3D_EINVAL, "kernel_class out of range or NULL output");
    DeviceGuard g(ctx->device);
    double ms = 0;
    int64_t n = 0;
    for (auto &ab : ctx->pending[kernel_class]) {
        cudaError_t e = cudaEventSynchronize(ab.second);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel timing");
        float t = 0.f;
        cudaEventElapsedTime(&t, ab.first, ab.second);
        ms += t;
        ++n;
        ctx->event_pool.push_back(ab.first);
        ctx->event_pool.push_back(ab.second);
    }
    ctx->pending[kernel_class].clear();
    *total_ms = ms;
    *launches = n;
    return B3D_OK;
}

b3d_status b3d_work_counters(b3d_ctx *ctx, int64_t *out) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    if (!out) return fail(ctx, B3D_EINVAL, "out is NULL");
    if (!ctx->d_stats) {
        for (int k = 0; k < kNumStats; ++k) out[k] = 0;
        return B3D_OK;
    }
    DeviceGuard g(ctx->device);
    unsigned long long h[kNumStats];
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h, ctx->d_stats, sizeof h, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_stats, 0, sizeof h);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "work counters");
    for (int k = 0; k < kNumStats; ++k) out[k] = (int64_t)h[k];
    return B3D_OK;
}

b3d_status b3d_sync(b3d_ctx *ctx, b3d_stream stream) {
    if (!ctx) return B3D_EINVAL;
    ctx->err.clear();
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    int flag = 0;
    e = cudaMemcpy(&flag, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "error flag read");
    if (flag) {
        cudaMemset(ctx->d_err, 0, sizeof(int));
        std::string what;
        if (flag & 1) what += " bounds check failed;";
        if (flag & 2) what += " bounded wait expired;";
        if (flag & 4) what += " resampling over all -inf scores;";
        return fail(ctx, B3D_EDEVICE, "device error flag " + std::to_string(flag) + ":" + what);
    }
    return B3D_OK;
}

}  // extern "C"

// ==========================================================================================
// Context hooks for the tracking server (b3d_server.cu); not part of the C ABI.
// ==========================================================================================
namespace b3d {

uint64_t ctx_used_bytes(b3d_ctx *ctx) { return ctx->used; }

void ctx_set_budget(b3d_ctx *ctx, uint64_t budget) { ctx->budget = budget; }

b3d_status ctx_alloc_bytes(b3d_ctx *ctx, size_t bytes, void **out, const char *what) {
    unsigned char *p = nullptr;
    DeviceGuard g(ctx->device);
    b3d_status st = dalloc(ctx, &p, bytes, what);
    *out = p;
    return st;
}

float *ctx_scene_poses(b3d_ctx *ctx) { return ctx->d_poses; }

int *ctx_err_flag(b3d_ctx *ctx) { return ctx->d_err; }

b3d_status ctx_prepare_shared_bg(b3d_ctx *ctx, cudaStream_t s) {
    if (!ctx->has_scene) return fail(ctx, B3D_EINVAL, "no scene");
    const size_t n_obj = ctx->obj_mesh.size();
    if (n_obj - 1 > (size_t)kMaxBgSources) return B3D_OK;  // too many objects: per-slot rendering
    const int64_t npx = (int64_t)ctx->cam.W * ctx->cam.H;
    DeviceGuard g(ctx->device);
    for (unsigned long long *z : ctx->objz) dfree(ctx, z);
    ctx->objz.assign(n_obj, nullptr);
    ctx->objz_ok.assign(n_obj, 0);
    for (size_t o = 0; o < n_obj; ++o) {
        b3d_status st = dalloc(ctx, &ctx->objz[o], (size_t)npx, "object z-buffer");
        if (st != B3D_OK) {
            for (unsigned long long *z : ctx->objz) dfree(ctx, z);
            ctx->objz.clear();
            ctx->objz_ok.clear();
            return st;
        }
    }
    (void)s;
    return B3D_OK;
}

void ctx_tracked_moved(b3d_ctx *ctx, int32_t n_slots) {
    if (ctx->objz.empty()) {
        bg_invalidate(ctx, -1);
        return;
    }
    for (int32_t o = 0; o < n_slots && o < (int32_t)ctx->obj_mesh.size(); ++o) bg_invalidate(ctx, o);
}

b3d_status ctx_build_slot_bgs(b3d_ctx *ctx, int32_t n_slots, cudaStream_t s) {
    if (ctx->objz.empty()) return B3D_OK;  // not prepared: ensure_bg renders each slot's background
    const int32_t n_obj = (int32_t)ctx->obj_mesh.size();
    const int64_t npx = (int64_t)ctx->cam.W * ctx->cam.H;
    bool any = false;
    for (int32_t k = 0; k < n_slots && k < n_obj; ++k) {
        const size_t i = (size_t)k + 1;
        if (i < ctx->bgc.size() && ctx->bgc[i].dirty && ctx->bgc[i].cap >= npx) any = true;
    }
    if (!any) return B3D_OK;
    DeviceGuard g(ctx->device);
    Timed tm(ctx, B3D_K_SCENE, s);
    for (int32_t o = 0; o < n_obj; ++o) {
        if (ctx->objz_ok[o]) continue;
        const MeshRec &m = ctx->meshes[ctx->obj_mesh[o]];
        launch_bg_clear(ctx->objz[o], npx, s);
        ++ctx->launches;
        if (m.n_full > 0) {
            launch_bg_raster(ctx->cam, view_of(m), ctx->d_poses + 16 * o, (int)ctx->tri_base[o], ctx->objz[o], s);
            ++ctx->launches;
        }
        ctx->objz_ok[o] = 1;
    }
    const unsigned long long *src[kMaxBgSources];
    for (int32_t k = 0; k < n_slots && k < n_obj; ++k) {
        BgCache &c = bg_cache(ctx, k);
        if (!c.dirty || c.cap < npx) continue;
        int n_src = 0;
        for (int32_t o = 0; o < n_obj; ++o)
            if (o != k && ctx->meshes[ctx->obj_mesh[o]].n_full > 0) src[n_src++] = ctx->objz[o];
        launch_bg_min(npx, src, n_src, c.bg, s);
        ++ctx->launches;
        c.dirty = false;
        c.lik_valid = c.grad_valid = c.nvalid = c.bgd_valid = false;
    }
    return check_launch(ctx, "shared backgrounds");
}

b3d_status ctx_prepare_slot(b3d_ctx *ctx, int32_t slot, const b3d_lik_params *lik, const b3d_c2f_schedule *sch,
                            cudaStream_t s) {
    b3d_status st = check_slot(ctx, slot);
    if (st != B3D_OK) return st;
    Lik L;
    if ((st = make_lik(ctx, lik, &L)) != B3D_OK) return st;
    DeviceGuard g(ctx->device);
    if ((st = ensure_bg(ctx, slot, s)) != B3D_OK) return st;
    if ((st = ensure_bg_lik(ctx, slot, lik, L, false, s)) != B3D_OK) return st;
    for (int t = 0; t < sch->n_stages; ++t) {
        float *rot = nullptr;
        if ((st = rotation_table(ctx, sch->stage[t], &rot, s)) != B3D_OK) return st;
    }
    return B3D_OK;
}

// Size the owner's batched-enumeration scratch and staging for n_items items of schedule
// sch, so batched calls up to that size allocate nothing (and never synchronise).
b3d_status owner_reserve(b3d_ctx *owner, int64_t n_items, const b3d_c2f_schedule *sch) {
    const int T = sch->n_stages;
    int64_t max_n = 1;
    for (int t = 0; t < T; ++t) {
        const b3d_stage &g = sch->stage[t];
        max_n = std::max<int64_t>(max_n, (int64_t)g.n_per_axis * g.n_per_axis * g.n_per_axis * g.n_rot);
    }
    DeviceGuard g(owner->device);
    b3d_status st = multi_scratch(owner, n_items * max_n, n_items * lse_blocks(max_n), n_items,
                                  n_items * sch->n_particles, T);
    if (st != B3D_OK) return st;
    unsigned char *h = nullptr;
    int slot = 0;
    st = batch_staging(owner, multi_layout(n_items, T).bytes, nullptr, &h, &slot);
    return st;
}

}  // namespace b3d
