// b3d_server.cu - the tracking server of include/b3d.h: sessions admitted under an HBM
// budget, depth frames queued per session and batched continuously across sessions.
//
// Host code only. Each frame's work runs in the library's kernels: the depth upload and
// observed-cloud build (b3d_set_observation), one batched coarse-to-fine enumeration over
// every tracked object of every frame in the batch (b3d_enumerate_multi, centres read
// from the device), and device-to-device copies that make the new estimates the scene
// poses of the next frame. The host never waits for a frame before issuing the next
// batch; a completion thread polls one event per batch.
//
// Threads: the caller's threads (open / close / submit / wait), one worker thread that
// forms and issues batches on the server's stream, one completion thread. Shared state is
// guarded by one mutex; a session's contexts and device buffers are touched only by the
// worker while the session has frames running, and by open / close / export / import
// while it has none.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "b3d.h"
#include "b3d_internal.h"

using namespace b3d;
using Clock = std::chrono::steady_clock;

namespace {

thread_local std::string g_srv_error;

b3d_status srv_fail(b3d_status st, const std::string &msg) {
    g_srv_error = msg;
    return st;
}

b3d_status srv_ok() {
    g_srv_error.clear();
    return B3D_OK;
}

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// SplitMix64 output function (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", 2014).
uint64_t splitmix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

struct Frame {
    int64_t ticket = 0, index = 0;
    int32_t sid = 0;
    int ring = 0;
    Clock::time_point t_submit, t_issue;
};

struct Session {
    int32_t id = 0;
    b3d_ctx *ctx = nullptr;
    int32_t n_obj = 0, n_track = 0, M = 0;
    int64_t npx = 0;
    float grid_frame[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    uint64_t seed = 0, reserved = 0;
    // device, owned by ctx: depth frame, particles [n_track][M][16], their scores and
    // proposal densities [n_track][M], estimates [n_track][16]
    float *d_depth = nullptr, *d_part = nullptr, *d_logw = nullptr, *d_logq = nullptr, *d_map = nullptr;
    // pinned host, one entry per queue slot: the submitted frame, its estimates, its error flag
    float *h_ring = nullptr;
    float *h_res = nullptr;
    int *h_err = nullptr;
    std::vector<int> ring_free;
    std::deque<Frame> queue;  // submitted, not yet taken by the worker
    int64_t next_index = 0;
    int running = 0;          // taken by the worker, not yet completed
    int writers = 0;          // submit calls copying into a queue slot
    bool closing = false;
    bool held = false;        // export / import in progress
};

struct Done {
    b3d_frame_result res;
    std::vector<float> poses;
};

struct Batch {
    cudaEvent_t ev = nullptr;
    std::vector<Frame> frames;
    int64_t hyps = 0;
    b3d_status status = B3D_OK;
    std::string msg;
};

void free_session_host(Session *x) {
    if (x->h_ring) cudaFreeHost(x->h_ring);
    if (x->h_res) cudaFreeHost(x->h_res);
    if (x->h_err) cudaFreeHost(x->h_err);
    x->h_ring = x->h_res = nullptr;
    x->h_err = nullptr;
}

}  // namespace

struct b3d_server {
    int device = 0;
    uint64_t budget = 0, reserved = 0, scratch = 0;
    b3d_server_config cfg{};
    int64_t hyp_per_item = 0;
    b3d_ctx *owner = nullptr;
    cudaStream_t s_work = nullptr, s_setup = nullptr;

    std::mutex mu;
    std::condition_variable cv_work, cv_comp, cv_done, cv_state;
    std::map<int32_t, std::unique_ptr<Session>> sessions;
    int32_t next_sid = 0;
    int64_t next_ticket = 1;
    std::unordered_map<int64_t, int32_t> pending;  // ticket -> session, not yet completed
    std::unordered_map<int64_t, Done> done;
    std::deque<int64_t> done_order;
    std::deque<Batch> inflight;
    std::vector<cudaEvent_t> ev_pool;
    int32_t rr = 0;
    bool paused = false, stop = false, failed = false;
    std::string fail_msg;
    b3d_server_stats stats{};
    std::mutex admit_mu;  // one session build at a time (admission accounting)
    std::thread worker, completer;
};

namespace {

// Record the result of frame f (lock held). status B3D_OK reads the frame's results from
// its queue slot; any other status completes it without results.
void finish_frame(b3d_server *S, const Frame &f, b3d_status status, Clock::time_point t_done, int batch_frames,
                  bool ran) {
    auto it = S->sessions.find(f.sid);
    Session *x = it == S->sessions.end() ? nullptr : it->second.get();
    Done d;
    memset(&d.res, 0, sizeof d.res);
    d.res.ticket = f.ticket;
    d.res.session = f.sid;
    d.res.frame_index = f.index;
    d.res.latency_ms = ms_between(f.t_submit, t_done);
    d.res.queue_ms = ran ? ms_between(f.t_submit, f.t_issue) : d.res.latency_ms;
    d.res.batch_frames = batch_frames;
    if (x) {
        d.res.n_track = x->n_track;
        if (status == B3D_OK) {
            if (x->h_err[f.ring] != 0) status = B3D_EDEVICE;
            const float *r = x->h_res + (size_t)f.ring * x->n_track * 16;
            d.poses.assign(r, r + (size_t)x->n_track * 16);
        }
        x->ring_free.push_back(f.ring);
        if (ran) --x->running;
    }
    d.res.status = status;
    if (status == B3D_OK) ++S->stats.frames_done;
    else ++S->stats.frames_failed;
    S->pending.erase(f.ticket);
    S->done.emplace(f.ticket, std::move(d));
    S->done_order.push_back(f.ticket);
}

// Cancel a session's queued frames (lock held).
void cancel_queued(b3d_server *S, Session *x, b3d_status status) {
    const auto now = Clock::now();
    while (!x->queue.empty()) {
        const Frame f = x->queue.front();
        x->queue.pop_front();
        finish_frame(S, f, status, now, 0, false);
    }
}

// Queue this batch's device work on the server's stream (no lock held).
b3d_status issue_batch(b3d_server *S, const std::vector<Frame> &frames, const std::vector<Session *> &sess,
                       std::string *msg) {
    cudaStream_t s = S->s_work;
    std::vector<b3d_c2f_item> items;
    b3d_status st;
    for (size_t i = 0; i < frames.size(); ++i) {
        Session *x = sess[i];
        const Frame &f = frames[i];
        cudaError_t e = cudaMemcpyAsync(x->d_depth, x->h_ring + (size_t)f.ring * x->npx, sizeof(float) * x->npx,
                                        cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) { *msg = std::string("depth upload: ") + cudaGetErrorString(e); return B3D_ECUDA; }
        if ((st = b3d_set_observation(x->ctx, x->d_depth, s)) != B3D_OK) {
            *msg = std::string("set_observation: ") + b3d_last_error(x->ctx);
            return st;
        }
        if ((st = ctx_build_slot_bgs(x->ctx, x->n_track, s)) != B3D_OK) {
            *msg = std::string("backgrounds: ") + b3d_last_error(x->ctx);
            return st;
        }
        float *poses = ctx_scene_poses(x->ctx);
        for (int32_t k = 0; k < x->n_track; ++k) {
            b3d_c2f_item it;
            memset(&it, 0, sizeof it);
            it.scene = x->ctx;
            it.obj_slot = k;
            it.centre_dev = poses + 16 * k;
            it.schedule = S->cfg.schedule;
            it.schedule.seed = b3d_frame_seed(x->seed, f.index, k);
            memcpy(it.schedule.grid_frame, x->grid_frame, sizeof x->grid_frame);
            it.particles_dev = x->d_part + (size_t)k * x->M * 16;
            it.logw_dev = x->d_logw + (size_t)k * x->M;
            it.logq_dev = x->d_logq + (size_t)k * x->M;
            it.map_dev = x->d_map + 16 * k;
            items.push_back(it);
        }
    }
    if ((st = b3d_enumerate_multi(S->owner, (int32_t)items.size(), items.data(), &S->cfg.lik, s)) != B3D_OK) {
        *msg = std::string("enumerate_multi: ") + b3d_last_error(S->owner);
        return st;
    }
    for (size_t i = 0; i < frames.size(); ++i) {
        Session *x = sess[i];
        const Frame &f = frames[i];
        const size_t pb = sizeof(float) * 16 * x->n_track;
        cudaError_t e = cudaMemcpyAsync(ctx_scene_poses(x->ctx), x->d_map, pb, cudaMemcpyDeviceToDevice, s);
        ctx_tracked_moved(x->ctx, x->n_track);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(x->h_res + (size_t)f.ring * x->n_track * 16, x->d_map, pb, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(x->h_err + f.ring, ctx_err_flag(x->ctx), sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctx_err_flag(x->ctx), 0, sizeof(int), s);
        if (e != cudaSuccess) { *msg = std::string("result copies: ") + cudaGetErrorString(e); return B3D_ECUDA; }
    }
    return B3D_OK;
}

// Every session that can take a frame has one queued (no reason to wait for more).
bool all_queued(b3d_server *S) {
    for (auto &kv : S->sessions) {
        const Session *x = kv.second.get();
        if (x->queue.empty() && !x->held && !x->closing) return false;
    }
    return true;
}

bool worker_ready(b3d_server *S) {
    if (S->stop) return true;
    if (S->paused || S->failed || (int)S->inflight.size() >= S->cfg.max_inflight) return false;
    for (auto &kv : S->sessions) {
        const Session *x = kv.second.get();
        if (!x->queue.empty() && !x->held && !x->closing) return true;
    }
    return false;
}

void worker_loop(b3d_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_work.wait_for(lk, std::chrono::milliseconds(50), [S] { return worker_ready(S); });
        if (S->stop) break;
        if (!worker_ready(S)) continue;
        if (!S->inflight.empty() && S->cfg.batch_linger_us > 0) {
            // the device is busy: let frames that are about to arrive join this batch
            const auto until = Clock::now() + std::chrono::microseconds(S->cfg.batch_linger_us);
            S->cv_work.wait_until(lk, until, [S] { return S->stop || S->paused || all_queued(S); });
            if (S->stop) break;
            if (!worker_ready(S)) continue;
        }
        // the oldest queued frame of each ready session, round-robin from S->rr
        std::vector<Frame> frames;
        std::vector<Session *> sess;
        int items = 0;
        int32_t last = -1;
        auto it = S->sessions.lower_bound(S->rr);
        for (size_t v = 0; v < S->sessions.size(); ++v, ++it) {
            if (it == S->sessions.end()) it = S->sessions.begin();
            Session *x = it->second.get();
            if (x->queue.empty() || x->held || x->closing) continue;
            if (items + x->n_track > S->cfg.max_batch_items) continue;
            if (S->cfg.max_batch_frames > 0 && (int32_t)frames.size() >= S->cfg.max_batch_frames) break;
            Frame f = x->queue.front();
            x->queue.pop_front();
            f.t_issue = Clock::now();
            ++x->running;
            items += x->n_track;
            frames.push_back(f);
            sess.push_back(x);
            last = x->id;
        }
        S->rr = last + 1;
        S->stats.max_batch_frames_seen = std::max<int32_t>(S->stats.max_batch_frames_seen, (int32_t)frames.size());
        cudaEvent_t ev = nullptr;
        if (!S->ev_pool.empty()) {
            ev = S->ev_pool.back();
            S->ev_pool.pop_back();
        }
        lk.unlock();
        Batch b;
        b.frames = frames;
        b.hyps = (int64_t)items * S->hyp_per_item;
        b.status = issue_batch(S, frames, sess, &b.msg);
        // the event also covers a batch that failed part-way, so its queue slots are
        // released only after the copies already queued have run
        if (!ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) ev = nullptr;
        if (!ev || cudaEventRecord(ev, S->s_work) != cudaSuccess) {
            cudaGetLastError();
            cudaStreamSynchronize(S->s_work);
            if (ev) cudaEventDestroy(ev);
            ev = nullptr;
        }
        b.ev = ev;
        lk.lock();
        S->inflight.push_back(std::move(b));
        S->cv_comp.notify_one();
    }
}

void completion_loop(b3d_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        S->cv_comp.wait_for(lk, std::chrono::milliseconds(50), [S] { return !S->inflight.empty() || S->stop; });
        if (S->inflight.empty()) {
            if (S->stop) break;
            continue;
        }
        cudaEvent_t ev = S->inflight.front().ev;
        const bool failed_before = S->failed;
        const double limit = S->cfg.device_timeout_ms;
        lk.unlock();
        b3d_status wst = B3D_OK;
        std::string wmsg;
        if (ev) {
            const auto t0 = Clock::now();
            for (;;) {
                const cudaError_t e = cudaEventQuery(ev);
                if (e == cudaSuccess) break;
                if (e != cudaErrorNotReady) {
                    wst = B3D_ECUDA;
                    wmsg = std::string("batch failed on the device: ") + cudaGetErrorString(e);
                    break;
                }
                if (failed_before || ms_between(t0, Clock::now()) > limit) {
                    wst = B3D_ETIMEOUT;
                    wmsg = "a batch did not finish within the device timeout";
                    break;
                }
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
        }
        const auto t_done = Clock::now();
        lk.lock();
        Batch b = std::move(S->inflight.front());
        S->inflight.pop_front();
        b3d_status fst = b.status != B3D_OK ? b.status : wst;
        if (b.status != B3D_OK) S->fail_msg = b.msg;
        if (wst != B3D_OK) {
            // the device did not finish this batch: stop serving; queue slots the device may
            // still read are never handed out again
            S->failed = true;
            S->fail_msg = wmsg;
            for (auto &kv : S->sessions) cancel_queued(S, kv.second.get(), B3D_ETIMEOUT);
        } else if (ev) {
            S->ev_pool.push_back(ev);
        }
        for (const Frame &f : b.frames) finish_frame(S, f, fst, t_done, (int)b.frames.size(), true);
        if (fst == B3D_OK) {
            ++S->stats.batches;
            S->stats.hypotheses += b.hyps;
        }
        S->cv_work.notify_one();
        S->cv_done.notify_all();
        S->cv_state.notify_all();
    }
}

b3d_status validate_config(const b3d_server_config *c) {
    if (!c) return srv_fail(B3D_EINVAL, "config is NULL");
    if (c->max_sessions < 1) return srv_fail(B3D_EINVAL, "max_sessions must be >= 1");
    if (c->max_batch_items < 1) return srv_fail(B3D_EINVAL, "max_batch_items must be >= 1");
    if (c->max_batch_frames < 0) return srv_fail(B3D_EINVAL, "max_batch_frames must be >= 0");
    if (c->max_inflight < 1 || c->max_inflight > 2) return srv_fail(B3D_EINVAL, "max_inflight must be 1 or 2");
    if (c->queue_depth < 1 || c->queue_depth > 64) return srv_fail(B3D_EINVAL, "queue_depth must be in [1, 64]");
    if (c->device_timeout_ms < 0) return srv_fail(B3D_EINVAL, "device_timeout_ms must be >= 0");
    if (c->batch_linger_us < 0 || c->batch_linger_us > 1000000)
        return srv_fail(B3D_EINVAL, "batch_linger_us must be in [0, 1000000]");
    const b3d_c2f_schedule &sch = c->schedule;
    if (sch.n_stages < 1 || sch.n_stages > B3D_MAX_STAGES) return srv_fail(B3D_EINVAL, "schedule.n_stages must be in [1, 8]");
    if (sch.n_particles < 1 || sch.n_particles > (1 << 20)) return srv_fail(B3D_EINVAL, "schedule.n_particles out of range");
    for (int t = 0; t < sch.n_stages; ++t) {
        const b3d_stage &g = sch.stage[t];
        if (g.n_per_axis < 1 || g.n_per_axis > 1024 || g.n_rot < 1)
            return srv_fail(B3D_EINVAL, "schedule stage " + std::to_string(t) + " is empty");
    }
    return B3D_OK;
}

b3d_status validate_desc(const b3d_server *S, const b3d_session_desc *d) {
    if (!d) return srv_fail(B3D_EINVAL, "desc is NULL");
    if (d->n_obj < 1 || d->n_track < 1 || d->n_track > d->n_obj)
        return srv_fail(B3D_EINVAL, "a session needs 1 <= n_track <= n_obj");
    if (d->n_track > S->cfg.max_batch_items)
        return srv_fail(B3D_EINVAL, "n_track exceeds the server's max_batch_items");
    if (!d->verts || !d->n_v || !d->faces || !d->n_f || !d->poses)
        return srv_fail(B3D_EINVAL, "verts, n_v, faces, n_f and poses must be non-NULL");
    for (int32_t k = 0; k < d->n_obj; ++k)
        if (!d->verts[k] || !d->faces[k]) return srv_fail(B3D_EINVAL, "object " + std::to_string(k) + " has no mesh");
    if (d->intr.width < 1 || d->intr.height < 1 || (int64_t)d->intr.width * d->intr.height > ((int64_t)1 << 26))
        return srv_fail(B3D_EINVAL, "image size must be >= 1x1 and at most 2^26 pixels");
    return B3D_OK;
}

// Build a session's context, scene, tracking state and queue slots, with its device
// memory limited to `cap` bytes (0: no limit).
b3d_status build_session(b3d_server *S, const b3d_session_desc *d, uint64_t cap, std::unique_ptr<Session> *out,
                         std::string *msg) {
    std::unique_ptr<Session> x(new Session());
    x->n_obj = d->n_obj;
    x->n_track = d->n_track;
    x->M = S->cfg.schedule.n_particles;
    x->npx = (int64_t)d->intr.width * d->intr.height;
    x->seed = d->seed;
    bool any = false;
    for (int i = 0; i < 9; ++i) any = any || d->grid_frame[i] != 0.f;
    memcpy(x->grid_frame, any ? d->grid_frame : S->cfg.schedule.grid_frame, sizeof x->grid_frame);
    b3d_ctx *ctx = nullptr;
    b3d_status st = b3d_create(&ctx, S->device, cap);
    if (st != B3D_OK) {
        *msg = b3d_last_error(nullptr);
        return st;
    }
    x->ctx = ctx;
    auto bail = [&](b3d_status s2, const std::string &m) {
        *msg = m;
        b3d_destroy(ctx);
        free_session_host(x.get());
        return s2;
    };
    cudaStream_t s = S->s_setup;
    std::vector<int32_t> mids((size_t)d->n_obj);
    for (int32_t k = 0; k < d->n_obj; ++k) {
        st = b3d_load_mesh(ctx, d->verts[k], d->n_v[k], d->faces[k], d->n_f[k], d->mesh_flags ? d->mesh_flags[k] : 0,
                           &mids[k]);
        if (st != B3D_OK) return bail(st, "object " + std::to_string(k) + ": " + b3d_last_error(ctx));
    }
    const size_t M = (size_t)x->M, nt = (size_t)x->n_track;
    void *p = nullptr;
    if ((st = ctx_alloc_bytes(ctx, sizeof(float) * x->npx, &p, "session depth frame")) != B3D_OK)
        return bail(st, b3d_last_error(ctx));
    x->d_depth = (float *)p;
    if ((st = ctx_alloc_bytes(ctx, sizeof(float) * nt * M * 16, &p, "session particles")) != B3D_OK)
        return bail(st, b3d_last_error(ctx));
    x->d_part = (float *)p;
    if ((st = ctx_alloc_bytes(ctx, sizeof(float) * nt * M, &p, "session particle scores")) != B3D_OK)
        return bail(st, b3d_last_error(ctx));
    x->d_logw = (float *)p;
    if ((st = ctx_alloc_bytes(ctx, sizeof(float) * nt * M, &p, "session proposal densities")) != B3D_OK)
        return bail(st, b3d_last_error(ctx));
    x->d_logq = (float *)p;
    if ((st = ctx_alloc_bytes(ctx, sizeof(float) * nt * 16, &p, "session estimates")) != B3D_OK)
        return bail(st, b3d_last_error(ctx));
    x->d_map = (float *)p;
    cudaMemsetAsync(x->d_depth, 0, sizeof(float) * x->npx, s);
    if ((st = b3d_set_scene(ctx, &d->intr, d->n_obj, mids.data(), d->poses, x->d_depth, s)) != B3D_OK)
        return bail(st, b3d_last_error(ctx));
    // tracking state before frame 0: every particle at the initial pose, scores 0
    std::vector<float> part(nt * M * 16);
    for (size_t k = 0; k < nt; ++k)
        for (size_t m = 0; m < M; ++m) memcpy(&part[(k * M + m) * 16], d->poses + 16 * k, 16 * sizeof(float));
    cudaMemcpyAsync(x->d_map, d->poses, sizeof(float) * nt * 16, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(x->d_part, part.data(), sizeof(float) * part.size(), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(x->d_logw, 0, sizeof(float) * nt * M, s);
    cudaMemsetAsync(x->d_logq, 0, sizeof(float) * nt * M, s);
    for (int32_t k = 0; k < d->n_track; ++k)
        if ((st = ctx_prepare_slot(ctx, k, &S->cfg.lik, &S->cfg.schedule, s)) != B3D_OK)
            return bail(st, "object " + std::to_string(k) + ": " + b3d_last_error(ctx));
    // one z-buffer per object: each frame re-renders the tracked objects once and the fixed
    // ones never, instead of every other object once per tracked slot
    if ((st = ctx_prepare_shared_bg(ctx, s)) != B3D_OK) return bail(st, b3d_last_error(ctx));
    if ((st = b3d_sync(ctx, s)) != B3D_OK) return bail(st, b3d_last_error(ctx));
    // everything the session's frames use is allocated now: freeze its budget there
    x->reserved = ctx_used_bytes(ctx);
    ctx_set_budget(ctx, x->reserved);
    const size_t Q = (size_t)S->cfg.queue_depth;
    if (cudaHostAlloc((void **)&x->h_ring, sizeof(float) * Q * x->npx, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void **)&x->h_res, sizeof(float) * Q * nt * 16, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void **)&x->h_err, sizeof(int) * Q, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return bail(B3D_ENOMEM, "pinned host allocation of the frame queue failed");
    }
    memset(x->h_err, 0, sizeof(int) * Q);
    for (int q = (int)Q - 1; q >= 0; --q) x->ring_free.push_back(q);
    *out = std::move(x);
    return B3D_OK;
}

Session *find_session(b3d_server *S, int32_t id) {
    auto it = S->sessions.find(id);
    return it == S->sessions.end() ? nullptr : it->second.get();
}

b3d_status take_result(b3d_server *S, int64_t ticket, b3d_frame_result *res, float *poses, int32_t cap) {
    auto it = S->done.find(ticket);
    const Done &d = it->second;
    if (poses && cap < (int32_t)d.poses.size())
        return srv_fail(B3D_EINVAL, "poses_capacity " + std::to_string(cap) + " < " + std::to_string(d.poses.size()));
    if (res) *res = d.res;
    if (poses && !d.poses.empty()) memcpy(poses, d.poses.data(), sizeof(float) * d.poses.size());
    S->done.erase(it);
    return srv_ok();
}

Clock::time_point deadline_of(int32_t timeout_ms) {
    return Clock::now() + std::chrono::milliseconds(std::max<int32_t>(0, timeout_ms));
}

}  // namespace

// ==========================================================================================
// C ABI
// ==========================================================================================
extern "C" {

uint64_t b3d_frame_seed(uint64_t seed, int64_t frame, int32_t obj) {
    return splitmix64(splitmix64(splitmix64(seed) ^ (uint64_t)frame) ^ (uint64_t)(uint32_t)obj);
}

const char *b3d_server_last_error(void) { return g_srv_error.c_str(); }

b3d_status b3d_server_create(b3d_server **out, int32_t device, uint64_t hbm_budget_bytes,
                             const b3d_server_config *cfg) {
    if (!out) return srv_fail(B3D_EINVAL, "out is NULL");
    *out = nullptr;
    b3d_status st = validate_config(cfg);
    if (st != B3D_OK) return st;
    std::unique_ptr<b3d_server> S(new (std::nothrow) b3d_server());
    if (!S) return srv_fail(B3D_ENOMEM, "host allocation failed");
    S->device = device;
    S->budget = hbm_budget_bytes;
    S->cfg = *cfg;
    if (S->cfg.device_timeout_ms == 0) S->cfg.device_timeout_ms = 60000;
    S->stats.hbm_budget = hbm_budget_bytes;
    for (int t = 0; t < cfg->schedule.n_stages; ++t) {
        const b3d_stage &g = cfg->schedule.stage[t];
        S->hyp_per_item += (int64_t)g.n_per_axis * g.n_per_axis * g.n_per_axis * g.n_rot;
    }
    if ((st = b3d_create(&S->owner, device, hbm_budget_bytes)) != B3D_OK)
        return srv_fail(st, b3d_last_error(nullptr));
    auto bail = [&](b3d_status s2, const std::string &m) {
        if (S->s_work) cudaStreamDestroy(S->s_work);
        if (S->s_setup) cudaStreamDestroy(S->s_setup);
        b3d_destroy(S->owner);
        return srv_fail(s2, m);
    };
    if (cfg->tuning.tile_w != 0 && (st = b3d_set_tuning(S->owner, &cfg->tuning)) != B3D_OK)
        return bail(st, std::string("tuning: ") + b3d_last_error(S->owner));
    // the batch scratch for max_batch_items items is reserved once, up front
    if ((st = owner_reserve(S->owner, cfg->max_batch_items, &cfg->schedule)) != B3D_OK)
        return bail(st, std::string("batch scratch: ") + b3d_last_error(S->owner));
    S->scratch = ctx_used_bytes(S->owner);
    ctx_set_budget(S->owner, S->scratch);
    S->reserved = S->scratch;
    S->stats.hbm_reserved = S->reserved;
    cudaSetDevice(device);
    if (cudaStreamCreateWithFlags(&S->s_work, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&S->s_setup, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return bail(B3D_ECUDA, "stream creation failed");
    }
    b3d_server *raw = S.get();
    raw->worker = std::thread(worker_loop, raw);
    raw->completer = std::thread(completion_loop, raw);
    *out = S.release();
    return srv_ok();
}

b3d_status b3d_server_destroy(b3d_server *S) {
    if (!S) return srv_fail(B3D_EINVAL, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        for (auto &kv : S->sessions) cancel_queued(S, kv.second.get(), B3D_ECLOSED);
        S->cv_work.notify_all();
        S->cv_comp.notify_all();
        S->cv_done.notify_all();
        S->cv_state.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    if (S->completer.joinable()) S->completer.join();
    const bool failed = S->failed;
    for (auto &kv : S->sessions) {
        Session *x = kv.second.get();
        if (failed) continue;  // the device may still read these; leave them
        b3d_destroy(x->ctx);
        free_session_host(x);
    }
    if (!failed) {
        for (cudaEvent_t e : S->ev_pool) cudaEventDestroy(e);
        cudaStreamDestroy(S->s_work);
        cudaStreamDestroy(S->s_setup);
        b3d_destroy(S->owner);
    }
    delete S;
    return srv_ok();
}

b3d_status b3d_session_open(b3d_server *S, const b3d_session_desc *desc, int32_t timeout_ms, int32_t *session_id) {
    if (!S || !session_id) return srv_fail(B3D_EINVAL, "server and session_id must be non-NULL");
    b3d_status st = validate_desc(S, desc);
    if (st != B3D_OK) return st;
    std::lock_guard<std::mutex> admit(S->admit_mu);
    const auto deadline = deadline_of(timeout_ms);
    for (;;) {
        uint64_t cap = 0;
        int64_t gen = 0;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop) return srv_fail(B3D_ECLOSED, "server is stopping");
            if (S->failed) return srv_fail(B3D_EDEVICE, "server failed: " + S->fail_msg);
            if (!S->cv_state.wait_until(lk, deadline, [S] {
                    return (int32_t)S->sessions.size() < S->cfg.max_sessions || S->stop;
                }))
                return srv_fail(B3D_EBUSY, "all " + std::to_string(S->cfg.max_sessions) + " session slots are in use");
            if (S->stop) return srv_fail(B3D_ECLOSED, "server is stopping");
            cap = S->budget == 0 ? 0 : (S->budget > S->reserved ? S->budget - S->reserved : 1);
            gen = (int64_t)S->reserved;
        }
        std::unique_ptr<Session> x;
        std::string msg;
        st = build_session(S, desc, cap, &x, &msg);
        if (st == B3D_OK) {
            std::lock_guard<std::mutex> lk(S->mu);
            const int32_t id = S->next_sid++;
            x->id = id;
            S->reserved += x->reserved;
            S->sessions[id] = std::move(x);
            S->stats.sessions = (int32_t)S->sessions.size();
            S->stats.hbm_reserved = S->reserved;
            *session_id = id;
            return srv_ok();
        }
        if (st != B3D_EBUDGET) return srv_fail(st, msg);
        // wait for a close to return memory, then try again
        std::unique_lock<std::mutex> lk(S->mu);
        if (!S->cv_state.wait_until(lk, deadline, [S, gen] { return (int64_t)S->reserved < gen || S->stop; }))
            return srv_fail(B3D_EBUDGET, "session does not fit in the HBM budget (" + std::to_string(S->reserved) +
                                             " of " + std::to_string(S->budget) + " bytes reserved): " + msg);
    }
}

b3d_status b3d_session_close(b3d_server *S, int32_t id) {
    if (!S) return srv_fail(B3D_EINVAL, "server is NULL");
    std::unique_ptr<Session> own;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        Session *x = find_session(S, id);
        if (!x) return srv_fail(B3D_ENOTFOUND, "no session " + std::to_string(id));
        x->closing = true;
        cancel_queued(S, x, B3D_ECLOSED);
        S->cv_done.notify_all();
        const auto deadline = Clock::now() + std::chrono::milliseconds(S->cfg.device_timeout_ms);
        if (!S->cv_state.wait_until(lk, deadline, [x] { return x->running == 0 && x->writers == 0 && !x->held; }))
            return srv_fail(B3D_ETIMEOUT, "session " + std::to_string(id) + " still has frames on the device");
        if (S->failed) return srv_fail(B3D_EDEVICE, "server failed: " + S->fail_msg);
        own = std::move(S->sessions[id]);
        S->sessions.erase(id);
    }
    b3d_destroy(own->ctx);
    free_session_host(own.get());
    std::lock_guard<std::mutex> lk(S->mu);
    S->reserved -= own->reserved;
    S->stats.sessions = (int32_t)S->sessions.size();
    S->stats.hbm_reserved = S->reserved;
    S->cv_state.notify_all();
    return srv_ok();
}

b3d_status b3d_frame_submit(b3d_server *S, int32_t id, const float *depth, int32_t timeout_ms, int64_t *ticket) {
    const auto t_submit = Clock::now();
    if (!S || !depth || !ticket) return srv_fail(B3D_EINVAL, "server, depth and ticket must be non-NULL");
    Session *x = nullptr;
    int ring = -1;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        x = find_session(S, id);
        if (!x) return srv_fail(B3D_ENOTFOUND, "no session " + std::to_string(id));
        if (S->failed) return srv_fail(B3D_EDEVICE, "server failed: " + S->fail_msg);
        const auto deadline = deadline_of(timeout_ms);
        if (!S->cv_state.wait_until(lk, deadline, [S, x] { return !x->ring_free.empty() || x->closing || S->stop || S->failed; }))
            return srv_fail(B3D_EBUSY, "session " + std::to_string(id) + " has queue_depth frames outstanding");
        if (x->closing || S->stop) return srv_fail(B3D_ECLOSED, "session is closing");
        if (S->failed) return srv_fail(B3D_EDEVICE, "server failed: " + S->fail_msg);
        ring = x->ring_free.back();
        x->ring_free.pop_back();
        ++x->writers;
    }
    memcpy(x->h_ring + (size_t)ring * x->npx, depth, sizeof(float) * x->npx);
    std::lock_guard<std::mutex> lk(S->mu);
    --x->writers;
    if (x->closing || S->stop) {
        x->ring_free.push_back(ring);
        S->cv_state.notify_all();
        return srv_fail(B3D_ECLOSED, "session is closing");
    }
    Frame f;
    f.ticket = S->next_ticket++;
    f.index = x->next_index++;
    f.sid = id;
    f.ring = ring;
    f.t_submit = t_submit;
    x->queue.push_back(f);
    S->pending[f.ticket] = id;
    *ticket = f.ticket;
    S->cv_work.notify_one();
    return srv_ok();
}

b3d_status b3d_frame_wait(b3d_server *S, int64_t ticket, int32_t timeout_ms, b3d_frame_result *res, float *poses,
                          int32_t poses_capacity) {
    if (!S) return srv_fail(B3D_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    if (!S->done.count(ticket) && !S->pending.count(ticket))
        return srv_fail(B3D_ENOTFOUND, "unknown or collected ticket " + std::to_string(ticket));
    const auto deadline = deadline_of(timeout_ms);
    if (!S->cv_done.wait_until(lk, deadline, [S, ticket] { return S->done.count(ticket) > 0; }))
        return srv_fail(B3D_ETIMEOUT, "frame " + std::to_string(ticket) + " not finished");
    return take_result(S, ticket, res, poses, poses_capacity);
}

b3d_status b3d_frame_next(b3d_server *S, int32_t timeout_ms, b3d_frame_result *res, float *poses,
                          int32_t poses_capacity) {
    if (!S) return srv_fail(B3D_EINVAL, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    auto first = [S]() -> int64_t {
        while (!S->done_order.empty()) {
            const int64_t t = S->done_order.front();
            if (S->done.count(t)) return t;
            S->done_order.pop_front();
        }
        return 0;
    };
    const auto deadline = deadline_of(timeout_ms);
    int64_t t = 0;
    if (!S->cv_done.wait_until(lk, deadline, [&] { return (t = first()) != 0; }))
        return srv_fail(B3D_ETIMEOUT, "no frame finished");
    return take_result(S, t, res, poses, poses_capacity);
}

b3d_status b3d_server_pause(b3d_server *S, int32_t paused) {
    if (!S) return srv_fail(B3D_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    S->paused = paused != 0;
    S->cv_work.notify_all();
    return srv_ok();
}

b3d_status b3d_server_get_stats(b3d_server *S, b3d_server_stats *out) {
    if (!S || !out) return srv_fail(B3D_EINVAL, "server and out must be non-NULL");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    uint64_t used = ctx_used_bytes(S->owner);
    for (auto &kv : S->sessions) used += ctx_used_bytes(kv.second->ctx);
    out->hbm_used = used;
    return srv_ok();
}

}  // extern "C"

namespace {

// Mark an idle session as held (no frame queued or running) for export / import.
b3d_status hold_idle(b3d_server *S, int32_t id, Session **out) {
    std::lock_guard<std::mutex> lk(S->mu);
    Session *x = find_session(S, id);
    if (!x) return srv_fail(B3D_ENOTFOUND, "no session " + std::to_string(id));
    if (S->failed) return srv_fail(B3D_EDEVICE, "server failed: " + S->fail_msg);
    if (x->closing || x->held || x->running || !x->queue.empty())
        return srv_fail(B3D_EBUSY, "session " + std::to_string(id) + " is not idle");
    x->held = true;
    *out = x;
    return B3D_OK;
}

void release_hold(b3d_server *S, Session *x) {
    std::lock_guard<std::mutex> lk(S->mu);
    x->held = false;
    S->cv_work.notify_one();
    S->cv_state.notify_all();
}

}  // namespace

extern "C" {

b3d_status b3d_session_export(b3d_server *S, int32_t id, float *poses, float *particles, float *logw,
                              int64_t *next_frame) {
    if (!S) return srv_fail(B3D_EINVAL, "server is NULL");
    Session *x = nullptr;
    b3d_status st = hold_idle(S, id, &x);
    if (st != B3D_OK) return st;
    cudaSetDevice(S->device);
    const size_t nt = (size_t)x->n_track, M = (size_t)x->M;
    cudaError_t e = cudaSuccess;
    if (poses) e = cudaMemcpy(poses, x->d_map, sizeof(float) * nt * 16, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && particles)
        e = cudaMemcpy(particles, x->d_part, sizeof(float) * nt * M * 16, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && logw) e = cudaMemcpy(logw, x->d_logw, sizeof(float) * nt * M, cudaMemcpyDeviceToHost);
    if (next_frame) *next_frame = x->next_index;
    release_hold(S, x);
    if (e != cudaSuccess) return srv_fail(B3D_ECUDA, std::string("export: ") + cudaGetErrorString(e));
    return srv_ok();
}

b3d_status b3d_session_import(b3d_server *S, int32_t id, const float *poses, const float *particles,
                              const float *logw, int64_t next_frame) {
    if (!S || !poses) return srv_fail(B3D_EINVAL, "server and poses must be non-NULL");
    if (next_frame < 0) return srv_fail(B3D_EINVAL, "next_frame must be >= 0");
    Session *x = nullptr;
    b3d_status st = hold_idle(S, id, &x);
    if (st != B3D_OK) return st;
    cudaSetDevice(S->device);
    const size_t nt = (size_t)x->n_track, M = (size_t)x->M;
    cudaError_t e = cudaMemcpy(x->d_map, poses, sizeof(float) * nt * 16, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(ctx_scene_poses(x->ctx), poses, sizeof(float) * nt * 16, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && particles)
        e = cudaMemcpy(x->d_part, particles, sizeof(float) * nt * M * 16, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && logw) e = cudaMemcpy(x->d_logw, logw, sizeof(float) * nt * M, cudaMemcpyHostToDevice);
    ctx_tracked_moved(x->ctx, x->n_track);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        x->next_index = next_frame;
    }
    release_hold(S, x);
    if (e != cudaSuccess) return srv_fail(B3D_ECUDA, std::string("import: ") + cudaGetErrorString(e));
    return srv_ok();
}

}  // extern "C"
