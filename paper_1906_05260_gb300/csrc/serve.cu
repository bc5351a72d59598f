// serve.cu -- frame-step serving runtime for many independent VIPER scenes.
//
// A server owns device-resident scenes admitted against a device-memory budget.
// Clients submit frame-step requests (bone poses + dt/substeps/iterations)
// for any scene at any time.  A dispatcher thread runs the multi-scene frame
// step (batch.cu): whenever fewer than two steps are in flight it takes the
// oldest waiting request of every scene without a frame in flight (those
// with the oldest request's schedule) and advances all of them with one
// launch sequence on the server's stream; requests that arrive meanwhile
// join the next step (continuous batching at frame granularity).  Completion
// is stamped by a host callback enqueued behind the step; latency is
// completion minus submission.
//
// Locking: server state is guarded by one mutex which is never held across a
// CUDA call that can wait for the GPU (host callbacks take the same mutex).
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "viper_impl.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    long long ticket = 0;
    float dt = 0;
    int substeps = 0, iterations = 0;
    std::vector<float> bq, bt;
    double t_submit = 0, t_done = 0;
};

struct Slot {
    int id = 0;
    viper_scene *sc = nullptr;
    size_t bytes = 0;
    int n_bones = 0;
    double units_per_substep = 0;  // rod vertices
    std::deque<Req *> queue;
    Req *inflight = nullptr;
    bool releasing = false;
    float4 *mesh = nullptr;  // rest, idx (int4 bits), weights, out: 4 n float4
    int n_mesh = 0;
};

struct Done {
    int status;
    double latency_ms;
};

}  // namespace

struct viper_server {
    size_t budget = 0, used = 0;
    int max_inflight = 1, inflight = 0;
    int steps_inflight = 0;
    long long steps = 0;
    viper_batch *batch = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::unordered_map<int, Slot *> slots;
    std::unordered_map<long long, Done> done;
    std::thread worker;
    bool stop = false;
    long long next_ticket = 1;
    int next_id = 1;
    std::vector<double> lat;
    long long frames = 0, failed = 0;
    double units = 0;
    Clock::time_point t0 = Clock::now();
};

namespace {

double ms_since(const viper_server *S) { return std::chrono::duration<double, std::milli>(Clock::now() - S->t0).count(); }

// Called with S->mu held.
void complete(viper_server *S, Slot *sl, Req *r, int status)
{
    r->t_done = ms_since(S);
    const double lat = r->t_done - r->t_submit;
    S->done[r->ticket] = Done{status, lat};
    if (status == VIPER_OK || status == VIPER_EOVERFLOW) {
        S->lat.push_back(lat);
        S->frames++;
        S->units += sl->units_per_substep * r->substeps;
    } else {
        S->failed++;
    }
    sl->inflight = nullptr;
    S->inflight--;
    delete r;
    S->cv_done.notify_all();
    S->cv_work.notify_one();
}

// Frames advanced by one multi-scene step, completed by its host callback.
struct StepCtx {
    viper_server *S;
    std::vector<std::pair<Slot *, Req *>> frames;
    std::vector<int> status;  // latched errors known when the step was queued
};

void CUDART_CB step_done(void *p)
{
    StepCtx *c = static_cast<StepCtx *>(p);
    {
        std::lock_guard<std::mutex> lk(c->S->mu);
        for (size_t i = 0; i < c->frames.size(); ++i) {
            Slot *sl = c->frames[i].first;
            int st = c->status[i];
            // the step mirrored the scene's error word to the host
            if (st == VIPER_OK) st = viper::scene_decode_err(*(volatile int *)sl->sc->h_err);
            complete(c->S, sl, c->frames[i].second, st);
        }
        c->S->steps_inflight--;
    }
    delete c;
}

// Queue one multi-scene step (no lock held).
void dispatch(viper_server *S, std::vector<std::pair<Slot *, Req *>> &todo)
{
    const int n = (int)todo.size();
    std::vector<viper_batch_item> items(n);
    for (int i = 0; i < n; ++i) {
        Slot *sl = todo[i].first;
        Req *r = todo[i].second;
        viper_batch_item &it = items[i];
        memset(&it, 0, sizeof(it));
        it.scene = sl->sc;
        if (sl->n_bones > 0) {
            it.bone_quat = r->bq.data();
            it.bone_trans = r->bt.data();
        }
        if (sl->n_mesh > 0) {
            const int m = sl->n_mesh;
            it.n_mesh = m;
            it.rest4 = (const float *)sl->mesh;
            it.idx4 = (const int *)(sl->mesh + m);
            it.w4 = (const float *)(sl->mesh + 2 * m);
            it.out4 = (float *)(sl->mesh + 3 * m);
        }
    }
    const Req *r0 = todo[0].second;
    StepCtx *c = new StepCtx{S, todo, std::vector<int>(n, VIPER_OK)};
    int rc = viper_batch_step(S->batch, items.data(), n, r0->dt, r0->substeps, r0->iterations, c->status.data());
    if (rc == VIPER_OK && cudaLaunchHostFunc((cudaStream_t)viper_batch_stream(S->batch), step_done, c) == cudaSuccess)
        return;
    if (rc == VIPER_OK) rc = VIPER_ECUDA;
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto &t : todo) complete(S, t.first, t.second, rc);
    S->steps_inflight--;
    delete c;
}

constexpr int kMaxSteps = 2;  // multi-scene steps in flight

void run(viper_server *S)
{
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        std::vector<Slot *> ready;
        if (S->steps_inflight < kMaxSteps)
            for (auto &kv : S->slots) {
                Slot *sl = kv.second;
                if (!sl->inflight && !sl->queue.empty()) ready.push_back(sl);
            }
        // oldest waiting request first; one step takes the requests sharing its schedule
        std::sort(ready.begin(), ready.end(), [](Slot *a, Slot *b) {
            return a->queue.front()->t_submit < b->queue.front()->t_submit;
        });
        std::vector<std::pair<Slot *, Req *>> todo;
        for (Slot *sl : ready) {
            if (S->inflight >= S->max_inflight) break;
            Req *r = sl->queue.front();
            if (!todo.empty()) {
                const Req *r0 = todo[0].second;
                if (r->dt != r0->dt || r->substeps != r0->substeps || r->iterations != r0->iterations) continue;
            }
            sl->queue.pop_front();
            sl->inflight = r;
            S->inflight++;
            todo.emplace_back(sl, r);
        }
        if (todo.empty()) {
            if (S->stop && S->steps_inflight == 0) return;
            S->cv_work.wait(lk);
            continue;
        }
        S->steps_inflight++;
        S->steps++;
        lk.unlock();
        dispatch(S, todo);
        lk.lock();
    }
}

void free_slot(Slot *sl)
{
    if (sl->sc) viper_scene_destroy(sl->sc);
    if (sl->mesh) cudaFree(sl->mesh);
    delete sl;
}

}  // namespace

extern "C" {

int viper_server_create(size_t budget_bytes, int max_inflight, viper_server **out)
{
    if (!out || max_inflight < 1 || budget_bytes == 0) return VIPER_EINVAL;
    viper_server *S = new viper_server();
    S->budget = budget_bytes;
    S->max_inflight = max_inflight;
    int rc = viper_batch_create(nullptr, &S->batch);
    if (rc != VIPER_OK) {
        delete S;
        return rc;
    }
    S->worker = std::thread(run, S);
    *out = S;
    return VIPER_OK;
}

void viper_server_destroy(viper_server *S)
{
    if (!S) return;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        for (auto &kv : S->slots) {
            for (Req *r : kv.second->queue) delete r;
            kv.second->queue.clear();
        }
        S->stop = true;
        S->cv_work.notify_all();
        S->cv_done.wait(lk, [&] { return S->inflight == 0 && S->steps_inflight == 0; });
    }
    S->worker.join();
    for (auto &kv : S->slots) free_slot(kv.second);
    viper_batch_destroy(S->batch);
    delete S;
}

int viper_server_admit(viper_server *S, const viper_scene_desc *desc, int n_mesh, const float *rest4,
                       const int *idx4, const float *w4, int solver_mode, float dt, int substeps,
                       int iterations, int *scene_id)
{
    if (!S || !desc || !scene_id || n_mesh < 0 || (n_mesh > 0 && (!rest4 || !idx4 || !w4))) return VIPER_EINVAL;
    size_t fp = viper_scene_footprint(desc);
    if (fp == 0) return VIPER_EINVAL;
    const size_t bytes = fp + 64 * (size_t)n_mesh + 4096;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->used + bytes > S->budget) return VIPER_EBUDGET;
        S->used += bytes;  // reserved while the scene is built
    }
    Slot *sl = new Slot();
    viper_scene_desc d = *desc;
    d.stream = viper_batch_stream(S->batch);  // scenes live on the server's stream
    int rc = viper_scene_create(&d, &sl->sc);
    if (rc == VIPER_OK && (solver_mode == VIPER_SOLVER_PLAIN || solver_mode == VIPER_SOLVER_FRAME)) {
        rc = viper_set_solver(sl->sc, solver_mode, 4, 256);
        if (rc != VIPER_OK && solver_mode == VIPER_SOLVER_FRAME) rc = VIPER_OK;  // not co-resident: batched
    }
    // scenes the multi-scene kernels cannot take run on their own: build their graph now
    if (rc == VIPER_OK && sl->sc->resident_nv != sl->sc->nv && dt > 0 && substeps > 0 && iterations >= 0)
        rc = viper_prepare(sl->sc, dt, substeps, iterations);
    if (rc == VIPER_OK && n_mesh > 0) {
        const size_t nb = sizeof(float4) * (size_t)n_mesh;
        if (cudaMalloc((void **)&sl->mesh, 4 * nb) != cudaSuccess) {
            cudaGetLastError();
            rc = VIPER_ENOMEM;
        } else if (cudaMemcpy(sl->mesh, rest4, nb, cudaMemcpyDefault) != cudaSuccess ||
                   cudaMemcpy(sl->mesh + n_mesh, idx4, nb, cudaMemcpyDefault) != cudaSuccess ||
                   cudaMemcpy(sl->mesh + 2 * n_mesh, w4, nb, cudaMemcpyDefault) != cudaSuccess) {
            rc = VIPER_ECUDA;
        }
        sl->n_mesh = n_mesh;
    }
    sl->n_bones = desc->n_bones;
    if (rc != VIPER_OK) {
        free_slot(sl);
        std::lock_guard<std::mutex> lk(S->mu);
        S->used -= bytes;
        return rc;
    }
    int nr = 0, nv = 0, ns = 0;
    viper_scene_counts(sl->sc, &nr, &nv, &ns);
    sl->units_per_substep = nv;
    sl->bytes = bytes;
    std::lock_guard<std::mutex> lk(S->mu);
    sl->id = S->next_id++;
    S->slots[sl->id] = sl;
    *scene_id = sl->id;
    return VIPER_OK;
}

int viper_server_submit(viper_server *S, int scene_id, const float *bone_quat, const float *bone_trans, float dt,
                        int substeps, int iterations, long long *ticket)
{
    if (!S || !ticket || !(dt > 0) || substeps <= 0 || iterations < 0) return VIPER_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->slots.find(scene_id);
    if (it == S->slots.end() || it->second->releasing) return VIPER_EINVAL;
    Slot *sl = it->second;
    if (sl->n_bones > 0 && (!bone_quat || !bone_trans)) return VIPER_EINVAL;
    Req *r = new Req();
    r->ticket = S->next_ticket++;
    r->dt = dt;
    r->substeps = substeps;
    r->iterations = iterations;
    if (sl->n_bones > 0) {
        r->bq.assign(bone_quat, bone_quat + 4 * sl->n_bones);
        r->bt.assign(bone_trans, bone_trans + 3 * sl->n_bones);
    }
    r->t_submit = ms_since(S);
    sl->queue.push_back(r);
    *ticket = r->ticket;
    S->cv_work.notify_one();
    return VIPER_OK;
}

int viper_server_wait(viper_server *S, long long ticket, double timeout_ms, int *status, double *latency_ms)
{
    if (!S) return VIPER_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto pred = [&] { return S->done.count(ticket) > 0; };
    if (!S->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), pred))
        return VIPER_ETIMEOUT;
    Done d = S->done[ticket];
    S->done.erase(ticket);
    if (status) *status = d.status;
    if (latency_ms) *latency_ms = d.latency_ms;
    return VIPER_OK;
}

int viper_server_release(viper_server *S, int scene_id)
{
    if (!S) return VIPER_EINVAL;
    Slot *sl = nullptr;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->slots.find(scene_id);
        if (it == S->slots.end()) return VIPER_EINVAL;
        sl = it->second;
        sl->releasing = true;
        S->cv_done.wait(lk, [&] { return sl->inflight == nullptr && sl->queue.empty(); });
        S->slots.erase(scene_id);
        S->used -= sl->bytes;
    }
    free_slot(sl);
    return VIPER_OK;
}

viper_scene *viper_server_scene(viper_server *S, int scene_id)
{
    if (!S) return nullptr;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->slots.find(scene_id);
    return it == S->slots.end() ? nullptr : it->second->sc;
}

int viper_server_mesh_out(viper_server *S, int scene_id, float *out4)
{
    if (!S || !out4) return VIPER_EINVAL;
    Slot *sl = nullptr;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        auto it = S->slots.find(scene_id);
        if (it == S->slots.end() || it->second->n_mesh == 0) return VIPER_EINVAL;
        sl = it->second;
        S->cv_done.wait(lk, [&] { return sl->inflight == nullptr && sl->queue.empty(); });
    }
    const size_t nb = sizeof(float4) * (size_t)sl->n_mesh;
    if (cudaStreamSynchronize(sl->sc->stream) != cudaSuccess) return VIPER_ECUDA;
    if (cudaMemcpy(out4, sl->mesh + 3 * sl->n_mesh, nb, cudaMemcpyDefault) != cudaSuccess) return VIPER_ECUDA;
    return VIPER_OK;
}

int viper_server_idle(viper_server *S, double timeout_ms)
{
    if (!S) return VIPER_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto pred = [&] {
        if (S->inflight) return false;
        for (auto &kv : S->slots)
            if (!kv.second->queue.empty()) return false;
        return true;
    };
    if (!S->cv_done.wait_for(lk, std::chrono::duration<double, std::milli>(timeout_ms), pred)) return VIPER_ETIMEOUT;
    return VIPER_OK;
}

int viper_server_get_stats(viper_server *S, viper_server_stats *st)
{
    if (!S || !st) return VIPER_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    memset(st, 0, sizeof(*st));
    st->frames = S->frames;
    st->failed = S->failed;
    st->rod_vertex_substeps = S->units;
    st->scenes = (int)S->slots.size();
    st->inflight = S->inflight;
    st->used_bytes = S->used;
    int q = 0;
    for (auto &kv : S->slots) q += (int)kv.second->queue.size();
    st->queued = q;
    st->steps = S->steps;
    if (!S->lat.empty()) {
        std::vector<double> v = S->lat;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            double k = p * (v.size() - 1);
            size_t i = (size_t)k;
            double f = k - i;
            return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
        };
        st->p50_ms = pct(0.50);
        st->p99_ms = pct(0.99);
        st->max_ms = v.back();
        double s = 0;
        for (double x : v) s += x;
        st->mean_ms = s / v.size();
    }
    return VIPER_OK;
}

int viper_server_reset_stats(viper_server *S)
{
    if (!S) return VIPER_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    S->lat.clear();
    S->frames = S->failed = 0;
    S->steps = 0;
    S->units = 0;
    return VIPER_OK;
}

}  // extern "C"
