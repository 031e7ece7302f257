// Continuous-batching request loop (ds_submit / ds_poll / ds_wait).
//
// ds_submit validates a request and queues it without waiting on the GPU.  A displacive request
// with an automatic Taylor order first needs x_max (Section III C): its reduction and the
// read-back into a pinned slot are queued on the context's planning stream, and a host callback
// marks the request planned.  One worker thread per context admits planned requests while the
// footprint of the requests in flight plus the candidate fits the context's budget: the queue is
// scanned from the oldest request, a request that does not fit is passed over by later ones at
// most kMaxBypass times (then everything waits for it), so nothing starves.  An admitted request
// runs on the least busy of the context's compute streams; requests whose cost (HBM footprint
// plus output) is at most the median of the recently admitted ones take the high-priority
// streams, so that small requests are not slowed by large ones sharing the GPU.  Completion is
// reported by a host callback queued behind the request's kernels (cudaLaunchHostFunc), which
// returns the footprint to the budget, timestamps the latency and wakes the worker and any
// waiter.  Every voxel of a request is computed by the same kernels with the same reduction order
// as an isolated request, so results do not depend on the mix.
//
// Host waits are bounded (ds_wait takes a timeout); no kernel of the path waits on another.
#include <algorithm>
#include <chrono>
#include <cstring>

#include "api_internal.h"

using namespace ds;

namespace {

constexpr int kServeStreams = 8;   // half of them at the highest stream priority
constexpr int kMaxBypass = 8;      // later requests admitted ahead of a waiting one, at most
constexpr int kPlanSlots = 1024;   // displacive requests planned concurrently
constexpr int kCostWindow = 64;    // admitted jobs in the median of the priority split

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

struct ServeJob {
    uint64_t ticket = 0;
    ds_ctx *ctx = nullptr;
    ds_model *model = nullptr;
    ds_qgrid q;
    ds_opts o;
    void *out = nullptr;
    size_t footprint = 0;
    double cost = 0.0;
    double xmax = -1.0;
    bool has_hint = false;
    TaylorHint hint;
    bool planned = false;       // Taylor order known (or not needed)
    int plan_slot = -1;         // pinned read-back slot while planning
    ds_status plan_status = DS_OK;
    int bypassed = 0;
    int stream_idx = -1;
    cudaStream_t stream = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double t_submit = 0.0, t_done = 0.0;
    bool done = false;
    ds_status status = DS_OK;
    ds_result_info info;
};

static void CUDART_CB job_done(void *arg) {
    ServeJob *j = (ServeJob *)arg;
    ds_ctx *ctx = j->ctx;
    std::lock_guard<std::mutex> g(ctx->mu);
    j->t_done = now_s();
    j->done = true;
    ctx->inflight_bytes -= j->footprint;
    if (j->stream_idx >= 0) ctx->stream_jobs[j->stream_idx]--;
    ctx->cv.notify_all();
}

// x_max of a displacive request has reached its pinned slot: order, footprint, cost
static void CUDART_CB job_planned(void *arg) {
    ServeJob *j = (ServeJob *)arg;
    ds_ctx *ctx = j->ctx;
    std::lock_guard<std::mutex> g(ctx->mu);
    const double *hx = ctx->plan_host + 16 * j->plan_slot;
    int P = 0;
    double umax = 0.0;
    // taylor_order_from_corners only formats a message on failure (no CUDA call)
    j->plan_status = taylor_order_from_corners(ctx, &j->o, hx, &P, &j->xmax, &umax);
    j->hint.P = P;
    j->hint.xmax = j->xmax;
    j->hint.umax = umax;
    j->has_hint = true;
    j->footprint = request_footprint(j->model, &j->q, &j->o, P);
    j->cost = (double)j->footprint;
    ctx->plan_free.push_back(j->plan_slot);
    j->plan_slot = -1;
    j->planned = true;
    ctx->cv.notify_all();
}

static void finish_failed(ServeJob *j, ds_status rc) {
    ds_ctx *ctx = j->ctx;
    std::lock_guard<std::mutex> g(ctx->mu);
    j->status = rc;
    j->t_done = now_s();
    j->done = true;
    ctx->inflight_bytes -= j->footprint;
    if (j->stream_idx >= 0) ctx->stream_jobs[j->stream_idx]--;
    ctx->cv.notify_all();
}

static void launch_job(ServeJob *j) {
    ds_model *M = j->model;
    Scratch ws(j->stream);
    cudaEventRecord(j->e0, j->stream);
    ds_status rc;
    const TaylorHint *h = j->has_hint ? &j->hint : nullptr;
    if (j->o.precision == DS_FP64)
        rc = enqueue_request<double>(M, &j->q, &j->o, (double *)j->out, j->stream, ws, &j->info, h);
    else
        rc = enqueue_request<float>(M, &j->q, &j->o, (float *)j->out, j->stream, ws, &j->info, h);
    cudaEventRecord(j->e1, j->stream);
    ws.release();
    if (rc == DS_OK && cudaLaunchHostFunc(j->stream, job_done, j) == cudaSuccess) return;
    // failed to queue: finish now with the error
    cudaStreamSynchronize(j->stream);
    finish_failed(j, rc != DS_OK ? rc : DS_ERR_CUDA);
}

// the next admissible job (ctx->mu held): the oldest planned job that fits, unless an older one
// that does not fit has been passed over kMaxBypass times already
static std::deque<ServeJob *>::iterator next_admissible(ds_ctx *ctx) {
    auto end = ctx->queue.end();
    for (auto it = ctx->queue.begin(); it != end; ++it) {
        ServeJob *j = *it;
        if (!j->planned) continue;
        if (j->plan_status != DS_OK) return it;  // finishes at once with its error
        if (ctx->inflight_bytes == 0 || ctx->inflight_bytes + j->footprint <= ctx->budget) return it;
        if (j->bypassed >= kMaxBypass) return end;
    }
    return end;
}

static void worker_loop(ds_ctx *ctx) {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(ctx->mu);
    const int nhi = (int)ctx->serve_streams.size() / 2;
    for (;;) {
        std::deque<ServeJob *>::iterator it;
        ctx->cv.wait(lk, [&] {
            if (ctx->stop) return true;
            if (ctx->paused || ctx->queue.empty()) return false;
            it = next_admissible(ctx);
            return it != ctx->queue.end();
        });
        if (ctx->stop) break;
        ServeJob *j = *it;
        // every planned job ahead of it that does not fit has been passed over once more
        for (auto k = ctx->queue.begin(); k != it; ++k)
            if ((*k)->planned) (*k)->bypassed++;
        ctx->queue.erase(it);
        if (j->plan_status != DS_OK) {
            const ds_status st = j->plan_status;
            lk.unlock();
            finish_failed(j, st);
            lk.lock();
            continue;
        }
        ctx->inflight_bytes += j->footprint;
        // priority class by cost against the median of the recent jobs, then the least busy stream
        std::vector<double> c(ctx->recent_cost.begin(), ctx->recent_cost.end());
        bool high = true;
        if (!c.empty()) {
            std::nth_element(c.begin(), c.begin() + c.size() / 2, c.end());
            high = j->cost <= c[c.size() / 2];
        }
        ctx->recent_cost.push_back(j->cost);
        if ((int)ctx->recent_cost.size() > kCostWindow) ctx->recent_cost.pop_front();
        const int lo = high ? 0 : nhi, hi = high ? nhi : (int)ctx->serve_streams.size();
        int best = lo;
        for (int s = lo; s < hi; ++s)
            if (ctx->stream_jobs[s] < ctx->stream_jobs[best]) best = s;
        j->stream_idx = best;
        ctx->stream_jobs[best]++;
        j->stream = ctx->serve_streams[best];
        lk.unlock();
        launch_job(j);
        lk.lock();
    }
}

static ds_status ensure_worker(ds_ctx *ctx) {
    std::lock_guard<std::mutex> g(ctx->mu);
    if (ctx->worker_started) return DS_OK;
    cudaSetDevice(ctx->device);
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    for (int i = 0; i < kServeStreams; ++i) {
        cudaStream_t s;
        const int prio = i < kServeStreams / 2 ? greatest : least;
        if (cudaStreamCreateWithPriority(&s, cudaStreamNonBlocking, prio) != cudaSuccess)
            return ds_fail(ctx, DS_ERR_CUDA, "stream creation failed");
        ctx->serve_streams.push_back(s);
        ctx->stream_jobs.push_back(0);
    }
    if (cudaStreamCreateWithFlags(&ctx->plan_stream, cudaStreamNonBlocking) != cudaSuccess)
        return ds_fail(ctx, DS_ERR_CUDA, "stream creation failed");
    if (cudaMallocHost(&ctx->plan_host, sizeof(double) * 16 * kPlanSlots) != cudaSuccess)
        return ds_fail(ctx, DS_ERR_OOM, "pinned planning buffer");
    for (int i = kPlanSlots - 1; i >= 0; --i) ctx->plan_free.push_back(i);
    ctx->stop = false;
    ctx->worker = std::thread(worker_loop, ctx);
    ctx->worker_started = true;
    return DS_OK;
}

void serving_shutdown(ds_ctx *ctx) {
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        if (!ctx->worker_started) return;
        ctx->stop = true;
        ctx->cv.notify_all();
    }
    ctx->worker.join();
    cudaSetDevice(ctx->device);
    if (ctx->plan_stream) {
        cudaStreamSynchronize(ctx->plan_stream);
        cudaStreamDestroy(ctx->plan_stream);
        ctx->plan_stream = nullptr;
    }
    for (cudaStream_t s : ctx->serve_streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    ctx->serve_streams.clear();
    ctx->stream_jobs.clear();
    std::lock_guard<std::mutex> g(ctx->mu);
    for (ServeJob *j : ctx->queue) ctx->jobs.erase(j->ticket), delete j;
    ctx->queue.clear();
    for (auto &kv : ctx->jobs) {
        cudaEventDestroy(kv.second->e0);
        cudaEventDestroy(kv.second->e1);
        delete kv.second;
    }
    ctx->jobs.clear();
    if (ctx->plan_host) cudaFreeHost(ctx->plan_host);
    ctx->plan_host = nullptr;
    ctx->plan_free.clear();
    ctx->recent_cost.clear();
    ctx->worker_started = false;
}

extern "C" ds_status ds_submit(ds_model *M, const ds_qgrid *q, const ds_opts *o, void *out, uint64_t *ticket) {
    if (!M) return DS_ERR_ARG;
    ds_ctx *ctx = M->ctx;
    if (!out || !ticket) return ds_fail(ctx, DS_ERR_ARG, "null output or ticket");
    ds_status rc = check_request(M, q, o);
    if (rc != DS_OK) return rc;
    int g0[3], cnt[3];
    rc = grid_indices(ctx, M, q, g0, cnt);
    if (rc != DS_OK) return rc;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return ds_fail(ctx, DS_ERR_CUDA, "cudaSetDevice");
    rc = ensure_worker(ctx);
    if (rc != DS_OK) return rc;
    ServeJob *j = new ServeJob();
    j->ctx = ctx;
    j->model = M;
    j->q = *q;
    j->o = *o;
    j->out = out;
    j->t_submit = now_s();
    memset(&j->info, 0, sizeof(j->info));
    const size_t esz = o->precision == DS_FP64 ? 8 : 4;
    const double out_bytes = (double)cnt[0] * cnt[1] * cnt[2] * esz;
    const bool plan = o->disorder == DS_DISP && o->taylor_order < 0;
    // the footprint of a displacive request with an automatic order is known once x_max is: until
    // then it is bounded by the order 60 limit for the refusal of oversized requests
    j->footprint = request_footprint(M, q, &j->o, plan ? 0 : o->taylor_order);
    if (j->footprint > ctx->budget) {
        const size_t fp = j->footprint;
        delete j;
        return ds_fail(ctx, DS_ERR_ADMISSION, "request needs about %zu bytes, budget %zu", fp, ctx->budget);
    }
    j->cost = (double)j->footprint + out_bytes;
    if (cudaEventCreate(&j->e0) != cudaSuccess || cudaEventCreate(&j->e1) != cudaSuccess) {
        delete j;
        return ds_fail(ctx, DS_ERR_CUDA, "event creation failed");
    }
    std::unique_lock<std::mutex> lk(ctx->mu);
    j->ticket = ctx->next_ticket++;
    ctx->jobs[j->ticket] = j;
    if (!plan) {
        j->planned = true;
    } else if (!ctx->plan_free.empty()) {
        // x_max on the planning stream, read back into a pinned slot; job_planned completes the plan
        j->plan_slot = ctx->plan_free.back();
        ctx->plan_free.pop_back();
        lk.unlock();
        Scratch ws(ctx->plan_stream);
        rc = queue_corner_xmax(M, q, o, ctx->plan_stream, ws, ctx->plan_host + 16 * j->plan_slot);
        ws.release();
        if (rc == DS_OK && cudaLaunchHostFunc(ctx->plan_stream, job_planned, j) != cudaSuccess) rc = DS_ERR_CUDA;
        lk.lock();
        if (rc != DS_OK) {
            ctx->plan_free.push_back(j->plan_slot);
            ctx->jobs.erase(j->ticket);
            cudaEventDestroy(j->e0);
            cudaEventDestroy(j->e1);
            delete j;
            return rc == DS_ERR_CUDA ? ds_fail(ctx, rc, "planning launch failed") : rc;
        }
    } else {
        // every planning slot busy: plan on this thread
        lk.unlock();
        Scratch ws(ctx->plan_stream);
        int P = 0;
        double umax = 0.0;
        rc = resolve_taylor_order(M, q, o, ctx->plan_stream, ws, &P, &j->xmax, &umax);
        ws.release();
        lk.lock();
        if (rc != DS_OK) {
            ctx->jobs.erase(j->ticket);
            cudaEventDestroy(j->e0);
            cudaEventDestroy(j->e1);
            delete j;
            return rc;
        }
        j->has_hint = true;
        j->hint.P = P;
        j->hint.xmax = j->xmax;
        j->hint.umax = umax;
        j->footprint = request_footprint(M, q, &j->o, P);
        j->cost = (double)j->footprint + out_bytes;
        j->planned = true;
    }
    ctx->queue.push_back(j);
    ctx->cv.notify_all();
    *ticket = j->ticket;
    return DS_OK;
}

// fills info of a finished job, returns its status and forgets it
static ds_status finish(ds_ctx *ctx, ServeJob *j, ds_result_info *info) {
    ds_status st = j->status;
    if (info) {
        *info = j->info;
        float ms = 0.f;
        if (st == DS_OK && cudaEventElapsedTime(&ms, j->e0, j->e1) == cudaSuccess) info->gpu_ms = ms;
        info->latency_ms = 1e3 * (j->t_done - j->t_submit);
        if (j->o.disorder == DS_DISP && j->xmax >= 0) info->x_max = j->xmax;
    }
    cudaEventDestroy(j->e0);
    cudaEventDestroy(j->e1);
    ctx->jobs.erase(j->ticket);
    delete j;
    return st;
}

extern "C" ds_status ds_poll(ds_ctx *ctx, uint64_t ticket, ds_result_info *info) {
    if (!ctx) return DS_ERR_ARG;
    std::unique_lock<std::mutex> lk(ctx->mu);
    auto it = ctx->jobs.find(ticket);
    if (it == ctx->jobs.end()) return ds_fail(ctx, DS_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    if (!it->second->done) return DS_ERR_STATE;
    return finish(ctx, it->second, info);
}

extern "C" ds_status ds_wait(ds_ctx *ctx, uint64_t ticket, double timeout_s, ds_result_info *info) {
    if (!ctx) return DS_ERR_ARG;
    std::unique_lock<std::mutex> lk(ctx->mu);
    auto it = ctx->jobs.find(ticket);
    if (it == ctx->jobs.end()) return ds_fail(ctx, DS_ERR_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    ServeJob *j = it->second;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0);
    if (!ctx->cv.wait_until(lk, deadline, [&] { return j->done; }))
        return ds_fail(ctx, DS_ERR_TIMEOUT, "ticket %llu not finished after %.3f s", (unsigned long long)ticket, timeout_s);
    return finish(ctx, j, info);
}

extern "C" ds_status ds_serving_pause(ds_ctx *ctx, int pause) {
    if (!ctx) return DS_ERR_ARG;
    std::lock_guard<std::mutex> g(ctx->mu);
    ctx->paused = pause != 0;
    ctx->cv.notify_all();
    return DS_OK;
}
