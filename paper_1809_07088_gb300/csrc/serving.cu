// Continuous-batching request loop (ds_submit / ds_poll / ds_wait).
//
// ds_submit plans a request on the caller's thread (validation, the Taylor order from x_max on
// the context's planning stream, the HBM footprint from request_footprint) and queues it.  One
// worker thread per context admits queued requests in arrival order whenever the footprint of
// the requests in flight plus the next one fits the context's budget, and launches each on one
// of the context's compute streams, so that the kernels of concurrent requests overlap on the
// GPU.  Completion is reported by a host callback queued behind the request's kernels
// (cudaLaunchHostFunc), which returns the footprint to the budget, timestamps the latency and
// wakes the worker and any waiter.  Every voxel of a request is computed by the same kernels
// with the same reduction order as an isolated request, so results do not depend on the mix.
//
// Host waits are bounded (ds_wait takes a timeout); no kernel of the path waits on another.
#include <chrono>
#include <cstring>

#include "api_internal.h"

using namespace ds;

namespace {

constexpr int kServeStreams = 8;

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
    double xmax = -1.0;
    bool has_hint = false;
    TaylorHint hint;
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
    ds_ctx *ctx = j->ctx;
    cudaStreamSynchronize(j->stream);
    std::lock_guard<std::mutex> g(ctx->mu);
    j->status = rc != DS_OK ? rc : DS_ERR_CUDA;
    j->t_done = now_s();
    j->done = true;
    ctx->inflight_bytes -= j->footprint;
    ctx->cv.notify_all();
}

static void worker_loop(ds_ctx *ctx) {
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(ctx->mu);
    int next = 0;
    for (;;) {
        ctx->cv.wait(lk, [&] {
            if (ctx->stop) return true;
            if (ctx->paused || ctx->queue.empty()) return false;
            const ServeJob *j = ctx->queue.front();
            return ctx->inflight_bytes == 0 || ctx->inflight_bytes + j->footprint <= ctx->budget;
        });
        if (ctx->stop) break;
        ServeJob *j = ctx->queue.front();
        ctx->queue.pop_front();
        ctx->inflight_bytes += j->footprint;
        j->stream = ctx->serve_streams[next];
        next = (next + 1) % (int)ctx->serve_streams.size();
        lk.unlock();
        launch_job(j);
        lk.lock();
    }
}

static ds_status ensure_worker(ds_ctx *ctx) {
    std::lock_guard<std::mutex> g(ctx->mu);
    if (ctx->worker_started) return DS_OK;
    cudaSetDevice(ctx->device);
    for (int i = 0; i < kServeStreams; ++i) {
        cudaStream_t s;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
            return ds_fail(ctx, DS_ERR_CUDA, "stream creation failed");
        ctx->serve_streams.push_back(s);
    }
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
    for (cudaStream_t s : ctx->serve_streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    ctx->serve_streams.clear();
    std::lock_guard<std::mutex> g(ctx->mu);
    for (ServeJob *j : ctx->queue) ctx->jobs.erase(j->ticket), delete j;
    ctx->queue.clear();
    for (auto &kv : ctx->jobs) {
        cudaEventDestroy(kv.second->e0);
        cudaEventDestroy(kv.second->e1);
        delete kv.second;
    }
    ctx->jobs.clear();
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
    int P = o->taylor_order;
    if (o->disorder == DS_DISP && P < 0) {
        Scratch ws(ctx->stream);
        double umax = 0.0;
        rc = resolve_taylor_order(M, q, o, ctx->stream, ws, &P, &j->xmax, &umax);
        ws.release();
        if (rc != DS_OK) {
            delete j;
            return rc;
        }
        j->has_hint = true;
        j->hint.P = P;
        j->hint.xmax = j->xmax;
        j->hint.umax = umax;
    }
    j->footprint = request_footprint(M, q, &j->o, P < 0 ? 0 : P);
    if (j->footprint > ctx->budget) {
        const size_t fp = j->footprint;
        delete j;
        return ds_fail(ctx, DS_ERR_ADMISSION, "request needs about %zu bytes, budget %zu", fp, ctx->budget);
    }
    if (cudaEventCreate(&j->e0) != cudaSuccess || cudaEventCreate(&j->e1) != cudaSuccess) {
        delete j;
        return ds_fail(ctx, DS_ERR_CUDA, "event creation failed");
    }
    std::lock_guard<std::mutex> g(ctx->mu);
    j->ticket = ctx->next_ticket++;
    ctx->jobs[j->ticket] = j;
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
