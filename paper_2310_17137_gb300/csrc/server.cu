// Continuous-batching server for GP solve + posterior-mean requests.
//
// Requests arrive at any time (ap_server_submit).  A scheduler admits them in
// arrival order as soon as a worker slot is free and the request's estimated
// device footprint fits in the HBM budget; memory and slots are returned the
// moment a request finishes, so later arrivals are admitted while earlier ones
// are still on the GPU.  Each worker owns a CUDA stream and runs its request's
// whole pipeline there -- copies in, FP64 block-Cholesky cache, Alg. 1 with one
// captured CUDA graph per epoch (the persistent tensor-core kernel in the
// low-precision form), posterior mean (Sec. 2), copy out -- so the work of
// different requests overlaps on the device.  Every per-request computation is
// deterministic (fixed-order reductions), so a result is the same alone and in
// a mix.  The paper has no serving component; this is the deployment shape of
// its solver.
#include <math.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ap_internal.cuh"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Job {
    int64_t id = 0;
    ap_request req;
    std::vector<float> ell;  // own copy of the lengthscales
    size_t reserve = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    ap_status status = AP_OK;
    int epochs = 0;
    double rel_res = 0.0;
    int compensated = 0;
    bool done = false;
    volatile int32_t cancel = 0;  // read by the solve between epochs
};

// Device bytes a request needs: inputs and outputs, the scaled inputs, the FP32
// inverse-factor cache, solve buffers, the tensor-core operands, and an FP64
// factorisation workspace of a few blocks (the context sizes its block groups to
// whatever is left of the reservation).
size_t estimate_bytes(const ap_request& r) {
    const int64_t n = r.n, d = r.d, M = r.M;
    const int64_t b = r.block < n ? r.block : n;
    const int64_t m = (n + b - 1) / b;
    const int64_t nt = (b + 63) / 64;
    const int64_t ntri = nt * (nt + 1) / 2;
    const int64_t D = d <= 4 ? 4 : (d <= 8 ? 8 : (d <= 12 ? 12 : (d <= 16 ? 16 : (d <= 24 ? 24 : 32))));
    const int64_t Cp = r.precision == AP_FP32 ? 1 : 16;
    size_t bytes = 0;
    bytes += (size_t)(n * d + 3 * n + M * d + M) * 4;            // caller data staged on the device
    bytes += (size_t)(2 * n * D) * 4;                              // Xs, Xs_lo
    bytes += (size_t)(m * ntri) * 64 * 64 * 4;                     // L^-1 cache
    bytes += (size_t)(4 * n * Cp) * 4 + (size_t)(nt * 64 + b) * Cp * 4;  // R, W, Bp, Tmp, Z, Delta
    if (r.precision != AP_FP32) {
        const int kd = ap::tc_kd((int)d);
        const int cpb = ap::tc_chunks_per_block(b);
        bytes += ap::tc_rows_bytes(m * ((b + 127) / 128), kd);  // row operands
        bytes += ap::tc_cols_bytes(m, cpb, kd);                 // column operands
        bytes += ap::tc_delta_bytes(cpb, 16);                   // Delta^T
        bytes += ap::tc_share_bytes(256, AP_MAX_RHS);           // boundary slots (up to 256 SMs)
    }
    bytes += (size_t)(M * D) * 4 + (size_t)(1 << 20);              // test inputs, partials
    const size_t ws_block = (size_t)(nt * 64) * (nt * 64) * 8 + (size_t)nt * 64 * 64 * 8;
    bytes += ws_block * (size_t)(m < 4 ? m : 4);                   // FP64 workspace
    return bytes + bytes / 16;                                     // slack
}

}  // namespace

struct ap_server {
    int device = 0;
    size_t budget = 0, reserved = 0;
    int slots = 1;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<Job*> pending;
    std::deque<Job*> admitted;
    std::unordered_map<int64_t, std::unique_ptr<Job>> jobs;
    int64_t next_id = 1;
    int idle = 0;
    bool stop = false;
    std::vector<std::thread> workers;
    std::thread scheduler;
};

namespace {

ap_status run_job(ap_server* srv, Job* j, cudaStream_t st) {
    const ap_request& r = j->req;
    float *X = nullptr, *Y = nullptr, *B = nullptr, *W = nullptr, *Xt = nullptr, *mu = nullptr;
    auto cleanup = [&]() {
        cudaFreeAsync(X, st);
        cudaFreeAsync(Y, st);
        cudaFreeAsync(B, st);
        cudaFreeAsync(W, st);
        cudaFreeAsync(Xt, st);
        cudaFreeAsync(mu, st);
        cudaStreamSynchronize(st);
        cudaGetLastError();
    };
    if (cudaMallocAsync((void**)&X, sizeof(float) * r.n * r.d, st) != cudaSuccess ||
        cudaMallocAsync((void**)&Y, sizeof(float) * r.n, st) != cudaSuccess ||
        cudaMallocAsync((void**)&B, sizeof(float) * r.n, st) != cudaSuccess ||
        cudaMallocAsync((void**)&W, sizeof(float) * r.n, st) != cudaSuccess ||
        cudaMallocAsync((void**)&Xt, sizeof(float) * r.M * r.d, st) != cudaSuccess ||
        cudaMallocAsync((void**)&mu, sizeof(float) * r.M, st) != cudaSuccess) {
        cleanup();
        return AP_ERR_NOMEM;
    }
    if (cudaMemcpyAsync(X, r.X_host, sizeof(float) * r.n * r.d, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(Y, r.y_host, sizeof(float) * r.n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(Xt, r.Xtest_host, sizeof(float) * r.M * r.d, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        ap::launch_assemble_rhs(Y, r.hyper.mean, nullptr, 0, 0, r.n, B, nullptr, st) != cudaSuccess) {
        cleanup();
        return AP_ERR_CUDA;
    }
    ap_opts o;
    ap_opts_default(&o);
    o.block = r.block;
    o.tol = r.tol;
    o.stop = r.stop;
    o.min_epochs = r.min_epochs;
    o.max_epochs = r.max_epochs;
    o.precision = r.precision;
    o.refine_every = r.refine_every > 0 ? r.refine_every : 4;
    o.stream = st;
    o.cancel = &j->cancel;
    const size_t inputs = sizeof(float) * (size_t)(r.n * r.d + 3 * r.n + r.M * r.d + r.M);
    o.hbm_budget = j->reserve > inputs ? j->reserve - inputs : 0;
    ap_hyper h = r.hyper;
    h.lengthscale = j->ell.data();
    ap_ctx* ctx = nullptr;
    ap_status s = ap_create(&ctx, X, r.n, r.d, &h, &o);
    if (s != AP_OK) {
        cleanup();
        return s;
    }
    ap_info info;
    memset(&info, 0, sizeof(info));
    s = j->cancel ? AP_ERR_CANCELLED : ap_solve(ctx, B, 1, nullptr, W, &info);
    j->epochs = info.epochs;
    j->rel_res = info.rel_res_true[0];
    j->compensated = info.compensated;
    if (s == AP_OK || s == AP_ERR_NOT_CONVERGED) {
        ap_status sp = ap_predict_mean(ctx, W, Xt, r.M, mu);
        if (sp != AP_OK) s = sp;
    }
    ap_destroy(ctx);
    if (s == AP_OK || s == AP_ERR_NOT_CONVERGED) {
        if (cudaMemcpyAsync(r.mean_host, mu, sizeof(float) * r.M, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            s = AP_ERR_CUDA;
    }
    cleanup();
    (void)srv;
    return s;
}

void worker_main(ap_server* srv) {
    cudaSetDevice(srv->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    while (true) {
        Job* j = nullptr;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            ++srv->idle;
            srv->cv_sched.notify_all();
            srv->cv_sched.wait(lk, [&] { return srv->stop || !srv->admitted.empty(); });
            --srv->idle;
            if (srv->stop && srv->admitted.empty()) break;
            j = srv->admitted.front();
            srv->admitted.pop_front();
            j->t_start = now_s();
        }
        const ap_status s = run_job(srv, j, st);
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            j->status = s;
            j->t_done = now_s();
            j->done = true;
            srv->reserved -= j->reserve;
        }
        srv->cv_sched.notify_all();
        srv->cv_done.notify_all();
    }
    cudaStreamDestroy(st);
}

// Admit pending requests in arrival order while a worker is idle and the
// request fits in what is left of the budget.
void scheduler_main(ap_server* srv) {
    std::unique_lock<std::mutex> lk(srv->mu);
    while (!srv->stop) {
        bool progressed = false;
        while (!srv->pending.empty()) {
            Job* j = srv->pending.front();
            const int free_workers = srv->idle - (int)srv->admitted.size();
            if (free_workers <= 0 || srv->reserved + j->reserve > srv->budget) break;
            srv->pending.pop_front();
            srv->reserved += j->reserve;
            srv->admitted.push_back(j);
            progressed = true;
        }
        if (progressed) srv->cv_sched.notify_all();
        srv->cv_sched.wait_for(lk, std::chrono::milliseconds(50));
    }
}

}  // namespace

extern "C" {

size_t ap_sizeof_request(void) { return sizeof(ap_request); }
size_t ap_sizeof_request_result(void) { return sizeof(ap_request_result); }

ap_status ap_server_create(ap_server** out, size_t hbm_budget, int32_t slots, int32_t device) {
    if (!out || slots < 1 || slots > 64 || hbm_budget == 0) return AP_ERR_INVALID_ARG;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return AP_ERR_CUDA;
    }
    // keep freed request memory in the process's pool instead of returning it
    // to the driver after every request (a per-process pool attribute)
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = (uint64_t)hbm_budget;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    ap_server* srv = new ap_server();
    srv->device = device;
    srv->budget = hbm_budget;
    srv->slots = slots;
    for (int i = 0; i < slots; ++i) srv->workers.emplace_back(worker_main, srv);
    srv->scheduler = std::thread(scheduler_main, srv);
    *out = srv;
    return AP_OK;
}

ap_status ap_server_submit(ap_server* srv, const ap_request* r, int64_t* id) {
    if (!srv || !r || !id || !r->X_host || !r->y_host || !r->Xtest_host || !r->mean_host) return AP_ERR_INVALID_ARG;
    if (r->n < 1 || r->d < 1 || r->d > AP_MAX_DIM || r->M < 1 || r->block < 1 || !r->hyper.lengthscale ||
        r->hyper.d != r->d)
        return AP_ERR_INVALID_ARG;
    std::unique_ptr<Job> j(new Job());
    j->req = *r;
    j->ell.assign(r->hyper.lengthscale, r->hyper.lengthscale + r->d);
    j->reserve = estimate_bytes(*r);
    if (j->reserve > srv->budget) return AP_ERR_NOMEM;
    j->t_submit = now_s();
    std::lock_guard<std::mutex> lk(srv->mu);
    j->id = srv->next_id++;
    *id = j->id;
    srv->pending.push_back(j.get());
    srv->jobs[j->id] = std::move(j);
    srv->cv_sched.notify_all();
    return AP_OK;
}

ap_status ap_server_poll(ap_server* srv, int64_t id, ap_request_result* res) {
    if (!srv || !res) return AP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    auto it = srv->jobs.find(id);
    if (it == srv->jobs.end()) return AP_ERR_INVALID_ARG;
    const Job* j = it->second.get();
    res->done = j->done ? 1 : 0;
    res->status = j->done ? j->status : AP_OK;
    res->epochs = j->epochs;
    res->rel_res = j->rel_res;
    res->queue_s = (j->t_start > 0 ? j->t_start : now_s()) - j->t_submit;
    res->latency_s = j->done ? j->t_done - j->t_submit : 0.0;
    res->reserved_bytes = j->reserve;
    res->started = j->t_start > 0 ? 1 : 0;
    res->compensated = j->compensated;
    return AP_OK;
}

ap_status ap_server_cancel(ap_server* srv, int64_t id) {
    if (!srv) return AP_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        auto it = srv->jobs.find(id);
        if (it == srv->jobs.end()) return AP_ERR_INVALID_ARG;
        Job* j = it->second.get();
        if (j->done) return AP_OK;
        j->cancel = 1;
        for (auto p = srv->pending.begin(); p != srv->pending.end(); ++p) {
            if (*p == j) {
                // never admitted: nothing reserved, nothing on the device
                srv->pending.erase(p);
                j->status = AP_ERR_CANCELLED;
                j->t_done = now_s();
                j->done = true;
                break;
            }
        }
    }
    srv->cv_done.notify_all();
    return AP_OK;
}

ap_status ap_server_wait(ap_server* srv, int64_t id, double timeout_s, ap_request_result* res) {
    if (!srv || !res) return AP_ERR_INVALID_ARG;
    {
        std::unique_lock<std::mutex> lk(srv->mu);
        auto it = srv->jobs.find(id);
        if (it == srv->jobs.end()) return AP_ERR_INVALID_ARG;
        Job* j = it->second.get();
        const bool ok = srv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return j->done; });
        if (!ok) return AP_ERR_TIMEOUT;
    }
    return ap_server_poll(srv, id, res);
}

void ap_server_destroy(ap_server* srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
        // requests never admitted are dropped
        srv->pending.clear();
    }
    srv->cv_sched.notify_all();
    for (auto& t : srv->workers) t.join();
    srv->scheduler.join();
    delete srv;
}

}  // extern "C"
