// Continuous-batching request server over the time-step library.
//
// Requests (a number of time steps, or one pressure solve, on a grid of its
// own) are queued in arrival order. A request is admitted as soon as a
// worker slot is free and its device memory (fields plus context workspace)
// fits in what is left of the budget; it then runs on its worker's CUDA
// stream, so admitted requests overlap on the GPU while later arrivals wait
// for slots and memory to free up. Admission is strictly first-in first-out,
// which bounds every request's wait. Each request's kernels are deterministic
// and touch only its own memory, so a result does not depend on what else
// was running.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "vof_internal.cuh"

namespace {

struct Job {
    unsigned long long id = 0;
    vof_request rq;
    size_t need = 0;
    vof_result res;
};

size_t field_bytes(const vof_grid& g, int kind) {
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const size_t nu = (size_t)(g.nx + 1) * g.ny * g.nz, nv = (size_t)g.nx * (g.ny + 1) * g.nz;
    if (kind == VOF_REQ_SOLVE) return 3 * n * sizeof(double);  // alpha, b, p
    return (5 * n + nu + nv + n) * sizeof(double);             // alpha, uc, vc, wc, p, u, v, w
}

}  // namespace

struct vof_server {
    int dev = 0;
    size_t budget = 0, used = 0;
    int slots = 1;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Job*> queue;
    std::map<unsigned long long, Job*> jobs;
    std::vector<std::thread> workers;
    bool stopping = false;
    unsigned long long next_id = 1;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// Runs one request on stream st; returns its status and fills the report.
vof_status run_job(Job* j, cudaStream_t st) {
    const vof_request& r = j->rq;
    const vof_grid& g = r.grid;
    const size_t n = (size_t)g.nx * g.ny * g.nz;
    const size_t nu = (size_t)(g.nx + 1) * g.ny * g.nz, nv = (size_t)g.nx * (g.ny + 1) * g.nz;
    const size_t D = sizeof(double);
    std::vector<void*> mem;
    auto A = [&](size_t bytes) -> double* {
        void* p = nullptr;
        if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        mem.push_back(p);
        return (double*)p;
    };
    auto release = [&]() {
        for (void* p : mem) cudaFreeAsync(p, st);
        cudaStreamSynchronize(st);
    };
    vof_status status = VOF_OK;
    vof_ctx* ctx = nullptr;
    // a request's context lives for one request: capturing and instantiating
    // a graph per request (from several workers at once) costs more than it
    // saves, so server contexts launch directly. They keep the built-in
    // launch shapes: shapes timed for one context alone favour more, smaller
    // blocks on the coarse levels, which lose when several requests share
    // the GPU (measured: 37-41 against 62 requests/s on the seeded mix)
    vof_solver sv = r.solver;
    sv.graph = VOF_GRAPH_OFF;
    sv.mg_tune = VOF_TUNE_OFF;
    const vof_status cs = vof_create(&g, &r.phys, &sv, 0, st, &ctx);
    if (cs != VOF_OK || !ctx) {
        cudaGetLastError();
        return cs != VOF_OK ? cs : VOF_ERR_OOM;
    }
    if (r.kind == VOF_REQ_SOLVE) {
        double *a = A(n * D), *b = A(n * D), *p = A(n * D);
        if (!a || !b || !p) {
            vof_destroy(ctx);
            release();
            return VOF_ERR_OOM;
        }
        cudaMemcpyAsync(a, r.alpha, n * D, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(b, r.b, n * D, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(p, r.p, n * D, cudaMemcpyHostToDevice, st);
        status = pressure_solve(ctx, a, b, p, &j->res.report);
        cudaMemcpyAsync(r.p, p, n * D, cudaMemcpyDeviceToHost, st);
    } else {
        double* d[8];
        const size_t sz[8] = {n, n, n, n, nu, nv, n, n};
        double* const h[8] = {r.alpha, r.uc, r.vc, r.wc, r.u, r.v, r.w, r.p};
        for (int q = 0; q < 8; ++q) {
            d[q] = A(sz[q] * D);
            if (!d[q]) {
                vof_destroy(ctx);
                release();
                return VOF_ERR_OOM;
            }
            cudaMemcpyAsync(d[q], h[q], sz[q] * D, cudaMemcpyHostToDevice, st);
        }
        for (int s = 0; s < r.n_steps && status == VOF_OK; ++s)
            status = step_entry(ctx, d[0], d[1], d[2], d[3], d[4], d[5], d[6], d[7], r.dt,
                                r.step0 + s, &j->res.report);
        for (int q = 0; q < 8; ++q)
            cudaMemcpyAsync(h[q], d[q], sz[q] * D, cudaMemcpyDeviceToHost, st);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        status = VOF_ERR_CUDA;
    }
    vof_destroy(ctx);
    release();
    return status;
}

void worker_main(vof_server* s) {
    cudaSetDevice(s->dev);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
        Job* j = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] {
                return (s->stopping && s->queue.empty()) ||
                       (!s->queue.empty() && s->used + s->queue.front()->need <= s->budget);
            });
            if (s->queue.empty()) break;  // stopping and drained
            j = s->queue.front();
            s->queue.pop_front();
            s->used += j->need;
            j->res.state = 1;
            j->res.t_admit = s->now();
        }
        const vof_status st_run = run_job(j, st);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->used -= j->need;
            j->res.status = st_run;
            j->res.t_finish = s->now();
            j->res.state = 2;
        }
        s->cv.notify_all();
    }
    cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

vof_status vof_server_create(size_t budget_bytes, int max_concurrent, vof_server** out) {
    if (!out || max_concurrent < 1 || max_concurrent > 64 || budget_bytes == 0) return VOF_ERR_ARG;
    *out = nullptr;
    vof_server* s = new vof_server();
    if (cudaGetDevice(&s->dev) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return VOF_ERR_CUDA;
    }
    s->budget = budget_bytes;
    s->slots = max_concurrent;
    // keep up to the budget cached in the device's default pool between
    // requests instead of returning it to the driver at every synchronisation
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, s->dev) == cudaSuccess) {
        unsigned long long keep = budget_bytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    for (int w = 0; w < max_concurrent; ++w) s->workers.emplace_back(worker_main, s);
    *out = s;
    return VOF_OK;
}

vof_status vof_submit(vof_server* s, const vof_request* rq, unsigned long long* id) {
    if (!s || !rq || !id) return VOF_ERR_ARG;
    if (rq->kind != VOF_REQ_STEP && rq->kind != VOF_REQ_SOLVE) return VOF_ERR_ARG;
    if (!rq->alpha || !rq->p || (rq->kind == VOF_REQ_SOLVE && !rq->b)) return VOF_ERR_ARG;
    if (rq->kind == VOF_REQ_STEP &&
        (!rq->uc || !rq->vc || !rq->wc || !rq->u || !rq->v || !rq->w || rq->n_steps < 1 ||
         !(rq->dt > 0.0)))
        return VOF_ERR_ARG;
    size_t ws = 0;
    if (vof_workspace_bytes(&rq->grid, &rq->solver, &ws) != VOF_OK) return VOF_ERR_ARG;
    const size_t need = ws + field_bytes(rq->grid, rq->kind);
    if (need > s->budget) return VOF_ERR_ADMISSION;  // could never be admitted
    Job* j = new Job();
    j->rq = *rq;
    j->need = need;
    std::memset(&j->res, 0, sizeof(j->res));
    j->res.status = -1;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stopping) {
            delete j;
            return VOF_ERR_ARG;
        }
        j->id = s->next_id++;
        j->res.t_submit = s->now();
        s->jobs[j->id] = j;
        s->queue.push_back(j);
        *id = j->id;
    }
    s->cv.notify_all();
    return VOF_OK;
}

vof_status vof_poll(vof_server* s, unsigned long long id, vof_result* res) {
    if (!s || !res) return VOF_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return VOF_ERR_ARG;
    *res = it->second->res;
    return VOF_OK;
}

vof_status vof_wait(vof_server* s, unsigned long long id, vof_result* res) {
    if (!s || !res) return VOF_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(id);
    if (it == s->jobs.end()) return VOF_ERR_ARG;
    Job* j = it->second;
    s->cv.wait(lk, [&] { return j->res.state == 2; });
    *res = j->res;
    return VOF_OK;
}

vof_status vof_server_destroy(vof_server* s) {
    if (!s) return VOF_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv.notify_all();
    for (auto& t : s->workers) t.join();
    for (auto& kv : s->jobs) delete kv.second;
    delete s;
    return VOF_OK;
}

}  // extern "C"
