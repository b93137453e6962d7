// Ensemble of independent ducts advanced together (one time step of every
// case per call). Each case keeps its context and its fields resident on the
// device; cases are dealt round-robin to worker threads, each driving its
// own CUDA stream, so the cases' kernels overlap on the GPU while every
// case's arithmetic stays exactly that of a solo run (deterministic
// reductions, private workspace).
#include <condition_variable>
#include <mutex>
#include <thread>
#include <vector>

#include "vof_internal.cuh"

struct vof_ensemble {
    int n = 0, nworkers = 0, dev = 0;
    std::vector<vof_ctx*> ctx;
    std::vector<cudaStream_t> streams;
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv_go, cv_done;
    unsigned long long generation = 0;
    int pending = 0;
    bool stopping = false;
    // arguments of the current step
    double* const* fields = nullptr;
    const double* dt = nullptr;
    long long step_index = 0;
    std::vector<vof_status> status;  // per case, of the last step
    vof_report* reports = nullptr;
};

namespace {

void ensemble_worker(vof_ensemble* e, int w) {
    cudaSetDevice(e->dev);
    unsigned long long seen = 0;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(e->mu);
            e->cv_go.wait(lk, [&] { return e->stopping || e->generation != seen; });
            if (e->stopping) return;
            seen = e->generation;
        }
        for (int c = w; c < e->n; c += e->nworkers) {
            double* const* f = e->fields + 8 * (size_t)c;
            vof_report* rep = e->reports ? e->reports + c : nullptr;
            const vof_status st = step_entry(e->ctx[c], f[0], f[1], f[2], f[3], f[4], f[5], f[6],
                                             f[7], e->dt[c], e->step_index, rep);
            e->status[c] = st;
        }
        cudaStreamSynchronize(e->streams[w]);
        {
            std::lock_guard<std::mutex> lk(e->mu);
            if (--e->pending == 0) e->cv_done.notify_all();
        }
    }
}

void destroy_all(vof_ensemble* e) {
    {
        std::lock_guard<std::mutex> lk(e->mu);
        e->stopping = true;
    }
    e->cv_go.notify_all();
    for (auto& t : e->workers) t.join();
    for (vof_ctx* c : e->ctx)
        if (c) vof_destroy(c);
    for (cudaStream_t s : e->streams)
        if (s) cudaStreamDestroy(s);
    delete e;
}

}  // namespace

extern "C" {

vof_status vof_ensemble_create(const vof_grid* grid, const vof_phys* phys, int n_phys,
                               const vof_solver* solver, int n_cases, int n_streams,
                               vof_ensemble** out) {
    if (!out || !grid || !phys || !solver || n_cases < 1 || n_streams < 1 || n_streams > 64 ||
        (n_phys != 1 && n_phys != n_cases))
        return VOF_ERR_ARG;
    *out = nullptr;
    vof_ensemble* e = new vof_ensemble();
    e->n = n_cases;
    e->nworkers = n_streams < n_cases ? n_streams : n_cases;
    if (cudaGetDevice(&e->dev) != cudaSuccess) {
        cudaGetLastError();
        delete e;
        return VOF_ERR_CUDA;
    }
    e->streams.assign(e->nworkers, nullptr);
    for (int w = 0; w < e->nworkers; ++w)
        if (cudaStreamCreateWithFlags(&e->streams[w], cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            destroy_all(e);
            return VOF_ERR_CUDA;
        }
    e->ctx.assign(n_cases, nullptr);
    e->status.assign(n_cases, VOF_OK);
    // the cases' solves keep their loops on the host: measured with 64 cases,
    // captured whole solves running side by side were slower (78 against
    // 64 ms per ensemble step on 16 streams)
    vof_solver sv = *solver;
    if (sv.graph == VOF_GRAPH_AUTO) sv.graph = VOF_GRAPH_CYCLE;
    for (int c = 0; c < n_cases; ++c) {
        const vof_status st = vof_create(grid, phys + (n_phys == 1 ? 0 : c), &sv, 0,
                                         e->streams[c % e->nworkers], &e->ctx[c]);
        if (st != VOF_OK) {
            destroy_all(e);
            return st;
        }
    }
    for (int w = 0; w < e->nworkers; ++w) e->workers.emplace_back(ensemble_worker, e, w);
    *out = e;
    return VOF_OK;
}

vof_status vof_ensemble_step(vof_ensemble* e, double* const* fields, const double* dt,
                             long long step_index, vof_status* status, vof_report* reports) {
    if (!e || !fields || !dt || step_index < 0) return VOF_ERR_ARG;
    for (int c = 0; c < 8 * e->n; ++c)
        if (!fields[c]) return VOF_ERR_ARG;
    {
        std::unique_lock<std::mutex> lk(e->mu);
        e->fields = fields;
        e->dt = dt;
        e->step_index = step_index;
        e->reports = reports;
        e->pending = e->nworkers;
        ++e->generation;
    }
    e->cv_go.notify_all();
    std::unique_lock<std::mutex> lk(e->mu);
    e->cv_done.wait(lk, [&] { return e->pending == 0; });
    vof_status first = VOF_OK;
    for (int c = 0; c < e->n; ++c) {
        if (status) status[c] = e->status[c];
        if (first == VOF_OK) first = e->status[c];
    }
    return first;
}

vof_status vof_ensemble_destroy(vof_ensemble* e) {
    if (!e) return VOF_ERR_ARG;
    destroy_all(e);
    return VOF_OK;
}

}  // extern "C"
