// Ensemble of independent ducts advanced together (one time step of every
// case per call). Each case keeps its context and its fields resident on the
// device, and every case's arithmetic is exactly that of a solo run
// (deterministic reductions, private workspace). Two ways to run the cases:
//
//  * batched (the default where the solver allows it): the cases' contexts
//    are carved from one arena at a fixed stride, and the pressure solves of
//    all cases run as one batched solve -- every multigrid operation of a
//    level, every Krylov update and reduction, one launch for all cases, the
//    V-cycle replayed from one CUDA graph -- between the per-case parts of
//    the step (advection to the right side before, correction after), which
//    worker threads launch on their own streams;
//  * streams: cases are dealt round-robin to worker threads, each driving its
//    own CUDA stream, so the cases' kernels overlap on the GPU.
#include <chrono>
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
    // batched solve
    bool batched = false;
    int phase = 0;  // what the workers run: 0 the whole step, 1 before the solve, 2 after it
    char* arena = nullptr;
    long long stride = 0;
    BatchSolveState* bs = nullptr;
    std::vector<int> run;
    std::vector<vof_status> solve_st;
    std::vector<vof_report> rep;
    double phase_ms[3] = {0.0, 0.0, 0.0};  // host time: before the solve, the solve, after it
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
            if (e->phase == 0) {
                vof_report* rep = e->reports ? e->reports + c : nullptr;
                e->status[c] = step_entry(e->ctx[c], f[0], f[1], f[2], f[3], f[4], f[5], f[6],
                                          f[7], e->dt[c], e->step_index, rep);
            } else if (e->phase == 1) {
                e->status[c] = step_pre_cfl(e->ctx[c], f, e->dt[c]);
            } else if (e->run[c]) {
                e->status[c] = step_post(e->ctx[c], f, e->dt[c], e->solve_st[c]);
            }
        }
        cudaStreamSynchronize(e->streams[w]);
        if (e->phase == 1) {
            // the CFL tests of the worker's cases, read back together; then the
            // rest of each case's step up to the solve, launched without a wait
            for (int c = w; c < e->n; c += e->nworkers)
                if (e->status[c] == VOF_OK)
                    e->status[c] = step_pre(e->ctx[c], e->fields + 8 * (size_t)c, e->dt[c],
                                            e->step_index);
            cudaStreamSynchronize(e->streams[w]);
        } else if (e->phase == 2) {
            for (int c = w; c < e->n; c += e->nworkers)
                if (e->run[c])
                    e->status[c] = step_post_report(e->ctx[c], e->solve_st[c], &e->rep[c]);
        }
        {
            std::lock_guard<std::mutex> lk(e->mu);
            if (--e->pending == 0) e->cv_done.notify_all();
        }
    }
}

// runs one phase on every worker and waits for all of them
void run_phase(vof_ensemble* e, int phase) {
    {
        std::unique_lock<std::mutex> lk(e->mu);
        e->phase = phase;
        e->pending = e->nworkers;
        ++e->generation;
    }
    e->cv_go.notify_all();
    std::unique_lock<std::mutex> lk(e->mu);
    e->cv_done.wait(lk, [&] { return e->pending == 0; });
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
    batch_solve_destroy(e->bs);
    if (e->arena) cudaFree(e->arena);
    for (cudaStream_t s : e->streams)
        if (s) cudaStreamDestroy(s);
    delete e;
}

// the contexts of a batched ensemble, carved from one arena; false (nothing
// left allocated) when the solver does not allow the batched solve or the
// contexts do not come out alike
bool create_batched(vof_ensemble* e, const vof_grid* grid, const vof_phys* phys, int n_phys,
                    const vof_solver* sv, vof_status* err) {
    *err = VOF_OK;
    // batched grids repeat a case's z blocks (at most nz) once per case
    if ((long long)grid->nz * e->n > 65535) return false;
    const long long S =
        (long long)((workspace_bytes(grid, sv) + (1u << 20) + 65535u) & ~(size_t)65535u);
    if (cudaMalloc((void**)&e->arena, (size_t)S * e->n) != cudaSuccess) {
        cudaGetLastError();
        e->arena = nullptr;
        *err = VOF_ERR_OOM;
        return false;
    }
    e->stride = S;
    bool ok = true;
    for (int c = 0; c < e->n && ok; ++c) {
        const vof_status st =
            create_in_arena(grid, phys + (n_phys == 1 ? 0 : c), sv, e->streams[c % e->nworkers],
                            e->arena + (size_t)c * S, (size_t)S, &e->ctx[c]);
        ok = st == VOF_OK && e->ctx[c]->arena_used == e->ctx[0]->arena_used;
        if (ok) e->ctx[c]->defer_dense = true;
        if (c == 0 && ok) ok = batch_solve_eligible(e->ctx[0]);
    }
    if (ok) {
        e->bs = batch_solve_create(e->ctx[0], e->n, S);
        ok = e->bs != nullptr;
    }
    if (!ok) {
        for (vof_ctx*& c : e->ctx)
            if (c) {
                c->defer_dense = false;
                vof_destroy(c);
                c = nullptr;
            }
        cudaFree(e->arena);
        e->arena = nullptr;
        return false;
    }
    e->run.assign(e->n, 0);
    e->solve_st.assign(e->n, VOF_OK);
    e->rep.assign(e->n, vof_report{});
    e->batched = true;
    return true;
}

}  // namespace

extern "C" {

vof_status vof_ensemble_create_mode(const vof_grid* grid, const vof_phys* phys, int n_phys,
                                    const vof_solver* solver, int n_cases, int n_streams,
                                    int mode, vof_ensemble** out) {
    if (!out || !grid || !phys || !solver || n_cases < 1 || n_streams < 1 || n_streams > 64 ||
        (n_phys != 1 && n_phys != n_cases) ||
        (mode != VOF_ENSEMBLE_AUTO && mode != VOF_ENSEMBLE_STREAMS &&
         mode != VOF_ENSEMBLE_BATCHED))
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
    if (mode != VOF_ENSEMBLE_STREAMS) {
        vof_status err = VOF_OK;
        if (!create_batched(e, grid, phys, n_phys, &sv, &err) && mode == VOF_ENSEMBLE_BATCHED) {
            destroy_all(e);
            return err != VOF_OK ? err : VOF_ERR_UNSUPPORTED;
        }
    }
    if (!e->batched)
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

vof_status vof_ensemble_create(const vof_grid* grid, const vof_phys* phys, int n_phys,
                               const vof_solver* solver, int n_cases, int n_streams,
                               vof_ensemble** out) {
    return vof_ensemble_create_mode(grid, phys, n_phys, solver, n_cases, n_streams,
                                    VOF_ENSEMBLE_AUTO, out);
}

vof_status vof_ensemble_batched(const vof_ensemble* e, int* batched) {
    if (!e || !batched) return VOF_ERR_ARG;
    *batched = e->batched ? 1 : 0;
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
    }
    using clk = std::chrono::steady_clock;
    auto ms_since = [](clk::time_point t0) {
        return std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    };
    if (!e->batched) {
        const auto t0 = clk::now();
        run_phase(e, 0);
        e->phase_ms[0] += ms_since(t0);
    } else {
        auto t0 = clk::now();
        run_phase(e, 1);
        e->phase_ms[0] += ms_since(t0);
        t0 = clk::now();
        for (int c = 0; c < e->n; ++c) {
            e->run[c] = e->status[c] == VOF_OK ? 1 : 0;
            e->rep[c] = vof_report{};
            e->solve_st[c] = VOF_OK;
        }
        const vof_status st = solve_mixed_batch(e->ctx[0], e->n, e->stride, e->run.data(), e->bs,
                                                e->solve_st.data(), e->rep.data(), e->ctx.data());
        if (st != VOF_OK)
            for (int c = 0; c < e->n; ++c)
                if (e->run[c]) e->status[c] = st;
        e->phase_ms[1] += ms_since(t0);
        t0 = clk::now();
        run_phase(e, 2);
        e->phase_ms[2] += ms_since(t0);
        if (reports)
            for (int c = 0; c < e->n; ++c)
                if (e->run[c]) reports[c] = e->rep[c];
    }
    vof_status first = VOF_OK;
    for (int c = 0; c < e->n; ++c) {
        if (status) status[c] = e->status[c];
        if (first == VOF_OK) first = e->status[c];
    }
    return first;
}

vof_status vof_ensemble_phase_ms(const vof_ensemble* e, double* ms) {
    if (!e || !ms) return VOF_ERR_ARG;
    for (int q = 0; q < 3; ++q) ms[q] = e->phase_ms[q];
    return VOF_OK;
}

vof_status vof_ensemble_launch_count(const vof_ensemble* e, long long* n) {
    if (!e || !n) return VOF_ERR_ARG;
    long long t = 0;
    for (const vof_ctx* c : e->ctx)
        if (c) t += c->nlaunch;
    *n = t;
    return VOF_OK;
}

vof_status vof_ensemble_destroy(vof_ensemble* e) {
    if (!e) return VOF_ERR_ARG;
    destroy_all(e);
    return VOF_OK;
}

}  // extern "C"
