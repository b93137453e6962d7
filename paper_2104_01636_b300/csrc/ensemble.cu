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
//
// In the batched mode with the solver's graph option left at AUTO, the whole
// ensemble step is one CUDA graph launch: the CFL test of every case (one
// launch and a device-side test), then, under a conditional IF node that the
// test opens, every case's step up to its solve (the cases' branches run
// side by side), the batched solve with its loops as conditional WHILE
// nodes steered on the device, and every case's correction. From 8 cases
// up the cases run in groups of consecutive cases (up to four) with a
// batched solve each: a group's part before its solve starts when the group
// before has ended its own, so it runs beside that group's solve. A step
// whose CFL test fails in any case is run again the host-driven way, which
// reports each case's status; nothing of the step has been launched by then.
// The graph is captured for the step's field pointers and time steps and the
// parity of the step index (the sweep order), and captured again when they
// change.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <vector>

#include "vof_internal.cuh"

// one captured ensemble step and what it was captured for
struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    std::vector<double*> f;  // the 8 n field pointers
    std::vector<double> dt;
    double* dt_d = nullptr;        // device copies the CFL test reads
    const double** uvw_d = nullptr;
    long long k_top = 0, k_body = 0;        // kernels per replay outside the solves' loops
    std::vector<long long> k_outer, k_inner;  // per case group: kernels per pass of its loops
};

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
    // the whole step as one graph: 1 in use, 0 host-driven, -1 capture failed
    int step_graph = 0;
    StepGraph sg[2];                           // by the parity of the step index
    cudaStream_t gst[2] = {nullptr, nullptr};  // capture origin, IF body
    cudaEvent_t ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
    // The cases in groups of consecutive cases, each with its own batched
    // solve, so that one group's solve runs beside the next group's part
    // before the solve (which starts when the group before has finished
    // its own). Per group: its solve's state, the origin of its branch, an
    // event at the end of its part before the solve; per group and worker:
    // the stream its cases launch on while the step is captured.
    int ngroups = 1;
    std::vector<BatchSolveState*> gbs;
    std::vector<cudaStream_t> gorig, gwork;
    std::vector<cudaEvent_t> ev_grp;
    unsigned long long* vmax_d = nullptr;  // per case: largest face-velocity magnitude (bits)
    int* abort_h = nullptr;                // mapped: the CFL test failed in some case
    int* abort_d = nullptr;
    // mapped: device clock (ns) at the step's start, after the parts before
    // the solves, after the solve, at the end
    unsigned long long* stamp_h = nullptr;
    unsigned long long* stamp_d = nullptr;
    long long graph_steps = 0, graph_kernels = 0;
};

namespace {

// The CFL test of every case in one launch (blockIdx.y: the case): the
// largest face-velocity magnitude, over the faces k_cfl reads, with the bit
// patterns of the magnitudes compared as integers (their order is that of the
// values, and a NaN sorts above every number).
__global__ void k_ens_vmax(Dims d, int per_x, int per_y, const double* const* __restrict__ uvw,
                           unsigned long long* __restrict__ vmax) {
    const int cs = blockIdx.y;
    const double* __restrict__ u = uvw[3 * cs];
    const double* __restrict__ v = uvw[3 * cs + 1];
    const double* __restrict__ w = uvw[3 * cs + 2];
    const int n = d.nx * d.ny * d.nz;
    constexpr unsigned long long MAG = 0x7FFFFFFFFFFFFFFFULL;
    auto mag = [](double x) { return (unsigned long long)__double_as_longlong(x) & MAG; };
    unsigned long long mb = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        const int i = c % d.nx, j = (c / d.nx) % d.ny, k = c / (d.nx * d.ny);
        if (i > 0 || per_x) mb = max(mb, mag(u[uid(d, i, j, k)]));
        if (j > 0 || per_y) mb = max(mb, mag(v[vid(d, i, j, k)]));
        mb = max(mb, mag(w[wid(d, i, j, k)]));
    }
    for (int o = 16; o > 0; o >>= 1) mb = max(mb, __shfl_xor_sync(0xffffffffu, mb, o));
    if ((threadIdx.x & 31) == 0 && mb) atomicMax(vmax + cs, mb);
}

// the test step_pre takes per case (a Courant number above 1 or not finite);
// the IF node opens only when every case passes
__global__ void k_ens_cfl_ctl(const unsigned long long* __restrict__ vmax,
                              const double* __restrict__ dt, int nc, double h, int* abort_flag,
                              cudaGraphConditionalHandle h_go) {
    int bad = 0;
    for (int i = threadIdx.x; i < nc; i += blockDim.x) {
        const double cfl = __longlong_as_double((long long)vmax[i]) * dt[i] / h;
        if (!isfinite(cfl) || cfl > 1.0) bad = 1;
    }
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        *abort_flag = bad;
        cudaGraphSetConditional(h_go, bad ? 0u : 1u);
    }
}

// the device's global clock (ns) into slot q, once the work before it is done
__global__ void k_stamp(unsigned long long* t, int q) {
    unsigned long long v;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
    t[q] = v;
}

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

// ---- the whole step as one graph ---------------------------------------------
// ensembles of at least this many cases run the captured step in groups:
// n / 4 groups, at most ENSEMBLE_MAX_GROUPS (measured with 64 cases of
// 48x48x96: 32.8, 31.5, 30.8 and 30.6 ms per step with 1, 2, 4 and 8 groups)
constexpr int ENSEMBLE_GROUP_MIN_CASES = 8;
constexpr int ENSEMBLE_MAX_GROUPS = 4;

// the first case of group g (g = ngroups: one past the last case)
int group_first(const vof_ensemble* e, int g) { return (int)((long long)g * e->n / e->ngroups); }

void free_step_graph(StepGraph& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.dt_d) cudaFree(g.dt_d);
    if (g.uvw_d) cudaFree((void*)g.uvw_d);
    g = StepGraph{};
}

// the streams, events and flags the captured step uses; false (the
// ensemble stays host-driven) when any is unavailable
bool step_graph_resources(vof_ensemble* e) {
    bool ok = true;
    for (cudaStream_t& s : e->gst)
        ok = ok && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    e->ngroups = e->n >= ENSEMBLE_GROUP_MIN_CASES ? std::min(ENSEMBLE_MAX_GROUPS, e->n / 4) : 1;
    const int G = e->ngroups;
    e->gbs.assign(G, nullptr);
    e->gorig.assign(G, nullptr);
    e->ev_grp.assign(G, nullptr);
    e->gwork.assign((size_t)G * e->nworkers, nullptr);
    for (int g = 0; g < G && ok; ++g) {
        e->gbs[g] = batch_solve_create(e->ctx[group_first(e, g)], group_first(e, g + 1) -
                                                                      group_first(e, g),
                                       e->stride);
        ok = e->gbs[g] != nullptr &&
             cudaStreamCreateWithFlags(&e->gorig[g], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&e->ev_grp[g], cudaEventDisableTiming) == cudaSuccess;
    }
    for (cudaStream_t& s : e->gwork)
        ok = ok && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
    // the groups' states encoded their TMA maps into the groups' first
    // contexts; case 0's context keeps those of the whole batch (the
    // host-driven solve)
    ok = ok && rho_path_batch_maps(e->ctx[0], e->n, e->stride) == VOF_OK;
    ok = ok && cudaEventCreateWithFlags(&e->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    e->ev_join.assign(e->nworkers, nullptr);
    for (cudaEvent_t& ev : e->ev_join)
        ok = ok && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaMalloc((void**)&e->vmax_d, sizeof(unsigned long long) * e->n) == cudaSuccess;
    ok = ok && cudaHostAlloc((void**)&e->abort_h, sizeof(int), cudaHostAllocMapped) == cudaSuccess &&
         cudaHostGetDevicePointer((void**)&e->abort_d, e->abort_h, 0) == cudaSuccess;
    ok = ok &&
         cudaHostAlloc((void**)&e->stamp_h, 4 * sizeof(unsigned long long), cudaHostAllocMapped) ==
             cudaSuccess &&
         cudaHostGetDevicePointer((void**)&e->stamp_d, e->stamp_h, 0) == cudaSuccess;
    cudaGetLastError();
    return ok;
}

void free_step_graph_resources(vof_ensemble* e) {
    for (StepGraph& g : e->sg) free_step_graph(g);
    for (cudaStream_t& s : e->gst)
        if (s) cudaStreamDestroy(s);
    for (BatchSolveState* b : e->gbs) batch_solve_destroy(b);
    for (cudaStream_t s : e->gorig)
        if (s) cudaStreamDestroy(s);
    for (cudaStream_t s : e->gwork)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t ev : e->ev_grp)
        if (ev) cudaEventDestroy(ev);
    if (e->ev_fork) cudaEventDestroy(e->ev_fork);
    for (cudaEvent_t ev : e->ev_join)
        if (ev) cudaEventDestroy(ev);
    if (e->vmax_d) cudaFree(e->vmax_d);
    if (e->abort_h) cudaFreeHost(e->abort_h);
    if (e->stamp_h) cudaFreeHost(e->stamp_h);
}

// group g's capture streams join the capture on s, and later join it again
void fork_to_group(vof_ensemble* e, int g, cudaStream_t s) {
    cudaEventRecord(e->ev_fork, s);
    for (int w = 0; w < e->nworkers; ++w)
        cudaStreamWaitEvent(e->gwork[(size_t)g * e->nworkers + w], e->ev_fork, 0);
}
void join_group(vof_ensemble* e, int g, cudaStream_t s) {
    for (int w = 0; w < e->nworkers; ++w) {
        cudaEventRecord(e->ev_join[w], e->gwork[(size_t)g * e->nworkers + w]);
        cudaStreamWaitEvent(s, e->ev_join[w], 0);
    }
}

// Captures the ensemble step for these fields, time steps and step parity
// into g. While the step is captured, each case's context launches on its
// group's stream for its worker, which joins the capture, so a group's cases
// are side-by-side branches of the graph; each group's batched solve is
// captured on the group's origin. False when capture is unavailable
// (nothing stays captured).
bool capture_step(vof_ensemble* e, StepGraph& g, double* const* fields, const double* dt,
                  long long step_index) {
    const int n = e->n, G = e->ngroups, nw = e->nworkers;
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    if (!g.dt_d && cudaMalloc((void**)&g.dt_d, sizeof(double) * n) != cudaSuccess) return false;
    if (!g.uvw_d && cudaMalloc((void**)&g.uvw_d, sizeof(double*) * 3 * n) != cudaSuccess)
        return false;
    std::vector<const double*> uvw(3 * (size_t)n);
    for (int c = 0; c < n; ++c)
        for (int q = 0; q < 3; ++q) uvw[3 * (size_t)c + q] = fields[8 * (size_t)c + 4 + q];
    if (cudaMemcpy(g.dt_d, dt, sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy((void*)g.uvw_d, uvw.data(), sizeof(double*) * 3 * n,
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return false;
    for (int q = 0; q < G; ++q)  // the solves' loop bodies are captured on these
        for (cudaStream_t& s : e->ctx[group_first(e, q)]->cap_st)
            if (!s && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
    const vof_ctx* m = e->ctx[0];
    std::vector<long long> n0(n);
    std::vector<cudaStream_t> st0(n);
    for (int c = 0; c < n; ++c) {
        n0[c] = e->ctx[c]->nlaunch;
        st0[c] = e->ctx[c]->st;
    }
    int grp = 0;
    for (int c = 0; c < n; ++c) {
        while (c >= group_first(e, grp + 1)) ++grp;
        e->ctx[c]->st = e->gwork[(size_t)grp * nw + c % nw];
    }
    cudaStream_t s0 = e->gst[0], sb = e->gst[1];
    if (cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        for (int c = 0; c < n; ++c) e->ctx[c]->st = st0[c];
        return false;
    }
    cudaGraph_t gt = capture_graph_of(s0);
    cudaGraphConditionalHandle h_go = 0;
    bool ok = gt && cudaGraphConditionalHandleCreate(&h_go, gt, 0, cudaGraphCondAssignDefault) ==
                        cudaSuccess;
    const int ncell = m->d.nx * m->d.ny * m->d.nz;
    const int bpc = std::max(1, std::min((ncell + 2047) / 2048, 1024));
    const int nthr = n < 1024 ? ((n + 31) / 32) * 32 : 1024;
    k_stamp<<<1, 1, 0, s0>>>(e->stamp_d, 0);
    cudaMemsetAsync(e->vmax_d, 0, sizeof(unsigned long long) * n, s0);
    k_ens_vmax<<<dim3(bpc, n), 256, 0, s0>>>(m->d, m->g.periodic_x, m->g.periodic_y, g.uvw_d,
                                             e->vmax_d);
    k_ens_cfl_ctl<<<1, nthr, 0, s0>>>(e->vmax_d, g.dt_d, n, m->g.h, e->abort_d, h_go);
    cudaGraph_t gif = ok ? capture_if(s0, h_go) : nullptr;
    ok = ok && gif &&
         cudaStreamBeginCaptureToGraph(sb, gif, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    std::vector<long long> kk(3 * (size_t)G, 0);
    if (ok) {
        cudaEventRecord(e->ev_fork, sb);
        for (int q = 0; q < G; ++q) {
            cudaStream_t o = e->gorig[q];
            // group q's part before the solve after group q - 1's
            cudaStreamWaitEvent(o, q == 0 ? e->ev_fork : e->ev_grp[q - 1], 0);
            const int c0 = group_first(e, q), c1 = group_first(e, q + 1);
            fork_to_group(e, q, o);
            for (int c = c0; c < c1; ++c)
                ok = step_pre_launch(e->ctx[c], fields + 8 * (size_t)c, dt[c], step_index) ==
                         VOF_OK &&
                     ok;
            join_group(e, q, o);
            cudaEventRecord(e->ev_grp[q], o);
            if (q == 0) k_stamp<<<1, 1, 0, o>>>(e->stamp_d, 1);
            vof_ctx* mq = e->ctx[c0];
            cudaStream_t sq = mq->st;
            mq->st = o;
            ok = ok && rho_path_batch_maps(mq, c1 - c0, e->stride) == VOF_OK;
            ok = capture_solve_mixed_batch(mq, c1 - c0, e->stride, e->gbs[q], &kk[3 * (size_t)q]) &&
                 ok;
            mq->st = sq;
            if (q == G - 1) k_stamp<<<1, 1, 0, o>>>(e->stamp_d, 2);
            fork_to_group(e, q, o);
            for (int c = c0; c < c1; ++c) {
                solve_tail_captured(e->ctx[c]);
                ok = step_post(e->ctx[c], fields + 8 * (size_t)c, dt[c], VOF_OK) == VOF_OK && ok;
            }
            join_group(e, q, o);
        }
        for (int q = 0; q < G; ++q) {
            cudaEventRecord(e->ev_grp[q], e->gorig[q]);
            cudaStreamWaitEvent(sb, e->ev_grp[q], 0);
        }
        k_stamp<<<1, 1, 0, sb>>>(e->stamp_d, 3);
        cudaGraph_t gb = nullptr;
        ok = cudaStreamEndCapture(sb, &gb) == cudaSuccess && ok;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(s0, &graph);
    ok = ok && ee == cudaSuccess && graph &&
         cudaGraphInstantiate(&g.exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    long long body = 0;
    for (int c = 0; c < n; ++c) {
        body += e->ctx[c]->nlaunch - n0[c];
        e->ctx[c]->nlaunch = n0[c];
        e->ctx[c]->st = st0[c];
    }
    // case 0's context keeps the TMA maps of the whole batch (host-driven steps)
    ok = rho_path_batch_maps(e->ctx[0], n, e->stride) == VOF_OK && ok;
    if (!ok) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
        return false;
    }
    g.k_top = 3;
    g.k_body = body + 3;
    g.k_outer.assign(G, 0);
    g.k_inner.assign(G, 0);
    for (int q = 0; q < G; ++q) {
        g.k_body += kk[3 * (size_t)q];
        g.k_outer[q] = kk[3 * (size_t)q + 1];
        g.k_inner[q] = kk[3 * (size_t)q + 2];
    }
    g.f.assign(fields, fields + 8 * (size_t)n);
    g.dt.assign(dt, dt + n);
    return true;
}

// One ensemble step as one graph launch. *done is false when the step has to
// run the host-driven way (a failed CFL test, or no graph).
void run_step_graph(vof_ensemble* e, double* const* fields, const double* dt,
                    long long step_index, vof_report* reports, bool* done) {
    *done = false;
    const int n = e->n;
    StepGraph& g = e->sg[step_index & 1];
    const bool same = g.exec && std::equal(g.f.begin(), g.f.end(), fields) &&
                      std::equal(g.dt.begin(), g.dt.end(), dt);
    if (!same && !capture_step(e, g, fields, dt, step_index)) {
        e->step_graph = -1;
        return;
    }
    for (vof_ctx* c : e->ctx) c->err.clear();
    cudaGraphLaunch(g.exec, e->gst[0]);
    const cudaError_t ce = cudaStreamSynchronize(e->gst[0]);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        for (int c = 0; c < n; ++c)
            e->status[c] = cuda_check(e->ctx[c], ce, "ensemble step graph");
        *done = true;
        return;
    }
    if (*e->abort_h) {
        e->graph_kernels += g.k_top;
        return;
    }
    e->graph_kernels += g.k_top + g.k_body;
    for (int q = 0; q < e->ngroups; ++q) {
        long long to = 0, ti = 0;
        batch_solve_trips(e->gbs[q], &to, &ti);
        e->graph_kernels += to * g.k_outer[q] + ti * g.k_inner[q];
    }
    ++e->graph_steps;
    const unsigned long long* t = e->stamp_h;
    for (int q = 0; q < 3; ++q) e->phase_ms[q] += (double)(t[q + 1] - t[q]) * 1e-6;
    for (int c = 0; c < n; ++c) {
        vof_report r{};
        const vof_status solve = captured_case_result(e->ctx[c], &r);
        e->status[c] = step_post_report(e->ctx[c], solve, &r);
        if (reports) reports[c] = r;
    }
    *done = true;
}

// the batched step driven from the host: the cases' parts before the solve
// on the worker streams, the batched solve with its loops on the host, the
// parts after it on the worker streams
void batched_host_step(vof_ensemble* e, vof_report* reports) {
    using clk = std::chrono::steady_clock;
    auto ms_since = [](clk::time_point t0) {
        return std::chrono::duration<double, std::milli>(clk::now() - t0).count();
    };
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

void destroy_all(vof_ensemble* e) {
    {
        std::lock_guard<std::mutex> lk(e->mu);
        e->stopping = true;
    }
    e->cv_go.notify_all();
    for (auto& t : e->workers) t.join();
    free_step_graph_resources(e);
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

// the batched solve's launch shapes, timed as the steps launch them: for
// each group through its first context (the step graph), or for every case
// through case 0's (host-driven steps)
vof_status tune_batched(vof_ensemble* e) {
    if (e->step_graph == 1) {
        for (int g = 0; g < e->ngroups; ++g) {
            const vof_status st = batch_solve_tune(e->ctx[group_first(e, g)], e->gbs[g], e->stride);
            if (st != VOF_OK) return st;
        }
        return VOF_OK;
    }
    return batch_solve_tune(e->ctx[0], e->bs, e->stride);
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
        // the batched step as one graph unless the solver asks for the
        // host-driven loops (VOF_GRAPH_CYCLE) or direct launches
        if (e->batched && solver->graph == VOF_GRAPH_AUTO)
            e->step_graph = step_graph_resources(e) ? 1 : -1;
        if (e->batched) {
            const vof_status st = tune_batched(e);
            if (st != VOF_OK) {
                destroy_all(e);
                return st;
            }
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
        bool done = false;
        if (e->step_graph > 0) run_step_graph(e, fields, dt, step_index, reports, &done);
        if (!done) batched_host_step(e, reports);
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

vof_status vof_ensemble_graph_steps(const vof_ensemble* e, long long* n) {
    if (!e || !n) return VOF_ERR_ARG;
    *n = e->graph_steps;
    return VOF_OK;
}

vof_status vof_ensemble_mg_shape(const vof_ensemble* e, int level, int shape[4]) {
    if (!e || !shape) return VOF_ERR_ARG;
    if (!e->batched) return VOF_ERR_UNSUPPORTED;
    return mg_shape_of(e->ctx[0], level, shape);
}

vof_status vof_ensemble_launch_count(const vof_ensemble* e, long long* n) {
    if (!e || !n) return VOF_ERR_ARG;
    long long t = e->graph_kernels;
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
