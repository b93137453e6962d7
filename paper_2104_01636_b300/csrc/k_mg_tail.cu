// Coarse tail of the mixed-precision multigrid cycle in one launch.
//
// Below some size a level's smoothing pass, restriction or dense coarsest
// solve takes a few microseconds of launch latency for well under a
// microsecond of work; the W-cycle visits those levels hundreds of times per
// time step. Here the whole cycle from a small level down (its smoothing
// passes, restrictions, the coarser levels' visits, the dense coarsest
// solve and the corrections on the way back up) runs as one kernel on one
// thread-block cluster: the CTAs of a cluster are co-scheduled on one GPC,
// so each operation spreads its cells over all threads of the cluster and
// the operations are separated by hardware cluster barriers
// (barrier.cluster arrive.release / wait.acquire) instead of kernel
// boundaries. The level arrays stay in global memory (a few MB, resident in
// L2); values written inside the launch are read back with L2 loads.
//
// The grid-wide variant (VOF_TAIL_GRID) runs the same program as one
// cooperative launch with one block on every SM, the operations separated
// by a grid-wide barrier: a counter in global memory that each block's
// first thread raises after a fence and then waits on with acquire loads.
// The counter only grows within a launch (operation o completes at
// (o + 1) x blocks) and is cleared before each launch. Every wait is
// bounded: a block that gives up sets the error flag and returns, so the
// others give up at their next barrier and the launch ends.
//
// The operations and their order come from the host (the same recursion as
// the launch-per-operation cycle, solver.cu) as a short program in device
// memory; the cell arithmetic is that of k_mg.cu (mg_cell.cuh), so the tail
// and the launch-per-operation cycle produce the same values.
#include <algorithm>

#include "mg_cell.cuh"
#include "vof_internal.cuh"

namespace {

constexpr int TAIL_THREADS = 1024;

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}

constexpr int GRID_WAIT_LIMIT = 1 << 21;  // acquire loads before a barrier wait gives up

// false once the wait gave up (the error flag is then set)
__device__ __forceinline__ bool grid_sync_bounded(unsigned* count, unsigned target, double* err) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        ok = 1;
        for (int it = 0;; ++it) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(count) : "memory");
            if (v >= target) break;
            if (it >= GRID_WAIT_LIMIT) {
                *err = 1.0;
                ok = 0;
                break;
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

__device__ __forceinline__ unsigned cluster_ctarank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

template <bool GRID>
__global__ void __launch_bounds__(TAIL_THREADS, 1)
    k_mg_tail(const TailProg* __restrict__ prog, const float* __restrict__ minv,
              unsigned* __restrict__ bar, double* __restrict__ err) {
    __shared__ float fs[DENSE_MAX];
    __shared__ TailProg sp;  // the program, read once
    {
        const int4* src = reinterpret_cast<const int4*>(prog);
        int4* dst = reinterpret_cast<int4*>(&sp);
        for (int e = threadIdx.x; e < (int)(sizeof(TailProg) / sizeof(int4)); e += blockDim.x)
            dst[e] = src[e];
        __syncthreads();
    }
    const int nthr = gridDim.x * blockDim.x;  // the grid: one cluster, or one block per SM
    const int gt = (int)(GRID ? blockIdx.x : cluster_ctarank()) * blockDim.x + threadIdx.x;
    const int nops = sp.nops;
    const float omega = sp.omega;
    const LdL2 ld;
    for (int o = 0; o < nops; ++o) {
        const TailOp op = sp.op[o];
        const TailLevel& L = sp.L[op.lev];
        const Dims d = L.d;
        if (op.kind == TAIL_SMOOTH) {
            // the cells of one colour, enumerated as x-pairs (2t, 2t+1) of
            // which one member has the colour (odd nx: the last pair may
            // have none)
            const TailLevel& C = sp.L[op.mode == 2 ? op.lev + 1 : op.lev];
            const Dims dc = C.d;
            const int hx = (d.nx + 1) >> 1;
            const int n = hx * d.ny * d.nz;
            for (int it = gt; it < n; it += nthr) {
                const int t = it % hx, r = it / hx, j = r % d.ny, k = r / d.ny;
                const int i = 2 * t + ((j + k + op.color) & 1);
                if (i >= d.nx) continue;
                if (op.mode == 1)
                    rbgs_cell<float, 1>(d, L.h2, L.bx, L.by, L.bz, L.x, L.x, L.f, i, j, k, dc,
                                        C.x, omega, ld);
                else if (op.mode == 2)
                    rbgs_cell<float, 2>(d, L.h2, L.bx, L.by, L.bz, L.x, L.x, L.f, i, j, k, dc,
                                        C.x, omega, ld);
                else
                    rbgs_cell<float, 0>(d, L.h2, L.bx, L.by, L.bz, L.x, L.x, L.f, i, j, k, dc,
                                        C.x, omega, ld);
            }
        } else if (op.kind == TAIL_RESTRICT) {
            const TailLevel& C = sp.L[op.lev + 1];
            const Dims dc = C.d;
            const int n = dc.nx * dc.ny * dc.nz;
            for (int it = gt; it < n; it += nthr) {
                const int I = it % dc.nx, r = it / dc.nx, J = r % dc.ny, K = r / dc.ny;
                restrict_cell(d, L.ih2, L.bx, L.by, L.bz, L.x, L.f, dc, C.f, I, J, K, ld);
            }
        } else {  // TAIL_DENSE: x = Minv f on the coarsest level, one warp per row
            const int n = d.nx * d.ny * d.nz;
            for (int e = threadIdx.x; e < n; e += blockDim.x) fs[e] = ld(L.f + e);
            __syncthreads();
            const int lane = threadIdx.x & 31, nw = nthr >> 5;
            for (int row = gt >> 5; row < n; row += nw) {
                const double s =
                    dense_row(minv + (long)row * n, [&](int j) { return fs[j]; }, n, lane);
                if (lane == 0) L.x[row] = (float)s;
            }
        }
        if (GRID) {
            if (!grid_sync_bounded(bar, (unsigned)(o + 1) * gridDim.x, err)) return;
        } else {
            cluster_sync_all();
        }
    }
}

}  // namespace

// Chooses the cluster (16 CTAs where the device schedules that many, else
// 8) and uploads the two programs (first visit from zero, later visits from
// the level's current x). Leaves c->tail_level at 0 when the tail cannot run.
vof_status mg_tail_setup(vof_ctx* c, int level, const TailProg* from_zero,
                         const TailProg* from_x, bool grid) {
    c->tail_level = 0;
    int cs = 0, gb = 0;
    if (grid) {
        // one resident block per SM, which a cooperative launch guarantees
        int coop = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->dev) != cudaSuccess ||
            !coop ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mg_tail<true>, TAIL_THREADS,
                                                          0) != cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            return VOF_OK;
        }
        gb = c->sm_count;
    } else if (cudaFuncSetAttribute(k_mg_tail<false>, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                    1) != cudaSuccess) {
        cudaGetLastError();
        return VOF_OK;
    }
    for (int want : {16, 8}) {
        if (grid) break;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = want;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(want);
        cfg.blockDim = dim3(TAIL_THREADS);
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, k_mg_tail<false>, &cfg) == cudaSuccess &&
            nclusters >= 1) {
            cs = want;
            break;
        }
        cudaGetLastError();
    }
    if (cs == 0 && gb == 0) return VOF_OK;
    TailProg* d = (TailProg*)dev_alloc(c, 2 * sizeof(TailProg) + 256);
    if (!d) return set_err(c, VOF_ERR_OOM, "allocation of the coarse-tail program failed");
    c->tail_bar = reinterpret_cast<unsigned*>(reinterpret_cast<char*>(d) + 2 * sizeof(TailProg));
    c->tail_host[0] = *from_zero;
    c->tail_host[1] = *from_x;
    if (cudaMemcpyAsync(d, c->tail_host, 2 * sizeof(TailProg), cudaMemcpyHostToDevice, c->st) !=
        cudaSuccess)
        return cuda_check(c, cudaGetLastError(), "coarse-tail program upload");
    c->tail_prog = d;
    c->tail_cluster = cs;
    c->tail_grid = gb;
    c->tail_level = level;
    return VOF_OK;
}

void mg_tail_run(vof_ctx* c, bool zero_start) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    if (c->tail_grid) {
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cfg.gridDim = dim3(c->tail_grid);
    } else {
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = c->tail_cluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(c->tail_cluster);
    }
    cfg.blockDim = dim3(TAIL_THREADS);
    cfg.stream = c->st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const TailProg* p = c->tail_prog + (zero_start ? 0 : 1);
    int m = timer_begin(c, T_COARSE);
    ++c->nlaunch;
    if (c->tail_grid) {
        cudaMemsetAsync(c->tail_bar, 0, sizeof(unsigned), c->st);
        cudaLaunchKernelEx(&cfg, k_mg_tail<true>, p, (const float*)c->dense_inv_f, c->tail_bar,
                           c->scal + S_ERR);
    } else {
        cudaLaunchKernelEx(&cfg, k_mg_tail<false>, p, (const float*)c->dense_inv_f, c->tail_bar,
                           c->scal + S_ERR);
    }
    timer_end(c, T_COARSE, m);
}
