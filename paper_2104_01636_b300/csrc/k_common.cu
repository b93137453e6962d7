// Launch geometry, the deterministic second pass of every reduction, and the
// host mirror of the device scalars.
#include <mutex>

#include "vof_internal.cuh"

Launch launch_cells(int nx, int ny, int nz, int sm_count) {
    Launch L;
    const int gx = (nx + TBX - 1) / TBX, gy = (ny + TBY - 1) / TBY;
    const int target = sm_count * 8;
    int gz = target / (gx * gy);
    if (gz < 1) gz = 1;
    if (gz > nz) gz = nz;
    while (gx * gy * gz > MAX_PARTIALS && gz > 1) --gz;
    L.kchunk = (nz + gz - 1) / gz;
    gz = (nz + L.kchunk - 1) / L.kchunk;
    L.grid = dim3(gx, gy, gz);
    L.block = dim3(TBX, TBY, 1);
    L.nblocks = gx * gy * gz;
    return L;
}

__global__ void k_finalize_sum(const double* __restrict__ part, int n, double* out, double scale) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    s = block_sum(s);
    if (threadIdx.x == 0) *out = s * scale;
}

__global__ void k_finalize_max(const double* __restrict__ part, int n, double* out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s = fmax(s, part[i]);
    s = block_max(s);
    if (threadIdx.x == 0) *out = s;
}

__global__ void k_finalize_dots_beta(const double* __restrict__ pa, const double* __restrict__ pb,
                                     int n, double* scal) {
    const double rz = sum_partials(pa, n);
    const double zq = sum_partials(pb, n);
    if (threadIdx.x == 0) {
        scal[S_RZ] = rz * 1.0;
        scal[S_ZQ] = zq * 1.0;
        const double pq = scal[S_PQ];  // of the previous direction
        scal[S_BETA] = pq > 0.0 ? -zq / pq : 0.0;
    }
}

__global__ void k_finalize_pq_alpha(const double* __restrict__ part, int n, double* scal) {
    const double pq = sum_partials(part, n);
    if (threadIdx.x == 0) {
        scal[S_PQ] = pq * 1.0;
        scal[S_ALPHA] = pq > 0.0 ? scal[S_RZ] / pq : 0.0;
    }
}

void finalize_dots_beta(vof_ctx* c, int nparts) {
    VOF_LAUNCH(c, k_finalize_dots_beta, 1, 1024, c->part + (size_t)S_RZ * MAX_PARTIALS,
               c->part + (size_t)S_ZQ * MAX_PARTIALS, nparts, c->scal);
}

void finalize_pq_alpha(vof_ctx* c, int nparts) {
    VOF_LAUNCH(c, k_finalize_pq_alpha, 1, 1024, c->part + (size_t)S_PQ * MAX_PARTIALS, nparts,
               c->scal);
}

void finalize_sum(vof_ctx* c, int slot, int nparts, int dst, double scale) {
    VOF_LAUNCH(c, k_finalize_sum, 1, 1024, c->part + (size_t)slot * MAX_PARTIALS, nparts,
                                          c->scal + dst, scale);
}

void finalize_max(vof_ctx* c, int slot, int nparts, int dst) {
    VOF_LAUNCH(c, k_finalize_max, 1, 1024, c->part + (size_t)slot * MAX_PARTIALS, nparts,
                                          c->scal + dst);
}

// ---- host mirror of the device scalars --------------------------------------
// A readback is a one-block kernel that writes the scalars into page-locked,
// mapped host memory, then a wait on the context stream. No copy engine is
// involved, so a readback never queues behind a large copy running on another
// stream (the copies of vof_step_host), and nothing is staged through
// pageable memory. The mirrors come from a process-wide arena that is never
// freed: freeing page-locked memory would synchronise the whole device.
namespace {
std::mutex g_mirror_mu;
std::vector<double*> g_mirror_free;

__global__ void k_to_mirror(const double* __restrict__ s, double* __restrict__ h, int n) {
    if ((int)threadIdx.x < n) h[threadIdx.x] = s[threadIdx.x];
    __threadfence_system();
}
}  // namespace

double* mirror_acquire() {
    std::lock_guard<std::mutex> lock(g_mirror_mu);
    if (g_mirror_free.empty()) {
        constexpr int SLOTS = 64;
        void* p = nullptr;
        if (cudaHostAlloc(&p, (size_t)SLOTS * MIRROR_DOUBLES * sizeof(double),
                          cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        for (int q = SLOTS - 1; q >= 0; --q) g_mirror_free.push_back((double*)p + q * MIRROR_DOUBLES);
    }
    double* p = g_mirror_free.back();
    g_mirror_free.pop_back();
    return p;
}

void mirror_release(double* p) {
    std::lock_guard<std::mutex> lock(g_mirror_mu);
    g_mirror_free.push_back(p);
}

void readback(vof_ctx* c) {
    if (c->hmirror_dev) {
        ++c->nlaunch;
        k_to_mirror<<<1, MIRROR_DOUBLES, 0, c->st>>>(c->scal, c->hmirror_dev, S_NSCALARS);
    } else {
        cudaMemcpyAsync(c->hbuf, c->scal, sizeof(double) * S_NSCALARS, cudaMemcpyDeviceToHost,
                        c->st);
    }
    cudaStreamSynchronize(c->st);
}
