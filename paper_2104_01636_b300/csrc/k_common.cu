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

template <bool B>
__global__ void k_finalize_sum(Bat t, const double* __restrict__ part, int n, double* out,
                               double scale) {
    const BatBlk bb = bat_blk<B>(t, blockIdx.x, gridDim.x);
    if (bb.off) return;
    part = bat_at<B>(t, bb.cs, part);
    out = bat_at<B>(t, bb.cs, out);
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

template <bool B>
__global__ void k_finalize_dots_beta(Bat t, const double* __restrict__ pa,
                                     const double* __restrict__ pb, int n, double* scal) {
    const BatBlk bb = bat_blk<B>(t, blockIdx.x, gridDim.x);
    if (bb.off) return;
    pa = bat_at<B>(t, bb.cs, pa);
    pb = bat_at<B>(t, bb.cs, pb);
    scal = bat_at<B>(t, bb.cs, scal);
    const double rz = sum_partials(pa, n);
    const double zq = sum_partials(pb, n);
    if (threadIdx.x == 0) {
        scal[S_RZ] = rz * 1.0;
        scal[S_ZQ] = zq * 1.0;
        const double pq = scal[S_PQ];  // of the previous direction
        scal[S_BETA] = pq > 0.0 ? -zq / pq : 0.0;
    }
}

template <bool B>
__global__ void k_finalize_pq_alpha(Bat t, const double* __restrict__ part, int n, double* scal) {
    const BatBlk bb = bat_blk<B>(t, blockIdx.x, gridDim.x);
    if (bb.off) return;
    part = bat_at<B>(t, bb.cs, part);
    scal = bat_at<B>(t, bb.cs, scal);
    const double pq = sum_partials(part, n);
    if (threadIdx.x == 0) {
        scal[S_PQ] = pq * 1.0;
        scal[S_ALPHA] = pq > 0.0 ? scal[S_RZ] / pq : 0.0;
    }
}

// x = 0 and dst = src on FP32 vectors of n4 float4s, batched along y (the
// batched solve's memset of e and copy of p; one case: a plain launch)
template <bool B>
__global__ void k_zero32x4(Bat t, int n4, float4* __restrict__ x) {
    const BatBlk bb = bat_blk<B>(t, blockIdx.y, gridDim.y);
    if (bb.off) return;
    x = bat_at<B>(t, bb.cs, x);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n4; c += gridDim.x * blockDim.x)
        x[c] = make_float4(0.f, 0.f, 0.f, 0.f);
}

template <bool B>
__global__ void k_copy32x4(Bat t, int n4, float4* __restrict__ dst, const float4* __restrict__ src) {
    const BatBlk bb = bat_blk<B>(t, blockIdx.y, gridDim.y);
    if (bb.off) return;
    dst = bat_at<B>(t, bb.cs, dst);
    src = bat_at<B>(t, bb.cs, src);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n4; c += gridDim.x * blockDim.x)
        dst[c] = src[c];
}

// every case's scalars into the mapped host mirror, MIRROR_DOUBLES per case
__global__ void k_to_mirror_bat(Bat t, const double* __restrict__ s, double* __restrict__ h,
                                int n) {
    const int cs = t.zb ? (int)blockIdx.x : 0;
    s = bat_at<true>(t, cs, s);
    if ((int)threadIdx.x < n) h[(size_t)cs * MIRROR_DOUBLES + threadIdx.x] = s[threadIdx.x];
    __threadfence_system();
}

void finalize_dots_beta(vof_ctx* c, int nparts) {
    dim3 g(1);
    const Bat b = bat_of(c, g.x);
    auto kern = b.zb ? k_finalize_dots_beta<true> : k_finalize_dots_beta<false>;
    VOF_LAUNCH(c, kern, g, 1024, b, c->part + (size_t)S_RZ * MAX_PARTIALS,
               c->part + (size_t)S_ZQ * MAX_PARTIALS, nparts, c->scal);
}

void finalize_pq_alpha(vof_ctx* c, int nparts) {
    dim3 g(1);
    const Bat b = bat_of(c, g.x);
    auto kern = b.zb ? k_finalize_pq_alpha<true> : k_finalize_pq_alpha<false>;
    VOF_LAUNCH(c, kern, g, 1024, b, c->part + (size_t)S_PQ * MAX_PARTIALS, nparts,
               c->scal);
}

void finalize_sum(vof_ctx* c, int slot, int nparts, int dst, double scale) {
    dim3 g(1);
    const Bat b = bat_of(c, g.x);
    auto kern = b.zb ? k_finalize_sum<true> : k_finalize_sum<false>;
    VOF_LAUNCH(c, kern, g, 1024, b, c->part + (size_t)slot * MAX_PARTIALS, nparts,
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

void readback_async(vof_ctx* c) {
    if (c->hmirror_dev) {
        ++c->nlaunch;
        k_to_mirror<<<1, MIRROR_DOUBLES, 0, c->st>>>(c->scal, c->hmirror_dev, S_NSCALARS);
    } else {
        cudaMemcpyAsync(c->hbuf, c->scal, sizeof(double) * S_NSCALARS, cudaMemcpyDeviceToHost,
                        c->st);
    }
}

void readback(vof_ctx* c) {
    readback_async(c);
    cudaStreamSynchronize(c->st);
}

static int flat_blocks4(int n4) {
    int b = (n4 + 255) / 256;
    return b < 1 ? 1 : (b > 1184 ? 1184 : b);
}

void launch_zero32_bat(vof_ctx* c, float* x, int n) {
    dim3 g(flat_blocks4(n / 4));
    const Bat b = bat_of(c, g.y);
    auto kern = b.zb ? k_zero32x4<true> : k_zero32x4<false>;
    VOF_LAUNCH(c, kern, g, 256, b, n / 4, (float4*)x);
}

void launch_copy32_bat(vof_ctx* c, float* dst, const float* src, int n) {
    dim3 g(flat_blocks4(n / 4));
    const Bat b = bat_of(c, g.y);
    auto kern = b.zb ? k_copy32x4<true> : k_copy32x4<false>;
    VOF_LAUNCH(c, kern, g, 256, b, n / 4, (float4*)dst, (const float4*)src);
}

// mirror_dev: the device address of a mapped page-locked buffer of
// c->bat_n x MIRROR_DOUBLES doubles; every case's scalars, not only the
// running ones, then a wait on the stream
void readback_batch(vof_ctx* c, double* mirror_dev) {
    dim3 g(1);
    Bat b = bat_of(c, g.x);
    b.act = nullptr;
    VOF_LAUNCH(c, k_to_mirror_bat, g, MIRROR_DOUBLES, b, c->scal, mirror_dev, (int)S_NSCALARS);
    cudaStreamSynchronize(c->st);
}
