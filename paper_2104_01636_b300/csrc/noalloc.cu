// y = A x for the pressure operator without any device allocation.
//
// vof_apply_operator needs a context, and a context allocates its workspace
// with cudaMalloc. This variant is for callers that cannot allocate device
// memory: hosts that reserve all device memory up front in their own arena
// (a cudaMalloc would fail or break their accounting), and latency-critical
// loops where an allocation could synchronise the device. The scratch it
// needs -- the face coefficients beta built from alpha -- lives in one fixed
// file-scope device array instead. The kernels are those of the context
// path (k_beta, k_apply_A), so both entry points give the same bits.
#include <mutex>

#include "vof_internal.cuh"

// Face coefficients of one call (x, then y, then z faces), shared by all calls.
static __device__ __align__(256) double g_noalloc_beta[VOF_NOALLOC_MAX_FACES];

namespace {

// The array's device address is a property of the CUDA context that loaded
// the module, not of the device ordinal: after cudaDeviceReset, or with a
// context of the caller's own, the same ordinal has another address. The
// cache is therefore keyed on the context's unique id (cuCtxGetId, which
// never repeats within a process), looked up through the runtime's driver
// entry points so the library needs no link against the driver library.
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);

struct AddrEntry {
    unsigned long long ctx_id;
    double* addr;
};

std::mutex g_mu;
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
AddrEntry g_cache[64];
int g_ncache = 0;

bool driver_fns() {
    if (g_ctx_current && g_ctx_id) return true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
        return false;
    g_ctx_current = (CtxGetCurrentFn)p;
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess || !p)
        return false;
    g_ctx_id = (CtxGetIdFn)p;
    return true;
}

// Device address of the scratch in the current context. The first lookup in
// a context may load the library's module (cudaGetSymbolAddress), so the
// first call in each context must not happen inside a stream capture.
vof_status scratch_in_current_context(double** out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!driver_fns()) {
        cudaGetLastError();
        return VOF_ERR_CUDA;
    }
    void* ctx = nullptr;
    if (g_ctx_current(&ctx) != 0) return VOF_ERR_CUDA;
    if (!ctx) {  // no context current on this thread yet: make the device's primary one current
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess ||
            g_ctx_current(&ctx) != 0 || !ctx) {
            cudaGetLastError();
            return VOF_ERR_CUDA;
        }
    }
    unsigned long long id = 0;
    if (g_ctx_id(ctx, &id) != 0) return VOF_ERR_CUDA;
    for (int e = 0; e < g_ncache; ++e)
        if (g_cache[e].ctx_id == id) {
            *out = g_cache[e].addr;
            return VOF_OK;
        }
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_beta) != cudaSuccess || !p) {
        cudaGetLastError();
        return VOF_ERR_CUDA;
    }
    // keep the newest entries: a process that cycles through more than 64
    // contexts re-looks-up the oldest ones
    if (g_ncache == 64) {
        for (int e = 1; e < 64; ++e) g_cache[e - 1] = g_cache[e];
        g_ncache = 63;
    }
    g_cache[g_ncache++] = {id, (double*)p};
    *out = (double*)p;
    return VOF_OK;
}

}  // namespace

extern "C" vof_status vof_apply_operator_noalloc(const vof_grid* grid, const vof_phys* phys,
                                                 const double* alpha, const double* x, double* y,
                                                 void* stream) {
    if (!alpha || !x || !y) return VOF_ERR_ARG;
    std::string why;
    if (!grid_ok(grid, why) || !phys_ok(phys)) return VOF_ERR_ARG;  // the checks of vof_create
    if (grid->periodic_x || grid->periodic_y) return VOF_ERR_UNSUPPORTED;
    const size_t nu = (size_t)(grid->nx + 1) * grid->ny * grid->nz;
    const size_t nv = (size_t)grid->nx * (grid->ny + 1) * grid->nz;
    const size_t nw = (size_t)grid->nx * grid->ny * grid->nz;
    if (nu + nv + nw > (size_t)VOF_NOALLOC_MAX_FACES) return VOF_ERR_ADMISSION;
    double* beta = nullptr;
    vof_status st = scratch_in_current_context(&beta);
    if (st != VOF_OK) return st;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return VOF_ERR_CUDA;
    }
    launch_beta_apply_raw(grid, phys, alpha, x, y, beta, beta + nu, beta + nu + nv, sms,
                          (cudaStream_t)stream);
    if (cudaGetLastError() != cudaSuccess) return VOF_ERR_CUDA;
    return VOF_OK;
}
