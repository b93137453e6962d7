// Internal declarations shared by the CUDA translation units of the library.
// Layout conventions are those of include/vof.h (x fastest, staggered faces,
// walls in x and y, periodic z).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/vof.h"

// ---------------------------------------------------------------------------
// launch geometry: 2-D thread tiles in (x, y) marching over a chunk of z
// planes, so every cell kernel has a bounded, SM-count-sized grid and
// per-block partial sums stay few enough for a one-block finalise.
// ---------------------------------------------------------------------------
constexpr int TBX = 32;
constexpr int TBY = 8;
constexpr int TB = TBX * TBY;
constexpr int MAX_PARTIALS = 4096;  // per reduction slot
constexpr int MIRROR_DOUBLES = 64;  // host mirror of the device scalars
constexpr int NSLOTS = 24;          // reduction slots in the partials buffer

struct Dims {
    int nx, ny, nz;
};

struct Launch {
    dim3 grid, block;
    int kchunk;
    int nblocks;
};

Launch launch_cells(int nx, int ny, int nz, int sm_count);

// every kernel launch of the library goes through this macro so the context
// can report how many of its kernels ran
#define VOF_LAUNCH(c, kernel, grid, block, ...)                \
    do {                                                       \
        ++(c)->nlaunch;                                        \
        kernel<<<(grid), (block), 0, (c)->st>>>(__VA_ARGS__);  \
    } while (0)

// index helpers (int32: vof_create rejects grids whose face counts overflow)
__host__ __device__ __forceinline__ int wrapk(int k, int nz) {
    return k < 0 ? k + nz : (k >= nz ? k - nz : k);
}
__host__ __device__ __forceinline__ int cid(const Dims& d, int i, int j, int k) {
    return i + d.nx * (j + d.ny * k);
}
__host__ __device__ __forceinline__ int uid(const Dims& d, int i, int j, int k) {
    return i + (d.nx + 1) * (j + d.ny * k);
}
__host__ __device__ __forceinline__ int vid(const Dims& d, int i, int j, int k) {
    return i + d.nx * (j + (d.ny + 1) * k);
}
__host__ __device__ __forceinline__ int wid(const Dims& d, int i, int j, int k) {
    return i + d.nx * (j + d.ny * k);
}

// Deterministic block sum (fixed shuffle tree, then fixed warp order).
// Every thread of the block must call it; the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh_bs[32];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) sh_bs[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
        v = tid < (nthreads + 31) / 32 ? sh_bs[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    __syncthreads();
    return v;
}
// the sum of n block partials by one block, in k_finalize_sum's order
// (every thread calls it; the result is valid in thread 0)
__device__ __forceinline__ double sum_partials(const double* __restrict__ part, int n) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    return block_sum(s);
}
__device__ __forceinline__ double block_max(double v) {
    __shared__ double sh_bm[32];
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    const int nthreads = blockDim.x * blockDim.y * blockDim.z;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((tid & 31) == 0) sh_bm[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
        v = tid < (nthreads + 31) / 32 ? sh_bm[tid] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    }
    __syncthreads();
    return v;
}
__device__ __forceinline__ int block_linear() {
    return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
}

// ---------------------------------------------------------------------------
// Batched launches: one launch runs a kernel of the pressure solve for every
// case of an ensemble. The cases' workspaces are carved from one arena at a
// fixed stride, so case c's arrays are case 0's moved by c * stride bytes. A
// batched launch repeats the solo grid once per case along one axis (z for
// the cell kernels, y for the flat vector kernels, x for the one-block
// finalisers); each block finds its case, its block index in the solo grid
// and its arrays from the Bat argument, so every case runs the blocks, and
// sums in the order, of its solo launch. A solo launch passes Bat{}.
// ---------------------------------------------------------------------------
struct Bat {
    int zb = 0;                // solo grid extent along the batched axis (0: a solo launch)
    long long stride = 0;      // bytes between consecutive cases' workspaces
    const int* act = nullptr;  // per case: 0 once its solve has finished (its blocks return)
};
struct BatBlk {
    int cs;    // the block's case
    int b;     // its index along the batched axis in the solo grid
    int g;     // the solo grid's extent along that axis
    bool off;  // its case has finished
};
// B: the kernel was instantiated for batched launches; the solo instantiation
// (B = false) compiles to the unbatched code
template <bool B>
__device__ __forceinline__ BatBlk bat_blk(const Bat& t, unsigned idx, unsigned dim) {
    BatBlk r;
    if (!B) {
        r.cs = 0;
        r.b = (int)idx;
        r.g = (int)dim;
        r.off = false;
        return r;
    }
    if (t.zb) {
        r.cs = (int)(idx / (unsigned)t.zb);
        r.b = (int)idx - r.cs * t.zb;
        r.g = t.zb;
    } else {
        r.cs = 0;
        r.b = (int)idx;
        r.g = (int)dim;
    }
    r.off = t.act != nullptr && t.act[r.cs] == 0;
    return r;
}
// the case's copy of a workspace array
template <bool B, class T>
__device__ __forceinline__ T* bat_at(const Bat& t, int cs, T* p) {
    if (!B) return p;
    return t.zb ? (T*)((const char*)p + (long long)cs * t.stride) : p;
}
// block_linear() of the solo grid, for a grid batched along z
__device__ __forceinline__ int block_linear_z(const BatBlk& bb) {
    return blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * bb.b);
}

// ---------------------------------------------------------------------------
// timing classes (CUDA events on the context stream, when enabled)
// ---------------------------------------------------------------------------
enum TimerClass {
    T_ADVECT = 0, T_SSF, T_PREDICT, T_RHS, T_SMOOTH0, T_SMOOTH, T_RESIDUAL, T_RESTRICT0,
    T_RESTRICT, T_PROLONG0, T_PROLONG, T_COARSE, T_KRYLOV, T_PROJECT, T_NCLASS
};

// ---------------------------------------------------------------------------
// multigrid level
// ---------------------------------------------------------------------------
struct Level {
    int idx = 0;  // 0 = fine grid
    Dims d;
    double h;
    int ncells;
    double *bx = nullptr, *by = nullptr, *bz = nullptr;  // face coefficients
    double *x = nullptr, *f = nullptr;                    // correction / right side
    float *bxf = nullptr, *byf = nullptr, *bzf = nullptr;  // FP32 copies (mixed)
    float *xf = nullptr, *ff = nullptr;
    // FP16 copies of the FP32 coefficients, read by the colour passes and
    // the restriction of a large coarse level (mixed cycle; see HALF_COEF_MIN_CELLS)
    __half *bxh = nullptr, *byh = nullptr, *bzh = nullptr;
    float hscale = 1.f;  // the FP16 copies hold beta / hscale (a power of two)
    void* rs = nullptr;  // residual scratch for full-weighting restriction (T per cell)
    void* rho = nullptr; // cell density (T per cell), levels >= 1 with density coarsening
    Launch L;
    // launch shape of the colour passes: a tiled pass takes pass_kchunk z
    // planes per thread (0: a quarter of L.kchunk), a narrow level's 1-D
    // blocks pass_block threads, and the 1-D restriction from it
    // restrict_block threads (mg_tune_shapes, vof_mg_set_shape; every shape
    // computes the same cells the same way)
    int pass_kchunk = 0;
    int pass_block = 256;
    int restrict_block = 256;
    bool tuned = false;
};

// ---------------------------------------------------------------------------
// coarse tail of the mixed cycle in one cluster launch (k_mg_tail.cu): the
// operations of the cycle from level tail_level down, as a program
// ---------------------------------------------------------------------------
// A coarse level of the mixed cycle with at least this many cells (and an
// even nx, constant prolongation) smooths and restricts with FP16 copies of
// its face coefficients: two thirds of a colour pass's bytes are
// coefficients, and from about 2^18 cells up the pass moves enough of them
// for the saving to show. Smaller levels are bound by latency and keep FP32,
// so the one-launch coarse tail (at most TAIL_MAX_CELLS) never sees them.
constexpr int HALF_COEF_MIN_CELLS = 1 << 18;
constexpr int TAIL_MAX_LEVELS = 16;
constexpr int TAIL_MAX_OPS = 256;
constexpr int TAIL_MAX_CELLS = 8192;  // largest level the cluster tail starts from
constexpr int TAIL_GRID_MAX_CELLS = 1 << 17;  // largest level the grid-wide tail starts from
enum TailKind { TAIL_SMOOTH = 0, TAIL_RESTRICT = 1, TAIL_DENSE = 2 };
struct TailLevel {
    Dims d;
    float h2, ih2;  // h^2 (smoother), 1/h^2 (restriction)
    const float *bx, *by, *bz;
    float *x, *f;
};
struct TailOp {
    unsigned char kind, lev, color, mode;  // lev: index relative to the tail level
};
struct alignas(16) TailProg {
    TailLevel L[TAIL_MAX_LEVELS];
    TailOp op[TAIL_MAX_OPS];
    int nops;
    float omega;
};

struct vof_ctx {
    vof_grid g;
    vof_phys ph;
    vof_solver sv;
    Dims d;
    cudaStream_t st = nullptr;
    int dev = 0;
    int sm_count = 148;
    size_t bytes = 0;
    std::vector<void*> allocs;
    Launch Lc;  // fine-grid cell launch

    // fine-grid workspace
    double *bx = nullptr, *by = nullptr, *bz = nullptr;    // beta on faces
    double *sx = nullptr, *sy = nullptr, *sz = nullptr;    // surface force (step)
    double *kappa = nullptr;                               // curvature (step)
    unsigned char *valid = nullptr, *cmask = nullptr, *has = nullptr;
    int* if_list = nullptr;   // interface cells of the current sweep
    int* if_count = nullptr;  // their number (device), then per plane-constant piece: counts, cursors
    int* if_perm = nullptr;   // the listed cells with a plane, ordered by piece
    unsigned char* if_piece = nullptr;  // per list entry: its piece (255: no plane)
    double *plane = nullptr;  // 4 per cell: n[3], d
    double *fx = nullptr, *fy = nullptr, *fz = nullptr;  // liquid fluxes / face accelerations
    double *uh[3] = {nullptr, nullptr, nullptr};          // cell intermediate velocity
    double *a1 = nullptr, *a2 = nullptr, *an = nullptr;  // alpha scratch
    double *b = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr;
    double* rhs = nullptr;  // assembled right side of the projection
    float *e32 = nullptr, *p32 = nullptr, *q32 = nullptr;  // inner FP32 Krylov (mixed)
    std::vector<Level> lv;
    double* coarse_scratch = nullptr;
    // dense inverse of the coarsest level (when it has <= DENSE_MAX cells)
    int dense_n = 0;
    double dense_shift = 0.0;  // s n / (1/h^2): regularising shift of the constants
    double *dense_a = nullptr, *dense_b = nullptr, *dense_inv = nullptr;
    float* dense_inv_f = nullptr;
    void* dense_w = nullptr;  // blocked Gauss-Jordan panels: 32x32 + 2 x 32 n entries

    double* part = nullptr;  // NSLOTS x MAX_PARTIALS block partials
    double* scal = nullptr;  // device scalars
    // host mirror of scal: a mapped page-locked slot (hmirror_dev its device
    // address), else hbuf_store
    double* hbuf = nullptr;
    double* hmirror_dev = nullptr;
    std::vector<double> hbuf_store = std::vector<double>(MIRROR_DOUBLES, 0.0);
    int* dflag = nullptr;    // device error flags

    // timing
    int timing = 0;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<int, int>>> ev_marks;  // class, (start, stop)
    double t_ms[T_NCLASS] = {0};
    long long t_n[T_NCLASS] = {0};

    // finest level of the mixed V-cycle with density-formed coefficients
    // (k_smooth_tma.cu): FP32 and FP16 density, second x buffer, TMA maps of
    // x (level-0 xf), x32b and rho16
    // mixed: FP32 cell velocities and alpha^n (viscous term of the predictor)
    float* u32[4] = {nullptr, nullptr, nullptr, nullptr};
    double *ptilde = nullptr, *pflow = nullptr;   // two-solve mode: p~ (kept) and p
    bool use_rho = false;
    float* rho32 = nullptr;   // also the mixed path's density for density coarsening
    void* rho16 = nullptr;    // FP16 density of the V-cycle's finest level (__half)
    double* rho64 = nullptr;  // FP64 path: finest-level density for density coarsening
    float* x32b = nullptr;
    int sweep_kchunk = 1;
    bool sweep_dot = false;  // the V-cycle's last sweep forms the Krylov dots
    alignas(64) unsigned char tmap[3][128];

    // the V-cycle captured once as a CUDA graph and replayed (state 0: not
    // tried yet, 1: ready, -1: capture unavailable, e.g. the legacy stream)
    cudaGraphExec_t vgraph = nullptr;
    long long vgraph_kernels = 0;
    int vgraph_state = 0;

    // the mixed solve captured once as a CUDA graph whose loops are
    // conditional WHILE nodes driven by device-side control kernels (state
    // 0: not tried, 1: ready, -1: unavailable); rebuilt when the right side
    // or the solution pointer changes
    // (two cached graphs: the two-solve mode alternates its solution pointer)
    struct SolveGraph {
        cudaGraphExec_t exec = nullptr;
        const double* b = nullptr;
        double* P = nullptr;
        long long k_fixed = 0, k_outer = 0, k_inner = 0;  // kernels per solve
        long long used = 0;
    } sgraph[2];
    long long sgraph_clock = 0;
    int sgraph_state = 0;
    cudaStream_t cap_st[2] = {nullptr, nullptr};  // streams capturing the loop bodies
    bool in_solve_capture = false;

    // coarse tail (0: not used); programs from zero / from the current x
    int tail_level = 0;
    int tail_cluster = 0;  // CTAs of the cluster tail, or 0
    int tail_grid = 0;     // blocks of the grid-wide tail (one per SM), or 0
    unsigned* tail_bar = nullptr;  // its barrier counter
    TailProg* tail_prog = nullptr;  // device copies of tail_host
    TailProg tail_host[2];

    // vof_step_host: the state on the device (alpha, uc, vc, wc, u, v, w, p),
    // allocated at the first call; a stream that copies it in and one that
    // copies it out beside the context stream, and the events ordering them
    double* hs[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaStream_t io_st[2] = {nullptr, nullptr};  // host to device, device to host
    cudaEvent_t io_ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t io_d2h[8] = {nullptr, nullptr, nullptr, nullptr,
                             nullptr, nullptr, nullptr, nullptr};  // last copy out, per field

    long long nlaunch = 0;  // kernels launched by this context
    std::string err;

    // workspace carved from an arena owned by an ensemble (nullptr: the
    // stream-ordered allocator); the ensemble's batched solve launches
    // through case 0's context with bat_n cases at bat_stride bytes apart
    char* arena = nullptr;
    size_t arena_size = 0, arena_used = 0;
    int bat_n = 1;
    long long bat_stride = 0;
    const int* bat_act = nullptr;
    bool defer_dense = false;  // the batched solve forms the dense coarsest inverse
};

// The batch of the context's launches: Bat{} for a single case; otherwise
// the grid extent axis_blocks is multiplied by the number of cases.
inline Bat bat_of(const vof_ctx* c, unsigned& axis_blocks) {
    Bat b;
    if (c->bat_n <= 1) return b;
    b.zb = (int)axis_blocks;
    b.stride = c->bat_stride;
    b.act = c->bat_act;
    axis_blocks *= (unsigned)c->bat_n;
    return b;
}

// ---------------------------------------------------------------------------
// programmatic dependent launch: a kernel launched by launch_pdl is set up
// while the previous kernel on the stream runs, and its blocks start as that
// kernel completes, which shortens the gap between the small kernels of the
// coarse multigrid levels. Such a kernel calls pdl_wait() before it touches
// global memory: it returns once the previous grid has completed and its
// writes are visible (at once for a kernel launched the ordinary way).
// Measured with an early trigger (griddepcontrol.launch_dependents at the
// top of each kernel) the step was slower: the waiting blocks held SM slots.
// The programmatic edges are kept inside the conditional bodies of the
// captured mixed solve as well.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class... KArgs, class... Args>
void launch_pdl(vof_ctx* c, void (*kern)(KArgs...), dim3 grid, dim3 block, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = c->st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    ++c->nlaunch;
    cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// scalar slots in ctx->scal
enum ScalarSlot {
    S_RR = 0,     // ||r||^2
    S_BB,         // ||b||^2
    S_PQ,         // p.q
    S_RZ,         // r.z
    S_ZQ,         // z.q
    S_ALPHA,      // CG step length
    S_BETA,       // CG direction update
    S_MEAN,       // mean removed
    S_VOL0, S_VOL1, S_CLIP0, S_CLIP1, S_CLIP2, S_MAXDIV, S_MAXU, S_FALLBACK, S_CFL, S_SUM,
    S_ERR,        // a kernel gave up a bounded wait (set to 1)
    // device-side control of the captured mixed solve (solver.cu)
    S_INNER, S_OUTER, S_RES, S_RES0, S_BNORM, S_THR, S_CAP, S_CONV, S_STATUS, S_ZERO, S_GUARD,
    // the same for each case of a batched solve captured whole: whether the
    // case takes part in the current refinement and in the inner loop
    S_OUTACT, S_INACT,
    S_NSCALARS
};
static_assert(S_NSCALARS <= MIRROR_DOUBLES, "the host mirror holds every device scalar");

// ---------------------------------------------------------------------------
// helpers implemented in capi.cu
// ---------------------------------------------------------------------------
vof_status set_err(vof_ctx* c, vof_status s, const std::string& msg);
void* dev_alloc(vof_ctx* c, size_t bytes);  // stream-ordered, freed by vof_destroy
vof_status cuda_check(vof_ctx* c, cudaError_t e, const char* what);
vof_status launch_check(vof_ctx* c, const char* what);
int timer_begin(vof_ctx* c, int cls);
void timer_end(vof_ctx* c, int cls, int mark);

// reductions (k_common.cu): sum / max of the block partials of slot into scal[dst]
// the device scalars into c->hbuf, then a wait on the context stream
void readback(vof_ctx* c);
// the same without the wait: c->hbuf is valid once the stream has reached it
void readback_async(vof_ctx* c);
double* mirror_acquire();
void mirror_release(double* p);
void finalize_sum(vof_ctx* c, int slot, int nparts, int dst, double scale);
// the inner FP32 CG's scalars with their reductions, one launch each:
// (z, r) -> S_RZ and (z, q) -> S_ZQ from the partials in slots S_RZ, S_ZQ,
// then beta; (p, q) -> S_PQ from slot S_PQ, then alpha
void finalize_dots_beta(vof_ctx* c, int nparts);
void finalize_pq_alpha(vof_ctx* c, int nparts);
void finalize_max(vof_ctx* c, int slot, int nparts, int dst);

// ---------------------------------------------------------------------------
// kernel launch wrappers
// ---------------------------------------------------------------------------
// poisson (k_poisson.cu)
void launch_beta(vof_ctx* c, const double* alpha);
// the face coefficients from alpha into caller-given storage, then y = A x
// with them: the kernels of launch_beta and launch_apply_A, without a context
void launch_beta_apply_raw(const vof_grid* g, const vof_phys* ph, const double* alpha,
                           const double* x, double* y, double* bx, double* by, double* bz,
                           int sm_count, cudaStream_t s);
// argument checks of vof_create for the grid and the physical properties
bool grid_ok(const vof_grid* g, std::string& why);
bool phys_ok(const vof_phys* p);
void launch_apply_A(vof_ctx* c, const Level& l, const double* x, double* y);
void launch_residual(vof_ctx* c, const Level& l, const double* x, const double* f, double* r,
                     int slot);
void launch_dot(vof_ctx* c, const double* x, const double* y, int n, int slot);
void launch_sub_mean(vof_ctx* c, double* x, int n, int slot_mean);
void launch_copy(vof_ctx* c, double* dst, const double* src, int n);
void launch_zero(vof_ctx* c, double* x, int n);
void launch_apply_A_dot(vof_ctx* c, const Level& l, const double* p, double* q, int slot);
void launch_cg_update(vof_ctx* c, int n, double* x, double* r, const double* p, const double* q,
                      int slot);
void launch_dot2(vof_ctx* c, int n, const double* z, const double* r, const double* q, int slot_a,
                 int slot_b);
void launch_p_update(vof_ctx* c, int n, double* p, const double* z);
void launch_scalar_alpha(vof_ctx* c);
void launch_scalar_beta(vof_ctx* c);

// multigrid (k_mg.cu), T = double (FP64 path) or float (mixed path)
// one red-black colour pass; mode 1: the first pass from a zero x, mode 2:
// the first pass after the coarse correction from level *coarse (folds in
// the prolongation)
template <class T> void mg_rbgs(vof_ctx* c, const Level& L, int color, int mode = 0,
                                const Level* coarse = nullptr);
template <class T> void mg_restrict(vof_ctx* c, const Level& fine, const Level& coarse);
template <class T> void mg_prolong(vof_ctx* c, const Level& coarse, const Level& fine);
template <class T> void mg_coarsen_beta(vof_ctx* c, const Level& fine, const Level& coarse);
template <class T> void mg_coarse(vof_ctx* c, const Level& L);
template <class T> void mg_zero(vof_ctx* c, const Level& L);
template <class T> void mg_dense_setup(vof_ctx* c, const Level& L);
// density coarsening: rho_c = mean of the eight children, faces 2 / (rho_L + rho_R)
template <class T> void mg_coarsen_density(vof_ctx* c, const T* rho_fine, const Level& fine,
                                           const Level& coarse);
constexpr int DENSE_MAX = 1536;  // largest coarsest level solved by the dense inverse
// The mixed solve's inner FP32 tolerance for a refinement that starts from
// relative residual res: max(INNER_TOL_FLOOR, 0.2 rtol / res) of its initial
// residual (the floor keeps the FP32 iteration above its rounding level)
constexpr double INNER_TOL_FLOOR = 1e-5;
void mg_to_f32(vof_ctx* c, const double* a, float* b, int n);
// inner FP32 Krylov of the mixed solve (k_mg.cu) and its FP64 residual (k_poisson.cu)
void k32_apply_A_dot(vof_ctx* c, const float* p, float* q, int slot);
// returns the number of block partials of (r, r) in slot; finalize false
// leaves their sum to the caller
int k32_cg_update(vof_ctx* c, int n, float* e, float* r, const float* p, const float* q, int slot,
                  bool finalize = true);
// (z, r) -> S_RZ, (z, q) -> S_ZQ and beta (finalize_dots_beta)
void k32_dot2(vof_ctx* c, int n, const float* z, const float* r, const float* q);
void k32_p_update(vof_ctx* c, int n, float* p, const float* z);
void k32_add_to_f64(vof_ctx* c, int n, const float* e, double* x);
void launch_residual_to32(vof_ctx* c, const double* x, const double* f, float* r32, int slot);
void mg_to_f64(vof_ctx* c, const float* a, double* b, int n);

// finest level of the mixed V-cycle from the cell density (k_smooth_tma.cu)
bool rho_path_eligible(const vof_grid* g, const vof_solver* sv, int nlevels);
vof_status rho_path_setup(vof_ctx* c);
vof_status rho_path_batch_maps(vof_ctx* c, int nc, long long case_stride);
void rho_sweep(vof_ctx* c, const float* src, float* dst, int c0, bool dot = false);
// one block waiting out a bounded wait on a barrier nothing completes
void wait_probe(vof_ctx* c, int limit);
void rho_restrict(vof_ctx* c);
void rho_apply_A_dot(vof_ctx* c, const float* p, float* q, int slot);
void mg_coarsen_beta_from64(vof_ctx* c, const Level& fine, const Level& coarse);
// FP16 copies of the FP32 coefficients of the levels that carry them
void mg_half_coefficients(vof_ctx* c);
// times the candidate launch shapes of the coarse levels' colour passes and
// narrow restrictions as launched for nb cases (nb > 1: the batched solve
// through this context, cases `stride` bytes apart, act_d their flags) and
// keeps the fastest in the levels; fills the levels' arrays with finite
// values first (the solve writes them before it reads them)
vof_status mg_tune_shapes(vof_ctx* c, int nb, long long stride, int* act_d);
// vof_mg_shape / vof_mg_set_shape for a context
vof_status mg_shape_of(const vof_ctx* c, int level, int shape[4]);
vof_status mg_set_shape(vof_ctx* c, int level, const int shape[3]);
// z planes per thread of a tiled colour pass of level L
int pass_kchunk_of(const Level& L);

// coarse tail (k_mg_tail.cu)
vof_status mg_tail_setup(vof_ctx* c, int level, const TailProg* from_zero, const TailProg* from_x,
                         bool grid);
void mg_tail_run(vof_ctx* c, bool zero_start);

// vof (k_vof.cu)
void launch_vof_mask_volume(vof_ctx* c, const double* alpha, int slot);
void launch_reconstruct(vof_ctx* c, const double* alpha);
void launch_face_flux(vof_ctx* c, int dir, const double* alpha, const double* vel, double dt,
                      double* flux);
void launch_vof_update(vof_ctx* c, int dir, const double* ain, double* aout, const double* vel,
                       const double* flux, double dt, int slot);
void launch_cfl(vof_ctx* c, const double* u, const double* v, const double* w, double dt, int slot);
void launch_volume(vof_ctx* c, const double* alpha, int slot);

// curvature and surface force (k_ssf.cu)
void launch_curvature(vof_ctx* c, const double* alpha, double* kappa, unsigned char* valid);
void launch_ssf_faces(vof_ctx* c, const double* alpha, const double* kappa,
                      const unsigned char* valid, double* sx, double* sy, double* sz, int slot);

// momentum (k_momentum.cu)
void launch_predict(vof_ctx* c, const double* alpha_n, const double* alpha_np1,
                    const double* const U[3], const double* u, const double* v, const double* w,
                    const double* fx, const double* fy, const double* fz, double dt,
                    double* const out[3]);
void launch_cell_to_face(vof_ctx* c, const double* uc, const double* vc, const double* wc,
                         double* u, double* v, double* w);

// projection (k_project.cu)
void launch_rhs(vof_ctx* c, const double* u, const double* v, const double* w, const double* sx,
                const double* sy, const double* sz, double dt, double* b, int slot);
void launch_lincomb(vof_ctx* c, int n, double a, const double* x, double b, const double* y,
                    double* out);  // out = a x + b y
void launch_correct(vof_ctx* c, const double* P, const double* sx, const double* sy,
                    const double* sz, double dt, const double* const Uh[3], double* const Uc[3],
                    double* u, double* v, double* w, int slot_div, int slot_u);

// solver driver (solver.cu)
vof_status solve_pressure(vof_ctx* c, const double* b_in, double* P, vof_report* rep);
// the mixed solve's setup (coefficients, mean-free b, its norm, the first
// FP64 residual into the scalars), as solve_pressure launches it
void solve_setup_mixed(vof_ctx* c, const double* b_in, double* P);
// the mixed solves of nc cases whose contexts were carved from one arena at
// stride bytes apart, launched through case 0's context m after every case's
// solve_setup_mixed (P: the contexts' c->p); run[i] = 0 leaves case i out.
// Per case: its status and its report's iters, refinements, res0, res, b_mean.
struct BatchSolveState;
vof_status solve_mixed_batch(vof_ctx* m, int nc, long long stride, const int* run,
                             BatchSolveState* bs, vof_status* status, vof_report* reps,
                             vof_ctx* const* cases);
BatchSolveState* batch_solve_create(vof_ctx* m, int nc, long long stride);
void batch_solve_destroy(BatchSolveState* bs);
// mg_tune_shapes for the batched launches of bs's cases through m
vof_status batch_solve_tune(vof_ctx* m, BatchSolveState* bs, long long stride);
// whether the batched solve supports contexts made with this solver
bool batch_solve_eligible(const vof_ctx* c);
// step_pre in two parts: the CFL reduction and its readback, launched without
// a wait, then (once the stream has finished them) its test and the rest
vof_status step_pre_cfl(vof_ctx* c, double* const f[8], double dt);
vof_status step_pre(vof_ctx* c, double* const f[8], double dt, long long step_index);
vof_status step_post(vof_ctx* c, double* const f[8], double dt, vof_status solve);
vof_status step_post_report(vof_ctx* c, vof_status solve, vof_report* report);
// step_pre's launches after its CFL test (the test taken elsewhere)
vof_status step_pre_launch(vof_ctx* c, double* const f[8], double dt, long long step_index);
// Captures, on m->st (which must be capturing), the batched mixed solve of
// nc cases whose setups have been captured before it: the dense coarsest
// inverses, then the loops of solve_mixed_batch as two nested conditional
// WHILE nodes whose per-case decisions are taken on the device. Each case's
// outcome is left in its scalars (S_INNER, S_OUTER, S_RES0, S_RES, S_CONV,
// S_STATUS, S_ZERO); the kernels launched per pass of the outer and inner
// loop bodies and the rest are counted into k[0..2] (rest, outer, inner).
// False when capture or conditional nodes are unavailable.
bool capture_solve_mixed_batch(vof_ctx* m, int nc, long long stride, BatchSolveState* bs,
                               long long k[3]);
// the outcome of case c's captured batched solve, from its scalars as the
// host mirror holds them after the step: report fields and status
vof_status captured_case_result(vof_ctx* c, vof_report* rep);
// passes of the two loop bodies in the last replay of that capture
void batch_solve_trips(const BatchSolveState* bs, long long* outer, long long* inner);
// after a captured batched solve, on case c's stream: P = 0 for a zero
// right side, then P made mean-free (the end of solve_mixed's graph)
void solve_tail_captured(vof_ctx* c);
// a conditional IF node on handle h after the work captured so far on s;
// later captures on s follow the node; returns its body graph (nullptr on
// failure)
cudaGraph_t capture_if(cudaStream_t s, cudaGraphConditionalHandle h);
// the graph being captured on s (nullptr when s is not capturing)
cudaGraph_t capture_graph_of(cudaStream_t s);
void launch_zero32_bat(vof_ctx* c, float* x, int n);                 // x = 0 (batched, masked)
void launch_copy32_bat(vof_ctx* c, float* dst, const float* src, int n);  // dst = src
void readback_batch(vof_ctx* c, double* mirror_dev);  // every case's scalars, then a wait
// the whole time step (the body of the exported step/vof_step); the
// library's own callers use this name, which no system library exports
vof_status step_entry(vof_ctx* c, double* alpha, double* uc, double* vc, double* wc, double* u,
                      double* v, double* w, double* p, double dt, long long step_index,
                      vof_report* report);
size_t mg_workspace_bytes(const vof_grid* g, const vof_solver* sv, int* nlevels);
// a context whose workspace comes from [arena, arena + arena_bytes) (capi.cu)
vof_status create_in_arena(const vof_grid* grid, const vof_phys* phys, const vof_solver* solver,
                           void* stream, void* arena, size_t arena_bytes, vof_ctx** out);
size_t workspace_bytes(const vof_grid* g, const vof_solver* sv);
vof_status mg_allocate(vof_ctx* c);
void mg_build_coefficients(vof_ctx* c);
