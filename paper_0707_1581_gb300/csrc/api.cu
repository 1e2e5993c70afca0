// api.cu -- host runtime and C ABI of the library (declared in include/flb.h).
//
// A context owns one or more boxes, their device buffers, a stream, the FP64
// statistics accumulators and (optionally) captured CUDA graphs of the time
// step.  All arithmetic of the method runs in the kernels; this file only
// validates parameters, derives the per-mode constants of the collision,
// allocates, launches and copies.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "flb.h"
#include "d2q9.cuh"
#include "diag_kernels.cuh"
#include "kernels.cuh"

using namespace flb;

namespace {

std::mutex g_create_err_mu;
std::string g_create_err;

size_t store_size(int store)
{
    switch (store) {
    case FLB_STORE_F64: return 8;
    case FLB_STORE_F32: return 4;
    case FLB_STORE_F16DEV:
    case FLB_STORE_BF16DEV:
    case FLB_STORE_BF16SR: return 2;
    }
    return 0;
}

struct Box {
    flb_config cfg;
    int Q = flb::Q;         // populations per site: 19 (D3Q19) or 9 (D2Q9)
    int64_t N = 0;          // sites
    int64_t plane = 0;      // elements between population planes (N rounded up to 64)
    void *buf[2] = {nullptr, nullptr};
    CollideConsts<float> Kf;
    CollideConsts<double> Kd;
    d2::CollideConsts<float> K2f;
    d2::CollideConsts<double> K2d;
    double *d_acc = nullptr;        // kAccWidth accumulators
    double *d_partial = nullptr;    // stats partials
    int stats_nb = 0;
    // structure factor (enabled when d_rho is set)
    void *d_rho = nullptr;                  // rho - rho0 per site, transform type
    void *d_X = nullptr;                    // half spectrum
    void *d_tw = nullptr;                   // twiddles
    uint16_t *d_shell_tab = nullptr;        // shell of every wave vector
    unsigned long long *d_sq_fixed = nullptr;   // nshells fixed-point sums of one sample, then the max word
    double *d_shell = nullptr;              // FP64 shell sums
    unsigned long long *d_count = nullptr;  // wave vectors per shell (fixed)
    std::vector<unsigned long long> count;  // the same on the host
    int nshells = 0;
    int sq_P = 0;                           // row stride of the half spectrum
    uint64_t sq_samples = 0;                // S(q) samples since the last reset
};

}  // namespace

// Device allocator of a context: the process-wide hook in effect when it was
// created (flb_set_device_allocator), else cudaMalloc / cudaFree.
struct DevAllocator {
    flb_dev_alloc_fn alloc = nullptr;
    flb_dev_free_fn free = nullptr;
    void *user = nullptr;
};

struct flb_ctx {
    DevAllocator A;
    std::vector<Box> boxes;
    int store = FLB_STORE_F32;
    int pattern = FLB_PATTERN_AB;
    int lattice = FLB_LATTICE_D3Q19;
    uint64_t step = 0;
    int cur = 0;                    // AB: buffer holding the current state
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Launch L;
    int graph_steps = 0;
    int64_t stats_every = 0;        // automatic statistics sample period (0: off)
    uint32_t *d_step = nullptr;
    void *d_bm = nullptr;           // FP64 Box-Muller tables (FP64 contexts)
    unsigned long long *d_viol = nullptr;   // bounds violations (checking build only)
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};   // by starting orientation
    // batched launch: per orientation, chunks of a BatchParams<S> (box table
    // passed as a kernel parameter) and the blocks each chunk launches
    struct Chunk {
        std::vector<unsigned char> params;
        int blocks = 0;
    };
    std::vector<Chunk> batch[2];
    bool noise = false, force = false;
    bool kin0 = true;               // every box has gamma_ghost = 0
    double *d_scratch = nullptr;    // canonical gather / moments staging
    size_t scratch_bytes = 0;
    // host-resident stepping: copy streams and per-chunk events
    cudaStream_t s_up = nullptr, s_down = nullptr;
    std::vector<cudaEvent_t> ev_up, ev_comp;
    cudaEvent_t ev_entry = nullptr, ev_done = nullptr;
    std::string err;
};

namespace {

// An NVTX range over a scope (header-only NVTX 3: a no-op unless a profiler
// is attached), so that timelines show the library's calls and graph replays.
struct NvtxRange {
    explicit NvtxRange(const char *m) { nvtxRangePushA(m); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

std::mutex g_alloc_mu;
DevAllocator g_alloc;

// Device memory of context c, through its allocator, ordered on its stream.
template <class T>
cudaError_t dev_malloc(flb_ctx *c, T **p, size_t bytes)
{
    if (c->A.alloc) {
        void *q = c->A.alloc(bytes, c->stream, c->A.user);
        *p = static_cast<T *>(q);
        return q ? cudaSuccess : cudaErrorMemoryAllocation;
    }
    void *q = nullptr;
    const cudaError_t e = cudaMalloc(&q, bytes);
    *p = static_cast<T *>(q);
    return e;
}

void dev_free(flb_ctx *c, void *p)
{
    if (!p) return;
    if (c->A.free) c->A.free(p, c->stream, c->A.user);
    else cudaFree(p);
}

int fail(flb_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    return code;
}

int cuda_fail(flb_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, FLB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(ctx, expr)                                                                                               \
    do {                                                                                                            \
        cudaError_t e_ = (expr);                                                                                    \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #expr);                                                  \
    } while (0)

void set_create_error(const std::string &m)
{
    std::lock_guard<std::mutex> lk(g_create_err_mu);
    g_create_err = m;
}

int validate(const flb_config &c, std::string &why)
{
    char b[256];
    if (c.stats_every < 0) {
        why = "stats_every must be >= 0";
        return FLB_EINVAL;
    }
    if (c.nx < 1 || c.ny < 1 || c.nz < 1) {
        snprintf(b, sizeof b, "box edges must be >= 1 (got %d x %d x %d)", c.nx, c.ny, c.nz);
        why = b;
        return FLB_EINVAL;
    }
    if ((int64_t)c.nx * c.ny * c.nz >= (int64_t(1) << 31)) {
        why = "nx*ny*nz must be below 2^31";
        return FLB_EINVAL;
    }
    if (!(c.rho0 > 0.0) || !std::isfinite(c.rho0)) {
        why = "rho0 must be positive";
        return FLB_EINVAL;
    }
    if (!(c.kT >= 0.0) || !std::isfinite(c.kT)) {
        why = "kT must be >= 0";
        return FLB_EINVAL;
    }
    const double g[3] = {c.gamma_shear, c.gamma_bulk, c.gamma_ghost};
    const char *gn[3] = {"gamma_shear", "gamma_bulk", "gamma_ghost"};
    for (int k = 0; k < 3; ++k) {
        if (!(std::fabs(g[k]) <= 1.0)) {
            snprintf(b, sizeof b, "%s = %g is outside the linear stability range [-1, 1]", gn[k], g[k]);
            why = b;
            return FLB_EINVAL;
        }
    }
    if (c.store < FLB_STORE_F64 || c.store > FLB_STORE_BF16SR) {
        why = "unknown store format";
        return FLB_EINVAL;
    }
    if (c.pattern != FLB_PATTERN_AB && c.pattern != FLB_PATTERN_AA) {
        why = "unknown streaming pattern";
        return FLB_EINVAL;
    }
    if (!std::isfinite(c.force_amp)) {
        why = "force_amp must be finite";
        return FLB_EINVAL;
    }
    if (c.sites_per_thread != 0 && c.sites_per_thread != 1 && c.sites_per_thread != 2 && c.sites_per_thread != 4) {
        why = "sites_per_thread must be 0, 1, 2 or 4";
        return FLB_EINVAL;
    }
    if (c.block_x < 0 || c.block_y < 0 || (c.block_x * (c.block_y ? c.block_y : 1)) > 256) {
        why = "block_x * block_y must be at most 256";
        return FLB_EINVAL;
    }
    if (c.graph_steps < 0) {
        why = "graph_steps must be >= 0";
        return FLB_EINVAL;
    }
    if (c.lattice != FLB_LATTICE_D3Q19 && c.lattice != FLB_LATTICE_D2Q9) {
        why = "unknown lattice";
        return FLB_EINVAL;
    }
    if (c.lattice == FLB_LATTICE_D2Q9 && c.nz != 1) {
        why = "a D2Q9 box has nz = 1";
        return FLB_EINVAL;
    }
    return FLB_OK;
}

// Per-mode constants of the collision (Sec. IV): gamma_k, sigma_k =
// sqrt(mu rho0 w_k (1 - gamma_k^2)) with mu = 3 kT (Sec. VI), folded with 1/w_k.
template <class R>
void fill_consts(const flb_config &c, CollideConsts<R> &K)
{
    std::memset(&K, 0, sizeof K);
    const double mu = 3.0 * c.kT;
    K.rho0 = (R)c.rho0;
    K.inv_rho0 = (R)(1.0 / c.rho0);
    for (int k = 0; k < Q; ++k) {
        double g = 1.0;
        if (k == 4) g = c.gamma_bulk;
        else if (k >= 5 && k <= 9) g = c.gamma_shear;
        else if (k >= 10) g = c.gamma_ghost;
        const double w = mode_norm(k);
        K.relax[k] = (R)(g / w);
        K.eq[k] = (R)((1.0 - g) / w);
        const bool thermal = k >= 4 && (k <= 9 || c.noise_ghosts);
        const double var = mu * c.rho0 * w * (1.0 - g * g);
        // the FP32 Box-Muller returns normals / sqrt(2 ln 2); its amplitudes carry the factor
        const double bm = sizeof(R) == 4 ? kBoxMullerF32Scale : 1.0;
        K.noise[k] = (R)(thermal && var > 0.0 ? bm * std::sqrt(var) / w : 0.0);
        if (k < 10) K.forcing[k] = (R)((1.0 + g) / (2.0 * w));
    }
    K.force_amp = (R)c.force_amp;
    K.force_phase = (R)(2.0 / c.nz);
    K.noise_rho_local = c.noise_rho_local;
    // Philox-4x32-10 key schedule (Salmon et al.): round r uses key + r (W0, W1)
    uint32_t k0 = (uint32_t)c.seed, k1 = (uint32_t)(c.seed >> 32);
    for (int r = 0; r < 10; ++r) {
        K.rk0[r] = k0;
        K.rk1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// The same constants for the D2Q9 modes of Table I: gamma_bulk for k = 3,
// gamma_shear for k = 4, 5, gamma_ghost for k = 6..8.
template <class R>
void fill_consts2(const flb_config &c, d2::CollideConsts<R> &K)
{
    std::memset(&K, 0, sizeof K);
    const double mu = 3.0 * c.kT;
    K.rho0 = (R)c.rho0;
    K.inv_rho0 = (R)(1.0 / c.rho0);
    for (int k = 0; k < d2::Q; ++k) {
        double g = 1.0;
        if (k == 3) g = c.gamma_bulk;
        else if (k == 4 || k == 5) g = c.gamma_shear;
        else if (k >= 6) g = c.gamma_ghost;
        const double w = d2::mode_norm(k);
        K.relax[k] = (R)(g / w);
        K.eq[k] = (R)((1.0 - g) / w);
        const bool thermal = k >= 3 && (k <= 5 || c.noise_ghosts);
        const double var = mu * c.rho0 * w * (1.0 - g * g);
        const double bm = sizeof(R) == 4 ? kBoxMullerF32Scale : 1.0;
        K.noise[k] = (R)(thermal && var > 0.0 ? bm * std::sqrt(var) / w : 0.0);
        if (k < 6) K.forcing[k] = (R)((1.0 + g) / (2.0 * w));
    }
    K.force_amp = (R)c.force_amp;
    K.force_phase = (R)(2.0 / c.ny);
    K.noise_rho_local = c.noise_rho_local;
    uint32_t k0 = (uint32_t)c.seed, k1 = (uint32_t)(c.seed >> 32);
    for (int r = 0; r < 10; ++r) {
        K.rk0[r] = k0;
        K.rk1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

bool is_d2(const flb_ctx *c);

template <class S>
BoxStep<S> make_step(const flb_ctx *c, const Box &b, int orient)
{
    BoxStep<S> s;
    std::memset(&s, 0, sizeof s);
    if (c->pattern == FLB_PATTERN_AB) {
        s.src = static_cast<const S *>(b.buf[orient]);
        s.dst = static_cast<S *>(b.buf[orient ^ 1]);
    } else {
        s.src = static_cast<const S *>(b.buf[0]);
        s.dst = static_cast<S *>(b.buf[0]);
    }
    s.nx = b.cfg.nx;
    s.ny = b.cfg.ny;
    s.nz = b.cfg.nz;
    s.z0 = 0;
    s.nzl = b.cfg.nz;
    s.plane = b.plane;
    s.replica = b.cfg.replica;
    const int sx = c->L.bx * c->L.V;
    s.gx = (b.cfg.nx + sx - 1) / sx;
    s.gy = (b.cfg.ny + c->L.by - 1) / c->L.by;
    if constexpr (sizeof(typename Storage<S>::R) == 8) s.K = b.Kd;
    else s.K = b.Kf;
#ifdef FLB_BOUNDS_CHECK
    s.viol = c->d_viol;
#endif
    return s;
}

int layout_of(const flb_ctx *c, uint64_t t)
{
    if (c->pattern == FLB_PATTERN_AB) return kAB;
    return (t & 1) ? kAAOdd : kAAEven;
}

// Current-state buffer of a box and the layout it is in at the context's step.
void *state_buf(const flb_ctx *c, const Box &b) { return c->pattern == FLB_PATTERN_AB ? b.buf[c->cur] : b.buf[0]; }

bool is_d2(const flb_ctx *c) { return c->lattice == FLB_LATTICE_D2Q9; }

// Kernel noise variant: 0 deterministic, 1 thermal, 2 thermal and gamma_ghost = 0 in every box.
int noise_mode(const flb_ctx *c) { return !c->noise ? 0 : (c->kin0 ? 2 : 1); }

template <class S>
d2::BoxStep<S> make_step2(const flb_ctx *c, const Box &b, int orient)
{
    d2::BoxStep<S> s;
    std::memset(&s, 0, sizeof s);
    if (c->pattern == FLB_PATTERN_AB) {
        s.src = static_cast<const S *>(b.buf[orient]);
        s.dst = static_cast<S *>(b.buf[orient ^ 1]);
    } else {
        s.src = static_cast<const S *>(b.buf[0]);
        s.dst = static_cast<S *>(b.buf[0]);
    }
    s.nx = b.cfg.nx;
    s.ny = b.cfg.ny;
    s.gx = (b.cfg.nx + c->L.bx - 1) / c->L.bx;
    s.plane = b.plane;
    s.replica = b.cfg.replica;
    if constexpr (sizeof(typename Storage<S>::R) == 8) s.K = b.K2d;
    else s.K = b.K2f;
#ifdef FLB_BOUNDS_CHECK
    s.viol = c->d_viol;
#endif
    return s;
}

// Slab unit of the host transfers: z-planes (D3Q19) or y-rows (D2Q9).
int64_t unit_sites(const Box &b) { return b.cfg.lattice == FLB_LATTICE_D2Q9 ? b.cfg.nx : (int64_t)b.cfg.nx * b.cfg.ny; }
int units(const Box &b) { return b.cfg.lattice == FLB_LATTICE_D2Q9 ? b.cfg.ny : b.cfg.nz; }

template <class S>
int upload_batch_tables(flb_ctx *c)
{
    constexpr int per_chunk = batch_chunk<S>();
    for (int o = 0; o < 2; ++o) {
        c->batch[o].clear();
        BatchParams<S> *P = nullptr;
        int blocks = 0;
        for (const Box &b : c->boxes) {
            if (!P || P->nboxes == per_chunk) {
                c->batch[o].emplace_back();
                flb_ctx::Chunk &ch = c->batch[o].back();
                ch.params.assign(sizeof(BatchParams<S>), 0);
                P = reinterpret_cast<BatchParams<S> *>(ch.params.data());
                blocks = 0;
            }
            BoxStep<S> s = make_step<S>(c, b, o);
            // densely packed threads: gx = x-groups per row, ceil(groups / T) blocks
            const int V = c->L.V == 4 && sizeof(S) * 4 > 16 ? 2 : c->L.V;
            const int T = c->L.bx * c->L.by;
            s.gx = b.cfg.nx / V;
            s.gy = b.cfg.ny;
            s.warprow = V > 1 && s.gx <= 32 && 32 % s.gx == 0;
            s.block0 = blocks;
            blocks += (int)(((int64_t)s.gx * b.cfg.ny * b.cfg.nz + T - 1) / T);
            P->boxes[P->nboxes++] = s;
            c->batch[o].back().blocks = blocks;
        }
    }
    return FLB_OK;
}

int refresh_batch_tables(flb_ctx *c)
{
    if (c->boxes.size() < 2 || is_d2(c)) return FLB_OK;
    switch (c->store) {
    case FLB_STORE_F64: return upload_batch_tables<double>(c);
    case FLB_STORE_F32: return upload_batch_tables<float>(c);
    case FLB_STORE_F16DEV: return upload_batch_tables<__half>(c);
    case FLB_STORE_BF16SR: return upload_batch_tables<bf16sr>(c);
    default: return upload_batch_tables<__nv_bfloat16>(c);
    }
}

template <class S>
cudaError_t enqueue_one_step_t(flb_ctx *c, int orient, int layout, const uint32_t *step_ptr, uint32_t step)
{
    if (is_d2(c)) {
        // D2Q9: one launch per box
        for (const Box &b : c->boxes) {
            const cudaError_t e = d2::launch_step<S>(make_step2<S>(c, b, orient), layout, c->noise, c->force, c->L.bx,
                                                     c->L.by, c->L.V, step_ptr, step, c->stream);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (c->boxes.size() == 1) {
        const BoxStep<S> s = make_step<S>(c, c->boxes[0], orient);
        return launch_step<S>(s, layout, noise_mode(c), c->force, c->L, step_ptr, step, c->stream);
    }
    for (const flb_ctx::Chunk &ch : c->batch[orient]) {
        const cudaError_t e = launch_step_batch<S>(*reinterpret_cast<const BatchParams<S> *>(ch.params.data()),
                                                   ch.blocks, layout, noise_mode(c), c->force, c->L, step_ptr, step,
                                                   c->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Enqueue the kernel of one time step.  orient = AB buffer holding the
// current state; step = absolute step (or offset from *step_ptr).
cudaError_t enqueue_one_step(flb_ctx *c, int orient, int layout, const uint32_t *step_ptr, uint32_t step)
{
    switch (c->store) {
    case FLB_STORE_F64: return enqueue_one_step_t<double>(c, orient, layout, step_ptr, step);
    case FLB_STORE_F32: return enqueue_one_step_t<float>(c, orient, layout, step_ptr, step);
    case FLB_STORE_F16DEV: return enqueue_one_step_t<__half>(c, orient, layout, step_ptr, step);
    case FLB_STORE_BF16SR: return enqueue_one_step_t<bf16sr>(c, orient, layout, step_ptr, step);
    default: return enqueue_one_step_t<__nv_bfloat16>(c, orient, layout, step_ptr, step);
    }
}

void drop_graphs(flb_ctx *c)
{
    for (auto &g : c->gexec) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

// Capture graph_steps steps starting in orientation `o` (AB buffer or AA
// parity), reading the absolute step from *d_step and advancing it at the end.
int capture_graph(flb_ctx *c, int o)
{
    cudaGraph_t g = nullptr;
    CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < c->graph_steps && e == cudaSuccess; ++k) {
        int orient, layout;
        if (c->pattern == FLB_PATTERN_AB) {
            orient = o ^ (k & 1);
            layout = kAB;
        } else {
            orient = 0;
            layout = ((o + k) & 1) ? kAAOdd : kAAEven;
        }
        e = enqueue_one_step(c, orient, layout, c->d_step, (uint32_t)k);
    }
    if (e == cudaSuccess) e = launch_advance_step(c->d_step, (uint32_t)c->graph_steps, c->stream);
    cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, e, "capturing the step graph");
    }
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->gexec[o], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
    return FLB_OK;
}

int ensure_scratch(flb_ctx *c, size_t bytes)
{
    if (c->scratch_bytes >= bytes) return FLB_OK;
    dev_free(c, c->d_scratch);
    c->d_scratch = nullptr;
    c->scratch_bytes = 0;
    if (dev_malloc(c, &c->d_scratch, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(c, FLB_ENOMEM, "cannot allocate the staging buffer");
    }
    c->scratch_bytes = bytes;
    return FLB_OK;
}

// Slab units (z-planes or y-rows) per slab so that `per_site` doubles per site fit in 256 MiB.
int slab_planes(const Box &b, int per_site)
{
    const int64_t plane_sites = unit_sites(b);
    int64_t nzc = (int64_t(256) << 20) / (8 * per_site * plane_sites);
    if (nzc < 1) nzc = 1;
    if (nzc > units(b)) nzc = units(b);
    return (int)nzc;
}

template <class S>
cudaError_t gather_t(flb_ctx *c, const Box &b, int layout, int z0, int nzc, double *out)
{
    if (is_d2(c))
        return d2::launch_gather<S>(static_cast<const S *>(state_buf(c, b)), b.plane, layout, b.cfg.nx, b.cfg.ny, z0,
                                    nzc, b.cfg.rho0, out, c->stream);
    return launch_gather<S>(static_cast<const S *>(state_buf(c, b)), b.plane, layout, b.cfg.nx, b.cfg.ny, b.cfg.nz,
                            z0, nzc, b.cfg.rho0, out, c->stream);
}

cudaError_t gather(flb_ctx *c, const Box &b, int layout, int z0, int nzc, double *out)
{
    switch (c->store) {
    case FLB_STORE_F64: return gather_t<double>(c, b, layout, z0, nzc, out);
    case FLB_STORE_F32: return gather_t<float>(c, b, layout, z0, nzc, out);
    case FLB_STORE_F16DEV: return gather_t<__half>(c, b, layout, z0, nzc, out);
    case FLB_STORE_BF16SR: return gather_t<bf16sr>(c, b, layout, z0, nzc, out);
    default: return gather_t<__nv_bfloat16>(c, b, layout, z0, nzc, out);
    }
}

template <class S>
cudaError_t gather_sites_t(flb_ctx *c, const Box &b, int layout, const int64_t *sites, int64_t n, double *out)
{
    if (is_d2(c))
        return d2::launch_gather_sites<S>(static_cast<const S *>(state_buf(c, b)), b.plane, layout, b.cfg.nx,
                                          b.cfg.ny, b.cfg.rho0, sites, n, out, c->stream);
    return launch_gather_sites<S>(static_cast<const S *>(state_buf(c, b)), b.plane, layout, b.cfg.nx, b.cfg.ny,
                                  b.cfg.nz, b.cfg.rho0, sites, n, out, c->stream);
}

cudaError_t gather_sites(flb_ctx *c, const Box &b, int layout, const int64_t *sites, int64_t n, double *out)
{
    switch (c->store) {
    case FLB_STORE_F64: return gather_sites_t<double>(c, b, layout, sites, n, out);
    case FLB_STORE_F32: return gather_sites_t<float>(c, b, layout, sites, n, out);
    case FLB_STORE_F16DEV: return gather_sites_t<__half>(c, b, layout, sites, n, out);
    case FLB_STORE_BF16SR: return gather_sites_t<bf16sr>(c, b, layout, sites, n, out);
    default: return gather_sites_t<__nv_bfloat16>(c, b, layout, sites, n, out);
    }
}

template <class S>
cudaError_t scatter_t(flb_ctx *c, Box &b, int layout, int z0, int nzc, const double *in, bool equilibrium)
{
    S *buf = static_cast<S *>(state_buf(c, b));
    if (is_d2(c)) {
        if (equilibrium)
            return d2::launch_init_equilibrium<S>(buf, b.plane, layout, b.cfg.nx, b.cfg.ny, z0, nzc, b.cfg.rho0, in,
                                                  c->stream);
        return d2::launch_scatter<S>(buf, b.plane, layout, b.cfg.nx, b.cfg.ny, z0, nzc, b.cfg.rho0, in, c->stream);
    }
    if (equilibrium)
        return launch_init_equilibrium<S>(buf, b.plane, layout, b.cfg.nx, b.cfg.ny, b.cfg.nz, z0, nzc, b.cfg.rho0, in,
                                          c->stream);
    return launch_scatter<S>(buf, b.plane, layout, b.cfg.nx, b.cfg.ny, b.cfg.nz, z0, nzc, b.cfg.rho0, in, c->stream);
}

cudaError_t scatter(flb_ctx *c, Box &b, int layout, int z0, int nzc, const double *in, bool equilibrium)
{
    switch (c->store) {
    case FLB_STORE_F64: return scatter_t<double>(c, b, layout, z0, nzc, in, equilibrium);
    case FLB_STORE_F32: return scatter_t<float>(c, b, layout, z0, nzc, in, equilibrium);
    case FLB_STORE_F16DEV: return scatter_t<__half>(c, b, layout, z0, nzc, in, equilibrium);
    case FLB_STORE_BF16SR: return scatter_t<bf16sr>(c, b, layout, z0, nzc, in, equilibrium);
    default: return scatter_t<__nv_bfloat16>(c, b, layout, z0, nzc, in, equilibrium);
    }
}

SqPlan sq_plan(const flb_ctx *c, const Box &b)
{
    const int nmax = std::max(b.cfg.nx, std::max(b.cfg.ny, b.cfg.nz));
    return SqPlan{b.cfg.nx, b.cfg.ny, b.cfg.nz, nmax, b.nshells, b.sq_P, c->store == FLB_STORE_F64,
                  b.d_rho, b.d_X, b.d_tw, b.d_shell, b.d_shell_tab, b.d_sq_fixed,
                  reinterpret_cast<uint32_t *>(b.d_sq_fixed + b.nshells)};
}

// One S(q) sample of a box whose density field the statistics pass has written.
cudaError_t sq_sample(flb_ctx *c, Box &b)
{
    cudaError_t e = launch_sq(sq_plan(c, b), c->stream);
    if (e == cudaSuccess) ++b.sq_samples;
    return e;
}

template <class S>
cudaError_t stats_t(flb_ctx *c, Box &b, int layout)
{
    using R = typename Storage<S>::R;
    const S *buf = static_cast<const S *>(state_buf(c, b));
    const bool two = is_d2(c);
    R *rho = static_cast<R *>(b.d_rho);
    cudaError_t e = two ? d2::launch_stats_partial<S>(buf, b.plane, layout, b.cfg.nx, b.cfg.ny, b.cfg.rho0,
                                                      b.d_partial, b.stats_nb, c->stream)
                        : launch_stats_partial<S>(buf, b.plane, layout, b.cfg.nx, b.cfg.ny, b.cfg.nz, b.cfg.rho0,
                                                  b.d_partial, b.stats_nb, rho, c->stream);
    if (e != cudaSuccess) return e;
    e = launch_stats_finish(b.d_partial, b.stats_nb, b.d_acc, c->stream);
    if (e != cudaSuccess || !rho) return e;
    if (two) {
        e = d2::launch_density<S>(buf, b.plane, layout, b.cfg.nx, b.cfg.ny, rho, c->stream);
        if (e != cudaSuccess) return e;
    }
    return sq_sample(c, b);
}

template <class S>
cudaError_t stats_batch_t(flb_ctx *c, int layout)
{
    const int nb = (int)c->boxes.size();
    for (int first = 0; first < nb; first += kStatsChunk) {
        const int n = std::min(kStatsChunk, nb - first);
        std::vector<unsigned char> tmem(sizeof(StatsTable<S>), 0);
        StatsTable<S> &T = *reinterpret_cast<StatsTable<S> *>(tmem.data());
        FinishTable F;
        std::memset(&F, 0, sizeof F);
        T.nboxes = F.nboxes = n;
        int blocks = 0;
        for (int i = 0; i < n; ++i) {
            const Box &b = c->boxes[first + i];
            StatsBox<S> &sb = T.box[i];
            sb.buf = static_cast<const S *>(state_buf(c, b));
            sb.partial = b.d_partial;
            sb.rho_out = static_cast<typename Storage<S>::R *>(b.d_rho);
            sb.plane = b.plane;
            sb.rho0 = b.cfg.rho0;
            sb.nx = b.cfg.nx;
            sb.ny = b.cfg.ny;
            sb.nz = b.cfg.nz;
            sb.nblocks = b.stats_nb;
            sb.block0 = blocks;
            blocks += b.stats_nb;
            F.box[i] = FinishBox{b.d_partial, b.d_acc, b.stats_nb, 0};
        }
        cudaError_t e = launch_stats_partial_batch<S>(T, blocks, layout, c->stream);
        if (e != cudaSuccess) return e;
        e = launch_stats_finish_batch(F, c->stream);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t stats_batch(flb_ctx *c, int layout)
{
    switch (c->store) {
    case FLB_STORE_F64: return stats_batch_t<double>(c, layout);
    case FLB_STORE_F32: return stats_batch_t<float>(c, layout);
    case FLB_STORE_F16DEV: return stats_batch_t<__half>(c, layout);
    case FLB_STORE_BF16SR: return stats_batch_t<bf16sr>(c, layout);
    default: return stats_batch_t<__nv_bfloat16>(c, layout);
    }
}

cudaError_t stats_box(flb_ctx *c, Box &b, int layout)
{
    switch (c->store) {
    case FLB_STORE_F64: return stats_t<double>(c, b, layout);
    case FLB_STORE_F32: return stats_t<float>(c, b, layout);
    case FLB_STORE_F16DEV: return stats_t<__half>(c, b, layout);
    case FLB_STORE_BF16SR: return stats_t<bf16sr>(c, b, layout);
    default: return stats_t<__nv_bfloat16>(c, b, layout);
    }
}

// Largest usable sites-per-thread <= V: the vector path needs nx % V == 0 in
// every box, at most 16-byte accesses (FP64: V <= 2) and whole warps (its
// neighbour exchange is a full-warp shuffle), i.e. bx * by % 32 == 0.
int usable_V(const flb_ctx *c, int V, int bx, int by)
{
    if ((bx * by) % 32 != 0) return 1;
    if (c->store == FLB_STORE_F64 && V > 2) V = 2;
    for (;;) {
        bool ok = true;
        for (const Box &b : c->boxes) ok = ok && (b.cfg.nx % V == 0);
        if (ok || V == 1) return V;
        V /= 2;
    }
}

// The row-exchange variant: one box, 4 sites per thread, 32-bit or smaller
// storage, each block row exactly one box row of whole warps, at most
// kXchWarps warps per row and kXchRows rows per block.
bool fullrow_ok(const flb_ctx *c, const Launch &L)
{
    if (c->boxes.size() != 1 || L.V != 4 || c->store == FLB_STORE_F64 || is_d2(c)) return false;
    const int nx = c->boxes[0].cfg.nx;
    return L.bx * L.V == nx && L.bx % 32 == 0 && L.bx / 32 <= kXchWarps && L.by <= kXchRows;
}

// The in-warp variant: one box, V > 1, each block row is one box row of
// bx lanes with bx dividing 32 (and whole warps), so rows tile the warps.
bool warprow_ok(const flb_ctx *c, const Launch &L)
{
    if (c->boxes.size() != 1 || L.V < 2 || is_d2(c)) return false;
    const int V = (c->store == FLB_STORE_F64 && L.V == 4) ? 2 : L.V;
    const int nx = c->boxes[0].cfg.nx;
    return L.bx * V == nx && 32 % L.bx == 0 && (L.bx * L.by) % 32 == 0;
}

void default_launch(flb_ctx *c)
{
    int maxnx = 1;
    for (const Box &b : c->boxes) maxnx = std::max(maxnx, b.cfg.nx);
    const flb_config &f = c->boxes[0].cfg;
    Launch L;
    if (is_d2(c)) {
        // warps along x, 256 threads; 4 sites per thread (2 for FP64) when nx allows
        int bx = 32;
        while (bx < maxnx && bx < 128) bx *= 2;
        L.bx = f.block_x ? f.block_x : bx;
        L.by = f.block_y ? f.block_y : std::max(1, 256 / L.bx);
        const int want = f.sites_per_thread ? f.sites_per_thread : (c->store == FLB_STORE_F64 ? 2 : 4);
        L.V = usable_V(c, want, L.bx, L.by);
        if (L.V == 2 && c->store != FLB_STORE_F64) L.V = 1;   // the D2Q9 vector kernel has V = 4 (FP64: 2)
        L.fullrow = false;
        c->L = L;
        return;
    }
    int want = f.sites_per_thread ? f.sites_per_thread : (c->store == FLB_STORE_F64 ? 2 : 4);
    if (!f.sites_per_thread) {
        // small boxes: fewer sites per thread until there are threads enough to
        // fill the GPU (~100k: 152 SMs x ~650), measured best for 32^3 and 64^3
        int64_t total = 0;
        for (const Box &b : c->boxes) total += b.N;
        while (want > 1 && total / want < 100000) want /= 2;
    }
    const int sites = (maxnx + want - 1) / want;
    int bx = 32;
    while (bx < sites && bx < 128) bx *= 2;
    // short rows in one box: a row of nx / V lanes, several rows per warp
    const int g = maxnx / want;
    if (c->boxes.size() == 1 && maxnx % want == 0 && g < 32 && 32 % g == 0) bx = g;
    L.bx = f.block_x ? f.block_x : bx;
    L.by = f.block_y ? f.block_y : std::max(1, 128 / L.bx);
    L.V = usable_V(c, want, L.bx, L.by);
    L.warprow = warprow_ok(c, L);
    L.fullrow = !L.warprow && fullrow_ok(c, L);
    c->L = L;
}

void free_box(flb_ctx *c, Box &b)
{
    for (void *&p : b.buf) {
        dev_free(c, p);
        p = nullptr;
    }
    dev_free(c, b.d_acc);
    dev_free(c, b.d_partial);
    dev_free(c, b.d_rho);
    dev_free(c, b.d_X);
    dev_free(c, b.d_tw);
    dev_free(c, b.d_shell_tab);
    dev_free(c, b.d_sq_fixed);
    dev_free(c, b.d_shell);
    dev_free(c, b.d_count);
    b.d_acc = b.d_partial = nullptr;
    b.d_rho = b.d_X = b.d_tw = nullptr;
    b.d_shell_tab = nullptr;
    b.d_sq_fixed = nullptr;
    b.d_shell = nullptr;
    b.d_count = nullptr;
}

int create_impl(const flb_config *cfgs, int nboxes, flb_ctx **out)
{
    if (!out) {
        set_create_error("out is NULL");
        return FLB_EINVAL;
    }
    *out = nullptr;
    if (!cfgs || nboxes < 1) {
        set_create_error("need at least one box configuration");
        return FLB_EINVAL;
    }
    for (int i = 0; i < nboxes; ++i) {
        std::string why;
        int rc = validate(cfgs[i], why);
        if (rc == FLB_OK && cfgs[i].lattice != cfgs[0].lattice) {
            why = "every box of a context has the same lattice";
            rc = FLB_EINVAL;
        }
        if (rc != FLB_OK) {
            set_create_error(nboxes > 1 ? "box " + std::to_string(i) + ": " + why : why);
            return rc;
        }
    }
    flb_ctx *c = new flb_ctx();
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        c->A = g_alloc;
    }
    c->store = cfgs[0].store;
    c->pattern = cfgs[0].pattern;
    c->lattice = cfgs[0].lattice;
    c->graph_steps = cfgs[0].graph_steps;
    c->stats_every = cfgs[0].stats_every;
    if (c->graph_steps & 1) c->graph_steps += 1;   // a graph must return to its starting orientation
    const size_t es = store_size(c->store);
    auto bail = [&](int code, const std::string &m) {
        set_create_error(m);
        flb_destroy(c);
        return code;
    };
    if (cfgs[0].stream) {
        c->stream = static_cast<cudaStream_t>(cfgs[0].stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return bail(FLB_ECUDA, "cannot create a CUDA stream (no usable GPU?)");
        }
        c->own_stream = true;
    }
    c->boxes.resize(nboxes);
    for (int i = 0; i < nboxes; ++i) {
        Box &b = c->boxes[i];
        b.cfg = cfgs[i];
        b.cfg.store = c->store;
        b.cfg.pattern = c->pattern;
        b.Q = c->lattice == FLB_LATTICE_D2Q9 ? d2::Q : flb::Q;
        b.N = (int64_t)b.cfg.nx * b.cfg.ny * b.cfg.nz;
        b.plane = (b.N + 63) / 64 * 64;
        if (b.Q == flb::Q) {
            fill_consts(b.cfg, b.Kf);
            fill_consts(b.cfg, b.Kd);
        } else {
            fill_consts2(b.cfg, b.K2f);
            fill_consts2(b.cfg, b.K2d);
        }
        if (b.cfg.kT > 0.0) c->noise = true;
        if (b.cfg.gamma_ghost != 0.0) c->kin0 = false;
        if (b.cfg.force_amp != 0.0) c->force = true;
        const size_t bytes = (size_t)b.Q * b.plane * es;
        const int nbuf = c->pattern == FLB_PATTERN_AB ? 2 : 1;
        for (int k = 0; k < nbuf; ++k) {
            if (dev_malloc(c, &b.buf[k], bytes) != cudaSuccess) {
                cudaGetLastError();
                return bail(FLB_ENOMEM, "cannot allocate " + std::to_string(bytes) + " bytes of populations");
            }
            // padding between planes is never read, but keep it defined
            if (cudaMemsetAsync(b.buf[k], 0, bytes, c->stream) != cudaSuccess) return bail(FLB_ECUDA, "cudaMemset");
        }
        b.stats_nb = stats_blocks(b.N, is_d2(c));
        if (dev_malloc(c, &b.d_acc, kAccWidth * sizeof(double)) != cudaSuccess ||
            dev_malloc(c, &b.d_partial, (size_t)b.stats_nb * kStatWidth * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return bail(FLB_ENOMEM, "cannot allocate statistics accumulators");
        }
        if (cudaMemsetAsync(b.d_acc, 0, kAccWidth * sizeof(double), c->stream) != cudaSuccess)
            return bail(FLB_ECUDA, "cudaMemset");
    }
    if (dev_malloc(c, &c->d_step, sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        return bail(FLB_ENOMEM, "cannot allocate the step counter");
    }
#ifdef FLB_BOUNDS_CHECK
    if (dev_malloc(c, &c->d_viol, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return bail(FLB_ENOMEM, "cannot allocate the bounds-violation counter");
    }
    if (cudaMemsetAsync(c->d_viol, 0, sizeof(unsigned long long), c->stream) != cudaSuccess)
        return bail(FLB_ECUDA, "cudaMemset");
#endif
    if (c->store == FLB_STORE_F64) {
        if (dev_malloc(c, &c->d_bm, kBoxMullerTableBytes) != cudaSuccess) {
            cudaGetLastError();
            return bail(FLB_ENOMEM, "cannot allocate the FP64 Box-Muller tables");
        }
        if (launch_bm_tables(c->d_bm, c->stream) != cudaSuccess) return bail(FLB_ECUDA, "filling the Box-Muller tables");
        for (Box &b : c->boxes) b.Kd.bm = b.K2d.bm = bm_tables_of(c->d_bm);
    }
    default_launch(c);
    if (refresh_batch_tables(c) != FLB_OK) return bail(FLB_ECUDA, c->err);
    for (int i = 0; i < nboxes; ++i) {
        int rc = flb_box_init_velocity(c, i, nullptr);
        if (rc != FLB_OK) return bail(rc, c->err);
    }
    *out = c;
    return FLB_OK;
}

template <class S>
cudaError_t z_profile_t(flb_ctx *c, const Box &b, double *out)
{
    if (is_d2(c))
        return d2::launch_y_profile<S>(static_cast<const S *>(state_buf(c, b)), b.plane, layout_of(c, c->step),
                                       b.cfg.nx, b.cfg.ny, b.cfg.rho0, out, c->stream);
    return launch_z_profile<S>(static_cast<const S *>(state_buf(c, b)), b.plane, layout_of(c, c->step), b.cfg.nx,
                               b.cfg.ny, b.cfg.nz, b.cfg.rho0, out, c->stream);
}

Box *box_of(flb_ctx *c, int box)
{
    if (!c || box < 0 || box >= (int)c->boxes.size()) return nullptr;
    return &c->boxes[box];
}

// One chunk of planes [z0, z1) of the stream-collide kernel of box b.
template <class S>
cudaError_t step_chunk_t(flb_ctx *c, const Box &b, int orient, int layout, int z0, int z1)
{
    BoxStep<S> s = make_step<S>(c, b, orient);
    s.z0 = z0;
    s.nzl = z1 - z0;
    return launch_step<S>(s, layout, noise_mode(c), c->force, c->L, nullptr, (uint32_t)c->step, c->stream);
}

cudaError_t step_chunk(flb_ctx *c, const Box &b, int orient, int layout, int z0, int z1)
{
    switch (c->store) {
    case FLB_STORE_F64: return step_chunk_t<double>(c, b, orient, layout, z0, z1);
    case FLB_STORE_F32: return step_chunk_t<float>(c, b, orient, layout, z0, z1);
    case FLB_STORE_F16DEV: return step_chunk_t<__half>(c, b, orient, layout, z0, z1);
    case FLB_STORE_BF16SR: return step_chunk_t<bf16sr>(c, b, orient, layout, z0, z1);
    default: return step_chunk_t<__nv_bfloat16>(c, b, orient, layout, z0, z1);
    }
}


}  // namespace

// ==========================================================================
// C ABI
// ==========================================================================
extern "C" {

void flb_config_init(flb_config *cfg)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->nx = cfg->ny = cfg->nz = 32;
    cfg->rho0 = 1.0;
    cfg->store = FLB_STORE_F32;
    cfg->pattern = FLB_PATTERN_AB;
    cfg->noise_ghosts = 1;
}

int flb_create(int nx, int ny, int nz, double rho0, double kT, double gamma_shear, double gamma_bulk,
               double gamma_ghost, uint64_t seed, flb_ctx **out)
{
    flb_config cfg;
    flb_config_init(&cfg);
    cfg.nx = nx;
    cfg.ny = ny;
    cfg.nz = nz;
    cfg.rho0 = rho0;
    cfg.kT = kT;
    cfg.gamma_shear = gamma_shear;
    cfg.gamma_bulk = gamma_bulk;
    cfg.gamma_ghost = gamma_ghost;
    cfg.seed = seed;
    return create_impl(&cfg, 1, out);
}

int flb_create_ex(const flb_config *cfg, flb_ctx **out) { return create_impl(cfg, 1, out); }

int flb_create_batch(const flb_config *cfgs, int nboxes, flb_ctx **out) { return create_impl(cfgs, nboxes, out); }

void flb_destroy(flb_ctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    for (Box &b : c->boxes) free_box(c, b);
    dev_free(c, c->d_step);
    dev_free(c, c->d_scratch);
    dev_free(c, c->d_bm);
    dev_free(c, c->d_viol);
    for (cudaEvent_t e : c->ev_up) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_comp) cudaEventDestroy(e);
    if (c->ev_entry) cudaEventDestroy(c->ev_entry);
    if (c->ev_done) cudaEventDestroy(c->ev_done);
    if (c->s_up) cudaStreamDestroy(c->s_up);
    if (c->s_down) cudaStreamDestroy(c->s_down);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    cudaGetLastError();
    delete c;
}

int flb_num_boxes(const flb_ctx *c) { return c ? (int)c->boxes.size() : 0; }

int flb_step(flb_ctx *c, int64_t nsteps)
{
    if (!c) return FLB_EINVAL;
    NvtxRange range("flb_step");
    if (nsteps < 0) return fail(c, FLB_EINVAL, "nsteps must be >= 0");
    if (c->step + (uint64_t)nsteps > 0xFFFFFFFFull)
        return fail(c, FLB_ERANGE, "the step counter is a 32-bit Philox counter word and would overflow");
    int64_t left = nsteps;
    const int64_t every = c->stats_every;
    bool counter_current = false;   // the device step counter equals c->step
    while (left > 0) {
        // the steps up to the next automatic sample (or all that are left)
        int64_t run = left;
        if (every > 0) run = std::min<int64_t>(run, every - (int64_t)(c->step % (uint64_t)every));
        left -= run;
        if (c->graph_steps > 0 && run >= c->graph_steps) {
            if (!counter_current) CK(c, launch_set_step(c->d_step, (uint32_t)c->step, c->stream));
            counter_current = true;
            while (run >= c->graph_steps) {
                const int o = c->pattern == FLB_PATTERN_AB ? c->cur : (int)(c->step & 1);
                if (!c->gexec[o]) {
                    int rc = capture_graph(c, o);
                    if (rc != FLB_OK) return rc;
                }
                {
                    NvtxRange replay("flb graph replay");
                    CK(c, cudaGraphLaunch(c->gexec[o], c->stream));
                }
                c->step += c->graph_steps;
                run -= c->graph_steps;
            }
        }
        for (; run > 0; --run) {
            CK(c, enqueue_one_step(c, c->cur, layout_of(c, c->step), nullptr, (uint32_t)c->step));
            if (c->pattern == FLB_PATTERN_AB) c->cur ^= 1;
            c->step += 1;
            counter_current = false;
        }
        if (every > 0 && c->step % (uint64_t)every == 0) {
            const int rc = flb_stats_sample(c);
            if (rc != FLB_OK) return rc;
        }
    }
    return FLB_OK;
}

int flb_box_step_host(flb_ctx *c, int box, void *host, int64_t nsteps)
{
    NvtxRange range("flb_box_step_host");
    Box *b = box_of(c, box);
    if (!b || !host || nsteps < 0) return fail(c, FLB_EINVAL, "bad box index, NULL state or nsteps < 0");
    if (is_d2(c)) return fail(c, FLB_EINVAL, "host-resident stepping is implemented for D3Q19 boxes");
    if (c->step + (uint64_t)nsteps > 0xFFFFFFFFull)
        return fail(c, FLB_ERANGE, "the step counter is a 32-bit Philox counter word and would overflow");
    if (nsteps == 0) return FLB_OK;
    const int nz = b->cfg.nz;
    // 32 to 128 chunks (one per 32 MB of state), at most one per plane: small
    // chunks shorten the stretches at the start and end of the call where only
    // one copy direction runs
    const int64_t state_bytes = (int64_t)b->Q * b->plane * (int64_t)store_size(c->store);
    const int K = (int)std::min<int64_t>(nz, std::clamp<int64_t>(state_bytes >> 25, 32, 128));
    if (!c->s_up) {
        CK(c, cudaStreamCreateWithFlags(&c->s_up, cudaStreamNonBlocking));
        CK(c, cudaStreamCreateWithFlags(&c->s_down, cudaStreamNonBlocking));
        CK(c, cudaEventCreateWithFlags(&c->ev_entry, cudaEventDisableTiming));
        CK(c, cudaEventCreateWithFlags(&c->ev_done, cudaEventDisableTiming));
    }
    while ((int)c->ev_up.size() < K) {
        cudaEvent_t e1, e2;
        CK(c, cudaEventCreateWithFlags(&e1, cudaEventDisableTiming));
        CK(c, cudaEventCreateWithFlags(&e2, cudaEventDisableTiming));
        c->ev_up.push_back(e1);
        c->ev_comp.push_back(e2);
    }
    std::vector<int> zb(K + 1);
    for (int k = 0; k <= K; ++k) zb[k] = (int)((int64_t)k * nz / K);
    const size_t es = store_size(c->store);
    const size_t pitch = (size_t)b->plane * es, nxy_bytes = (size_t)b->cfg.nx * b->cfg.ny * es;
    const int Q19 = b->Q;
    char *h = static_cast<char *>(host);
    const int orient = c->cur;
    const int layout = layout_of(c, c->step);
    char *src = static_cast<char *>(state_buf(c, *b));
    // earlier work on the context's stream comes first
    CK(c, cudaEventRecord(c->ev_entry, c->stream));
    CK(c, cudaStreamWaitEvent(c->s_up, c->ev_entry, 0));
    // a chunk's step reads its own planes and, except in the AA even step, one
    // plane on each side (periodic): upload the last chunk first, then compute
    // chunks 0, 1, ... as their neighbours arrive
    const bool local = layout == kAAEven;
    for (int n = 0; n < K; ++n) {
        const int k = local ? n : (n + K - 1) % K;
        const size_t off = (size_t)zb[k] * nxy_bytes, w = (size_t)(zb[k + 1] - zb[k]) * nxy_bytes;
        CK(c, cudaMemcpy2DAsync(src + off, pitch, h + off, pitch, w, Q19, cudaMemcpyHostToDevice, c->s_up));
        CK(c, cudaEventRecord(c->ev_up[k], c->s_up));
    }
    for (int k = 0; k < K; ++k) {
        if (local || K == 1) {
            CK(c, cudaStreamWaitEvent(c->stream, c->ev_up[k], 0));
        } else {
            for (int d = -1; d <= 1; ++d) CK(c, cudaStreamWaitEvent(c->stream, c->ev_up[(k + d + K) % K], 0));
        }
        CK(c, step_chunk(c, *b, orient, layout, zb[k], zb[k + 1]));
        CK(c, cudaEventRecord(c->ev_comp[k], c->stream));
    }
    if (c->pattern == FLB_PATTERN_AB) c->cur ^= 1;
    c->step += 1;
    // further steps on the device
    for (int64_t left = nsteps - 1; left > 0; --left) {
        CK(c, enqueue_one_step(c, c->cur, layout_of(c, c->step), nullptr, (uint32_t)c->step));
        if (c->pattern == FLB_PATTERN_AB) c->cur ^= 1;
        c->step += 1;
    }
    CK(c, cudaEventRecord(c->ev_done, c->stream));
    // downloads: after one step a chunk is final once the computes that write
    // it are done (its own; in the AA odd step also its neighbours'), so they
    // are issued in the order the chunks become final (chunk 0 of an AA odd
    // step waits for the last compute)
    char *dst = static_cast<char *>(state_buf(c, *b));
    std::vector<int> dorder(K);
    for (int k = 0; k < K; ++k) dorder[k] = k;
    if (nsteps == 1 && layout == kAAOdd && K > 1) std::rotate(dorder.begin(), dorder.begin() + 1, dorder.end());
    for (int k : dorder) {
        if (nsteps > 1) {
            CK(c, cudaStreamWaitEvent(c->s_down, c->ev_done, 0));
        } else if (layout == kAAOdd && K > 1) {
            for (int d = -1; d <= 1; ++d) CK(c, cudaStreamWaitEvent(c->s_down, c->ev_comp[(k + d + K) % K], 0));
        } else {
            CK(c, cudaStreamWaitEvent(c->s_down, c->ev_comp[k], 0));
        }
        const size_t off = (size_t)zb[k] * nxy_bytes, w = (size_t)(zb[k + 1] - zb[k]) * nxy_bytes;
        CK(c, cudaMemcpy2DAsync(h + off, pitch, dst + off, pitch, w, Q19, cudaMemcpyDeviceToHost, c->s_down));
    }
    CK(c, cudaStreamSynchronize(c->s_down));
    // the context's stream must not run ahead of the downloads' reads of the state
    CK(c, cudaEventRecord(c->ev_done, c->s_down));
    CK(c, cudaStreamWaitEvent(c->stream, c->ev_done, 0));
    return FLB_OK;
}

int flb_sync(flb_ctx *c)
{
    if (!c) return FLB_EINVAL;
    CK(c, cudaStreamSynchronize(c->stream));
    return FLB_OK;
}

int flb_get_step(const flb_ctx *c, uint64_t *step)
{
    if (!c || !step) return FLB_EINVAL;
    *step = c->step;
    return FLB_OK;
}

int flb_box_get_populations(flb_ctx *c, int box, double *n)
{
    Box *b = box_of(c, box);
    if (!b || !n) return fail(c, FLB_EINVAL, "bad box index or NULL output");
    const int Qb = b->Q;
    const int nzc = slab_planes(*b, Qb);
    const int64_t plane_sites = unit_sites(*b);
    int rc = ensure_scratch(c, (size_t)Qb * nzc * plane_sites * sizeof(double));
    if (rc) return rc;
    const int layout = layout_of(c, c->step);
    for (int z0 = 0; z0 < units(*b); z0 += nzc) {
        const int nz_here = std::min(nzc, units(*b) - z0);
        const int64_t slab = nz_here * plane_sites;
        CK(c, gather(c, *b, layout, z0, nz_here, c->d_scratch));
        CK(c, cudaMemcpy2DAsync(n + z0 * plane_sites, b->N * sizeof(double), c->d_scratch, slab * sizeof(double),
                                slab * sizeof(double), Qb, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return FLB_OK;
}

int flb_get_populations(flb_ctx *c, double *n) { return flb_box_get_populations(c, 0, n); }

int flb_box_get_sites(flb_ctx *c, int box, const int64_t *sites, int64_t nsites, double *out)
{
    Box *b = box_of(c, box);
    if (!b || nsites < 0 || (nsites > 0 && (!sites || !out))) return fail(c, FLB_EINVAL, "bad arguments");
    if (nsites == 0) return FLB_OK;
    for (int64_t s = 0; s < nsites; ++s)
        if (sites[s] < 0 || sites[s] >= b->N) return fail(c, FLB_EINVAL, "site index out of range");
    const int Qb = b->Q;
    const size_t need = (size_t)nsites * (Qb + 1) * sizeof(double);
    int rc = ensure_scratch(c, need);
    if (rc) return rc;
    int64_t *d_sites = reinterpret_cast<int64_t *>(c->d_scratch + (size_t)nsites * Qb);
    CK(c, cudaMemcpyAsync(d_sites, sites, nsites * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
    CK(c, gather_sites(c, *b, layout_of(c, c->step), d_sites, nsites, c->d_scratch));
    CK(c, cudaMemcpyAsync(out, c->d_scratch, (size_t)nsites * Qb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return FLB_OK;
}

static int put_field(flb_ctx *c, int box, const double *src, int ncomp, bool equilibrium)
{
    Box *b = box_of(c, box);
    if (!b) return fail(c, FLB_EINVAL, "bad box index");
    if (!src && !equilibrium) return fail(c, FLB_EINVAL, "NULL populations");
    if (!src) {
        // rest equilibrium: every stored deviation n_i - rho0 a_i is +0 in every
        // format, and every slot holds one population, so the state is all zero bits
        CK(c, cudaMemsetAsync(state_buf(c, *b), 0, (size_t)b->Q * b->plane * store_size(c->store), c->stream));
        CK(c, cudaStreamSynchronize(c->stream));
        return FLB_OK;
    }
    if (ncomp < 0) ncomp = b->Q;                       // populations
    const int nzc = slab_planes(*b, b->Q);
    const int64_t plane_sites = unit_sites(*b);
    int rc = ensure_scratch(c, (size_t)b->Q * nzc * plane_sites * sizeof(double));
    if (rc) return rc;
    const int layout = layout_of(c, c->step);
    for (int z0 = 0; z0 < units(*b); z0 += nzc) {
        const int nz_here = std::min(nzc, units(*b) - z0);
        const int64_t slab = nz_here * plane_sites;
        const double *in = nullptr;
        if (src) {
            CK(c, cudaMemcpy2DAsync(c->d_scratch, slab * sizeof(double), src + z0 * plane_sites,
                                    b->N * sizeof(double), slab * sizeof(double), ncomp, cudaMemcpyHostToDevice,
                                    c->stream));
            in = c->d_scratch;
        }
        CK(c, scatter(c, *b, layout, z0, nz_here, in, equilibrium));
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return FLB_OK;
}

int flb_box_set_populations(flb_ctx *c, int box, const double *n) { return put_field(c, box, n, -1, false); }
int flb_set_populations(flb_ctx *c, const double *n) { return flb_box_set_populations(c, 0, n); }

int flb_box_init_velocity(flb_ctx *c, int box, const double *u)
{
    return put_field(c, box, u, c && c->lattice == FLB_LATTICE_D2Q9 ? 2 : 3, true);
}
int flb_init_velocity(flb_ctx *c, const double *u) { return flb_box_init_velocity(c, 0, u); }

int flb_box_moments(flb_ctx *c, int box, double *rho, double *j, double *Pi)
{
    Box *b = box_of(c, box);
    if (!b) return fail(c, FLB_EINVAL, "bad box index");
    const bool two = is_d2(c);
    const int nd = two ? 2 : 3, npi = two ? 3 : 6;      // velocity and stress components
    const int per_site = b->Q + 1 + nd + npi;
    const int nzc = slab_planes(*b, per_site);
    const int64_t plane_sites = unit_sites(*b);
    const int64_t slab_max = nzc * plane_sites;
    int rc = ensure_scratch(c, (size_t)per_site * slab_max * sizeof(double));
    if (rc) return rc;
    const int layout = layout_of(c, c->step);
    double *pop = c->d_scratch;
    for (int z0 = 0; z0 < units(*b); z0 += nzc) {
        const int nz_here = std::min(nzc, units(*b) - z0);
        const int64_t slab = nz_here * plane_sites;
        double *mrho = pop + b->Q * slab, *mj = mrho + slab, *mpi = mj + nd * slab;
        CK(c, gather(c, *b, layout, z0, nz_here, pop));
        if (two)
            CK(c, d2::launch_moments(pop, slab, b->cfg.nx, b->cfg.ny, z0, b->cfg.force_amp, mrho, mj, mpi, c->stream));
        else
            CK(c, launch_moments(pop, slab, b->cfg.nx, b->cfg.ny, b->cfg.nz, z0, b->cfg.force_amp, mrho, mj, mpi,
                                 c->stream));
        const size_t w = slab * sizeof(double), hp = b->N * sizeof(double);
        if (rho) CK(c, cudaMemcpyAsync(rho + z0 * plane_sites, mrho, w, cudaMemcpyDeviceToHost, c->stream));
        if (j) CK(c, cudaMemcpy2DAsync(j + z0 * plane_sites, hp, mj, w, w, nd, cudaMemcpyDeviceToHost, c->stream));
        if (Pi) CK(c, cudaMemcpy2DAsync(Pi + z0 * plane_sites, hp, mpi, w, w, npi, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(c, cudaStreamSynchronize(c->stream));
    return FLB_OK;
}

int flb_moments(flb_ctx *c, double *rho, double *j, double *Pi) { return flb_box_moments(c, 0, rho, j, Pi); }

int flb_box_z_profile(flb_ctx *c, int box, double *rho, double *j)
{
    Box *b = box_of(c, box);
    if (!b) return fail(c, FLB_EINVAL, "bad box index");
    const int nz = units(*b);            // z-planes, or y-rows of a D2Q9 box
    int rc = ensure_scratch(c, (size_t)4 * nz * sizeof(double));
    if (rc) return rc;
    cudaError_t e;
    switch (c->store) {
    case FLB_STORE_F64: e = z_profile_t<double>(c, *b, c->d_scratch); break;
    case FLB_STORE_F32: e = z_profile_t<float>(c, *b, c->d_scratch); break;
    case FLB_STORE_F16DEV: e = z_profile_t<__half>(c, *b, c->d_scratch); break;
    case FLB_STORE_BF16SR: e = z_profile_t<bf16sr>(c, *b, c->d_scratch); break;
    default: e = z_profile_t<__nv_bfloat16>(c, *b, c->d_scratch); break;
    }
    CK(c, e);
    std::vector<double> h(4 * (size_t)nz);
    CK(c, cudaMemcpyAsync(h.data(), c->d_scratch, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    for (int z = 0; z < nz; ++z) {
        if (rho) rho[z] = h[z];
        if (j) {
            // half-step momentum with a body force (see flb_box_moments)
            const double half_force = 0.5 * b->cfg.force_amp * std::sin(2.0 * M_PI * z / nz);
            j[z] = h[nz + 3 * z] + half_force;
            j[nz + z] = h[nz + 3 * z + 1];
            j[2 * nz + z] = h[nz + 3 * z + 2];
        }
    }
    return FLB_OK;
}

int flb_stats_reset(flb_ctx *c)
{
    if (!c) return FLB_EINVAL;
    for (Box &b : c->boxes) {
        CK(c, cudaMemsetAsync(b.d_acc, 0, kAccWidth * sizeof(double), c->stream));
        if (b.d_shell) {
            CK(c, cudaMemsetAsync(b.d_shell, 0, b.nshells * sizeof(double), c->stream));
            b.sq_samples = 0;
        }
    }
    return FLB_OK;
}

int flb_stats_sample(flb_ctx *c)
{
    if (!c) return FLB_EINVAL;
    NvtxRange range("flb_stats_sample");
    const int layout = layout_of(c, c->step);
    if (c->boxes.size() > 1 && !is_d2(c)) {
        // a batch: mode sums of every box in two launches (which also write the
        // density of the boxes with S(q) enabled), then S(q) per such box
        CK(c, stats_batch(c, layout));
        for (Box &b : c->boxes)
            if (b.d_rho) CK(c, sq_sample(c, b));
        return FLB_OK;
    }
    for (Box &b : c->boxes) CK(c, stats_box(c, b, layout));
    return FLB_OK;
}

int flb_box_mode_stats(flb_ctx *c, int box, flb_mode_stats_t *out)
{
    Box *b = box_of(c, box);
    if (!b || !out) return fail(c, FLB_EINVAL, "bad box index or NULL output");
    double acc[kAccWidth];
    CK(c, cudaMemcpyAsync(acc, b->d_acc, sizeof acc, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    std::memset(out, 0, sizeof *out);
    const double ns = acc[kAccCount];
    out->nsamples = (uint64_t)ns;
    out->nsites = (uint64_t)b->N;
    const double mu = 3.0 * b->cfg.kT;
    const double denom = ns * (double)b->N;
    const bool two = b->Q == d2::Q;
    for (int k = 0; k < b->Q; ++k) {
        const double w = two ? d2::mode_norm(k) : mode_norm(k);
        out->mode_m2[k] = ns > 0 ? acc[kAccSums + k] / denom : 0.0;
        out->mode_ratio[k] = (ns > 0 && mu > 0) ? out->mode_m2[k] / (mu * b->cfg.rho0 * w) : 0.0;
    }
    for (int a = 0; a < (two ? 2 : 3); ++a) {
        out->u2[a] = ns > 0 ? acc[kAccSums + 19 + a] / denom : 0.0;
        out->u2_ratio[a] = (ns > 0 && b->cfg.kT > 0) ? out->u2[a] * b->cfg.rho0 / b->cfg.kT : 0.0;
    }
    out->mass_first = acc[kAccFirst];
    out->mass_last = acc[kAccLast];
    for (int a = 0; a < 3; ++a) {
        out->momentum_first[a] = acc[kAccFirst + 1 + a];
        out->momentum_last[a] = acc[kAccLast + 1 + a];
    }
    out->nonfinite = (uint64_t)acc[kAccSums + 26];
    return FLB_OK;
}

int flb_mode_stats(flb_ctx *c, flb_mode_stats_t *out) { return flb_box_mode_stats(c, 0, out); }

int flb_box_enable_structure_factor(flb_ctx *c, int box)
{
    Box *b = box_of(c, box);
    if (!b) return fail(c, FLB_EINVAL, "bad box index");
    if (b->d_rho) return FLB_OK;
    const int nx = b->cfg.nx, ny = b->cfg.ny, nz = b->cfg.nz;
    const bool dbl = c->store == FLB_STORE_F64;
    const int nmax = std::max(nx, std::max(ny, nz));
    if (nmax > 4096 || !sq_supported(nx, ny, nz, dbl))
        return fail(c, FLB_EINVAL, dbl ? "structure factor of an FP64 context supports edges up to 2048"
                                       : "structure factor supports edges up to 4096");
    b->nshells = sq_shells(nx, ny, nz);
    b->sq_P = sq_row_stride(nx, dbl);
    const size_t eb = sq_elem_bytes(dbl);
    const size_t half = (size_t)b->sq_P * ny * nz;
    if (dev_malloc(c, &b->d_rho, (size_t)b->N * eb) != cudaSuccess ||
        dev_malloc(c, &b->d_X, half * 2 * eb) != cudaSuccess ||
        dev_malloc(c, &b->d_tw, (size_t)(nx + ny + nz) * 2 * eb) != cudaSuccess ||
        dev_malloc(c, &b->d_shell_tab, (size_t)sq_table_elems(nx, ny, nz, dbl) * sizeof(uint16_t)) != cudaSuccess ||
        dev_malloc(c, &b->d_sq_fixed, (size_t)(b->nshells + 1) * sizeof(unsigned long long)) != cudaSuccess ||
        dev_malloc(c, &b->d_shell, b->nshells * sizeof(double)) != cudaSuccess ||
        dev_malloc(c, &b->d_count, b->nshells * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        for (void *p : {b->d_rho, b->d_X, b->d_tw, (void *)b->d_shell_tab, (void *)b->d_sq_fixed, (void *)b->d_shell,
                        (void *)b->d_count})
            dev_free(c, p);
        b->d_rho = b->d_X = b->d_tw = nullptr;
        b->d_shell_tab = nullptr;
        b->d_sq_fixed = nullptr;
        b->d_shell = nullptr;
        b->d_count = nullptr;
        return fail(c, FLB_ENOMEM, "cannot allocate the structure-factor workspace");
    }
    CK(c, cudaMemsetAsync(b->d_shell, 0, b->nshells * sizeof(double), c->stream));
    b->sq_samples = 0;
    CK(c, sq_init(sq_plan(c, *b), b->d_count, c->stream));
    b->count.assign(b->nshells, 0ull);
    CK(c, cudaMemcpyAsync(b->count.data(), b->d_count, b->nshells * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return FLB_OK;
}

int flb_enable_structure_factor(flb_ctx *c) { return flb_box_enable_structure_factor(c, 0); }

int flb_structure_factor(flb_ctx *c, double *S, int nshells) { return flb_box_structure_factor(c, 0, S, nullptr, nshells); }

int flb_box_structure_factor(flb_ctx *c, int box, double *S, int64_t *count, int nshells)
{
    Box *b = box_of(c, box);
    if (!b || nshells < 0) return fail(c, FLB_EINVAL, "bad box index or shell count");
    if (!b->d_rho) return fail(c, FLB_EINVAL, "structure factor not enabled for this box");
    std::vector<double> sum(b->nshells);
    CK(c, cudaMemcpyAsync(sum.data(), b->d_shell, b->nshells * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    const double ns = (double)b->sq_samples;
    for (int s = 0; s < nshells; ++s) {
        const unsigned long long n = s < b->nshells ? b->count[s] : 0ull;
        if (S) S[s] = (n > 0 && ns > 0) ? sum[s] / ((double)n * ns) : 0.0;
        if (count) count[s] = (int64_t)n;
    }
    return FLB_OK;
}

int flb_box_state_bytes(const flb_ctx *c, int box, size_t *bytes)
{
    if (!c || !bytes || box < 0 || box >= (int)c->boxes.size()) return FLB_EINVAL;
    *bytes = (size_t)c->boxes[box].Q * c->boxes[box].plane * store_size(c->store);
    return FLB_OK;
}

int flb_box_state_download(flb_ctx *c, int box, void *host)
{
    Box *b = box_of(c, box);
    if (!b || !host) return fail(c, FLB_EINVAL, "bad box index or NULL buffer");
    const size_t bytes = (size_t)b->Q * b->plane * store_size(c->store);
    CK(c, cudaMemcpyAsync(host, state_buf(c, *b), bytes, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return FLB_OK;
}

int flb_box_state_upload(flb_ctx *c, int box, const void *host)
{
    Box *b = box_of(c, box);
    if (!b || !host) return fail(c, FLB_EINVAL, "bad box index or NULL buffer");
    const size_t bytes = (size_t)b->Q * b->plane * store_size(c->store);
    CK(c, cudaMemcpyAsync(state_buf(c, *b), host, bytes, cudaMemcpyHostToDevice, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    return FLB_OK;
}

namespace {
struct CkptHeader {
    char magic[8];
    uint32_t version, nboxes;
    int32_t store, pattern, cur, pad;
    uint64_t step;
};
}  // namespace

int flb_save(flb_ctx *c, const char *path)
{
    if (!c || !path) return FLB_EINVAL;
    FILE *f = fopen(path, "wb");
    if (!f) return fail(c, FLB_EIO, std::string("cannot open ") + path);
    CkptHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, "FLBCKPT1", 8);
    h.version = 1;
    h.nboxes = (uint32_t)c->boxes.size();
    h.store = c->store;
    h.pattern = c->pattern;
    h.cur = c->cur;
    h.step = c->step;
    bool ok = fwrite(&h, sizeof h, 1, f) == 1;
    std::vector<char> host;
    for (int i = 0; ok && i < (int)c->boxes.size(); ++i) {
        ok = fwrite(&c->boxes[i].cfg, sizeof(flb_config), 1, f) == 1;
        size_t bytes = 0;
        flb_box_state_bytes(c, i, &bytes);
        host.resize(bytes);
        if (ok && flb_box_state_download(c, i, host.data()) != FLB_OK) {
            fclose(f);
            return FLB_ECUDA;
        }
        ok = ok && fwrite(host.data(), 1, bytes, f) == bytes;
    }
    ok = (fclose(f) == 0) && ok;
    return ok ? FLB_OK : fail(c, FLB_EIO, std::string("cannot write ") + path);
}

namespace {
// The physics of a saved box must be the context's: its size and lattice fix
// the layout, and rho0, kT, the eigenvalues, the noise variants, the force,
// the seed and the replica id fix the dynamics and the noise stream that a
// resumed run continues.  Launch shape, graphs, sampling and stream are
// run-time choices and may differ.
const char *ckpt_mismatch(const flb_config &a, const flb_config &b)
{
    if (a.nx != b.nx || a.ny != b.ny || a.nz != b.nz || a.lattice != b.lattice) return "box sizes or lattice";
    if (a.rho0 != b.rho0 || a.kT != b.kT) return "rho0 or kT";
    if (a.gamma_shear != b.gamma_shear || a.gamma_bulk != b.gamma_bulk || a.gamma_ghost != b.gamma_ghost)
        return "eigenvalues";
    if (a.seed != b.seed || a.replica != b.replica) return "seed or replica id";
    if (a.noise_ghosts != b.noise_ghosts || a.noise_rho_local != b.noise_rho_local) return "noise variant";
    if (a.force_amp != b.force_amp) return "force amplitude";
    return nullptr;
}
}  // namespace

int flb_load(flb_ctx *c, const char *path)
{
    if (!c || !path) return FLB_EINVAL;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(c, FLB_EIO, std::string("cannot open ") + path);
    CkptHeader h;
    bool ok = fread(&h, sizeof h, 1, f) == 1 && std::memcmp(h.magic, "FLBCKPT1", 8) == 0 && h.version == 1;
    if (!ok || h.nboxes != c->boxes.size() || h.store != c->store || h.pattern != c->pattern) {
        fclose(f);
        return fail(c, FLB_EIO, "checkpoint does not match this context (format, boxes or pattern)");
    }
    // AB keeps the current buffer index 0 or 1; AA has one buffer
    const bool cur_ok = c->pattern == FLB_PATTERN_AB ? (h.cur == 0 || h.cur == 1) : h.cur == 0;
    if (!cur_ok || h.step > 0xFFFFFFFFull) {
        fclose(f);
        return fail(c, FLB_EIO, "corrupt checkpoint header (buffer index or step counter out of range)");
    }
    // every box is read and checked into host memory before any is uploaded,
    // so a bad file leaves the context as it was
    std::vector<std::vector<char>> host(h.nboxes);
    for (uint32_t i = 0; i < h.nboxes; ++i) {
        flb_config saved;
        if (fread(&saved, sizeof(flb_config), 1, f) != 1) {
            ok = false;
            break;
        }
        if (const char *what = ckpt_mismatch(saved, c->boxes[i].cfg)) {
            fclose(f);
            return fail(c, FLB_EIO, std::string("checkpoint box ") + std::to_string(i) + " differs from this context: " + what);
        }
        size_t bytes = 0;
        flb_box_state_bytes(c, (int)i, &bytes);
        host[i].resize(bytes);
        if (fread(host[i].data(), 1, bytes, f) != bytes) {
            ok = false;
            break;
        }
    }
    fclose(f);
    if (!ok) return fail(c, FLB_EIO, std::string("truncated checkpoint ") + path);
    // the states go into the buffer that will be current
    const int saved_cur = c->cur;
    c->cur = h.cur;
    for (uint32_t i = 0; i < h.nboxes; ++i) {
        int rc = flb_box_state_upload(c, (int)i, host[i].data());
        if (rc != FLB_OK) {
            c->cur = saved_cur;
            return rc;
        }
    }
    c->step = h.step;
    return FLB_OK;
}

int flb_get_launch(const flb_ctx *c, int *V, int *bx, int *by)
{
    if (!c) return FLB_EINVAL;
    if (V) *V = c->L.V;
    if (bx) *bx = c->L.bx;
    if (by) *by = c->L.by;
    return FLB_OK;
}

}  // extern "C"

namespace {
int tune_shapes(flb_ctx *c, int trials, float *best_out)
{
    if (!c) return FLB_EINVAL;
    if (trials < 1) trials = 1;
    const int nb = (int)c->boxes.size();
    int maxnx = 1;
    for (const Box &b : c->boxes) maxnx = std::max(maxnx, b.cfg.nx);
    // back up every box's current state (device to device) and the step counter
    std::vector<void *> backup(nb, nullptr);
    for (int i = 0; i < nb; ++i) {
        size_t bytes = 0;
        flb_box_state_bytes(c, i, &bytes);
        if (dev_malloc(c, &backup[i], bytes) != cudaSuccess) {
            cudaGetLastError();
            for (void *p : backup) dev_free(c, p);
            return fail(c, FLB_ENOMEM, "autotune needs a copy of the state");
        }
        CK(c, cudaMemcpyAsync(backup[i], state_buf(c, c->boxes[i]), bytes, cudaMemcpyDeviceToDevice, c->stream));
    }
    const uint64_t step0 = c->step;
    const int cur0 = c->cur;
    const Launch keep = c->L;
    const int keep_graph = c->graph_steps;
    c->graph_steps = 0;
    Launch best = keep;
    float best_ms = 1e30f;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int Vs[3] = {1, 2, 4};
    const int shapes[9][2] = {{32, 4}, {64, 2}, {64, 4}, {128, 1}, {128, 2}, {256, 1}, {16, 8}, {16, 16}, {32, 8}};
    int rc = FLB_OK;
    for (int vi = 0; vi < 3 && rc == FLB_OK; ++vi) {
        for (int si = 0; si < 9 && rc == FLB_OK; ++si) {
            Launch L;
            L.V = Vs[vi];
            L.bx = shapes[si][0];
            L.by = shapes[si][1];
            if (usable_V(c, L.V, L.bx, L.by) != L.V) continue;
            // the D2Q9 vector kernel has one width per format
            if (is_d2(c) && L.V != 1 && L.V != (c->store == FLB_STORE_F64 ? 2 : 4)) continue;
            L.warprow = warprow_ok(c, L);
            L.fullrow = !L.warprow && fullrow_ok(c, L);
            if (L.bx * L.V > 2 * std::max(32, maxnx)) continue;   // mostly idle threads
            c->L = L;
            if ((rc = refresh_batch_tables(c)) != FLB_OK) break;
            rc = flb_step(c, 2);   // warm-up
            if (rc != FLB_OK) break;
            cudaEventRecord(e0, c->stream);
            rc = flb_step(c, 2 * trials);
            cudaEventRecord(e1, c->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = cuda_fail(c, cudaGetLastError(), "autotune");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best_ms) {
                best_ms = ms;
                best = L;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // restore state, counter and orientation
    c->step = step0;
    c->cur = cur0;
    for (int i = 0; i < nb; ++i) {
        size_t bytes = 0;
        flb_box_state_bytes(c, i, &bytes);
        cudaMemcpyAsync(state_buf(c, c->boxes[i]), backup[i], bytes, cudaMemcpyDeviceToDevice, c->stream);
    }
    cudaStreamSynchronize(c->stream);
    for (void *p : backup) dev_free(c, p);
    c->L = rc == FLB_OK ? best : keep;
    c->graph_steps = keep_graph;
    drop_graphs(c);
    int rc2 = refresh_batch_tables(c);
    if (best_out) *best_out = best_ms;
    return rc != FLB_OK ? rc : rc2;
}

}  // namespace

extern "C" {

int flb_box_check_finite(flb_ctx *c, int box, uint64_t *nonfinite)
{
    Box *b = box_of(c, box);
    if (!b) return fail(c, FLB_EINVAL, "bad box index");
    int rc = ensure_scratch(c, sizeof(unsigned long long));
    if (rc) return rc;
    unsigned long long *d_count = reinterpret_cast<unsigned long long *>(c->d_scratch);
    CK(c, cudaMemsetAsync(d_count, 0, sizeof *d_count, c->stream));
    CK(c, launch_count_nonfinite(state_buf(c, *b), (int64_t)b->Q * b->plane, c->store, d_count, c->stream));
    unsigned long long h = 0;
    CK(c, cudaMemcpyAsync(&h, d_count, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    if (nonfinite) *nonfinite = h;
    return h ? fail(c, FLB_ENONFINITE, std::to_string(h) + " non-finite populations") : FLB_OK;
}

int flb_get_pattern(const flb_ctx *c, int *pattern)
{
    if (!c || !pattern) return FLB_EINVAL;
    *pattern = c->pattern;
    return FLB_OK;
}

int flb_set_pattern(flb_ctx *c, int pattern)
{
    if (!c) return FLB_EINVAL;
    if (pattern != FLB_PATTERN_AB && pattern != FLB_PATTERN_AA) return fail(c, FLB_EINVAL, "unknown streaming pattern");
    if (pattern == c->pattern) return FLB_OK;
    const size_t es = store_size(c->store);
    const int aa_layout = (c->step & 1) ? kAAOdd : kAAEven;
    const bool two = is_d2(c);
    if (pattern == FLB_PATTERN_AB) {
        // AA -> AB: a second buffer per box receives the AB layout and becomes current
        for (Box &b : c->boxes) {
            if (!b.buf[1]) {
                const size_t bytes = (size_t)b.Q * b.plane * es;
                if (dev_malloc(c, &b.buf[1], bytes) != cudaSuccess) {
                    cudaGetLastError();
                    return fail(c, FLB_ENOMEM, "the two-buffer pattern needs a second state buffer");
                }
                CK(c, cudaMemsetAsync(b.buf[1], 0, bytes, c->stream));
            }
        }
        for (Box &b : c->boxes)
            CK(c, launch_relayout(b.buf[0], aa_layout, b.buf[1], kAB, es, b.plane, b.cfg.nx, b.cfg.ny, b.cfg.nz, two,
                                  c->stream));
        c->cur = 1;
    } else {
        // AB -> AA: the other buffer receives the AA layout and becomes the only one
        for (Box &b : c->boxes) {
            CK(c, launch_relayout(b.buf[c->cur], kAB, b.buf[c->cur ^ 1], aa_layout, es, b.plane, b.cfg.nx, b.cfg.ny,
                                  b.cfg.nz, two, c->stream));
        }
        CK(c, cudaStreamSynchronize(c->stream));
        for (Box &b : c->boxes) {
            if (c->cur == 0) std::swap(b.buf[0], b.buf[1]);
            dev_free(c, b.buf[1]);
            b.buf[1] = nullptr;
        }
        c->cur = 0;
    }
    c->pattern = pattern;
    for (Box &b : c->boxes) b.cfg.pattern = pattern;
    drop_graphs(c);
    int rc = refresh_batch_tables(c);
    if (rc != FLB_OK) return rc;
    CK(c, cudaStreamSynchronize(c->stream));
    return FLB_OK;
}

int flb_set_launch(flb_ctx *c, int V, int bx, int by)
{
    if (!c) return FLB_EINVAL;
    if ((V != 1 && V != 2 && V != 4) || bx < 1 || by < 1 || bx * by > 256)
        return fail(c, FLB_EINVAL, "sites per thread must be 1, 2 or 4 and block_x * block_y at most 256");
    if (usable_V(c, V, bx, by) != V) return fail(c, FLB_EINVAL, "this launch shape does not fit the boxes");
    if (is_d2(c) && V != 1 && V != (c->store == FLB_STORE_F64 ? 2 : 4))
        return fail(c, FLB_EINVAL, "the D2Q9 vector kernel takes 4 sites per thread (2 for FP64)");
    Launch L;
    L.V = V;
    L.bx = bx;
    L.by = by;
    L.warprow = warprow_ok(c, L);
    L.fullrow = !L.warprow && fullrow_ok(c, L);
    c->L = L;
    drop_graphs(c);
    return refresh_batch_tables(c);
}

int flb_autotune(flb_ctx *c, int trials)
{
    if (!c) return FLB_EINVAL;
    return tune_shapes(c, trials, nullptr);
}

int flb_autotune_ex(flb_ctx *c, int trials, int flags)
{
    NvtxRange range("flb_autotune");
    if (!c) return FLB_EINVAL;
    float ms0 = 0.f, ms1 = 0.f;
    int rc = tune_shapes(c, trials, &ms0);
    if (rc != FLB_OK || !(flags & FLB_TUNE_PATTERN)) return rc;
    const int p0 = c->pattern;
    const Launch L0 = c->L;
    rc = flb_set_pattern(c, p0 == FLB_PATTERN_AB ? FLB_PATTERN_AA : FLB_PATTERN_AB);
    if (rc == FLB_ENOMEM) return FLB_OK;   // no room for the two-buffer pattern: keep the current one
    if (rc != FLB_OK) return rc;
    rc = tune_shapes(c, trials, &ms1);
    if (rc != FLB_OK) return rc;
    if (ms1 >= ms0) {
        rc = flb_set_pattern(c, p0);
        if (rc != FLB_OK) return rc;
        c->L = L0;
        rc = refresh_batch_tables(c);
    }
    return rc;
}

static bool positive_finite(double v) { return std::isfinite(v) && v > 0.0; }

int flb_gammas_from_viscosities(double eta, double zeta, double rho, double b, double h, double *gamma_shear,
                                double *gamma_bulk)
{
    if (!positive_finite(eta) || !positive_finite(zeta) || !positive_finite(rho) || !positive_finite(b) ||
        !positive_finite(h) || !gamma_shear || !gamma_bulk)
        return FLB_EINVAL;
    const double cs2_hat = 1.0 / 3.0;
    const double eta_hat = eta * h / (rho * b * b * cs2_hat);
    const double zeta_hat = zeta * h / (rho * b * b * cs2_hat);
    *gamma_shear = (2.0 * eta_hat - 1.0) / (2.0 * eta_hat + 1.0);
    *gamma_bulk = (3.0 * zeta_hat - 1.0) / (3.0 * zeta_hat + 1.0);
    return FLB_OK;
}

int flb_lattice_kT(double kT, double rho, double b, double h, double rho0, double *kT_lattice)
{
    if (!positive_finite(kT) || !positive_finite(rho) || !positive_finite(b) || !positive_finite(h) ||
        !positive_finite(rho0) || !kT_lattice)
        return FLB_EINVAL;
    *kT_lattice = rho0 * kT * h * h / (rho * b * b * b * b * b);
    return FLB_OK;
}

int flb_lattice_params(int d, double eta, double zeta, double kT, double rho, double b, double h, double rho0,
                       double *gamma_shear, double *gamma_bulk, double *kT_lattice)
{
    if ((d != 2 && d != 3) || !positive_finite(eta) || !positive_finite(zeta) || !positive_finite(rho) ||
        !positive_finite(b) || !positive_finite(h) || !positive_finite(rho0) || !(kT >= 0.0) || !std::isfinite(kT) ||
        !gamma_shear || !gamma_bulk || !kT_lattice)
        return FLB_EINVAL;
    const double cs2_hat = 1.0 / 3.0;
    const double eta_hat = eta * h / (rho * b * b * cs2_hat);
    const double zeta_hat = zeta * h / (rho * b * b * cs2_hat);
    *gamma_shear = (2.0 * eta_hat - 1.0) / (2.0 * eta_hat + 1.0);
    *gamma_bulk = (d * zeta_hat - 1.0) / (d * zeta_hat + 1.0);
    *kT_lattice = rho0 * kT * h * h / (rho * std::pow(b, d + 2));
    return FLB_OK;
}

int flb_bounds_violations(flb_ctx *c, uint64_t *count)
{
    if (!c || !count) return FLB_EINVAL;
#ifdef FLB_BOUNDS_CHECK
    unsigned long long v = 0;
    CK(c, cudaMemcpyAsync(&v, c->d_viol, sizeof v, cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    *count = v;
    return FLB_OK;
#else
    *count = 0;
    return fail(c, FLB_EINVAL, "this library was built without bounds checks (FLB_BOUNDS_CHECK)");
#endif
}

int flb_bounds_selftest(flb_ctx *c)
{
    if (!c) return FLB_EINVAL;
#ifdef FLB_BOUNDS_CHECK
    const Box &b = c->boxes[0];
    CK(c, launch_guard_selftest(state_buf(c, b), (int64_t)b.Q * b.plane * (int64_t)store_size(c->store), c->d_viol,
                                c->stream));
    return FLB_OK;
#else
    return fail(c, FLB_EINVAL, "this library was built without bounds checks (FLB_BOUNDS_CHECK)");
#endif
}

int flb_set_device_allocator(flb_dev_alloc_fn alloc, flb_dev_free_fn free_fn, void *user)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) return FLB_EINVAL;
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.free = free_fn;
    g_alloc.user = alloc ? user : nullptr;
    return FLB_OK;
}

const char *flb_last_error(const flb_ctx *c) { return c ? c->err.c_str() : "NULL context"; }

const char *flb_create_error(void)
{
    static thread_local std::string copy;
    std::lock_guard<std::mutex> lk(g_create_err_mu);
    copy = g_create_err;
    return copy.c_str();
}

int flb_version(char *buf, int len)
{
    if (!buf || len < 1) return FLB_EINVAL;
    snprintf(buf, (size_t)len, "flb 0.2 (D3Q19 and D2Q9 fluctuating LB; sm_103a; CUDA %d)", CUDART_VERSION);
    return FLB_OK;
}

}  // extern "C"
