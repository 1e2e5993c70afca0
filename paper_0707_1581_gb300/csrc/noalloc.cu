// noalloc.cu -- mode statistics of caller-owned populations, with no device
// allocation.
//
// The ordinary statistics path (flb_stats_sample) reduces through a per-box
// partial-sum buffer the context allocates.  This entry point serves callers
// that must not allocate device memory themselves or through a library:
// cudaMalloc synchronises the whole device and can fail under memory
// pressure, and some hosts (plugins inside another application's fixed
// memory budget, loops that must never stall) hand a library only the buffers
// it reads and writes.  Its scratch is a fixed array in this file instead.
#include <mutex>

#include "flb.h"
#include "diag_kernels.cuh"
#include "kernels.cuh"

namespace flb {
namespace {

// Each block reduces up to kSitesPerBlock sites into one row of partial sums,
// so a box of at most FLB_NOALLOC_MAX_SITES sites needs at most kMaxBlocks rows.
constexpr int64_t kSitesPerBlock = 8192;
constexpr int kMaxBlocks = (int)(FLB_NOALLOC_MAX_SITES / kSitesPerBlock);
static_assert((int64_t)kMaxBlocks * kSitesPerBlock == FLB_NOALLOC_MAX_SITES, "whole blocks");

// Partial sums, kMaxBlocks x kStatWidth doubles (432 KiB); every device that
// loads the library keeps one copy until the process exits.  Each call
// overwrites the rows it uses, so nothing needs clearing.
static __device__ __align__(256) double g_noalloc_partial[kMaxBlocks * kStatWidth];

// Device address of g_noalloc_partial, resolved once per device context.  In
// host code the symbol itself is only a host-side stand-in, not a device
// address.  cudaDeviceReset destroys the context and with it the module that
// holds the array; the next context loads it again, possibly elsewhere, so the
// cached address is tagged with the id of the context it was resolved in and
// resolved again when the current context's id differs.
constexpr int kMaxDevices = 128;
std::mutex g_addr_mu;
double *g_addr[kMaxDevices] = {};
unsigned long long g_ctx_id[kMaxDevices] = {};

// cuCtxGetCurrent / cuCtxGetId through the runtime's driver entry points (the
// library links only the CUDA runtime).  Both are plain queries.
typedef int (*PfnCtxGetCurrent)(void **);
typedef int (*PfnCtxGetId)(void *, unsigned long long *);
PfnCtxGetCurrent g_ctx_get_current = nullptr;
PfnCtxGetId g_ctx_get_id = nullptr;
std::once_flag g_entry_once;

// Id of the calling thread's current context, 0 if there is none or the
// driver cannot say (then the address is resolved on every call).
unsigned long long current_ctx_id()
{
    std::call_once(g_entry_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<PfnCtxGetCurrent>(fn);
        fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<PfnCtxGetId>(fn);
        cudaGetLastError();
    });
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != 0 || !ctx) return 0;
    if (g_ctx_get_id(ctx, &id) != 0) return 0;
    return id;
}

// Sum the partial rows in block order and write (not add) the totals.
__global__ void k_stats_write(const double *__restrict__ partial, int nblocks, double *__restrict__ out)
{
    const int k = threadIdx.x;
    if (k < kStatWidth) {
        double v = 0.0;
        for (int b = 0; b < nblocks; ++b) v += partial[(int64_t)b * kStatWidth + k];
        out[k] = v;
    }
}

template <class S>
cudaError_t sums_t(const void *pop, int64_t plane, int nx, int ny, int nz, double rho0, double *partial, int nblocks,
                   double *out, cudaStream_t st)
{
    cudaError_t e = launch_stats_partial<S>(static_cast<const S *>(pop), plane, kAAEven, nx, ny, nz, rho0, partial,
                                            nblocks, nullptr, st);
    if (e != cudaSuccess) return e;
    k_stats_write<<<1, 32, 0, st>>>(partial, nblocks, out);
    return cudaGetLastError();
}

}  // namespace
}  // namespace flb

extern "C" int flb_mode_sums_noalloc(const void *populations, int store, int64_t plane, int nx, int ny, int nz,
                                     double rho0, double *sums, void *stream)
{
    using namespace flb;
    if (!populations || !sums) return FLB_EINVAL;
    if (store < FLB_STORE_F64 || store > FLB_STORE_BF16SR) return FLB_EINVAL;
    if (store == FLB_STORE_BF16SR) store = FLB_STORE_BF16DEV;   // same bits; only the rounding differs
    if (nx < 1 || ny < 1 || nz < 1 || !(rho0 > 0.0)) return FLB_EINVAL;
    const int64_t N = (int64_t)nx * ny * nz;
    if (N > FLB_NOALLOC_MAX_SITES) return FLB_ERANGE;
    if (plane < N) return FLB_EINVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return FLB_ECUDA;
    }
    double *partial = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_addr_mu);
        const unsigned long long id = current_ctx_id();
        if (!g_addr[dev] || id == 0 || id != g_ctx_id[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_partial) != cudaSuccess || !p) {
                cudaGetLastError();
                g_addr[dev] = nullptr;
                return FLB_ECUDA;
            }
            g_addr[dev] = static_cast<double *>(p);
            g_ctx_id[dev] = current_ctx_id();   // the symbol lookup made the context current if it was not
        }
        partial = g_addr[dev];
    }
    const int nblocks = (int)((N + kSitesPerBlock - 1) / kSitesPerBlock);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    switch (store) {
    case FLB_STORE_F64: e = sums_t<double>(populations, plane, nx, ny, nz, rho0, partial, nblocks, sums, st); break;
    case FLB_STORE_F32: e = sums_t<float>(populations, plane, nx, ny, nz, rho0, partial, nblocks, sums, st); break;
    case FLB_STORE_F16DEV: e = sums_t<__half>(populations, plane, nx, ny, nz, rho0, partial, nblocks, sums, st); break;
    default: e = sums_t<__nv_bfloat16>(populations, plane, nx, ny, nz, rho0, partial, nblocks, sums, st); break;
    }
    return e == cudaSuccess ? FLB_OK : FLB_ECUDA;
}
