// rng.cu -- the device generator on its own, for checking it directly: the
// Philox-4x32-10 words and the Box-Muller normals that the stream-collide
// kernels draw (the same __device__ functions of d3q19.cuh), computed for
// arrays of counters or sites and copied to the host.
#include <cuda_runtime.h>

#include <vector>

#include "flb.h"
#include "d3q19.cuh"
#include "internal.h"

namespace flb {
namespace {

__global__ void k_philox(const uint32_t *__restrict__ ctr, const uint32_t *__restrict__ key, int64_t n,
                         uint32_t *__restrict__ out)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        uint32_t rk0[10], rk1[10];
        uint32_t k0 = key[2 * s], k1 = key[2 * s + 1];
        for (int r = 0; r < 10; ++r) {
            rk0[r] = k0;
            rk1[r] = k1;
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const Words4 w = philox4x32_10(ctr[4 * s], ctr[4 * s + 1], ctr[4 * s + 2], ctr[4 * s + 3], rk0, rk1);
        out[4 * s] = w.x;
        out[4 * s + 1] = w.y;
        out[4 * s + 2] = w.z;
        out[4 * s + 3] = w.w;
    }
}

// The sixteen normals of sites site0 .. site0 + n - 1 at (step, replica), in the
// compute type R; the FP32 ones are scaled back by sqrt(2 ln 2) (the kernels
// fold that factor into the noise amplitudes instead).
template <class R>
__global__ void k_normals(uint64_t seed, uint32_t step, uint32_t replica, uint32_t site0, int64_t n,
                          const BoxMullerTables T, double *__restrict__ out)
{
    uint32_t rk0[10], rk1[10];
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk0[r] = k0;
        rk1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    const double scale = sizeof(R) == 4 ? kBoxMullerF32Scale : 1.0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        R g[16];
        gaussians15<R>(site0 + (uint32_t)s, step, replica, rk0, rk1, T, g);
        for (int k = 0; k < 16; ++k) out[16 * s + k] = scale * (double)g[k];
    }
}

int grid_of(int64_t n)
{
    int64_t g = (n + 255) / 256;
    return (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
}

}  // namespace
}  // namespace flb

extern "C" {

int flb_philox4x32_10(const uint32_t *ctr, const uint32_t *key, int64_t n, uint32_t *out)
{
    if (n < 0 || (n > 0 && (!ctr || !key || !out))) return FLB_EINVAL;
    if (n == 0) return FLB_OK;
    uint32_t *d = nullptr;
    const size_t words = (size_t)n * 10;   // ctr 4n, key 2n, out 4n
    if (cudaMalloc(&d, words * sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        return FLB_ENOMEM;
    }
    int rc = FLB_OK;
    if (cudaMemcpy(d, ctr, 4 * n * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d + 4 * n, key, 2 * n * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = FLB_ECUDA;
    if (rc == FLB_OK) {
        flb::k_philox<<<flb::grid_of(n), 256>>>(d, d + 4 * n, n, d + 6 * n);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(out, d + 6 * n, 4 * n * sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = FLB_ECUDA;
    }
    cudaFree(d);
    cudaGetLastError();
    return rc;
}

int flb_normals(uint64_t seed, uint32_t step, uint32_t replica, uint32_t site0, int64_t nsites, int fp64,
                double *out)
{
    if (nsites < 0 || (nsites > 0 && !out) || (uint64_t)site0 + (uint64_t)nsites > 0x100000000ull) return FLB_EINVAL;
    if (nsites == 0) return FLB_OK;
    double *d = nullptr;
    const size_t nout = (size_t)nsites * 16 * sizeof(double);
    if (cudaMalloc(&d, nout + flb::kBoxMullerTableBytes) != cudaSuccess) {
        cudaGetLastError();
        return FLB_ENOMEM;
    }
    void *tables = reinterpret_cast<char *>(d) + nout;   // nout is a multiple of 128 bytes
    int rc = FLB_OK;
    if (fp64) {
        if (flb::launch_bm_tables(tables, 0) != cudaSuccess) rc = FLB_ECUDA;
        else
            flb::k_normals<double><<<flb::grid_of(nsites), 256>>>(seed, step, replica, site0, nsites,
                                                                   flb::bm_tables_of(tables), d);
    } else {
        flb::k_normals<float><<<flb::grid_of(nsites), 256>>>(seed, step, replica, site0, nsites,
                                                              flb::BoxMullerTables{nullptr, nullptr}, d);
    }
    if (rc == FLB_OK && (cudaGetLastError() != cudaSuccess ||
                         cudaMemcpy(out, d, nout, cudaMemcpyDeviceToHost) != cudaSuccess))
        rc = FLB_ECUDA;
    cudaFree(d);
    cudaGetLastError();
    return rc;
}

}  // extern "C"
