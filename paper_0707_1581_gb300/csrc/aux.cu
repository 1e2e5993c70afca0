// aux.cu -- kernels outside the time step: moments of gathered populations,
// the second pass of the statistics reduction, the device step counter, and
// the static structure factor (density field, 3-D DFT, shell sums).
#include "d2q9.cuh"
#include "d2q9_diag.cuh"
#include "diag_kernels.cuh"
#include "kernels.cuh"

namespace flb {

// --------------------------------------------------------------------------
// Streaming-pattern conversion: every stored element moves from the slot that
// holds the canonical population in layout `from` to its slot in layout `to`
// (a permutation of raw bits; src and dst are different buffers).
// --------------------------------------------------------------------------
template <class T, bool D2>
__global__ void k_relayout(const T *__restrict__ src, int from, T *__restrict__ dst, int to, int64_t plane, int nx,
                           int ny, int nz)
{
    const int64_t N = (int64_t)nx * ny * nz;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
        const int si = (int)s;
        const int x = si % nx, row = si / nx, y = row % ny, z = row / ny;
        if constexpr (D2) {
#pragma unroll
            for (int i = 0; i < d2::Q; ++i) {
                const d2::Slot2 a = d2::canonical_slot(from, i, x, y, nx, ny);
                const d2::Slot2 b = d2::canonical_slot(to, i, x, y, nx, ny);
                dst[(int64_t)b.q * plane + b.y * nx + b.x] = src[(int64_t)a.q * plane + a.y * nx + a.x];
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const Slot a = canonical_slot(from, i, x, y, z, nx, ny, nz);
                const Slot b = canonical_slot(to, i, x, y, z, nx, ny, nz);
                dst[(int64_t)b.q * plane + ((int64_t)b.z * ny + b.y) * nx + b.x] =
                    src[(int64_t)a.q * plane + ((int64_t)a.z * ny + a.y) * nx + a.x];
            }
        }
    }
}

template <class T>
cudaError_t relayout_t(const void *src, int from, void *dst, int to, int64_t plane, int nx, int ny, int nz, bool d2,
                       cudaStream_t st)
{
    int64_t g = ((int64_t)nx * ny * nz + 255) / 256;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    if (d2)
        k_relayout<T, true><<<(int)g, 256, 0, st>>>(static_cast<const T *>(src), from, static_cast<T *>(dst), to, plane,
                                                     nx, ny, nz);
    else
        k_relayout<T, false><<<(int)g, 256, 0, st>>>(static_cast<const T *>(src), from, static_cast<T *>(dst), to,
                                                      plane, nx, ny, nz);
    return cudaGetLastError();
}

// Non-finite stored values (all exponent bits set), counted from the raw bits.
template <class T>
__global__ void k_count_nonfinite(const T *__restrict__ buf, int64_t n, T expmask, unsigned long long *__restrict__ count)
{
    unsigned long long c = 0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x)
        c += (buf[s] & expmask) == expmask;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

cudaError_t launch_count_nonfinite(const void *buf, int64_t n, int store, unsigned long long *count, cudaStream_t st)
{
    int64_t g = (n + 255) / 256;
    if (g > 2432) g = 2432;
    if (g < 1) g = 1;
    switch (store) {
    case 0:   // FP64
        k_count_nonfinite<unsigned long long><<<(int)g, 256, 0, st>>>(static_cast<const unsigned long long *>(buf), n,
                                                                       0x7ff0000000000000ull, count);
        break;
    case 1:   // FP32
        k_count_nonfinite<uint32_t><<<(int)g, 256, 0, st>>>(static_cast<const uint32_t *>(buf), n, 0x7f800000u, count);
        break;
    case 2:   // binary16
        k_count_nonfinite<uint16_t><<<(int)g, 256, 0, st>>>(static_cast<const uint16_t *>(buf), n, (uint16_t)0x7c00,
                                                             count);
        break;
    default:  // bfloat16 (both roundings)
        k_count_nonfinite<uint16_t><<<(int)g, 256, 0, st>>>(static_cast<const uint16_t *>(buf), n, (uint16_t)0x7f80,
                                                             count);
        break;
    }
    return cudaGetLastError();
}

cudaError_t launch_relayout(const void *src, int from, void *dst, int to, size_t elem, int64_t plane, int nx, int ny,
                            int nz, bool d2, cudaStream_t st)
{
    switch (elem) {
    case 2: return relayout_t<uint16_t>(src, from, dst, to, plane, nx, ny, nz, d2, st);
    case 4: return relayout_t<uint32_t>(src, from, dst, to, plane, nx, ny, nz, d2, st);
    case 8: return relayout_t<uint64_t>(src, from, dst, to, plane, nx, ny, nz, d2, st);
    }
    return cudaErrorInvalidValue;
}

__global__ void k_advance_step(uint32_t *step_ptr, uint32_t by) { *step_ptr += by; }

__global__ void k_bm_tables(double *r, double2 *cs)
{
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < 65536u; k += gridDim.x * blockDim.x) {
        double rr, c, s;
        box_muller_entry(k, rr, c, s);
        r[k] = rr;
        cs[k] = make_double2(c, s);
    }
}

__global__ void k_guard_selftest(const unsigned char *buf, int64_t bytes, unsigned long long *viol)
{
    // spans of one byte-sized element in a one-plane view of the buffer
    span_ok<unsigned char, 1>(buf, bytes, buf - 1, 1, viol);
    span_ok<unsigned char, 1>(buf, bytes, buf + bytes, 1, viol);
    span_ok<unsigned char, 1>(buf, bytes, buf + bytes - 1, 1, viol);   // the last byte: inside
}

cudaError_t launch_guard_selftest(const void *buf, int64_t bytes, unsigned long long *viol, cudaStream_t st)
{
    k_guard_selftest<<<1, 1, 0, st>>>(static_cast<const unsigned char *>(buf), bytes, viol);
    return cudaGetLastError();
}

cudaError_t launch_bm_tables(void *tables, cudaStream_t st)
{
    double *r = static_cast<double *>(tables);
    k_bm_tables<<<256, 256, 0, st>>>(r, reinterpret_cast<double2 *>(r + 65536));
    return cudaGetLastError();
}

__global__ void k_set_step(uint32_t *step_ptr, uint32_t value) { *step_ptr = value; }

cudaError_t launch_advance_step(uint32_t *step_ptr, uint32_t by, cudaStream_t st)
{
    k_advance_step<<<1, 1, 0, st>>>(step_ptr, by);
    return cudaGetLastError();
}

cudaError_t launch_set_step(uint32_t *step_ptr, uint32_t value, cudaStream_t st)
{
    k_set_step<<<1, 1, 0, st>>>(step_ptr, value);
    return cudaGetLastError();
}

// rho = sum_i n_i, j = sum_i n_i c_i + F/2, Pi = sum_i n_i c_ia c_ib (xx, yy, zz, xy, yz, zx).
__global__ void k_moments(const double *__restrict__ n, int64_t slab, int nx, int ny, int nz, int z0,
                          double force_amp, double *__restrict__ rho, double *__restrict__ j, double *__restrict__ Pi)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < slab; s += (int64_t)gridDim.x * blockDim.x) {
        double r = 0, jx = 0, jy = 0, jz = 0, pxx = 0, pyy = 0, pzz = 0, pxy = 0, pyz = 0, pzx = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double v = n[i * slab + s];
            const double cx = vel_x(i), cy = vel_y(i), cz = vel_z(i);
            r += v;
            jx += v * cx;
            jy += v * cy;
            jz += v * cz;
            pxx += v * cx * cx;
            pyy += v * cy * cy;
            pzz += v * cz * cz;
            pxy += v * cx * cy;
            pyz += v * cy * cz;
            pzx += v * cz * cx;
        }
        if (force_amp != 0.0) {
            const int z = z0 + (int)s / (nx * ny);
            jx += 0.5 * force_amp * sinpi(2.0 * z / nz);
        }
        if (rho) rho[s] = r;
        if (j) {
            j[s] = jx;
            j[slab + s] = jy;
            j[2 * slab + s] = jz;
        }
        if (Pi) {
            Pi[s] = pxx;
            Pi[slab + s] = pyy;
            Pi[2 * slab + s] = pzz;
            Pi[3 * slab + s] = pxy;
            Pi[4 * slab + s] = pyz;
            Pi[5 * slab + s] = pzx;
        }
    }
}

cudaError_t launch_moments(const double *n, int64_t slab, int nx, int ny, int nz, int z0, double force_amp, double *rho,
                           double *j, double *Pi, cudaStream_t st)
{
    int64_t g = (slab + 255) / 256;
    if (g > 4096) g = 4096;
    k_moments<<<(int)g, 256, 0, st>>>(n, slab, nx, ny, nz, z0, force_amp, rho, j, Pi);
    return cudaGetLastError();
}

// At least 8 sites per thread (so the per-block reduction is amortised), and
// whole waves of the statistics kernel, whose blocks stride over the rows.
// D3Q19: one wave -- the kernel takes 120-128 registers, so an SM holds two
// of its 256-thread blocks (at 512^3, 1.68 ms per sample against 1.78 ms with
// the blocks of 4.5 waves).  D2Q9 (64-70 registers, three blocks per SM):
// three waves on 152 SMs, as before.
int stats_blocks(int64_t nsites, bool d2q9)
{
    // 2 x the SMs of the device current at first use
    static const int cap3 = [] {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
            cudaGetLastError();
            sms = 152;
        }
        return 2 * sms;
    }();
    const int cap = d2q9 ? 1368 : cap3;
    int64_t g = (nsites + 2047) / 2048;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

// One block of 32 x 8 threads: thread (k, j) sums rows j, j + 8, j + 16, ...
// of column k of the partials, then thread (k, 0) adds the eight sums in
// order -- a fixed order, so the result does not depend on scheduling.  It
// adds the column to the running sums, and thread 0 records the sample's total
// mass and momentum.
constexpr int kFinishRows = 8;
__device__ __forceinline__ void stats_finish_block(const double *__restrict__ partial, int nblocks,
                                                   double *__restrict__ acc)
{
    __shared__ double part[kFinishRows][32];
    __shared__ double col[kStatWidth];
    const int k = threadIdx.x, j = threadIdx.y;
    double v = 0.0;
    if (k < kStatWidth)
        for (int b = j; b < nblocks; b += kFinishRows) v += partial[(int64_t)b * kStatWidth + k];
    part[j][k] = v;
    __syncthreads();
    if (j == 0 && k < kStatWidth) {
        double s = 0.0;
#pragma unroll
        for (int r = 0; r < kFinishRows; ++r) s += part[r][k];
        col[k] = s;
        acc[kAccSums + k] += s;
    }
    __syncthreads();
    if (k == 0 && j == 0) {
        const bool first = acc[kAccCount] == 0.0;
        for (int c = 0; c < 4; ++c) {
            const double v = col[22 + c];
            if (first) acc[kAccFirst + c] = v;
            acc[kAccLast + c] = v;
        }
        acc[kAccCount] += 1.0;
    }
}

__global__ void __launch_bounds__(32 * kFinishRows) k_stats_finish(const double *__restrict__ partial, int nblocks,
                                                                    double *__restrict__ acc)
{
    stats_finish_block(partial, nblocks, acc);
}

// One block per box of a batch.
__global__ void __launch_bounds__(32 * kFinishRows) k_stats_finish_batch(const __grid_constant__ FinishTable T)
{
    const FinishBox &B = T.box[blockIdx.x];
    stats_finish_block(B.partial, B.nblocks, B.acc);
}

cudaError_t launch_stats_finish_batch(const FinishTable &T, cudaStream_t st)
{
    k_stats_finish_batch<<<T.nboxes, dim3(32, kFinishRows), 0, st>>>(T);
    return cudaGetLastError();
}

cudaError_t launch_stats_finish(const double *partial, int nblocks, double *acc, cudaStream_t st)
{
    k_stats_finish<<<1, dim3(32, kFinishRows), 0, st>>>(partial, nblocks, acc);
    return cudaGetLastError();
}

}  // namespace flb
