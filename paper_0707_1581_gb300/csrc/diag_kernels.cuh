// diag_kernels.cuh -- D3Q19 kernels outside the time step, templated on the
// storage format S: canonical gather/scatter of the populations, the rest or
// velocity-field initialisation, the per-block statistics pass, plane profiles
// and the density field of S(q); with their launch wrappers.  The
// step_<format>.cu files instantiate them (FLB_INSTANTIATE).
#pragma once

#include "d3q19.cuh"
#include "internal.h"

namespace flb {

namespace diag {
inline int grid_for(int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    return (int)g;
}
}  // namespace diag

// --------------------------------------------------------------------------
// Canonical gather / scatter over a slab of z-planes [z0, z0 + nzc).
// out[i][local] = n_i(r) as FP64 (deviation formats add rho0 a_i back).
// --------------------------------------------------------------------------
template <class S>
__global__ void k_gather(const S *__restrict__ buf, int64_t plane, int layout, int nx, int ny, int nz, int z0,
                         int nzc, double rho0, double *__restrict__ out)
{
    const int64_t slab = (int64_t)nzc * ny * nx;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < slab; s += (int64_t)gridDim.x * blockDim.x) {
        const int si = (int)s;   // < nx*ny*nz < 2^31: 32-bit index arithmetic
        const int x = si % nx;
        const int row = si / nx;
        const int y = row % ny;
        const int z = z0 + row / ny;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const Slot sl = canonical_slot(layout, i, x, y, z, nx, ny, nz);
            const int64_t idx = (int64_t)sl.q * plane + ((int64_t)sl.z * ny + sl.y) * nx + sl.x;
            double v = Storage<S>::to_double(buf[idx]);
            if (Storage<S>::dev) v += rho0 * weight(i);
            out[i * slab + s] = v;
        }
    }
}

// Canonical populations at a list of sites: out[s][i] = n_i(sites[s]).
template <class S>
__global__ void k_gather_sites(const S *__restrict__ buf, int64_t plane, int layout, int nx, int ny, int nz,
                               double rho0, const int64_t *__restrict__ sites, int64_t nsites, double *__restrict__ out)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nsites; s += (int64_t)gridDim.x * blockDim.x) {
        const int site = (int)sites[s];
        const int x = site % nx;
        const int row = site / nx;
        const int y = row % ny;
        const int z = row / ny;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const Slot sl = canonical_slot(layout, i, x, y, z, nx, ny, nz);
            double v = Storage<S>::to_double(buf[(int64_t)sl.q * plane + ((int64_t)sl.z * ny + sl.y) * nx + sl.x]);
            if (Storage<S>::dev) v += rho0 * weight(i);
            out[s * Q + i] = v;
        }
    }
}

template <class S>
__global__ void k_scatter(S *__restrict__ buf, int64_t plane, int layout, int nx, int ny, int nz, int z0, int nzc,
                          double rho0, const double *__restrict__ in)
{
    const int64_t slab = (int64_t)nzc * ny * nx;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < slab; s += (int64_t)gridDim.x * blockDim.x) {
        const int si = (int)s;   // < nx*ny*nz < 2^31: 32-bit index arithmetic
        const int x = si % nx;
        const int row = si / nx;
        const int y = row % ny;
        const int z = z0 + row / ny;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const Slot sl = canonical_slot(layout, i, x, y, z, nx, ny, nz);
            const int64_t idx = (int64_t)sl.q * plane + ((int64_t)sl.z * ny + sl.y) * nx + sl.x;
            double v = in[i * slab + s];
            if (Storage<S>::dev) v -= rho0 * weight(i);
            buf[idx] = Storage<S>::from_double(v);
        }
    }
}

// n_i = n_i^eq(rho0, u) of Eq. derived_equil_distrib (sigma_2 = 1/3) written
// as canonical populations of a slab; u = NULL means rest.
template <class S>
__global__ void k_init_equilibrium(S *__restrict__ buf, int64_t plane, int layout, int nx, int ny, int nz, int z0,
                                   int nzc, double rho0, const double *__restrict__ u)
{
    const int64_t slab = (int64_t)nzc * ny * nx;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < slab; s += (int64_t)gridDim.x * blockDim.x) {
        const int si = (int)s;   // < nx*ny*nz < 2^31: 32-bit index arithmetic
        const int x = si % nx;
        const int row = si / nx;
        const int y = row % ny;
        const int z = z0 + row / ny;
        double ux = 0.0, uy = 0.0, uz = 0.0;
        if (u) {
            ux = u[s];
            uy = u[slab + s];
            uz = u[2 * slab + s];
        }
        const double u2 = ux * ux + uy * uy + uz * uz;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double cu = vel_x(i) * ux + vel_y(i) * uy + vel_z(i) * uz;
            // deviation from rho0 a_i, computed without cancellation
            const double dev = rho0 * weight(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * u2);
            const double v = Storage<S>::dev ? dev : rho0 * weight(i) + dev;
            const Slot sl = canonical_slot(layout, i, x, y, z, nx, ny, nz);
            const int64_t idx = (int64_t)sl.q * plane + ((int64_t)sl.z * ny + sl.y) * nx + sl.x;
            buf[idx] = Storage<S>::from_double(v);
        }
    }
}

// rho, j (+ F/2) and Pi of gathered canonical populations (FP64).
__global__ void k_moments(const double *__restrict__ n, int64_t slab, int nx, int ny, int nz, int z0, double force_amp,
                          double *__restrict__ rho, double *__restrict__ j, double *__restrict__ Pi);

// --------------------------------------------------------------------------
// Statistics: per-block partial sums over the sites of one box, then a
// single-block pass that adds them, in a fixed order, to the FP64
// accumulators of the box.  Entries of a partial (kStatWidth doubles):
//   [0..18] sum_r m_k(n - rho0 a)^2, [19..21] sum (j/rho)^2, [22] sum rho,
//   [23..25] sum j, [26] non-finite count.
// --------------------------------------------------------------------------
constexpr int kStatWidth = 27;

// Raw vector of the statistics pass's aligned loads (four 4- or 2-byte elements).
template <int BYTES>
struct StatsVec;
template <>
struct StatsVec<16> {
    using T = uint4;
};
template <>
struct StatsVec<8> {
    using T = uint2;
};

// Block `bid` of `nb` blocks of one box (blockDim.x <= 256, whole warps): its
// rows' sums into row bid of partial.
template <class S>
__device__ __forceinline__ void stats_pass(const S *__restrict__ buf, int64_t plane, int layout, int nx, int ny, int nz,
                                           double rho0, double *__restrict__ partial, int bid, int nb,
                                           typename Storage<S>::R *__restrict__ rho_out)
{
    // Per site everything runs in the compute type R on the stored deviations
    // n_i - rho0 a_i.  Each lane keeps R partial sums of about 16 sites; at
    // warp-uniform points a warp adds its lanes' partials (fixed butterfly
    // order) and lane 0 adds the result to the warp's FP64 row in shared
    // memory, so FP64 arithmetic and the FP64 registers stay off the per-site
    // path.  Every order is fixed: the result is bitwise reproducible.
    using R = typename Storage<S>::R;
    constexpr int kWarps = 8;
    __shared__ double wsum[kWarps][kStatWidth];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = lane; k < kStatWidth; k += 32) wsum[warp][k] = 0.0;
    __syncwarp();
    R part[kStatWidth - 1];
#pragma unroll
    for (int k = 0; k < kStatWidth - 1; ++k) part[k] = R(0);
    unsigned sites_ok = 0, nonfinite = 0;
    auto flush = [&]() {   // every lane of the warp calls it
#pragma unroll
        for (int k = 0; k < kStatWidth - 1; ++k) {
            R v = part[k];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) wsum[warp][k] += (double)v;
            part[k] = R(0);
        }
    };
    // returns rho - rho0 of the site (non-finite if a population is)
    auto accumulate = [&](R (&d)[Q]) -> R {
        bool finite = true;
#pragma unroll
        for (int i = 0; i < Q; ++i) finite = finite && isfinite(d[i]);
        if (!finite) {
            ++nonfinite;
            R r = R(0);
#pragma unroll
            for (int i = 0; i < Q; ++i) r += d[i];
            return r;
        }
        R m[Q];
        forward_modes<R>(d, m);   // m0 = rho - rho0, m1..3 = j
#pragma unroll
        for (int k = 0; k < Q; ++k) part[k] += m[k] * m[k];
        const R inv_rho = R(1) / (R(rho0) + m[0]);
        const R ux = m[1] * inv_rho, uy = m[2] * inv_rho, uz = m[3] * inv_rho;
        part[19] += ux * ux;
        part[20] += uy * uy;
        part[21] += uz * uz;
        part[22] += m[0];
        part[23] += m[1];
        part[24] += m[2];
        part[25] += m[3];
        ++sites_ok;
        return m[0];
    };
    const int nxy = nx * ny;
    constexpr int V = 4;
    bool done = false;
    if constexpr (sizeof(S) <= 4) {
      // whole groups per row, and every group's address aligned for the
      // vector loads (the library's planes are multiples of 64 elements; a
      // caller's buffer of the allocation-free entry point may not be)
      if (nx % V == 0 && plane % V == 0 && reinterpret_cast<uintptr_t>(buf) % (sizeof(S) * V) == 0) {
        // Four x-consecutive sites per lane, one aligned 16- or 8-byte load per
        // plane; the x-shifted planes take the element beyond the group from
        // the neighbouring lane (which owns the adjacent group unless the group
        // starts or ends a row or the lane is at a warp edge), else from one
        // scalar load that every lane issues with its vector.  Groups are
        // dealt to the blocks in a block-uniform stride, so every lane of a
        // warp reaches every shuffle and flush.
        using T = typename StatsVec<sizeof(S) * V>::T;
        const int gx = nx / V;
        const int64_t total = (int64_t)gx * ny * nz;
        int since = 0;
        for (int64_t g0 = (int64_t)bid * blockDim.x; g0 < total; g0 += (int64_t)nb * blockDim.x) {
            const int64_t gi = g0 + threadIdx.x;
            const bool valid = gi < total;
            const int g = (int)(valid ? gi : total - 1);
            const int x0 = V * (g % gx), row = g / gx;
            const int y = row % ny, z = row / ny;
            const int yo[3] = {(y == 0 ? ny - 1 : y - 1) * nx, y * nx, (y == ny - 1 ? 0 : y + 1) * nx};
            const int zo[3] = {(z == 0 ? nz - 1 : z - 1) * nxy, z * nxy, (z == nz - 1 ? 0 : z + 1) * nxy};
            const bool shl = lane > 0 && x0 != 0, shr = lane < 31 && x0 + V != nx;
            const int x_lload = shl ? x0 : (x0 == 0 ? nx - 1 : x0 - 1);        // x0 - 1 (periodic)
            const int x_rload = shr ? x0 + V - 1 : (x0 + V == nx ? 0 : x0 + V);  // x0 + V (periodic)
            S raw[Q][V];
            S edge[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                // canonical slot: AA even slot i at r; AB slot i, AA odd slot opposite(i), at r - c_i
                const bool own = layout == kAAEven;
                const int q = layout == kAAOdd ? opposite(i) : i;
                const int ro = own ? zo[1] + yo[1] : zo[1 - vel_z(i)] + yo[1 - vel_y(i)];
                const S *base = buf + (int64_t)q * plane + ro;
                const T w = __ldg(reinterpret_cast<const T *>(base + x0));
                const S *e = reinterpret_cast<const S *>(&w);
#pragma unroll
                for (int v = 0; v < V; ++v) raw[i][v] = e[v];
                edge[i] = vel_x(i) > 0 ? base[x_lload] : (vel_x(i) < 0 ? base[x_rload] : raw[i][0]);
            }
            R d[V][Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int cx = layout == kAAEven ? 0 : vel_x(i);
                if (cx == 0) {
#pragma unroll
                    for (int v = 0; v < V; ++v) d[v][i] = Storage<S>::load(raw[i][v]);
                } else if (cx > 0) {   // canonical n_i(x) sits at x - 1
                    const R via = __shfl_up_sync(0xffffffffu, Storage<S>::load(raw[i][V - 1]), 1);
                    d[0][i] = shl ? via : Storage<S>::load(edge[i]);
#pragma unroll
                    for (int v = 1; v < V; ++v) d[v][i] = Storage<S>::load(raw[i][v - 1]);
                } else {               // at x + 1
                    const R via = __shfl_down_sync(0xffffffffu, Storage<S>::load(raw[i][0]), 1);
#pragma unroll
                    for (int v = 0; v < V - 1; ++v) d[v][i] = Storage<S>::load(raw[i][v + 1]);
                    d[V - 1][i] = shr ? via : Storage<S>::load(edge[i]);
                }
            }
            if (valid) {
                R r[V];
#pragma unroll
                for (int v = 0; v < V; ++v) r[v] = accumulate(d[v]);
                if (rho_out) {
                    R *o = rho_out + (int64_t)zo[1] + yo[1] + x0;   // 4 R-aligned: nx % 4 == 0
                    if constexpr (sizeof(R) == 4 && V == 4) *reinterpret_cast<float4 *>(o) = make_float4(r[0], r[1], r[2], r[3]);
                    else {
#pragma unroll
                        for (int v = 0; v < V; ++v) o[v] = r[v];
                    }
                }
            }
            if (++since == 4) {
                flush();
                since = 0;
            }
        }
        done = true;
      }
    }
    if (!done) {
        // rows (y, z) are spread over the blocks, x over the threads (several
        // short rows per block at a time): the nine neighbour rows and the
        // x-neighbours are selects, no division per site
        const int nrows = ny * nz;
        const int tpr = nx < (int)blockDim.x ? nx : (int)blockDim.x;   // threads per row
        const int rpi = (int)blockDim.x / tpr;                          // rows per block and iteration
        const int tr = (int)threadIdx.x / tpr, tx = (int)threadIdx.x % tpr;
        const int per_iter = (nx + tpr - 1) / tpr;                      // sites of a lane per iteration, at most
        const int every = per_iter >= 16 ? 1 : 16 / per_iter;           // iterations between flushes
        int since = 0;
        for (int row0 = bid * rpi; row0 < nrows; row0 += nb * rpi) {   // the same trip count for the whole block
            const int row = row0 + tr;
            if (tr < rpi && row < nrows) {
                const int y = row % ny, z = row / ny;
                const int yo[3] = {(y == 0 ? ny - 1 : y - 1) * nx, y * nx, (y == ny - 1 ? 0 : y + 1) * nx};
                const int zo[3] = {(z == 0 ? nz - 1 : z - 1) * nxy, z * nxy, (z == nz - 1 ? 0 : z + 1) * nxy};
                for (int x = tx; x < nx; x += tpr) {
                    const int xo[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};   // x - 1, x, x + 1
                    R d[Q];
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        const bool own = layout == kAAEven;
                        const int q = layout == kAAOdd ? opposite(i) : i;
                        const int off =
                            own ? zo[1] + yo[1] + x : zo[1 - vel_z(i)] + yo[1 - vel_y(i)] + xo[1 - vel_x(i)];
                        d[i] = Storage<S>::load(buf[(int64_t)q * plane + off]);
                    }
                    const R r = accumulate(d);
                    if (rho_out) rho_out[(int64_t)zo[1] + yo[1] + x] = r;
                }
            }
            if (++since == every) {
                flush();
                since = 0;
            }
        }
    }
    flush();
    // counts: sum of rho = sum of (rho - rho0) + rho0 per site; non-finite sites
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        sites_ok += __shfl_xor_sync(0xffffffffu, sites_ok, off);
        nonfinite += __shfl_xor_sync(0xffffffffu, nonfinite, off);
    }
    if (lane == 0) {
        wsum[warp][22] += rho0 * (double)sites_ok;
        wsum[warp][26] += (double)nonfinite;
    }
    __syncthreads();
    // block sum over the warps' rows in a fixed order
    if (threadIdx.x < kStatWidth) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += wsum[w][threadIdx.x];
        partial[(int64_t)bid * kStatWidth + threadIdx.x] = v;
    }
}

template <class S>
__global__ void __launch_bounds__(256) k_stats_partial(const S *__restrict__ buf, int64_t plane, int layout, int nx,
                                                       int ny, int nz, double rho0, double *__restrict__ partial,
                                                       typename Storage<S>::R *__restrict__ rho_out)
{
    stats_pass<S>(buf, plane, layout, nx, ny, nz, rho0, partial, (int)blockIdx.x, (int)gridDim.x, rho_out);
}

// All boxes of a batch in one launch: the box table is a kernel parameter;
// a block finds its box by a block-uniform binary search on block0.
template <class S>
struct StatsBox {
    const S *buf;
    double *partial;
    typename Storage<S>::R *rho_out;   // NULL, or rho - rho0 of every site (structure factor enabled)
    int64_t plane;
    double rho0;
    int nx, ny, nz;
    int nblocks;   // blocks (partial rows) of this box
    int block0;    // its first block in the launch
    int pad_;
};

template <class S>
struct StatsTable {
    int nboxes;
    int pad_;
    StatsBox<S> box[kStatsChunk];
};

template <class S>
__global__ void __launch_bounds__(256) k_stats_partial_batch(const __grid_constant__ StatsTable<S> T, int layout)
{
    int lo = 0, hi = T.nboxes - 1;
    const int b = (int)blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.box[mid].block0 <= b) lo = mid;
        else hi = mid - 1;
    }
    const StatsBox<S> &B = T.box[lo];
    stats_pass<S>(B.buf, B.plane, layout, B.nx, B.ny, B.nz, B.rho0, B.partial, b - B.block0, B.nblocks, B.rho_out);
}

// Means over each z-plane of rho and j = sum_i n_i c_i (FP64 sums of the
// stored values): one block per plane.  out[z] = <rho>, out[nz + 3 z + a] = <j_a>.
template <class S>
__global__ void __launch_bounds__(256) k_z_profile(const S *__restrict__ buf, int64_t plane, int layout, int nx, int ny,
                                                   int nz, double rho0, double *__restrict__ out)
{
    const int z = blockIdx.x;
    const int nxy = nx * ny;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int s = threadIdx.x; s < nxy; s += blockDim.x) {
        const int x = s % nx, y = s / nx;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const Slot sl = canonical_slot(layout, i, x, y, z, nx, ny, nz);
            double v = Storage<S>::to_double(buf[(int64_t)sl.q * plane + ((int64_t)sl.z * ny + sl.y) * nx + sl.x]);
            if (Storage<S>::dev) v += rho0 * weight(i);
            acc[0] += v;
            acc[1] += vel_x(i) * v;
            acc[2] += vel_y(i) * v;
            acc[3] += vel_z(i) * v;
        }
    }
    __shared__ double red[4][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double v = acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
        v /= (double)nxy;
        if (threadIdx.x == 0) out[z] = v;
        else out[nz + 3 * z + threadIdx.x - 1] = v;
    }
}

// rho(r) - rho0 of the canonical state as a complex FP64 field (for S(q)).
// Sums nblocks partials (fixed order) and adds them to acc[kStatWidth];
// also records the first and last total mass and momentum of the samples
// (acc layout described in internal.h).
__global__ void k_stats_finish(const double *__restrict__ partial, int nblocks, double *__restrict__ acc);


template <class S>
cudaError_t launch_gather(const S *buf, int64_t plane, int layout, int nx, int ny, int nz, int z0, int nzc,
                          double rho0, double *out, cudaStream_t st)
{
    const int64_t n = (int64_t)nx * ny * nzc;
    k_gather<S><<<diag::grid_for(n, 256), 256, 0, st>>>(buf, plane, layout, nx, ny, nz, z0, nzc, rho0, out);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_gather_sites(const S *buf, int64_t plane, int layout, int nx, int ny, int nz, double rho0,
                                const int64_t *sites, int64_t nsites, double *out, cudaStream_t st)
{
    k_gather_sites<S><<<diag::grid_for(nsites, 128), 128, 0, st>>>(buf, plane, layout, nx, ny, nz, rho0, sites,
                                                                      nsites, out);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_scatter(S *buf, int64_t plane, int layout, int nx, int ny, int nz, int z0, int nzc, double rho0,
                           const double *in, cudaStream_t st)
{
    const int64_t n = (int64_t)nx * ny * nzc;
    k_scatter<S><<<diag::grid_for(n, 256), 256, 0, st>>>(buf, plane, layout, nx, ny, nz, z0, nzc, rho0, in);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_init_equilibrium(S *buf, int64_t plane, int layout, int nx, int ny, int nz, int z0, int nzc,
                                    double rho0, const double *u, cudaStream_t st)
{
    const int64_t n = (int64_t)nx * ny * nzc;
    k_init_equilibrium<S><<<diag::grid_for(n, 256), 256, 0, st>>>(buf, plane, layout, nx, ny, nz, z0, nzc, rho0,
                                                                     u);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_stats_partial(const S *buf, int64_t plane, int layout, int nx, int ny, int nz, double rho0,
                                 double *partial, int nblocks, typename Storage<S>::R *rho_out, cudaStream_t st)
{
    k_stats_partial<S><<<nblocks, 256, 0, st>>>(buf, plane, layout, nx, ny, nz, rho0, partial, rho_out);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_stats_partial_batch(const StatsTable<S> &T, int total_blocks, int layout, cudaStream_t st)
{
    k_stats_partial_batch<S><<<total_blocks, 256, 0, st>>>(T, layout);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_z_profile(const S *buf, int64_t plane, int layout, int nx, int ny, int nz, double rho0, double *out,
                             cudaStream_t st)
{
    k_z_profile<S><<<nz, 256, 0, st>>>(buf, plane, layout, nx, ny, nz, rho0, out);
    return cudaGetLastError();
}


}  // namespace flb
