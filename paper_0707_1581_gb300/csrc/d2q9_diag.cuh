// d2q9_diag.cuh -- the D2Q9 kernels outside the time step: gather and scatter
// of canonical populations, the equilibrium initialisation, the statistics
// pass, row profiles and the density field of S(q) (Table I lattice, the same
// conventions as the D3Q19 diagnostics).
#pragma once

#include "d2q9.cuh"

namespace flb {
namespace d2 {

// Where the canonical pre-collision n_i(x, y) lives (same rules as D3Q19).
struct Slot2 {
    int q, x, y;
};

__device__ __forceinline__ Slot2 canonical_slot(int layout, int i, int x, int y, int nx, int ny)
{
    if (layout == kAAEven) return Slot2{i, x, y};
    return Slot2{layout == kAB ? i : opposite(i), wrap_add(x, -vel_x(i), nx), wrap_add(y, -vel_y(i), ny)};
}

// Canonical FP64 populations of rows [y0, y0 + nyc): out[i][local].
template <class S>
__global__ void k_gather(const S *__restrict__ buf, int64_t plane, int layout, int nx, int ny, int y0, int nyc,
                         double rho0, double *__restrict__ out)
{
    const int64_t slab = (int64_t)nyc * nx;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < slab; s += (int64_t)gridDim.x * blockDim.x) {
        const int si = (int)s;
        const int x = si % nx, y = y0 + si / nx;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const Slot2 sl = canonical_slot(layout, i, x, y, nx, ny);
            out[i * slab + s] = Storage<S>::to_double(buf[(int64_t)sl.q * plane + sl.y * nx + sl.x]) + rho0 * weight(i);
        }
    }
}

template <class S>
__global__ void k_gather_sites(const S *__restrict__ buf, int64_t plane, int layout, int nx, int ny, double rho0,
                               const int64_t *__restrict__ sites, int64_t nsites, double *__restrict__ out)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nsites; s += (int64_t)gridDim.x * blockDim.x) {
        const int site = (int)sites[s];
        const int x = site % nx, y = site / nx;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const Slot2 sl = canonical_slot(layout, i, x, y, nx, ny);
            out[s * Q + i] = Storage<S>::to_double(buf[(int64_t)sl.q * plane + sl.y * nx + sl.x]) + rho0 * weight(i);
        }
    }
}

template <class S>
__global__ void k_scatter(S *__restrict__ buf, int64_t plane, int layout, int nx, int ny, int y0, int nyc,
                          double rho0, const double *__restrict__ in)
{
    const int64_t slab = (int64_t)nyc * nx;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < slab; s += (int64_t)gridDim.x * blockDim.x) {
        const int si = (int)s;
        const int x = si % nx, y = y0 + si / nx;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const Slot2 sl = canonical_slot(layout, i, x, y, nx, ny);
            buf[(int64_t)sl.q * plane + sl.y * nx + sl.x] = Storage<S>::from_double(in[i * slab + s] - rho0 * weight(i));
        }
    }
}

// n = n^eq(rho0, u) (Eq. derived_equil_distrib, d = 2) for rows [y0, y0 + nyc); u[2][slab] or NULL (rest).
template <class S>
__global__ void k_init_equilibrium(S *__restrict__ buf, int64_t plane, int layout, int nx, int ny, int y0, int nyc,
                                   double rho0, const double *__restrict__ u)
{
    const int64_t slab = (int64_t)nyc * nx;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < slab; s += (int64_t)gridDim.x * blockDim.x) {
        const int si = (int)s;
        const int x = si % nx, y = y0 + si / nx;
        const double ux = u ? u[s] : 0.0, uy = u ? u[slab + s] : 0.0;
        const double u2 = ux * ux + uy * uy;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double cu = vel_x(i) * ux + vel_y(i) * uy;
            const double dev = rho0 * weight(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * u2);
            const Slot2 sl = canonical_slot(layout, i, x, y, nx, ny);
            buf[(int64_t)sl.q * plane + sl.y * nx + sl.x] = Storage<S>::from_double(dev);
        }
    }
}

// rho, j (+ F/2 along x) and Pi (xx, yy, xy) of gathered canonical populations.
__global__ void k_moments(const double *__restrict__ n, int64_t slab, int nx, int ny, int y0, double force_amp,
                          double *__restrict__ rho, double *__restrict__ j, double *__restrict__ Pi);

// Statistics partials in the D3Q19 layout of kStatWidth entries: [0..8] mode
// sums (9..18 zero), [19..20] sum u_a^2 ([21] zero), [22] sum rho, [23..24]
// sum j ([25] zero), [26] non-finite count.
template <class S>
__global__ void __launch_bounds__(256) k_stats_partial(const S *__restrict__ buf, int64_t plane, int layout, int nx,
                                                       int ny, double rho0, double *__restrict__ partial)
{
    // As the D3Q19 pass: R partials of 16 sites per lane, summed across the
    // warp at block-uniform points into per-warp FP64 rows (fixed orders).
    using R = typename Storage<S>::R;
    constexpr int W = 27, kWarps = 8;
    __shared__ double wsum[kWarps][W];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = lane; k < W; k += 32) wsum[warp][k] = 0.0;
    __syncwarp();
    const int64_t N = (int64_t)nx * ny;
    R part[W - 1];
#pragma unroll
    for (int k = 0; k < W - 1; ++k) part[k] = R(0);
    unsigned sites_ok = 0, nonfinite = 0;
    auto flush = [&]() {   // every lane of the warp calls it
#pragma unroll
        for (int k = 0; k < W - 1; ++k) {
            R v = part[k];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
            if (lane == 0) wsum[warp][k] += (double)v;
            part[k] = R(0);
        }
    };
    auto accumulate = [&](R (&d)[Q]) {
        bool finite = true;
#pragma unroll
        for (int i = 0; i < Q; ++i) finite = finite && isfinite(d[i]);
        if (!finite) {
            ++nonfinite;
            return;
        }
        const R sx = d[1] + d[2], dx = d[1] - d[2], sy = d[3] + d[4], dy = d[3] - d[4];
        const R sa = d[5] + d[6], da = d[5] - d[6], sb = d[7] + d[8], db = d[7] - d[8];
        const R A = sx + sy, Dg = sa + sb;
        R m[Q];
        m[0] = d[0] + A + Dg;
        m[1] = dx + (da + db);
        m[2] = dy + (da - db);
        m[3] = (A - R(2) * d[0]) + R(4) * Dg;
        m[4] = sx - sy;
        m[5] = sa - sb;
        m[6] = R(2) * (da + db) - dx;
        m[7] = R(2) * (da - db) - dy;
        m[8] = (R(2) * d[0] - R(4) * A) + R(8) * Dg;
#pragma unroll
        for (int k = 0; k < Q; ++k) part[k] += m[k] * m[k];
        const R inv_rho = R(1) / (R(rho0) + m[0]);
        const R ux = m[1] * inv_rho, uy = m[2] * inv_rho;
        part[19] += ux * ux;
        part[20] += uy * uy;
        part[22] += m[0];
        part[23] += m[1];
        part[24] += m[2];
        ++sites_ok;
    };
    constexpr int V = 4;
    bool done = false;
    if constexpr (sizeof(S) <= 4) {
      // four x-consecutive sites per lane with one aligned load per plane and
      // the x-shift by warp shuffle, as in the D3Q19 pass
      if (nx % V == 0 && plane % V == 0 && reinterpret_cast<uintptr_t>(buf) % (sizeof(S) * V) == 0) {
        using T = typename RawVec2<sizeof(S) * V>::T;
        const int gx = nx / V;
        const int64_t total = (int64_t)gx * ny;
        int since = 0;
        for (int64_t g0 = (int64_t)blockIdx.x * blockDim.x; g0 < total; g0 += (int64_t)gridDim.x * blockDim.x) {
            const int64_t gi = g0 + threadIdx.x;
            const bool valid = gi < total;
            const int g = (int)(valid ? gi : total - 1);
            const int x0 = V * (g % gx), y = g / gx;
            const int yo[3] = {(y == 0 ? ny - 1 : y - 1) * nx, y * nx, (y == ny - 1 ? 0 : y + 1) * nx};
            const bool shl = lane > 0 && x0 != 0, shr = lane < 31 && x0 + V != nx;
            const int x_lload = shl ? x0 : (x0 == 0 ? nx - 1 : x0 - 1);
            const int x_rload = shr ? x0 + V - 1 : (x0 + V == nx ? 0 : x0 + V);
            S raw[Q][V];
            S edge[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const bool own = layout == kAAEven;
                const int q = layout == kAAOdd ? opposite(i) : i;
                const S *base = buf + (int64_t)q * plane + (own ? yo[1] : yo[1 - vel_y(i)]);
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
                } else if (cx > 0) {
                    const R via = __shfl_up_sync(0xffffffffu, Storage<S>::load(raw[i][V - 1]), 1);
                    d[0][i] = shl ? via : Storage<S>::load(edge[i]);
#pragma unroll
                    for (int v = 1; v < V; ++v) d[v][i] = Storage<S>::load(raw[i][v - 1]);
                } else {
                    const R via = __shfl_down_sync(0xffffffffu, Storage<S>::load(raw[i][0]), 1);
#pragma unroll
                    for (int v = 0; v < V - 1; ++v) d[v][i] = Storage<S>::load(raw[i][v + 1]);
                    d[V - 1][i] = shr ? via : Storage<S>::load(edge[i]);
                }
            }
            if (valid) {
#pragma unroll
                for (int v = 0; v < V; ++v) accumulate(d[v]);
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
        int since = 0;
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t s0 = blockIdx.x * (int64_t)blockDim.x; s0 < N; s0 += stride) {   // block-uniform trip count
            const int64_t s = s0 + threadIdx.x;
            if (s < N) {
                const int si = (int)s;
                const int x = si % nx, y = si / nx;
                R d[Q];
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const Slot2 sl = canonical_slot(layout, i, x, y, nx, ny);
                    d[i] = Storage<S>::load(buf[(int64_t)sl.q * plane + sl.y * nx + sl.x]);
                }
                accumulate(d);
            }
            if (++since == 16) {
                flush();
                since = 0;
            }
        }
    }
    flush();
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
    if (threadIdx.x < W) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += wsum[w][threadIdx.x];
        partial[(int64_t)blockIdx.x * W + threadIdx.x] = v;
    }
}

// Row means of rho and j along y: one block per row.  out[y] = <rho>,
// out[ny + 3 y + a] = <j_a> (a = 0, 1; the third entry is 0).
template <class S>
__global__ void __launch_bounds__(256) k_y_profile(const S *__restrict__ buf, int64_t plane, int layout, int nx, int ny,
                                                   double rho0, double *__restrict__ out)
{
    const int y = blockIdx.x;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const Slot2 sl = canonical_slot(layout, i, x, y, nx, ny);
            const double v = Storage<S>::to_double(buf[(int64_t)sl.q * plane + sl.y * nx + sl.x]) + rho0 * weight(i);
            acc[0] += v;
            acc[1] += vel_x(i) * v;
            acc[2] += vel_y(i) * v;
        }
    }
    __shared__ double red[3][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double v = acc[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double v = 0.0;
        if (threadIdx.x < 3)
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
        v /= (double)nx;
        if (threadIdx.x == 0) out[y] = v;
        else out[ny + 3 * y + threadIdx.x - 1] = v;
    }
}

// rho(r) - rho0 (the sum of the stored deviations) in the compute type, the
// input of S(q).
template <class S>
__global__ void k_density(const S *__restrict__ buf, int64_t plane, int layout, int nx, int ny,
                          typename Storage<S>::R *__restrict__ field)
{
    using R = typename Storage<S>::R;
    const int64_t N = (int64_t)nx * ny;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < N; s += (int64_t)gridDim.x * blockDim.x) {
        const int si = (int)s;
        const int x = si % nx, y = si / nx;
        R r = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const Slot2 sl = canonical_slot(layout, i, x, y, nx, ny);
            r += Storage<S>::load(buf[(int64_t)sl.q * plane + sl.y * nx + sl.x]);
        }
        field[s] = r;
    }
}

}  // namespace d2
}  // namespace flb
