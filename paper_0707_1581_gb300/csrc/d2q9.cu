// d2q9.cu -- launch wrappers of the D2Q9 kernels (d2q9.cuh) for every
// storage format, and the FP64 moments of gathered D2Q9 populations.
#include "d2q9.cuh"
#include "d2q9_diag.cuh"

namespace flb {
namespace d2 {

namespace {

int grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    if (g > 4096) g = 4096;
    return g < 1 ? 1 : (int)g;
}

template <class S, int LAYOUT>
cudaError_t step_layout(const BoxStep<S> &b, bool noise, bool force, dim3 grid, dim3 block, const uint32_t *p,
                        uint32_t t, cudaStream_t st)
{
    if (noise && force) k_stream_collide<S, LAYOUT, true, true><<<grid, block, 0, st>>>(b, p, t);
    else if (noise) k_stream_collide<S, LAYOUT, true, false><<<grid, block, 0, st>>>(b, p, t);
    else if (force) k_stream_collide<S, LAYOUT, false, true><<<grid, block, 0, st>>>(b, p, t);
    else k_stream_collide<S, LAYOUT, false, false><<<grid, block, 0, st>>>(b, p, t);
    return cudaGetLastError();
}

// V sites per thread: 16-byte accesses for 4-byte formats, 8-byte for 16-bit, V = 2 for FP64.
template <class S>
constexpr int vec_width()
{
    return sizeof(S) == 8 ? 2 : 4;
}

template <class S, int LAYOUT>
cudaError_t step_layout_vec(const BoxStep<S> &b, bool noise, bool force, dim3 grid, dim3 block, const uint32_t *p,
                            uint32_t t, cudaStream_t st)
{
    constexpr int V = vec_width<S>();
    if (noise && force) k_stream_collide_vec<S, LAYOUT, true, true, V><<<grid, block, 0, st>>>(b, p, t);
    else if (noise) k_stream_collide_vec<S, LAYOUT, true, false, V><<<grid, block, 0, st>>>(b, p, t);
    else if (force) k_stream_collide_vec<S, LAYOUT, false, true, V><<<grid, block, 0, st>>>(b, p, t);
    else k_stream_collide_vec<S, LAYOUT, false, false, V><<<grid, block, 0, st>>>(b, p, t);
    return cudaGetLastError();
}

}  // namespace

template <class S>
cudaError_t launch_step(const BoxStep<S> &b, int layout, bool noise, bool force, int bx, int by, int V,
                        const uint32_t *step_ptr, uint32_t step, cudaStream_t st)
{
    if (V > 1) {
        // vectorised: needs nx % V == 0 and whole warps
        constexpr int W = vec_width<S>();
        const int T = bx * by;
        if (b.nx % W != 0 || T % 32 != 0 || T > 256) return cudaErrorInvalidValue;
        const int64_t items = (int64_t)(b.nx / W) * b.ny;
        const dim3 grid((unsigned)((items + T - 1) / T)), block(bx, by, 1);
        switch (layout) {
        case kAB: return step_layout_vec<S, kAB>(b, noise, force, grid, block, step_ptr, step, st);
        case kAAEven: return step_layout_vec<S, kAAEven>(b, noise, force, grid, block, step_ptr, step, st);
        default: return step_layout_vec<S, kAAOdd>(b, noise, force, grid, block, step_ptr, step, st);
        }
    }
    const int gy = (b.ny + by - 1) / by;
    const int64_t blocks = (int64_t)b.gx * gy;
    if (blocks > 0x7FFFFFFF || bx * by > 256 || bx < 1 || by < 1) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)blocks), block(bx, by, 1);
    switch (layout) {
    case kAB: return step_layout<S, kAB>(b, noise, force, grid, block, step_ptr, step, st);
    case kAAEven: return step_layout<S, kAAEven>(b, noise, force, grid, block, step_ptr, step, st);
    default: return step_layout<S, kAAOdd>(b, noise, force, grid, block, step_ptr, step, st);
    }
}

template <class S>
cudaError_t launch_gather(const S *buf, int64_t plane, int layout, int nx, int ny, int y0, int nyc, double rho0,
                          double *out, cudaStream_t st)
{
    k_gather<S><<<grid_for((int64_t)nx * nyc, 256), 256, 0, st>>>(buf, plane, layout, nx, ny, y0, nyc, rho0, out);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_gather_sites(const S *buf, int64_t plane, int layout, int nx, int ny, double rho0,
                                const int64_t *sites, int64_t nsites, double *out, cudaStream_t st)
{
    k_gather_sites<S><<<grid_for(nsites, 256), 256, 0, st>>>(buf, plane, layout, nx, ny, rho0, sites, nsites, out);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_scatter(S *buf, int64_t plane, int layout, int nx, int ny, int y0, int nyc, double rho0,
                           const double *in, cudaStream_t st)
{
    k_scatter<S><<<grid_for((int64_t)nx * nyc, 256), 256, 0, st>>>(buf, plane, layout, nx, ny, y0, nyc, rho0, in);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_init_equilibrium(S *buf, int64_t plane, int layout, int nx, int ny, int y0, int nyc, double rho0,
                                    const double *u, cudaStream_t st)
{
    k_init_equilibrium<S><<<grid_for((int64_t)nx * nyc, 256), 256, 0, st>>>(buf, plane, layout, nx, ny, y0, nyc,
                                                                           rho0, u);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_stats_partial(const S *buf, int64_t plane, int layout, int nx, int ny, double rho0,
                                 double *partial, int nblocks, cudaStream_t st)
{
    k_stats_partial<S><<<nblocks, 256, 0, st>>>(buf, plane, layout, nx, ny, rho0, partial);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_y_profile(const S *buf, int64_t plane, int layout, int nx, int ny, double rho0, double *out,
                             cudaStream_t st)
{
    k_y_profile<S><<<ny, 256, 0, st>>>(buf, plane, layout, nx, ny, rho0, out);
    return cudaGetLastError();
}

template <class S>
cudaError_t launch_density(const S *buf, int64_t plane, int layout, int nx, int ny, typename Storage<S>::R *field,
                           cudaStream_t st)
{
    k_density<S><<<grid_for((int64_t)nx * ny, 256), 256, 0, st>>>(buf, plane, layout, nx, ny, field);
    return cudaGetLastError();
}

__global__ void k_moments(const double *__restrict__ n, int64_t slab, int nx, int ny, int y0, double force_amp,
                          double *__restrict__ rho, double *__restrict__ j, double *__restrict__ Pi)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < slab; s += (int64_t)gridDim.x * blockDim.x) {
        double r = 0, jx = 0, jy = 0, pxx = 0, pyy = 0, pxy = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double v = n[i * slab + s];
            const double cx = vel_x(i), cy = vel_y(i);
            r += v;
            jx += v * cx;
            jy += v * cy;
            pxx += v * cx * cx;
            pyy += v * cy * cy;
            pxy += v * cx * cy;
        }
        if (force_amp != 0.0) {
            const int y = y0 + (int)(s / nx);
            jx += 0.5 * force_amp * sinpi(2.0 * y / ny);
        }
        if (rho) rho[s] = r;
        if (j) {
            j[s] = jx;
            j[slab + s] = jy;
        }
        if (Pi) {
            Pi[s] = pxx;
            Pi[slab + s] = pyy;
            Pi[2 * slab + s] = pxy;
        }
    }
}

cudaError_t launch_moments(const double *n, int64_t slab, int nx, int ny, int y0, double force_amp, double *rho,
                           double *j, double *Pi, cudaStream_t st)
{
    k_moments<<<grid_for(slab, 256), 256, 0, st>>>(n, slab, nx, ny, y0, force_amp, rho, j, Pi);
    return cudaGetLastError();
}

#define FLB_D2_INSTANTIATE(S)                                                                                       \
    template cudaError_t launch_step<S>(const BoxStep<S> &, int, bool, bool, int, int, int, const uint32_t *,      \
                                        uint32_t, cudaStream_t);                                                    \
    template cudaError_t launch_gather<S>(const S *, int64_t, int, int, int, int, int, double, double *,           \
                                          cudaStream_t);                                                            \
    template cudaError_t launch_gather_sites<S>(const S *, int64_t, int, int, int, double, const int64_t *,        \
                                                int64_t, double *, cudaStream_t);                                   \
    template cudaError_t launch_scatter<S>(S *, int64_t, int, int, int, int, int, double, const double *,          \
                                           cudaStream_t);                                                           \
    template cudaError_t launch_init_equilibrium<S>(S *, int64_t, int, int, int, int, int, double, const double *, \
                                                    cudaStream_t);                                                  \
    template cudaError_t launch_stats_partial<S>(const S *, int64_t, int, int, int, double, double *, int,         \
                                                 cudaStream_t);                                                     \
    template cudaError_t launch_y_profile<S>(const S *, int64_t, int, int, int, double, double *, cudaStream_t);   \
    template cudaError_t launch_density<S>(const S *, int64_t, int, int, int, typename Storage<S>::R *, cudaStream_t);

FLB_D2_INSTANTIATE(double)
FLB_D2_INSTANTIATE(float)
FLB_D2_INSTANTIATE(__half)
FLB_D2_INSTANTIATE(__nv_bfloat16)
FLB_D2_INSTANTIATE(bf16sr)

}  // namespace d2
}  // namespace flb
