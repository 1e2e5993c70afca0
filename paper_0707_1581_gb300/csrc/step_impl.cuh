// step_impl.cuh -- launch wrappers of the templated kernels; included by the
// step_<format>.cu files, each of which instantiates them for one storage
// format so the formats compile in parallel.
#pragma once

#include "diag_kernels.cuh"
#include "kernels.cuh"

namespace flb {

namespace detail {

template <class S, int LAYOUT, int NOISE, bool FORCE, int V>
cudaError_t step_one(const BoxStep<S> &b, const Launch &L, const uint32_t *step_ptr, uint32_t step, cudaStream_t st)
{
    const int sites_x = L.bx * V;
    dim3 grid((b.nx + sites_x - 1) / sites_x, (b.ny + L.by - 1) / L.by, b.nzl);
    dim3 block(L.bx, L.by, 1);
    if constexpr (V == 4 && sizeof(S) <= 4) {
        if (L.fullrow) {
            if (L.by == 1 && (uint64_t)Q * (uint64_t)b.plane < (1ull << 32)) {
                if constexpr (Storage<S>::stochastic) {
                    if (L.bx <= 128) {   // the register-capped kernel takes at most 128 threads a block
                        k_stream_collide_row4<S, LAYOUT, NOISE, FORCE, V><<<grid, block, 0, st>>>(b, step_ptr, step);
                        return cudaGetLastError();
                    }
                }
                k_stream_collide<S, LAYOUT, NOISE, FORCE, V, true, false, true><<<grid, block, 0, st>>>(b, step_ptr, step);
            } else {
                k_stream_collide<S, LAYOUT, NOISE, FORCE, V, true><<<grid, block, 0, st>>>(b, step_ptr, step);
            }
            return cudaGetLastError();
        }
    }
    if constexpr (V > 1) {
        if (L.warprow) {
            k_stream_collide<S, LAYOUT, NOISE, FORCE, V, false, true><<<grid, block, 0, st>>>(b, step_ptr, step);
            return cudaGetLastError();
        }
    }
    k_stream_collide<S, LAYOUT, NOISE, FORCE, V><<<grid, block, 0, st>>>(b, step_ptr, step);
    return cudaGetLastError();
}

template <class S, int LAYOUT, int NOISE, bool FORCE, int V>
cudaError_t step_batch(const BatchParams<S> &P, int total_blocks, const Launch &L, const uint32_t *step_ptr,
                       uint32_t step, cudaStream_t st)
{
    dim3 block(L.bx, L.by, 1);
    k_stream_collide_batch<S, LAYOUT, NOISE, FORCE, V><<<total_blocks, block, 0, st>>>(P, step_ptr, step);
    return cudaGetLastError();
}

template <class S, int LAYOUT, int NOISE, bool FORCE>
cudaError_t step_v(const BoxStep<S> &b, const Launch &L, const uint32_t *p, uint32_t t, cudaStream_t st)
{
    switch (L.V) {
    case 1: return step_one<S, LAYOUT, NOISE, FORCE, 1>(b, L, p, t, st);
    case 2: return step_one<S, LAYOUT, NOISE, FORCE, 2>(b, L, p, t, st);
    case 4: return step_one<S, LAYOUT, NOISE, FORCE, (sizeof(S) * 4 > 16 ? 2 : 4)>(b, L, p, t, st);
    }
    return cudaErrorInvalidValue;
}

template <class S, int LAYOUT, int NOISE, bool FORCE>
cudaError_t batch_v(const BatchParams<S> &P, int tb, const Launch &L, const uint32_t *p, uint32_t t, cudaStream_t st)
{
    switch (L.V) {
    case 1: return step_batch<S, LAYOUT, NOISE, FORCE, 1>(P, tb, L, p, t, st);
    case 2: return step_batch<S, LAYOUT, NOISE, FORCE, 2>(P, tb, L, p, t, st);
    case 4: return step_batch<S, LAYOUT, NOISE, FORCE, (sizeof(S) * 4 > 16 ? 2 : 4)>(P, tb, L, p, t, st);
    }
    return cudaErrorInvalidValue;
}

template <class S, int LAYOUT>
cudaError_t step_nf(const BoxStep<S> &b, int noise, bool force, const Launch &L, const uint32_t *p, uint32_t t,
                    cudaStream_t st)
{
    if (noise == 2) return force ? step_v<S, LAYOUT, 2, true>(b, L, p, t, st) : step_v<S, LAYOUT, 2, false>(b, L, p, t, st);
    if (noise) return force ? step_v<S, LAYOUT, 1, true>(b, L, p, t, st) : step_v<S, LAYOUT, 1, false>(b, L, p, t, st);
    return force ? step_v<S, LAYOUT, 0, true>(b, L, p, t, st) : step_v<S, LAYOUT, 0, false>(b, L, p, t, st);
}

template <class S, int LAYOUT>
cudaError_t batch_nf(const BatchParams<S> &P, int tb, int noise, bool force, const Launch &L, const uint32_t *p,
                     uint32_t t, cudaStream_t st)
{
    if (noise == 2)
        return force ? batch_v<S, LAYOUT, 2, true>(P, tb, L, p, t, st) : batch_v<S, LAYOUT, 2, false>(P, tb, L, p, t, st);
    if (noise)
        return force ? batch_v<S, LAYOUT, 1, true>(P, tb, L, p, t, st) : batch_v<S, LAYOUT, 1, false>(P, tb, L, p, t, st);
    return force ? batch_v<S, LAYOUT, 0, true>(P, tb, L, p, t, st) : batch_v<S, LAYOUT, 0, false>(P, tb, L, p, t, st);
}

inline int grid_for(int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace detail

template <class S>
cudaError_t launch_step(const BoxStep<S> &b, int layout, int noise, bool force, const Launch &L,
                        const uint32_t *step_ptr, uint32_t step, cudaStream_t st)
{
    switch (layout) {
    case kAB: return detail::step_nf<S, kAB>(b, noise, force, L, step_ptr, step, st);
    case kAAEven: return detail::step_nf<S, kAAEven>(b, noise, force, L, step_ptr, step, st);
    case kAAOdd: return detail::step_nf<S, kAAOdd>(b, noise, force, L, step_ptr, step, st);
    }
    return cudaErrorInvalidValue;
}

template <class S>
cudaError_t launch_step_batch(const BatchParams<S> &P, int total_blocks, int layout, int noise, bool force,
                              const Launch &L, const uint32_t *step_ptr, uint32_t step, cudaStream_t st)
{
    switch (layout) {
    case kAB: return detail::batch_nf<S, kAB>(P, total_blocks, noise, force, L, step_ptr, step, st);
    case kAAEven: return detail::batch_nf<S, kAAEven>(P, total_blocks, noise, force, L, step_ptr, step, st);
    case kAAOdd: return detail::batch_nf<S, kAAOdd>(P, total_blocks, noise, force, L, step_ptr, step, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace flb

// The stream-collide kernels of one storage format S and one layout L
// (instantiated in step_<format>_<layout>.cu, so the 15 kernel TUs compile in
// parallel); the dispatching TU declares them extern.
#define FLB_LAYOUT_FUNCS(PREFIX, S, L)                                                                              \
    namespace flb {                                                                                                 \
    namespace detail {                                                                                              \
    PREFIX template cudaError_t step_nf<S, L>(const BoxStep<S> &, int, bool, const Launch &, const uint32_t *,      \
                                              uint32_t, cudaStream_t);                                              \
    PREFIX template cudaError_t batch_nf<S, L>(const BatchParams<S> &, int, int, bool, const Launch &,              \
                                               const uint32_t *, uint32_t, cudaStream_t);                           \
    }                                                                                                               \
    }
#define FLB_INSTANTIATE_LAYOUT(S, L) FLB_LAYOUT_FUNCS(, S, L)

#define FLB_INSTANTIATE(S)                                                                                          \
    FLB_LAYOUT_FUNCS(extern, S, kAB)                                                                                \
    FLB_LAYOUT_FUNCS(extern, S, kAAEven)                                                                            \
    FLB_LAYOUT_FUNCS(extern, S, kAAOdd)                                                                             \
    namespace flb {                                                                                                 \
    template cudaError_t launch_step<S>(const BoxStep<S> &, int, int, bool, const Launch &, const uint32_t *,       \
                                        uint32_t, cudaStream_t);                                                    \
    template cudaError_t launch_step_batch<S>(const BatchParams<S> &, int, int, int, bool, const Launch &,         \
                                              const uint32_t *, uint32_t, cudaStream_t);                            \
    template cudaError_t launch_gather<S>(const S *, int64_t, int, int, int, int, int, int, double, double *,      \
                                          cudaStream_t);                                                            \
    template cudaError_t launch_gather_sites<S>(const S *, int64_t, int, int, int, int, double, const int64_t *,    \
                                                int64_t, double *, cudaStream_t);                                   \
    template cudaError_t launch_scatter<S>(S *, int64_t, int, int, int, int, int, int, double, const double *,     \
                                           cudaStream_t);                                                           \
    template cudaError_t launch_init_equilibrium<S>(S *, int64_t, int, int, int, int, int, int, double,            \
                                                    const double *, cudaStream_t);                                  \
    template cudaError_t launch_stats_partial<S>(const S *, int64_t, int, int, int, int, double, double *, int,    \
                                                 typename Storage<S>::R *, cudaStream_t);                           \
    template cudaError_t launch_stats_partial_batch<S>(const StatsTable<S> &, int, int, cudaStream_t);             \
    template cudaError_t launch_z_profile<S>(const S *, int64_t, int, int, int, int, double, double *, cudaStream_t); \
    }
