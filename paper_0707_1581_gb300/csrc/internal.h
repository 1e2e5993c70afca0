// internal.h -- declarations shared by the .cu files of the library (not part
// of the C ABI).  The launch_* wrappers are instantiated once per storage
// format in step_<format>.cu; the host runtime (api.cu) calls them.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "d3q19.cuh"

namespace flb {

template <class S>
struct BoxStep;
template <class S>
struct BatchParams;

// Accumulator block of one box (doubles): [0, kStatWidth) running sums of the
// partials, then the sample count, then first/last mass and momentum.
constexpr int kAccSums = 0;
constexpr int kAccCount = 27;       // number of samples (stored as double)
constexpr int kAccFirst = 28;       // mass, jx, jy, jz at the first sample
constexpr int kAccLast = 32;        // mass, jx, jy, jz at the last sample
constexpr int kAccWidth = 36;

// Launch shape of the stream-collide kernels.
struct Launch {
    int V = 1;        // x-consecutive sites per thread
    int bx = 64;      // block threads along x
    int by = 4;       // block threads along y
    bool fullrow = false;   // one box, bx * V == nx, whole warps: edge exchange inside the block
    bool warprow = false;   // one box, bx * V == nx, bx divides 32: rows tile the warps, shuffles only
};

// The FP64 Box-Muller tables (BoxMullerTables): r[65536] then cs[65536] in one
// allocation of kBoxMullerTableBytes, filled by one launch.
constexpr size_t kBoxMullerTableBytes = 65536 * (sizeof(double) + sizeof(double2));
cudaError_t launch_bm_tables(void *tables, cudaStream_t st);
inline BoxMullerTables bm_tables_of(void *tables)
{
    const double *r = static_cast<const double *>(tables);
    return BoxMullerTables{r, reinterpret_cast<const double2 *>(r + 65536)};
}

// The guard of the checking build on two spans just outside a buffer of `bytes`
// bytes (one element before it, one past its end): two violations, no access.
cudaError_t launch_guard_selftest(const void *buf, int64_t bytes, unsigned long long *viol, cudaStream_t st);

// noise: 0 deterministic, 1 thermal, 2 thermal with gamma_ghost = 0 in every box.
template <class S>
cudaError_t launch_step(const BoxStep<S> &b, int layout, int noise, bool force, const Launch &L,
                        const uint32_t *step_ptr, uint32_t step, cudaStream_t st);

template <class S>
cudaError_t launch_step_batch(const BatchParams<S> &P, int total_blocks, int layout, int noise, bool force,
                              const Launch &L, const uint32_t *step_ptr, uint32_t step, cudaStream_t st);

template <class S>
cudaError_t launch_gather(const S *buf, int64_t plane, int layout, int nx, int ny, int nz, int z0, int nzc,
                          double rho0, double *out, cudaStream_t st);

template <class S>
cudaError_t launch_gather_sites(const S *buf, int64_t plane, int layout, int nx, int ny, int nz, double rho0,
                                const int64_t *sites, int64_t nsites, double *out, cudaStream_t st);

template <class S>
cudaError_t launch_scatter(S *buf, int64_t plane, int layout, int nx, int ny, int nz, int z0, int nzc, double rho0,
                           const double *in, cudaStream_t st);

template <class S>
cudaError_t launch_init_equilibrium(S *buf, int64_t plane, int layout, int nx, int ny, int nz, int z0, int nzc,
                                    double rho0, const double *u, cudaStream_t st);

// Blocks used by launch_stats_partial (size of the partial-sum scratch /
// kStatWidth); depends only on the box size, the lattice and the device.
int stats_blocks(int64_t nsites, bool d2q9);

// rho_out (NULL: not written): rho - rho0 of every site, in the compute type,
// [z][y][x] contiguous (the input of the structure factor).
template <class S>
cudaError_t launch_stats_partial(const S *buf, int64_t plane, int layout, int nx, int ny, int nz, double rho0,
                                 double *partial, int nblocks, typename Storage<S>::R *rho_out, cudaStream_t st);

cudaError_t launch_stats_finish(const double *partial, int nblocks, double *acc, cudaStream_t st);

// Statistics of every box of a batch in two launches (box tables as kernel parameters).
constexpr int kStatsChunk = 256;   // boxes per launch
template <class S>
struct StatsTable;
template <class S>
cudaError_t launch_stats_partial_batch(const StatsTable<S> &T, int total_blocks, int layout, cudaStream_t st);
struct FinishBox {
    const double *partial;
    double *acc;
    int nblocks;
    int pad_;
};
struct FinishTable {
    int nboxes;
    int pad_;
    FinishBox box[kStatsChunk];
};
cudaError_t launch_stats_finish_batch(const FinishTable &T, cudaStream_t st);

cudaError_t launch_moments(const double *n, int64_t slab, int nx, int ny, int nz, int z0, double force_amp,
                           double *rho, double *j, double *Pi, cudaStream_t st);

cudaError_t launch_advance_step(uint32_t *step_ptr, uint32_t by, cudaStream_t st);

// Counts the stored values of a state buffer (n elements, format `store` =
// flb_store_t) whose exponent bits are all set; adds the count to *count.
cudaError_t launch_count_nonfinite(const void *buf, int64_t n, int store, unsigned long long *count, cudaStream_t st);

// Moves every stored element of a box from its layout-`from` slot to its
// layout-`to` slot (raw bits, elem bytes each; src != dst); d2 selects D2Q9.
cudaError_t launch_relayout(const void *src, int from, void *dst, int to, size_t elem, int64_t plane, int nx, int ny,
                            int nz, bool d2, cudaStream_t st);
cudaError_t launch_set_step(uint32_t *step_ptr, uint32_t value, cudaStream_t st);

template <class S>
cudaError_t launch_z_profile(const S *buf, int64_t plane, int layout, int nx, int ny, int nz, double rho0, double *out,
                             cudaStream_t st);

// Static structure factor (sq.cu).  The density deviation rho - rho0 of a box
// (written by the statistics pass, or for D2Q9 by d2::launch_density) in the
// transform type (FP64 for the FP64 format, else FP32) is transformed to its
// half spectrum and |.|^2 / N is added into FP64 shell sums.
struct SqRadices {
    int n;          // number of stages
    int r[20];      // radix of each stage
};
struct SqShells {
    double *sum;                    // nshells FP64 sums over the samples
    unsigned long long *fixed;      // FP32 transform: nshells fixed-point sums of one sample
    uint32_t *maxbits;              // FP32 transform: bits of the sample's largest |rho - rho0|
    int nshells;
    int nx, ny, nz, nmax;
};
struct SqPlan {
    int nx, ny, nz, nmax, nshells;
    int P;              // row stride (complex elements) of the half spectrum, >= nx / 2 + 1
    bool dbl;           // FP64 transform
    void *rho;          // nx ny nz reals: rho - rho0
    void *X;            // P ny nz complex: the half spectrum
    void *tw;           // nx + ny + nz complex: exp(-2 pi i m / L) for the three lengths
    double *shell_sum;  // nshells
    uint16_t *shell_tab;  // sq_table_elems entries: the shell of every half-spectrum wave vector
    unsigned long long *shell_fixed;   // nshells (FP32 transform scratch)
    uint32_t *maxbits;                 // one word (FP32 transform scratch)
};
int sq_shells(int nx, int ny, int nz);
int sq_row_stride(int nx, bool dbl);
size_t sq_elem_bytes(bool dbl);
bool sq_supported(int nx, int ny, int nz, bool dbl);
int64_t sq_table_elems(int nx, int ny, int nz, bool dbl);
// Twiddles, the shell table, and the wave vectors per shell into
// count[nshells] (once per box).
cudaError_t sq_init(const SqPlan &p, unsigned long long *count, cudaStream_t st);
// One sample: transform p.rho and add its shells to p.shell_sum.
cudaError_t launch_sq(const SqPlan &p, cudaStream_t st);

// D2Q9 boxes (d2q9.cu): one site per thread, rows [y0, y0 + nyc) as the slab unit.
namespace d2 {
template <class S>
struct BoxStep;

// V > 1: the vectorised kernel (4 sites per thread, 2 for FP64; nx % that == 0, whole warps).
template <class S>
cudaError_t launch_step(const BoxStep<S> &b, int layout, bool noise, bool force, int bx, int by, int V,
                        const uint32_t *step_ptr, uint32_t step, cudaStream_t st);
template <class S>
cudaError_t launch_gather(const S *buf, int64_t plane, int layout, int nx, int ny, int y0, int nyc, double rho0,
                          double *out, cudaStream_t st);
template <class S>
cudaError_t launch_gather_sites(const S *buf, int64_t plane, int layout, int nx, int ny, double rho0,
                                const int64_t *sites, int64_t nsites, double *out, cudaStream_t st);
template <class S>
cudaError_t launch_scatter(S *buf, int64_t plane, int layout, int nx, int ny, int y0, int nyc, double rho0,
                           const double *in, cudaStream_t st);
template <class S>
cudaError_t launch_init_equilibrium(S *buf, int64_t plane, int layout, int nx, int ny, int y0, int nyc, double rho0,
                                    const double *u, cudaStream_t st);
template <class S>
cudaError_t launch_stats_partial(const S *buf, int64_t plane, int layout, int nx, int ny, double rho0,
                                 double *partial, int nblocks, cudaStream_t st);
template <class S>
cudaError_t launch_y_profile(const S *buf, int64_t plane, int layout, int nx, int ny, double rho0, double *out,
                             cudaStream_t st);
template <class S>
cudaError_t launch_density(const S *buf, int64_t plane, int layout, int nx, int ny, typename Storage<S>::R *field,
                           cudaStream_t st);
cudaError_t launch_moments(const double *n, int64_t slab, int nx, int ny, int y0, double force_amp, double *rho,
                           double *j, double *Pi, cudaStream_t st);
}  // namespace d2

}  // namespace flb
