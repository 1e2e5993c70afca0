/*
 * flb.h -- C ABI of the GB300 fluctuating lattice Boltzmann library (D3Q19 and D2Q9).
 *
 * The library advances the fluctuating lattice Boltzmann equation of
 * Duenweg, Schiller and Ladd (arXiv:0707.1581) on periodic boxes, one GPU,
 * every step in hand-written sm_103a CUDA kernels:
 *
 *   n_i(r + c_i, t + 1) = n*_i(r, t)                          (Sec. I, Eq. LBE)
 *   m_k = sum_i e_ki n_i                                      (Table II)
 *   m*_k = m_k^eq + gamma_k (m_k - m_k^eq) + sigma_k r_k      (Sec. IV, Eq. updaterule)
 *   sigma_k = sqrt(mu rho0 w_k (1 - gamma_k^2)),  mu = 3 k_B T (Eq. FDT; Sec. VI)
 *   n*_i = a_i sum_k e_ki m*_k / w_k                          (Sec. III, Eqs. x_s, evectors_orthonormal)
 *
 * Conventions shared by every entry point:
 *  - Units are lattice units, b = h = 1 (Sec. VI).  c_s^2 = 1/3.
 *  - Velocity order i = 0..18: rest; +x, -x, +y, -y, +z, -z; (1,1,0), (-1,-1,0),
 *    (1,-1,0), (-1,1,0); (0,1,1), (0,-1,-1), (0,1,-1), (0,-1,1); (1,0,1),
 *    (-1,0,-1), (-1,0,1), (1,0,-1).  The paper fixes only the speeds (Sec. II).
 *  - Mode order k = 0..18 and basis e_ki: Table II of the paper.
 *  - Eigenvalues (Sec. IV): gamma_k = 1 for k <= 3, gamma_bulk for k = 4,
 *    gamma_shear for k = 5..9, gamma_ghost for k = 10..18; |gamma| <= 1.
 *  - Fields on the host are [component][z][y][x] with x fastest, N = nx*ny*nz.
 *    "Canonical populations" are the pre-collision n_i(r, t) at the context's
 *    current step t, as FP64, whatever the storage format on the device.
 *  - Gaussian numbers (the paper only asks for zero mean, unit variance):
 *    Philox-4x32-10 (Salmon et al., SC'11), key (lo32(seed), hi32(seed)),
 *    counter (site = x + nx (y + ny z), step t, replica, block b = 0..1);
 *    word p = 4b + j gives one Box-Muller pair from its two 16-bit halves,
 *    u1 = (lo16 + 1/2) 2^-16, u2 = (hi16 + 1/2) 2^-16:
 *    normals 2p, 2p+1 = R cos(2 pi u2), R sin(2 pi u2), R = sqrt(-2 ln u1).
 *    Mode k >= 4 uses normal number k - 4 of the sixteen.
 *  - Every call returns FLB_OK (0) or a negative FLB_E* code; the message is
 *    kept in the context (flb_last_error).  Host pointers are owned by the
 *    caller and never retained.  Device memory is owned by the context.
 *  - A context is not thread-safe.  Output calls synchronise its stream;
 *    flb_step only enqueues work (errors of the kernels surface at the next
 *    synchronising call).
 */
#ifndef FLB_H
#define FLB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FLB_OK 0
#define FLB_EINVAL (-1)       /* a parameter is out of range (message says which) */
#define FLB_ENOMEM (-2)       /* device or host allocation failed */
#define FLB_ECUDA (-3)        /* a CUDA runtime call or kernel failed */
#define FLB_ETIMEOUT (-4)     /* a bounded device wait ran out (reserved: no call of this version waits on the device with a bound) */
#define FLB_ENONFINITE (-5)   /* non-finite populations were found */
#define FLB_ERANGE (-6)       /* the step counter would pass 2^32 - 1 */
#define FLB_EIO (-7)          /* checkpoint file could not be read or written */

/* Storage format of the populations in device memory.  Every format stores
 * the deviation n_i - rho0 a_i from the rest equilibrium, rounded to nearest
 * even, so its resolution follows the size of the deviation.  Collisions run
 * in FP64 for FLB_STORE_F64 and in FP32 otherwise.  FLB_STORE_BF16SR holds
 * the bits of FLB_STORE_BF16DEV but rounds every post-collision value
 * stochastically, so that the rounding error has zero mean: the FP32 value's
 * bit pattern plus 16 random bits, low half cleared.  The bits are
 * Philox-4x32-10 blocks 2, 3, 4 of (site, step, replica) with the key of the
 * noise; population i takes word (i mod 8) / 2 of block 2 + i / 8, low half
 * for even i.  States set from the host are rounded to nearest.  The
 * allocation-free statistics call reads this format as FLB_STORE_BF16DEV. */
typedef enum {
    FLB_STORE_F64 = 0,
    FLB_STORE_F32 = 1,
    FLB_STORE_F16DEV = 2,
    FLB_STORE_BF16DEV = 3,
    FLB_STORE_BF16SR = 4       /* bfloat16 deviation written with stochastic rounding */
} flb_store_t;

/* Streaming pattern: AB = two buffers, each step pulls from one and writes the
 * other; AA = one buffer updated in place, even steps touch only their own
 * site, odd steps read and write the neighbour slots. */
typedef enum { FLB_PATTERN_AB = 0, FLB_PATTERN_AA = 1 } flb_pattern_t;

/* Lattice.  D3Q19 (Table II) is the default.  D2Q9 (Table I) boxes are
 * nx x ny with nz = 1: velocity order rest; +x, -x, +y, -y; (1,1), (-1,-1),
 * (1,-1), (-1,1); weights 4/9, 1/9, 1/36; modes k = 0..8 of Table I with
 * gamma_bulk for k = 3, gamma_shear for k = 4, 5, gamma_ghost for k = 6..8;
 * mode k >= 3 uses normal k - 3 of Philox block 0 (one call per site); the
 * body force is F_x(y) = force_amp sin(2 pi y / ny).  Every per-box call
 * then works with 9 populations, 2 velocity components and 3 stress
 * components (xx, yy, xy); the batch and graph machinery are shared; the
 * kernel takes 4 sites per thread (2 for FP64), or 1 when nx is not a
 * multiple of that.  Host arrays of a
 * D2Q9 box: populations n[9][ny][nx], velocities u[2][ny][nx], j[2][N],
 * Pi[3][N] (xx, yy, xy); flb_box_z_profile averages rows along y (rho[ny],
 * j[3][ny] with a zero third row); flb_mode_stats_t fills modes 0..8 and
 * velocity components 0..1. */
typedef enum { FLB_LATTICE_D3Q19 = 0, FLB_LATTICE_D2Q9 = 1 } flb_lattice_t;

typedef struct {
    int nx, ny, nz;            /* box edge lengths, each >= 1, nx*ny*nz < 2^31 */
    double rho0;               /* mean density, > 0 */
    double kT;                 /* k_B T >= 0; mu = 3 kT (Sec. VI); 0 = deterministic LB */
    double gamma_shear;        /* modes 5..9, in [-1, 1] */
    double gamma_bulk;         /* mode 4, in [-1, 1] */
    double gamma_ghost;        /* modes 10..18, in [-1, 1] */
    uint64_t seed;             /* Philox key */
    uint32_t replica;          /* Philox counter word 2 (ensemble member id) */
    int store;                 /* flb_store_t */
    int pattern;               /* flb_pattern_t */
    int noise_ghosts;          /* 1: thermalize the kinetic modes too (Sec. IV, the
                                  detailed-balance rule); 0: stress modes only */
    int noise_rho_local;       /* 0: variance mu rho0 w_k; 1: mu rho(r) w_k (Sec. III) */
    double force_amp;          /* body force F_x(z) = force_amp sin(2 pi z / nz) per step */
    int sites_per_thread;      /* 0 = automatic (4, FP64 2; halved while the boxes' sites
                                  over it stay below 100,000 threads); else 1, 2 or 4
                                  (x-consecutive sites) */
    int block_x, block_y;      /* 0 = automatic; else the CUDA block shape */
    int graph_steps;           /* steps per captured CUDA graph; 0 = plain launches */
    int lattice;               /* flb_lattice_t; every box of a context has the same lattice */
    int stats_every;           /* k > 0: flb_step takes a statistics sample (flb_stats_sample) after
                                  every step that brings the step counter to a multiple of k, between
                                  graph replays; 0 = samples only on request */
    void *stream;              /* cudaStream_t to run on; NULL = a stream owned by the context */
} flb_config;

/* Statistics accumulated on the device (FP64) by flb_stats_sample. */
typedef struct {
    uint64_t nsamples;         /* number of sampled steps */
    uint64_t nsites;           /* sites per sample */
    double mode_m2[19];        /* mean over samples and sites of (sum_i e_ki (n_i - rho0 a_i))^2 */
    double mode_ratio[19];     /* mode_m2[k] / (mu rho0 w_k); 0 when kT = 0 (Sec. III, Eq. modeprob) */
    double u2[3];              /* mean of (j_alpha / rho)^2 */
    double u2_ratio[3];        /* u2 rho0 / kT (Sec. V: k_B T / rho0 per component); 0 when kT = 0 */
    double mass_first, mass_last;            /* total mass at the first / last sample */
    double momentum_first[3], momentum_last[3];
    uint64_t nonfinite;        /* non-finite populations seen over all samples */
} flb_mode_stats_t;

typedef struct flb_ctx flb_ctx;

/* Fills *cfg with defaults: 32^3, rho0 = 1, kT = 0, all gamma = 0, seed 0,
 * FP32 storage, AB pattern, noise_ghosts = 1, automatic launch shape. */
void flb_config_init(flb_config *cfg);

/* Creates one box at rest equilibrium n_i = rho0 a_i, step 0.  The nine
 * scalars of the method: box, rho0, k_B T, gamma_shear, gamma_bulk,
 * gamma_ghost (Sec. IV eigenvalue assignment) and the Philox seed.  FP32
 * storage, AB pattern.  Errors: FLB_EINVAL (|gamma| > 1 -- the linear stability
 * limit of Sec. IV --, kT < 0, rho0 <= 0, an edge < 1, nx*ny*nz >= 2^31),
 * FLB_ENOMEM, FLB_ECUDA.  *out is NULL on error. */
int flb_create(int nx, int ny, int nz, double rho0, double kT, double gamma_shear,
               double gamma_bulk, double gamma_ghost, uint64_t seed, flb_ctx **out);

/* As flb_create with every option of flb_config. */
int flb_create_ex(const flb_config *cfg, flb_ctx **out);

/* A batch of nboxes independent boxes (ensemble replicas and boxes of
 * different sizes and parameters) advanced together by one kernel launch per
 * step.  All boxes share store, pattern, launch shape and graph_steps (taken
 * from cfgs[0]); each keeps its own size, rho0, kT, gammas, seed, replica and
 * force.  Per-box calls take the box index 0..nboxes-1. */
int flb_create_batch(const flb_config *cfgs, int nboxes, flb_ctx **out);

/* Frees every device and host resource of the context (NULL is accepted). */
void flb_destroy(flb_ctx *ctx);

/* Number of boxes of the context (1 unless made by flb_create_batch). */
int flb_num_boxes(const flb_ctx *ctx);

/* Enqueues nsteps time steps (Eq. LBE with the collision of Sec. IV) of every
 * box.  Asynchronous.  FLB_ERANGE if the step counter would pass 2^32 - 1
 * (it is a Philox counter word); FLB_EINVAL if nsteps < 0. */
int flb_step(flb_ctx *ctx, int64_t nsteps);

/* Host-resident stepping of box `box`: `host` holds its raw state (the bytes
 * of flb_box_state_download, flb_box_state_bytes long; pinned memory for full
 * speed).  The call uploads it, advances the context by nsteps (Eq. LBE with
 * the collision of Sec. IV) and writes the new state back to `host`.  The
 * first step runs in z-chunks as the planes arrive, on a copy stream beside the
 * compute stream, and the downloads start chunk by chunk as the step finishes
 * them, so the two copy directions and the kernel overlap.  Other boxes of a
 * batch do not advance their state, but the step counter is shared.  D3Q19 only
 * (FLB_EINVAL for D2Q9).  Synchronises. */
int flb_box_step_host(flb_ctx *ctx, int box, void *host, int64_t nsteps);

/* Page-locked host memory for host-resident state (flb_box_step_host) or any
 * other staging: nbytes (> 0) of zeroed memory, mapped with transparent huge
 * pages where the system offers them (aligned to the huge-page size when
 * nbytes spans one), faulted in and registered with the CUDA driver, so the
 * copy engines stream it at the host link's rate from the first transfer on.
 * *out receives the buffer; the caller owns it and releases it with
 * flb_host_free (which takes exactly a pointer this call returned; NULL is
 * accepted).  FLB_EINVAL (NULL out, nbytes = 0, or a pointer not from
 * flb_host_alloc), FLB_ENOMEM (the mapping failed), FLB_ECUDA (the driver did
 * not register it; no GPU).  Thread-safe. */
int flb_host_alloc(size_t nbytes, void **out);
int flb_host_free(void *ptr);

/* Device-memory hook.  Every device buffer a context owns (populations,
 * statistics accumulators, staging, structure-factor workspace, the copies the
 * autotuner and the pattern conversion make) is taken from alloc(bytes,
 * stream, user) and returned through free(ptr, stream, user), stream being the
 * context's cudaStream_t: a caching allocator can order reuse on it (the
 * Python binding installs torch's).  alloc returns NULL on failure (the call
 * then fails with FLB_ENOMEM) and memory aligned to at least 256 bytes.  The
 * hook is process-wide and is captured by each context at creation, so it must
 * stay valid until those contexts are destroyed; flb_destroy synchronises the
 * stream before freeing.  Both NULL restores cudaMalloc / cudaFree; one NULL
 * is FLB_EINVAL.  The context-free calls (flb_philox4x32_10, flb_normals)
 * always use cudaMalloc.  Thread-safe. */
/* Bounds checks (a debugging build: the library compiled with
 * FLB_BOUNDS_CHECK, `build(check=True)`, libflb_check.so).  There every global
 * access of the stream-collide kernels checks its span against the buffer it
 * addresses; a span outside is counted and the access is not made.
 * flb_bounds_violations gives the context's count; flb_bounds_selftest makes
 * the guard check two spans just outside box 0's buffer (and one inside),
 * adding exactly 2 to the count without touching memory.  In the ordinary
 * build both return FLB_EINVAL (*count = 0). */
int flb_bounds_violations(flb_ctx *ctx, uint64_t *count);
int flb_bounds_selftest(flb_ctx *ctx);

typedef void *(*flb_dev_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*flb_dev_free_fn)(void *ptr, void *stream, void *user);
int flb_set_device_allocator(flb_dev_alloc_fn alloc, flb_dev_free_fn free_fn, void *user);

/* Waits for all work enqueued on the context's stream. */
int flb_sync(flb_ctx *ctx);

/* Current step t of the context (all boxes share it). */
int flb_get_step(const flb_ctx *ctx, uint64_t *step);

/* Canonical pre-collision populations of box `box` at the current step,
 * written to the host array n[19][nz][ny][nx] (FP64).  Synchronises. */
int flb_box_get_populations(flb_ctx *ctx, int box, double *n);
int flb_get_populations(flb_ctx *ctx, double *n);                 /* box 0 */

/* Canonical pre-collision populations of box `box` at nsites chosen sites:
 * sites[s] is the site index x + nx (y + ny z) (each in [0, N)), and
 * out[s][19] receives n_i at that site (host arrays, FP64).  For checking large
 * boxes without copying every population.  Synchronises. */
int flb_box_get_sites(flb_ctx *ctx, int box, const int64_t *sites, int64_t nsites, double *out);

/* Replaces the state of box `box` by the canonical pre-collision populations
 * n[19][nz][ny][nx] (host, FP64), interpreted at the current step.  Values are
 * rounded to the storage format.  Synchronises. */
int flb_box_set_populations(flb_ctx *ctx, int box, const double *n);
int flb_set_populations(flb_ctx *ctx, const double *n);           /* box 0 */

/* Sets box `box` to n_i = n_i^eq(rho0, u(r)) of Eq. derived_equil_distrib (with
 * sigma_2 = c_s^2), from the host field u[3][nz][ny][nx]; u = NULL means rest. */
int flb_box_init_velocity(flb_ctx *ctx, int box, const double *u);
int flb_init_velocity(flb_ctx *ctx, const double *u);             /* box 0 */

/* Hydrodynamic moments of the canonical state (Sec. I, Eqs. defrho, defj,
 * defstress): rho[N] = sum_i n_i, j[3][N] = sum_i n_i c_i (plus F/2 when a
 * body force is set: the half-step momentum), Pi[6][N] = sum_i n_i c_ia c_ib in
 * the order xx, yy, zz, xy, yz, zx.  Any pointer may be NULL.  Host arrays.
 * Synchronises. */
int flb_box_moments(flb_ctx *ctx, int box, double *rho, double *j, double *Pi);
int flb_moments(flb_ctx *ctx, double *rho, double *j, double *Pi); /* box 0 */

/* Plane averages along z of the canonical state: rho[z] = mean over x, y of
 * sum_i n_i, and j[3][nz] = mean over x, y of sum_i n_i c_i (plus F/2 with a
 * body force) (Sec. I, Eqs. defrho, defj), FP64 sums of the stored values.
 * For flows that vary only along z (shear waves, Kolmogorov flow).  Host
 * arrays; either may be NULL.  Synchronises. */
int flb_box_z_profile(flb_ctx *ctx, int box, double *rho, double *j);

/* Statistics.  flb_stats_sample enqueues one sample of every box at the
 * current step: per-mode second moments of n - rho0 a_i, velocity variance,
 * total mass and momentum and the non-finite count, accumulated in FP64 on the
 * device; and, for boxes whose structure factor is enabled, |FFT(rho)|^2.
 * flb_box_mode_stats reads and normalises them (synchronises). */
int flb_stats_reset(flb_ctx *ctx);
int flb_stats_sample(flb_ctx *ctx);
int flb_box_mode_stats(flb_ctx *ctx, int box, flb_mode_stats_t *out);
int flb_mode_stats(flb_ctx *ctx, flb_mode_stats_t *out);          /* box 0 */

/* Health check of box `box`: counts the stored populations that are not
 * finite (infinite or NaN, from the raw bits of the storage format) and writes
 * the count to *nonfinite (may be NULL).  FLB_OK if there are none,
 * FLB_ENONFINITE otherwise.  Synchronises. */
int flb_box_check_finite(flb_ctx *ctx, int box, uint64_t *nonfinite);

/* Static structure factor S(q) = <|sum_r (rho(r) - <rho>) e^{-i q.r}|^2> / N
 * (Sec. V: flat at mu rho0 = rho0 k_B T / c_s^2 for the isothermal ideal gas,
 * Eq. mpeos).  flb_box_enable_structure_factor allocates the FFT workspace of a
 * box (complex FP64, 16 N bytes); later samples accumulate S(q).
 * flb_box_structure_factor writes the shell averages: shell s holds the q != 0
 * with s <= |q| / dq < s + 1, dq = 2 pi / max(nx, ny, nz); S[s] is the mean and
 * count[s] the number of wave vectors (either pointer may be NULL), for
 * s = 0..nshells-1.  Divide by mu rho0 for the ratio. */
int flb_box_enable_structure_factor(flb_ctx *ctx, int box);
int flb_box_structure_factor(flb_ctx *ctx, int box, double *S, int64_t *count, int nshells);
/* Box 0, shell means only. */
int flb_enable_structure_factor(flb_ctx *ctx);
int flb_structure_factor(flb_ctx *ctx, double *S, int nshells);

/* Raw device state of box `box` (the deviations n_i - rho0 a_i in the storage
 * format and layout the kernels use, valid at the current step): size in bytes, and
 * copies to / from a host buffer of that size (pinned memory is fastest).
 * Upload keeps the current step.  Synchronises. */
int flb_box_state_bytes(const flb_ctx *ctx, int box, size_t *bytes);
int flb_box_state_download(flb_ctx *ctx, int box, void *host);
int flb_box_state_upload(flb_ctx *ctx, int box, const void *host);

/* Checkpoint of every box (parameters, step counter, raw state) to a file and
 * back.  Philox is counter-based, so a run continued from a checkpoint is
 * bitwise identical to an uninterrupted one.  flb_load requires a context of
 * the same format, pattern and number of boxes, and boxes of the same size,
 * lattice, rho0, kT, eigenvalues, noise variants, force, seed and replica id
 * (launch shape, graphs, sampling and stream may differ).  It reads and checks
 * the whole file before it uploads anything, so on any error the context is
 * left unchanged.  FLB_EIO on file errors, a mismatch, or a corrupt header
 * (buffer index other than 0 or 1 -- 0 for AA --, step counter >= 2^32). */
int flb_save(flb_ctx *ctx, const char *path);
int flb_load(flb_ctx *ctx, const char *path);

/* Launch configuration in use, and a measured choice: flb_autotune times every
 * candidate (sites per thread x block shape) for `trials` steps each on the
 * context's own state (which it restores afterwards) and keeps the fastest. */
int flb_get_launch(const flb_ctx *ctx, int *sites_per_thread, int *block_x, int *block_y);
/* Sets the launch shape (for instance one that flb_autotune chose earlier for
 * the same boxes); FLB_EINVAL if it does not fit the boxes (sites per thread
 * must divide every nx and blocks of more than one site per thread must be
 * whole warps). */
int flb_set_launch(flb_ctx *ctx, int sites_per_thread, int block_x, int block_y);
int flb_autotune(flb_ctx *ctx, int trials);

/* flb_autotune_ex with flags = FLB_TUNE_PATTERN also times the other streaming
 * pattern (converting the state there and back with flb_set_pattern, skipped
 * when the two-buffer pattern does not fit in memory) and keeps the faster
 * pattern with its fastest launch shape.  The state and the step counter are
 * unchanged. */
#define FLB_TUNE_PATTERN 1
int flb_autotune_ex(flb_ctx *ctx, int trials, int flags);

/* Streaming pattern of the context.  flb_set_pattern converts every box in
 * place of the canonical state: each stored element moves, bit for bit, from
 * its slot in the current layout to its slot in the other (AB allocates the
 * second buffer of every box, FLB_ENOMEM if it does not fit; AA frees it).
 * Graphs are recaptured on the next flb_step.  Synchronises. */
int flb_get_pattern(const flb_ctx *ctx, int *pattern);
int flb_set_pattern(flb_ctx *ctx, int pattern);

/* The device generator on its own (the functions the kernels call), for
 * checking it directly.  flb_philox4x32_10: Philox-4x32-10 (Salmon et al.,
 * SC'11) of n counters ctr[n][4] under keys key[n][2], words to out[n][4].
 * flb_normals: the sixteen normals of sites site0 .. site0 + nsites - 1 at
 * (step, replica) under `seed`, as the noise of the collision draws them
 * (Philox blocks 0, 1; word p gives normals 2p, 2p + 1 by Box-Muller from its
 * 16-bit halves), out[nsites][16]; fp64 = 1 the FP64 kernels' normals, 0 the
 * FP32 kernels' (hardware log2/sin/cos).  Host arrays; the GPU computes.
 * FLB_EINVAL on bad sizes or pointers, FLB_ENOMEM, FLB_ECUDA. */
int flb_philox4x32_10(const uint32_t *ctr, const uint32_t *key, int64_t n, uint32_t *out);
int flb_normals(uint64_t seed, uint32_t step, uint32_t replica, uint32_t site0, int64_t nsites, int fp64,
                double *out);

/* Physical units (Sec. VI).  With lattice spacing b and time step h, the
 * nondimensional viscosities are eta_hat = eta h / (rho b^2 c_hat_s^2) and
 * zeta_hat = zeta h / (rho b^2 c_hat_s^2) (c_hat_s^2 = 1/3), and the eigenvalues
 * that realise them are gamma_shear = (2 eta_hat - 1) / (2 eta_hat + 1) and
 * gamma_bulk = (3 zeta_hat - 1) / (3 zeta_hat + 1).  FLB_EINVAL if a input is
 * not positive and finite.  Host only; no GPU needed. */
int flb_gammas_from_viscosities(double eta, double zeta, double rho, double b, double h, double *gamma_shear,
                                double *gamma_bulk);

/* Lattice-unit k_B T for the library from physical k_B T, mass density rho,
 * lattice spacing b and time step h: the fluctuation parameter of Sec. VI,
 * mu = k_B T h^2 / (c_hat_s^2 b^5) per unit density, is 3 kT_lattice / rho0, so
 * kT_lattice = rho0 k_B T h^2 / (rho b^5).  rho0 is the lattice density the
 * context will use (usually 1).  FLB_EINVAL on a non-positive or non-finite
 * input.  Host only. */
int flb_lattice_kT(double kT, double rho, double b, double h, double rho0, double *kT_lattice);

/* Both conversions for a lattice of dimension d (2 for D2Q9, 3 for D3Q19):
 * gamma_shear = (2 eta_hat - 1) / (2 eta_hat + 1) (Eq. shearviscosity has no
 * d), gamma_bulk = (d zeta_hat - 1) / (d zeta_hat + 1) (Eq. bulkviscosity,
 * zeta = h rho c_s^2 / d (1 + gamma_bulk) / (1 - gamma_bulk)), and
 * kT_lattice = rho0 k_B T h^2 / (rho b^(d+2)) (rho is a mass per b^d).
 * kT = 0 gives kT_lattice = 0.  FLB_EINVAL if d is not 2 or 3, kT < 0, or
 * another input is not positive and finite.  Host only. */
int flb_lattice_params(int d, double eta, double zeta, double kT, double rho, double b, double h, double rho0,
                       double *gamma_shear, double *gamma_bulk, double *kT_lattice);

/* Largest box, in sites, that flb_mode_sums_noalloc accepts. */
#define FLB_NOALLOC_MAX_SITES 16777216

/* Mode and velocity sums of caller-owned device populations, with no device
 * allocation.  The paper has no counterpart; this is a service for callers that
 * must not allocate device memory: cudaMalloc synchronises the whole device and
 * can fail under memory pressure, and some hosts (plugins inside another
 * application's fixed memory budget, loops that must never stall) give a
 * library only the buffers it reads and writes.
 *   populations  device array of the deviations n_i - rho0 a_i of canonical
 *                populations (the library's storage convention, e.g. a raw
 *                state of an AA context at an even step), planes [19][nz][ny][nx]
 *                of `plane` elements each (plane >= nx*ny*nz), in format `store`
 *                (FLB_STORE_BF16SR is accepted and read as FLB_STORE_BF16DEV:
 *                the stored bits are the same, only their rounding differed)
 *   sums         device array of 27 doubles, overwritten with, over all sites:
 *                [0..18] sum of m_k^2, m_k = sum_i e_ki (n_i - rho0 a_i) with the
 *                library's 19 mode vectors (those of flb_mode_stats),
 *                [19..21] sum of (j_alpha / rho)^2, [22] sum of rho,
 *                [23..25] sum of j, [26] number of sites with non-finite values
 *   stream       cudaStream_t (NULL = the default stream); the call only
 *                enqueues work and returns.
 * Scratch is one static device array of FLB_NOALLOC_MAX_SITES / 8192 rows of
 * partial sums (432 KiB) that every GPU which loads the library keeps until the
 * process exits.  It is shared by every call and keeps the last call's
 * contents; each call overwrites the rows it uses.  Calls that overlap on the
 * GPU (other streams, or other host threads) race on it and must be ordered.
 * The first call on a device resolves the array's device address; make that
 * first call before any stream capture.  The address is kept per device and
 * resolved again when the device's context changes (after cudaDeviceReset the
 * next call resolves it in the new context).  Returns FLB_ERANGE if nx*ny*nz exceeds
 * FLB_NOALLOC_MAX_SITES, FLB_EINVAL for NULL pointers, an unknown format,
 * sizes < 1, rho0 <= 0 or plane < nx*ny*nz, FLB_ECUDA on a CUDA error. */
int flb_mode_sums_noalloc(const void *populations, int store, int64_t plane, int nx, int ny, int nz, double rho0,
                          double *sums, void *stream);

/* Message of the last failed call on this context ("" if none). */
const char *flb_last_error(const flb_ctx *ctx);

/* Message of the last failed flb_create* (which has no context to hold it). */
const char *flb_create_error(void);

/* Library and device description: writes at most len bytes of a NUL-terminated
 * string (library version, compiled architecture). */
int flb_version(char *buf, int len);

#ifdef __cplusplus
}
#endif

#endif /* FLB_H */
