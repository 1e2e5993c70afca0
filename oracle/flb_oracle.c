/*
 * flb_oracle.c -- plain FP64 CPU oracle of the fluctuating lattice Boltzmann
 * update on D3Q19 (Duenweg, Schiller, Ladd, "Statistical mechanics of the
 * fluctuating lattice Boltzmann equation", arXiv:0707.1581).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA path is checked against.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * table or constant with the CUDA library: every table below is written out
 * here from the paper.
 *
 * What it computes, per time step t and per lattice site r (Sec. I, Eq. LBE):
 *   1. modes        m_k = sum_i e_ki n_i                      (Table II, Sec. III)
 *   2. equilibrium  n_i^eq(rho, u), u = j / rho               (Eq. derived_equil_distrib)
 *                   m_k^eq = sum_i e_ki n_i^eq
 *   3. collision    m*_k = m_k^eq + gamma_k (m_k - m_k^eq) + sigma_k r_k, k >= 4
 *                   m*_k = m_k for the conserved modes k <= 3  (Eqs. updaterule, FDT)
 *                   sigma_k = sqrt(mu rho0 w_k (1 - gamma_k^2)), mu = 3 k_B T
 *   4. back         n*_i = a_i sum_k e_ki m*_k / w_k           (Eqs. x_s, evectors_orthonormal)
 *   5. streaming    n_i(r + c_i, t + 1) = n*_i(r, t)           (Eq. LBE, push form)
 * The transforms are the literal 19 x 19 loops; no factorisation, no fusion.
 *
 * Readings taken where the paper is silent or leaves a choice open:
 *  - velocity order: rest; +x,-x,+y,-y,+z,-z; then the (x,y), (y,z), (z,x)
 *    diagonals, each as (+,+),(-,-),(+,-),(-,+) in that cyclic index order;
 *  - the variance of a population uses the mean density rho0 (the low-velocity
 *    limit of Sec. III taken at the mean density); a switch selects the local rho;
 *  - mu = 3 k_B T in lattice units b = h = 1 (Sec. VI, with c_s^2 = 1/3);
 *  - the Gaussian numbers r_k come from Philox-4x32-10 (Salmon et al., SC'11)
 *    keyed by (seed) with counter (site, step, replica, block 0..1), two
 *    16-bit uniforms u = (h + 1/2) 2^-16 per word and the Box-Muller
 *    transform;
 *  - body force: second-order moment-space forcing (the paper has none);
 *  - reduced-precision storage is emulated by rounding n - rho0 a_i to the
 *    storage format after each step (the paper has no storage format);
 *  - stochastic rounding to bfloat16 (store 4): the deviation is first rounded
 *    to binary32 (the precision the GPU collides in), then r, 16 bits from
 *    Philox blocks 2..4 of (site, step, replica), is added to its bit pattern
 *    and the low 16 bits are dropped; population i takes word (i mod 8) / 2
 *    of block 2 + i / 8, low half for even i, high half for odd i.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19

/* ------------------------------------------------------------------------ */
/* D3Q19 velocity set and weights (Sec. II, end: a^0 = 1/3, a^1 = 1/18,      */
/* a^sqrt2 = 1/36, c_s^2 = 1/3).                                              */
/* ------------------------------------------------------------------------ */
static const int VEL[Q][3] = {
    {0, 0, 0},
    {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
    {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1},
    {1, 0, 1},  {-1, 0, -1}, {-1, 0, 1}, {1, 0, -1},
};

static double weight_of(int i)
{
    int c2 = VEL[i][0] * VEL[i][0] + VEL[i][1] * VEL[i][1] + VEL[i][2] * VEL[i][2];
    if (c2 == 0) return 1.0 / 3.0;
    if (c2 == 1) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

static const double CS2 = 1.0 / 3.0;

/* Table II: the polynomial e_k(c) of row k, evaluated at velocity c. */
static double table2_poly(int k, const int c[3])
{
    double x = c[0], y = c[1], z = c[2];
    double c2 = x * x + y * y + z * z;
    switch (k) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return z;
    case 4: return c2 - 1.0;
    case 5: return 3.0 * x * x - c2;
    case 6: return y * y - z * z;
    case 7: return x * y;
    case 8: return y * z;
    case 9: return z * x;
    case 10: return (3.0 * c2 - 5.0) * x;
    case 11: return (3.0 * c2 - 5.0) * y;
    case 12: return (3.0 * c2 - 5.0) * z;
    case 13: return (y * y - z * z) * x;
    case 14: return (z * z - x * x) * y;
    case 15: return (x * x - y * y) * z;
    case 16: return 3.0 * c2 * c2 - 6.0 * c2 + 1.0;
    case 17: return (2.0 * c2 - 3.0) * (3.0 * x * x - c2);
    case 18: return (2.0 * c2 - 3.0) * (y * y - z * z);
    }
    return 0.0;
}

typedef struct {
    double a[Q];      /* weights a^{c_i} */
    double e[Q][Q];   /* e[k][i] = e_ki (unscaled basis, Table II) */
    double w[Q];      /* w_k = sum_i a_i e_ki^2 (Sec. III) */
} lattice_t;

static void build_lattice(lattice_t *L)
{
    for (int i = 0; i < Q; ++i) L->a[i] = weight_of(i);
    for (int k = 0; k < Q; ++k) {
        double wk = 0.0;
        for (int i = 0; i < Q; ++i) {
            L->e[k][i] = table2_poly(k, VEL[i]);
            wk += L->a[i] * L->e[k][i] * L->e[k][i];
        }
        L->w[k] = wk;
    }
}

/* Export of the tables, so the tests can pin them against the paper. */
void ora_lattice(int *c /*19*3*/, double *a /*19*/, double *e /*19*19, [k][i]*/, double *w /*19*/)
{
    lattice_t L;
    build_lattice(&L);
    for (int i = 0; i < Q; ++i) {
        for (int d = 0; d < 3; ++d) c[3 * i + d] = VEL[i][d];
        a[i] = L.a[i];
    }
    for (int k = 0; k < Q; ++k) {
        w[k] = L.w[k];
        for (int i = 0; i < Q; ++i) e[k * Q + i] = L.e[k][i];
    }
}

/* ------------------------------------------------------------------------ */
/* Philox-4x32-10, from the published description (Salmon, Moraes, Dror,   */
/* Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds  */
/* of two 32x32->64 bit multiplications with a Weyl-sequence key schedule.  */
/* ------------------------------------------------------------------------ */
static const uint32_t PHILOX_M0 = 0xD2511F53u;
static const uint32_t PHILOX_M1 = 0xCD9E8D57u;
static const uint32_t PHILOX_W0 = 0x9E3779B9u;   /* golden ratio */
static const uint32_t PHILOX_W1 = 0xBB67AE85u;   /* sqrt(3) - 1 */

void ora_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        uint32_t n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* 16-bit value -> uniform in (0,1): u = (h + 1/2) * 2^-16.  The 2^16 values
 * (2h+1) 2^-17 are exact in binary32 and binary64. */
double ora_uniform16(uint32_t h)
{
    return ((double)(h & 0xFFFFu) + 0.5) * (1.0 / 65536.0);
}

/* Sixteen standard normals for one (site, step, replica): Philox blocks
 * b = 0, 1 with counter (site, step, replica, b) and key (lo32(seed),
 * hi32(seed)) give eight words; word p = 4b + j feeds one Box-Muller pair
 * with u1 from its low and u2 from its high 16 bits:
 *   R = sqrt(-2 ln u1),  g[2p] = R cos(2 pi u2),  g[2p+1] = R sin(2 pi u2). */
void ora_gaussians(uint64_t seed, uint32_t site, uint32_t step, uint32_t replica, double g[16])
{
    const double two_pi = 6.283185307179586476925286766559;
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint32_t b = 0; b < 2; ++b) {
        uint32_t ctr[4] = {site, step, replica, b};
        uint32_t w[4];
        ora_philox4x32_10(ctr, key, w);
        for (int j = 0; j < 4; ++j) {
            const int p = 4 * (int)b + j;
            double u1 = ora_uniform16(w[j] & 0xFFFFu);
            double u2 = ora_uniform16(w[j] >> 16);
            double R = sqrt(-2.0 * log(u1));
            g[2 * p] = R * cos(two_pi * u2);
            g[2 * p + 1] = R * sin(two_pi * u2);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Collision.                                                               */
/* ------------------------------------------------------------------------ */
typedef struct {
    int nx, ny, nz;
    double rho0;
    double kT;
    double gamma[Q];       /* per-mode eigenvalue; modes 0..3 are forced to 1 */
    uint64_t seed;
    uint32_t replica;
    int noise_ghosts;      /* 1: thermalize the kinetic modes too (Sec. IV); 0: stress modes only */
    int noise_rho_local;   /* 0: variance mu rho0 w_k; 1: mu rho(r) w_k */
    double force_amp;      /* F_x(z) = force_amp sin(2 pi z / nz), F_y = F_z = 0 */
    int store;             /* 0 exact FP64; 2 FP16 deviation; 3 BF16 deviation; 4 BF16 stochastic */
} ora_params;

/* Eq. derived_equil_distrib with sigma_2 = c_s^2 = 1/3. */
static void equilibrium(const double rho, const double u[3], const double a[Q], double neq[Q])
{
    double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; ++i) {
        double cu = VEL[i][0] * u[0] + VEL[i][1] * u[1] + VEL[i][2] * u[2];
        neq[i] = rho * a[i] * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - u2 / (2.0 * CS2));
    }
}

void ora_equilibrium_field(int64_t nsites, const double *rho, const double *u /*[3][N]*/, double *n /*[19][N]*/)
{
    lattice_t L;
    build_lattice(&L);
    for (int64_t s = 0; s < nsites; ++s) {
        double uu[3] = {u[s], u[nsites + s], u[2 * nsites + s]};
        double neq[Q];
        equilibrium(rho[s], uu, L.a, neq);
        for (int i = 0; i < Q; ++i) n[(int64_t)i * nsites + s] = neq[i];
    }
}

/* One collision at one site.  g[] holds the 16 normals of this (site, step);
 * mode k >= 4 uses g[k - 4].  F is the body force density per step. */
static void collide(const ora_params *p, const lattice_t *L, const double n[Q],
                    const double g[16], const double F[3], double nstar[Q])
{
    double m[Q], meq[Q], ms[Q], neq[Q];
    for (int k = 0; k < Q; ++k) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) s += L->e[k][i] * n[i];
        m[k] = s;
    }
    double rho = m[0];
    double j[3] = {m[1], m[2], m[3]};
    /* with a force the equilibrium velocity is taken at the half step */
    double u[3] = {(j[0] + 0.5 * F[0]) / rho, (j[1] + 0.5 * F[1]) / rho, (j[2] + 0.5 * F[2]) / rho};
    equilibrium(rho, u, L->a, neq);
    for (int k = 0; k < Q; ++k) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) s += L->e[k][i] * neq[i];
        meq[k] = s;
    }
    /* source of the second moment, S = u F + F u, in the stress modes 4..9:
     * S_k = sum_i e_ki a_i (c_i.u)(c_i.F) / c_s^4 projected the same way as n_eq */
    double Smode[Q];
    for (int k = 0; k < Q; ++k) Smode[k] = 0.0;
    if (F[0] != 0.0 || F[1] != 0.0 || F[2] != 0.0) {
        double S[3][3];
        for (int al = 0; al < 3; ++al)
            for (int be = 0; be < 3; ++be) S[al][be] = u[al] * F[be] + F[al] * u[be];
        /* the stress modes of Table II are linear in sum_i n_i c_ia c_ib and
         * sum_i n_i; a population set with second moment S and no mass,
         * momentum or ghost content is n_i = a_i (c_ia c_ib - c_s^2 d_ab) S_ab / (2 c_s^4) */
        double nS[Q];
        for (int i = 0; i < Q; ++i) {
            double acc = 0.0;
            for (int al = 0; al < 3; ++al)
                for (int be = 0; be < 3; ++be)
                    acc += (VEL[i][al] * VEL[i][be] - (al == be ? CS2 : 0.0)) * S[al][be];
            nS[i] = L->a[i] * acc / (2.0 * CS2 * CS2);
        }
        for (int k = 0; k < Q; ++k) {
            double s = 0.0;
            for (int i = 0; i < Q; ++i) s += L->e[k][i] * nS[i];
            Smode[k] = s;
        }
    }
    double mu = 3.0 * p->kT;
    double rho_var = p->noise_rho_local ? rho : p->rho0;
    for (int k = 0; k < Q; ++k) {
        if (k <= 3) {
            ms[k] = m[k];
            continue;
        }
        double gk = p->gamma[k];
        double v = meq[k] + gk * (m[k] - meq[k]) + 0.5 * (1.0 + gk) * Smode[k];
        int thermal = (k <= 9) || p->noise_ghosts;
        if (p->kT > 0.0 && thermal) {
            double sigma = sqrt(mu * rho_var * L->w[k] * (1.0 - gk * gk));
            v += sigma * g[k - 4];
        }
        ms[k] = v;
    }
    ms[1] += F[0];
    ms[2] += F[1];
    ms[3] += F[2];
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int k = 0; k < Q; ++k) s += L->e[k][i] * ms[k] / L->w[k];
        nstar[i] = L->a[i] * s;
    }
}

static void fill_gamma(const ora_params *p, double gam[Q])
{
    for (int k = 0; k < Q; ++k) gam[k] = (k <= 3) ? 1.0 : p->gamma[k];
}

/* Single-site collision, exported for the single-site tests.  If g is NULL
 * the normals are drawn for (site, step) of the parameter set. */
void ora_collide_site(const ora_params *p_in, const double n[Q], uint32_t site, uint32_t step,
                      const double F[3], const double *g_in, double nstar[Q])
{
    ora_params p = *p_in;
    fill_gamma(p_in, p.gamma);
    lattice_t L;
    build_lattice(&L);
    double g[16];
    if (g_in) memcpy(g, g_in, sizeof g);
    else ora_gaussians(p.seed, site, step, p.replica, g);
    double Fz[3] = {0.0, 0.0, 0.0};
    collide(&p, &L, n, g, F ? F : Fz, nstar);
}

/* ------------------------------------------------------------------------ */
/* Reduced-precision storage emulation: round to nearest, ties to even,     */
/* to a binary format with `p` significand bits and minimum normal          */
/* exponent `emin` (IEEE 754 binary16: p=11, emin=-14; bfloat16: p=8,       */
/* emin=-126), with gradual underflow and overflow to infinity.             */
/* ------------------------------------------------------------------------ */
static double round_to_format(double x, int p, int emin, double maxval)
{
    if (x == 0.0 || !isfinite(x)) return x;
    int e;
    frexp(x, &e);                 /* x = f 2^e, 0.5 <= |f| < 1 */
    int ex = e - 1;               /* x = g 2^ex, 1 <= |g| < 2 */
    if (ex < emin) ex = emin;     /* subnormal range: fixed quantum */
    double quantum = ldexp(1.0, ex - (p - 1));
    double r = nearbyint(x / quantum) * quantum;   /* default mode: ties to even */
    if (fabs(r) > maxval) r = copysign(INFINITY, x);
    return r;
}

double ora_round_f16(double x) { return round_to_format(x, 11, -14, 65504.0); }
double ora_round_bf16(double x) { return round_to_format(x, 8, -126, 3.3895313892515355e38); }

/* Stochastic rounding of x to bfloat16 with the 16 random bits r: x is
 * rounded to binary32 (ties to even), r is added to its bit pattern and the
 * low 16 bits are cleared.  The result is the bfloat16 neighbour above |x|
 * with probability (low 16 bits of x) / 2^16, else the one below.
 * Non-finite values round to nearest. */
double ora_sr_bf16(double x, uint32_t r)
{
    float f = (float)x;
    uint32_t b;
    memcpy(&b, &f, sizeof b);
    if ((b & 0x7F800000u) == 0x7F800000u) return ora_round_bf16(x);
    b = (b + (r & 0xFFFFu)) & 0xFFFF0000u;
    memcpy(&f, &b, sizeof f);
    return (double)f;
}

/* The 24 16-bit values of Philox blocks 2, 3, 4 of (site, step, replica):
 * r[p] is word (p mod 8) / 2 of block 2 + p / 8, low half for even p. */
void ora_sr_bits(uint64_t seed, uint32_t site, uint32_t step, uint32_t replica, uint32_t r[24])
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (uint32_t b = 0; b < 3; ++b) {
        uint32_t ctr[4] = {site, step, replica, 2 + b};
        uint32_t w[4];
        ora_philox4x32_10(ctr, key, w);
        for (int j = 0; j < 4; ++j) {
            r[8 * b + 2 * j] = w[j] & 0xFFFFu;
            r[8 * b + 2 * j + 1] = w[j] >> 16;
        }
    }
}

/* Rounds a whole state to the storage format (nearest even; the stochastic
 * format is rounded to nearest here, as the library does when a state is set). */
void ora_quantize(const ora_params *p, double *n)
{
    if (p->store != 2 && p->store != 3 && p->store != 4) return;
    lattice_t L;
    build_lattice(&L);
    int64_t N = (int64_t)p->nx * p->ny * p->nz;
    for (int i = 0; i < Q; ++i) {
        double base = p->rho0 * L.a[i];
        for (int64_t s = 0; s < N; ++s) {
            double d = n[(int64_t)i * N + s] - base;
            d = (p->store == 2) ? ora_round_f16(d) : ora_round_bf16(d);
            n[(int64_t)i * N + s] = base + d;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Time stepping: collide every site, then push-stream with periodic wrap.  */
/* n holds the pre-collision populations n[i][z][y][x] at step t0 on entry */
/* and at step t0 + nsteps on return.                                       */
/* ------------------------------------------------------------------------ */
static int wrap(int v, int n) { v %= n; return v < 0 ? v + n : v; }

int ora_run(const ora_params *p_in, double *n, uint32_t t0, uint32_t nsteps)
{
    ora_params p = *p_in;
    fill_gamma(p_in, p.gamma);
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    if (nx < 1 || ny < 1 || nz < 1) return -1;
    const int64_t N = (int64_t)nx * ny * nz;
    double *next = (double *)malloc(sizeof(double) * Q * (size_t)N);
    if (!next) return -2;
    lattice_t L;
    build_lattice(&L);
    const double two_pi = 6.283185307179586476925286766559;
    ora_quantize(&p, n);
    for (uint32_t t = t0; t < t0 + nsteps; ++t) {
#pragma omp parallel for schedule(static)
        for (int z = 0; z < nz; ++z) {
            for (int y = 0; y < ny; ++y) {
                for (int x = 0; x < nx; ++x) {
                    int64_t s = x + (int64_t)nx * (y + (int64_t)ny * z);
                    double loc[Q], out[Q], g[16];
                    for (int i = 0; i < Q; ++i) loc[i] = n[(int64_t)i * N + s];
                    if (p.kT > 0.0) ora_gaussians(p.seed, (uint32_t)s, t, p.replica, g);
                    else memset(g, 0, sizeof g);
                    double F[3] = {p.force_amp * sin(two_pi * (double)z / (double)nz), 0.0, 0.0};
                    collide(&p, &L, loc, g, F, out);
                    if (p.store == 4) {
                        uint32_t r[24];
                        ora_sr_bits(p.seed, (uint32_t)s, t, p.replica, r);
                        for (int i = 0; i < Q; ++i) {
                            double base = p.rho0 * L.a[i];
                            out[i] = base + ora_sr_bf16(out[i] - base, r[i]);
                        }
                    }
                    for (int i = 0; i < Q; ++i) {
                        int xd = wrap(x + VEL[i][0], nx);
                        int yd = wrap(y + VEL[i][1], ny);
                        int zd = wrap(z + VEL[i][2], nz);
                        int64_t sd = xd + (int64_t)nx * (yd + (int64_t)ny * zd);
                        next[(int64_t)i * N + sd] = out[i];
                    }
                }
            }
        }
        memcpy(n, next, sizeof(double) * Q * (size_t)N);
        if (p.store != 4) ora_quantize(&p, n);   /* store 4 rounded each value where it was computed */
    }
    free(next);
    return 0;
}

int ora_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Batch helpers for the tests: n independent Philox calls, and the sixteen
 * normals of sites 0..nsites-1 at one (step, replica). */
void ora_philox_many(const uint32_t *ctr /*[n][4]*/, const uint32_t *key /*[n][2]*/, int64_t n,
                     uint32_t *out /*[n][4]*/)
{
    for (int64_t s = 0; s < n; ++s) ora_philox4x32_10(ctr + 4 * s, key + 2 * s, out + 4 * s);
}

void ora_gaussians_many(uint64_t seed, uint32_t step, uint32_t replica, int64_t nsites,
                        double *g /*[nsites][16]*/)
{
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < nsites; ++s) ora_gaussians(seed, (uint32_t)s, step, replica, g + 16 * s);
}

/* Collision only (no streaming) of every site of a field at one step: the
 * single-site tests of Sec. IV draw many independent collisions this way. */
void ora_collide_field(const ora_params *p_in, const double *n /*[19][N]*/, uint32_t step,
                       double *out /*[19][N]*/)
{
    ora_params p = *p_in;
    fill_gamma(p_in, p.gamma);
    lattice_t L;
    build_lattice(&L);
    const double two_pi = 6.283185307179586476925286766559;
    const int64_t N = (int64_t)p.nx * p.ny * p.nz;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < N; ++s) {
        double loc[Q], res[Q], g[16];
        for (int i = 0; i < Q; ++i) loc[i] = n[(int64_t)i * N + s];
        if (p.kT > 0.0) ora_gaussians(p.seed, (uint32_t)s, step, p.replica, g);
        else memset(g, 0, sizeof g);
        int z = (int)(s / ((int64_t)p.nx * p.ny));
        double F[3] = {p.force_amp * sin(two_pi * (double)z / (double)p.nz), 0.0, 0.0};
        collide(&p, &L, loc, g, F, res);
        for (int i = 0; i < Q; ++i) out[(int64_t)i * N + s] = res[i];
    }
}

/* ora_run that also records the pre-collision state after every step:
 * trace[t][19][N] for t = 1..nsteps. */
int ora_run_trace(const ora_params *p, double *n, uint32_t t0, uint32_t nsteps, double *trace)
{
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    for (uint32_t t = 0; t < nsteps; ++t) {
        int rc = ora_run(p, n, t0 + t, 1);
        if (rc) return rc;
        memcpy(trace + (int64_t)t * Q * N, n, sizeof(double) * Q * (size_t)N);
    }
    return 0;
}
