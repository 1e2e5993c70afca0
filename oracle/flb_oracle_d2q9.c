/*
 * flb_oracle_d2q9.c -- plain FP64 CPU oracle of the fluctuating lattice
 * Boltzmann update on D2Q9 (Duenweg, Schiller, Ladd, arXiv:0707.1581,
 * Table I).
 *
 * TEST INFRASTRUCTURE ONLY, like flb_oracle.c next to it (whose Philox
 * generator, Box-Muller normals and rounding helpers it calls): only the
 * tests and the smoke check may load it, and it shares nothing with the CUDA
 * library.
 *
 * Per time step t and site r = (x, y) of an nx x ny periodic box:
 *   1. modes        m_k = sum_i e_ki n_i                      (Table I, Sec. III)
 *   2. equilibrium  n_i^eq(rho, u), u = j / rho (2-D)         (Eq. derived_equil_distrib)
 *                   m_k^eq = sum_i e_ki n_i^eq
 *   3. collision    m*_k = m_k^eq + gamma_k (m_k - m_k^eq) + sigma_k r_k, k >= 3
 *                   m*_k = m_k for the conserved modes k <= 2  (Eqs. updaterule, FDT)
 *                   sigma_k = sqrt(mu rho0 w_k (1 - gamma_k^2)), mu = 3 k_B T
 *   4. back         n*_i = a_i sum_k e_ki m*_k / w_k
 *   5. streaming    n_i(r + c_i, t + 1) = n*_i(r, t)           (Eq. LBE, push form)
 * Literal 9 x 9 loops, no factorisation.
 *
 * Readings taken where the paper is silent or leaves a choice open:
 *  - velocity order: rest; +x, -x, +y, -y; (1,1), (-1,-1), (1,-1), (-1,1);
 *  - eigenvalues: gamma_bulk for mode 3, gamma_shear for modes 4 and 5,
 *    gamma_ghost for the kinetic modes 6..8;
 *  - normals: the first block of the D3Q19 generator, i.e. Philox-4x32-10
 *    with counter (site x + nx y, step, replica, 0); mode k uses g[k - 3];
 *  - body force F = (F0 sin(2 pi y / ny), 0), the same second-order
 *    moment-space forcing as the D3Q19 oracle;
 *  - reduced-precision storage rounds n - rho0 a_i after each step; the
 *    stochastic bfloat16 format (store 4) rounds each post-collision value
 *    with the bits of ora_sr_bits, as the D3Q19 oracle does.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q9 9

void ora_gaussians(uint64_t seed, uint32_t site, uint32_t step, uint32_t replica, double g[16]);
double ora_round_f16(double x);
double ora_round_bf16(double x);
double ora_sr_bf16(double x, uint32_t r);
void ora_sr_bits(uint64_t seed, uint32_t site, uint32_t step, uint32_t replica, uint32_t r[24]);

/* D2Q9 velocities; weights a^0 = 4/9, a^1 = 1/9, a^sqrt2 = 1/36, c_s^2 = 1/3 (Sec. II). */
static const int VEL2[Q9][2] = {
    {0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, -1}, {1, -1}, {-1, 1},
};

static double weight2(int i)
{
    int c2 = VEL2[i][0] * VEL2[i][0] + VEL2[i][1] * VEL2[i][1];
    if (c2 == 0) return 4.0 / 9.0;
    if (c2 == 1) return 1.0 / 9.0;
    return 1.0 / 36.0;
}

static const double CS2_2 = 1.0 / 3.0;

/* Table I: the polynomial e_k(c) of row k at velocity c. */
static double table1_poly(int k, const int c[2])
{
    double x = c[0], y = c[1];
    double c2 = x * x + y * y;
    switch (k) {
    case 0: return 1.0;
    case 1: return x;
    case 2: return y;
    case 3: return 3.0 * c2 - 2.0;
    case 4: return 2.0 * x * x - c2;
    case 5: return x * y;
    case 6: return (3.0 * c2 - 4.0) * x;
    case 7: return (3.0 * c2 - 4.0) * y;
    case 8: return 9.0 * c2 * c2 - 15.0 * c2 + 2.0;
    }
    return 0.0;
}

typedef struct {
    double a[Q9];
    double e[Q9][Q9];   /* e[k][i] */
    double w[Q9];       /* w_k = sum_i a_i e_ki^2 */
} lattice2_t;

static void build_lattice2(lattice2_t *L)
{
    for (int i = 0; i < Q9; ++i) L->a[i] = weight2(i);
    for (int k = 0; k < Q9; ++k) {
        double wk = 0.0;
        for (int i = 0; i < Q9; ++i) {
            L->e[k][i] = table1_poly(k, VEL2[i]);
            wk += L->a[i] * L->e[k][i] * L->e[k][i];
        }
        L->w[k] = wk;
    }
}

void ora2_lattice(int *c /*9*2*/, double *a /*9*/, double *e /*9*9, [k][i]*/, double *w /*9*/)
{
    lattice2_t L;
    build_lattice2(&L);
    for (int i = 0; i < Q9; ++i) {
        c[2 * i] = VEL2[i][0];
        c[2 * i + 1] = VEL2[i][1];
        a[i] = L.a[i];
    }
    for (int k = 0; k < Q9; ++k) {
        w[k] = L.w[k];
        for (int i = 0; i < Q9; ++i) e[k * Q9 + i] = L.e[k][i];
    }
}

typedef struct {
    int nx, ny;
    double rho0;
    double kT;
    double gamma[Q9];      /* modes 0..2 are forced to 1 */
    uint64_t seed;
    uint32_t replica;
    int noise_ghosts;      /* 1: thermalize the kinetic modes 6..8 too */
    int noise_rho_local;   /* 0: variance mu rho0 w_k; 1: mu rho(r) w_k */
    double force_amp;      /* F_x(y) = force_amp sin(2 pi y / ny) */
    int store;             /* 0 exact FP64; 2 FP16 deviation; 3 BF16 deviation; 4 BF16 stochastic */
} ora2_params;

/* Eq. derived_equil_distrib in two dimensions, sigma_2 = c_s^2 = 1/3. */
static void equilibrium2(double rho, const double u[2], const double a[Q9], double neq[Q9])
{
    double u2 = u[0] * u[0] + u[1] * u[1];
    for (int i = 0; i < Q9; ++i) {
        double cu = VEL2[i][0] * u[0] + VEL2[i][1] * u[1];
        neq[i] = rho * a[i] * (1.0 + cu / CS2_2 + cu * cu / (2.0 * CS2_2 * CS2_2) - u2 / (2.0 * CS2_2));
    }
}

void ora2_equilibrium_field(int64_t nsites, const double *rho, const double *u /*[2][N]*/, double *n /*[9][N]*/)
{
    lattice2_t L;
    build_lattice2(&L);
    for (int64_t s = 0; s < nsites; ++s) {
        double uu[2] = {u[s], u[nsites + s]};
        double neq[Q9];
        equilibrium2(rho[s], uu, L.a, neq);
        for (int i = 0; i < Q9; ++i) n[(int64_t)i * nsites + s] = neq[i];
    }
}

static void collide2(const ora2_params *p, const lattice2_t *L, const double n[Q9], const double g[16],
                     const double F[2], double nstar[Q9])
{
    double m[Q9], meq[Q9], ms[Q9], neq[Q9], Smode[Q9];
    for (int k = 0; k < Q9; ++k) {
        double s = 0.0;
        for (int i = 0; i < Q9; ++i) s += L->e[k][i] * n[i];
        m[k] = s;
    }
    double rho = m[0];
    double u[2] = {(m[1] + 0.5 * F[0]) / rho, (m[2] + 0.5 * F[1]) / rho};
    equilibrium2(rho, u, L->a, neq);
    for (int k = 0; k < Q9; ++k) {
        double s = 0.0;
        for (int i = 0; i < Q9; ++i) s += L->e[k][i] * neq[i];
        meq[k] = s;
    }
    for (int k = 0; k < Q9; ++k) Smode[k] = 0.0;
    if (F[0] != 0.0 || F[1] != 0.0) {
        /* second-moment source S = u F + F u carried by the population set
         * a_i (c_ia c_ib - c_s^2 d_ab) S_ab / (2 c_s^4) (no mass, momentum or ghosts) */
        double S[2][2], nS[Q9];
        for (int al = 0; al < 2; ++al)
            for (int be = 0; be < 2; ++be) S[al][be] = u[al] * F[be] + F[al] * u[be];
        for (int i = 0; i < Q9; ++i) {
            double acc = 0.0;
            for (int al = 0; al < 2; ++al)
                for (int be = 0; be < 2; ++be)
                    acc += (VEL2[i][al] * VEL2[i][be] - (al == be ? CS2_2 : 0.0)) * S[al][be];
            nS[i] = L->a[i] * acc / (2.0 * CS2_2 * CS2_2);
        }
        for (int k = 0; k < Q9; ++k) {
            double s = 0.0;
            for (int i = 0; i < Q9; ++i) s += L->e[k][i] * nS[i];
            Smode[k] = s;
        }
    }
    double mu = 3.0 * p->kT;
    double rho_var = p->noise_rho_local ? rho : p->rho0;
    for (int k = 0; k < Q9; ++k) {
        if (k <= 2) {
            ms[k] = m[k];
            continue;
        }
        double gk = p->gamma[k];
        double v = meq[k] + gk * (m[k] - meq[k]) + 0.5 * (1.0 + gk) * Smode[k];
        int thermal = (k <= 5) || p->noise_ghosts;
        if (p->kT > 0.0 && thermal) v += sqrt(mu * rho_var * L->w[k] * (1.0 - gk * gk)) * g[k - 3];
        ms[k] = v;
    }
    ms[1] += F[0];
    ms[2] += F[1];
    for (int i = 0; i < Q9; ++i) {
        double s = 0.0;
        for (int k = 0; k < Q9; ++k) s += L->e[k][i] * ms[k] / L->w[k];
        nstar[i] = L->a[i] * s;
    }
}

static void fill_gamma2(const ora2_params *in, ora2_params *p)
{
    *p = *in;
    for (int k = 0; k <= 2; ++k) p->gamma[k] = 1.0;
}

void ora2_collide_site(const ora2_params *p_in, const double n[Q9], uint32_t site, uint32_t step, const double F[2],
                       const double *g_in, double nstar[Q9])
{
    ora2_params p;
    fill_gamma2(p_in, &p);
    lattice2_t L;
    build_lattice2(&L);
    double g[16];
    if (g_in) memcpy(g, g_in, sizeof g);
    else ora_gaussians(p.seed, site, step, p.replica, g);
    double Fz[2] = {0.0, 0.0};
    collide2(&p, &L, n, g, F ? F : Fz, nstar);
}

void ora2_quantize(const ora2_params *p, double *n)
{
    if (p->store != 2 && p->store != 3 && p->store != 4) return;
    lattice2_t L;
    build_lattice2(&L);
    int64_t N = (int64_t)p->nx * p->ny;
    for (int i = 0; i < Q9; ++i) {
        double base = p->rho0 * L.a[i];
        for (int64_t s = 0; s < N; ++s) {
            double d = n[(int64_t)i * N + s] - base;
            d = (p->store == 2) ? ora_round_f16(d) : ora_round_bf16(d);
            n[(int64_t)i * N + s] = base + d;
        }
    }
}

static int wrap2(int v, int n) { v %= n; return v < 0 ? v + n : v; }

/* n[9][y][x]: pre-collision populations at step t0 on entry, t0 + nsteps on return. */
int ora2_run(const ora2_params *p_in, double *n, uint32_t t0, uint32_t nsteps)
{
    ora2_params p;
    fill_gamma2(p_in, &p);
    const int nx = p.nx, ny = p.ny;
    if (nx < 1 || ny < 1) return -1;
    const int64_t N = (int64_t)nx * ny;
    double *next = (double *)malloc(sizeof(double) * Q9 * (size_t)N);
    if (!next) return -2;
    lattice2_t L;
    build_lattice2(&L);
    const double two_pi = 6.283185307179586476925286766559;
    ora2_quantize(&p, n);
    for (uint32_t t = t0; t < t0 + nsteps; ++t) {
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y) {
            for (int x = 0; x < nx; ++x) {
                int64_t s = x + (int64_t)nx * y;
                double loc[Q9], out[Q9], g[16];
                for (int i = 0; i < Q9; ++i) loc[i] = n[(int64_t)i * N + s];
                if (p.kT > 0.0) ora_gaussians(p.seed, (uint32_t)s, t, p.replica, g);
                else memset(g, 0, sizeof g);
                double F[2] = {p.force_amp * sin(two_pi * (double)y / (double)ny), 0.0};
                collide2(&p, &L, loc, g, F, out);
                if (p.store == 4) {
                    uint32_t r[24];
                    ora_sr_bits(p.seed, (uint32_t)s, t, p.replica, r);
                    for (int i = 0; i < Q9; ++i) {
                        double base = p.rho0 * L.a[i];
                        out[i] = base + ora_sr_bf16(out[i] - base, r[i]);
                    }
                }
                for (int i = 0; i < Q9; ++i) {
                    int xd = wrap2(x + VEL2[i][0], nx);
                    int yd = wrap2(y + VEL2[i][1], ny);
                    next[(int64_t)i * N + xd + (int64_t)nx * yd] = out[i];
                }
            }
        }
        memcpy(n, next, sizeof(double) * Q9 * (size_t)N);
        if (p.store != 4) ora2_quantize(&p, n);
    }
    free(next);
    return 0;
}

/* Collision only at every site of a field, one step (single-site statistics). */
void ora2_collide_field(const ora2_params *p_in, const double *n /*[9][N]*/, uint32_t step, double *out /*[9][N]*/)
{
    ora2_params p;
    fill_gamma2(p_in, &p);
    lattice2_t L;
    build_lattice2(&L);
    const double two_pi = 6.283185307179586476925286766559;
    const int64_t N = (int64_t)p.nx * p.ny;
#pragma omp parallel for schedule(static)
    for (int64_t s = 0; s < N; ++s) {
        double loc[Q9], res[Q9], g[16];
        for (int i = 0; i < Q9; ++i) loc[i] = n[(int64_t)i * N + s];
        if (p.kT > 0.0) ora_gaussians(p.seed, (uint32_t)s, step, p.replica, g);
        else memset(g, 0, sizeof g);
        int y = (int)(s / p.nx);
        double F[2] = {p.force_amp * sin(two_pi * (double)y / (double)p.ny), 0.0};
        collide2(&p, &L, loc, g, F, res);
        for (int i = 0; i < Q9; ++i) out[(int64_t)i * N + s] = res[i];
    }
}
