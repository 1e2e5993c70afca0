// d3q19.cuh -- device-side arithmetic of the fluctuating D3Q19 update.
//
// Everything a stream-collide kernel does at one site, written for registers:
//   * the D3Q19 velocity set and weights (Sec. II of arXiv:0707.1581);
//   * the Table II mode transform and its inverse, factorised over the nine
//     pairs of opposite velocities (even modes see only pair sums, odd modes
//     only pair differences), so each transform costs ~60 adds instead of
//     the 207 nonzeros of the 19x19 matrix;
//   * the collision of Sec. IV: conserved modes kept, the stress modes relaxed
//     towards the equilibrium of Eq. derived_equil_distrib, the kinetic modes
//     relaxed towards zero, each plus Gaussian noise of amplitude
//     sqrt(mu rho0 w_k (1 - gamma_k^2)) (Eqs. updaterule, FDT);
//   * Philox-4x32-10 (Salmon et al., SC'11), two 16-bit uniforms per word, and
//     the Box-Muller transform: two Philox calls give the 15 normals of a site.
// The scale factors 1/w_k and the noise amplitudes are folded into per-mode
// constants computed once on the host, so relaxation + noise is two or three
// FMAs per mode.
#pragma once

#include <type_traits>

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace flb {

constexpr int Q = 19;

// Velocity order: rest; +x,-x,+y,-y,+z,-z; (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0);
// (0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1); (1,0,1),(-1,0,-1),(-1,0,1),(1,0,-1).
// Odd i >= 1 and i + 1 are opposite.
__host__ __device__ constexpr int vel_x(int i)
{
    constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1};
    return t[i];
}
__host__ __device__ constexpr int vel_y(int i)
{
    constexpr int t[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 1, -1, 1, -1, 0, 0, 0, 0};
    return t[i];
}
__host__ __device__ constexpr int vel_z(int i)
{
    constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int opposite(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// Weights a^{c_i}: 1/3 (rest), 1/18 (|c| = 1), 1/36 (|c| = sqrt 2).
__host__ __device__ constexpr double weight(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

// Norms w_k of the Table II basis vectors.
__host__ __device__ constexpr double mode_norm(int k)
{
    constexpr double t[Q] = {1.0,       1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, 2.0 / 3.0, 4.0 / 3.0, 4.0 / 9.0,
                             1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 2.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0, 2.0 / 9.0,
                             2.0 / 9.0, 2.0 / 9.0, 2.0,       4.0 / 3.0, 4.0 / 9.0};
    return t[k];
}

// Per-box constants of the collision, in the compute type R.
//   relax[k] = gamma_k / w_k,  eq[k] = (1 - gamma_k) / w_k,
//   noise[k] = sigma_k / w_k (times kBoxMullerF32Scale in FP32, see box_muller),
//   forcing[k] = (1 + gamma_k) / (2 w_k)  (k = 4..9)
// The 2^16 values each Box-Muller factor of the FP64 generator can take (its
// uniforms have 16 bits): r[k] = sqrt(-2 ln u) and cs[k] = (cos, sin)(2 pi u)
// at u = (k + 1/2) 2^-16.  Filled once per context by k_bm_tables with the
// same double-precision expressions the inline form evaluates, so a normal
// from the tables is bitwise the one computed in place; GB300's FP64 rate
// makes the accurate log and sincos the FP64 kernel's largest cost, and the
// 1.5 MB of tables stay in L2.
struct BoxMullerTables {
    const double *r;
    const double2 *cs;
};

// Only the FP64 constants carry the tables (a base class, so that the FP32
// constants keep the layout, and the kernels the constant loads, they had).
template <class R>
struct CollideTables {
};
template <>
struct CollideTables<double> {
    BoxMullerTables bm;
};
__device__ __forceinline__ BoxMullerTables bm_of(const CollideTables<float> &) { return BoxMullerTables{nullptr, nullptr}; }
__device__ __forceinline__ const BoxMullerTables &bm_of(const CollideTables<double> &K) { return K.bm; }

__device__ __forceinline__ void box_muller_entry(uint32_t k, double &r, double &c, double &s)
{
    const double u = ((double)k + 0.5) * 0x1p-16;
    r = sqrt(-2.0 * log(u));
    sincospi(2.0 * u, &s, &c);
}

template <class R>
struct CollideConsts : CollideTables<R> {
    R rho0;
    R inv_rho0;
    R relax[Q];
    R eq[Q];
    R noise[Q];
    R forcing[10];
    R force_amp;      // F_x(z) = force_amp sin(2 pi z / nz)
    R force_phase;    // 2 / nz (sin(pi * force_phase * z))
    int noise_rho_local;
    uint32_t rk0[10];  // Philox round keys k0 + r * 0x9E3779B9, r = 0..9
    uint32_t rk1[10];  // Philox round keys k1 + r * 0xBB67AE85
};

__device__ __forceinline__ float sin_pi(float x) { return sinpif(x); }
__device__ __forceinline__ double sin_pi(double x) { return sinpi(x); }

// --------------------------------------------------------------------------
// Philox-4x32-10 and Box-Muller.
// --------------------------------------------------------------------------
struct Words4 {
    uint32_t x, y, z, w;
};

// rk0/rk1 hold the ten round keys of the Weyl schedule (key + r W), computed
// once per box on the host, so a round is two 32x32->64 multiplies and two
// three-input XORs.
__device__ __forceinline__ Words4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                const uint32_t (&rk0)[10], const uint32_t (&rk1)[10])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk0[r];
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk1[r];
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
    }
    return Words4{c0, c1, c2, c3};
}

__device__ __forceinline__ float sqrt_approx(float x)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// The hardware log2, sine and cosine with denormals flushed: their inputs here
// (u1 >= 2^-17, |angle| < pi) never need the denormal handling of the
// non-flushing forms.
__device__ __forceinline__ float log2_approx(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void sincos_approx(float x, float &s, float &c)
{
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(s) : "f"(x));
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(c) : "f"(x));
}

// 1 / x: the hardware approximation in FP32 (at most 1 ulp off; the density
// it inverts is rho0 plus a small deviation, never 0 or denormal), exact
// division in FP64.
__device__ __forceinline__ float recip(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// Two sites in the two FP32 lanes of a float2: sm_100+ adds, multiplies and
// fuses a pair of FP32 operands in one instruction (__fadd2_rn, __fmul2_rn,
// __ffma2_rn, each lane rounded as the scalar operation), so the collision of
// two sites at once issues about half the FP32 instructions.  The 16-bit
// formats, bound by instruction issue, gain 6-7 %.
struct F2 {
    float2 v;
    __device__ __forceinline__ F2() {}
    __device__ __forceinline__ explicit F2(float a) : v(make_float2(a, a)) {}
    __device__ __forceinline__ F2(float a, float b) : v(make_float2(a, b)) {}
};
__device__ __forceinline__ F2 mk2(float2 v) { F2 r; r.v = v; return r; }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) { return mk2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator-(F2 a) { return F2(-a.v.x, -a.v.y); }
__device__ __forceinline__ F2 operator-(F2 a, F2 b) { return mk2(__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y))); }
__device__ __forceinline__ F2 operator*(F2 a, F2 b) { return mk2(__fmul2_rn(a.v, b.v)); }
__device__ __forceinline__ F2 operator*(float a, F2 b) { return F2(a) * b; }
__device__ __forceinline__ F2 operator*(F2 a, float b) { return a * F2(b); }
__device__ __forceinline__ F2 operator+(float a, F2 b) { return F2(a) + b; }
__device__ __forceinline__ F2 operator+(F2 a, float b) { return a + F2(b); }
__device__ __forceinline__ F2 &operator+=(F2 &a, F2 b) { a = a + b; return a; }
__device__ __forceinline__ F2 &operator*=(F2 &a, F2 b) { a = a * b; return a; }
// fma_r / sqrt_r: the operation in the compute type (paired, FP32 or FP64)
__device__ __forceinline__ F2 fma_r(F2 a, F2 b, F2 c) { return mk2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ float fma_r(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_r(double a, double b, double c) { return ::fma(a, b, c); }
__device__ __forceinline__ F2 sqrt_r(F2 x) { return F2(sqrtf(x.v.x), sqrtf(x.v.y)); }
__device__ __forceinline__ float sqrt_r(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_r(double x) { return ::sqrt(x); }
__device__ __forceinline__ F2 recip(F2 x) { return F2(recip(x.v.x), recip(x.v.y)); }

// One Box-Muller pair from one Philox word: u1 = (lo16 + 1/2) 2^-16 drives
// the radius, u2 = (hi16 + 1/2) 2^-16 the angle.
//
// FP32 variant, with the hardware approximations of log2 and sin/cos.  It
// returns the normals divided by sqrt(2 ln 2) -- radius sqrt(-log2 u1) instead
// of sqrt(-2 ln u1) -- and the FP32 noise amplitudes carry that factor (set on
// the host), which saves a multiply per pair.  u1 is built as the float
// 1 + lo16 2^-16 minus (1 - 2^-17), and u2 - 1/2 as 1 + hi16 2^-16 minus
// (3/2 - 2^-17): the first difference is representable, so the subtraction is
// exact; the second is folded with the factor 2 pi into one FMA (angle error
// below 1e-6 rad, under the error of the hardware sine).  The angle is taken
// in (-pi, pi), where sin.approx is most accurate: cos(2 pi u) =
// -cos(2 pi (u - 1/2)), sin(2 pi u) = -sin(2 pi (u - 1/2)).  u1 <= 1 - 2^-17,
// so log2 u1 <= -1.1e-5, far below the error of the hardware log2 near 1; its
// absolute value (a free operand modifier) only guards the square root.
constexpr double kBoxMullerF32Scale = 1.1774100225154747;   // sqrt(2 ln 2)

__device__ __forceinline__ void box_muller(uint32_t w, float &g0, float &g1)
{
    const float u1 = __uint_as_float(((w << 7) & 0x007fff80u) | 0x3f800000u) - (1.0f - 0x1p-17f);
    const float v2 = __uint_as_float(((w >> 9) & 0x007fff80u) | 0x3f800000u);      // 1 + hi16 2^-16
    const float angle = fmaf(v2, 6.2831853071795865f, -(1.5f - 0x1p-17f) * 6.2831853071795865f);
    const float R = sqrt_approx(fabsf(log2_approx(u1)));
    float s, c;
    sincos_approx(angle, s, c);
    g0 = -R * c;
    g1 = -R * s;
}

// FP64 variant: the accurate double-precision factors, read from the tables
// (box_muller_entry of the 16-bit halves: lo16 gives the radius, hi16 the angle).
__device__ __forceinline__ void box_muller(uint32_t w, double &g0, double &g1, const BoxMullerTables &T)
{
    const double R = __ldg(T.r + (w & 0xFFFFu));
    const double2 cs = __ldg(T.cs + (w >> 16));
    g0 = R * cs.x;
    g1 = R * cs.y;
}
__device__ __forceinline__ void box_muller(uint32_t w, float &g0, float &g1, const BoxMullerTables &)
{
    box_muller(w, g0, g1);
}

// The sixteen normals of (site, step, replica): Philox blocks b = 0, 1, word
// p = 4b + j gives g[2p], g[2p+1]; g[k - 4] drives mode k (g[15] is unused).
template <class R>
__device__ __forceinline__ void gaussians15(uint32_t site, uint32_t step, uint32_t replica, const uint32_t (&rk0)[10],
                                            const uint32_t (&rk1)[10], const BoxMullerTables &T, R (&g)[16])
{
#pragma unroll
    for (uint32_t b = 0; b < 2; ++b) {
        const Words4 w = philox4x32_10(site, step, replica, b, rk0, rk1);
        box_muller(w.x, g[8 * b + 0], g[8 * b + 1], T);
        box_muller(w.y, g[8 * b + 2], g[8 * b + 3], T);
        box_muller(w.z, g[8 * b + 4], g[8 * b + 5], T);
        box_muller(w.w, g[8 * b + 6], g[8 * b + 7], T);
    }
}

// --------------------------------------------------------------------------
// Forward transform m_k = sum_i e_ki f_i (Table II), on the pair sums s and
// differences d of opposite velocities.
// --------------------------------------------------------------------------
template <class R>
__device__ __forceinline__ void modes_from_pairs(R n0, R sx, R dx, R sy, R dy, R sz, R dz, R sxyp, R dxyp, R sxym,
                                                 R dxym, R syzp, R dyzp, R syzm, R dyzm, R szxp, R dzxp, R szxm,
                                                 R dzxm, R (&m)[Q])
{
    const R A = sx + sy + sz;
    const R Sxy = sxyp + sxym, Syz = syzp + syzm, Szx = szxp + szxm;
    const R Dg = Sxy + Syz + Szx;
    const R m0 = n0 + A + Dg;                              // rho (or rho - rho0)
    const R m4 = Dg - n0;                                  // c^2 - 1
    const R m16 = (n0 + Dg) - R(2) * A;                    // 3c^4 - 6c^2 + 1
    const R P = R(2) * sx - (sy + sz);
    const R Qd = (Sxy + Szx) - R(2) * Syz;
    const R m5 = P + Qd;                                   // 3cx^2 - c^2
    const R m17 = Qd - P;                                  // (2c^2-3)(3cx^2-c^2)
    const R R1 = sy - sz, R2 = Sxy - Szx;
    const R m6 = R1 + R2;                                  // cy^2 - cz^2
    const R m18 = R2 - R1;                                 // (2c^2-3)(cy^2-cz^2)
    const R m7 = sxyp - sxym;                              // cx cy
    const R m8 = syzp - syzm;                              // cy cz
    const R m9 = szxp - szxm;                              // cz cx

    const R a1 = dxyp + dxym, a2 = dxyp - dxym;
    const R b1 = dyzp + dyzm, b2 = dyzp - dyzm;
    const R c1 = dzxp + dzxm, c2 = dzxp - dzxm;
    const R Ux = a1 + c2, Uy = a2 + b1, Uz = b2 + c1;
    const R jx = dx + Ux, jy = dy + Uy, jz = dz + Uz;      // m1..m3
    const R m10 = Ux - R(2) * dx;                          // (3c^2-5) cx
    const R m11 = Uy - R(2) * dy;
    const R m12 = Uz - R(2) * dz;
    const R m13 = a1 - c2;                                 // (cy^2-cz^2) cx
    const R m14 = b1 - a2;                                 // (cz^2-cx^2) cy
    const R m15 = c1 - b2;                                 // (cx^2-cy^2) cz

    m[0] = m0;
    m[1] = jx;
    m[2] = jy;
    m[3] = jz;
    m[4] = m4;
    m[5] = m5;
    m[6] = m6;
    m[7] = m7;
    m[8] = m8;
    m[9] = m9;
    m[10] = m10;
    m[11] = m11;
    m[12] = m12;
    m[13] = m13;
    m[14] = m14;
    m[15] = m15;
    m[16] = m16;
    m[17] = m17;
    m[18] = m18;
}


template <class R>
__device__ __forceinline__ void forward_modes(const R (&f)[Q], R (&m)[Q])
{
    modes_from_pairs<R>(f[0], f[1] + f[2], f[1] - f[2], f[3] + f[4], f[3] - f[4], f[5] + f[6], f[5] - f[6],
                        f[7] + f[8], f[7] - f[8], f[9] + f[10], f[9] - f[10], f[11] + f[12], f[11] - f[12],
                        f[13] + f[14], f[13] - f[14], f[15] + f[16], f[15] - f[16], f[17] + f[18], f[17] - f[18], m);
}

// --------------------------------------------------------------------------
// The collision of one site, in place on f[19], which holds the deviations
// n_i - rho0 a_i (so m_0 = rho - rho0; modes k >= 1 equal those of n).
//   Fx  = body force density of this site along x (used when FORCE).
// R = F2 collides two sites at once (site = their two indices; constants K
// in FP32): the same operations, lane by lane.
// --------------------------------------------------------------------------
// NOISE: 0 = deterministic, 1 = thermal noise, 2 = thermal noise with
// gamma_ghost = 0 (the kinetic modes carry only their noise, so their forward
// transform and relaxation are skipped).
template <class R, int NOISE, bool FORCE, class KR, class SiteT>
__device__ __forceinline__ void collide(R (&f)[Q], const CollideConsts<KR> &K, SiteT site, uint32_t step,
                                        uint32_t replica, R Fx)
{
    constexpr bool kin0 = NOISE == 2;
    R m[Q];
    forward_modes<R>(f, m);
    const R m0 = m[0], jx = m[1], jy = m[2], jz = m[3], m4 = m[4], m5 = m[5], m6 = m[6], m7 = m[7], m8 = m[8];
    const R m9 = m[9], m10 = m[10], m11 = m[11], m12 = m[12], m13 = m[13], m14 = m[14], m15 = m[15];
    const R m16 = m[16], m17 = m[17], m18 = m[18];

    // --- equilibrium stress modes of Eq. derived_equil_distrib ---
    const R rho = K.rho0 + m0;
    const R inv_rho = recip(rho);
    const R px = FORCE ? jx + R(0.5) * Fx : jx;            // rho u (half-step momentum)
    const R ux = px * inv_rho, uy = jy * inv_rho, uz = jz * inv_rho;
    const R exx = px * ux, eyy = jy * uy, ezz = jz * uz;
    const R eq4 = exx + eyy + ezz;                         // rho u^2
    const R eq5 = R(3) * exx - eq4;                        // rho (3 ux^2 - u^2)
    const R eq6 = eyy - ezz;                               // rho (uy^2 - uz^2)
    const R eq7 = px * uy, eq8 = jy * uz, eq9 = jz * ux;   // rho u_a u_b

    // --- relaxation (+ noise, + forcing), scaled by 1/w_k for the inverse ---
    R t[Q];
    t[0] = m0;
    t[1] = R(3) * (FORCE ? jx + Fx : jx);
    t[2] = R(3) * jy;
    t[3] = R(3) * jz;
    t[4] = K.relax[4] * m4 + K.eq[4] * eq4;
    t[5] = K.relax[5] * m5 + K.eq[5] * eq5;
    t[6] = K.relax[6] * m6 + K.eq[6] * eq6;
    t[7] = K.relax[7] * m7 + K.eq[7] * eq7;
    t[8] = K.relax[8] * m8 + K.eq[8] * eq8;
    t[9] = K.relax[9] * m9 + K.eq[9] * eq9;
    if constexpr (kin0) {
#pragma unroll
        for (int k = 10; k < Q; ++k) t[k] = R(0);
    } else {
        t[10] = K.relax[10] * m10;
        t[11] = K.relax[11] * m11;
        t[12] = K.relax[12] * m12;
        t[13] = K.relax[13] * m13;
        t[14] = K.relax[14] * m14;
        t[15] = K.relax[15] * m15;
        t[16] = K.relax[16] * m16;
        t[17] = K.relax[17] * m17;
        t[18] = K.relax[18] * m18;
    }
    if (FORCE) {
        // source S = uF + Fu of the second moment, F = (Fx, 0, 0)
        const R uF = ux * Fx;
        t[4] += K.forcing[4] * (R(2) * uF);
        t[5] += K.forcing[5] * (R(4) * uF);
        t[7] += K.forcing[7] * (uy * Fx);
        t[9] += K.forcing[9] * (uz * Fx);
    }
    if (NOISE) {
        R g[16];
        if constexpr (std::is_same<R, F2>::value) {   // a pair of sites: each its own normals
            float ga[16], gb[16];
            gaussians15<float>(site.x, step, replica, K.rk0, K.rk1, bm_of(K), ga);
            gaussians15<float>(site.y, step, replica, K.rk0, K.rk1, bm_of(K), gb);
#pragma unroll
            for (int k = 0; k < 16; ++k) g[k] = R(ga[k], gb[k]);
        } else {
            gaussians15<R>(site, step, replica, K.rk0, K.rk1, bm_of(K), g);
        }
        if (K.noise_rho_local) {
            // variance mu rho w_k with the local density
            const R scale = sqrt_r(rho * K.inv_rho0);
#pragma unroll
            for (int k = 0; k < 15; ++k) g[k] *= scale;
        }
#pragma unroll
        for (int k = 4; k < Q; ++k) t[k] += K.noise[k] * g[k - 4];
    }

    // --- inverse transform n*_i = a_i sum_k e_ki t_k, per opposite pair ---
    const R D = t[0] + t[4] + t[16];
    const R Pp = t[5] + t[17], Rp = t[6] + t[18];
    const R Pm = t[5] - t[17], Rm = t[6] - t[18];
    const R X = t[0] - R(2) * t[16];
    const R Ex = X + R(2) * Pm;
    const R Ey = (X - Pm) + Rm;
    const R Ez = (X - Pm) - Rm;
    const R DP = D + Pp;
    const R Exy = DP + Rp, Ezx = DP - Rp;
    const R Eyz = D - R(2) * Pp;
    const R Ox = t[1] - R(2) * t[10];
    const R Oy = t[2] - R(2) * t[11];
    const R Oz = t[3] - R(2) * t[12];
    const R U1 = t[1] + t[10], U2 = t[2] + t[11], U3 = t[3] + t[12];
    const R Oxyp = (U1 + U2) + (t[13] - t[14]);
    const R Oxym = (U1 - U2) + (t[13] + t[14]);
    const R Oyzp = (U2 + U3) + (t[14] - t[15]);
    const R Oyzm = (U2 - U3) + (t[14] + t[15]);
    const R Ozxp = (U1 + U3) + (t[15] - t[13]);
    const R Ozxm = (U3 - U1) + (t[13] + t[15]);

    const R w0 = R(1.0 / 3.0), w1 = R(1.0 / 18.0), w2 = R(1.0 / 36.0);
    f[0] = w0 * ((t[0] - t[4]) + t[16]);
    {
        const R e = w1 * (Ex);
        f[1] = fma_r(w1, Ox, e);
        f[2] = fma_r(-w1, Ox, e);
    }
    {
        const R e = w1 * (Ey);
        f[3] = fma_r(w1, Oy, e);
        f[4] = fma_r(-w1, Oy, e);
    }
    {
        const R e = w1 * (Ez);
        f[5] = fma_r(w1, Oz, e);
        f[6] = fma_r(-w1, Oz, e);
    }
    {
        const R e = w2 * (Exy + t[7]);
        f[7] = fma_r(w2, Oxyp, e);
        f[8] = fma_r(-w2, Oxyp, e);
    }
    {
        const R e = w2 * (Exy - t[7]);
        f[9] = fma_r(w2, Oxym, e);
        f[10] = fma_r(-w2, Oxym, e);
    }
    {
        const R e = w2 * (Eyz + t[8]);
        f[11] = fma_r(w2, Oyzp, e);
        f[12] = fma_r(-w2, Oyzp, e);
    }
    {
        const R e = w2 * (Eyz - t[8]);
        f[13] = fma_r(w2, Oyzm, e);
        f[14] = fma_r(-w2, Oyzm, e);
    }
    {
        const R e = w2 * (Ezx + t[9]);
        f[15] = fma_r(w2, Ozxp, e);
        f[16] = fma_r(-w2, Ozxp, e);
    }
    {
        const R e = w2 * (Ezx - t[9]);
        f[17] = fma_r(w2, Ozxm, e);
        f[18] = fma_r(-w2, Ozxm, e);
    }
}

// --------------------------------------------------------------------------
// Storage formats.  Every format holds the deviation n_i - rho0 a_i from the
// rest equilibrium, so the resolution follows the size of the deviation (for
// FP32: 2^-24 of |n_i - rho0 a_i| instead of 2^-24 of rho0 a_i), the rounding
// of the weights never touches rho0 a_i, and the collision needs no offset.
// load() gives the deviation in the compute type, store() rounds it back.
// --------------------------------------------------------------------------
template <class S>
struct Storage;

template <>
struct Storage<double> {
    using R = double;
    static constexpr bool dev = true;
    static constexpr bool stochastic = false;
    __device__ static R load(double v) { return v; }
    __device__ static double store(R v) { return v; }
    __device__ static double from_double(double v) { return v; }
    __device__ static double to_double(double v) { return v; }
};
template <>
struct Storage<float> {
    using R = float;
    static constexpr bool dev = true;
    static constexpr bool stochastic = false;
    __device__ static R load(float v) { return v; }
    __device__ static float store(R v) { return v; }
    __device__ static float from_double(double v) { return (float)v; }
    __device__ static double to_double(float v) { return (double)v; }
};
template <>
struct Storage<__half> {
    using R = float;
    static constexpr bool dev = true;
    static constexpr bool stochastic = false;
    __device__ static R load(__half v) { return __half2float(v); }
    __device__ static __half store(R v) { return __float2half_rn(v); }
    __device__ static __half from_double(double v) { return __double2half(v); }
    __device__ static double to_double(__half v) { return (double)__half2float(v); }
};
template <>
struct Storage<__nv_bfloat16> {
    using R = float;
    static constexpr bool dev = true;
    static constexpr bool stochastic = false;
    __device__ static R load(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ static __nv_bfloat16 store(R v) { return __float2bfloat16_rn(v); }
    __device__ static __nv_bfloat16 from_double(double v) { return __double2bfloat16(v); }
    __device__ static double to_double(__nv_bfloat16 v) { return (double)__bfloat162float(v); }
};

// bfloat16 deviations written with stochastic rounding (FLB_STORE_BF16SR): the
// same 16-bit pattern as __nv_bfloat16, a distinct type so that the kernels
// round every post-collision value with random bits before storing it.
struct bf16sr {
    uint16_t bits;
};
template <>
struct Storage<bf16sr> {
    using R = float;
    static constexpr bool dev = true;
    static constexpr bool stochastic = true;
    __device__ static R load(bf16sr v) { return __uint_as_float((uint32_t)v.bits << 16); }
    // the upper 16 bits: stochastic_round has already added the random bits
    // below them (and left non-finite values as they were, which stay
    // non-finite when cut)
    __device__ static bf16sr store(R v) { return bf16sr{(unsigned short)(__float_as_uint(v) >> 16)}; }
    __device__ static bf16sr from_double(double v) { return bf16sr{__bfloat16_as_ushort(__double2bfloat16(v))}; }
    __device__ static double to_double(bf16sr v) { return (double)load(v); }
};

// Read-only cached load of one stored element (the 16-bit pattern for bf16sr).
template <class S>
__device__ __forceinline__ S load_ro(const S *p)
{
    return __ldg(p);
}
template <>
__device__ __forceinline__ bf16sr load_ro<bf16sr>(const bf16sr *p)
{
    return bf16sr{__ldg(reinterpret_cast<const unsigned short *>(p))};
}

// Stochastic rounding of x to bfloat16 with 16 random bits r: r is added to
// the bit pattern, and cutting the low 16 bits (the store of the stochastic
// format) completes it, so |x| rounds up with probability (low 16 bits) / 2^16
// and the expected result is x.  For finite x only: the carry of a NaN
// pattern can reach the sign bit.
__device__ __forceinline__ float sr_bf16_bits(float x, uint32_t r)
{
    return __uint_as_float(__float_as_uint(x) + r);
}

// For the stochastic format: rounds the NQ post-collision deviations of one
// site with the 16-bit values of Philox blocks 2, 3, ... of (site, step,
// replica); population i takes word (i mod 8) / 2 of block 2 + i / 8, low
// half for even i.  A site whose sum is finite has only finite values and
// takes the plain path; otherwise every non-finite value is left as it is.
// No-op for the other formats.
template <class S, int NQ, class R>
__device__ __forceinline__ void stochastic_round(R (&f)[NQ], uint32_t site, uint32_t step, uint32_t replica,
                                                 const uint32_t (&rk0)[10], const uint32_t (&rk1)[10])
{
    if constexpr (Storage<S>::stochastic) {
        uint32_t r[NQ];
#pragma unroll
        for (int b = 0; b < (NQ + 7) / 8; ++b) {
            const Words4 w = philox4x32_10(site, step, replica, 2u + (uint32_t)b, rk0, rk1);
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int p = 8 * b; p < 8 * b + 8 && p < NQ; ++p) r[p] = p & 1 ? ws[(p & 7) >> 1] >> 16 : ws[(p & 7) >> 1] & 0xffffu;
        }
        R sum = f[0];
#pragma unroll
        for (int i = 1; i < NQ; ++i) sum += f[i];
        if (fabsf(sum) <= 3.402823466e38f) {   // false for NaN and infinities
#pragma unroll
            for (int p = 0; p < NQ; ++p) f[p] = sr_bf16_bits(f[p], r[p]);
        } else {
#pragma unroll
            for (int p = 0; p < NQ; ++p)
                if (fabsf(f[p]) <= 3.402823466e38f) f[p] = sr_bf16_bits(f[p], r[p]);
        }
    }
}

// --------------------------------------------------------------------------
// Bounds checks of the checking build (compiled with FLB_BOUNDS_CHECK; the
// ordinary build compiles them away).  Every global access of a stream-collide
// kernel passes its span [p, p + n) through a guard against the Q planes of
// the buffer it addresses; a span outside counts one violation in a device
// word and the access is not made (a load reads the buffer's first elements,
// a store is dropped), so a bad index is reported instead of faulting.
// --------------------------------------------------------------------------
template <class S, int NQ>
__device__ __forceinline__ bool span_ok(const S *base, int64_t plane, const S *p, int n, unsigned long long *viol)
{
    const bool ok = p >= base && p + n <= base + (int64_t)NQ * plane;
    if (!ok && viol) atomicAdd(viol, 1ull);
    return ok;
}

#ifdef FLB_BOUNDS_CHECK
#define FLB_VIOL_FIELD unsigned long long *viol;   /* violation counter of the checking build */
#define FLB_GUARD_LD(B, p, n) (span_ok<S, Q>((B).src, (B).plane, (p), (n), (B).viol) ? (p) : (B).src)
#define FLB_GUARD_ST(B, p, n) span_ok<S, Q>((B).dst, (B).plane, (p), (n), (B).viol)
#else
#define FLB_VIOL_FIELD
#define FLB_GUARD_LD(B, p, n) (p)
#define FLB_GUARD_ST(B, p, n) true
#endif

// --------------------------------------------------------------------------
// Where the canonical pre-collision population n_i(r, t) lives in device memory.
//   AB (pull):     slot i at r - c_i of the current buffer (it holds the
//                  post-collision values of the previous step at their origin).
//   AA, t even:    slot i at r.
//   AA, t odd:     slot opposite(i) at r - c_i.
// --------------------------------------------------------------------------
enum Layout : int { kAB = 0, kAAEven = 1, kAAOdd = 2 };

__host__ __device__ inline int wrap_add(int v, int d, int n)
{
    v += d;
    return v < 0 ? v + n : (v >= n ? v - n : v);
}

struct Slot {
    int q;
    int x, y, z;
};

__device__ __forceinline__ Slot canonical_slot(int layout, int i, int x, int y, int z, int nx, int ny, int nz)
{
    if (layout == kAAEven) return Slot{i, x, y, z};
    const int xs = wrap_add(x, -vel_x(i), nx), ys = wrap_add(y, -vel_y(i), ny), zs = wrap_add(z, -vel_z(i), nz);
    return Slot{layout == kAB ? i : opposite(i), xs, ys, zs};
}

}  // namespace flb
