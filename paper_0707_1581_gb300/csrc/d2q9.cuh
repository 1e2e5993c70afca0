// d2q9.cuh -- the fluctuating update on the D2Q9 lattice (Table I of
// arXiv:0707.1581): per-site arithmetic and the kernels of the D2Q9 boxes.
//
// The method is the one of the D3Q19 path (Sec. IV: conserved modes kept,
// stress modes relaxed towards the equilibrium of Eq. derived_equil_distrib,
// kinetic modes towards zero, each plus Gaussian noise of amplitude
// sqrt(mu rho0 w_k (1 - gamma_k^2)), Eqs. updaterule and FDT) on the nine
// velocities of D2Q9 with the basis of Table I.  Six modes are thermalized,
// so one Philox-4x32-10 call (counter block 0, the first block of the D3Q19
// generator) gives the normals: word j feeds normals 2j and 2j + 1, mode k
// uses normal k - 3.
//
// A box is nx x ny (nz = 1); populations are stored as planes [q][y][x] of
// deviations n_i - rho0 a_i, like the D3Q19 formats, in the AB (pull) or AA
// (in-place) pattern.  The vectorised kernel takes 4 sites per thread (2 for
// FP64), the scalar one 1 (for nx not a multiple of 4): at 72 bytes per FP32
// site update the update is bound by HBM bandwidth well before the ~250 lane
// instructions of its arithmetic.
#pragma once

#include "d3q19.cuh"
#include "internal.h"

namespace flb {
namespace d2 {

constexpr int Q = 9;

template <int BYTES>
struct RawVec2;
template <>
struct RawVec2<8> {
    using T = uint2;
};
template <>
struct RawVec2<16> {
    using T = uint4;
};

// Velocity order: rest; +x, -x, +y, -y; (1,1), (-1,-1), (1,-1), (-1,1).
// Odd i and i + 1 are opposite.
__host__ __device__ constexpr int vel_x(int i)
{
    constexpr int t[Q] = {0, 1, -1, 0, 0, 1, -1, 1, -1};
    return t[i];
}
__host__ __device__ constexpr int vel_y(int i)
{
    constexpr int t[Q] = {0, 0, 0, 1, -1, 1, -1, -1, 1};
    return t[i];
}
__host__ __device__ constexpr int opposite(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// Weights 4/9 (rest), 1/9 (|c| = 1), 1/36 (|c| = sqrt 2): the solution of
// Eqs. wi0-wi4 on these speeds with sigma_2 = c_s^2 = 1/3.
__host__ __device__ constexpr double weight(int i) { return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }

// Norms w_k of the Table I basis vectors.
__host__ __device__ constexpr double mode_norm(int k)
{
    constexpr double t[Q] = {1.0, 1.0 / 3.0, 1.0 / 3.0, 4.0, 4.0 / 9.0, 1.0 / 9.0, 2.0 / 3.0, 2.0 / 3.0, 16.0};
    return t[k];
}

// Per-box constants in the compute type R (host-filled):
//   relax[k] = gamma_k / w_k, eq[k] = (1 - gamma_k) / w_k, noise[k] = sigma_k / w_k
//   (times kBoxMullerF32Scale in FP32), forcing[k] = (1 + gamma_k) / (2 w_k), k = 3..5.
template <class R>
struct CollideConsts : CollideTables<R> {
    R rho0;
    R inv_rho0;
    R relax[Q];
    R eq[Q];
    R noise[Q];
    R forcing[6];
    R force_amp;      // F_x(y) = force_amp sin(2 pi y / ny)
    R force_phase;    // 2 / ny
    int noise_rho_local;
    uint32_t rk0[10];
    uint32_t rk1[10];
};

// Collision of one site, in place on the deviations f[9] (m_0 = rho - rho0).
// R = F2 collides two sites at once (site = their two indices; K in FP32).
template <class R, bool NOISE, bool FORCE, class KR, class SiteT>
__device__ __forceinline__ void collide(R (&f)[Q], const CollideConsts<KR> &K, SiteT site, uint32_t step,
                                        uint32_t replica, R Fx)
{
    // Table I transform on the sums s and differences d of opposite pairs
    const R sx = f[1] + f[2], dx = f[1] - f[2];
    const R sy = f[3] + f[4], dy = f[3] - f[4];
    const R sa = f[5] + f[6], da = f[5] - f[6];      // (1,1) / (-1,-1)
    const R sb = f[7] + f[8], db = f[7] - f[8];      // (1,-1) / (-1,1)
    const R A = sx + sy, Dg = sa + sb;
    const R m0 = f[0] + A + Dg;                      // rho - rho0
    const R jx = dx + (da + db);
    const R jy = dy + (da - db);
    const R m3 = (A - R(2) * f[0]) + R(4) * Dg;      // 3c^2 - 2
    const R m4 = sx - sy;                            // 2cx^2 - c^2
    const R m5 = sa - sb;                            // cx cy
    const R m6 = R(2) * (da + db) - dx;              // (3c^2 - 4) cx
    const R m7 = R(2) * (da - db) - dy;              // (3c^2 - 4) cy
    const R m8 = (R(2) * f[0] - R(4) * A) + R(8) * Dg;   // 9c^4 - 15c^2 + 2

    // equilibrium of the stress modes, rho u u with u at the half step
    const R rho = K.rho0 + m0;
    const R inv_rho = recip(rho);
    const R px = FORCE ? jx + R(0.5) * Fx : jx;
    const R ux = px * inv_rho, uy = jy * inv_rho;
    const R exx = px * ux, eyy = jy * uy;
    const R eq3 = R(3) * (exx + eyy);
    const R eq4 = exx - eyy;
    const R eq5 = px * uy;

    R t[Q];
    t[0] = m0;
    t[1] = R(3) * (FORCE ? jx + Fx : jx);
    t[2] = R(3) * jy;
    t[3] = K.relax[3] * m3 + K.eq[3] * eq3;
    t[4] = K.relax[4] * m4 + K.eq[4] * eq4;
    t[5] = K.relax[5] * m5 + K.eq[5] * eq5;
    t[6] = K.relax[6] * m6;
    t[7] = K.relax[7] * m7;
    t[8] = K.relax[8] * m8;
    if (FORCE) {
        // source S = uF + Fu, F = (Fx, 0): modes 3, 4, 5 see 3 tr S, S_xx - S_yy, S_xy
        const R uF = ux * Fx;
        t[3] += K.forcing[3] * (R(6) * uF);
        t[4] += K.forcing[4] * (R(2) * uF);
        t[5] += K.forcing[5] * (uy * Fx);
    }
    if (NOISE) {
        R g[6];
        if constexpr (std::is_same<R, F2>::value) {   // a pair of sites: each its own normals
            float ga[6], gb[6];
            const Words4 wa = philox4x32_10(site.x, step, replica, 0u, K.rk0, K.rk1);
            const Words4 wb = philox4x32_10(site.y, step, replica, 0u, K.rk0, K.rk1);
            box_muller(wa.x, ga[0], ga[1]);
            box_muller(wa.y, ga[2], ga[3]);
            box_muller(wa.z, ga[4], ga[5]);
            box_muller(wb.x, gb[0], gb[1]);
            box_muller(wb.y, gb[2], gb[3]);
            box_muller(wb.z, gb[4], gb[5]);
#pragma unroll
            for (int k = 0; k < 6; ++k) g[k] = R(ga[k], gb[k]);
        } else {
            const Words4 w = philox4x32_10(site, step, replica, 0u, K.rk0, K.rk1);
            box_muller(w.x, g[0], g[1], bm_of(K));
            box_muller(w.y, g[2], g[3], bm_of(K));
            box_muller(w.z, g[4], g[5], bm_of(K));
        }
        if (K.noise_rho_local) {
            const R scale = sqrt_r(rho * K.inv_rho0);
#pragma unroll
            for (int k = 0; k < 6; ++k) g[k] *= scale;
        }
#pragma unroll
        for (int k = 3; k < Q; ++k) t[k] += K.noise[k] * g[k - 3];
    }

    // n*_i = a_i sum_k e_ki t_k, per opposite pair
    const R ax = (t[0] + t[3]) - R(4) * t[8];
    const R dg = (t[0] + R(4) * t[3]) + R(8) * t[8];
    const R w0 = R(4.0 / 9.0), w1 = R(1.0 / 9.0), w2 = R(1.0 / 36.0);
    f[0] = w0 * ((t[0] - R(2) * t[3]) + R(2) * t[8]);
    {
        const R e = w1 * (ax + t[4]), o = w1 * (t[1] - t[6]);
        f[1] = e + o;
        f[2] = e - o;
    }
    {
        const R e = w1 * (ax - t[4]), o = w1 * (t[2] - t[7]);
        f[3] = e + o;
        f[4] = e - o;
    }
    const R o6 = R(2) * t[6], o7 = R(2) * t[7];
    {
        const R e = w2 * (dg + t[5]), o = w2 * ((t[1] + t[2]) + (o6 + o7));
        f[5] = e + o;
        f[6] = e - o;
    }
    {
        const R e = w2 * (dg - t[5]), o = w2 * ((t[1] - t[2]) + (o6 - o7));
        f[7] = e + o;
        f[8] = e - o;
    }
}

template <class S>
struct BoxStep {
    const S *src;
    S *dst;
    int nx, ny;
    int gx;                    // blocks along x
    int pad_;
    int64_t plane;
    uint32_t replica;
    CollideConsts<typename Storage<S>::R> K;
    FLB_VIOL_FIELD
};

// One thread per site; blockIdx.x enumerates (x block, y block).
//   AB      pull n_i(r) from slot i at r - c_i of src, store n*_i(r) in slot i at r of dst.
//   AA even read slot i at r, store n*_i(r) in slot opposite(i) at r.
//   AA odd  read slot opposite(i) at r - c_i, store n*_i(r) in slot i at r + c_i.
template <class S, int LAYOUT, bool NOISE, bool FORCE>
__global__ void __launch_bounds__(256) k_stream_collide(const BoxStep<S> B, const uint32_t *step_ptr, uint32_t step)
{
    using R = typename Storage<S>::R;
    const int bxi = blockIdx.x % B.gx, byi = blockIdx.x / B.gx;
    const int x = bxi * blockDim.x + threadIdx.x;
    const int y = byi * blockDim.y + threadIdx.y;
    if (x >= B.nx || y >= B.ny) return;
    if (step_ptr) step += *step_ptr;
    const int nx = B.nx, ny = B.ny;
    const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    auto xsel = [&](int c) { return c > 0 ? xm : (c < 0 ? xp : x); };        // x - c
    auto ysel = [&](int c) { return c > 0 ? ym : (c < 0 ? yp : y); };
    auto xpush = [&](int c) { return c > 0 ? xp : (c < 0 ? xm : x); };      // x + c
    auto ypush = [&](int c) { return c > 0 ? yp : (c < 0 ? ym : y); };
    const int site = y * nx + x;
    R f[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int idx = site, slot = i;
        if (LAYOUT != kAAEven) {
            idx = ysel(vel_y(i)) * nx + xsel(vel_x(i));
            slot = LAYOUT == kAB ? i : opposite(i);
        }
        const S *p = B.src + (int64_t)slot * B.plane + idx;
        f[i] = Storage<S>::load(load_ro(FLB_GUARD_LD(B, p, 1)));
    }
    R Fx = R(0);
    if (FORCE) Fx = B.K.force_amp * sin_pi(B.K.force_phase * R(y));
    collide<R, NOISE, FORCE>(f, B.K, (uint32_t)site, step, B.replica, Fx);
    stochastic_round<S>(f, (uint32_t)site, step, B.replica, B.K.rk0, B.K.rk1);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        int idx = site, slot = i;
        if (LAYOUT == kAAEven) slot = opposite(i);
        else if (LAYOUT == kAAOdd) idx = ypush(vel_y(i)) * nx + xpush(vel_x(i));
        S *p = B.dst + (int64_t)slot * B.plane + idx;
        if (FLB_GUARD_ST(B, p, 1)) *p = Storage<S>::store(f[i]);
    }
}

// Vectorised form: thread item k = blockIdx.x T + tid owns the V sites
// x0 = V (k mod gx) .. x0 + V - 1 of row y = k / gx (gx = nx / V, nx % V == 0,
// whole warps), so every plane is read and written with aligned V-wide
// accesses.  The +-1 x-shift comes by warp shuffle from the neighbouring lane
// (which owns the adjacent group whenever the group is not at a row end),
// else by one scalar access; all lanes reach every shuffle.
template <class S, int V>
__device__ __forceinline__ void load_vec2(const S *p, S (&out)[V])
{
    using T = typename RawVec2<sizeof(S) * V>::T;
    const T raw = __ldg(reinterpret_cast<const T *>(p));
    const S *e = reinterpret_cast<const S *>(&raw);
#pragma unroll
    for (int v = 0; v < V; ++v) out[v] = e[v];
}

template <class S, int V>
__device__ __forceinline__ void store_vec2(S *p, const S (&in)[V])
{
    using T = typename RawVec2<sizeof(S) * V>::T;
    T raw;
    S *e = reinterpret_cast<S *>(&raw);
#pragma unroll
    for (int v = 0; v < V; ++v) e[v] = in[v];
    *reinterpret_cast<T *>(p) = raw;
}

template <class S, int LAYOUT, bool NOISE, bool FORCE, int V>
__global__ void __launch_bounds__(256, sizeof(typename Storage<S>::R) == 4 ? (sizeof(S) == 2 ? 3 : 4) : 1)
k_stream_collide_vec(const BoxStep<S> B, const uint32_t *step_ptr, uint32_t step)
{
    using R = typename Storage<S>::R;
    const int nx = B.nx, ny = B.ny, gx = nx / V;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31;
    const int item = (int)blockIdx.x * (int)(blockDim.x * blockDim.y) + tid;
    const bool active = item < gx * ny;
    const int it = active ? item : gx * ny - 1;       // idle lanes work on the last group, store nothing
    const int x0 = V * (it % gx), y = it / gx;
    if (step_ptr) step += __ldg(step_ptr);
    const int yo[3] = {(y == 0 ? ny - 1 : y - 1) * nx, y * nx, (y == ny - 1 ? 0 : y + 1) * nx};   // rows y-1, y, y+1
    const bool shl = lane > 0 && x0 != 0;             // lane - 1 owns x0 - V .. x0 - 1
    const bool shr = lane < 31 && x0 + V != nx;       // lane + 1 owns x0 + V ..
    const int x_left = x0 == 0 ? nx - 1 : x0 - 1, x_right = x0 + V == nx ? 0 : x0 + V;
    const int x_lload = shl ? x0 : x_left, x_rload = shr ? x0 + V - 1 : x_right;
    S raw[Q][V];
    S edge[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = vel_x(i), cy = vel_y(i);
        int ro = yo[1], slot = i;
        if (LAYOUT != kAAEven) {
            ro = yo[1 - cy];                           // pull from r - c_i
            slot = LAYOUT == kAB ? i : opposite(i);
        }
        const S *base = B.src + (int64_t)slot * B.plane + ro;
        load_vec2<S, V>(FLB_GUARD_LD(B, base + x0, V), raw[i]);
        if (LAYOUT != kAAEven && cx > 0) edge[i] = load_ro(FLB_GUARD_LD(B, base + x_lload, 1));
        if (LAYOUT != kAAEven && cx < 0) edge[i] = load_ro(FLB_GUARD_LD(B, base + x_rload, 1));
    }
    R f[V][Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = vel_x(i);
        if (LAYOUT == kAAEven || cx == 0) {
#pragma unroll
            for (int v = 0; v < V; ++v) f[v][i] = Storage<S>::load(raw[i][v]);
        } else if (cx > 0) {
            const R via = __shfl_up_sync(0xffffffffu, Storage<S>::load(raw[i][V - 1]), 1);
            f[0][i] = shl ? via : Storage<S>::load(edge[i]);
#pragma unroll
            for (int v = 1; v < V; ++v) f[v][i] = Storage<S>::load(raw[i][v - 1]);
        } else {
            const R via = __shfl_down_sync(0xffffffffu, Storage<S>::load(raw[i][0]), 1);
#pragma unroll
            for (int v = 0; v < V - 1; ++v) f[v][i] = Storage<S>::load(raw[i][v + 1]);
            f[V - 1][i] = shr ? via : Storage<S>::load(edge[i]);
        }
    }
    R Fx = R(0);
    if (FORCE) Fx = B.K.force_amp * sin_pi(B.K.force_phase * R(y));
    const uint32_t site0 = (uint32_t)(yo[1] + x0);
#pragma unroll
    // 16-bit formats: two sites per collision in the paired FP32 instructions
    if constexpr (sizeof(R) == 4 && sizeof(S) == 2 && V % 2 == 0) {
#pragma unroll
        for (int v = 0; v < V; v += 2) {
            F2 p[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) p[i] = F2(f[v][i], f[v + 1][i]);
            collide<F2, NOISE, FORCE>(p, B.K, make_uint2(site0 + v, site0 + v + 1), step, B.replica, F2(Fx));
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                f[v][i] = p[i].v.x;
                f[v + 1][i] = p[i].v.y;
            }
        }
    } else {
#pragma unroll
        for (int v = 0; v < V; ++v) collide<R, NOISE, FORCE>(f[v], B.K, site0 + v, step, B.replica, Fx);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) stochastic_round<S>(f[v], site0 + v, step, B.replica, B.K.rk0, B.K.rk1);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = vel_x(i), cy = vel_y(i);
        if (LAYOUT != kAAOdd) {
            // AB: slot i at r; AA even: slot opposite(i) at r
            S *base = B.dst + (int64_t)(LAYOUT == kAB ? i : opposite(i)) * B.plane + yo[1];
            S out[V];
#pragma unroll
            for (int v = 0; v < V; ++v) out[v] = Storage<S>::store(f[v][i]);
            if (active && FLB_GUARD_ST(B, base + x0, V)) store_vec2<S, V>(base + x0, out);
            continue;
        }
        // AA odd: population i goes to slot i at r + c_i
        S *base = B.dst + (int64_t)i * B.plane + yo[1 + cy];
        S out[V];
        if (cx == 0) {
#pragma unroll
            for (int v = 0; v < V; ++v) out[v] = Storage<S>::store(f[v][i]);
            if (active && FLB_GUARD_ST(B, base + x0, V)) store_vec2<S, V>(base + x0, out);
        } else if (cx > 0) {   // site x goes to x + 1
            const R from_left = __shfl_up_sync(0xffffffffu, f[V - 1][i], 1);
            out[0] = Storage<S>::store(from_left);
#pragma unroll
            for (int v = 1; v < V; ++v) out[v] = Storage<S>::store(f[v - 1][i]);
            if (active && shl && FLB_GUARD_ST(B, base + x0, V)) store_vec2<S, V>(base + x0, out);
#pragma unroll
            for (int v = 1; v < V; ++v)
                if (active && !shl && FLB_GUARD_ST(B, base + x0 + v, 1)) base[x0 + v] = out[v];
            if (active && !shr && FLB_GUARD_ST(B, base + x_right, 1)) base[x_right] = Storage<S>::store(f[V - 1][i]);
        } else {               // site x goes to x - 1
            const R from_right = __shfl_down_sync(0xffffffffu, f[0][i], 1);
#pragma unroll
            for (int v = 0; v < V - 1; ++v) out[v] = Storage<S>::store(f[v + 1][i]);
            out[V - 1] = Storage<S>::store(from_right);
            if (active && shr && FLB_GUARD_ST(B, base + x0, V)) store_vec2<S, V>(base + x0, out);
#pragma unroll
            for (int v = 0; v < V - 1; ++v)
                if (active && !shr && FLB_GUARD_ST(B, base + x0 + v, 1)) base[x0 + v] = out[v];
            if (active && !shl && FLB_GUARD_ST(B, base + x_left, 1)) base[x_left] = Storage<S>::store(f[0][i]);
        }
    }
}

}  // namespace d2
}  // namespace flb
