// kernels.cuh -- the stream-collide kernels of the fluctuating D3Q19 library
// (single box and batched), templated on the storage format S; the kernels
// outside the time step are in diag_kernels.cuh.  The step_<format>_<layout>.cu
// files instantiate them; the host runtime calls the launch_* wrappers declared
// in internal.h.
#pragma once

#include "d3q19.cuh"
#include "internal.h"

namespace flb {

// --------------------------------------------------------------------------
// Stream-collide.
// One thread updates V x-consecutive sites of one row (y, z) of one box.
//   AB      pull n_i(r) from slot i at r - c_i of src, store n*_i(r) in slot i at r of dst.
//   AA even read slot i at r, store n*_i(r) in slot opposite(i) at r (in place).
//   AA odd  read slot opposite(i) at r - c_i, store n*_i(r) in slot i at r + c_i (in place).
// In the AA steps every thread writes exactly the locations it read, so the
// in-place update has no races whatever the launch shape.
// --------------------------------------------------------------------------
template <class S>
struct BoxStep {
    const S *src;
    S *dst;
    int nx, ny, nz;
    int warprow;               // batched launch: nx / V divides 32, rows tile the warps (see update_vec)
    int64_t plane;             // elements between population planes
    uint32_t replica;
    int gx, gy;                // blocks along x and y of this box (batched launch)
    int block0;                // first block of this box in a batched launch
    int z0, nzl;               // single-box launch: planes z0 .. z0 + nzl - 1 (grid.z = nzl)
    CollideConsts<typename Storage<S>::R> K;
    FLB_VIOL_FIELD
};

template <class S, int LAYOUT, int NOISE, bool FORCE, int V>
__device__ __forceinline__ void update_sites(const BoxStep<S> &B, int x0, int y, int z, uint32_t step)
{
    using R = typename Storage<S>::R;
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    // row offsets (in sites) of the nine (y', z') rows the stencil touches
    auto row = [&](int yy, int zz) { return (zz * ny + yy) * nx; };
    auto ysel = [&](int c) { return c > 0 ? ym : (c < 0 ? yp : y); };   // y - c
    auto zsel = [&](int c) { return c > 0 ? zm : (c < 0 ? zp : z); };   // z - c
    auto ysel_push = [&](int c) { return c > 0 ? yp : (c < 0 ? ym : y); };  // y + c
    auto zsel_push = [&](int c) { return c > 0 ? zp : (c < 0 ? zm : z); };
    R Fx = R(0);
    if (FORCE) Fx = B.K.force_amp * sin_pi(B.K.force_phase * R(z));
    const uint32_t site_row = (uint32_t)row(y, z);

#pragma unroll
    for (int v = 0; v < V; ++v) {
        const int x = x0 + v;
        if (x >= nx) break;
        const int xm = x == 0 ? nx - 1 : x - 1, xp = x == nx - 1 ? 0 : x + 1;
        auto xsel = [&](int c) { return c > 0 ? xm : (c < 0 ? xp : x); };
        auto xsel_push = [&](int c) { return c > 0 ? xp : (c < 0 ? xm : x); };
        R f[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            int idx, slot;
            if (LAYOUT == kAAEven) {
                idx = (int)site_row + x;
                slot = i;
            } else {
                idx = row(ysel(vel_y(i)), zsel(vel_z(i))) + xsel(vel_x(i));
                slot = LAYOUT == kAB ? i : opposite(i);
            }
            const S *p = B.src + (int64_t)slot * B.plane + idx;
            f[i] = Storage<S>::load(load_ro(FLB_GUARD_LD(B, p, 1)));
        }
        collide<R, NOISE, FORCE>(f, B.K, site_row + (uint32_t)x, step, B.replica, Fx);
        stochastic_round<S>(f, site_row + (uint32_t)x, step, B.replica, B.K.rk0, B.K.rk1);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            int idx, slot;
            if (LAYOUT == kAB) {
                idx = (int)site_row + x;
                slot = i;
            } else if (LAYOUT == kAAEven) {
                idx = (int)site_row + x;
                slot = opposite(i);
            } else {
                idx = row(ysel_push(vel_y(i)), zsel_push(vel_z(i))) + xsel_push(vel_x(i));
                slot = i;
            }
            S *p = B.dst + (int64_t)slot * B.plane + idx;
            if (FLB_GUARD_ST(B, p, 1)) *p = Storage<S>::store(f[i]);
        }
    }
}

// --------------------------------------------------------------------------
// Vectorised update: one thread owns V x-consecutive sites x0..x0+V-1 of row
// (y, z) (nx % V == 0, x0 % V == 0), so every population plane is read and
// written with one aligned V-wide access.  A shift of the source (pull) or
// destination (AA odd push) by c_x = +-1 is resolved with a warp shuffle of the
// neighbouring thread's edge element; only threads at a row end or a warp or
// block-row edge fall back to one scalar access for that element.  All 32
// lanes of a warp reach every shuffle (inactive lanes work on a clamped,
// in-bounds position and skip their stores).
// --------------------------------------------------------------------------
template <int BYTES>
struct RawVec;
template <>
struct RawVec<4> {
    using T = uint32_t;
};
template <>
struct RawVec<8> {
    using T = uint2;
};
template <>
struct RawVec<16> {
    using T = uint4;
};

template <class S, int V>
__device__ __forceinline__ void load_vec(const S *p, S (&out)[V])
{
    using T = typename RawVec<sizeof(S) * V>::T;
    const T raw = __ldg(reinterpret_cast<const T *>(p));
    const S *e = reinterpret_cast<const S *>(&raw);
#pragma unroll
    for (int v = 0; v < V; ++v) out[v] = e[v];
}

template <class S, int V>
__device__ __forceinline__ void store_vec(S *p, const S (&in)[V])
{
    using T = typename RawVec<sizeof(S) * V>::T;
    T raw;
    S *e = reinterpret_cast<S *>(&raw);
#pragma unroll
    for (int v = 0; v < V; ++v) e[v] = in[v];
    *reinterpret_cast<T *>(p) = raw;
}

// Stores guarded by a predicate without a branch, so that the edge lanes of
// a warp do not split it (hand-written PTX: one predicated st.global).
__device__ __forceinline__ void st_if(bool p, void *a, uint16_t v)
{
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %0, 0;\n @q st.global.b16 [%1], %2;\n}" ::"r"((int)p), "l"(a),
                 "h"(v)
                 : "memory");
}
__device__ __forceinline__ void st_if(bool p, void *a, uint32_t v)
{
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %0, 0;\n @q st.global.b32 [%1], %2;\n}" ::"r"((int)p), "l"(a),
                 "r"(v)
                 : "memory");
}
__device__ __forceinline__ void st_if(bool p, void *a, uint64_t v)
{
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %0, 0;\n @q st.global.b64 [%1], %2;\n}" ::"r"((int)p), "l"(a),
                 "l"(v)
                 : "memory");
}
__device__ __forceinline__ void st_if(bool p, void *a, uint2 v)
{
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %0, 0;\n @q st.global.v2.b32 [%1], {%2, %3};\n}" ::"r"((int)p),
                 "l"(a), "r"(v.x), "r"(v.y)
                 : "memory");
}
__device__ __forceinline__ void st_if(bool p, void *a, uint4 v)
{
    asm volatile("{\n .reg .pred q;\n setp.ne.b32 q, %0, 0;\n @q st.global.v4.b32 [%1], {%2, %3, %4, %5};\n}" ::"r"((int)p),
                 "l"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

template <int BYTES>
struct RawScalar;
template <>
struct RawScalar<2> {
    using T = uint16_t;
};
template <>
struct RawScalar<4> {
    using T = uint32_t;
};
template <>
struct RawScalar<8> {
    using T = uint64_t;
};

// One element if p.
template <class S>
__device__ __forceinline__ void store_one_if(bool p, S *a, S v)
{
    using T = typename RawScalar<sizeof(S)>::T;
    st_if(p, a, *reinterpret_cast<const T *>(&v));
}

// V elements (aligned) if p.
template <class S, int V>
__device__ __forceinline__ void store_vec_if(bool p, S *a, const S (&in)[V])
{
    using T = typename RawVec<sizeof(S) * V>::T;
    T raw;
    S *e = reinterpret_cast<S *>(&raw);
#pragma unroll
    for (int v = 0; v < V; ++v) e[v] = in[v];
    st_if(p, a, raw);
}

// V elements (aligned) if p, as an ordinary store: for the whole-vector stores
// the compiler can fold the address arithmetic into the store's addressing.
template <class S, int V>
__device__ __forceinline__ void store_vec_when(bool p, S *a, const S (&in)[V])
{
    if (p) store_vec<S, V>(a, in);
}

template <class R>
__device__ __forceinline__ R shfl_up1(R v)
{
    return __shfl_up_sync(0xffffffffu, v, 1);
}
template <class R>
__device__ __forceinline__ R shfl_down1(R v)
{
    return __shfl_down_sync(0xffffffffu, v, 1);
}

// Row-edge exchange of a block whose rows are covered by whole warps: slot
// [ty][i][w] of warp w in block row ty, for the load phase (l*) and the store
// phase (s*).  At most kXchRows block rows and kXchWarps warps per row.
constexpr int kXchRows = 2, kXchWarps = 8;
template <class R>
struct RowExchange {
    R l_last[kXchRows][Q][kXchWarps];    // last element of each warp's vector (pull from x - 1)
    R l_first[kXchRows][Q][kXchWarps];   // first element (pull from x + 1)
    R s_last[kXchRows][Q][kXchWarps];    // value pushed to x + 1 across the warp edge
    R s_first[kXchRows][Q][kXchWarps];   // value pushed to x - 1 across the warp edge
};

// FULLROW: every block row is exactly one box row (blockDim.x * V == nx, whole
// warps), so the neighbour of every edge element is in the block: shuffles
// inside a warp, the exchange above across warps (and around the periodic
// row end), and every lane reads and writes only whole aligned vectors.
// WARPROW: the converse -- a row is g = nx / V consecutive lanes and g divides
// 32, so rows tile the warps and the periodic neighbour of a row end is in the
// same warp: every neighbour element comes by an indexed shuffle (lane - 1,
// or lane + g - 1 at the row start; lane + 1, or lane - g + 1 at the row end),
// with no edge access and no shared memory.
// OFF32: every element offset of the box's buffer (Q planes) fits in 32 bits,
// so an address is one 32-bit offset (slot, row and x together) added to the
// buffer pointer, instead of 64-bit arithmetic per access.
template <class S, int LAYOUT, int NOISE, bool FORCE, int V, bool FULLROW = false, bool WARPROW = false,
          bool OFF32 = false>
__device__ __forceinline__ void update_vec(const BoxStep<S> &B, int x0, int y, int z, bool active, bool left_in_warp,
                                           bool right_in_warp, uint32_t step,
                                           RowExchange<typename Storage<S>::R> *xch = nullptr)
{
    static_assert(!(FULLROW && WARPROW), "one row-exchange variant at a time");
    using R = typename Storage<S>::R;
    // element (slot, row offset + x) of the source / destination buffer
    auto src_at = [&](int slot, int off) -> const S * {
        if constexpr (OFF32) return B.src + ((uint32_t)slot * (uint32_t)B.plane + (uint32_t)off);
        else return B.src + (int64_t)slot * B.plane + off;
    };
    auto dst_at = [&](int slot, int off) -> S * {
        if constexpr (OFF32) return B.dst + ((uint32_t)slot * (uint32_t)B.plane + (uint32_t)off);
        else return B.dst + (int64_t)slot * B.plane + off;
    };
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    // row offsets: yo[1 + d] = ((y + d) mod ny) nx, zo[1 + d] = ((z + d) mod nz) nx ny
    const int yo[3] = {(y == 0 ? ny - 1 : y - 1) * nx, y * nx, (y == ny - 1 ? 0 : y + 1) * nx};
    const int nxy = nx * ny;
    const int zo[3] = {(z == 0 ? nz - 1 : z - 1) * nxy, z * nxy, (z == nz - 1 ? 0 : z + 1) * nxy};
    // a neighbour's element comes by shuffle only inside the same row
    const bool shl = left_in_warp && x0 != 0;          // lane - 1 owns x0 - V .. x0 - 1
    const bool shr = right_in_warp && x0 + V != nx;    // lane + 1 owns x0 + V .. x0 + 2V - 1
    const int x_left = x0 == 0 ? nx - 1 : x0 - 1;      // element left of the group (periodic)
    const int x_right = x0 + V == nx ? 0 : x0 + V;     // element right of the group (periodic)
    // every lane reads its edge element with the vector (no wait behind the
    // shuffle, no divergence); lanes that get it by shuffle re-read a word of
    // their own vector instead
    const int x_lload = shl ? x0 : x_left;
    const int x_rload = shr ? x0 + V - 1 : x_right;

    // 1. issue every load of the 19 planes (vector + edge element) before
    //    any shuffle, so that all of them are in flight together
    S raw[Q][V];
    S edge[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = vel_x(i), cy = vel_y(i), cz = vel_z(i);
        int ro, slot;
        if (LAYOUT == kAAEven) {
            ro = zo[1] + yo[1];
            slot = i;
        } else {
            ro = zo[1 - cz] + yo[1 - cy];   // pull from r - c_i
            slot = LAYOUT == kAB ? i : opposite(i);
        }
        load_vec<S, V>(FLB_GUARD_LD(B, src_at(slot, ro + x0), V), raw[i]);
        if (!FULLROW && !WARPROW && LAYOUT != kAAEven && cx > 0) edge[i] = load_ro(FLB_GUARD_LD(B, src_at(slot, ro + x_lload), 1));
        if (!FULLROW && !WARPROW && LAYOUT != kAAEven && cx < 0) edge[i] = load_ro(FLB_GUARD_LD(B, src_at(slot, ro + x_rload), 1));
    }
    const int lane = (threadIdx.y * blockDim.x + threadIdx.x) & 31;
    // WARPROW source lanes of the left (x - 1) and right (x + 1) neighbour, periodic in the row
    const int gl = nx / V;
    const int lane_l = WARPROW ? (x0 != 0 ? lane - 1 : lane + gl - 1) : 0;
    const int lane_r = WARPROW ? (x0 + V != nx ? lane + 1 : lane - gl + 1) : 0;
    const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5, row_t = threadIdx.y;
    if (FULLROW && LAYOUT != kAAEven) {
        // publish each warp's edge elements, then read the neighbours' (periodic in the row)
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (vel_x(i) > 0 && lane == 31) xch->l_last[row_t][i][warp] = Storage<S>::load(raw[i][V - 1]);
            if (vel_x(i) < 0 && lane == 0) xch->l_first[row_t][i][warp] = Storage<S>::load(raw[i][0]);
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (vel_x(i) > 0) edge[i] = Storage<S>::store(xch->l_last[row_t][i][warp == 0 ? nwarp - 1 : warp - 1]);
            if (vel_x(i) < 0) edge[i] = Storage<S>::store(xch->l_first[row_t][i][warp == nwarp - 1 ? 0 : warp + 1]);
        }
    }
    // 2. shift the planes with c_x != 0 by one site
    const bool use_left = FULLROW ? lane != 0 : shl;
    const bool use_right = FULLROW ? lane != 31 : shr;
    R f[V][Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = vel_x(i);
        if (LAYOUT == kAAEven || cx == 0) {
#pragma unroll
            for (int v = 0; v < V; ++v) f[v][i] = Storage<S>::load(raw[i][v]);
        } else if (cx > 0) {   // pull from x - 1
            if constexpr (WARPROW) {
                f[0][i] = __shfl_sync(0xffffffffu, Storage<S>::load(raw[i][V - 1]), lane_l);
            } else {
                const R via = shfl_up1(Storage<S>::load(raw[i][V - 1]));
                f[0][i] = use_left ? via : Storage<S>::load(edge[i]);
            }
#pragma unroll
            for (int v = 1; v < V; ++v) f[v][i] = Storage<S>::load(raw[i][v - 1]);
        } else {               // pull from x + 1
#pragma unroll
            for (int v = 0; v < V - 1; ++v) f[v][i] = Storage<S>::load(raw[i][v + 1]);
            if constexpr (WARPROW) {
                f[V - 1][i] = __shfl_sync(0xffffffffu, Storage<S>::load(raw[i][0]), lane_r);
            } else {
                const R via = shfl_down1(Storage<S>::load(raw[i][0]));
                f[V - 1][i] = use_right ? via : Storage<S>::load(edge[i]);
            }
        }
    }

    R Fx = R(0);
    if (FORCE) Fx = B.K.force_amp * sin_pi(B.K.force_phase * R(z));
    const uint32_t site0 = (uint32_t)(zo[1] + yo[1]) + (uint32_t)x0;
    // 16-bit formats (issue-bound): two sites per collision in the paired FP32
    // instructions; FP32 storage is bound by HBM and keeps the one-site form,
    // whose odd AA step measured faster
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

    R pushed[Q];   // FULLROW, AA odd: the value crossing into this warp's vector from the neighbour warp
    if (FULLROW && LAYOUT == kAAOdd) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (vel_x(i) > 0 && lane == 31) xch->s_last[row_t][i][warp] = f[V - 1][i];
            if (vel_x(i) < 0 && lane == 0) xch->s_first[row_t][i][warp] = f[0][i];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            pushed[i] = R(0);
            if (vel_x(i) > 0) pushed[i] = xch->s_last[row_t][i][warp == 0 ? nwarp - 1 : warp - 1];
            if (vel_x(i) < 0) pushed[i] = xch->s_first[row_t][i][warp == nwarp - 1 ? 0 : warp + 1];
        }
    }
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int cx = vel_x(i), cy = vel_y(i), cz = vel_z(i);
        if (WARPROW && LAYOUT == kAAOdd && cx != 0) {
            // whole aligned vectors: the element crossing a lane edge comes from the neighbour lane
            S *base = B.dst + (int64_t)i * B.plane + zo[1 + cz] + yo[1 + cy];
            S out[V];
            if (cx > 0) {   // site x goes to x + 1
                out[0] = Storage<S>::store(__shfl_sync(0xffffffffu, f[V - 1][i], lane_l));
#pragma unroll
                for (int v = 1; v < V; ++v) out[v] = Storage<S>::store(f[v - 1][i]);
            } else {        // site x goes to x - 1
#pragma unroll
                for (int v = 0; v < V - 1; ++v) out[v] = Storage<S>::store(f[v + 1][i]);
                out[V - 1] = Storage<S>::store(__shfl_sync(0xffffffffu, f[0][i], lane_r));
            }
            store_vec_when<S, V>(active && FLB_GUARD_ST(B, base + x0, V), base + x0, out);
            continue;
        }
        if (FULLROW && LAYOUT == kAAOdd && cx != 0) {
            // whole aligned vectors only: the element that crosses the warp edge came through the exchange
            S out[V];
            if (cx > 0) {   // site x goes to x + 1
                const R from_left = shfl_up1(f[V - 1][i]);
                out[0] = Storage<S>::store(lane == 0 ? pushed[i] : from_left);
#pragma unroll
                for (int v = 1; v < V; ++v) out[v] = Storage<S>::store(f[v - 1][i]);
            } else {        // site x goes to x - 1
                const R from_right = shfl_down1(f[0][i]);
#pragma unroll
                for (int v = 0; v < V - 1; ++v) out[v] = Storage<S>::store(f[v + 1][i]);
                out[V - 1] = Storage<S>::store(lane == 31 ? pushed[i] : from_right);
            }
            S *p = dst_at(i, zo[1 + cz] + yo[1 + cy] + x0);
            store_vec_when<S, V>(active && FLB_GUARD_ST(B, p, V), p, out);
            continue;
        }
        if (LAYOUT != kAAOdd) {
            // AB: slot i at r;  AA even: slot opposite(i) at r
            S *p = dst_at(LAYOUT == kAB ? i : opposite(i), zo[1] + yo[1] + x0);
            S out[V];
#pragma unroll
            for (int v = 0; v < V; ++v) out[v] = Storage<S>::store(f[v][i]);
            store_vec_when<S, V>(active && FLB_GUARD_ST(B, p, V), p, out);
        } else {
            // AA odd: push population i to slot i at r + c_i
            S *base = B.dst + (int64_t)i * B.plane + zo[1 + cz] + yo[1 + cy];
            if (cx == 0) {
                S out[V];
#pragma unroll
                for (int v = 0; v < V; ++v) out[v] = Storage<S>::store(f[v][i]);
                store_vec_if<S, V>(active && FLB_GUARD_ST(B, base + x0, V), base + x0, out);
            } else if (cx > 0) {   // site x goes to x + 1
                const R from_left = shfl_up1(f[V - 1][i]);
                S out[V];
                out[0] = Storage<S>::store(from_left);
#pragma unroll
                for (int v = 1; v < V; ++v) out[v] = Storage<S>::store(f[v - 1][i]);
                store_vec_if<S, V>(active && shl && FLB_GUARD_ST(B, base + x0, V), base + x0, out);
                // without the left neighbour: elements x0+1 .. x0+V-1 one by one
#pragma unroll
                for (int v = 1; v < V; ++v) store_one_if<S>(active && !shl && FLB_GUARD_ST(B, base + x0 + v, 1), base + x0 + v, out[v]);
                store_one_if<S>(active && !shr && FLB_GUARD_ST(B, base + x_right, 1), base + x_right, Storage<S>::store(f[V - 1][i]));
            } else {               // site x goes to x - 1
                const R from_right = shfl_down1(f[0][i]);
                S out[V];
#pragma unroll
                for (int v = 0; v < V - 1; ++v) out[v] = Storage<S>::store(f[v + 1][i]);
                out[V - 1] = Storage<S>::store(from_right);
                store_vec_if<S, V>(active && shr && FLB_GUARD_ST(B, base + x0, V), base + x0, out);
#pragma unroll
                for (int v = 0; v < V - 1; ++v) store_one_if<S>(active && !shr && FLB_GUARD_ST(B, base + x0 + v, 1), base + x0 + v, out[v]);
                store_one_if<S>(active && !shl && FLB_GUARD_ST(B, base + x_left, 1), base + x_left, Storage<S>::store(f[0][i]));
            }
        }
    }
}

// Lane bookkeeping of a (bx, by) block for update_vec: the thread left
// (right) of (tx, ty) in the row is lane - 1 (+ 1) of the same warp unless tx
// or the lane sits on an edge.
struct LaneEdges {
    bool left, right;
};
__device__ __forceinline__ LaneEdges lane_edges()
{
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int lane = tid & 31;
    return LaneEdges{threadIdx.x > 0 && lane > 0, threadIdx.x + 1 < blockDim.x && lane < 31};
}

__device__ __forceinline__ uint32_t step_of(const uint32_t *step_ptr, uint32_t step)
{
    return step_ptr ? __ldg(step_ptr) + step : step;
}

// One box: grid (gx, gy, nz), block (bx, by); thread (tx, ty) updates the V
// sites x0 = V (blockIdx.x bx + tx) .. x0 + V - 1 of row (y, z).  V = 1 is the
// general scalar path; V > 1 needs nx % V == 0.  UROW (FULLROW with by = 1
// and a buffer of fewer than 2^32 elements): the block is one whole box row,
// y = blockIdx.y, so the row offsets of the nine neighbour rows are the same
// for the whole block, and every address is one 32-bit element offset.
template <class S, int LAYOUT, int NOISE, bool FORCE, int V, bool FULLROW, bool WARPROW, bool UROW>
__device__ __forceinline__ void stream_collide_box(const BoxStep<S> &B, const uint32_t *step_ptr, uint32_t step)
{
    static_assert(!UROW || FULLROW, "UROW is a FULLROW launch");
    int x0 = V * (blockIdx.x * blockDim.x + threadIdx.x);
    int y = UROW ? (int)blockIdx.y : (int)(blockIdx.y * blockDim.y + threadIdx.y);
    const int z = B.z0 + (int)blockIdx.z;
    if constexpr (V == 1) {
        if (x0 >= B.nx || y >= B.ny) return;
        update_sites<S, LAYOUT, NOISE, FORCE, 1>(B, x0, y, z, step_of(step_ptr, step));
    } else {
        const bool active = x0 < B.nx && y < B.ny;
        if (!active) {   // stay in the warp for the shuffles, on an in-bounds position
            x0 = min(x0, B.nx - V);
            y = min(y, B.ny - 1);
        }
        const LaneEdges e = lane_edges();
        if constexpr (FULLROW) {
            __shared__ RowExchange<typename Storage<S>::R> xch;
            update_vec<S, LAYOUT, NOISE, FORCE, V, true, false, UROW>(B, x0, y, z, active, e.left, e.right,
                                                                      step_of(step_ptr, step), &xch);
        } else if constexpr (WARPROW) {
            update_vec<S, LAYOUT, NOISE, FORCE, V, false, true>(B, x0, y, z, active, e.left, e.right,
                                                                step_of(step_ptr, step));
        } else {
            update_vec<S, LAYOUT, NOISE, FORCE, V>(B, x0, y, z, active, e.left, e.right, step_of(step_ptr, step));
        }
    }
}

template <class S, int LAYOUT, int NOISE, bool FORCE, int V, bool FULLROW = false, bool WARPROW = false,
          bool UROW = false>
__global__ void __launch_bounds__(256) k_stream_collide(const BoxStep<S> B, const uint32_t *step_ptr, uint32_t step)
{
    stream_collide_box<S, LAYOUT, NOISE, FORCE, V, FULLROW, WARPROW, UROW>(B, step_ptr, step);
}

// The one-row launch of the stochastically rounded format, held to four
// 128-thread blocks per SM (at most 128 registers): left free, its AA odd step
// took 130 registers, which left room for three blocks, and ran 15 % slower.
template <class S, int LAYOUT, int NOISE, bool FORCE, int V>
__global__ void __launch_bounds__(128, 4) k_stream_collide_row4(const BoxStep<S> B, const uint32_t *step_ptr,
                                                                uint32_t step)
{
    stream_collide_box<S, LAYOUT, NOISE, FORCE, V, true, false, true>(B, step_ptr, step);
}

// Many boxes in one 1-D grid: box b owns blocks [block0, block0 + ceil(gx ny nz / T)),
// T threads per block.  Inside a box the threads are packed densely: thread
// item k = (block - block0) T + tid owns the V sites of x-group k mod gx
// (gx = nx / V groups per row) of row k / gx, so a warp may span several
// short rows and no lane idles at a row end; the lanes at a row start or end
// exchange through edge loads instead of shuffles.  The box table is a kernel
// parameter (constant bank, at most ~31 KB); batches larger than one table
// are split into several launches.
template <class S>
constexpr int batch_chunk()
{
    constexpr int n = (int)(31000 / sizeof(BoxStep<S>));
    return n > 64 ? 64 : n;
}

template <class S>
struct BatchParams {
    int nboxes;
    int pad_;
    BoxStep<S> boxes[batch_chunk<S>()];
};

template <class S, int LAYOUT, int NOISE, bool FORCE, int V>
__global__ void __launch_bounds__(256) k_stream_collide_batch(const __grid_constant__ BatchParams<S> P,
                                                              const uint32_t *step_ptr, uint32_t step)
{
    // last box with block0 <= blockIdx.x (the same for the whole block)
    int lo = 0, hi = P.nboxes - 1;
    const int b = (int)blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.boxes[mid].block0 <= b) lo = mid;
        else hi = mid - 1;
    }
    const BoxStep<S> &sb = P.boxes[lo];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int total = sb.gx * sb.ny * sb.nz;                 // x-groups of the box
    const int item = (b - sb.block0) * (int)(blockDim.x * blockDim.y) + tid;
    const bool active = item < total;
    const int it = active ? item : total - 1;                // idle lanes work on the last group, store nothing
    const int xg = it % sb.gx, row = it / sb.gx;
    const int y = row % sb.ny, z = row / sb.ny;
    const int x0 = V * xg;
    if constexpr (V == 1) {
        if (!active) return;
        update_sites<S, LAYOUT, NOISE, FORCE, 1>(sb, x0, y, z, step_of(step_ptr, step));
    } else {
        // consecutive lanes own consecutive x-groups: lane - 1 holds x0 - V whenever x0 > 0
        const int lane = tid & 31;
        if (sb.warprow)
            update_vec<S, LAYOUT, NOISE, FORCE, V, false, true>(sb, x0, y, z, active, lane > 0, lane < 31,
                                                                step_of(step_ptr, step));
        else
            update_vec<S, LAYOUT, NOISE, FORCE, V>(sb, x0, y, z, active, lane > 0, lane < 31, step_of(step_ptr, step));
    }
}

__global__ void k_advance_step(uint32_t *step_ptr, uint32_t by);

}  // namespace flb
