// sq.cu -- the static structure factor S(q) = <|sum_r drho(r) e^{-i q.r}|^2> / N
// of Sec. V (the isothermal ideal gas of Eq. mpeos has S(q) = mu rho0 at every
// q != 0), accumulated into shells of |q| on the device.
//
// Input: the real density deviation drho(r) = rho(r) - rho0 of one box, written
// by the statistics pass (D3Q19) or the D2Q9 density kernel, in the transform
// type T: FP32 for the formats that collide in FP32, FP64 for the FP64 format.
// The transform runs in T; the shell sums are FP64.
//
// Three passes, each reading and writing the field once:
//   x   real rows -> half spectrum X[z][y][kx], kx = 0 .. nx/2 (row stride P):
//       two real rows are transformed as one complex row (a + i b) and
//       separated afterwards;
//   y   tiles of W consecutive kx columns of one z-plane: every row of the tile
//       is one contiguous W-element segment, so loads and stores coalesce; the
//       W lines along y are transformed in shared memory and written back;
//   z   the same tiles along z for one y; instead of being written back, each
//       |X(q)|^2 / N goes into its shell (weight 2 for the kx that stand for
//       the mirrored -q as well).
// FP32 transforms sum into 64-bit fixed point per sample (see to_fixed), so
// their shell sums are the same bits whatever the order of the additions.
// Each line transform is a mixed-radix Stockham FFT (self-sorting, ping-pong
// in shared memory) with radices 8, 4, 2, 3, 5, 7 done in registers and any
// larger prime factor p by a direct p-point sum; the twiddles
// exp(-2 pi i m / L) are computed once in FP64 and rounded to T.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>

#include "internal.h"

namespace flb {
namespace {

template <class T>
struct alignas(2 * sizeof(T)) Cx {
    T x, y;
};

template <class T>
__device__ __forceinline__ Cx<T> cadd(Cx<T> a, Cx<T> b)
{
    return Cx<T>{a.x + b.x, a.y + b.y};
}
template <class T>
__device__ __forceinline__ Cx<T> csub(Cx<T> a, Cx<T> b)
{
    return Cx<T>{a.x - b.x, a.y - b.y};
}
template <class T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b)
{
    return Cx<T>{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// n / d and n mod d for 0 <= n < 2^24 and d >= 1, by the FP32 reciprocal and
// one correction step (the estimate is off by at most one).
struct Div {
    int d;
    float inv;
    __device__ __forceinline__ explicit Div(int d_) : d(d_), inv(1.0f / (float)d_) {}
    __device__ __forceinline__ int quot(int n, int &rem) const
    {
        int q = __float2int_rz((float)n * inv);
        int r = n - q * d;
        if (r < 0) {
            --q;
            r += d;
        } else if (r >= d) {
            ++q;
            r -= d;
        }
        rem = r;
        return q;
    }
};

// 4-point DFT in place: X_q = sum_r v_r (-i)^(r q)
template <class T>
__device__ __forceinline__ void dft4(Cx<T> &v0, Cx<T> &v1, Cx<T> &v2, Cx<T> &v3)
{
    const Cx<T> t0 = cadd(v0, v2), t1 = csub(v0, v2);
    const Cx<T> t2 = cadd(v1, v3), d = csub(v1, v3);
    const Cx<T> t3 = Cx<T>{d.y, -d.x};   // (v1 - v3) (-i)
    v0 = cadd(t0, t2);
    v1 = cadd(t1, t3);
    v2 = csub(t0, t2);
    v3 = csub(t1, t3);
}

// Position of element n of a line in shared memory: one unused slot after
// every 32 elements, so that the strided accesses of the first Stockham
// stages spread over the banks (0.57 of the shared-memory wavefronts of an
// unpadded 512-point line), while three blocks of 512-point tiles with their
// shell sums still fit in an SM.  A line of L elements spans line_span(L) slots.
__device__ __forceinline__ int pidx(int n) { return n + (n >> 5); }
__host__ __device__ constexpr int line_span(int L) { return L + (L >> 5) + 1; }

// R-point DFT of v in registers: v[q] <- sum_r v[r] exp(-2 pi i r q / R); tw
// holds exp(-2 pi i m / L) for m < L (R divides L).
template <class T, int R>
__device__ __forceinline__ void dft_small(Cx<T> (&v)[R], const Cx<T> *tw, int L)
{
    if constexpr (R == 2) {
        const Cx<T> a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        dft4(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 8) {
        // two 4-point DFTs of the even and odd elements, combined with
        // exp(-2 pi i k / 8), k = 0..3
        Cx<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
        Cx<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
        dft4(e0, e1, e2, e3);
        dft4(o0, o1, o2, o3);
        const T h = T(0.70710678118654752440);
        const Cx<T> w1 = Cx<T>{h * (o1.x + o1.y), h * (o1.y - o1.x)};     // (1 - i)/sqrt 2
        const Cx<T> w2 = Cx<T>{o2.y, -o2.x};                              // -i
        const Cx<T> w3 = Cx<T>{h * (o3.y - o3.x), -h * (o3.x + o3.y)};    // -(1 + i)/sqrt 2
        v[0] = cadd(e0, o0);
        v[4] = csub(e0, o0);
        v[1] = cadd(e1, w1);
        v[5] = csub(e1, w1);
        v[2] = cadd(e2, w2);
        v[6] = csub(e2, w2);
        v[3] = cadd(e3, w3);
        v[7] = csub(e3, w3);
    } else {
        const int step = L / R;
        Cx<T> out[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            Cx<T> acc = v[0];
#pragma unroll
            for (int r = 1; r < R; ++r) acc = cadd(acc, cmul(v[r], tw[((r * q) % R) * step]));
            out[q] = acc;
        }
#pragma unroll
        for (int q = 0; q < R; ++q) v[q] = out[q];
    }
}

// One Stockham stage of radix R over nl lines of length L (line stride Ls in
// shared memory): with Ns the product of the radices already done, butterfly
// j takes the R elements j + r L/R, twiddles element r by exp(-2 pi i r k / (Ns
// R)), k = j mod Ns, and stores its R outputs at (j - k) R + k + q Ns.  A
// thread keeps one j (and its twiddles) for the whole stage and walks the
// lines, so the index arithmetic is done once per stage.
template <class T, int R>
__device__ __forceinline__ void butterfly(const Cx<T> *__restrict__ s, Cx<T> *__restrict__ d, const Cx<T> *tw,
                                          const Cx<T> (&twr)[R], int L, int M, int j, int o, int Ns)
{
    Cx<T> v[R];
    v[0] = s[pidx(j)];
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmul(s[pidx(j + r * M)], twr[r]);
    dft_small<T, R>(v, tw, L);
#pragma unroll
    for (int q = 0; q < R; ++q) d[pidx(o + q * Ns)] = v[q];
}

template <class T, int R>
__device__ __forceinline__ void stage(const Cx<T> *__restrict__ src, Cx<T> *__restrict__ dst, const Cx<T> *tw, int L,
                                      int Ls, int Ns, int nl)
{
    const int M = L / R;
    const int ts = L / (Ns * R);
    const int bd = blockDim.x, tid = threadIdx.x;
    // threads per line: M when M <= bd (lines in parallel), else bd (j in steps of bd)
    const int lpp = M <= bd ? bd / M : 1;
    const int jt = M <= bd ? tid % M : tid;
    const int l0 = M <= bd ? tid / M : 0;
    if (l0 >= lpp) return;
    for (int j = jt; j < M; j += (M <= bd ? M : bd)) {
        const int k = j % Ns;
        Cx<T> twr[R];
#pragma unroll
        for (int r = 1; r < R; ++r) twr[r] = tw[r * k * ts];
        const int o = (j - k) * R + k;
        for (int line = l0; line < nl; line += lpp)
            butterfly<T, R>(src + line * Ls, dst + line * Ls, tw, twr, L, M, j, o, Ns);
    }
}

// The same stage for a prime radix R > 7 (a direct R-point sum per output).
template <class T>
__device__ void stage_generic(const Cx<T> *__restrict__ src, Cx<T> *__restrict__ dst, const Cx<T> *tw, int L, int Ls,
                              int Ns, int nl, int R)
{
    const int M = L / R;
    const int ts = L / (Ns * R);
    const int step = L / R;
    const int total = nl * M;
    for (int w = threadIdx.x; w < total; w += blockDim.x) {
        const int line = w / M, j = w - line * M;
        const int k = j % Ns;
        const Cx<T> *s = src + line * Ls;
        Cx<T> *d = dst + line * Ls;
        const int o = (j - k) * R + k;
        for (int q = 0; q < R; ++q) {
            Cx<T> acc = s[pidx(j)];
            int m = 0;   // (r q) mod R
            for (int r = 1; r < R; ++r) {
                m += q;
                if (m >= R) m -= R;
                acc = cadd(acc, cmul(cmul(s[pidx(j + r * M)], tw[r * k * ts]), tw[m * step]));
            }
            d[pidx(o + q * Ns)] = acc;
        }
    }
}

// Stages s0 .. s1 - 1 of the transform of nl lines held in a (line stride
// Ls), Ns the product of the radices before s0; returns the buffer (a or b)
// that holds the result.  Each stage ends with a block barrier.
template <class T>
__device__ Cx<T> *fft_stages(Cx<T> *a, Cx<T> *b, const Cx<T> *tw, int L, int Ls, int nl, const SqRadices &rd, int s0,
                             int s1, int Ns)
{
    Cx<T> *src = a, *dst = b;
    for (int s = s0; s < s1; ++s) {
        const int R = rd.r[s];
        switch (R) {
        case 2: stage<T, 2>(src, dst, tw, L, Ls, Ns, nl); break;
        case 3: stage<T, 3>(src, dst, tw, L, Ls, Ns, nl); break;
        case 4: stage<T, 4>(src, dst, tw, L, Ls, Ns, nl); break;
        case 5: stage<T, 5>(src, dst, tw, L, Ls, Ns, nl); break;
        case 7: stage<T, 7>(src, dst, tw, L, Ls, Ns, nl); break;
        case 8: stage<T, 8>(src, dst, tw, L, Ls, Ns, nl); break;
        default: stage_generic<T>(src, dst, tw, L, Ls, Ns, nl, R); break;
        }
        __syncthreads();
        Cx<T> *t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

// The whole transform of nl lines held in a.
template <class T>
__device__ Cx<T> *fft_lines(Cx<T> *a, Cx<T> *b, const Cx<T> *tw, int L, int Ls, int nl, const SqRadices &rd)
{
    return fft_stages<T>(a, b, tw, L, Ls, nl, rd, 0, rd.n, 1);
}

__host__ __device__ constexpr bool pow2_radix(int r) { return r == 2 || r == 4 || r == 8; }

// The first Stockham stage (Ns = 1: no twiddles) read straight from a tile of
// global memory: butterfly j of column c takes rows j + r M (M = L / R) and
// writes d[c Ls + pidx(j R + q)].  Columns at or past Hx are zeros.
template <class T, int R>
__device__ __forceinline__ void stage_first_global(const Cx<T> *base, int64_t sline, int c0, int Hx, int lgW, int L,
                                                   int Ls, Cx<T> *d, const Cx<T> *tw)
{
    const int W = 1 << lgW, M = L / R;
    for (int w = threadIdx.x; w < W * M; w += blockDim.x) {
        const int c = w & (W - 1), j = w >> lgW;
        const bool in = c0 + c < Hx;
        Cx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in ? base[(int64_t)(j + r * M) * sline + c] : Cx<T>{T(0), T(0)};
        dft_small<T, R>(v, tw, L);
#pragma unroll
        for (int q = 0; q < R; ++q) d[c * Ls + pidx(j * R + q)] = v[q];
    }
}

// The last Stockham stage (Ns = L / R) written straight to the tile in global
// memory: butterfly j twiddles element r by exp(-2 pi i r j / L), and its
// outputs are the elements j + q M in natural order.
template <class T, int R>
__device__ __forceinline__ void stage_last_global(const Cx<T> *s, int L, int Ls, int lgW, Cx<T> *base, int64_t sline,
                                                  int c0, int Hx, const Cx<T> *tw)
{
    const int W = 1 << lgW, M = L / R;
    for (int w = threadIdx.x; w < W * M; w += blockDim.x) {
        const int c = w & (W - 1), j = w >> lgW;
        Cx<T> v[R];
        v[0] = s[c * Ls + pidx(j)];
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(s[c * Ls + pidx(j + r * M)], tw[r * j]);
        dft_small<T, R>(v, tw, L);
        if (c0 + c < Hx) {
#pragma unroll
            for (int q = 0; q < R; ++q) base[(int64_t)(j + q * M) * sline + c] = v[q];
        }
    }
}

template <class T>
__device__ __forceinline__ void first_global(int R, const Cx<T> *base, int64_t sline, int c0, int Hx, int lgW, int L,
                                             int Ls, Cx<T> *d, const Cx<T> *tw)
{
    switch (R) {
    case 2: stage_first_global<T, 2>(base, sline, c0, Hx, lgW, L, Ls, d, tw); break;
    case 4: stage_first_global<T, 4>(base, sline, c0, Hx, lgW, L, Ls, d, tw); break;
    default: stage_first_global<T, 8>(base, sline, c0, Hx, lgW, L, Ls, d, tw); break;
    }
}

template <class T>
__device__ __forceinline__ void last_global(int R, const Cx<T> *s, int L, int Ls, int lgW, Cx<T> *base, int64_t sline,
                                            int c0, int Hx, const Cx<T> *tw)
{
    switch (R) {
    case 2: stage_last_global<T, 2>(s, L, Ls, lgW, base, sline, c0, Hx, tw); break;
    case 4: stage_last_global<T, 4>(s, L, Ls, lgW, base, sline, c0, Hx, tw); break;
    default: stage_last_global<T, 8>(s, L, Ls, lgW, base, sline, c0, Hx, tw); break;
    }
}

// exp(-2 pi i m / L), m < L, for the three lengths (consecutive in tw).
template <class T>
__global__ void k_sq_twiddles(Cx<T> *__restrict__ tw, int nx, int ny, int nz)
{
    const int total = nx + ny + nz;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int L = i < nx ? nx : (i < nx + ny ? ny : nz);
        const int m = i < nx ? i : (i < nx + ny ? i - nx : i - nx - ny);
        double s, c;
        sincospi(-2.0 * (double)m / (double)L, &s, &c);
        tw[i] = Cx<T>{(T)c, (T)s};
    }
}

// Shell of the wave vector with integer components (kx, ky, kz):
// floor(nmax |f|), f_a = k_a / n_a with k_a taken in (-n_a/2, n_a/2].  An FP32
// estimate decides unless it lies within 4e-3 of an integer (its error is below
// 2.2e-3 for nmax <= 4096: reciprocal edges, three squares, an approximate
// reciprocal square root); there the FP64 formula ((fx^2 + fy^2) + fz^2,
// correctly rounded square root, times nmax) decides.
struct ShellGeom {
    int nx, ny, nz, nmax;
    float inx, iny, inz;
    __device__ __forceinline__ ShellGeom(int nx_, int ny_, int nz_, int nmax_)
        : nx(nx_), ny(ny_), nz(nz_), nmax(nmax_), inx(1.0f / (float)nx_), iny(1.0f / (float)ny_),
          inz(1.0f / (float)nz_)
    {
    }
    __device__ __forceinline__ static int sgn(int k, int n) { return k <= n / 2 ? k : k - n; }
    // FP32 estimate of |f|^2 (fy^2 + fz^2 first: it is shared along a row of kx)
    __device__ __forceinline__ float fyz2(int ky, int kz) const
    {
        const float fy = (float)sgn(ky, ny) * iny, fz = (float)sgn(kz, nz) * inz;
        return fy * fy + fz * fz;
    }
    __device__ __forceinline__ int shell(int kx, int ky, int kz, float yz2) const
    {
        const float fx = (float)sgn(kx, nx) * inx;
        const float v = fx * fx + yz2;
        const float t = v > 0.0f ? (float)nmax * (v * rsqrtf(v)) : 0.0f;
        if (fabsf(t - rintf(t)) > 4e-3f) return (int)floorf(t);
        const double dx = (double)sgn(kx, nx) / (double)nx, dy = (double)sgn(ky, ny) / (double)ny,
                     dz = (double)sgn(kz, nz) / (double)nz;
        const double w = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        return (int)floor(__dmul_rn((double)nmax, __dsqrt_rn(w)));
    }
};

// The half-spectrum column kx stands for kx and its mirror nx - kx, except kx
// = 0 and, for even nx, kx = nx / 2.
__device__ __forceinline__ int mirror_weight(int kx, int nx) { return (kx == 0 || 2 * kx == nx) ? 1 : 2; }

// The shell of every wave vector of the half spectrum, once per box, in the
// order the z pass visits them (the 512-point FP32 z pass: entry ((o ntiles +
// t) W + c) nz + kz; otherwise as follows): entry ((o ntiles + t) nz + e) W + c holds the
// shell of (kx = t W + c, ky = o, kz = e lmul mod nz), or kNoShell for q = 0
// and for the padding columns kx >= nx/2 + 1; and the wave vectors per shell
// (the mirrored columns counted twice).  The z pass gives thread position e
// the wave number kz = e lmul mod nz (lmul odd and prime to nz), so that the
// lanes of a warp, whose kz are lmul apart, fall in different shells and
// their shared-memory additions rarely collide.
constexpr uint16_t kNoShell = 0xFFFF;

__global__ void k_sq_shells(int nx, int ny, int nz, int nmax, int nshells, int lgW, int lmul, bool natural,
                            uint16_t *__restrict__ tab, unsigned long long *__restrict__ count)
{
    extern __shared__ unsigned long long scount[];
    const ShellGeom G(nx, ny, nz, nmax);
    for (int s = threadIdx.x; s < nshells; s += blockDim.x) scount[s] = 0ull;
    __syncthreads();
    const int W = 1 << lgW;
    const int Hx = nx / 2 + 1;
    const int ntiles = (Hx + W - 1) / W;
    const int64_t total = (int64_t)ntiles * W * ny * nz;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int c, kz;
        int64_t item;
        if (natural) {   // [item][c][kz]: the fused last stage of the 512-point z pass
            kz = (int)(e % nz);
            const int64_t r = e / nz;
            c = (int)(r & (W - 1));
            item = r >> lgW;
        } else {         // [item][position][c], kz = position lmul mod nz
            c = (int)(e & (W - 1));
            const int64_t r = e >> lgW;
            const int pos = (int)(r % nz);
            kz = (int)(((int64_t)pos * lmul) % nz);
            item = r / nz;
        }
        const int t = (int)(item % ntiles), ky = (int)(item / ntiles);
        const int kx = t * W + c;
        int s = kNoShell;
        if (kx < Hx && !(kx == 0 && ky == 0 && kz == 0)) {
            s = G.shell(kx, ky, kz, G.fyz2(ky, kz));
            if (s >= nshells) s = kNoShell;
        }
        tab[e] = (uint16_t)s;
        if (s != kNoShell) atomicAdd(&scount[s], (unsigned long long)mirror_weight(kx, nx));
    }
    __syncthreads();
    for (int s = threadIdx.x; s < nshells; s += blockDim.x)
        if (scount[s]) atomicAdd(&count[s], scount[s]);
}

// FP32 transforms add |X|^2 / N into 64-bit fixed-point shell sums: integer
// additions, so the sums do not depend on the order of the additions (and the
// FP64 pipe, slow on this part, stays out of the per-element path).  The unit
// 2^lu is fixed per sample from the largest |rho - rho0| of the field, m:
// every term is at most sum_r (rho - rho0)^2 <= N m^2 (Parseval), so with
// 2^(lu + 62) >= N m^2 no sum of a sample can overflow, and one unit is
// below 2^-62 N m^2 (a relative error of about 1e-9 of a shell sum).
__device__ __forceinline__ int sq_unit_log2(uint32_t maxbits, int64_t N)
{
    int cl2n = 0;
    while (((int64_t)1 << cl2n) < N) ++cl2n;
    const int em = (int)(maxbits >> 23) - 127;   // m < 2^(em + 1)
    return cl2n + 2 * (em + 1) - 62;
}

// floor(f / 2^lu) for finite f >= 0, from the bits of f
__device__ __forceinline__ unsigned long long to_fixed(float f, int lu)
{
    const uint32_t b = __float_as_uint(f);
    const int e = (int)(b >> 23);
    const uint64_t m = e ? (uint64_t)((b & 0x7FFFFFu) | 0x800000u) : (uint64_t)(b & 0x7FFFFFu);
    const int sh = (e ? e : 1) - 150 - lu;   // f = m 2^(e - 150)
    if (sh >= 0) return m << sh;             // sh <= 38 for every term bounded as above
    return sh > -64 ? m >> -sh : 0ull;
}

// The x pass's first Stockham stage (power-of-two radix R) read straight from
// the real rows: butterfly j of complex line p takes x = j + r M (M = nx / R)
// of rows row0 + 2p (real part) and row0 + 2p + 1 (imaginary part).
template <class T, int R>
__device__ __forceinline__ void x_first_global(const T *__restrict__ rho, int64_t row0, int64_t nrows, int nx,
                                               int npair, int Ls, Cx<T> *d, const Cx<T> *tw, uint32_t &mb)
{
    const int M = nx / R;
    const Div dM(M);
    for (int w = threadIdx.x; w < npair * M; w += blockDim.x) {
        int j;
        const int p = dM.quot(w, j);
        const int64_t ra = row0 + 2 * p, rb = ra + 1;
        Cx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int x = j + r * M;
            v[r] = Cx<T>{ra < nrows ? rho[ra * nx + x] : T(0), rb < nrows ? rho[rb * nx + x] : T(0)};
        }
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                mb = max(mb, max(__float_as_uint(v[r].x) & 0x7FFFFFFFu, __float_as_uint(v[r].y) & 0x7FFFFFFFu));
        }
        dft_small<T, R>(v, tw, nx);
#pragma unroll
        for (int q = 0; q < R; ++q) d[p * Ls + pidx(j * R + q)] = v[q];
    }
}

// x pass: rows row0 .. of the real field, two per complex line.
template <class T>
__global__ void __launch_bounds__(256, 3) k_sq_x(const T *__restrict__ rho, Cx<T> *__restrict__ X, int nx, int64_t nrows,
                                              int P, const Cx<T> *__restrict__ twg, SqRadices rd, int npair,
                                              uint32_t *__restrict__ maxbits)
{
    uint32_t mb = 0;   // FP32: bits of the largest |rho - rho0| seen by this thread
    extern __shared__ __align__(16) unsigned char sq_smem[];
    Cx<T> *tw = reinterpret_cast<Cx<T> *>(sq_smem);
    const int Ls = line_span(nx);
    Cx<T> *a = tw + nx;
    Cx<T> *b = a + npair * Ls;
    for (int m = threadIdx.x; m < nx; m += blockDim.x) tw[m] = twg[m];
    const int64_t row0 = (int64_t)blockIdx.x * 2 * npair;
    const bool fuse_first = rd.n >= 1 && pow2_radix(rd.r[0]);
    if (fuse_first) {
        // the first radix applied as the rows are read
        switch (rd.r[0]) {
        case 2: x_first_global<T, 2>(rho, row0, nrows, nx, npair, Ls, a, tw, mb); break;
        case 4: x_first_global<T, 4>(rho, row0, nrows, nx, npair, Ls, a, tw, mb); break;
        default: x_first_global<T, 8>(rho, row0, nrows, nx, npair, Ls, a, tw, mb); break;
        }
    } else if (nx % 2 == 0) {
        // the block's 2 npair rows are contiguous in rho: read them as one
        // span, two elements per load, eight loads in flight per thread
        const int half = nx / 2;
        const Div dh(half);
        const int64_t nel = (int64_t)nrows * nx;
        const int tot = 2 * npair * half;
        constexpr int kB = 8;
        for (int e0 = threadIdx.x; e0 < tot; e0 += kB * blockDim.x) {
            Cx<T> v[kB];
#pragma unroll
            for (int q = 0; q < kB; ++q) {
                const int e = e0 + q * blockDim.x;
                const int64_t g = row0 * nx + 2 * (int64_t)e;   // rows are contiguous: element 2 e of the span
                v[q] = (e < tot && g < nel) ? *reinterpret_cast<const Cx<T> *>(rho + g) : Cx<T>{T(0), T(0)};
            }
            if constexpr (sizeof(T) == 4) {
#pragma unroll
                for (int q = 0; q < kB; ++q)
                    mb = max(mb, max(__float_as_uint(v[q].x) & 0x7FFFFFFFu, __float_as_uint(v[q].y) & 0x7FFFFFFFu));
            }
#pragma unroll
            for (int q = 0; q < kB; ++q) {
                const int e = e0 + q * blockDim.x;
                if (e < tot) {
                    int xh;
                    const int r = dh.quot(e, xh);   // local row, element pair xh
                    // elements 2 xh and 2 xh + 1 are adjacent (no gap after an odd index)
                    T *dstp = reinterpret_cast<T *>(a + (r >> 1) * Ls + pidx(2 * xh)) + (r & 1);
                    dstp[0] = v[q].x;   // element 2 xh of row r: re (even row) or im (odd row)
                    dstp[2] = v[q].y;   // element 2 xh + 1
                }
            }
        }
    } else {
        const Div dn(nx);
        for (int e = threadIdx.x; e < npair * nx; e += blockDim.x) {
            int x;
            const int p = dn.quot(e, x);
            const int64_t ra = row0 + 2 * p, rb = ra + 1;
            const T re = ra < nrows ? rho[ra * nx + x] : T(0);
            const T im = rb < nrows ? rho[rb * nx + x] : T(0);
            if constexpr (sizeof(T) == 4)
                mb = max(mb, max(__float_as_uint(re) & 0x7FFFFFFFu, __float_as_uint(im) & 0x7FFFFFFFu));
            a[p * Ls + pidx(x)] = Cx<T>{re, im};
        }
    }
    if constexpr (sizeof(T) == 4) {
        // NaN bits order above every finite value and infinity
        mb = __reduce_max_sync(0xffffffffu, mb);
        if ((threadIdx.x & 31) == 0 && mb) atomicMax(maxbits, mb);
    }
    __syncthreads();
    const Cx<T> *Z = fft_stages<T>(a, b, tw, nx, Ls, npair, rd, fuse_first ? 1 : 0, rd.n, fuse_first ? rd.r[0] : 1);
    const int Hx = nx / 2 + 1;
    const Div dH(Hx);
    for (int e = threadIdx.x; e < npair * Hx; e += blockDim.x) {
        int k;
        const int p = dH.quot(e, k);
        const int64_t ra = row0 + 2 * p, rb = ra + 1;
        if (ra >= nrows) continue;
        const Cx<T> z = Z[p * Ls + pidx(k)];
        const Cx<T> zm = Z[p * Ls + pidx(k == 0 ? 0 : nx - k)];   // Z(-k)
        // row a: (Z(k) + conj Z(-k)) / 2;  row b: (Z(k) - conj Z(-k)) / (2 i)
        X[ra * P + k] = Cx<T>{T(0.5) * (z.x + zm.x), T(0.5) * (z.y - zm.y)};
        if (rb < nrows) X[rb * P + k] = Cx<T>{T(0.5) * (z.y + zm.y), T(-0.5) * (z.x - zm.x)};
    }
}

// z pass: the shells of the transformed tile F (W columns kx = c0 .. c0 + W
// - 1 of line stride Ls, ky = item / ntiles).  Element (kx, ky, kz = l): a
// thread takes one kz and the W columns in order; along kx the shell changes
// slowly, so a run of equal shells is summed in a register and added to the
// block's sum once.
// WC > 0: W = WC known at compile time (the 512-point kernel's 8 columns).
template <class T, int WC = 0>
__device__ __forceinline__ void accumulate_tile(const Cx<T> *F, int Ls, int L, int lgW, int c0, int64_t item,
                                                const SqShells &sh, const uint16_t *__restrict__ tab, T inv_n,
                                                int lmul, int lu, unsigned long long *fsum, double *dsum)
{
    const int W = WC > 0 ? WC : 1 << lgW;
    const T inv_n2 = T(2) * inv_n;   // a column that stands for -q too
    const uint16_t *trow = tab + item * (int64_t)L * W;
    const int lstep = (int)(((int64_t)blockDim.x * lmul) % L);
    int l = (int)(((int64_t)threadIdx.x * lmul) % L);   // kz of position e
    for (int e = threadIdx.x; e < L; e += blockDim.x, l = (l + lstep >= L ? l + lstep - L : l + lstep)) {
        uint16_t sv[16];
        if (W >= 8) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h * 8 < W) {
                    const uint4 u = *reinterpret_cast<const uint4 *>(trow + e * W + 8 * h);
                    const uint16_t *pu = reinterpret_cast<const uint16_t *>(&u);
#pragma unroll
                    for (int q = 0; q < 8; ++q) sv[8 * h + q] = pu[q];
                }
            }
        } else {
            for (int c = 0; c < W; ++c) sv[c] = trow[e * W + c];
        }
        int cur = -1;
        T run = T(0);   // at most W values, in column order: the same sum on every run
        // no branch on the data: every column is read (padding columns hold
        // zeros), and the addition of a finished run is a predicated atomic
#pragma unroll
        for (int c = 0; c < (WC > 0 ? WC : 16); ++c) {
            if (WC == 0 && c >= W) break;
            const int s = sv[c];
            const Cx<T> v = F[c * Ls + pidx(l)];
            const int kx = c0 + c;
            const T p = (v.x * v.x + v.y * v.y) * ((kx == 0 || 2 * kx == sh.nx) ? inv_n : inv_n2);
            const bool valid = s != kNoShell;
            const bool flush = valid && s != cur && cur >= 0;
            if constexpr (sizeof(T) == 4) {
                const unsigned long long add = to_fixed(run, lu);
                if (flush) atomicAdd(&fsum[cur], add);
            } else {
                if (flush) atomicAdd(&dsum[cur], run);
            }
            const bool start = valid && s != cur;
            run = start ? p : (valid ? run + p : run);
            cur = start ? s : cur;
        }
        if (cur >= 0) {
            if constexpr (sizeof(T) == 4) atomicAdd(&fsum[cur], to_fixed(run, lu));
            else atomicAdd(&dsum[cur], run);
        }
    }
}

// y pass (ACC = false: transform and write back) and z pass (ACC = true:
// transform and add into the shells).  Item (tile t, outer o) covers the
// columns kx = t W .. t W + W - 1 (< Hx) and the L elements at X[o souter + l
// sline + kx]; the y pass has o = z, the z pass o = y.
template <class T, bool ACC>
__global__ void __launch_bounds__(256, 3) k_sq_lines(Cx<T> *__restrict__ X, int L, int64_t sline, int64_t souter,
                                                  int nouter, int Hx, int lgW, const Cx<T> *__restrict__ twg,
                                                  SqRadices rd, SqShells sh, const uint16_t *__restrict__ tab, T inv_n,
                                                  int lmul)
{
    const int W = 1 << lgW;
    extern __shared__ __align__(16) unsigned char sq_smem[];
    Cx<T> *tw = reinterpret_cast<Cx<T> *>(sq_smem);
    const int Ls = line_span(L);
    Cx<T> *a = tw + L;
    Cx<T> *b = a + W * Ls;
    // ACC: the block's shell sums, FP64 (FP64 transform) or fixed point (FP32)
    double *dsum = reinterpret_cast<double *>(b + W * Ls);
    unsigned long long *fsum = reinterpret_cast<unsigned long long *>(dsum);
    for (int m = threadIdx.x; m < L; m += blockDim.x) tw[m] = twg[m];
    if constexpr (ACC) {
        for (int s = threadIdx.x; s < sh.nshells; s += blockDim.x) {
            if constexpr (sizeof(T) == 4) fsum[s] = 0ull;
            else dsum[s] = 0.0;
        }
    }
    int lu = 0;
    if constexpr (ACC && sizeof(T) == 4) lu = sq_unit_log2(*sh.maxbits, (int64_t)sh.nx * sh.ny * sh.nz);
    const int ntiles = (Hx + W - 1) / W;
    const int64_t items = (int64_t)ntiles * nouter;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int t = (int)(item % ntiles), o = (int)(item / ntiles);
        const int c0 = t * W;
        Cx<T> *base = X + o * souter + c0;
        __syncthreads();   // the previous item's readers of a and b are done
        // a power-of-two first radix is applied as the tile is read (the
        // loads of a butterfly are its registers); a power-of-two last radix
        // of the y pass writes straight back to global memory
        const bool fuse_first = rd.n >= 1 && pow2_radix(rd.r[0]);
        const bool fuse_last = !ACC && rd.n >= 2 && pow2_radix(rd.r[rd.n - 1]);
        if (fuse_first) {
            first_global<T>(rd.r[0], base, sline, c0, Hx, lgW, L, Ls, a, tw);
        } else {
            // eight loads in flight per thread, then the shared-memory stores
            constexpr int kB = 8;
            const int tot = W * L;
            for (int e0 = threadIdx.x; e0 < tot; e0 += kB * blockDim.x) {
                Cx<T> v[kB];
#pragma unroll
                for (int q = 0; q < kB; ++q) {
                    const int e = e0 + q * blockDim.x;
                    const int l = e >> lgW, c = e & (W - 1);
                    v[q] = (e < tot && c0 + c < Hx) ? base[l * sline + c] : Cx<T>{T(0), T(0)};
                }
#pragma unroll
                for (int q = 0; q < kB; ++q) {
                    const int e = e0 + q * blockDim.x;
                    if (e < tot) a[(e & (W - 1)) * Ls + pidx(e >> lgW)] = v[q];
                }
            }
        }
        __syncthreads();
        const int s0 = fuse_first ? 1 : 0, s1 = fuse_last ? rd.n - 1 : rd.n;
        const Cx<T> *F = fft_stages<T>(a, b, tw, L, Ls, W, rd, s0, s1, fuse_first ? rd.r[0] : 1);
        if constexpr (!ACC) {
            if (fuse_last) {
                last_global<T>(rd.r[rd.n - 1], F, L, Ls, lgW, base, sline, c0, Hx, tw);
            } else {
                for (int e = threadIdx.x; e < W * L; e += blockDim.x) {
                    const int l = e >> lgW, c = e & (W - 1);
                    if (c0 + c < Hx) base[l * sline + c] = F[c * Ls + pidx(l)];
                }
            }
        } else {
            accumulate_tile<T>(F, Ls, L, lgW, c0, item, sh, tab, inv_n, lmul, lu, fsum, dsum);
        }
    }
    if constexpr (ACC) {
        __syncthreads();
        for (int s = threadIdx.x; s < sh.nshells; s += blockDim.x) {
            if constexpr (sizeof(T) == 4) {
                if (fsum[s]) atomicAdd(&sh.fixed[s], fsum[s]);
            } else {
                if (dsum[s] != 0.0) atomicAdd(&sh.sum[s], dsum[s]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// 512-point lines, FP32: the same three radix-8 Stockham stages as above for
// eight lines per block of 256 threads (two butterflies per thread and stage),
// with the index arithmetic of the general stages turned into constants.  With
// M = 64 and one padding slot after every 32 elements, pidx(j + 64 r) =
// pidx(j) + 66 r; a stage's outputs o + q Ns sit at constant offsets from one
// base (Ns = 8: o = 64 m + k, pidx(o + 8 q) = o + 2 m + 8 q + q / 4; Ns = 64:
// o = j).  Every butterfly does the operations of the general path in the same
// order, so the results are the same bits.
// ---------------------------------------------------------------------------
constexpr int kL512 = 512;
constexpr int kLs512 = line_span(512);

// The twiddles of the two twiddled stages, laid out in the order the lanes of
// a warp read them (consecutive lanes, consecutive entries: no bank
// conflicts): t[(r - 1) 64 + j] = w^(r j) (Ns = 64), then t[448 + (r - 1) 8 +
// k] = w^(8 r k) (Ns = 8), w = exp(-2 pi i / 512); 504 entries, copied from
// the 512-entry table, so the values are the same.
constexpr int kTw8 = 448;
template <class T>
__device__ __forceinline__ void load_twiddles512(Cx<T> *t, const Cx<T> *__restrict__ twg)
{
    for (int m = threadIdx.x; m < kTw8 + 56; m += blockDim.x) {
        const int r = (m < kTw8 ? m >> 6 : (m - kTw8) >> 3) + 1;
        const int e = m < kTw8 ? r * (m & 63) : 8 * r * ((m - kTw8) & 7);
        t[m] = twg[e];
    }
}

// Stage Ns = NS (8 or 64) of the eight lines in s, into d.
template <class T, int NS>
__device__ __forceinline__ void stage512(const Cx<T> *__restrict__ s, Cx<T> *__restrict__ d, const Cx<T> *tw)
{
    static_assert(NS == 8 || NS == 64, "the twiddled stages");
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int w = (int)threadIdx.x + it * 256;
        const int c = w >> 6, j = w & 63;
        const int k = j & (NS - 1);
        const Cx<T> *sl = s + c * kLs512 + pidx(j);
        Cx<T> v[8];
        v[0] = sl[0];
#pragma unroll
        for (int r = 1; r < 8; ++r)
            v[r] = cmul(sl[66 * r], NS == 8 ? tw[kTw8 + (r - 1) * 8 + k] : tw[(r - 1) * 64 + j]);   // w^(r k 512/(8 NS))
        dft_small<T, 8>(v, tw, kL512);
        Cx<T> *dl = d + c * kLs512;
        if constexpr (NS == 8) {
            const int o = (j - k) * 8 + k;
            const int base = o + ((o >> 6) << 1);
#pragma unroll
            for (int q = 0; q < 8; ++q) dl[base + 8 * q + (q >> 2)] = v[q];
        } else {
            const int base = pidx(j);
#pragma unroll
            for (int q = 0; q < 8; ++q) dl[base + 66 * q] = v[q];
        }
    }
}

// The same stage in place: every thread reads (and twiddles) the inputs of
// its two butterflies, the block waits, then each writes its outputs over the
// lines, so one buffer serves all stages.  The caller waits again before the
// next stage reads.
template <class T, int NS>
__device__ __forceinline__ void stage512_inplace(Cx<T> *a, const Cx<T> *tw)
{
    static_assert(NS == 8 || NS == 64, "the twiddled stages");
    Cx<T> v[2][8];
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int w = (int)threadIdx.x + it * 256;
        const int c = w >> 6, j = w & 63;
        const int k = j & (NS - 1);
        const Cx<T> *sl = a + c * kLs512 + pidx(j);
        v[it][0] = sl[0];
#pragma unroll
        for (int r = 1; r < 8; ++r)
            v[it][r] = cmul(sl[66 * r], NS == 8 ? tw[kTw8 + (r - 1) * 8 + k] : tw[(r - 1) * 64 + j]);
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int w = (int)threadIdx.x + it * 256;
        const int c = w >> 6, j = w & 63;
        const int k = j & (NS - 1);
        dft_small<T, 8>(v[it], tw, kL512);
        Cx<T> *dl = a + c * kLs512;
        if constexpr (NS == 8) {
            const int o = (j - k) * 8 + k;
            const int base = o + ((o >> 6) << 1);
#pragma unroll
            for (int q = 0; q < 8; ++q) dl[base + 8 * q + (q >> 2)] = v[it][q];
        } else {
            const int base = pidx(j);
#pragma unroll
            for (int q = 0; q < 8; ++q) dl[base + 66 * q] = v[it][q];
        }
    }
}

// First stage (Ns = 1) read from a tile of 8 columns in global memory:
// butterfly j of column c takes rows j + 64 r; pidx(8 j + q) = 8 j + q + j / 4.
template <class T>
__device__ __forceinline__ void first512_global(const Cx<T> *base, int64_t sline, int c0, int Hx, Cx<T> *d,
                                                const Cx<T> *tw)
{
    const int64_t s64 = 64 * sline;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int w = (int)threadIdx.x + it * 256;
        const int c = w & 7, j = w >> 3;
        const bool in = c0 + c < Hx;
        const Cx<T> *p = base + (int64_t)j * sline + c;
        Cx<T> v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = in ? p[r * s64] : Cx<T>{T(0), T(0)};
        dft_small<T, 8>(v, tw, kL512);
        Cx<T> *dl = d + c * kLs512 + 8 * j + (j >> 2);
#pragma unroll
        for (int q = 0; q < 8; ++q) dl[q] = v[q];
    }
}

// Last stage (Ns = 64) written to the tile in global memory, natural order.
template <class T>
__device__ __forceinline__ void last512_global(const Cx<T> *s, Cx<T> *base, int64_t sline, int c0, int Hx,
                                               const Cx<T> *tw)
{
    const int64_t s64 = 64 * sline;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int w = (int)threadIdx.x + it * 256;
        const int c = w & 7, j = w >> 3;
        const Cx<T> *sl = s + c * kLs512 + pidx(j);
        Cx<T> v[8];
        v[0] = sl[0];
#pragma unroll
        for (int r = 1; r < 8; ++r) v[r] = cmul(sl[66 * r], tw[(r - 1) * 64 + j]);   // w^(r j)
        dft_small<T, 8>(v, tw, kL512);
        if (c0 + c < Hx) {
            Cx<T> *p = base + (int64_t)j * sline + c;
#pragma unroll
            for (int q = 0; q < 8; ++q) p[q * s64] = v[q];
        }
    }
}

// The z pass's last stage (Ns = 64) with the shell sums, FP32: butterfly (c,
// j) yields X(kx = c0 + c, ky, kz = j + 64 q), q = 0..7.  A warp's 32 lanes
// share c and hold 32 consecutive j, so for each q their kz are consecutive
// and on one side of the Nyquist plane: |q| and its shell are monotonic across
// the lanes and equal shells form runs of lanes.  A segmented sum over the
// lanes (five shuffle steps, in lane order) gives each run's total to its last
// lane, which adds it, in fixed point, to the block's sum.  The shell table is
// in natural order, [item][c][kz].
template <class T>
__device__ __forceinline__ void last512_shells(const Cx<T> *a, const Cx<T> *tw, int c0, int64_t item,
                                               const SqShells &sh, const uint16_t *__restrict__ tab, T inv_n, int lu,
                                               unsigned long long *fsum)
{
    const int lane = (int)threadIdx.x & 31;
    const T inv_n2 = T(2) * inv_n;   // a column that stands for -q too
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int w = (int)threadIdx.x + it * 256;
        const int c = w >> 6, j = w & 63;
        const Cx<T> *sl = a + c * kLs512 + pidx(j);
        Cx<T> v[8];
        v[0] = sl[0];
#pragma unroll
        for (int r = 1; r < 8; ++r) v[r] = cmul(sl[66 * r], tw[(r - 1) * 64 + j]);   // w^(r j)
        dft_small<T, 8>(v, tw, kL512);
        const int kx = c0 + c;
        const T wgt = (kx == 0 || 2 * kx == sh.nx) ? inv_n : inv_n2;
        const uint16_t *trow = tab + (item * 8 + c) * kL512 + j;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int s = trow[64 * q];
            T p = (v[q].x * v[q].x + v[q].y * v[q].y) * wgt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const T pu = __shfl_up_sync(0xffffffffu, p, d);
                const int su = __shfl_up_sync(0xffffffffu, s, d);
                if (lane >= d && su == s) p += pu;
            }
            const int sn = __shfl_down_sync(0xffffffffu, s, 1);
            const unsigned long long add = to_fixed(p, lu);
            if ((lane == 31 || sn != s) && s != kNoShell) atomicAdd(&fsum[s], add);
        }
    }
}

// x pass of a 512-wide box: sixteen real rows per block as eight complex lines.
template <class T>
__global__ void __launch_bounds__(256, 4) k_sq_x512(const T *__restrict__ rho, Cx<T> *__restrict__ X, int64_t nrows,
                                                 int P, const Cx<T> *__restrict__ twg, uint32_t *__restrict__ maxbits)
{
    constexpr int nx = kL512, npair = 8;
    uint32_t mb = 0;
    extern __shared__ __align__(16) unsigned char sq_smem[];
    Cx<T> *tw = reinterpret_cast<Cx<T> *>(sq_smem);
    Cx<T> *a = tw + nx;
    load_twiddles512<T>(tw, twg);
    const int64_t row0 = (int64_t)blockIdx.x * 2 * npair;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const int w = (int)threadIdx.x + it * 256;
        const int p = w >> 6, j = w & 63;
        const int64_t ra = row0 + 2 * p, rb = ra + 1;
        const T *pa = rho + ra * nx + j, *pb = pa + nx;
        Cx<T> v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = Cx<T>{ra < nrows ? pa[64 * r] : T(0), rb < nrows ? pb[64 * r] : T(0)};
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int r = 0; r < 8; ++r)
                mb = max(mb, max(__float_as_uint(v[r].x) & 0x7FFFFFFFu, __float_as_uint(v[r].y) & 0x7FFFFFFFu));
        }
        dft_small<T, 8>(v, tw, nx);
        Cx<T> *dl = a + p * kLs512 + 8 * j + (j >> 2);
#pragma unroll
        for (int q = 0; q < 8; ++q) dl[q] = v[q];
    }
    if constexpr (sizeof(T) == 4) {
        mb = __reduce_max_sync(0xffffffffu, mb);
        if ((threadIdx.x & 31) == 0 && mb) atomicMax(maxbits, mb);
    }
    __syncthreads();
    stage512_inplace<T, 8>(a, tw);
    __syncthreads();
    stage512_inplace<T, 64>(a, tw);
    __syncthreads();
    const Cx<T> *Z = a;
    constexpr int Hx = nx / 2 + 1;
    for (int e = threadIdx.x; e < npair * Hx; e += blockDim.x) {
        const int p = e / Hx, k = e - p * Hx;
        const int64_t ra = row0 + 2 * p, rb = ra + 1;
        if (ra >= nrows) continue;
        const Cx<T> z = Z[p * kLs512 + pidx(k)];
        const Cx<T> zm = Z[p * kLs512 + pidx(k == 0 ? 0 : nx - k)];   // Z(-k)
        X[ra * P + k] = Cx<T>{T(0.5) * (z.x + zm.x), T(0.5) * (z.y - zm.y)};
        if (rb < nrows) X[rb * P + k] = Cx<T>{T(0.5) * (z.y + zm.y), T(-0.5) * (z.x - zm.x)};
    }
}

// y pass (ACC = false) and z pass (ACC = true) of 512-point lines, tiles of 8
// columns: the general kernel's work with the stages above.
template <class T, bool ACC>
__global__ void __launch_bounds__(256, 4) k_sq_lines512(Cx<T> *__restrict__ X, int64_t sline, int64_t souter,
                                                     int nouter, int Hx, const Cx<T> *__restrict__ twg, SqShells sh,
                                                     const uint16_t *__restrict__ tab, T inv_n, int lmul)
{
    constexpr int L = kL512, W = 8;
    static_assert(!ACC || sizeof(T) == 4, "fixed-point shell sums: the FP32 transform");
    extern __shared__ __align__(16) unsigned char sq_smem[];
    Cx<T> *tw = reinterpret_cast<Cx<T> *>(sq_smem);
    Cx<T> *a = tw + L;
    double *dsum = reinterpret_cast<double *>(a + W * kLs512);
    unsigned long long *fsum = reinterpret_cast<unsigned long long *>(dsum);
    load_twiddles512<T>(tw, twg);
    if constexpr (ACC) {
        for (int s = threadIdx.x; s < sh.nshells; s += blockDim.x) {
            if constexpr (sizeof(T) == 4) fsum[s] = 0ull;
            else dsum[s] = 0.0;
        }
    }
    int lu = 0;
    if constexpr (ACC && sizeof(T) == 4) lu = sq_unit_log2(*sh.maxbits, (int64_t)sh.nx * sh.ny * sh.nz);
    const int ntiles = (Hx + W - 1) / W;
    const int64_t items = (int64_t)ntiles * nouter;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int t = (int)(item % ntiles), o = (int)(item / ntiles);
        const int c0 = t * W;
        Cx<T> *base = X + o * souter + c0;
        __syncthreads();   // the previous item's readers of a are done
        first512_global<T>(base, sline, c0, Hx, a, tw);
        __syncthreads();
        stage512_inplace<T, 8>(a, tw);
        __syncthreads();
        if constexpr (!ACC) {
            last512_global<T>(a, base, sline, c0, Hx, tw);
        } else {
            last512_shells<T>(a, tw, c0, item, sh, tab, inv_n, lu, fsum);
        }
    }
    if constexpr (ACC) {
        __syncthreads();
        for (int s = threadIdx.x; s < sh.nshells; s += blockDim.x) {
            if constexpr (sizeof(T) == 4) {
                if (fsum[s]) atomicAdd(&sh.fixed[s], fsum[s]);
            } else {
                if (dsum[s] != 0.0) atomicAdd(&sh.sum[s], dsum[s]);
            }
        }
    }
}

// FP32 transform, after the z pass: the sample's fixed-point shell sums times
// 2^lu into the FP64 sums, and the sample's scratch cleared for the next one.
// A non-finite field (max bits at or above those of infinity) gives NaN sums.
__global__ void k_sq_finish(SqShells sh)
{
    const uint32_t mb = *sh.maxbits;
    const int lu = sq_unit_log2(mb, (int64_t)sh.nx * sh.ny * sh.nz);
    const bool bad = mb >= 0x7F800000u;
    for (int s = threadIdx.x; s < sh.nshells; s += blockDim.x) {
        sh.sum[s] += bad ? __longlong_as_double(0x7FF8000000000000ll) : ldexp((double)sh.fixed[s], lu);
        sh.fixed[s] = 0ull;
    }
    __syncthreads();
    if (threadIdx.x == 0) *sh.maxbits = 0u;
}

// Radices of L: eights, then fours, then 2, 3, 5, 7 and the remaining primes
// in increasing order.
SqRadices radices_of(int L)
{
    SqRadices rd{};
    int n = L;
    auto push = [&](int r) { rd.r[rd.n++] = r; };
    while (n % 8 == 0) {
        push(8);
        n /= 8;
    }
    while (n % 4 == 0) {
        push(4);
        n /= 4;
    }
    for (int p : {2, 3, 5, 7})
        while (n % p == 0) {
            push(p);
            n /= p;
        }
    for (int p = 11; n > 1; p += 2)
        while (n % p == 0) {
            push(p);
            n /= p;
        }
    return rd;
}

// An odd multiplier near 17 that is prime to L (so e -> e m mod L permutes
// 0 .. L-1): lanes 17 apart in kz, and 17 * 8 bytes apart in shared memory,
// which spreads a warp's loads over the banks.
int kz_multiplier(int L)
{
    for (int m = 17;; m += 2) {
        int a = m, b = L;
        while (b) {
            const int t = a % b;
            a = b;
            b = t;
        }
        if (a == 1) return L == 1 ? 1 : m % L;
    }
}

int log2_of(int w)
{
    int l = 0;
    while ((1 << (l + 1)) <= w) ++l;
    return l;
}

constexpr int kSqThreads = 256;
constexpr size_t kSqLineBudget = 72 * 1024;   // shared memory for the lines of one block

template <class T>
int lines_per_block(int L, int cap)
{
    const size_t per = 2 * (size_t)line_span(L) * sizeof(Cx<T>);
    int w = (int)std::max<size_t>(1, kSqLineBudget / per);
    w = std::min(w, cap);
    int p = 1;
    while (2 * p <= w) p *= 2;
    return p;
}

// columns per tile: up to 128 bytes of a row
template <class T>
constexpr int tile_cap()
{
    return (int)(128 / sizeof(Cx<T>));
}

template <class T>
size_t lines_smem(int L, int W, int nshells, bool acc)
{
    size_t s = (size_t)L * sizeof(Cx<T>) + 2 * (size_t)W * line_span(L) * sizeof(Cx<T>);
    if (acc) s += (size_t)nshells * sizeof(double);   // FP64 or 64-bit fixed-point sums
    return s;
}

// The 512-point kernels: the twiddles, one buffer of eight lines, the shell sums.
template <class T>
size_t smem512(int nshells)
{
    return (size_t)kL512 * sizeof(Cx<T>) + 8 * (size_t)kLs512 * sizeof(Cx<T>) + (size_t)nshells * sizeof(double);
}

template <class T>
size_t x_smem(int nx, int npair)
{
    return (size_t)nx * sizeof(Cx<T>) + 2 * (size_t)npair * line_span(nx) * sizeof(Cx<T>);
}

int max_smem()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
        cudaGetLastError();
        return 48 * 1024;
    }
    return v;
}

template <class T>
bool fits(int nx, int ny, int nz, int nshells)
{
    const size_t lim = (size_t)max_smem();
    const int npair = lines_per_block<T>(nx, 16);
    return x_smem<T>(nx, npair) <= lim &&
           lines_smem<T>(ny, lines_per_block<T>(ny, tile_cap<T>()), 0, false) <= lim &&
           lines_smem<T>(nz, lines_per_block<T>(nz, tile_cap<T>()), nshells, true) <= lim;
}

template <class T, class K>
cudaError_t set_smem(K kernel, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <class T>
cudaError_t run(const SqPlan &p, cudaStream_t st)
{
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int Hx = nx / 2 + 1;
    const Cx<T> *tw = static_cast<const Cx<T> *>(p.tw);
    Cx<T> *X = static_cast<Cx<T> *>(p.X);
    const SqShells sh{p.shell_sum, p.shell_fixed, p.maxbits, p.nshells, nx, ny, nz, p.nmax};
    const T inv_n = T(1.0 / ((double)nx * ny * nz));
    // x pass
    {
        const int npair = lines_per_block<T>(nx, 16);
        const size_t smem = x_smem<T>(nx, npair);
        const int64_t nrows = (int64_t)ny * nz;
        const int64_t grid = (nrows + 2 * npair - 1) / (2 * npair);
        cudaError_t e;
        bool fixed512 = false;
        if constexpr (sizeof(T) == 4) {
            if (nx == kL512 && npair == 8) {
                const size_t smem1 = smem512<T>(0);
                if ((e = set_smem<T>(k_sq_x512<T>, smem1)) != cudaSuccess) return e;
                k_sq_x512<T><<<(unsigned)grid, kSqThreads, smem1, st>>>(static_cast<const T *>(p.rho), X, nrows, p.P,
                                                                          tw, p.maxbits);
                fixed512 = true;
            }
        }
        if (!fixed512) {
            if ((e = set_smem<T>(k_sq_x<T>, smem)) != cudaSuccess) return e;
            k_sq_x<T><<<(unsigned)grid, kSqThreads, smem, st>>>(static_cast<const T *>(p.rho), X, nx, nrows, p.P, tw,
                                                                  radices_of(nx), npair, p.maxbits);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // y pass
    if (ny > 1) {
        const int W = lines_per_block<T>(ny, tile_cap<T>());
        const size_t smem = lines_smem<T>(ny, W, 0, false);
        const int64_t items = (int64_t)((Hx + W - 1) / W) * nz;
        const unsigned grid = (unsigned)std::min<int64_t>(items, 1 << 30);
        cudaError_t e;
        bool fixed512 = false;
        if constexpr (sizeof(T) == 4) {
            if (ny == kL512 && W == 8) {
                const size_t smem1 = smem512<T>(0);
                if ((e = set_smem<T>(k_sq_lines512<T, false>, smem1)) != cudaSuccess) return e;
                k_sq_lines512<T, false><<<grid, kSqThreads, smem1, st>>>(X, (int64_t)p.P, (int64_t)p.P * ny, nz, Hx,
                                                                        tw + nx, sh, nullptr, inv_n, 1);
                fixed512 = true;
            }
        }
        if (!fixed512) {
            if ((e = set_smem<T>(k_sq_lines<T, false>, smem)) != cudaSuccess) return e;
            k_sq_lines<T, false><<<grid, kSqThreads, smem, st>>>(X, ny, (int64_t)p.P, (int64_t)p.P * ny, nz, Hx,
                                                                log2_of(W), tw + nx, radices_of(ny), sh, nullptr,
                                                                inv_n, 1);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    // z pass with the shell sums: a grid of at most the resident blocks, each
    // looping over items, so that each block adds its shells to global memory once
    {
        const int W = lines_per_block<T>(nz, tile_cap<T>());
        const size_t smem = lines_smem<T>(nz, W, p.nshells, true);
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t items = (int64_t)((Hx + W - 1) / W) * ny;
        // at most the resident blocks, each looping over items
        auto grid_of = [&](auto kernel, size_t bytes) -> int64_t {
            int per_sm = 1;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kSqThreads, bytes);
            return std::max<int64_t>(1, std::min<int64_t>(items, (int64_t)std::max(per_sm, 1) * sms));
        };
        cudaError_t e;
        bool fixed512 = false;
        if constexpr (sizeof(T) == 4) {
            if (nz == kL512 && W == 8) {
                const size_t smem1 = smem512<T>(p.nshells);
                if ((e = set_smem<T>(k_sq_lines512<T, true>, smem1)) != cudaSuccess) return e;
                k_sq_lines512<T, true><<<(unsigned)grid_of(k_sq_lines512<T, true>, smem1), kSqThreads, smem1, st>>>(
                    X, (int64_t)p.P * ny, (int64_t)p.P, ny, Hx, tw + nx + ny, sh, p.shell_tab, inv_n,
                    kz_multiplier(nz));
                fixed512 = true;
            }
        }
        if (!fixed512) {
            if ((e = set_smem<T>(k_sq_lines<T, true>, smem)) != cudaSuccess) return e;
            k_sq_lines<T, true><<<(unsigned)grid_of(k_sq_lines<T, true>, smem), kSqThreads, smem, st>>>(
                X, nz, (int64_t)p.P * ny, (int64_t)p.P, ny, Hx, log2_of(W), tw + nx + ny, radices_of(nz), sh,
                p.shell_tab, inv_n, kz_multiplier(nz));
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if constexpr (sizeof(T) == 4) {
        k_sq_finish<<<1, 256, 0, st>>>(sh);
        return cudaGetLastError();
    }
    return cudaSuccess;
}

}  // namespace

int sq_shells(int nx, int ny, int nz)
{
    const int nmax = std::max(nx, std::max(ny, nz));
    return (int)std::ceil(std::sqrt(3.0) * nmax / 2.0) + 2;
}

int sq_row_stride(int nx, bool dbl)
{
    const int Hx = nx / 2 + 1;
    const int a = dbl ? tile_cap<double>() : tile_cap<float>();
    return (Hx + a - 1) / a * a;
}

size_t sq_elem_bytes(bool dbl) { return dbl ? sizeof(double) : sizeof(float); }

bool sq_supported(int nx, int ny, int nz, bool dbl)
{
    const int nshells = sq_shells(nx, ny, nz);
    return dbl ? fits<double>(nx, ny, nz, nshells) : fits<float>(nx, ny, nz, nshells);
}

namespace {
// the z pass's tile width, which fixes the table layout
int z_tile(int nz, bool dbl)
{
    return dbl ? lines_per_block<double>(nz, tile_cap<double>()) : lines_per_block<float>(nz, tile_cap<float>());
}
// the z pass takes the fused 512-point kernel (natural table order)
bool z_fixed512(int nz, bool dbl) { return !dbl && nz == kL512 && z_tile(nz, dbl) == 8; }
}  // namespace

int64_t sq_table_elems(int nx, int ny, int nz, bool dbl)
{
    const int W = z_tile(nz, dbl);
    const int Hx = nx / 2 + 1;
    return (int64_t)((Hx + W - 1) / W) * W * ny * nz;
}

cudaError_t sq_init(const SqPlan &p, unsigned long long *count, cudaStream_t st)
{
    const int total = p.nx + p.ny + p.nz;
    const int g = std::max(1, std::min(1024, (total + 255) / 256));
    if (p.dbl) k_sq_twiddles<double><<<g, 256, 0, st>>>(static_cast<Cx<double> *>(p.tw), p.nx, p.ny, p.nz);
    else k_sq_twiddles<float><<<g, 256, 0, st>>>(static_cast<Cx<float> *>(p.tw), p.nx, p.ny, p.nz);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(count, 0, (size_t)p.nshells * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(p.shell_fixed, 0, (size_t)p.nshells * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(p.maxbits, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const int64_t n = sq_table_elems(p.nx, p.ny, p.nz, p.dbl);
    const int64_t cg = std::max<int64_t>(1, std::min<int64_t>(2048, (n + 255) / 256));
    const size_t smem = (size_t)p.nshells * sizeof(unsigned long long);
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(k_sq_shells, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_sq_shells<<<(unsigned)cg, 256, smem, st>>>(p.nx, p.ny, p.nz, p.nmax, p.nshells, log2_of(z_tile(p.nz, p.dbl)),
                                                  kz_multiplier(p.nz), z_fixed512(p.nz, p.dbl), p.shell_tab, count);
    return cudaGetLastError();
}

cudaError_t launch_sq(const SqPlan &p, cudaStream_t st) { return p.dbl ? run<double>(p, st) : run<float>(p, st); }

}  // namespace flb
