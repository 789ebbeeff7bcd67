// dct.cu -- the 2D discrete cosine transform of real images on the radix-2
// passes: the DCT-II forward and its inverse, the DCT-III (further down).
// Section 5 names the DCT among the transforms the method extends to,
// without giving an algorithm.  This file uses the well-known
// reduction of a length-N DCT-II to one length-N complex DFT (Makhoul, IEEE
// Trans. ASSP 1980), on the same scramble + butterfly engine as the FFT:
//
//  * reorder: v[i] = x[2i] for i < N/2, v[N-1-i] = x[2i+1] -- the even
//    samples ascending, then the odd ones descending;
//  * V = DFT_N(v) (forward, W_N = e^{-2 pi i / N}: the radix-2 DIT stages);
//  * X[k] = Re(e^{-i pi k / (2N)} V[k]).
//
// Two real lines a, b share one complex line z = v_a + i v_b ("two for one"):
// with Z = DFT(z) and k' = (N - k) mod N,
//   X_a[k] = (c (Zr[k] + Zr[k']) + s (Zi[k] - Zi[k'])) / 2
//   X_b[k] = (c (Zi[k] + Zi[k']) + s (Zr[k'] - Zr[k])) / 2,
//   (c, s) = (cos, sin)(pi k / (2N)),
// and the outputs at k' use (c, s) swapped.  So a real image costs half the
// butterflies of a complex one, and each pass moves 4 bytes per pixel in
// and 4 out.  The row pass pairs rows 2j and 2j+1; the column pass pairs
// columns 2q and 2q+1, which are adjacent floats: the real image read as a
// complex image of half the width.  The reorder is fused into the first
// (scrambled) read, the pairing and rotation into the last write.
//
// Definition computed (unnormalised, the oracle's):
//   X[k][l] = sum_m sum_n x[m][n] cos(pi k (2m+1) / (2R)) cos(pi l (2n+1) / (2C)).
//
// Kernels, forward / inverse:
//  * line_dct_kernel / line_idct_kernel: any line length, row or column
//    pass; the pairing of outputs (k, N-k) goes through shared memory;
//  * row_dct_kernel / row_idct_kernel: rows of 2^10 .. 2^14 points, 32
//    values per thread, loads, pairing and stores in registers;
//  * col_dct_tma_kernel / col_idct_tma_kernel: persistent TMA-fed column
//    passes for columns of 2^11 points;
//  * col_dct_tma64_kernel / col_idct_tma64_kernel: columns of 2^12 points on
//    the 6-stage engine of the complex column pass;
//  * col_dct_pack_l2_kernel (col_group.cuh): forward columns of 2^13 and
//    2^14 points on a cluster of 2 or 4 CTAs, two real columns per complex
//    line; col_idct_pair_kernel and col_idct_l2_kernel: the inverse.
#include <cmath>

#include "col_group.cuh"
#include "line_fft.cuh"
#include "passes.h"

namespace fft2d {

namespace {

// Where position i of the reordered line reads the real line from.
__device__ __forceinline__ int dct_src(int i, int N)
{
    return i < N / 2 ? 2 * i : 2 * (N - 1 - i) + 1;
}

struct DctIO {
    const float *in;
    float *out;
    long long rows, cols;   // real image shape, row-major, pitch = cols
};

// Complex value at reordered position i of complex line (line0 + lb) (row
// pass: real rows 2(line0+lb) and 2(line0+lb)+1) or complex column
// (line0 + w) (column pass: real columns 2(line0+w), 2(line0+w)+1).
template <class C, bool ROW>
__device__ __forceinline__ float2 dct_load(const DctIO &d, long long line0, int lb, int i, int w)
{
    const int s = dct_src(i, C::N);
    if constexpr (ROW) {
        const long long ra = 2 * (line0 + lb);
        return make_float2(__ldg(d.in + ra * d.cols + s), __ldg(d.in + (ra + 1) * d.cols + s));
    } else {
        const float2 *p = reinterpret_cast<const float2 *>(d.in);
        return __ldg(p + (long long)s * (d.cols / 2) + line0 + w);
    }
}

// dct_pair (col_group.cuh): the outputs at k and k' = (N - k) mod N of
// the two real lines of a complex line, from Z[k] and Z[k'].

template <class C, bool ROW>
__device__ __forceinline__ void dct_store(const DctIO &d, long long line0, int lb, int w, int k,
                                          float2 x)
{
    if constexpr (ROW) {
        const long long ra = 2 * (line0 + lb);
        d.out[ra * d.cols + k] = x.x;
        d.out[(ra + 1) * d.cols + k] = x.y;
    } else {
        reinterpret_cast<float2 *>(d.out)[(long long)k * (d.cols / 2) + line0 + w] = x;
    }
}

// One CTA: LB complex lines (row pass) or W complex columns (column pass)
// of N = 2^L points.  nlines = complex lines of the pass (rows/2 or cols/2);
// tw = the axis's per-stage rotation factors, post = (cos, sin)(pi k/(2N)),
// k = 0..N/2.
template <class C, bool ROW>
__global__ void __launch_bounds__(C::T, C::MINB) line_dct_kernel(const DctIO d,
                                                                 const float2 *__restrict__ tw,
                                                                 const float2 *__restrict__ post,
                                                                 long long nlines, float scale)
{
    extern __shared__ float2 sm[];
    using G0 = Grp<C, 0>;
    const int tid = threadIdx.x;
    const long long line0 = (long long)blockIdx.x * (ROW ? C::LB : C::W);
    const long long nvalid = nlines - line0;
    float2 a[C::EPT];

    // group 0: reordered, scrambled read (unit (r, h) sits at position
    // p = r | h << G, which holds v[rev(p)]), first stages
#pragma unroll
    for (int v = 0; v < G0::V; v++) {
        const int u = tid + v * C::T;
        const int w = u & (C::W - 1);
        const int u2 = u >> C::KW;
        const int hib = u2 & ((1 << G0::HB) - 1);
        const int lb = u2 >> G0::HB;
        const bool ok = ROW ? lb < nvalid : w < nvalid;
#pragma unroll
        for (int r = 0; r < G0::R; r++) {
            const int i = (brev_c(r, G0::G) << G0::HB) | hib;
            a[v * G0::R + r] = ok ? dct_load<C, ROW>(d, line0, lb, i, w) : make_float2(0.f, 0.f);
        }
    }
#pragma unroll
    for (int v = 0; v < G0::V; v++)
        run_stages<C, 0, false>(a, v, 0, tw, C::L);

    if constexpr (C::NG == 1) {
        // the whole line is one unit: Z[r] = a[v R + r] in natural order
#pragma unroll
        for (int v = 0; v < G0::V; v++) {
            const int u = tid + v * C::T;
            const int w = u & (C::W - 1);
            const int lb = (u >> C::KW) >> G0::HB;
            if (ROW ? lb >= nvalid : w >= nvalid)
                continue;
#pragma unroll
            for (int k = 0; k <= C::N / 2; k++) {
                const int kp = (C::N - k) & (C::N - 1);
                float2 xk, xp;
                dct_pair(a[v * G0::R + k], a[v * G0::R + kp], __ldg(post + k), scale, xk, xp);
                dct_store<C, ROW>(d, line0, lb, w, k, xk);
                if (kp != k)
                    dct_store<C, ROW>(d, line0, lb, w, kp, xp);
            }
        }
    } else {
        // exchange into the swizzled layout, the middle groups
#pragma unroll
        for (int v = 0; v < G0::V; v++) {
            const int u = tid + v * C::T;
            const int w = u & (C::W - 1);
            const int u2 = u >> C::KW;
            const int hib = u2 & ((1 << G0::HB) - 1);
            const int lb = u2 >> G0::HB;
            const int hi = brev_rt(hib, G0::HB);
#pragma unroll
            for (int r = 0; r < G0::R; r++)
                sm[sidx<C>(lb, r | (hi << G0::G), w)] = a[v * G0::R + r];
        }
        __syncthreads();
        if constexpr (C::NG >= 3) {
            group_smem<C, 1, false>(a, sm, tw, C::L);
            __syncthreads();
        }
        if constexpr (C::NG >= 4) {
            group_smem<C, 2, false>(a, sm, tw, C::L);
            __syncthreads();
        }
        // last group, then the spectrum in natural order in shared memory
        using Gl = Grp<C, C::NG - 1>;
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
            const int u = tid + v * C::T;
            const int w = u & (C::W - 1);
            const int u2 = u >> C::KW;
            const int lo = u2 & ((1 << Gl::S0) - 1);
            const int lb = u2 >> Gl::S0;
#pragma unroll
            for (int r = 0; r < Gl::R; r++)
                a[v * Gl::R + r] = sm[sidx<C>(lb, lo | (r << Gl::S0), w)];
        }
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
            const int u = tid + v * C::T;
            const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
            run_stages<C, C::NG - 1, false>(a, v, lo, tw, C::L);
        }
        __syncthreads();   // every swizzled slot has been read
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
            const int u = tid + v * C::T;
            const int w = u & (C::W - 1);
            const int u2 = u >> C::KW;
            const int lo = u2 & ((1 << Gl::S0) - 1);
            const int lb = u2 >> Gl::S0;
#pragma unroll
            for (int r = 0; r < Gl::R; r++)
                sm[((((lb << C::L) | lo | (r << Gl::S0))) << C::KW) | w] = a[v * Gl::R + r];
        }
        __syncthreads();
        // pairs (k, N - k): item q -> line block / column and k in [0, N/2);
        // k = 0 also finishes k = N/2 (both pair with themselves)
        constexpr int HALF = C::N / 2;
#pragma unroll
        for (int t = 0; t < C::EPT / 2; t++) {
            const int q = tid + t * C::T;
            const int w = ROW ? 0 : q & (C::W - 1);
            const int rest = ROW ? q : q >> C::KW;
            const int lb = ROW ? rest / HALF : 0;
            const int k = rest % HALF;
            if (ROW ? lb >= nvalid : w >= nvalid)
                continue;
            const float2 *line = sm + ((long long)lb << (C::L + C::KW)) + w;
            float2 xk, xp;
            if (k == 0) {
                dct_pair(line[0], line[0], __ldg(post), scale, xk, xp);
                dct_store<C, ROW>(d, line0, lb, w, 0, xk);
                const float2 zh = line[HALF << C::KW];
                dct_pair(zh, zh, __ldg(post + HALF), scale, xk, xp);
                dct_store<C, ROW>(d, line0, lb, w, HALF, xk);
            } else {
                dct_pair(line[k << C::KW], line[(C::N - k) << C::KW], __ldg(post + k), scale, xk,
                         xp);
                dct_store<C, ROW>(d, line0, lb, w, k, xk);
                dct_store<C, ROW>(d, line0, lb, w, C::N - k, xp);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Inverse (DCT-III, the oracle's x[n] = (1/N)(X[0] + 2 sum_k X[k]
// cos(pi k (2n+1) / (2N)))) through one inverse DFT:
//   V[k] = exp(i pi k / (2N)) (X[k] - i X[N-k])   (X[N] = 0),
//   v = IDFT(V),  x[2n] = v[n],  x[2n+1] = v[N-1-n].
// Two real lines a, b share the complex line z = X_a + i X_b; since the
// IDFT is linear, Z[k] = V_a[k] + i V_b[k] gives v_a + i v_b:
//   Z[k]   = (c + i s) ((X_a[k] + X_b[N-k]) + i (X_b[k] - X_a[N-k])),
//   Z[N-k] = (s + i c) ((X_a[N-k] + X_b[k]) + i (X_b[N-k] - X_a[k])),
// (c, s) = (cos, sin)(pi k / (2N)); Z[0] = z[0].
__device__ __forceinline__ void idct_pre(float2 za, float2 zb, float2 cs, float2 &yk, float2 &yp)
{
    const float ux = za.x + zb.y, uy = za.y - zb.x;
    const float vx = zb.x + za.y, vy = zb.y - za.x;
    yk = make_float2(cs.x * ux - cs.y * uy, cs.y * ux + cs.x * uy);
    yp = make_float2(cs.y * vx - cs.x * vy, cs.x * vx + cs.y * vy);
}

// The un-reordering store of v[n] and v[N-1-n] (n < N/2) of complex line lb
// (rows: real rows 2(line0+lb), +1; columns: complex column line0 + w).
template <bool ROW>
__device__ __forceinline__ void idct_store(const DctIO &d, long long line0, int lb, int w, int n,
                                           float2 zn, float2 zm, float scale)
{
    if constexpr (ROW) {
        const long long ra = 2 * (line0 + lb);
        reinterpret_cast<float2 *>(d.out + ra * d.cols)[n] = make_float2(zn.x * scale, zm.x * scale);
        reinterpret_cast<float2 *>(d.out + (ra + 1) * d.cols)[n] =
            make_float2(zn.y * scale, zm.y * scale);
    } else {
        float2 *o = reinterpret_cast<float2 *>(d.out) + line0 + w;
        o[(long long)(2 * n) * (d.cols / 2)] = make_float2(zn.x * scale, zn.y * scale);
        o[(long long)(2 * n + 1) * (d.cols / 2)] = make_float2(zm.x * scale, zm.y * scale);
    }
}

// The inverse pass for any line length: the spectrum lines land in shared
// memory in natural order, are pre-rotated in place (pairs k, N-k), run
// through the radix-2 stages from there (conjugate rotation factors), come
// back in natural order and leave un-reordered.
template <class C, bool ROW>
__global__ void __launch_bounds__(C::T, C::MINB) line_idct_kernel(const DctIO d,
                                                                  const float2 *__restrict__ tw,
                                                                  const float2 *__restrict__ post,
                                                                  long long nlines, float scale)
{
    extern __shared__ float2 sm[];
    constexpr int HALF = C::N / 2;
    const int tid = threadIdx.x;
    const long long line0 = (long long)blockIdx.x * (ROW ? C::LB : C::W);
    const long long nvalid = nlines - line0;
    for (int e = tid; e < C::E; e += C::T) {
        const int w = e & (C::W - 1);
        const int k = (e >> C::KW) & (C::N - 1);
        const int lb = e >> (C::L + C::KW);
        float2 z = make_float2(0.f, 0.f);
        if (ROW ? lb < nvalid : w < nvalid) {
            if constexpr (ROW) {
                const long long ra = 2 * (line0 + lb);
                z = make_float2(__ldg(d.in + ra * d.cols + k), __ldg(d.in + (ra + 1) * d.cols + k));
            } else {
                z = __ldg(reinterpret_cast<const float2 *>(d.in) + (long long)k * (d.cols / 2) +
                          line0 + w);
            }
        }
        sm[e] = z;
    }
    __syncthreads();
    // pre-rotation: item q -> line block / column and k in [0, N/2); k = 0
    // also handles k = N/2
#pragma unroll
    for (int t = 0; t < C::EPT / 2; t++) {
        const int q = tid + t * C::T;
        const int w = ROW ? 0 : q & (C::W - 1);
        const int rest = ROW ? q : q >> C::KW;
        const int lb = ROW ? rest / HALF : 0;
        const int k = rest % HALF;
        float2 *line = sm + ((long long)lb << (C::L + C::KW)) + w;
        float2 yk, yp;
        if (k == 0) {
            const float2 zh = line[HALF << C::KW];
            idct_pre(zh, zh, __ldg(post + HALF), yk, yp);
            line[HALF << C::KW] = yk;
        } else {
            idct_pre(line[k << C::KW], line[(C::N - k) << C::KW], __ldg(post + k), yk, yp);
            line[k << C::KW] = yk;
            line[(C::N - k) << C::KW] = yp;
        }
    }
    __syncthreads();
    float2 a[C::EPT];
    if constexpr (C::NG == 1) {
        using G0 = Grp<C, 0>;
#pragma unroll
        for (int v = 0; v < G0::V; v++) {
            const int u = tid + v * C::T;
            const int w = u & (C::W - 1);
            const int lb = u >> C::KW;
#pragma unroll
            for (int r = 0; r < G0::R; r++)
                a[v * G0::R + r] = sm[(((lb << C::L) | brev_c(r, G0::G)) << C::KW) | w];
            run_stages<C, 0, false>(a, v, 0, tw, C::L);
            if (ROW ? lb >= nvalid : w >= nvalid)
                continue;
#pragma unroll
            for (int n = 0; n < HALF; n++)
                idct_store<ROW>(d, line0, lb, w, n, a[v * G0::R + n], a[v * G0::R + C::N - 1 - n],
                                scale);
        }
    } else {
        group_first_smem<C, false>(a, sm, tw, C::L);
        __syncthreads();
        if constexpr (C::NG >= 3) {
            group_smem<C, 1, false>(a, sm, tw, C::L);
            __syncthreads();
        }
        if constexpr (C::NG >= 4) {
            group_smem<C, 2, false>(a, sm, tw, C::L);
            __syncthreads();
        }
        using Gl = Grp<C, C::NG - 1>;
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
            const int u = tid + v * C::T;
            const int w = u & (C::W - 1);
            const int u2 = u >> C::KW;
            const int lo = u2 & ((1 << Gl::S0) - 1);
            const int lb = u2 >> Gl::S0;
#pragma unroll
            for (int r = 0; r < Gl::R; r++)
                a[v * Gl::R + r] = sm[sidx<C>(lb, lo | (r << Gl::S0), w)];
        }
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
            const int u = tid + v * C::T;
            const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
            run_stages<C, C::NG - 1, false>(a, v, lo, tw, C::L);
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
            const int u = tid + v * C::T;
            const int w = u & (C::W - 1);
            const int u2 = u >> C::KW;
            const int lo = u2 & ((1 << Gl::S0) - 1);
            const int lb = u2 >> Gl::S0;
#pragma unroll
            for (int r = 0; r < Gl::R; r++)
                sm[((((lb << C::L) | lo | (r << Gl::S0))) << C::KW) | w] = a[v * Gl::R + r];
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < C::EPT / 2; t++) {
            const int q = tid + t * C::T;
            const int w = ROW ? 0 : q & (C::W - 1);
            const int rest = ROW ? q : q >> C::KW;
            const int lb = ROW ? rest / HALF : 0;
            const int n = rest % HALF;
            if (ROW ? lb >= nvalid : w >= nvalid)
                continue;
            const float2 *line = sm + ((long long)lb << (C::L + C::KW)) + w;
            idct_store<ROW>(d, line0, lb, w, n, line[n << C::KW], line[(C::N - 1 - n) << C::KW],
                            scale);
        }
    }
}

template <class C, bool ROW>
cudaError_t idct_launch(const DctIO &d, const float2 *tw, const float2 *post, long long nlines,
                        float scale, cudaStream_t s)
{
    auto k = line_idct_kernel<C, ROW>;
    constexpr int bytes = C::E * 8;
    if (bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess)
            return e;
    }
    const long long per = ROW ? C::LB : C::W;
    const unsigned grid = (unsigned)((nlines + per - 1) / per);
    k<<<grid, C::T, bytes, s>>>(d, tw, post, nlines, scale);
    return cudaGetLastError();
}

// The last stage group of a line: unit lo (0 <= lo < M = 2^S0) holds rows
// lo + M r, r < R.  Output k pairs with N - k, i.e. row lo + M r of unit lo
// with row (M - lo) + M (R-1-r) of unit M - lo (unit 0 pairs with itself,
// r with R - r).  The M units of a line are dealt out V to a thread so that
// every pair stays inside one thread: with Q = 2M/V, thread j (0 <= j < M/V)
// takes, for t < V/2, the offsets t Q + j (register unit 2t) and t Q + Q - j
// (unit 2t+1) -- unit 2t pairs with unit 2(V/2-1-t)+1 -- and thread 0 the
// offsets t Q and t Q + Q/2, which pair among themselves.
template <class C>
__device__ __forceinline__ int dct_unit_lo(int v, int j)
{
    using Gl = Grp<C, C::NG - 1>;
    constexpr int Q = 2 * (1 << Gl::S0) / Gl::V;
    const int t = v >> 1;
    if (j != 0)
        return t * Q + ((v & 1) ? Q - j : j);
    return t * Q + ((v & 1) ? Q / 2 : 0);
}

// Whether unit v of every thread holds rows with offset below M/2.
template <class C>
__host__ __device__ constexpr bool dct_unit_low(int v)
{
    using Gl = Grp<C, C::NG - 1>;
    return Gl::V == 2 ? v == 0 : (v >> 1) < Gl::V / 4;
}

// The rotations (cos, sin)(pi q / 32), q < 16, passed by value to the
// paired kernels (they sit in the constant bank).  Row lo + M r of a line of
// N = M R points needs (cos, sin)(pi (lo + M r) / (2N)), the table entry of
// lo rotated by pi r / (2R) = pi q / 32 with q = r 16 / R: one complex
// product instead of a table load per output pair.  Both factors are FP32
// roundings of FP64 values, so the product is within a few units in the last
// place of the exact rotation.
struct DctRot {
    float2 r[16];
};

__device__ __forceinline__ float2 rot_mul(float2 b, float2 t)
{
    return make_float2(b.x * t.x - b.y * t.y, b.y * t.x + b.x * t.y);
}

// Rows p of za and N - p of zb, cs = (cos, sin)(pi p / (2N)): the outputs at
// both, from the one below N/2 (cos and sin swap between p and N - p).
__device__ __forceinline__ void dct_pair_rows(float2 &za, float2 &zb, float2 cs, bool a_low,
                                              float scale)
{
    float2 xk, xp;
    if (a_low) {
        dct_pair(za, zb, cs, scale, xk, xp);
        za = xk;
        zb = xp;
    } else {
        dct_pair(zb, za, make_float2(cs.y, cs.x), scale, xk, xp);
        zb = xk;
        za = xp;
    }
}

// Units UA and UB (UA may equal UB) whose rows r and R-1-r pair, UA at an
// offset whose rotation is `base`; rows r < RMAX of UA.
template <class C, int UA, int UB, int RMAX>
__device__ __forceinline__ void dct_pair_units(float2 (&a)[C::EPT], float2 base,
                                               const DctRot &rot, float scale)
{
    using Gl = Grp<C, C::NG - 1>;
    constexpr int R = Gl::R;
#pragma unroll
    for (int r = 0; r < RMAX; r++)
        dct_pair_rows(a[UA * R + r], a[UB * R + R - 1 - r], rot_mul(base, rot.r[r * (16 / R)]),
                      r < R / 2, scale);
}

// Unit U of offset 0: rows M r, pairs (r, R - r); rows 0 and N/2 pair with
// themselves.
template <class C, int U>
__device__ __forceinline__ void dct_pair_unit0(float2 (&a)[C::EPT], const DctRot &rot,
                                               float scale)
{
    using Gl = Grp<C, C::NG - 1>;
    constexpr int R = Gl::R;
    float2 xk, xp;
    dct_pair(a[U * R], a[U * R], make_float2(1.f, 0.f), scale, xk, xp);
    a[U * R] = xk;
    dct_pair(a[U * R + R / 2], a[U * R + R / 2], rot.r[8], scale, xk, xp);
    a[U * R + R / 2] = xk;
#pragma unroll
    for (int r = 1; r < R / 2; r++) {
        dct_pair(a[U * R + r], a[U * R + R - r], rot.r[r * (16 / R)], scale, xk, xp);
        a[U * R + r] = xk;
        a[U * R + R - r] = xp;
    }
}

template <class C, int T0>
__device__ __forceinline__ void dct_pairs_j_side0(float2 (&a)[C::EPT], int j,
                                                  const float2 *__restrict__ post,
                                                  const DctRot &rot, float scale)
{
    using Gl = Grp<C, C::NG - 1>;
    constexpr int V = Gl::V, Q = 2 * (1 << Gl::S0) / V, R = Gl::R;
    if constexpr (T0 < V / 2) {
        dct_pair_units<C, 2 * T0, 2 * (V / 2 - 1 - T0) + 1, R>(a, __ldg(post + T0 * Q + j), rot,
                                                               scale);
        dct_pairs_j_side0<C, T0 + 1>(a, j, post, rot, scale);
    }
}

// Thread 0's units: side 0 (offsets t Q) pair t <-> V/2 - t, side 1
// (offsets t Q + Q/2) pair t <-> V/2 - 1 - t.
template <class C, int T0>
__device__ __forceinline__ void dct_pairs_0(float2 (&a)[C::EPT], const float2 *__restrict__ post,
                                            const DctRot &rot, float scale)
{
    using Gl = Grp<C, C::NG - 1>;
    constexpr int V = Gl::V, Q = 2 * (1 << Gl::S0) / V, R = Gl::R;
    if constexpr (T0 < V / 2) {
        constexpr int P0 = V / 2 - T0, P1 = V / 2 - 1 - T0;
        if constexpr (T0 == 0)
            dct_pair_unit0<C, 0>(a, rot, scale);
        else if constexpr (T0 < P0)
            dct_pair_units<C, 2 * T0, 2 * P0, R>(a, __ldg(post + T0 * Q), rot, scale);
        else if constexpr (T0 == P0)
            dct_pair_units<C, 2 * T0, 2 * T0, R / 2>(a, __ldg(post + T0 * Q), rot, scale);
        if constexpr (T0 < P1)
            dct_pair_units<C, 2 * T0 + 1, 2 * P1 + 1, R>(a, __ldg(post + T0 * Q + Q / 2), rot,
                                                         scale);
        else if constexpr (T0 == P1)
            dct_pair_units<C, 2 * T0 + 1, 2 * T0 + 1, R / 2>(a, __ldg(post + T0 * Q + Q / 2), rot,
                                                             scale);
        dct_pairs_0<C, T0 + 1>(a, post, rot, scale);
    }
}

// Pair and rotate every output of the thread's last-group units (natural
// order spectrum Z in, DCT outputs X out, same registers).  post: the
// axis's table, read at the units' offsets only.
template <class C>
__device__ __forceinline__ void dct_pairs(float2 (&a)[C::EPT], int j,
                                          const float2 *__restrict__ post, const DctRot &rot,
                                          float scale)
{
    if (j != 0)
        dct_pairs_j_side0<C, 0>(a, j, post, rot, scale);
    else
        dct_pairs_0<C, 0>(a, post, rot, scale);
}

// The table of (cos, sin)(pi q / 32), built once in FP64.
const DctRot &dct_rot_table()
{
    static const DctRot t = [] {
        DctRot r{};
        for (int q = 0; q < 16; q++) {
            const double ang = 3.14159265358979323846264338327950288 * q / 32.0;
            r.r[q] = make_float2(q == 0 ? 1.f : (float)std::cos(ang), q == 0 ? 0.f : (float)std::sin(ang));
        }
        return r;
    }();
    return t;
}

// ---------------------------------------------------------------------------
// Row pass with vector loads and the pairing in registers (rows of 2^10 ..
// 2^14 points, 32 values per thread).  One 8-byte load at x[2i] of a real
// row brings v[i] and v[N-1-i].  In group 0 a thread therefore takes the
// units hib and 2^HB - 1 - hib of one line: position i = top + hib of the
// first pairs with N-1-i of the second (register r <-> r ^ (R-1)), and
// the loads of the two real rows of the complex line fill both units.  The
// last group is dealt out as in the column pass (dct_unit_lo), so each
// thread rotates its pairs (k, N-k) in registers and stores the two real
// rows' outputs directly.
template <class C>
__global__ void __launch_bounds__(C::T, C::MINB) row_dct_kernel(const DctIO d,
                                                                const float2 *__restrict__ tw,
                                                                const float2 *__restrict__ post,
                                                                const DctRot rot,
                                                                long long nlines, float scale)
{
    using G0 = Grp<C, 0>;
    using Gl = Grp<C, C::NG - 1>;
    static_assert(C::KW == 0 && C::NG >= 2 && G0::V == 2, "rows, two stage groups, 2 units");
    constexpr int HH = 1 << (G0::HB - 1);           // group-0 threads per line
    constexpr int P = (1 << Gl::S0) / Gl::V;        // last-group threads per line
    static_assert(HH * C::LB == C::T && P * C::LB == C::T, "threads cover the line blocks");
    extern __shared__ float2 sm[];
    const int tid = threadIdx.x;
    const long long line0 = (long long)blockIdx.x * C::LB;
    const long long nvalid = nlines - line0;
    float2 a[C::EPT];
    {
        const int lb = tid / HH;
        const int h = tid & (HH - 1);
        const int h1 = 2 * HH - 1 - h;
        const bool ok = lb < nvalid;
        const float *ra = d.in + 2 * (line0 + lb) * d.cols;
        const float *rb = ra + d.cols;
#pragma unroll
        for (int r = 0; r < G0::R; r += 2) {   // top(r) < N/2 exactly for even r
            const int top = brev_c(r, G0::G) << G0::HB;
            const int rc = r ^ (G0::R - 1);
            float2 fa = make_float2(0.f, 0.f), fb = fa, ga = fa, gb = fa;
            if (ok) {
                fa = __ldg(reinterpret_cast<const float2 *>(ra + 2 * (top + h)));
                fb = __ldg(reinterpret_cast<const float2 *>(rb + 2 * (top + h)));
                ga = __ldg(reinterpret_cast<const float2 *>(ra + 2 * (top + h1)));
                gb = __ldg(reinterpret_cast<const float2 *>(rb + 2 * (top + h1)));
            }
            a[r] = make_float2(fa.x, fb.x);                  // unit 0, position top + h
            a[G0::R + rc] = make_float2(fa.y, fb.y);         // unit 1, N-1-(top + h)
            a[G0::R + r] = make_float2(ga.x, gb.x);          // unit 1, position top + h1
            a[rc] = make_float2(ga.y, gb.y);                 // unit 0, N-1-(top + h1)
        }
#pragma unroll
        for (int v = 0; v < 2; v++)
            run_stages<C, 0, false>(a, v, 0, tw, C::L);
#pragma unroll
        for (int v = 0; v < 2; v++) {
            const int hi = brev_rt(v ? h1 : h, G0::HB);
#pragma unroll
            for (int r = 0; r < G0::R; r++)
                sm[sidx<C>(lb, r | (hi << G0::G), 0)] = a[v * G0::R + r];
        }
    }
    __syncthreads();
    if constexpr (C::NG >= 3) {
        group_smem<C, 1, false>(a, sm, tw, C::L);
        __syncthreads();
    }
    if constexpr (C::NG >= 4) {
        group_smem<C, 2, false>(a, sm, tw, C::L);
        __syncthreads();
    }
    const int lb = tid / P;
    const int j = tid % P;
#pragma unroll
    for (int v = 0; v < Gl::V; v++) {
        const int lo = dct_unit_lo<C>(v, j);
#pragma unroll
        for (int r = 0; r < Gl::R; r++)
            a[v * Gl::R + r] = sm[sidx<C>(lb, lo | (r << Gl::S0), 0)];
    }
#pragma unroll
    for (int v = 0; v < Gl::V; v++)
        run_stages<C, C::NG - 1, false>(a, v, dct_unit_lo<C>(v, j), tw, C::L);
    dct_pairs<C>(a, j, post, rot, scale);
    if (lb >= nvalid)
        return;
    float *oa = d.out + 2 * (line0 + lb) * d.cols;
    float *ob = oa + d.cols;
#pragma unroll
    for (int v = 0; v < Gl::V; v++) {
        const int lo = dct_unit_lo<C>(v, j);
#pragma unroll
        for (int r = 0; r < Gl::R; r++) {
            const int p = lo + (r << Gl::S0);
            oa[p] = a[v * Gl::R + r].x;
            ob[p] = a[v * Gl::R + r].y;
        }
    }
}

template <class C>
cudaError_t row_dct_launch(const DctIO &d, const float2 *tw, const float2 *post, long long nlines,
                           float scale, cudaStream_t s)
{
    auto k = row_dct_kernel<C>;
    constexpr int bytes = C::SMEM_BYTES;
    if (bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess)
            return e;
    }
    const unsigned grid = (unsigned)((nlines + C::LB - 1) / C::LB);
    k<<<grid, C::T, bytes, s>>>(d, tw, post, dct_rot_table(), nlines, scale);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Persistent TMA-fed column pass of the DCT (columns of 2^11 and 2^12 points,
// tiles of W complex columns = 2W real columns).
//
// The reorder needs no gather table: two tensor maps see the image's even
// rows and its odd rows (row stride 2 ld), so one TMA load brings
// x[0], x[2], .., x[N-2] = v[0 .. N/2) in order (the "even region") and
// another x[1], x[3], .., x[N-1] = v[N-1], v[N-2], .., v[N/2] (the "odd
// region", reversed).  Group 0 then gathers v[i] scrambled from the even
// region (i < N/2) or from odd-region slot N-1-i; which one is fixed by the
// register index.  As in the complex column pass, the next tile's even rows
// land in a prefetch region while the current tile is worked on and its odd
// rows in the lower half of the tile region once the last group has read it.
//
// The last group holds rows lo + r 2^S0 of a unit.  Output k pairs with
// N - k, i.e. unit lo with unit 2^S0 - lo (reversed r), so the units are
// dealt out such that each thread owns both members of its pairs
// (dct_unit_lo); the pairing and rotation then run in registers.  Units
// with lo < 2^(S0-1) leave through a staging buffer and one TMA store, the
// others with per-thread stores.
template <class C>
struct DctCol {
    using Gl = Grp<C, C::NG - 1>;
    static constexpr int HALF = C::N / 2;                  // rows of one parity
    static constexpr int BY = HALF < 256 ? HALF : 256;     // rows per block of a parity map
    static constexpr int NZ = HALF / BY;
    static constexpr int HVALS = HALF * C::W;              // values of one parity region
    static constexpr int TW_OFF = C::E + HVALS;
    static constexpr int SMEM_BYTES = (TW_OFF + C::N) * 8;
    static constexpr uint32_t HBYTES = (uint32_t)HVALS * 8u;
    static constexpr uint32_t TW_BYTES = (uint32_t)C::N * 8u;   // N-1 entries + padding
    static constexpr int M = 1 << Gl::S0;                  // rows of one store block
    static constexpr int QROWS = M / 2;
    static_assert(C::LB == 1 && C::NG >= 2, "one line block, two stage groups at least");
    static_assert(M == 256, "store blocks are the 256-row blocks of the store map");
    static_assert(((C::T * (Gl::V / 2)) >> C::KW) == QROWS, "threads cover half the row offsets");
    static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
};

// maps: even rows (me), odd rows (mo), each x = complex column, y = row
// pair within a block of BY, z = block, box W x BY x NZ; omap: the output as
// complex columns, x, row within a 256-row block, block, box W x 128 x N/256.
template <class C>
__global__ void __launch_bounds__(C::T, 1) col_dct_tma_kernel(
    const __grid_constant__ CUtensorMap me, const __grid_constant__ CUtensorMap mo,
    const __grid_constant__ CUtensorMap omap, float2 *out, long long ld, int ntiles,
    const float2 *__restrict__ tw, const float2 *__restrict__ post, const DctRot rot, float scale,
    int *err, int withhold)
{
    using D = DctCol<C>;
    using G0 = Grp<C, 0>;
    using Gl = Grp<C, C::NG - 1>;
    extern __shared__ __align__(1024) float2 sm[];
    __shared__ __align__(8) uint64_t bar_even, bar_odd;
    const int tid = threadIdx.x;
    int tile = blockIdx.x;
    float2 *pref = sm + C::E;          // even region
    float2 *stw = sm + D::TW_OFF;      // rotation factors, loaded once
    float2 *stage = sm + C::E / 2;     // staging half of the tile region
    if (tid == 0) {
        mbar_init(&bar_even, 1);
        mbar_init(&bar_odd, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0 && tile < ntiles) {
        mbar_expect_tx(&bar_even, D::TW_BYTES);
        bulk_load(stw, tw, D::TW_BYTES, &bar_even);
        mbar_arrive_expect_tx(&bar_even, D::HBYTES);
        tma_load_3d(pref, &me, tile * C::W, 0, 0, &bar_even);
        if (!(withhold && blockIdx.x == 0)) {   // self-test: the first odd rows never come
            mbar_arrive_expect_tx(&bar_odd, D::HBYTES);
            tma_load_3d(sm, &mo, tile * C::W, 0, 0, &bar_odd);
        }
    }
    uint32_t parity = 0;
    const int j = tid >> C::KW;
    float2 a[C::EPT];
    for (; tile < ntiles; tile += gridDim.x) {
        const int next = tile + gridDim.x;
        const bool ok = mbar_wait_bounded(&bar_even, parity) && mbar_wait_bounded(&bar_odd, parity);
        if (__syncthreads_or(ok ? 0 : 1)) {
            if (tid == 0) {
                atomicExch(err, kDevErrTmaTimeout);
                bulk_wait_all();
            }
            mbar_wait_bounded(&bar_even, parity);
            mbar_wait_bounded(&bar_odd, parity);
            return;
        }
        parity ^= 1;
        // group 0: v[i] from the even region (i < N/2) or odd-region slot N-1-i
#pragma unroll
        for (int v = 0; v < G0::V; v++) {
            const int u = tid + v * C::T;
            const int w = u & (C::W - 1);
            const int hib = (u >> C::KW) & ((1 << G0::HB) - 1);
#pragma unroll
            for (int r = 0; r < G0::R; r++) {
                const int i = (brev_c(r, G0::G) << G0::HB) | hib;
                a[v * G0::R + r] = (brev_c(r, G0::G) << G0::HB) < D::HALF
                                       ? pref[i * C::W + w]
                                       : sm[(C::N - 1 - i) * C::W + w];
            }
        }
#pragma unroll
        for (int v = 0; v < G0::V; v++)
            run_stages<C, 0, false, true>(a, v, 0, stw, C::L);
        fence_proxy_async_smem();
        if (tid == 0)
            bulk_wait_read_all();   // the previous tile's staging half is free
        __syncthreads();            // both regions have been read
        if (tid == 0 && next < ntiles) {
            mbar_arrive_expect_tx(&bar_even, D::HBYTES);
            tma_load_3d(pref, &me, next * C::W, 0, 0, &bar_even);
        }
#pragma unroll
        for (int v = 0; v < G0::V; v++) {
            const int u = tid + v * C::T;
            const int w = u & (C::W - 1);
            const int hib = (u >> C::KW) & ((1 << G0::HB) - 1);
            const int hi = brev_rt(hib, G0::HB);
#pragma unroll
            for (int r = 0; r < G0::R; r++)
                sm[sidx<C>(0, r | (hi << G0::G), w)] = a[v * G0::R + r];
        }
        __syncthreads();
        if constexpr (C::NG >= 3) {
            group_smem<C, 1, false, false, true>(a, sm, stw, C::L);
            __syncthreads();
        }
        if constexpr (C::NG >= 4) {
            group_smem<C, 2, false, false, true>(a, sm, stw, C::L);
            __syncthreads();
        }
        // last group: units dealt out in pairs
        const int w = tid & (C::W - 1);
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
            const int lo = dct_unit_lo<C>(v, j);
#pragma unroll
            for (int r = 0; r < Gl::R; r++)
                a[v * Gl::R + r] = sm[sidx<C>(0, lo | (r << Gl::S0), w)];
        }
        fence_proxy_async_smem();
        __syncthreads();   // the tile region is free
        if (tid == 0 && next < ntiles) {
            mbar_arrive_expect_tx(&bar_odd, D::HBYTES);
            tma_load_3d(sm, &mo, next * C::W, 0, 0, &bar_odd);
        }
#pragma unroll
        for (int v = 0; v < Gl::V; v++)
            run_stages<C, C::NG - 1, false, true>(a, v, dct_unit_lo<C>(v, j), stw, C::L);
        dct_pairs<C>(a, j, post, rot, scale);
        // units with row offsets below M/2: staging + one TMA store
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
            if (!dct_unit_low<C>(v))
                continue;
            const int q = dct_unit_lo<C>(v, j) & (D::QROWS - 1);
#pragma unroll
            for (int r = 0; r < Gl::R; r++)
                stage[((r * D::QROWS) | q) * C::W + w] = a[v * Gl::R + r];
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tma_store_3d(&omap, tile * C::W, 0, 0, stage);
            bulk_commit();
        }
        // the others: per-thread stores
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
            if (dct_unit_low<C>(v))
                continue;
            float2 *dst = out + (long long)dct_unit_lo<C>(v, j) * ld + (long long)tile * C::W + w;
#pragma unroll
            for (int r = 0; r < Gl::R; r++)
                st_stream(dst + (long long)(r << Gl::S0) * ld, a[v * Gl::R + r]);
        }
    }
    if (tid == 0)
        bulk_wait_all();   // shared memory stays valid until the stores are done
}

// The TMA-fed DCT column pass when the image allows it: complex width a
// multiple of W, 16-byte aligned buffers and table, a status word; returns
// cudaErrorNotSupported otherwise (the caller then runs the plain kernel).
template <class C>
cudaError_t dct_col_tma_launch(const DctIO &d, const float2 *tw, const float2 *post, float scale,
                               int *err, int withhold, cudaStream_t s)
{
    using D = DctCol<C>;
    const long long cc = d.cols / 2;   // complex columns
    if (!err || cc % C::W != 0 || (reinterpret_cast<uintptr_t>(d.in) & 15) ||
        (reinterpret_cast<uintptr_t>(d.out) & 15) || (reinterpret_cast<uintptr_t>(tw) & 15) ||
        (cc * 8) % 16 != 0 || !tensor_maps_available())
        return cudaErrorNotSupported;
    const float2 *in = reinterpret_cast<const float2 *>(d.in);
    float2 *out = reinterpret_cast<float2 *>(d.out);
    CUtensorMap me, mo, omap;
    if (!encode_map_xyz(&me, in, cc, D::BY, D::NZ, 2 * cc, 2 * cc * D::BY, C::W, D::BY, D::NZ) ||
        !encode_map_xyz(&mo, in + cc, cc, D::BY, D::NZ, 2 * cc, 2 * cc * D::BY, C::W, D::BY,
                        D::NZ) ||
        !encode_map_xyz(&omap, out, cc, 256, C::N / 256, cc, cc * 256, C::W, D::QROWS,
                        C::N / 256))
        return cudaErrorNotSupported;
    auto k = col_dct_tma_kernel<C>;
    constexpr int SMEM = D::SMEM_BYTES;
    static DeviceCache attr_set;
    const int dev = device_current();
    if (!attr_set.get(dev)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess)
            return e;
        attr_set.set(dev, 1);
    }
    const int ntiles = (int)(cc / C::W);
    int grid = device_sm_count();
    if (grid > ntiles)
        grid = ntiles;
    k<<<grid, C::T, SMEM, s>>>(me, mo, omap, out, cc, ntiles, tw, post, dct_rot_table(), scale,
                               err, withhold);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Forward DCT columns of 4096 points on the engine of the complex column
// pass (two groups of 6 stages, 256 threads x 64 values), two real columns
// per complex line, tiles of W complex = 2W real columns.  The even rows
// (v[0..N/2)) arrive in the prefetch region and the odd rows (v[N/2..N),
// reversed) in the first half of the tile region, as two TMA loads.
// After the last group thread (lo, w) holds Z[k], k = lo + 64 r.  The
// mirror N - k lies in thread 64 - lo at index 63 - r (lo != 0) or in the
// same thread at 64 - r (lo = 0), so each thread with lo != 0 hands its
// values r >= 32 through the staging half of shared memory to the thread
// that pairs them, and every thread forms X[k] and X[N-k] for its r < 32
// (dct_pair); k = N/2 pairs with itself.  X[k] (rows 0..N/2-1) and X[N-k]
// (rows N/2..N-1; k = 0 has no mirror row) leave by one TMA store each.
template <class C>
__global__ void __launch_bounds__(C::T, 1) col_dct_tma64_kernel(
    const __grid_constant__ CUtensorMap me, const __grid_constant__ CUtensorMap mo,
    const __grid_constant__ CUtensorMap omap, int ntiles, const float2 *__restrict__ tw,
    const float2 *__restrict__ post, float scale, int *err, int withhold)
{
    using S = TmaSplit<C>;
    using G0 = Grp<C, 0>;
    using Gl = Grp<C, C::NG - 1>;
    constexpr int N = C::N, HALF = N / 2, R = Gl::R;
    static_assert(C::NG == 2 && Gl::V == 1 && C::T == (1 << (Gl::S0 + C::KW)) &&
                      (R << Gl::S0) == N,
                  "one unit of R values per thread, k = lo + 2^S0 r");
    extern __shared__ __align__(1024) float2 sm[];
    __shared__ __align__(8) uint64_t bar_early, bar_late;
    __shared__ float2 rot_base[R / 2];   // (cos, sin)(pi 2^S0 r / (2N)), r < R/2
    const int tid = threadIdx.x;
    float2 *stw = sm + S::TW_OFF;
    float2 *stage = sm + C::E / 2;
    const int w = tid & (C::W - 1);
    const int lo = tid >> C::KW;
    auto issue_early = [&](int t) {
        mbar_arrive_expect_tx(&bar_early, S::EARLY_BYTES);
        tma_load_3d(sm + C::E, &me, t * C::W, 0, 0, &bar_early);
    };
    auto issue_late = [&](int t) {
        mbar_arrive_expect_tx(&bar_late, S::LATE_BYTES);
        tma_load_3d(sm, &mo, t * C::W, 0, 0, &bar_late);
    };
    if (tid == 0) {
        mbar_init(&bar_early, 1);
        mbar_init(&bar_late, 1);
        fence_mbar_init();
    }
    for (int j = tid; j < R / 2; j += C::T)
        rot_base[j] = __ldg(post + (j << Gl::S0));
    const float2 rot_lo = __ldg(post + lo);
    __syncthreads();
    int tile = (int)blockIdx.x;
    int n_early = 0, n_late = 0, w_early = 0, w_late = 0;
    if (tile < ntiles) {
        if (tid == 0) {
            mbar_expect_tx(&bar_early, S::TW_BYTES);
            bulk_load(stw, tw, S::TW_BYTES, &bar_early);
            issue_early(tile);
            if (!(withhold && blockIdx.x == 0))   // self-test: the first odd rows never come
                issue_late(tile);
        }
        n_early = n_late = 1;
    }
    bool lost = false;
    float2 a[C::EPT];
    for (; tile < ntiles; tile += gridDim.x) {
        const int next = tile + gridDim.x;
        const bool ok = mbar_wait_bounded(&bar_early, (uint32_t)(w_early & 1)) &&
                        mbar_wait_bounded(&bar_late, (uint32_t)(w_late & 1));
        if (__syncthreads_or(ok ? 0 : 1)) {
            lost = true;
            break;
        }
        w_early++;
        w_late++;
        // group 0: scrambled gather of the reordered line (odd rows backwards)
        {
            const float2 *pref = sm + C::E;
#pragma unroll
            for (int v = 0; v < G0::V; v++) {
                const int u = tid + v * C::T;
                const int hib = (u >> C::KW) & ((1 << G0::HB) - 1);
#pragma unroll
                for (int r = 0; r < G0::R; r++) {
                    const int top = brev_c(r, G0::G) << G0::HB;   // compile-time
                    a[v * G0::R + r] = top < HALF ? pref[(top | hib) * C::W + w]
                                                  : sm[(N - 1 - (top | hib)) * C::W + w];
                }
            }
        }
#pragma unroll
        for (int v = 0; v < G0::V; v++)
            run_stages<C, 0, false, true>(a, v, 0, stw, C::L);
        fence_proxy_async_smem();
        if (tid == 0)
            bulk_wait_read_all();   // the previous tile's stores have read the staging half
        __syncthreads();            // both input regions have been read
        if (tid == 0 && next < ntiles)
            issue_early(next);
        if (next < ntiles)
            n_early++;
#pragma unroll
        for (int v = 0; v < G0::V; v++) {
            const int u = tid + v * C::T;
            const int hib = (u >> C::KW) & ((1 << G0::HB) - 1);
            const int hi = brev_rt(hib, G0::HB);
#pragma unroll
            for (int r = 0; r < G0::R; r++)
                sm[sidx<C>(0, r | (hi << G0::G), w)] = a[v * G0::R + r];
        }
        __syncthreads();
        group_last_read<C>(a, sm);
        fence_proxy_async_smem();
        __syncthreads();   // the tile region is free: the next tile's odd rows
        if (tid == 0 && next < ntiles)
            issue_late(next);
        if (next < ntiles)
            n_late++;
        run_stages<C, C::NG - 1, false, true>(a, 0, lo, stw, C::L);
        // values r >= R/2 to the thread that pairs them: N - k is thread
        // 2^S0 - lo, index R - 1 - r
        if (lo != 0) {
            const int tid_r = (((1 << Gl::S0) - lo) << C::KW) | w;
#pragma unroll
            for (int r = R / 2; r < R; r++)
                stage[(R - 1 - r) * C::T + tid_r] = a[r];
        }
        __syncthreads();
        float2 xmid = make_float2(0.f, 0.f);
        if (lo == 0) {   // k = N/2 pairs with itself
            float2 xq;
            dct_pair(a[R / 2], a[R / 2], __ldg(post + HALF), scale, xmid, xq);
        }
#pragma unroll
        for (int r = 0; r < R / 2; r++) {
            const float2 zk = a[r];
            const float2 zp = lo != 0 ? stage[r * C::T + tid] : (r == 0 ? zk : a[R - r]);
            const float2 rb = rot_base[r];
            const float2 cs = make_float2(rb.x * rot_lo.x - rb.y * rot_lo.y,
                                          rb.x * rot_lo.y + rb.y * rot_lo.x);
            float2 xk, xp;
            dct_pair(zk, zp, cs, scale, xk, xp);
            a[r] = xk;
            a[r == 0 ? R / 2 : R - r] = xp;   // the slot zp came from (lo = 0)
        }
        __syncthreads();   // the handed values have been read
        // X[k], rows k < N/2
#pragma unroll
        for (int r = 0; r < R / 2; r++)
            stage[((r << Gl::S0) | lo) * C::W + w] = a[r];
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tma_store_3d(&omap, tile * C::W, 0, 0, stage);
            bulk_commit();
            bulk_wait_read_all();
        }
        __syncthreads();
        // X[N - k] at rows N/2 + s, s = N/2 - k; X[N/2] at s = 0
#pragma unroll
        for (int r = 0; r < R / 2; r++)
            if (lo != 0 || r != 0)
                stage[(HALF - ((r << Gl::S0) | lo)) * C::W + w] = a[r == 0 ? R / 2 : R - r];
        if (lo == 0)
            stage[w] = xmid;
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tma_store_3d(&omap, tile * C::W, 0, HALF / 256, stage);
            bulk_commit();
        }
    }
    if (__syncthreads_or(lost ? 1 : 0)) {
        if (tid == 0)
            atomicExch(err, kDevErrTmaTimeout);
        // let transfers still in flight land before the CTA leaves
        if (n_early > w_early)
            mbar_wait_bounded(&bar_early, (uint32_t)(w_early & 1));
        if (n_late > w_late)
            mbar_wait_bounded(&bar_late, (uint32_t)(w_late & 1));
    }
    if (tid == 0)
        bulk_wait_all();   // shared memory stays valid until the stores are done
}

// The kernel above for forward DCT columns of 4096 points when the image
// allows it; cudaErrorNotSupported (nothing launched) otherwise.
cudaError_t dct_col_tma64_launch(const DctIO &d, const float2 *tw, const float2 *post,
                                 float scale, int *err, int withhold, cudaStream_t s)
{
    using C = LineCfg<12, 2, 0, 64, 6>;
    using S = TmaSplit<C>;
    constexpr int HALF = C::N / 2;
    const long long cc = d.cols / 2;   // complex columns
    if (!err || d.rows != C::N || cc % C::W != 0 || (reinterpret_cast<uintptr_t>(d.in) & 15) ||
        (reinterpret_cast<uintptr_t>(d.out) & 15) || (reinterpret_cast<uintptr_t>(tw) & 15) ||
        !tensor_maps_available())
        return cudaErrorNotSupported;
    const float2 *in = reinterpret_cast<const float2 *>(d.in);
    float2 *out = reinterpret_cast<float2 *>(d.out);
    CUtensorMap me, mo, omap;
    if (!encode_map_xyz(&me, in, cc, 256, HALF / 256, 2 * cc, 2 * cc * 256, C::W, 256,
                        HALF / 256) ||
        !encode_map_xyz(&mo, in + cc, cc, 256, HALF / 256, 2 * cc, 2 * cc * 256, C::W, 256,
                        HALF / 256) ||
        !encode_map_xyz(&omap, out, cc, 256, C::N / 256, cc, cc * 256, C::W, 256, HALF / 256))
        return cudaErrorNotSupported;
    static_assert((uint32_t)HALF * C::W * 8u == S::EARLY_BYTES &&
                      S::EARLY_BYTES == S::LATE_BYTES,
                  "each parity fills one half of the split");
    auto k = col_dct_tma64_kernel<C>;
    constexpr int SMEM = S::SMEM_BYTES;
    static DeviceCache attr_set;
    const int dev = device_current();
    if (!attr_set.get(dev)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess)
            return e;
        attr_set.set(dev, 1);
    }
    const int ntiles = (int)(cc / C::W);
    int grid = device_sm_count();
    if (grid > ntiles)
        grid = ntiles;
    k<<<grid, C::T, SMEM, s>>>(me, mo, omap, ntiles, tw, post, scale, err, withhold);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Inverse DCT columns of 4096 points on the same engine, two real columns per
// complex line: with (c, s) = (cos, sin)(pi k / (2N)) and X' = X[N - k]
// (X[N] = 0), V_a = (c + i s)(X_a - i X'_a), V_b likewise, Z = V_a + i V_b,
// and v_a + i v_b = IDFT(Z) (the plan's conjugate factors).  The tile arrives
// in natural order (rows 0..N/2-1 in the prefetch region, the others in the
// tile region), so group 0 reads X[k] and X[N-k] of its scrambled positions
// straight from shared memory.  Outputs: x[2n] = v[n] (n < N/2) and
// x[2n+1] = v[N-1-n], one TMA store over the even rows and one over the odd
// rows (reversed in staging).
template <class C>
__global__ void __launch_bounds__(C::T, 1) col_idct_tma64_kernel(
    const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap oe,
    const __grid_constant__ CUtensorMap oo, int ntiles, const float2 *__restrict__ tw,
    const float2 *__restrict__ post, float scale, int *err, int withhold)
{
    using S = TmaSplit<C>;
    using G0 = Grp<C, 0>;
    using Gl = Grp<C, C::NG - 1>;
    constexpr int N = C::N, HALF = N / 2, R = Gl::R;
    static_assert(C::NG == 2 && Gl::V == 1 && G0::V == 1 && C::T == (1 << (Gl::S0 + C::KW)) &&
                      (R << Gl::S0) == N && G0::R == R,
                  "one unit of R values per thread in both groups");
    extern __shared__ __align__(1024) float2 sm[];
    __shared__ __align__(8) uint64_t bar_early, bar_late;
    __shared__ float2 rot_top[G0::R];   // (cos, sin)(pi top(r) / (2N)), top(r) = rev(r) 2^HB
    const int tid = threadIdx.x;
    float2 *stw = sm + S::TW_OFF;
    float2 *stage = sm + C::E / 2;
    const float2 *pref = sm + C::E;
    const int w = tid & (C::W - 1);
    const int hib = (tid >> C::KW) & ((1 << G0::HB) - 1);
    const int lo = (tid >> C::KW) & ((1 << Gl::S0) - 1);
    if (tid == 0) {
        mbar_init(&bar_early, 1);
        mbar_init(&bar_late, 1);
        fence_mbar_init();
    }
    for (int j = tid; j < G0::R; j += C::T) {
        const int top = brev_rt(j, G0::G) << G0::HB;
        const float2 p = __ldg(post + (top <= HALF ? top : N - top));
        rot_top[j] = top <= HALF ? p : make_float2(p.y, p.x);
    }
    const float2 rot_hib = __ldg(post + hib);
    __syncthreads();
    int tile = (int)blockIdx.x;
    int n_early = 0, n_late = 0, w_early = 0, w_late = 0;
    if (tile < ntiles) {
        if (tid == 0) {
            mbar_expect_tx(&bar_early, S::TW_BYTES);
            bulk_load(stw, tw, S::TW_BYTES, &bar_early);
            split_issue_early<C>(sm, &map, tile * C::W, &bar_early);
            if (!(withhold && blockIdx.x == 0))   // self-test: the first second half never comes
                split_issue_late<C>(sm, &map, tile * C::W, &bar_late);
        }
        n_early = n_late = 1;
    }
    bool lost = false;
    float2 a[C::EPT];
    auto xrow = [&](int k) { return k < HALF ? pref[k * C::W + w] : sm[(k - HALF) * C::W + w]; };
    for (; tile < ntiles; tile += gridDim.x) {
        const int next = tile + gridDim.x;
        const bool ok = mbar_wait_bounded(&bar_early, (uint32_t)(w_early & 1)) &&
                        mbar_wait_bounded(&bar_late, (uint32_t)(w_late & 1));
        if (__syncthreads_or(ok ? 0 : 1)) {
            lost = true;
            break;
        }
        w_early++;
        w_late++;
        // group 0: scrambled gather of the spectrum rows k and N - k,
        // pre-rotated into Z[k]
#pragma unroll
        for (int r = 0; r < G0::R; r++) {
            const int k = (brev_c(r, G0::G) << G0::HB) | hib;
            const float2 xn = xrow(k);
            float2 xm = xrow((N - k) & (N - 1));
            if (k == 0)
                xm = make_float2(0.f, 0.f);   // X[N] = 0
            const float2 rt = rot_top[r];
            const float c = rt.x * rot_hib.x - rt.y * rot_hib.y;
            const float sn = rt.x * rot_hib.y + rt.y * rot_hib.x;
            a[r] = make_float2(c * xn.x + sn * xm.x - sn * xn.y + c * xm.y,
                               sn * xn.x - c * xm.x + c * xn.y + sn * xm.y);
        }
        run_stages<C, 0, false, true>(a, 0, 0, stw, C::L);
        fence_proxy_async_smem();
        if (tid == 0)
            bulk_wait_read_all();   // the previous tile's stores have read the staging half
        __syncthreads();            // both input regions have been read
        if (tid == 0 && next < ntiles)
            split_issue_early<C>(sm, &map, next * C::W, &bar_early);
        if (next < ntiles)
            n_early++;
        {
            const int hi = brev_rt(hib, G0::HB);
#pragma unroll
            for (int r = 0; r < G0::R; r++)
                sm[sidx<C>(0, r | (hi << G0::G), w)] = a[r];
        }
        __syncthreads();
        group_last_read<C>(a, sm);
        fence_proxy_async_smem();
        __syncthreads();   // the tile region is free: the next tile's second half
        if (tid == 0 && next < ntiles)
            split_issue_late<C>(sm, &map, next * C::W, &bar_late);
        if (next < ntiles)
            n_late++;
        run_stages<C, C::NG - 1, false, true>(a, 0, lo, stw, C::L);
        // v[k], k = lo + 2^S0 r: the even rows take k < N/2 in order
#pragma unroll
        for (int r = 0; r < R / 2; r++)
            stage[((r << Gl::S0) | lo) * C::W + w] = make_float2(a[r].x * scale, a[r].y * scale);
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tma_store_3d(&oe, tile * C::W, 0, 0, stage);
            bulk_commit();
            bulk_wait_read_all();
        }
        __syncthreads();
        // the odd rows take k >= N/2 at slot N - 1 - k
#pragma unroll
        for (int r = R / 2; r < R; r++)
            stage[(N - 1 - ((r << Gl::S0) | lo)) * C::W + w] =
                make_float2(a[r].x * scale, a[r].y * scale);
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tma_store_3d(&oo, tile * C::W, 0, 0, stage);
            bulk_commit();
        }
    }
    if (__syncthreads_or(lost ? 1 : 0)) {
        if (tid == 0)
            atomicExch(err, kDevErrTmaTimeout);
        // let transfers still in flight land before the CTA leaves
        if (n_early > w_early)
            mbar_wait_bounded(&bar_early, (uint32_t)(w_early & 1));
        if (n_late > w_late)
            mbar_wait_bounded(&bar_late, (uint32_t)(w_late & 1));
    }
    if (tid == 0)
        bulk_wait_all();   // shared memory stays valid until the stores are done
}

// The kernel above for inverse DCT columns of 4096 points when the image
// allows it; cudaErrorNotSupported (nothing launched) otherwise.
cudaError_t idct_col_tma64_launch(const DctIO &d, const float2 *tw, const float2 *post,
                                  float scale, int *err, int withhold, cudaStream_t s)
{
    using C = LineCfg<12, 2, 0, 64, 6>;
    using S = TmaSplit<C>;
    constexpr int HALF = C::N / 2;
    const long long cc = d.cols / 2;   // complex columns
    if (!err || d.rows != C::N || cc % C::W != 0 || (reinterpret_cast<uintptr_t>(d.in) & 15) ||
        (reinterpret_cast<uintptr_t>(d.out) & 15) || (reinterpret_cast<uintptr_t>(tw) & 15) ||
        !tensor_maps_available())
        return cudaErrorNotSupported;
    const float2 *in = reinterpret_cast<const float2 *>(d.in);
    float2 *out = reinterpret_cast<float2 *>(d.out);
    CUtensorMap map, oe, oo;
    if (!encode_col_map(&map, in, C::N, (int)cc, cc, C::W, S::BOX, S::NB) ||
        !encode_map_xyz(&oe, out, cc, 256, HALF / 256, 2 * cc, 2 * cc * 256, C::W, 256,
                        HALF / 256) ||
        !encode_map_xyz(&oo, out + cc, cc, 256, HALF / 256, 2 * cc, 2 * cc * 256, C::W, 256,
                        HALF / 256))
        return cudaErrorNotSupported;
    auto k = col_idct_tma64_kernel<C>;
    constexpr int SMEM = S::SMEM_BYTES;
    static DeviceCache attr_set;
    const int dev = device_current();
    if (!attr_set.get(dev)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess)
            return e;
        attr_set.set(dev, 1);
    }
    const int ntiles = (int)(cc / C::W);
    int grid = device_sm_count();
    if (grid > ntiles)
        grid = ntiles;
    k<<<grid, C::T, SMEM, s>>>(map, oe, oo, ntiles, tw, post, scale, err, withhold);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Tile geometry of the inverse DCT column pass over a CTA pair (below): the
// local engine's 2^L rows in two halves of whole 256-row blocks.
template <class C>
struct DctPair {
    using S = TmaSplit<C>;
    using GC = GroupCol<C, 1>;
    static constexpr int HALF_ROWS = C::N / 2;               // local rows per map
    static constexpr uint32_t HBYTES = (uint32_t)HALF_ROWS * C::W * 8u;
    static constexpr int NBH = HALF_ROWS / S::BOX;           // 256-row blocks per map
    static_assert(C::L == 12 && C::W == 4, "the 4096-row engine, 4 complex columns");
    static_assert(HBYTES == S::EARLY_BYTES && HBYTES == S::LATE_BYTES, "two halves of the split");
};

// Forward DCT columns of 16384 points on the four-CTA cluster kernel with
// the exchange through L2 (col_dct_l2_kernel, one complex line per real
// column), for widths of 4 mod 8 real columns (the packed kernel above takes
// multiples of 8); cudaErrorNotSupported (nothing launched) when the image
// does not allow it.  The kernel runs in place: its tiles are 4 real columns, so
// every access is half of a 32-byte sector, and a store merges into a
// sector that the load of the same tile (and of the neighbouring tile, in
// flight at the same time) has just brought into L2.  Out of place the
// stores would fall on sectors not in L2 (measured 3.38 ms against 1.35 ms
// at 16384^2, with 25 % more DRAM reads), so an out-of-place call copies the
// input to the output first (one device-to-device copy).
cudaError_t dct_col_quad_launch(const DctIO &din, const float2 *tw, const float2 *post,
                                float scale, int *err, int withhold, cudaStream_t s)
{
    using C = LineCfg<12, 2, 0, 64, 6>;
    using S = TmaSplit<C>;
    using GC = GroupCol<C, 2>;
    constexpr int CS = GC::CS;
    const long long cc = din.cols / 2;   // 8-byte elements per row
    if (!err || din.rows != (long long)CS * C::N || din.cols % C::W != 0 ||
        (reinterpret_cast<uintptr_t>(din.in) & 15) || (reinterpret_cast<uintptr_t>(din.out) & 15) ||
        (reinterpret_cast<uintptr_t>(tw) & 15) || !tensor_maps_available())
        return cudaErrorNotSupported;
    const DctIO d{din.out, din.out, din.rows, din.cols};
    const float2 *in = reinterpret_cast<const float2 *>(d.in);
    float2 *out = reinterpret_cast<float2 *>(d.out);
    constexpr int HALF = C::N / 2;   // rows of each half of a CTA's local line
    DctL2Maps m;
    for (int r = 0; r < CS; r++)
        if (!encode_col_map(&m.early[r], in + 2 * r * cc, HALF, (int)cc, 2 * CS * cc, C::W / 2,
                            S::BOX, HALF / S::BOX) ||
            !encode_col_map(&m.late[r], in + (2 * CS - 1 - 2 * r) * cc, HALF, (int)cc, 2 * CS * cc,
                            C::W / 2, S::BOX, HALF / S::BOX))
            return cudaErrorNotSupported;
    if (!encode_col_map(&m.out, out, (int)d.rows, (int)cc, cc, C::W / 2, S::BOX, GC::OUT_BOX_Z))
        return cudaErrorNotSupported;
    auto k = col_dct_l2_kernel<C, 2>;
    constexpr int SMEM = S::SMEM_BYTES;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(C::T);
    cfg.dynamicSmemBytes = SMEM;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    static DeviceCache groups;
    const int dev = device_current();
    if (!groups.get(dev)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess)
            return e;
        cfg.gridDim = dim3((unsigned)(CS * (device_sm_count() / CS)));
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
        if (e != cudaSuccess)
            return e;
        groups.set(dev, n > 0 ? n : 1);
    }
    const int ntiles = (int)(d.cols / C::W);
    const int ng = groups.get(dev) < ntiles ? groups.get(dev) : ntiles;
    if (din.in != din.out) {
        cudaError_t e = cudaMemcpyAsync(din.out, din.in, (size_t)(din.rows * din.cols) * sizeof(float),
                                        cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess)
            return e;
    }
    void *xbuf = nullptr;
    cudaError_t e = scratch_take(&xbuf, (size_t)ng * GC::L2_SCRATCH_VALS * sizeof(float2), s);
    if (e != cudaSuccess)
        return e;
    cfg.gridDim = dim3((unsigned)(CS * ng));
    e = cudaLaunchKernelEx(&cfg, k, m, tw, post, ntiles, scale, err, withhold,
                           static_cast<float2 *>(xbuf));
    const cudaError_t f = cudaFreeAsync(xbuf, s);
    return e != cudaSuccess ? e : f;
}

// Forward DCT columns of 2^(12+CL) points (8192: a CTA pair, 16384: four
// CTAs) with two real columns per complex line on the cluster kernel with
// the exchange through L2 (col_dct_pack_l2_kernel): tiles of 8 real
// columns, 32-byte rows, in place or out of place; cudaErrorNotSupported
// (nothing launched) when the image does not allow it.
template <int CL>
cudaError_t dct_col_pack_launch(const DctIO &d, const float2 *tw, const float2 *post,
                                float scale, int *err, int withhold, cudaStream_t s)
{
    using C = LineCfg<12, 2, 0, 64, 6>;
    using S = TmaSplit<C>;
    using GC = GroupCol<C, CL>;
    constexpr int CS = GC::CS;
    const long long cc = d.cols / 2;   // complex columns: pairs of real columns
    if (!err || d.rows != (long long)CS * C::N || d.cols % (2 * C::W) != 0 ||
        (reinterpret_cast<uintptr_t>(d.in) & 15) || (reinterpret_cast<uintptr_t>(d.out) & 15) ||
        (reinterpret_cast<uintptr_t>(tw) & 15) || !tensor_maps_available())
        return cudaErrorNotSupported;
    const float2 *in = reinterpret_cast<const float2 *>(d.in);
    float2 *out = reinterpret_cast<float2 *>(d.out);
    constexpr int HALF = C::N / 2;   // rows of each half of a CTA's local line
    DctPackMaps m;
    for (int r = 0; r < CS; r++)
        if (!encode_col_map(&m.early[r], in + 2 * r * cc, HALF, (int)cc, 2 * CS * cc, C::W, S::BOX,
                            HALF / S::BOX) ||
            !encode_col_map(&m.late[r], in + (2 * CS - 1 - 2 * r) * cc, HALF, (int)cc, 2 * CS * cc,
                            C::W, S::BOX, HALF / S::BOX))
            return cudaErrorNotSupported;
    if (!encode_col_map(&m.out, out, (int)d.rows, (int)cc, cc, C::W, S::BOX, GC::OUT_BOX_Z) ||
        !encode_map_xyz(&m.out2, out, cc, (int)d.rows, 1, cc, cc * d.rows, C::W, S::BOX, 1))
        return cudaErrorNotSupported;
    m.mid_row = out + (d.rows / 2) * cc;
    auto k = col_dct_pack_l2_kernel<C, CL>;
    constexpr int SMEM = S::SMEM_BYTES;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(C::T);
    cfg.dynamicSmemBytes = SMEM;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    static DeviceCache groups;
    const int dev = device_current();
    if (!groups.get(dev)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess)
            return e;
        cfg.gridDim = dim3((unsigned)(CS * (device_sm_count() / CS)));
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
        if (e != cudaSuccess)
            return e;
        groups.set(dev, n > 0 ? n : 1);
    }
    const int ntiles = (int)(cc / C::W);
    const int ng = groups.get(dev) < ntiles ? groups.get(dev) : ntiles;
    void *xbuf = nullptr;
    cudaError_t e = scratch_take(
        &xbuf, (size_t)ng * (size_t)(GC::L2_SCRATCH_VALS + GC::MIRROR_VALS) * sizeof(float2), s);
    if (e != cudaSuccess)
        return e;
    cfg.gridDim = dim3((unsigned)(CS * ng));
    e = cudaLaunchKernelEx(&cfg, k, m, tw, post, ntiles, scale, err, withhold,
                           static_cast<float2 *>(xbuf));
    const cudaError_t f = cudaFreeAsync(xbuf, s);
    return e != cudaSuccess ? e : f;
}

// Inverse DCT columns of 16384 points on the same four-CTA kernel
// (col_idct_l2_kernel, one real line per complex line), in place for the
// same reason as the forward pass; cudaErrorNotSupported (nothing launched)
// when the image does not allow it.
cudaError_t idct_col_quad_launch(const DctIO &din, const float2 *tw, const float2 *post,
                                 float scale, int *err, int withhold, cudaStream_t s)
{
    using C = LineCfg<12, 2, 0, 64, 6>;
    using S = TmaSplit<C>;
    using GC = GroupCol<C, 2>;
    constexpr int CS = GC::CS;
    const long long cc = din.cols / 2;   // 8-byte elements per row
    if (!err || din.rows != (long long)CS * C::N || din.cols % C::W != 0 ||
        (reinterpret_cast<uintptr_t>(din.in) & 15) || (reinterpret_cast<uintptr_t>(din.out) & 15) ||
        (reinterpret_cast<uintptr_t>(tw) & 15) || !tensor_maps_available())
        return cudaErrorNotSupported;
    const DctIO d{din.out, din.out, din.rows, din.cols};
    const float2 *in = reinterpret_cast<const float2 *>(d.in);
    float2 *out = reinterpret_cast<float2 *>(d.out);
    IdctL2Maps m;
    for (int r = 0; r < CS; r++)
        if (!encode_col_map(&m.rows[r], in + r * cc, C::N, (int)cc, CS * cc, C::W / 2, S::BOX,
                            S::NB))
            return cudaErrorNotSupported;
    if (!encode_col_map(&m.even, out, (int)(d.rows / 2), (int)cc, 2 * cc, C::W / 2, S::BOX,
                        GC::OUT_BOX_Z) ||
        !encode_col_map(&m.odd, out + cc, (int)(d.rows / 2), (int)cc, 2 * cc, C::W / 2, S::BOX,
                        GC::OUT_BOX_Z))
        return cudaErrorNotSupported;
    auto k = col_idct_l2_kernel<C, 2>;
    constexpr int SMEM = S::SMEM_BYTES;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(C::T);
    cfg.dynamicSmemBytes = SMEM;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    static DeviceCache groups;
    const int dev = device_current();
    if (!groups.get(dev)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess)
            return e;
        cfg.gridDim = dim3((unsigned)(CS * (device_sm_count() / CS)));
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
        if (e != cudaSuccess)
            return e;
        groups.set(dev, n > 0 ? n : 1);
    }
    const int ntiles = (int)(d.cols / C::W);
    const int ng = groups.get(dev) < ntiles ? groups.get(dev) : ntiles;
    if (din.in != din.out) {
        cudaError_t e = cudaMemcpyAsync(din.out, din.in, (size_t)(din.rows * din.cols) * sizeof(float),
                                        cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess)
            return e;
    }
    void *xbuf = nullptr;
    cudaError_t e = scratch_take(&xbuf, (size_t)ng * GC::L2_SCRATCH_VALS * sizeof(float2), s);
    if (e != cudaSuccess)
        return e;
    cfg.gridDim = dim3((unsigned)(CS * ng));
    e = cudaLaunchKernelEx(&cfg, k, m, tw, post, ntiles, scale, err, withhold,
                           static_cast<float2 *>(xbuf));
    const cudaError_t f = cudaFreeAsync(xbuf, s);
    return e != cudaSuccess ? e : f;
}

template <class C, bool ROW>
cudaError_t dct_launch(const DctIO &d, const float2 *tw, const float2 *post, long long nlines,
                       float scale, cudaStream_t s)
{
    auto k = line_dct_kernel<C, ROW>;
    const int bytes = C::SMEM_BYTES;
    if (bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess)
            return e;
    }
    const long long per = ROW ? C::LB : C::W;
    const unsigned grid = (unsigned)((nlines + per - 1) / per);
    k<<<grid, C::T, bytes, s>>>(d, tw, post, nlines, scale);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fast inverse passes (rows of 2^10 .. 2^14 points; TMA-fed columns of 2^11
// and 2^12 points).  The pre-rotation pairs spectrum entries k and N - k of
// a line.  In the first stage group, position i = top(r) + hib (top(r) =
// brev(r) 2^HB) pairs with N - i = top(r ^ (R-1)) + (2^HB - hib), so a
// thread takes the units hib = h and 2^HB - h (h < 2^(HB-1)); thread 0 the
// units 0 and 2^(HB-1), each paired with itself.  The rotation of position
// top(r) + h is that of h turned by pi brev(r) / (2R) (a DctRot entry).
template <class C>
__device__ __forceinline__ void idct_pre_units(float2 (&a)[C::EPT], int h,
                                               const float2 *__restrict__ post, const DctRot &rot)
{
    using G0 = Grp<C, 0>;
    constexpr int R = G0::R, G = G0::G, HH = 1 << (G0::HB - 1), QS = 16 / R;
    float2 yk, yp;
    if (h != 0) {
        const float2 b0 = __ldg(post + h), b1 = __ldg(post + (2 * HH - h));
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int rc = r ^ (R - 1);
            if (brev_c(r, G) < R / 2) {
                idct_pre(a[r], a[R + rc], rot_mul(b0, rot.r[brev_c(r, G) * QS]), yk, yp);
                a[r] = yk;
                a[R + rc] = yp;
            } else {
                idct_pre(a[R + rc], a[r], rot_mul(b1, rot.r[brev_c(rc, G) * QS]), yk, yp);
                a[R + rc] = yk;
                a[r] = yp;
            }
        }
    } else {
        // unit 0: positions brev(r) 2^HB; b <-> R - b, k = 0 left alone,
        // k = N/2 (b = R/2) paired with itself
#pragma unroll
        for (int b = 1; b < R / 2; b++) {
            const int r = brev_c(b, G), r2 = brev_c(R - b, G);
            idct_pre(a[r], a[r2], rot.r[b * QS], yk, yp);
            a[r] = yk;
            a[r2] = yp;
        }
        idct_pre(a[brev_c(R / 2, G)], a[brev_c(R / 2, G)], rot.r[8], yk, yp);
        a[brev_c(R / 2, G)] = yk;
        // unit 1: positions top(r) + 2^(HB-1), pairs (r, r ^ (R-1))
        const float2 bh = __ldg(post + HH);
#pragma unroll
        for (int r = 0; r < R; r++) {
            if (brev_c(r, G) >= R / 2)
                continue;
            const int rc = r ^ (R - 1);
            idct_pre(a[R + r], a[R + rc], rot_mul(bh, rot.r[brev_c(r, G) * QS]), yk, yp);
            a[R + r] = yk;
            a[R + rc] = yp;
        }
    }
}

// Inverse row pass: scalar loads of the two spectrum rows, pre-rotation in
// registers, the stages, and a last group dealt out in complementary units
// (offsets t Q + j and t Q + Q - 1 - j, Q = 2M/V): position n pairs with
// N - 1 - n, so each thread writes x[2n] = v[n], x[2n+1] = v[N-1-n] of both
// real rows with 8-byte stores.
template <class C>
__global__ void __launch_bounds__(C::T, C::MINB) row_idct_kernel(const DctIO d,
                                                                 const float2 *__restrict__ tw,
                                                                 const float2 *__restrict__ post,
                                                                 const DctRot rot,
                                                                 long long nlines, float scale)
{
    using G0 = Grp<C, 0>;
    using Gl = Grp<C, C::NG - 1>;
    static_assert(C::KW == 0 && C::NG >= 2 && G0::V == 2, "rows, two stage groups, 2 units");
    constexpr int HH = 1 << (G0::HB - 1);
    constexpr int M = 1 << Gl::S0, V = Gl::V, R = Gl::R, Q = 2 * M / V, P = M / V;
    static_assert(HH * C::LB == C::T && P * C::LB == C::T, "threads cover the line blocks");
    extern __shared__ float2 sm[];
    const int tid = threadIdx.x;
    const long long line0 = (long long)blockIdx.x * C::LB;
    const long long nvalid = nlines - line0;
    float2 a[C::EPT];
    {
        const int lb = tid / HH;
        const int h = tid & (HH - 1);
        const int h1 = h == 0 ? HH : 2 * HH - h;
        const bool ok = lb < nvalid;
        const float *ra = d.in + 2 * (line0 + lb) * d.cols;
        const float *rb = ra + d.cols;
#pragma unroll
        for (int r = 0; r < G0::R; r++) {
            const int top = brev_c(r, G0::G) << G0::HB;
            a[r] = ok ? make_float2(__ldg(ra + top + h), __ldg(rb + top + h)) : make_float2(0.f, 0.f);
            a[G0::R + r] = ok ? make_float2(__ldg(ra + top + h1), __ldg(rb + top + h1))
                              : make_float2(0.f, 0.f);
        }
        idct_pre_units<C>(a, h, post, rot);
#pragma unroll
        for (int v = 0; v < 2; v++)
            run_stages<C, 0, false>(a, v, 0, tw, C::L);
#pragma unroll
        for (int v = 0; v < 2; v++) {
            const int hi = brev_rt(v ? h1 : h, G0::HB);
#pragma unroll
            for (int r = 0; r < G0::R; r++)
                sm[sidx<C>(lb, r | (hi << G0::G), 0)] = a[v * G0::R + r];
        }
    }
    __syncthreads();
    if constexpr (C::NG >= 3) {
        group_smem<C, 1, false>(a, sm, tw, C::L);
        __syncthreads();
    }
    if constexpr (C::NG >= 4) {
        group_smem<C, 2, false>(a, sm, tw, C::L);
        __syncthreads();
    }
    const int lb = tid / P;
    const int j = tid % P;
#pragma unroll
    for (int v = 0; v < V; v++) {
        const int lo = (v >> 1) * Q + ((v & 1) ? Q - 1 - j : j);
#pragma unroll
        for (int r = 0; r < R; r++)
            a[v * R + r] = sm[sidx<C>(lb, lo | (r << Gl::S0), 0)];
        run_stages<C, C::NG - 1, false>(a, v, lo, tw, C::L);
    }
    if (lb >= nvalid)
        return;
    float2 *oa = reinterpret_cast<float2 *>(d.out + 2 * (line0 + lb) * d.cols);
    float2 *ob = reinterpret_cast<float2 *>(d.out + (2 * (line0 + lb) + 1) * d.cols);
#pragma unroll
    for (int t = 0; t < V / 2; t++) {
#pragma unroll
        for (int r = 0; r < R; r++) {
            const float2 za = a[(2 * t) * R + r];                       // n = t Q + j + M r
            const float2 zb = a[(2 * (V / 2 - 1 - t) + 1) * R + R - 1 - r];   // N - 1 - n
            if (r < R / 2) {
                const int n = t * Q + j + M * r;
                oa[n] = make_float2(za.x * scale, zb.x * scale);
                ob[n] = make_float2(za.y * scale, zb.y * scale);
            } else {
                const int n = C::N - 1 - (t * Q + j + M * r);
                oa[n] = make_float2(zb.x * scale, za.x * scale);
                ob[n] = make_float2(zb.y * scale, za.y * scale);
            }
        }
    }
}

template <class C>
cudaError_t row_idct_launch(const DctIO &d, const float2 *tw, const float2 *post,
                            long long nlines, float scale, cudaStream_t s)
{
    auto k = row_idct_kernel<C>;
    constexpr int bytes = C::SMEM_BYTES;
    if (bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess)
            return e;
    }
    const unsigned grid = (unsigned)((nlines + C::LB - 1) / C::LB);
    k<<<grid, C::T, bytes, s>>>(d, tw, post, dct_rot_table(), nlines, scale);
    return cudaGetLastError();
}

// Inverse column pass, persistent and TMA-fed like the complex column pass
// (natural-order tiles, the next tile's first half prefetched).  Group 0
// gathers the units of idct_pre_units from the tile and pre-rotates them;
// the last group keeps the natural units.  Output row 2n takes v[n] and row
// 2n+1 takes v[N-1-n]: the rows below N/2 of the transformed tile go
// through a staging buffer and one TMA store over the even output rows
// (row stride 2 ld), the others with per-thread stores to the odd rows.
// maps: map (the input, 256-row blocks, box W x 256 x NB), oe (the even
// output rows, box W x BY x NZ as DctCol).
template <class C>
__global__ void __launch_bounds__(C::T, 1) col_idct_tma_kernel(
    const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap oe, float2 *out,
    long long ld, int ntiles, const float2 *__restrict__ tw, const float2 *__restrict__ post,
    const DctRot rot, float scale, int *err, int withhold)
{
    using S = TmaSplit<C>;
    using G0 = Grp<C, 0>;
    using Gl = Grp<C, C::NG - 1>;
    constexpr int HH = 1 << (G0::HB - 1);
    static_assert(C::LB == 1 && C::NG >= 2 && G0::V == 2, "one line block, 2 group-0 units");
    static_assert((C::T >> C::KW) == HH, "threads cover half the group-0 units");
    static_assert((1 << G0::HB) <= S::BOX, "box index must depend on the register only");
    static_assert(S::LATE_BYTES <= (uint32_t)C::E * 4u, "late boxes leave the staging half free");
    extern __shared__ __align__(1024) float2 sm[];
    __shared__ __align__(8) uint64_t bar_early, bar_late;
    const int tid = threadIdx.x;
    int tile = blockIdx.x;
    const float2 *pref = sm + C::E;
    float2 *stw = sm + S::TW_OFF;
    float2 *stage = sm + C::E / 2;
    if (tid == 0) {
        mbar_init(&bar_early, 1);
        mbar_init(&bar_late, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0 && tile < ntiles) {
        mbar_expect_tx(&bar_early, S::TW_BYTES);
        bulk_load(stw, tw, S::TW_BYTES, &bar_early);
        split_issue_early<C>(sm, &map, tile * C::W, &bar_early);
        if (!(withhold && blockIdx.x == 0))   // self-test: the first late half never comes
            split_issue_late<C>(sm, &map, tile * C::W, &bar_late);
    }
    uint32_t parity = 0;
    const int w = tid & (C::W - 1);
    const int h = tid >> C::KW;
    const int h1 = h == 0 ? HH : 2 * HH - h;
    float2 a[C::EPT];
    for (; tile < ntiles; tile += gridDim.x) {
        const int next = tile + gridDim.x;
        const bool ok = mbar_wait_bounded(&bar_early, parity) && mbar_wait_bounded(&bar_late, parity);
        if (__syncthreads_or(ok ? 0 : 1)) {
            if (tid == 0) {
                atomicExch(err, kDevErrTmaTimeout);
                bulk_wait_all();
            }
            mbar_wait_bounded(&bar_early, parity);
            mbar_wait_bounded(&bar_late, parity);
            return;
        }
        parity ^= 1;
#pragma unroll
        for (int v = 0; v < 2; v++) {
            const int hib = v ? h1 : h;
#pragma unroll
            for (int r = 0; r < G0::R; r++) {
                const int top = brev_c(r, G0::G) << G0::HB;   // compile-time
                const int k = top / S::BOX;
                const float2 *bx = k < S::NB ? pref + k * S::BOX_VALS : sm + (k - S::NB) * S::BOX_VALS;
                a[v * G0::R + r] = bx[((top % S::BOX) | hib) * C::W + w];
            }
        }
        idct_pre_units<C>(a, h, post, rot);
#pragma unroll
        for (int v = 0; v < 2; v++)
            run_stages<C, 0, false, true>(a, v, 0, stw, C::L);
        fence_proxy_async_smem();
        if (tid == 0)
            bulk_wait_read_all();   // the previous tile's staging half is free
        __syncthreads();            // both regions have been read
        if (tid == 0 && next < ntiles)
            split_issue_early<C>(sm, &map, next * C::W, &bar_early);
#pragma unroll
        for (int v = 0; v < 2; v++) {
            const int hi = brev_rt(v ? h1 : h, G0::HB);
#pragma unroll
            for (int r = 0; r < G0::R; r++)
                sm[sidx<C>(0, r | (hi << G0::G), w)] = a[v * G0::R + r];
        }
        __syncthreads();
        if constexpr (C::NG >= 3) {
            group_smem<C, 1, false, false, true>(a, sm, stw, C::L);
            __syncthreads();
        }
        if constexpr (C::NG >= 4) {
            group_smem<C, 2, false, false, true>(a, sm, stw, C::L);
            __syncthreads();
        }
        group_last_read<C>(a, sm);
        fence_proxy_async_smem();
        __syncthreads();   // the tile region is free
        if (tid == 0 && next < ntiles)
            split_issue_late<C>(sm, &map, next * C::W, &bar_late);
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
            const int u = tid + v * C::T;
            const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
            run_stages<C, C::NG - 1, false, true>(a, v, lo, stw, C::L);
        }
        // positions below N/2 (r < R/2): staging slot p W + w, one TMA store
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
            const int u = tid + v * C::T;
            const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
#pragma unroll
            for (int r = 0; r < Gl::R / 2; r++) {
                const float2 x = a[v * Gl::R + r];
                stage[(lo + (r << Gl::S0)) * C::W + w] = make_float2(x.x * scale, x.y * scale);
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tma_store_3d(&oe, tile * C::W, 0, 0, stage);
            bulk_commit();
        }
        // the others: odd output rows 2 (N-1-p) + 1
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
            const int u = tid + v * C::T;
            const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
            float2 *dst = out + (long long)tile * C::W + w;
#pragma unroll
            for (int r = Gl::R / 2; r < Gl::R; r++) {
                const int p = lo + (r << Gl::S0);
                const float2 x = a[v * Gl::R + r];
                st_stream(dst + (long long)(2 * (C::N - 1 - p) + 1) * ld,
                          make_float2(x.x * scale, x.y * scale));
            }
        }
    }
    if (tid == 0)
        bulk_wait_all();
}

// ---------------------------------------------------------------------------
// Inverse DCT column pass for columns of 2^(L+1) points over a CTA pair.
// CTA b runs the DIT half of the inverse DFT whose inputs are the spectrum
// positions k = 2m + b (the rows of parity b, one tensor map with twice the
// row pitch).  The pre-rotation pairs k with N - k, which has the same
// parity, so it stays inside the CTA: in local positions m pairs with
// 2^L - m for b = 0 (m = 0 alone, m = 2^(L-1) with itself) and with
// 2^L - 1 - m for b = 1.  A thread takes the group-0 units h and, for b = 0,
// 2^HB - h (unit 0 with 2^(HB-1), both paired within themselves) or, for
// b = 1, 2^HB - 1 - h.  After stages 1..L and the exchange round of stage
// L+1, CTA b holds v[n] and v[n + 2^L] for n in [b 2^(L-1), (b+1) 2^(L-1));
// x[2n] = v[n] and x[2n'+1] = v[N-1-n'] are two contiguous ranges of the
// even and the odd output rows, each staged and stored with one TMA store.
template <class C>
__global__ void __launch_bounds__(C::T, 1) col_idct_pair_kernel(
    const __grid_constant__ CUtensorMap m0, const __grid_constant__ CUtensorMap m1,
    const __grid_constant__ CUtensorMap oe, const __grid_constant__ CUtensorMap oo, int ntiles,
    const float2 *__restrict__ tw, const float2 *__restrict__ post, float scale, int *err,
    int withhold)
{
    namespace cg = cooperative_groups;
    using S = TmaSplit<C>;
    using GC = GroupCol<C, 1>;
    using G0 = Grp<C, 0>;
    using Gl = Grp<C, C::NG - 1>;
    constexpr int N = 2 * C::N;
    constexpr int R = G0::R, HH = 1 << (G0::HB - 1);
    static_assert(G0::V == 2 && (C::T >> C::KW) == HH, "threads cover half the group-0 units");
    extern __shared__ __align__(1024) float2 sm[];
    __shared__ __align__(8) uint64_t bar_early, bar_late, bar_recv;
    __shared__ int lost_flag[2];
    cg::cluster_group cluster = cg::this_cluster();
    const int b = (int)cluster.block_rank();
    const int tid = threadIdx.x;
    const int nclusters = (int)gridDim.x / 2;
    const CUtensorMap *lmap = b == 0 ? &m0 : &m1;
    float2 *stw = sm + S::TW_OFF;
    float2 *recvb = sm;
    float2 *sendb = sm + C::E / 2;
    const uint32_t peer_recv = mapa_shared(smem_addr(recvb), (uint32_t)(b ^ 1));
    const uint32_t peer_bar = mapa_shared(smem_addr(&bar_recv), (uint32_t)(b ^ 1));
    const int w = tid & (C::W - 1);
    const int h = tid >> C::KW;
    const int h1 = b == 0 ? (h == 0 ? HH : 2 * HH - h) : 2 * HH - 1 - h;
    int lost_recv = 0;
    int tile = (int)blockIdx.x / 2;
    if (tid == 0) {
        mbar_init(&bar_early, 1);
        mbar_init(&bar_late, 1);
        mbar_init(&bar_recv, 1);
        fence_mbar_init();
    }
    __syncthreads();
    int n_early = 0, n_late = 0, w_early = 0, w_late = 0;
    if (tile < ntiles) {
        if (tid == 0) {
            mbar_expect_tx(&bar_early, S::TW_BYTES);
            bulk_load(stw, tw, S::TW_BYTES, &bar_early);
            split_issue_early<C>(sm, lmap, tile * C::W, &bar_early);
            if (!(withhold && blockIdx.x == 0))   // self-test: the first late half never comes
                split_issue_late<C>(sm, lmap, tile * C::W, &bar_late);
        }
        n_early = n_late = 1;
    }
    bool lost = false;
    int w_recv = 0;
    float2 a[C::EPT];
    for (; tile < ntiles; tile += nclusters) {
        const int next = tile + nclusters;
        const bool ok = mbar_wait_bounded(&bar_early, (uint32_t)(w_early & 1)) &&
                        mbar_wait_bounded(&bar_late, (uint32_t)(w_late & 1));
        const int lost_here = __syncthreads_or((ok ? 0 : 1) | lost_recv);
        if (tid == 0) {
            if (!lost_recv)
                mbar_arrive_expect_tx(&bar_recv, GC::XBYTES);
            lost_flag[b] = lost_here;
            *cluster.map_shared_rank(lost_flag + b, b ^ 1) = lost_here;
        }
        if (!lost_here) {
            w_early++;
            w_late++;
#pragma unroll
            for (int v = 0; v < 2; v++) {
                const int hib = v ? h1 : h;
#pragma unroll
                for (int r = 0; r < R; r++) {
                    const int top = brev_c(r, G0::G) << G0::HB;   // compile-time
                    const int kb = top / S::BOX;
                    const float2 *bx = kb < S::NB ? sm + C::E + kb * S::BOX_VALS
                                                  : sm + (kb - S::NB) * S::BOX_VALS;
                    a[v * R + r] = bx[((top % S::BOX) | hib) * C::W + w];
                }
            }
            // pre-rotation of the pairs (k, N - k), k = 2 (local position) + b
            float2 yk, yp;
            if (b == 1 || h != 0) {
#pragma unroll
                for (int r = 0; r < R; r++) {
                    const int rc = r ^ (R - 1);
                    if (brev_c(r, G0::G) < R / 2) {
                        const int ks = 2 * ((brev_c(r, G0::G) << G0::HB) + h) + b;
                        idct_pre(a[r], a[R + rc], __ldg(post + ks), yk, yp);
                        a[r] = yk;
                        a[R + rc] = yp;
                    } else {
                        const int ks = 2 * ((brev_c(rc, G0::G) << G0::HB) + h1) + b;
                        idct_pre(a[R + rc], a[r], __ldg(post + ks), yk, yp);
                        a[R + rc] = yk;
                        a[r] = yp;
                    }
                }
            } else {
                // b = 0, h = 0: unit 0 (positions brev(r) 2^HB) pairs b' with
                // R - b' (k = 0 alone, k = N/2 with itself); unit HH pairs r
                // with r ^ (R - 1)
#pragma unroll
                for (int bb = 1; bb < R / 2; bb++) {
                    const int r = brev_c(bb, G0::G), r2 = brev_c(R - bb, G0::G);
                    idct_pre(a[r], a[r2], __ldg(post + 2 * (bb << G0::HB)), yk, yp);
                    a[r] = yk;
                    a[r2] = yp;
                }
                constexpr int r8 = brev_c(R / 2, G0::G);
                idct_pre(a[r8], a[r8], __ldg(post + N / 2), yk, yp);
                a[r8] = yk;
#pragma unroll
                for (int r = 0; r < R; r++) {
                    if (brev_c(r, G0::G) >= R / 2)
                        continue;
                    const int rc = r ^ (R - 1);
                    idct_pre(a[R + r], a[R + rc],
                             __ldg(post + 2 * ((brev_c(r, G0::G) << G0::HB) + HH)), yk, yp);
                    a[R + r] = yk;
                    a[R + rc] = yp;
                }
            }
#pragma unroll
            for (int v = 0; v < 2; v++)
                run_stages<C, 0, false, true>(a, v, 0, stw, C::L);
            fence_proxy_async_smem();
            if (tid == 0)
                bulk_wait_read_all();   // the previous tile's stores have read the staging
            __syncthreads();
            if (tid == 0 && next < ntiles)
                split_issue_early<C>(sm, lmap, next * C::W, &bar_early);
            if (next < ntiles)
                n_early++;
#pragma unroll
            for (int v = 0; v < 2; v++) {
                const int hi = brev_rt(v ? h1 : h, G0::HB);
#pragma unroll
                for (int r = 0; r < R; r++)
                    sm[sidx<C>(0, r | (hi << G0::G), w)] = a[v * R + r];
            }
            __syncthreads();
            group_smem<C, 1, false, false, true>(a, sm, stw, C::L);
            __syncthreads();
            group_last_read<C>(a, sm);
            __syncthreads();   // the tile region is free
        }
        cluster_arrive_release();   // A0
        float2 wk[16];
        if (!lost_here) {
#pragma unroll
            for (int v = 0; v < Gl::V; v++) {
                const int u = tid + v * C::T;
                const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
                run_stages<C, C::NG - 1, false, true>(a, v, lo, stw, C::L);
            }
            group_round_send<C, 0>(a, sendb, b);
            fence_proxy_async_smem();
        }
        __syncthreads();
        group_round_twiddles<C, 0>(wk, tw, b * (Gl::R / 2));
        cluster_wait_acquire();
        if (lost_flag[0] | lost_flag[1]) {
            lost = true;
            break;
        }
        if (tid == 0)
            bulk_copy_to_peer(peer_recv, sendb, GC::XBYTES, peer_bar);
        lost_recv = mbar_wait_bounded(&bar_recv, (uint32_t)(w_recv & 1)) ? 0 : 1;
        if (!lost_recv)
            w_recv++;
        cluster_arrive_release();   // B0: the partner's send buffer has been read
        // stage L+1: a[t 16 + v 8 + i] = v[n + 2^L t], n = lo_v + 2^S0 (8b + i)
        group_round_compute<C, 0>(a, recvb, wk, b);
        fence_proxy_async_smem();
        __syncthreads();   // the receive buffer has been read
        if (tid == 0 && next < ntiles)
            split_issue_late<C>(sm, lmap, next * C::W, &bar_late);
        if (next < ntiles)
            n_late++;
        cluster_wait_acquire();   // B0: this CTA's send buffer is free for staging
        // x[2n] = v[n]: even rows n in [b 2^(L-1), ...), one store; then
        // x[2j+1] = v[N-1-j] = v[n + 2^L] for j = 2^L - 1 - n: odd rows
        // j in [2^(L-1) (1 - b), ...), staged in reverse
#pragma unroll
        for (int t = 0; t < 2; t++) {
            if (t == 1) {
                if (tid == 0)
                    bulk_wait_read_all();
                __syncthreads();
            }
#pragma unroll
            for (int v = 0; v < Gl::V; v++) {
                const int lo = ((tid + v * C::T) >> C::KW) & ((1 << Gl::S0) - 1);
#pragma unroll
                for (int i = 0; i < 8; i++) {
                    const int off = (i << Gl::S0) | lo;   // n - b 2^(L-1)
                    const int slot = t == 0 ? off : (C::N / 2 - 1) - off;
                    const float2 x = a[t * 16 + v * 8 + i];
                    sendb[slot * C::W + w] = make_float2(x.x * scale, x.y * scale);
                }
            }
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                if (t == 0)
                    tma_store_3d(&oe, tile * C::W, 0, b * (C::N / 2 / S::BOX), sendb);
                else
                    tma_store_3d(&oo, tile * C::W, 0, (1 - b) * (C::N / 2 / S::BOX), sendb);
                bulk_commit();
            }
        }
    }

    if (__syncthreads_or((lost || lost_recv) ? 1 : 0)) {
        if (tid == 0)
            atomicExch(err, kDevErrTmaTimeout);
        if (n_early > w_early)
            mbar_wait_bounded(&bar_early, (uint32_t)(w_early & 1));
        if (n_late > w_late)
            mbar_wait_bounded(&bar_late, (uint32_t)(w_late & 1));
        if (lost_recv)
            mbar_wait_bounded(&bar_recv, (uint32_t)(w_recv & 1));
    }
    if (tid == 0)
        bulk_wait_all();
}

// The pair kernel for inverse DCT columns of 8192 points when the image
// allows it; cudaErrorNotSupported otherwise.
cudaError_t idct_col_pair_launch(const DctIO &d, const float2 *tw, const float2 *post,
                                 float scale, int *err, int withhold, cudaStream_t s)
{
    using C = LineCfg<12, 2, 0, 32>;
    using S = TmaSplit<C>;
    using D = DctPair<C>;
    const long long cc = d.cols / 2;
    if (!err || d.rows != 2 * C::N || cc % C::W != 0 || (reinterpret_cast<uintptr_t>(d.in) & 15) ||
        (reinterpret_cast<uintptr_t>(d.out) & 15) || (reinterpret_cast<uintptr_t>(tw) & 15) ||
        (cc * 8) % 16 != 0 || !tensor_maps_available())
        return cudaErrorNotSupported;
    const float2 *in = reinterpret_cast<const float2 *>(d.in);
    float2 *out = reinterpret_cast<float2 *>(d.out);
    CUtensorMap lm[2], oe, oo;
    for (int b = 0; b < 2; b++)
        if (!encode_col_map(&lm[b], in + b * cc, C::N, (int)cc, 2 * cc, C::W, S::BOX, S::NB))
            return cudaErrorNotSupported;
    if (!encode_col_map(&oe, out, C::N, (int)cc, 2 * cc, C::W, S::BOX, D::NBH) ||
        !encode_col_map(&oo, out + cc, C::N, (int)cc, 2 * cc, C::W, S::BOX, D::NBH))
        return cudaErrorNotSupported;
    auto k = col_idct_pair_kernel<C>;
    constexpr int SMEM = S::SMEM_BYTES;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(C::T);
    cfg.dynamicSmemBytes = SMEM;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    static DeviceCache pairs;
    const int dev = device_current();
    if (!pairs.get(dev)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess)
            return e;
        cfg.gridDim = dim3((unsigned)(2 * (device_sm_count() / 2)));
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
        if (e != cudaSuccess)
            return e;
        pairs.set(dev, n > 0 ? n : 1);
    }
    const int ntiles = (int)(cc / C::W);
    const int np = pairs.get(dev) < ntiles ? pairs.get(dev) : ntiles;
    cfg.gridDim = dim3((unsigned)(2 * np));
    return cudaLaunchKernelEx(&cfg, k, lm[0], lm[1], oe, oo, ntiles, tw, post, scale, err,
                              withhold);
}

template <class C>
cudaError_t idct_col_tma_launch(const DctIO &d, const float2 *tw, const float2 *post, float scale,
                                int *err, int withhold, cudaStream_t s)
{
    using S = TmaSplit<C>;
    using D = DctCol<C>;
    const long long cc = d.cols / 2;
    if (!err || cc % C::W != 0 || (reinterpret_cast<uintptr_t>(d.in) & 15) ||
        (reinterpret_cast<uintptr_t>(d.out) & 15) || (reinterpret_cast<uintptr_t>(tw) & 15) ||
        (cc * 8) % 16 != 0 || !tensor_maps_available())
        return cudaErrorNotSupported;
    const float2 *in = reinterpret_cast<const float2 *>(d.in);
    float2 *out = reinterpret_cast<float2 *>(d.out);
    CUtensorMap map, oe;
    if (!encode_map_xyz(&map, in, cc, 256, C::N / 256, cc, cc * 256, C::W, S::BOX, S::NB) ||
        !encode_map_xyz(&oe, out, cc, D::BY, D::NZ, 2 * cc, 2 * cc * D::BY, C::W, D::BY, D::NZ))
        return cudaErrorNotSupported;
    auto k = col_idct_tma_kernel<C>;
    constexpr int SMEM = S::SMEM_BYTES;
    static DeviceCache attr_set;
    const int dev = device_current();
    if (!attr_set.get(dev)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess)
            return e;
        attr_set.set(dev, 1);
    }
    const int ntiles = (int)(cc / C::W);
    int grid = device_sm_count();
    if (grid > ntiles)
        grid = ntiles;
    k<<<grid, C::T, SMEM, s>>>(map, oe, out, cc, ntiles, tw, post, dct_rot_table(), scale, err,
                               withhold);
    return cudaGetLastError();
}

template <int L>
cudaError_t dct_dispatch(bool row, bool inverse, const DctIO &d, const float2 *tw,
                         const float2 *post, float scale, int *err, int withhold, cudaStream_t s)
{
    if (withhold) {   // the self-test runs on the TMA-fed column kernels only
        if (row)
            return cudaErrorNotSupported;
        if constexpr (L == 12)
            return inverse ? idct_col_tma64_launch(d, tw, post, scale, err, 1, s)
                           : dct_col_tma64_launch(d, tw, post, scale, err, 1, s);
        if constexpr (L == 11 || L == 12)
            return inverse ? idct_col_tma_launch<LineCfg<L, col_kw(L), 0, 32>>(d, tw, post, scale,
                                                                                err, 1, s)
                           : dct_col_tma_launch<LineCfg<L, col_kw(L), 0, 32>>(d, tw, post, scale,
                                                                               err, 1, s);
        if constexpr (L == 13)
            return inverse ? idct_col_pair_launch(d, tw, post, scale, err, 1, s)
                           : dct_col_pack_launch<1>(d, tw, post, scale, err, 1, s);
        if constexpr (L == 14) {
            if (inverse)
                return idct_col_quad_launch(d, tw, post, scale, err, 1, s);
            const cudaError_t e = dct_col_pack_launch<2>(d, tw, post, scale, err, 1, s);
            return e != cudaErrorNotSupported ? e
                                              : dct_col_quad_launch(d, tw, post, scale, err, 1, s);
        }
        return cudaErrorNotSupported;
    }
    if (inverse) {
        if (row) {
            if constexpr (L >= 10)
                return row_idct_launch<LineCfg<L, 0, row_kb(L), 32>>(d, tw, post, d.rows / 2,
                                                                     scale, s);
            return idct_launch<LineCfg<L, 0, row_kb(L)>, true>(d, tw, post, d.rows / 2, scale, s);
        }
        if constexpr (L == 12) {
            const cudaError_t e = idct_col_tma64_launch(d, tw, post, scale, err, 0, s);
            if (e != cudaErrorNotSupported)
                return e;
        }
        if constexpr (L == 11) {
            const cudaError_t e =
                idct_col_tma_launch<LineCfg<L, col_kw(L), 0, 32>>(d, tw, post, scale, err, 0, s);
            if (e != cudaErrorNotSupported)
                return e;
        }
        if constexpr (L == 13) {
            const cudaError_t e = idct_col_pair_launch(d, tw, post, scale, err, 0, s);
            if (e != cudaErrorNotSupported)
                return e;
        }
        if constexpr (L == 14) {
            const cudaError_t e = idct_col_quad_launch(d, tw, post, scale, err, 0, s);
            if (e != cudaErrorNotSupported)
                return e;
        }
        return idct_launch<LineCfg<L, col_kw(L), 0>, false>(d, tw, post, d.cols / 2, scale, s);
    }
    if (row) {
        if constexpr (L >= 10)
            return row_dct_launch<LineCfg<L, 0, row_kb(L), 32>>(d, tw, post, d.rows / 2, scale, s);
        return dct_launch<LineCfg<L, 0, row_kb(L)>, true>(d, tw, post, d.rows / 2, scale, s);
    }
    if constexpr (L == 12) {
        const cudaError_t e = dct_col_tma64_launch(d, tw, post, scale, err, 0, s);
        if (e != cudaErrorNotSupported)
            return e;
    }
    if constexpr (L == 11) {
        const cudaError_t e =
            dct_col_tma_launch<LineCfg<L, col_kw(L), 0, 32>>(d, tw, post, scale, err, 0, s);
        if (e != cudaErrorNotSupported)
            return e;
    }
    if constexpr (L == 13 || L == 14) {
        const cudaError_t e = dct_col_pack_launch<L - 12>(d, tw, post, scale, err, 0, s);
        if (e != cudaErrorNotSupported)
            return e;
    }
    if constexpr (L == 14) {
        const cudaError_t e = dct_col_quad_launch(d, tw, post, scale, err, 0, s);
        if (e != cudaErrorNotSupported)
            return e;
    }
    return dct_launch<LineCfg<L, col_kw(L), 0>, false>(d, tw, post, d.cols / 2, scale, s);
}

}  // namespace

cudaError_t launch_dct_pass(bool row, bool inverse, int L, const float *in, float *out, int rows,
                            int cols, const float2 *tw, const float2 *post, float scale, int *err,
                            cudaStream_t s, int withhold)
{
    const DctIO d{in, out, rows, cols};
    switch (L) {
    case 1: return dct_dispatch<1>(row, inverse, d, tw, post, scale, err, withhold, s);
    case 2: return dct_dispatch<2>(row, inverse, d, tw, post, scale, err, withhold, s);
    case 3: return dct_dispatch<3>(row, inverse, d, tw, post, scale, err, withhold, s);
    case 4: return dct_dispatch<4>(row, inverse, d, tw, post, scale, err, withhold, s);
    case 5: return dct_dispatch<5>(row, inverse, d, tw, post, scale, err, withhold, s);
    case 6: return dct_dispatch<6>(row, inverse, d, tw, post, scale, err, withhold, s);
    case 7: return dct_dispatch<7>(row, inverse, d, tw, post, scale, err, withhold, s);
    case 8: return dct_dispatch<8>(row, inverse, d, tw, post, scale, err, withhold, s);
    case 9: return dct_dispatch<9>(row, inverse, d, tw, post, scale, err, withhold, s);
    case 10: return dct_dispatch<10>(row, inverse, d, tw, post, scale, err, withhold, s);
    case 11: return dct_dispatch<11>(row, inverse, d, tw, post, scale, err, withhold, s);
    case 12: return dct_dispatch<12>(row, inverse, d, tw, post, scale, err, withhold, s);
    case 13: return dct_dispatch<13>(row, inverse, d, tw, post, scale, err, withhold, s);
    case 14: return dct_dispatch<14>(row, inverse, d, tw, post, scale, err, withhold, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fft2d
