// dct.cu -- the 2D discrete cosine transform (DCT-II) of real images on the
// radix-2 passes: Section 5 names the DCT among the transforms the method
// extends to, without giving an algorithm.  This file uses the well-known
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

// The outputs at k and k' = (N - k) mod N of the two real lines of a
// complex line, from Z[k] and Z[k'] (see the header); (c, s) belong to k.
__device__ __forceinline__ void dct_pair(float2 zk, float2 zp, float2 cs, float scale,
                                         float2 &xk, float2 &xp)
{
    const float c = cs.x * 0.5f * scale, s = cs.y * 0.5f * scale;
    const float sr = zk.x + zp.x, dr = zp.x - zk.x;   // Zr[k] + Zr[k'], Zr[k'] - Zr[k]
    const float si = zk.y + zp.y, di = zk.y - zp.y;   // Zi[k] + Zi[k'], Zi[k] - Zi[k']
    xk = make_float2(c * sr + s * di, c * si + s * dr);     // (X_a[k], X_b[k])
    xp = make_float2(s * sr - c * di, s * si - c * dr);     // (X_a[k'], X_b[k'])
}

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

template <int L>
cudaError_t dct_dispatch(bool row, const DctIO &d, const float2 *tw, const float2 *post,
                         float scale, cudaStream_t s)
{
    if (row)
        return dct_launch<LineCfg<L, 0, row_kb(L)>, true>(d, tw, post, d.rows / 2, scale, s);
    return dct_launch<LineCfg<L, col_kw(L), 0>, false>(d, tw, post, d.cols / 2, scale, s);
}

}  // namespace

cudaError_t launch_dct_pass(bool row, int L, const float *in, float *out, int rows, int cols,
                            const float2 *tw, const float2 *post, float scale, cudaStream_t s)
{
    const DctIO d{in, out, rows, cols};
    switch (L) {
    case 1: return dct_dispatch<1>(row, d, tw, post, scale, s);
    case 2: return dct_dispatch<2>(row, d, tw, post, scale, s);
    case 3: return dct_dispatch<3>(row, d, tw, post, scale, s);
    case 4: return dct_dispatch<4>(row, d, tw, post, scale, s);
    case 5: return dct_dispatch<5>(row, d, tw, post, scale, s);
    case 6: return dct_dispatch<6>(row, d, tw, post, scale, s);
    case 7: return dct_dispatch<7>(row, d, tw, post, scale, s);
    case 8: return dct_dispatch<8>(row, d, tw, post, scale, s);
    case 9: return dct_dispatch<9>(row, d, tw, post, scale, s);
    case 10: return dct_dispatch<10>(row, d, tw, post, scale, s);
    case 11: return dct_dispatch<11>(row, d, tw, post, scale, s);
    case 12: return dct_dispatch<12>(row, d, tw, post, scale, s);
    case 13: return dct_dispatch<13>(row, d, tw, post, scale, s);
    case 14: return dct_dispatch<14>(row, d, tw, post, scale, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fft2d
