// kernels_h16.cu -- half2 storage with a power-of-two exponent per line:
// the row and column passes (FP32 butterflies and exchanges, half2 global
// traffic) and the pack / unpack conversions between complex64 and that
// format.
#include <cuda_fp16.h>

#include "line_fft.cuh"
#include "passes.h"

namespace fft2d {

namespace {

template <class C, bool ROW, bool GENERIC>
cudaError_t h16_launch(const H16PassArgs &a, cudaStream_t s)
{
    auto k = ROW ? row_pass_kernel<C, GENERIC, StoreH16> : col_pass_kernel<C, GENERIC, StoreH16>;
    const int bytes = LineSmem<C, ROW, StoreH16>::BYTES;
    if (bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess)
            return e;
    }
    const int lines = ROW ? a.rows : a.cols;
    const int per = ROW ? C::LB : C::W;
    const unsigned grid = (unsigned)((lines + per - 1) / per);
    StoreH16 io{a.in, a.out, a.in_exp, a.in_axis, a.out_exp};
    k<<<grid, C::T, bytes, s>>>(io, a.tw, lines, a.ld, a.scale, a.nst);
    return cudaGetLastError();
}

template <int L>
cudaError_t h16_dispatch(bool row, const H16PassArgs &a, cudaStream_t s)
{
    if (row) {
        // 8192-point rows: 32 values per thread (256 threads), as for complex64
        using C = LineCfg<L, 0, row_kb(L), L == 13 ? 32 : 16>;
        return a.rows % C::LB ? h16_launch<C, true, true>(a, s) : h16_launch<C, true, false>(a, s);
    }
    using C = LineCfg<L, col_kw(L), 0>;
    if constexpr (L >= 12) {
        // from 4096 rows the single-CTA tile would be 2 or fewer columns
        // wide (8 bytes of half2 per row): split 8-column tiles over a
        // cluster of 2, 4 or 8 CTAs instead (32-byte row segments)
        using CC = ClusterColCfg<L, 3, L - 11>;
        if (a.cols % CC::W == 0) {
            StoreH16 io{a.in, a.out, a.in_exp, a.in_axis, a.out_exp};
            return launch_cluster_kernel<CC, StoreH16>(io, a.tw, a.cols, a.ld, a.scale, a.nst, s);
        }
    }
    return a.cols % C::W ? h16_launch<C, false, true>(a, s) : h16_launch<C, false, false>(a, s);
}

// complex64 -> half2 + one exponent per row (the pass exponent rule: the
// row's largest component magnitude M = f 2^k gives e = k - 14).
__global__ void h16_pack_kernel(const float2 *in, __half2 *out, int *exp_rows, int cols)
{
    __shared__ int smax;
    const long long row = blockIdx.x;
    const float2 *src = in + row * cols;
    if (threadIdx.x == 0)
        smax = 0;
    __syncthreads();
    float m = 0.f;
    for (int i = threadIdx.x; i < cols; i += blockDim.x) {
        const float2 v = src[i];
        m = fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    atomicMax(&smax, __float_as_int(m));
    __syncthreads();
    const int e = line_exponent(__int_as_float(smax));
    const float f = pow2f(-e);
    for (int i = threadIdx.x; i < cols; i += blockDim.x) {
        const float2 v = src[i];
        out[row * cols + i] = __floats2half2_rn(v.x * f, v.y * f);
    }
    if (threadIdx.x == 0)
        exp_rows[row] = e;
}

__global__ void h16_unpack_kernel(const __half2 *in, const int *exps, int axis, float2 *out,
                                  int rows, int cols)
{
    const long long n = (long long)rows * cols;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const long long r = k / cols, c = k - r * cols;
        const float f = pow2f(exps[axis == 0 ? r : c]);
        const float2 q = __half22float2(in[k]);
        out[k] = make_float2(q.x * f, q.y * f);
    }
}

}  // namespace

cudaError_t launch_pass_h16(bool row, int L, const H16PassArgs &a, cudaStream_t s)
{
    switch (L) {
    case 1: return h16_dispatch<1>(row, a, s);
    case 2: return h16_dispatch<2>(row, a, s);
    case 3: return h16_dispatch<3>(row, a, s);
    case 4: return h16_dispatch<4>(row, a, s);
    case 5: return h16_dispatch<5>(row, a, s);
    case 6: return h16_dispatch<6>(row, a, s);
    case 7: return h16_dispatch<7>(row, a, s);
    case 8: return h16_dispatch<8>(row, a, s);
    case 9: return h16_dispatch<9>(row, a, s);
    case 10: return h16_dispatch<10>(row, a, s);
    case 11: return h16_dispatch<11>(row, a, s);
    case 12: return h16_dispatch<12>(row, a, s);
    case 13: return h16_dispatch<13>(row, a, s);
    case 14: return h16_dispatch<14>(row, a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_h16_pack(const float2 *in, __half2 *out, int *exp_rows, int rows, int cols,
                            cudaStream_t s)
{
    h16_pack_kernel<<<rows, 256, 0, s>>>(in, out, exp_rows, cols);
    return cudaGetLastError();
}

cudaError_t launch_h16_unpack(const __half2 *in, const int *exps, int axis, float2 *out,
                              int rows, int cols, cudaStream_t s)
{
    const long long n = (long long)rows * cols;
    long long blocks = (n + 255) / 256;
    if (blocks > 4096)
        blocks = 4096;
    h16_unpack_kernel<<<(unsigned)blocks, 256, 0, s>>>(in, exps, axis, out, rows, cols);
    return cudaGetLastError();
}

}  // namespace fft2d
