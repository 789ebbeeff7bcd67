// kernels_h16.cu -- half2 storage with a power-of-two exponent per line:
// the row and column passes (FP32 butterflies and exchanges, half2 global
// traffic) and the pack / unpack conversions between complex64 and that
// format.
#include <type_traits>

#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include "col_group.cuh"
#include "col_h16.cuh"
#include "line_fft.cuh"
#include "passes.h"

namespace fft2d {

namespace {

template <class C, bool ROW, bool GENERIC, int IA>
cudaError_t h16_launch_axis(const H16PassArgs &a, cudaStream_t s)
{
    using IO = StoreH16T<IA>;
    auto k = ROW ? row_pass_kernel<C, GENERIC, IO> : col_pass_kernel<C, GENERIC, IO>;
    const int bytes = LineSmem<C, ROW, IO>::BYTES;
    if (bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess)
            return e;
    }
    const int lines = ROW ? a.rows : a.cols;
    const int per = ROW ? C::LB : C::W;
    const unsigned grid = (unsigned)((lines + per - 1) / per);
    IO io{a.in, a.out, a.in_exp, a.in_axis, a.out_exp};
    k<<<grid, C::T, bytes, s>>>(io, a.tw, lines, a.ld, a.scale, a.nst);
    return cudaGetLastError();
}

// The input's exponent axis becomes a compile-time choice, so a line's
// exponent is loaded once per unit where it runs along the line.
template <class C, bool ROW, bool GENERIC>
cudaError_t h16_launch(const H16PassArgs &a, cudaStream_t s)
{
    return a.in_axis == 0 ? h16_launch_axis<C, ROW, GENERIC, 0>(a, s)
                          : h16_launch_axis<C, ROW, GENERIC, 1>(a, s);
}

// 3D tensor map over a half2 image (4-byte elements): x = column, y = row
// within a block of 256 rows, z = block; box W x box_y x box_z.
bool encode_h16_col_map(CUtensorMap *map, const __half2 *base, int rows, int cols, long long ld,
                        int W, int box_y, int box_z)
{
    static PFN_cuTensorMapEncodeTiled_v12000 enc = [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        return static_cast<PFN_cuTensorMapEncodeTiled_v12000>(nullptr);
    }();
    if (!enc || (reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 4) & 15) || rows % 256 != 0)
        return false;
    cuuint64_t dims[3] = {(cuuint64_t)cols, 256, (cuuint64_t)(rows / 256)};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 4, (cuuint64_t)ld * 4 * 256};
    cuuint32_t box[3] = {(cuuint32_t)W, (cuuint32_t)box_y, (cuuint32_t)box_z};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<__half2 *>(base), dims, strides,
               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// The persistent TMA-fed half2 column pass (col_h16.cuh) for columns of
// 2^L rows in 4-column tiles.  Returns cudaErrorNotSupported (nothing
// launched) when the buffers or shape cannot feed it: the caller then takes
// another kernel.
template <int L>
cudaError_t h16_launch_col_tma(const H16PassArgs &a, cudaStream_t s)
{
    using C = LineCfg<L, 2, 0, 64, 6>;   // two groups of 6 stages, as the complex64 pass
    using H = H16Col<C>;
    if (a.in_axis != 0 || a.nst != L || !a.err || a.cols % C::W != 0 ||
        (reinterpret_cast<uintptr_t>(a.tw) & 15))
        return cudaErrorNotSupported;
    CUtensorMap map, omap;
    if (!encode_h16_col_map(&map, a.in, a.rows, a.cols, a.ld, C::W, H::BOX, H::NB) ||
        !encode_h16_col_map(&omap, a.out, a.rows, a.cols, a.ld, C::W, H::BOX, H::NBOX))
        return cudaErrorNotSupported;
    auto k = col_h16_tma_kernel<C>;
    static DeviceCache ready;
    const int d = device_current();
    if (!ready.get(d)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             H::SMEM_BYTES);
        if (e != cudaSuccess)
            return e;
        ready.set(d, 1);
    }
    const int ntiles = a.cols / C::W;
    int grid = device_sm_count();
    if (grid > ntiles)
        grid = ntiles;
    k<<<grid, C::T, H::SMEM_BYTES, s>>>(map, omap, a.tw, a.in_exp, a.out_exp, a.cols, a.scale,
                                        a.err);
    return cudaGetLastError();
}

// Columns of 2^(12+CL) rows on a cluster of 2^CL CTAs (col_group_l2_kernel,
// half2 storage): the 4096-row engine on each CTA's rows, the last CL stages
// after an exchange through a stream-ordered scratch block in L2.
// cudaErrorNotSupported (nothing launched) when the buffers or shape cannot
// feed it.
template <int CL>
cudaError_t h16_launch_col_group(const H16PassArgs &a, cudaStream_t s)
{
    // local engine: two groups of 6 stages for the pair (0.484 against 0.510
    // ms per 8192^2 transform), three of 4 for four CTAs (2.47 against 2.53
    // ms per 16384^2 transform; 2.33 against 2.44 ms with 16-byte exchange
    // slots)
    using C = typename std::conditional<CL == 1, LineCfg<12, 2, 0, 64, 6>, LineCfg<12, 2, 0, 32>>::type;
    using GH = GroupH16<C>;
    using GC = GroupCol<C, CL>;
    constexpr int CS = 1 << CL;
    if (a.in_axis != 0 || a.nst != 12 + CL || !a.err || a.cols % C::W != 0 ||
        a.rows != (C::N << CL) || (reinterpret_cast<uintptr_t>(a.tw) & 15))
        return cudaErrorNotSupported;
    CUtensorMap m[4], om;
    for (int r = 0; r < CS; r++)
        if (!encode_h16_col_map(&m[r], a.in + r * a.ld, a.rows / CS, a.cols, CS * a.ld, C::W,
                                GH::BOX, GH::NB))
            return cudaErrorNotSupported;
    for (int r = CS; r < 4; r++)
        m[r] = m[0];
    if (!encode_h16_col_map(&om, a.out, a.rows, a.cols, a.ld, C::W, GH::BOX, GC::OUT_BOX_Z))
        return cudaErrorNotSupported;
    auto k = col_group_l2_kernel<C, CL, true>;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3(C::T);
    cfg.dynamicSmemBytes = GH::SMEM_BYTES;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    static DeviceCache groups;
    const int d = device_current();
    if (!groups.get(d)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             GH::SMEM_BYTES);
        if (e != cudaSuccess)
            return e;
        cfg.gridDim = dim3((unsigned)(CS * (device_sm_count() / CS)));
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
        if (e != cudaSuccess)
            return e;
        groups.set(d, n > 0 ? n : 1);
    }
    const int ntiles = a.cols / C::W;
    const int ng = groups.get(d) < ntiles ? groups.get(d) : ntiles;
    void *xbuf = nullptr;
    cudaError_t e = scratch_take(&xbuf, (size_t)ng * GC::L2_SCRATCH_VALS * sizeof(float2), s);
    if (e != cudaSuccess)
        return e;
    cfg.gridDim = dim3((unsigned)(CS * ng));
    e = cudaLaunchKernelEx(&cfg, k, m[0], m[1], m[2], m[3], om, a.tw, a.cols, a.scale, a.err, 0,
                           static_cast<float2 *>(xbuf), GroupIO{a.in_exp, a.out_exp});
    const cudaError_t f = cudaFreeAsync(xbuf, s);
    return e != cudaSuccess ? e : f;
}

template <int L>
cudaError_t h16_dispatch(bool row, const H16PassArgs &a, cudaStream_t s)
{
    if (row) {
        if constexpr (L >= 13) {
            // rows of 8192 and 16384 points: groups of 5 stages, 32 values a
            // thread (three groups instead of four), as for complex64
            using C5 = LineCfg<L, 0, 0, 32, 5>;
            return h16_launch<C5, true, false>(a, s);
        } else {
            using C = LineCfg<L, 0, row_kb(L), 16>;
            return a.rows % C::LB ? h16_launch<C, true, true>(a, s)
                                  : h16_launch<C, true, false>(a, s);
        }
    }
    using C = LineCfg<L, col_kw(L), 0>;
    if constexpr (L == 12) {
        const cudaError_t e = h16_launch_col_tma<L>(a, s);
        if (e != cudaErrorNotSupported)
            return e;
    }
    if constexpr (L == 13 || L == 14) {
        const cudaError_t e = h16_launch_col_group<L - 12>(a, s);
        if (e != cudaErrorNotSupported)
            return e;
    }
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
