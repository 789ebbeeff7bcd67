// kernels_col.cu -- column pass instantiations: every column of an image is a
// line of rows = 2^L points spaced one row pitch apart; a CTA owns a tile of
// W adjacent whole columns, so each global access reads or writes W*8
// contiguous bytes of a row and the whole column stays on chip.
#include <cudaTypedefs.h>

#include <mutex>

#include "line_fft.cuh"
#include "passes.h"

namespace fft2d {

namespace {

constexpr int kMaxDev = 64;

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

int current_device() { return device_current(); }
int sm_count() { return device_sm_count(); }

}  // namespace

int device_current()
{
    int d = 0;
    cudaGetDevice(&d);
    return d < 0 || d >= kMaxDev ? 0 : d;
}

int device_sm_count()
{
    static int cache[kMaxDev] = {};
    const int d = device_current();
    if (!cache[d]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d);
        cache[d] = n > 0 ? n : 1;
    }
    return cache[d];
}

// 2^14 values (128 KB of shared memory) per CTA from 1024-point columns up;
// 16 to 64 columns per CTA below.
static constexpr int col_kw(int L)
{
    return L >= 10 ? 14 - L : (13 - L < 4 ? 4 : (13 - L > 6 ? 6 : 13 - L));
}

int col_width(int L) { return 1 << col_kw(L); }

// One CTA waits, with the same bounded wait as the TMA pipeline, on an
// mbarrier phase that nothing completes, then records the timeout.
__global__ void selftest_timeout_kernel(int *err, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int lost = mbar_wait_bounded(&bar, 0, limit_ns) ? 0 : 1;
    if (__syncthreads_or(lost) && threadIdx.x == 0)
        atomicExch(err, kDevErrTmaTimeout);
}

cudaError_t launch_selftest_timeout(int *err, cudaStream_t s)
{
    selftest_timeout_kernel<<<1, 32, 0, s>>>(err, 20000000ull);   // 20 ms
    return cudaGetLastError();
}

template <int L, bool GENERIC>
static cudaError_t col_launch(const PassArgs &a, cudaStream_t s)
{
    using C = LineCfg<L, col_kw(L), 0>;
    auto k = col_pass_kernel<C, GENERIC>;
    const int dev_bytes = C::SMEM_BYTES;
    if (dev_bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             dev_bytes);
        if (e != cudaSuccess)
            return e;
    }
    const unsigned grid = (unsigned)((a.cols + C::W - 1) / C::W);
    k<<<grid, C::T, dev_bytes, s>>>(a.in, a.out, a.tw, a.cols, a.ld, a.scale, a.nst);
    return cudaGetLastError();
}

// Persistent TMA-fed variant (see col_tma_kernel): whole tiles only, input
// 16-byte aligned, row pitch a multiple of 16 bytes.
// Values per thread of the TMA column kernel: 32 for tiles of 2^14 values
// (512 threads of up to 128 registers), 16 below.
static constexpr int col_tma_ept(int L) { return L >= 10 ? 32 : 16; }

template <int L>
static cudaError_t col_launch_tma(const PassArgs &a, cudaStream_t s, bool *used)
{
    using C = LineCfg<L, col_kw(L), 0, col_tma_ept(L)>;
    *used = false;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || (reinterpret_cast<uintptr_t>(a.in) & 15) || ((a.ld * 8) & 15))
        return cudaSuccess;
    CUtensorMap map;
    const int box_rows = C::N < 256 ? C::N : 256;
    cuuint64_t dims[2] = {(cuuint64_t)a.cols, (cuuint64_t)a.rows};
    cuuint64_t strides[1] = {(cuuint64_t)a.ld * 8};
    cuuint32_t box[2] = {(cuuint32_t)C::W, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<float2 *>(a.in), dims,
                     strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return cudaSuccess;   // not expressible as a tensor map: plain kernel
    auto k = col_tma2_kernel<C>;
    constexpr int SMEM = TmaSplit<C>::SMEM_BYTES;
    static int occ[kMaxDev] = {};
    const int d = current_device();
    if (!occ[d]) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SMEM);
        if (e != cudaSuccess)
            return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, C::T, SMEM);
        if (e != cudaSuccess)
            return e;
        occ[d] = o > 0 ? o : 1;
    }
    const int ntiles = a.cols / C::W;
    int grid = sm_count() * occ[d];
    if (grid > ntiles)
        grid = ntiles;
    k<<<grid, C::T, SMEM, s>>>(map, a.out, a.tw, a.cols, a.ld, a.scale, a.err);
    *used = true;
    return cudaGetLastError();
}

template <int L>
static cudaError_t col_dispatch(const PassArgs &a, cudaStream_t s)
{
    const bool generic = a.partial || a.cols < col_width(L);
    if constexpr (L >= 9 && L <= 12) {
        if (!generic && a.err) {
            bool used = false;
            cudaError_t e = col_launch_tma<L>(a, s, &used);
            if (e != cudaSuccess || used)
                return e;
        }
    }
    return generic ? col_launch<L, true>(a, s) : col_launch<L, false>(a, s);
}

cudaError_t launch_col_pass(int L, const PassArgs &a, cudaStream_t s)
{
    switch (L) {
    case 1: return col_dispatch<1>(a, s);
    case 2: return col_dispatch<2>(a, s);
    case 3: return col_dispatch<3>(a, s);
    case 4: return col_dispatch<4>(a, s);
    case 5: return col_dispatch<5>(a, s);
    case 6: return col_dispatch<6>(a, s);
    case 7: return col_dispatch<7>(a, s);
    case 8: return col_dispatch<8>(a, s);
    case 9: return col_dispatch<9>(a, s);
    case 10: return col_dispatch<10>(a, s);
    case 11: return col_dispatch<11>(a, s);
    case 12: return col_dispatch<12>(a, s);
    case 13: return col_dispatch<13>(a, s);
    case 14: return col_dispatch<14>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fft2d
