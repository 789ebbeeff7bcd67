// kernels_row.cu -- row pass instantiations: every row of an image is one line
// of cols = 2^L points (contiguous), LB rows per CTA, 256 threads per CTA up to
// 4096-point rows.
#include "line_fft.cuh"
#include "passes.h"

namespace fft2d {

static constexpr int row_kb(int L) { return L <= 12 ? 12 - L : 0; }
// values per thread (32 measured no faster for 4096-point rows)
static constexpr int row_ept(int) { return 16; }

int row_lines_per_cta(int L) { return 1 << row_kb(L); }

template <int L, bool GENERIC>
static cudaError_t row_launch(const PassArgs &a, cudaStream_t s)
{
    using C = LineCfg<L, 0, row_kb(L), row_ept(L)>;
    auto k = row_pass_kernel<C, GENERIC>;
    const int dev_bytes = C::SMEM_BYTES;
    if (dev_bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             dev_bytes);
        if (e != cudaSuccess)
            return e;
    }
    const unsigned grid = (unsigned)((a.rows + C::LB - 1) / C::LB);
    k<<<grid, C::T, dev_bytes, s>>>(a.in, a.out, a.tw, a.rows, a.ld, a.scale, a.nst);
    return cudaGetLastError();
}

// Persistent TMA-fed variant (row_tma_kernel): whole blocks of LB rows only,
// input 16-byte aligned, row pitch a multiple of 16 bytes.
template <int L>
static cudaError_t row_launch_tma(const PassArgs &a, cudaStream_t s, bool *used)
{
    using C = LineCfg<L, 0, row_kb(L)>;
    constexpr int SMEM = RowTma<C>::SMEM_BYTES;
    *used = false;
    if ((reinterpret_cast<uintptr_t>(a.in) & 15) || ((a.ld * 8) & 15) || a.rows % C::LB)
        return cudaSuccess;
    auto k = row_tma_kernel<C>;
    constexpr int kMaxDev = 64;
    static int occ[kMaxDev] = {};
    const int d = device_current();
    if (!occ[d]) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess)
            return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, C::T, SMEM);
        if (e != cudaSuccess)
            return e;
        occ[d] = o > 0 ? o : 1;
    }
    const int ntiles = a.rows / C::LB;
    int grid = device_sm_count() * occ[d];
    if (grid > ntiles)
        grid = ntiles;
    k<<<grid, C::T, SMEM, s>>>(a.in, a.out, a.tw, a.rows, a.ld, a.scale, a.err);
    *used = true;
    return cudaGetLastError();
}

// The plain kernel keeps 4 CTAs of 256 threads on every SM, which already
// overlaps loads with compute; the TMA variant's double buffer costs one CTA
// per SM and measured slower at 4096 points, so it serves only on request
// (row_variant == 1).
template <int L>
static cudaError_t row_dispatch(const PassArgs &a, cudaStream_t s)
{
    const bool generic = a.partial || a.rows < row_lines_per_cta(L);
    if constexpr (L >= 5 && L <= 13) {
        if (!generic && a.err && a.variant == 1) {
            bool used = false;
            cudaError_t e = row_launch_tma<L>(a, s, &used);
            if (e != cudaSuccess || used)
                return e;
        }
    }
    return generic ? row_launch<L, true>(a, s) : row_launch<L, false>(a, s);
}

cudaError_t launch_row_pass(int L, const PassArgs &a, cudaStream_t s)
{
    switch (L) {
    case 1: return row_dispatch<1>(a, s);
    case 2: return row_dispatch<2>(a, s);
    case 3: return row_dispatch<3>(a, s);
    case 4: return row_dispatch<4>(a, s);
    case 5: return row_dispatch<5>(a, s);
    case 6: return row_dispatch<6>(a, s);
    case 7: return row_dispatch<7>(a, s);
    case 8: return row_dispatch<8>(a, s);
    case 9: return row_dispatch<9>(a, s);
    case 10: return row_dispatch<10>(a, s);
    case 11: return row_dispatch<11>(a, s);
    case 12: return row_dispatch<12>(a, s);
    case 13: return row_dispatch<13>(a, s);
    case 14: return row_dispatch<14>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fft2d
