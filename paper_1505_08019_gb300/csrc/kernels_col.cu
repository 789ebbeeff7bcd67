// kernels_col.cu -- column pass instantiations: every column of an image is a
// line of rows = 2^L points spaced one row pitch apart; a CTA owns a tile of
// W adjacent whole columns, so each global access reads or writes W*8
// contiguous bytes of a row and the whole column stays on chip.
#include "line_fft.cuh"
#include "passes.h"

namespace fft2d {

// 2^14 values (128 KB of shared memory) per CTA from 1024-point columns up;
// 16 to 64 columns per CTA below.
static constexpr int col_kw(int L)
{
    return L >= 10 ? 14 - L : (13 - L < 4 ? 4 : (13 - L > 6 ? 6 : 13 - L));
}

int col_width(int L) { return 1 << col_kw(L); }

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

template <int L>
static cudaError_t col_dispatch(const PassArgs &a, cudaStream_t s)
{
    const bool generic = a.partial || a.cols < col_width(L);
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
