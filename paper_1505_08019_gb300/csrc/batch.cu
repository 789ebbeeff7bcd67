// batch.cu -- grouped launches for many independent images of uneven shapes.
//
// Every image is a separate 2D transform (Section 2: rows and columns of one
// image are independent, and so are images).  Instead of two launches per
// image, the images are grouped by axis length: one launch runs the row pass
// of every image whose rows have 2^L points, another the column pass of every
// image whose columns have 2^L points.  A small job table travels as a kernel
// parameter; each CTA finds its image by binary search over the table's CTA
// offsets and then runs exactly the per-CTA work of the single-image kernels,
// so a batched image is bit-for-bit the image transformed alone.
#include <type_traits>

#include "line_fft.cuh"
#include "passes.h"

namespace fft2d {

namespace {

template <class Table>
__device__ __forceinline__ int find_job(const Table &t)
{
    int lo = 0, hi = t.n - 1;
    const int b = (int)blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t.job[mid].first_cta <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <class C>
__global__ void __launch_bounds__(C::T, C::MINB) row_batch_kernel(const __grid_constant__ BatchTable t)
{
    const BatchJob &jb = t.job[find_job(t)];
    const long long r0 = (long long)((int)blockIdx.x - jb.first_cta) * C::LB;
    line_fft<C, true, true, StoreC64>(StoreC64{jb.in, jb.out}, Geo{r0, 1, 0, jb.ld}, jb.tw,
                                      jb.scale, C::L, jb.lines - r0);
}

template <class C>
__global__ void __launch_bounds__(C::T, C::MINB) col_batch_kernel(const __grid_constant__ BatchTable t)
{
    const BatchJob &jb = t.job[find_job(t)];
    const long long c0 = (long long)((int)blockIdx.x - jb.first_cta) * C::W;
    line_fft<C, false, true, StoreC64>(StoreC64{jb.in, jb.out}, Geo{0, 1, c0, jb.ld}, jb.tw,
                                       jb.scale, C::L, jb.lines - c0);
}

// Half2 jobs: per-line exponents in and out (StoreH16T), the input's
// exponent axis fixed for the launch.
template <class C, bool ROW, int IA>
__global__ void __launch_bounds__(C::T, C::MINB) h16_batch_kernel(const __grid_constant__ BatchTableH16 t)
{
    using IO = StoreH16T<IA>;
    const BatchJobH16 &jb = t.job[find_job(t)];
    const long long l0 = (long long)((int)blockIdx.x - jb.first_cta) * (ROW ? C::LB : C::W);
    const IO io{jb.in, jb.out, jb.in_exp, IA, jb.out_exp};
    const Geo g = ROW ? Geo{l0, 1, 0, jb.ld} : Geo{0, 1, l0, jb.ld};
    line_fft<C, ROW, true, IO>(io, g, jb.tw, jb.scale, C::L, jb.lines - l0);
}

template <class C, bool ROW, int IA>
cudaError_t batch_launch_h16(BatchTableH16 &t, cudaStream_t s)
{
    auto k = h16_batch_kernel<C, ROW, IA>;
    const int per = ROW ? C::LB : C::W;
    int ctas = 0;
    for (int i = 0; i < t.n; i++) {
        t.job[i].first_cta = ctas;
        ctas += (t.job[i].lines + per - 1) / per;
    }
    if (ctas == 0)
        return cudaSuccess;
    constexpr int SMEM = LineSmem<C, ROW, StoreH16T<IA>>::BYTES;
    if (SMEM > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess)
            return e;
    }
    k<<<ctas, C::T, SMEM, s>>>(t);
    return cudaGetLastError();
}

// The single-image half2 passes' CTA shapes (kernels_h16.cu): rows as for
// complex64, plain column tiles of 2^col_kw(L) columns.
template <int L>
cudaError_t batch_dispatch_h16(bool row, BatchTableH16 &t, int in_axis, cudaStream_t s)
{
    if (row) {
        using C = LineCfg<L, 0, row_kb(L), L == 13 ? 32 : 16>;
        return in_axis == 0 ? batch_launch_h16<C, true, 0>(t, s) : batch_launch_h16<C, true, 1>(t, s);
    }
    using C = LineCfg<L, col_kw(L), 0>;
    return in_axis == 0 ? batch_launch_h16<C, false, 0>(t, s) : batch_launch_h16<C, false, 1>(t, s);
}

template <class C, bool ROW>
cudaError_t batch_launch(BatchTable &t, cudaStream_t s)
{
    auto k = ROW ? row_batch_kernel<C> : col_batch_kernel<C>;
    const int per = ROW ? C::LB : C::W;
    int ctas = 0;
    for (int i = 0; i < t.n; i++) {
        t.job[i].first_cta = ctas;
        ctas += (t.job[i].lines + per - 1) / per;
    }
    if (ctas == 0)
        return cudaSuccess;
    if (C::SMEM_BYTES > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM_BYTES);
        if (e != cudaSuccess)
            return e;
    }
    k<<<ctas, C::T, C::SMEM_BYTES, s>>>(t);
    return cudaGetLastError();
}

// Grouped persistent TMA column pass: a load and a store tensor map per
// image; not used when some image cannot be described by them (alignment,
// partial tiles).  Store mode: 0 TMA stores, 1 per-thread stores, 2 half of
// each (TMA stores need tma_store_ok; otherwise per-thread stores).
template <class C, int MODE>
cudaError_t batch_launch_tma(const BatchTable &t, int *err, cudaStream_t s, bool *used)
{
    *used = false;
    static thread_local BatchTmaTable tt;
    if (t.n > kBatchTmaMaxJobs || !err || (reinterpret_cast<uintptr_t>(t.job[0].tw) & 15))
        return cudaSuccess;
    // one unit a thread (groups of 6 stages): the half of each tile that
    // leaves by TMA is its first N/2 rows, one box of the load map's shape
    constexpr bool ROWHALF = Grp<C, C::NG - 1>::V == 1;
    int tiles = 0;
    for (int i = 0; i < t.n; i++) {
        const BatchJob &j = t.job[i];
        if (j.lines % C::W != 0 ||
            !encode_col_map(&tt.map[i], j.in, C::N, j.lines, j.ld, C::W, TmaSplit<C>::BOX,
                            TmaSplit<C>::NB) ||
            !encode_col_map(&tt.omap[i], j.out, C::N, j.lines, j.ld, C::W,
                            ROWHALF ? TmaSplit<C>::BOX : tma_store_rows(C::L),
                            ROWHALF ? TmaSplit<C>::NB : TmaSplit<C>::NBOX))
            return cudaSuccess;
        tt.out[i] = j.out;
        tt.ld[i] = j.ld;
        tt.scale[i] = j.scale;
        tt.first_tile[i] = tiles;
        tiles += j.lines / C::W;
    }
    tt.first_tile[t.n] = tiles;
    tt.n = t.n;
    if (tiles == 0) {
        *used = true;
        return cudaSuccess;
    }
    constexpr bool TS = ROWHALF ? MODE == 2 : (MODE != 1 && tma_store_ok<C>());
    auto k = col_tma2_batch_kernel<C, TS, TS && MODE == 2>;
    constexpr int SMEM = TmaSplit<C>::SMEM_BYTES;
    constexpr int kMaxDev = 64;
    static DeviceCache occ;
    const int d = device_current();
    if (!occ.get(d)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess)
            return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, C::T, SMEM);
        if (e != cudaSuccess)
            return e;
        occ.set(d, o > 0 ? o : 1);
    }
    int grid = device_sm_count() * occ.get(d);
    if (grid > tiles)
        grid = tiles;
    k<<<grid, C::T, SMEM, s>>>(tt, t.job[0].tw, err);
    *used = true;
    return cudaGetLastError();
}

template <int L>
cudaError_t batch_dispatch(bool row, BatchTable &t, int variant, int *err, cudaStream_t s)
{
    if (row) {
        if (variant == 1 && L >= 5)
            return batch_launch<LineCfg<L, 0, row_kb(L), 32>, true>(t, s);
        return batch_launch<LineCfg<L, 0, row_kb(L)>, true>(t, s);
    }
    if constexpr (L >= 9 && L <= 12) {
        if (variant >= 2 && variant <= 4) {
            using C = LineCfg<L, col_kw(L), 0, col_tma_ept(L)>;
            // half of each: 4096 rows in two groups of 6 stages, as the
            // single-image default
            using CH = typename std::conditional<L == 12, LineCfg<L, col_kw(L), 0, 64, 6>, C>::type;
            // per-thread stores: 2048 rows in two groups (6 + 5), as the
            // single-image default
            using CS = typename std::conditional<L == 11, LineCfg<L, col_kw(L), 0, 64, 6>, C>::type;
            bool used = false;
            cudaError_t e = variant == 2   ? batch_launch_tma<C, 0>(t, err, s, &used)
                            : variant == 3 ? batch_launch_tma<CS, 1>(t, err, s, &used)
                                           : batch_launch_tma<CH, 2>(t, err, s, &used);
            if (e != cudaSuccess || used)
                return e;
        }
    }
    if constexpr (L >= 5 && col_kw(L) >= 3) {
        if (variant == 1)
            return batch_launch<LineCfg<L, col_kw(L) - 1, 0>, false>(t, s);
    }
    return batch_launch<LineCfg<L, col_kw(L), 0>, false>(t, s);
}

}  // namespace

// Defaults, from timings on a GB300 (the batch autotuner can override them):
// per-thread stores for 1024- and 2048-row columns, half of each for 4096.
int batch_default_variant(bool row, int L)
{
    if (row)
        return 0;
    if (L == 10 || L == 11)
        return 3;
    if (L == 12)
        return 4;
    return L == 9 ? 2 : 0;
}

const char *batch_variant_name(bool row, int variant)
{
    static const char *rn[kBatchRowVariants] = {"plain", "plain32"};
    static const char *cn[kBatchColVariants] = {"plain", "narrow", "tma", "tmast", "tmah"};
    if (row)
        return variant >= 0 && variant < kBatchRowVariants ? rn[variant] : "";
    return variant >= 0 && variant < kBatchColVariants ? cn[variant] : "";
}

cudaError_t launch_batch_pass_h16(bool row, int L, BatchTableH16 &t, int in_axis, cudaStream_t s)
{
    switch (L) {
    case 1: return batch_dispatch_h16<1>(row, t, in_axis, s);
    case 2: return batch_dispatch_h16<2>(row, t, in_axis, s);
    case 3: return batch_dispatch_h16<3>(row, t, in_axis, s);
    case 4: return batch_dispatch_h16<4>(row, t, in_axis, s);
    case 5: return batch_dispatch_h16<5>(row, t, in_axis, s);
    case 6: return batch_dispatch_h16<6>(row, t, in_axis, s);
    case 7: return batch_dispatch_h16<7>(row, t, in_axis, s);
    case 8: return batch_dispatch_h16<8>(row, t, in_axis, s);
    case 9: return batch_dispatch_h16<9>(row, t, in_axis, s);
    case 10: return batch_dispatch_h16<10>(row, t, in_axis, s);
    case 11: return batch_dispatch_h16<11>(row, t, in_axis, s);
    case 12: return batch_dispatch_h16<12>(row, t, in_axis, s);
    case 13: return batch_dispatch_h16<13>(row, t, in_axis, s);
    case 14: return batch_dispatch_h16<14>(row, t, in_axis, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_pass(bool row, int L, BatchTable &t, int variant, int *err,
                              cudaStream_t s)
{
    switch (L) {
    case 1: return batch_dispatch<1>(row, t, variant, err, s);
    case 2: return batch_dispatch<2>(row, t, variant, err, s);
    case 3: return batch_dispatch<3>(row, t, variant, err, s);
    case 4: return batch_dispatch<4>(row, t, variant, err, s);
    case 5: return batch_dispatch<5>(row, t, variant, err, s);
    case 6: return batch_dispatch<6>(row, t, variant, err, s);
    case 7: return batch_dispatch<7>(row, t, variant, err, s);
    case 8: return batch_dispatch<8>(row, t, variant, err, s);
    case 9: return batch_dispatch<9>(row, t, variant, err, s);
    case 10: return batch_dispatch<10>(row, t, variant, err, s);
    case 11: return batch_dispatch<11>(row, t, variant, err, s);
    case 12: return batch_dispatch<12>(row, t, variant, err, s);
    case 13: return batch_dispatch<13>(row, t, variant, err, s);
    case 14: return batch_dispatch<14>(row, t, variant, err, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace fft2d
