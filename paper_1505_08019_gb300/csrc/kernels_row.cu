// kernels_row.cu -- row pass kernel variants: every row of an image is one
// line of cols = 2^L contiguous points.
//
// Variants per line length (the autotuner picks among the usable ones):
//   0  plain   : LB = 2^row_kb(L) rows per CTA, 256 threads x 16 values,
//                scrambled global loads (the default)
//   1  plain32 : the same rows per CTA with 32 values per thread
//   2  plain2x : twice the rows per CTA (two line blocks in flight)
//   3  tma     : persistent, double-buffered TMA bulk loads (16-byte aligned,
//                dense whole blocks only)
//   4  split   : persistent, one row per CTA at a time with the next row's
//                first half prefetched (rows of 4096..16384 points)
#include <cstring>

#include "line_fft.cuh"
#include "passes.h"

namespace fft2d {

int row_lines_per_cta(int L) { return 1 << row_kb(L); }

namespace {

template <class C, bool GENERIC>
cudaError_t row_launch(const PassArgs &a, cudaStream_t s)
{
    auto k = row_pass_kernel<C, GENERIC, StoreC64>;
    const int dev_bytes = LineSmem<C, true, StoreC64>::BYTES;
    if (dev_bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             dev_bytes);
        if (e != cudaSuccess)
            return e;
    }
    const unsigned grid = (unsigned)((a.rows + C::LB - 1) / C::LB);
    k<<<grid, C::T, dev_bytes, s>>>(StoreC64{a.in, a.out}, a.tw, a.rows, a.ld, a.scale, a.nst);
    return cudaGetLastError();
}

template <class C>
cudaError_t row_launch_any(const PassArgs &a, cudaStream_t s)
{
    const bool generic = a.partial || a.rows % C::LB != 0;
    return generic ? row_launch<C, true>(a, s) : row_launch<C, false>(a, s);
}

template <class C>
bool row_tma_usable(const PassArgs &a)
{
    return !a.partial && a.err && !(reinterpret_cast<uintptr_t>(a.in) & 15) &&
           !((a.ld * 8) & 15) && a.rows % C::LB == 0;
}

template <class C>
cudaError_t row_launch_tma(const PassArgs &a, cudaStream_t s)
{
    constexpr int SMEM = RowTma<C>::SMEM_BYTES;
    auto k = row_tma_kernel<C>;
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
    const int ntiles = a.rows / C::LB;
    int grid = device_sm_count() * occ.get(d);
    if (grid > ntiles)
        grid = ntiles;
    k<<<grid, C::T, SMEM, s>>>(a.in, a.out, a.tw, a.rows, a.ld, a.scale, a.err);
    return cudaGetLastError();
}

// Persistent row pass for long rows, one row (LB = 1) per CTA at a time.
// Shared memory holds the row region (the exchange buffer) and a prefetch
// region of half a row.  A row arrives as two bulk copies: its first half
// into the prefetch region as soon as group 0 has gathered the previous row,
// its second half into the lower half of the row region once the last group
// has read the previous row from there.  Group 0 finds position i in the
// prefetch region (i < N/2) or in the row region (i >= N/2); which one is
// fixed by the register index.  Rotation factors come from global memory
// (a 16384-point table is 128 KB).
template <class C>
struct RowSplit {
    static constexpr int HALF = C::E / 2;
    static constexpr int SMEM_BYTES = (C::E + HALF) * 8;
    static constexpr uint32_t HALF_BYTES = (uint32_t)HALF * 8u;
    static_assert(C::LB == 1 && C::KW == 0 && C::NG >= 2, "one row per CTA, two stage groups");
    static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
};

template <class C>
__device__ __forceinline__ void row_split_issue(float2 *dst, const float2 *src, uint64_t *bar)
{
    mbar_arrive_expect_tx(bar, RowSplit<C>::HALF_BYTES);
    bulk_load(dst, src, RowSplit<C>::HALF_BYTES, bar);
}

template <class C>
__global__ void __launch_bounds__(C::T, 1) row_split_kernel(const float2 *in, float2 *out,
                                                            const float2 *__restrict__ tw,
                                                            int rows, long long ld, float scale,
                                                            int *err)
{
    using S = RowSplit<C>;
    using G0 = Grp<C, 0>;
    extern __shared__ __align__(128) float2 sm[];
    __shared__ __align__(8) uint64_t bar_early, bar_late;
    float2 *pref = sm + C::E;
    const int tid = threadIdx.x;
    int row = blockIdx.x;
    if (tid == 0) {
        mbar_init(&bar_early, 1);
        mbar_init(&bar_late, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0 && row < rows) {
        row_split_issue<C>(pref, in + (long long)row * ld, &bar_early);
        row_split_issue<C>(sm, in + (long long)row * ld + S::HALF, &bar_late);
    }
    uint32_t parity = 0;
    float2 a[C::EPT];
    for (; row < rows; row += gridDim.x) {
        const int next = row + gridDim.x;
        const bool ok = mbar_wait_bounded(&bar_early, parity) && mbar_wait_bounded(&bar_late, parity);
        if (__syncthreads_or(ok ? 0 : 1)) {
            if (tid == 0)
                atomicExch(err, kDevErrTmaTimeout);
            mbar_wait_bounded(&bar_early, parity);
            mbar_wait_bounded(&bar_late, parity);
            return;
        }
        parity ^= 1;
#pragma unroll
        for (int v = 0; v < G0::V; v++) {
            const int hib = (tid + v * C::T) & ((1 << G0::HB) - 1);
#pragma unroll
            for (int r = 0; r < G0::R; r++) {
                const int top = brev_c(r, G0::G) << G0::HB;   // compile-time
                a[v * G0::R + r] = top < S::HALF ? pref[top | hib] : sm[(top - S::HALF) | hib];
            }
        }
#pragma unroll
        for (int v = 0; v < G0::V; v++)
            run_stages<C, 0, false>(a, v, 0, tw, C::L);
        fence_proxy_async_smem();
        __syncthreads();   // both regions have been read
        if (tid == 0 && next < rows)
            row_split_issue<C>(pref, in + (long long)next * ld, &bar_early);
#pragma unroll
        for (int v = 0; v < G0::V; v++) {
            const int hib = (tid + v * C::T) & ((1 << G0::HB) - 1);
            const int hi = brev_rt(hib, G0::HB);
#pragma unroll
            for (int r = 0; r < G0::R; r++)
                sm[sidx<C>(0, r | (hi << G0::G), 0)] = a[v * G0::R + r];
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
        group_last_read<C>(a, sm);
        fence_proxy_async_smem();
        __syncthreads();   // the row region is free
        if (tid == 0 && next < rows)
            row_split_issue<C>(sm, in + (long long)next * ld + S::HALF, &bar_late);
        group_last_finish<C, false>(a, out + (long long)row * ld, tw, 1, scale, C::L);
    }
}

template <class C>
bool row_split_usable(const PassArgs &a)
{
    return !a.partial && a.err && !(reinterpret_cast<uintptr_t>(a.in) & 15) &&
           !((a.ld * 8) & 15);
}

template <class C>
cudaError_t row_launch_split(const PassArgs &a, cudaStream_t s)
{
    constexpr int SMEM = RowSplit<C>::SMEM_BYTES;
    auto k = row_split_kernel<C>;
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
    if (grid > a.rows)
        grid = a.rows;
    k<<<grid, C::T, SMEM, s>>>(a.in, a.out, a.tw, a.rows, a.ld, a.scale, a.err);
    return cudaGetLastError();
}

bool always(const PassArgs &) { return true; }
bool whole_stages(const PassArgs &a) { return !a.partial; }

template <int L>
struct RowVariants {
    using Plain = LineCfg<L, 0, row_kb(L), 16>;
    using Plain32 = LineCfg<L, 0, row_kb(L), 32>;
    static constexpr int KB2 = row_kb(L) + 1;
    using Plain2x = LineCfg<L, 0, KB2, 16>;
    static constexpr bool HAS32 = L >= 5 && Plain32::E >= 32;
    static constexpr bool HAS2X = L >= 5 && L <= 13 && Plain2x::E * 8 <= 128 * 1024;
    static constexpr bool HASTMA = L >= 5 && L <= 13;
    static constexpr bool HASSPLIT = L >= 12;
    // groups of 5 stages (32 values a thread) where they save a group:
    // 512, 1024, 8192 and 16384 points
    using G5 = LineCfg<L, 0, row_kb(L), 32, 5>;
    static constexpr bool HASG5 = (L == 9 || L == 10 || L == 13 || L == 14) && G5::E >= 32;
    using Split5 = LineCfg<L, 0, 0, 32, 5>;
    static constexpr bool HASSPLIT5 = L >= 13;

    struct Table {
        Variant v[7];
        int n = 0;
    };
    static Table build()
    {
        Table t;
        t.v[t.n++] = {"plain", 1 << row_kb(L), 16, always, row_launch_any<Plain>};
        if constexpr (HAS32)
            t.v[t.n++] = {"plain32", 1 << row_kb(L), 32, whole_stages, row_launch_any<Plain32>};
        if constexpr (HAS2X)
            t.v[t.n++] = {"plain2x", 1 << KB2, 16, whole_stages, row_launch_any<Plain2x>};
        if constexpr (HASTMA)
            t.v[t.n++] = {"tma", 1 << row_kb(L), 16, row_tma_usable<Plain>, row_launch_tma<Plain>};
        if constexpr (HASSPLIT)
            t.v[t.n++] = {"split", 1, 16, row_split_usable<Plain>, row_launch_split<Plain>};
        if constexpr (HASG5)
            t.v[t.n++] = {"plain32g5", 1 << row_kb(L), 32, whole_stages, row_launch_any<G5>};
        if constexpr (HASSPLIT5)
            t.v[t.n++] = {"split32g5", 1, 32, row_split_usable<Split5>, row_launch_split<Split5>};
        return t;
    }
    static const Variant *table(int *n)
    {
        static const Table t = build();
        *n = t.n;
        return t.v;
    }
};

}  // namespace

const Variant *row_variants(int L, int *n)
{
    switch (L) {
    case 1: return RowVariants<1>::table(n);
    case 2: return RowVariants<2>::table(n);
    case 3: return RowVariants<3>::table(n);
    case 4: return RowVariants<4>::table(n);
    case 5: return RowVariants<5>::table(n);
    case 6: return RowVariants<6>::table(n);
    case 7: return RowVariants<7>::table(n);
    case 8: return RowVariants<8>::table(n);
    case 9: return RowVariants<9>::table(n);
    case 10: return RowVariants<10>::table(n);
    case 11: return RowVariants<11>::table(n);
    case 12: return RowVariants<12>::table(n);
    case 13: return RowVariants<13>::table(n);
    case 14: return RowVariants<14>::table(n);
    default: *n = 0; return nullptr;
    }
}

// plain everywhere except 8192- and 16384-point rows, where groups of 5
// stages (32 values a thread, three groups instead of four) measured faster:
// 0.183 against 0.218 ms (8192^2, "plain32") and 0.906 against 1.04 ms
// (16384^2, "split")
int row_default_variant(int L)
{
    if (L != 13 && L != 14)
        return 0;
    int n = 0;
    const Variant *v = row_variants(L, &n);
    for (int i = 0; i < n; i++)
        if (std::strcmp(v[i].name, "plain32g5") == 0)
            return i;
    return 0;
}

cudaError_t launch_row_pass(int L, const PassArgs &a, cudaStream_t s)
{
    int n = 0;
    const Variant *v = row_variants(L, &n);
    if (!v || n == 0)
        return cudaErrorInvalidValue;
    int i = a.variant >= 0 && a.variant < n ? a.variant : row_default_variant(L);
    if (!v[i].usable(a))
        i = 0;   // the plain kernel serves every case
    return v[i].launch(a, s);
}

}  // namespace fft2d
