// kernels_col.cu -- column pass instantiations: every column of an image is a
// line of rows = 2^L points spaced one row pitch apart; a CTA owns a tile of
// W adjacent whole columns, so each global access reads or writes W*8
// contiguous bytes of a row and the whole column stays on chip.
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "col_group.cuh"
#include "col_tmem.cuh"
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
    static DeviceCache cache;
    const int d = device_current();
    if (!cache.get(d)) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d);
        cache.set(d, n > 0 ? n : 1);
    }
    return cache.get(d);
}


int col_width(int L) { return 1 << col_kw(L); }

bool encode_col_map(CUtensorMap *map, const float2 *base, int rows, int cols, long long ld, int W,
                    int box_y, int box_z)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || (reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 8) & 15) || rows % 256 != 0)
        return false;
    cuuint64_t dims[3] = {(cuuint64_t)cols, 256, (cuuint64_t)(rows / 256)};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 8, (cuuint64_t)ld * 8 * 256};
    cuuint32_t box[3] = {(cuuint32_t)W, (cuuint32_t)box_y, (cuuint32_t)box_z};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<float2 *>(base), dims, strides,
               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

bool encode_map_xyz(CUtensorMap *map, const void *base, long long xdim, int ydim, int zdim,
                    long long ystride, long long zstride, int box_x, int box_y, int box_z)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || (reinterpret_cast<uintptr_t>(base) & 15) || ((ystride * 8) & 15) ||
        ((zstride * 8) & 15))
        return false;
    cuuint64_t dims[3] = {(cuuint64_t)xdim, (cuuint64_t)ydim, (cuuint64_t)zdim};
    cuuint64_t strides[2] = {(cuuint64_t)ystride * 8, (cuuint64_t)zstride * 8};
    cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, (cuuint32_t)box_z};
    cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<void *>(base), dims, strides,
               box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

bool tensor_maps_available() { return tensor_map_encoder() != nullptr; }

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

namespace {

template <class C, bool GENERIC>
cudaError_t col_launch(const PassArgs &a, cudaStream_t s)
{
    auto k = col_pass_kernel<C, GENERIC, StoreC64>;
    const int dev_bytes = LineSmem<C, false, StoreC64>::BYTES;
    if (dev_bytes > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             dev_bytes);
        if (e != cudaSuccess)
            return e;
    }
    const unsigned grid = (unsigned)((a.cols + C::W - 1) / C::W);
    k<<<grid, C::T, dev_bytes, s>>>(StoreC64{a.in, a.out}, a.tw, a.cols, a.ld, a.scale, a.nst);
    return cudaGetLastError();
}

template <class C>
cudaError_t col_launch_any(const PassArgs &a, cudaStream_t s)
{
    const bool generic = a.partial || a.cols % C::W != 0;
    return generic ? col_launch<C, true>(a, s) : col_launch<C, false>(a, s);
}

template <class C>
bool col_tma_usable(const PassArgs &a)
{
    return !a.partial && a.err && tensor_map_encoder() &&
           !(reinterpret_cast<uintptr_t>(a.in) & 15) && !(reinterpret_cast<uintptr_t>(a.out) & 15) &&
           !(reinterpret_cast<uintptr_t>(a.tw) & 15) && !((a.ld * 8) & 15) && a.cols % C::W == 0;
}

// Persistent TMA-fed column pass (col_tma2_kernel), with TMA stores (TS),
// per-thread stores, or half of each (TS and HYB).  Falls back to the plain
// kernel if a tile cannot be described by a tensor map.
template <class C, bool TS, bool HYB = false>
cudaError_t col_launch_tma(const PassArgs &a, cudaStream_t s)
{
    CUtensorMap map, omap;
    using S = TmaSplit<C>;
    // store boxes: half a 256-row block per box (4-stage groups), or the
    // first half of the tile in one box (one unit a thread)
    constexpr bool ROWHALF = Grp<C, C::NG - 1>::V == 1;
    if (!encode_col_map(&map, a.in, a.rows, a.cols, a.ld, C::W, S::BOX, S::NB) ||
        !encode_col_map(&omap, a.out, a.rows, a.cols, a.ld, C::W,
                        ROWHALF ? S::BOX : tma_store_rows(C::L), ROWHALF ? S::NB : S::NBOX))
        return col_launch_any<LineCfg<C::L, C::KW, 0>>(a, s);
    auto k = col_tma2_kernel<C, TS, HYB>;
    constexpr int SMEM = TmaSplit<C>::SMEM_BYTES;
    static DeviceCache occ;
    const int d = current_device();
    if (!occ.get(d)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SMEM);
        if (e != cudaSuccess)
            return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, C::T, SMEM);
        if (e != cudaSuccess)
            return e;
        occ.set(d, o > 0 ? o : 1);
    }
    const int ntiles = a.cols / C::W;
    int grid = sm_count() * occ.get(d);
    if (grid > ntiles)
        grid = ntiles;
    k<<<grid, C::T, SMEM, s>>>(map, omap, a.out, a.tw, a.cols, a.ld, a.scale, a.err,
                               a.withhold);
    return cudaGetLastError();
}

// Persistent column pass with the next tile parked in TMEM (col_tmem_kernel):
// TMA loads into a landing region, whole-tile TMA store.  Falls back to the
// plain kernel if a tile cannot be described by a tensor map.
template <class C>
cudaError_t col_launch_tmem(const PassArgs &a, cudaStream_t s)
{
    CUtensorMap map, omap;
    using S = TmaSplit<C>;
    if (!encode_col_map(&map, a.in, a.rows, a.cols, a.ld, C::W, S::BOX, S::NB) ||
        !encode_col_map(&omap, a.out, a.rows, a.cols, a.ld, C::W, S::BOX, S::NBOX))
        return col_launch_any<LineCfg<C::L, C::KW, 0>>(a, s);
    auto k = col_tmem_kernel<C>;
    constexpr int SMEM = S::SMEM_BYTES;
    static DeviceCache occ;
    const int d = current_device();
    if (!occ.get(d)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SMEM);
        if (e != cudaSuccess)
            return e;
        int o = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k, C::T, SMEM);
        if (e != cudaSuccess)
            return e;
        occ.set(d, o > 0 ? o : 1);
    }
    const int ntiles = a.cols / C::W;
    int grid = sm_count() * occ.get(d);
    if (grid > ntiles)
        grid = ntiles;
    k<<<grid, C::T, SMEM, s>>>(map, omap, a.out, a.tw, a.cols, a.ld, a.scale, a.err,
                               a.withhold);
    return cudaGetLastError();
}

// Column pass over 2^(L+CL)-row columns split over a cluster of 2^CL CTAs
// (col_group_kernel, local engine C of 2^L rows): one load map per row
// residue modulo 2^CL, one store map, a persistent grid of as many clusters
// as can be resident at once.
template <class C, int CL>
bool col_group_usable(const PassArgs &a)
{
    return col_tma_usable<C>(a) && a.rows == (C::N << CL);
}

template <class C, int CL>
cudaError_t col_launch_group(const PassArgs &a, cudaStream_t s)
{
    using S = TmaSplit<C>;
    using GC = GroupCol<C, CL>;
    constexpr int CS = 1 << CL;
    CUtensorMap m[4], om;
    for (int r = 0; r < CS; r++)
        if (!encode_col_map(&m[r], a.in + r * a.ld, a.rows / CS, a.cols, CS * a.ld, C::W, S::BOX,
                            S::NB))
            return col_launch_any<LineCfg<C::L + CL, C::KW, 0>>(a, s);
    for (int r = CS; r < 4; r++)
        m[r] = m[0];
    if (!encode_col_map(&om, a.out, a.rows, a.cols, a.ld, C::W, S::BOX, GC::OUT_BOX_Z))
        return col_launch_any<LineCfg<C::L + CL, C::KW, 0>>(a, s);
    auto k = col_group_kernel<C, CL>;
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
    const int d = current_device();
    if (!groups.get(d)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SMEM);
        if (e != cudaSuccess)
            return e;
        cfg.gridDim = dim3((unsigned)(CS * (sm_count() / CS)));
        int n = 0;
        e = cudaOccupancyMaxActiveClusters(&n, k, &cfg);
        if (e != cudaSuccess)
            return e;
        groups.set(d, n > 0 ? n : 1);
    }
    const int ntiles = a.cols / C::W;
    const int ng = groups.get(d) < ntiles ? groups.get(d) : ntiles;
    cfg.gridDim = dim3((unsigned)(CS * ng));
    return cudaLaunchKernelEx(&cfg, k, m[0], m[1], m[2], m[3], om, a.tw, a.cols, a.scale, a.err,
                              a.withhold);
}


// Column pass over 2^(L+CL)-row columns on clusters of 2^CL CTAs with the
// exchange rounds through L2 (col_group_l2_kernel); the same tensor maps and
// persistent grid as col_launch_group.
template <class C, int CL>
cudaError_t col_launch_group_l2(const PassArgs &a, cudaStream_t s)
{
    using S = TmaSplit<C>;
    using GC = GroupCol<C, CL>;
    constexpr int CS = 1 << CL;
    CUtensorMap m[4], om;
    for (int r = 0; r < CS; r++)
        if (!encode_col_map(&m[r], a.in + r * a.ld, a.rows / CS, a.cols, CS * a.ld, C::W, S::BOX,
                            S::NB))
            return col_launch_any<LineCfg<C::L + CL, C::KW, 0>>(a, s);
    for (int r = CS; r < 4; r++)
        m[r] = m[0];
    if (!encode_col_map(&om, a.out, a.rows, a.cols, a.ld, C::W, S::BOX, GC::OUT_BOX_Z))
        return col_launch_any<LineCfg<C::L + CL, C::KW, 0>>(a, s);
    auto k = col_group_l2_kernel<C, CL, false>;
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
    const int d = current_device();
    if (!groups.get(d)) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             SMEM);
        if (e != cudaSuccess)
            return e;
        cfg.gridDim = dim3((unsigned)(CS * (sm_count() / CS)));
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
    e = cudaLaunchKernelEx(&cfg, k, m[0], m[1], m[2], m[3], om, a.tw, a.cols, a.scale, a.err,
                           a.withhold, static_cast<float2 *>(xbuf), GroupIO{nullptr, nullptr});
    const cudaError_t f = cudaFreeAsync(xbuf, s);
    return e != cudaSuccess ? e : f;
}

template <class CC>
bool col_cluster_usable(const PassArgs &a)
{
    return !a.partial && a.cols % CC::W == 0;
}

// Cluster column pass (col_cluster_kernel): CS CTAs share a tile, the last
// log2(CS) stages run through distributed shared memory.
template <class CC>
cudaError_t col_launch_cluster(const PassArgs &a, cudaStream_t s)
{
    return launch_cluster_kernel<CC, StoreC64>(StoreC64{a.in, a.out}, a.tw, a.cols, a.ld, a.scale,
                                               a.nst, s);
}

bool always(const PassArgs &) { return true; }
bool whole_stages(const PassArgs &a) { return !a.partial; }


template <int L>
struct ColVariants {
    using Plain = LineCfg<L, col_kw(L), 0>;
    static constexpr bool HASTMA = L >= 9 && L <= 12;
    static constexpr bool HASTMEM = HASTMA && col_tma_ept(L) == 32;
    using PairLocal = LineCfg<12, 2, 0, 32>;
    using PairLocal6 = LineCfg<12, 2, 0, 64, 6>;
    using Tma32 = LineCfg<L, col_kw(L), 0, col_tma_ept(L)>;
    using Tma16 = LineCfg<L, col_kw(L), 0, 16>;
    using Tma64 = LineCfg<L, col_kw(L), 0, 64, 6>;
    static constexpr int KWN = col_kw(L) - 1;                 // narrower tiles
    static constexpr bool HASNARROW = L >= 5 && KWN >= 2;

    using Narrow = LineCfg<L, (KWN >= 0 ? KWN : 0), 0>;
    // cluster shapes: W = 8 over 2 (2048 rows) or 4 (4096 rows) CTAs;
    // W = 4 over 2 or 4 CTAs for 8192 and 16384 rows
    static constexpr int CKW = L <= 12 ? 3 : 2;
    static constexpr int CC_ = L <= 11 ? 1 : (L == 12 ? 2 : (L == 13 ? 1 : 2));
    static constexpr bool HASCLUSTER = L >= 11;
    using Clu = ClusterColCfg<(L >= 11 ? L : 11), CKW, CC_>;
    // 8-column tiles over 4 or 8 CTAs for 8192 and 16384 rows
    static constexpr bool HASCLUSTER8 = L >= 13;
    using Clu8 = ClusterColCfg<(L >= 13 ? L : 13), 3, (L >= 13 ? L - 11 : 2)>;

    struct Table {
        Variant v[12];
        int n = 0;
    };
    static Table build()
    {
        Table t;
        t.v[t.n++] = {"plain", Plain::W, 16, always, col_launch_any<Plain>};
        if constexpr (HASTMA) {
            // TMA loads with TMA stores where the tile shape allows them, the
            // same engine with per-thread stores, and (lines of 1024..4096)
            // 16 values per thread
            constexpr bool TS32 = tma_store_ok<Tma32>();
            t.v[t.n++] = {Tma32::EPT == 32 ? "tma32" : "tma", Tma32::W, Tma32::EPT,
                          col_tma_usable<Tma32>, col_launch_tma<Tma32, TS32>, true};
            if constexpr (TS32)
                t.v[t.n++] = {Tma32::EPT == 32 ? "tma32st" : "tmast", Tma32::W, Tma32::EPT,
                              col_tma_usable<Tma32>, col_launch_tma<Tma32, false>, true};
            if constexpr (Tma32::EPT == 32)
                t.v[t.n++] = {"tma16", Tma16::W, 16, col_tma_usable<Tma16>,
                              col_launch_tma<Tma16, tma_store_ok<Tma16>()>, true};
        }
        if constexpr (HASNARROW)
            t.v[t.n++] = {"narrow", Narrow::W, 16, whole_stages, col_launch_any<Narrow>};
        if constexpr (HASCLUSTER)
            t.v[t.n++] = {"cluster", Clu::W, 16, col_cluster_usable<Clu>, col_launch_cluster<Clu>};
        if constexpr (HASCLUSTER8)
            t.v[t.n++] = {"cluster8", Clu8::W, 16, col_cluster_usable<Clu8>,
                          col_launch_cluster<Clu8>};
        // the TMA engine with the next tile parked in TMEM (32 values a thread)
        if constexpr (HASTMEM)
            t.v[t.n++] = {"tmem", Tma32::W, 32, col_tma_usable<Tma32>, col_launch_tmem<Tma32>,
                          true};
        // half of each tile through TMA stores, half through per-thread stores
        if constexpr (HASTMEM && tma_store_ok<Tma32>())
            t.v[t.n++] = {"tma32h", Tma32::W, 32, col_tma_usable<Tma32>,
                          col_launch_tma<Tma32, true, true>, true};
        // 4096 rows in two groups of 6 stages (256 threads x 64 values): one
        // exchange through shared memory per tile instead of two
        if constexpr (L == 12)
            t.v[t.n++] = {"tma64", Tma64::W, 64, col_tma_usable<Tma64>,
                          col_launch_tma<Tma64, true, true>, true};
        // 1024 and 2048 rows in two groups (6 + 4, 6 + 5), per-thread stores
        if constexpr (L == 10 || L == 11)
            t.v[t.n++] = {"tma64st", Tma64::W, 64, col_tma_usable<Tma64>,
                          col_launch_tma<Tma64, false>, true};
        // 8192 and 16384 rows: 4-column tiles over a cluster of 2 or 4 CTAs,
        // the 4096-row engine on each CTA's rows and the last one or two
        // stages through bulk copies between the CTAs' shared memories
        if constexpr (L == 13)
            t.v[t.n++] = {"pair", PairLocal::W, 32, col_group_usable<PairLocal, 1>,
                          col_launch_group<PairLocal, 1>, true};
        if constexpr (L == 14)
            t.v[t.n++] = {"quad", PairLocal::W, 32, col_group_usable<PairLocal, 2>,
                          col_launch_group<PairLocal, 2>, true};
        // the same with the exchange through L2 (a scratch buffer; four CTAs
        // in one radix-4 round) and the local engine in two groups of 6
        // stages (256 threads x 64 values)
        if constexpr (L == 13)
            t.v[t.n++] = {"pairl2", PairLocal6::W, 64, col_group_usable<PairLocal6, 1>,
                          col_launch_group_l2<PairLocal6, 1>, true};
        if constexpr (L == 14)
            t.v[t.n++] = {"quadl2", PairLocal6::W, 64, col_group_usable<PairLocal6, 2>,
                          col_launch_group_l2<PairLocal6, 2>, true};
        return t;
    }
    static const Variant *table(int *n)
    {
        static const Table t = build();
        *n = t.n;
        return t.v;
    }
    static int index_of(const char *name)
    {
        int n = 0;
        const Variant *v = table(&n);
        for (int i = 0; i < n; i++)
            if (std::strcmp(v[i].name, name) == 0)
                return i;
        return 0;
    }
    // The default per column length, from timings of every variant on a
    // GB300 (512..4096 rows, square and 1:4 images): narrow tiles for 512 and
    // 1024 rows; the TMA pass in two groups of 6 stages with per-thread
    // stores for 2048, and with half TMA / half per-thread stores for 4096.
    static int preferred()
    {
        if constexpr (L == 9 || L == 10)
            return index_of("narrow");
        else if constexpr (L == 11)
            return index_of("tma64st");   // 20.7 vs 22.5 us for "tma32st" at 2048^2
        else if constexpr (L == 12)
            return index_of("tma64");     // 61.8 vs 66.0 us for "tma32h" at 4096^2
        else if constexpr (L == 13)
            return index_of("pairl2");    // 4-column tiles over a CTA pair (0.316 vs 0.334 ms for "pair")
        else if constexpr (L == 14)
            return index_of("quadl2");    // 4-column tiles over 4 CTAs (1.24 vs 1.83 ms for "quad")
        else
            return 0;
    }
};

}  // namespace

const Variant *col_variants(int L, int *n)
{
    switch (L) {
    case 1: return ColVariants<1>::table(n);
    case 2: return ColVariants<2>::table(n);
    case 3: return ColVariants<3>::table(n);
    case 4: return ColVariants<4>::table(n);
    case 5: return ColVariants<5>::table(n);
    case 6: return ColVariants<6>::table(n);
    case 7: return ColVariants<7>::table(n);
    case 8: return ColVariants<8>::table(n);
    case 9: return ColVariants<9>::table(n);
    case 10: return ColVariants<10>::table(n);
    case 11: return ColVariants<11>::table(n);
    case 12: return ColVariants<12>::table(n);
    case 13: return ColVariants<13>::table(n);
    case 14: return ColVariants<14>::table(n);
    default: *n = 0; return nullptr;
    }
}

int col_default_variant(int L)
{
    switch (L) {
    case 9: return ColVariants<9>::preferred();
    case 10: return ColVariants<10>::preferred();
    case 11: return ColVariants<11>::preferred();
    case 12: return ColVariants<12>::preferred();
    case 13: return ColVariants<13>::preferred();
    case 14: return ColVariants<14>::preferred();
    default: return 0;
    }
}

namespace {

// The variant launch_col_pass runs for these arguments (nullptr: none).
const Variant *select_col_variant(int L, const PassArgs &a)
{
    int n = 0;
    const Variant *v = col_variants(L, &n);
    if (!v || n == 0)
        return nullptr;
    int i = a.variant >= 0 && a.variant < n ? a.variant : col_default_variant(L);
    if (!v[i].usable(a))
        i = 0;   // the plain kernel serves every case
    return &v[i];
}

}  // namespace

cudaError_t launch_col_pass(int L, const PassArgs &a, cudaStream_t s)
{
    const Variant *v = select_col_variant(L, a);
    return v ? v->launch(a, s) : cudaErrorInvalidValue;
}

bool col_pass_is_tma_fed(int L, const PassArgs &a)
{
    const Variant *v = select_col_variant(L, a);
    return v && v->tma_fed;
}

// Stream-ordered scratch for the exchange rounds of col_group_l2_kernel,
// from a memory pool of the library's own per device (kept cached: its
// release threshold is unlimited, so after the first calls taking and
// returning a block costs no driver allocation).  A block is taken on the
// launch's stream and given back on it after the launch, so launches on
// different streams never share one, and under stream capture the pair
// becomes graph memory nodes.
cudaError_t scratch_take(void **p, size_t bytes, cudaStream_t s)
{
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static cudaMemPool_t pool[kMaxDev] = {};
    const int d = device_current();
    {
        std::lock_guard<std::mutex> g(mu);
        if (!pool[d]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = d;
            cudaMemPool_t mp;
            cudaError_t e = cudaMemPoolCreate(&mp, &props);
            if (e != cudaSuccess)
                return e;
            uint64_t keep = ~0ull;
            e = cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep);
            if (e != cudaSuccess) {
                cudaMemPoolDestroy(mp);
                return e;
            }
            pool[d] = mp;
        }
    }
    return cudaMallocFromPoolAsync(p, bytes, pool[d], s);
}

}  // namespace fft2d
