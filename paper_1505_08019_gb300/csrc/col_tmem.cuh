// col_tmem.cuh -- persistent column pass that parks the next tile in tensor
// memory (TMEM).
//
// Same arithmetic, stage grouping and tile shape as col_tma2_body (a tile of
// W whole columns of 2^L rows, 512 threads x 32 values, three groups of
// radix-2 DIT stages, Section 2 eqs. 2-3 / Section 3.1 eq. 4, scramble of
// Section 3.2 fused into the first read), but a different use of on-chip
// memory:
//
//  * The next tile streams, one half at a time, into a 64 KB landing region
//    P by TMA.  As soon as a half has landed -- at a point where the current
//    tile sits in shared memory between two stage groups and the registers
//    are free -- every thread copies its own group-0 inputs out of P
//    (scrambled, exactly the values it will need) into its private TMEM
//    columns, and P is refilled.  Early half = the even register indices r of
//    each group-0 unit (rows whose top bit is 0), late half = the odd ones.
//  * The 128 KB tile region is therefore only the exchange buffer between
//    groups and, at the end, the staging buffer of the whole finished tile,
//    which leaves with ONE TMA store and no wait in the middle of the last
//    group.
//  * Group 0 of the next tile reads its 32 values back with one tcgen05.ld.
//
// TMEM use: 64 32-bit columns per thread (32 complex values), 4 warps per
// lane quadrant -> 256 columns per CTA (one CTA per SM: the 224 KB of shared
// memory guarantee it).  Every wait is bounded; on a timeout the kernel
// records kDevErrTmaTimeout, lets the transfer in flight land, drains its
// stores and frees its TMEM before returning.
#pragma once

#include "line_fft.cuh"
#include "tmem.cuh"

namespace fft2d {

template <class C>
struct TmemCol {
    using S = TmaSplit<C>;
    using G0 = Grp<C, 0>;
    static constexpr int WARPS = C::T / 32;
    static constexpr uint32_t COLS_PER_THREAD = 2u * C::EPT;   // re, im of EPT values
    static constexpr uint32_t HALF_COLS = COLS_PER_THREAD / 2;
    static constexpr uint32_t TMEM_COLS = (uint32_t)(WARPS / 4) * COLS_PER_THREAD;
    static constexpr bool even_r_is_early()
    {
        for (int r = 0; r < G0::R; r++) {
            const int k = (brev_c(r, G0::G) << G0::HB) / S::BOX;
            if ((k < S::NB) != (r % 2 == 0))
                return false;
        }
        return true;
    }
    static_assert(C::EPT == 32 && C::NG == 3 && C::LB == 1, "512 threads x 32 values, 3 groups");
    static_assert(WARPS % 4 == 0, "whole lane quadrants");
    static_assert(TMEM_COLS >= 32 && TMEM_COLS <= 512 && (TMEM_COLS & (TMEM_COLS - 1)) == 0,
                  "TMEM allocation is a power of two from 32 to 512 columns");
    static_assert(G0::V * (G0::R / 2) * 2 == 32, "each half is 32 columns of a thread");
    static_assert(even_r_is_early(), "the early boxes hold exactly the even register indices");
};

// Copy this thread's group-0 inputs of one half (H = 0 early, 1 late) of the
// tile in P into its TMEM columns [H*32, H*32 + 32).
template <class C, int H>
__device__ __forceinline__ void tmem_drain_half(const float2 *P, uint32_t taddr)
{
    using Gp = Grp<C, 0>;
    using S = TmaSplit<C>;
    const int tid = threadIdx.x;
    uint32_t f[32];
#pragma unroll
    for (int v = 0; v < Gp::V; v++) {
        const int u = tid + v * C::T;
        const int w = u & (C::W - 1);
        const int hib = (u >> C::KW) & ((1 << Gp::HB) - 1);
#pragma unroll
        for (int i = 0; i < Gp::R / 2; i++) {
            const int r = 2 * i + H;
            const int top = brev_c(r, Gp::G) << Gp::HB;      // compile-time
            const int k = top / S::BOX - H * S::NB;
            const float2 x = P[k * S::BOX_VALS + ((top % S::BOX) | hib) * C::W + w];
            const int idx = v * (Gp::R / 2) + i;
            f[2 * idx] = __float_as_uint(x.x);
            f[2 * idx + 1] = __float_as_uint(x.y);
        }
    }
    tmem_st32(taddr + (uint32_t)(H * 32), f);
}

// Group-0 values of the tile parked in TMEM -> registers.
template <class C>
__device__ __forceinline__ void tmem_fetch_tile(float2 (&a)[C::EPT], uint32_t taddr)
{
    using Gp = Grp<C, 0>;
    uint32_t f[64];
    tmem_ld64(taddr, f);
#pragma unroll
    for (int v = 0; v < Gp::V; v++) {
#pragma unroll
        for (int r = 0; r < Gp::R; r++) {
            const int idx = (r & 1) * 16 + v * (Gp::R / 2) + (r >> 1);
            a[v * Gp::R + r] = make_float2(__uint_as_float(f[2 * idx]), __uint_as_float(f[2 * idx + 1]));
        }
    }
}

template <class C>
__device__ __forceinline__ void tmem_issue_half(float2 *P, const CUtensorMap *map, int c0, int h,
                                                uint64_t *bar)
{
    using S = TmaSplit<C>;
    mbar_arrive_expect_tx(bar, h == 0 ? S::EARLY_BYTES : S::LATE_BYTES);
    tma_load_3d(P, map, c0, 0, h == 0 ? 0 : S::NB, bar);
}

// Persistent body: CTA b takes tiles b, b + grid, ...  Shared memory: tile
// region T (E values), landing region P (E/2), rotation factors.  omap's box
// is the whole tile (W x 256 x N/256), stored from T in natural row order.
// withhold (self-test): CTA 0 does not issue its first tile's late half.
template <class C, class Src>
__device__ __forceinline__ void col_tmem_body(const Src &src, int ntiles,
                                              const float2 *__restrict__ tw, int *err,
                                              int withhold)
{
    using S = TmaSplit<C>;
    using TC = TmemCol<C>;
    using Gl = Grp<C, C::NG - 1>;
    extern __shared__ __align__(1024) float2 sm[];
    __shared__ __align__(8) uint64_t bar_early, bar_late;
    __shared__ uint32_t tmem_base;
    float2 *T = sm;
    float2 *P = sm + C::E;
    float2 *stw = sm + S::TW_OFF;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const int grid = (int)gridDim.x;
    int tile = blockIdx.x;
    if (tile >= ntiles)
        return;   // whole CTA, before anything is allocated

    if (warp == 0) {
        tmem_alloc(&tmem_base, TC::TMEM_COLS);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(&bar_early, 1);
        mbar_init(&bar_late, 1);
        fence_mbar_init();
    }
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const uint32_t taddr = tmem_base + ((uint32_t)((warp & 3) * 32) << 16) +
                           (uint32_t)(warp >> 2) * TC::COLS_PER_THREAD;

    // which transfer a timed-out CTA must still let land: 0 none, 1 early, 2 late
    int pending = 0;
    uint32_t pending_parity = 0;
    bool lost = false;

    // prologue: the first tile (and the rotation factors) through P into TMEM
    if (tid == 0) {
        mbar_expect_tx(&bar_early, S::TW_BYTES);
        bulk_load(stw, tw, S::TW_BYTES, &bar_early);
        tmem_issue_half<C>(P, src.tmap(tile), src.col(tile), 0, &bar_early);
    }
    lost = __syncthreads_or(mbar_wait_bounded(&bar_early, 0) ? 0 : 1);
    if (lost) {
        pending = 1;
    } else {
        tmem_drain_half<C, 0>(P, taddr);
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0 && !(withhold && blockIdx.x == 0))
            tmem_issue_half<C>(P, src.tmap(tile), src.col(tile), 1, &bar_late);
        lost = __syncthreads_or(mbar_wait_bounded(&bar_late, 0) ? 0 : 1);
        if (lost) {
            pending = 2;
        } else {
            tmem_drain_half<C, 1>(P, taddr);
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0 && tile + grid < ntiles)
                tmem_issue_half<C>(P, src.tmap(tile + grid), src.col(tile + grid), 0, &bar_early);
        }
    }

    float2 a[C::EPT];
    for (int it = 0; !lost && tile < ntiles; tile += grid, it++) {
        const int next = tile + grid;
        const uint32_t pn = (uint32_t)((it + 1) & 1);   // phase parity of the next tile's halves

        // group 0 from TMEM, then the exchange into T (once the previous
        // tile's store has finished reading it)
        tmem_fetch_tile<C>(a, taddr);
#pragma unroll
        for (int v = 0; v < Grp<C, 0>::V; v++)
            run_stages<C, 0, false, true>(a, v, 0, stw, C::L);
        if (tid == 0)
            bulk_wait_read_all();
        __syncthreads();
        {
            using Gp = Grp<C, 0>;
#pragma unroll
            for (int v = 0; v < Gp::V; v++) {
                const int u = tid + v * C::T;
                const int w = u & (C::W - 1);
                const int hib = (u >> C::KW) & ((1 << Gp::HB) - 1);
                const int hi = brev_rt(hib, Gp::HB);
#pragma unroll
                for (int r = 0; r < Gp::R; r++)
                    T[sidx<C>(0, r | (hi << Gp::G), w)] = a[v * Gp::R + r];
            }
        }
        __syncthreads();
        group_smem<C, 1, false, false, true>(a, T, stw, C::L);
        __syncthreads();

        // the next tile's early half: P -> TMEM, then its late half -> P
        if (next < ntiles) {
            lost = __syncthreads_or(mbar_wait_bounded(&bar_early, pn) ? 0 : 1);
            if (lost) {
                pending = 1;
                pending_parity = pn;
                break;
            }
            tmem_drain_half<C, 0>(P, taddr);
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0)
                tmem_issue_half<C>(P, src.tmap(next), src.col(next), 1, &bar_late);
        }

        // last group: read, stages, stage the whole tile in T, one TMA store
        group_last_read<C>(a, T);
        __syncthreads();
        const float scale = src.scl(tile);
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
            const int u = tid + v * C::T;
            const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
            run_stages<C, C::NG - 1, false, true>(a, v, lo, stw, C::L);
        }
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
            const int u = tid + v * C::T;
            const int w = u & (C::W - 1);
            const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
#pragma unroll
            for (int r = 0; r < Gl::R; r++) {
                const float2 x = a[v * Gl::R + r];
                T[(lo | (r << Gl::S0)) * C::W + w] = make_float2(x.x * scale, x.y * scale);
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tma_store_3d(src.omap(tile), src.col(tile), 0, 0, T);
            bulk_commit();
        }

        // the next tile's late half: P -> TMEM, then the early half after it
        if (next < ntiles) {
            lost = __syncthreads_or(mbar_wait_bounded(&bar_late, pn) ? 0 : 1);
            if (lost) {
                pending = 2;
                pending_parity = pn;
                break;
            }
            tmem_drain_half<C, 1>(P, taddr);
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0 && next + grid < ntiles)
                tmem_issue_half<C>(P, src.tmap(next + grid), src.col(next + grid), 0, &bar_early);
        }
    }

    if (lost) {
        if (tid == 0)
            atomicExch(err, kDevErrTmaTimeout);
        // the transfer that timed out may still land in P: give it time
        if (pending == 1)
            mbar_wait_bounded(&bar_early, pending_parity);
        else if (pending == 2)
            mbar_wait_bounded(&bar_late, pending_parity);
    }
    if (tid == 0)
        bulk_wait_all();   // shared memory stays valid until the stores are done
    tmem_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tmem_fence_after_sync();
        tmem_dealloc(tmem_base, TC::TMEM_COLS);
    }
}

template <class C>
__global__ void __launch_bounds__(C::T, 1) col_tmem_kernel(const __grid_constant__ CUtensorMap map,
                                                           const __grid_constant__ CUtensorMap omap,
                                                           float2 *out,
                                                           const float2 *__restrict__ tw,
                                                           int cols, long long ld, float scale,
                                                           int *err, int withhold)
{
    const TilesOneImage src{&map, &omap, out, ld, scale, C::W};
    col_tmem_body<C>(src, cols / C::W, tw, err, withhold);
}

}  // namespace fft2d
