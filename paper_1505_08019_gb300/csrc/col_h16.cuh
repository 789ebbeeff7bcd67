// col_h16.cuh -- persistent TMA-fed column pass for half2 storage (one
// power-of-two exponent per line, FP32 arithmetic).
//
// The arithmetic is the FP32 column engine's (a tile of W = 4 whole columns
// of 2^L rows; 256 threads x 64 values in two groups of radix-2 DIT stages,
// or 512 x 32 in three,
// Section 2 eqs. 2-3 / Section 3.1 eq. 4, the scramble of Section 3.2 fused
// into the first read), so the results are those of the complex64 column
// pass on the dequantised input, rounded once to half precision at the end.
// Only the storage differs:
//
//  * The tile arrives as half2 (4 bytes a pixel): its first half (the early
//    256-row blocks) in a prefetch region, its second half at the start of
//    the FP32 exchange region once the previous tile's last group has read
//    it, both by TMA with 16-byte box rows.
//  * Group 0 gathers it scrambled, widens each value to FP32 and applies its
//    row's input scale 2^e (the row pass's exponents, converted once per CTA
//    into a table of factors in shared memory).
//  * After the last group, the CTA max-reduces |component| per column
//    (warp shuffles, then one shared atomic per warp and column), picks each
//    column's exponent (e = k - 14 for a maximum of f 2^k, f in [0.5, 1)),
//    stages the finished tile as half2 in the upper half of the exchange
//    region in natural row order and stores it with one TMA store, which
//    drains while the next tile's group 0 runs.
//
// Every mbarrier wait is bounded; on a timeout the kernel records
// kDevErrTmaTimeout, drains its stores and lets the transfers in flight land
// before it returns.
#pragma once

#include "line_fft.cuh"

namespace fft2d {

template <class C>
struct H16Col {
    static constexpr int BOX = 256;                         // rows per TMA block
    static constexpr int NBOX = C::N / BOX;
    static constexpr int NB = NBOX / 2;                     // early blocks
    static constexpr int BOXV = BOX * C::W;                 // half2 values per block
    static constexpr int X_BYTES = C::E * 8;                // FP32 exchange region
    static constexpr int PREF_OFF = X_BYTES;                // early half of the next tile
    static constexpr uint32_t EARLY_BYTES = (uint32_t)NB * BOXV * 4u;
    static constexpr uint32_t LATE_BYTES = (uint32_t)(NBOX - NB) * BOXV * 4u;
    static constexpr int TW_OFF = PREF_OFF + (int)EARLY_BYTES;   // rotation factors
    static constexpr uint32_t TW_BYTES = (uint32_t)C::N * 8u;     // N-1 entries + padding
    static constexpr int RF_OFF = TW_OFF + (int)TW_BYTES;         // 2^e of every image row
    static constexpr int SMEM_BYTES = RF_OFF + C::N * 4;
    static constexpr int STAGE_OFF = X_BYTES / 2;           // finished half2 tile
    static_assert(C::W == 4 && C::LB == 1 &&
                      ((C::EPT == 32 && C::NG == 3) || (C::EPT == 64 && C::NG == 2)),
                  "4-column tiles; 512 threads x 32 values in three stage groups or 256 x 64 "
                  "in two");
    static_assert(NB >= 1 && 2 * NB == NBOX, "two equal halves of whole blocks");
    static_assert(LATE_BYTES <= (uint32_t)STAGE_OFF, "the late half and the staging never overlap");
    static_assert(STAGE_OFF + C::E * 4 <= X_BYTES, "the staging fits in the exchange region");
    static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
};

template <class C>
__device__ __forceinline__ void h16_issue(void *dst, const CUtensorMap *map, int c0, int z,
                                          uint32_t bytes, uint64_t *bar)
{
    mbar_arrive_expect_tx(bar, bytes);
    tma_load_3d(dst, map, c0, 0, z, bar);
}

// map: load map over the half2 input (box 4 x 256 x NB); omap: store map over
// the half2 output (box 4 x 256 x NBOX, the whole tile); tw: the column
// axis's rotation factors (N entries with padding); row_exp: the input's
// exponent of every row; out_exp: one exponent per output column.
template <class C>
__global__ void __launch_bounds__(C::T, 1) col_h16_tma_kernel(const __grid_constant__ CUtensorMap map,
                                                              const __grid_constant__ CUtensorMap omap,
                                                              const float2 *__restrict__ tw,
                                                              const int *__restrict__ row_exp,
                                                              int *out_exp, int cols, float scale,
                                                              int *err)
{
    using H = H16Col<C>;
    using G0 = Grp<C, 0>;
    using GL = Grp<C, C::NG - 1>;
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar_early, bar_late;
    __shared__ int sred[C::W];
    float2 *sm = reinterpret_cast<float2 *>(smraw);
    const __half2 *pref = reinterpret_cast<const __half2 *>(smraw + H::PREF_OFF);
    const __half2 *late = reinterpret_cast<const __half2 *>(smraw);
    float2 *stw = reinterpret_cast<float2 *>(smraw + H::TW_OFF);
    float *rf = reinterpret_cast<float *>(smraw + H::RF_OFF);
    __half2 *stage = reinterpret_cast<__half2 *>(smraw + H::STAGE_OFF);
    const int ntiles = cols / C::W;
    const int tid = threadIdx.x;
    int tile = blockIdx.x;
    if (tid == 0) {
        mbar_init(&bar_early, 1);
        mbar_init(&bar_late, 1);
        fence_mbar_init();
    }
    if (tid < C::W)
        sred[tid] = 0;
    for (int i = tid; i < C::N; i += C::T)
        rf[i] = pow2f(row_exp[i]);
    __syncthreads();
    if (tid == 0 && tile < ntiles) {
        mbar_expect_tx(&bar_early, H::TW_BYTES);
        bulk_load(stw, tw, H::TW_BYTES, &bar_early);
        h16_issue<C>(smraw + H::PREF_OFF, &map, tile * C::W, 0, H::EARLY_BYTES, &bar_early);
        h16_issue<C>(smraw, &map, tile * C::W, H::NB, H::LATE_BYTES, &bar_late);
    }
    uint32_t parity = 0;
    float2 a[C::EPT];
    for (; tile < ntiles; tile += gridDim.x) {
        const int next = tile + gridDim.x;
        const int c0 = tile * C::W;
        const bool ok = mbar_wait_bounded(&bar_early, parity) && mbar_wait_bounded(&bar_late, parity);
        if (__syncthreads_or(ok ? 0 : 1)) {
            if (tid == 0) {
                atomicExch(err, kDevErrTmaTimeout);
                bulk_wait_all();
            }
            mbar_wait_bounded(&bar_early, parity);
            mbar_wait_bounded(&bar_late, parity);
            return;
        }
        parity ^= 1;
        // group 0: scrambled gather of the half2 tile, widened and scaled by
        // the row factors
#pragma unroll
        for (int v = 0; v < G0::V; v++) {
            const int u = tid + v * C::T;
            const int w = u & (C::W - 1);
            const int hib = (u >> C::KW) & ((1 << G0::HB) - 1);
#pragma unroll
            for (int r = 0; r < G0::R; r++) {
                const int top = brev_c(r, G0::G) << G0::HB;   // compile-time
                const int k = top / H::BOX;
                const int in_box = ((top % H::BOX) | hib) * C::W + w;
                const __half2 *bx = k < H::NB ? pref + k * H::BOXV : late + (k - H::NB) * H::BOXV;
                const float2 q = __half22float2(bx[in_box]);
                const float f = rf[top | hib];
                a[v * G0::R + r] = make_float2(q.x * f, q.y * f);
            }
        }
#pragma unroll
        for (int v = 0; v < G0::V; v++)
            run_stages<C, 0, false, true>(a, v, 0, stw, C::L);
        fence_proxy_async_smem();
        if (tid == 0)
            bulk_wait_read_all();   // the previous tile's staging has been stored
        __syncthreads();            // every slot of both input regions has been read
        if (tid == 0 && next < ntiles)
            h16_issue<C>(smraw + H::PREF_OFF, &map, next * C::W, 0, H::EARLY_BYTES, &bar_early);
#pragma unroll
        for (int v = 0; v < G0::V; v++) {
            const int u = tid + v * C::T;
            const int w = u & (C::W - 1);
            const int hib = (u >> C::KW) & ((1 << G0::HB) - 1);
            const int hi = brev_rt(hib, G0::HB);
#pragma unroll
            for (int r = 0; r < G0::R; r++)
                sm[sidx<C>(0, r | (hi << G0::G), w)] = a[v * G0::R + r];
        }
        __syncthreads();
        if constexpr (C::NG >= 3) {
            group_smem<C, 1, false, false, true>(a, sm, stw, C::L);
            __syncthreads();
        }
        group_last_read<C>(a, sm);
        fence_proxy_async_smem();
        __syncthreads();   // the exchange region is free
        if (tid == 0 && next < ntiles)
            h16_issue<C>(smraw, &map, next * C::W, H::NB, H::LATE_BYTES, &bar_late);
        // the last group, then the column maxima (a thread's values all
        // belong to column w = tid mod W)
        float m = 0.f;
#pragma unroll
        for (int v = 0; v < GL::V; v++) {
            const int u = tid + v * C::T;
            const int lo = (u >> C::KW) & ((1 << GL::S0) - 1);
            run_stages<C, C::NG - 1, false, true>(a, v, lo, stw, C::L);
#pragma unroll
            for (int r = 0; r < GL::R; r++)
                m = fmaxf(m, fmaxf(fabsf(a[v * GL::R + r].x), fabsf(a[v * GL::R + r].y)));
        }
        m = warp_line_max<C::KW, 5>(m);
        if ((tid & (31 & ~(C::W - 1))) == 0)
            atomicMax(&sred[tid & (C::W - 1)], __float_as_int(m * scale));
        __syncthreads();
        const int w = tid & (C::W - 1);
        const int e = line_exponent(__int_as_float(sred[w]));
        const float f = scale * pow2f(-e);
#pragma unroll
        for (int v = 0; v < GL::V; v++) {
            const int u = tid + v * C::T;
            const int lo = (u >> C::KW) & ((1 << GL::S0) - 1);
#pragma unroll
            for (int r = 0; r < GL::R; r++) {
                const float2 x = a[v * GL::R + r];
                stage[((r << GL::S0) | lo) * C::W + w] = __floats2half2_rn(x.x * f, x.y * f);
            }
        }
        if (tid < C::W)
            out_exp[c0 + tid] = e;
        fence_proxy_async_smem();
        __syncthreads();   // staging complete; every thread has read sred
        if (tid < C::W)
            sred[tid] = 0;
        if (tid == 0) {
            tma_store_3d(&omap, c0, 0, 0, stage);
            bulk_commit();
        }
    }
    if (tid == 0)
        bulk_wait_all();   // shared memory stays valid until the stores are done
}

}  // namespace fft2d
