// col_pair.cuh -- persistent column pass for columns of 2^(L+1) rows whose
// 4-column tile is too large for one SM, split over a cluster of two CTAs.
//
// The DIT structure (Section 2 eqs. 2-3) splits the transform without any
// extra pass over memory.  After the scramble, positions p < 2^L hold the
// even rows and positions p >= 2^L the odd rows, each in the bit-reversed
// order of a 2^L-point line, and stages 1..L never mix the two halves.  So
// CTA b of the pair loads rows 2m + b of the tile by TMA (a tensor map with
// twice the row pitch), runs stages 1..L on them with the same engine as the
// single-CTA column pass (col_tma2_body: prefetch region, three stage
// groups, rotation factors in shared memory) and ends with Y_b[k], k < 2^L,
// in registers.  The last stage pairs Y_0[k] and Y_1[k]:
//     X[k] = Y_0[k] + W^k Y_1[k],   X[k + 2^L] = Y_0[k] - W^k Y_1[k],
// W = W_{2^(L+1)}.  Thread t holds the same indices k in both CTAs, so the
// two twins exchange half of their values: CTA b keeps the k of its half
// (top bit of k/2^(L-1) equal to b).  Each thread writes the partner's half
// into a send buffer, one thread moves the whole buffer into the partner's
// shared memory with a single bulk copy that completes on the partner's
// mbarrier, and each CTA then runs the last stage on its half and writes
// rows k and k + 2^L of it with two TMA stores.
//
// Cluster barriers have no time limit, so both CTAs always execute the same
// sequence of them: a CTA that lost a TMA transfer still reaches the next
// cluster barrier, where the two exchange a "lost" flag and leave together.
#pragma once

#include <cooperative_groups.h>

#include "line_fft.cuh"

namespace fft2d {

__device__ __forceinline__ void cluster_arrive_release()
{
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}

__device__ __forceinline__ void cluster_wait_acquire()
{
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// Bulk copy from this CTA's shared memory into another CTA's (dst and its
// mbarrier are shared::cluster addresses); completes on that mbarrier.
__device__ __forceinline__ void bulk_copy_to_peer(uint32_t dst, const void *src, uint32_t bytes,
                                                  uint32_t peer_bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(dst),
        "r"(smem_addr(src)), "r"(bytes), "r"(peer_bar)
        : "memory");
}

// Tile geometry of the pair kernel for a local engine C (2^L rows, W
// columns, 512 threads x 32 values).
template <class C>
struct PairCol {
    using S = TmaSplit<C>;
    using Gl = Grp<C, C::NG - 1>;
    static constexpr int L = C::L;                        // local stages
    static constexpr int NL = C::N;                       // local rows
    static constexpr int HALF_R = Gl::R / 2;              // register indices of one output half
    static constexpr int RECV = Gl::V * HALF_R;           // values received per thread
    static constexpr int OUT_BOX_Z = (NL / 2) / S::BOX;   // 256-row blocks of one output half
    static constexpr uint32_t XBYTES = (uint32_t)RECV * C::T * 8u;   // values exchanged per CTA
    static_assert(C::EPT == 32 && C::NG == 3 && C::LB == 1, "512 threads x 32 values, 3 groups");
    static_assert(Gl::S0 + Gl::G == L && (NL >> Gl::S0) == Gl::R,
                  "the last group's register index is the top bits of k");
    static_assert(RECV * C::T * 8 <= C::E * 4, "the receive buffer fits in half the tile region");
    static_assert((NL / 2) % S::BOX == 0, "output halves are whole 256-row blocks");
};

// C: the local engine; CTA rank b of the cluster.  lmap: this CTA's load map
// (rows b, b+2, ... of the image; box W x 256 x NB); omap: store map over the
// output (box W x 256 x OUT_BOX_Z); twl: rotation factors of the local stages
// (2^L entries, padding included); tw_last: W_{2^(L+1)}^k, k < 2^L.
template <class C>
__device__ __forceinline__ void col_pair_body(const CUtensorMap *lmap, const CUtensorMap *omap,
                                              int ntiles, const float2 *__restrict__ twl,
                                              const float2 *__restrict__ tw_last, float scale,
                                              int *err, int withhold)
{
    namespace cg = cooperative_groups;
    using S = TmaSplit<C>;
    using PC = PairCol<C>;
    using Gl = Grp<C, C::NG - 1>;
    extern __shared__ __align__(1024) float2 sm[];
    __shared__ __align__(8) uint64_t bar_early, bar_late, bar_recv;
    __shared__ int lost_flag[2];   // [0] this CTA, [1] written by the partner
    cg::cluster_group cluster = cg::this_cluster();
    const int b = (int)cluster.block_rank();
    const int tid = threadIdx.x;
    const int nclusters = (int)gridDim.x / 2;
    float2 *stw = sm + S::TW_OFF;
    // after the last read of a tile: the lower half of the tile region
    // receives the partner's values, the upper half holds the values sent
    // and then stages the output
    float2 *recvb = sm;
    float2 *sendb = sm + C::E / 2;
    const uint32_t peer_recv = mapa_shared(smem_addr(recvb), (uint32_t)(b ^ 1));
    const uint32_t peer_bar = mapa_shared(smem_addr(&bar_recv), (uint32_t)(b ^ 1));
    int *peer_flag = cluster.map_shared_rank(lost_flag + 1, b ^ 1);   // its slot [1]
    int lost_recv = 0;
    int tile = (int)blockIdx.x / 2;

    if (tid == 0) {
        mbar_init(&bar_early, 1);
        mbar_init(&bar_late, 1);
        mbar_init(&bar_recv, 1);
        fence_mbar_init();
    }
    __syncthreads();
    // issued / waited phases of each mbarrier (thread 0 issues, all wait)
    int n_early = 0, n_late = 0, w_early = 0, w_late = 0;
    if (tile < ntiles) {
        if (tid == 0) {
            mbar_expect_tx(&bar_early, S::TW_BYTES);
            bulk_load(stw, twl, S::TW_BYTES, &bar_early);
            split_issue_early<C>(sm, lmap, tile * C::W, &bar_early);
            // (self-test: CTA 0 withholds its first late boxes)
            if (!(withhold && blockIdx.x == 0))
                split_issue_late<C>(sm, lmap, tile * C::W, &bar_late);
        }
        n_early = n_late = 1;
    }
    bool lost = false;
    int w_recv = 0;   // completed phases of bar_recv
    float2 a[C::EPT];
    for (; tile < ntiles; tile += nclusters) {
        const int next = tile + nclusters;
        const bool ok = mbar_wait_bounded(&bar_early, (uint32_t)(w_early & 1)) &&
                        mbar_wait_bounded(&bar_late, (uint32_t)(w_late & 1));
        // a receive that timed out on the previous tile counts as lost too
        const int lost_here = __syncthreads_or((ok ? 0 : 1) | lost_recv);
        // the "lost" flags for cluster barrier X1 and the arming of the
        // receive mbarrier, early so the remote flag store is long done
        // when X1 is arrived at (the partner reads the flag after X1 and
        // writes the next one only after X2)
        if (tid == 0) {
            if (!lost_recv)   // (a phase that timed out may still be open)
                mbar_arrive_expect_tx(&bar_recv, PC::XBYTES);
            lost_flag[0] = lost_here;
            *peer_flag = lost_here;
        }
        if (!lost_here) {
            w_early++;
            w_late++;
            group_first_split<C>(
                a, sm, stw,
                [&] {
                    if (tid == 0)
                        bulk_wait_read_all();   // the previous tile's stores have read T
                },
                [&] {
                    if (tid == 0 && next < ntiles)
                        split_issue_early<C>(sm, lmap, next * C::W, &bar_early);
                });
            if (next < ntiles)
                n_early++;
            __syncthreads();
            group_smem<C, 1, false, false, true>(a, sm, stw, C::L);
            __syncthreads();
            group_last_read<C>(a, sm);
            __syncthreads();   // the tile region is free
        }
        // cluster barrier X1, arrive: this CTA's tile region is free and its
        // receive mbarrier armed; the "lost" flags travel with it
        cluster_arrive_release();
        float2 wk[PC::RECV];
        if (!lost_here) {
#pragma unroll
            for (int v = 0; v < Gl::V; v++) {
                const int u = tid + v * C::T;
                const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
                run_stages<C, C::NG - 1, false, true>(a, v, lo, stw, C::L);
            }
            // the partner's half -- register index r with top bit != b --
            // into the send buffer, slot (v * HALF_R + (r mod HALF_R)) * T + tid
#pragma unroll
            for (int v = 0; v < Gl::V; v++) {
#pragma unroll
                for (int i = 0; i < PC::HALF_R; i++) {
                    const float2 lo_half = a[v * Gl::R + i], hi_half = a[v * Gl::R + PC::HALF_R + i];
                    sendb[(v * PC::HALF_R + i) * C::T + tid] = b == 0 ? hi_half : lo_half;
                }
            }
            fence_proxy_async_smem();
        }
        __syncthreads();   // the send buffer is complete
        // rotation factors of the last stage, W^k for this CTA's k (read from
        // global memory; their latency hides behind the cluster barrier)
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
            const int u = tid + v * C::T;
            const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
#pragma unroll
            for (int i = 0; i < PC::HALF_R; i++) {
                const int k = lo | ((b * PC::HALF_R + i) << Gl::S0);
                wk[v * PC::HALF_R + i] = __ldg(tw_last + k);
            }
        }
        cluster_wait_acquire();
        if (lost_flag[0] | lost_flag[1]) {
            lost = true;
            break;
        }
        // the partner's tile region is free: one bulk copy of the send
        // buffer into it, completing on the partner's receive mbarrier
        if (tid == 0)
            bulk_copy_to_peer(peer_recv, sendb, PC::XBYTES, peer_bar);
        lost_recv = mbar_wait_bounded(&bar_recv, (uint32_t)(w_recv & 1)) ? 0 : 1;
        if (!lost_recv)
            w_recv++;
        // cluster barrier X2, arrive: the partner's send buffer has been read
        cluster_arrive_release();

        // the last stage on this CTA's half
        float2 o[2][PC::RECV];
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
#pragma unroll
            for (int i = 0; i < PC::HALF_R; i++) {
                const int j = v * PC::HALF_R + i;
                const float2 lo_half = a[v * Gl::R + i], hi_half = a[v * Gl::R + PC::HALF_R + i];
                const float2 mine = b == 0 ? lo_half : hi_half;
                const float2 theirs = recvb[j * C::T + tid];
                float2 x0 = b == 0 ? mine : theirs;
                float2 x1 = b == 0 ? theirs : mine;
                butterfly_w(x0, x1, wk[j]);
                o[0][j] = make_float2(x0.x * scale, x0.y * scale);
                o[1][j] = make_float2(x1.x * scale, x1.y * scale);
            }
        }
        fence_proxy_async_smem();
        __syncthreads();   // the receive buffer has been read
        if (tid == 0 && next < ntiles)
            split_issue_late<C>(sm, lmap, next * C::W, &bar_late);
        if (next < ntiles)
            n_late++;
        // X2, wait: this CTA's send buffer is free for staging
        cluster_wait_acquire();

        // rows k and k + 2^L of this half: two TMA stores from the staging
        // buffer (the send buffer)
#pragma unroll
        for (int h = 0; h < 2; h++) {
            if (h == 1) {
                if (tid == 0)
                    bulk_wait_read_all();
                __syncthreads();
            }
#pragma unroll
            for (int v = 0; v < Gl::V; v++) {
                const int u = tid + v * C::T;
                const int w = u & (C::W - 1);
                const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
#pragma unroll
                for (int i = 0; i < PC::HALF_R; i++)
                    sendb[((i << Gl::S0) | lo) * C::W + w] = o[h][v * PC::HALF_R + i];
            }
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                // rows h 2^L + b 2^(L-1) + [0, 2^(L-1)): 256-row blocks from z
                const int z = (h * PC::NL + b * (PC::NL / 2)) / S::BOX;
                tma_store_3d(omap, tile * C::W, 0, z, sendb);
                bulk_commit();
            }
        }
    }

    if (__syncthreads_or((lost || lost_recv) ? 1 : 0)) {
        if (tid == 0)
            atomicExch(err, kDevErrTmaTimeout);
        // let transfers still in flight land before the CTA leaves
        if (n_early > w_early)
            mbar_wait_bounded(&bar_early, (uint32_t)(w_early & 1));
        if (n_late > w_late)
            mbar_wait_bounded(&bar_late, (uint32_t)(w_late & 1));
        if (lost_recv)
            mbar_wait_bounded(&bar_recv, (uint32_t)(w_recv & 1));
    }
    if (tid == 0)
        bulk_wait_all();   // shared memory stays valid until the stores are done
}

template <class C>
__global__ void __launch_bounds__(C::T, 1) col_pair_kernel(const __grid_constant__ CUtensorMap map0,
                                                           const __grid_constant__ CUtensorMap map1,
                                                           const __grid_constant__ CUtensorMap omap,
                                                           const float2 *__restrict__ tw,
                                                           int cols, float scale, int *err,
                                                           int withhold)
{
    const bool odd = (cooperative_groups::this_cluster().block_rank() & 1) != 0;
    // the local stages use entries [0, 2^L) of the table, the last stage
    // entries 2^L - 1 + k (stage L+1 starts at offset 2^L - 1)
    col_pair_body<C>(odd ? &map1 : &map0, &omap, cols / C::W, tw, tw + (C::N - 1), scale, err,
                     withhold);
}

}  // namespace fft2d
