// col_group.cuh -- persistent column pass for columns of 2^(L+c) rows whose
// 4-column tile is too large for one SM, split over a cluster of CS = 2^c
// CTAs (c = 1: a CTA pair for 8192 rows; c = 2: four CTAs for 16384 rows).
//
// The DIT structure (Section 2 eqs. 2-3) splits the transform without any
// extra pass over memory.  After the scramble, the positions P = k + 2^L q,
// k < 2^L, q < CS, with the same q hold the rows m = CS m' + rev_c(q) in the
// bit-reversed order of a 2^L-point line, and stages 1..L never mix
// different q.  So CTA q of the cluster loads rows CS m' + rev_c(q) of the
// tile by TMA (a tensor map with CS times the row pitch), runs stages 1..L
// on them with the same engine as the single-CTA column pass (prefetch
// region, three stage groups, rotation factors in shared memory) and ends
// with Y_q[k], k < 2^L, in registers.  The last c stages each pair values
// of two CTAs: stage L+1+j pairs positions that differ in bit L+j, i.e. the
// CTAs q and q ^ 2^j, with
//     X[P] = Y[P] + W^i Y[P + 2^(L+j)],  X[P + 2^(L+j)] = Y[P] - W^i Y[P + 2^(L+j)],
// W = W_{2^(L+j+1)}, i = P mod 2^(L+j).  Thread t holds the same indices k
// in every CTA, so in round j the two partners split the k that are still
// theirs by bit L-1-j of k: each keeps one half and hands the values of the
// other half to its partner.  After c rounds CTA q holds, for a contiguous
// quarter (c = 2) or half (c = 1) of the k, all CS outputs X[k + 2^L t] and
// writes them with TMA stores.
//
// Two kernels move the values.  col_group_kernel: one thread moves a send
// buffer into the partner's shared memory with a single bulk copy that
// completes on the partner's mbarrier, two cluster barriers per round.
// col_group_l2_kernel (the default): the values go through a scratch block
// in global memory, resident in L2, one cluster barrier per exchange, and
// four CTAs exchange once and run both cross stages together (radix 4).
// Only the second has a half2 storage mode (H16): the tile arrives as half2
// (16-byte TMA box rows) and group 0 widens each value with its row's factor
// 2^e, as in the single-CTA half2 column pass; at the end every CTA
// max-reduces its part of each column, the partial maxima travel to every
// CTA of the cluster through one more cluster barrier, and all CTAs pick the
// same exponent per column before staging their ranges as half2.
//
// Cluster barriers have no time limit, so every CTA always executes the same
// sequence of them: a CTA that lost a TMA transfer still reaches the first
// cluster barrier of the tile, where all CTAs have exchanged "lost" flags,
// and the whole cluster leaves together.
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

// Tile geometry of the group kernels for a local engine C (2^L rows, W
// columns; 512 threads x 32 values in three stage groups, or 256 x 64 in
// two) and a cluster of 2^CL CTAs.
template <class C, int CL>
struct GroupCol {
    using S = TmaSplit<C>;
    using Gl = Grp<C, C::NG - 1>;
    static constexpr int CS = 1 << CL;
    static constexpr int L = C::L;                        // local stages
    static constexpr int NL = C::N;                       // rows held by one CTA
    static constexpr int XVALS = C::EPT / 2;              // values exchanged per thread per round
    static constexpr uint32_t XBYTES = (uint32_t)XVALS * C::T * 8u;   // per CTA per round
    static constexpr int KEEP_R = Gl::R >> CL;            // register indices r kept at the end
    static constexpr int OUT_ROWS = NL / CS;              // rows k of one CTA's output range
    static constexpr int OUT_BOX_Z = OUT_ROWS / S::BOX;   // 256-row blocks of one range
    static constexpr int STAGE_T = (C::E / 2) / (OUT_ROWS * C::W);   // ranges per staging fill
    // values a thread keeps per output t at the end (all its units)
    static constexpr int KEEP_V = Gl::V * KEEP_R;
    // scratch of the L2 exchange per cluster (col_group_l2_kernel): two
    // tiles' slots, CS XVALS T values (pair) or CS^2 KEEP_V T (four CTAs)
    static constexpr long long L2_SCRATCH_VALS =
        CL == 2 ? 2LL * CS * CS * KEEP_V * C::T : 2LL * CS * XVALS * C::T;
    // the mirror exchange of the paired forward DCT per cluster, after the
    // slots above: per CTA a receive region of CS/2 output blocks, KEEP_V
    // values per thread each
    static constexpr long long MIRROR_VALS = (long long)CS * (CS / 2) * KEEP_V * C::T;
    static_assert(C::LB == 1 && ((C::EPT == 32 && C::NG == 3) || (C::EPT == 64 && C::NG == 2)),
                  "512 threads x 32 values in 3 groups, or 256 x 64 in 2");
    static_assert(CL >= 1 && CL <= 2, "two or four CTAs");
    static_assert(Gl::S0 + Gl::G == L && (NL >> Gl::S0) == Gl::R,
                  "the last group's register index is the top bits of k");
    static_assert(Gl::V * (Gl::R / 2) == XVALS, "half of a thread's values per round");
    static_assert(XBYTES <= (uint32_t)C::E * 4u, "the receive buffer fits in half the tile region");
    static_assert(OUT_ROWS % S::BOX == 0, "output ranges are whole 256-row blocks");
    static_assert(STAGE_T >= 1 && CS % STAGE_T == 0, "whole output ranges per staging fill");
};

// One exchange round J of the last CL stages.  On entry s[] holds, for the
// 2^J outputs t and the register indices r in [rb, rb + NK) of both units v,
// s[t * 2 NK + v NK + (r - rb)] (NK = 16 >> J); on return it holds the same
// for 2^(J+1) outputs and the half [rk, rk + NK/2) kept by this CTA.
// Twiddles wk[] were loaded for the kept half, in the order of the loop.
template <class C, int J>
__device__ __forceinline__ void group_round_compute(float2 (&s)[32], const float2 *recv,
                                                    const float2 (&wk)[16], int bitj)
{
    using Gl = Grp<C, C::NG - 1>;
    constexpr int NT = 1 << J;
    constexpr int NK = Gl::R >> J;
    constexpr int NH = NK / 2;
    const int tid = threadIdx.x;
    float2 n[32];
#pragma unroll
    for (int t = 0; t < NT; t++) {
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
#pragma unroll
            for (int ih = 0; ih < NH; ih++) {
                const int j = (t * Gl::V + v) * NH + ih;     // send / receive slot, twiddle
                const float2 lo_half = s[t * 2 * NK + v * NK + ih];
                const float2 hi_half = s[t * 2 * NK + v * NK + NH + ih];
                const float2 mine = bitj == 0 ? lo_half : hi_half;
                const float2 theirs = recv[j * C::T + tid];
                float2 x0 = bitj == 0 ? mine : theirs;
                float2 x1 = bitj == 0 ? theirs : mine;
                butterfly_w(x0, x1, wk[j]);
                n[t * 2 * NH + v * NH + ih] = x0;                 // output t (bit L+J clear)
                n[(t + NT) * 2 * NH + v * NH + ih] = x1;          // output t + 2^J
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 32; i++)
        s[i] = n[i];
}

// The half of round J's values this CTA gives away, into the send buffer.
template <class C, int J>
__device__ __forceinline__ void group_round_send(const float2 (&s)[32], float2 *sendb, int bitj)
{
    using Gl = Grp<C, C::NG - 1>;
    constexpr int NT = 1 << J;
    constexpr int NK = Gl::R >> J;
    constexpr int NH = NK / 2;
    const int tid = threadIdx.x;
#pragma unroll
    for (int t = 0; t < NT; t++) {
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
#pragma unroll
            for (int ih = 0; ih < NH; ih++) {
                const int j = (t * Gl::V + v) * NH + ih;
                const float2 lo_half = s[t * 2 * NK + v * NK + ih];
                const float2 hi_half = s[t * 2 * NK + v * NK + NH + ih];
                sendb[j * C::T + tid] = bitj == 0 ? hi_half : lo_half;
            }
        }
    }
}

// Rotation factors of round J for the kept half: W_{2^(L+J+1)}^i with
// i = k + 2^L t, read from the plan's table (stage L+J+1 starts at entry
// 2^(L+J) - 1), k = lo_v + 2^S0 r for the kept r.
template <class C, int J, int NW>
__device__ __forceinline__ void group_round_twiddles(float2 (&wk)[NW],
                                                     const float2 *__restrict__ tw, int rk)
{
    using Gl = Grp<C, C::NG - 1>;
    constexpr int NT = 1 << J;
    constexpr int NH = (Gl::R >> J) / 2;
    const float2 *tws = tw + ((1 << (C::L + J)) - 1);
    const int tid = threadIdx.x;
#pragma unroll
    for (int t = 0; t < NT; t++) {
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
            const int u = tid + v * C::T;
            const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
#pragma unroll
            for (int ih = 0; ih < NH; ih++) {
                const int k = lo | ((rk + ih) << Gl::S0);
                wk[(t * Gl::V + v) * NH + ih] = __ldg(tws + k + (t << C::L));
            }
        }
    }
}

// Slot pair m (slots 2m and 2m + 1) of this thread in an exchange region of
// global memory: rt is the region's start plus threadIdx.x, and the pair is
// the 16 bytes at float2 offset 2 (m T + tid), contiguous over the threads.
template <class C>
__device__ __forceinline__ float4 *slot_pair(float2 *rt, int m)
{
    return reinterpret_cast<float4 *>(rt + 2 * m * C::T + threadIdx.x);
}
template <class C>
__device__ __forceinline__ const float4 *slot_pair(const float2 *rt, int m)
{
    return reinterpret_cast<const float4 *>(rt + 2 * m * C::T + threadIdx.x);
}

// The same two steps of round J with the exchanged values in global memory
// (region rt = its start plus threadIdx.x), written and read through L2
// only: slot j of this thread at rt + j T (8-byte accesses), or with VEC
// two slots per 16-byte access (slot_pair).  Measured: VEC speeds up the
// half2 kernels (16384^2 FP16 transform 2.51 -> 2.31 ms) and slows the
// complex64 ones down (8192^2 column pass 0.317 -> 0.326 ms, more spills).
template <class C, int J, bool VEC, int NA>
__device__ __forceinline__ void group_round_send_g(const float2 (&s)[NA], float2 *rt, int bitj)
{
    using Gl = Grp<C, C::NG - 1>;
    constexpr int NT = 1 << J;
    constexpr int NK = Gl::R >> J;
    constexpr int NH = NK / 2;
    static_assert(NA == C::EPT, "a thread's values");
#pragma unroll
    for (int t = 0; t < NT; t++) {
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
            if constexpr (VEC) {
#pragma unroll
                for (int ih = 0; ih < NH; ih += 2) {
                    const int j = (t * Gl::V + v) * NH + ih;
                    const int b = (t * Gl::V + v) * NK + ih;
                    const float2 x0 = bitj == 0 ? s[b + NH] : s[b];
                    const float2 x1 = bitj == 0 ? s[b + NH + 1] : s[b + 1];
                    __stcg(slot_pair<C>(rt, j / 2), make_float4(x0.x, x0.y, x1.x, x1.y));
                }
            } else {
#pragma unroll
                for (int ih = 0; ih < NH; ih++) {
                    const int j = (t * Gl::V + v) * NH + ih;
                    const float2 lo_half = s[(t * Gl::V + v) * NK + ih];
                    const float2 hi_half = s[(t * Gl::V + v) * NK + NH + ih];
                    __stcg(rt + j * C::T, bitj == 0 ? hi_half : lo_half);
                }
            }
        }
    }
}

template <class C, int J, bool VEC, int NA, int NW>
__device__ __forceinline__ void group_round_compute_g(float2 (&s)[NA], const float2 *rt,
                                                      const float2 (&wk)[NW], int bitj)
{
    using Gl = Grp<C, C::NG - 1>;
    constexpr int NT = 1 << J;
    constexpr int NK = Gl::R >> J;
    constexpr int NH = NK / 2;
    static_assert(NA == C::EPT && NW >= NT * Gl::V * NH, "a thread's values and factors");
    static_assert(NH % 2 == 0, "whole slot pairs");
    float2 n[NA];
#pragma unroll
    for (int t = 0; t < NT; t++) {
#pragma unroll
        for (int v = 0; v < Gl::V; v++) {
#pragma unroll
            for (int ih = 0; ih < NH; ih++) {
                const int j = (t * Gl::V + v) * NH + ih;
                const float2 lo_half = s[(t * Gl::V + v) * NK + ih];
                const float2 hi_half = s[(t * Gl::V + v) * NK + NH + ih];
                const float2 mine = bitj == 0 ? lo_half : hi_half;
                float2 theirs;
                if constexpr (VEC) {
                    const float4 tp = __ldcg(slot_pair<C>(rt, j / 2));
                    theirs = (j & 1) ? make_float2(tp.z, tp.w) : make_float2(tp.x, tp.y);
                } else {
                    theirs = __ldcg(rt + j * C::T);
                }
                float2 x0 = bitj == 0 ? mine : theirs;
                float2 x1 = bitj == 0 ? theirs : mine;
                butterfly_w(x0, x1, wk[j]);
                n[(t * Gl::V + v) * NH + ih] = x0;                 // output t
                n[((t + NT) * Gl::V + v) * NH + ih] = x1;          // output t + 2^J
            }
        }
    }
#pragma unroll
    for (int i = 0; i < NA; i++)
        s[i] = n[i];
}

// Shared-memory layout of the half2 group kernel (byte offsets): the FP32
// tile / exchange region, the early half of the next half2 tile, the
// rotation factors, the factors 2^e of this CTA's rows.
template <class C>
struct GroupH16 {
    static constexpr int BOX = 256;
    static constexpr int NBOX = C::N / BOX;
    static constexpr int NB = NBOX / 2;
    static constexpr int BOXV = BOX * C::W;                  // half2 values per block
    static constexpr uint32_t HALF_BYTES = (uint32_t)NB * BOXV * 4u;
    static constexpr int PREF_OFF = C::E * 8;
    static constexpr int TW_OFF = PREF_OFF + (int)HALF_BYTES;
    static constexpr int RF_OFF = TW_OFF + C::N * 8;
    static constexpr int SMEM_BYTES = RF_OFF + C::N * 4;
    static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
};

// Storage of the group kernel's input and output: complex64, or half2 with
// the input's exponents per row (row_exp) and the output's per column.
struct GroupIO {
    const int *row_exp;
    int *out_exp;
    float2 *mid_row = nullptr;   // paired forward DCT: output row N/2
};

// The "two for one" split of Z = DFT(v_a + i v_b) into the DCT-II outputs of
// the real lines a and b (Makhoul's reduction): from Z[k], Z[k'] (k' = N - k)
// and (c, s) = (cos, sin)(pi k / (2N)),
//   xk = (X_a[k], X_b[k]),  xp = (X_a[k'], X_b[k']),  both times scale.
__device__ __forceinline__ void dct_pair(float2 zk, float2 zp, float2 cs, float scale,
                                         float2 &xk, float2 &xp)
{
    const float c = cs.x * 0.5f * scale, s = cs.y * 0.5f * scale;
    const float sr = zk.x + zp.x, dr = zp.x - zk.x;   // Zr[k] + Zr[k'], Zr[k'] - Zr[k]
    const float si = zk.y + zp.y, di = zk.y - zp.y;   // Zi[k] + Zi[k'], Zi[k] - Zi[k']
    xk = make_float2(c * sr + s * di, c * si + s * dr);     // (X_a[k], X_b[k])
    xp = make_float2(s * sr - c * di, s * si - c * dr);     // (X_a[k'], X_b[k'])
}

// C: the local engine; cluster of 2^CL CTAs, this CTA's rank q.  lmap: this
// CTA's load map (rows CS m + rev_CL(q) of the image; box W x 256 x NB);
// omap: store map over the output (box W x 256 x OUT_BOX_Z); tw: the plan's
// rotation-factor table of the column axis (2^(L+CL) entries with padding:
// the local stages read entries [0, 2^L), round j stage L+1+j).
template <class C, int CL>
__device__ __forceinline__ void col_group_body(const CUtensorMap *lmap, const CUtensorMap *omap,
                                               int ntiles, const float2 *__restrict__ tw,
                                               float scale, int *err, int withhold)
{
    namespace cg = cooperative_groups;
    using S = TmaSplit<C>;
    using GC = GroupCol<C, CL>;
    using Gl = Grp<C, C::NG - 1>;
    constexpr int CS = GC::CS;
    extern __shared__ __align__(1024) float2 sm[];
    __shared__ __align__(8) uint64_t bar_early, bar_late, bar_recv;
    __shared__ int lost_flag[CS];   // slot p: written by CTA p of the cluster
    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank();
    const int tid = threadIdx.x;
    const int nclusters = (int)gridDim.x / CS;
    float2 *stw = sm + S::TW_OFF;
    // the first and second half of a tile's TMA boxes
    auto issue_early = [&](int t) { split_issue_early<C>(sm, lmap, t * C::W, &bar_early); };
    auto issue_late = [&](int t) { split_issue_late<C>(sm, lmap, t * C::W, &bar_late); };
    // after the last read of a tile: the lower half of the tile region
    // receives the partner's values, the upper half holds the values sent
    // and then stages the output
    float2 *recvb = sm;
    float2 *sendb = sm + C::E / 2;
    uint32_t peer_recv[CL], peer_bar[CL];
#pragma unroll
    for (int j = 0; j < CL; j++) {
        peer_recv[j] = mapa_shared(smem_addr(recvb), (uint32_t)(q ^ (1 << j)));
        peer_bar[j] = mapa_shared(smem_addr(&bar_recv), (uint32_t)(q ^ (1 << j)));
    }
    // the k this CTA keeps at the end: register indices [rk_end, rk_end + KEEP_R)
    int rk_end = 0;
#pragma unroll
    for (int j = 0; j < CL; j++)
        rk_end += ((q >> j) & 1) * ((Gl::R >> j) / 2);
    const int k_base = rk_end << Gl::S0;   // first row k of this CTA's output ranges
    int lost_recv = 0;
    int tile = (int)blockIdx.x / CS;

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
            bulk_load(stw, tw, S::TW_BYTES, &bar_early);
            issue_early(tile);
            // (self-test: CTA 0 withholds its first late boxes)
            if (!(withhold && blockIdx.x == 0))
                issue_late(tile);
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
        // the "lost" flags for the first cluster barrier and the arming of
        // the receive mbarrier, early so the remote flag stores are long done
        // when that barrier is arrived at (the peers read the flags after it
        // and the next ones are written only after the tile's second barrier)
        if (tid == 0) {
            if (!lost_recv)   // (a phase that timed out may still be open)
                mbar_arrive_expect_tx(&bar_recv, GC::XBYTES);
#pragma unroll
            for (int p = 0; p < CS; p++)
                *cluster.map_shared_rank(lost_flag + q, p) = lost_here;
        }
        if (!lost_here) {
            w_early++;
            w_late++;
            group_first_split<C>(
                a, sm, stw,
                [&] {
                    if (tid == 0)
                        bulk_wait_read_all();   // the previous tile's stores have read it
                },
                [&] {
                    if (tid == 0 && next < ntiles)
                        issue_early(next);
                });
            if (next < ntiles)
                n_early++;
            __syncthreads();
            group_smem<C, 1, false, false, true>(a, sm, stw, C::L);
            __syncthreads();
            group_last_read<C>(a, sm);
            __syncthreads();   // the tile region is free
        }
        // cluster barrier A0, arrive: this CTA's tile region is free and its
        // receive mbarrier armed; the "lost" flags travel with it
        cluster_arrive_release();
        float2 wk[16];
        if (!lost_here) {
#pragma unroll
            for (int v = 0; v < Gl::V; v++) {
                const int u = tid + v * C::T;
                const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
                run_stages<C, C::NG - 1, false, true>(a, v, lo, stw, C::L);
            }
            group_round_send<C, 0>(a, sendb, q & 1);
            fence_proxy_async_smem();
        }
        __syncthreads();   // the send buffer is complete
        group_round_twiddles<C, 0>(wk, tw, (q & 1) * (Gl::R / 2));
        cluster_wait_acquire();
        {
            int any = 0;
#pragma unroll
            for (int p = 0; p < CS; p++)
                any |= lost_flag[p];
            if (any) {
                lost = true;
                break;
            }
        }
        // round 0: the partner's receive region is free; one bulk copy of
        // the send buffer into it, completing on the partner's mbarrier
        if (tid == 0)
            bulk_copy_to_peer(peer_recv[0], sendb, GC::XBYTES, peer_bar[0]);
        lost_recv = mbar_wait_bounded(&bar_recv, (uint32_t)(w_recv & 1)) ? 0 : 1;
        if (!lost_recv)
            w_recv++;
        // cluster barrier B0, arrive: the partner's send buffer has been read
        // (half2, last round: after the column maxima, further down)
        cluster_arrive_release();
        group_round_compute<C, 0>(a, recvb, wk, q & 1);
        if constexpr (CL == 2) {
            const int rk1 = ((q & 1) * (Gl::R / 2)) + ((q >> 1) & 1) * (Gl::R / 4);
            group_round_twiddles<C, 1>(wk, tw, rk1);
            fence_proxy_async_smem();
            __syncthreads();   // the receive buffer has been read
            if (tid == 0 && !lost_recv)
                mbar_arrive_expect_tx(&bar_recv, GC::XBYTES);
            cluster_wait_acquire();   // B0: this CTA's send buffer is free
            group_round_send<C, 1>(a, sendb, (q >> 1) & 1);
            fence_proxy_async_smem();
            __syncthreads();   // the send buffer is complete
            // cluster barrier A1: every receive region is free and armed
            cluster_arrive_release();
            cluster_wait_acquire();
            if (tid == 0)
                bulk_copy_to_peer(peer_recv[1], sendb, GC::XBYTES, peer_bar[1]);
            const int lr = mbar_wait_bounded(&bar_recv, (uint32_t)(w_recv & 1)) ? 0 : 1;
            if (!lr)
                w_recv++;
            lost_recv |= lr;
            // cluster barrier B1, arrive: the partner's send buffer has been read
            cluster_arrive_release();
            group_round_compute<C, 1>(a, recvb, wk, (q >> 1) & 1);
        }
        fence_proxy_async_smem();
        __syncthreads();   // the receive buffer has been read
        if (tid == 0 && next < ntiles)
            issue_late(next);
        if (next < ntiles)
            n_late++;
        // the last B barrier, wait: this CTA's send buffer is free for staging
        cluster_wait_acquire();

        // outputs t = 0 .. CS-1: rows k_base + [0, OUT_ROWS) + 2^L t, STAGE_T
        // ranges per fill of the staging buffer (the send buffer), each
        // range one TMA store
#pragma unroll
        for (int f = 0; f < CS / GC::STAGE_T; f++) {
            if (f > 0) {
                if (tid == 0)
                    bulk_wait_read_all();
                __syncthreads();
            }
#pragma unroll
            for (int ts = 0; ts < GC::STAGE_T; ts++) {
                const int t = f * GC::STAGE_T + ts;
#pragma unroll
                for (int v = 0; v < Gl::V; v++) {
                    const int u = tid + v * C::T;
                    const int w = u & (C::W - 1);
                    const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
#pragma unroll
                    for (int i = 0; i < GC::KEEP_R; i++) {
                        const float2 x = a[t * 2 * GC::KEEP_R + v * GC::KEEP_R + i];
                        sendb[(ts * GC::OUT_ROWS + ((i << Gl::S0) | lo)) * C::W + w] =
                            make_float2(x.x * scale, x.y * scale);
                    }
                }
            }
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
#pragma unroll
                for (int ts = 0; ts < GC::STAGE_T; ts++) {
                    const int t = f * GC::STAGE_T + ts;
                    const int z = ((t << C::L) + k_base) / S::BOX;
                    tma_store_3d(omap, tile * C::W, 0, z, sendb + ts * GC::OUT_ROWS * C::W);
                }
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

// rank q loads map[rev_CL(q)] -- the rows of residue rev_CL(q) mod 2^CL
template <class C, int CL>
__global__ void __launch_bounds__(C::T, 1) col_group_kernel(const __grid_constant__ CUtensorMap map0,
                                                            const __grid_constant__ CUtensorMap map1,
                                                            const __grid_constant__ CUtensorMap map2,
                                                            const __grid_constant__ CUtensorMap map3,
                                                            const __grid_constant__ CUtensorMap omap,
                                                            const float2 *__restrict__ tw,
                                                            int cols, float scale, int *err,
                                                            int withhold)
{
    const int q = (int)cooperative_groups::this_cluster().block_rank();
    const int res = brev_rt(q, CL);
    const CUtensorMap *m = res == 0 ? &map0 : res == 1 ? &map1 : res == 2 ? &map2 : &map3;
    col_group_body<C, CL>(m, &omap, cols / C::W, tw, scale, err, withhold);
}

// The same column pass with the exchange rounds through a scratch buffer in
// global memory (resident in L2) instead of bulk copies between shared
// memories.  Every CTA writes the values it gives away into its slots of the
// buffer (contiguous per thread index), the cluster barrier (release /
// acquire at cluster scope) makes the writes visible, and the partners read
// them straight into registers.  Nothing of the exchange lives in shared
// memory, so the tile region is free as soon as the last group has read it:
// the next tile's second half is requested then, and one cluster barrier per
// exchange suffices (against two with bulk copies, which must wait until the
// receiving region is free and again until the copy has left).  The output
// leaves through TMA stores from the staging half of the tile region.
//
// Four CTAs (c = 2) run both cross stages after a single exchange: CTA q
// sends each partner p the values at p's final rows k (KEEP_V per thread) and
// receives the three partners' values at its own, then runs stage L+1 on
// the pairs of blocks (0, 1), (2, 3) and stage L+2 on (0, 2), (1, 3) in
// registers -- the same butterflies on the same operands as two rounds of
// pairwise swaps, with one barrier and 96 KB each way per CTA instead of two
// and 128 KB.
//
// Slots alternate per tile: a slot is written again only after the next
// tile's barrier, which every reader arrives at after its reads of the slot.
// The "lost" flags alternate per tile for the same reason.  xbuf: per
// cluster of the launch, 2 CS XVALS T values (pair) or 2 CS^2 KEEP_V T
// (four CTAs), cluster-major; it belongs to this launch alone.
//
// DCT == 1: the forward DCT-II of real columns (Section 5's similar transforms;
// the reduction of a length-N DCT-II to a length-N complex DFT of the
// reordered line v[j] = x[2j], v[N-1-j] = x[2j+1], X[k] = Re(e^{-i pi k /
// (2N)} V[k]), Makhoul 1980), one complex line per real column, imaginary
// part zero: no pairing of outputs (k, N-k) is needed.  A tile is W real
// columns; CTA q's local line u[m] = v[CS m + rev(q)] is, for m < NL/2, the
// rows 2 CS m + 2 rev(q) (lmap) and for m >= NL/2 the rows
// 2 CS (NL-1-m) + 2 CS - 1 - 2 rev(q) read backwards (lmap2: ascending rows
// 2 CS m' + 2 CS - 1 - 2 rev(q)); both maps have 2-float (8-byte) elements,
// W/2 per box row.  The outputs X[k] (post = (cos, sin)(pi k / (2N)),
// k <= N/2) leave as floats through the real output map omap.
//
// DCT == 2: the inverse, DCT-III, of real columns, one real line per complex
// line: V[k] = e^{i pi k / (2N)} (X[k] - i X[N-k]) (X[N] = 0), v = IDFT(V)
// (the plan's conjugate rotation factors), x[2n] = v[n], x[2n+1] =
// v[N-1-n].  CTA q's local line holds k = CS m + rev(q), the rows of that
// residue (lmap, ascending); X[N-k] lies in the rows of residue
// (CS - rev(q)) mod CS read backwards (lmap2): index NL-1-m, or (NL-m) mod
// NL for residue 0, where m = 0 takes X[N] = 0.  Outputs n < N/2 go to the
// even rows (omap: rows 2n'), the others in reverse order to the odd rows
// (omap2: rows 2n'+1).
//
// DCT == 3: the forward DCT-II with two real columns per complex line (the
// "two for one" split, dct_pair): a tile is W complex = 2W real columns
// (32-byte rows), the local line is gathered as in DCT == 1 from complex
// maps (lmap ascending, lmap2 backwards), so half the butterflies of DCT ==
// 1 per real column.  Output K needs Z[K] and Z[N-K].  CTA q holds K = NL t
// + k_base + row (row < OUT_ROWS); N - K is row OUT_ROWS - row of block
// CS-1-t in CTA CS-1-q (k_base(q) + k_base(CS-1-q) = NL - OUT_ROWS), except
// for row 0, whose mirror is row 0 of the CTA with k_base = NL - k_base(q)
// (CTA 0 and the CTA at NL/2: itself; CTAs 2 and 3 of four: each other).  So
// every CTA forms the pairs of its blocks t < CS/2 and sends its blocks t >=
// CS/2 through a second exchange in L2 to the thread that holds the mirror
// (unit 2^S0 - lo, index KEEP_R-1-i; KEEP_R-i for lo = 0).  X[K] leaves by
// TMA from the staged ranges, X[N-K] from the ranges staged in reverse
// through omap2 (W x 256 boxes at any row; the one row past the image, the
// mirror of K = 0, is outside the map and not written); X[N/2], which pairs
// with itself, is stored by CTA 0's threads of row 0 (io.mid_row).
template <class C, int CL, bool H16, int DCT = 0>
__device__ __forceinline__ void col_group_l2_body(const CUtensorMap *lmap, const CUtensorMap *omap,
                                                  int ntiles, const float2 *__restrict__ tw,
                                                  float scale, int *err, int withhold,
                                                  float2 *xbuf, const GroupIO &io,
                                                  const CUtensorMap *lmap2 = nullptr,
                                                  const float2 *__restrict__ post = nullptr,
                                                  const CUtensorMap *omap2 = nullptr)
{
    namespace cg = cooperative_groups;
    using S = TmaSplit<C>;
    using GC = GroupCol<C, CL>;
    using GH = GroupH16<C>;
    using Gl = Grp<C, C::NG - 1>;
    using G0 = Grp<C, 0>;
    constexpr int CS = GC::CS;
    constexpr int XV = GC::XVALS * C::T;   // values given away per CTA per round
    extern __shared__ __align__(1024) float2 sm[];
    __shared__ __align__(8) uint64_t bar_early, bar_late;
    __shared__ int lost_flag[2][CS];       // [tile parity][slot p: written by CTA p]
    __shared__ int cmax[2][CS][C::W];      // half2: [tile parity][CTA p's partial column maxima]
    __shared__ int cmax_local[C::W];
    // DCT == 3: (cos, sin)(pi B / (2N)) of the block starts B = NL t + k_base
    // + 2^S0 i of this CTA's paired outputs (t < CS/2); a thread multiplies
    // them by its own (cos, sin)(pi lo / (2N)) (within a few ulp of the table)
    __shared__ float2 rot_base[DCT == 3 ? (1 << CL) / 2 * (Grp<C, C::NG - 1>::R >> CL) : 1];
    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank();
    const int tid = threadIdx.x;
    const int nclusters = (int)gridDim.x / CS;
    const int cid = (int)blockIdx.x / CS;
    unsigned char *smb = reinterpret_cast<unsigned char *>(sm);
    float2 *stw = H16 ? reinterpret_cast<float2 *>(smb + GH::TW_OFF) : sm + S::TW_OFF;
    float *rf = reinterpret_cast<float *>(smb + GH::RF_OFF);
    const uint32_t tw_bytes = H16 ? (uint32_t)C::N * 8u : S::TW_BYTES;
    float2 *stage = sm + C::E / 2;
    static_assert(!(H16 && DCT), "one storage mode");
    constexpr uint32_t DCT_HALF_BYTES = (uint32_t)(C::N / 2) * C::W * 4u;   // floats
    constexpr int DCT_HALF_FLOATS = (C::N / 2) * C::W;
    // the first and second half of a tile's TMA boxes
    auto issue_early = [&](int t) {
        if constexpr (DCT == 1) {
            mbar_arrive_expect_tx(&bar_early, DCT_HALF_BYTES);
            tma_load_3d(sm + C::E, lmap, t * (C::W / 2), 0, 0, &bar_early);
        } else if constexpr (DCT == 3) {
            mbar_arrive_expect_tx(&bar_early, S::EARLY_BYTES);
            tma_load_3d(sm + C::E, lmap, t * C::W, 0, 0, &bar_early);
        } else if constexpr (DCT == 2) {
            // first halves of the natural and the mirrored rows
            float *pf = reinterpret_cast<float *>(sm + C::E);
            mbar_arrive_expect_tx(&bar_early, 2 * DCT_HALF_BYTES);
            tma_load_3d(pf, lmap, t * (C::W / 2), 0, 0, &bar_early);
            tma_load_3d(pf + DCT_HALF_FLOATS, lmap2, t * (C::W / 2), 0, 0, &bar_early);
        } else if constexpr (H16) {
            mbar_arrive_expect_tx(&bar_early, GH::HALF_BYTES);
            tma_load_3d(smb + GH::PREF_OFF, lmap, t * C::W, 0, 0, &bar_early);
        } else {
            split_issue_early<C>(sm, lmap, t * C::W, &bar_early);
        }
    };
    auto issue_late = [&](int t) {
        if constexpr (DCT == 1) {
            mbar_arrive_expect_tx(&bar_late, DCT_HALF_BYTES);
            tma_load_3d(sm, lmap2, t * (C::W / 2), 0, 0, &bar_late);
        } else if constexpr (DCT == 3) {
            mbar_arrive_expect_tx(&bar_late, S::LATE_BYTES);
            tma_load_3d(sm, lmap2, t * C::W, 0, 0, &bar_late);
        } else if constexpr (DCT == 2) {
            // second halves, at the start of the tile region
            float *lf = reinterpret_cast<float *>(sm);
            mbar_arrive_expect_tx(&bar_late, 2 * DCT_HALF_BYTES);
            tma_load_3d(lf, lmap, t * (C::W / 2), 0, S::NB, &bar_late);
            tma_load_3d(lf + DCT_HALF_FLOATS, lmap2, t * (C::W / 2), 0, S::NB, &bar_late);
        } else if constexpr (H16) {
            mbar_arrive_expect_tx(&bar_late, GH::HALF_BYTES);
            tma_load_3d(smb, lmap, t * C::W, 0, GH::NB, &bar_late);
        } else {
            split_issue_late<C>(sm, lmap, t * C::W, &bar_late);
        }
    };
    // four CTAs exchange once per tile (both cross stages, radix 4); slots
    // [tile parity][source][destination][KEEP_V values][T]
    constexpr bool R4 = CL == 2;
    constexpr bool VEC = H16;   // 16-byte exchange slots (see group_round_send_g)
    constexpr int R4V = GC::KEEP_V;                       // values per source and destination
    constexpr long long XSTRIDE = GC::L2_SCRATCH_VALS + (DCT == 3 ? GC::MIRROR_VALS : 0);
    float2 *xb = xbuf + (long long)cid * XSTRIDE + tid;
    int rk_end = 0;
#pragma unroll
    for (int j = 0; j < CL; j++)
        rk_end += ((q >> j) & 1) * ((Gl::R >> j) / 2);
    const int k_base = rk_end << Gl::S0;   // first row k of this CTA's output ranges
    int tile = cid;

    if (tid == 0) {
        mbar_init(&bar_early, 1);
        mbar_init(&bar_late, 1);
        fence_mbar_init();
    }
    float2 rot_lo = make_float2(1.f, 0.f);
    if constexpr (DCT == 3) {
        constexpr int KR = GC::KEEP_R;
        for (int j = tid; j < CS / 2 * KR; j += C::T)
            rot_base[j] = __ldg(post + ((j / KR) << C::L) + k_base + ((j % KR) << Gl::S0));
        rot_lo = __ldg(post + ((tid >> C::KW) & ((1 << Gl::S0) - 1)));
    }
    if constexpr (H16) {
        // the factors of this CTA's rows CS m + rev_CL(q)
        const int res = brev_rt(q, CL);
        for (int i = tid; i < C::N; i += C::T)
            rf[i] = pow2f(io.row_exp[(long long)i * CS + res]);
        if (tid < C::W)
            cmax_local[tid] = 0;
    }
    __syncthreads();
    int n_early = 0, n_late = 0, w_early = 0, w_late = 0;
    if (tile < ntiles) {
        if (tid == 0) {
            mbar_expect_tx(&bar_early, tw_bytes);
            bulk_load(stw, tw, tw_bytes, &bar_early);
            issue_early(tile);
            // (self-test: CTA 0 withholds its first late boxes)
            if (!(withhold && blockIdx.x == 0))
                issue_late(tile);
        }
        n_early = n_late = 1;
    }
    bool lost = false;
    float2 a[C::EPT];
    for (int it = 0; tile < ntiles; tile += nclusters, it++) {
        const int next = tile + nclusters;
        const int par = it & 1;
        const bool ok = mbar_wait_bounded(&bar_early, (uint32_t)(w_early & 1)) &&
                        mbar_wait_bounded(&bar_late, (uint32_t)(w_late & 1));
        const int lost_here = __syncthreads_or(ok ? 0 : 1);
        if (tid == 0) {
#pragma unroll
            for (int p = 0; p < CS; p++)
                *cluster.map_shared_rank(&lost_flag[par][q], p) = lost_here;
        }
        // round 0 slots: alternate per tile for a pair, slot 0 for four CTAs
        float2 *x0 = xb + (CL == 1 ? par : 0) * (CS * XV);
        if (!lost_here) {
            w_early++;
            w_late++;
            if constexpr (DCT == 2) {
                // group 0: scrambled gather of the spectrum rows k = CS i +
                // res and their mirrors N - k, pre-rotated into V[k]
                const int res = brev_rt(q, CL);
                constexpr int NN = C::N << CL;
                const float *pn = reinterpret_cast<const float *>(sm + C::E);
                const float *pm = pn + DCT_HALF_FLOATS;
                const float *ln = reinterpret_cast<const float *>(sm);
                const float *lm = ln + DCT_HALF_FLOATS;
#pragma unroll
                for (int v = 0; v < G0::V; v++) {
                    const int u = tid + v * C::T;
                    const int w = u & (C::W - 1);
                    const int hib = (u >> C::KW) & ((1 << G0::HB) - 1);
#pragma unroll
                    for (int r = 0; r < G0::R; r++) {
                        const int top = brev_c(r, G0::G) << G0::HB;   // compile-time
                        const int i = top | hib;
                        const float xn = top < C::N / 2 ? pn[i * C::W + w]
                                                        : ln[(i - C::N / 2) * C::W + w];
                        const int j = res == 0 ? ((C::N - i) & (C::N - 1)) : C::N - 1 - i;
                        float xm = j < C::N / 2 ? pm[j * C::W + w] : lm[(j - C::N / 2) * C::W + w];
                        if (res == 0 && i == 0)
                            xm = 0.f;   // X[N] = 0
                        const int k = CS * i + res;
                        const float2 cs = k <= NN / 2 ? __ldg(post + k) : __ldg(post + (NN - k));
                        const float c = k <= NN / 2 ? cs.x : cs.y;
                        const float sn = k <= NN / 2 ? cs.y : cs.x;
                        a[v * G0::R + r] = make_float2(c * xn + sn * xm, sn * xn - c * xm);
                    }
                }
#pragma unroll
                for (int v = 0; v < G0::V; v++)
                    run_stages<C, 0, false, true>(a, v, 0, stw, C::L);
                fence_proxy_async_smem();
                if (tid == 0)
                    bulk_wait_read_all();   // the previous tile's stores have read it
                __syncthreads();            // every slot of both input regions has been read
                if (tid == 0 && next < ntiles)
                    issue_early(next);
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
            } else if constexpr (DCT == 3) {
                // group 0: scrambled gather of the reordered pairs of real
                // columns (the second half of the local line read backwards)
                const float2 *pref = sm + C::E;
                const float2 *late = sm;
#pragma unroll
                for (int v = 0; v < G0::V; v++) {
                    const int u = tid + v * C::T;
                    const int w = u & (C::W - 1);
                    const int hib = (u >> C::KW) & ((1 << G0::HB) - 1);
#pragma unroll
                    for (int r = 0; r < G0::R; r++) {
                        const int top = brev_c(r, G0::G) << G0::HB;   // compile-time
                        a[v * G0::R + r] = top < C::N / 2 ? pref[(top | hib) * C::W + w]
                                                          : late[(C::N - 1 - (top | hib)) * C::W + w];
                    }
                }
#pragma unroll
                for (int v = 0; v < G0::V; v++)
                    run_stages<C, 0, false, true>(a, v, 0, stw, C::L);
                fence_proxy_async_smem();
                if (tid == 0)
                    bulk_wait_read_all();   // the previous tile's stores have read it
                __syncthreads();            // every slot of both input regions has been read
                if (tid == 0 && next < ntiles)
                    issue_early(next);
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
            } else if constexpr (DCT == 1) {
                // group 0: scrambled gather of the reordered real columns
                // (the second half of the local line read backwards), as
                // complex values with imaginary part zero
                const float *pref = reinterpret_cast<const float *>(sm + C::E);
                const float *late = reinterpret_cast<const float *>(sm);
#pragma unroll
                for (int v = 0; v < G0::V; v++) {
                    const int u = tid + v * C::T;
                    const int w = u & (C::W - 1);
                    const int hib = (u >> C::KW) & ((1 << G0::HB) - 1);
#pragma unroll
                    for (int r = 0; r < G0::R; r++) {
                        const int top = brev_c(r, G0::G) << G0::HB;   // compile-time
                        const float x = top < C::N / 2 ? pref[(top | hib) * C::W + w]
                                                       : late[(C::N - 1 - (top | hib)) * C::W + w];
                        a[v * G0::R + r] = make_float2(x, 0.f);
                    }
                }
#pragma unroll
                for (int v = 0; v < G0::V; v++)
                    run_stages<C, 0, false, true>(a, v, 0, stw, C::L);
                fence_proxy_async_smem();
                if (tid == 0)
                    bulk_wait_read_all();   // the previous tile's stores have read it
                __syncthreads();            // every slot of both input regions has been read
                if (tid == 0 && next < ntiles)
                    issue_early(next);
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
            } else if constexpr (H16) {
                // group 0: scrambled gather of the half2 tile, widened and
                // scaled by the row factors
                const __half2 *pref = reinterpret_cast<const __half2 *>(smb + GH::PREF_OFF);
                const __half2 *late = reinterpret_cast<const __half2 *>(smb);
#pragma unroll
                for (int v = 0; v < G0::V; v++) {
                    const int u = tid + v * C::T;
                    const int w = u & (C::W - 1);
                    const int hib = (u >> C::KW) & ((1 << G0::HB) - 1);
#pragma unroll
                    for (int r = 0; r < G0::R; r++) {
                        const int top = brev_c(r, G0::G) << G0::HB;   // compile-time
                        const int kb = top / GH::BOX;
                        const int in_box = ((top % GH::BOX) | hib) * C::W + w;
                        const __half2 *bx = kb < GH::NB ? pref + kb * GH::BOXV
                                                        : late + (kb - GH::NB) * GH::BOXV;
                        const float2 hv = __half22float2(bx[in_box]);
                        const float f = rf[top | hib];
                        a[v * G0::R + r] = make_float2(hv.x * f, hv.y * f);
                    }
                }
#pragma unroll
                for (int v = 0; v < G0::V; v++)
                    run_stages<C, 0, false, true>(a, v, 0, stw, C::L);
                fence_proxy_async_smem();
                if (tid == 0)
                    bulk_wait_read_all();   // the previous tile's stores have read it
                __syncthreads();            // every slot of both input regions has been read
                if (tid == 0 && next < ntiles)
                    issue_early(next);
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
            } else {
                group_first_split<C>(
                    a, sm, stw,
                    [&] {
                        if (tid == 0)
                            bulk_wait_read_all();   // the previous tile's stores have read it
                    },
                    [&] {
                        if (tid == 0 && next < ntiles)
                            issue_early(next);
                    });
            }
            if (next < ntiles)
                n_early++;
            __syncthreads();
            if constexpr (C::NG >= 3) {
                group_smem<C, 1, false, false, true>(a, sm, stw, C::L);
                __syncthreads();
            }
            group_last_read<C>(a, sm);
            fence_proxy_async_smem();
            __syncthreads();   // the tile region is free: the next tile's second half
            if (tid == 0 && next < ntiles)
                issue_late(next);
            if (next < ntiles)
                n_late++;
#pragma unroll
            for (int v = 0; v < Gl::V; v++) {
                const int u = tid + v * C::T;
                const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
                run_stages<C, C::NG - 1, false, true>(a, v, lo, stw, C::L);
            }
            if constexpr (R4) {
                // value r of unit v goes to the CTA whose final rows hold k's
                // top bits r: p = bit G-1 of r | bit G-2 of r << 1
                float2 *src = xb + par * (CS * CS * R4V * C::T) + q * (CS * R4V * C::T);
                static_assert(GC::KEEP_R % 2 == 0, "whole slot pairs");
#pragma unroll
                for (int v = 0; v < Gl::V; v++) {
                    if constexpr (VEC) {
#pragma unroll
                        for (int r = 0; r < Gl::R; r += 2) {
                            const int p =
                                ((r >> (Gl::G - 1)) & 1) | (((r >> (Gl::G - 2)) & 1) << 1);
                            const int sl = p * R4V + v * GC::KEEP_R + (r & (GC::KEEP_R - 1));
                            const float2 x0 = a[v * Gl::R + r], x1 = a[v * Gl::R + r + 1];
                            if (p != q)
                                __stcg(slot_pair<C>(src, sl / 2),
                                       make_float4(x0.x, x0.y, x1.x, x1.y));
                        }
                    } else {
#pragma unroll
                        for (int r = 0; r < Gl::R; r++) {
                            const int p =
                                ((r >> (Gl::G - 1)) & 1) | (((r >> (Gl::G - 2)) & 1) << 1);
                            if (p != q)
                                __stcg(src + (p * R4V + v * GC::KEEP_R + (r & (GC::KEEP_R - 1))) *
                                                 C::T,
                                       a[v * Gl::R + r]);
                        }
                    }
                }
            } else {
                float2 *mine = x0 + q * XV;
                group_round_send_g<C, 0, VEC>(a, mine, q & 1);
            }
        }
        // round 0 barrier: the flags and the values given away are visible
        cluster_arrive_release();
        float2 wk[R4 ? 2 * R4V : GC::XVALS];
        if constexpr (R4) {
            // stage L+1 and L+2 factors of this CTA's V x KEEP_R rows k
#pragma unroll
            for (int v = 0; v < Gl::V; v++) {
                const int u = tid + v * C::T;
                const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
#pragma unroll
                for (int i = 0; i < GC::KEEP_R; i++) {
                    const int k = lo | ((rk_end + i) << Gl::S0);
                    wk[v * GC::KEEP_R + i] = __ldg(tw + ((1 << C::L) - 1) + k);
                    wk[R4V + v * GC::KEEP_R + i] = __ldg(tw + ((1 << (C::L + 1)) - 1) + k);
                }
            }
        } else {
            group_round_twiddles<C, 0>(wk, tw, (q & 1) * (Gl::R / 2));
        }
        cluster_wait_acquire();
        {
            int any = 0;
#pragma unroll
            for (int p = 0; p < CS; p++)
                any |= lost_flag[par][p];
            if (any) {
                lost = true;
                break;
            }
        }
        if constexpr (R4) {
            // Y_t (t = 0..3, the four CTAs' blocks) at this CTA's rows k:
            // stage L+1 pairs (Y0, Y1) and (Y2, Y3) with W_{2^(L+1)}^k,
            // stage L+2 pairs (Z0, Z2) with W_{2^(L+2)}^k and (Z1, Z3) with
            // W_{2^(L+2)}^(k + 2^L), a quarter turn of it; outputs
            // X_t = a[t * R4V + v * KEEP_R + i] at rows k + 2^L t
            const float pq = -ld_tw<false>(tw + 2).y;
            const float2 *base = xb + par * (CS * CS * R4V * C::T) + q * (R4V * C::T);
            // this CTA's own rows: r = rk_end + i, rk_end = (q & 1) R/2 + (q >> 1) R/4
            auto own = [&](int v, int i) {
                const float2 o0 = a[v * Gl::R + 0 * (Gl::R / 4) + i];
                const float2 o1 = a[v * Gl::R + 2 * (Gl::R / 4) + i];
                const float2 o2 = a[v * Gl::R + 1 * (Gl::R / 4) + i];
                const float2 o3 = a[v * Gl::R + 3 * (Gl::R / 4) + i];
                return q == 0 ? o0 : q == 1 ? o1 : q == 2 ? o2 : o3;
            };
            float2 y[4][R4V];
            if constexpr (VEC) {
#pragma unroll
                for (int v = 0; v < Gl::V; v++) {
#pragma unroll
                    for (int i = 0; i < GC::KEEP_R; i += 2) {
                        const int jj = v * GC::KEEP_R + i;
                        const float2 own0 = own(v, i), own1 = own(v, i + 1);
#pragma unroll
                        for (int t = 0; t < CS; t++) {
                            float4 tp = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (t != q)
                                tp = __ldcg(slot_pair<C>(base, (t * CS * R4V + jj) / 2));
                            y[t][jj] = t == q ? own0 : make_float2(tp.x, tp.y);
                            y[t][jj + 1] = t == q ? own1 : make_float2(tp.z, tp.w);
                        }
                    }
                }
            } else {
#pragma unroll
                for (int v = 0; v < Gl::V; v++) {
#pragma unroll
                    for (int i = 0; i < GC::KEEP_R; i++) {
                        const int jj = v * GC::KEEP_R + i;
                        const float2 o = own(v, i);
#pragma unroll
                        for (int t = 0; t < CS; t++)
                            y[t][jj] = t == q ? o : __ldcg(base + (t * CS * R4V + jj) * C::T);
                    }
                }
            }
#pragma unroll
            for (int jj = 0; jj < R4V; jj++) {
                float2 z0 = y[0][jj], z1 = y[1][jj], z2 = y[2][jj], z3 = y[3][jj];
                butterfly_w(z0, z1, wk[jj]);
                butterfly_w(z2, z3, wk[jj]);
                butterfly_w(z0, z2, wk[R4V + jj]);
                butterfly_w(z1, z3, quarter_turn(wk[R4V + jj], pq));
                a[0 * R4V + jj] = z0;
                a[1 * R4V + jj] = z1;
                a[2 * R4V + jj] = z2;
                a[3 * R4V + jj] = z3;
            }
        } else {
            const float2 *theirs = x0 + (q ^ 1) * XV;
            group_round_compute_g<C, 0, VEC>(a, theirs, wk, q & 1);
        }
        if constexpr (DCT == 3) {
            constexpr int NN = C::N << CL;   // line length
            constexpr int HT = CS / 2;       // blocks t < HT are paired here
            constexpr int KR = GC::KEEP_R;
            constexpr int MREG = HT * GC::KEEP_V * C::T;
            static_assert(Gl::V == 1 && C::T == (1 << (Gl::S0 + C::KW)), "one unit per thread");
            float2 *mb = xbuf + (long long)cid * XSTRIDE + GC::L2_SCRATCH_VALS;
            const int w = tid & (C::W - 1);
            const int lo = tid >> C::KW;
            {
                // blocks t >= HT to CTA CS-1-q, each value in the slot of
                // the thread and index that pair it
                float2 *dst = mb + (CS - 1 - q) * MREG;
                const int tid_r = ((((1 << Gl::S0) - lo) & ((1 << Gl::S0) - 1)) << C::KW) | w;
#pragma unroll
                for (int t = HT; t < CS; t++) {
#pragma unroll
                    for (int i = 0; i < KR; i++) {
                        if (lo == 0 && i == 0)
                            continue;
                        const int i_r = lo != 0 ? KR - 1 - i : KR - i;
                        __stcg(dst + ((CS - 1 - t) * KR + i_r) * C::T + tid_r, a[t * KR + i]);
                    }
                }
                // row 0 of CTAs 2 and 3 of four: the other one pairs it
                if (CL == 2 && q >= 2 && lo == 0) {
                    float2 *d2 = mb + (q ^ 1) * MREG;
#pragma unroll
                    for (int t = HT; t < CS; t++)
                        __stcg(d2 + (CS - 1 - t) * KR * C::T + w, a[t * KR]);
                }
            }
            cluster_arrive_release();   // the mirror values are visible
            float2 r0[CS];              // row 0 of every block
#pragma unroll
            for (int t = 0; t < CS; t++)
                r0[t] = a[t * KR];
            if (q == 0 && lo == 0) {
                // K = N/2: row 0 of block HT in CTA 0, its own mirror
                float2 xk, xp;
                dct_pair(r0[HT], r0[HT], __ldg(post + NN / 2), scale, xk, xp);
                st_stream(io.mid_row + (long long)tile * C::W + w, xk);
            }
            cluster_wait_acquire();
            const float2 *src = mb + q * MREG + tid;
#pragma unroll
            for (int t = 0; t < HT; t++) {
#pragma unroll
                for (int i = 0; i < KR; i++) {
                    const float2 zk = a[t * KR + i];
                    float2 zp;
                    if (i == 0 && lo == 0 && q == 0)
                        zp = t == 0 ? zk : r0[CS - t];   // K = 0 and NL t: CTA 0's own
                    else if (i == 0 && lo == 0 && k_base == C::N / 2)
                        zp = r0[CS - 1 - t];             // k = NL/2 mirrors itself
                    else
                        zp = __ldcg(src + (t * KR + i) * C::T);
                    const float2 rb = rot_base[t * KR + i];
                    const float2 cs = make_float2(rb.x * rot_lo.x - rb.y * rot_lo.y,
                                                  rb.x * rot_lo.y + rb.y * rot_lo.x);
                    float2 xk, xp;
                    dct_pair(zk, zp, cs, scale, xk, xp);
                    a[t * KR + i] = xk;
                    a[(t + HT) * KR + i] = xp;
                }
            }
            // X[K] of blocks t < HT: one staging fill, one TMA store per range
#pragma unroll
            for (int t = 0; t < HT; t++)
#pragma unroll
                for (int i = 0; i < KR; i++)
                    stage[(t * GC::OUT_ROWS + ((i << Gl::S0) | lo)) * C::W + w] = a[t * KR + i];
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
#pragma unroll
                for (int t = 0; t < HT; t++)
                    tma_store_3d(omap, tile * C::W, 0, ((t << C::L) + k_base) / S::BOX,
                                 stage + t * GC::OUT_ROWS * C::W);
                bulk_commit();
                bulk_wait_read_all();
            }
            __syncthreads();
            // X[N-K]: the same ranges in reverse, rows y0 + s, y0 = N - NL t
            // - k_base - OUT_ROWS + 1, in 256-row boxes of omap2
#pragma unroll
            for (int t = 0; t < HT; t++)
#pragma unroll
                for (int i = 0; i < KR; i++)
                    stage[(t * GC::OUT_ROWS + GC::OUT_ROWS - 1 - ((i << Gl::S0) | lo)) * C::W + w] =
                        a[(t + HT) * KR + i];
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
#pragma unroll
                for (int t = 0; t < HT; t++) {
                    const int y0 = NN - (t << C::L) - k_base - GC::OUT_ROWS + 1;
#pragma unroll
                    for (int j = 0; j < GC::OUT_BOX_Z; j++)
                        tma_store_3d(omap2, tile * C::W, y0 + j * S::BOX, 0,
                                     stage + (t * GC::OUT_ROWS + j * S::BOX) * C::W);
                }
                bulk_commit();
            }
            continue;
        }
        if constexpr (DCT == 2) {
            // x[2n] = Re v[n] (n < N/2, the even rows), x[2(N-1-n)+1] = Re
            // v[n] (the odd rows, in reverse order within a range)
            float *fst = reinterpret_cast<float *>(stage);
#pragma unroll
            for (int t = 0; t < CS; t++) {
                const bool odd = t >= CS / 2;
#pragma unroll
                for (int v = 0; v < Gl::V; v++) {
                    const int u = tid + v * C::T;
                    const int w = u & (C::W - 1);
                    const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
#pragma unroll
                    for (int i = 0; i < GC::KEEP_R; i++) {
                        const int row = (i << Gl::S0) | lo;
                        const int slot = odd ? GC::OUT_ROWS - 1 - row : row;
                        fst[(t * GC::OUT_ROWS + slot) * C::W + w] =
                            a[(t * Gl::V + v) * GC::KEEP_R + i].x * scale;
                    }
                }
            }
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
                constexpr int NN = C::N << CL;
#pragma unroll
                for (int t = 0; t < CS; t++) {
                    const int n0 = (t << C::L) + k_base;
                    if (t < CS / 2)
                        tma_store_3d(omap, tile * (C::W / 2), 0, n0 / S::BOX,
                                     fst + t * GC::OUT_ROWS * C::W);
                    else
                        tma_store_3d(omap2, tile * (C::W / 2), 0,
                                     (NN - n0 - GC::OUT_ROWS) / S::BOX,
                                     fst + t * GC::OUT_ROWS * C::W);
                }
                bulk_commit();
            }
            continue;
        }
        if constexpr (DCT == 1) {
            // X[K] = cos(theta) Re V[K] + sin(theta) Im V[K], theta = pi K /
            // (2N), K = k + 2^L t; (cos, sin) of K > N/2 is (sin, cos) of N - K
            constexpr int NN = C::N << CL;
            float *fst = reinterpret_cast<float *>(stage);
#pragma unroll
            for (int t = 0; t < CS; t++) {
#pragma unroll
                for (int v = 0; v < Gl::V; v++) {
                    const int u = tid + v * C::T;
                    const int w = u & (C::W - 1);
                    const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
#pragma unroll
                    for (int i = 0; i < GC::KEEP_R; i++) {
                        const int row = (i << Gl::S0) | lo;
                        const int K = (t << C::L) + k_base + row;
                        const float2 cs = K <= NN / 2 ? __ldg(post + K) : __ldg(post + (NN - K));
                        const float c = K <= NN / 2 ? cs.x : cs.y;
                        const float sn = K <= NN / 2 ? cs.y : cs.x;
                        const float2 z = a[(t * Gl::V + v) * GC::KEEP_R + i];
                        fst[(t * GC::OUT_ROWS + row) * C::W + w] = (c * z.x + sn * z.y) * scale;
                    }
                }
            }
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
#pragma unroll
                for (int t = 0; t < CS; t++) {
                    const int z = ((t << C::L) + k_base) / S::BOX;
                    tma_store_3d(omap, tile * (C::W / 2), 0, z,
                                 fst + t * GC::OUT_ROWS * C::W);
                }
                bulk_commit();
            }
            continue;
        }
        if constexpr (H16) {
            // this CTA's part of each column's largest |component| (a
            // thread's values all belong to column tid mod W) to every CTA of
            // the cluster, one more cluster barrier, then every CTA picks the
            // same exponent per column and stages all its ranges as half2
            float m = 0.f;
#pragma unroll
            for (int i = 0; i < C::EPT; i++)
                m = fmaxf(m, fmaxf(fabsf(a[i].x), fabsf(a[i].y)));
            m = warp_line_max<C::KW, 5>(m);
            if ((tid & (31 & ~(C::W - 1))) == 0)
                atomicMax(&cmax_local[tid & (C::W - 1)], __float_as_int(m * scale));
            __syncthreads();
            if (tid < C::W) {
                const int mine = cmax_local[tid];
                cmax_local[tid] = 0;
#pragma unroll
                for (int p = 0; p < CS; p++)
                    *cluster.map_shared_rank(&cmax[par][q][tid], p) = mine;
            }
            cluster_arrive_release();
            cluster_wait_acquire();
            const int w = tid & (C::W - 1);
            int mb = 0;
#pragma unroll
            for (int p = 0; p < CS; p++)
                mb = max(mb, cmax[par][p][w]);
            const int e = line_exponent(__int_as_float(mb));
            const float f = scale * pow2f(-e);
            __half2 *hst = reinterpret_cast<__half2 *>(stage);
#pragma unroll
            for (int t = 0; t < CS; t++) {
#pragma unroll
                for (int v = 0; v < Gl::V; v++) {
                    const int u = tid + v * C::T;
                    const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
#pragma unroll
                    for (int i = 0; i < GC::KEEP_R; i++) {
                        const float2 x = a[(t * Gl::V + v) * GC::KEEP_R + i];
                        hst[(t * GC::OUT_ROWS + ((i << Gl::S0) | lo)) * C::W + w] =
                            __floats2half2_rn(x.x * f, x.y * f);
                    }
                }
            }
            if (q == 0 && tid < C::W)
                io.out_exp[tile * C::W + tid] = e;
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
#pragma unroll
                for (int t = 0; t < CS; t++) {
                    const int z = ((t << C::L) + k_base) / S::BOX;
                    tma_store_3d(omap, tile * C::W, 0, z, hst + t * GC::OUT_ROWS * C::W);
                }
                bulk_commit();
            }
            continue;
        }
        // outputs t = 0 .. CS-1: rows k_base + [0, OUT_ROWS) + 2^L t, STAGE_T
        // ranges per fill of the staging half, each range one TMA store
#pragma unroll
        for (int f = 0; f < CS / GC::STAGE_T; f++) {
            if (f > 0) {
                if (tid == 0)
                    bulk_wait_read_all();
                __syncthreads();
            }
#pragma unroll
            for (int ts = 0; ts < GC::STAGE_T; ts++) {
                const int t = f * GC::STAGE_T + ts;
#pragma unroll
                for (int v = 0; v < Gl::V; v++) {
                    const int u = tid + v * C::T;
                    const int w = u & (C::W - 1);
                    const int lo = (u >> C::KW) & ((1 << Gl::S0) - 1);
#pragma unroll
                    for (int i = 0; i < GC::KEEP_R; i++) {
                        const float2 x = a[(t * Gl::V + v) * GC::KEEP_R + i];
                        stage[(ts * GC::OUT_ROWS + ((i << Gl::S0) | lo)) * C::W + w] =
                            make_float2(x.x * scale, x.y * scale);
                    }
                }
            }
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0) {
#pragma unroll
                for (int ts = 0; ts < GC::STAGE_T; ts++) {
                    const int t = f * GC::STAGE_T + ts;
                    const int z = ((t << C::L) + k_base) / S::BOX;
                    tma_store_3d(omap, tile * C::W, 0, z, stage + ts * GC::OUT_ROWS * C::W);
                }
                bulk_commit();
            }
        }
    }

    if (__syncthreads_or(lost ? 1 : 0)) {
        if (tid == 0)
            atomicExch(err, kDevErrTmaTimeout);
        // let transfers still in flight land before the CTA leaves
        if (n_early > w_early)
            mbar_wait_bounded(&bar_early, (uint32_t)(w_early & 1));
        if (n_late > w_late)
            mbar_wait_bounded(&bar_late, (uint32_t)(w_late & 1));
    }
    if (tid == 0)
        bulk_wait_all();   // shared memory stays valid until the stores are done
}

// The forward DCT-II column pass of real columns on the same kernel (DCT
// mode above): per residue rev(q) a map of the ascending rows (first half of
// the local line) and one of the rows read backwards (second half).
struct DctL2Maps {
    CUtensorMap early[4], late[4];
    CUtensorMap out;
};

template <class C, int CL>
__global__ void __launch_bounds__(C::T, 1) col_dct_l2_kernel(const __grid_constant__ DctL2Maps maps,
                                                             const float2 *__restrict__ tw,
                                                             const float2 *__restrict__ post,
                                                             int ntiles, float scale, int *err,
                                                             int withhold, float2 *xbuf)
{
    const int q = (int)cooperative_groups::this_cluster().block_rank();
    const int res = brev_rt(q, CL);
    col_group_l2_body<C, CL, false, 1>(&maps.early[res], &maps.out, ntiles, tw, scale, err,
                                       withhold, xbuf, GroupIO{nullptr, nullptr}, &maps.late[res],
                                       post);
}

// The forward DCT-II column pass with two real columns per complex line
// (DCT == 3 above): per residue the complex maps of the ascending and the
// backwards rows, the output map of whole ranges, the any-row map of the
// reversed ranges, and the output row N/2.
struct DctPackMaps {
    CUtensorMap early[4], late[4];
    CUtensorMap out, out2;
    float2 *mid_row;
};

template <class C, int CL>
__global__ void __launch_bounds__(C::T, 1) col_dct_pack_l2_kernel(
    const __grid_constant__ DctPackMaps maps, const float2 *__restrict__ tw,
    const float2 *__restrict__ post, int ntiles, float scale, int *err, int withhold,
    float2 *xbuf)
{
    const int q = (int)cooperative_groups::this_cluster().block_rank();
    const int res = brev_rt(q, CL);
    col_group_l2_body<C, CL, false, 3>(&maps.early[res], &maps.out, ntiles, tw, scale, err,
                                       withhold, xbuf, GroupIO{nullptr, nullptr, maps.mid_row},
                                       &maps.late[res], post, &maps.out2);
}

// The inverse DCT-III column pass of real columns (DCT == 2 above): per
// residue a map of its rows (the mirror of residue r is residue (CS-r) mod
// CS), and store maps over the even and the odd rows of the output.
struct IdctL2Maps {
    CUtensorMap rows[4];
    CUtensorMap even, odd;
};

template <class C, int CL>
__global__ void __launch_bounds__(C::T, 1) col_idct_l2_kernel(const __grid_constant__ IdctL2Maps maps,
                                                              const float2 *__restrict__ tw,
                                                              const float2 *__restrict__ post,
                                                              int ntiles, float scale, int *err,
                                                              int withhold, float2 *xbuf)
{
    constexpr int CS = 1 << CL;
    const int q = (int)cooperative_groups::this_cluster().block_rank();
    const int res = brev_rt(q, CL);
    col_group_l2_body<C, CL, false, 2>(&maps.rows[res], &maps.even, ntiles, tw, scale, err,
                                       withhold, xbuf, GroupIO{nullptr, nullptr},
                                       &maps.rows[(CS - res) & (CS - 1)], post, &maps.odd);
}

template <class C, int CL, bool H16 = false>
__global__ void __launch_bounds__(C::T, 1) col_group_l2_kernel(const __grid_constant__ CUtensorMap map0,
                                                               const __grid_constant__ CUtensorMap map1,
                                                               const __grid_constant__ CUtensorMap map2,
                                                               const __grid_constant__ CUtensorMap map3,
                                                               const __grid_constant__ CUtensorMap omap,
                                                               const float2 *__restrict__ tw,
                                                               int cols, float scale, int *err,
                                                               int withhold, float2 *xbuf,
                                                               const GroupIO io)
{
    const int q = (int)cooperative_groups::this_cluster().block_rank();
    const int res = brev_rt(q, CL);
    const CUtensorMap *m = res == 0 ? &map0 : res == 1 ? &map1 : res == 2 ? &map2 : &map3;
    col_group_l2_body<C, CL, H16>(m, &omap, cols / C::W, tw, scale, err, withhold, xbuf, io);
}

}  // namespace fft2d
