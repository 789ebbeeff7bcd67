// line_fft.cuh -- the per-CTA radix-2 decimation-in-time engine shared by the
// row pass and the column pass of the 2D FFT.
//
// What one CTA computes (Section 2 eqs. 2-3, Section 3.1 eq. 4, Section 3.2):
// LB separate lines ("line blocks") of N = 2^L points, each block holding W
// interleaved lines, i.e. LB*W independent length-N transforms.  Each line is
// scrambled (bit-reversed) and then run through stages s = 1..L of N/2
// butterflies
//     X(j) = Xe(j) + W_{2^s}^j Xo(j),   X(j + 2^(s-1)) = Xe(j) - W_{2^s}^j Xo(j)
// on the in-place positions p of the scrambled line.
//
// GB300 mapping (not the paper's one-render-per-stage design):
//  * Stage fusion: stage s touches bit s-1 of the position p, so the stages
//    are cut into groups of <= 4 consecutive stages (bits [S0, S0+G)).  In a
//    group each thread holds, in registers, "units" of 2^G positions that
//    differ only in those bits and runs the group's G stages on them without
//    any memory traffic.  Between groups the line goes through shared memory
//    once.  Every thread always holds 16 complex values.
//  * Fused scramble: group 0 reads global memory directly.  Its unit with
//    register index r and "hi" bits h sits at position p = r | h << G, which
//    holds input element rev_L(p) = rev_G(r) << (L-G) | rev(h).  Threads are
//    numbered by rev(h), so for each r a warp reads consecutive elements:
//    the bit reversal costs no extra pass and no uncoalesced access.
//  * The last group's positions p = lo | r << S0 are the natural output
//    order, so the store is coalesced too.
//  * Shared memory is XOR-swizzled so that both the scrambled group-0 writes
//    (lanes differ in the top bits of p) and the later accesses (lanes differ
//    in the low bits of p) are free of bank conflicts.
//  * Twiddles come from a per-stage table (stage s holds W_{2^s}^j for
//    j < 2^(s-1) at offset 2^(s-1)-1; the paper's "log(N) rows" secondary
//    texture, compacted), built in FP64 on the host and rounded to FP32.  In
//    a group after the first, lanes read consecutive entries.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fft2d {

__host__ __device__ constexpr int brev_c(int v, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; b++)
        if (v & (1 << b))
            r |= 1 << (bits - 1 - b);
    return r;
}

__device__ __forceinline__ int brev_rt(int v, int bits)
{
    return bits == 0 ? 0 : (int)(__brev((unsigned)v) >> (32 - bits));
}

// Geometry of one CTA's work: lines of 2^L points, 2^KW interleaved lines
// (adjacent in memory: the column pass), 2^KB separate line blocks (the row
// pass), 16 values per thread.
template <int L_, int KW_, int KB_>
struct LineCfg {
    static constexpr int L = L_, KW = KW_, KB = KB_;
    static constexpr int N = 1 << L, W = 1 << KW, LB = 1 << KB;
    static constexpr int E = N * W * LB;
    static constexpr int T = E / 16;
    static constexpr int NG = (L + 3) / 4;
    // lanes of a half-warp that are not spent on the interleave index
    static constexpr int K = KW >= 4 ? 0 : 4 - KW;
    static constexpr bool SWZ = K > 0 && L >= 2 * K;
    static constexpr int SMEM_BYTES = NG > 1 ? E * 8 : 0;
    static_assert(L >= 1 && L <= 14, "line length out of range");
    static_assert(E >= 16, "CTA must hold at least 16 values");
};

// Group GI of the stage groups: bits [S0, S0 + G) of p.
template <class C, int GI>
struct Grp {
    static constexpr int S0 = 4 * GI;
    static constexpr int G = (C::L - S0) < 4 ? (C::L - S0) : 4;
    static constexpr int R = 1 << G;             // values per unit
    static constexpr int V = 16 / R;             // units per thread
    static constexpr int HB = C::L - S0 - G;     // bits above the group
};

// Shared-memory slot of (line block lb, position p, interleaved line w).
template <class C>
__device__ __forceinline__ int sidx(int lb, int p, int w)
{
    int q = p;
    if constexpr (C::SWZ)
        q = p ^ ((p >> (C::L - C::K)) & ((1 << C::K) - 1));
    return (((lb << C::L) | q) << C::KW) | w;
}

// Stages S0+1 .. S0+G on unit v of a[]: pairs (r, r + 2^t) at stage S0+1+t use
// W_{2^s}^j with j = lo + (r mod 2^t) 2^S0.
template <class C, int GI, bool GENERIC>
__device__ __forceinline__ void run_stages(float2 (&a)[16], int v, int lo,
                                           const float2 *__restrict__ tw, int nst)
{
    using Gp = Grp<C, GI>;
#pragma unroll
    for (int t = 0; t < Gp::G; t++) {
        const int s = Gp::S0 + 1 + t;
        if (GENERIC && s > nst)
            return;
        const float2 *tws = tw + ((1 << (s - 1)) - 1);
#pragma unroll
        for (int r = 0; r < Gp::R; r++) {
            if (r & (1 << t))
                continue;
            const int jc = (r & ((1 << t) - 1)) << Gp::S0;
            float2 &x0 = a[v * Gp::R + r];
            float2 &x1 = a[v * Gp::R + (r | (1 << t))];
            float2 m;
            if (GI == 0 && jc == 0) {
                m = x1;   // W = 1
            } else {
                const float2 w = __ldg(tws + lo + jc);
                m.x = w.x * x1.x - w.y * x1.y;
                m.y = w.x * x1.y + w.y * x1.x;
            }
            x1 = make_float2(x0.x - m.x, x0.y - m.y);
            x0 = make_float2(x0.x + m.x, x0.y + m.y);
        }
    }
}

// Group 0: scrambled global load, first stages, then either the final store
// (single group, L <= 4) or the write to shared memory.
template <class C, bool ROW, bool GENERIC>
__device__ __forceinline__ void group_first(float2 (&a)[16], float2 *sm, const float2 *in,
                                            float2 *out, const float2 *__restrict__ tw,
                                            long long ld, float scale, int nst,
                                            long long nvalid)
{
    using Gp = Grp<C, 0>;
    const int tid = threadIdx.x;
#pragma unroll
    for (int v = 0; v < Gp::V; v++) {
        const int u = tid + v * C::T;
        const int w = u & (C::W - 1);
        const int u2 = u >> C::KW;
        const int hib = u2 & ((1 << Gp::HB) - 1);
        const int lb = u2 >> Gp::HB;
        const bool ok = !GENERIC || (ROW ? lb < nvalid : w < nvalid);
        const float2 *src = ROW ? in + (long long)lb * ld + hib : in + (long long)hib * ld + w;
#pragma unroll
        for (int r = 0; r < Gp::R; r++) {
            const int off = brev_c(r, Gp::G) << Gp::HB;
            a[v * Gp::R + r] = ok ? src[ROW ? (long long)off : (long long)off * ld]
                                  : make_float2(0.f, 0.f);
        }
    }
#pragma unroll
    for (int v = 0; v < Gp::V; v++)
        run_stages<C, 0, GENERIC>(a, v, 0, tw, nst);
#pragma unroll
    for (int v = 0; v < Gp::V; v++) {
        const int u = tid + v * C::T;
        const int w = u & (C::W - 1);
        const int u2 = u >> C::KW;
        const int hib = u2 & ((1 << Gp::HB) - 1);
        const int lb = u2 >> Gp::HB;
        if constexpr (C::NG == 1) {
            // whole line in this unit: positions p = r are the output order
            const bool ok = !GENERIC || (ROW ? lb < nvalid : w < nvalid);
            if (ok) {
                float2 *dst = ROW ? out + (long long)lb * ld : out + w;
#pragma unroll
                for (int r = 0; r < Gp::R; r++) {
                    const float2 x = a[v * Gp::R + r];
                    dst[ROW ? (long long)r : (long long)r * ld] =
                        make_float2(x.x * scale, x.y * scale);
                }
            }
        } else {
            const int hi = brev_rt(hib, Gp::HB);
#pragma unroll
            for (int r = 0; r < Gp::R; r++)
                sm[sidx<C>(lb, r | (hi << Gp::G), w)] = a[v * Gp::R + r];
        }
    }
}

// Group GI >= 1: read units from shared memory, run the group's stages, then
// write back in place (middle group) or store to global memory (last group).
template <class C, int GI, bool ROW, bool GENERIC>
__device__ __forceinline__ void group_smem(float2 (&a)[16], float2 *sm, float2 *out,
                                           const float2 *__restrict__ tw, long long ld,
                                           float scale, int nst, long long nvalid)
{
    using Gp = Grp<C, GI>;
    constexpr bool LAST = (GI == C::NG - 1);
    const int tid = threadIdx.x;
#pragma unroll
    for (int v = 0; v < Gp::V; v++) {
        const int u = tid + v * C::T;
        const int w = u & (C::W - 1);
        const int u2 = u >> C::KW;
        const int lo = u2 & ((1 << Gp::S0) - 1);
        const int hi = (u2 >> Gp::S0) & ((1 << Gp::HB) - 1);
        const int lb = u2 >> (Gp::S0 + Gp::HB);
#pragma unroll
        for (int r = 0; r < Gp::R; r++)
            a[v * Gp::R + r] = sm[sidx<C>(lb, lo | (r << Gp::S0) | (hi << (Gp::S0 + Gp::G)), w)];
    }
#pragma unroll
    for (int v = 0; v < Gp::V; v++) {
        const int u = tid + v * C::T;
        const int lo = (u >> C::KW) & ((1 << Gp::S0) - 1);
        run_stages<C, GI, GENERIC>(a, v, lo, tw, nst);
    }
#pragma unroll
    for (int v = 0; v < Gp::V; v++) {
        const int u = tid + v * C::T;
        const int w = u & (C::W - 1);
        const int u2 = u >> C::KW;
        const int lo = u2 & ((1 << Gp::S0) - 1);
        const int hi = (u2 >> Gp::S0) & ((1 << Gp::HB) - 1);
        const int lb = u2 >> (Gp::S0 + Gp::HB);
        if constexpr (LAST) {
            const bool ok = !GENERIC || (ROW ? lb < nvalid : w < nvalid);
            if (ok) {
                float2 *dst = ROW ? out + (long long)lb * ld + lo : out + (long long)lo * ld + w;
#pragma unroll
                for (int r = 0; r < Gp::R; r++) {
                    const int off = r << Gp::S0;
                    const float2 x = a[v * Gp::R + r];
                    dst[ROW ? (long long)off : (long long)off * ld] =
                        make_float2(x.x * scale, x.y * scale);
                }
            }
        } else {
#pragma unroll
            for (int r = 0; r < Gp::R; r++)
                sm[sidx<C>(lb, lo | (r << Gp::S0) | (hi << (Gp::S0 + Gp::G)), w)] =
                    a[v * Gp::R + r];
        }
    }
}

// The whole line transform of one CTA.  in/out point at the CTA's first line
// (row pass: first row of its block; column pass: first column of its tile).
// ld is the image row pitch in complex elements.  nvalid (GENERIC only) is the
// number of line blocks (ROW) or interleaved lines (column pass) that exist.
template <class C, bool ROW, bool GENERIC>
__device__ __forceinline__ void line_fft(const float2 *in, float2 *out,
                                         const float2 *__restrict__ tw, long long ld,
                                         float scale, int nst, long long nvalid)
{
    extern __shared__ float2 sm[];
    float2 a[16];
    group_first<C, ROW, GENERIC>(a, sm, in, out, tw, ld, scale, nst, nvalid);
    if constexpr (C::NG >= 2) {
        __syncthreads();
        if constexpr (C::NG >= 3) {
            group_smem<C, 1, ROW, GENERIC>(a, sm, out, tw, ld, scale, nst, nvalid);
            __syncthreads();
        }
        if constexpr (C::NG >= 4) {
            group_smem<C, 2, ROW, GENERIC>(a, sm, out, tw, ld, scale, nst, nvalid);
            __syncthreads();
        }
        group_smem<C, C::NG - 1, ROW, GENERIC>(a, sm, out, tw, ld, scale, nst, nvalid);
    }
}

// Row pass: CTA b transforms rows [b*LB, b*LB + LB).  ld = row pitch.
template <class C, bool GENERIC>
__global__ void __launch_bounds__(C::T) row_pass_kernel(const float2 *in, float2 *out,
                                                        const float2 *__restrict__ tw,
                                                        int rows, long long ld, float scale,
                                                        int nst)
{
    const long long r0 = (long long)blockIdx.x * C::LB;
    line_fft<C, true, GENERIC>(in + r0 * ld, out + r0 * ld, tw, ld, scale, nst, rows - r0);
}

// Column pass: CTA b transforms columns [b*W, b*W + W), each of `rows`=2^L
// points spaced ld apart.
template <class C, bool GENERIC>
__global__ void __launch_bounds__(C::T) col_pass_kernel(const float2 *in, float2 *out,
                                                        const float2 *__restrict__ tw,
                                                        int cols, long long ld, float scale,
                                                        int nst)
{
    const long long c0 = (long long)blockIdx.x * C::W;
    line_fft<C, false, GENERIC>(in + c0, out + c0, tw, ld, scale, nst, cols - c0);
}

}  // namespace fft2d
