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

#include <cooperative_groups.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "async_copy.cuh"
#include "passes.h"

namespace fft2d {

__host__ __device__ constexpr int brev_c(int v, int bits)
{
    int r = 0;
    for (int b = 0; b < bits; b++)
        if (v & (1 << b))
            r |= 1 << (bits - 1 - b);
    return r;
}

// Image data is read exactly once: keep it out of L1 so that the rotation
// factor table, which every CTA re-reads, stays resident there.
__device__ __forceinline__ float2 ld_stream(const float2 *p)
{
    float2 v;
    asm volatile("ld.global.L1::no_allocate.v2.f32 {%0, %1}, [%2];"
                 : "=f"(v.x), "=f"(v.y)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ int brev_rt(int v, int bits)
{
    return bits == 0 ? 0 : (int)(__brev((unsigned)v) >> (32 - bits));
}

// Geometry of one CTA's work: lines of 2^L points, 2^KW interleaved lines
// (adjacent in memory: the column pass), 2^KB separate line blocks (the row
// pass), EPT (16, 32 or 64) values per thread, stage groups of GS stages (4;
// 5 with 32 values a thread; 6 with 64: one unit of 2^GS values, fewer
// groups and so fewer exchanges through shared memory, e.g. two instead of
// three groups for lines of 2^12 points with GS = 6).  The grouping changes
// where values wait between stages, not the butterflies, so every GS gives
// the same bits.
template <int L_, int KW_, int KB_, int EPT_ = 16, int GS_ = 4>
struct LineCfg {
    static constexpr int L = L_, KW = KW_, KB = KB_, EPT = EPT_, GS = GS_;
    static constexpr int N = 1 << L, W = 1 << KW, LB = 1 << KB;
    static constexpr int E = N * W * LB;
    static constexpr int T = E / EPT;
    static constexpr int NG = (L + GS - 1) / GS;
    static_assert(GS == 4 || (GS == 5 && EPT == 32) || (GS == 6 && EPT == 64),
                  "groups of 4 stages, 5 with 32 values a thread or 6 with 64");
    // lanes of a half-warp that are not spent on the interleave index
    static constexpr int K = KW >= 4 ? 0 : 4 - KW;
    static constexpr bool SWZ = K > 0 && L >= 2 * K;
    static constexpr int SMEM_BYTES = NG > 1 ? E * 8 : 0;
    // resident CTAs per SM asked of the register allocator: 64 registers a
    // thread with 16 values, 128 with 32, up to 255 with 64
    static constexpr int REGS = EPT == 16 ? 64 : (EPT == 32 ? 128 : 255);
    static constexpr int MINB = 65536 / (T * REGS) > 0 ? 65536 / (T * REGS) : 1;
    static_assert(L >= 1 && L <= 14, "line length out of range");
    static_assert(E >= EPT, "CTA must hold at least one thread's values");
    static_assert(EPT == 16 || EPT == 32 || EPT == 64, "16, 32 or 64 values per thread");
};

// A group of G consecutive stages S0+1 .. S0+G (bits [S0, S0 + G) of p) on
// lines of 2^L points.
template <int L, int S0_, int G_, int EPT = 16>
struct GrpSG {
    static constexpr int S0 = S0_;
    static constexpr int G = G_;
    static constexpr int R = 1 << G;             // values per unit
    static constexpr int V = EPT / R;            // units per thread
    static constexpr int HB = L - S0 - G;        // bits above the group
};

// Group GI of the stage groups of a CTA config: bits [GS GI, GS GI + G).
template <class C, int GI>
struct Grp : GrpSG<C::L, C::GS * GI, ((C::L - C::GS * GI) < C::GS ? (C::L - C::GS * GI) : C::GS),
                   C::EPT> {};

// Shared-memory slot of (line block lb, position p, interleaved line w).
template <class C>
__device__ __forceinline__ int sidx(int lb, int p, int w)
{
    int q = p;
    if constexpr (C::SWZ)
        q = p ^ ((p >> (C::L - C::K)) & ((1 << C::K) - 1));
    return (((lb << C::L) | q) << C::KW) | w;
}

// Rotation factor load: from global memory through the read-only path, or
// from a copy of the table in shared memory (TWS).
template <bool TWS>
__device__ __forceinline__ float2 ld_tw(const float2 *p)
{
    if constexpr (TWS)
        return *p;
    else
        return __ldg(p);
}

// One radix-2 butterfly (x0, x1) <- (x0 + W x1, x0 - W x1) with a fixed
// rounding sequence, so that every kernel variant -- whatever the compiler
// would otherwise contract -- produces the same bits.  Six fused
// multiply-adds: the sum y = x0 + W x1 takes two per component (x0 + the
// first partial product, then + the second), and the difference follows
// from it as 2 x0 - y (exact doubling, one rounding), instead of forming W x1
// and then both the sum and the difference (eight operations).
__device__ __forceinline__ void butterfly_w(float2 &x0, float2 &x1, float2 w)
{
    const float2 y = make_float2(__fmaf_rn(-w.y, x1.y, __fmaf_rn(w.x, x1.x, x0.x)),
                                 __fmaf_rn(w.y, x1.x, __fmaf_rn(w.x, x1.y, x0.y)));
    x1 = make_float2(__fmaf_rn(2.0f, x0.x, -y.x), __fmaf_rn(2.0f, x0.y, -y.y));
    x0 = y;
}

// Stages S0+1 .. S0+G on unit v of a[]: pairs (r, r + 2^t) at stage S0+1+t use
// W_{2^s}^j with j = lo + m 2^S0, m = r mod 2^t.
//
// Half of each stage's rotation factors come from the other half: for
// m >= 2^(t-1), j = j0 + 2^(s-2) with j0 = lo + (m - 2^(t-1)) 2^S0, and
// W_{2^s}^{j0 + 2^(s-2)} = W_4^1 W_{2^s}^{j0} -- a quarter turn, -i forward
// and +i inverse, exact in floating point (a swap and a sign).  The plan's
// tables hold the same values bit for bit (they are built with exact
// quarter-turn symmetry), so a unit loads 2^(t-1) factors instead of 2^t
// and the results do not change.  The turn's sign p = -Im W_4^1 (+1 forward,
// -1 inverse) is read once from the stage-2 entry of the table; adding 0
// turns the -0 of p * 0 into the table's +0.
__device__ __forceinline__ float2 quarter_turn(float2 w, float p)
{
    return make_float2(__fmaf_rn(p, w.y, 0.0f), __fmaf_rn(-p, w.x, 0.0f));
}

template <class Gp, bool FIRST, bool GENERIC, bool TWS = false, int NA>
__device__ __forceinline__ void run_stages_g(float2 (&a)[NA], int v, int lo,
                                             const float2 *__restrict__ tw, int nst)
{
    float p = 0.f;
    if constexpr (Gp::G >= 2)
        p = -ld_tw<TWS>(tw + 2).y;
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
            const int m = r & ((1 << t) - 1);
            float2 &x0 = a[v * Gp::R + r];
            float2 &x1 = a[v * Gp::R + (r | (1 << t))];
            if (FIRST && m == 0 && t < 4) {   // W = 1 (a 5th stage of group 0 takes the
                                              // table's W^0 as a 4-stage grouping does)
                const float2 d = x1;
                x1 = make_float2(__fsub_rn(x0.x, d.x), __fsub_rn(x0.y, d.y));
                x0 = make_float2(__fadd_rn(x0.x, d.x), __fadd_rn(x0.y, d.y));
            } else if (t >= 1 && m >= (1 << (t - 1))) {   // a quarter turn of a lower entry
                const int m0 = m - (1 << (t - 1));
                const float2 w0 = (FIRST && m0 == 0) ? make_float2(1.0f, 0.0f)
                                                     : ld_tw<TWS>(tws + lo + (m0 << Gp::S0));
                butterfly_w(x0, x1, quarter_turn(w0, p));
            } else {
                butterfly_w(x0, x1, ld_tw<TWS>(tws + lo + (m << Gp::S0)));
            }
        }
    }
}

template <class C, int GI, bool GENERIC, bool TWS = false>
__device__ __forceinline__ void run_stages(float2 (&a)[C::EPT], int v, int lo,
                                           const float2 *__restrict__ tw, int nst)
{
    run_stages_g<Grp<C, GI>, GI == 0, GENERIC, TWS>(a, v, lo, tw, nst);
}

// ---------------------------------------------------------------------------
// Global-memory storage of the image, used by the load of group 0 and the
// store of the last group (everything in between is FP32 in registers and
// shared memory).
//
//  * StoreC64: complex64, float2 per pixel.
//  * StoreH16: half2 per pixel, each line carrying a power-of-two exponent:
//    pixel = q * 2^e.  The input's exponents are per row (in_axis 0) or per
//    column (in_axis 1); the pass writes one exponent per line it owns (row
//    pass: per row, column pass: per column), chosen from that line's largest
//    component magnitude M as e = k - 14 where M = f 2^k, f in [0.5, 1), so
//    every stored |q| < 2^14, well inside half precision's range.
struct StoreC64 {
    static constexpr bool H16 = false;
    static constexpr int AXIS = -1;
    using T = float2;
    const float2 *in;
    float2 *out;
};

// IA: the input's exponent axis when fixed at compile time (0 per row, 1 per
// column), -1 when it is taken from in_axis at run time.
template <int IA = -1>
struct StoreH16T {
    static constexpr bool H16 = true;
    static constexpr int AXIS = IA;
    using T = __half2;
    const __half2 *in;
    __half2 *out;
    const int *in_exp;   // exponents of the input lines
    int in_axis;         // 0: one per row, 1: one per column
    int *out_exp;        // exponents of this pass's output lines
    __device__ __forceinline__ int axis() const { return IA >= 0 ? IA : in_axis; }
};
using StoreH16 = StoreH16T<-1>;

// 2^e as a float (exact), e clamped to the normal range.
__device__ __forceinline__ float pow2f(int e)
{
    e = e < -126 ? -126 : (e > 127 ? 127 : e);
    return __int_as_float((127 + e) << 23);
}

// Exponent of a line from its largest component magnitude (see StoreH16).
__device__ __forceinline__ int line_exponent(float m)
{
    const int bits = __float_as_int(m);
    const int ebits = (bits >> 23) & 0xff;
    if (ebits == 0)
        return 0;                       // zero (or subnormal) line
    return (ebits - 126) - 14;          // m = f 2^(ebits-126), f in [0.5, 1)
}

// Where the CTA's elements live: element i of line lb (row pass) is pixel
// (r0 + lb, i); element i of interleaved line w (column pass) is pixel
// (r0 + i * rstep, c0 + w).  ld = row pitch in pixels.
struct Geo {
    long long r0, rstep, c0, ld;
};

template <bool ROW>
__device__ __forceinline__ long long pix(const Geo &g, int lb, int i, int w)
{
    return ROW ? (g.r0 + lb) * g.ld + i : (g.r0 + (long long)i * g.rstep) * g.ld + g.c0 + w;
}

// Whether every value of one unit of group 0 (one line block lb, one
// interleaved line w) shares its input exponent: the exponent runs along the
// line being transformed.
template <class IO, bool ROW>
struct H16PerUnit {
    static constexpr bool value = IO::H16 && ((ROW && IO::AXIS == 0) || (!ROW && IO::AXIS == 1));
};

// 2^e of the input line holding element i of line (lb, w).
template <class IO, bool ROW>
__device__ __forceinline__ float in_factor(const IO &io, const Geo &g, int lb, int i, int w)
{
    const long long line = io.axis() == 0 ? (ROW ? g.r0 + lb : g.r0 + (long long)i * g.rstep)
                                          : (ROW ? (long long)i : g.c0 + w);
    return pow2f(io.in_exp[line]);
}

// Element i of line (lb, w); for half2 storage, f is its line's 2^e when
// the caller already knows it (H16PerUnit), else 0.
template <class IO, bool ROW>
__device__ __forceinline__ float2 load_pix(const IO &io, const Geo &g, int lb, int i, int w,
                                           float f = 0.f)
{
    const long long k = pix<ROW>(g, lb, i, w);
    if constexpr (IO::H16) {
        const float2 q = __half22float2(io.in[k]);
        if constexpr (!H16PerUnit<IO, ROW>::value)
            f = in_factor<IO, ROW>(io, g, lb, i, w);
        return make_float2(q.x * f, q.y * f);
    } else {
        return ld_stream(io.in + k);
    }
}

// Max of m over the lanes of a warp that hold values of the same output
// line, for a line index that is constant over the lane bits [B0, B1):
// afterwards the lane with those bits clear holds the maximum.
template <int B0, int B1>
__device__ __forceinline__ float warp_line_max(float m)
{
#pragma unroll
    for (int b = B0; b < B1; b++)
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1 << b));
    return m;
}

// Store the units of a finished line group.  For half2 storage each line's
// exponent is chosen first: the largest |component| of every line is
// max-reduced in shared memory (sred, one int per line, zeroed at kernel
// start), which costs one barrier; the thread holding position 0 of a line
// writes its exponent.  pos(v, r) is the position of value r of unit v.
template <class C, bool ROW, bool GENERIC, class IO, class Gp, class Pos>
__device__ __forceinline__ void store_units(float2 (&a)[C::EPT], const IO &io, const Geo &g,
                                            float scale, long long nvalid, int *sred,
                                            Pos pos)
{
    const int tid = threadIdx.x;
    if constexpr (IO::H16) {
        // lanes of a warp that share an output line: row pass, lanes that
        // differ only in the unit bits below the group's start (the line
        // block is the unit index above them); column pass, lanes that
        // differ only above the interleave bits (the line is u mod W)
        constexpr int S0 = Gp::S0;
        constexpr int RB0 = 0, RB1 = C::NG == 1 ? 0 : (S0 < 5 ? S0 : 5);
        constexpr int CB0 = C::KW < 5 ? C::KW : 5, CB1 = 5;
        constexpr int B0 = ROW ? RB0 : CB0, B1 = ROW ? RB1 : CB1;
        constexpr unsigned LMASK = ((1u << B1) - 1u) & ~((1u << B0) - 1u);
#pragma unroll
        for (int v = 0; v < Gp::V; v++) {
            const int u = tid + v * C::T;
            const int w = u & (C::W - 1);
            const int lb = ROW ? pos(v, 0) >> C::L : 0;
            const bool ok = !GENERIC || (ROW ? lb < nvalid : w < nvalid);
            float m = 0.f;
#pragma unroll
            for (int r = 0; r < Gp::R; r++)
                m = fmaxf(m, fmaxf(fabsf(a[v * Gp::R + r].x), fabsf(a[v * Gp::R + r].y)));
            m = warp_line_max<B0, B1>(m);
            if (ok && (tid & LMASK) == 0)
                atomicMax(sred + (ROW ? lb : w), __float_as_int(m * scale));
        }
        __syncthreads();
    }
#pragma unroll
    for (int v = 0; v < Gp::V; v++) {
        const int u = tid + v * C::T;
        const int w = u & (C::W - 1);
        const int lb = ROW ? pos(v, 0) >> C::L : 0;
        const bool ok = !GENERIC || (ROW ? lb < nvalid : w < nvalid);
        if (!ok)
            continue;
        float f = scale;
        int e = 0;
        if constexpr (IO::H16) {
            e = line_exponent(__int_as_float(sred[ROW ? lb : w]));
            f = scale * pow2f(-e);
        }
#pragma unroll
        for (int r = 0; r < Gp::R; r++) {
            const int p = pos(v, r) & (C::N - 1);
            const float2 x = a[v * Gp::R + r];
            const long long k = pix<ROW>(g, lb, p, w);
            if constexpr (IO::H16) {
                io.out[k] = __floats2half2_rn(x.x * f, x.y * f);
                if (p == 0)
                    io.out_exp[ROW ? g.r0 + lb : g.c0 + w] = e;
            } else {
                io.out[k] = make_float2(x.x * f, x.y * f);
            }
        }
    }
}

// Group 0: scrambled global load, first stages, then either the final store
// (single group, L <= 4) or the write to shared memory.
template <class C, bool ROW, bool GENERIC, class IO>
__device__ __forceinline__ void group_first(float2 (&a)[C::EPT], float2 *sm, const IO &io,
                                            const Geo &g, const float2 *__restrict__ tw,
                                            float scale, int nst, long long nvalid, int *sred)
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
        float f = 0.f;
        if constexpr (H16PerUnit<IO, ROW>::value)
            f = ok ? in_factor<IO, ROW>(io, g, lb, 0, w) : 0.f;
#pragma unroll
        for (int r = 0; r < Gp::R; r++) {
            const int i = (brev_c(r, Gp::G) << Gp::HB) | hib;
            a[v * Gp::R + r] = ok ? load_pix<IO, ROW>(io, g, lb, i, w, f) : make_float2(0.f, 0.f);
        }
    }
#pragma unroll
    for (int v = 0; v < Gp::V; v++)
        run_stages<C, 0, GENERIC>(a, v, 0, tw, nst);
    if constexpr (C::NG == 1) {
        // the whole line is in one unit: positions p = r are the output order
        store_units<C, ROW, GENERIC, IO, Gp>(a, io, g, scale, nvalid, sred, [&](int v, int r) {
            const int u = tid + v * C::T;
            const int lb = (u >> C::KW) >> Gp::HB;
            return (lb << C::L) | r;
        });
    } else {
#pragma unroll
        for (int v = 0; v < Gp::V; v++) {
            const int u = tid + v * C::T;
            const int w = u & (C::W - 1);
            const int u2 = u >> C::KW;
            const int hib = u2 & ((1 << Gp::HB) - 1);
            const int lb = u2 >> Gp::HB;
            const int hi = brev_rt(hib, Gp::HB);
#pragma unroll
            for (int r = 0; r < Gp::R; r++)
                sm[sidx<C>(lb, r | (hi << Gp::G), w)] = a[v * Gp::R + r];
        }
    }
}

// Group GI >= 1 that stays in shared memory: read units, run the group's
// stages, write back in place (a middle group) or, for the last group with
// TO_SMEM, leave the finished lines in natural order, slot k*W + w (used by
// the cluster column pass, whose last stages run across CTAs).
template <class C, int GI, bool GENERIC, bool TO_SMEM = false, bool TWS = false>
__device__ __forceinline__ void group_smem(float2 (&a)[C::EPT], float2 *sm,
                                           const float2 *__restrict__ tw, int nst)
{
    using Gp = Grp<C, GI>;
    constexpr bool LAST = (GI == C::NG - 1);
    static_assert(!LAST || TO_SMEM, "the last group with a global store is group_last");
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
        run_stages<C, GI, GENERIC, TWS>(a, v, lo, tw, nst);
    }
    if constexpr (LAST && TO_SMEM) {
        // the natural-order slots differ from the swizzled ones just read
        if constexpr (C::SWZ)
            __syncthreads();
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
#pragma unroll
            for (int r = 0; r < Gp::R; r++)
                sm[((lo | (r << Gp::S0)) << C::KW) | w] = a[v * Gp::R + r];
        } else {
#pragma unroll
            for (int r = 0; r < Gp::R; r++)
                sm[sidx<C>(lb, lo | (r << Gp::S0) | (hi << (Gp::S0 + Gp::G)), w)] =
                    a[v * Gp::R + r];
        }
    }
}

// The last group (GI = NG-1 >= 1): read units from shared memory, run the
// group's stages, store natural-order positions p = lo | r << S0 to global.
template <class C, bool ROW, bool GENERIC, class IO, bool TWS = false>
__device__ __forceinline__ void group_last(float2 (&a)[C::EPT], float2 *sm, const IO &io,
                                           const Geo &g, const float2 *__restrict__ tw,
                                           float scale, int nst, long long nvalid, int *sred)
{
    using Gp = Grp<C, C::NG - 1>;
    static_assert(Gp::HB == 0, "last group");
    const int tid = threadIdx.x;
#pragma unroll
    for (int v = 0; v < Gp::V; v++) {
        const int u = tid + v * C::T;
        const int w = u & (C::W - 1);
        const int u2 = u >> C::KW;
        const int lo = u2 & ((1 << Gp::S0) - 1);
        const int lb = u2 >> Gp::S0;
#pragma unroll
        for (int r = 0; r < Gp::R; r++)
            a[v * Gp::R + r] = sm[sidx<C>(lb, lo | (r << Gp::S0), w)];
    }
#pragma unroll
    for (int v = 0; v < Gp::V; v++) {
        const int u = tid + v * C::T;
        const int lo = (u >> C::KW) & ((1 << Gp::S0) - 1);
        run_stages<C, C::NG - 1, GENERIC, TWS>(a, v, lo, tw, nst);
    }
    store_units<C, ROW, GENERIC, IO, Gp>(a, io, g, scale, nvalid, sred, [&](int v, int r) {
        const int u = tid + v * C::T;
        const int u2 = u >> C::KW;
        const int lo = u2 & ((1 << Gp::S0) - 1);
        const int lb = u2 >> Gp::S0;
        return (lb << C::L) | lo | (r << Gp::S0);
    });
}

// Shared memory of a line_fft CTA: the exchange buffer, then (half2 storage)
// one int per output line for the exponent reduction.
template <class C, bool ROW, class IO>
struct LineSmem {
    static constexpr int RED_INTS = IO::H16 ? (ROW ? C::LB : C::W) : 0;
    static constexpr int BYTES = C::SMEM_BYTES + RED_INTS * 4;
};

// The whole line transform of one CTA.  nvalid (GENERIC only) is the number
// of line blocks (ROW) or interleaved lines (column pass) that exist.
template <class C, bool ROW, bool GENERIC, class IO>
__device__ __forceinline__ void line_fft(const IO &io, const Geo &g,
                                         const float2 *__restrict__ tw, float scale, int nst,
                                         long long nvalid)
{
    extern __shared__ float2 sm[];
    int *sred = reinterpret_cast<int *>(sm + C::E * (C::NG > 1 ? 1 : 0));
    if constexpr (IO::H16) {
        for (int i = threadIdx.x; i < LineSmem<C, ROW, IO>::RED_INTS; i += C::T)
            sred[i] = 0;
        if constexpr (C::NG == 1)
            __syncthreads();
    }
    float2 a[C::EPT];
    group_first<C, ROW, GENERIC, IO>(a, sm, io, g, tw, scale, nst, nvalid, sred);
    if constexpr (C::NG >= 2) {
        __syncthreads();
        if constexpr (C::NG >= 3) {
            group_smem<C, 1, GENERIC>(a, sm, tw, nst);
            __syncthreads();
        }
        if constexpr (C::NG >= 4) {
            group_smem<C, 2, GENERIC>(a, sm, tw, nst);
            __syncthreads();
        }
        group_last<C, ROW, GENERIC, IO>(a, sm, io, g, tw, scale, nst, nvalid, sred);
    }
}

// Row pass: CTA b transforms rows [b*LB, b*LB + LB).  ld = row pitch.
template <class C, bool GENERIC, class IO = StoreC64>
__global__ void __launch_bounds__(C::T, C::MINB) row_pass_kernel(const IO io,
                                                                 const float2 *__restrict__ tw,
                                                                 int rows, long long ld,
                                                                 float scale, int nst)
{
    const long long r0 = (long long)blockIdx.x * C::LB;
    const Geo g{r0, 1, 0, ld};
    line_fft<C, true, GENERIC, IO>(io, g, tw, scale, nst, rows - r0);
}

// Column pass: CTA b transforms columns [b*W, b*W + W), each of `rows`=2^L
// points spaced ld apart.
template <class C, bool GENERIC, class IO = StoreC64>
__global__ void __launch_bounds__(C::T, C::MINB) col_pass_kernel(const IO io,
                                                                 const float2 *__restrict__ tw,
                                                                 int cols, long long ld,
                                                                 float scale, int nst)
{
    const long long c0 = (long long)blockIdx.x * C::W;
    const Geo g{0, 1, c0, ld};
    line_fft<C, false, GENERIC, IO>(io, g, tw, scale, nst, cols - c0);
}

// ---------------------------------------------------------------------------
// Pieces of the TMA-fed kernels: the tile arrives in shared memory in natural
// order (TMA boxes or bulk copies), group 0 gathers it scrambled from there,
// and the last group is split so the caller can recycle shared memory
// between reading it and storing to global memory.

// Group 0 from a natural-order tile in shared memory, slot
// ((lb << L) | i) * W + w for element i of interleaved line w of line block
// lb; ends with the swizzled exchange layout in the same buffer.
template <class C, bool GENERIC, bool TWS = false>
__device__ __forceinline__ void group_first_smem(float2 (&a)[C::EPT], float2 *sm,
                                                 const float2 *__restrict__ tw, int nst)
{
    using Gp = Grp<C, 0>;
    static_assert(C::NG >= 2, "tile engine needs two groups");
    const int tid = threadIdx.x;
#pragma unroll
    for (int v = 0; v < Gp::V; v++) {
        const int u = tid + v * C::T;
        const int w = u & (C::W - 1);
        const int u2 = u >> C::KW;
        const int hib = u2 & ((1 << Gp::HB) - 1);
        const int lb = u2 >> Gp::HB;
#pragma unroll
        for (int r = 0; r < Gp::R; r++) {
            const int i = (brev_c(r, Gp::G) << Gp::HB) | hib;
            a[v * Gp::R + r] = sm[(((lb << C::L) | i) << C::KW) | w];
        }
    }
#pragma unroll
    for (int v = 0; v < Gp::V; v++)
        run_stages<C, 0, GENERIC, TWS>(a, v, 0, tw, nst);
    __syncthreads();   // every natural-order slot has been read
#pragma unroll
    for (int v = 0; v < Gp::V; v++) {
        const int u = tid + v * C::T;
        const int w = u & (C::W - 1);
        const int u2 = u >> C::KW;
        const int hib = u2 & ((1 << Gp::HB) - 1);
        const int lb = u2 >> Gp::HB;
        const int hi = brev_rt(hib, Gp::HB);
#pragma unroll
        for (int r = 0; r < Gp::R; r++)
            sm[sidx<C>(lb, r | (hi << Gp::G), w)] = a[v * Gp::R + r];
    }
}

// Last group, split in two so the caller can recycle shared memory in
// between: read the units into registers ...
template <class C>
__device__ __forceinline__ void group_last_read(float2 (&a)[C::EPT], const float2 *sm)
{
    using Gp = Grp<C, C::NG - 1>;
    static_assert(Gp::HB == 0, "last group");
    const int tid = threadIdx.x;
#pragma unroll
    for (int v = 0; v < Gp::V; v++) {
        const int u = tid + v * C::T;
        const int w = u & (C::W - 1);
        const int lo = (u >> C::KW) & ((1 << Gp::S0) - 1);
#pragma unroll
        for (int r = 0; r < Gp::R; r++)
            a[v * Gp::R + r] = sm[sidx<C>(0, lo | (r << Gp::S0), w)];
    }
}

// ... then run its stages and store rows lo + r 2^S0 of the tile.
__device__ __forceinline__ void st_stream(float2 *p, float2 v)
{
    asm volatile("st.global.cs.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v.x), "f"(v.y) : "memory");
}

template <class C, bool GENERIC, bool TWS = false>
__device__ __forceinline__ void group_last_finish(float2 (&a)[C::EPT], float2 *out,
                                                  const float2 *__restrict__ tw, long long ld,
                                                  float scale, int nst)
{
    using Gp = Grp<C, C::NG - 1>;
    const int tid = threadIdx.x;
#pragma unroll
    for (int v = 0; v < Gp::V; v++) {
        const int u = tid + v * C::T;
        const int lo = (u >> C::KW) & ((1 << Gp::S0) - 1);
        run_stages<C, C::NG - 1, GENERIC, TWS>(a, v, lo, tw, nst);
    }
#pragma unroll
    for (int v = 0; v < Gp::V; v++) {
        const int u = tid + v * C::T;
        const int w = u & (C::W - 1);
        const int lo = (u >> C::KW) & ((1 << Gp::S0) - 1);
        float2 *dst = out + (long long)lo * ld + w;
#pragma unroll
        for (int r = 0; r < Gp::R; r++) {
            const float2 x = a[v * Gp::R + r];
            st_stream(dst + (long long)(r << Gp::S0) * ld, make_float2(x.x * scale, x.y * scale));
        }
    }
}

// ... or run its stages and hand the tile to TMA stores, half at a time,
// through a staging buffer of E/2 values, so that the stores drain while the
// CTA computes (the per-thread global stores of group_last_finish issue one
// request per W-column row segment and stall the CTA until they leave).
// The units split in two halves by their top index bit, which is bit S0-1 of
// the row offset lo; half h is therefore rows (k << S0) | (h << (S0-1)) + q,
// q < 2^(S0-1): one box of W x 2^(S0-1) x (N >> S0) of the 3D store map
// (x = column, y = row within a 2^S0-row block, z = block) at y = h 2^(S0-1).
// The staging slot of (k, q, w) is ((k << (S0-1)) | q) * W + w.  Before overwriting the buffer
// with the second half, the issuing thread waits until the first half's
// stores have read it; the second half is still being read when this
// returns, so the caller waits (bulk_wait_read_all by thread 0, then a CTA
// barrier) before it next writes the buffer.
template <class C>
constexpr bool tma_store_ok()
{
    using Gp = Grp<C, C::NG - 1>;
    return C::NG >= 2 && C::LB == 1 && Gp::V >= 2 &&
           ((C::T * (Gp::V / 2)) >> C::KW) == (1 << (Gp::S0 - 1)) &&
           (1 << (Gp::S0 - 1)) == tma_store_rows(C::L);
}

template <class C, bool TWS = false>
__device__ __forceinline__ void group_last_finish_tma(float2 (&a)[C::EPT], float2 *stage,
                                                      const CUtensorMap *omap, int c0,
                                                      const float2 *__restrict__ tw, float scale,
                                                      int nst)
{
    using Gp = Grp<C, C::NG - 1>;
    constexpr int S0 = Gp::S0;
    constexpr int HALF = Gp::V / 2;
    constexpr int QROWS = 1 << (S0 - 1);
    static_assert(Gp::V >= 2 && C::LB == 1, "two halves of whole units, one line block");
    static_assert((1 << S0) == 256, "store blocks are the 256-row blocks of the tensor maps");
    static_assert(((C::T * HALF) >> C::KW) == QROWS, "the top unit bit is row bit S0-1");
    const int tid = threadIdx.x;
#pragma unroll
    for (int h = 0; h < 2; h++) {
#pragma unroll
        for (int v = h * HALF; v < (h + 1) * HALF; v++) {
            const int u = tid + v * C::T;
            const int lo = (u >> C::KW) & ((1 << S0) - 1);
            run_stages<C, C::NG - 1, false, TWS>(a, v, lo, tw, nst);
        }
        if (h == 1) {
            if (tid == 0)
                bulk_wait_read_all();
            __syncthreads();
        }
#pragma unroll
        for (int v = h * HALF; v < (h + 1) * HALF; v++) {
            const int u = tid + v * C::T;
            const int w = u & (C::W - 1);
            const int q = (u >> C::KW) & (QROWS - 1);
#pragma unroll
            for (int r = 0; r < Gp::R; r++) {
                const float2 x = a[v * Gp::R + r];
                stage[((r * QROWS) | q) * C::W + w] = make_float2(x.x * scale, x.y * scale);
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tma_store_3d(omap, c0, h << (S0 - 1), 0, stage);   // box W x QROWS x NBX
            bulk_commit();
        }
    }
}

// ... or split the store work between the two store paths of the SM: the
// first half of the units goes out through the staging buffer and one TMA
// store (as above), the second half straight from registers with
// per-thread stores, so neither the TMA unit nor the load/store unit carries
// all 2^L row segments of the tile and nothing waits for the staging buffer
// in the middle of the group.
template <class C, bool TWS = false>
__device__ __forceinline__ void group_last_finish_hybrid(float2 (&a)[C::EPT], float2 *stage,
                                                         const CUtensorMap *omap, int c0,
                                                         float2 *out, long long ld,
                                                         const float2 *__restrict__ tw,
                                                         float scale, int nst)
{
    using Gp = Grp<C, C::NG - 1>;
    constexpr int S0 = Gp::S0;
    constexpr int HALF = Gp::V / 2;
    constexpr int QROWS = 1 << (S0 - 1);
    static_assert(Gp::V >= 2 && C::LB == 1, "two halves of whole units, one line block");
    static_assert((1 << S0) == 256, "store blocks are the 256-row blocks of the tensor maps");
    static_assert(((C::T * HALF) >> C::KW) == QROWS, "the top unit bit is row bit S0-1");
    const int tid = threadIdx.x;
#pragma unroll
    for (int v = 0; v < HALF; v++) {
        const int u = tid + v * C::T;
        const int lo = (u >> C::KW) & ((1 << S0) - 1);
        run_stages<C, C::NG - 1, false, TWS>(a, v, lo, tw, nst);
    }
#pragma unroll
    for (int v = 0; v < HALF; v++) {
        const int u = tid + v * C::T;
        const int w = u & (C::W - 1);
        const int q = (u >> C::KW) & (QROWS - 1);
#pragma unroll
        for (int r = 0; r < Gp::R; r++) {
            const float2 x = a[v * Gp::R + r];
            stage[((r * QROWS) | q) * C::W + w] = make_float2(x.x * scale, x.y * scale);
        }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
        tma_store_3d(omap, c0, 0, 0, stage);   // box W x QROWS x NBX
        bulk_commit();
    }
#pragma unroll
    for (int v = HALF; v < Gp::V; v++) {
        const int u = tid + v * C::T;
        const int lo = (u >> C::KW) & ((1 << S0) - 1);
        run_stages<C, C::NG - 1, false, TWS>(a, v, lo, tw, nst);
    }
#pragma unroll
    for (int v = HALF; v < Gp::V; v++) {
        const int u = tid + v * C::T;
        const int w = u & (C::W - 1);
        const int lo = (u >> C::KW) & ((1 << S0) - 1);
        float2 *dst = out + (long long)lo * ld + w;
#pragma unroll
        for (int r = 0; r < Gp::R; r++) {
            const float2 x = a[v * Gp::R + r];
            st_stream(dst + (long long)(r << S0) * ld, make_float2(x.x * scale, x.y * scale));
        }
    }
}

// ... or, with one unit a thread (groups of 6 stages, 64 values a thread:
// the last group's unit holds rows lo + r 2^S0, r < R), split the unit by
// its values: rows [0, N/2) (r < R/2) go out through the staging buffer and
// one TMA store (box W x 256 x N/512 of the load map's shape, rows 0 ..
// N/2-1 of the tile), rows [N/2, N) straight from registers.
template <class C, bool TWS = false>
__device__ __forceinline__ void group_last_finish_rowhalf(float2 (&a)[C::EPT], float2 *stage,
                                                          const CUtensorMap *omap, int c0,
                                                          float2 *out, long long ld,
                                                          const float2 *__restrict__ tw,
                                                          float scale, int nst)
{
    using Gp = Grp<C, C::NG - 1>;
    constexpr int S0 = Gp::S0;
    static_assert(Gp::V == 1 && Gp::HB == 0 && C::LB == 1, "one unit a thread, the last group");
    const int tid = threadIdx.x;
    const int w = tid & (C::W - 1);
    const int lo = (tid >> C::KW) & ((1 << S0) - 1);
    run_stages<C, C::NG - 1, false, TWS>(a, 0, lo, tw, nst);
#pragma unroll
    for (int r = 0; r < Gp::R / 2; r++) {
        const float2 x = a[r];
        stage[((r << S0) | lo) * C::W + w] = make_float2(x.x * scale, x.y * scale);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
        tma_store_3d(omap, c0, 0, 0, stage);   // rows 0 .. N/2-1
        bulk_commit();
    }
    float2 *dst = out + (long long)lo * ld + w;
#pragma unroll
    for (int r = Gp::R / 2; r < Gp::R; r++) {
        const float2 x = a[r];
        st_stream(dst + (long long)(r << S0) * ld, make_float2(x.x * scale, x.y * scale));
    }
}

// ---------------------------------------------------------------------------
// Persistent row pass fed by TMA bulk copies, double buffered: while a CTA
// transforms its current block of LB rows in one shared-memory buffer, the
// next block streams into the other.  The block's rows arrive in natural
// order and group 0 gathers them scrambled from shared memory.
template <class C>
struct RowTma {
    static constexpr int SMEM_BYTES = 2 * C::E * 8;
    static constexpr uint32_t ROW_BYTES = (uint32_t)C::N * 8u;
    static constexpr uint32_t TILE_BYTES = (uint32_t)C::E * 8u;
};

template <class C>
__device__ __forceinline__ void row_issue(float2 *buf, const float2 *in, long long ld, int tile,
                                          uint64_t *bar)
{
    mbar_arrive_expect_tx(bar, RowTma<C>::TILE_BYTES);
    const float2 *src = in + (long long)tile * C::LB * ld;
    if (ld == C::N) {
        bulk_load(buf, src, RowTma<C>::TILE_BYTES, bar);   // dense rows: one copy
    } else {
        for (int lb = 0; lb < C::LB; lb++)
            bulk_load(buf + lb * C::N, src + lb * ld, RowTma<C>::ROW_BYTES, bar);
    }
}

// in must be 16-byte aligned, ld even, rows a multiple of LB.
template <class C>
__global__ void __launch_bounds__(C::T, C::MINB) row_tma_kernel(const float2 *in, float2 *out,
                                                                const float2 *__restrict__ tw,
                                                                int rows, long long ld,
                                                                float scale, int *err)
{
    extern __shared__ __align__(1024) float2 sm[];
    __shared__ __align__(8) uint64_t bar[2];
    const int ntiles = rows / C::LB;
    const int tid = threadIdx.x;
    int tile = blockIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0) {
        if (tile < ntiles)
            row_issue<C>(sm, in, ld, tile, &bar[0]);
        if (tile + (int)gridDim.x < ntiles)
            row_issue<C>(sm + C::E, in, ld, tile + gridDim.x, &bar[1]);
    }
    float2 a[C::EPT];
    for (int it = 0; tile < ntiles; tile += gridDim.x, it++) {
        const int b = it & 1;
        const uint32_t parity = (it >> 1) & 1;
        float2 *buf = sm + b * C::E;
        const int lost = mbar_wait_bounded(&bar[b], parity) ? 0 : 1;
        if (__syncthreads_or(lost)) {
            if (tid == 0)
                atomicExch(err, kDevErrTmaTimeout);
            // let transfers in flight land before the CTA leaves
            mbar_wait_bounded(&bar[b], parity);
            if (tile + (int)gridDim.x < ntiles)
                mbar_wait_bounded(&bar[b ^ 1], ((it + 1) >> 1) & 1);
            return;
        }
        group_first_smem<C, false>(a, buf, tw, C::L);
        __syncthreads();
        if constexpr (C::NG >= 3) {
            group_smem<C, 1, false>(a, buf, tw, C::L);
            __syncthreads();
        }
        if constexpr (C::NG >= 4) {
            group_smem<C, 2, false>(a, buf, tw, C::L);
            __syncthreads();
        }
        group_last<C, true, false, StoreC64>(a, buf, StoreC64{in, out},
                                             Geo{(long long)tile * C::LB, 1, 0, ld}, tw, scale,
                                             C::L, C::LB, nullptr);
        fence_proxy_async_smem();
        __syncthreads();   // this buffer is free again
        const int nn = tile + 2 * (int)gridDim.x;
        if (tid == 0 && nn < ntiles)
            row_issue<C>(buf, in, ld, nn, &bar[b]);
    }
}

// ---------------------------------------------------------------------------
// Column pass with an early prefetch.  Shared memory holds the tile region
// (the exchange buffer, one tile) and a prefetch region of half a tile.  The
// tile is seen through a 3D tensor map (x = column, y = row within a block
// of BOX = 256 rows, z = block), so each half moves with one TMA
// instruction: blocks 0..NB-1 of the NEXT tile land in the prefetch region as
// soon as group 0 has gathered the current tile into registers -- while the
// remaining groups still work -- and blocks NB.. land at the start of the
// tile region once the last group has read it.  Group 0 of a tile finds
// block k in the prefetch region (k < NB) or in the tile region (k >= NB); k
// depends only on the register index, so the split costs no extra address
// arithmetic.
template <class C>
struct TmaSplit {
    static constexpr int BOX = C::N < 256 ? C::N : 256;             // rows per block
    static constexpr int NBOX = C::N / BOX;
    static constexpr int BOX_VALS = BOX * C::W;
    static constexpr int NB = NBOX / 2;                              // early blocks
    static constexpr int TW_VALS = C::N - 1;                         // twiddle table copy
    static constexpr int TW_OFF = C::E + NB * BOX_VALS;
    static constexpr int SMEM_BYTES = (TW_OFF + TW_VALS + 1) * 8;
    static constexpr uint32_t TW_BYTES = (uint32_t)(TW_VALS + 1) * 8u;   // with padding
    static constexpr uint32_t EARLY_BYTES = (uint32_t)NB * BOX_VALS * 8u;
    static constexpr uint32_t LATE_BYTES = (uint32_t)(NBOX - NB) * BOX_VALS * 8u;
    static_assert(NB >= 1 && 2 * NB == NBOX, "two equal halves of whole blocks");
    static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
};

// Load tensor map box of the split tile: W x BOX x NB (one half).
template <class C>
__device__ __forceinline__ void split_issue_early(float2 *sm, const CUtensorMap *map, int c0,
                                                  uint64_t *bar)
{
    mbar_arrive_expect_tx(bar, TmaSplit<C>::EARLY_BYTES);
    tma_load_3d(sm + C::E, map, c0, 0, 0, bar);
}

template <class C>
__device__ __forceinline__ void split_issue_late(float2 *sm, const CUtensorMap *map, int c0,
                                                 uint64_t *bar)
{
    mbar_arrive_expect_tx(bar, TmaSplit<C>::LATE_BYTES);
    tma_load_3d(sm, map, c0, 0, TmaSplit<C>::NB, bar);
}

// Group 0 from the split tile (see above), ending with the swizzled exchange
// layout in the tile region.  `before_barrier` runs just before the barrier
// that follows the gather; `after_reads` runs once every thread has gathered
// its values (the prefetch region is then free).
template <class C, class F0, class F>
__device__ __forceinline__ void group_first_split(float2 (&a)[C::EPT], float2 *sm,
                                                  const float2 *__restrict__ tw, F0 before_barrier,
                                                  F after_reads)
{
    using Gp = Grp<C, 0>;
    using S = TmaSplit<C>;
    static_assert(C::NG >= 2 && C::LB == 1, "tile engine needs two groups, one line block");
    static_assert((1 << Gp::HB) <= S::BOX, "box index must depend on the register only");
    const float2 *pref = sm + C::E;
    const int tid = threadIdx.x;
#pragma unroll
    for (int v = 0; v < Gp::V; v++) {
        const int u = tid + v * C::T;
        const int w = u & (C::W - 1);
        const int hib = (u >> C::KW) & ((1 << Gp::HB) - 1);
#pragma unroll
        for (int r = 0; r < Gp::R; r++) {
            const int top = brev_c(r, Gp::G) << Gp::HB;     // compile-time
            const int k = top / S::BOX;
            const int in_box = ((top % S::BOX) | hib) * C::W + w;
            const float2 *bx = k < S::NB ? pref + k * S::BOX_VALS : sm + (k - S::NB) * S::BOX_VALS;
            a[v * Gp::R + r] = bx[in_box];
        }
    }
#pragma unroll
    for (int v = 0; v < Gp::V; v++)
        run_stages<C, 0, false, true>(a, v, 0, tw, C::L);
    fence_proxy_async_smem();
    before_barrier();  // what it waits for holds for every thread after the barrier
    __syncthreads();   // every slot of both regions has been read
    after_reads();
#pragma unroll
    for (int v = 0; v < Gp::V; v++) {
        const int u = tid + v * C::T;
        const int w = u & (C::W - 1);
        const int hib = (u >> C::KW) & ((1 << Gp::HB) - 1);
        const int hi = brev_rt(hib, Gp::HB);
#pragma unroll
        for (int r = 0; r < Gp::R; r++)
            sm[sidx<C>(0, r | (hi << Gp::G), w)] = a[v * Gp::R + r];
    }
}

// Where the persistent TMA column kernel finds tile t: the tensor maps and
// first column of its TMA boxes (load map over the input, store map over the
// output), the output pointer of its first column, the image row pitch and
// the output scale.
struct TilesOneImage {
    const CUtensorMap *map;
    const CUtensorMap *omap_;
    float2 *out;
    long long ld;
    float scale;
    int W;
    __device__ const CUtensorMap *tmap(int) const { return map; }
    __device__ const CUtensorMap *omap(int) const { return omap_; }
    __device__ int col(int t) const { return t * W; }
    __device__ float2 *dst(int t) const { return out + (long long)t * W; }
    __device__ long long pitch(int) const { return ld; }
    __device__ float scl(int) const { return scale; }
};

// Persistent column pass: CTA b takes tiles b, b + grid, ...  Shared memory:
// the tile region (E values; the next tile's late boxes land in its lower
// half), the prefetch region (the next tile's early boxes), the rotation
// factors.  With TS (TMA stores) the upper half of the tile region is also
// the staging buffer of the finished tile, drained while the next tile's
// group 0 runs; otherwise each thread stores its results directly.
// withhold (self-test): CTA 0 does not issue its first tile's late boxes,
// so its first wait runs out and the kernel takes its timeout path.
// HYB (with TS): the last group stores half the tile through TMA and half
// with per-thread stores (group_last_finish_hybrid).
template <class C, bool TS, class Src, bool HYB = false>
__device__ __forceinline__ void col_tma2_body(const Src &src, int ntiles,
                                              const float2 *__restrict__ tw, int *err,
                                              int withhold = 0)
{
    static_assert(!TS || TmaSplit<C>::LATE_BYTES <= (uint32_t)C::E * 4u,
                  "late boxes must leave the staging half free");
    extern __shared__ __align__(1024) float2 sm[];
    __shared__ __align__(8) uint64_t bar_early, bar_late;
    const int tid = threadIdx.x;
    int tile = blockIdx.x;
    if (tid == 0) {
        mbar_init(&bar_early, 1);
        mbar_init(&bar_late, 1);
        fence_mbar_init();
    }
    __syncthreads();
    // the rotation factors (N entries, the last one padding) stay in shared
    // memory for the CTA's whole life; they arrive with the first tile
    float2 *stw = sm + TmaSplit<C>::TW_OFF;
    if (tid == 0 && tile < ntiles) {
        mbar_expect_tx(&bar_early, TmaSplit<C>::TW_BYTES);
        bulk_load(stw, tw, TmaSplit<C>::TW_BYTES, &bar_early);
        split_issue_early<C>(sm, src.tmap(tile), src.col(tile), &bar_early);
        if (!(withhold && blockIdx.x == 0))
            split_issue_late<C>(sm, src.tmap(tile), src.col(tile), &bar_late);
    }
    uint32_t parity = 0;
    float2 a[C::EPT];
    for (; tile < ntiles; tile += gridDim.x) {
        const int next = tile + gridDim.x;
        const bool ok = mbar_wait_bounded(&bar_early, parity) && mbar_wait_bounded(&bar_late, parity);
        if (__syncthreads_or(ok ? 0 : 1)) {
            if (tid == 0) {
                atomicExch(err, kDevErrTmaTimeout);
                if constexpr (TS)
                    bulk_wait_all();
            }
            // let late transfers land before the CTA leaves
            mbar_wait_bounded(&bar_early, parity);
            mbar_wait_bounded(&bar_late, parity);
            return;
        }
        parity ^= 1;
        group_first_split<C>(
            a, sm, stw,
            [&] {
                if constexpr (TS) {
                    if (tid == 0)
                        bulk_wait_read_all();   // the previous tile's staging half is free
                }
            },
            [&] {
                if (tid == 0 && next < ntiles)
                    split_issue_early<C>(sm, src.tmap(next), src.col(next), &bar_early);
            });
        __syncthreads();
        if constexpr (C::NG >= 3) {
            group_smem<C, 1, false, false, true>(a, sm, stw, C::L);
            __syncthreads();
        }
        if constexpr (C::NG >= 4) {
            group_smem<C, 2, false, false, true>(a, sm, stw, C::L);
            __syncthreads();
        }
        group_last_read<C>(a, sm);
        fence_proxy_async_smem();
        __syncthreads();   // the tile region is free
        if (tid == 0 && next < ntiles)
            split_issue_late<C>(sm, src.tmap(next), src.col(next), &bar_late);
        if constexpr (TS && HYB && Grp<C, C::NG - 1>::V == 1)
            group_last_finish_rowhalf<C, true>(a, sm + C::E / 2, src.omap(tile), src.col(tile),
                                               src.dst(tile), src.pitch(tile), stw, src.scl(tile),
                                               C::L);
        else if constexpr (TS && HYB)
            group_last_finish_hybrid<C, true>(a, sm + C::E / 2, src.omap(tile), src.col(tile),
                                              src.dst(tile), src.pitch(tile), stw, src.scl(tile),
                                              C::L);
        else if constexpr (TS)
            group_last_finish_tma<C, true>(a, sm + C::E / 2, src.omap(tile), src.col(tile), stw,
                                           src.scl(tile), C::L);
        else
            group_last_finish<C, false, true>(a, src.dst(tile), stw, src.pitch(tile),
                                              src.scl(tile), C::L);
    }
    if constexpr (TS) {
        if (tid == 0)
            bulk_wait_all();   // shared memory stays valid until the stores are done
    }
}

template <class C, bool TS, bool HYB = false>
__global__ void __launch_bounds__(C::T, 1) col_tma2_kernel(const __grid_constant__ CUtensorMap map,
                                                           const __grid_constant__ CUtensorMap omap,
                                                           float2 *out,
                                                           const float2 *__restrict__ tw,
                                                           int cols, long long ld, float scale,
                                                           int *err, int withhold)
{
    const TilesOneImage src{&map, &omap, out, ld, scale, C::W};
    col_tma2_body<C, TS, TilesOneImage, HYB>(src, cols / C::W, tw, err, withhold);
}

// The same kernel over the column tiles of many images of one column length
// (a batch group): tile g belongs to the image whose first_tile range holds
// it; each image brings its own tensor maps, output, pitch and scale.
struct TilesBatch {
    const BatchTmaTable *t;
    int W;
    __device__ int job(int g) const
    {
        int lo = 0, hi = t->n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (t->first_tile[mid] <= g)
                lo = mid;
            else
                hi = mid - 1;
        }
        return lo;
    }
    __device__ const CUtensorMap *tmap(int g) const { return &t->map[job(g)]; }
    __device__ const CUtensorMap *omap(int g) const { return &t->omap[job(g)]; }
    __device__ int col(int g) const { return (g - t->first_tile[job(g)]) * W; }
    __device__ float2 *dst(int g) const
    {
        const int j = job(g);
        return t->out[j] + (long long)(g - t->first_tile[j]) * W;
    }
    __device__ long long pitch(int g) const { return t->ld[job(g)]; }
    __device__ float scl(int g) const { return t->scale[job(g)]; }
};

template <class C, bool TS, bool HYB = false>
__global__ void __launch_bounds__(C::T, 1) col_tma2_batch_kernel(const __grid_constant__ BatchTmaTable t,
                                                                 const float2 *__restrict__ tw,
                                                                 int *err)
{
    const TilesBatch src{&t, C::W};
    col_tma2_body<C, TS, TilesBatch, HYB>(src, t.first_tile[t.n], tw, err);
}

// ---------------------------------------------------------------------------
// Column pass split over a thread-block cluster of CS = 2^c CTAs.
//
// A tile of W adjacent columns of 2^L rows is too large for one CTA when the
// tile is wide enough for full 64-128 byte row segments.  The DIT structure
// splits it without any extra pass over memory: after the scramble, the
// positions p in [b 2^(L-c), (b+1) 2^(L-c)) hold exactly the rows
// m = CS m' + rev_c(b), in the order p = b 2^(L-c) + rev_{L-c}(m').  So CTA
// b of the cluster loads every CS-th row (starting at rev_c(b)), runs stages
// 1 .. L-c on them locally (the ordinary engine with a CS-times row pitch)
// and leaves its 2^(L-c)-point results in shared memory in natural order.
// Stages L-c+1 .. L pair positions that differ only in their top c bits,
// i.e. values held by different CTAs: after a cluster barrier each CTA
// gathers, through distributed shared memory, the CS values of its share of
// the output rows (lo in [b 2^(L-2c), (b+1) 2^(L-2c))), runs those last c
// stages in registers and stores rows lo + r 2^(L-c), r < CS.
template <int L_, int KW_, int C_>
struct ClusterColCfg {
    static constexpr int L = L_, KW = KW_, c = C_;
    static constexpr int CS = 1 << c;
    using Local = LineCfg<L - c, KW, 0>;
    using Cross = GrpSG<L, L - c, c>;
    static constexpr int T = Local::T;
    static constexpr int W = Local::W;
    static constexpr int NL = Local::N;          // rows held by one CTA
    static constexpr int SMEM_BYTES = Local::E * 8;
    static_assert(c >= 1 && c <= 4, "cluster of 2 to 16 CTAs");
    static_assert(Local::NG >= 2, "local line must span at least two groups");
};

// Shared memory of a cluster CTA: its rows of the tile, then (half2
// storage) one int per column for the cluster-wide exponent reduction.
template <class CC, class IO>
struct ClusterSmem {
    static constexpr int BYTES = CC::SMEM_BYTES + (IO::H16 ? CC::W * 4 : 0);
};

template <class CC, bool GENERIC, class IO = StoreC64>
__global__ void __launch_bounds__(CC::T) col_cluster_kernel(const IO io,
                                                            const float2 *__restrict__ tw,
                                                            int cols, long long ld,
                                                            float scale, int nst)
{
    namespace cg = cooperative_groups;
    using LC = typename CC::Local;
    using X = typename CC::Cross;
    extern __shared__ float2 sm[];
    int *sred = reinterpret_cast<int *>(sm + LC::E);
    cg::cluster_group cluster = cg::this_cluster();
    const int b = (int)cluster.block_rank();
    const long long c0 = (long long)(blockIdx.x / CC::CS) * CC::W;
    const long long nvalid = cols - c0;
    const int tid = threadIdx.x;
    float2 a[CC::Local::EPT];
    if constexpr (IO::H16) {
        for (int i = tid; i < CC::W; i += CC::T)
            sred[i] = 0;
    }

    // stages 1 .. L-c on this CTA's rows
    group_first<LC, false, GENERIC, IO>(a, sm, io,
                                        Geo{(long long)brev_rt(b, CC::c), CC::CS, c0, ld}, tw,
                                        1.0f, nst, nvalid, nullptr);
    __syncthreads();
    if constexpr (LC::NG >= 3) {
        group_smem<LC, 1, GENERIC>(a, sm, tw, nst);
        __syncthreads();
    }
    if constexpr (LC::NG >= 4) {
        group_smem<LC, 2, GENERIC>(a, sm, tw, nst);
        __syncthreads();
    }
    group_smem<LC, LC::NG - 1, GENERIC, true>(a, sm, tw, nst);
    cluster.sync();

    // stages L-c+1 .. L across the cluster
#pragma unroll
    for (int v = 0; v < X::V; v++) {
        const int u = tid + v * CC::T;
        const int w = u & (CC::W - 1);
        const int lo = b * (CC::NL / CC::CS) + (u >> CC::KW);
#pragma unroll
        for (int r = 0; r < CC::CS; r++) {
            const float2 *peer = cluster.map_shared_rank(sm, r);
            a[v * X::R + r] = peer[lo * CC::W + w];
        }
    }
    if constexpr (!IO::H16)
        cluster.sync();   // no CTA leaves while a peer may still read its smem
#pragma unroll
    for (int v = 0; v < X::V; v++) {
        const int u = tid + v * CC::T;
        const int lo = b * (CC::NL / CC::CS) + (u >> CC::KW);
        run_stages_g<X, false, GENERIC>(a, v, lo, tw, nst);
    }
    if constexpr (IO::H16) {
        // a column's exponent depends on all CS CTAs' rows of it: each CTA
        // max-reduces its part into sred, then reads every peer's value
#pragma unroll
        for (int v = 0; v < X::V; v++) {
            const int u = tid + v * CC::T;
            const int w = u & (CC::W - 1);
            float m = 0.f;
#pragma unroll
            for (int r = 0; r < CC::CS; r++)
                m = fmaxf(m, fmaxf(fabsf(a[v * X::R + r].x), fabsf(a[v * X::R + r].y)));
            if (!GENERIC || w < nvalid)
                atomicMax(sred + w, __float_as_int(m * scale));
        }
        cluster.sync();   // gathers done, partial maxima final
    }
#pragma unroll
    for (int v = 0; v < X::V; v++) {
        const int u = tid + v * CC::T;
        const int w = u & (CC::W - 1);
        const int lo = b * (CC::NL / CC::CS) + (u >> CC::KW);
        if (GENERIC && w >= nvalid)
            continue;
        float f = scale;
        int e = 0;
        if constexpr (IO::H16) {
            int mb = 0;
#pragma unroll
            for (int r = 0; r < CC::CS; r++) {
                const int *peer = cluster.map_shared_rank(sred, r);
                mb = max(mb, peer[w]);
            }
            e = line_exponent(__int_as_float(mb));
            f = scale * pow2f(-e);
        }
#pragma unroll
        for (int r = 0; r < CC::CS; r++) {
            const float2 x = a[v * X::R + r];
            const long long k = ((long long)lo + (long long)r * CC::NL) * ld + c0 + w;
            if constexpr (IO::H16) {
                io.out[k] = __floats2half2_rn(x.x * f, x.y * f);
                if (lo == 0 && r == 0)
                    io.out_exp[c0 + w] = e;
            } else {
                io.out[k] = make_float2(x.x * f, x.y * f);
            }
        }
    }
    if constexpr (IO::H16)
        cluster.sync();   // peers are done reading this CTA's maxima
}

// Host-side launch of a cluster column pass (cluster dimension attribute,
// shared-memory opt-in).  Defined here so both storage formats share it.
template <class CC, class IO>
inline cudaError_t launch_cluster_kernel(const IO &io, const float2 *tw, int cols, long long ld,
                                         float scale, int nst, cudaStream_t s)
{
    auto k = col_cluster_kernel<CC, false, IO>;
    constexpr int SMEM = ClusterSmem<CC, IO>::BYTES;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e == cudaSuccess && CC::CS > 8)
        e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess)
        return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CC::CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(cols / CC::W * CC::CS));
    cfg.blockDim = dim3(CC::T);
    cfg.dynamicSmemBytes = SMEM;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, io, tw, cols, ld, scale, nst);
}

}  // namespace fft2d
