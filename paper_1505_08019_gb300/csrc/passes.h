// passes.h -- host-side entry points of the row and column pass kernels.
#pragma once

#include <atomic>

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace fft2d {

// An NVTX range for the host-side span of one library call or pass launch
// (shown by Nsight Systems / Nsight Compute when attached; a no-op stub
// otherwise).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// One int per device (index from device_current(), below 64), computed on
// first use by the launching thread; threads that race on the first use
// compute and store the same value.
struct DeviceCache {
    std::atomic<int> v[64];
    int get(int d) const { return v[d].load(std::memory_order_relaxed); }
    void set(int d, int x) { v[d].store(x, std::memory_order_relaxed); }
};

// Arguments common to both passes (complex64 storage, FP32 arithmetic).
struct PassArgs {
    const float2 *in;    // device, first pixel of the image
    float2 *out;         // device, may equal in
    const float2 *tw;    // device, per-stage rotation factors of this axis: 2^L - 1
                         // entries and one padding entry, 16-byte aligned
    int rows, cols;      // image shape
    long long ld;        // row pitch in pixels (== cols for a dense image)
    float scale;         // multiplies every stored value (1 or 1/(rows*cols))
    int nst;             // stages to run on this axis (partial debug view)
    bool partial;        // nst < log2(axis length)
    int *err;            // device status word (bounded-wait timeouts)
    int variant = -1;    // kernel variant index (-1: the default for this size)
    int withhold = 0;    // self-test: CTA 0 does not issue its first tile's second TMA load
};

// One way to run a pass for one line length (see kernels_row.cu and
// kernels_col.cu for the lists).  `usable` says whether it can serve these
// arguments (alignment, whole tiles, ...); the plain variant 0 serves all.
struct Variant {
    const char *name;
    int shape;     // rows per CTA (row pass) or adjacent columns per tile (column pass)
    int ept;       // values per thread
    bool (*usable)(const PassArgs &);
    cudaError_t (*launch)(const PassArgs &, cudaStream_t);
    bool tma_fed = false;   // persistent TMA-fed kernel: honours PassArgs::withhold
};
const Variant *row_variants(int L, int *n);
const Variant *col_variants(int L, int *n);
int row_default_variant(int L);
int col_default_variant(int L);

// Per-size CTA shapes of the plain kernels: log2 of the rows per CTA of the
// row pass (256 threads per CTA up to 4096-point rows) and log2 of the
// adjacent columns per CTA of the column pass (2^14 values per CTA from
// 1024-point columns up, 16 to 64 columns below).
constexpr int row_kb(int L) { return L <= 12 ? 12 - L : 0; }
constexpr int col_kw(int L)
{
    return L >= 10 ? 14 - L : (13 - L < 4 ? 4 : (13 - L > 6 ? 6 : 13 - L));
}

// Values per thread of the TMA column kernel: 32 for tiles of 2^14 values
// (512 threads of up to 128 registers), 16 below.
constexpr int col_tma_ept(int L) { return L >= 10 ? 32 : 16; }

// Rows of one TMA store box of the persistent column pass: half of the 2^8
// rows that one unit of its last stage group spans (lines of 2^9..2^12).
constexpr int tma_store_rows(int) { return 128; }

// Lines per CTA of the row pass and interleaved columns per CTA of the
// column pass for an axis of 2^L points.
int row_lines_per_cta(int L);
int col_width(int L);

// Half2 storage with one power-of-two exponent per line (kernels_h16.cu).
struct H16PassArgs {
    const __half2 *in;
    __half2 *out;
    const float2 *tw;
    int rows, cols;
    long long ld;
    float scale;
    int nst;
    const int *in_exp;   // input exponents, one per row (in_axis 0) or column (1)
    int in_axis;
    int *out_exp;        // output exponents: per row (row pass) or column (column pass)
    int *err = nullptr;  // device status word (bounded waits of the TMA-fed column pass)
};
cudaError_t launch_pass_h16(bool row, int L, const H16PassArgs &a, cudaStream_t s);
cudaError_t launch_h16_pack(const float2 *in, __half2 *out, int *exp_rows, int rows, int cols,
                            cudaStream_t s);
cudaError_t launch_h16_unpack(const __half2 *in, const int *exps, int axis, float2 *out,
                              int rows, int cols, cudaStream_t s);

// Gaussian low-pass multiply of an unshifted spectrum (filter.cu).
cudaError_t launch_lowpass(bool half2, void *x, int rows, int cols, float sigma_r, float sigma_c,
                           cudaStream_t s);

// Grouped launches over many images (batch.cu): one job per image, passed
// by value as a kernel parameter.
constexpr int kBatchMaxJobs = 128;
struct BatchJob {
    const float2 *in;
    float2 *out;
    const float2 *tw;
    long long ld;
    int lines;       // rows (row pass) or columns (column pass) of the image
    int first_cta;   // filled by launch_batch_pass
    float scale;
};
struct BatchTable {
    int n;
    BatchJob job[kBatchMaxJobs];
};
// Job table of the grouped TMA column kernel: a load and a store tensor map
// per image (a kernel parameter, well inside the 32 KB parameter limit).
constexpr int kBatchTmaMaxJobs = 64;
struct BatchTmaTable {   // 128-byte aligned through CUtensorMap
    CUtensorMap map[kBatchTmaMaxJobs];
    CUtensorMap omap[kBatchTmaMaxJobs];
    float2 *out[kBatchTmaMaxJobs];
    long long ld[kBatchTmaMaxJobs];
    float scale[kBatchTmaMaxJobs];
    int first_tile[kBatchTmaMaxJobs + 1];
    int n;
};

// What the serving loop needs to see of a plan (fft2d_api.cpp): shape,
// direction, the device rotation-factor tables of both axes and the status
// word.  False for a null plan.
struct PlanView {
    int rows, cols, Lr, Lc, dtype, dir;
    const float2 *tw_rows, *tw_cols;
    int *err;
};
bool plan_view(const void *plan, PlanView *v);

// Grouped launches of half2 images (batch.cu): the same per-CTA work as the
// single-image half2 passes, one job per image.
constexpr int kBatchH16MaxJobs = 64;
struct BatchJobH16 {
    const __half2 *in;
    __half2 *out;
    const float2 *tw;
    const int *in_exp;   // exponents of the input lines (the group's input axis)
    int *out_exp;        // exponents of this pass's output lines (per row / column)
    long long ld;
    int lines;           // rows (row pass) or columns (column pass) of the image
    int first_cta;       // filled by launch_batch_pass_h16
    float scale;
};
struct BatchTableH16 {
    int n;
    BatchJobH16 job[kBatchH16MaxJobs];
};
// One launch for every job of `t` whose axis has 2^L points; in_axis: the
// jobs' input exponent axis (0 one per row, 1 one per column).
cudaError_t launch_batch_pass_h16(bool row, int L, BatchTableH16 &t, int in_axis, cudaStream_t s);

// Grouped-launch variants: rows 0 plain, 1 plain32; columns 0 plain,
// 1 narrow (half-width tiles), 2 tma (persistent, TMA-fed, TMA stores;
// 512..4096 rows), 3 tmast (the same with per-thread stores), 4 tmah (half
// of each tile through TMA stores, half through per-thread stores).
constexpr int kBatchRowVariants = 2;
constexpr int kBatchColVariants = 5;
int batch_default_variant(bool row, int L);
const char *batch_variant_name(bool row, int variant);

// One launch for every job of `t` whose axis has 2^L points (all jobs of one
// direction: they share the rotation-factor table of job 0).  err: status
// word for bounded waits.  A variant that cannot serve the jobs falls back
// to the plain grouped kernel.
cudaError_t launch_batch_pass(bool row, int L, BatchTable &t, int variant, int *err,
                              cudaStream_t s);

// 3D tensor map over a column-pass image of 8-byte elements (rows a
// multiple of 256): x = column, y = row within a block of 256 rows, z =
// block; box W x box_y x box_z.
bool encode_col_map(CUtensorMap *map, const float2 *base, int rows, int cols, long long ld, int W,
                    int box_y, int box_z);

// 2D DCT of a real FP32 image (dct.cu): one pass along the rows (row =
// true: lines of cols = 2^L points, in -> out) or along the columns (lines
// of rows = 2^L points), DCT-II forward or its inverse (DCT-III, unscaled:
// the caller passes the 1/N factors in `scale`).  Two real lines share one
// complex line of the radix-2 engine.  tw: this axis's per-stage table of
// the direction (conjugated for the inverse); post: the axis's
// (cos, sin)(pi k / (2N)), k = 0..N/2.  rows, cols >= 2; in may equal out.
// err: the plan's device status word (bounded waits of the TMA-fed kernels).
// withhold (self-test, column pass only): run the TMA-fed column kernel with
// CTA 0's first second-half load never issued; cudaErrorNotSupported when
// this pass does not run on such a kernel.
cudaError_t launch_dct_pass(bool row, bool inverse, int L, const float *in, float *out, int rows,
                            int cols, const float2 *tw, const float2 *post, float scale, int *err,
                            cudaStream_t s, int withhold = 0);

// 3D tensor map over 8-byte elements: x = element within a row (xdim), y
// (ydim rows, ystride elements apart), z (zdim blocks, zstride elements
// apart); box box_x x box_y x box_z.  False if the driver's encoder is
// missing or rejects the description (base 16-byte aligned, strides
// multiples of 16 bytes).
bool encode_map_xyz(CUtensorMap *map, const void *base, long long xdim, int ydim, int zdim,
                    long long ystride, long long zstride, int box_x, int box_y, int box_z);
bool tensor_maps_available();

cudaError_t launch_row_pass(int L, const PassArgs &a, cudaStream_t s);

// Stream-ordered device scratch from the library's own memory pool of the
// current device (kernels_col.cu): taken on `s` (cudaMallocFromPoolAsync),
// given back by the caller with cudaFreeAsync on `s` after its launches.
// The pool keeps what it has allocated, so after the first calls no driver
// allocation happens; launches on different streams never share a block.
cudaError_t scratch_take(void **p, size_t bytes, cudaStream_t s);

// Streaming multiprocessors of the current device (cached per device).
int device_sm_count();

int device_current();
cudaError_t launch_selftest_timeout(int *err, cudaStream_t s);
cudaError_t launch_col_pass(int L, const PassArgs &a, cudaStream_t s);
// Whether the column-pass kernel that launch_col_pass would run for these
// arguments is a TMA-fed one (the only kernels with the withhold self-test).
bool col_pass_is_tma_fed(int L, const PassArgs &a);

}  // namespace fft2d
