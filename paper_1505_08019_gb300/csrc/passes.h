// passes.h -- host-side entry points of the row and column pass kernels.
#pragma once

#include <cuda_runtime.h>

namespace fft2d {

// Arguments common to both passes (complex64 storage, FP32 arithmetic).
struct PassArgs {
    const float2 *in;    // device, first pixel of the image
    float2 *out;         // device, may equal in
    const float2 *tw;    // device, per-stage rotation factors of this axis
    int rows, cols;      // image shape
    long long ld;        // row pitch in pixels (== cols for a dense image)
    float scale;         // multiplies every stored value (1 or 1/(rows*cols))
    int nst;             // stages to run on this axis (partial debug view)
    bool partial;        // nst < log2(axis length)
    int *err;            // device status word (bounded-wait timeouts)
    int variant = 0;     // kernel variant (0 = default for this size)
};

// Lines per CTA of the row pass and interleaved columns per CTA of the
// column pass for an axis of 2^L points.
int row_lines_per_cta(int L);
int col_width(int L);

cudaError_t launch_row_pass(int L, const PassArgs &a, cudaStream_t s);

// Streaming multiprocessors of the current device (cached per device).
int device_sm_count();
int device_current();
cudaError_t launch_selftest_timeout(int *err, cudaStream_t s);
cudaError_t launch_col_pass(int L, const PassArgs &a, cudaStream_t s);

}  // namespace fft2d
