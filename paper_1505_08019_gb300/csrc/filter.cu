// filter.cu -- Gaussian low-pass multiply of an unshifted 2D spectrum, the
// "filter" step of the FFT -> filter -> inverse FFT image operation (the
// paper's motivating use, image filtering, Section 1).
//
// H[k][l] = exp(-d_k^2 / (2 s_r^2)) * exp(-d_l^2 / (2 s_c^2)),
// d_k = min(k, rows - k), d_l = min(l, cols - l), with s_r, s_c the caller's
// widths in frequency bins (side/8 in the serving workload).  H is real and
// <= 1, so for half2 storage the per-column exponents stay valid.
#include <cuda_fp16.h>

#include "passes.h"

namespace fft2d {

namespace {

__device__ __forceinline__ float gauss_factor(int k, int n, float inv2s2)
{
    const int d = k < n - k ? k : n - k;
    return expf(-(float)d * (float)d * inv2s2);
}

template <class T>
__global__ void lowpass_kernel(T *x, int rows, int cols, float inv2sr2, float inv2sc2)
{
    const int row = blockIdx.y;
    const float hr = gauss_factor(row, rows, inv2sr2);
    T *line = x + (long long)row * cols;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
        const float h = hr * gauss_factor(c, cols, inv2sc2);
        if constexpr (sizeof(T) == 8) {
            const float2 v = reinterpret_cast<float2 *>(line)[c];
            reinterpret_cast<float2 *>(line)[c] = make_float2(v.x * h, v.y * h);
        } else {
            const float2 v = __half22float2(reinterpret_cast<__half2 *>(line)[c]);
            reinterpret_cast<__half2 *>(line)[c] = __floats2half2_rn(v.x * h, v.y * h);
        }
    }
}

}  // namespace

cudaError_t launch_lowpass(bool half2, void *x, int rows, int cols, float sigma_r, float sigma_c,
                           cudaStream_t s)
{
    const float ir = 1.0f / (2.0f * sigma_r * sigma_r);
    const float ic = 1.0f / (2.0f * sigma_c * sigma_c);
    const int threads = 256;
    int bx = (cols + threads - 1) / threads;
    if (bx > 16)
        bx = 16;
    dim3 grid((unsigned)bx, (unsigned)rows);
    if (half2)
        lowpass_kernel<__half2><<<grid, threads, 0, s>>>(static_cast<__half2 *>(x), rows, cols, ir, ic);
    else
        lowpass_kernel<float2><<<grid, threads, 0, s>>>(static_cast<float2 *>(x), rows, cols, ir, ic);
    return cudaGetLastError();
}

}  // namespace fft2d
