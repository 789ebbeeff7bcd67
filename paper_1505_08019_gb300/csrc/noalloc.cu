// noalloc.cu -- the 2D transform for callers that cannot allocate device memory.
//
// fft2d_exec needs a plan, and a plan allocates device memory (its rotation
// factor tables and its status word).  Some callers cannot allocate: a
// plug-in inside a host application that owns every byte of the device
// through its own memory manager (a cudaMalloc behind its back breaks its
// accounting, or fails because it has reserved the whole device), code in a
// process whose caching allocator already holds the free memory, and
// latency-bound paths where cudaMalloc's implicit device synchronisation is
// not allowed.  fft2d_exec_noalloc serves them: the same row and column pass
// kernels run with their tables and status word taken from one file-scope
// device array that exists from the moment the library is loaded on a device
// until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "fft2d.h"
#include "passes.h"

namespace {

constexpr int kMaxDevices = 64;
// entries per axis table: 2^L - 1 rotation factors plus one padding entry
// (the persistent column pass copies 2^L entries with one 16-byte-multiple
// bulk copy, so every table starts on a 16-byte boundary)
constexpr int kTableVals = FFT2D_NOALLOC_MAX_SIDE;

// The shared scratch: both axes' rotation factors and the status word the
// column kernel writes when a bounded wait gives up.  About 64 KB.
struct NoAllocScratch {
    float2 tw_rows[kTableVals];
    float2 tw_cols[kTableVals];
    int status;
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of g_noalloc_scratch, looked up once per device (in host
// code the symbol name is only a stand-in, not a device address).
NoAllocScratch *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_setup_mu;

// Per-stage table of an axis of 2^L points (stage s at offset 2^(s-1)-1,
// entry j = W_{2^s}^j), computed in FP64 with sincospi -- exact at the
// quarter turns -- and rounded to FP32.  Also clears the status word.
__global__ void noalloc_fill_tables(NoAllocScratch *s, int Lr, int Lc, int dir)
{
    const int n_rows_tab = (1 << Lc) - 1;
    const int n_cols_tab = (1 << Lr) - 1;
    const int total = n_rows_tab + n_cols_tab;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += gridDim.x * blockDim.x) {
        const bool row_tab = idx < n_rows_tab;
        const int e = row_tab ? idx : idx - n_rows_tab;
        const int sm1 = 31 - __clz(e + 1);            // s - 1
        const int j = e + 1 - (1 << sm1);
        double sn, cs;
        sincospi((double)j / (double)(1 << sm1), &sn, &cs);   // angle 2*pi*j/2^s
        const float2 w = make_float2((float)cs, (float)(dir == FFT2D_FORWARD ? -sn : sn));
        if (row_tab)
            s->tw_rows[e] = w;
        else
            s->tw_cols[e] = w;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        s->status = 0;
}

int log2_pow2(int n)
{
    int L = 0;
    while ((1 << L) < n)
        L++;
    return L;
}

}  // namespace

extern "C" {

fft2d_status fft2d_exec_noalloc(int rows, int cols, int dir, const void *in, void *out,
                                void *stream)
{
    if (!in || !out || (dir != FFT2D_FORWARD && dir != FFT2D_INVERSE))
        return FFT2D_ERR_ARG;
    if (rows < 1 || cols < 1 || (rows & (rows - 1)) || (cols & (cols - 1)))
        return FFT2D_ERR_NOT_POW2;
    if (rows > FFT2D_NOALLOC_MAX_SIDE || cols > FFT2D_NOALLOC_MAX_SIDE)
        return FFT2D_ERR_TOO_LARGE;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return FFT2D_ERR_CUDA;
    NoAllocScratch *scratch;
    {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_scratch_ptr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return FFT2D_ERR_CUDA;
            g_scratch_ptr[dev] = static_cast<NoAllocScratch *>(p);
        }
        scratch = g_scratch_ptr[dev];
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int Lr = log2_pow2(rows), Lc = log2_pow2(cols);
    noalloc_fill_tables<<<16, 256, 0, st>>>(scratch, Lr, Lc, dir);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return FFT2D_ERR_CUDA;

    fft2d::PassArgs a;
    a.rows = rows;
    a.cols = cols;
    a.ld = cols;
    a.err = &scratch->status;
    a.partial = false;
    const float inv_scale = (float)(1.0 / ((double)rows * (double)cols));
    // row pass: in -> out (a length-1 row is the identity)
    if (Lc == 0) {
        if (in != out) {
            e = cudaMemcpyAsync(out, in, (size_t)rows * cols * sizeof(float2),
                                cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess)
                return FFT2D_ERR_CUDA;
        }
    } else {
        a.in = static_cast<const float2 *>(in);
        a.out = static_cast<float2 *>(out);
        a.tw = scratch->tw_rows;
        a.nst = Lc;
        a.scale = (Lr == 0 && dir == FFT2D_INVERSE) ? inv_scale : 1.0f;
        e = fft2d::launch_row_pass(Lc, a, st);
        if (e != cudaSuccess)
            return FFT2D_ERR_CUDA;
    }
    // column pass: in place on out
    if (Lr > 0) {
        a.in = static_cast<const float2 *>(out);
        a.out = static_cast<float2 *>(out);
        a.tw = scratch->tw_cols;
        a.nst = Lr;
        a.scale = dir == FFT2D_INVERSE ? inv_scale : 1.0f;
        e = fft2d::launch_col_pass(Lr, a, st);
        if (e != cudaSuccess)
            return FFT2D_ERR_CUDA;
    }
    return FFT2D_OK;
}

}  // extern "C"
