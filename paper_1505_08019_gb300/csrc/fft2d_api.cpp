// fft2d_api.cpp -- the C ABI declared in include/fft2d.h: plans, rotation
// factor tables, and the two-launch execution of the 2D transform.
#include "fft2d.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>
#include <tuple>
#include <vector>

#include "passes.h"

struct fft2d_plan_s {
    int rows, cols, Lr, Lc, dtype, dir, device;
    // Per-stage rotation factors of each axis (stage s: W_{2^s}^j, j < 2^(s-1),
    // at offset 2^(s-1)-1), already conjugated for the inverse direction.
    float2 *tw_rows;   // table for the row pass: lines of cols points
    float2 *tw_cols;   // table for the column pass: lines of rows points
    void *staging;     // device image buffer for fft2d_exec_host (lazy)
    int *dev_err;      // device status word set by bounded waits in the kernels
    int row_variant;   // kernel variant of each pass (-1: per-size default)
    int col_variant;
    int *exp_rows;     // half2 plans: exponents of the row pass output, one per row
    float2 *post_rows; // DCT plans: (cos, sin)(pi k / (2 cols)), k = 0 .. cols/2
    float2 *post_cols; // DCT plans: (cos, sin)(pi k / (2 rows)), k = 0 .. rows/2
};

namespace fft2d {

bool plan_view(const void *plan, PlanView *v)
{
    const fft2d_plan_s *p = static_cast<const fft2d_plan_s *>(plan);
    if (!p || !v)
        return false;
    *v = PlanView{p->rows, p->cols, p->Lr, p->Lc, p->dtype, p->dir, p->tw_rows, p->tw_cols,
                  p->dev_err};
    return true;
}

}  // namespace fft2d

namespace {

thread_local char g_last_error[256] = "";

fft2d_status cuda_fail(cudaError_t e, const char *what)
{
    std::snprintf(g_last_error, sizeof g_last_error, "%s: %s", what, cudaGetErrorString(e));
    return FFT2D_ERR_CUDA;
}

int log2_exact(int n)
{
    int L = 0;
    while ((1 << L) < n)
        L++;
    return L;
}

// W_M^j = exp(-2*pi*i*j/M) in FP64 with exact symmetry: the angle is reduced
// to the first octant with integer arithmetic, so quarter turns are exact
// (1, -i, -1, i) and symmetric entries are bitwise mirror images.
void twiddle_fp64(long long j, long long M, double *c, double *s)
{
    j %= M;
    // n in [0, M): fold by symmetries of cos/sin of 2*pi*n/M
    long long n = j;
    double sgn_s = 1.0, sgn_c = 1.0;
    bool swap = false;
    if (2 * n > M) {          // (pi, 2pi): sin negative
        n = M - n;
        sgn_s = -1.0;
    }
    if (4 * n > M) {          // (pi/2, pi]: cos negative
        n = M / 2 - n;        // M is even whenever 4n > M can hold with n <= M/2
        sgn_c = -1.0;
    }
    if (8 * n > M) {          // (pi/4, pi/2]: swap cos and sin
        n = M / 4 - n;
        swap = true;
    }
    double cc, ss;
    if (n == 0) {
        cc = 1.0;
        ss = 0.0;
    } else {
        const double ang = 2.0 * 3.14159265358979323846264338327950288 * (double)n / (double)M;
        cc = std::cos(ang);
        ss = std::sin(ang);
    }
    if (swap) {
        double t = cc;
        cc = ss;
        ss = t;
    }
    *c = sgn_c * cc;
    *s = sgn_s * ss;
}

// Per-stage table for an axis of 2^L points: N-1 entries.  Forward entries
// are W = cos(theta) - i sin(theta); inverse entries are the conjugates.
std::vector<float2> stage_table(int L, int dir)
{
    const long long N = 1LL << L;
    std::vector<float2> t((size_t)(N > 1 ? N - 1 : 1));
    for (int s = 1; s <= L; s++) {
        const long long half = 1LL << (s - 1);
        for (long long j = 0; j < half; j++) {
            double c, sn;
            twiddle_fp64(j, 1LL << s, &c, &sn);
            const double im = (dir == FFT2D_FORWARD) ? -sn : sn;
            t[(size_t)(half - 1 + j)] = make_float2((float)c, (float)im);
        }
    }
    return t;
}

// Post-rotation table of the DCT-II along an axis of N = 2^L points:
// (cos, sin)(pi k / (2N)) for k = 0 .. N/2, i.e. angles 2 pi k / (4N) up to
// pi/4, from the same octant-reduced FP64 evaluation as the stage tables
// (k = 0 is exactly (1, 0)).
std::vector<float2> dct_post_table(int L)
{
    const long long N = 1LL << L;
    std::vector<float2> t((size_t)(N / 2 + 1));
    for (long long k = 0; k <= N / 2; k++) {
        double c, sn;
        twiddle_fp64(k, 4 * N, &c, &sn);
        t[(size_t)k] = make_float2((float)c, (float)sn);
    }
    return t;
}

// Bytes of one image of the plan's storage type (C64 and DCT plans).
size_t image_bytes(const fft2d_plan_s *p)
{
    return (size_t)p->rows * p->cols * (p->dtype == FFT2D_R32_DCT2 ? sizeof(float) : sizeof(float2));
}

fft2d_status check_shape(int rows, int cols)
{
    if (rows < 1 || cols < 1 || (rows & (rows - 1)) || (cols & (cols - 1)))
        return FFT2D_ERR_NOT_POW2;
    if (rows > FFT2D_MAX_SIDE || cols > FFT2D_MAX_SIDE)
        return FFT2D_ERR_TOO_LARGE;
    return FFT2D_OK;
}

fft2d_status check_device(const fft2d_plan_s *p)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    if (dev != p->device) {
        std::snprintf(g_last_error, sizeof g_last_error,
                      "plan belongs to device %d, current device is %d", p->device, dev);
        return FFT2D_ERR_ARG;
    }
    return FFT2D_OK;
}

// One pass over the image.  nst < 0: all stages of that axis.
fft2d_status run_pass(const fft2d_plan_s *p, int pass, const void *in, void *out, int nst,
                      bool allow_scale, cudaStream_t st, int withhold = 0)
{
    fft2d::NvtxRange range(pass == FFT2D_PASS_ROWS ? "fft2d row pass" : "fft2d column pass");
    fft2d::PassArgs a;
    a.withhold = withhold;
    a.in = static_cast<const float2 *>(in);
    a.out = static_cast<float2 *>(out);
    a.rows = p->rows;
    a.cols = p->cols;
    a.ld = p->cols;
    a.scale = 1.0f;
    a.err = p->dev_err;
    a.variant = (pass == FFT2D_PASS_ROWS) ? p->row_variant : p->col_variant;
    const int L = (pass == FFT2D_PASS_ROWS) ? p->Lc : p->Lr;
    a.nst = nst < 0 ? L : nst;
    a.partial = a.nst < L;
    if (L == 0) {
        // A length-1 axis is the identity.  The inverse scale is applied by the
        // other axis's pass (the row pass when rows == 1, see below).
        if (in != out) {
            cudaError_t e = cudaMemcpyAsync(out, in, (size_t)p->rows * p->cols * sizeof(float2),
                                            cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess)
                return cuda_fail(e, "cudaMemcpyAsync");
        }
        return FFT2D_OK;
    }
    cudaError_t e;
    if (pass == FFT2D_PASS_ROWS) {
        a.tw = p->tw_rows;
        // inverse of an image with one row: the row pass is the last pass
        if (p->Lr == 0 && p->dir == FFT2D_INVERSE && allow_scale)
            a.scale = 1.0f / (float)((double)p->rows * p->cols);
        e = fft2d::launch_row_pass(L, a, st);
    } else {
        a.tw = p->tw_cols;
        if (p->dir == FFT2D_INVERSE && allow_scale)
            a.scale = (float)(1.0 / ((double)p->rows * (double)p->cols));
        if (withhold && !fft2d::col_pass_is_tma_fed(L, a)) {
            std::snprintf(g_last_error, sizeof g_last_error,
                          "the column pass of this plan does not run on a TMA-fed kernel");
            return FFT2D_ERR_ARG;
        }
        e = fft2d::launch_col_pass(L, a, st);
    }
    if (e != cudaSuccess)
        return cuda_fail(e, pass == FFT2D_PASS_ROWS ? "row pass launch" : "column pass launch");
    return FFT2D_OK;
}

// One DCT-II pass of a DCT plan (rows: lines of cols points; columns: lines
// of rows points).
fft2d_status run_dct_pass(const fft2d_plan_s *p, int pass, const void *in, void *out,
                          cudaStream_t st)
{
    fft2d::NvtxRange range(pass == FFT2D_PASS_ROWS ? "fft2d dct rows" : "fft2d dct cols");
    const bool row = pass == FFT2D_PASS_ROWS;
    const bool inverse = p->dir == FFT2D_INVERSE;
    // the inverse's 1/(rows cols) rides on the column pass, as for the FFT
    const float scale = (inverse && !row) ? (float)(1.0 / ((double)p->rows * p->cols)) : 1.0f;
    cudaError_t e = fft2d::launch_dct_pass(row, inverse, row ? p->Lc : p->Lr,
                                           static_cast<const float *>(in),
                                           static_cast<float *>(out), p->rows, p->cols,
                                           row ? p->tw_rows : p->tw_cols,
                                           row ? p->post_rows : p->post_cols, scale,
                                           p->dev_err, st);
    if (e != cudaSuccess)
        return cuda_fail(e, row ? "DCT row pass launch" : "DCT column pass launch");
    return FFT2D_OK;
}

fft2d_status exec_impl(const fft2d_plan_s *p, const void *in, void *out, int rs, int cs,
                       cudaStream_t st)
{
    if (p->dtype == FFT2D_R32_DCT2) {
        fft2d_status s = run_dct_pass(p, FFT2D_PASS_ROWS, in, out, st);
        if (s != FFT2D_OK)
            return s;
        return run_dct_pass(p, FFT2D_PASS_COLS, out, out, st);
    }
    const bool full = (rs < 0 || rs == p->Lc) && (cs < 0 || cs == p->Lr);
    fft2d_status s = run_pass(p, FFT2D_PASS_ROWS, in, out, rs, full, st);
    if (s != FFT2D_OK)
        return s;
    if (p->Lr == 0)
        return FFT2D_OK;   // one row: nothing along the columns
    return run_pass(p, FFT2D_PASS_COLS, out, out, cs, full, st);
}

// ---------------------------------------------------------------- autotuning
// Winners of past tunings, keyed by (device, pass, log2 axis length, number
// of lines): later plans of the same shape start from them.  Optionally
// mirrored in the text file named by the FFT2D_TUNE_CACHE environment
// variable, one "device-name<TAB>pass<TAB>L<TAB>lines<TAB>variant-name" line
// per entry, so that a new process does not have to tune again.
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_tuned;
bool g_tune_file_loaded = false;

std::string device_name(int dev)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return "unknown";
    return prop.name;
}

int variant_index(int pass, int L, const char *name)
{
    int n = 0;
    const fft2d::Variant *v =
        pass == FFT2D_PASS_ROWS ? fft2d::row_variants(L, &n) : fft2d::col_variants(L, &n);
    for (int i = 0; i < n; i++)
        if (std::strcmp(v[i].name, name) == 0)
            return i;
    return -1;
}

void load_tune_file_locked(int dev)
{
    if (g_tune_file_loaded)
        return;
    g_tune_file_loaded = true;
    const char *path = std::getenv("FFT2D_TUNE_CACHE");
    if (!path || !*path)
        return;
    FILE *f = std::fopen(path, "r");
    if (!f)
        return;
    const std::string me = device_name(dev);
    char line[512];
    while (std::fgets(line, sizeof line, f)) {
        char name[256], var[64];
        int pass, L, lines;
        if (std::sscanf(line, "%255[^\t]\t%d\t%d\t%d\t%63s", name, &pass, &L, &lines, var) != 5)
            continue;
        if (me != name || L < 1 || L > 14)
            continue;
        const int idx = variant_index(pass, L, var);
        if (idx >= 0)
            g_tuned[std::make_tuple(dev, pass, L, lines)] = idx;
    }
    std::fclose(f);
}

void save_tune_file_locked()
{
    const char *path = std::getenv("FFT2D_TUNE_CACHE");
    if (!path || !*path)
        return;
    FILE *f = std::fopen(path, "w");
    if (!f)
        return;
    for (const auto &kv : g_tuned) {
        const int dev = std::get<0>(kv.first), pass = std::get<1>(kv.first);
        const int L = std::get<2>(kv.first), lines = std::get<3>(kv.first);
        int n = 0;
        const fft2d::Variant *v =
            pass == FFT2D_PASS_ROWS ? fft2d::row_variants(L, &n) : fft2d::col_variants(L, &n);
        if (kv.second < 0 || kv.second >= n)
            continue;
        std::fprintf(f, "%s\t%d\t%d\t%d\t%s\n", device_name(dev).c_str(), pass, L, lines,
                     v[kv.second].name);
    }
    std::fclose(f);
}

void apply_tuned(fft2d_plan_s *p)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    load_tune_file_locked(p->device);
    auto r = g_tuned.find(std::make_tuple(p->device, (int)FFT2D_PASS_ROWS, p->Lc, p->rows));
    if (r != g_tuned.end())
        p->row_variant = r->second;
    auto c = g_tuned.find(std::make_tuple(p->device, (int)FFT2D_PASS_COLS, p->Lr, p->cols));
    if (c != g_tuned.end())
        p->col_variant = c->second;
}

}  // namespace

namespace {

// Device buffers, streams and events of the pipelined host path, one set per
// device, grown on demand and kept for the life of the process.  One call at
// a time uses a device's set (the mutex).
// Device image buffers of the host pipeline: images in flight between
// upload, transform and download.  A forward transform and its chained
// inverse hold two at once, so three pairs stay in flight with six.
constexpr int kHostSlots = 6;
constexpr int kHostMaxDev = 64;

struct HostPipe {
    std::mutex mu;
    void *slot[kHostSlots] = {};
    size_t slot_bytes = 0;
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t in_ready[kHostSlots] = {}, done[kHostSlots] = {}, freed[kHostSlots] = {};
    cudaEvent_t start = nullptr, join_up = nullptr, join_down = nullptr;
    // download of the i-th image of a call: an upload of a later image of
    // the same call that reads the same host buffer waits for it
    std::vector<cudaEvent_t> image_out;
    bool ready = false;
};

HostPipe g_host_pipe[kHostMaxDev];

cudaError_t host_pipe_prepare(HostPipe &hp, size_t bytes)
{
    cudaError_t e = cudaSuccess;
    if (!hp.ready) {
        e = cudaStreamCreateWithFlags(&hp.up, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaStreamCreateWithFlags(&hp.down, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&hp.start, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&hp.join_up, cudaEventDisableTiming);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&hp.join_down, cudaEventDisableTiming);
        for (int k = 0; k < kHostSlots && e == cudaSuccess; k++) {
            e = cudaEventCreateWithFlags(&hp.in_ready[k], cudaEventDisableTiming);
            if (e == cudaSuccess)
                e = cudaEventCreateWithFlags(&hp.done[k], cudaEventDisableTiming);
            if (e == cudaSuccess)
                e = cudaEventCreateWithFlags(&hp.freed[k], cudaEventDisableTiming);
        }
        if (e != cudaSuccess)
            return e;
        hp.ready = true;
    }
    if (bytes > hp.slot_bytes) {
        for (int k = 0; k < kHostSlots; k++) {
            cudaFree(hp.slot[k]);
            hp.slot[k] = nullptr;
        }
        hp.slot_bytes = 0;
        for (int k = 0; k < kHostSlots; k++) {
            e = cudaMalloc(&hp.slot[k], bytes);
            if (e != cudaSuccess) {
                for (int j = 0; j < kHostSlots; j++) {
                    cudaFree(hp.slot[j]);
                    hp.slot[j] = nullptr;
                }
                return e;
            }
        }
        hp.slot_bytes = bytes;
    }
    return cudaSuccess;
}

}  // namespace

namespace {

// Grouped-launch variant for (pass, L): tuned winner (key pass + 2) or the
// default.
int batch_variant(int device, int pass, int L)
{
    std::lock_guard<std::mutex> lock(g_tune_mu);
    load_tune_file_locked(device);
    auto it = g_tuned.find(std::make_tuple(device, pass + 2, L, 0));
    if (it != g_tuned.end())
        return it->second;
    return fft2d::batch_default_variant(pass == FFT2D_PASS_ROWS, L);
}

// Internal streams of the grouped executor, one set per (device, caller
// stream) so that batches issued on different streams still overlap: the
// groups of one pass are independent, so they run on kBatchLanes streams at
// once (the tail of one launch overlaps the start of the next); the column
// pass starts after every row group, and the caller's stream waits for
// everything.
constexpr int kBatchLanes = 4;
struct BatchLanes {
    std::mutex mu;
    cudaStream_t s[kBatchLanes] = {};
    cudaEvent_t fork = nullptr, ev[kBatchLanes] = {};
    bool ready = false;
};
std::mutex g_batch_lanes_mu;
std::map<std::pair<int, cudaStream_t>, BatchLanes *> g_batch_lanes;   // kept for the process

BatchLanes *batch_lanes(int dev, cudaStream_t st)
{
    std::lock_guard<std::mutex> lock(g_batch_lanes_mu);
    BatchLanes *&bl = g_batch_lanes[std::make_pair(dev, st)];
    if (!bl)
        bl = new (std::nothrow) BatchLanes();
    return bl;
}

cudaError_t batch_lanes_prepare(BatchLanes &bl)
{
    if (bl.ready)
        return cudaSuccess;
    cudaError_t e = cudaEventCreateWithFlags(&bl.fork, cudaEventDisableTiming);
    for (int k = 0; k < kBatchLanes && e == cudaSuccess; k++) {
        e = cudaStreamCreateWithFlags(&bl.s[k], cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&bl.ev[k], cudaEventDisableTiming);
    }
    if (e == cudaSuccess)
        bl.ready = true;
    return e;
}

// Every lane waits for `from` (one stream) ...
cudaError_t lanes_wait_stream(BatchLanes &bl, cudaStream_t from)
{
    cudaError_t e = cudaEventRecord(bl.fork, from);
    for (int k = 0; k < kBatchLanes && e == cudaSuccess; k++)
        e = cudaStreamWaitEvent(bl.s[k], bl.fork, 0);
    return e;
}

// ... and `to` waits for every lane.
cudaError_t stream_wait_lanes(BatchLanes &bl, cudaStream_t to)
{
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < kBatchLanes && e == cudaSuccess; k++) {
        e = cudaEventRecord(bl.ev[k], bl.s[k]);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(to, bl.ev[k], 0);
    }
    return e;
}

// Run the grouped passes of a batch.  With `timing` set, every (pass, L,
// direction) group is launched once per variant and timed on `st`, and the
// fastest variant per (pass, L) is recorded (the batch autotuner);
// otherwise each group runs once with its chosen variant, the groups of a
// pass spread over the device's internal lanes.
fft2d_status batched_impl(int n, const fft2d_plan_t *plans, const void *const *in,
                          void *const *out, cudaStream_t st, bool timing)
{
    fft2d::NvtxRange range(timing ? "fft2d batched autotune" : "fft2d batched");
    BatchLanes *bl = nullptr;
    std::unique_lock<std::mutex> lanes_lock;
    if (!timing && n > 0) {
        bl = batch_lanes(plans[0]->device, st);
        if (!bl)
            return FFT2D_ERR_OOM;
        lanes_lock = std::unique_lock<std::mutex>(bl->mu);
        cudaError_t e = batch_lanes_prepare(*bl);
        if (e == cudaSuccess)
            e = lanes_wait_stream(*bl, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "batch lanes");
    }
    int group = 0;
    static thread_local fft2d::BatchTable table;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (timing && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        return cuda_fail(cudaGetLastError(), "cudaEventCreate");
    std::map<std::pair<int, int>, std::vector<float>> times;   // (pass, L) -> ms per variant
    fft2d_status result = FFT2D_OK;
    for (int pass = 0; pass < 2 && result == FFT2D_OK; pass++) {
        const bool row = pass == FFT2D_PASS_ROWS;
        if (bl && !row) {
            // the column pass starts once every row group has finished
            cudaError_t e = stream_wait_lanes(*bl, bl->s[0]);
            if (e == cudaSuccess)
                e = lanes_wait_stream(*bl, bl->s[0]);
            if (e != cudaSuccess) {
                result = cuda_fail(e, "batch lanes");
                break;
            }
        }
        for (int L = 1; L <= 14 && result == FFT2D_OK; L++) {
            for (int dir = -1; dir <= 1 && result == FFT2D_OK; dir += 2) {
                table.n = 0;
                int *err = nullptr;
                int first = -1;
                for (int i = 0; i <= n; i++) {
                    const bool flush = (i == n) || table.n == fft2d::kBatchTmaMaxJobs;
                    if (flush && table.n > 0) {
                        const int nv = row ? fft2d::kBatchRowVariants : fft2d::kBatchColVariants;
                        if (!timing && L >= 13) {
                            // lines of 8192 and 16384 points: each image's
                            // single-image pass (the cluster column kernels,
                            // the 5-stage-group rows), the same bits
                            cudaStream_t ls = bl->s[group++ % kBatchLanes];
                            cudaError_t e = cudaSuccess;
                            for (int jj = 0; jj < table.n && e == cudaSuccess; jj++) {
                                const fft2d::BatchJob &j = table.job[jj];
                                fft2d::PassArgs a;
                                a.in = j.in;
                                a.out = j.out;
                                a.tw = j.tw;
                                a.rows = row ? j.lines : (1 << L);
                                a.cols = row ? (1 << L) : j.lines;
                                a.ld = j.ld;
                                a.scale = j.scale;
                                a.nst = L;
                                a.partial = false;
                                a.err = err;
                                e = row ? fft2d::launch_row_pass(L, a, ls)
                                        : fft2d::launch_col_pass(L, a, ls);
                            }
                            if (e != cudaSuccess) {
                                result = cuda_fail(e, "batched pass");
                                break;
                            }
                        } else if (!timing) {
                            const int v = batch_variant(plans[first]->device, pass, L);
                            cudaStream_t ls = bl->s[group++ % kBatchLanes];
                            cudaError_t e = fft2d::launch_batch_pass(row, L, table, v, err, ls);
                            if (e != cudaSuccess) {
                                result = cuda_fail(e, "batched pass");
                                break;
                            }
                        } else {
                            auto &tv = times[std::make_pair(pass, L)];
                            tv.resize(nv, 0.f);
                            for (int v = 0; v < nv && result == FFT2D_OK; v++) {
                                cudaError_t e = fft2d::launch_batch_pass(row, L, table, v, err, st);
                                if (e == cudaSuccess)
                                    e = cudaEventRecord(e0, st);
                                for (int r = 0; r < 3 && e == cudaSuccess; r++)
                                    e = fft2d::launch_batch_pass(row, L, table, v, err, st);
                                if (e == cudaSuccess)
                                    e = cudaEventRecord(e1, st);
                                if (e == cudaSuccess)
                                    e = cudaEventSynchronize(e1);
                                float ms = 0.f;
                                if (e == cudaSuccess)
                                    e = cudaEventElapsedTime(&ms, e0, e1);
                                if (e != cudaSuccess)
                                    result = cuda_fail(e, "batched tuning");
                                tv[v] += ms;
                            }
                        }
                        table.n = 0;
                    }
                    if (i == n)
                        break;
                    const fft2d_plan_s *p = plans[i];
                    if (p->Lr == 0 || p->Lc == 0 || (row ? p->Lc : p->Lr) != L || p->dir != dir)
                        continue;
                    if (first < 0) {
                        first = i;
                        err = p->dev_err;
                    }
                    fft2d::BatchJob &j = table.job[table.n++];
                    j.in = static_cast<const float2 *>(row ? in[i] : out[i]);
                    j.out = static_cast<float2 *>(out[i]);
                    j.tw = row ? p->tw_rows : p->tw_cols;
                    j.ld = p->cols;
                    j.lines = row ? p->rows : p->cols;
                    j.first_cta = 0;
                    j.scale = (!row && p->dir == FFT2D_INVERSE)
                                  ? (float)(1.0 / ((double)p->rows * (double)p->cols))
                                  : 1.0f;
                }
            }
        }
    }
    if (bl) {
        cudaError_t e = stream_wait_lanes(*bl, st);
        if (e != cudaSuccess && result == FFT2D_OK)
            result = cuda_fail(e, "batch lanes");
    }
    if (timing) {
        if (result == FFT2D_OK && n > 0) {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            load_tune_file_locked(plans[0]->device);
            for (auto &kv : times) {
                const auto &tv = kv.second;
                int best = 0;
                for (int v = 1; v < (int)tv.size(); v++)
                    if (tv[v] < tv[best])
                        best = v;
                g_tuned[std::make_tuple(plans[0]->device, kv.first.first + 2, kv.first.second, 0)] =
                    best;
            }
            save_tune_file_locked();
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    return result;
}

fft2d_status batched_check(int n, const fft2d_plan_t *plans, const void *const *in,
                           void *const *out)
{
    if (n < 0 || (n > 0 && (!plans || !in || !out)))
        return FFT2D_ERR_ARG;
    for (int i = 0; i < n; i++)
        if (!plans[i] || !in[i] || !out[i] || plans[i]->dtype != FFT2D_C64)
            return FFT2D_ERR_ARG;
    for (int i = 0; i < n; i++) {
        fft2d_status s = check_device(plans[i]);
        if (s != FFT2D_OK)
            return s;
    }
    return FFT2D_OK;
}

}  // namespace

extern "C" {

int fft2d_version(void) { return 100; }

const char *fft2d_strerror(int status)
{
    switch (status) {
    case FFT2D_OK: return "ok";
    case FFT2D_ERR_ARG: return "invalid argument";
    case FFT2D_ERR_NOT_POW2: return "image side is not a power of two";
    case FFT2D_ERR_TOO_LARGE: return "image side exceeds FFT2D_MAX_SIDE";
    case FFT2D_ERR_OOM: return "out of memory";
    case FFT2D_ERR_CUDA: return "CUDA error";
    case FFT2D_ERR_TIMEOUT: return "bounded device wait timed out";
    case FFT2D_ERR_BUDGET: return "request exceeds the memory budget";
    case FFT2D_ERR_UNSUPPORTED: return "not supported by this build";
    default: return "unknown status";
    }
}

const char *fft2d_last_error(void) { return g_last_error; }

fft2d_status fft2d_plan(int rows, int cols, int dtype, int dir, fft2d_plan_t *out)
{
    if (!out)
        return FFT2D_ERR_ARG;
    *out = nullptr;
    fft2d_status st = check_shape(rows, cols);
    if (st != FFT2D_OK)
        return st;
    if (dir != FFT2D_FORWARD && dir != FFT2D_INVERSE)
        return FFT2D_ERR_ARG;
    if (dtype != FFT2D_C64 && dtype != FFT2D_C32H && dtype != FFT2D_R32_DCT2)
        return FFT2D_ERR_ARG;
    if ((dtype == FFT2D_C32H || dtype == FFT2D_R32_DCT2) && (rows < 2 || cols < 2))
        return FFT2D_ERR_UNSUPPORTED;
    fft2d_plan_s *p = new (std::nothrow) fft2d_plan_s();
    if (!p)
        return FFT2D_ERR_OOM;
    p->rows = rows;
    p->cols = cols;
    p->Lr = log2_exact(rows);
    p->Lc = log2_exact(cols);
    p->dtype = dtype;
    p->dir = dir;
    p->row_variant = -1;
    p->col_variant = -1;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "cudaGetDevice");
    }
    std::vector<float2> tr = stage_table(p->Lc, dir), tc = stage_table(p->Lr, dir);
    // one padding entry: kernels may copy 2^L entries (a multiple of 16 bytes)
    tr.push_back(make_float2(0.f, 0.f));
    tc.push_back(make_float2(0.f, 0.f));
    e = cudaMalloc(&p->tw_rows, tr.size() * sizeof(float2));
    if (e == cudaSuccess)
        e = cudaMalloc(&p->tw_cols, tc.size() * sizeof(float2));
    if (e != cudaSuccess) {
        cudaFree(p->tw_rows);
        delete p;
        cuda_fail(e, "cudaMalloc twiddles");
        return FFT2D_ERR_OOM;
    }
    e = cudaMalloc(&p->dev_err, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(p->tw_rows);
        cudaFree(p->tw_cols);
        delete p;
        cuda_fail(e, "cudaMalloc status word");
        return FFT2D_ERR_OOM;
    }
    e = cudaMemcpy(p->tw_rows, tr.data(), tr.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(p->tw_cols, tc.data(), tc.size() * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemset(p->dev_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(p->tw_rows);
        cudaFree(p->tw_cols);
        cudaFree(p->dev_err);
        delete p;
        return cuda_fail(e, "cudaMemcpy twiddles");
    }
    if (dtype == FFT2D_C32H) {
        e = cudaMalloc(&p->exp_rows, sizeof(int) * (size_t)rows);
        if (e != cudaSuccess) {
            cudaFree(p->tw_rows);
            cudaFree(p->tw_cols);
            cudaFree(p->dev_err);
            delete p;
            cuda_fail(e, "cudaMalloc exponents");
            return FFT2D_ERR_OOM;
        }
    }
    if (dtype == FFT2D_R32_DCT2) {
        const std::vector<float2> pr = dct_post_table(p->Lc), pc = dct_post_table(p->Lr);
        e = cudaMalloc(&p->post_rows, pr.size() * sizeof(float2));
        if (e == cudaSuccess)
            e = cudaMalloc(&p->post_cols, pc.size() * sizeof(float2));
        if (e == cudaSuccess)
            e = cudaMemcpy(p->post_rows, pr.data(), pr.size() * sizeof(float2),
                           cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(p->post_cols, pc.data(), pc.size() * sizeof(float2),
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            fft2d_destroy(p);
            return cuda_fail(e, "DCT post-rotation tables");
        }
        *out = p;
        return FFT2D_OK;
    }
    apply_tuned(p);
    *out = p;
    return FFT2D_OK;
}

fft2d_status fft2d_autotune(fft2d_plan_t p, void *stream)
{
    if (!p || p->dtype == FFT2D_R32_DCT2)
        return FFT2D_ERR_ARG;
    fft2d_status s = check_device(p);
    if (s != FFT2D_OK)
        return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = (size_t)p->rows * p->cols * sizeof(float2);
    void *a = nullptr, *b = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&a, bytes);
    if (e == cudaSuccess)
        e = cudaMalloc(&b, bytes);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(a, 0, bytes, st);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    fft2d_status result = FFT2D_OK;
    for (int pass = 0; pass < 2 && e == cudaSuccess; pass++) {
        const int L = pass == FFT2D_PASS_ROWS ? p->Lc : p->Lr;
        if (L == 0)
            continue;
        int n = 0;
        const fft2d::Variant *v =
            pass == FFT2D_PASS_ROWS ? fft2d::row_variants(L, &n) : fft2d::col_variants(L, &n);
        fft2d::PassArgs args;
        args.in = static_cast<const float2 *>(pass == FFT2D_PASS_ROWS ? a : b);
        args.out = static_cast<float2 *>(b);
        args.tw = pass == FFT2D_PASS_ROWS ? p->tw_rows : p->tw_cols;
        args.rows = p->rows;
        args.cols = p->cols;
        args.ld = p->cols;
        args.scale = 1.0f;
        args.nst = L;
        args.partial = false;
        args.err = p->dev_err;
        int best = -1;
        float best_ms = 0.f;
        for (int i = 0; i < n && e == cudaSuccess; i++) {
            args.variant = i;
            if (!v[i].usable(args))
                continue;
            for (int w = 0; w < 2 && e == cudaSuccess; w++)
                e = v[i].launch(args, st);
            const int reps = 5;
            if (e == cudaSuccess)
                e = cudaEventRecord(e0, st);
            for (int r = 0; r < reps && e == cudaSuccess; r++)
                e = v[i].launch(args, st);
            if (e == cudaSuccess)
                e = cudaEventRecord(e1, st);
            if (e == cudaSuccess)
                e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess)
                e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && (best < 0 || ms < best_ms)) {
                best = i;
                best_ms = ms;
            }
        }
        if (e == cudaSuccess && best >= 0) {
            const int lines = pass == FFT2D_PASS_ROWS ? p->rows : p->cols;
            if (pass == FFT2D_PASS_ROWS)
                p->row_variant = best;
            else
                p->col_variant = best;
            std::lock_guard<std::mutex> lock(g_tune_mu);
            load_tune_file_locked(p->device);
            g_tuned[std::make_tuple(p->device, pass, L, lines)] = best;
            save_tune_file_locked();
        }
    }
    if (e != cudaSuccess)
        result = cuda_fail(e, "fft2d_autotune");
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    cudaFree(a);
    cudaFree(b);
    // a timeout during tuning is not the caller's business: clear the word
    cudaMemset(p->dev_err, 0, sizeof(int));
    return result;
}

fft2d_status fft2d_exec_h16(fft2d_plan_t p, const void *in, const int *in_exp, int in_axis,
                            void *out, int *out_exp, void *stream)
{
    if (!p || !in || !in_exp || !out || !out_exp || p->dtype != FFT2D_C32H ||
        (in_axis != FFT2D_PASS_ROWS && in_axis != FFT2D_PASS_COLS))
        return FFT2D_ERR_ARG;
    fft2d_status s = check_device(p);
    if (s != FFT2D_OK)
        return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    fft2d::H16PassArgs a;
    a.rows = p->rows;
    a.cols = p->cols;
    a.ld = p->cols;
    // row pass: in -> out, per-row exponents into the plan
    a.in = static_cast<const __half2 *>(in);
    a.out = static_cast<__half2 *>(out);
    a.tw = p->tw_rows;
    a.scale = 1.0f;
    a.nst = p->Lc;
    a.in_exp = in_exp;
    a.in_axis = in_axis;
    a.out_exp = p->exp_rows;
    a.err = p->dev_err;
    cudaError_t e = fft2d::launch_pass_h16(true, p->Lc, a, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "half2 row pass");
    // column pass: out -> out, per-column exponents to the caller
    a.in = static_cast<const __half2 *>(out);
    a.tw = p->tw_cols;
    a.scale = p->dir == FFT2D_INVERSE ? (float)(1.0 / ((double)p->rows * (double)p->cols)) : 1.0f;
    a.nst = p->Lr;
    a.in_exp = p->exp_rows;
    a.in_axis = FFT2D_PASS_ROWS;
    a.out_exp = out_exp;
    e = fft2d::launch_pass_h16(false, p->Lr, a, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "half2 column pass");
    return FFT2D_OK;
}

fft2d_status fft2d_h16_pack(int rows, int cols, const void *in, void *out, int *out_exp,
                            void *stream)
{
    if (!in || !out || !out_exp || rows < 1 || cols < 1)
        return FFT2D_ERR_ARG;
    cudaError_t e = fft2d::launch_h16_pack(static_cast<const float2 *>(in),
                                           static_cast<__half2 *>(out), out_exp, rows, cols,
                                           static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FFT2D_OK : cuda_fail(e, "fft2d_h16_pack");
}

fft2d_status fft2d_h16_unpack(int rows, int cols, const void *in, const int *exps, int axis,
                              void *out, void *stream)
{
    if (!in || !exps || !out || rows < 1 || cols < 1 ||
        (axis != FFT2D_PASS_ROWS && axis != FFT2D_PASS_COLS))
        return FFT2D_ERR_ARG;
    cudaError_t e = fft2d::launch_h16_unpack(static_cast<const __half2 *>(in), exps, axis,
                                             static_cast<float2 *>(out), rows, cols,
                                             static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FFT2D_OK : cuda_fail(e, "fft2d_h16_unpack");
}

fft2d_status fft2d_lowpass(int rows, int cols, int dtype, void *data, float sigma_rows,
                           float sigma_cols, void *stream)
{
    if (!data || rows < 1 || cols < 1 || !(sigma_rows > 0.f) || !(sigma_cols > 0.f) ||
        (dtype != FFT2D_C64 && dtype != FFT2D_C32H))
        return FFT2D_ERR_ARG;
    cudaError_t e = fft2d::launch_lowpass(dtype == FFT2D_C32H, data, rows, cols, sigma_rows,
                                          sigma_cols, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? FFT2D_OK : cuda_fail(e, "fft2d_lowpass");
}

int fft2d_variant_count(int pass, int L)
{
    if ((pass != FFT2D_PASS_ROWS && pass != FFT2D_PASS_COLS) || L < 1 || L > 14)
        return 0;
    int n = 0;
    if (pass == FFT2D_PASS_ROWS)
        fft2d::row_variants(L, &n);
    else
        fft2d::col_variants(L, &n);
    return n;
}

const char *fft2d_variant_name(int pass, int L, int index)
{
    const int n = fft2d_variant_count(pass, L);
    if (index < 0 || index >= n)
        return "";
    int m = 0;
    const fft2d::Variant *v =
        pass == FFT2D_PASS_ROWS ? fft2d::row_variants(L, &m) : fft2d::col_variants(L, &m);
    return v[index].name;
}

fft2d_status fft2d_plan_set_variant(fft2d_plan_t p, int pass, int variant)
{
    if (!p || (pass != FFT2D_PASS_ROWS && pass != FFT2D_PASS_COLS) ||
        p->dtype == FFT2D_R32_DCT2)
        return FFT2D_ERR_ARG;
    const int L = pass == FFT2D_PASS_ROWS ? p->Lc : p->Lr;
    if (variant < -1 || variant >= fft2d_variant_count(pass, L) + (L == 0 ? 1 : 0))
        return FFT2D_ERR_ARG;
    if (pass == FFT2D_PASS_ROWS)
        p->row_variant = variant;
    else
        p->col_variant = variant;
    return FFT2D_OK;
}

fft2d_status fft2d_plan_describe(fft2d_plan_t p, char *buf, int len)
{
    if (!p || !buf || len <= 0)
        return FFT2D_ERR_ARG;
    if (p->dtype == FFT2D_R32_DCT2) {
        const char *kind = p->dir == FFT2D_INVERSE ? "dct3" : "dct2";
        std::snprintf(buf, (size_t)len, "rows:%s(lines=%d,points=%d) cols:%s(lines=%d,points=%d)",
                      kind, p->rows / 2, p->cols, kind, p->cols / 2, p->rows);
        return FFT2D_OK;
    }
    std::string out;
    for (int pass = 0; pass < 2; pass++) {
        const int L = pass == FFT2D_PASS_ROWS ? p->Lc : p->Lr;
        out += pass == FFT2D_PASS_ROWS ? "rows:" : " cols:";
        if (L == 0) {
            out += "identity";
            continue;
        }
        int n = 0;
        const fft2d::Variant *v =
            pass == FFT2D_PASS_ROWS ? fft2d::row_variants(L, &n) : fft2d::col_variants(L, &n);
        int i = pass == FFT2D_PASS_ROWS ? p->row_variant : p->col_variant;
        const bool tuned = i >= 0;
        if (i < 0 || i >= n)
            i = pass == FFT2D_PASS_ROWS ? fft2d::row_default_variant(L)
                                        : fft2d::col_default_variant(L);
        char tmp[96];
        std::snprintf(tmp, sizeof tmp, "%s(shape=%d,ept=%d,%s)", v[i].name, v[i].shape, v[i].ept,
                      tuned ? "tuned" : "default");
        out += tmp;
    }
    std::snprintf(buf, (size_t)len, "%s", out.c_str());
    return FFT2D_OK;
}

fft2d_status fft2d_destroy(fft2d_plan_t p)
{
    if (!p)
        return FFT2D_OK;
    cudaFree(p->tw_rows);
    cudaFree(p->tw_cols);
    cudaFree(p->dev_err);
    if (p->exp_rows)
        cudaFree(p->exp_rows);
    cudaFree(p->post_rows);
    cudaFree(p->post_cols);
    if (p->staging)
        cudaFree(p->staging);
    delete p;
    return FFT2D_OK;
}

fft2d_status fft2d_selftest_timeout(fft2d_plan_t p, void *stream)
{
    if (!p)
        return FFT2D_ERR_ARG;
    fft2d_status s = check_device(p);
    if (s != FFT2D_OK)
        return s;
    cudaError_t e = fft2d::launch_selftest_timeout(p->dev_err, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess)
        return cuda_fail(e, "self-test launch");
    return FFT2D_OK;
}

fft2d_status fft2d_sync_status(fft2d_plan_t p)
{
    if (!p)
        return FFT2D_ERR_ARG;
    fft2d_status s = check_device(p);
    if (s != FFT2D_OK)
        return s;
    int h = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(&h, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_fail(e, "fft2d_sync_status");
    if (h != 0) {
        cudaMemset(p->dev_err, 0, sizeof(int));
        std::snprintf(g_last_error, sizeof g_last_error,
                      "a bounded device wait gave up (code %d)", h);
        return FFT2D_ERR_TIMEOUT;
    }
    return FFT2D_OK;
}

fft2d_status fft2d_stage_table(int L, int dir, float *out)
{
    if (!out || L < 0 || L > 14 || (dir != FFT2D_FORWARD && dir != FFT2D_INVERSE))
        return FFT2D_ERR_ARG;
    std::vector<float2> t = stage_table(L, dir);
    const size_t n = (L > 0) ? ((size_t)1 << L) - 1 : 0;
    std::memcpy(out, t.data(), n * sizeof(float2));
    return FFT2D_OK;
}

fft2d_status fft2d_plan_info(fft2d_plan_t p, int *rows, int *cols, int *dtype, int *dir)
{
    if (!p)
        return FFT2D_ERR_ARG;
    if (rows)
        *rows = p->rows;
    if (cols)
        *cols = p->cols;
    if (dtype)
        *dtype = p->dtype;
    if (dir)
        *dir = p->dir;
    return FFT2D_OK;
}

fft2d_status fft2d_exec(fft2d_plan_t p, const void *in, void *out, void *stream)
{
    if (!p || !in || !out || (p->dtype != FFT2D_C64 && p->dtype != FFT2D_R32_DCT2))
        return FFT2D_ERR_ARG;
    fft2d_status s = check_device(p);
    if (s != FFT2D_OK)
        return s;
    return exec_impl(p, in, out, -1, -1, static_cast<cudaStream_t>(stream));
}

fft2d_status fft2d_selftest_withheld_load(fft2d_plan_t p, const void *in, void *out,
                                          void *stream)
{
    if (!p || !in || !out || (p->dtype != FFT2D_C64 && p->dtype != FFT2D_R32_DCT2) || p->Lr == 0)
        return FFT2D_ERR_ARG;
    fft2d_status s = check_device(p);
    if (s != FFT2D_OK)
        return s;
    if (p->dtype == FFT2D_R32_DCT2) {
        const bool inverse = p->dir == FFT2D_INVERSE;
        const float scale = inverse ? (float)(1.0 / ((double)p->rows * p->cols)) : 1.0f;
        cudaError_t e = fft2d::launch_dct_pass(false, inverse, p->Lr, static_cast<const float *>(in),
                                               static_cast<float *>(out), p->rows, p->cols,
                                               p->tw_cols, p->post_cols, scale, p->dev_err,
                                               static_cast<cudaStream_t>(stream), 1);
        if (e == cudaErrorNotSupported) {
            std::snprintf(g_last_error, sizeof g_last_error,
                          "the column pass of this plan does not run on a TMA-fed kernel");
            return FFT2D_ERR_ARG;
        }
        if (e != cudaSuccess)
            return cuda_fail(e, "DCT column pass launch");
        return FFT2D_OK;
    }
    return run_pass(p, FFT2D_PASS_COLS, in, out, -1, true, static_cast<cudaStream_t>(stream), 1);
}

fft2d_status fft2d_exec_pass(fft2d_plan_t p, int pass, const void *in, void *out, void *stream)
{
    if (!p || !in || !out || (pass != FFT2D_PASS_ROWS && pass != FFT2D_PASS_COLS) ||
        (p->dtype != FFT2D_C64 && p->dtype != FFT2D_R32_DCT2))
        return FFT2D_ERR_ARG;
    fft2d_status s = check_device(p);
    if (s != FFT2D_OK)
        return s;
    if (p->dtype == FFT2D_R32_DCT2)
        return run_dct_pass(p, pass, in, out, static_cast<cudaStream_t>(stream));
    return run_pass(p, pass, in, out, -1, true, static_cast<cudaStream_t>(stream));
}

fft2d_status fft2d_exec_stages(fft2d_plan_t p, const void *in, void *out, int row_stages,
                               int col_stages, void *stream)
{
    if (!p || !in || !out || p->dtype != FFT2D_C64)
        return FFT2D_ERR_ARG;
    if (row_stages < 0 || row_stages > p->Lc || col_stages < 0 || col_stages > p->Lr)
        return FFT2D_ERR_ARG;
    fft2d_status s = check_device(p);
    if (s != FFT2D_OK)
        return s;
    return exec_impl(p, in, out, row_stages, col_stages, static_cast<cudaStream_t>(stream));
}

fft2d_status fft2d_exec_host(fft2d_plan_t p, const void *in_host, void *out_host, void *stream)
{
    if (!p || !in_host || !out_host || (p->dtype != FFT2D_C64 && p->dtype != FFT2D_R32_DCT2))
        return FFT2D_ERR_ARG;
    fft2d_status s = check_device(p);
    if (s != FFT2D_OK)
        return s;
    const size_t bytes = image_bytes(p);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!p->staging) {
        cudaError_t e = cudaMalloc(&p->staging, bytes);
        if (e != cudaSuccess) {
            p->staging = nullptr;
            cuda_fail(e, "cudaMalloc staging");
            return FFT2D_ERR_OOM;
        }
    }
    cudaError_t e = cudaMemcpyAsync(p->staging, in_host, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync H2D");
    s = exec_impl(p, p->staging, p->staging, -1, -1, st);
    if (s != FFT2D_OK)
        return s;
    e = cudaMemcpyAsync(out_host, p->staging, bytes, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaMemcpyAsync D2H");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaStreamSynchronize");
    return FFT2D_OK;
}

namespace {

// Queue the pipelined host transforms of fft2d_exec_host_many(_async) on the
// device's host pipeline; the caller holds hp.mu.  On return (success or
// not) `st` is ordered after every copy queued here.
fft2d_status host_many_enqueue(HostPipe &hp, int n, const fft2d_plan_t *plans,
                               const void *const *in_host, void *const *out_host, cudaStream_t st)
{
    fft2d::NvtxRange range("fft2d host pipeline");
    size_t bytes = 0;
    for (int i = 0; i < n; i++) {
        const size_t b = image_bytes(plans[i]);
        bytes = b > bytes ? b : bytes;
    }
    cudaError_t e = host_pipe_prepare(hp, bytes);
    if (e != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? (cuda_fail(e, "cudaMalloc host pipeline"), FFT2D_ERR_OOM)
                                              : cuda_fail(e, "host pipeline setup");
    while ((int)hp.image_out.size() < n) {
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess)
            return cuda_fail(e, "host pipeline events");
        hp.image_out.push_back(ev);
    }
    fft2d_status result = FFT2D_OK;
    // the copies start after the work already queued on the caller's stream
    e = cudaEventRecord(hp.start, st);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(hp.up, hp.start, 0);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(hp.down, hp.start, 0);
    if (e != cudaSuccess)
        result = cuda_fail(e, "host pipeline ordering");
    // image i uses slot i % kHostSlots: upload on `up`, transform on the
    // caller's stream, download on `down`.  The upload into a slot waits for
    // the last download from it (of this call or an earlier one), and for the
    // download of an earlier image of this call whose output it reads.
    for (int i = 0; i < n && result == FFT2D_OK; i++) {
        const int k = i % kHostSlots;
        const fft2d_plan_s *p = plans[i];
        const size_t b = image_bytes(p);
        // an image whose input is the previous image's output (a forward
        // transform followed by its inverse) starts from the device copy of
        // that output, still in the previous slot: no upload
        const bool chained = i > 0 && in_host[i] == out_host[i - 1] && b == image_bytes(plans[i - 1]);
        const int kp = (i + kHostSlots - 1) % kHostSlots;
        if (chained) {
            e = cudaStreamWaitEvent(st, hp.freed[k], 0);
        } else {
            e = cudaStreamWaitEvent(hp.up, hp.freed[k], 0);
            for (int j = i - 1; j >= 0 && e == cudaSuccess; j--) {
                if (out_host[j] == in_host[i]) {
                    e = cudaStreamWaitEvent(hp.up, hp.image_out[j], 0);
                    break;
                }
            }
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hp.slot[k], in_host[i], b, cudaMemcpyHostToDevice, hp.up);
            if (e == cudaSuccess)
                e = cudaEventRecord(hp.in_ready[k], hp.up);
            if (e == cudaSuccess)
                e = cudaStreamWaitEvent(st, hp.in_ready[k], 0);
        }
        if (e != cudaSuccess) {
            result = cuda_fail(e, "host pipeline upload");
            break;
        }
        result = exec_impl(p, chained ? hp.slot[kp] : hp.slot[k], hp.slot[k], -1, -1, st);
        if (result != FFT2D_OK)
            break;
        // the output of an image that the next image of the call both starts
        // from (chained) and overwrites on the host can never be observed
        // there: it is not copied back
        const bool dead = i + 1 < n && in_host[i + 1] == out_host[i] &&
                          out_host[i + 1] == out_host[i] && image_bytes(plans[i + 1]) == b;
        e = cudaEventRecord(hp.done[k], st);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(hp.down, hp.done[k], 0);
        if (e == cudaSuccess && !dead)
            e = cudaMemcpyAsync(out_host[i], hp.slot[k], b, cudaMemcpyDeviceToHost, hp.down);
        if (e == cudaSuccess)
            e = cudaEventRecord(hp.freed[k], hp.down);
        // the previous slot was read by this transform: it is free once this
        // download (which follows the transform) is done
        if (e == cudaSuccess && chained)
            e = cudaEventRecord(hp.freed[kp], hp.down);
        if (e == cudaSuccess)
            e = cudaEventRecord(hp.image_out[i], hp.down);
        if (e != cudaSuccess)
            result = cuda_fail(e, "host pipeline download");
    }
    // join both copy streams into the caller's stream
    e = cudaEventRecord(hp.join_up, hp.up);
    if (e == cudaSuccess)
        e = cudaEventRecord(hp.join_down, hp.down);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(st, hp.join_up, 0);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(st, hp.join_down, 0);
    if (e != cudaSuccess && result == FFT2D_OK)
        result = cuda_fail(e, "host pipeline join");
    return result;
}

fft2d_status host_many_check(int n, const fft2d_plan_t *plans, const void *const *in_host,
                             void *const *out_host, HostPipe **hp)
{
    if (n < 0 || (n > 0 && (!plans || !in_host || !out_host)))
        return FFT2D_ERR_ARG;
    for (int i = 0; i < n; i++) {
        if (!plans[i] || !in_host[i] || !out_host[i] ||
            (plans[i]->dtype != FFT2D_C64 && plans[i]->dtype != FFT2D_R32_DCT2))
            return FFT2D_ERR_ARG;
        fft2d_status s = check_device(plans[i]);
        if (s != FFT2D_OK)
            return s;
    }
    if (n == 0)
        return FFT2D_OK;
    const int dev = plans[0]->device;
    if (dev < 0 || dev >= kHostMaxDev)
        return FFT2D_ERR_ARG;
    *hp = &g_host_pipe[dev];
    return FFT2D_OK;
}

// Wait for everything a failed enqueue may have left in flight.
void host_many_drain(HostPipe &hp, cudaStream_t st)
{
    cudaStreamSynchronize(hp.up);
    cudaStreamSynchronize(st);
    cudaStreamSynchronize(hp.down);
}

}  // namespace

fft2d_status fft2d_exec_host_many(int n, const fft2d_plan_t *plans, const void *const *in_host,
                                  void *const *out_host, void *stream)
{
    HostPipe *hp = nullptr;
    fft2d_status s = host_many_check(n, plans, in_host, out_host, &hp);
    if (s != FFT2D_OK || n == 0)
        return s;
    std::lock_guard<std::mutex> lock(hp->mu);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    fft2d_status result = host_many_enqueue(*hp, n, plans, in_host, out_host, st);
    // synchronous: every queued copy and transform has finished on return,
    // also after a failure (the slots may then be reused)
    cudaError_t e1 = cudaStreamSynchronize(hp->up);
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaError_t e3 = cudaStreamSynchronize(hp->down);
    if (result == FFT2D_OK && (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess))
        result = cuda_fail(e1 != cudaSuccess ? e1 : (e2 != cudaSuccess ? e2 : e3),
                           "cudaStreamSynchronize");
    return result;
}

fft2d_status fft2d_exec_host_many_async(int n, const fft2d_plan_t *plans,
                                        const void *const *in_host, void *const *out_host,
                                        void *stream)
{
    HostPipe *hp = nullptr;
    fft2d_status s = host_many_check(n, plans, in_host, out_host, &hp);
    if (s != FFT2D_OK || n == 0)
        return s;
    std::lock_guard<std::mutex> lock(hp->mu);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    fft2d_status result = host_many_enqueue(*hp, n, plans, in_host, out_host, st);
    if (result != FFT2D_OK)
        host_many_drain(*hp, st);
    return result;
}

fft2d_status fft2d_exec_batched(int n, const fft2d_plan_t *plans, const void *const *in,
                                void *const *out, void *stream)
{
    fft2d_status s = batched_check(n, plans, in, out);
    if (s != FFT2D_OK)
        return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // images with a length-1 side take the single-image path
    for (int i = 0; i < n; i++) {
        if (plans[i]->Lr == 0 || plans[i]->Lc == 0) {
            s = exec_impl(plans[i], in[i], out[i], -1, -1, st);
            if (s != FFT2D_OK)
                return s;
        }
    }
    return batched_impl(n, plans, in, out, st, false);
}

int fft2d_batch_variant_count(int pass)
{
    if (pass == FFT2D_PASS_ROWS)
        return fft2d::kBatchRowVariants;
    return pass == FFT2D_PASS_COLS ? fft2d::kBatchColVariants : 0;
}

const char *fft2d_batch_variant_name(int pass, int index)
{
    if (index < 0 || index >= fft2d_batch_variant_count(pass))
        return "";
    return fft2d::batch_variant_name(pass == FFT2D_PASS_ROWS, index);
}

int fft2d_batch_get_variant(int pass, int L)
{
    int dev = 0;
    if (fft2d_batch_variant_count(pass) == 0 || L < 1 || L > 14 ||
        cudaGetDevice(&dev) != cudaSuccess)
        return -1;
    return batch_variant(dev, pass, L);
}

fft2d_status fft2d_batch_set_variant(int pass, int L, int variant)
{
    const int n = fft2d_batch_variant_count(pass);
    if (n == 0 || L < 1 || L > 14 || variant < -1 || variant >= n)
        return FFT2D_ERR_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lock(g_tune_mu);
    load_tune_file_locked(dev);
    const auto key = std::make_tuple(dev, pass + 2, L, 0);
    if (variant < 0)
        g_tuned.erase(key);
    else
        g_tuned[key] = variant;
    return FFT2D_OK;
}

fft2d_status fft2d_autotune_batched(int n, const fft2d_plan_t *plans, const void *const *in,
                                    void *const *out, void *stream)
{
    fft2d_status s = batched_check(n, plans, in, out);
    if (s != FFT2D_OK)
        return s;
    s = batched_impl(n, plans, in, out, static_cast<cudaStream_t>(stream), true);
    for (int i = 0; i < n; i++)
        cudaMemset(plans[i]->dev_err, 0, sizeof(int));
    return s;
}

}  // extern "C"
