// serve.cpp -- a continuous-batching request loop for 2D FFT work.
//
// Clients submit requests (a forward FFT, or FFT -> Gaussian low-pass ->
// inverse FFT) on host buffers.  One scheduler thread:
//   * admits queued requests in arrival order while the device memory they
//     need fits the HBM budget (buffers come from a resident pool; a request
//     that could never fit is refused at submission);
//   * launches everything admitted so far as one batch on an idle stream:
//     host->device copies, grouped FFT launches for the complex64 work
//     (fft2d_exec_batched) and for the half2 work (one launch per pass and
//     axis length; images with 4096+ rows on the TMA-fed half2 column pass
//     one at a time), the low-pass multiply, the inverse, device->host
//     copies, then an event;
//   * keeps several batches in flight on different streams, so requests that
//     arrive while others run are admitted as memory frees up and their work
//     overlaps on the device;
//   * polls the events, stamps completion times, returns buffers to the pool.
// Plans (rotation-factor tables) stay resident for the server's lifetime.
//
// A simulation mode runs the same admission and batching logic with no CUDA
// calls at all (modelled device time), so it can be tested without a GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <new>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "fft2d.h"
#include "passes.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    unsigned long long ticket;
    fft2d_request r;
    size_t bytes;                 // device memory this request holds while in flight
    Clock::time_point t_submit;
    Clock::time_point t_done;
    void *buf_c64 = nullptr;      // device complex64 image (FFT2D_C64)
    void *buf_h16 = nullptr;      // device half2 image (FFT2D_C32H)
    int *exps = nullptr;          // device exponents (FFT2D_C32H): input rows, row-pass
                                  // output rows, result columns (2 rows + cols ints)
    fft2d_status status = FFT2D_OK;
    bool done = false;
};

struct Batch {
    std::vector<Req *> reqs;
    int stream = -1;
    cudaEvent_t ev = nullptr;
    Clock::time_point sim_ready;  // simulation: modelled completion time
};

size_t exps_bytes(const fft2d_request &r) { return (size_t)(2 * r.rows + r.cols) * 4; }

size_t request_bytes(const fft2d_request &r)
{
    const size_t px = (size_t)r.rows * r.cols;
    return r.dtype == FFT2D_C32H ? px * 4 + exps_bytes(r) : px * 8;
}

// Half2 work of a batch phase: image i of `reqs` (in place in its buf_h16)
// from exponents in_exp (per row if in_axis == 0, else per column) through
// its row-pass exponents to its column exponents, with plans[i].  Columns of
// 4096+ rows take the single-image half2 passes (TMA-fed column pass), the
// rest grouped launches -- one per (pass, axis length) -- with the same CTA
// shapes, so every image gets the same bits either way.
cudaError_t h16_phase(const std::vector<Req *> &reqs, const std::vector<fft2d_plan_t> &plans,
                      int in_axis, cudaStream_t st)
{
    static thread_local fft2d::BatchTableH16 table;
    const size_t n = reqs.size();
    std::vector<fft2d::PlanView> pv(n);
    for (size_t i = 0; i < n; i++)
        if (!fft2d::plan_view(plans[i], &pv[i]))
            return cudaErrorInvalidValue;
    auto in_exp = [&](size_t i) {
        const Req *q = reqs[i];
        return in_axis == 0 ? q->exps : q->exps + 2 * q->r.rows;
    };
    auto grouped = [&](size_t i) { return pv[i].Lr < 12; };
    // the large images, one at a time
    for (size_t i = 0; i < n; i++) {
        if (grouped(i))
            continue;
        const Req *q = reqs[i];
        const fft2d::PlanView &v = pv[i];
        fft2d::H16PassArgs a;
        a.in = static_cast<const __half2 *>(q->buf_h16);
        a.out = static_cast<__half2 *>(q->buf_h16);
        a.rows = v.rows;
        a.cols = v.cols;
        a.ld = v.cols;
        a.tw = v.tw_rows;
        a.scale = 1.0f;
        a.nst = v.Lc;
        a.in_exp = in_exp(i);
        a.in_axis = in_axis;
        a.out_exp = q->exps + v.rows;
        a.err = v.err;
        cudaError_t e = fft2d::launch_pass_h16(true, v.Lc, a, st);
        if (e != cudaSuccess)
            return e;
        a.tw = v.tw_cols;
        a.nst = v.Lr;
        a.scale = v.dir == FFT2D_INVERSE ? (float)(1.0 / ((double)v.rows * (double)v.cols)) : 1.0f;
        a.in_exp = q->exps + v.rows;
        a.in_axis = FFT2D_PASS_ROWS;
        a.out_exp = q->exps + 2 * v.rows;
        e = fft2d::launch_pass_h16(false, v.Lr, a, st);
        if (e != cudaSuccess)
            return e;
    }
    // the rest: row groups by row length, then column groups by column length
    for (int pass = 0; pass < 2; pass++) {
        const bool row = pass == 0;
        for (int L = 1; L <= 14; L++) {
            table.n = 0;
            for (size_t i = 0; i <= n; i++) {
                const bool flush = i == n || table.n == fft2d::kBatchH16MaxJobs;
                if (flush && table.n > 0) {
                    cudaError_t e = fft2d::launch_batch_pass_h16(row, L, table,
                                                                 row ? in_axis : 0, st);
                    if (e != cudaSuccess)
                        return e;
                    table.n = 0;
                }
                if (i == n)
                    break;
                const fft2d::PlanView &v = pv[i];
                if (!grouped(i) || (row ? v.Lc : v.Lr) != L)
                    continue;
                const Req *q = reqs[i];
                fft2d::BatchJobH16 &j = table.job[table.n++];
                j.in = static_cast<const __half2 *>(q->buf_h16);
                j.out = static_cast<__half2 *>(q->buf_h16);
                j.tw = row ? v.tw_rows : v.tw_cols;
                j.in_exp = row ? in_exp(i) : q->exps + v.rows;
                j.out_exp = row ? q->exps + v.rows : q->exps + 2 * v.rows;
                j.ld = v.cols;
                j.lines = row ? v.rows : v.cols;
                j.first_cta = 0;
                j.scale = (!row && v.dir == FFT2D_INVERSE)
                              ? (float)(1.0 / ((double)v.rows * (double)v.cols))
                              : 1.0f;
            }
        }
    }
    return cudaSuccess;
}

bool pow2(int n) { return n >= 1 && !(n & (n - 1)); }

}  // namespace

struct fft2d_server_s {
    size_t budget;
    int nstreams;
    bool simulate;
    int device = 0;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stopping = false;
    std::thread worker;

    unsigned long long next_ticket = 1;
    std::deque<Req *> queue;                          // submitted, not admitted
    std::unordered_map<unsigned long long, Req *> all;
    std::vector<Batch> inflight;
    std::vector<cudaStream_t> streams;
    std::vector<bool> stream_busy;

    // memory accounting (device bytes held: in use + pooled)
    size_t used = 0, pooled = 0, peak = 0;
    std::multimap<size_t, void *> pool;               // free device buffers by size

    std::map<std::tuple<int, int, int, int>, fft2d_plan_t> plans;

    // statistics
    std::vector<double> latencies_ms;
    long long rejected = 0, batches = 0, batched_reqs = 0;
    Clock::time_point first_submit{}, last_done{};
    bool any_submit = false;

    // ------------------------------------------------------------- memory
    // Take a buffer of at least `need` bytes from the pool, or allocate one if
    // the budget allows.  Returns nullptr (without waiting) when it cannot.
    // With `exact`, a pooled buffer is taken only if it has exactly `need`
    // bytes.
    void *acquire(size_t need, bool exact = false)
    {
        auto it = pool.lower_bound(need);
        if (it != pool.end() && (exact ? it->first == need : it->first <= 2 * need)) {
            void *p = it->second;
            pooled -= it->first;
            used += it->first;
            sizes[p] = it->first;
            pool.erase(it);
            return p;
        }
        // make room by releasing pooled buffers that do not fit this request
        while (used + pooled + need > budget && !pool.empty()) {
            auto big = std::prev(pool.end());
            if (!simulate)
                cudaFree(big->second);
            else
                std::free(big->second);
            pooled -= big->first;
            pool.erase(big);
        }
        if (used + pooled + need > budget)
            return nullptr;
        void *p = nullptr;
        if (simulate) {
            p = std::malloc(1);
        } else if (cudaMalloc(&p, need) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        used += need;
        sizes[p] = need;
        peak = std::max(peak, used + pooled);
        return p;
    }
    std::unordered_map<void *, size_t> sizes;

    void release(void *p)
    {
        if (!p)
            return;
        const size_t n = sizes[p];
        sizes.erase(p);
        used -= n;
        pooled += n;
        pool.emplace(n, p);
    }

    bool try_admit(Req *q, bool exact)
    {
        const size_t px = (size_t)q->r.rows * q->r.cols;
        if (q->r.dtype == FFT2D_C64) {
            q->buf_c64 = acquire(px * 8, exact);
            return q->buf_c64 != nullptr;
        }
        q->buf_h16 = acquire(px * 4, exact);
        q->exps = static_cast<int *>(acquire(exps_bytes(q->r), exact));
        if (!q->buf_h16 || !q->exps) {
            release(q->buf_h16);
            release(q->exps);
            q->buf_h16 = nullptr;
            q->exps = nullptr;
            return false;
        }
        return true;
    }

    void free_pool()
    {
        for (auto &kv : pool) {
            if (simulate)
                std::free(kv.second);
            else
                cudaFree(kv.second);
        }
        pool.clear();
        pooled = 0;
    }

    // Admit q if its buffers fit the budget now.  A pooled buffer taken for
    // one of q's buffers may be up to twice as large as asked; when nothing
    // is in use (no request in flight), that surplus could be all that keeps
    // q's other buffers out, and no completion would ever change it.  In that
    // case the pool is released and q gets buffers of exactly its sizes,
    // which fit because submission refuses requests larger than the budget.
    bool admit(Req *q)
    {
        if (try_admit(q, false))
            return true;
        if (used != 0)
            return false;   // wait for in-flight work to return memory
        free_pool();
        return try_admit(q, true);
    }

    void free_req(Req *q)
    {
        release(q->buf_c64);
        release(q->buf_h16);
        release(q->exps);
        q->buf_c64 = q->buf_h16 = nullptr;
        q->exps = nullptr;
    }

    fft2d_plan_t plan(int rows, int cols, int dtype, int dir)
    {
        auto key = std::make_tuple(rows, cols, dtype, dir);
        auto it = plans.find(key);
        if (it != plans.end())
            return it->second;
        fft2d_plan_t p = nullptr;
        if (fft2d_plan(rows, cols, dtype, dir, &p) != FFT2D_OK)
            return nullptr;
        plans[key] = p;
        return p;
    }

    // ------------------------------------------------------------- launch
    fft2d_status launch(Batch &b)
    {
        fft2d::NvtxRange range("fft2d serve batch");
        cudaStream_t st = streams[b.stream];
        std::vector<Req *> c64, h16;
        for (Req *q : b.reqs)
            (q->r.dtype == FFT2D_C64 ? c64 : h16).push_back(q);
        for (Req *q : b.reqs) {
            const size_t px = (size_t)q->r.rows * q->r.cols;
            cudaError_t e;
            if (q->r.dtype == FFT2D_C64) {
                e = cudaMemcpyAsync(q->buf_c64, q->r.in, px * 8, cudaMemcpyHostToDevice, st);
            } else {
                e = cudaMemcpyAsync(q->buf_h16, q->r.in, px * 4, cudaMemcpyHostToDevice, st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(q->exps, q->r.in_exp, (size_t)q->r.rows * 4,
                                        cudaMemcpyHostToDevice, st);
            }
            if (e != cudaSuccess)
                return FFT2D_ERR_CUDA;
        }
        // forward: complex64 through fft2d_exec_batched, half2 grouped
        std::vector<fft2d_plan_t> fp;
        std::vector<const void *> fin;
        std::vector<void *> fout;
        for (Req *q : c64) {
            fft2d_plan_t p = plan(q->r.rows, q->r.cols, FFT2D_C64, FFT2D_FORWARD);
            if (!p)
                return FFT2D_ERR_OOM;
            fp.push_back(p);
            fin.push_back(q->buf_c64);
            fout.push_back(q->buf_c64);
        }
        fft2d_status s = FFT2D_OK;
        if (!fp.empty())
            s = fft2d_exec_batched((int)fp.size(), fp.data(), fin.data(), fout.data(), st);
        if (s != FFT2D_OK)
            return s;
        std::vector<fft2d_plan_t> hp;
        for (Req *q : h16) {
            fft2d_plan_t p = plan(q->r.rows, q->r.cols, FFT2D_C32H, FFT2D_FORWARD);
            if (!p)
                return FFT2D_ERR_OOM;
            hp.push_back(p);
        }
        if (!h16.empty() && h16_phase(h16, hp, FFT2D_PASS_ROWS, st) != cudaSuccess)
            return FFT2D_ERR_CUDA;
        // low-pass, then the inverse of the filtered spectra
        std::vector<fft2d_plan_t> ip;
        std::vector<const void *> iin;
        std::vector<void *> iout;
        for (Req *q : c64) {
            if (q->r.op != FFT2D_OP_LOWPASS)
                continue;
            if (fft2d::launch_lowpass(false, q->buf_c64, q->r.rows, q->r.cols,
                                      q->r.rows / 8.0f, q->r.cols / 8.0f, st) != cudaSuccess)
                return FFT2D_ERR_CUDA;
            fft2d_plan_t p = plan(q->r.rows, q->r.cols, FFT2D_C64, FFT2D_INVERSE);
            if (!p)
                return FFT2D_ERR_OOM;
            ip.push_back(p);
            iin.push_back(q->buf_c64);
            iout.push_back(q->buf_c64);
        }
        if (!ip.empty())
            s = fft2d_exec_batched((int)ip.size(), ip.data(), iin.data(), iout.data(), st);
        if (s != FFT2D_OK)
            return s;
        std::vector<Req *> h16f;
        std::vector<fft2d_plan_t> hip;
        for (Req *q : h16) {
            if (q->r.op != FFT2D_OP_LOWPASS)
                continue;
            const int R = q->r.rows, C = q->r.cols;
            if (fft2d::launch_lowpass(true, q->buf_h16, R, C, R / 8.0f, C / 8.0f, st) !=
                cudaSuccess)
                return FFT2D_ERR_CUDA;
            fft2d_plan_t p = plan(R, C, FFT2D_C32H, FFT2D_INVERSE);
            if (!p)
                return FFT2D_ERR_OOM;
            h16f.push_back(q);
            hip.push_back(p);
        }
        // the inverse reads the spectrum's per-column exponents and writes
        // new per-column exponents into the same vector
        if (!h16f.empty() && h16_phase(h16f, hip, FFT2D_PASS_COLS, st) != cudaSuccess)
            return FFT2D_ERR_CUDA;
        for (Req *q : b.reqs) {
            const size_t px = (size_t)q->r.rows * q->r.cols;
            cudaError_t e;
            if (q->r.dtype == FFT2D_C64) {
                e = cudaMemcpyAsync(q->r.out, q->buf_c64, px * 8, cudaMemcpyDeviceToHost, st);
            } else {
                e = cudaMemcpyAsync(q->r.out, q->buf_h16, px * 4, cudaMemcpyDeviceToHost, st);
                if (e == cudaSuccess)
                    e = cudaMemcpyAsync(q->r.out_exp, q->exps + 2 * q->r.rows,
                                        (size_t)q->r.cols * 4, cudaMemcpyDeviceToHost, st);
            }
            if (e != cudaSuccess)
                return FFT2D_ERR_CUDA;
        }
        if (cudaEventRecord(b.ev, st) != cudaSuccess)
            return FFT2D_ERR_CUDA;
        return FFT2D_OK;
    }

    // Modelled device time of a batch in simulation mode: 2 us per request
    // plus 1 ns per byte moved.
    static Clock::duration sim_time(const Batch &b)
    {
        double us = 0;
        for (const Req *q : b.reqs)
            us += 2.0 + (double)q->bytes * 1e-3;
        return std::chrono::microseconds((long long)us);
    }

    // ------------------------------------------------------------- loop
    void complete(Batch &b, fft2d_status s)
    {
        const auto now = Clock::now();
        for (Req *q : b.reqs) {
            q->t_done = now;
            q->status = s;
            q->done = true;
            free_req(q);
            latencies_ms.push_back(
                std::chrono::duration<double, std::milli>(now - q->t_submit).count());
        }
        last_done = now;
        stream_busy[b.stream] = false;
        if (b.ev)
            cudaEventDestroy(b.ev);
        b.ev = nullptr;
    }

    void run()
    {
        if (!simulate)
            cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            // 1. retire finished batches
            bool progressed = false;
            for (size_t i = 0; i < inflight.size();) {
                Batch &b = inflight[i];
                bool fin;
                if (simulate)
                    fin = Clock::now() >= b.sim_ready;
                else
                    fin = cudaEventQuery(b.ev) != cudaErrorNotReady;
                if (fin) {
                    const fft2d_status s =
                        simulate || cudaEventQuery(b.ev) == cudaSuccess ? FFT2D_OK : FFT2D_ERR_CUDA;
                    complete(b, s);
                    inflight.erase(inflight.begin() + i);
                    progressed = true;
                } else {
                    i++;
                }
            }
            if (progressed)
                cv_done.notify_all();
            // 2. admit and launch on an idle stream
            int idle = -1;
            for (int k = 0; k < nstreams; k++)
                if (!stream_busy[k]) {
                    idle = k;
                    break;
                }
            if (idle >= 0 && !queue.empty()) {
                Batch b;
                b.stream = idle;
                while (!queue.empty() && b.reqs.size() < 128) {
                    Req *q = queue.front();
                    if (!admit(q))
                        break;   // wait for memory; keep arrival order
                    queue.pop_front();
                    b.reqs.push_back(q);
                }
                if (!b.reqs.empty()) {
                    stream_busy[idle] = true;
                    batches++;
                    batched_reqs += (long long)b.reqs.size();
                    fft2d_status s = FFT2D_OK;
                    if (simulate) {
                        b.sim_ready = Clock::now() + sim_time(b);
                    } else if (cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming) !=
                               cudaSuccess) {
                        s = FFT2D_ERR_CUDA;
                    } else {
                        lk.unlock();   // launches need no lock: buffers are owned
                        s = launch(b);
                        lk.lock();
                    }
                    if (s != FFT2D_OK) {
                        if (b.ev)
                            cudaStreamSynchronize(streams[b.stream]);
                        complete(b, s);
                        cv_done.notify_all();
                    } else {
                        inflight.push_back(b);
                    }
                    continue;
                }
            }
            if (stopping && queue.empty() && inflight.empty())
                break;
            // 3. wait for new work or poll the device again shortly
            cv_work.wait_for(lk, std::chrono::microseconds(inflight.empty() ? 1000 : 20));
        }
    }
};

extern "C" {

fft2d_status fft2d_serve_create(size_t hbm_budget_bytes, int streams, int flags,
                                fft2d_server_t *out)
{
    if (!out || hbm_budget_bytes == 0 || streams < 1 || streams > 16)
        return FFT2D_ERR_ARG;
    *out = nullptr;
    fft2d_server_s *s = new (std::nothrow) fft2d_server_s();
    if (!s)
        return FFT2D_ERR_OOM;
    s->budget = hbm_budget_bytes;
    s->nstreams = streams;
    s->simulate = (flags & FFT2D_SERVE_SIMULATE) != 0;
    s->streams.assign(streams, nullptr);
    s->stream_busy.assign(streams, false);
    if (!s->simulate) {
        if (cudaGetDevice(&s->device) != cudaSuccess) {
            delete s;
            return FFT2D_ERR_CUDA;
        }
        for (int k = 0; k < streams; k++) {
            if (cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking) != cudaSuccess) {
                for (int j = 0; j < k; j++)
                    cudaStreamDestroy(s->streams[j]);
                delete s;
                return FFT2D_ERR_CUDA;
            }
        }
    }
    s->worker = std::thread([s] { s->run(); });
    *out = s;
    return FFT2D_OK;
}

fft2d_status fft2d_serve_submit(fft2d_server_t s, const fft2d_request *req,
                                unsigned long long *ticket)
{
    if (!s || !req || !ticket)
        return FFT2D_ERR_ARG;
    const fft2d_request &r = *req;
    if ((r.op != FFT2D_OP_FORWARD && r.op != FFT2D_OP_LOWPASS) || !r.in || !r.out ||
        (r.dtype != FFT2D_C64 && r.dtype != FFT2D_C32H))
        return FFT2D_ERR_ARG;
    if (!pow2(r.rows) || !pow2(r.cols))
        return FFT2D_ERR_NOT_POW2;
    if (r.rows > FFT2D_MAX_SIDE || r.cols > FFT2D_MAX_SIDE)
        return FFT2D_ERR_TOO_LARGE;
    if (r.dtype == FFT2D_C32H && (r.rows < 2 || r.cols < 2))
        return FFT2D_ERR_UNSUPPORTED;
    if (r.dtype == FFT2D_C32H && (!r.in_exp || !r.out_exp))
        return FFT2D_ERR_ARG;
    Req *q = new (std::nothrow) Req();
    if (!q)
        return FFT2D_ERR_OOM;
    q->r = r;
    q->bytes = request_bytes(r);
    q->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        // a request larger than the whole budget could never be admitted
        if (q->bytes > s->budget) {
            s->rejected++;
            delete q;
            return FFT2D_ERR_BUDGET;
        }
        if (!s->any_submit) {
            s->first_submit = q->t_submit;
            s->any_submit = true;
        }
        q->ticket = s->next_ticket++;
        s->all[q->ticket] = q;
        s->queue.push_back(q);
        *ticket = q->ticket;
    }
    s->cv_work.notify_one();
    return FFT2D_OK;
}

fft2d_status fft2d_serve_wait(fft2d_server_t s, unsigned long long ticket, int timeout_ms,
                              double *latency_ms)
{
    if (!s)
        return FFT2D_ERR_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end())
        return FFT2D_ERR_ARG;
    Req *q = it->second;
    const auto pred = [q] { return q->done; };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, pred);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
        return FFT2D_ERR_TIMEOUT;
    if (latency_ms)
        *latency_ms = std::chrono::duration<double, std::milli>(q->t_done - q->t_submit).count();
    const fft2d_status st = q->status;
    s->all.erase(it);
    delete q;
    return st;
}

fft2d_status fft2d_serve_stats_get(fft2d_server_t s, fft2d_serve_stats *out)
{
    if (!s || !out)
        return FFT2D_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof *out);
    std::vector<double> v = s->latencies_ms;
    out->completed = (long long)v.size();
    out->rejected = s->rejected;
    out->submitted = (long long)(s->next_ticket - 1) + s->rejected;
    out->queued = (long long)s->queue.size();
    out->peak_device_bytes = (long long)s->peak;
    out->batches = s->batches;
    out->mean_batch_size = s->batches ? (double)s->batched_reqs / (double)s->batches : 0.0;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto pct = [&v](double p) {
            const size_t i = (size_t)std::min((double)v.size() - 1, p * (double)(v.size() - 1) + 0.5);
            return v[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = v.back();
        double sum = 0;
        for (double x : v)
            sum += x;
        out->mean_ms = sum / (double)v.size();
        const double span =
            std::chrono::duration<double>(s->last_done - s->first_submit).count();
        out->throughput_rps = span > 0 ? (double)v.size() / span : 0.0;
    }
    return FFT2D_OK;
}

fft2d_status fft2d_serve_destroy(fft2d_server_t s)
{
    if (!s)
        return FFT2D_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable())
        s->worker.join();
    for (auto &kv : s->all)
        delete kv.second;
    s->free_pool();
    for (auto &kv : s->plans)
        fft2d_destroy(kv.second);
    if (!s->simulate)
        for (cudaStream_t st : s->streams)
            if (st)
                cudaStreamDestroy(st);
    delete s;
    return FFT2D_OK;
}

}  // extern "C"
