// cg_stream.cu -- streaming server: pinned host rings, continuous batching
// across instrument streams under a device-memory budget, running averages
// on the device, in-order result delivery with latency statistics.
//
// Paper ("Data Capture and Processing"): the digitiser streams into a ring
// buffer in host memory, the GPU processes batches asynchronously, finished
// batches are sorted back into time order, and the ring overflows if the
// production rate exceeds the consumption rate.  One scheduler thread per
// server drives every stream: it harvests finished batches (CUDA events),
// admits streams whose batch buffers fit the budget, and launches a batch
// whenever a stream has frames waiting and a free batch buffer.  Each batch
// buffer owns a CUDA stream, so copies and kernels of different batches and
// different instruments overlap on the device.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "cg_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s()
{
    return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

cg_status sfail(cg_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    cg::set_last_error(buf);
    return st;
}

// Latency histogram: logarithmic bins 1 % wide from 100 ns to 1000 s.
struct LatencyHist {
    static constexpr double kLo = 1e-7;
    static constexpr double kLogRatio = 0.00995033085316809;   // ln(1.01)
    std::vector<int64_t> bins = std::vector<int64_t>(2400, 0);
    int64_t n = 0;
    double maxv = 0;
    void add(double v)
    {
        int b = 0;
        if (v > kLo) b = static_cast<int>(std::log(v / kLo) / kLogRatio) + 1;
        if (b >= static_cast<int>(bins.size())) b = static_cast<int>(bins.size()) - 1;
        ++bins[b];
        ++n;
        maxv = std::max(maxv, v);
    }
    // upper edge of the bin holding the q-quantile
    double quantile(double q) const
    {
        if (n == 0) return 0;
        const int64_t want = static_cast<int64_t>(std::ceil(q * static_cast<double>(n)));
        int64_t acc = 0;
        for (size_t b = 0; b < bins.size(); ++b) {
            acc += bins[b];
            if (acc >= want) return b == 0 ? kLo : std::min(maxv, kLo * std::exp(kLogRatio * static_cast<double>(b)));
        }
        return maxv;
    }
};

// One device batch buffer: its CUDA stream, completion event, device outputs
// and pinned host staging of the results.
struct Batch {
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    int16_t* d_frames = nullptr;
    float *d_amps = nullptr, *d_params = nullptr, *d_rss = nullptr;
    int16_t *d_iters = nullptr, *d_status = nullptr;
    float *h_amps = nullptr, *h_params = nullptr, *h_rss = nullptr;
    int16_t *h_iters = nullptr, *h_status = nullptr;
    int64_t first = 0;   // ordinal of the batch's first frame
    int m = 0;
    bool done = false;
};

constexpr int kMinBuffers = 2;
constexpr int kMaxBuffers = 4;
constexpr double kDrainTimeoutS = 30.0;

// FP64 sums of y_k = amps_k / ref_k (k < T), of the four parameters and of
// the frame count over converged frames, per running-average window; a batch
// spans at most two windows, accumulated into slots (window & 1).
__global__ void __launch_bounds__(256) window_sum_kernel(const float* __restrict__ amps,
                                                          const float* __restrict__ inv_ref,
                                                          const float* __restrict__ params,
                                                          const int16_t* __restrict__ status, int m, int T,
                                                          int64_t ord0, int64_t W, double* __restrict__ acc)
{
    __shared__ double red[2][256];
    const int j = blockIdx.x;   // column: y_k (k < T), parameter (T..T+3), count (T+4)
    const int64_t w0 = ord0 / W;
    double s0 = 0.0, s1 = 0.0;
    for (int f = threadIdx.x; f < m; f += blockDim.x) {
        if ((status[f] & 3) != 0) continue;
        double v;
        if (j < T)
            v = static_cast<double>(amps[static_cast<int64_t>(f) * T + j]) * static_cast<double>(inv_ref[j]);
        else if (j < T + 4)
            v = static_cast<double>(params[static_cast<int64_t>(f) * 4 + (j - T)]);
        else
            v = 1.0;
        if ((ord0 + f) / W == w0)
            s0 += v;
        else
            s1 += v;
    }
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            red[0][threadIdx.x] += red[0][threadIdx.x + w];
            red[1][threadIdx.x] += red[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int cols = T + 5;
        atomicAdd(&acc[(w0 & 1) * cols + j], red[0][0]);
        if (red[1][0] != 0.0) atomicAdd(&acc[((w0 + 1) & 1) * cols + j], red[1][0]);
    }
}

}  // namespace

struct cg_server_s;

struct cg_stream_s {
    cg_server_s* srv = nullptr;
    cg_plan_s* plan = nullptr;
    int N = 0, T = 0, batch = 0;
    double max_delay = 0;
    int64_t W = 0;
    // ring of C frames (pinned) with per-frame metadata and result slots;
    // ordinals grow without bound, position = ordinal % C
    int64_t C = 0;
    int16_t* ring = nullptr;
    std::vector<uint64_t> seq;
    std::vector<double> t_arr;
    std::vector<cg_result> res;
    std::vector<float> res_amps;
    // guarded by mu
    int64_t head = 0;     // next ordinal pushed
    int64_t ready = 0;    // results ready below this ordinal
    int64_t tail = 0;     // next ordinal polled
    bool flush = false;
    cg_status err = CG_OK;
    std::string err_msg;
    int64_t pushed = 0, dropped = 0, done = 0, polled = 0, batches = 0;
    double t_first_push = -1, t_last_done = 0;
    int64_t bytes_done = 0;
    LatencyHist hist;
    int64_t last_win = -1, last_win_count = 0;
    std::vector<double> last_mean_y, last_mean_p;
    bool admitted = false;
    std::mutex mu;
    std::condition_variable cv;
    // scheduler thread only
    int64_t sched = 0;
    std::deque<Batch*> inflight;
    std::vector<Batch*> buffers, free_bufs;
    size_t buf_bytes = 0;
    double* d_acc = nullptr;     // [2][T + 5]
    cudaStream_t aux = nullptr;
    int64_t win_next = 0;                 // next window to harvest
    std::deque<int64_t> win_frames;       // frames completed in windows win_next, win_next + 1, ...
    // destruction handshake
    std::atomic<bool> destroying{false};
    std::atomic<bool> dead{false};
};

struct cg_server_s {
    int device = 0;
    size_t budget = 0, used = 0;
    std::vector<cg_stream_s*> streams;
    std::mutex mu;
    std::condition_variable cv;     // wakes the scheduler
    std::condition_variable cv_dead;
    std::thread th;
    std::atomic<bool> stop{false};
    std::atomic<double> throttle{0.0};
    std::atomic<bool> hold{false};
    std::atomic<int> fail_launch{0};
};

namespace {

void set_err(cg_stream_s* st, cg_status e, const std::string& msg)
{
    std::lock_guard<std::mutex> lk(st->mu);
    if (st->err == CG_OK) {
        st->err = e;
        st->err_msg = msg;
    }
    st->cv.notify_all();
}

void free_batch(Batch* b)
{
    if (!b) return;
    if (b->cs) cudaStreamSynchronize(b->cs);
    cudaFree(b->d_frames);
    cudaFree(b->d_amps);
    cudaFree(b->d_params);
    cudaFree(b->d_rss);
    cudaFree(b->d_iters);
    cudaFree(b->d_status);
    cudaFreeHost(b->h_amps);
    cudaFreeHost(b->h_params);
    cudaFreeHost(b->h_rss);
    cudaFreeHost(b->h_iters);
    cudaFreeHost(b->h_status);
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->cs) cudaStreamDestroy(b->cs);
    delete b;
}

size_t batch_device_bytes(int m, int N, int T)
{
    return static_cast<size_t>(m) * (2 * static_cast<size_t>(N) + 4 * static_cast<size_t>(T) + 16 + 4 + 2 + 2);
}

Batch* alloc_batch(int m, int N, int T)
{
    Batch* b = new (std::nothrow) Batch;
    if (!b) return nullptr;
    const size_t M = static_cast<size_t>(m);
    bool ok = cudaStreamCreateWithFlags(&b->cs, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc(&b->d_frames, M * N * 2) == cudaSuccess && cudaMalloc(&b->d_amps, M * T * 4) == cudaSuccess &&
              cudaMalloc(&b->d_params, M * 16) == cudaSuccess && cudaMalloc(&b->d_rss, M * 4) == cudaSuccess &&
              cudaMalloc(&b->d_iters, M * 2) == cudaSuccess && cudaMalloc(&b->d_status, M * 2) == cudaSuccess &&
              cudaMallocHost(&b->h_amps, M * T * 4) == cudaSuccess && cudaMallocHost(&b->h_params, M * 16) == cudaSuccess &&
              cudaMallocHost(&b->h_rss, M * 4) == cudaSuccess && cudaMallocHost(&b->h_iters, M * 2) == cudaSuccess &&
              cudaMallocHost(&b->h_status, M * 2) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_batch(b);
        return nullptr;
    }
    return b;
}

// Grants batch buffers from the budget: kMinBuffers to admit, then one more
// at a time (up to kMaxBuffers) while the stream has a backlog.
bool grant_buffers(cg_server_s* s, cg_stream_s* st)
{
    const int have = static_cast<int>(st->buffers.size());
    if (have >= kMaxBuffers) return false;
    int want;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (have == 0) {
            if (s->used + kMinBuffers * st->buf_bytes > s->budget) return false;
            want = kMinBuffers;
        } else {
            if (s->used + st->buf_bytes > s->budget) return false;
            want = 1;
        }
        s->used += want * st->buf_bytes;
    }
    int got = 0;
    for (; got < want; ++got) {
        Batch* b = alloc_batch(st->batch, st->N, st->T);
        if (!b) break;
        st->buffers.push_back(b);
        st->free_bufs.push_back(b);
    }
    if (got < want) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->used -= (want - got) * st->buf_bytes;
    }
    if (have == 0 && got < kMinBuffers) {
        for (Batch* b : st->buffers) free_batch(b);
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->used -= got * st->buf_bytes;
        }
        st->buffers.clear();
        st->free_bufs.clear();
        set_err(st, CG_ERR_NOMEM, "device allocation of the batch buffers failed");
        return false;
    }
    if (have == 0) {
        std::lock_guard<std::mutex> lk(st->mu);
        st->admitted = true;
    }
    return got > 0;
}

// Finished batches: results into the ring's result slots, window sums, and
// the in-order prefix made ready for polling.
bool harvest(cg_server_s* s, cg_stream_s* st)
{
    if (s->hold.load()) return false;
    bool progress = false;
    for (Batch* b : st->inflight) {
        if (b->done) continue;
        const cudaError_t q = cudaEventQuery(b->ev);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) {
            set_err(st, CG_ERR_CUDA, std::string("batch failed: ") + cudaGetErrorString(q));
            return progress;
        }
        const int64_t C = st->C;
        nvtxRangePushA("cg stream: deliver");
        for (int i = 0; i < b->m; ++i) {
            const int64_t pos = (b->first + i) % C;
            cg_result& r = st->res[pos];
            r.seq = st->seq[pos];
            r.t_arrival = st->t_arr[pos];
            std::memcpy(r.params, b->h_params + 4 * i, 16);
            r.rss = b->h_rss[i];
            r.iters = b->h_iters[i];
            r.status = b->h_status[i];
        }
        for (int i = 0; i < b->m; ++i) {
            const int64_t pos = (b->first + i) % C;
            std::memcpy(&st->res_amps[pos * st->T], b->h_amps + static_cast<size_t>(i) * st->T, 4 * st->T);
        }
        nvtxRangePop();
        // running-average windows touched by this batch
        const int64_t w0 = b->first / st->W, w1 = (b->first + b->m - 1) / st->W;
        for (int64_t w = w0; w <= w1; ++w) {
            const int64_t lo = std::max(b->first, w * st->W), hi = std::min(b->first + b->m, (w + 1) * st->W);
            const int64_t k = w - st->win_next;
            while (static_cast<int64_t>(st->win_frames.size()) <= k) st->win_frames.push_back(0);
            st->win_frames[k] += hi - lo;
        }
        b->done = true;
        progress = true;
    }
    // complete windows, in order: read the slot's sums, then clear it
    while (!st->win_frames.empty() && st->win_frames.front() == st->W) {
        const int cols = st->T + 5;
        std::vector<double> h(cols);
        double* slot = st->d_acc + (st->win_next & 1) * cols;
        cudaError_t e = cudaMemcpyAsync(h.data(), slot, sizeof(double) * cols, cudaMemcpyDeviceToHost, st->aux);
        if (e == cudaSuccess) e = cudaMemsetAsync(slot, 0, sizeof(double) * cols, st->aux);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st->aux);
        if (e != cudaSuccess) {
            set_err(st, CG_ERR_CUDA, std::string("running averages: ") + cudaGetErrorString(e));
            return progress;
        }
        {
            std::lock_guard<std::mutex> lk(st->mu);
            const double cnt = h[cols - 1];
            st->last_win = st->win_next;
            st->last_win_count = static_cast<int64_t>(cnt);
            st->last_mean_y.assign(st->T, NAN);
            st->last_mean_p.assign(4, NAN);
            if (cnt > 0) {
                for (int k = 0; k < st->T; ++k) st->last_mean_y[k] = h[k] / cnt;
                for (int k = 0; k < 4; ++k) st->last_mean_p[k] = h[st->T + k] / cnt;
            }
        }
        st->win_frames.pop_front();
        ++st->win_next;
        progress = true;
    }
    // in-order prefix of finished batches becomes ready
    while (!st->inflight.empty() && st->inflight.front()->done) {
        Batch* b = st->inflight.front();
        st->inflight.pop_front();
        const double t = now_s();
        {
            std::lock_guard<std::mutex> lk(st->mu);
            for (int i = 0; i < b->m; ++i) {
                cg_result& r = st->res[(b->first + i) % st->C];
                r.t_done = t;
                st->hist.add(t - r.t_arrival);
            }
            st->ready = b->first + b->m;
            st->done += b->m;
            st->batches += 1;
            st->bytes_done += static_cast<int64_t>(b->m) * st->N * 2;
            st->t_last_done = t;
        }
        st->cv.notify_all();
        b->done = false;
        st->free_bufs.push_back(b);
        progress = true;
    }
    return progress;
}

// Launches batches while frames wait and batch buffers are free.
bool launch(cg_server_s* s, cg_stream_s* st)
{
    bool progress = false;
    while (!st->free_bufs.empty()) {
        int64_t avail;
        bool flush;
        double t_oldest = 0;
        {
            std::lock_guard<std::mutex> lk(st->mu);
            if (st->err != CG_OK) return progress;
            avail = st->head - st->sched;
            flush = st->flush;
            if (avail > 0) t_oldest = st->t_arr[st->sched % st->C];
        }
        if (avail <= 0) break;
        int64_t m = std::min<int64_t>(avail, st->batch);
        // a batch spans at most two running-average windows, and the window
        // two ahead of the oldest unharvested one must not be touched yet
        const int64_t w_first = st->sched / st->W;
        m = std::min<int64_t>(m, (w_first + 2) * st->W - st->sched);
        const int64_t w_last = (st->sched + m - 1) / st->W;
        if (w_last > st->win_next + 1) break;
        if (m < st->batch && !flush && now_s() - t_oldest < st->max_delay) break;
        const double thr = s->throttle.load();
        if (thr > 0) std::this_thread::sleep_for(std::chrono::duration<double>(thr));
        int inj = s->fail_launch.load();
        while (inj > 0 && !s->fail_launch.compare_exchange_weak(inj, inj - 1)) {
        }
        if (inj > 0) {
            set_err(st, CG_ERR_CUDA, "batch launch failed (injected)");
            return progress;
        }
        Batch* b = st->free_bufs.back();
        st->free_bufs.pop_back();
        b->first = st->sched;
        b->m = static_cast<int>(m);
        b->done = false;
        const int N = st->N, T = st->T;
        const int64_t pos = st->sched % st->C;
        const int64_t n1 = std::min<int64_t>(m, st->C - pos);
        // NVTX ranges mark the scheduler's stages on the host timeline (a
        // profiler shows them; without one they cost a function call)
        nvtxRangePushA("cg stream: copy frames");
        cudaError_t e = cudaMemcpyAsync(b->d_frames, st->ring + pos * N, static_cast<size_t>(n1) * N * 2,
                                        cudaMemcpyHostToDevice, b->cs);
        if (e == cudaSuccess && m > n1)
            e = cudaMemcpyAsync(b->d_frames + n1 * N, st->ring, static_cast<size_t>(m - n1) * N * 2,
                                cudaMemcpyHostToDevice, b->cs);
        nvtxRangePop();
        if (e != cudaSuccess) {
            set_err(st, CG_ERR_CUDA, std::string("frame copy: ") + cudaGetErrorString(e));
            return progress;
        }
        nvtxRangePushA("cg stream: process");
        const cg_status ps = cg_process(st->plan, b->d_frames, m, b->d_amps, nullptr, b->d_params, b->d_rss,
                                        b->d_iters, b->d_status, b->cs);
        if (ps != CG_OK) {
            nvtxRangePop();
            set_err(st, ps, std::string("cg_process: ") + cg_last_error());
            return progress;
        }
        window_sum_kernel<<<T + 5, 256, 0, b->cs>>>(b->d_amps, st->plan->d.inv_ref, b->d_params, b->d_status,
                                                    static_cast<int>(m), T, st->sched, st->W, st->d_acc);
        e = cudaGetLastError();
        nvtxRangePop();
        nvtxRangePushA("cg stream: copy results");
        const size_t M = static_cast<size_t>(m);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_params, b->d_params, M * 16, cudaMemcpyDeviceToHost, b->cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_rss, b->d_rss, M * 4, cudaMemcpyDeviceToHost, b->cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_iters, b->d_iters, M * 2, cudaMemcpyDeviceToHost, b->cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_status, b->d_status, M * 2, cudaMemcpyDeviceToHost, b->cs);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->h_amps, b->d_amps, M * T * 4, cudaMemcpyDeviceToHost, b->cs);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev, b->cs);
        nvtxRangePop();
        if (e != cudaSuccess) {
            set_err(st, CG_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
            return progress;
        }
        st->sched += m;
        st->inflight.push_back(b);
        progress = true;
    }
    return progress;
}

// Waits (bounded) for a stream's batches and frees its device resources.
void retire(cg_server_s* s, cg_stream_s* st)
{
    const double t_end = now_s() + kDrainTimeoutS;
    for (Batch* b : st->inflight)
        while (cudaEventQuery(b->ev) == cudaErrorNotReady && now_s() < t_end)
            std::this_thread::sleep_for(std::chrono::microseconds(100));
    st->inflight.clear();
    for (Batch* b : st->buffers) free_batch(b);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->used -= st->buffers.size() * st->buf_bytes;
    }
    st->buffers.clear();
    st->free_bufs.clear();
    if (st->aux) cudaStreamSynchronize(st->aux);
    cudaFree(st->d_acc);
    st->d_acc = nullptr;
    if (st->aux) cudaStreamDestroy(st->aux);
    st->aux = nullptr;
}

void scheduler(cg_server_s* s)
{
    cudaSetDevice(s->device);
    while (!s->stop.load()) {
        std::vector<cg_stream_s*> list;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            list = s->streams;
        }
        bool progress = false, busy = false;
        for (cg_stream_s* st : list) {
            if (st->destroying.load()) {
                retire(s, st);
                {
                    std::lock_guard<std::mutex> lk(s->mu);
                    s->streams.erase(std::find(s->streams.begin(), s->streams.end(), st));
                    st->dead.store(true);
                }
                s->cv_dead.notify_all();
                progress = true;
                continue;
            }
            if (st->buffers.empty() || (st->free_bufs.empty() && st->buffers.size() < kMaxBuffers)) {
                int64_t backlog;
                {
                    std::lock_guard<std::mutex> lk(st->mu);
                    backlog = st->head - st->sched;
                }
                if (st->buffers.empty() || backlog >= st->batch) progress |= grant_buffers(s, st);
            }
            progress |= harvest(s, st);
            progress |= launch(s, st);
            busy |= !st->inflight.empty();
        }
        if (!progress) {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop.load()) break;
            // batches in flight: poll their events often; otherwise sleep
            // until a push, flush, create or destroy wakes the scheduler
            s->cv.wait_for(lk, busy ? std::chrono::microseconds(20) : std::chrono::microseconds(500));
        }
    }
    std::vector<cg_stream_s*> rest;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        rest = s->streams;
    }
    for (cg_stream_s* st : rest) retire(s, st);
}

void wake(cg_server_s* s)
{
    std::lock_guard<std::mutex> lk(s->mu);
    s->cv.notify_all();
}

}  // namespace

extern "C" {

double cg_clock(void) { return now_s(); }

cg_status cg_server_create(cg_server_t* out, size_t budget)
{
    if (!out) return sfail(CG_ERR_ARG, "server is NULL");
    *out = nullptr;
    if (budget == 0) return sfail(CG_ERR_ARG, "device_budget_bytes must be > 0");
    cg_server_s* s = new (std::nothrow) cg_server_s;
    if (!s) return sfail(CG_ERR_NOMEM, "host allocation failed");
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return sfail(CG_ERR_CUDA, "no CUDA device");
    }
    s->budget = budget;
    try {
        s->th = std::thread(scheduler, s);
    } catch (...) {
        delete s;
        return sfail(CG_ERR_NOMEM, "cannot start the scheduler thread");
    }
    *out = s;
    return CG_OK;
}

cg_status cg_server_destroy(cg_server_t s)
{
    if (!s) return CG_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop.store(true);
        s->cv.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    for (cg_stream_s* st : s->streams) {
        if (st->ring) cudaFreeHost(st->ring);
        delete st;
    }
    delete s;
    return CG_OK;
}

cg_status cg_server_inject(cg_server_t s, int what, double value)
{
    if (!s) return sfail(CG_ERR_ARG, "server is NULL");
    switch (what) {
    case CG_INJECT_THROTTLE_S: s->throttle.store(value > 0 ? value : 0.0); break;
    case CG_INJECT_HOLD: s->hold.store(value != 0.0); break;
    case CG_INJECT_FAIL_LAUNCH: s->fail_launch.store(value > 0 ? static_cast<int>(value) : 0); break;
    default: return sfail(CG_ERR_ARG, "unknown injection %d", what);
    }
    wake(s);
    return CG_OK;
}

cg_status cg_stream_create(cg_stream_t* out, cg_server_t s, cg_plan_t plan, size_t ring_bytes, int batch,
                           double max_delay, int64_t W)
{
    if (!out) return sfail(CG_ERR_ARG, "stream is NULL");
    *out = nullptr;
    if (!s || !plan) return sfail(CG_ERR_ARG, "server or plan is NULL");
    if (batch < 1 || batch > (1 << 24)) return sfail(CG_ERR_ARG, "batch_frames must be in [1, 2^24]");
    if (!(max_delay >= 0.0)) return sfail(CG_ERR_ARG, "max_delay_s must be >= 0");
    if (W < 1) return sfail(CG_ERR_ARG, "avg_window must be >= 1");
    if (plan->device != s->device) return sfail(CG_ERR_ARG, "plan and server are on different devices");
    const int N = plan->N, T = plan->T;
    const int64_t C = static_cast<int64_t>(ring_bytes / (2 * static_cast<size_t>(N)));
    if (C < 2 * static_cast<int64_t>(batch)) return sfail(CG_ERR_ARG, "ring_bytes must hold at least two batches");
    const size_t bb = batch_device_bytes(batch, N, T);
    if (kMinBuffers * bb > s->budget)
        return sfail(CG_ERR_UNSUPPORTED, "two batch buffers (%zu bytes) exceed the server budget", kMinBuffers * bb);
    cg_stream_s* st = new (std::nothrow) cg_stream_s;
    if (!st) return sfail(CG_ERR_NOMEM, "host allocation failed");
    st->srv = s;
    st->plan = plan;
    st->N = N;
    st->T = T;
    st->batch = batch;
    st->max_delay = max_delay;
    st->W = W;
    st->C = C;
    st->buf_bytes = bb;
    cudaError_t e = cudaMallocHost(&st->ring, static_cast<size_t>(C) * N * 2);
    if (e == cudaSuccess) e = cudaMalloc(&st->d_acc, sizeof(double) * 2 * (T + 5));
    if (e == cudaSuccess) e = cudaMemset(st->d_acc, 0, sizeof(double) * 2 * (T + 5));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st->aux, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        if (st->ring) cudaFreeHost(st->ring);
        cudaFree(st->d_acc);
        if (st->aux) cudaStreamDestroy(st->aux);
        delete st;
        return sfail(e == cudaErrorMemoryAllocation ? CG_ERR_NOMEM : CG_ERR_CUDA, "stream ring: %s",
                     cudaGetErrorString(e));
    }
    try {
        st->seq.resize(C);
        st->t_arr.resize(C);
        st->res.resize(C);
        st->res_amps.resize(static_cast<size_t>(C) * T);
    } catch (...) {
        cudaFreeHost(st->ring);
        cudaFree(st->d_acc);
        cudaStreamDestroy(st->aux);
        delete st;
        return sfail(CG_ERR_NOMEM, "host allocation failed");
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->streams.push_back(st);
        s->cv.notify_all();
    }
    *out = st;
    return CG_OK;
}

cg_status cg_stream_push(cg_stream_t st, const int16_t* frames, int64_t n, uint64_t first_seq, double t_arrival)
{
    if (!st) return sfail(CG_ERR_ARG, "stream is NULL");
    if (n < 0 || (n > 0 && !frames)) return sfail(CG_ERR_ARG, "bad frames / n");
    if (n == 0) return CG_OK;
    const double t = t_arrival < 0 ? now_s() : t_arrival;
    int64_t h;
    {
        std::lock_guard<std::mutex> lk(st->mu);
        if (st->err != CG_OK) return sfail(st->err, "stream failed earlier: %s", st->err_msg.c_str());
        if (n > st->C - (st->head - st->tail)) {
            st->dropped += n;
            return sfail(CG_ERR_OVERFLOW, "ring full: %lld frames dropped (%lld in total)",
                         static_cast<long long>(n), static_cast<long long>(st->dropped));
        }
        h = st->head;
    }
    // single producer: [head, head + n) is not visible to the scheduler yet
    const int N = st->N;
    const int64_t pos = h % st->C;
    const int64_t n1 = std::min<int64_t>(n, st->C - pos);
    std::memcpy(st->ring + pos * N, frames, static_cast<size_t>(n1) * N * 2);
    if (n > n1) std::memcpy(st->ring, frames + n1 * N, static_cast<size_t>(n - n1) * N * 2);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t p = (h + i) % st->C;
        st->seq[p] = first_seq + static_cast<uint64_t>(i);
        st->t_arr[p] = t;
    }
    {
        std::lock_guard<std::mutex> lk(st->mu);
        st->head += n;
        st->pushed += n;
        if (st->t_first_push < 0) st->t_first_push = t;
    }
    wake(st->srv);
    return CG_OK;
}

cg_status cg_stream_poll(cg_stream_t st, cg_result* recs, float* amps, int64_t cap, int64_t* n_out, double timeout)
{
    if (!st || !recs || !n_out) return sfail(CG_ERR_ARG, "NULL argument");
    *n_out = 0;
    if (cap < 1) return sfail(CG_ERR_ARG, "cap must be >= 1");
    std::unique_lock<std::mutex> lk(st->mu);
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(timeout > 0 ? timeout : 0.0));
    st->cv.wait_until(lk, deadline, [&] { return st->ready > st->tail || st->err != CG_OK; });
    const int64_t k = std::min<int64_t>(cap, st->ready - st->tail);
    for (int64_t i = 0; i < k; ++i) {
        const int64_t p = (st->tail + i) % st->C;
        recs[i] = st->res[p];
        if (amps) std::memcpy(amps + i * st->T, &st->res_amps[p * st->T], 4 * st->T);
    }
    st->tail += k;
    st->polled += k;
    *n_out = k;
    if (k > 0) return CG_OK;
    if (st->err != CG_OK) return sfail(st->err, "stream failed: %s", st->err_msg.c_str());
    return sfail(CG_ERR_TIMEOUT, "no result within %.3f s", timeout);
}

cg_status cg_stream_flush(cg_stream_t st, double timeout)
{
    if (!st) return sfail(CG_ERR_ARG, "stream is NULL");
    int64_t target;
    {
        std::lock_guard<std::mutex> lk(st->mu);
        st->flush = true;
        target = st->head;
    }
    wake(st->srv);
    std::unique_lock<std::mutex> lk(st->mu);
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(timeout > 0 ? timeout : 0.0));
    const bool ok = st->cv.wait_until(lk, deadline, [&] { return st->ready >= target || st->err != CG_OK; });
    st->flush = false;
    if (st->err != CG_OK) return sfail(st->err, "stream failed: %s", st->err_msg.c_str());
    if (!ok) return sfail(CG_ERR_TIMEOUT, "flush did not complete within %.3f s", timeout);
    return CG_OK;
}

cg_status cg_stream_stats(cg_stream_t st, cg_stream_stats_t* o)
{
    if (!st || !o) return sfail(CG_ERR_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(st->mu);
    o->frames_pushed = st->pushed;
    o->frames_dropped = st->dropped;
    o->frames_done = st->done;
    o->frames_polled = st->polled;
    o->batches = st->batches;
    o->latency_p50_s = st->hist.quantile(0.50);
    o->latency_p99_s = st->hist.quantile(0.99);
    o->latency_max_s = st->hist.maxv;
    const double span = st->t_last_done - st->t_first_push;
    o->input_bytes_per_s = (span > 0 && st->t_first_push >= 0) ? static_cast<double>(st->bytes_done) / span : 0.0;
    o->admitted = st->admitted ? 1 : 0;
    o->window_index = st->last_win;
    o->window_frames = st->last_win_count;
    return CG_OK;
}

cg_status cg_stream_window(cg_stream_t st, int64_t* index, int64_t* count, double* mean_y, double* mean_p)
{
    if (!st) return sfail(CG_ERR_ARG, "stream is NULL");
    std::lock_guard<std::mutex> lk(st->mu);
    if (index) *index = st->last_win;
    if (count) *count = st->last_win_count;
    if (st->last_win >= 0) {
        if (mean_y) std::memcpy(mean_y, st->last_mean_y.data(), sizeof(double) * st->T);
        if (mean_p) std::memcpy(mean_p, st->last_mean_p.data(), sizeof(double) * 4);
    }
    return CG_OK;
}

cg_status cg_stream_destroy(cg_stream_t st)
{
    if (!st) return CG_OK;
    cg_server_s* s = st->srv;
    st->destroying.store(true);
    {
        std::unique_lock<std::mutex> lk(s->mu);
        s->cv.notify_all();
        const bool ok = s->cv_dead.wait_for(lk, std::chrono::duration<double>(kDrainTimeoutS + 5.0),
                                            [&] { return st->dead.load() || s->stop.load(); });
        if (!ok) return sfail(CG_ERR_TIMEOUT, "the scheduler did not release the stream in time");
        if (!st->dead.load()) return CG_OK;   // server stopping: it frees the stream
    }
    cudaFreeHost(st->ring);
    delete st;
    return CG_OK;
}

}  // extern "C"
