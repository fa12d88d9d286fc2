// hb_serve.cu -- continuous-batching server for many concurrent video streams (an
// extension around the estimator; the paper processes one frame at a time).
//
// A persistent request-loop thread takes frames in arrival order from all open streams,
// packs as many as fit (up to max_batch frames and the batch's low-pass capacity) into a
// batch of mixed sizes and level counts, and enqueues the whole batch on one of two
// CUDA streams: host->device copies of the frames, one batched analysis launch (a job
// table maps CTAs to frames), one posterior launch over the low-pass pixels of all
// frames, one batched synthesis launch, device->host copies of THb and SO2, and a host
// callback that marks the frames done.  While one batch is on the GPU the loop builds
// and enqueues the next on another stream (kBatchSlots batches in flight), so consecutive
// batches overlap on the device and frames that arrive meanwhile join the next batch as
// soon as a batch slot frees.  Every stream owns a ring of frame slots (pinned host and device buffers)
// allocated at open time against the server's device-memory budget; the operator and
// grid constants are shared by all streams and stay resident.
#include "hb.h"
#include "hb_common.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

using hb::BayesParams;
using hb::BayesRec;
using hb::FrameJob;
using hb::TransformParams;

namespace {

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum SlotState { FREE = 0, QUEUED, RUNNING, DONE, HELD };

// Optional host-side timeline (compile with -DHB_SERVE_TRACE): per batch the time its frames
// were taken from the queue, the time the enqueue of its copies and launches returned, the
// time its completion callback ran, and its frames' longest wait in the queue; a summary goes
// to stderr when the server is destroyed.
#ifdef HB_SERVE_TRACE
struct TraceRec {
    double formed, enqueued, done, max_wait;
    int frames;
};
#endif

struct Slot {
    unsigned char* h_in = nullptr;
    float* h_thb = nullptr;
    float* h_so2 = nullptr;
    unsigned char* d_in = nullptr;
    float* d_thb = nullptr;
    float* d_so2 = nullptr;
    int state = FREE;
    uint64_t tag = 0;
    double t_submit = 0.0, t_done = 0.0;
};

struct Stream {
    bool open = false;
    int W = 0, H = 0, levels = 0;
    size_t row = 0;        // packed input row bytes
    long npix_ll = 0;
    int tiles_x = 0;
    TransformParams tp{};
    std::vector<Slot> slots;
    size_t dev_bytes = 0;
};

struct Batch {
    cudaStream_t s = nullptr;
    FrameJob* h_jobs = nullptr;  // pinned
    FrameJob* d_jobs = nullptr;
    BayesRec* d_rec = nullptr;
    float2* d_chat = nullptr;
    float* d_partial = nullptr;
    unsigned* d_count = nullptr;
    std::vector<std::pair<int, int>> members;  // (stream, slot)
    bool busy = false;
    struct hb_server* srv = nullptr;
#ifdef HB_SERVE_TRACE
    TraceRec tr{};
#endif
};

struct Done {
    int stream, slot;
};

// Batches in flight at once (each on its own CUDA stream).  Under load most batches are
// small -- frames arrive one by one and a free batch slot takes whatever is queued -- so
// the server's rate is set by how many batches overlap: their copies, launches and
// completion callbacks.
#ifndef HB_SERVE_BATCH_SLOTS
#define HB_SERVE_BATCH_SLOTS 4
#endif
constexpr int kBatchSlots = HB_SERVE_BATCH_SLOTS;

}  // namespace

struct hb_server {
    int device = 0;
    int fmt = 1;
    int ll_intensity = 0;  // HB_LOWPASS_INTENSITY
    BayesParams bp{};
    float M[6] = {0};
    float2* d_lut = nullptr;
    float4* d_rowtab = nullptr;  // the closed-form row sums' table (BayesParams::row_tab)
    size_t budget = 0, used = 0;
    int max_batch = 1;
    long cap_ll = 0;
    int nbatch_slots = kBatchSlots;
    std::vector<Stream> streams;  // capacity reserved up front: elements never move
    Batch batches[kBatchSlots];
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<std::pair<int, int>> queue;  // (stream, slot) in arrival order
    std::deque<Done> done;
    std::thread loop;
    bool stop = false;
    bool paused = false;
    hb_status loop_error = HB_OK;
    long n_batches = 0, n_frames = 0, max_batch_seen = 0;
    double sum_batch = 0.0;
#ifdef HB_SERVE_TRACE
    std::vector<TraceRec> trace;  // under mu
#endif
};

// Shared with hb_api.cu: the FP64 preparation of the operator and grid constants.
namespace hb {
void prepare_constants(const hb_mixing* mix, const hb_grid* grid, double lambda, unsigned flags, float M[6],
                       BayesParams& bp);
}

namespace {

void CUDART_CB batch_done(void* arg) {
    Batch* b = static_cast<Batch*>(arg);
    hb_server* srv = b->srv;
    const double t = now_ms();
    {
        std::lock_guard<std::mutex> lk(srv->mu);
#ifdef HB_SERVE_TRACE
        b->tr.done = t;
        srv->trace.push_back(b->tr);
#endif
        for (auto& m : b->members) {
            Slot& sl = srv->streams[m.first].slots[m.second];
            sl.state = DONE;
            sl.t_done = t;
            srv->done.push_back(Done{m.first, m.second});
        }
        b->members.clear();
        b->busy = false;
    }
    srv->cv_work.notify_all();
    srv->cv_done.notify_all();
}

// Enqueue one batch; called by the loop thread without the lock held.
cudaError_t run_batch(hb_server* srv, Batch& b) {
    hb::NvtxRange r("hb_serve.batch");
    cudaStream_t s = b.s;
    int tiles = 0;
    long ll = 0;
    const int nj = (int)b.members.size();
    for (int j = 0; j < nj; ++j) {
        Stream& st = srv->streams[b.members[j].first];
        Slot& sl = st.slots[b.members[j].second];
        cudaError_t e = cudaMemcpyAsync(sl.d_in, sl.h_in, st.row * st.H, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
        FrameJob& job = b.h_jobs[j];
        job.tp = st.tp;
        job.frame = sl.d_in;
        job.stride = st.row;
        job.thb = sl.d_thb;
        job.so2 = sl.d_so2;
        job.ll_offset = ll;
        job.tile_begin = tiles;
        job.tiles_x = st.tiles_x;
        tiles += st.tiles_x * st.tp.hl;
        ll += st.npix_ll;
    }
    cudaError_t e = cudaMemcpyAsync(b.d_jobs, b.h_jobs, sizeof(FrameJob) * nj, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = hb::launch_batch_analysis(srv->bp, b.d_jobs, nj, tiles, srv->d_lut, b.d_rec, s);
    if (e == cudaSuccess)
        e = hb::launch_posterior(srv->bp, b.d_rec, ll, hb::PosteriorScratch{b.d_partial, b.d_count, hb::kMaxParts},
                                 b.d_chat, nullptr, 1.f, false, s);
    if (e == cudaSuccess) e = hb::launch_batch_synthesis(b.d_jobs, nj, tiles, srv->d_lut, b.d_chat, s);
    for (int j = 0; e == cudaSuccess && j < nj; ++j) {
        Stream& st = srv->streams[b.members[j].first];
        Slot& sl = st.slots[b.members[j].second];
        const size_t px = (size_t)st.W * st.H;
        e = cudaMemcpyAsync(sl.h_thb, sl.d_thb, px * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_so2, sl.d_so2, px * 4, cudaMemcpyDeviceToHost, s);
    }
#ifdef HB_SERVE_TRACE
    b.tr.enqueued = now_ms();  // before the callback is enqueued, so the callback sees it
#endif
    if (e == cudaSuccess) e = cudaLaunchHostFunc(s, batch_done, &b);
    return e;
}

void loop_main(hb_server* srv) {
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    while (true) {
        Batch* b = nullptr;
        srv->cv_work.wait(lk, [&] {
            if (srv->stop) return true;
            if (srv->paused || srv->queue.empty()) return false;
            for (int k = 0; k < srv->nbatch_slots; ++k)
                if (!srv->batches[k].busy) return true;
            return false;
        });
        if (srv->stop) break;
        for (int k = 0; k < srv->nbatch_slots && !b; ++k)
            if (!srv->batches[k].busy) b = &srv->batches[k];
        long ll = 0;
        while (!srv->queue.empty() && (int)b->members.size() < srv->max_batch) {
            const auto m = srv->queue.front();
            const long need = srv->streams[m.first].npix_ll;
            if (!b->members.empty() && ll + need > srv->cap_ll) break;
            srv->queue.pop_front();
            ll += need;
            srv->streams[m.first].slots[m.second].state = RUNNING;
            b->members.push_back(m);
        }
        b->busy = true;
#ifdef HB_SERVE_TRACE
        b->tr = TraceRec{now_ms(), 0.0, 0.0, 0.0, (int)b->members.size()};
        for (auto& m : b->members) {
            const double w = b->tr.formed - srv->streams[m.first].slots[m.second].t_submit;
            if (w > b->tr.max_wait) b->tr.max_wait = w;
        }
#endif
        srv->n_batches++;
        srv->n_frames += (long)b->members.size();
        srv->sum_batch += (double)b->members.size();
        if ((long)b->members.size() > srv->max_batch_seen) srv->max_batch_seen = (long)b->members.size();
        lk.unlock();
        const cudaError_t e = run_batch(srv, *b);
        lk.lock();
        if (e != cudaSuccess) {
            // the batch never completes: report its frames as done with the error recorded
            srv->loop_error = HB_ERR_CUDA;
            for (auto& m : b->members) {
                srv->streams[m.first].slots[m.second].state = DONE;
                srv->done.push_back(Done{m.first, m.second});
            }
            b->members.clear();
            b->busy = false;
            cudaGetLastError();
            srv->cv_done.notify_all();
        }
    }
}

void free_slot(Slot& sl) {
    cudaFreeHost(sl.h_in);
    cudaFreeHost(sl.h_thb);
    cudaFreeHost(sl.h_so2);
    cudaFree(sl.d_in);
    cudaFree(sl.d_thb);
    cudaFree(sl.d_so2);
    sl = Slot();
}

constexpr int kMaxStreams = 256;

size_t batch_bytes(long cap_ll) {
    return (sizeof(BayesRec) + sizeof(float2) + sizeof(float) * 3 * hb::kMaxParts + sizeof(unsigned)) * cap_ll +
           sizeof(FrameJob) * hb::kMaxBatchJobs;
}

#ifdef HB_SERVE_TRACE
// Percentiles of the batches' phases and the slowest batches, to stderr.
void trace_summary(hb_server* srv) {
    std::lock_guard<std::mutex> lk(srv->mu);
    std::vector<TraceRec>& t = srv->trace;
    if (t.empty()) return;
    auto pct = [&](std::vector<double> v, double q) {
        std::sort(v.begin(), v.end());
        return v[(size_t)std::min<double>(v.size() - 1, q * (v.size() - 1) + 0.5)];
    };
    std::vector<double> wait, enq, gpu, total;
    for (auto& r : t) {
        wait.push_back(r.max_wait);
        enq.push_back(r.enqueued - r.formed);
        gpu.push_back(r.done - r.enqueued);
        total.push_back(r.done - r.formed + r.max_wait);
    }
    std::fprintf(stderr, "hb_serve trace: %zu batches\n", t.size());
    const char* names[4] = {"queue wait", "enqueue", "enqueued->callback", "frame worst"};
    std::vector<double>* vs[4] = {&wait, &enq, &gpu, &total};
    for (int k = 0; k < 4; ++k)
        std::fprintf(stderr, "  %-20s p50 %8.3f p90 %8.3f p99 %8.3f max %8.3f ms\n", names[k], pct(*vs[k], 0.5),
                     pct(*vs[k], 0.9), pct(*vs[k], 0.99), pct(*vs[k], 1.0));
    std::vector<size_t> idx(t.size());
    for (size_t i = 0; i < idx.size(); ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](size_t a, size_t b) { return total[a] > total[b]; });
    const double t0 = t.front().formed;
    for (size_t k = 0; k < idx.size() && k < 12; ++k) {
        const TraceRec& r = t[idx[k]];
        std::fprintf(stderr, "  slow: at %9.3f ms frames %2d wait %7.3f enqueue %7.3f gpu+cb %7.3f\n", r.formed - t0,
                     r.frames, r.max_wait, r.enqueued - r.formed, r.done - r.enqueued);
    }
}
#endif

}  // namespace

extern "C" {

hb_status hb_server_create(const hb_mixing* mix, const hb_grid* grid, double lambda, unsigned flags, int in_format,
                           size_t budget_bytes, int max_batch, long batch_lowpass_pixels, hb_server** out) {
    if (!out) return HB_ERR_ARG;
    *out = nullptr;
    if (!mix || !grid) return HB_ERR_ARG;
    if (in_format != HB_IN_F32_HWC && in_format != HB_IN_U8_HWC) return HB_ERR_ARG;
    if (flags & ~(unsigned)(HB_LAMBDA_ABSOLUTE | HB_FULL_GRID | HB_ILLUMINATION | HB_LOWPASS_INTENSITY |
                            HB_SERVE_SEQUENTIAL))
        return HB_ERR_ARG;
    if (max_batch < 1 || max_batch > hb::kMaxBatchJobs || batch_lowpass_pixels < 1) return HB_ERR_ARG;
    if (grid->n0 < 1 || grid->n1 < 1 || !(grid->hi0 >= grid->lo0) || !(grid->hi1 >= grid->lo1) ||
        !(grid->sigma_l > 0.0))
        return HB_ERR_SHAPE;
    if (!std::isfinite(lambda) || lambda < 0.0) return HB_ERR_ARG;
    hb_server* srv = new (std::nothrow) hb_server();
    if (!srv) return HB_ERR_OOM;
    if (cudaGetDevice(&srv->device) != cudaSuccess) {
        cudaGetLastError();
        delete srv;
        return HB_ERR_CUDA;
    }
    srv->fmt = in_format;
    srv->budget = budget_bytes;
    srv->max_batch = max_batch;
    srv->cap_ll = batch_lowpass_pixels;
    srv->nbatch_slots = (flags & HB_SERVE_SEQUENTIAL) ? 1 : kBatchSlots;
    srv->ll_intensity = (flags & HB_LOWPASS_INTENSITY) ? 1 : 0;
    hb::prepare_constants(mix, grid, lambda, flags & (HB_LAMBDA_ABSOLUTE | HB_FULL_GRID | HB_ILLUMINATION), srv->M,
                          srv->bp);
    std::vector<float4> rowtab;
    if (!hb::row_table(srv->bp, rowtab)) rowtab.clear();
    const size_t need =
        (size_t)srv->nbatch_slots * batch_bytes(srv->cap_ll) + 256 * sizeof(float2) + sizeof(float4) * rowtab.size();
    if (need > budget_bytes) {
        delete srv;
        return HB_ERR_BUDGET;
    }
    float2 lut[256];
    for (int k = 0; k < 256; ++k) {
        const double y = -std::log((double)(k > 0 ? k : 1) / 255.0);
        const float hi = (float)y;
        lut[k] = make_float2(hi, (float)(y - (double)hi));
    }
    bool ok = cudaMalloc(&srv->d_lut, sizeof(lut)) == cudaSuccess &&
              cudaMemcpy(srv->d_lut, lut, sizeof(lut), cudaMemcpyHostToDevice) == cudaSuccess;
    if (ok && !rowtab.empty()) {
        ok = cudaMalloc(&srv->d_rowtab, sizeof(float4) * rowtab.size()) == cudaSuccess &&
             cudaMemcpy(srv->d_rowtab, rowtab.data(), sizeof(float4) * rowtab.size(), cudaMemcpyHostToDevice) ==
                 cudaSuccess;
        if (ok) srv->bp.row_tab = srv->d_rowtab;
    }
    for (int k = 0; ok && k < srv->nbatch_slots; ++k) {
        Batch& b = srv->batches[k];
        b.srv = srv;
        const long c = srv->cap_ll;
        ok = cudaStreamCreateWithFlags(&b.s, cudaStreamNonBlocking) == cudaSuccess &&
             cudaMallocHost(&b.h_jobs, sizeof(FrameJob) * hb::kMaxBatchJobs) == cudaSuccess &&
             cudaMalloc(&b.d_jobs, sizeof(FrameJob) * hb::kMaxBatchJobs) == cudaSuccess &&
             cudaMalloc(&b.d_rec, sizeof(BayesRec) * c) == cudaSuccess &&
             cudaMalloc(&b.d_chat, sizeof(float2) * c) == cudaSuccess &&
             cudaMalloc(&b.d_partial, sizeof(float) * 3 * hb::kMaxParts * c) == cudaSuccess &&
             cudaMalloc(&b.d_count, sizeof(unsigned) * c) == cudaSuccess &&
             cudaMemset(b.d_count, 0, sizeof(unsigned) * c) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        hb_server_destroy(srv);
        return HB_ERR_OOM;
    }
    srv->used = need;
    srv->streams.reserve(kMaxStreams);
    srv->loop = std::thread(loop_main, srv);
    *out = srv;
    return HB_OK;
}

void hb_server_destroy(hb_server* srv) {
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    if (srv->loop.joinable()) srv->loop.join();
#ifdef HB_SERVE_TRACE
    for (auto& b : srv->batches)
        if (b.s) cudaStreamSynchronize(b.s);
    trace_summary(srv);
#endif
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(srv->device);
    for (auto& b : srv->batches)
        if (b.s) cudaStreamSynchronize(b.s);
    for (auto& st : srv->streams)
        for (auto& sl : st.slots) free_slot(sl);
    for (auto& b : srv->batches) {
        if (b.s) cudaStreamDestroy(b.s);
        cudaFreeHost(b.h_jobs);
        cudaFree(b.d_jobs);
        cudaFree(b.d_rec);
        cudaFree(b.d_chat);
        cudaFree(b.d_partial);
        cudaFree(b.d_count);
    }
    cudaFree(srv->d_lut);
    cudaFree(srv->d_rowtab);
    cudaGetLastError();
    if (prev >= 0) cudaSetDevice(prev);
    delete srv;
}

hb_status hb_stream_open(hb_server* srv, int width, int height, int levels, int slots, int* stream_id) {
    if (!srv || !stream_id || slots < 1 || slots > 64) return HB_ERR_ARG;
    *stream_id = -1;
    if (width <= 0 || height <= 0 || levels < 0 || levels > 4) return HB_ERR_SHAPE;
    Stream st;
    const int B = 1 << levels;
    st.W = width;
    st.H = height;
    st.levels = levels;
    const size_t es = srv->fmt == HB_IN_U8_HWC ? 1 : 4;
    st.row = (size_t)width * 3 * es;
    TransformParams& tp = st.tp;
    tp.H = height;
    tp.W = width;
    tp.levels = levels;
    tp.fmt = srv->fmt;
    tp.eps = 1e-6f;
    tp.hl = (height + B - 1) / B;
    tp.wl = (width + B - 1) / B;
    tp.tile_w = hb::kThreads;
    tp.tikhonov_lowpass = 0;
    tp.ll_intensity = srv->ll_intensity;
    for (int k = 0; k < 6; ++k) tp.M[k] = srv->M[k];
    st.npix_ll = (long)tp.hl * tp.wl;
    const int cols = hb::tile_cols(levels, tp.ll_intensity);
    st.tiles_x = (tp.wl * B + cols - 1) / cols;
    if (st.npix_ll > srv->cap_ll) return HB_ERR_SHAPE;
    const size_t px = (size_t)width * height;
    st.dev_bytes = (size_t)slots * (st.row * height + 2 * px * 4);
    std::lock_guard<std::mutex> lk(srv->mu);
    if (srv->used + st.dev_bytes > srv->budget) return HB_ERR_BUDGET;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(srv->device);
    st.slots.resize(slots);
    bool ok = true;
    for (auto& sl : st.slots) {
        ok = ok && cudaMallocHost(&sl.h_in, st.row * height) == cudaSuccess &&
             cudaMallocHost(&sl.h_thb, px * 4) == cudaSuccess && cudaMallocHost(&sl.h_so2, px * 4) == cudaSuccess &&
             cudaMalloc(&sl.d_in, st.row * height) == cudaSuccess && cudaMalloc(&sl.d_thb, px * 4) == cudaSuccess &&
             cudaMalloc(&sl.d_so2, px * 4) == cudaSuccess;
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (!ok) {
        cudaGetLastError();
        for (auto& sl : st.slots) free_slot(sl);
        return HB_ERR_OOM;
    }
    st.open = true;
    int id = -1;
    for (int k = 0; k < (int)srv->streams.size(); ++k)
        if (!srv->streams[k].open && srv->streams[k].slots.empty()) {
            id = k;
            break;
        }
    if (id < 0) {
        if ((int)srv->streams.size() >= kMaxStreams) {
            for (auto& sl : st.slots) free_slot(sl);
            return HB_ERR_STATE;
        }
        id = (int)srv->streams.size();
        srv->streams.push_back(Stream());
    }
    srv->streams[id] = std::move(st);
    srv->used += srv->streams[id].dev_bytes;
    *stream_id = id;
    return HB_OK;
}

hb_status hb_stream_close(hb_server* srv, int stream_id) {
    if (!srv) return HB_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (stream_id < 0 || stream_id >= (int)srv->streams.size() || !srv->streams[stream_id].open) return HB_ERR_ARG;
    Stream& st = srv->streams[stream_id];
    for (auto& sl : st.slots)
        if (sl.state != FREE) return HB_ERR_STATE;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(srv->device);
    for (auto& sl : st.slots) free_slot(sl);
    if (prev >= 0) cudaSetDevice(prev);
    st.slots.clear();
    st.open = false;
    srv->used -= st.dev_bytes;
    st.dev_bytes = 0;
    return HB_OK;
}

hb_status hb_submit(hb_server* srv, int stream_id, const void* frame_host, size_t row_stride_bytes, uint64_t tag) {
    const double t = now_ms();
    if (!srv || !frame_host) return HB_ERR_ARG;
    Slot* slot = nullptr;
    int slot_id = -1;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        if (stream_id < 0 || stream_id >= (int)srv->streams.size() || !srv->streams[stream_id].open)
            return HB_ERR_ARG;
        Stream& st = srv->streams[stream_id];
        if (row_stride_bytes < st.row) return HB_ERR_ARG;
        for (int k = 0; k < (int)st.slots.size(); ++k)
            if (st.slots[k].state == FREE) {
                slot_id = k;
                break;
            }
        if (slot_id < 0) return HB_ERR_STATE;  // every slot of the stream is busy: poll and release first
        slot = &st.slots[slot_id];
        slot->state = QUEUED + 100;             // reserved while the frame is copied in
    }
    const Stream& st = srv->streams[stream_id];
    for (int r = 0; r < st.H; ++r)
        std::memcpy(slot->h_in + (size_t)r * st.row, static_cast<const unsigned char*>(frame_host) + r * row_stride_bytes,
                    st.row);
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        slot->state = QUEUED;
        slot->tag = tag;
        slot->t_submit = t;
        srv->queue.emplace_back(stream_id, slot_id);
    }
    srv->cv_work.notify_all();
    return HB_OK;
}

hb_status hb_poll(hb_server* srv, hb_result* out, int max_results, int* n_out, int wait_us) {
    if (!srv || !n_out || max_results < 0 || (max_results > 0 && !out)) return HB_ERR_ARG;
    *n_out = 0;
    std::unique_lock<std::mutex> lk(srv->mu);
    if (srv->done.empty() && wait_us > 0)
        srv->cv_done.wait_for(lk, std::chrono::microseconds(wait_us), [&] { return !srv->done.empty(); });
    int n = 0;
    while (n < max_results && !srv->done.empty()) {
        const Done d = srv->done.front();
        srv->done.pop_front();
        Slot& sl = srv->streams[d.stream].slots[d.slot];
        sl.state = HELD;
        hb_result& r = out[n++];
        r.stream_id = d.stream;
        r.slot = d.slot;
        r.tag = sl.tag;
        r.latency_ms = sl.t_done - sl.t_submit;
        r.thb_host = sl.h_thb;
        r.so2_host = sl.h_so2;
    }
    *n_out = n;
    return srv->loop_error;
}

hb_status hb_release(hb_server* srv, int stream_id, int slot) {
    if (!srv) return HB_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    if (stream_id < 0 || stream_id >= (int)srv->streams.size() || !srv->streams[stream_id].open) return HB_ERR_ARG;
    Stream& st = srv->streams[stream_id];
    if (slot < 0 || slot >= (int)st.slots.size() || st.slots[slot].state != HELD) return HB_ERR_STATE;
    st.slots[slot].state = FREE;
    return HB_OK;
}

hb_status hb_server_pause(hb_server* srv, int paused) {
    if (!srv) return HB_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->paused = paused != 0;
    }
    srv->cv_work.notify_all();
    return HB_OK;
}

hb_status hb_server_drain(hb_server* srv, int timeout_ms) {
    if (!srv || timeout_ms < 0) return HB_ERR_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto idle = [&] {
        if (!srv->queue.empty()) return false;
        for (int k = 0; k < srv->nbatch_slots; ++k)
            if (srv->batches[k].busy) return false;
        for (const Stream& st : srv->streams)
            for (const Slot& sl : st.slots)
                if (sl.state == QUEUED + 100) return false;  // a frame still being copied in
        return true;
    };
    // a frame leaving the copy-in state notifies only the loop, so re-check at least every millisecond
    const auto end = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    while (!idle()) {
        const auto now = std::chrono::steady_clock::now();
        if (now >= end) return HB_ERR_TIMEOUT;
        srv->cv_done.wait_for(lk, std::min<std::chrono::steady_clock::duration>(end - now, std::chrono::milliseconds(1)));
    }
    return srv->loop_error;
}

hb_status hb_server_stats(hb_server* srv, hb_server_info* out) {
    if (!srv || !out) return HB_ERR_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    out->batches = srv->n_batches;
    out->frames = srv->n_frames;
    out->max_batch_frames = srv->max_batch_seen;
    out->mean_batch_frames = srv->n_batches ? srv->sum_batch / srv->n_batches : 0.0;
    out->bytes_in_use = srv->used;
    out->budget_bytes = srv->budget;
    out->queued = (long)srv->queue.size();
    return HB_OK;
}

}  // extern "C"
