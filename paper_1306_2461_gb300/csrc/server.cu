// Serving loop: camera streams of mixed resolutions, continuous batching on one GPU.
//
// Each stream delivers frames in order; every frame after the first gives the field
// from the previous frame to it. The stream's previous-frame pyramid stays resident on
// the device and is the first image of the next pair, so each field processes one new
// image (computing scheme 1 of Sect. 2.4). Streams are admitted against an HBM budget
// (their workspace plus two staging buffers).
//
// A worker thread forms "ticks": the next pending frame of every stream that has one
// (at most max_batch pairs) goes into one batched launch (tuned as of_compute_batch). Frames that
// arrive while ticks run join the next tick as soon as fewer than max_inflight ticks
// are on the device; their host-to-device copies run on a copy stream and overlap the
// running tick's compute, and the next tick's kernel follows the previous one on the
// compute stream with no host round trip in between. Completed ticks are retired in
// order and their results, with host timestamps (arrival, launch, completion), are
// handed to of_server_poll.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "of_engine.h"
#include "of_internal.cuh"

namespace {

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    const void *frame;
    float *u, *v;
    uint64_t tag;
    int64_t arrival_ns;
};

struct Stream {
    bool open = false;
    int32_t H = 0, W = 0;
    of_handle h = nullptr;
    void *raw[2] = {nullptr, nullptr};   // device staging of the last two frames
    size_t frame_bytes = 0, bytes = 0;   // one frame; everything this stream holds
    int64_t frames = 0;                  // frames taken into ticks so far
    int64_t last_reader[2] = {-1, -1};   // tick that last read each staging buffer
    int64_t last_tick = -1;              // last tick that holds work of this stream
    std::deque<Request> queue;
};

struct Tick {
    int64_t seq = 0;
    int slot = 0;
    cudaEvent_t copied = nullptr, done = nullptr;
    int64_t launch_ns = 0;
    std::vector<of_result> results;
};

constexpr int kMaxQueue = 256;

}  // namespace

struct of_server {
    of_server_config cfg;
    of_plan method;
    int device = 0;
    cudaStream_t compute = nullptr, copy = nullptr;
    std::vector<Stream> streams;
    uint64_t used = 0;
    std::vector<of::BatchSlot> slots;
    std::vector<cudaEvent_t> ev_copied, ev_done;   // one pair per slot
    std::deque<Tick> inflight;
    std::deque<of_result> done;
    int64_t next_seq = 0, retired = -1;
    size_t rr = 0;                                 // round-robin start for fairness
    int64_t pending = 0;                           // submitted, not yet in a tick
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    int error = OF_OK;
    // statistics
    int64_t ticks = 0, pairs = 0;
};

namespace {

bool in_flight(const of_server *s, int64_t seq) { return seq > s->retired; }

cudaEvent_t done_event_of(of_server *s, int64_t seq)
{
    for (auto &t : s->inflight)
        if (t.seq == seq) return t.done;
    return nullptr;
}

void retire(of_server *s)
{
    while (!s->inflight.empty()) {
        Tick &t = s->inflight.front();
        const cudaError_t q = cudaEventQuery(t.done);
        if (q == cudaErrorNotReady) break;
        const int64_t tnow = now_ns();
        const int st = q == cudaSuccess ? OF_OK : OF_ECUDA;
        if (q != cudaSuccess) {
            cudaGetLastError();
            s->error = OF_ECUDA;
        }
        for (auto &r : t.results) {
            r.done_ns = tnow;
            r.launch_ns = t.launch_ns;
            if (r.status == OF_OK) r.status = st;
            s->done.push_back(r);
        }
        s->retired = t.seq;
        s->inflight.pop_front();
        s->cv_done.notify_all();
    }
}

// Take the next frame of every stream that has one into a new tick and launch it.
int form_tick(of_server *s)
{
    const int slot = (int)(s->next_seq % s->cfg.max_inflight);
    Tick t;
    t.seq = s->next_seq;
    t.slot = slot;
    t.copied = s->ev_copied[slot];
    t.done = s->ev_done[slot];
    std::vector<of_handle> hs;
    std::vector<const void *> I1s, I2s;
    std::vector<float *> us, vs;
    const size_t n = s->streams.size();
    bool any = false;
    for (size_t k = 0; k < n && (int)hs.size() < s->cfg.max_batch; ++k) {
        Stream &st = s->streams[(s->rr + k) % n];
        if (!st.open || st.queue.empty()) continue;
        const Request rq = st.queue.front();
        st.queue.pop_front();
        --s->pending;
        const int b = (int)(st.frames % 2);
        // the staging buffer is free once the tick that last read it is done
        if (st.last_reader[b] >= 0 && in_flight(s, st.last_reader[b])) {
            cudaEvent_t e = done_event_of(s, st.last_reader[b]);
            if (e && cudaStreamWaitEvent(s->copy, e, 0) != cudaSuccess) return OF_ECUDA;
        }
        if (cudaMemcpyAsync(st.raw[b], rq.frame, st.frame_bytes, cudaMemcpyHostToDevice, s->copy) != cudaSuccess)
            return OF_ECUDA;
        of_result r;
        memset(&r, 0, sizeof(r));
        r.stream = (int32_t)((s->rr + k) % n);
        r.tag = rq.tag;
        r.arrival_ns = rq.arrival_ns;
        r.status = OF_OK;
        if (st.frames == 0) {
            r.has_field = 0;   // first frame: staged, no field yet
        } else {
            r.has_field = 1;
            hs.push_back(st.h);
            I1s.push_back(st.frames == 1 ? st.raw[1 - b] : nullptr);   // then reuse the resident pyramid
            I2s.push_back(st.raw[b]);
            us.push_back(rq.u);
            vs.push_back(rq.v);
            if (st.frames == 1) st.last_reader[1 - b] = t.seq;
        }
        st.last_reader[b] = t.seq;
        st.last_tick = t.seq;
        st.frames += 1;
        t.results.push_back(r);
        any = true;
    }
    if (!any) return OF_OK;
    s->rr = (s->rr + 1) % (n ? n : 1);
    if (cudaEventRecord(t.copied, s->copy) != cudaSuccess || cudaStreamWaitEvent(s->compute, t.copied, 0) != cudaSuccess)
        return OF_ECUDA;
    for (auto &r : t.results) r.batch = (int32_t)hs.size();
    if (!hs.empty()) {
        const int rc = of::batch_run_slot(s->slots[slot], (int32_t)hs.size(), hs.data(), I1s.data(), I2s.data(),
                                          us.data(), vs.data(), s->compute);
        if (rc) return rc;
        s->pairs += (int64_t)hs.size();
    }
    if (cudaEventRecord(t.done, s->compute) != cudaSuccess) return OF_ECUDA;
    t.launch_ns = now_ns();
    s->inflight.push_back(std::move(t));
    ++s->next_seq;
    ++s->ticks;
    return OF_OK;
}

void worker_main(of_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        retire(s);
        if (s->pending > 0 && (int)s->inflight.size() < s->cfg.max_inflight && s->error == OF_OK) {
            const int rc = form_tick(s);
            if (rc) s->error = rc;
            continue;
        }
        if (!s->inflight.empty())
            s->cv_work.wait_for(lk, std::chrono::microseconds(20));
        else
            s->cv_work.wait(lk, [s] { return s->stop || s->pending > 0; });
    }
}

void free_stream(Stream &st)
{
    if (st.h) of_destroy(st.h);
    for (auto &p : st.raw)
        if (p) cudaFree(p);
    st = Stream();
}

}  // namespace

extern "C" {

void of_server_config_init(of_server_config *c)
{
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->levels = 3;
    c->radius = 4;
    c->iterations = 5;
    c->in_format = OF_U16;
    c->in_bits = 12;
    c->storage = OF_F16;
    c->fp64_cond = 1e3f;
    c->flags = 0;
    c->hbm_budget_bytes = 8ull << 30;
    c->max_batch = 64;
    c->max_inflight = 2;
}

int of_server_create(const of_server_config *c, of_server_t *out)
{
    if (!out) return OF_EINVAL;
    *out = nullptr;
    if (!c || c->max_batch < 1 || c->max_batch > 4096 || c->max_inflight < 1 || c->max_inflight > 8) return OF_EINVAL;
    of_plan m;
    of_plan_init(&m, 64, 64);
    m.levels = c->levels;
    m.radius = c->radius;
    m.iterations = c->iterations;
    m.in_format = c->in_format;
    m.in_bits = c->in_bits;
    m.storage = c->storage;
    m.fp64_cond = c->fp64_cond;
    m.flags = c->flags & ~OF_FLAG_NO_GRAPH;
    if (of_plan_validate(&m) != OF_OK) return OF_EINVAL;
    of_server *s = new (std::nothrow) of_server();
    if (!s) return OF_ENOMEM;
    s->cfg = *c;
    s->method = m;
    cudaGetDevice(&s->device);
    int rc = OF_OK;
    if (cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking) != cudaSuccess)
        rc = OF_ECUDA;
    const int phases = m.levels + m.levels * m.iterations;   // an upper bound on the pyramid phases
    s->slots.resize(c->max_inflight);
    s->ev_copied.assign(c->max_inflight, nullptr);
    s->ev_done.assign(c->max_inflight, nullptr);
    for (int i = 0; rc == OF_OK && i < c->max_inflight; ++i) {
        rc = of::batch_slot_init(s->slots[i], c->max_batch, phases);
        if (rc == OF_OK && (cudaEventCreateWithFlags(&s->ev_copied[i], cudaEventDisableTiming) != cudaSuccess ||
                            cudaEventCreateWithFlags(&s->ev_done[i], cudaEventDisableTiming) != cudaSuccess))
            rc = OF_ECUDA;
    }
    if (rc != OF_OK) {
        of_server_destroy(s);
        return rc;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return OF_OK;
}

int of_server_open_stream(of_server_t s, int32_t H, int32_t W, int32_t *id)
{
    if (!s || !id) return OF_EINVAL;
    *id = -1;
    of_plan p = s->method;
    p.H = H;
    p.W = W;
    if (of_plan_validate(&p) != OF_OK) return OF_EINVAL;
    size_t ws = 0;
    of_workspace_bytes(&p, &ws);
    const size_t frame = (size_t)H * W * (p.in_format == OF_U8 ? 1 : 2);
    const size_t need = ws + 2 * ((frame + 255) / 256 * 256);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->used + need > s->cfg.hbm_budget_bytes) return OF_ENOMEM;   // admission by HBM budget
    Stream st;
    st.H = H;
    st.W = W;
    st.frame_bytes = frame;
    st.bytes = need;
    int rc = of_create(&p, &st.h);
    for (int b = 0; rc == OF_OK && b < 2; ++b)
        if (of::dev_malloc(&st.raw[b], frame) != cudaSuccess) {
            cudaGetLastError();
            rc = OF_ENOMEM;
        }
    if (rc != OF_OK) {
        free_stream(st);
        return rc;
    }
    st.open = true;
    size_t slot = 0;
    while (slot < s->streams.size() && s->streams[slot].open) ++slot;
    if (slot == s->streams.size()) s->streams.emplace_back();
    s->streams[slot] = st;
    s->used += need;
    *id = (int32_t)slot;
    return OF_OK;
}

int of_server_close_stream(of_server_t s, int32_t id)
{
    if (!s) return OF_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (id < 0 || (size_t)id >= s->streams.size() || !s->streams[id].open) return OF_EINVAL;
    Stream &st = s->streams[id];
    if (!st.queue.empty()) return OF_EBUSY;
    // wait (bounded) for the ticks that hold work of this stream to retire
    const int64_t last = st.last_tick;
    if (!s->cv_done.wait_for(lk, std::chrono::seconds(30), [&] { return s->retired >= last || s->error; }))
        return OF_ETIMEOUT;
    s->used -= st.bytes;
    free_stream(st);
    return OF_OK;
}

int of_server_submit(of_server_t s, int32_t id, const void *frame, float *u, float *v, uint64_t tag,
                     int64_t arrival_ns)
{
    if (!s || !frame) return OF_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->error) return s->error;
    if (id < 0 || (size_t)id >= s->streams.size() || !s->streams[id].open) return OF_EINVAL;
    Stream &st = s->streams[id];
    const bool first = st.frames == 0 && st.queue.empty();
    if (!first && (!u || !v)) return OF_EINVAL;
    if ((int)st.queue.size() >= kMaxQueue) return OF_EBUSY;
    st.queue.push_back(Request{frame, u, v, tag, arrival_ns ? arrival_ns : now_ns()});
    ++s->pending;
    s->cv_work.notify_one();
    return OF_OK;
}

int of_server_poll(of_server_t s, of_result *out, int32_t max, int32_t *n, int32_t timeout_us)
{
    if (!s || !n || (max > 0 && !out) || max < 0) return OF_EINVAL;
    *n = 0;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && timeout_us > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [s] { return !s->done.empty() || s->error; });
    while (*n < max && !s->done.empty()) {
        out[(*n)++] = s->done.front();
        s->done.pop_front();
    }
    return s->error;
}

int of_server_drain(of_server_t s, int32_t timeout_ms)
{
    if (!s) return OF_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms), [s] {
        return (s->pending == 0 && s->inflight.empty()) || s->error;
    });
    if (s->error) return s->error;
    return ok ? OF_OK : OF_ETIMEOUT;
}

int of_server_stats(of_server_t s, int64_t *ticks, int64_t *pairs, uint64_t *hbm_used)
{
    if (!s) return OF_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (ticks) *ticks = s->ticks;
    if (pairs) *pairs = s->pairs;
    if (hbm_used) *hbm_used = s->used;
    return OF_OK;
}

int64_t of_server_now_ns(void) { return now_ns(); }

int of_server_destroy(of_server_t s)
{
    if (!s) return OF_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    if (s->compute) cudaStreamSynchronize(s->compute);
    if (s->copy) cudaStreamSynchronize(s->copy);
    for (auto &st : s->streams)
        if (st.open) free_stream(st);
    for (auto &sl : s->slots) of::batch_slot_free(sl);
    for (auto e : s->ev_copied)
        if (e) cudaEventDestroy(e);
    for (auto e : s->ev_done)
        if (e) cudaEventDestroy(e);
    if (s->compute) cudaStreamDestroy(s->compute);
    if (s->copy) cudaStreamDestroy(s->copy);
    delete s;
    return OF_OK;
}

}  // extern "C"
