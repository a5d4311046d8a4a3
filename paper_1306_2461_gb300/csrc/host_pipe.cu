// of_compute_batch_host: of_compute_batch from and to host buffers, with the copies
// overlapped with the launches (Sect. 3.3: the fields of a batch are independent, so the
// pairs can be uploaded, computed and downloaded chunk by chunk).
#include <math.h>

#include <algorithm>
#include <map>
#include <vector>

#include "of_engine.h"

using namespace of;

// Level-0 megapixels of the default chunk of of_compute_batch_host.
#ifndef OF_HOST_CHUNK_MPX
#define OF_HOST_CHUNK_MPX 8.0
#endif

// ------------------------------------------------------ host-buffer pipelined form
// of_compute_batch_host: the batch in chunks; chunk k's upload runs on a copy stream,
// its launches after that upload on one of two compute streams (the caller's for even
// chunks, the pipeline's own for odd ones), and its download on a second copy stream
// after the launches, so that uploads, launches and downloads of neighbouring chunks
// overlap and one chunk's launches fill the last, partly empty waves of the other's.
// Events order the four streams; the caller's stream waits for the last download
// before the call's completion.
namespace {

// The pipeline's streams of the calling thread on the current device (the second compute
// stream and the two copy streams), kept until the thread exits: captured launches are
// cached per stream, so the compute stream must outlive a call for the next call to replay
// them, and it is the thread's own, so that no other thread queues work on it while a
// launch sequence is being captured there. Keeping the copy streams saves creating two
// streams per call.
struct PipeStreams {
    cudaStream_t compute = nullptr, up = nullptr, down = nullptr;
};

struct ThreadStreams {
    std::map<int, PipeStreams> s;
    ~ThreadStreams()
    {
        for (auto &kv : s)   // pending work still runs
            for (cudaStream_t x : {kv.second.compute, kv.second.up, kv.second.down})
                if (x) cudaStreamDestroy(x);
    }
};

const PipeStreams *pipe_streams()
{
    thread_local ThreadStreams streams;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    auto it = streams.s.find(dev);
    if (it != streams.s.end()) return &it->second;
    PipeStreams p;
    if (cudaStreamCreateWithFlags(&p.compute, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p.up, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p.down, cudaStreamNonBlocking) != cudaSuccess) {
        for (cudaStream_t x : {p.compute, p.up, p.down})
            if (x) cudaStreamDestroy(x);
        return nullptr;
    }
    return &(streams.s[dev] = p);
}

struct HostPipe {
    cudaStream_t up = nullptr, down = nullptr;
    std::vector<cudaEvent_t> ev;
    ~HostPipe()
    {
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);   // released once recorded work completes
    }
    cudaEvent_t make()
    {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        ev.push_back(e);
        return e;
    }
};

}  // namespace

extern "C" int of_compute_batch_host(int32_t n, const of_handle *hs, const void *const *hI1s, const void *const *hI2s,
                                     float *const *hus, float *const *hvs, void *const *dI1s, void *const *dI2s,
                                     float *const *dus, float *const *dvs, of_stream_t stream, int32_t chunk)
{
    if (n == 0) return OF_OK;
    if (n < 0 || n > 65536 || !hs || !hI1s || !hI2s || !hus || !hvs || !dI1s || !dI2s || !dus || !dvs || chunk < 0)
        return OF_EINVAL;
    std::vector<of_handle> seen(hs, hs + n);
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return OF_EINVAL;   // a handle twice
    for (int i = 0; i < n; ++i) {
        if (!hs[i] || !hI2s[i] || !hus[i] || !hvs[i] || !dI2s[i] || !dus[i] || !dvs[i] || (hI1s[i] && !dI1s[i]))
            return OF_EINVAL;
        if (!same_method(hs[i]->plan, hs[0]->plan) || hs[i]->device != hs[0]->device)
            return OF_EINVAL;
        if (!hI1s[i] && !hs[i]->has_prev) return OF_ESTATE;
    }
    // default: chunks of about eight 1024^2 pairs, at most 24 of them (measured on 64 such
    // pairs, fields/s for 3, 4, 6, 8, 11, 16, 22, 32 pairs per chunk: 9343, 9434, 9517, 9656,
    // 9430, 9146, 8782, 7915; from 8 pairs on, a chunk's launches have the tiles for strips),
    // the first and the last two a quarter and a half of that, so that the pipeline fills
    // (first upload) and drains (last launches and downloads) in less time
    int per = chunk;
    std::vector<int> sizes;
    if (per <= 0) {
        double px = 0.0;
        for (int i = 0; i < n; ++i) px += (double)hs[i]->plan.H * hs[i]->plan.W;
        per = (int)lround(OF_HOST_CHUNK_MPX * 1048576.0 / (px / n));
        per = std::max(per, std::max(1, (n + 23) / 24));
        const int q = std::max(1, per / 4), h = std::max(1, per / 2);
        if (per >= 4 && n >= 2 * (q + h) + per) {
            sizes = {q, h};
            int rest = n - 2 * (q + h);
            while (rest > 0) {
                sizes.push_back(std::min(per, rest));
                rest -= per;
            }
            sizes.push_back(h);
            sizes.push_back(q);
        }
    }
    if (sizes.empty())
        for (int off = 0; off < n; off += per) sizes.push_back(std::min(per, n - off));
    const int nch = (int)sizes.size();
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const PipeStreams *ps = pipe_streams();
    if (!ps) return OF_ECUDA;
    cudaStream_t aux = nch > 1 ? ps->compute : st;
    HostPipe pp;
    pp.up = ps->up;
    pp.down = ps->down;
    cudaEvent_t start = pp.make();
    if (!start || cudaEventRecord(start, st) != cudaSuccess || cudaStreamWaitEvent(pp.up, start, 0) != cudaSuccess ||
        cudaStreamWaitEvent(pp.down, start, 0) != cudaSuccess ||
        (aux != st && cudaStreamWaitEvent(aux, start, 0) != cudaSuccess))
        return OF_ECUDA;
    // After an error past this point, `st` is made to wait for everything already queued
    // on the pipeline's streams before the call returns, so that a caller who synchronises
    // `st` after the error may free or reuse the buffers of the earlier chunks.
    auto fail = [&](int rc) {
        for (cudaStream_t x : {pp.up, aux, pp.down}) {
            if (x == st) continue;
            cudaEvent_t j = pp.make();
            if (!j || cudaEventRecord(j, x) != cudaSuccess || cudaStreamWaitEvent(st, j, 0) != cudaSuccess)
                cudaStreamSynchronize(x);   // cannot be ordered on the device: wait here
        }
        return rc;
    };
    const size_t in_elem = hs[0]->plan.in_format == OF_U8 ? 1 : 2;
    std::vector<const void *> d1(*std::max_element(sizes.begin(), sizes.end()));
    for (int c = 0, off = 0; c < nch; off += sizes[c], ++c) {
        const int cnt = sizes[c];
        for (int i = off; i < off + cnt; ++i) {
            const size_t px = (size_t)hs[i]->plan.H * hs[i]->plan.W;
            if ((hI1s[i] && cudaMemcpyAsync(dI1s[i], hI1s[i], px * in_elem, cudaMemcpyHostToDevice, pp.up) != cudaSuccess) ||
                cudaMemcpyAsync(dI2s[i], hI2s[i], px * in_elem, cudaMemcpyHostToDevice, pp.up) != cudaSuccess)
                return fail(OF_ECUDA);
            d1[i - off] = hI1s[i] ? dI1s[i] : nullptr;
        }
        cudaStream_t cs = (c & 1) ? aux : st;
        cudaEvent_t in = pp.make(), done = pp.make();
        if (!in || !done || cudaEventRecord(in, pp.up) != cudaSuccess || cudaStreamWaitEvent(cs, in, 0) != cudaSuccess)
            return fail(OF_ECUDA);
        const Tuning t = tuning_for(hs[0]->plan, batch_size_class(cnt, hs + off));
        const int rc = run_batch(cnt, hs + off, d1.data(), dI2s + off, dus + off, dvs + off, cs, t);
        if (rc != OF_OK) return fail(rc);
        if (cudaEventRecord(done, cs) != cudaSuccess || cudaStreamWaitEvent(pp.down, done, 0) != cudaSuccess)
            return fail(OF_ECUDA);
        for (int i = off; i < off + cnt; ++i) {
            const size_t bytes = (size_t)hs[i]->plan.H * hs[i]->plan.W * sizeof(float);
            if (cudaMemcpyAsync(hus[i], dus[i], bytes, cudaMemcpyDeviceToHost, pp.down) != cudaSuccess ||
                cudaMemcpyAsync(hvs[i], dvs[i], bytes, cudaMemcpyDeviceToHost, pp.down) != cudaSuccess)
                return fail(OF_ECUDA);
        }
    }
    cudaEvent_t end = pp.make();
    if (!end || cudaEventRecord(end, pp.down) != cudaSuccess || cudaStreamWaitEvent(st, end, 0) != cudaSuccess)
        return fail(OF_ECUDA);
    return OF_OK;
}
