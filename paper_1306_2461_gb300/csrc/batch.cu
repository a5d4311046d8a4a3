// of_compute_batch: many independent pairs (each field is independent of the others,
// Sect. 3.3) per CUDA graph replay: one ordinary launch per phase (pyramid pass,
// iteration) over all pairs' tiles, optionally in concurrent sequences over parts of
// the batch, or one persistent cooperative launch with grid barriers (batch_device.cuh).
// This file builds the work lists and the phase arguments, caches the captured launches
// and records the handles' state.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "batch_device.cuh"

// Strips of the phase launches shrink while a launch would have fewer blocks than this
// many per resident block slot.
#ifndef OF_STRIP_WAVES
#define OF_STRIP_WAVES 2
#endif

namespace of {

// The bounded-wait test kernel (of_debug_wait_timeout) runs the barrier's wait loop on
// a counter that nothing increments.
__global__ void wait_test_kernel(const unsigned int *word, int *status, long long timeout_ns)
{
    if (threadIdx.x == 0 && blockIdx.x == 0 && !bounded_wait_ge(word, 1u, nullptr, timeout_ns))
        *status = DEV_TIMEOUT;
}

cudaError_t launch_wait_timeout(int *flag, int *status, long long timeout_ns, cudaStream_t s)
{
    wait_test_kernel<<<1, 32, 0, s>>>(reinterpret_cast<const unsigned int *>(flag), status, timeout_ns);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ host side
namespace {

// A captured batch: its device descriptors, barrier words and graph.
struct BatchEntry {
    std::vector<char> key;              // host image of the descriptors + stream
    char *dev = nullptr;                // pairs | prefix | barrier | abort
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t done = nullptr;
    BatchHdr hdr;
    void *fn = nullptr;
    dim3 grid;
    size_t smem = 0;
    int device = -1;
    uint64_t last_use = 0;
    // phase launches: what to launch again when no graph could be captured
    int phased = 0;
    std::vector<BatchPair> pairs;
    of_plan plan;
    Tuning tuning;
};

constexpr int BATCH_CACHE = 64;   // captured batches kept (a host pipeline call takes one per chunk)
std::mutex g_mu;
BatchEntry g_cache[BATCH_CACHE];
uint64_t g_clock = 0;

void release(BatchEntry &e)
{
    if (e.done) cudaEventSynchronize(e.done);
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.done) cudaEventDestroy(e.done);
    if (e.dev) cudaFree(e.dev);
    e = BatchEntry();
}

cudaError_t launch_direct(const BatchEntry &e, cudaStream_t st)
{
    cudaError_t err = cudaMemsetAsync(e.hdr.barrier, 0, 2 * sizeof(unsigned int), st);
    if (err != cudaSuccess) return err;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = e.grid;
    cfg.blockDim = dim3(LK_THREADS);
    cfg.dynamicSmemBytes = e.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {(void *)&e.hdr};
    return cudaLaunchKernelExC(&cfg, e.fn, args);
}

}  // namespace

}  // namespace of

using namespace of;

namespace of {

bool same_method(const of_plan &a, const of_plan &b)
{
    return a.levels == b.levels && a.radius == b.radius && a.iterations == b.iterations &&
           a.in_format == b.in_format && a.in_bits == b.in_bits && a.storage == b.storage &&
           a.fp64_cond == b.fp64_cond &&
           (a.flags & (OF_FLAG_GATHER | OF_FLAG_ZNSSD | OF_FLAG_I1GRAD)) ==
               (b.flags & (OF_FLAG_GATHER | OF_FLAG_ZNSSD | OF_FLAG_I1GRAD));
}

// The host image of one batch: descriptors, work-list prefix sums, slots, launch shape.
struct BatchBuild {
    std::vector<BatchPair> pairs;
    std::vector<int32_t> prefix;
    std::vector<int> s1, s2;
    int nphases = 0, npyr = 0, max_items = 0;
};

static int build_batch(int32_t n, const of_handle *hs, const void *const *I1s, const void *const *I2s,
                       float *const *us, float *const *vs, BatchBuild &b)
{
    if (n < 0 || n > 65536 || !hs || !I1s || !I2s || !us || !vs) return OF_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!hs[i] || !I2s[i] || !us[i] || !vs[i]) return OF_EINVAL;
        if (!same_method(hs[i]->plan, hs[0]->plan)) return OF_EINVAL;
        if (!I1s[i] && !hs[i]->has_prev) return OF_ESTATE;
        if (hs[i]->device != hs[0]->device) return OF_EINVAL;
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return OF_EINVAL;
    }
    const of_plan &p0 = hs[0]->plan;
    const int L = p0.levels;
    const bool zn = (p0.flags & OF_FLAG_ZNSSD) != 0;
    b.npyr = zn ? L : (L > 1 ? L - 1 : 1);
    b.nphases = b.npyr + L * p0.iterations;
    b.pairs.assign(n, BatchPair());
    b.prefix.assign((size_t)b.nphases * (n + 1), 0);
    b.s1.assign(n, 0);
    b.s2.assign(n, 1);
    for (int i = 0; i < n; ++i) {
        of_ctx *h = hs[i];
        b.s1[i] = I1s[i] ? 0 : h->prev_slot;
        b.s2[i] = I1s[i] ? 1 : 1 - h->prev_slot;
        BatchPair &bp = b.pairs[i];
        memset(&bp, 0, sizeof(bp));
        bp.raw[0] = I1s[i];
        bp.raw[1] = I2s[i];
        bp.u = us[i];
        bp.v = vs[i];
        bp.pyr[0] = h->pyr[b.s1[i]];
        bp.pyr[1] = h->pyr[b.s2[i]];
        bp.flow[0] = h->flow[0];
        bp.flow[1] = h->flow[1];
        bp.status = h->status;
        bp.hess = h->hess;
        bp.first_image = I1s[i] ? 0 : 1;
        for (int l = 0; l < L; ++l) {
            bp.H[l] = h->lay.H[l];
            bp.W[l] = h->lay.W[l];
            bp.pitch[l] = h->lay.pitch[l];
            bp.off[l] = h->lay.level_off[l];
        }
    }
    b.max_items = 0;
    for (int ph = 0; ph < b.nphases; ++ph) {
        int32_t *pre = &b.prefix[(size_t)ph * (n + 1)];
        pre[0] = 0;
        for (int i = 0; i < n; ++i) {
            const BatchPair &bp = b.pairs[i];
            int64_t cnt;
            if (ph < b.npyr && zn && ph == 0) {
                cnt = (int64_t)((bp.W[0] + ZN_T - 1) / ZN_T) * ((bp.H[0] + ZN_T - 1) / ZN_T) * (2 - bp.first_image);
            } else if (ph < b.npyr) {
                const int ls = zn ? ph - 1 : ph;
                const int Ho = (bp.H[ls] + 1) / 2, Wo = (bp.W[ls] + 1) / 2;
                cnt = (int64_t)((Wo + PYR_TW - 1) / PYR_TW) * ((Ho + PYR_TH - 1) / PYR_TH) * (2 - bp.first_image);
            } else {
                const int l = L - 1 - (ph - b.npyr) / p0.iterations;
                cnt = (int64_t)((bp.W[l] + LK_TW - 1) / LK_TW) * ((bp.H[l] + LK_TH - 1) / LK_TH);
            }
            if (pre[i] + cnt > INT32_MAX) return OF_EINVAL;
            pre[i + 1] = (int32_t)(pre[i] + cnt);
        }
        if (pre[n] > b.max_items) b.max_items = pre[n];
    }
    return OF_OK;
}

static void fill_header(BatchHdr &hd, const of_plan &p0, const BatchBuild &b, char *dev, size_t bar_off)
{
    const size_t pairs_bytes = sizeof(BatchPair) * b.pairs.size();
    hd.pairs = reinterpret_cast<const BatchPair *>(dev);
    hd.prefix = reinterpret_cast<const int32_t *>(dev + pairs_bytes);
    hd.barrier = reinterpret_cast<unsigned int *>(dev + bar_off);
    hd.abort = reinterpret_cast<int *>(dev + bar_off + sizeof(unsigned int));
    hd.npairs = (int32_t)b.pairs.size();
    hd.levels = p0.levels;
    hd.iterations = p0.iterations;
    hd.radius = p0.radius;
    hd.nphases = b.nphases;
    hd.npyr = b.npyr;
    hd.fp64_cond = p0.fp64_cond;
    hd.timeout_ns = BARRIER_TIMEOUT_NS;
    hd.znssd = (p0.flags & OF_FLAG_ZNSSD) ? 1 : 0;
}

static size_t bar_offset(const BatchBuild &b)
{
    return (sizeof(BatchPair) * b.pairs.size() + sizeof(int32_t) * b.prefix.size() + 255) / 256 * 256;
}

// Grid size of the persistent kernel: every block resident at once (cooperative),
// at most blocks_per_sm per SM when that is > 0.
static int grid_for(void *fn, size_t smem, int device, int max_items, int blocks_per_sm, dim3 &grid)
{
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, LK_THREADS, smem) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || per_sm < 1)
        return OF_ECUDA;
    if (blocks_per_sm > 0 && blocks_per_sm < per_sm) per_sm = blocks_per_sm;
    int g = per_sm * sms;
    if (g > max_items) g = max_items > 0 ? max_items : 1;
    grid = dim3(g);
    return OF_OK;
}

// The persistent kernel and its shared memory for a method (it gathers its taps: the
// TMA staging of the phase launches needs tensor maps in parameter space).
struct Resolved {
    void *fn;
    size_t smem;
};
static Resolved resolve(const of_plan &p0, const Tuning &t)
{
    Resolved r;
    if (t.generic_sums) {
        r.fn = batch_kernel_generic(p0.in_format, p0.storage);
        r.smem = batch_smem_generic(p0.radius);
    } else {
        r.fn = batch_kernel_for(p0.in_format, p0.storage, p0.radius);
        r.smem = batch_smem_bytes(p0.radius, false);
    }
    return r;
}

// The method for all pairs of a batch as ordinary launches, one per phase and group of
// up to PHASE_PAIRS pairs (the per-pair arguments are kernel parameters): pyramid passes
// (after the normalisation of Eq. 2 when the plan asks for it), then the iterations
// level by level. Stream order separates the phases; there is no grid-wide barrier.
static cudaError_t enqueue_chain(const BatchPair *pairs, int n, const of_plan &p0, const Tuning &t,
                                 cudaStream_t st)
{
    const int L = p0.levels;
    const bool zn = (p0.flags & OF_FLAG_ZNSSD) != 0;
    const int32_t stage = (!t.generic_sums && !(p0.flags & OF_FLAG_GATHER) && t.stage_i2) ? 1 : 0;
    // L2 prefetch distance of the iteration launches: t.prefetch blocks per SM ahead
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int32_t prefetch_ahead = sms * t.prefetch;
    // iteration tile height: the tuned one for the grouped sums of a specialised radius
    const int tile_h = (t.tile_h == ALT_TH && !t.generic_sums && radius_specialised(p0.radius)) ? ALT_TH : LK_TH;
    // tiles per block of the fixed-radius kernels (the run-time-radius kernel takes one)
    const int strip = (!t.generic_sums && radius_specialised(p0.radius)) ? strip_len(tuning_strip(t)) : 1;
    cudaError_t e;
    for (int g0 = 0; g0 < n; g0 += PHASE_PAIRS) {
        const int m = n - g0 < PHASE_PAIRS ? n - g0 : PHASE_PAIRS;
        const BatchPair *bp = pairs + g0;
        if (zn) {
            ZnPhase Z;
            memset(&Z, 0, sizeof(Z));
            Z.npairs = m;
            for (int i = 0; i < m; ++i) {
                ZnArgs &z = Z.a[i];
                z.H = bp[i].H[0];
                z.W = bp[i].W[0];
                z.src_pitch = bp[i].W[0];
                z.dst_pitch = bp[i].pitch[0];
                z.tiles_x = (z.W + ZN_T - 1) / ZN_T;
                z.tiles = z.tiles_x * ((z.H + ZN_T - 1) / ZN_T);
                z.first_image = bp[i].first_image;
                for (int k = 0; k < 2; ++k) {
                    z.src[k] = bp[i].raw[k];
                    z.dst[k] = bp[i].pyr[k] + bp[i].off[0];
                }
                Z.prefix[i + 1] = Z.prefix[i] + z.tiles * (2 - z.first_image);
            }
            if ((e = launch_phase_zn(Z, p0.in_format, p0.storage, st)) != cudaSuccess) return e;
        }
        // pyramid passes: level ls -> ls + 1; without the normalisation the first pass
        // reads the camera images and stores level 0 as well
        for (int ls = 0; ls < (L > 1 ? L - 1 : (zn ? 0 : 1)); ++ls) {
            const bool first = !zn && ls == 0;
            PyrPhase Q;
            memset(&Q, 0, sizeof(Q));
            Q.npairs = m;
            for (int i = 0; i < m; ++i) {
                PyrArgs &a = Q.a[i];
                const int ld = ls + 1;
                a.H = bp[i].H[ls];
                a.W = bp[i].W[ls];
                a.Ho = (a.H + 1) / 2;
                a.Wo = (a.W + 1) / 2;
                a.dst_pitch = ld < L ? bp[i].pitch[ld] : 0;
                a.tiles_x = (a.Wo + PYR_TW - 1) / PYR_TW;
                a.tiles = a.tiles_x * ((a.Ho + PYR_TH - 1) / PYR_TH);
                a.first_image = bp[i].first_image;
                for (int k = 0; k < 2; ++k) {
                    a.dst[k] = ld < L ? bp[i].pyr[k] + bp[i].off[ld] : nullptr;
                    a.dst0[k] = first ? bp[i].pyr[k] + bp[i].off[0] : nullptr;
                    a.src[k] = first ? bp[i].raw[k] : bp[i].pyr[k] + bp[i].off[ls];
                }
                a.src_pitch = first ? bp[i].W[0] : bp[i].pitch[ls];
                a.dst0_pitch = first ? bp[i].pitch[0] : 0;
                Q.prefix[i + 1] = Q.prefix[i] + a.tiles * (2 - a.first_image);
            }
            if ((e = launch_phase_pyr(Q, first, p0.in_format, p0.storage, st)) != cudaSuccess) return e;
        }
        // iterations, coarsest level first; flow buffers ping-pong (one swap per launch). With
        // fusion 2, iterations it and it + 1 of a level (it >= 1) run as one launch.
        const bool i1grad = (p0.flags & OF_FLAG_I1GRAD) != 0;
        const bool fuse = t.fusion == 2 && !i1grad;
        int cur = 0;
        for (int k = 0; k < L * p0.iterations; ++k, cur = 1 - cur) {
            const int l = L - 1 - k / p0.iterations, it = k % p0.iterations;
            const bool two = fuse && it >= 1 && it + 1 < p0.iterations;   // iterations it, it + 1
            const int last = two ? it + 1 : it;   // the iteration whose estimate this launch writes
            if (i1grad && it == 0) {
                // the variant's window matrices of this level, from I1 alone
                HessPhase Hp;
                memset(&Hp, 0, sizeof(Hp));
                Hp.npairs = m;
                for (int i = 0; i < m; ++i) {
                    HessArgs &h = Hp.a[i];
                    h.I1 = bp[i].pyr[0] + bp[i].off[l];
                    h.H = bp[i].H[l];
                    h.W = bp[i].W[l];
                    h.pitch = bp[i].pitch[l];
                    h.hess = bp[i].hess;
                    h.hess_pitch = bp[i].pitch[l];
                    h.tiles_x = (h.W + LK_TW - 1) / LK_TW;
                    h.tiles = h.tiles_x * ((h.H + I1_TH - 1) / I1_TH);
                    Hp.prefix[i + 1] = Hp.prefix[i] + h.tiles;
                }
                if ((e = launch_phase_hess(Hp, level_elem(p0, l), p0.radius, t.generic_sums != 0, st)) != cudaSuccess)
                    return e;
            }
            IterPhase I;
            memset(&I, 0, sizeof(I));
            I.npairs = m;
            I.ahead = prefetch_ahead;
            // strips as long as the tuning's while the launch keeps OF_STRIP_WAVES blocks per
            // resident block slot (4 per SM) or more; the fields do not depend on the strip length
            int kl = strip;
            if (kl > 1) {
                long tiles_l = 0;
                for (int i = 0; i < m; ++i)
                    tiles_l += strip_units(bp[i].H[l], bp[i].W[l], tile_h, 1);
                while (kl > 1 && tiles_l < (long)kl * OF_STRIP_WAVES * 4 * sms) kl /= 2;
            }
            for (int i = 0; i < m; ++i) {
                IterArgs &a = I.a[i];
                a.I1 = bp[i].pyr[0] + bp[i].off[l];
                a.I2 = bp[i].pyr[1] + bp[i].off[l];
                a.H = bp[i].H[l];
                a.W = bp[i].W[l];
                a.pitch = bp[i].pitch[l];
                a.fin = bp[i].flow[cur];
                a.fin_pitch = bp[i].pitch[l];
                if (it == 0 && l == L - 1) {
                    a.mode = FLOW_ZERO;
                } else if (it == 0) {
                    a.mode = FLOW_UPSAMPLE;
                    a.fin_pitch = bp[i].pitch[l + 1];
                    a.Hc = bp[i].H[l + 1];
                    a.Wc = bp[i].W[l + 1];
                } else {
                    a.mode = FLOW_SAME;
                }
                if (l == 0 && last == p0.iterations - 1) {
                    a.u_out = bp[i].u;
                    a.v_out = bp[i].v;
                } else {
                    a.fout = bp[i].flow[1 - cur];
                    a.fout_pitch = bp[i].pitch[l];
                }
                a.tiles_x = (a.W + LK_TW - 1) / LK_TW;
                // the variant's kernels and the fused kernel have their own tile height
                const int th = i1grad ? I1_TH : (two ? LK_TH : tile_h);
                a.strip = (i1grad || two) ? 1 : kl;
                a.tiles = strip_units(a.H, a.W, th, a.strip);
                a.status = bp[i].status;
                a.stage_i2 = (i1grad || two) ? 0 : stage;   // the fused kernel gathers
                if (a.stage_i2) fill_stage_maps(a, I.m[i], level_elem(p0, l), p0.radius, tile_h);   // else gathered
                a.hess = bp[i].hess;
                a.hess_pitch = bp[i].pitch[l];
                I.prefix[i + 1] = I.prefix[i] + a.tiles;
            }
            e = i1grad ? launch_phase_i1_iter(I, level_elem(p0, l), p0.radius, t.generic_sums != 0, p0.fp64_cond, st)
                : two  ? launch_phase_iter2(I, level_elem(p0, l), p0.radius, p0.fp64_cond, st)
                       : launch_phase_iter(I, level_elem(p0, l), p0.radius, t.generic_sums != 0, p0.fp64_cond, tile_h,
                                           st);
            if (e != cudaSuccess) return e;
            if (two) ++k;   // both iterations done
        }
    }
    return cudaSuccess;
}

// Side streams and events of the concurrent launch sequences, per calling thread and
// device, kept until the thread exits (work still queued on them runs to completion).
// Batches launched directly (no graph) from different threads therefore queue their
// extra sequences on different streams and do not wait for one another; a thread's own
// batches share its side streams. Inside a capture the forks become graph branches.
struct Forks {
    cudaStream_t s[3] = {};
    cudaEvent_t fork = nullptr, join[3] = {};
};

struct ThreadForks {
    std::map<int, Forks> all;
    ~ThreadForks()
    {
        for (auto &kv : all) {
            Forks &f = kv.second;
            if (f.fork) cudaEventDestroy(f.fork);
            for (int b = 0; b < 3; ++b) {
                if (f.s[b]) cudaStreamDestroy(f.s[b]);
                if (f.join[b]) cudaEventDestroy(f.join[b]);
            }
        }
    }
};

static Forks *forks_for_device()
{
    thread_local ThreadForks forks;
    std::map<int, Forks> &all = forks.all;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    auto it = all.find(dev);
    if (it != all.end()) return &it->second;
    Forks f;
    bool ok = cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming) == cudaSuccess;
    for (int b = 0; b < 3 && ok; ++b)
        ok = cudaStreamCreateWithFlags(&f.s[b], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&f.join[b], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        if (f.fork) cudaEventDestroy(f.fork);
        for (int b = 0; b < 3; ++b) {
            if (f.s[b]) cudaStreamDestroy(f.s[b]);
            if (f.join[b]) cudaEventDestroy(f.join[b]);
        }
        return nullptr;
    }
    return &(all[dev] = f);
}

// The phase launches of a batch on `st`. With branches > 1 the pairs are split into that
// many runs of about equal level-0 pixel counts whose launch sequences are forked from
// `st` onto side streams and joined back (inside a capture they become parallel branches
// of one graph): each run's launches fill the last waves of the others'.
static cudaError_t enqueue_phased(const std::vector<BatchPair> &pairs, const of_plan &p0, const Tuning &t,
                                  cudaStream_t st, int branches)
{
    const int n = (int)pairs.size();
    const int nb = branches < n ? branches : n;
    if (nb <= 1) return enqueue_chain(pairs.data(), n, p0, t, st);
    Forks *f = forks_for_device();
    if (!f) return cudaErrorUnknown;
    double total = 0.0;
    for (const BatchPair &bp : pairs) total += (double)bp.H[0] * bp.W[0];
    int bound[5] = {0};
    {
        double acc = 0.0;
        int k = 1;
        for (int i = 0; i < n && k < nb; ++i) {
            acc += (double)pairs[i].H[0] * pairs[i].W[0];
            // run k - 1 ends after pair i once it holds its share; every run keeps a pair
            if (acc >= total * k / nb && i + 1 >= k && n - (i + 1) >= nb - k) bound[k++] = i + 1;
        }
        for (; k < nb; ++k) bound[k] = bound[k - 1] + 1;   // shares not reached: one pair each
        bound[nb] = n;
    }
    cudaError_t e = cudaEventRecord(f->fork, st);
    for (int b = 1; b < nb && e == cudaSuccess; ++b) e = cudaStreamWaitEvent(f->s[b - 1], f->fork, 0);
    for (int b = 0; b < nb && e == cudaSuccess; ++b)
        e = enqueue_chain(pairs.data() + bound[b], bound[b + 1] - bound[b], p0, t, b ? f->s[b - 1] : st);
    // join every side stream, also after an error, so that no forked work is left unjoined
    for (int b = 1; b < nb; ++b) {
        const cudaError_t j = cudaEventRecord(f->join[b - 1], f->s[b - 1]) == cudaSuccess
                                  ? cudaStreamWaitEvent(st, f->join[b - 1], 0)
                                  : cudaErrorUnknown;
        if (e == cudaSuccess) e = j;
    }
    return e;
}

// The variant with the first image's gradient runs as phase launches only (it has no
// persistent form) and gathers its 4 taps (no staging).
static Tuning effective(const of_plan &p0, Tuning t)
{
    if (p0.flags & OF_FLAG_I1GRAD) {
        t.phased = 1;
        t.blocks_per_sm = 0;
        t.stage_i2 = 0;
        t.tile_h = 0;
        t.fusion = 0;
    }
    if (!t.phased || t.generic_sums || !radius_specialised(p0.radius) || (t.tile_h != 0 && t.tile_h != LK_TH))
        t.fusion = 0;
    return t;
}

static int commit_state(int32_t n, const of_handle *hs, const BatchBuild &b, cudaStream_t st)
{
    for (int i = 0; i < n; ++i) {
        of_ctx *h = hs[i];
        h->prev_slot = b.s2[i];
        h->has_prev = true;
        h->last_s1 = b.s1[i];
        h->last_s2 = b.s2[i];
        h->computed = true;
        if (cudaEventRecord(h->done, st) != cudaSuccess) return OF_ECUDA;
    }
    return OF_OK;
}

// ------------------------------------------------------------- reusable slots
int batch_slot_init(BatchSlot &s, int max_pairs, int max_phases)
{
    s.max_pairs = max_pairs;
    s.max_phases = max_phases;
    const size_t bytes = (sizeof(BatchPair) * max_pairs + sizeof(int32_t) * (size_t)max_phases * (max_pairs + 1) +
                          255) / 256 * 256;
    s.desc_bytes = bytes;
    if (dev_malloc((void **)&s.dev, bytes + 256) != cudaSuccess) {
        cudaGetLastError();
        return OF_ENOMEM;
    }
    if (cudaMallocHost((void **)&s.host, bytes) != cudaSuccess ||
        cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        batch_slot_free(s);
        return OF_ENOMEM;
    }
    return OF_OK;
}

void batch_slot_free(BatchSlot &s)
{
    if (s.done) cudaEventSynchronize(s.done);
    if (s.done) cudaEventDestroy(s.done);
    if (s.host) cudaFreeHost(s.host);
    if (s.dev) cudaFree(s.dev);
    s = BatchSlot();
}

// One persistent launch on `st` from a preallocated slot: the descriptors go through
// the slot's pinned buffer with one asynchronous copy; no allocation, no graph. The
// slot must not be in use by an unfinished launch (its `done` event).
int batch_run_slot(BatchSlot &slot, int32_t n, const of_handle *hs, const void *const *I1s, const void *const *I2s,
                   float *const *us, float *const *vs, cudaStream_t st)
{
    if (n == 0) return OF_OK;
    BatchBuild b;
    int rc = build_batch(n, hs, I1s, I2s, us, vs, b);
    if (rc) return rc;
    if (n > slot.max_pairs || b.nphases > slot.max_phases) return OF_EINVAL;
    const of_plan &p0 = hs[0]->plan;
    const size_t pairs_bytes = sizeof(BatchPair) * n, prefix_bytes = sizeof(int32_t) * b.prefix.size();
    const size_t bar_off = bar_offset(b);
    memcpy(slot.host, b.pairs.data(), pairs_bytes);
    memcpy(slot.host + pairs_bytes, b.prefix.data(), prefix_bytes);
    const Tuning t = effective(p0, tuning_for(p0, batch_size_class(n, hs)));
    if (t.phased) {
        if (enqueue_phased(b.pairs, p0, t, st, 1) != cudaSuccess || cudaEventRecord(slot.done, st) != cudaSuccess)
            return OF_ECUDA;
        return commit_state(n, hs, b, st);
    }
    const Resolved rv = resolve(p0, t);
    BatchHdr hd;
    fill_header(hd, p0, b, slot.dev, bar_off);
    void *fn = rv.fn;
    const size_t smem = rv.smem;
    dim3 grid;
    if ((rc = grid_for(fn, smem, hs[0]->device, b.max_items, t.blocks_per_sm, grid))) return rc;
    if (cudaMemcpyAsync(slot.dev, slot.host, pairs_bytes + prefix_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(hd.barrier, 0, 2 * sizeof(unsigned int), st) != cudaSuccess)
        return OF_ECUDA;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(LK_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *args[] = {(void *)&hd};
    if (cudaLaunchKernelExC(&cfg, fn, args) != cudaSuccess || cudaEventRecord(slot.done, st) != cudaSuccess)
        return OF_ECUDA;
    return commit_state(n, hs, b, st);
}

}  // namespace of

namespace of {

// One batched launch with an explicit tuning, through the cache of captured launches.
int run_batch(int32_t n, const of_handle *hs, const void *const *I1s, const void *const *I2s, float *const *us,
              float *const *vs, cudaStream_t st, const Tuning &t_in)
{
    if (n == 0) return OF_OK;
    if (!hs || !hs[0]) return OF_EINVAL;
    const Tuning t = effective(hs[0]->plan, t_in);
    BatchBuild b;
    int rc = build_batch(n, hs, I1s, I2s, us, vs, b);
    if (rc) return rc;
    const of_plan &p0 = hs[0]->plan;
    const size_t pairs_bytes = sizeof(BatchPair) * n, prefix_bytes = sizeof(int32_t) * b.prefix.size();
    std::vector<char> key(pairs_bytes + prefix_bytes + sizeof(st) + 7 * sizeof(int));
    {
        char *k = key.data();
        memcpy(k, b.pairs.data(), pairs_bytes);
        memcpy(k + pairs_bytes, b.prefix.data(), prefix_bytes);
        memcpy(k + pairs_bytes + prefix_bytes, &st, sizeof(st));
        const int extra[7] = {p0.radius,
                              (int)(p0.iterations * 16 + (p0.flags & (OF_FLAG_GATHER | OF_FLAG_ZNSSD | OF_FLAG_I1GRAD))),
                              hs[0]->device, t.generic_sums, t.stage_i2,
                              t.blocks_per_sm + 256 * t.phased + 65536 * t.prefetch + (1 << 24) * (t.tile_h != 0),
                              t.phased ? t.branches + 16 * t.fusion + 256 * tuning_strip(t) : 0};
        memcpy(k + pairs_bytes + prefix_bytes + sizeof(st), extra, sizeof(extra));
    }

    std::lock_guard<std::mutex> lk(g_mu);
    ++g_clock;
    BatchEntry *e = nullptr;
    for (auto &c : g_cache)
        if (c.dev && c.key == key) e = &c;
    if (!e) {
        BatchEntry *slot = &g_cache[0];
        for (auto &c : g_cache) {
            if (!c.dev) { slot = &c; break; }
            if (c.last_use < slot->last_use) slot = &c;
        }
        release(*slot);
        BatchEntry &ne = *slot;
        ne.key = key;
        ne.device = hs[0]->device;
        const size_t bar_off = bar_offset(b);
        cudaError_t err = cudaMalloc((void **)&ne.dev, bar_off + 256);
        if (err != cudaSuccess) {
            cudaGetLastError();
            ne = BatchEntry();
            return err == cudaErrorMemoryAllocation ? OF_ENOMEM : OF_ECUDA;
        }
        if (cudaMemcpy(ne.dev, b.pairs.data(), pairs_bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(ne.dev + pairs_bytes, b.prefix.data(), prefix_bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaEventCreateWithFlags(&ne.done, cudaEventDisableTiming) != cudaSuccess) {
            release(ne);
            return OF_ECUDA;
        }
        const Resolved rv = resolve(p0, t);
        fill_header(ne.hdr, p0, b, ne.dev, bar_off);
        ne.fn = rv.fn;
        ne.smem = rv.smem;
        ne.phased = t.phased;
        ne.plan = p0;
        ne.tuning = t;
        if (t.phased) ne.pairs = b.pairs;
        if ((rc = grid_for(ne.fn, ne.smem, ne.device, b.max_items, t.blocks_per_sm, ne.grid))) {
            release(ne);
            return rc;
        }
        // capture [reset barrier, persistent kernel] or the phase launches as a graph when
        // the stream allows it
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        const bool graphs = st != nullptr && !(p0.flags & OF_FLAG_NO_GRAPH) &&
                            cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
        if (graphs) {
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const cudaError_t le = ne.phased ? enqueue_phased(ne.pairs, ne.plan, ne.tuning, st, ne.tuning.branches)
                                                 : launch_direct(ne, st);
                const cudaError_t ce = cudaStreamEndCapture(st, &g);
                if (le == cudaSuccess && ce == cudaSuccess && g &&
                    cudaGraphInstantiate(&ne.exec, g, 0) != cudaSuccess)
                    ne.exec = nullptr;
                if (g) cudaGraphDestroy(g);
            }
            cudaGetLastError();   // a failed capture falls back to direct launches
        }
        e = &ne;
    }
    e->last_use = g_clock;
    cudaError_t err = e->exec ? cudaGraphLaunch(e->exec, st)
                              : (e->phased ? enqueue_phased(e->pairs, e->plan, e->tuning, st, e->tuning.branches)
                                           : launch_direct(*e, st));
    if (err != cudaSuccess) return OF_ECUDA;
    if (cudaEventRecord(e->done, st) != cudaSuccess) return OF_ECUDA;
    return commit_state(n, hs, b, st);
}

}  // namespace of

extern "C" int of_compute_batch(int32_t n, const of_handle *hs, const void *const *I1s, const void *const *I2s,
                                float *const *us, float *const *vs, of_stream_t stream)
{
    if (n <= 0) return n == 0 ? OF_OK : OF_EINVAL;
    if (!hs || !hs[0]) return OF_EINVAL;
    const Tuning t = tuning_for(hs[0]->plan, batch_size_class(n, hs));
    return run_batch(n, hs, I1s, I2s, us, vs, reinterpret_cast<cudaStream_t>(stream), t);
}
