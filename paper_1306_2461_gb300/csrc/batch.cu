// of_compute_batch: many independent pairs (each field is independent of the others,
// Sect. 3.3) in ONE persistent cooperative launch, replayed from a CUDA graph.
//
// The method's steps for all pairs are cut into phases: the pyramid passes, then the
// iterations level by level (coarsest first). Within a phase, the tiles of all pairs
// form one flat work list that the resident blocks stride through, so small levels of
// one pair share the GPU with large levels of another; a grid-wide barrier separates
// phases (an iteration reads the whole previous iterate through its window halo). The
// barrier's wait is bounded: past its time limit a block records OF_ETIMEOUT in every
// pair's status word, raises an abort flag that releases the other blocks, and returns.
#include <string.h>

#include <mutex>
#include <vector>

#include "of_engine.h"
#include "of_internal.cuh"
#include "of_kernels.cuh"

namespace of {

struct BatchPair {
    const void *raw[2];                 // caller images (raw[0] == NULL: first image reused)
    float *u, *v;                       // caller outputs
    char *pyr[2];                       // pyramid slots of the first and second image
    float2 *flow[2];                    // ping-pong flow buffers
    int *status;                        // the handle's device status word
    int32_t first_image;                // 0: build both pyramids, 1: only the second
    int32_t H[MAX_LEVELS], W[MAX_LEVELS], pitch[MAX_LEVELS];
    uint64_t off[MAX_LEVELS];
};

struct BatchHdr {
    const BatchPair *pairs;
    const int32_t *prefix;              // nphases x (npairs + 1) work-item prefix sums
    unsigned int *barrier;              // arrival counter, zeroed before each launch
    int *abort;                         // set when a block gave up waiting
    int32_t npairs, levels, iterations, radius, nphases, npyr;
    float fp64_cond;
    long long timeout_ns;
};

constexpr long long BARRIER_TIMEOUT_NS = 2000000000LL;   // 2 s per phase

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Spin until *word >= target, *abort != 0, or timeout_ns elapses (a matching iteration
// cap bounds the loop even if the timer stalls). Returns true when the target was reached.
__device__ bool bounded_wait_ge(const volatile unsigned int *word, unsigned int target, const volatile int *abort,
                                long long timeout_ns)
{
    const unsigned long long t0 = gtimer();
    const long long cap = timeout_ns / 32 + 100000;
    for (long long it = 0;; ++it) {
        if (*word >= target) return true;
        if (abort && *abort) return false;
        if ((long long)(gtimer() - t0) > timeout_ns || it > cap) return false;
        __nanosleep(32);
    }
}

__device__ bool grid_barrier(const BatchHdr &hd, unsigned int target)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(hd.barrier, 1u);
        bool ok = bounded_wait_ge(hd.barrier, target, hd.abort, hd.timeout_ns);
        if (!ok && atomicExch(hd.abort, 1) == 0) {
            for (int i = 0; i < hd.npairs; ++i) atomicExch(hd.pairs[i].status, DEV_TIMEOUT);
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ int find_pair(const int32_t *pre, int n, int item)
{
    int lo = 0, hi = n - 1;   // largest i with pre[i] <= item
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <typename Tin, typename T>
__global__ void __launch_bounds__(LK_THREADS) batch_kernel(BatchHdr hd)
{
    extern __shared__ float smem[];
    const int P = hd.npairs;
    for (int phase = 0; phase < hd.nphases; ++phase) {
        const int32_t *pre = hd.prefix + (size_t)phase * (P + 1);
        const int total = pre[P];
        for (int item = blockIdx.x; item < total; item += gridDim.x) {
            const int pi = find_pair(pre, P, item);
            const BatchPair &bp = hd.pairs[pi];
            const int j = item - pre[pi];
            if (phase < hd.npyr) {
                // pyramid pass `phase`: level phase -> phase + 1 (the first pass reads raw)
                const int ls = phase, ld = phase + 1;
                PyrArgs a;
                a.H = bp.H[ls];
                a.W = bp.W[ls];
                a.Ho = (a.H + 1) / 2;
                a.Wo = (a.W + 1) / 2;
                a.dst_pitch = ld < hd.levels ? bp.pitch[ld] : 0;
                a.tiles_x = (a.Wo + PYR_TW - 1) / PYR_TW;
                a.tiles = a.tiles_x * ((a.Ho + PYR_TH - 1) / PYR_TH);
                const int img = bp.first_image + j / a.tiles;
                const int tile = j - (j / a.tiles) * a.tiles;
                for (int k = 0; k < 2; ++k) {
                    a.dst[k] = ld < hd.levels ? bp.pyr[k] + bp.off[ld] : nullptr;
                    a.dst0[k] = bp.pyr[k] + bp.off[0];
                }
                if (phase == 0) {
                    a.src[0] = bp.raw[0];
                    a.src[1] = bp.raw[1];
                    a.src_pitch = bp.W[0];
                    a.dst0_pitch = bp.pitch[0];
                    pyr_tile_smem<Tin, T, true, true>(a, tile, img, smem);   // caller images: read-only
                } else {
                    a.src[0] = bp.pyr[0] + bp.off[ls];
                    a.src[1] = bp.pyr[1] + bp.off[ls];
                    a.src_pitch = bp.pitch[ls];
                    pyr_tile_smem<T, T, false, false>(a, tile, img, smem);
                }
            } else {
                const int k = phase - hd.npyr;
                const int l = hd.levels - 1 - k / hd.iterations;
                const int it = k - (k / hd.iterations) * hd.iterations;
                const int cur = k & 1;
                IterArgs a;
                a.I1 = bp.pyr[0] + bp.off[l];
                a.I2 = bp.pyr[1] + bp.off[l];
                a.H = bp.H[l];
                a.W = bp.W[l];
                a.pitch = bp.pitch[l];
                a.fin = bp.flow[cur];
                a.fin_pitch = bp.pitch[l];
                a.Hc = a.Wc = 0;
                if (it == 0 && l == hd.levels - 1) {
                    a.mode = FLOW_ZERO;
                } else if (it == 0) {
                    a.mode = FLOW_UPSAMPLE;
                    a.fin_pitch = bp.pitch[l + 1];
                    a.Hc = bp.H[l + 1];
                    a.Wc = bp.W[l + 1];
                } else {
                    a.mode = FLOW_SAME;
                }
                if (l == 0 && it == hd.iterations - 1) {
                    a.fout = nullptr;
                    a.u_out = bp.u;
                    a.v_out = bp.v;
                } else {
                    a.fout = bp.flow[1 - cur];
                    a.fout_pitch = bp.pitch[l];
                    a.u_out = a.v_out = nullptr;
                }
                a.tiles_x = (a.W + LK_TW - 1) / LK_TW;
                a.tiles = 0;
                if (l == 0) lk_tile<Tin, false>(a, j, hd.radius, hd.fp64_cond, smem);
                else lk_tile<T, false>(a, j, hd.radius, hd.fp64_cond, smem);
            }
        }
        if (phase + 1 < hd.nphases && !grid_barrier(hd, (unsigned int)(phase + 1) * gridDim.x)) return;
    }
}

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

static size_t batch_smem_bytes(int r)
{
    const size_t lk = sizeof(float) * lk_smem_floats(r), pyr = sizeof(float) * PYR_SMEM_FLOATS;
    return lk > pyr ? lk : pyr;
}

template <typename Tin, typename T> static void *kernel_ptr() { return (void *)batch_kernel<Tin, T>; }

static void *batch_kernel_for(int in_format, int storage)
{
    if (in_format == OF_U8) {
        if (storage == OF_F32) return kernel_ptr<uint8_t, float>();
        if (storage == OF_F16) return kernel_ptr<uint8_t, __half>();
        return kernel_ptr<uint8_t, __nv_bfloat16>();
    }
    if (storage == OF_F32) return kernel_ptr<uint16_t, float>();
    if (storage == OF_F16) return kernel_ptr<uint16_t, __half>();
    return kernel_ptr<uint16_t, __nv_bfloat16>();
}

cudaError_t configure_batch_kernels()
{
    const int bytes = (int)batch_smem_bytes(MAX_RADIUS);
    for (int f = 0; f < 2; ++f)
        for (int s = 0; s < 3; ++s) {
            cudaError_t e = cudaFuncSetAttribute(batch_kernel_for(f, s), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 bytes);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
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
};

constexpr int BATCH_CACHE = 8;
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

static bool same_method(const of_plan &a, const of_plan &b)
{
    return a.levels == b.levels && a.radius == b.radius && a.iterations == b.iterations &&
           a.in_format == b.in_format && a.in_bits == b.in_bits && a.storage == b.storage &&
           a.fp64_cond == b.fp64_cond;
}

extern "C" int of_compute_batch(int32_t n, const of_handle *hs, const void *const *I1s, const void *const *I2s,
                                float *const *us, float *const *vs, of_stream_t stream)
{
    if (n == 0) return OF_OK;
    if (n < 0 || n > 65536 || !hs || !I1s || !I2s || !us || !vs) return OF_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (!hs[i] || !I2s[i] || !us[i] || !vs[i]) return OF_EINVAL;
        if (!same_method(hs[i]->plan, hs[0]->plan)) return OF_EINVAL;
        if (!I1s[i] && !hs[i]->has_prev) return OF_ESTATE;
        if (hs[i]->device != hs[0]->device) return OF_EINVAL;
        for (int j = 0; j < i; ++j)
            if (hs[j] == hs[i]) return OF_EINVAL;
    }
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const of_plan &p0 = hs[0]->plan;
    const int L = p0.levels, npyr = L > 1 ? L - 1 : 1, nphases = npyr + L * p0.iterations;

    // descriptors
    std::vector<BatchPair> pairs(n);
    std::vector<int32_t> prefix((size_t)nphases * (n + 1));
    std::vector<int> s1(n), s2(n);
    for (int i = 0; i < n; ++i) {
        of_ctx *h = hs[i];
        s1[i] = I1s[i] ? 0 : h->prev_slot;
        s2[i] = I1s[i] ? 1 : 1 - h->prev_slot;
        BatchPair &bp = pairs[i];
        memset(&bp, 0, sizeof(bp));
        bp.raw[0] = I1s[i];
        bp.raw[1] = I2s[i];
        bp.u = us[i];
        bp.v = vs[i];
        bp.pyr[0] = h->pyr[s1[i]];
        bp.pyr[1] = h->pyr[s2[i]];
        bp.flow[0] = h->flow[0];
        bp.flow[1] = h->flow[1];
        bp.status = h->status;
        bp.first_image = I1s[i] ? 0 : 1;
        for (int l = 0; l < L; ++l) {
            bp.H[l] = h->lay.H[l];
            bp.W[l] = h->lay.W[l];
            bp.pitch[l] = h->lay.pitch[l];
            bp.off[l] = h->lay.level_off[l];
        }
    }
    int max_items = 0;
    for (int ph = 0; ph < nphases; ++ph) {
        int32_t *pre = &prefix[(size_t)ph * (n + 1)];
        pre[0] = 0;
        for (int i = 0; i < n; ++i) {
            const BatchPair &bp = pairs[i];
            int64_t cnt;
            if (ph < npyr) {
                const int Ho = (bp.H[ph] + 1) / 2, Wo = (bp.W[ph] + 1) / 2;
                cnt = (int64_t)((Wo + PYR_TW - 1) / PYR_TW) * ((Ho + PYR_TH - 1) / PYR_TH) * (2 - bp.first_image);
            } else {
                const int l = L - 1 - (ph - npyr) / p0.iterations;
                cnt = (int64_t)((bp.W[l] + LK_TW - 1) / LK_TW) * ((bp.H[l] + LK_TH - 1) / LK_TH);
            }
            if (pre[i] + cnt > INT32_MAX) return OF_EINVAL;
            pre[i + 1] = (int32_t)(pre[i] + cnt);
        }
        if (pre[n] > max_items) max_items = pre[n];
    }
    const size_t pairs_bytes = sizeof(BatchPair) * n, prefix_bytes = sizeof(int32_t) * prefix.size();
    std::vector<char> key(pairs_bytes + prefix_bytes + sizeof(st) + 3 * sizeof(int));
    {
        char *k = key.data();
        memcpy(k, pairs.data(), pairs_bytes);
        memcpy(k + pairs_bytes, prefix.data(), prefix_bytes);
        memcpy(k + pairs_bytes + prefix_bytes, &st, sizeof(st));
        const int extra[3] = {p0.radius, p0.iterations, hs[0]->device};
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
        const size_t bar_off = (pairs_bytes + prefix_bytes + 255) / 256 * 256;
        cudaError_t err = cudaMalloc((void **)&ne.dev, bar_off + 256);
        if (err != cudaSuccess) {
            cudaGetLastError();
            ne = BatchEntry();
            return err == cudaErrorMemoryAllocation ? OF_ENOMEM : OF_ECUDA;
        }
        if (cudaMemcpy(ne.dev, pairs.data(), pairs_bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(ne.dev + pairs_bytes, prefix.data(), prefix_bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaEventCreateWithFlags(&ne.done, cudaEventDisableTiming) != cudaSuccess) {
            release(ne);
            return OF_ECUDA;
        }
        BatchHdr &hd = ne.hdr;
        hd.pairs = reinterpret_cast<const BatchPair *>(ne.dev);
        hd.prefix = reinterpret_cast<const int32_t *>(ne.dev + pairs_bytes);
        hd.barrier = reinterpret_cast<unsigned int *>(ne.dev + bar_off);
        hd.abort = reinterpret_cast<int *>(ne.dev + bar_off + sizeof(unsigned int));
        hd.npairs = n;
        hd.levels = L;
        hd.iterations = p0.iterations;
        hd.radius = p0.radius;
        hd.nphases = nphases;
        hd.npyr = npyr;
        hd.fp64_cond = p0.fp64_cond;
        hd.timeout_ns = BARRIER_TIMEOUT_NS;
        ne.fn = batch_kernel_for(p0.in_format, p0.storage);
        ne.smem = batch_smem_bytes(p0.radius);
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ne.fn, LK_THREADS, ne.smem) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ne.device) != cudaSuccess || per_sm < 1) {
            release(ne);
            return OF_ECUDA;
        }
        int grid = per_sm * sms;
        if (grid > max_items) grid = max_items > 0 ? max_items : 1;
        ne.grid = dim3(grid);
        // capture [reset barrier, persistent kernel] as a graph when the stream allows it
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        const bool graphs = st != nullptr && !(p0.flags & OF_FLAG_NO_GRAPH) &&
                            cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
        if (graphs) {
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const cudaError_t le = launch_direct(ne, st);
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
    cudaError_t err = e->exec ? cudaGraphLaunch(e->exec, st) : launch_direct(*e, st);
    if (err != cudaSuccess) return OF_ECUDA;
    if (cudaEventRecord(e->done, st) != cudaSuccess) return OF_ECUDA;
    for (int i = 0; i < n; ++i) {
        of_ctx *h = hs[i];
        h->prev_slot = s2[i];
        h->has_prev = true;
        h->last_s1 = s1[i];
        h->last_s2 = s2[i];
        h->computed = true;
        if (cudaEventRecord(h->done, st) != cudaSuccess) return OF_ECUDA;
    }
    return OF_OK;
}
