// C ABI of libof (include/of.h): plan validation, workspace layout, the per-pair launch
// sequence of the coarse-to-fine method (Sect. 2.4), CUDA-graph replay, status words.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>

#include "of_engine.h"
#include "of_internal.cuh"

using namespace of;

namespace {

constexpr int kPitchAlign = 64;       // elements per row are a multiple of this (>= 128 B)
constexpr size_t kAlign = 256;        // byte alignment of every buffer in the workspace

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
int pitch_of(int W) { return (W + kPitchAlign - 1) / kPitchAlign * kPitchAlign; }

int map_cuda(cudaError_t e) { return e == cudaSuccess ? OF_OK : (e == cudaErrorMemoryAllocation ? OF_ENOMEM : OF_ECUDA); }

std::mutex g_dev_mu;
bool g_dev_configured[256];

int configure_device()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return OF_ECUDA;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (dev < 0 || dev >= 256) return OF_ECUDA;
    if (g_dev_configured[dev]) return OF_OK;
    if (configure_lk_kernels() != cudaSuccess) return OF_ECUDA;
    g_dev_configured[dev] = true;
    return OF_OK;
}

}  // namespace

namespace of {

static std::atomic<int> g_fail_allocs{0};

cudaError_t dev_malloc(void **p, size_t bytes)
{
    int n = g_fail_allocs.load();
    while (n > 0) {
        if (g_fail_allocs.compare_exchange_weak(n, n - 1)) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMalloc(p, bytes);
}

// Layout of one plan's workspace (all offsets 256-byte aligned):
//   pyramid slot 0 | pyramid slot 1 | flow buffer 0 | flow buffer 1 | status word
//   [| window matrices (OF_FLAG_I1GRAD: one float4 per pixel of level 0, reused per level)]
// A pyramid slot holds levels 0..L-1 of one image: level 0 in the input's integer
// format, levels >= 1 at the storage precision. A flow buffer holds the interleaved
// (u, v) float2 field of the largest level.
void layout_plan(const of_plan &p, Layout &L)
{
    memset(&L, 0, sizeof(L));
    L.levels = p.levels;
    int H = p.H, W = p.W;
    size_t off = 0;
    for (int l = 0; l < p.levels; ++l) {
        L.H[l] = H;
        L.W[l] = W;
        L.pitch[l] = pitch_of(W);
        L.level_off[l] = off;
        off = align_up(off + (size_t)L.pitch[l] * H * elem_bytes(level_elem(p, l)), kAlign);
        H = (H + 1) / 2;
        W = (W + 1) / 2;
    }
    L.pyr_bytes = off;
    L.flow_bytes = align_up((size_t)L.pitch[0] * L.H[0] * sizeof(float2), kAlign);
    L.hess_off = 2 * L.pyr_bytes + 2 * L.flow_bytes + kAlign;
    L.hess_bytes = (p.flags & OF_FLAG_I1GRAD) ? align_up((size_t)L.pitch[0] * L.H[0] * sizeof(float4), kAlign) : 0;
    L.total = L.hess_off + L.hess_bytes;
}

void assign_workspace(of_ctx *h, char *ws)
{
    const Layout &L = h->lay;
    h->ws = ws;
    h->pyr[0] = ws;
    h->pyr[1] = ws + L.pyr_bytes;
    h->flow[0] = reinterpret_cast<float2 *>(ws + 2 * L.pyr_bytes);
    h->flow[1] = reinterpret_cast<float2 *>(ws + 2 * L.pyr_bytes + L.flow_bytes);
    h->status = reinterpret_cast<int *>(ws + 2 * L.pyr_bytes + 2 * L.flow_bytes);
    h->hess = L.hess_bytes ? reinterpret_cast<float4 *>(ws + L.hess_off) : nullptr;
}

// Queue the whole method for one pair (Sect. 2.4): pyramids, then n iterations on every
// level from the coarsest (zero start) to level 0, the first iteration of each finer
// level reading the coarser result through the x2 upsampling.
cudaError_t enqueue_pair(of_ctx *h, const void *I1, const void *I2, float *u, float *v, int s1, int s2,
                         cudaStream_t st)
{
    const of_plan &p = h->plan;
    const Layout &L = h->lay;
    cudaError_t e;
    // pyramids: first pass (raw -> level 0 and level 1), then one pass per further
    // level; with the normalisation of Eq. 2, a normalisation pass (raw -> level 0) and
    // then one reduction per level from level 0
    {
        const int sl[2] = {s1, s2};
        PyrArgs a;
        memset(&a, 0, sizeof(a));
        a.first_image = I1 ? 0 : 1;
        int lfirst;   // first level reduced by pyr_down
        if (p.flags & OF_FLAG_ZNSSD) {
            ZnArgs z;
            memset(&z, 0, sizeof(z));
            z.src[0] = I1;
            z.src[1] = I2;
            for (int k = 0; k < 2; ++k) z.dst[k] = h->pyr[sl[k]] + L.level_off[0];
            z.H = L.H[0];
            z.W = L.W[0];
            z.src_pitch = L.W[0];
            z.dst_pitch = L.pitch[0];
            z.first_image = a.first_image;
            z.tiles_x = (z.W + ZN_T - 1) / ZN_T;
            z.tiles = z.tiles_x * ((z.H + ZN_T - 1) / ZN_T);
            if ((e = launch_znssd(z, p.in_format, p.storage, st)) != cudaSuccess) return e;
            lfirst = 0;
        } else {
            a.src[0] = I1;
            a.src[1] = I2;
            for (int k = 0; k < 2; ++k) {
                a.dst0[k] = h->pyr[sl[k]] + L.level_off[0];
                a.dst[k] = p.levels > 1 ? h->pyr[sl[k]] + L.level_off[1] : nullptr;
            }
            a.H = L.H[0];
            a.W = L.W[0];
            a.src_pitch = L.W[0];
            a.dst0_pitch = L.pitch[0];
            a.Ho = (L.H[0] + 1) / 2;
            a.Wo = (L.W[0] + 1) / 2;
            a.dst_pitch = p.levels > 1 ? L.pitch[1] : 0;
            a.tiles_x = (a.Wo + PYR_TW - 1) / PYR_TW;
            a.tiles = a.tiles_x * ((a.Ho + PYR_TH - 1) / PYR_TH);
            if ((e = launch_pyr_first(a, p.in_format, p.storage, st)) != cudaSuccess) return e;
            lfirst = 1;
        }
        for (int l = lfirst; l + 1 < p.levels; ++l) {
            for (int k = 0; k < 2; ++k) {
                a.src[k] = h->pyr[sl[k]] + L.level_off[l];
                a.dst0[k] = nullptr;
                a.dst[k] = h->pyr[sl[k]] + L.level_off[l + 1];
            }
            a.H = L.H[l];
            a.W = L.W[l];
            a.src_pitch = L.pitch[l];
            a.Ho = L.H[l + 1];
            a.Wo = L.W[l + 1];
            a.dst_pitch = L.pitch[l + 1];
            a.tiles_x = (a.Wo + PYR_TW - 1) / PYR_TW;
            a.tiles = a.tiles_x * ((a.Ho + PYR_TH - 1) / PYR_TH);
            if ((e = launch_pyr_down(a, p.storage, st)) != cudaSuccess) return e;
        }
    }
    // iterations
    const bool i1grad = (p.flags & OF_FLAG_I1GRAD) != 0;
    int cur = 0;
    for (int l = p.levels - 1; l >= 0; --l) {
        if (i1grad) {
            // the variant's window matrix of this level, from I1 alone
            HessArgs ha;
            ha.I1 = h->pyr[s1] + L.level_off[l];
            ha.H = L.H[l];
            ha.W = L.W[l];
            ha.pitch = L.pitch[l];
            ha.hess = h->hess;
            ha.hess_pitch = L.pitch[l];
            ha.tiles_x = (ha.W + LK_TW - 1) / LK_TW;
            ha.tiles = ha.tiles_x * ((ha.H + I1_TH - 1) / I1_TH);
            if ((e = launch_i1_hess(ha, level_elem(p, l), p.radius, st)) != cudaSuccess) return e;
        }
        for (int it = 0; it < p.iterations; ++it) {
            IterArgs a;
            memset(&a, 0, sizeof(a));
            a.I1 = h->pyr[s1] + L.level_off[l];
            a.I2 = h->pyr[s2] + L.level_off[l];
            a.H = L.H[l];
            a.W = L.W[l];
            a.pitch = L.pitch[l];
            if (it == 0 && l == p.levels - 1) {
                a.mode = FLOW_ZERO;
            } else if (it == 0) {
                a.mode = FLOW_UPSAMPLE;
                a.fin = h->flow[cur];
                a.fin_pitch = L.pitch[l + 1];
                a.Hc = L.H[l + 1];
                a.Wc = L.W[l + 1];
            } else {
                a.mode = FLOW_SAME;
                a.fin = h->flow[cur];
                a.fin_pitch = L.pitch[l];
            }
            const bool last = (l == 0 && it == p.iterations - 1);
            if (last) {
                a.u_out = u;
                a.v_out = v;
            } else {
                a.fout = h->flow[1 - cur];
                a.fout_pitch = L.pitch[l];
            }
            a.tiles_x = (a.W + LK_TW - 1) / LK_TW;
            const int th = i1grad ? I1_TH : LK_TH;   // the variant's kernels have their own tile height
            a.strip = 1;   // one tile per block: the most blocks for one pair
            a.tiles = strip_units(a.H, a.W, th, a.strip);
            a.status = h->status;
            a.stage_i2 = !(p.flags & OF_FLAG_GATHER) && !i1grad ? 1 : 0;
            StageMaps maps;
            memset(&maps, 0, sizeof(maps));
            if (a.stage_i2) fill_stage_maps(a, maps, level_elem(p, l), p.radius, LK_TH);   // else gathered
            if (i1grad) {
                a.hess = h->hess;
                a.hess_pitch = L.pitch[l];
                e = launch_i1_iter(a, level_elem(p, l), p.radius, p.fp64_cond, st);
            } else {
                e = launch_lk_iter(a, maps, level_elem(p, l), p.radius, p.fp64_cond, st);
            }
            if (e != cudaSuccess) return e;
            cur = 1 - cur;
        }
    }
    return cudaSuccess;
}

}  // namespace of

// ----------------------------------------------------------------------- C ABI
extern "C" {

void of_plan_init(of_plan *p, int32_t H, int32_t W)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->H = H;
    p->W = W;
    p->levels = 3;
    p->radius = 4;
    p->iterations = 5;
    p->in_format = OF_U8;
    p->in_bits = 8;
    p->storage = OF_F32;
    p->fp64_cond = 1e3f;
    p->flags = 0;
}

int of_plan_validate(const of_plan *p)
{
    if (!p) return OF_EINVAL;
    if (p->H < 1 || p->W < 1 || p->H > 32768 || p->W > 32768) return OF_EINVAL;
    if ((int64_t)p->H * p->W > (int64_t(1) << 28)) return OF_EINVAL;
    if (p->levels < 1 || p->levels > MAX_LEVELS) return OF_EINVAL;
    if (p->radius < 1 || p->radius > MAX_RADIUS) return OF_EINVAL;
    if (p->iterations < 1 || p->iterations > 1000) return OF_EINVAL;
    if (p->in_format == OF_U8) {
        if (p->in_bits < 1 || p->in_bits > 8) return OF_EINVAL;
    } else if (p->in_format == OF_U16) {
        if (p->in_bits < 1 || p->in_bits > 16) return OF_EINVAL;
    } else {
        return OF_EINVAL;
    }
    if (p->storage != OF_F32 && p->storage != OF_F16 && p->storage != OF_BF16) return OF_EINVAL;
    if (!(p->fp64_cond >= 0.0f) || isinf(p->fp64_cond)) return OF_EINVAL;
    if (p->flags & ~(OF_FLAG_NO_GRAPH | OF_FLAG_GATHER | OF_FLAG_ZNSSD | OF_FLAG_I1GRAD)) return OF_EINVAL;
    return OF_OK;
}

int of_plan_check(const of_plan *p, float max_disp_px, int *ok)
{
    if (!p || !ok || p->levels < 1 || p->levels > MAX_LEVELS || !(max_disp_px >= 0.0f)) return OF_EINVAL;
    // Eq. 1: (dx)_max / 2^(n_lev - 1) < 3 px
    *ok = ((double)max_disp_px / ldexp(1.0, p->levels - 1)) < 3.0 ? 1 : 0;
    return OF_OK;
}

int of_level_size(const of_plan *p, int32_t level, int32_t *Hl, int32_t *Wl)
{
    if (of_plan_validate(p) != OF_OK || !Hl || !Wl || level < 0 || level >= p->levels) return OF_EINVAL;
    int H = p->H, W = p->W;
    for (int l = 0; l < level; ++l) {
        H = (H + 1) / 2;
        W = (W + 1) / 2;
    }
    *Hl = H;
    *Wl = W;
    return OF_OK;
}

int of_workspace_bytes(const of_plan *p, size_t *bytes)
{
    if (of_plan_validate(p) != OF_OK || !bytes) return OF_EINVAL;
    Layout L;
    layout_plan(*p, L);
    *bytes = L.total;
    return OF_OK;
}

int of_create(const of_plan *p, of_handle *out)
{
    if (!out) return OF_EINVAL;
    *out = nullptr;
    if (of_plan_validate(p) != OF_OK) return OF_EINVAL;
    int rc = configure_device();
    if (rc) return rc;
    of_ctx *h = new (std::nothrow) of_ctx();
    if (!h) return OF_ENOMEM;
    h->plan = *p;
    layout_plan(*p, h->lay);
    cudaGetDevice(&h->device);
    cudaError_t e = dev_malloc((void **)&h->ws, h->lay.total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return map_cuda(e);
    }
    assign_workspace(h, h->ws);
    if ((e = cudaMemset(h->status, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&h->ctl, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaDeviceSynchronize()) != cudaSuccess) {
        of_destroy(h);
        return map_cuda(e);
    }
    *out = h;
    return OF_OK;
}

int of_compute(of_handle h, const void *I1, const void *I2, float *u, float *v, of_stream_t stream)
{
    if (!h || !I2 || !u || !v) return OF_EINVAL;
    if (!I1 && !h->has_prev) return OF_ESTATE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int s1, s2;
    if (I1) {
        s1 = 0;
        s2 = 1;
    } else {
        s1 = h->prev_slot;
        s2 = 1 - h->prev_slot;
    }
    int rc = run_pair(h, I1, I2, u, v, s1, s2, st);
    if (rc) return rc;
    h->prev_slot = s2;
    h->has_prev = true;
    h->last_s1 = s1;
    h->last_s2 = s2;
    h->computed = true;
    return map_cuda(cudaEventRecord(h->done, st));
}

int of_sync_status(of_handle h)
{
    if (!h) return OF_EINVAL;
    int host = 0;
    if (cudaEventSynchronize(h->done) != cudaSuccess) return OF_ECUDA;
    if (cudaMemcpyAsync(&host, h->status, sizeof(int), cudaMemcpyDeviceToHost, h->ctl) != cudaSuccess ||
        cudaMemsetAsync(h->status, 0, sizeof(int), h->ctl) != cudaSuccess || cudaStreamSynchronize(h->ctl) != cudaSuccess)
        return OF_ECUDA;
    if (host == DEV_TIMEOUT) return OF_ETIMEOUT;
    if (host != DEV_OK) return OF_EDEVICE;
    return OF_OK;
}

int of_destroy(of_handle h)
{
    if (!h) return OF_OK;
    int rc = OF_OK;
    if (h->done && cudaEventSynchronize(h->done) != cudaSuccess) rc = OF_ECUDA;
    drop_graphs(h);
    if (h->ctl) cudaStreamDestroy(h->ctl);
    if (h->done) cudaEventDestroy(h->done);
    if (h->ws && cudaFree(h->ws) != cudaSuccess) rc = OF_ECUDA;
    delete h;
    return rc;
}

int of_get_level(of_handle h, int32_t which, int32_t level, float *dst, of_stream_t stream)
{
    if (!h || !dst || which < 0 || which > 1 || level < 0 || level >= h->plan.levels) return OF_EINVAL;
    if (!h->computed) return OF_ESTATE;
    Level l;
    l.ptr = h->pyr[which == 0 ? h->last_s1 : h->last_s2] + h->lay.level_off[level];
    l.H = h->lay.H[level];
    l.W = h->lay.W[level];
    l.pitch = h->lay.pitch[level];
    return map_cuda(launch_level_to_f32(l, level_elem(h->plan, level), dst, reinterpret_cast<cudaStream_t>(stream)));
}

int of_window_sums(const float *ch, int32_t H, int32_t W, int32_t r, float *out, of_stream_t stream)
{
    if (!ch || !out || H < 1 || W < 1 || r < 1 || r > MAX_RADIUS || (int64_t)H * W > (int64_t(1) << 28))
        return OF_EINVAL;
    int rc = configure_device();
    if (rc) return rc;
    return map_cuda(launch_window_sums(ch, H, W, r, out, reinterpret_cast<cudaStream_t>(stream)));
}

int of_debug_wait_timeout(int32_t timeout_us)
{
    if (timeout_us < 1 || timeout_us > 10000000) return OF_EINVAL;
    int *buf = nullptr;
    cudaStream_t s = nullptr;
    int host = 0, rc = OF_OK;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return OF_ECUDA;
    if (cudaMalloc((void **)&buf, 2 * sizeof(int)) != cudaSuccess) {
        cudaStreamDestroy(s);
        return OF_ENOMEM;
    }
    if (cudaMemsetAsync(buf, 0, 2 * sizeof(int), s) != cudaSuccess ||
        launch_wait_timeout(buf, buf + 1, (long long)timeout_us * 1000, s) != cudaSuccess ||
        cudaMemcpyAsync(&host, buf + 1, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        rc = OF_ECUDA;
    cudaFree(buf);
    cudaStreamDestroy(s);
    if (rc) return rc;
    return host == DEV_TIMEOUT ? OF_ETIMEOUT : (host == DEV_OK ? OF_OK : OF_EDEVICE);
}

const char *of_status_string(int s)
{
    switch (s) {
    case OF_OK: return "ok";
    case OF_EINVAL: return "invalid argument";
    case OF_ENOMEM: return "out of device memory or over the memory budget";
    case OF_ECUDA: return "CUDA runtime error";
    case OF_EDEVICE: return "device-side check failed";
    case OF_ETIMEOUT: return "bounded device wait timed out";
    case OF_ESTATE: return "missing state (no previous frame)";
    case OF_EBUSY: return "queue or slot pool full";
    default: return "unknown status";
    }
}

int of_version(void) { return 100; }

int of_debug_fail_allocs(int32_t n) { return of::g_fail_allocs.exchange(n < 0 ? 0 : n); }

}  // extern "C"
