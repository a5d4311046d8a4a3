// Device side of the persistent batched launch: descriptors, the bounded grid barrier
// and the kernel (instantiated per window radius in the radius_*.cu files).
//
// The method's steps for all pairs are cut into phases: the pyramid passes, then the
// iterations level by level (coarsest first). Within a phase, the tiles of all pairs
// form one flat work list that the resident blocks stride through, so small levels of
// one pair share the GPU with large levels of another; a grid-wide barrier separates
// phases (an iteration reads the whole previous iterate through its window halo). The
// barrier's wait is bounded: past its time limit a block records OF_ETIMEOUT in every
// pair's status word, raises an abort flag that releases the other blocks, and returns.
#pragma once

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
    float4 *hess;                       // window matrices of the first-image-gradient variant (or NULL)
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
    int32_t znssd;                      // phase 0 normalises the images (Eq. 2)
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
__device__ __forceinline__ bool bounded_wait_ge(const volatile unsigned int *word, unsigned int target, const volatile int *abort,
                                long long timeout_ns)
{
    const unsigned long long t0 = gtimer();
    const long long cap = timeout_ns / 256 + 100000;
    for (long long it = 0;; ++it) {
        if (*word >= target) return true;
        if (abort && *abort) return false;
        if ((long long)(gtimer() - t0) > timeout_ns || it > cap) return false;
        __nanosleep(256);
    }
}

__device__ __forceinline__ bool grid_barrier(const BatchHdr &hd, unsigned int target)
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

template <typename Tin, typename T, int R>
__global__ void __launch_bounds__(LK_THREADS, batch_min_blocks<R>()) batch_kernel(BatchHdr hd)
{
    extern __shared__ float4 smem4[];
    float *smem = reinterpret_cast<float *>(smem4);
    const int P = hd.npairs;
    uint32_t mbar_phase = 0;
    bool live = true;   // false once a staging copy timed out: the block only keeps the barrier
    lk_tile_prepare<R>(smem);
    for (int phase = 0; phase < hd.nphases; ++phase) {
        const int32_t *pre = hd.prefix + (size_t)phase * (P + 1);
        const int total = pre[P];
        for (int item = blockIdx.x; live && item < total; item += gridDim.x) {
            const int pi = find_pair(pre, P, item);
            const BatchPair &bp = hd.pairs[pi];
            const int j = item - pre[pi];
            if (phase < hd.npyr) {
                if (hd.znssd && phase == 0) {
                    // local normalisation (Eq. 2): raw -> level 0 at the storage precision
                    ZnArgs z;
                    z.H = bp.H[0];
                    z.W = bp.W[0];
                    z.src_pitch = bp.W[0];
                    z.dst_pitch = bp.pitch[0];
                    z.tiles_x = (z.W + ZN_T - 1) / ZN_T;
                    z.tiles = z.tiles_x * ((z.H + ZN_T - 1) / ZN_T);
                    z.first_image = bp.first_image;
                    for (int k = 0; k < 2; ++k) {
                        z.src[k] = bp.raw[k];
                        z.dst[k] = bp.pyr[k] + bp.off[0];
                    }
                    const int img = bp.first_image + j / z.tiles;
                    znssd_tile<Tin, T, true>(z, j - (j / z.tiles) * z.tiles, img, smem);   // caller images: read-only
                    continue;
                }
                // pyramid pass: level ls -> ls + 1 (the first pass of the plain path reads raw)
                const int ls = hd.znssd ? phase - 1 : phase, ld = ls + 1;
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
                if (!hd.znssd && phase == 0) {
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
                a.hess = nullptr;
                a.hess_pitch = 0;
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
                a.strip = 1;
                a.status = bp.status;
                a.stage_i2 = 0;   // no tensor maps: the TMA staging needs them in parameter space
                if (l == 0 && !hd.znssd)
                    live = lk_tile<Tin, false, R, -1, LK_TH, false>(a, nullptr, j, hd.radius, hd.fp64_cond, smem, mbar_phase);
                else
                    live = lk_tile<T, false, R, -1, LK_TH, false>(a, nullptr, j, hd.radius, hd.fp64_cond, smem, mbar_phase);
            }
        }
        if (phase + 1 < hd.nphases && !grid_barrier(hd, (unsigned int)(phase + 1) * gridDim.x)) return;
    }
}

}  // namespace of
