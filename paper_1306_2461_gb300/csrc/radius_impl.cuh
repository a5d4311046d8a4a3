// Kernels and launchers for one window radius. Each radius_<R>.cu defines OF_RADIUS
// and includes this file; radius 0 is the generic kernel (radius given at run time).
#pragma once

#include "batch_device.cuh"
#include "i1grad_kernels.cuh"
#include "of_internal.cuh"
#include "of_kernels.cuh"

#ifndef OF_RADIUS
#error "define OF_RADIUS before including radius_impl.cuh"
#endif

namespace of {

template <typename T, int R>
__global__ void __launch_bounds__(LK_THREADS, lk_min_blocks<R>())
lk_iter_kernel(const __grid_constant__ IterArgs a, const __grid_constant__ StageMaps m, int r, float fp64_cond)
{
    extern __shared__ __align__(128) float4 smem4[];
    float *smem = reinterpret_cast<float *>(smem4);
    uint32_t phase = 0;
    lk_tile_prepare<R>(smem);
    lk_tile<T, true, R, -1, LK_TH, false>(a, &m, blockIdx.x, r, fp64_cond, smem, phase);   // a.strip is 1
}

// One iteration of up to PHASE_PAIRS pairs on one level: block b runs tile
// b - prefix[p] of pair p. The same tile code as lk_iter_kernel, so the same results.
template <typename T, int R, int MODE, int TH>
__global__ void __launch_bounds__(LK_THREADS, lk_min_blocks<R, TH>())
phase_iter_kernel(const __grid_constant__ IterPhase P, int r, float fp64_cond)
{
    extern __shared__ __align__(128) float4 smem4[];
    float *smem = reinterpret_cast<float *>(smem4);
    if constexpr (R != 0) {
        const int t2 = blockIdx.x + P.ahead;
        if (P.ahead > 0 && t2 < P.prefix[P.npairs]) {
            const int q = phase_pair(P.prefix, P.npairs, t2);
            prefetch_tile<T, MODE, TH>(P.a[q], t2 - P.prefix[q], R);
        }
    }
    const int p = phase_pair(P.prefix, P.npairs, blockIdx.x);
    uint32_t phase = 0;
    lk_tile_prepare<R, TH>(smem);
    lk_tile<T, true, R, MODE, TH>(P.a[p], &P.m[p], blockIdx.x - P.prefix[p], r, fp64_cond, smem, phase);
}

// Two same-level iterations of up to PHASE_PAIRS pairs in one launch (iteration fusion
// depth 2): block b runs both on tile b - prefix[p] of pair p (tile height LK_TH).
template <int R> constexpr int fused2_min_blocks()
{
    if constexpr (R == 0) {
        return 1;
    } else {
        constexpr int b = 233472 / (4 * Fused2<R, LK_TH>::SMEM_FLOATS + 1024);
        return b < 1 ? 1 : (b > 2 ? 2 : b);
    }
}
template <typename T, int R>
__global__ void __launch_bounds__(LK_THREADS, fused2_min_blocks<R>())
phase_iter2_kernel(const __grid_constant__ IterPhase P, float fp64_cond)
{
    extern __shared__ __align__(128) float4 smem4[];
    if constexpr (R != 0) {
        const int p = phase_pair(P.prefix, P.npairs, blockIdx.x);
        lk_tile_fused2<T, true, R, LK_TH>(P.a[p], blockIdx.x - P.prefix[p], fp64_cond,
                                          reinterpret_cast<float *>(smem4));
    }
}

// The window sums of five given planes, through the same passes as the iteration tile.
template <int R>
__global__ void __launch_bounds__(LK_THREADS)
window_sums_kernel(const float *ch, int H, int W, int r, int tiles_x, float *out)
{
    extern __shared__ float4 smem4[];
    float *smem = reinterpret_cast<float *>(smem4);
    const int tile = blockIdx.x;
    const int ty0 = (tile / tiles_x) * LK_TH, tx0 = (tile % tiles_x) * LK_TW;
    const size_t N = (size_t)H * W;
    if constexpr (R == 0) {
        const int RH = LK_TH + 2 * r, RW = LK_TW + 2 * r;
        const int plane = RH * RW;
        float *P = smem, *S = smem + 5 * plane;
        for (int i = threadIdx.x; i < plane; i += blockDim.x) {
            const int ry = i / RW, rx = i - ry * RW;
            const int y = ty0 - r + ry, x = tx0 - r + rx;
            const bool in = y >= 0 && y < H && x >= 0 && x < W;
            for (int c = 0; c < 5; ++c) P[c * plane + i] = in ? ch[c * N + (size_t)y * W + x] : 0.0f;
        }
        __syncthreads();
        box_hsum(P, S, RH, RW, r);
        __syncthreads();
        for (int i = threadIdx.x; i < LK_TH * LK_TW; i += blockDim.x) {
            const int ty = i / LK_TW, tx = i % LK_TW;
            const int y = ty0 + ty, x = tx0 + tx;
            if (y >= H || x >= W) continue;
            float s[5];
            box_vsum(S, RH, r, ty, tx, s);
            for (int c = 0; c < 5; ++c) out[c * N + (size_t)y * W + x] = s[c];
        }
    } else {
        // the planes of the iteration tile: channels (0, 1) and (2, 3) as float2 pairs, 4 alone
        using F = FixedTile<R>;
        float2 *P01 = reinterpret_cast<float2 *>(smem);
        float2 *P23 = P01 + F::PAIR_PLANE;
        float *P4 = reinterpret_cast<float *>(P23 + F::PAIR_PLANE);
        for (int i = threadIdx.x; i < F::RH * F::RWE; i += blockDim.x) {
            const int ry = i / F::RWE, rx = i - ry * F::RWE;
            const int y = ty0 - R + ry, x = tx0 - F::RE + rx;
            const bool in = y >= 0 && y < H && x >= 0 && x < W;
            float c[5];
            for (int k = 0; k < 5; ++k) c[k] = in ? ch[k * N + (size_t)y * W + x] : 0.0f;
            P01[ry * F::RWP2 + rx] = make_float2(c[0], c[1]);
            P23[ry * F::RWP2 + rx] = make_float2(c[2], c[3]);
            P4[ry * F::RWP1 + rx] = c[4];
        }
        __syncthreads();
        box_h_pairs<R, LK_TH>(P01);
        box_h_pairs<R, LK_TH>(P23);
        box_h_single<R, LK_TH>(P4);
        __syncthreads();
        constexpr int VR = v_rows<R, LK_TH>();
        for (int i = threadIdx.x; i < LK_TW * (LK_TH / VR); i += blockDim.x) {
            const int tx = i % LK_TW, g = i / LK_TW;
            const int x = tx0 + tx;
            if (x >= W) continue;
            float2 s01[VR], s23[VR];
            float s4[VR];
            box_v_planes<R, LK_TH>(P01, P23, P4, g, tx, s01, s23, s4);
            for (int j = 0; j < VR; ++j) {
                const int y = ty0 + VR * g + j;
                if (y >= H) break;
                const float s[5] = {s01[j].x, s01[j].y, s23[j].x, s23[j].y, s4[j]};
                for (int c = 0; c < 5; ++c) out[c * N + (size_t)y * W + x] = s[c];
            }
        }
    }
}

template <int R> size_t radius_smem_bytes(int r, bool stage_i2)
{
    const size_t lk = sizeof(float) * (size_t)lk_tile_smem_floats<R>(r, stage_i2);
    size_t pyr = sizeof(float) * (size_t)PYR_SMEM_FLOATS;
    const size_t zn = sizeof(float) * (size_t)ZN_SMEM_FLOATS;
    if (zn > pyr) pyr = zn;
    return lk > pyr ? lk : pyr;
}

template <typename T, int R>
static cudaError_t lk_for(const IterArgs &a, const StageMaps &m, int r, float fp64_cond, cudaStream_t s)
{
    lk_iter_kernel<T, R><<<a.tiles, LK_THREADS,
                           sizeof(float) * lk_tile_smem_floats<R>(r, a.stage_i2 != 0, (int)sizeof(T)), s>>>(
        a, m, r, fp64_cond);
    return cudaGetLastError();
}

template <int R>
cudaError_t lk_launch(const IterArgs &a, const StageMaps &m, int elem, int r, float fp64_cond, cudaStream_t s)
{
    switch (elem) {
    case ET_U8: return lk_for<uint8_t, R>(a, m, r, fp64_cond, s);
    case ET_U16: return lk_for<uint16_t, R>(a, m, r, fp64_cond, s);
    case ET_F32: return lk_for<float, R>(a, m, r, fp64_cond, s);
    case ET_F16: return lk_for<__half, R>(a, m, r, fp64_cond, s);
    default: return lk_for<__nv_bfloat16, R>(a, m, r, fp64_cond, s);
    }
}

template <int R> cudaError_t ws_launch(const float *ch, int H, int W, int r, float *out, cudaStream_t s)
{
    const int tiles_x = (W + LK_TW - 1) / LK_TW, tiles_y = (H + LK_TH - 1) / LK_TH;
    window_sums_kernel<R><<<tiles_x * tiles_y, LK_THREADS, sizeof(float) * lk_tile_smem_floats<R>(r, false), s>>>(
        ch, H, W, r, tiles_x, out);
    return cudaGetLastError();
}

// The flow mode is the same for every pair of a phase: one kernel per mode (and per
// tile height; the run-time-radius kernel has only the default height).
template <typename T, int R, int TH>
static cudaError_t phase_for_th(const IterPhase &P, int r, float fp64_cond, cudaStream_t s)
{
    bool stage = false;   // shared memory for the staged window if any pair stages
    for (int i = 0; i < P.npairs; ++i) stage = stage || P.a[i].stage_i2 != 0;
    const size_t smem = sizeof(float) * lk_tile_smem_floats<R, TH>(r, stage, (int)sizeof(T));
    const int blocks = P.prefix[P.npairs];
    switch (P.a[0].mode) {
    case FLOW_ZERO: phase_iter_kernel<T, R, FLOW_ZERO, TH><<<blocks, LK_THREADS, smem, s>>>(P, r, fp64_cond); break;
    case FLOW_SAME: phase_iter_kernel<T, R, FLOW_SAME, TH><<<blocks, LK_THREADS, smem, s>>>(P, r, fp64_cond); break;
    default: phase_iter_kernel<T, R, FLOW_UPSAMPLE, TH><<<blocks, LK_THREADS, smem, s>>>(P, r, fp64_cond); break;
    }
    return cudaGetLastError();
}

template <typename T, int R>
static cudaError_t phase_for(const IterPhase &P, int r, float fp64_cond, int tile_h, cudaStream_t s)
{
    if constexpr (R != 0) {
        if (tile_h == ALT_TH) return phase_for_th<T, R, ALT_TH>(P, r, fp64_cond, s);
    }
    return phase_for_th<T, R, LK_TH>(P, r, fp64_cond, s);
}

template <int R>
cudaError_t phase_launch(const IterPhase &P, int elem, int r, float fp64_cond, int tile_h, cudaStream_t s)
{
    if (P.prefix[P.npairs] == 0) return cudaSuccess;
    switch (elem) {
    case ET_U8: return phase_for<uint8_t, R>(P, r, fp64_cond, tile_h, s);
    case ET_U16: return phase_for<uint16_t, R>(P, r, fp64_cond, tile_h, s);
    case ET_F32: return phase_for<float, R>(P, r, fp64_cond, tile_h, s);
    case ET_F16: return phase_for<__half, R>(P, r, fp64_cond, tile_h, s);
    default: return phase_for<__nv_bfloat16, R>(P, r, fp64_cond, tile_h, s);
    }
}

template <int R> size_t fused2_smem_bytes()
{
    if constexpr (R == 0) return 0;
    else return sizeof(float) * (size_t)Fused2<R, LK_TH>::SMEM_FLOATS;
}

template <typename T, int R> static cudaError_t phase2_for(const IterPhase &P, float fp64_cond, cudaStream_t s)
{
    phase_iter2_kernel<T, R><<<P.prefix[P.npairs], LK_THREADS, fused2_smem_bytes<R>(), s>>>(P, fp64_cond);
    return cudaGetLastError();
}

template <int R> cudaError_t phase2_launch(const IterPhase &P, int elem, float fp64_cond, cudaStream_t s)
{
    if constexpr (R == 0) {
        return cudaErrorInvalidValue;   // fusion needs a fixed-radius kernel
    } else {
        if (P.prefix[P.npairs] == 0) return cudaSuccess;
        switch (elem) {
        case ET_U8: return phase2_for<uint8_t, R>(P, fp64_cond, s);
        case ET_U16: return phase2_for<uint16_t, R>(P, fp64_cond, s);
        case ET_F32: return phase2_for<float, R>(P, fp64_cond, s);
        case ET_F16: return phase2_for<__half, R>(P, fp64_cond, s);
        default: return phase2_for<__nv_bfloat16, R>(P, fp64_cond, s);
        }
    }
}

template <typename T, int R> static cudaError_t i1h_for(const HessArgs &a, int r, cudaStream_t s)
{
    i1_hess_kernel<T, R><<<a.tiles, LK_THREADS, sizeof(float) * i1_smem_floats<R>(r, 3), s>>>(a, r);
    return cudaGetLastError();
}

template <int R> cudaError_t i1h_launch(const HessArgs &a, int elem, int r, cudaStream_t s)
{
    switch (elem) {
    case ET_U8: return i1h_for<uint8_t, R>(a, r, s);
    case ET_U16: return i1h_for<uint16_t, R>(a, r, s);
    case ET_F32: return i1h_for<float, R>(a, r, s);
    case ET_F16: return i1h_for<__half, R>(a, r, s);
    default: return i1h_for<__nv_bfloat16, R>(a, r, s);
    }
}

template <typename T, int R> static cudaError_t i1_for(const IterArgs &a, int r, float fp64_cond, cudaStream_t s)
{
    i1_iter_kernel<T, R><<<a.tiles, LK_THREADS, sizeof(float) * i1_smem_floats<R>(r, 2), s>>>(a, r, fp64_cond);
    return cudaGetLastError();
}

template <int R> cudaError_t i1_launch(const IterArgs &a, int elem, int r, float fp64_cond, cudaStream_t s)
{
    switch (elem) {
    case ET_U8: return i1_for<uint8_t, R>(a, r, fp64_cond, s);
    case ET_U16: return i1_for<uint16_t, R>(a, r, fp64_cond, s);
    case ET_F32: return i1_for<float, R>(a, r, fp64_cond, s);
    case ET_F16: return i1_for<__half, R>(a, r, fp64_cond, s);
    default: return i1_for<__nv_bfloat16, R>(a, r, fp64_cond, s);
    }
}

template <typename T, int R> static cudaError_t phase_hess_for(const HessPhase &P, int r, cudaStream_t s)
{
    phase_hess_kernel<T, R><<<P.prefix[P.npairs], LK_THREADS, sizeof(float) * i1_smem_floats<R>(r, 3), s>>>(P, r);
    return cudaGetLastError();
}

template <int R> cudaError_t phase_hess_launch(const HessPhase &P, int elem, int r, cudaStream_t s)
{
    if (P.prefix[P.npairs] == 0) return cudaSuccess;
    switch (elem) {
    case ET_U8: return phase_hess_for<uint8_t, R>(P, r, s);
    case ET_U16: return phase_hess_for<uint16_t, R>(P, r, s);
    case ET_F32: return phase_hess_for<float, R>(P, r, s);
    case ET_F16: return phase_hess_for<__half, R>(P, r, s);
    default: return phase_hess_for<__nv_bfloat16, R>(P, r, s);
    }
}

template <typename T, int R>
static cudaError_t phase_i1_for(const IterPhase &P, int r, float fp64_cond, cudaStream_t s)
{
    phase_i1_iter_kernel<T, R><<<P.prefix[P.npairs], LK_THREADS, sizeof(float) * i1_smem_floats<R>(r, 2), s>>>(
        P, r, fp64_cond);
    return cudaGetLastError();
}

template <int R> cudaError_t phase_i1_launch(const IterPhase &P, int elem, int r, float fp64_cond, cudaStream_t s)
{
    if (P.prefix[P.npairs] == 0) return cudaSuccess;
    switch (elem) {
    case ET_U8: return phase_i1_for<uint8_t, R>(P, r, fp64_cond, s);
    case ET_U16: return phase_i1_for<uint16_t, R>(P, r, fp64_cond, s);
    case ET_F32: return phase_i1_for<float, R>(P, r, fp64_cond, s);
    case ET_F16: return phase_i1_for<__half, R>(P, r, fp64_cond, s);
    default: return phase_i1_for<__nv_bfloat16, R>(P, r, fp64_cond, s);
    }
}

// The tensor maps of the staged fixed-radius tile of height TH: the estimate in boxes
// of the tile's region (RWP2 x RH elements of 8 bytes) and I2 in boxes of the window.
template <int R, int TH> static bool stage_maps_th(const IterArgs &a, StageMaps &m, int elem)
{
    using F = FixedTile<R, TH>;
    const int S = elem_bytes(elem);
    if (a.mode == FLOW_SAME &&
        !encode_tile_map(&m.flow, ET_FLOW2, a.fin, a.W, a.H, (size_t)a.fin_pitch * 8, F::RWP2, F::FLOW_BH))
        return false;
    return encode_tile_map(&m.i2, elem, a.I2, a.W, a.H, (size_t)a.pitch * S, F::win_w(S), F::WIN_H);
}

template <int R> bool radius_stage_maps(const IterArgs &a, StageMaps &m, int elem, int tile_h)
{
    if constexpr (R == 0) {
        return false;
    } else {
        return tile_h == ALT_TH ? stage_maps_th<R, ALT_TH>(a, m, elem) : stage_maps_th<R, LK_TH>(a, m, elem);
    }
}

template <int R> void *batch_kernel_ptr(int in_format, int storage)
{
    if (in_format == OF_U8) {
        if (storage == OF_F32) return (void *)batch_kernel<uint8_t, float, R>;
        if (storage == OF_F16) return (void *)batch_kernel<uint8_t, __half, R>;
        return (void *)batch_kernel<uint8_t, __nv_bfloat16, R>;
    }
    if (storage == OF_F32) return (void *)batch_kernel<uint16_t, float, R>;
    if (storage == OF_F16) return (void *)batch_kernel<uint16_t, __half, R>;
    return (void *)batch_kernel<uint16_t, __nv_bfloat16, R>;
}

// Raise the dynamic shared memory limit of this radius's kernels on the current device.
template <int R> cudaError_t radius_configure()
{
    const int bytes = (int)radius_smem_bytes<R>(R == 0 ? MAX_RADIUS : R, true);
    cudaError_t e;
#define OF_SET(fn) if ((e = cudaFuncSetAttribute((const void *)(fn), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) != cudaSuccess) return e
    OF_SET((lk_iter_kernel<uint8_t, R>));
    OF_SET((lk_iter_kernel<uint16_t, R>));
    OF_SET((lk_iter_kernel<float, R>));
    OF_SET((lk_iter_kernel<__half, R>));
    OF_SET((lk_iter_kernel<__nv_bfloat16, R>));
#define OF_SET_PH(T) OF_SET((phase_iter_kernel<T, R, FLOW_ZERO, LK_TH>)); OF_SET((phase_iter_kernel<T, R, FLOW_SAME, LK_TH>)); \
    OF_SET((phase_iter_kernel<T, R, FLOW_UPSAMPLE, LK_TH>))
    OF_SET_PH(uint8_t);
    OF_SET_PH(uint16_t);
    OF_SET_PH(float);
    OF_SET_PH(__half);
    OF_SET_PH(__nv_bfloat16);
#undef OF_SET_PH
    if constexpr (R != 0) {   // the other tile height of the phase kernels
        const int alt = (int)sizeof(float) * lk_tile_smem_floats<R, ALT_TH>(R, true);
#define OF_SET_ALT(T)                                                                                       \
    for (const void *fn : {(const void *)phase_iter_kernel<T, R, FLOW_ZERO, ALT_TH>,                        \
                           (const void *)phase_iter_kernel<T, R, FLOW_SAME, ALT_TH>,                        \
                           (const void *)phase_iter_kernel<T, R, FLOW_UPSAMPLE, ALT_TH>})                   \
        if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, alt)) != cudaSuccess) \
            return e;
        OF_SET_ALT(uint8_t)
        OF_SET_ALT(uint16_t)
        OF_SET_ALT(float)
        OF_SET_ALT(__half)
        OF_SET_ALT(__nv_bfloat16)
#undef OF_SET_ALT
    }
    OF_SET((window_sums_kernel<R>));
    if constexpr (R != 0) {   // the fused two-iteration kernels
        const int fb = (int)fused2_smem_bytes<R>();
        for (const void *fn : {(const void *)phase_iter2_kernel<uint8_t, R>, (const void *)phase_iter2_kernel<uint16_t, R>,
                               (const void *)phase_iter2_kernel<float, R>, (const void *)phase_iter2_kernel<__half, R>,
                               (const void *)phase_iter2_kernel<__nv_bfloat16, R>})
            if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, fb)) != cudaSuccess) return e;
    }
    {
        const int r = R == 0 ? MAX_RADIUS : R;
        const int hb = (int)sizeof(float) * i1_smem_floats<R>(r, 3), ib = (int)sizeof(float) * i1_smem_floats<R>(r, 2);
#define OF_SET_I1(T)                                                                                       \
    if ((e = cudaFuncSetAttribute((const void *)i1_hess_kernel<T, R>,                                     \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, hb)) != cudaSuccess ||     \
        (e = cudaFuncSetAttribute((const void *)i1_iter_kernel<T, R>,                                     \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, ib)) != cudaSuccess ||     \
        (e = cudaFuncSetAttribute((const void *)phase_hess_kernel<T, R>,                                  \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, hb)) != cudaSuccess ||     \
        (e = cudaFuncSetAttribute((const void *)phase_i1_iter_kernel<T, R>,                               \
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, ib)) != cudaSuccess)       \
        return e;
        OF_SET_I1(uint8_t)
        OF_SET_I1(uint16_t)
        OF_SET_I1(float)
        OF_SET_I1(__half)
        OF_SET_I1(__nv_bfloat16)
#undef OF_SET_I1
    }
    for (int f = 0; f < 2; ++f)
        for (int st = 0; st < 3; ++st) OF_SET(batch_kernel_ptr<R>(f, st));
#undef OF_SET
    return cudaSuccess;
}

template cudaError_t lk_launch<OF_RADIUS>(const IterArgs &, const StageMaps &, int, int, float, cudaStream_t);
template cudaError_t ws_launch<OF_RADIUS>(const float *, int, int, int, float *, cudaStream_t);
template cudaError_t i1h_launch<OF_RADIUS>(const HessArgs &, int, int, cudaStream_t);
template cudaError_t phase_launch<OF_RADIUS>(const IterPhase &, int, int, float, int, cudaStream_t);
template cudaError_t phase_hess_launch<OF_RADIUS>(const HessPhase &, int, int, cudaStream_t);
template cudaError_t phase_i1_launch<OF_RADIUS>(const IterPhase &, int, int, float, cudaStream_t);
template cudaError_t i1_launch<OF_RADIUS>(const IterArgs &, int, int, float, cudaStream_t);
template void *batch_kernel_ptr<OF_RADIUS>(int, int);
template bool radius_stage_maps<OF_RADIUS>(const IterArgs &, StageMaps &, int, int);
template cudaError_t phase2_launch<OF_RADIUS>(const IterPhase &, int, float, cudaStream_t);
template cudaError_t radius_configure<OF_RADIUS>();
template size_t radius_smem_bytes<OF_RADIUS>(int, bool);

}  // namespace of
