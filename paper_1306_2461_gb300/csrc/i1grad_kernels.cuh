// The variant of the iteration linearised with the FIRST image's gradient (the FOLKI
// lineage the method of Sect. 2.4 comes from): g1 = central difference of I1 at integer
// pixels, indices clamped, halved. The window matrix [Sa Sb; Sb Sc] = sum over the
// window of g1 g1^T then depends on I1 only: i1_hess_kernel sums it once per level, and
// each iteration forms and sums only the two right-hand-side channels
//     g1 e~,  e~ = I1 - I2(x + u_k) + g1 . (u_k - u_ref),
// then solves [Sa Sb; Sb Sc] (u_{k+1} - u_ref) = sum g1 e~ with the guard of solve2.
#pragma once

#include "of_internal.cuh"
#include "of_kernels.cuh"

namespace of {

// I1 at (x, y) and its central-difference gradient (neighbour indices clamped).
template <bool NC, typename T>
__device__ __forceinline__ void i1_grad(const T *I1, int pitch, int H, int W, int x, int y, float &c, float &gx,
                                        float &gy)
{
    const T *row = I1 + y * pitch;
    c = ldf<NC>(row + x);
    const float xm = ldf<NC>(row + max(x - 1, 0)), xp = ldf<NC>(row + min(x + 1, W - 1));
    const float ym = ldf<NC>(I1 + max(y - 1, 0) * pitch + x), yp = ldf<NC>(I1 + min(y + 1, H - 1) * pitch + x);
    gx = (xp - xm) * 0.5f;
    gy = (yp - ym) * 0.5f;
}

template <int R> inline __host__ __device__ int i1_smem_floats(int r, int channels)
{
    if constexpr (R == 0) {
        const int RH = I1_TH + 2 * r, RW = LK_TW + 2 * r;
        return channels * (RH * RW + RH * LK_TW);
    } else {
        return channels * FixedTile<R, I1_TH>::PLANE;
    }
}

// Plane stride and row length of the product planes (padded rows for a fixed radius).
template <int R> __device__ __forceinline__ int i1_plane(int RH, int RW)
{
    if constexpr (R == 0) return RH * RW;
    else return FixedTile<R, I1_TH>::PLANE;
}
template <int R> __device__ __forceinline__ int i1_rowlen(int RW)
{
    if constexpr (R == 0) return RW;
    else return FixedTile<R, I1_TH>::RWP;
}

// Window matrix of one level: (Sa, Sb, Sc, 0) at every pixel of one output tile.
template <typename T, int R>
__device__ __forceinline__ void i1_hess_tile(const HessArgs &a, int tile, int r, float *smem)
{
    const int tyi = tile / a.tiles_x;
    const int ty0 = tyi * I1_TH, tx0 = (tile - tyi * a.tiles_x) * LK_TW;
    const T *I1 = static_cast<const T *>(a.I1);
    const int rr = R == 0 ? r : R;
    const int RH = I1_TH + 2 * rr, RW = LK_TW + 2 * rr;
    const int plane = i1_plane<R>(RH, RW);
    const int rowlen = i1_rowlen<R>(RW);
    for (int i = threadIdx.x; i < RH * RW; i += LK_THREADS) {
        const int ry = i / RW, rx = i - ry * RW;
        const int y = ty0 - rr + ry, x = tx0 - rr + rx;
        float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f;
        if ((unsigned)y < (unsigned)a.H && (unsigned)x < (unsigned)a.W) {
            float c, gx, gy;
            i1_grad<true>(I1, a.pitch, a.H, a.W, x, y, c, gx, gy);
            p0 = gx * gx;
            p1 = gx * gy;
            p2 = gy * gy;
        }
        float *q = smem + ry * rowlen + rx;
        q[0] = p0;
        q[plane] = p1;
        q[2 * plane] = p2;
    }
    __syncthreads();
    if constexpr (R == 0) {
        float *S = smem + 3 * plane;
        box_hsum<3>(smem, S, RH, RW, r);
        __syncthreads();
        for (int i = threadIdx.x; i < I1_TH * LK_TW; i += LK_THREADS) {
            const int ty = i / LK_TW, tx = i - ty * LK_TW;
            const int y = ty0 + ty, x = tx0 + tx;
            if (y >= a.H || x >= a.W) continue;
            float s[3];
            box_vsum<3>(S, RH, r, ty, tx, s);
            a.hess[(size_t)y * a.hess_pitch + x] = make_float4(s[0], s[1], s[2], 0.0f);
        }
    } else {
        box_h_inplace<R, 3, I1_TH>(smem);
        for (int i = threadIdx.x; i < LK_TW * (I1_TH / 4); i += LK_THREADS) {
            const int tx = i % LK_TW, g = i / LK_TW;
            const int x = tx0 + tx;
            if (x >= a.W || ty0 + 4 * g >= a.H) continue;
            float s[3][4];
            box_v4<R, 3, I1_TH>(smem, g, tx, s);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int y = ty0 + 4 * g + j;
                if (y >= a.H) break;
                a.hess[(size_t)y * a.hess_pitch + x] = make_float4(s[0][j], s[1][j], s[2][j], 0.0f);
            }
        }
    }
}

// One iteration of the variant on one output tile.
template <typename T, int R>
__device__ __forceinline__ void i1_iter_tile(const IterArgs &a, int tile, int r, float fp64_cond, float *smem)
{
    const int tyi = tile / a.tiles_x;
    const int ty0 = tyi * I1_TH, tx0 = (tile - tyi * a.tiles_x) * LK_TW;
    const T *I1 = static_cast<const T *>(a.I1);
    const T *I2 = static_cast<const T *>(a.I2);
    const float2 ref = flow_at<true>(a, min(tx0 + LK_TW / 2, a.W - 1), min(ty0 + I1_TH / 2, a.H - 1));
    const int rr = R == 0 ? r : R;
    const int RH = I1_TH + 2 * rr, RW = LK_TW + 2 * rr;
    const int plane = i1_plane<R>(RH, RW);
    const int rowlen = i1_rowlen<R>(RW);
    const int nreg = RH * RW;
    // the current estimates of S1 region pixels are loaded before any is used
    constexpr int S1 = 4;
#pragma unroll 1
    for (int i0 = threadIdx.x; i0 < nreg; i0 += S1 * LK_THREADS) {
        float2 f[S1];
        bool in[S1];
#pragma unroll
        for (int k = 0; k < S1; ++k) {
            const int i = i0 + k * LK_THREADS;
            const int ry = i / RW, rx = i - ry * RW;
            const int y = ty0 - rr + ry, x = tx0 - rr + rx;
            in[k] = i < nreg && (unsigned)y < (unsigned)a.H && (unsigned)x < (unsigned)a.W;
            f[k] = in[k] ? flow_at<true>(a, x, y) : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int k = 0; k < S1; ++k) {
            const int i = i0 + k * LK_THREADS;
            if (i >= nreg) break;
            const int ry = i / RW, rx = i - ry * RW;
            const int y = ty0 - rr + ry, x = tx0 - rr + rx;
            float p0 = 0.0f, p1 = 0.0f;
            if (in[k]) {
                float c, gx, gy;
                i1_grad<true>(I1, a.pitch, a.H, a.W, x, y, c, gx, gy);
                const float Iw = bil_at<true>(I2, a.pitch, a.H, a.W, x, y, f[k].x, f[k].y);
                const float e = resid(c, Iw, gx, gy, f[k].x - ref.x, f[k].y - ref.y);
                p0 = gx * e;
                p1 = gy * e;
            }
            float *q = smem + ry * rowlen + rx;
            q[0] = p0;
            q[plane] = p1;
        }
    }
    __syncthreads();
    auto finish = [&](int x, int y, float d, float e) {
        const float4 h = __ldg(a.hess + (size_t)y * a.hess_pitch + x);
        const float s[5] = {h.x, h.y, h.z, d, e};
        float xu, xv;
        const float2 f = solve2(s, fp64_cond, xu, xv) ? make_float2(ref.x + xu, ref.y + xv) : flow_at<true>(a, x, y);
        if (a.fout) {
            a.fout[(size_t)y * a.fout_pitch + x] = f;
        } else {
            a.u_out[(size_t)y * a.W + x] = f.x;
            a.v_out[(size_t)y * a.W + x] = f.y;
        }
    };
    if constexpr (R == 0) {
        float *S = smem + 2 * plane;
        box_hsum<2>(smem, S, RH, RW, r);
        __syncthreads();
        for (int i = threadIdx.x; i < I1_TH * LK_TW; i += LK_THREADS) {
            const int ty = i / LK_TW, tx = i - ty * LK_TW;
            const int y = ty0 + ty, x = tx0 + tx;
            if (y >= a.H || x >= a.W) continue;
            float s[2];
            box_vsum<2>(S, RH, r, ty, tx, s);
            finish(x, y, s[0], s[1]);
        }
    } else {
        box_h_inplace<R, 2, I1_TH>(smem);
#pragma unroll 1
        for (int i = threadIdx.x; i < LK_TW * (I1_TH / 4); i += LK_THREADS) {
            const int tx = i % LK_TW, g = i / LK_TW;
            const int x = tx0 + tx;
            if (x >= a.W || ty0 + 4 * g >= a.H) continue;
            float s[2][4];
            box_v4<R, 2, I1_TH>(smem, g, tx, s);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int y = ty0 + 4 * g + j;
                if (y >= a.H) break;
                finish(x, y, s[0][j], s[1][j]);
            }
        }
    }
}

template <typename T, int R>
__global__ void __launch_bounds__(LK_THREADS) i1_hess_kernel(HessArgs a, int r)
{
    extern __shared__ float4 smem4[];
    i1_hess_tile<T, R>(a, blockIdx.x, r, reinterpret_cast<float *>(smem4));
}

#ifndef OF_I1_MIN_BLOCKS
#define OF_I1_MIN_BLOCKS 6
#endif
template <typename T, int R>
__global__ void __launch_bounds__(LK_THREADS, OF_I1_MIN_BLOCKS) i1_iter_kernel(IterArgs a, int r, float fp64_cond)
{
    extern __shared__ float4 smem4[];
    i1_iter_tile<T, R>(a, blockIdx.x, r, fp64_cond, reinterpret_cast<float *>(smem4));
}

// The same over the tiles of up to PHASE_PAIRS pairs (batched form).
template <typename T, int R>
__global__ void __launch_bounds__(LK_THREADS) phase_hess_kernel(const __grid_constant__ HessPhase P, int r)
{
    extern __shared__ float4 smem4[];
    const int p = phase_pair(P.prefix, P.npairs, blockIdx.x);
    i1_hess_tile<T, R>(P.a[p], blockIdx.x - P.prefix[p], r, reinterpret_cast<float *>(smem4));
}

template <typename T, int R>
__global__ void __launch_bounds__(LK_THREADS, OF_I1_MIN_BLOCKS)
phase_i1_iter_kernel(const __grid_constant__ IterPhase P, int r, float fp64_cond)
{
    extern __shared__ float4 smem4[];
    if constexpr (R != 0) {
        const int t2 = blockIdx.x + P.ahead;
        if (P.ahead > 0 && t2 < P.prefix[P.npairs]) {
            const int q = phase_pair(P.prefix, P.npairs, t2);
            prefetch_tile<T, -1, I1_TH>(P.a[q], t2 - P.prefix[q], R);
        }
    }
    const int p = phase_pair(P.prefix, P.npairs, blockIdx.x);
    i1_iter_tile<T, R>(P.a[p], blockIdx.x - P.prefix[p], r, fp64_cond, reinterpret_cast<float *>(smem4));
}

}  // namespace of
