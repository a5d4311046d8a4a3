// Device tile functions shared by the per-level kernels and the persistent batched
// kernel: one pyramid-reduction tile and one Gauss-Newton iteration tile.
#pragma once

#include "of_internal.cuh"

namespace of {

// Loads. NC = true reads through the non-coherent read-only path (__ldg): only for
// data no thread writes during the kernel. The persistent batched kernel reads levels
// and flows that other blocks wrote earlier in the same launch, so it uses NC = false.
template <bool NC, typename T> __device__ __forceinline__ T ld(const T *p)
{
    if constexpr (NC) return __ldg(p);
    else return *p;
}
template <bool NC> __device__ __forceinline__ float ldf(const uint8_t *p) { return (float)ld<NC>(p); }
template <bool NC> __device__ __forceinline__ float ldf(const uint16_t *p) { return (float)ld<NC>(p); }
template <bool NC> __device__ __forceinline__ float ldf(const float *p) { return ld<NC>(p); }
template <bool NC> __device__ __forceinline__ float ldf(const __half *p)
{
    if constexpr (NC) return __half2float(__ldg(p));
    else return __half2float(*p);
}
template <bool NC> __device__ __forceinline__ float ldf(const __nv_bfloat16 *p)
{
    if constexpr (NC) return __bfloat162float(__ldg(p));
    else return __bfloat162float(*p);
}

__device__ __forceinline__ int clampi(int a, int lo, int hi) { return a < lo ? lo : (a > hi ? hi : a); }

// ------------------------------------------------------------------ pyramid tile
// Shared memory: PYR_SMEM_FLOATS floats.
constexpr int PYR_RH = 2 * PYR_TH + 3;
constexpr int PYR_RW = 2 * PYR_TW + 3;
constexpr int PYR_SMEM_FLOATS = PYR_RH * PYR_RW + PYR_RH * PYR_TW;

// One output tile (PYR_TH x PYR_TW at level l+1) of image `img` (0/1) of a pair.
// FIRST: the source is the raw camera image; level 0 is stored as well, unchanged in
// the camera's integer format.
template <typename Tin, typename Tout, bool FIRST, bool NC>
__device__ __forceinline__ void pyr_tile_smem(const PyrArgs &a, int tile, int img, float *smem)
{
    float *s_in = smem;                      // PYR_RH x PYR_RW
    float *s_h = smem + PYR_RH * PYR_RW;     // PYR_RH x PYR_TW
    const int ty0 = (tile / a.tiles_x) * PYR_TH;
    const int tx0 = (tile - (tile / a.tiles_x) * a.tiles_x) * PYR_TW;
    const int ys = 2 * ty0 - 2, xs = 2 * tx0 - 2;
    const Tin *src = static_cast<const Tin *>(img ? a.src[1] : a.src[0]);
    __syncthreads();   // the previous tile's readers of smem are done
    for (int i = threadIdx.x; i < PYR_RH * PYR_RW; i += blockDim.x) {
        const int r = i / PYR_RW, c = i - r * PYR_RW;
        const int y = clampi(ys + r, 0, a.H - 1), x = clampi(xs + c, 0, a.W - 1);
        s_in[i] = ldf<NC>(src + (size_t)y * a.src_pitch + x);
    }
    __syncthreads();
    if (FIRST) {
        Tin *d0 = static_cast<Tin *>(img ? a.dst0[1] : a.dst0[0]);
        for (int i = threadIdx.x; i < 4 * PYR_TH * PYR_TW; i += blockDim.x) {
            const int r = i / (2 * PYR_TW), c = i - r * (2 * PYR_TW);
            const int y = 2 * ty0 + r, x = 2 * tx0 + c;
            if (y < a.H && x < a.W)
                d0[(size_t)y * a.dst0_pitch + x] = to_elem<Tin>(s_in[(r + 2) * PYR_RW + c + 2]);
        }
    }
    Tout *d = static_cast<Tout *>(img ? a.dst[1] : a.dst[0]);
    if (d == nullptr) return;   // one-level plan: level 0 only (uniform per block)
    for (int i = threadIdx.x; i < PYR_RH * PYR_TW; i += blockDim.x) {
        const int r = i / PYR_TW, j = i - r * PYR_TW;
        const float *q = s_in + r * PYR_RW + 2 * j;
        s_h[i] = q[0] + 4.0f * q[1] + 6.0f * q[2] + 4.0f * q[3] + q[4];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < PYR_TH * PYR_TW; i += blockDim.x) {
        const int r = i / PYR_TW, j = i - r * PYR_TW;
        const int y = ty0 + r, x = tx0 + j;
        if (y < a.Ho && x < a.Wo) {
            const float *q = s_h + 2 * r * PYR_TW + j;
            const float s = q[0] + 4.0f * q[PYR_TW] + 6.0f * q[2 * PYR_TW] + 4.0f * q[3 * PYR_TW] + q[4 * PYR_TW];
            d[(size_t)y * a.dst_pitch + x] = to_elem<Tout>(s * (1.0f / 256.0f));
        }
    }
}

template <typename Tin, typename Tout, bool FIRST>
__device__ __forceinline__ void pyr_tile(const PyrArgs &a, int tile, int img)
{
    __shared__ float smem[PYR_SMEM_FLOATS];
    pyr_tile_smem<Tin, Tout, FIRST, true>(a, tile, img, smem);
}

// ------------------------------------------------------------ iteration helpers
__device__ __forceinline__ float lerpf(float p, float q, float t) { return (1.0f - t) * p + t * q; }

// Bilinear sample with the position clamped to [0, W-1] x [0, H-1].
template <bool NC, typename T>
__device__ __forceinline__ float bil(const T *I, int pitch, int H, int W, float x, float y)
{
    x = fminf(fmaxf(x, 0.0f), (float)(W - 1));
    y = fminf(fmaxf(y, 0.0f), (float)(H - 1));
    const float fx = floorf(x), fy = floorf(y);
    const int x0 = (int)fx, y0 = (int)fy;
    const int x1 = min(x0 + 1, W - 1), y1 = min(y0 + 1, H - 1);
    const float ax = x - fx, ay = y - fy;
    const T *r0 = I + (size_t)y0 * pitch, *r1 = I + (size_t)y1 * pitch;
    return lerpf(lerpf(ldf<NC>(r0 + x0), ldf<NC>(r0 + x1), ax), lerpf(ldf<NC>(r1 + x0), ldf<NC>(r1 + x1), ax), ay);
}

// I2 at p = (px, py) and its gradient at p: central difference of the bilinear samples
// at p +- (1, 0) and p +- (0, 1). Away from the border the 12 distinct taps of the 4x4
// neighbourhood are read once; near it each sample is clamped on its own.
template <bool NC, typename T>
__device__ __forceinline__ void sample_grad(const T *I, int pitch, int H, int W, float px, float py,
                                            float &Iw, float &gx, float &gy)
{
    if (px >= 1.0f && py >= 1.0f && px < (float)(W - 2) && py < (float)(H - 2)) {
        const float fx = floorf(px), fy = floorf(py);
        const int x0 = (int)fx, y0 = (int)fy;
        const float ax = px - fx, ay = py - fy;
        const T *rm = I + (size_t)(y0 - 1) * pitch + x0;
        const T *r0 = rm + pitch, *r1 = r0 + pitch, *r2 = r1 + pitch;
        const float a0 = ldf<NC>(rm), a1 = ldf<NC>(rm + 1);
        const float bm = ldf<NC>(r0 - 1), b0 = ldf<NC>(r0), b1 = ldf<NC>(r0 + 1), b2 = ldf<NC>(r0 + 2);
        const float cm = ldf<NC>(r1 - 1), c0 = ldf<NC>(r1), c1 = ldf<NC>(r1 + 1), c2 = ldf<NC>(r1 + 2);
        const float d0 = ldf<NC>(r2), d1 = ldf<NC>(r2 + 1);
        const float top = lerpf(b0, b1, ax), bot = lerpf(c0, c1, ax);
        Iw = lerpf(top, bot, ay);
        gx = (lerpf(lerpf(b1, b2, ax), lerpf(c1, c2, ax), ay) - lerpf(lerpf(bm, b0, ax), lerpf(cm, c0, ax), ay)) * 0.5f;
        gy = (lerpf(bot, lerpf(d0, d1, ax), ay) - lerpf(lerpf(a0, a1, ax), top, ay)) * 0.5f;
    } else {
        Iw = bil<NC>(I, pitch, H, W, px, py);
        gx = (bil<NC>(I, pitch, H, W, px + 1.0f, py) - bil<NC>(I, pitch, H, W, px - 1.0f, py)) * 0.5f;
        gy = (bil<NC>(I, pitch, H, W, px, py + 1.0f) - bil<NC>(I, pitch, H, W, px, py - 1.0f)) * 0.5f;
    }
}

// Current estimate at (x, y) of the level being iterated.
template <bool NC>
__device__ __forceinline__ float2 flow_at(const IterArgs &a, int x, int y)
{
    if (a.mode == FLOW_ZERO) return make_float2(0.0f, 0.0f);
    if (a.mode == FLOW_SAME) return ld<NC>(a.fin + (size_t)y * a.fin_pitch + x);
    // 2 * bilinear(coarse; x/2, y/2): weights are 0 or 1/2, indices clamped
    const int x0 = x >> 1, y0 = y >> 1;
    const int x1 = min(x0 + 1, a.Wc - 1), y1 = min(y0 + 1, a.Hc - 1);
    const float ax = (x & 1) ? 0.5f : 0.0f, ay = (y & 1) ? 0.5f : 0.0f;
    const float2 f00 = ld<NC>(a.fin + (size_t)y0 * a.fin_pitch + x0);
    const float2 f01 = ld<NC>(a.fin + (size_t)y0 * a.fin_pitch + x1);
    const float2 f10 = ld<NC>(a.fin + (size_t)y1 * a.fin_pitch + x0);
    const float2 f11 = ld<NC>(a.fin + (size_t)y1 * a.fin_pitch + x1);
    return make_float2(2.0f * lerpf(lerpf(f00.x, f01.x, ax), lerpf(f10.x, f11.x, ax), ay),
                       2.0f * lerpf(lerpf(f00.y, f01.y, ax), lerpf(f10.y, f11.y, ax), ay));
}

// Horizontal pass of the box sums: S[c][ry][tx] = sum_{k=0..2r} P[c][ry][tx+k], left to right.
__device__ __forceinline__ void box_hsum(const float *P, float *S, int RH, int RW, int r)
{
    const int n = RH * LK_TW;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int ry = i / LK_TW, tx = i - ry * LK_TW;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            const float *q = P + (size_t)c * RH * RW + ry * RW + tx;
            float s = 0.0f;
            for (int k = 0; k <= 2 * r; ++k) s += q[k];
            S[c * n + i] = s;
        }
    }
}

// Vertical pass at output (ty, tx): sums of S over rows ty..ty+2r, top to bottom.
__device__ __forceinline__ void box_vsum(const float *S, int RH, int r, int ty, int tx, float s[5])
{
    const int n = RH * LK_TW;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        const float *q = S + c * n + ty * LK_TW + tx;
        float acc = 0.0f;
        for (int k = 0; k <= 2 * r; ++k) acc += q[k * LK_TW];
        s[c] = acc;
    }
}

// Solve [a b; b c] x = [d; e]. Returns false (keep the estimate) when tr <= 0 or
// det <= 1e-6 tr^2. Pixels with tr^2/det above fp64_cond (or det <= 0) are solved in
// FP64 from the FP32 sums; fp64_cond == 0 keeps everything in FP32.
__device__ __forceinline__ bool solve2(const float s[5], float fp64_cond, float &xu, float &xv)
{
    const float a = s[0], b = s[1], c = s[2], d = s[3], e = s[4];
    const float tr = a + c;
    if (!(tr > 0.0f)) return false;
    const float det = fmaf(a, c, -(b * b));
    if (fp64_cond > 0.0f && !(det * fp64_cond > tr * tr)) {
        const double A = a, B = b, C = c, D = d, E = e;
        const double T = A + C, dt = A * C - B * B;
        if (!(dt > 1e-6 * T * T)) return false;
        xu = (float)((C * D - B * E) / dt);
        xv = (float)((A * E - B * D) / dt);
        return true;
    }
    if (!(det > 1e-6f * tr * tr)) return false;
    const float inv = 1.0f / det;
    xu = (c * d - b * e) * inv;
    xv = (a * e - b * d) * inv;
    return true;
}

inline __host__ __device__ int lk_smem_floats(int r)
{
    const int RH = LK_TH + 2 * r, RW = LK_TW + 2 * r;
    return 5 * (RH * RW + RH * LK_TW);
}

// ---------------------------------------------------------------- iteration tile
// One Gauss-Newton iteration (Sect. 2.4) on one LK_TH x LK_TW output tile. Per pixel of
// the tile plus an r-pixel halo: warp I2 by the current estimate, take the gradient of
// I2 there, form e~ = I1 - I2w + g.(u - u_ref) and the five products; then box sums
// (rows, then columns) and the 2x2 solve for the new estimate u_ref + x.
// u_ref is the estimate at the tile centre: the equations are exact for any constant
// reference, and subtracting one keeps the FP32 right-hand side small.
template <typename T, bool NC>
__device__ __forceinline__ void lk_tile(const IterArgs &a, int tile, int r, float fp64_cond, float *smem)
{
    const int RH = LK_TH + 2 * r, RW = LK_TW + 2 * r;
    const int plane = RH * RW;
    float *P = smem;
    float *S = smem + 5 * plane;
    const int tyi = tile / a.tiles_x;
    const int ty0 = tyi * LK_TH, tx0 = (tile - tyi * a.tiles_x) * LK_TW;
    const float2 ref = flow_at<NC>(a, min(tx0 + LK_TW / 2, a.W - 1), min(ty0 + LK_TH / 2, a.H - 1));
    const T *I1 = static_cast<const T *>(a.I1);
    const T *I2 = static_cast<const T *>(a.I2);
    __syncthreads();   // the previous tile's readers of smem are done
    for (int i = threadIdx.x; i < plane; i += blockDim.x) {
        const int ry = i / RW, rx = i - ry * RW;
        const int y = ty0 - r + ry, x = tx0 - r + rx;
        float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f, p3 = 0.0f, p4 = 0.0f;
        if (y >= 0 && y < a.H && x >= 0 && x < a.W) {
            const float2 f = flow_at<NC>(a, x, y);
            float Iw, gx, gy;
            sample_grad<NC>(I2, a.pitch, a.H, a.W, (float)x + f.x, (float)y + f.y, Iw, gx, gy);
            const float e = ldf<NC>(I1 + (size_t)y * a.pitch + x) - Iw + gx * (f.x - ref.x) + gy * (f.y - ref.y);
            p0 = gx * gx;
            p1 = gx * gy;
            p2 = gy * gy;
            p3 = gx * e;
            p4 = gy * e;
        }
        P[i] = p0;
        P[plane + i] = p1;
        P[2 * plane + i] = p2;
        P[3 * plane + i] = p3;
        P[4 * plane + i] = p4;
    }
    __syncthreads();
    box_hsum(P, S, RH, RW, r);
    __syncthreads();
    for (int i = threadIdx.x; i < LK_TH * LK_TW; i += blockDim.x) {
        const int ty = i / LK_TW, tx = i - ty * LK_TW;
        const int y = ty0 + ty, x = tx0 + tx;
        if (y >= a.H || x >= a.W) continue;
        float s[5];
        box_vsum(S, RH, r, ty, tx, s);
        float2 f = flow_at<NC>(a, x, y);
        float xu, xv;
        if (solve2(s, fp64_cond, xu, xv)) f = make_float2(ref.x + xu, ref.y + xv);
        if (a.fout) {
            a.fout[(size_t)y * a.fout_pitch + x] = f;
        } else {
            a.u_out[(size_t)y * a.W + x] = f.x;
            a.v_out[(size_t)y * a.W + x] = f.y;
        }
    }
}

}  // namespace of
