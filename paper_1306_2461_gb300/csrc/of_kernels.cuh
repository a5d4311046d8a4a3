// Device tile functions shared by the per-level kernels and the persistent batched
// kernel: one pyramid-reduction tile and one Gauss-Newton iteration tile.
#pragma once

#include <float.h>

#include <climits>

#include "async_copy.cuh"
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

// The pair of block b in a phase launch: the largest p with prefix[p] <= b.
__device__ __forceinline__ int phase_pair(const int32_t *prefix, int n, int b)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// L2 prefetch of row `slot` of the rectangle [y0, y1) x [x0, x1) of a pitched image
// (elements of `elem` bytes), clamped to the image. Rows of the pyramid and flow buffers
// start 16-byte aligned and span pitch * elem bytes, a multiple of 16, so the widened
// range stays inside the row.
__device__ __forceinline__ void prefetch_row(const void *base, int pitch, int elem, int H, int W, int y0, int y1,
                                             int x0, int x1, int slot)
{
    y0 = max(y0, 0);
    y1 = min(y1, H);
    x0 = max(x0, 0);
    x1 = min(x1, W);
    if (x0 >= x1 || slot < 0 || slot >= y1 - y0) return;
    const char *row = static_cast<const char *>(base) + (size_t)(y0 + slot) * pitch * elem;
    const uintptr_t s = reinterpret_cast<uintptr_t>(row + (size_t)x0 * elem) & ~uintptr_t(15);
    const uintptr_t e = (reinterpret_cast<uintptr_t>(row + (size_t)x1 * elem) + 15) & ~uintptr_t(15);
    prefetch_l2(reinterpret_cast<const void *>(s), (uint32_t)(e - s));
}

// Warm L2 with what the block that runs iteration tile `tile` will read first: its region
// (tile + r-pixel halo) of the current estimate (flow mode MODE, or a.mode at run time when
// MODE < 0), of I1, of I2 widened by PF_MARGIN pixels for the displacement, and of the
// variant's window matrices (a.hess, when set). Threads [0, 64) take the estimate's rows,
// [64, 128) I1's, [128, 192) I2's, [192, 256) the window matrices'.
constexpr int PF_MARGIN = 8;
template <typename T, int MODE, int TH = LK_TH>
__device__ __forceinline__ void prefetch_tile(const IterArgs &a, int tile, int r)
{
    const int tyi = tile / a.tiles_x;
    const int ty0 = tyi * TH - r, tx0 = (tile - tyi * a.tiles_x) * LK_TW - r;
    const int ty1 = ty0 + TH + 2 * r, tx1 = tx0 + LK_TW + 2 * r;
    const int t = threadIdx.x;
    const int mode = MODE >= 0 ? MODE : a.mode;
    if (t < 64) {
        if (mode == FLOW_SAME)
            prefetch_row(a.fin, a.fin_pitch, 8, a.H, a.W, ty0, ty1, tx0, tx1, t);
        else if (mode == FLOW_UPSAMPLE)
            prefetch_row(a.fin, a.fin_pitch, 8, a.Hc, a.Wc, ty0 >> 1, (ty1 >> 1) + 2, tx0 >> 1, (tx1 >> 1) + 2, t);
    } else if (t < 128) {
        prefetch_row(a.I1, a.pitch, (int)sizeof(T), a.H, a.W, ty0 - 1, ty1 + 1, tx0 - 1, tx1 + 1, t - 64);
    } else if (t < 192) {
        prefetch_row(a.I2, a.pitch, (int)sizeof(T), a.H, a.W, ty0 - PF_MARGIN, ty1 + PF_MARGIN, tx0 - PF_MARGIN,
                     tx1 + PF_MARGIN, t - 128);
    } else if (a.hess) {
        prefetch_row(a.hess, a.hess_pitch, 16, a.H, a.W, ty0 + r, ty1 - r, tx0 + r, tx1 - r, t - 192);
    }
}

// [1 4 6 4 1] . (a, b, c, d, e), with its roundings fixed: (a + e) + 4 (b + d) + 6 c.
__device__ __forceinline__ float binom5(float a, float b, float c, float d, float e)
{
    return fmaf(6.0f, c, fmaf(4.0f, __fadd_rn(b, d), __fadd_rn(a, e)));
}

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
        // the tile's level-0 pixels, as they are: 16-byte chunks straight from the camera
        // image when its rows allow it and the tile lies inside the image, else element
        // by element from shared memory (the same values either way)
        constexpr int E = 16 / (int)sizeof(Tin);
        constexpr int CPR = 2 * PYR_TW / E;   // chunks per tile row
        const bool chunks = 2 * tx0 + 2 * PYR_TW <= a.W && 2 * ty0 + 2 * PYR_TH <= a.H &&
                            (a.src_pitch * (int)sizeof(Tin)) % 16 == 0 && (a.dst0_pitch * (int)sizeof(Tin)) % 16 == 0 &&
                            (reinterpret_cast<uintptr_t>(src) & 15) == 0 && (reinterpret_cast<uintptr_t>(d0) & 15) == 0;
        if (chunks) {
            for (int i = threadIdx.x; i < 2 * PYR_TH * CPR; i += blockDim.x) {
                const int r = i / CPR, c = i - r * CPR;
                const int y = 2 * ty0 + r, x = 2 * tx0 + c * E;
                *reinterpret_cast<uint4 *>(d0 + (size_t)y * a.dst0_pitch + x) =
                    ld<NC>(reinterpret_cast<const uint4 *>(src + (size_t)y * a.src_pitch + x));
            }
        } else {
            for (int i = threadIdx.x; i < 4 * PYR_TH * PYR_TW; i += blockDim.x) {
                const int r = i / (2 * PYR_TW), c = i - r * (2 * PYR_TW);
                const int y = 2 * ty0 + r, x = 2 * tx0 + c;
                if (y < a.H && x < a.W)
                    d0[(size_t)y * a.dst0_pitch + x] = to_elem<Tin>(s_in[(r + 2) * PYR_RW + c + 2]);
            }
        }
    }
    Tout *d = static_cast<Tout *>(img ? a.dst[1] : a.dst[0]);
    if (d == nullptr) return;   // one-level plan: level 0 only (uniform per block)
    for (int i = threadIdx.x; i < PYR_RH * PYR_TW; i += blockDim.x) {
        const int r = i / PYR_TW, j = i - r * PYR_TW;
        const float *q = s_in + r * PYR_RW + 2 * j;
        s_h[i] = binom5(q[0], q[1], q[2], q[3], q[4]);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < PYR_TH * PYR_TW; i += blockDim.x) {
        const int r = i / PYR_TW, j = i - r * PYR_TW;
        const int y = ty0 + r, x = tx0 + j;
        if (y < a.Ho && x < a.Wo) {
            const float *q = s_h + 2 * r * PYR_TW + j;
            const float s = binom5(q[0], q[PYR_TW], q[2 * PYR_TW], q[3 * PYR_TW], q[4 * PYR_TW]);
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

// ---------------------------------------------------------- normalisation tile
// Eq. 2 on one ZN_T x ZN_T tile: window sums S1 = sum I and S2 = sum I^2 over the
// (2*ZN_RADIUS+1)^2 window clipped to the image (n pixels) in exact integer arithmetic,
// then out = (n I - S1) / sqrt(n S2 - S1^2 + n^2 eps) in FP32.
constexpr int ZN_RR = ZN_T + 2 * ZN_RADIUS;
constexpr int ZN_SMEM_FLOATS = ZN_RR * ZN_RR + ZN_RR * ZN_T + 2 * ZN_RR * ZN_T;

template <typename Tin, typename Tout, bool NC>
__device__ __forceinline__ void znssd_tile(const ZnArgs &a, int tile, int img, float *smem)
{
    unsigned int *s_raw = reinterpret_cast<unsigned int *>(smem);                 // ZN_RR x ZN_RR
    unsigned int *s_h1 = s_raw + ZN_RR * ZN_RR;                                   // ZN_RR x ZN_T
    unsigned long long *s_h2 = reinterpret_cast<unsigned long long *>(s_h1 + ZN_RR * ZN_T);
    const int ty0 = (tile / a.tiles_x) * ZN_T;
    const int tx0 = (tile - (tile / a.tiles_x) * a.tiles_x) * ZN_T;
    const Tin *src = static_cast<const Tin *>(img ? a.src[1] : a.src[0]);
    Tout *dst = static_cast<Tout *>(img ? a.dst[1] : a.dst[0]);
    __syncthreads();   // the previous tile's readers of smem are done
    for (int i = threadIdx.x; i < ZN_RR * ZN_RR; i += blockDim.x) {
        const int ry = i / ZN_RR, rx = i - ry * ZN_RR;
        const int y = ty0 - ZN_RADIUS + ry, x = tx0 - ZN_RADIUS + rx;
        s_raw[i] = ((unsigned)y < (unsigned)a.H && (unsigned)x < (unsigned)a.W)
                       ? (unsigned int)ld<NC>(src + ((size_t)y * a.src_pitch + x))
                       : 0u;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ZN_RR * ZN_T; i += blockDim.x) {
        const int ry = i / ZN_T, tx = i - ry * ZN_T;
        const unsigned int *q = s_raw + ry * ZN_RR + tx;
        unsigned int h1 = 0;
        unsigned long long h2 = 0;
#pragma unroll
        for (int k = 0; k <= 2 * ZN_RADIUS; ++k) {
            h1 += q[k];
            h2 += (unsigned long long)q[k] * q[k];
        }
        s_h1[i] = h1;
        s_h2[i] = h2;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < ZN_T * ZN_T; i += blockDim.x) {
        const int ty = i / ZN_T, tx = i - ty * ZN_T;
        const int y = ty0 + ty, x = tx0 + tx;
        if (y >= a.H || x >= a.W) continue;
        long long s1 = 0, s2 = 0;
#pragma unroll
        for (int k = 0; k <= 2 * ZN_RADIUS; ++k) {
            s1 += s_h1[(ty + k) * ZN_T + tx];
            s2 += (long long)s_h2[(ty + k) * ZN_T + tx];
        }
        const long long n = (long long)(min(x + ZN_RADIUS, a.W - 1) - max(x - ZN_RADIUS, 0) + 1) *
                            (min(y + ZN_RADIUS, a.H - 1) - max(y - ZN_RADIUS, 0) + 1);
        const long long I = s_raw[(ty + ZN_RADIUS) * ZN_RR + tx + ZN_RADIUS];
        const float num = (float)(n * I - s1);
        const float rad = (float)(n * s2 - s1 * s1 + n * n * ZN_EPS);
        dst[(size_t)y * a.dst_pitch + x] = to_elem<Tout>(num / sqrtf(rad));
    }
}

// ------------------------------------------------------------ iteration helpers
// The arithmetic below is written with explicit fused and unfused operations so that
// every code path that computes a quantity (per-pair and batched kernels, gathered and
// staged taps) rounds it the same way, whatever the compiler would contract.
__device__ __forceinline__ float lerpf(float p, float q, float t) { return fmaf(t, q, __fmul_rn(1.0f - t, p)); }

// e~ = I1 - I2w + gx dx + gy dy (dx, dy: current estimate minus the tile's reference).
__device__ __forceinline__ float resid(float i1, float Iw, float gx, float gy, float dx, float dy)
{
    return fmaf(gy, dy, fmaf(gx, dx, __fsub_rn(i1, Iw)));
}

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
        const int o = (y0 - 1) * pitch + x0;
        const T *rm = I + o, *r0 = I + (o + pitch), *r1 = I + (o + 2 * pitch), *r2 = I + (o + 3 * pitch);
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

// Current estimate at (x, y) of the level being iterated, for a flow mode known at
// compile time (offsets in 32 bits: a level holds fewer than 2^31 elements).
template <bool NC, int MODE>
__device__ __forceinline__ float2 flow_at_m(const IterArgs &a, int x, int y)
{
    if constexpr (MODE == FLOW_ZERO) {
        return make_float2(0.0f, 0.0f);
    } else if constexpr (MODE == FLOW_SAME) {
        return ld<NC>(a.fin + (y * a.fin_pitch + x));
    } else {
        // 2 * bilinear(coarse; x/2, y/2): weights are 0 or 1/2, indices clamped
        const int x0 = x >> 1, y0 = y >> 1;
        const int x1 = min(x0 + 1, a.Wc - 1), y1 = min(y0 + 1, a.Hc - 1);
        const float ax = (x & 1) ? 0.5f : 0.0f, ay = (y & 1) ? 0.5f : 0.0f;
        const float2 *r0 = a.fin + y0 * a.fin_pitch, *r1 = a.fin + y1 * a.fin_pitch;
        const float2 f00 = ld<NC>(r0 + x0), f01 = ld<NC>(r0 + x1);
        const float2 f10 = ld<NC>(r1 + x0), f11 = ld<NC>(r1 + x1);
        return make_float2(2.0f * lerpf(lerpf(f00.x, f01.x, ax), lerpf(f10.x, f11.x, ax), ay),
                           2.0f * lerpf(lerpf(f00.y, f01.y, ax), lerpf(f10.y, f11.y, ax), ay));
    }
}

// The same with the mode read at run time.
template <bool NC>
__device__ __forceinline__ float2 flow_at(const IterArgs &a, int x, int y)
{
    if (a.mode == FLOW_ZERO) return flow_at_m<NC, FLOW_ZERO>(a, x, y);
    if (a.mode == FLOW_SAME) return flow_at_m<NC, FLOW_SAME>(a, x, y);
    return flow_at_m<NC, FLOW_UPSAMPLE>(a, x, y);
}

// MODE < 0: read the mode at run time.
template <bool NC, int MODE>
__device__ __forceinline__ float2 flow_mode(const IterArgs &a, int x, int y)
{
    if constexpr (MODE < 0) return flow_at<NC>(a, x, y);
    else return flow_at_m<NC, MODE>(a, x, y);
}

// Horizontal pass of the box sums of C planes: S[c][ry][tx] = sum_{k=0..2r} P[c][ry][tx+k], left to right.
template <int C = 5>
__device__ __forceinline__ void box_hsum(const float *P, float *S, int RH, int RW, int r)
{
    const int n = RH * LK_TW;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int ry = i / LK_TW, tx = i - ry * LK_TW;
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float *q = P + (size_t)c * RH * RW + ry * RW + tx;
            float s = 0.0f;
            for (int k = 0; k <= 2 * r; ++k) s += q[k];
            S[c * n + i] = s;
        }
    }
}

// Vertical pass at output (ty, tx): sums of S over rows ty..ty+2r, top to bottom.
template <int C = 5>
__device__ __forceinline__ void box_vsum(const float *S, int RH, int r, int ty, int tx, float s[C])
{
    const int n = RH * LK_TW;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float *q = S + c * n + ty * LK_TW + tx;
        float acc = 0.0f;
        for (int k = 0; k <= 2 * r; ++k) acc += q[k * LK_TW];
        s[c] = acc;
    }
}

// Solve [a b; b c] x = [d; e]. Returns false (keep the estimate) when tr <= 0 or
// det <= 1e-6 tr^2. Pixels with tr^2/det above fp64_cond (or det <= 0) form the
// determinant and the numerators in FP64 from the FP32 sums; fp64_cond == 0 keeps
// everything in FP32.
__device__ __forceinline__ bool solve2(const float s[5], float fp64_cond, float &xu, float &xv)
{
    const float a = s[0], b = s[1], c = s[2], d = s[3], e = s[4];
    const float tr = a + c;
    if (!(tr > 0.0f)) return false;
    const float det = fmaf(a, c, -__fmul_rn(b, b));
    if (fp64_cond > 0.0f && !(det * fp64_cond > tr * tr)) {
        // ill-conditioned: the determinant and the numerators, where the cancellation
        // is, in FP64 from the FP32 sums (the products are exact, one rounding each);
        // the final divisions in FP32
        const double A = a, B = b, C = c, D = d, E = e;
        const double T = A + C, dt = fma(A, C, -__dmul_rn(B, B));
        if (!(dt > 1e-6 * T * T)) return false;
        const float fdt = (float)dt;
        if (!(fdt >= FLT_MIN)) return false;
        xu = __fdiv_rn((float)fma(C, D, -__dmul_rn(B, E)), fdt);
        xv = __fdiv_rn((float)fma(A, E, -__dmul_rn(B, D)), fdt);
        return true;
    }
    if (!(det > 1e-6f * tr * tr)) return false;
    const float inv = __fdividef(1.0f, det);   // det < 2^126 for any sums of 16-bit data
    xu = fmaf(c, d, -__fmul_rn(b, e)) * inv;
    xv = fmaf(a, e, -__fmul_rn(b, d)) * inv;
    return true;
}

inline __host__ __device__ int lk_smem_floats(int r)   // generic tile
{
    const int RH = LK_TH + 2 * r, RW = LK_TW + 2 * r;
    return 5 * (RH * RW + RH * LK_TW);
}

// ----------------------------------------------------------- generic iteration tile
// One Gauss-Newton iteration (Sect. 2.4) on one LK_TH x LK_TW output tile, for any
// window radius r given at run time (the fixed-radius tile below is the fast path). Per pixel of
// the tile plus an r-pixel halo: warp I2 by the current estimate, take the gradient of
// I2 there, form e~ = I1 - I2w + g.(u - u_ref) and the five products; then box sums
// (rows, then columns) and the 2x2 solve for the new estimate u_ref + x.
// u_ref is the estimate at the tile centre: the equations are exact for any constant
// reference, and subtracting one keeps the FP32 right-hand side small.
template <typename T, bool NC>
__device__ __forceinline__ void lk_tile_generic(const IterArgs &a, int tile, int r, float fp64_cond, float *smem)
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
            const float e = resid(ldf<NC>(I1 + (size_t)y * a.pitch + x), Iw, gx, gy, f.x - ref.x, f.y - ref.y);
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
        float xu, xv;
        const float2 f = solve2(s, fp64_cond, xu, xv) ? make_float2(ref.x + xu, ref.y + xv) : flow_at<NC>(a, x, y);
        if (a.fout) {
            a.fout[(size_t)y * a.fout_pitch + x] = f;
        } else {
            a.u_out[(size_t)y * a.W + x] = f.x;
            a.v_out[(size_t)y * a.W + x] = f.y;
        }
    }
}


// ------------------------------------------------------- fixed-radius iteration tile
// The same iteration with the window radius R known at compile time (R >= 2). Box
// sums are formed for groups of 4 consecutive outputs at once: the 2R-2 terms in the
// middle of the 4 windows are added once and shared, each output adds its own 3 edge
// terms (4.25 additions per output and channel for R = 4, instead of 8). Groups start
// at multiples of 4 in image coordinates (tiles are multiples of 4 wide and high), so
// the order of the additions depends only on the pixel's position, not on the tiling:
// the batched and the per-pair launches give the same bits.
template <int R, int TH = LK_TH> struct FixedTile {
    static_assert(R >= 2, "the grouped box sums need 2R >= 4");
    static constexpr int W = 2 * R + 1;                // window width
    static constexpr int NV4 = (2 * R + 4 + 3) / 4;    // float4 loads for 4 outputs' windows
    static constexpr int RH = TH + 2 * R;              // region rows (tile + halo)
    static constexpr int RW = LK_TW + 2 * R;           // region columns
    static constexpr int RWP = LK_TW + 4 * NV4 - 4;    // padded row length (>= RW, multiple of 4)
    static constexpr int PLANE = RH * RWP;
    static constexpr int NREG = RH * RW;               // region pixels
    static constexpr int PER = (NREG + LK_THREADS - 1) / LK_THREADS;   // region pixels per thread
    // Staging of I2 (a.stage_i2): a window of the tile's region shifted by the tile's
    // reference flow and widened by STAGE_MARGIN pixels (plus the 4x4 tap footprint and
    // 16-byte alignment of its rows), in the storage type. WIN_BYTES holds it for 1- and
    // 2-byte types; a larger window (FP32 storage) is not staged.
    static constexpr int STAGE_MARGIN = 6;
    static constexpr int WIN_ROWS = TH + 2 * R + 2 * STAGE_MARGIN + 4;
    static constexpr int WIN_BYTES = WIN_ROWS * 2 * (LK_TW + 2 * R + 2 * STAGE_MARGIN + 4 + 16);
    static_assert(PLANE % 4 == 0, "the barrier and the window after the planes must be 16-byte aligned");
    static constexpr int OFF_BAR = 5 * PLANE;       // 8-byte mbarrier
    static constexpr int OFF_WIN = OFF_BAR + 4;     // 16-byte aligned staging window
    static constexpr int SMEM_NOSTAGE = OFF_WIN;    // launches without I2 staging
    static constexpr int SMEM_FLOATS = OFF_WIN + (WIN_BYTES + 15) / 16 * 4;
#ifndef OF_LK_MIN_BLOCKS
#define OF_LK_MIN_BLOCKS 5   // resident blocks per SM the fixed-radius kernels are compiled for (R <= 6)
#endif
    // resident blocks per SM the kernels are compiled for: the measured choice for the
    // default tile height, else as many as the shared memory holds (at most 5)
    static constexpr int SMEM_FIT = 233472 / (4 * (5 * PLANE + 4) + 1024);
    static constexpr int MIN_BLOCKS =
        TH == LK_TH ? (R <= 6 ? OF_LK_MIN_BLOCKS : 2) : (SMEM_FIT < 1 ? 1 : (SMEM_FIT > 5 ? 5 : SMEM_FIT));
};

constexpr long long STAGE_TIMEOUT_NS = 200000000LL;   // 0.2 s for one tile's row copies

template <typename T> __device__ __forceinline__ float ld_smem_elem(const unsigned char *p)
{
    return ldf<false>(reinterpret_cast<const T *>(p));
}

// The interior branch of sample_grad with its 12 taps read from the staged window (rows
// wy0.., columns wx0.., `rowbytes` per row). Returns false, reading nothing, when the
// 4x4 footprint of (px, py) is not inside both the window and the image's interior.
template <typename T>
__device__ __forceinline__ bool sample_grad_win(const unsigned char *win, int rowbytes, int wx0, int wy0, int wx1,
                                                int wy1, int H, int W, float px, float py, float &Iw, float &gx,
                                                float &gy)
{
    if (!(px >= 1.0f && py >= 1.0f && px < (float)(W - 2) && py < (float)(H - 2))) return false;
    const float fx = floorf(px), fy = floorf(py);
    const int x0 = (int)fx, y0 = (int)fy;
    if (x0 - 1 < wx0 || x0 + 2 >= wx1 || y0 - 1 < wy0 || y0 + 2 >= wy1) return false;
    const float ax = px - fx, ay = py - fy;
    constexpr int S = (int)sizeof(T);
    const unsigned char *rm = win + (y0 - 1 - wy0) * rowbytes + (x0 - wx0) * S;
    const unsigned char *r0 = rm + rowbytes, *r1 = r0 + rowbytes, *r2 = r1 + rowbytes;
    const float a0 = ld_smem_elem<T>(rm), a1 = ld_smem_elem<T>(rm + S);
    const float bm = ld_smem_elem<T>(r0 - S), b0 = ld_smem_elem<T>(r0), b1 = ld_smem_elem<T>(r0 + S),
                b2 = ld_smem_elem<T>(r0 + 2 * S);
    const float cm = ld_smem_elem<T>(r1 - S), c0 = ld_smem_elem<T>(r1), c1 = ld_smem_elem<T>(r1 + S),
                c2 = ld_smem_elem<T>(r1 + 2 * S);
    const float d0 = ld_smem_elem<T>(r2), d1 = ld_smem_elem<T>(r2 + S);
    const float top = lerpf(b0, b1, ax), bot = lerpf(c0, c1, ax);
    Iw = lerpf(top, bot, ay);
    gx = (lerpf(lerpf(b1, b2, ax), lerpf(c1, c2, ax), ay) - lerpf(lerpf(bm, b0, ax), lerpf(cm, c0, ax), ay)) * 0.5f;
    gy = (lerpf(bot, lerpf(d0, d1, ax), ay) - lerpf(lerpf(a0, a1, ax), top, ay)) * 0.5f;
    return true;
}

// o[j] = sum_{k=0}^{2R} v[j+k], j = 0..3, from v[0 .. 2R+3].
template <int R>
__device__ __forceinline__ void box4(const float *v, float o[4])
{
    float m = v[3];
#pragma unroll
    for (int k = 4; k <= 2 * R; ++k) m += v[k];
    o[0] = ((v[0] + v[1]) + v[2]) + m;
    o[1] = ((v[1] + v[2]) + m) + v[2 * R + 1];
    o[2] = ((v[2] + m) + v[2 * R + 1]) + v[2 * R + 2];
    o[3] = ((m + v[2 * R + 1]) + v[2 * R + 2]) + v[2 * R + 3];
}

// Horizontal pass, in place: row ry of plane c (c < C) becomes, at columns
// 0..LK_TW-1, the window sums of the outputs of that row.
template <int R, int C = 5, int TH = LK_TH>
__device__ __forceinline__ void box_h_inplace(float *P)
{
    using F = FixedTile<R, TH>;
    constexpr int NG = LK_TW / 4;
    static_assert(32 % NG == 0 && LK_THREADS % 32 == 0, "a row's items must lie in one warp");
    constexpr int NITEMS = F::RH * NG;
    constexpr int IT = (NITEMS + LK_THREADS - 1) / LK_THREADS;
#pragma unroll 1
    for (int c = 0; c < C; ++c) {
        float *Pc = P + c * F::PLANE;
        float4 res[IT];
#pragma unroll
        for (int k = 0; k < IT; ++k) {
            const int i = threadIdx.x + k * LK_THREADS;
            if (i < NITEMS) {
                const int ry = i / NG, g = i % NG;
                const float4 *src = reinterpret_cast<const float4 *>(Pc + ry * F::RWP + 4 * g);
                float v[4 * F::NV4];
#pragma unroll
                for (int q = 0; q < F::NV4; ++q) {
                    const float4 t = src[q];
                    v[4 * q] = t.x;
                    v[4 * q + 1] = t.y;
                    v[4 * q + 2] = t.z;
                    v[4 * q + 3] = t.w;
                }
                float o[4];
                box4<R>(v, o);
                res[k] = make_float4(o[0], o[1], o[2], o[3]);
            }
        }
        // Item i covers row i / NG: the NG = 16 items of a row are 16 consecutive lanes
        // of one warp (in every pass), so only that warp reads what it overwrites.
        __syncwarp();
#pragma unroll
        for (int k = 0; k < IT; ++k) {
            const int i = threadIdx.x + k * LK_THREADS;
            if (i < NITEMS) {
                const int ry = i / NG, g = i % NG;
                *reinterpret_cast<float4 *>(Pc + ry * F::RWP + 4 * g) = res[k];
            }
        }
    }
    __syncthreads();
}

// Vertical pass for the 4 outputs (rows 4g..4g+3, column tx) of each of C channels.
template <int R, int C = 5, int TH = LK_TH>
__device__ __forceinline__ void box_v4(const float *P, int g, int tx, float s[C][4])
{
    using F = FixedTile<R, TH>;
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float *col = P + c * F::PLANE + 4 * g * F::RWP + tx;
        float v[2 * R + 4];
#pragma unroll
        for (int q = 0; q < 2 * R + 4; ++q) v[q] = col[q * F::RWP];
        box4<R>(v, s[c]);
    }
}

// The tile's mbarrier: initialised once per block, before the first tile.
template <int R, int TH = LK_TH> __device__ __forceinline__ void lk_tile_init(float *smem)
{
    if (threadIdx.x == 0) {
        mbar_init(reinterpret_cast<uint64_t *>(smem + FixedTile<R, TH>::OFF_BAR), 1);
        fence_proxy_async_smem();
    }
    __syncthreads();
}

// Returns false if the staging copy did not complete in time (then OF_ETIMEOUT is in
// *a.status, nothing of the tile was written, and the block must stop).
template <typename T, bool NC, int R, int MODE, int TH = LK_TH>
__device__ __forceinline__ bool lk_tile_fixed(const IterArgs &a, int tile, float fp64_cond, float *smem,
                                              uint32_t &phase)
{
    using F = FixedTile<R, TH>;
    float *P = smem;
    unsigned char *win = reinterpret_cast<unsigned char *>(smem + F::OFF_WIN);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + F::OFF_BAR);
    const int tyi = tile / a.tiles_x;
    const int ty0 = tyi * TH, tx0 = (tile - tyi * a.tiles_x) * LK_TW;
    const float2 ref = flow_mode<NC, MODE>(a, min(tx0 + LK_TW / 2, a.W - 1), min(ty0 + TH / 2, a.H - 1));
    const T *I1 = static_cast<const T *>(a.I1);
    const T *I2 = static_cast<const T *>(a.I2);
    __syncthreads();   // the previous tile's readers of smem are done
    // Staging: the window of I2 around the tile's region displaced by the reference flow,
    // row by row with bulk copies (raw storage type, 16-byte aligned rows, clamped to the
    // image's rows and to the padded row length). The window is the same for every thread.
    int wx0 = 0, wx1 = 0, wy0 = 0, wy1 = 0, rowbytes = 0;
    bool staged = false;
    if (a.stage_i2) {
        constexpr int E = 16 / (int)sizeof(T);   // elements per 16-byte chunk
        const int ox = __float2int_rn(fminf(fmaxf(ref.x, -(float)a.W), (float)a.W));
        const int oy = __float2int_rn(fminf(fmaxf(ref.y, -(float)a.H), (float)a.H));
        wx0 = max(tx0 - R - F::STAGE_MARGIN + ox - 1, 0) / E * E;
        wx1 = (min(tx0 + LK_TW + R + F::STAGE_MARGIN + ox + 3, a.pitch) + E - 1) / E * E;   // pitch: multiple of E
        wy0 = max(ty0 - R - F::STAGE_MARGIN + oy - 1, 0);
        wy1 = min(ty0 + TH + R + F::STAGE_MARGIN + oy + 3, a.H);
        rowbytes = (wx1 - wx0) * (int)sizeof(T);
        const int rows = wy1 - wy0;
        staged = wx1 > wx0 && rows > 0 && rows * rowbytes <= F::WIN_BYTES;
        if (staged) {
            if (threadIdx.x < 32) {
                if (threadIdx.x == 0) {
                    fence_proxy_async_smem();
                    mbar_arrive_expect_tx(bar, (uint32_t)(rows * rowbytes));
                }
                __syncwarp();
                fence_proxy_async_global();
                for (int k = threadIdx.x; k < rows; k += 32)
                    bulk_g2s(win + k * rowbytes, I2 + (size_t)(wy0 + k) * a.pitch + wx0, (uint32_t)rowbytes, bar);
            }
            const bool done = mbar_wait_bounded(bar, phase, STAGE_TIMEOUT_NS);
            phase ^= 1u;
            if (__syncthreads_or(!done)) {
                if (threadIdx.x == 0 && a.status) atomicExch(a.status, DEV_TIMEOUT);
                return false;
            }
        }
    }
    // stage 1: products over the tile and its R-pixel halo. The current estimates of
    // S1 pixels are loaded before any of them is used, so that their latencies overlap.
    constexpr int S1 = 3;   // measured: 1, 2, 3, 4, 6, 12 -> 3 is fastest
#pragma unroll 1
    for (int k0 = 0; k0 < F::PER; k0 += S1) {
        float2 f[S1];
        bool in[S1];
#pragma unroll
        for (int u = 0; u < S1; ++u) {
            const int i = threadIdx.x + (k0 + u) * LK_THREADS;
            const int ry = i / F::RW, rx = i - ry * F::RW;
            const int y = ty0 - R + ry, x = tx0 - R + rx;
            in[u] = i < F::NREG && (unsigned)y < (unsigned)a.H && (unsigned)x < (unsigned)a.W;
            f[u] = in[u] ? flow_mode<NC, MODE>(a, x, y) : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int u = 0; u < S1; ++u) {
            const int i = threadIdx.x + (k0 + u) * LK_THREADS;
            if (i >= F::NREG) break;
            const int ry = i / F::RW, rx = i - ry * F::RW;
            const int y = ty0 - R + ry, x = tx0 - R + rx;
            float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f, p3 = 0.0f, p4 = 0.0f;
            if (in[u]) {
                float Iw, gx, gy;
                const float px = (float)x + f[u].x, py = (float)y + f[u].y;
                if (!(staged && sample_grad_win<T>(win, rowbytes, wx0, wy0, wx1, wy1, a.H, a.W, px, py, Iw, gx, gy)))
                    sample_grad<NC>(I2, a.pitch, a.H, a.W, px, py, Iw, gx, gy);
                const float e = resid(ldf<NC>(I1 + (y * a.pitch + x)), Iw, gx, gy, f[u].x - ref.x, f[u].y - ref.y);
                p0 = gx * gx;
                p1 = gx * gy;
                p2 = gy * gy;
                p3 = gx * e;
                p4 = gy * e;
            }
            float *q = P + ry * F::RWP + rx;
            q[0] = p0;
            q[F::PLANE] = p1;
            q[2 * F::PLANE] = p2;
            q[3 * F::PLANE] = p3;
            q[4 * F::PLANE] = p4;
        }
    }
    __syncthreads();
    box_h_inplace<R, 5, TH>(P);
    // vertical sums, solve and write, 4 rows of one column per item
    constexpr int VITEMS = LK_TW * (TH / 4);
#pragma unroll 1
    for (int i = threadIdx.x; i < VITEMS; i += LK_THREADS) {
        const int tx = i % LK_TW, g = i / LK_TW;
        const int x = tx0 + tx;
        if (x >= a.W || ty0 + 4 * g >= a.H) continue;
        float s[5][4];
        box_v4<R, 5, TH>(P, g, tx, s);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int y = ty0 + 4 * g + j;
            if (y >= a.H) break;
            const float sj[5] = {s[0][j], s[1][j], s[2][j], s[3][j], s[4][j]};
            float xu, xv;
            const float2 f = solve2(sj, fp64_cond, xu, xv) ? make_float2(ref.x + xu, ref.y + xv) : flow_mode<NC, MODE>(a, x, y);
            if (a.fout) {
                a.fout[(size_t)y * a.fout_pitch + x] = f;
            } else {
                a.u_out[(size_t)y * a.W + x] = f.x;
                a.v_out[(size_t)y * a.W + x] = f.y;
            }
        }
    }
    return true;
}

// The iteration tile for radius R (0 = generic, radius r at run time). MODE: the flow
// mode when it is known at compile time (-1: read a.mode at run time). Returns false
// when the block must stop (a staging copy timed out; recorded in *a.status).
template <typename T, bool NC, int R, int MODE = -1, int TH = LK_TH>
__device__ __forceinline__ bool lk_tile(const IterArgs &a, int tile, int r, float fp64_cond, float *smem,
                                        uint32_t &phase)
{
    if constexpr (R == 0) {
        lk_tile_generic<T, NC>(a, tile, r, fp64_cond, smem);
        return true;
    } else {
        return lk_tile_fixed<T, NC, R, MODE, TH>(a, tile, fp64_cond, smem, phase);
    }
}

template <int R, int TH = LK_TH> __device__ __forceinline__ void lk_tile_prepare(float *smem)
{
    if constexpr (R != 0) lk_tile_init<R, TH>(smem);
}

template <int R, int TH = LK_TH> constexpr int lk_min_blocks()
{
    if constexpr (R == 0) return 2;
    else return FixedTile<R, TH>::MIN_BLOCKS;
}

#ifndef OF_BATCH_MIN_BLOCKS
#define OF_BATCH_MIN_BLOCKS 3
#endif
// Resident blocks per SM the persistent kernel is compiled for (its register cap).
template <int R> constexpr int batch_min_blocks()
{
    constexpr int m = lk_min_blocks<R>();
    return m < OF_BATCH_MIN_BLOCKS ? m : OF_BATCH_MIN_BLOCKS;
}

template <int R, int TH = LK_TH> inline __host__ __device__ int lk_tile_smem_floats(int r, bool stage_i2)
{
    if constexpr (R == 0) return lk_smem_floats(r);
    else return stage_i2 ? FixedTile<R, TH>::SMEM_FLOATS : FixedTile<R, TH>::SMEM_NOSTAGE;
}

}  // namespace of
