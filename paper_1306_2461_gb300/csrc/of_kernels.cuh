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
// An output tile of PYR_TW x PYR_TH at level l+1 reads rows 2 ty0 - 2 .. 2 ty0 + 2 PYR_TH
// (PYR_RH rows) of level l and, per row, PYR_RWS(T) columns starting one 16-byte chunk
// left of 2 tx0 (the 5-tap window needs 2 tx0 - 2 .. 2 tx0 + 2 PYR_TW).
constexpr int PYR_RH = 2 * PYR_TH + 3;
template <typename T> constexpr int pyr_chunk() { return 16 / (int)sizeof(T); }   // elements per 16 bytes
template <typename T> constexpr int pyr_rws() { return 2 * PYR_TW + 2 * pyr_chunk<T>(); }
template <typename T> constexpr int pyr_smem_floats() { return PYR_RH * pyr_rws<T>() + PYR_RH * PYR_TW; }
constexpr int PYR_SMEM_FLOATS = PYR_RH * (2 * PYR_TW + 32) + PYR_RH * PYR_TW;   // the largest (8-bit input)

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

// L1 prefetch of the 128-byte lines of the rectangle [y0, y1) x [x0, x1) of a pitched
// image (elements of `elem` bytes), clamped to the image: line `slot` of at most `lpr`
// per row (slot < (y1 - y0) lpr; a row's lines past its last column are skipped), so
// that threads [0, (y1 - y0) lpr) take one line each.
__device__ __forceinline__ void prefetch_lines_l1(const void *base, int pitch, int elem, int H, int W, int y0,
                                                  int y1, int x0, int x1, int lpr, int slot)
{
    const int row = slot / lpr, line = slot - row * lpr;
    const int y = y0 + row;
    x0 = max(x0, 0);
    x1 = min(x1, W);
    if (x0 >= x1 || y < 0 || y >= min(y1, H)) return;
    const char *r = static_cast<const char *>(base) + (size_t)y * pitch * elem;
    const uintptr_t s = (reinterpret_cast<uintptr_t>(r + (size_t)x0 * elem) & ~uintptr_t(127)) + 128u * line;
    if (s > reinterpret_cast<uintptr_t>(r + (size_t)(x1 - 1) * elem)) return;
    asm volatile("prefetch.global.L1 [%0];" ::"l"(s));
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
    const int uy = tile / a.tiles_x;   // a work unit: its first tile
    const int ty0 = uy * strip_len(a.strip) * TH - r, tx0 = (tile - uy * a.tiles_x) * LK_TW - r;
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

// The elements of one 16-byte chunk as floats.
template <typename T> __device__ __forceinline__ void chunk_to_f(const uint4 &w, float *o)
{
    const T *e = reinterpret_cast<const T *>(&w);
#pragma unroll
    for (int k = 0; k < pyr_chunk<T>(); ++k) o[k] = ldf<false>(e + k);
}

// One output tile (PYR_TW x PYR_TH at level l+1) of image `img` (0/1) of a pair.
// FIRST: the source is the raw camera image; level 0 is stored as well, unchanged in
// the camera's integer format. Rows are read in 16-byte chunks (each thread one chunk at a
// time, converted to FP32 in shared memory once); the chunks of FIRST's level-0 copy are
// stored from the same registers. Chunks that cross the image border, or all of them when
// a row is not 16-byte aligned, are read element by element with clamped coordinates.
// Then the horizontal and the vertical binomial, 4 outputs per thread with 16-byte
// shared-memory accesses.
template <typename Tin, typename Tout, bool FIRST, bool NC>
__device__ __forceinline__ void pyr_tile_smem(const PyrArgs &a, int tile, int img, float *smem)
{
    constexpr int CH = pyr_chunk<Tin>();
    constexpr int RWS = pyr_rws<Tin>();
    constexpr int NCH = RWS / CH;   // chunks per row
    float *s_in = smem;                          // PYR_RH x RWS
    float *s_h = smem + PYR_RH * RWS;           // PYR_RH x PYR_TW
    const int ty0 = (tile / a.tiles_x) * PYR_TH;
    const int tx0 = (tile - (tile / a.tiles_x) * a.tiles_x) * PYR_TW;
    const int ys = 2 * ty0 - 2, cs = 2 * tx0 - CH;
    const Tin *src = static_cast<const Tin *>(img ? a.src[1] : a.src[0]);
    Tin *d0 = FIRST ? static_cast<Tin *>(img ? a.dst0[1] : a.dst0[0]) : nullptr;
    const bool vsrc = (a.src_pitch * (int)sizeof(Tin)) % 16 == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0;
    const bool vdst = FIRST && (a.dst0_pitch * (int)sizeof(Tin)) % 16 == 0 && (reinterpret_cast<uintptr_t>(d0) & 15) == 0;
    __syncthreads();   // the previous tile's readers of smem are done
    for (int i = threadIdx.x; i < PYR_RH * NCH; i += blockDim.x) {
        const int r = i / NCH, k = i - r * NCH;
        const int y = ys + r, c0 = cs + k * CH;
        float v[CH];
        const bool inside = vsrc && (unsigned)y < (unsigned)a.H && c0 >= 0 && c0 + CH <= a.W;
        if (inside) {
            const uint4 w = ld<NC>(reinterpret_cast<const uint4 *>(src + ((size_t)y * a.src_pitch + c0)));
            chunk_to_f<Tin>(w, v);
            // level 0 as it is: the tile's rows 2 ty0 .. 2 ty0 + 2 PYR_TH - 1, columns 2 tx0 ..
            if (FIRST && vdst && r >= 2 && r < 2 + 2 * PYR_TH && k >= 1 && k <= 2 * PYR_TW / CH)
                *reinterpret_cast<uint4 *>(d0 + ((size_t)y * a.dst0_pitch + c0)) = w;
        } else {
            const int yc = clampi(y, 0, a.H - 1);
#pragma unroll
            for (int e = 0; e < CH; ++e)
                v[e] = ldf<NC>(src + ((size_t)yc * a.src_pitch + clampi(c0 + e, 0, a.W - 1)));
        }
        if (FIRST && !(inside && vdst) && r >= 2 && r < 2 + 2 * PYR_TH && k >= 1 && k <= 2 * PYR_TW / CH &&
            (unsigned)y < (unsigned)a.H) {
#pragma unroll
            for (int e = 0; e < CH; ++e)
                if ((unsigned)(c0 + e) < (unsigned)a.W) d0[(size_t)y * a.dst0_pitch + c0 + e] = to_elem<Tin>(v[e]);
        }
        float4 *q = reinterpret_cast<float4 *>(s_in + r * RWS + k * CH);
#pragma unroll
        for (int e = 0; e < CH / 4; ++e) q[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
    }
    __syncthreads();
    Tout *d = static_cast<Tout *>(img ? a.dst[1] : a.dst[0]);
    if (d == nullptr) return;   // one-level plan: level 0 only (uniform per block)
    // horizontal: outputs 4g .. 4g + 3 of a row read columns 8g - 2 + CH .. 8g + 8 + CH
    // (image 2 (tx0 + 4g) - 2 ..), from the 16 floats starting at column 8g + CH - 4
    constexpr int NG = PYR_TW / 4;
    for (int i = threadIdx.x; i < PYR_RH * NG; i += blockDim.x) {
        const int r = i / NG, g = i - r * NG;
        const float4 *q = reinterpret_cast<const float4 *>(s_in + r * RWS + 8 * g + CH - 4);
        float v[16];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float4 t = q[e];
            v[4 * e] = t.x;
            v[4 * e + 1] = t.y;
            v[4 * e + 2] = t.z;
            v[4 * e + 3] = t.w;
        }
        float o[4];
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) o[jj] = binom5(v[2 + 2 * jj], v[3 + 2 * jj], v[4 + 2 * jj], v[5 + 2 * jj], v[6 + 2 * jj]);
        *reinterpret_cast<float4 *>(s_h + r * PYR_TW + 4 * g) = make_float4(o[0], o[1], o[2], o[3]);
    }
    __syncthreads();
    // vertical: output row i reads rows 2i .. 2i + 4 of s_h
    for (int i = threadIdx.x; i < PYR_TH * NG; i += blockDim.x) {
        const int r = i / NG, g = i - r * NG;
        const int y = ty0 + r, x = tx0 + 4 * g;
        if (y >= a.Ho || x >= a.Wo) continue;
        float4 c[5];
#pragma unroll
        for (int e = 0; e < 5; ++e) c[e] = *reinterpret_cast<const float4 *>(s_h + (2 * r + e) * PYR_TW + 4 * g);
        const float o0 = binom5(c[0].x, c[1].x, c[2].x, c[3].x, c[4].x) * (1.0f / 256.0f);
        const float o1 = binom5(c[0].y, c[1].y, c[2].y, c[3].y, c[4].y) * (1.0f / 256.0f);
        const float o2 = binom5(c[0].z, c[1].z, c[2].z, c[3].z, c[4].z) * (1.0f / 256.0f);
        const float o3 = binom5(c[0].w, c[1].w, c[2].w, c[3].w, c[4].w) * (1.0f / 256.0f);
        Tout *row = d + (size_t)y * a.dst_pitch + x;
        row[0] = to_elem<Tout>(o0);
        if (x + 1 < a.Wo) row[1] = to_elem<Tout>(o1);
        if (x + 2 < a.Wo) row[2] = to_elem<Tout>(o2);
        if (x + 3 < a.Wo) row[3] = to_elem<Tout>(o3);
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

// Packed FP32 pairs: sm_100 and later issue two FP32 additions, multiplications or fused
// multiply-adds as one instruction, each component rounded exactly as the scalar
// operation. The iteration tile runs its arithmetic on pairs of pixels (or of channels)
// with these, so it computes the same bits as the scalar code with half the FP32
// instructions. A difference a - b is formed as fma(b, -1, a), the same single rounding.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
// lerpf on both components; omt = 1 - t
__device__ __forceinline__ float2 lerp2(float2 p, float2 q, float2 t, float2 omt) { return fma2(t, q, mul2(omt, p)); }
__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return add2(a, b); }

// A sample position x + u is held as the integer x + floor(u) and the fraction
// u - floor(u), which FP32 gives exactly for u >= 0 and within 2^-25 for u < 0: the
// interpolation weights carry the flow's own precision rather than the rounding of the
// sum x + u in FP32 (half an ulp of x + u, about 1.5e-5 px at a few hundred pixels). The integer part wraps around in 32 bits, so that a flow too
// large for an int (floor(u) saturated) never passes a test for a range of the image or
// of a staged window; where the result is clamped instead, floor(u) is first limited
// to +-2^20 (the position is then far outside the image, on the same side).
__device__ __forceinline__ int pos_floor(int x, float fu)
{
    return (int)((unsigned)x + (unsigned)__float2int_rz(fu));
}
__device__ __forceinline__ int pos_floor_clamped(int x, float fu)
{
    return x + max(min(__float2int_rz(fu), 1 << 20), -(1 << 20));
}
// The upper bound of (unsigned)(x0 - 1) for a position whose 4 x 4 tap footprint
// (x0 - 1 .. x0 + 2) lies inside an extent of n pixels.
__device__ __forceinline__ unsigned interior_span(int n) { return n > 3 ? (unsigned)(n - 3) : 0u; }

// Bilinear sample at the position (x0 + ax, y0 + ay), ax, ay in [0, 1) (x0, y0 not
// wrapped), clamped to [0, W-1] x [0, H-1], the right and bottom neighbours clamped.
template <bool NC, typename T>
__device__ __forceinline__ float bil(const T *I, int pitch, int H, int W, int x0, float ax, int y0, float ay)
{
    // a position left of 0 or at or right of W - 1 clamps to the end pixel, fraction 0
    ax = (unsigned)x0 < (unsigned)(W - 1) ? ax : 0.0f;
    ay = (unsigned)y0 < (unsigned)(H - 1) ? ay : 0.0f;
    x0 = min(max(x0, 0), W - 1);
    y0 = min(max(y0, 0), H - 1);
    const int x1 = min(x0 + 1, W - 1), y1 = min(y0 + 1, H - 1);
    const T *r0 = I + (size_t)y0 * pitch, *r1 = I + (size_t)y1 * pitch;
    return lerpf(lerpf(ldf<NC>(r0 + x0), ldf<NC>(r0 + x1), ax), lerpf(ldf<NC>(r1 + x0), ldf<NC>(r1 + x1), ax), ay);
}

// I2 bilinear at (x + u, y + v), the position clamped to the image.
template <bool NC, typename T>
__device__ __forceinline__ float bil_at(const T *I, int pitch, int H, int W, int x, int y, float u, float v)
{
    const float fu = floorf(u), fv = floorf(v);
    return bil<NC>(I, pitch, H, W, pos_floor_clamped(x, fu), u - fu, pos_floor_clamped(y, fv), v - fv);
}

// sample_grad by five clamped bilinear samples. Where no sample is clamped these are the
// interior branch's interpolations in the same order, so the two agree bit for bit.
template <bool NC, typename T>
__device__ __forceinline__ void sample_grad_clamped(const T *I, int pitch, int H, int W, int x, int y, float u,
                                                    float v, float &Iw, float &gx, float &gy)
{
    const float fu = floorf(u), fv = floorf(v);
    const float ax = u - fu, ay = v - fv;
    const int bx = pos_floor_clamped(x, fu), by = pos_floor_clamped(y, fv);
    Iw = bil<NC>(I, pitch, H, W, bx, ax, by, ay);
    gx = (bil<NC>(I, pitch, H, W, bx + 1, ax, by, ay) - bil<NC>(I, pitch, H, W, bx - 1, ax, by, ay)) * 0.5f;
    gy = (bil<NC>(I, pitch, H, W, bx, ax, by + 1, ay) - bil<NC>(I, pitch, H, W, bx, ax, by - 1, ay)) * 0.5f;
}

// I2 at p = (x + u, y + v) and its gradient at p: central difference of the bilinear
// samples at p +- (1, 0) and p +- (0, 1). Away from the border the 12 distinct taps of
// the 4x4 neighbourhood are read once; near it each sample is clamped on its own.
template <bool NC, typename T>
__device__ __forceinline__ void sample_grad(const T *I, int pitch, int H, int W, int x, int y, float u, float v,
                                            float &Iw, float &gx, float &gy)
{
    const float fu = floorf(u), fv = floorf(v);
    const float ax = u - fu, ay = v - fv;
    const int x0 = pos_floor(x, fu), y0 = pos_floor(y, fv);
    if ((unsigned)x0 - 1u < interior_span(W) && (unsigned)y0 - 1u < interior_span(H)) {
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
        sample_grad_clamped<NC>(I, pitch, H, W, x, y, u, v, Iw, gx, gy);
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
            sample_grad<NC>(I2, a.pitch, a.H, a.W, x, y, f.x, f.y, Iw, gx, gy);
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
template <int R, int TH = LK_TH, int TW = LK_TW> struct FixedTile {
    static_assert(R >= 2, "the grouped box sums need 2R >= 4");
    static constexpr int W = 2 * R + 1;                // window width
    static constexpr int NV4 = (2 * R + 4 + 3) / 4;    // float4 loads for 4 outputs' windows
    static constexpr int RH = TH + 2 * R;              // region rows (tile + halo)
    static constexpr int RW = TW + 2 * R;              // region columns
    static constexpr int RWP = TW + 4 * NV4 - 4;       // padded row length (>= RW, multiple of 4)
    static constexpr int PLANE = RH * RWP;
    static constexpr int NREG = RH * RW;               // region pixels
    static constexpr int PER = (NREG + LK_THREADS - 1) / LK_THREADS;   // region pixels per thread
    // Staging (a.stage_i2): one TMA box of I2, the window of the tile's region shifted by
    // the rounded estimate at the tile's centre and widened by STAGE_MARGIN pixels plus the 4x4
    // tap footprint (and, for the alignment of its first column, E - 1 columns), in the
    // storage type: WIN_W(S) x WIN_H elements of S bytes, rows WIN_W(S) elements apart.
    // A pixel whose taps leave it reads them from global memory instead.
    static constexpr int STAGE_MARGIN = 6;
    static constexpr int WIN_H = TH + 2 * R + 2 * STAGE_MARGIN + 4;
    static constexpr int win_w(int S)
    {
        return (TW + 2 * ((R + 1) / 2 * 2) + 2 * STAGE_MARGIN + 4 + 16 / S - 1 + 16 / S - 1) / (16 / S) * (16 / S);
    }
    static constexpr int win_bytes(int S) { return win_w(S) * WIN_H * S; }
    // Product planes of the iteration tile. Stage 1 computes pixel pairs (x, x+1) with x
    // even in image coordinates, so the region starts RE = R rounded up to even pixels
    // left of the tile and is RWE columns wide; a window's first column is then OFF =
    // RE - R columns into the region. Channels 0 and 1 share one plane of float2 (P01),
    // channels 2 and 3 another (P23), channel 4 has a plane of floats (P4), so that the
    // box sums add two channels per instruction. Row lengths: RWP1 floats for P4 (a
    // multiple of 4), RWP2 float2 for the pair planes (2 mod 4, so that the float4 reads
    // of a quarter warp of the horizontal pass fall in distinct banks).
    static constexpr int RE = (R + 1) / 2 * 2;
    static constexpr int OFF = RE - R;
    static constexpr int RWE = TW + 2 * RE;
    static constexpr int NVE = (OFF + 2 * R + 4 + 3) / 4;   // float4 column groups read per 4 outputs
    static_assert(TW % 4 == 0 && TW / 4 <= 32, "4-output groups, a row's groups in one warp");
    static_assert(TW - 4 + 4 * NVE <= RWE, "the horizontal pass reads computed columns only");
    static constexpr int RWP1 = RWE;
    static constexpr int RWP2 = RWE + 2;
    static_assert(RWP1 % 4 == 0 && RWP2 % 4 == 2, "row lengths");
    static constexpr int PAIR_PLANE = RH * RWP2;             // float2 per pair plane
    static constexpr int PLANES = 4 * PAIR_PLANE + RH * RWP1;  // floats of the three planes
    static_assert(PLANES % 4 == 0, "the barrier after the planes must be 8-byte aligned");
    static constexpr int OFF_BAR = PLANES;                    // 8-byte mbarrier
    static constexpr int OFF_WREF = OFF_BAR + 2;              // a strip's tile-centre estimates (4 float2)
    static constexpr int OFF_WIN = (OFF_WREF + 8 + 31) / 32 * 32;   // 128-byte aligned staging window
    static constexpr int SMEM_NOSTAGE = OFF_WIN;              // launches without staging
    static constexpr int smem_staged(int S) { return OFF_WIN + (win_bytes(S) + 15) / 16 * 4; }
    static constexpr int SMEM_FLOATS = smem_staged(4);        // the largest (FP32 storage)
    // The staged flow estimate: TMA boxes of RWP2 x FLOW_BH 8-byte elements written over
    // P01. Where row 2R (the first below the 2R rows a tile of a strip takes over from the
    // tile above) starts on a 128-byte boundary (R a multiple of 4), boxes of 2R rows when
    // they tile TH, so that every row of a region is staged (RH / 2R boxes for a strip's
    // first tile, TH / 2R for the others), else one box of TH rows at row 2R; elsewhere one
    // box of TH rows at row 0 for a strip's first tile, the other rows' estimates read from
    // global memory.
    static constexpr bool FLOW_BOX_BELOW = (2 * R * RWP2 * 8) % 128 == 0;
    static constexpr int FLOW_BH = FLOW_BOX_BELOW && TH % (2 * R) == 0 ? 2 * R : TH;
    static constexpr int FLOW_BOX_BYTES = RWP2 * FLOW_BH * 8;
#ifndef OF_LK_MIN_BLOCKS
#define OF_LK_MIN_BLOCKS 4   // resident blocks per SM the fixed-radius kernels are compiled for (R <= 6)
#endif
    // resident blocks per SM the kernels are compiled for: the measured choice for the
    // default tile height, else as many as the shared memory holds (at most 5)
    static constexpr int SMEM_FIT = 233472 / (4 * (PLANES + 4) + 1024);
    static constexpr int MIN_BLOCKS =
        TH == LK_TH ? (R <= 6 ? OF_LK_MIN_BLOCKS : 2) : (SMEM_FIT < 1 ? 1 : (SMEM_FIT > 5 ? 5 : SMEM_FIT));
};

// Staged tile, while its boxes land: 0 no prefetch, 1 warm L2 with the region's I1 rows,
// 2 bring the region's I1 lines (and, upsampling, the coarser estimate's) into L1. With 4
// resident blocks per SM their lines (4.6 KB per 64 x 24 tile of 16-bit data) fit in what
// the shared-memory carve-out leaves of L1; 2 measured 1.9% faster per batch step than 0.
#ifndef OF_PREFETCH_I1
#define OF_PREFETCH_I1 2
#endif
// Strips: request a later tile's window of I2 while the tile above finishes (1), or at
// the tile's own staging (0).
#ifndef OF_EARLY_WINDOW
#define OF_EARLY_WINDOW 1
#endif
constexpr long long STAGE_TIMEOUT_NS = 200000000LL;   // 0.2 s for one tile's staging copies

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

// --------------------------------------------------- pixel-pair and channel-pair passes
// Two horizontally adjacent pixels (x even) of a level image, as floats (exact for every
// storage type; the second is 0 when q is false, and then only the first is read).
template <bool NC> __device__ __forceinline__ float2 ld_pair(const uint8_t *p, bool q)
{
    if (!q) return f2(ldf<NC>(p), 0.0f);
    const uchar2 w = ld<NC>(reinterpret_cast<const uchar2 *>(p));
    return f2((float)w.x, (float)w.y);
}
template <bool NC> __device__ __forceinline__ float2 ld_pair(const uint16_t *p, bool q)
{
    if (!q) return f2(ldf<NC>(p), 0.0f);
    const ushort2 w = ld<NC>(reinterpret_cast<const ushort2 *>(p));
    return f2((float)w.x, (float)w.y);
}
template <bool NC> __device__ __forceinline__ float2 ld_pair(const float *p, bool q)
{
    if (!q) return f2(ldf<NC>(p), 0.0f);
    return ld<NC>(reinterpret_cast<const float2 *>(p));
}
template <bool NC> __device__ __forceinline__ float2 ld_pair(const __half *p, bool q)
{
    if (!q) return f2(ldf<NC>(p), 0.0f);
    const __half2 w = ld<NC>(reinterpret_cast<const __half2 *>(p));
    return __half22float2(w);
}
template <bool NC> __device__ __forceinline__ float2 ld_pair(const __nv_bfloat16 *p, bool q)
{
    if (!q) return f2(ldf<NC>(p), 0.0f);
    const __nv_bfloat162 w = ld<NC>(reinterpret_cast<const __nv_bfloat162 *>(p));
    return __bfloat1622float2(w);
}

// The current estimates of the pixel pair (x, y), (x + 1, y) (x even; the second only
// when q): one 16-byte load of the same-level flow, else pixel by pixel.
template <bool NC, int MODE>
__device__ __forceinline__ void flow_pair(const IterArgs &a, int x, int y, bool q, float2 &fp, float2 &fq)
{
    if (MODE == FLOW_SAME || (MODE < 0 && a.mode == FLOW_SAME)) {
        if (q) {
            const float4 w = ld<NC>(reinterpret_cast<const float4 *>(a.fin + (y * a.fin_pitch + x)));
            fp = f2(w.x, w.y);
            fq = f2(w.z, w.w);
            return;
        }
    }
    if (MODE == FLOW_UPSAMPLE || (MODE < 0 && a.mode == FLOW_UPSAMPLE)) {
        // flow_at_m's upsampling for x (weight 0) and x + 1 (weight 1/2), which share
        // their four coarse samples (x even), computed on both at once
        const int x0 = x >> 1, y0 = y >> 1;
        const int x1 = min(x0 + 1, a.Wc - 1), y1 = min(y0 + 1, a.Hc - 1);
        const float ay = (y & 1) ? 0.5f : 0.0f;
        const float2 *r0 = a.fin + y0 * a.fin_pitch, *r1 = a.fin + y1 * a.fin_pitch;
        const float2 f00 = ld<NC>(r0 + x0), f01 = ld<NC>(r0 + x1);
        const float2 f10 = ld<NC>(r1 + x0), f11 = ld<NC>(r1 + x1);
        const float2 T = f2(0.0f, 0.5f), OT = f2(1.0f, 0.5f), AY = f2(ay, ay), OY = f2(1.0f - ay, 1.0f - ay);
        const float2 two = f2(2.0f, 2.0f);
        const float2 ux = mul2(two, lerp2(lerp2(f2(f00.x, f00.x), f2(f01.x, f01.x), T, OT),
                                          lerp2(f2(f10.x, f10.x), f2(f11.x, f11.x), T, OT), AY, OY));
        const float2 uy = mul2(two, lerp2(lerp2(f2(f00.y, f00.y), f2(f01.y, f01.y), T, OT),
                                          lerp2(f2(f10.y, f10.y), f2(f11.y, f11.y), T, OT), AY, OY));
        fp = f2(ux.x, uy.x);
        fq = q ? f2(ux.y, uy.y) : f2(0.0f, 0.0f);
        return;
    }
    fp = flow_mode<NC, MODE>(a, x, y);
    fq = q ? flow_mode<NC, MODE>(a, x + 1, y) : f2(0.0f, 0.0f);
}

// The 4 x 4 tap footprint of the position with integer part (x0, y0) lies inside the image.
__device__ __forceinline__ bool interior(int x0, int y0, unsigned wspan, unsigned hspan)
{
    return (unsigned)x0 - 1u < wspan && (unsigned)y0 - 1u < hspan;
}

// The interior branch of sample_grad for two sample positions at once (integer parts
// (xp, yp) and (xq, yq), fractions AX, AY), with every operation of the scalar form on
// both components. The 12 taps of each come from the staged window (win: WW x WH
// elements, first element at image (wx0, wy0)) when `inwin`, else from global memory.
template <bool NC, int WW, typename T>
__device__ __forceinline__ void sample_grad2(const T *I, int pitch, const T *win, bool inwin, int cpx, int cpy,
                                             int cqx, int cqy, int xp, int yp, int xq, int yq, float2 AX, float2 AY,
                                             float2 &IW, float2 &GX, float2 &GY)
{
    const float2 one = f2(1.0f, 1.0f);
    const float2 OX = sub2(one, AX), OY = sub2(one, AY);
    float2 A0, A1, BM, B0, B1, B2, CM, C0, C1, C2, D0, D1;
    if (inwin) {
        // (cpx, cpy), (cqx, cqy): the taps' top-left corner (x0 - 1, y0 - 1) in the window;
        // rows WW elements apart: every tap at a constant offset from it
        const T *p = win + (cpy * WW + cpx + 1), *q = win + (cqy * WW + cqx + 1);
        A0 = f2(ldf<false>(p), ldf<false>(q));
        A1 = f2(ldf<false>(p + 1), ldf<false>(q + 1));
        BM = f2(ldf<false>(p + WW - 1), ldf<false>(q + WW - 1));
        B0 = f2(ldf<false>(p + WW), ldf<false>(q + WW));
        B1 = f2(ldf<false>(p + WW + 1), ldf<false>(q + WW + 1));
        B2 = f2(ldf<false>(p + WW + 2), ldf<false>(q + WW + 2));
        CM = f2(ldf<false>(p + 2 * WW - 1), ldf<false>(q + 2 * WW - 1));
        C0 = f2(ldf<false>(p + 2 * WW), ldf<false>(q + 2 * WW));
        C1 = f2(ldf<false>(p + 2 * WW + 1), ldf<false>(q + 2 * WW + 1));
        C2 = f2(ldf<false>(p + 2 * WW + 2), ldf<false>(q + 2 * WW + 2));
        D0 = f2(ldf<false>(p + 3 * WW), ldf<false>(q + 3 * WW));
        D1 = f2(ldf<false>(p + 3 * WW + 1), ldf<false>(q + 3 * WW + 1));
    } else {
        const int op = (yp - 1) * pitch + xp, oq = (yq - 1) * pitch + xq;
        const T *mp = I + op, *mq = I + oq;
        const T *p0 = I + (op + pitch), *q0 = I + (oq + pitch);
        const T *p1 = I + (op + 2 * pitch), *q1 = I + (oq + 2 * pitch);
        const T *p2 = I + (op + 3 * pitch), *q2 = I + (oq + 3 * pitch);
        A0 = f2(ldf<NC>(mp), ldf<NC>(mq));
        A1 = f2(ldf<NC>(mp + 1), ldf<NC>(mq + 1));
        BM = f2(ldf<NC>(p0 - 1), ldf<NC>(q0 - 1));
        B0 = f2(ldf<NC>(p0), ldf<NC>(q0));
        B1 = f2(ldf<NC>(p0 + 1), ldf<NC>(q0 + 1));
        B2 = f2(ldf<NC>(p0 + 2), ldf<NC>(q0 + 2));
        CM = f2(ldf<NC>(p1 - 1), ldf<NC>(q1 - 1));
        C0 = f2(ldf<NC>(p1), ldf<NC>(q1));
        C1 = f2(ldf<NC>(p1 + 1), ldf<NC>(q1 + 1));
        C2 = f2(ldf<NC>(p1 + 2), ldf<NC>(q1 + 2));
        D0 = f2(ldf<NC>(p2), ldf<NC>(q2));
        D1 = f2(ldf<NC>(p2 + 1), ldf<NC>(q2 + 1));
    }
    const float2 TOP = lerp2(B0, B1, AX, OX), BOT = lerp2(C0, C1, AX, OX);
    IW = lerp2(TOP, BOT, AY, OY);
    const float2 half = f2(0.5f, 0.5f);
    GX = mul2(sub2(lerp2(lerp2(B1, B2, AX, OX), lerp2(C1, C2, AX, OX), AY, OY),
                   lerp2(lerp2(BM, B0, AX, OX), lerp2(CM, C0, AX, OX), AY, OY)),
              half);
    GY = mul2(sub2(lerp2(BOT, lerp2(D0, D1, AX, OX), AY, OY), lerp2(lerp2(A0, A1, AX, OX), TOP, AY, OY)), half);
}

// o[j] = sum_{k=0}^{2R} v[OFF+j+k], j = 0..3, the additions in box4's order (floats or
// float2 pairs of channels).
template <int R, int OFF, typename V>
__device__ __forceinline__ void box4v(const V *v, V o[4])
{
    V m = v[OFF + 3];
#pragma unroll
    for (int k = 4; k <= 2 * R; ++k) m = vadd(m, v[OFF + k]);
    o[0] = vadd(vadd(vadd(v[OFF], v[OFF + 1]), v[OFF + 2]), m);
    o[1] = vadd(vadd(vadd(v[OFF + 1], v[OFF + 2]), m), v[OFF + 2 * R + 1]);
    o[2] = vadd(vadd(vadd(v[OFF + 2], m), v[OFF + 2 * R + 1]), v[OFF + 2 * R + 2]);
    o[3] = vadd(vadd(vadd(m, v[OFF + 2 * R + 1]), v[OFF + 2 * R + 2]), v[OFF + 2 * R + 3]);
}

// Horizontal pass of one pair plane, in place, over rows r0..RH-1: row ry becomes, at
// columns 0..TW-1, the window sums of its outputs (two channels per float2). Chunk c of
// rows goes to warp (c + woff) mod WARPS. For 64-wide tiles a warp takes
// two rows and a quarter warp 4 groups of 4 outputs of each (with rows RWP2 = 2 mod 4
// float2 long, its 16-byte reads hit distinct banks); other widths take one row per warp,
// one group per lane. Each row is read and rewritten by one warp.
template <int R, int TH, int TW = LK_TW>
__device__ __forceinline__ void box_h_pairs(float2 *P, int r0 = 0, int woff = 0)
{
    using F = FixedTile<R, TH, TW>;
    static_assert(LK_THREADS % 32 == 0, "whole warps");
    constexpr int WARPS = LK_THREADS / 32;
    constexpr int RW4 = F::RWP2 / 2;   // float4 per row
    const int lane = threadIdx.x & 31;
    constexpr bool TWO = TW == 64;
    constexpr int NG = TW / 4;
    const int rsub = TWO ? (lane >> 2) & 1 : 0, g = TWO ? (((lane >> 3) << 2) | (lane & 3)) : lane;
    const int rows = TWO ? (F::RH - r0) / 2 : F::RH - r0;   // warp-sized chunks (r0, RH - r0 even)
#pragma unroll 1
    for (int chunk = ((threadIdx.x >> 5) + WARPS - woff) % WARPS; chunk < rows; chunk += WARPS) {
        const bool act = TWO || g < NG;
        float4 *row = reinterpret_cast<float4 *>(P) + ((r0 + (TWO ? 2 * chunk + rsub : chunk)) * RW4 + 2 * g);
        float2 o[4];
        if (act) {
            float2 v[4 * F::NVE];
#pragma unroll
            for (int q = 0; q < 2 * F::NVE; ++q) {
                const float4 t = row[q];
                v[2 * q] = f2(t.x, t.y);
                v[2 * q + 1] = f2(t.z, t.w);
            }
            box4v<R, F::OFF>(v, o);
        }
        __syncwarp();
        if (act) {
            row[0] = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
            row[1] = make_float4(o[2].x, o[2].y, o[3].x, o[3].y);
        }
    }
}

// Horizontal pass of the float plane P4, in place, over rows r0..RH-1: for 64-wide tiles
// the 16 items of a row in 16 lanes, else one row per warp.
template <int R, int TH, int TW = LK_TW>
__device__ __forceinline__ void box_h_single(float *P, int r0 = 0)
{
    using F = FixedTile<R, TH, TW>;
    constexpr int NG = TW / 4;
    if constexpr (TW == LK_TW && NG == 16) {
        constexpr int IT = (F::RH * NG + LK_THREADS - 1) / LK_THREADS;
        const int nitems = (F::RH - r0) * NG;
        float4 res[IT];
#pragma unroll
        for (int k = 0; k < IT; ++k) {
            const int i = threadIdx.x + k * LK_THREADS;
            if (i < nitems) {
                const int ry = r0 + i / NG, g = i % NG;
                const float4 *src = reinterpret_cast<const float4 *>(P + ry * F::RWP1 + 4 * g);
                float v[4 * F::NVE];
#pragma unroll
                for (int q = 0; q < F::NVE; ++q) {
                    const float4 t = src[q];
                    v[4 * q] = t.x;
                    v[4 * q + 1] = t.y;
                    v[4 * q + 2] = t.z;
                    v[4 * q + 3] = t.w;
                }
                float o[4];
                box4v<R, F::OFF>(v, o);
                res[k] = make_float4(o[0], o[1], o[2], o[3]);
            }
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < IT; ++k) {
            const int i = threadIdx.x + k * LK_THREADS;
            if (i < nitems) {
                const int ry = r0 + i / NG, g = i % NG;
                *reinterpret_cast<float4 *>(P + ry * F::RWP1 + 4 * g) = res[k];
            }
        }
    } else {
        constexpr int WARPS = LK_THREADS / 32;
        const int g = threadIdx.x & 31;
#pragma unroll 1
        for (int ry = r0 + (threadIdx.x >> 5); ry < F::RH; ry += WARPS) {
            float4 *row = reinterpret_cast<float4 *>(P + ry * F::RWP1 + 4 * g);
            float o[4];
            if (g < NG) {
                float v[4 * F::NVE];
#pragma unroll
                for (int q = 0; q < F::NVE; ++q) {
                    const float4 t = row[q];
                    v[4 * q] = t.x;
                    v[4 * q + 1] = t.y;
                    v[4 * q + 2] = t.z;
                    v[4 * q + 3] = t.w;
                }
                box4v<R, F::OFF>(v, o);
            }
            __syncwarp();
            if (g < NG) row[0] = make_float4(o[0], o[1], o[2], o[3]);
        }
    }
}

// o[j] = sum_{k=0}^{2R} v[j+k], j = 0..5, from v[0 .. 2R+5] (R >= 3): the rows 5..2R that
// all six windows share summed once, the others as partial sums from either end.
template <int R, typename V>
__device__ __forceinline__ void box6v(const V *v, V o[6])
{
    static_assert(R >= 3, "six windows with a shared middle");
    V m = v[5];
#pragma unroll
    for (int k = 6; k <= 2 * R; ++k) m = vadd(m, v[k]);
    V lf[5], rt[6];
    lf[4] = v[4];
#pragma unroll
    for (int j = 3; j >= 0; --j) lf[j] = vadd(v[j], lf[j + 1]);
    rt[1] = v[2 * R + 1];
#pragma unroll
    for (int j = 2; j <= 5; ++j) rt[j] = vadd(rt[j - 1], v[2 * R + j]);
    o[0] = vadd(lf[0], m);
#pragma unroll
    for (int j = 1; j <= 4; ++j) o[j] = vadd(vadd(lf[j], m), rt[j]);
    o[5] = vadd(m, rt[5]);
}

// Output rows per item of the vertical pass: 6 where they tile the tile height (for TH =
// 24 one item per thread of a 256-thread block), else 4.
template <int R, int TH> constexpr int v_rows() { return (TH % 6 == 0 && R >= 3) ? 6 : 4; }

// Vertical pass for the VR = v_rows outputs of item g (rows VR g .. VR g + VR - 1, column
// tx): sums of the three planes.
template <int R, int TH, int TW = LK_TW>
__device__ __forceinline__ void box_v_planes(const float2 *P01, const float2 *P23, const float *P4, int g, int tx,
                                             float2 s01[v_rows<R, TH>()], float2 s23[v_rows<R, TH>()],
                                             float s4[v_rows<R, TH>()])
{
    using F = FixedTile<R, TH, TW>;
    constexpr int VR = v_rows<R, TH>(), NV = 2 * R + VR;
    {
        float2 v[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = P01[(VR * g + q) * F::RWP2 + tx];
        if constexpr (VR == 6) box6v<R>(v, s01);
        else box4v<R, 0>(v, s01);
    }
    {
        float2 v[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = P23[(VR * g + q) * F::RWP2 + tx];
        if constexpr (VR == 6) box6v<R>(v, s23);
        else box4v<R, 0>(v, s23);
    }
    {
        float v[NV];
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q] = P4[(VR * g + q) * F::RWP1 + tx];
        if constexpr (VR == 6) box6v<R>(v, s4);
        else box4v<R, 0>(v, s4);
    }
}

// Stage 1 of the fixed-radius tile for the pixel pair (x, y), (x + 1, y): warp I2 by the
// current estimate, its gradient there, e~ and the five products, on both pixels at
// once when both sample the interior (taps from the staged window or global memory),
// pixel by pixel near the border or at the image's last column. sflow: the pair's staged
// estimates (NULL: read them from fin). Out-of-image pixels get zero products. Returns the
// products in the planes' layout.
template <typename T, bool NC, int MODE, int WW>
__device__ __forceinline__ void stage1_pair(const IterArgs &a, int x, int y, float2 ref, const float4 *sflow,
                                            const T *win, bool win_in_image, int wx0, int wy0, int WH, float4 &s01,
                                            float4 &s23, float2 &s4)
{
    s01 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    s23 = s01;
    s4 = f2(0.0f, 0.0f);
    const bool rowin = (unsigned)y < (unsigned)a.H;
    const bool inp = rowin && (unsigned)x < (unsigned)a.W;
    const bool inq = rowin && (unsigned)(x + 1) < (unsigned)a.W;   // implies inp (x even)
    if (!inp) return;
    const T *I1 = static_cast<const T *>(a.I1);
    const T *I2 = static_cast<const T *>(a.I2);
    float2 fp, fq;
    if (sflow) {
        const float4 w = *sflow;   // zeros beyond the image
        fp = f2(w.x, w.y);
        fq = f2(w.z, w.w);
    } else {
        flow_pair<NC, MODE>(a, x, y, inq, fp, fq);
    }
    const float2 i1 = ld_pair<NC>(I1 + (y * a.pitch + x), inq);
    float2 IW, GX, GY;
    // The positions' integer parts and fractions (exact; pos_floor). Both pixels sample
    // the interior (their 4x4 footprints inside the image) and, with a staged window, the
    // footprints' corners (x0 - 1, y0 - 1) inside it. When the whole window lies inside
    // the image, a footprint inside the window is inside the image, which is the interior
    // condition, so only the window is tested.
    const float2 FU = f2(floorf(fp.x), floorf(fq.x)), FV = f2(floorf(fp.y), floorf(fq.y));
    const float2 AX = sub2(f2(fp.x, fq.x), FU), AY = sub2(f2(fp.y, fq.y), FV);
    const int xp = pos_floor(x, FU.x), yp = pos_floor(y, FV.x);
    const int xq = pos_floor(x + 1, FU.y), yq = pos_floor(y, FV.y);
    const int cpx = (int)((unsigned)xp - 1u - (unsigned)wx0), cpy = (int)((unsigned)yp - 1u - (unsigned)wy0);
    const int cqx = (int)((unsigned)xq - 1u - (unsigned)wx0), cqy = (int)((unsigned)yq - 1u - (unsigned)wy0);
    const bool inwin = win && (unsigned)cpx < (unsigned)(WW - 3) && (unsigned)cqx < (unsigned)(WW - 3) &&
                       (unsigned)cpy < (unsigned)(WH - 3) && (unsigned)cqy < (unsigned)(WH - 3);
    const unsigned ws = interior_span(a.W), hs = interior_span(a.H);
    if (inq && (win_in_image ? inwin : (interior(xp, yp, ws, hs) && interior(xq, yq, ws, hs)))) {
        sample_grad2<NC, WW>(I2, a.pitch, win, inwin, cpx, cpy, cqx, cqy, xp, yp, xq, yq, AX, AY, IW, GX, GY);
    } else {
        float iw0, gx0, gy0, iw1 = 0.0f, gx1 = 0.0f, gy1 = 0.0f;
        sample_grad_clamped<NC>(I2, a.pitch, a.H, a.W, x, y, fp.x, fp.y, iw0, gx0, gy0);
        if (inq) sample_grad_clamped<NC>(I2, a.pitch, a.H, a.W, x + 1, y, fq.x, fq.y, iw1, gx1, gy1);
        IW = f2(iw0, iw1);
        GX = f2(gx0, gx1);
        GY = f2(gy0, gy1);
    }
    const float2 DX = sub2(f2(fp.x, fq.x), f2(ref.x, ref.x)), DY = sub2(f2(fp.y, fq.y), f2(ref.y, ref.y));
    const float2 E = fma2(GY, DY, fma2(GX, DX, sub2(i1, IW)));
    const float2 q0 = mul2(GX, GX), q1 = mul2(GX, GY), q2 = mul2(GY, GY), q3 = mul2(GX, E), q4 = mul2(GY, E);
    if (inq) {
        s01 = make_float4(q0.x, q1.x, q0.y, q1.y);
        s23 = make_float4(q2.x, q3.x, q2.y, q3.y);
        s4 = q4;
    } else {
        s01 = make_float4(q0.x, q1.x, 0.0f, 0.0f);
        s23 = make_float4(q2.x, q3.x, 0.0f, 0.0f);
        s4 = f2(q4.x, 0.0f);
    }
}

// The estimate that places the staged window of the 64 x TH tile at (tx0, ty0): the one at
// the tile's centre.
template <bool NC, int MODE, int TH>
__device__ __forceinline__ float2 win_ref(const IterArgs &a, int tx0, int ty0)
{
    return flow_mode<NC, MODE>(a, min(tx0 + LK_TW / 2, a.W - 1), min(ty0 + TH / 2, a.H - 1));
}

// First element (wx0, wy0) of the staged window of the tile at (tx0, ty0) for the estimate
// w at its centre: the tile's region displaced by w rounded, widened by the margin and the
// tap footprint, wx0 rounded down to a multiple of 16 bytes.
template <int R, int TH, int S>
__device__ __forceinline__ void win_origin(const IterArgs &a, int tx0, int ty0, float2 w, int &wx0, int &wy0)
{
    using F = FixedTile<R, TH>;
    constexpr int E = 16 / S;
    const int ox = __float2int_rn(fminf(fmaxf(w.x, -(float)a.W), (float)a.W));
    const int oy = __float2int_rn(fminf(fmaxf(w.y, -(float)a.H), (float)a.H));
    const int wx = tx0 - F::RE + ox - F::STAGE_MARGIN - 2;
    wx0 = (wx >= 0 ? wx / E : -((-wx + E - 1) / E)) * E;
    wy0 = ty0 - R + oy - F::STAGE_MARGIN - 2;
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

// One tile of a work unit (lk_tile_fixed). A tile after the first of its strip takes over
// region rows 0..2R-1 from the tile above; CM = 0: a first tile, 1: a later one, 2: as
// `carry_rt` says at run time (one body for both, the loop of a strip). At CM 2 with
// staging, wrefs[0] is this tile's window estimate (win_ref) and wrefs[1] the next one's
// when `next` (a tile of the same strip follows): that tile's window is then requested as
// soon as this tile's stage 1 is done, and a later tile of a strip requests only its flow
// boxes. Returns false if a staging copy did not complete in time.
template <typename T, bool NC, int R, int MODE, int TH, int CM>
__device__ __forceinline__ bool lk_tile_step(const IterArgs &a, const StageMaps *maps, int tx0, int ty0, float2 ref,
                                             float fp64_cond, float *smem, uint32_t &phase, bool carry_rt,
                                             const float2 *wrefs = nullptr, bool next = false)
{
    const bool CARRY = CM == 2 ? carry_rt : CM == 1;
    using F = FixedTile<R, TH>;
    unsigned char *win = reinterpret_cast<unsigned char *>(smem + F::OFF_WIN);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + F::OFF_BAR);
    constexpr int S = (int)sizeof(T);
    constexpr int WW = F::win_w(S);
    constexpr bool SAME = MODE == FLOW_SAME;
    float2 *P01 = reinterpret_cast<float2 *>(smem);
    float2 *P23 = P01 + F::PAIR_PLANE;
    float *P4 = reinterpret_cast<float *>(P23 + F::PAIR_PLANE);
    const bool staged = maps && a.stage_i2 != 0;
    const int r0 = CARRY ? 2 * R : 0;   // the first region row this tile computes
    __syncthreads();   // the previous tile's readers of smem are done
    if (CARRY) {
        // region rows TH .. TH+2R-1 of the tile above are rows 0 .. 2R-1 of this one:
        // their window sums along x (columns 0..TW-1 of each plane) move up
        constexpr int Q2 = LK_TW / 2, Q1 = LK_TW / 4;   // float4 per row: pair planes, P4
        constexpr int N = 2 * R * (2 * Q2 + Q1);
        for (int i = threadIdx.x; i < N; i += LK_THREADS) {
            const int row = i / (2 * Q2 + Q1), c = i - row * (2 * Q2 + Q1);
            float4 *dst, *src;
            if (c < 2 * Q2) {
                float2 *P = c < Q2 ? P01 : P23;
                const int q = c < Q2 ? c : c - Q2;
                dst = reinterpret_cast<float4 *>(P + row * F::RWP2) + q;
                src = reinterpret_cast<float4 *>(P + (row + TH) * F::RWP2) + q;
            } else {
                dst = reinterpret_cast<float4 *>(P4 + row * F::RWP1) + (c - 2 * Q2);
                src = reinterpret_cast<float4 *>(P4 + (row + TH) * F::RWP1) + (c - 2 * Q2);
            }
            *dst = *src;
        }
        __syncthreads();
    }
    // Staging (a.stage_i2): one TMA box of I2, the tile's window displaced by the
    // rounded estimate at the tile's centre, and at FLOW_SAME the boxes of the current
    // estimate over the rows this tile computes (FixedTile::FLOW_BH), written over plane
    // P01: stage 1 reads each pair's estimate there before storing the pair's products
    // in the same place (the estimates of rows no box covers are read from global memory).
    const bool box = SAME && staged && (!CARRY || F::FLOW_BOX_BELOW);
    constexpr bool ALL = F::FLOW_BH == 2 * R;   // boxes cover a first tile's whole region
    const int bx0 = CARRY ? 2 * R : 0;          // first row of the boxes; rows below brow_end read them
    const int nbox = !box ? 0 : (CARRY ? TH / F::FLOW_BH : (ALL ? F::RH / F::FLOW_BH : 1));
    const int brow_end = box ? ((CARRY || ALL) ? F::RH : TH) : 0;
    int wx0 = 0, wy0 = 0;
    if (staged) {
        // a later tile of a strip: its window was requested by the tile above
        const bool early = OF_EARLY_WINDOW && CM == 2 && CARRY;
        win_origin<R, TH, S>(a, tx0, ty0, CM == 2 ? wrefs[0] : win_ref<NC, MODE, TH>(a, tx0, ty0), wx0, wy0);
        if (threadIdx.x == 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, (uint32_t)((early ? 0 : F::win_bytes(S)) + nbox * F::FLOW_BOX_BYTES));
            for (int b = 0; b < nbox; ++b)
                tma_load_2d(P01 + (bx0 + b * F::FLOW_BH) * F::RWP2, &maps->flow, tx0 - F::RE,
                            ty0 - R + bx0 + b * F::FLOW_BH, bar);
            if (!early) tma_load_2d(win, &maps->i2, wx0, wy0, bar);
        }
#if OF_PREFETCH_I1 == 1
        // while the boxes land: warm L2 with the region's rows of I1 (read by stage 1)
        if (threadIdx.x >= 32 && threadIdx.x < 32 + F::RH - r0)
            prefetch_row(a.I1, a.pitch, S, a.H, a.W, ty0 - R + r0, ty0 - R + F::RH, tx0 - F::RE,
                         tx0 - F::RE + F::RWE, threadIdx.x - 32);
#elif OF_PREFETCH_I1 == 2
        // while the boxes land: bring the lines of I1 that stage 1 reads into L1, and at
        // the first iteration of a level those of the coarser estimate it upsamples
        {
            constexpr int LPR = (F::RWE * S + 127) / 128 + 1;
            constexpr int CRH = F::RH / 2 + 2, CLPR = ((F::RWE / 2 + 2) * 8 + 127) / 128 + 1;
            const int n1 = (F::RH - r0) * LPR;
            const int n = n1 + (MODE == FLOW_UPSAMPLE ? CRH * CLPR : 0);
            for (int i = threadIdx.x; i < n; i += LK_THREADS) {
                if (i < n1)
                    prefetch_lines_l1(a.I1, a.pitch, S, a.H, a.W, ty0 - R + r0, ty0 - R + F::RH, tx0 - F::RE,
                                      tx0 - F::RE + F::RWE, LPR, i);
                else
                    prefetch_lines_l1(a.fin, a.fin_pitch, 8, a.Hc, a.Wc, (ty0 - R) >> 1,
                                      ((ty0 - R) >> 1) + CRH, (tx0 - F::RE) >> 1,
                                      ((tx0 - F::RE) >> 1) + F::RWE / 2 + 2, CLPR, i - n1);
            }
        }
#endif
        bool done = mbar_wait_bounded(bar, phase, STAGE_TIMEOUT_NS);
        if (__syncthreads_or(!done)) {
            // give the copies in flight a further bounded wait before the block leaves
            if (!done) mbar_wait_bounded(bar, phase, STAGE_TIMEOUT_NS);
            if (threadIdx.x == 0 && a.status) atomicExch(a.status, DEV_TIMEOUT);
            return false;
        }
        phase ^= 1u;
    }
    // stage 1: products over region rows r0..RH-1 (the tile and its halo), by pixel pairs
    constexpr int NPR = F::RWE / 2;   // pairs per region row
    const T *wt = staged ? reinterpret_cast<const T *>(win) : nullptr;
    const bool win_in_image = staged && wx0 >= 0 && wy0 >= 0 && wx0 + WW <= a.W && wy0 + F::WIN_H <= a.H;
    auto pair = [&](int ry, int cx) {
        const int k2 = ry * (F::RWP2 / 2) + cx;   // float4 slot of the pair in the pair planes
        float4 s01, s23;
        float2 s4;
        stage1_pair<T, NC, MODE, WW>(a, tx0 - F::RE + 2 * cx, ty0 - R + ry, ref,
                                     ry < brow_end ? reinterpret_cast<const float4 *>(P01) + k2 : nullptr, wt,
                                     win_in_image, wx0, wy0, F::WIN_H, s01, s23, s4);
        reinterpret_cast<float4 *>(P01)[k2] = s01;
        reinterpret_cast<float4 *>(P23)[k2] = s23;
        reinterpret_cast<float2 *>(P4)[ry * (F::RWP1 / 2) + cx] = s4;
    };
    if constexpr (CM == 2) {
        // strips: thread t takes pixel pair cx = t mod NPR of rows r0 + t / NPR, then RPI
        // rows further each round, so that what depends on the pair's column is the same on
        // every row it takes (5% fewer instructions per pixel-iteration at r = 4)
        constexpr int RPI = LK_THREADS / NPR;   // rows per round
        const int cx = threadIdx.x % NPR, rs = threadIdx.x / NPR;
        if (rs < RPI) {
#pragma unroll 1
            for (int ry = r0 + rs; ry < F::RH; ry += RPI) pair(ry, cx);
        }
    } else {
        // single tiles: pair j = threadIdx.x + k LK_THREADS is (row ry, pair cx) of the rows
        // computed, stepped without a division (LK_THREADS = DY rows + DX pairs); it
        // compiles without spills where the form above does not
        constexpr int DY = LK_THREADS / NPR, DX = LK_THREADS % NPR;
        const int npair = (F::RH - r0) * NPR;
        int ry = r0 + threadIdx.x / NPR, cx = threadIdx.x % NPR;
#pragma unroll 1
        for (int j = threadIdx.x; j < npair; j += LK_THREADS) {
            pair(ry, cx);
            ry += DY;
            cx += DX;
            if (cx >= NPR) {
                cx -= NPR;
                ++ry;
            }
        }
    }
    __syncthreads();
    if constexpr (CM == 2 && OF_EARLY_WINDOW) {
        // the window is free: request the next tile's, which lands while this tile
        // finishes (the barrier's next phase completes only on that tile's arrival)
        if (staged && next && threadIdx.x == 0) {
            int nx0, ny0;
            win_origin<R, TH, S>(a, tx0, ty0 + TH, wrefs[1], nx0, ny0);
            fence_proxy_async_smem();
            mbar_expect_tx(bar, (uint32_t)F::win_bytes(S));
            tma_load_2d(win, &maps->i2, nx0, ny0, bar);
        }
    }
    // P23's chunks start at warp 4, so that when the rows leave some warps an extra chunk
    // of P01 and of P4 (24 rows: 12 chunks and 384 items) the other warps take P23's
    box_h_pairs<R, TH>(P01, r0);
    box_h_pairs<R, TH>(P23, r0, LK_THREADS / 64);
    box_h_single<R, TH>(P4, r0);
    __syncthreads();
    // vertical sums, solve and write, VR rows of one column per item
    constexpr int VR = v_rows<R, TH>();
    constexpr int VITEMS = LK_TW * (TH / VR);
#pragma unroll 1
    for (int i = threadIdx.x; i < VITEMS; i += LK_THREADS) {
        const int tx = i % LK_TW, g = i / LK_TW;
        const int x = tx0 + tx;
        if (x >= a.W || ty0 + VR * g >= a.H) continue;
        float2 s01[VR], s23[VR];
        float s4[VR];
        box_v_planes<R, TH>(P01, P23, P4, g, tx, s01, s23, s4);
#pragma unroll
        for (int j = 0; j < VR; ++j) {
            const int y = ty0 + VR * g + j;
            if (y >= a.H) break;
            const float sj[5] = {s01[j].x, s01[j].y, s23[j].x, s23[j].y, s4[j]};
            float xu, xv;
            const float2 f = solve2(sj, fp64_cond, xu, xv) ? make_float2(ref.x + xu, ref.y + xv)
                                                           : flow_mode<NC, MODE>(a, x, y);
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

// One work unit of the fixed-radius iteration: the a.strip (1, 2 or 4) vertically
// consecutive 64 x TH tiles of one column of tiles starting at tile row a.strip * (unit /
// tiles_x), inside one group of REF_GROUP tile rows. All tiles of a group take the same
// reference flow (the estimate at the group's centre column and row), so the products of
// a region row do not depend on which tile computes them: the tiles after the first take
// over the last 2R rows of window sums along x from the tile above instead of computing
// their stage 1 and horizontal pass again, and the fields are the same bit for bit for
// every a.strip. MULTI = false: a kernel whose units are single tiles (a.strip 1). Returns
// false if a staging copy did not complete in time (then OF_ETIMEOUT is in *a.status,
// nothing more of the unit was written, and the block must stop).
template <typename T, bool NC, int R, int MODE, int TH = LK_TH, bool MULTI = true>
__device__ __forceinline__ bool lk_tile_fixed(const IterArgs &a, const StageMaps *maps, int unit, float fp64_cond,
                                              float *smem, uint32_t &phase)
{
    using F = FixedTile<R, TH>;
    static_assert(REF_GROUP % 4 == 0, "strips of 1, 2 or 4 tiles inside a group");
    static_assert(TH >= 2 * R && TH % 2 == 0, "the rows taken over lie below the tile above's own 2R first rows");
    const int K = strip_len(a.strip);
    const int uy = unit / a.tiles_x;
    const int tx0 = (unit - uy * a.tiles_x) * LK_TW;
    const int t_first = uy * K, t_end = min(t_first + K, (a.H + TH - 1) / TH);
    const int gy0 = t_first / REF_GROUP * REF_GROUP * TH;
    const float2 ref = flow_mode<NC, MODE>(a, min(tx0 + LK_TW / 2, a.W - 1), min(gy0 + REF_GROUP * TH / 2, a.H - 1));
    if constexpr (!MULTI) {   // one tile per unit (a.strip 1)
        return lk_tile_step<T, NC, R, MODE, TH, 0>(a, maps, tx0, t_first * TH, ref, fp64_cond, smem, phase, false);
    } else {
        // the window estimates of the strip's tiles (strip_len: at most the 4 slots at
        // OFF_WREF), loaded together before the first tile's staging
        float2 *wrefs = reinterpret_cast<float2 *>(smem + F::OFF_WREF);
        if (maps && a.stage_i2 && (int)threadIdx.x < t_end - t_first)
            wrefs[threadIdx.x] = win_ref<NC, MODE, TH>(a, tx0, (t_first + (int)threadIdx.x) * TH);
#pragma unroll 1
        for (int t = t_first; t < t_end; ++t)
            if (!lk_tile_step<T, NC, R, MODE, TH, 2>(a, maps, tx0, t * TH, ref, fp64_cond, smem, phase, t > t_first,
                                                     wrefs + (t - t_first), t + 1 < t_end))
                return false;
        return true;
    }
}

// ------------------------------------------------ two iterations fused in one tile
// Iterations k+1 and k+2 (same level, FLOW_SAME) of one 64 x TH output tile in one block,
// the iteration fusion depth 2 of the batched launch. Step A computes iteration k+1 on the
// tile's whole region (the RWE x RH pixels the tile's window sums read, rounded up to
// whole 4-row groups) as a tile of that size of its own, from the estimate in global
// memory, and keeps the result in shared memory (buffer FB, laid out like plane P01).
// Step B computes iteration k+2 on the tile from FB. Each step takes its reference
// flow at the tile's centre (step A from the estimate of iteration k, step B from FB's),
// so the fused fields equal the unfused ones up to rounding (the region's pixels belong
// to neighbouring tiles, whose references differ). The taps are gathered from global
// memory; the region's rows are read twice as wide a halo as one iteration needs.
template <int R, int TH> struct Fused2 {
    using B = FixedTile<R, TH>;                        // step B: the tile
    static constexpr int THA = (B::RH + 3) / 4 * 4;    // step A's output rows (B's region rows)
    static constexpr int TWA = B::RWE;                 // step A's output columns (B's region columns)
    using A = FixedTile<R, THA, TWA>;
    static constexpr int FB_FLOATS = 2 * B::PAIR_PLANE;    // B::RH x B::RWP2 float2
    static_assert(B::PLANES <= A::PLANES, "step B reuses step A's planes");
    static constexpr int SMEM_FLOATS = A::PLANES + FB_FLOATS;
};

template <typename T, bool NC, int R, int TH>
__device__ __forceinline__ void lk_tile_fused2(const IterArgs &a, int tile, float fp64_cond, float *smem)
{
    using X = Fused2<R, TH>;
    using A = typename X::A;
    using B = typename X::B;
    float2 *P01 = reinterpret_cast<float2 *>(smem);
    float2 *FB = reinterpret_cast<float2 *>(smem + A::PLANES);
    const int tyi = tile / a.tiles_x;
    const int ty0 = tyi * TH, tx0 = (tile - tyi * a.tiles_x) * LK_TW;
    const int ax0 = tx0 - B::RE, ay0 = ty0 - R;   // step A's output origin: B's region
    const int cxr = min(tx0 + LK_TW / 2, a.W - 1), cyr = min(ty0 + TH / 2, a.H - 1);
    // ---------------- step A: iteration k+1 on B's region, into FB
    {
        const float2 ref = flow_at_m<NC, FLOW_SAME>(a, cxr, cyr);
        float2 *Q01 = P01;
        float2 *Q23 = Q01 + A::PAIR_PLANE;
        float *Q4 = reinterpret_cast<float *>(Q23 + A::PAIR_PLANE);
        constexpr int NPR = A::RWE / 2, NPAIR = A::RH * NPR;
        constexpr int DY = LK_THREADS / NPR, DX = LK_THREADS % NPR;
        int ry = threadIdx.x / NPR, cx = threadIdx.x % NPR;
        __syncthreads();
#pragma unroll 1
        for (int j = threadIdx.x; j < NPAIR; j += LK_THREADS) {
            const int k2 = ry * (A::RWP2 / 2) + cx;
            float4 s01, s23;
            float2 s4;
            stage1_pair<T, NC, FLOW_SAME, 1>(a, ax0 - A::RE + 2 * cx, ay0 - R + ry, ref, nullptr, nullptr, false, 0,
                                             0, 0, s01, s23, s4);
            reinterpret_cast<float4 *>(Q01)[k2] = s01;
            reinterpret_cast<float4 *>(Q23)[k2] = s23;
            reinterpret_cast<float2 *>(Q4)[ry * (A::RWP1 / 2) + cx] = s4;
            ry += DY;
            cx += DX;
            if (cx >= NPR) {
                cx -= NPR;
                ++ry;
            }
        }
        __syncthreads();
        box_h_pairs<R, X::THA, X::TWA>(Q01);
        box_h_pairs<R, X::THA, X::TWA>(Q23);
        box_h_single<R, X::THA, X::TWA>(Q4);
        __syncthreads();
        constexpr int VRA = v_rows<R, X::THA>();
        constexpr int VITEMS = X::TWA * (X::THA / VRA);
#pragma unroll 1
        for (int i = threadIdx.x; i < VITEMS; i += LK_THREADS) {
            const int tx = i % X::TWA, g = i / X::TWA;
            const int x = ax0 + tx;
            float2 s01[VRA], s23[VRA];
            float s4[VRA];
            box_v_planes<R, X::THA, X::TWA>(Q01, Q23, Q4, g, tx, s01, s23, s4);
#pragma unroll
            for (int jj = 0; jj < VRA; ++jj) {
                const int ryb = VRA * g + jj, y = ay0 + ryb;
                if (ryb >= B::RH) break;
                float2 f = f2(0.0f, 0.0f);   // outside the image: never read by step B
                if ((unsigned)x < (unsigned)a.W && (unsigned)y < (unsigned)a.H) {
                    const float sj[5] = {s01[jj].x, s01[jj].y, s23[jj].x, s23[jj].y, s4[jj]};
                    float xu, xv;
                    f = solve2(sj, fp64_cond, xu, xv) ? make_float2(ref.x + xu, ref.y + xv)
                                                      : flow_at_m<NC, FLOW_SAME>(a, x, y);
                }
                FB[ryb * B::RWP2 + tx] = f;
            }
        }
        __syncthreads();
    }
    // ---------------- step B: iteration k+2 on the tile, from FB
    {
        const float2 ref = FB[(cyr - ay0) * B::RWP2 + (cxr - ax0)];
        float2 *P23 = P01 + B::PAIR_PLANE;
        float *P4 = reinterpret_cast<float *>(P23 + B::PAIR_PLANE);
        constexpr int NPR = B::RWE / 2, NPAIR = B::RH * NPR;
        constexpr int DY = LK_THREADS / NPR, DX = LK_THREADS % NPR;
        int ry = threadIdx.x / NPR, cx = threadIdx.x % NPR;
#pragma unroll 1
        for (int j = threadIdx.x; j < NPAIR; j += LK_THREADS) {
            const int k2 = ry * (B::RWP2 / 2) + cx;
            float4 s01, s23;
            float2 s4;
            stage1_pair<T, NC, FLOW_SAME, 1>(a, tx0 - B::RE + 2 * cx, ty0 - R + ry, ref,
                                             reinterpret_cast<const float4 *>(FB) + k2, nullptr, false, 0, 0, 0, s01,
                                             s23, s4);
            reinterpret_cast<float4 *>(P01)[k2] = s01;
            reinterpret_cast<float4 *>(P23)[k2] = s23;
            reinterpret_cast<float2 *>(P4)[ry * (B::RWP1 / 2) + cx] = s4;
            ry += DY;
            cx += DX;
            if (cx >= NPR) {
                cx -= NPR;
                ++ry;
            }
        }
        __syncthreads();
        box_h_pairs<R, TH>(P01);
        box_h_pairs<R, TH>(P23);
        box_h_single<R, TH>(P4);
        __syncthreads();
        constexpr int VR = v_rows<R, TH>();
        constexpr int VITEMS = LK_TW * (TH / VR);
#pragma unroll 1
        for (int i = threadIdx.x; i < VITEMS; i += LK_THREADS) {
            const int tx = i % LK_TW, g = i / LK_TW;
            const int x = tx0 + tx;
            if (x >= a.W || ty0 + VR * g >= a.H) continue;
            float2 s01[VR], s23[VR];
            float s4[VR];
            box_v_planes<R, TH>(P01, P23, P4, g, tx, s01, s23, s4);
#pragma unroll
            for (int jj = 0; jj < VR; ++jj) {
                const int y = ty0 + VR * g + jj;
                if (y >= a.H) break;
                const float sj[5] = {s01[jj].x, s01[jj].y, s23[jj].x, s23[jj].y, s4[jj]};
                float xu, xv;
                const float2 f = solve2(sj, fp64_cond, xu, xv) ? make_float2(ref.x + xu, ref.y + xv)
                                                               : FB[(y - ay0) * B::RWP2 + (x - ax0)];
                if (a.fout) {
                    a.fout[(size_t)y * a.fout_pitch + x] = f;
                } else {
                    a.u_out[(size_t)y * a.W + x] = f.x;
                    a.v_out[(size_t)y * a.W + x] = f.y;
                }
            }
        }
    }
}

// The iteration tile for radius R (0 = generic, radius r at run time). MODE: the flow
// mode when it is known at compile time (-1: read a.mode at run time). maps: the staging
// tensor maps in parameter space (NULL: gather from global memory). Returns false when
// the block must stop (a staging copy timed out; recorded in *a.status).
template <typename T, bool NC, int R, int MODE = -1, int TH = LK_TH, bool MULTI = true>
__device__ __forceinline__ bool lk_tile(const IterArgs &a, const StageMaps *maps, int tile, int r, float fp64_cond,
                                        float *smem, uint32_t &phase)
{
    if constexpr (R == 0) {
        lk_tile_generic<T, NC>(a, tile, r, fp64_cond, smem);
        return true;
    } else {
        return lk_tile_fixed<T, NC, R, MODE, TH, MULTI>(a, maps, tile, fp64_cond, smem, phase);
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

// Dynamic shared memory of the iteration tile (floats); elem_bytes: the level image's
// element size (the staged window's).
template <int R, int TH = LK_TH>
inline __host__ __device__ int lk_tile_smem_floats(int r, bool stage_i2, int elem_bytes = 4)
{
    if constexpr (R == 0) return lk_smem_floats(r);
    else return stage_i2 ? FixedTile<R, TH>::smem_staged(elem_bytes) : FixedTile<R, TH>::SMEM_NOSTAGE;
}

}  // namespace of
