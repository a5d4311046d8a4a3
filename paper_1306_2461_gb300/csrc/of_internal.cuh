// Internal declarations of libof: storage types, level descriptors, kernel launchers.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/of.h"

namespace of {

// Device status word values (written by kernels, read by of_sync_status).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_BAD_INDEX = 2 };

// ---------------------------------------------------------------- storage types
template <typename T> struct Store;
template <> struct Store<float> {
    static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ float to_f(float x) { return x; }
    static __device__ __forceinline__ float from_f(float x) { return x; }
};
template <> struct Store<__half> {
    static __device__ __forceinline__ float ld(const __half *p) { return __half2float(__ldg(p)); }
    static __device__ __forceinline__ float to_f(__half x) { return __half2float(x); }
    static __device__ __forceinline__ __half from_f(float x) { return __float2half_rn(x); }
};
template <> struct Store<__nv_bfloat16> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    static __device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
    static __device__ __forceinline__ __nv_bfloat16 from_f(float x) { return __float2bfloat16_rn(x); }
};

inline int storage_bytes(int storage) { return storage == OF_F32 ? 4 : 2; }

// Element type of one pyramid level. Level 0 keeps the camera's integer format (exact,
// at most 2 bytes per pixel); the reduced levels use the plan's storage precision.
enum ElemType : int { ET_U8 = 0, ET_U16 = 1, ET_F32 = 2, ET_F16 = 3, ET_BF16 = 4 };
inline int elem_bytes(int et) { return et == ET_U8 ? 1 : (et == ET_F32 ? 4 : 2); }
inline int raw_elem(int in_format) { return in_format == OF_U8 ? ET_U8 : ET_U16; }
inline int storage_elem(int storage) { return storage == OF_F32 ? ET_F32 : (storage == OF_F16 ? ET_F16 : ET_BF16); }
inline int level_elem(const of_plan &p, int level)
{
    return (level == 0 && !(p.flags & OF_FLAG_ZNSSD)) ? raw_elem(p.in_format) : storage_elem(p.storage);
}

template <typename T> __device__ __forceinline__ T to_elem(float x);
template <> __device__ __forceinline__ float to_elem<float>(float x) { return x; }
template <> __device__ __forceinline__ __half to_elem<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 to_elem<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ uint8_t to_elem<uint8_t>(float x) { return (uint8_t)__float2uint_rn(x); }
template <> __device__ __forceinline__ uint16_t to_elem<uint16_t>(float x) { return (uint16_t)__float2uint_rn(x); }

// One image level in HBM: row-major, `pitch` elements per row.
struct Level {
    void *ptr;
    int32_t H, W, pitch;
};

// Flow input modes of one iteration.
enum FlowMode : int {
    FLOW_ZERO = 0,     // coarsest level, first iteration: u = v = 0
    FLOW_SAME = 1,     // previous iterate on this level
    FLOW_UPSAMPLE = 2  // first iteration of a finer level: 2 * bilinear(coarse, x/2, y/2)
};

// Arguments of one Gauss-Newton iteration on one level of one pair.
struct IterArgs {
    const void *I1;          // level image of the first frame (storage type)
    const void *I2;          // level image of the second frame
    int32_t H, W, pitch;     // level size, image pitch (elements)
    const float2 *fin;       // input flow (FLOW_SAME: this level; FLOW_UPSAMPLE: coarse level)
    int32_t fin_pitch;       // float2 elements per row of fin
    int32_t Hc, Wc;          // coarse level size (FLOW_UPSAMPLE)
    int32_t mode;            // FlowMode
    float2 *fout;            // output flow (interleaved), or NULL when writing u/v planes
    int32_t fout_pitch;
    float *u_out, *v_out;    // final planes, pitch W (used when fout == NULL)
    int32_t tiles_x;         // tiles along x (for flattened work lists)
    int32_t tiles;           // work units in this level (tiles, or strips of `strip` tiles)
    int32_t strip;           // fixed-radius tile: tiles per work unit along y (1, 2 or 4; others mean 1)
    int *status;             // the handle's device status word (errors only)
    int32_t stage_i2;        // stage the tile's I2 window (and, at FLOW_SAME, its estimate) in shared
                             // memory with the TMA copies of the launch's StageMaps (fixed-radius tile)
    const float4 *hess;      // first-image-gradient variant: window matrix (Sa, Sb, Sc, 0) of this level
    int32_t hess_pitch;      // float4 elements per row of hess
};

// Tensor maps of the staged iteration tile, passed as kernel parameters (TMA reads them
// from parameter space).
struct StageMaps {
    CUtensorMap flow;        // fin (8-byte elements, W x H) in boxes of rows of the tile's region (FLOW_SAME)
    CUtensorMap i2;          // I2 (storage type, W x H) in boxes of the tile's window
};

// Arguments of the per-level window-matrix pass of the first-image-gradient variant.
struct HessArgs {
    const void *I1;          // level image of the first frame
    int32_t H, W, pitch;
    float4 *hess;            // output: (Sa, Sb, Sc, 0) per pixel
    int32_t hess_pitch;
    int32_t tiles_x, tiles;
};

// Arguments of one pyramid reduction (both images of a pair at once).
struct PyrArgs {
    const void *src[2];      // raw input (first pass) or level l (storage type)
    void *dst0[2];           // level 0 copy of the raw input (first pass; NULL otherwise)
    void *dst[2];            // level l+1 output (NULL when levels == 1 in the first pass)
    int32_t H, W;            // source size
    int32_t src_pitch;       // elements
    int32_t dst0_pitch;
    int32_t Ho, Wo, dst_pitch;
    int32_t first_image;     // 0: both images, 1: only the second (first reused)
    int32_t tiles_x, tiles;  // output tiles of one image
};

// Arguments of the local normalisation (Eq. 2) of both images of a pair.
struct ZnArgs {
    const void *src[2];      // raw camera images (pitch W)
    void *dst[2];            // level 0 of the pyramid slots (storage type)
    int32_t H, W, src_pitch, dst_pitch;
    int32_t first_image;     // 0: both images, 1: only the second
    int32_t tiles_x, tiles;
};
constexpr int ZN_RADIUS = 5;          // Sect. 2.4: a radius of 5 pixels
constexpr int ZN_T = 32;              // output tile
constexpr int ZN_EPS = 1;             // added to the local variance (counts squared)

// One launch of a phase of the batched method over up to PHASE_PAIRS pairs: the pairs'
// arguments travel as a kernel parameter (constant space, warp-uniform), and block b
// works on tile b - prefix[p] of the pair p with prefix[p] <= b < prefix[p + 1].
constexpr int PHASE_PAIRS = 64;
template <typename A> struct Phase {
    int32_t npairs;
    int32_t ahead;                      // iteration phases: warm L2 for tile b + ahead (0: off)
    int32_t prefix[PHASE_PAIRS + 1];
    A a[PHASE_PAIRS];
};
struct IterPhase : Phase<IterArgs> {
    StageMaps m[PHASE_PAIRS];           // pair p's tensor maps when a[p].stage_i2
};
using PyrPhase = Phase<PyrArgs>;
using ZnPhase = Phase<ZnArgs>;
using HessPhase = Phase<HessArgs>;
static_assert(sizeof(IterPhase) <= 32000 && sizeof(PyrPhase) <= 32000, "kernel parameters are limited to 32 KB");

// Tile shapes.
constexpr int LK_TW = 64;    // iteration output tile width
// Iteration output tile: 64 x 24 at 4 blocks of 256 threads per SM (measured on the 1024^2,
// r = 4 batch with staging and strips of 4 tiles: 64 x 24 5.54 ms per step, 64 x 32 at 3
// blocks 6.01, 64 x 16 at 5 blocks (48 registers, spills) 6.95; before strips, 64 x 20 at 4
// blocks 7.11 and, with 512-thread blocks at 2 per SM, 64 x 56 6.75 against 6.66 for 64 x 24).
// At 24 rows the vertical pass's six-row items are one per thread. The height can be set at
// build time (a multiple of 4).
#ifndef OF_LK_TH
#define OF_LK_TH 24
#endif
constexpr int LK_TH = OF_LK_TH;
static_assert(LK_TH % 4 == 0, "the vertical box pass takes 4 rows at a time");
// The other iteration tile height the tuning can choose for the phase launches (64 x ALT_TH).
#ifndef OF_ALT_TH
#define OF_ALT_TH 32
#endif
constexpr int ALT_TH = OF_ALT_TH;
static_assert(ALT_TH % 4 == 0 && ALT_TH != LK_TH, "a multiple of 4 other than LK_TH");
// The fixed-radius iteration tile takes its reference flow per group of REF_GROUP tile
// rows of a column of tiles, and a work unit is a strip of strip_len(strip) consecutive
// tiles of one column inside one group (the tiles after the first take over the window
// sums of the rows they share with the tile above).
constexpr int REF_GROUP = 4;
inline __host__ __device__ int strip_len(int strip) { return strip == 2 || strip == 4 ? strip : 1; }
inline __host__ __device__ int strip_units(int H, int W, int tile_h, int strip)
{
    const int tx = (W + LK_TW - 1) / LK_TW, ty = (H + tile_h - 1) / tile_h, k = strip_len(strip);
    return tx * ((ty + k - 1) / k);
}

// Output tile height of the first-image-gradient variant's kernels (two product planes,
// so a taller tile still leaves room for many blocks per SM).
#ifndef OF_I1_TH
#define OF_I1_TH 32
#endif
constexpr int I1_TH = OF_I1_TH;
static_assert(I1_TH % 4 == 0, "the vertical box pass takes 4 rows at a time");
#ifndef OF_LK_THREADS
#define OF_LK_THREADS 256
#endif
constexpr int LK_THREADS = OF_LK_THREADS;   // threads per iteration / batch block
constexpr int PYR_TW = 64;   // pyramid output tile
constexpr int PYR_TH = 16;
constexpr int PYR_THREADS = 256;
#ifndef OF_MAX_RADIUS
#define OF_MAX_RADIUS 16
#endif
constexpr int MAX_RADIUS = OF_MAX_RADIUS;

// Window radii with a kernel specialised at compile time (the workloads' and the
// paper's radii); any other radius runs the generic kernel.
#define OF_RADII(X) X(2) X(3) X(4) X(5) X(6) X(8) X(10)

inline bool radius_specialised(int r)
{
#define OF_IS_RADIUS(R) if (r == R) return true;
    OF_RADII(OF_IS_RADIUS)
#undef OF_IS_RADIUS
    return false;
}

// ------------------------------------------------------------------- launchers
// All return cudaGetLastError() of their launch.
cudaError_t launch_pyr_first(const PyrArgs &a, int in_format, int storage, cudaStream_t s);
cudaError_t launch_pyr_down(const PyrArgs &a, int storage, cudaStream_t s);
cudaError_t launch_znssd(const ZnArgs &a, int in_format, int storage, cudaStream_t s);
cudaError_t launch_lk_iter(const IterArgs &a, const StageMaps &m, int elem, int radius, float fp64_cond,
                           cudaStream_t s);
cudaError_t launch_window_sums(const float *ch, int H, int W, int r, float *out, cudaStream_t s);
// The variant linearised with the first image's gradient: window matrix of one level,
// then iterations that read it from a.hess.
cudaError_t launch_i1_hess(const HessArgs &a, int elem, int radius, cudaStream_t s);
cudaError_t launch_i1_iter(const IterArgs &a, int elem, int radius, float fp64_cond, cudaStream_t s);
// Phase launches of the batched method (grid = P.prefix[P.npairs] blocks).
cudaError_t launch_phase_pyr(const PyrPhase &P, bool first, int in_format, int storage, cudaStream_t s);
cudaError_t launch_phase_zn(const ZnPhase &P, int in_format, int storage, cudaStream_t s);
cudaError_t launch_phase_iter(const IterPhase &P, int elem, int radius, bool generic, float fp64_cond, int tile_h,
                              cudaStream_t s);
// Two same-level FLOW_SAME iterations in one launch per tile (fixed radii, tile height
// LK_TH, taps gathered); the arguments are those of the second iteration's output and
// the first's input.
cudaError_t launch_phase_iter2(const IterPhase &P, int elem, int radius, float fp64_cond, cudaStream_t s);
// The first-image-gradient variant: window matrices of one level, then its iterations.
cudaError_t launch_phase_hess(const HessPhase &P, int elem, int radius, bool generic, cudaStream_t s);
cudaError_t launch_phase_i1_iter(const IterPhase &P, int elem, int radius, bool generic, float fp64_cond,
                                 cudaStream_t s);
void *batch_kernel_for(int in_format, int storage, int radius);
size_t batch_smem_bytes(int radius, bool stage_i2);
void *batch_kernel_generic(int in_format, int storage);   // the run-time-radius kernel
size_t batch_smem_generic(int radius);
cudaError_t launch_level_to_f32(const Level &l, int elem, float *dst, cudaStream_t s);
cudaError_t launch_wait_timeout(int *flag, int *status, long long timeout_ns, cudaStream_t s);
cudaError_t configure_lk_kernels();   // all kernels with dynamic shared memory, current device
// Fill a.tm_flow and a.tm_i2 for the staged fixed-radius tile of this radius and tile
// height (level image type elem). Returns false (and clears a.stage_i2) when the radius
// has no fixed-radius kernel or the tensor maps cannot be encoded; the tile then
// gathers from global memory.
bool fill_stage_maps(IterArgs &a, StageMaps &m, int elem, int radius, int tile_h);
// Encode a 2-D tiled tensor map: W x H elements of elem_bytes with rows pitch_bytes apart,
// boxes of box_w x box_h, zero fill outside. False if the driver entry point is missing or
// the encoding fails.
bool encode_tile_map(CUtensorMap *m, int elem, const void *base, int W, int H, size_t pitch_bytes, int box_w,
                     int box_h);
// Element type code for an 8-byte flow element in encode_tile_map.
constexpr int ET_FLOW2 = 100;

// Per-radius instantiations (radius_<R>.cu; R = 0 is the generic kernel).
template <int R>
cudaError_t lk_launch(const IterArgs &a, const StageMaps &m, int elem, int r, float fp64_cond, cudaStream_t s);
template <int R> cudaError_t ws_launch(const float *ch, int H, int W, int r, float *out, cudaStream_t s);
template <int R> cudaError_t i1h_launch(const HessArgs &a, int elem, int r, cudaStream_t s);
template <int R> cudaError_t phase_launch(const IterPhase &P, int elem, int r, float fp64_cond, int tile_h, cudaStream_t s);
template <int R> cudaError_t phase_hess_launch(const HessPhase &P, int elem, int r, cudaStream_t s);
template <int R> cudaError_t phase_i1_launch(const IterPhase &P, int elem, int r, float fp64_cond, cudaStream_t s);
template <int R> cudaError_t i1_launch(const IterArgs &a, int elem, int r, float fp64_cond, cudaStream_t s);
template <int R> void *batch_kernel_ptr(int in_format, int storage);
template <int R> cudaError_t radius_configure();
template <int R> size_t radius_smem_bytes(int r, bool stage_i2);
template <int R> bool radius_stage_maps(const IterArgs &a, StageMaps &m, int elem, int tile_h);
template <int R> cudaError_t phase2_launch(const IterPhase &P, int elem, float fp64_cond, cudaStream_t s);

}  // namespace of
