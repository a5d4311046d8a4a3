// Pyramid construction (Sect. 2.4, Fig. 3: each level is the one below reduced by 4 in
// area). A level is the level below low-passed with the separable binomial
// [1 4 6 4 1]/16 (clamp-to-edge taps) with the even samples kept, so a level of n pixels
// along an axis has ceil(n/2) at the next.
//
// The first pass reads the raw camera counts (uint8/uint16) once, stores level 0 as they
// are (the camera's integers are exact in at most 2 bytes, no more than an FP16 copy),
// and computes level 1 from them in the same kernel, stored at the plan's precision;
// level 0 is never read back to build level 1. Later passes reduce one level each.
// Both images of a pair are processed by one launch (blockIdx.y selects the image).
#include "of_internal.cuh"
#include "of_kernels.cuh"

namespace of {

template <typename Tin, typename Tout, bool FIRST>
__global__ void __launch_bounds__(PYR_THREADS) pyr_kernel(PyrArgs a)
{
    pyr_tile<Tin, Tout, FIRST>(a, blockIdx.x, blockIdx.y + a.first_image);
}

template <typename Tout>
static cudaError_t first_for(const PyrArgs &a, int in_format, cudaStream_t s)
{
    dim3 grid(a.tiles, 2 - a.first_image);
    if (in_format == OF_U8)
        pyr_kernel<uint8_t, Tout, true><<<grid, PYR_THREADS, 0, s>>>(a);
    else
        pyr_kernel<uint16_t, Tout, true><<<grid, PYR_THREADS, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pyr_first(const PyrArgs &a, int in_format, int storage, cudaStream_t s)
{
    switch (storage) {
    case OF_F32: return first_for<float>(a, in_format, s);
    case OF_F16: return first_for<__half>(a, in_format, s);
    default: return first_for<__nv_bfloat16>(a, in_format, s);
    }
}

cudaError_t launch_pyr_down(const PyrArgs &a, int storage, cudaStream_t s)
{
    dim3 grid(a.tiles, 2 - a.first_image);
    switch (storage) {
    case OF_F32: pyr_kernel<float, float, false><<<grid, PYR_THREADS, 0, s>>>(a); break;
    case OF_F16: pyr_kernel<__half, __half, false><<<grid, PYR_THREADS, 0, s>>>(a); break;
    default: pyr_kernel<__nv_bfloat16, __nv_bfloat16, false><<<grid, PYR_THREADS, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256) znssd_kernel(ZnArgs a)
{
    __shared__ float smem[ZN_SMEM_FLOATS];
    znssd_tile<Tin, Tout, true>(a, blockIdx.x, blockIdx.y + a.first_image, smem);
}

template <typename Tout> static cudaError_t zn_for(const ZnArgs &a, int in_format, cudaStream_t s)
{
    dim3 grid(a.tiles, 2 - a.first_image);
    if (in_format == OF_U8) znssd_kernel<uint8_t, Tout><<<grid, 256, 0, s>>>(a);
    else znssd_kernel<uint16_t, Tout><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_znssd(const ZnArgs &a, int in_format, int storage, cudaStream_t s)
{
    switch (storage) {
    case OF_F32: return zn_for<float>(a, in_format, s);
    case OF_F16: return zn_for<__half>(a, in_format, s);
    default: return zn_for<__nv_bfloat16>(a, in_format, s);
    }
}

// ------------------------------------------------------------ phase launches
// One pyramid pass of up to PHASE_PAIRS pairs (both images, or only the second when the
// first is reused); the pairs' arguments are a kernel parameter.
template <typename Tin, typename Tout, bool FIRST>
__global__ void __launch_bounds__(PYR_THREADS) phase_pyr_kernel(const __grid_constant__ PyrPhase P)
{
    const int p = phase_pair(P.prefix, P.npairs, blockIdx.x);
    const PyrArgs &a = P.a[p];
    const int j = blockIdx.x - P.prefix[p];
    const int img = a.first_image + j / a.tiles;
    pyr_tile<Tin, Tout, FIRST>(a, j - (j / a.tiles) * a.tiles, img);
}

template <typename Tout>
static cudaError_t phase_first_for(const PyrPhase &P, int in_format, cudaStream_t s)
{
    if (in_format == OF_U8)
        phase_pyr_kernel<uint8_t, Tout, true><<<P.prefix[P.npairs], PYR_THREADS, 0, s>>>(P);
    else
        phase_pyr_kernel<uint16_t, Tout, true><<<P.prefix[P.npairs], PYR_THREADS, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_phase_pyr(const PyrPhase &P, bool first, int in_format, int storage, cudaStream_t s)
{
    const int blocks = P.prefix[P.npairs];
    if (blocks == 0) return cudaSuccess;
    if (first) {
        switch (storage) {
        case OF_F32: return phase_first_for<float>(P, in_format, s);
        case OF_F16: return phase_first_for<__half>(P, in_format, s);
        default: return phase_first_for<__nv_bfloat16>(P, in_format, s);
        }
    }
    switch (storage) {
    case OF_F32: phase_pyr_kernel<float, float, false><<<blocks, PYR_THREADS, 0, s>>>(P); break;
    case OF_F16: phase_pyr_kernel<__half, __half, false><<<blocks, PYR_THREADS, 0, s>>>(P); break;
    default: phase_pyr_kernel<__nv_bfloat16, __nv_bfloat16, false><<<blocks, PYR_THREADS, 0, s>>>(P); break;
    }
    return cudaGetLastError();
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(256) phase_zn_kernel(const __grid_constant__ ZnPhase P)
{
    __shared__ float smem[ZN_SMEM_FLOATS];
    const int p = phase_pair(P.prefix, P.npairs, blockIdx.x);
    const ZnArgs &a = P.a[p];
    const int j = blockIdx.x - P.prefix[p];
    znssd_tile<Tin, Tout, true>(a, j - (j / a.tiles) * a.tiles, a.first_image + j / a.tiles, smem);
}

template <typename Tout> static cudaError_t phase_zn_for(const ZnPhase &P, int in_format, cudaStream_t s)
{
    if (in_format == OF_U8) phase_zn_kernel<uint8_t, Tout><<<P.prefix[P.npairs], 256, 0, s>>>(P);
    else phase_zn_kernel<uint16_t, Tout><<<P.prefix[P.npairs], 256, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_phase_zn(const ZnPhase &P, int in_format, int storage, cudaStream_t s)
{
    if (P.prefix[P.npairs] == 0) return cudaSuccess;
    switch (storage) {
    case OF_F32: return phase_zn_for<float>(P, in_format, s);
    case OF_F16: return phase_zn_for<__half>(P, in_format, s);
    default: return phase_zn_for<__nv_bfloat16>(P, in_format, s);
    }
}

template <typename T>
__global__ void level_to_f32_kernel(Level l, float *dst)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x < l.W) dst[(size_t)y * l.W + x] = ldf<true>(static_cast<const T *>(l.ptr) + (size_t)y * l.pitch + x);
}

cudaError_t launch_level_to_f32(const Level &l, int elem, float *dst, cudaStream_t s)
{
    dim3 grid((l.W + 255) / 256, l.H);
    switch (elem) {
    case ET_U8: level_to_f32_kernel<uint8_t><<<grid, 256, 0, s>>>(l, dst); break;
    case ET_U16: level_to_f32_kernel<uint16_t><<<grid, 256, 0, s>>>(l, dst); break;
    case ET_F32: level_to_f32_kernel<float><<<grid, 256, 0, s>>>(l, dst); break;
    case ET_F16: level_to_f32_kernel<__half><<<grid, 256, 0, s>>>(l, dst); break;
    default: level_to_f32_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(l, dst); break;
    }
    return cudaGetLastError();
}

}  // namespace of
