// Per-level Gauss-Newton iteration kernel (Sect. 2.4) and the window-sum step on its own.
#include "of_internal.cuh"
#include "of_kernels.cuh"

namespace of {

template <typename T>
__global__ void __launch_bounds__(LK_THREADS) lk_iter_kernel(IterArgs a, int r, float fp64_cond)
{
    extern __shared__ float smem[];
    lk_tile<T, true>(a, blockIdx.x, r, fp64_cond, smem);
}

template <typename T>
static cudaError_t lk_for(const IterArgs &a, int r, float fp64_cond, cudaStream_t s)
{
    const size_t smem = sizeof(float) * lk_smem_floats(r);
    lk_iter_kernel<T><<<a.tiles, LK_THREADS, smem, s>>>(a, r, fp64_cond);
    return cudaGetLastError();
}

cudaError_t launch_lk_iter(const IterArgs &a, int elem, int radius, float fp64_cond, cudaStream_t s)
{
    switch (elem) {
    case ET_U8: return lk_for<uint8_t>(a, radius, fp64_cond, s);
    case ET_U16: return lk_for<uint16_t>(a, radius, fp64_cond, s);
    case ET_F32: return lk_for<float>(a, radius, fp64_cond, s);
    case ET_F16: return lk_for<__half>(a, radius, fp64_cond, s);
    default: return lk_for<__nv_bfloat16>(a, radius, fp64_cond, s);
    }
}

// The box sums of five given planes, through the same two passes as lk_tile.
__global__ void __launch_bounds__(LK_THREADS)
window_sums_kernel(const float *ch, int H, int W, int r, int tiles_x, float *out)
{
    extern __shared__ float smem[];
    const int RH = LK_TH + 2 * r, RW = LK_TW + 2 * r;
    const int plane = RH * RW;
    float *P = smem, *S = smem + 5 * plane;
    const int tile = blockIdx.x;
    const int ty0 = (tile / tiles_x) * LK_TH, tx0 = (tile % tiles_x) * LK_TW;
    const size_t N = (size_t)H * W;
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
}

cudaError_t launch_window_sums(const float *ch, int H, int W, int r, float *out, cudaStream_t s)
{
    const int tiles_x = (W + LK_TW - 1) / LK_TW, tiles_y = (H + LK_TH - 1) / LK_TH;
    const size_t smem = sizeof(float) * lk_smem_floats(r);
    window_sums_kernel<<<tiles_x * tiles_y, LK_THREADS, smem, s>>>(ch, H, W, r, tiles_x, out);
    return cudaGetLastError();
}

// Raise the dynamic shared memory limit of every kernel that takes the iteration tile's
// buffer, on the current device (once per device and process).
cudaError_t configure_lk_kernels()
{
    const int bytes = (int)lk_smem_bytes(MAX_RADIUS);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(lk_iter_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    if ((e = cudaFuncSetAttribute(lk_iter_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    if ((e = cudaFuncSetAttribute(lk_iter_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)))
        return e;
    if ((e = cudaFuncSetAttribute(lk_iter_kernel<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    if ((e = cudaFuncSetAttribute(lk_iter_kernel<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    return cudaFuncSetAttribute(window_sums_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace of
