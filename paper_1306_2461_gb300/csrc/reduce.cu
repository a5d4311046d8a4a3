// Reductions over a displacement field for the recirculation-bubble surface of Eq. 3
// (Sect. 3.2): the number of vectors whose streamwise component is at most T_v, and the
// minimum and maximum of a (mean) field, from which T_v = (min + max) / 2.
#include "of_internal.cuh"

namespace of {

constexpr int RED_THREADS = 256;

__global__ void __launch_bounds__(RED_THREADS) count_le_kernel(const float *u, long long n, float Tv,
                                                                unsigned long long *count)
{
    __shared__ unsigned int s[RED_THREADS / 32];
    unsigned int c = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) c += u[i] <= Tv;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned int t = threadIdx.x < RED_THREADS / 32 ? s[threadIdx.x] : 0u;
        t = __reduce_add_sync(0xffffffffu, t);
        if (threadIdx.x == 0 && t) atomicAdd(count, (unsigned long long)t);
    }
}

// Order-preserving map from float to unsigned (NaN excluded by the callers' data).
__device__ __forceinline__ unsigned int f2key(float f)
{
    const unsigned int b = __float_as_uint(f);
    return (b >> 31) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key2f(unsigned int k)
{
    return __uint_as_float((k >> 31) ? (k & 0x7fffffffu) : ~k);
}

__global__ void minmax_init_kernel(unsigned int *mm)
{
    mm[0] = 0xffffffffu;   // min key
    mm[1] = 0u;            // max key
}

__global__ void __launch_bounds__(RED_THREADS) minmax_kernel(const float *f, long long n, unsigned int *mm)
{
    __shared__ unsigned int s_lo[RED_THREADS / 32], s_hi[RED_THREADS / 32];
    unsigned int lo = 0xffffffffu, hi = 0u;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float v = f[i];
        if (v == v) {
            const unsigned int k = f2key(v);
            lo = min(lo, k);
            hi = max(hi, k);
        }
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((threadIdx.x & 31) == 0) {
        s_lo[threadIdx.x >> 5] = lo;
        s_hi[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        unsigned int a = threadIdx.x < RED_THREADS / 32 ? s_lo[threadIdx.x] : 0xffffffffu;
        unsigned int b = threadIdx.x < RED_THREADS / 32 ? s_hi[threadIdx.x] : 0u;
        a = __reduce_min_sync(0xffffffffu, a);
        b = __reduce_max_sync(0xffffffffu, b);
        if (threadIdx.x == 0) {
            atomicMin(&mm[0], a);
            atomicMax(&mm[1], b);
        }
    }
}

__global__ void minmax_decode_kernel(unsigned int *mm)
{
    float *out = reinterpret_cast<float *>(mm);
    const unsigned int a = mm[0], b = mm[1];
    out[0] = a == 0xffffffffu ? __int_as_float(0x7fc00000) : key2f(a);   // NaN if the field had no number
    out[1] = b == 0u ? __int_as_float(0x7fc00000) : key2f(b);
}

static int reduce_grid(long long n)
{
    int sms = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (n + RED_THREADS - 1) / RED_THREADS;
    const long long cap = (long long)sms * 8;
    return (int)(want < cap ? (want < 1 ? 1 : want) : cap);
}

}  // namespace of

using namespace of;

extern "C" int of_sbubble_count(const float *u, int32_t H, int32_t W, float Tv, unsigned long long *count,
                                of_stream_t stream)
{
    if (!u || !count || H < 1 || W < 1 || !(Tv == Tv)) return OF_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const long long n = (long long)H * W;
    if (cudaMemsetAsync(count, 0, sizeof(unsigned long long), st) != cudaSuccess) return OF_ECUDA;
    count_le_kernel<<<reduce_grid(n), RED_THREADS, 0, st>>>(u, n, Tv, count);
    return cudaGetLastError() == cudaSuccess ? OF_OK : OF_ECUDA;
}

extern "C" int of_field_minmax(const float *field, int32_t H, int32_t W, float *minmax, of_stream_t stream)
{
    if (!field || !minmax || H < 1 || W < 1) return OF_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const long long n = (long long)H * W;
    unsigned int *mm = reinterpret_cast<unsigned int *>(minmax);
    minmax_init_kernel<<<1, 1, 0, st>>>(mm);
    minmax_kernel<<<reduce_grid(n), RED_THREADS, 0, st>>>(field, n, mm);
    minmax_decode_kernel<<<1, 1, 0, st>>>(mm);
    return cudaGetLastError() == cudaSuccess ? OF_OK : OF_ECUDA;
}
