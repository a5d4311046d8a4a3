// Dispatch of the iteration, window-sum and batch kernels to their per-radius
// instantiations (radius_<R>.cu): a specialised kernel for the radii listed in
// OF_RADII, the generic one (radius at run time) for any other.
#include <cudaTypedefs.h>

#include <mutex>

#include "of_internal.cuh"

namespace of {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

bool encode_tile_map(CUtensorMap *m, int elem, const void *base, int W, int H, size_t pitch_bytes, int box_w,
                     int box_h)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || !base || W < 1 || H < 1 || box_w < 1 || box_h < 1 || box_w > 256 || box_h > 256) return false;
    CUtensorMapDataType dt;
    switch (elem) {
    case ET_U8: dt = CU_TENSOR_MAP_DATA_TYPE_UINT8; break;
    case ET_U16: dt = CU_TENSOR_MAP_DATA_TYPE_UINT16; break;
    case ET_F32: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
    case ET_F16: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
    case ET_BF16: dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
    case ET_FLOW2: dt = CU_TENSOR_MAP_DATA_TYPE_UINT64; break;
    default: return false;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

#define OF_CASE_SMAP(R) \
    case R: ok = radius_stage_maps<R>(a, m, elem, tile_h); break;
bool fill_stage_maps(IterArgs &a, StageMaps &m, int elem, int radius, int tile_h)
{
    bool ok = false;
    if (a.stage_i2) {
        switch (radius) {
            OF_RADII(OF_CASE_SMAP)
        default: ok = false;
        }
    }
    if (!ok) a.stage_i2 = 0;
    return ok;
}

#define OF_CASE_LK(R) \
    case R: return lk_launch<R>(a, m, elem, radius, fp64_cond, s);
cudaError_t launch_lk_iter(const IterArgs &a, const StageMaps &m, int elem, int radius, float fp64_cond,
                           cudaStream_t s)
{
    switch (radius) {
        OF_RADII(OF_CASE_LK)
    default: return lk_launch<0>(a, m, elem, radius, fp64_cond, s);
    }
}

#define OF_CASE_WS(R) \
    case R: return ws_launch<R>(ch, H, W, r, out, s);
cudaError_t launch_window_sums(const float *ch, int H, int W, int r, float *out, cudaStream_t s)
{
    switch (r) {
        OF_RADII(OF_CASE_WS)
    default: return ws_launch<0>(ch, H, W, r, out, s);
    }
}

#define OF_CASE_I1H(R) \
    case R: return i1h_launch<R>(a, elem, radius, s);
cudaError_t launch_i1_hess(const HessArgs &a, int elem, int radius, cudaStream_t s)
{
    switch (radius) {
        OF_RADII(OF_CASE_I1H)
    default: return i1h_launch<0>(a, elem, radius, s);
    }
}

#define OF_CASE_I1(R) \
    case R: return i1_launch<R>(a, elem, radius, fp64_cond, s);
cudaError_t launch_i1_iter(const IterArgs &a, int elem, int radius, float fp64_cond, cudaStream_t s)
{
    switch (radius) {
        OF_RADII(OF_CASE_I1)
    default: return i1_launch<0>(a, elem, radius, fp64_cond, s);
    }
}

#define OF_CASE_PH(R) \
    case R: return phase_launch<R>(P, elem, radius, fp64_cond, tile_h, s);
cudaError_t launch_phase_iter(const IterPhase &P, int elem, int radius, bool generic, float fp64_cond, int tile_h,
                              cudaStream_t s)
{
    if (generic) return phase_launch<0>(P, elem, radius, fp64_cond, LK_TH, s);
    switch (radius) {
        OF_RADII(OF_CASE_PH)
    default: return phase_launch<0>(P, elem, radius, fp64_cond, LK_TH, s);
    }
}

#define OF_CASE_PH2(R) \
    case R: return phase2_launch<R>(P, elem, fp64_cond, s);
cudaError_t launch_phase_iter2(const IterPhase &P, int elem, int radius, float fp64_cond, cudaStream_t s)
{
    switch (radius) {
        OF_RADII(OF_CASE_PH2)
    default: return cudaErrorInvalidValue;
    }
}

#define OF_CASE_PHH(R) \
    case R: return phase_hess_launch<R>(P, elem, radius, s);
cudaError_t launch_phase_hess(const HessPhase &P, int elem, int radius, bool generic, cudaStream_t s)
{
    if (generic) return phase_hess_launch<0>(P, elem, radius, s);
    switch (radius) {
        OF_RADII(OF_CASE_PHH)
    default: return phase_hess_launch<0>(P, elem, radius, s);
    }
}

#define OF_CASE_PHI(R) \
    case R: return phase_i1_launch<R>(P, elem, radius, fp64_cond, s);
cudaError_t launch_phase_i1_iter(const IterPhase &P, int elem, int radius, bool generic, float fp64_cond,
                                 cudaStream_t s)
{
    if (generic) return phase_i1_launch<0>(P, elem, radius, fp64_cond, s);
    switch (radius) {
        OF_RADII(OF_CASE_PHI)
    default: return phase_i1_launch<0>(P, elem, radius, fp64_cond, s);
    }
}

#define OF_CASE_BK(R) \
    case R: return batch_kernel_ptr<R>(in_format, storage);
void *batch_kernel_for(int in_format, int storage, int radius)
{
    switch (radius) {
        OF_RADII(OF_CASE_BK)
    default: return batch_kernel_ptr<0>(in_format, storage);
    }
}

#define OF_CASE_SM(R) \
    case R: return radius_smem_bytes<R>(radius, stage_i2);
size_t batch_smem_bytes(int radius, bool stage_i2)
{
    switch (radius) {
        OF_RADII(OF_CASE_SM)
    default: return radius_smem_bytes<0>(radius, stage_i2);
    }
}

void *batch_kernel_generic(int in_format, int storage) { return batch_kernel_ptr<0>(in_format, storage); }
size_t batch_smem_generic(int radius) { return radius_smem_bytes<0>(radius, false); }

#define OF_CFG(R) \
    if ((e = radius_configure<R>()) != cudaSuccess) return e;
cudaError_t configure_lk_kernels()
{
    cudaError_t e;
    OF_RADII(OF_CFG)
    OF_CFG(0)
    return cudaSuccess;
}

}  // namespace of
