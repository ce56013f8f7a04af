// Dispatch of the splat launch by output type (the kernels of each type are
// instantiated in splat_<type>.cu from splat.cuh) and the splat's shared
// memory size.
#include "splat.cuh"

namespace spx {

size_t splat_smem_bytes(int edge, int tile, int warp_scratch, int rec_buf_bytes) {
    return smem_layout(edge, tile, warp_scratch, rec_buf_bytes).total;
}

cudaError_t launch_splat_f32(const KernelArgs &a, cudaStream_t st);
cudaError_t launch_splat_f16(const KernelArgs &a, cudaStream_t st);
cudaError_t launch_splat_bf16(const KernelArgs &a, cudaStream_t st);
cudaError_t launch_splat_u8(const KernelArgs &a, cudaStream_t st);
cudaError_t launch_splat_u16(const KernelArgs &a, cudaStream_t st);

cudaError_t launch_splat(const KernelArgs &a, int32_t out_dtype, cudaStream_t st, cudaEvent_t const *ev) {
    cudaError_t e;
    switch (out_dtype) {
    case SYNTHPIX_F32: e = launch_splat_f32(a, st); break;
    case SYNTHPIX_F16: e = launch_splat_f16(a, st); break;
    case SYNTHPIX_BF16: e = launch_splat_bf16(a, st); break;
    case SYNTHPIX_U8: e = launch_splat_u8(a, st); break;
    default: e = launch_splat_u16(a, st); break;
    }
    if (e != cudaSuccess) return e;
    if (ev && ev[5]) cudaEventRecord(ev[5], st);
    return cudaGetLastError();
}

}  // namespace spx
