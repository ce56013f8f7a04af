// k_splat and k_finish for __nv_bfloat16 outputs (device code in splat.cuh).
#include "splat.cuh"

namespace spx {

cudaError_t launch_splat_bf16(const KernelArgs &a, cudaStream_t st) { return launch_splat_t<__nv_bfloat16>(a, st); }

}  // namespace spx
