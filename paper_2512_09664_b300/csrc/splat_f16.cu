// k_splat and k_finish for __half outputs (device code in splat.cuh).
#include "splat.cuh"

namespace spx {

cudaError_t launch_splat_f16(const KernelArgs &a, cudaStream_t st) { return launch_splat_t<__half>(a, st); }

}  // namespace spx
