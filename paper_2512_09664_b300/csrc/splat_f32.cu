// k_splat and k_finish for float outputs (device code in splat.cuh).
#include "splat.cuh"

namespace spx {

cudaError_t launch_splat_f32(const KernelArgs &a, cudaStream_t st) { return launch_splat_t<float>(a, st); }

}  // namespace spx
