// k_splat and k_finish for uint8_t outputs (device code in splat.cuh).
#include "splat.cuh"

namespace spx {

cudaError_t launch_splat_u8(const KernelArgs &a, cudaStream_t st) { return launch_splat_t<uint8_t>(a, st); }

}  // namespace spx
