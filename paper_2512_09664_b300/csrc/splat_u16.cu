// k_splat and k_finish for uint16_t outputs (device code in splat.cuh).
#include "splat.cuh"

namespace spx {

cudaError_t launch_splat_u16(const KernelArgs &a, cudaStream_t st) { return launch_splat_t<uint16_t>(a, st); }

}  // namespace spx
