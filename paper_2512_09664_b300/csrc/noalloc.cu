// synthpix_render_pairs_noalloc: the render call for callers that cannot
// allocate device memory.  Some host applications own all device memory
// through their own allocator and do not let libraries call cudaMalloc
// (plugin hosts, embedded runtimes with a fixed memory budget), and some
// loops cannot afford the device synchronisation cudaMalloc may imply.  Such
// callers pass only their inputs and outputs; the scratch memory the render
// needs lives in the fixed array below, compiled into the library.
#include <cstdio>
#include <mutex>

#include "synthpix.h"

// The scratch of the no-allocation entry point.  Every GPU that loads the
// library holds these SYNTHPIX_NOALLOC_SCRATCH_BYTES until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SYNTHPIX_NOALLOC_SCRATCH_BYTES];

namespace spx {
int set_error(int code, const char *msg);
int render_workspace_need(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs, int32_t n_pairs,
                          size_t *need);
// synthpix_render_pairs with the kernels launched one by one (no CUDA graph,
// whose instantiation may allocate)
int render_pairs_direct(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                        const synthpix_pair_desc *pairs_dev, int32_t n_pairs, const float *flows, void *images,
                        void *workspace, size_t workspace_bytes, void *stream);
}

namespace {

constexpr int kMaxDevices = 256;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  Host code only
// sees a host-side stand-in under the array's name, so the address is looked
// up once per device with that device current, and cached.
int scratch_address(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof(msg), "no-allocation render: cudaGetDevice failed: %s", cudaGetErrorString(e));
        return spx::set_error(SYNTHPIX_ECUDA, msg);
    }
    if (dev < 0 || dev >= kMaxDevices) return spx::set_error(SYNTHPIX_ECUDA, "no-allocation render: device index out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            char msg[256];
            snprintf(msg, sizeof(msg), "no-allocation render: cudaGetSymbolAddress failed: %s",
                     cudaGetErrorString(e));
            return spx::set_error(SYNTHPIX_ECUDA, msg);
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SYNTHPIX_OK;
}

}  // namespace

extern "C" int synthpix_render_pairs_noalloc(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                                             const synthpix_pair_desc *pairs_dev, int32_t n_pairs,
                                             const float *flows, void *images, void *stream) {
    // validation and the scratch size come from the host descriptors alone: the
    // plan of the tile edge the render itself resolves (batch->tile, or the
    // default edge for 0), checked the way the render checks it
    size_t need = 0;
    const int prc = spx::render_workspace_need(batch, pairs, n_pairs, &need);
    if (prc != SYNTHPIX_OK) return prc;  // invalid descriptors: the plan's own status and message
    if (n_pairs == 0) return spx::set_error(SYNTHPIX_OK, "");
    if (need > (size_t)SYNTHPIX_NOALLOC_SCRATCH_BYTES) {
        char msg[256];
        snprintf(msg, sizeof(msg),
                 "no-allocation render: this batch needs %zu bytes of scratch, more than the %zu the library "
                 "holds; split the batch or use synthpix_render_pairs with a workspace",
                 need, (size_t)SYNTHPIX_NOALLOC_SCRATCH_BYTES);
        return spx::set_error(SYNTHPIX_EWORKSPACE, msg);
    }
    void *scratch = nullptr;
    const int rc = scratch_address(&scratch);
    if (rc != SYNTHPIX_OK) return rc;
    // the render clears what must start at zero (its bin counters) itself;
    // everything else in the scratch is written before it is read
    return spx::render_pairs_direct(batch, pairs, pairs_dev, n_pairs, flows, images, scratch,
                                    (size_t)SYNTHPIX_NOALLOC_SCRATCH_BYTES, stream);
}
