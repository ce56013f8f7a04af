// Launch interface between the host entry points (api.cu) and the kernels
// (prep.cu: plan, seeding + advection, binning; splat.cu: the splat).
#pragma once

#include <memory>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace spx {

// Everything one render launch sequence reads or writes (passed by value).
struct KernelArgs {
    const synthpix_pair_desc *descs;  // device copy of the descriptors (16-byte aligned)
    const PairPlan *plan;             // device plan (k_plan)
    const int32_t *check;             // 1 when the device plan matches the host's
    int32_t n_pairs;
    int32_t tile;                     // largest tile edge of the batch's pairs (launch shapes, shared memory)
    int64_t n_part;                   // particles of all pairs
    int64_t n_tiles;                  // (pair, frame, tile) work items
    int64_t n_chunks;                 // particle chunks (kChunk particles of one pair)
    uint64_t seed;
    PhiloxKeys keys;                  // round keys of seed
    float dt;
    int32_t n_substeps;
    int32_t integrator;
    int32_t quant_bits;
    const float *flows;
    void *images;
    float4 *pos0, *pos1;              // split positions of frames 1 and 2
    float2 *sa;                       // (sigma, Ieff * 2 pi sigma^2)
    float4 *shape;                    // ext: [2][n_part] (sigma_x, sigma_y, rho, amplitude) per frame;
                                      // sigma_x < 0: hidden from that frame
    int32_t ext;                      // 1: per-frame shapes (general shapes, variation or hiding)
    int32_t general;                  // 1: bins hold RecordG (general-shape splat)
    float hide_prob;                  // probability of hiding a particle from a frame
    uint32_t *carry;                  // k_splat: carry words, carry_stride per CTA (wrapped fixed-point sums)
    int64_t carry_stride;
    int32_t out_of_plane;             // 1: a w grid follows each flow grid; z moves along the path
    uint32_t *count, *off, *cursor;   // per (pair, frame, tile)
    ItemInfo *items;                  // per (pair, frame, tile): the splat's work items
    Record *rec;                      // bins
    Record *adv;                      // tiled advection: frame-2 records by frame-1 bin slot (sigma < 0: none)
    int32_t tiled;                    // seeded renders, records placed into fixed-capacity bins (fixed_caps):
                                      // 2: k_seed_place advects each particle and places both frames;
                                      // 1: k_seed_place places frame 1, the tiled advection (k_advect)
                                      // makes and places frame 2; 0: k_seed_advect and a counting sort
    uint32_t *ovf;                    // [2]: a fixed bin of frame 1 / frame 2 overflowed (zeroed by k_plan)
    int32_t rebin;                    // 1: launch k_rebin after each placement (0: no bin can overflow)
    uint32_t *ticket;                 // work-queue counter of the persistent splat
    int32_t smem_edge;                // capacity edge of the on-chip tile (tile + 2 max radius)
    int32_t warp_scratch;             // floats of per-warp window scratch
    const float *blur_w;              // [n_pairs][kBlurStride] normalised taps w[|k|]
    int32_t rec_buf_bytes;            // bytes of the staged-record region (at most rec_buf_bytes_for(tile))
    int32_t reg_epilogue;             // 1: full 128 x 128 tiles finish with the register blur
    int32_t inter_dtype;              // SYNTHPIX_F32: fused; F16 / BF16: intermediate frames
    void *inter;                      // 16-bit intermediate frames (non-fused path)
    const float *particles_in;        // NULL or [n_part][3] (x0, y0, d) replacing the seeded values
    float *particles_out;             // NULL, or export only: [n_part][3] (x, y, d) of frame export_frame
    int32_t export_frame;             // 0: the seeded (frame-1) positions; 1: the advected (frame-2) ones
    // adjoint
    const float *grad_images;         // dL/d(images), FP32, same packing as the images
    float *grad_flows;                // NULL or dL/d(flows), accumulated
    float *grad_particles;            // NULL or [n_part][3] dL/d(x0, y0, d)
    float4 *grad_frames;              // [n_part][2]: dL/d(x, y, sigma) of each frame's splat
    float4 *states;                   // NULL, or [n_part][n_substeps]: the split position (fx, fy, ix, iy) at
                                      // the start of each substep, written by the per-particle advection for
                                      // the adjoint (which then does not recompute them)
};

// The splat's work item t (t = tile_base + frame ntiles + tile).  With fixed
// bins the item holds the bin's capacity and the count is the bin's counter
// (records were placed at slots 0 .. min(counter, capacity) - 1), unless the
// frame was binned again exactly after an overflow (k_rebin wrote the item).
__device__ __forceinline__ ItemInfo work_item(const KernelArgs &a, int64_t t) {
    ItemInfo it = a.items[t];
    if (a.tiled) {  // the three loads are independent of the item's
        const uint32_t n = a.count[t], o0 = a.ovf[0], o1 = a.ovf[1];
        if ((it.frame ? o1 : o0) == 0u) it.count = min(it.count, n);
    }
    return it;
}

constexpr int kStageEvents = 6;

// Counts the library's kernel launches (synthpix_launch_count); every launch
// of the library goes through launch_kernel, which calls it.
void count_launch();
uint64_t launch_total();

// A kernel launch held back for a CUDA graph: the kernel, its shape and a
// copy of its arguments (params points into `args`).
struct RecordedLaunch {
    const void *func;
    unsigned grid, block;
    size_t smem;
    std::shared_ptr<void> args;
    std::vector<void *> params;
};
// While a render's launch sequence is recorded on this thread, launch_kernel
// appends to it instead of launching (api.cu submits the sequence as one
// CUDA graph).
extern thread_local std::vector<RecordedLaunch> *t_recording;

// Launch a kernel of the library (or record it, see t_recording); returns
// the launch's error.  (Programmatic dependent launch was measured: a
// replayed render took 12 us longer with it, so the kernels are launched
// plainly.)
template <typename... P, typename... A>
inline cudaError_t launch_kernel(void (*kernel)(P...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                                  A &&...args) {
    if (t_recording) {
        using Tuple = std::tuple<P...>;
        auto tup = std::make_shared<Tuple>(static_cast<A &&>(args)...);
        RecordedLaunch r;
        r.func = reinterpret_cast<const void *>(kernel);
        r.grid = grid;
        r.block = block;
        r.smem = smem;
        r.params = std::apply([](auto &...e) { return std::vector<void *>{static_cast<void *>(&e)...}; }, *tup);
        r.args = std::move(tup);
        t_recording->push_back(std::move(r));
        return cudaSuccess;
    }
    kernel<<<grid, block, smem, st>>>(static_cast<A &&>(args)...);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) count_launch();
    return e;
}
constexpr int kSplatThreads = 256;      // k_splat below tile 128, k_finish
constexpr int kSplatMaxThreads = 1024;  // k_splat at tile 128 (one CTA per SM)
constexpr int kStageDesc = (int)sizeof(synthpix_pair_desc);  // staged header: descriptor (160),
constexpr int kStagePlan = kStageDesc + (int)sizeof(PairPlan);  // plan (64),
constexpr int kStageHeader = kStagePlan + 128;                  // blur taps (128)
// k_splat stages two headers (the current and the next item's) and one
// region of binned records: the next item's records are copied in once the
// current item's are splatted, behind its finishing steps.
constexpr int kRecBufBytes = 2 * 10240 - 2 * kStageHeader;       // the record region (tiles up to 64)
constexpr int kRecBufBytesLarge = 2 * 13312 - 2 * kStageHeader;  // the same at tile 128 (two CTAs per SM; one
                                                                  // chunk for most items of 512 x 512 frames)
constexpr int kSplatRpt = 3;  // records per thread of one chunk of round particles (splat_chunk)
// records of rec_bytes bytes per staged chunk of a record region
__host__ __device__ constexpr int rec_cap(int buf_bytes, int rec_bytes = 24) { return (buf_bytes - 32) / rec_bytes; }
// threads of a k_splat CTA at a tile edge: 512 at tile 128 (two CTAs per
// SM), else 256 (several CTAs per SM hide each other's barriers)
__host__ __device__ constexpr int splat_threads(int tile) { return tile >= 128 ? 512 : 256; }
// k_splat CTAs the carry words are laid out for: a bound on SMs times the
// CTAs an SM holds at 64 registers a thread (65536 / (64 NT)), and never
// more than the batch's work items; the launch is clamped to it
constexpr int kCarrySms = 160;
__host__ __device__ constexpr int64_t splat_max_ctas(int tile, int64_t n_items) {
    const int64_t m = (int64_t)kCarrySms * (1024 / splat_threads(tile));
    return n_items < m ? n_items : m;
}
// Row pitch capacity of the accumulator for a capacity edge E (tile + 2 max
// radius): the aligned widths stay within E + 6.
__host__ __device__ inline int pitch_cap(int E) { return ((E + 3) & ~3) + 4; }
__host__ __device__ constexpr int rec_buf_bytes_for(int tile) { return tile >= 128 ? kRecBufBytesLarge : kRecBufBytes; }
constexpr size_t kMaxSmemBytes = 227 * 1024;  // dynamic shared memory of one CTA

// count: NULL, or the per-(pair, frame, tile) bin counts, zeroed by the plan launch
// ticket: the splat's work-queue counter, followed by the two overflow flags of the fixed bins.
// pf_flows: NULL, or the flows of a batch whose flow grids take at most
// kPrefetchMaxBytes in all (pf_planes floats per node: 2, or 3 with the
// out-of-plane grid); a CTA per pair of the plan launch then asks the L2 to
// fetch the pair's grid, so that the flow gathers of the next kernels hit L2.
constexpr int64_t kPrefetchMaxBytes = 32LL << 20;    // a quarter of the 126 MB L2
constexpr int64_t kPrefetchPieceBytes = 64LL << 10;  // per bulk-prefetch instruction (one lane)
cudaError_t launch_plan(const synthpix_pair_desc *descs, int32_t n_pairs, const TileRule &rule, int32_t fused,
                        PairPlan *plan, const Layout &L, int32_t *check, float *blur_w, uint32_t *ticket,
                        uint32_t *count, const float *pf_flows, int32_t pf_planes, cudaStream_t st);
// ev: NULL or kStageEvents events recorded at the stage boundaries.
cudaError_t launch_prep(const KernelArgs &a, cudaStream_t st, cudaEvent_t const *ev);
cudaError_t launch_splat(const KernelArgs &a, int32_t out_dtype, cudaStream_t st, cudaEvent_t const *ev);
size_t splat_smem_bytes(int edge, int tile, int warp_scratch, int rec_buf_bytes);
// export only (a.particles_out set): k_seed_advect exports the particles of frame a.export_frame
cudaError_t launch_seed_only(const KernelArgs &a, cudaStream_t st);
// adjoint: splat gradients per (particle, frame), then the reverse advection
cudaError_t launch_adjoint(const KernelArgs &a, cudaStream_t st);
constexpr int kMaxAdjointSubsteps = 64;

}  // namespace spx
