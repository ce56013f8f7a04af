/*
 * synthpix.h — C ABI of the B300 (sm_103a) PIV image-pair renderer.
 *
 * The library renders synthetic Particle Image Velocimetry image pairs from a
 * prescribed flow field, the method of SynthPix (arXiv 2512.09664, Section 2):
 * particles are seeded over the image, moved by the flow for the second
 * frame, each drawn as the Gaussian particle image of Eq. 1, summed, and the
 * frames finished with illumination non-uniformity, noise, blur and
 * quantisation (the imaging parameters listed in the Abstract and in
 * Section 2 "Configuration file").
 *
 * Conventions used by every entry point
 *  - Pixel (i, j) covers [j, j+1) x [i, i+1); x is the column, y the row
 *    (downwards).  Frames are row-major [H][W].
 *  - Flow grids are float32 [flow_h][flow_w][2] holding (u, v) in pixels per
 *    frame, nodes at cell centres ((l + 1/2) W / flow_w, (k + 1/2) H / flow_h),
 *    interpolated bilinearly with indices clamped to the grid.
 *  - sigma = d / 4 for a particle of diameter d; the particle image is
 *    integrated over each pixel (separable erf differences) on the window
 *    [floor(x - 1.5 d), floor(x + 1.5 d)]^2, the 3 d + 1 patch of Section 2
 *    "Efficient rasterization".  General particles (Eq. 1 with
 *    sigma_x = d / 4, sigma_y = d_y / 4 and correlation rho) are integrated
 *    over each pixel too, on the window floor(x +- 1.5 d) by
 *    floor(y +- 1.5 d_y); their integrated image is
 *    Ieff 2 pi sigma_x sigma_y sqrt(1 - rho^2).
 *  - Random numbers: Philox4x32-10 keyed by the batch seed; the output of a
 *    pair depends only on (seed, pair_id, its descriptor, its flow grid).
 *  - All device pointers are owned by the caller.  The library allocates no
 *    device memory and keeps no per-call state; it only reads the caller's
 *    inputs and writes the caller's outputs and workspace.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *    default stream).  They never synchronise the device and never trap; on
 *    error they return a negative status before launching anything, and
 *    synthpix_last_error() describes it.
 */
#ifndef SYNTHPIX_H
#define SYNTHPIX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SYNTHPIX_ABI_VERSION 3

/* ---- status codes ------------------------------------------------------ */
#define SYNTHPIX_OK            0
#define SYNTHPIX_EINVAL       -1  /* a descriptor or argument is out of range      */
#define SYNTHPIX_EWORKSPACE   -2  /* workspace pointer NULL / too small / unaligned */
#define SYNTHPIX_ECUDA        -3  /* a CUDA call or launch failed                   */
#define SYNTHPIX_EUNSUPPORTED -4  /* valid but not supported (reserved fields set)  */

/* ---- element types (out_dtype, inter_dtype) ----------------------------- */
#define SYNTHPIX_F32  0
#define SYNTHPIX_F16  1
#define SYNTHPIX_BF16 2
#define SYNTHPIX_U8   3
#define SYNTHPIX_U16  4

/* ---- integrators -------------------------------------------------------- */
#define SYNTHPIX_RK4   0
#define SYNTHPIX_EULER 1

/* sheet models (pair->sheet_model) */
#define SYNTHPIX_SHEET_GAUSSIAN 0
#define SYNTHPIX_SHEET_REMARK   1

/* batch flags */
#define SYNTHPIX_FLAG_GATHER_ADVECT 1  /* advect every particle by direct flow-grid gathers
                                          and bin both frames by a counting sort instead
                                          of the fixed-capacity bins (same result)       */
#define SYNTHPIX_FLAG_TILED_ADVECT  4  /* advect tile by tile from flow windows staged on
                                          chip instead of per particle while seeding
                                          (same result); excludes GATHER_ADVECT          */
#define SYNTHPIX_FLAG_OUT_OF_PLANE  2  /* out-of-plane motion (Remark "out-of-focus": a
                                          three-dimensional flow): each pair's flow grid
                                          is followed in `flows`, at flow_offset +
                                          2 flow_h flow_w, by flow_h x flow_w floats w,
                                          the out-of-plane velocity in units of z per
                                          frame on the same nodes.  z moves along the
                                          particle's path (the same RK4 / Euler stages
                                          as x, y) and frame 2's intensity uses the
                                          moved z.  Such renders advect per particle. */

/*
 * Per-pair acquisition parameters (Abstract: seeding density, particle image
 * size, illumination non-uniformity, noise, blur, timing; Section 2 "Sampling
 * the particles": parameters drawn uniformly from configured intervals).
 * 160 bytes, naturally aligned; reserved fields must be zero.
 */
typedef struct synthpix_pair_desc {
    int32_t  height, width;      /* frame size in pixels, 1..32768                   */
    int64_t  image_offset;       /* element offset of frame 1 in the output buffer;
                                    frame 2 follows at image_offset + height*width   */
    int64_t  flow_offset;        /* float offset of this pair's flow grid in `flows`;
                                    pairs may share a grid (F flows for B pairs)     */
    int32_t  flow_h, flow_w;     /* flow grid nodes, 1..32768                         */
    uint64_t pair_id;            /* Philox counter words of this pair                 */
    uint32_t n_particles;        /* particles of frame 1: floor(ppp * H * W)          */
    int32_t  d_dist;             /* 0: d ~ U[d_min, d_max]; 1: N(d_mu, d_sigma)
                                    clipped to [d_min, d_max]                         */
    float d_min, d_max;          /* particle diameter bounds, px; 0 < d_min <= d_max <= 32 */
    float d_mu, d_sigma;         /* normal diameter parameters (d_dist = 1)           */
    float i_min, i_max;          /* peak intensity I0 of Eq. 1 ~ U[i_min, i_max]       */
    float z_min, z_max;          /* out-of-plane position ~ U[z_min, z_max]            */
    float sheet_sigma;           /* laser sheet: Gaussian I = I0 exp(-z^2/(2 s^2)), or the
                                    thickness dz0 of the Remark form (sheet_model);
                                    <= 0 disables the attenuation                     */
    float illum_min, illum_max;  /* illumination field L in [illum_min, illum_max]:
                                    L = min + (max-min) sin^2(pi (j+.5)/W) sin^2(pi (i+.5)/H) */
    float noise_sigma;           /* additive Gaussian noise std (full scale 1.0)      */
    float blur_sigma;            /* Gaussian blur std in px (radius ceil(3 sigma)), 0..8 */
    /* General particle shapes and second-image variation (text after Eq. 1:
       sigma_x, sigma_y, rho drawn per particle from intervals; each parameter
       of the second image varies by a zero-mean Gaussian).  All zero: round
       particles, the same parameters in both frames.  Drawn from Philox
       stream 2 (hiding words, normals of the d and I0 changes) and stream 3
       (d_y, rho, normals of the d_y and rho changes).  Any non-zero field
       (or batch->hide_prob > 0) makes the render advect per particle; d_y or
       rho non-zero in any pair selects the general-shape splat (32-byte
       bin records, per-pixel quadrature when rho != 0).                       */
    float dy_min, dy_max;        /* diameter along y, sigma_y = d_y / 4, d_y ~ U[dy_min,
                                    dy_max]; 0, 0: d_y = d.  Else 0 < dy_min <= dy_max <= 32 */
    float rho_min, rho_max;      /* correlation of Eq. 1 ~ U[rho_min, rho_max],
                                    -0.95 <= rho_min <= rho_max <= 0.95              */
    float jitter_d;              /* std (px) of the frame-2 change of d and of d_y (drawn
                                    independently; with d_y = d one change for both),
                                    the results clamped to [d_min, d_max] / [dy_min, dy_max] */
    float jitter_i;              /* std of the frame-2 change of I0, clamped to [i_min, i_max] */
    float jitter_rho;            /* std of the frame-2 change of rho, clamped to its interval */
    /* Out-of-focus intensity (Remark "out-of-focus").                          */
    int32_t sheet_model;         /* SYNTHPIX_SHEET_GAUSSIAN (0): exp(-z^2 / (2 sheet_sigma^2));
                                    SYNTHPIX_SHEET_REMARK (1): the Remark's
                                    exp(-|2 z^2 / sheet_sigma^2|^sheet_shape / sqrt(2 pi)),
                                    I0 drawn in [i_min, i_max] playing the scattering
                                    efficiency q                                       */
    float sheet_shape;           /* shape factor s of the Remark form, 0 < s <= 16
                                    (ignored, may be 0, for the Gaussian sheet)        */
    int32_t reserved[6];         /* must be zero                                       */
} synthpix_pair_desc;

/*
 * Batch-wide settings.  64 bytes; reserved fields must be zero.
 */
typedef struct synthpix_batch_desc {
    uint64_t seed;               /* Philox key                                         */
    int32_t  out_dtype;          /* SYNTHPIX_F32/F16/BF16 (values of B, unclipped) or
                                    SYNTHPIX_U8/U16 (codes clamp(rint(B*M),0,M))        */
    int32_t  quant_bits;         /* 0 for float outputs; 1..8 for U8; 1..16 for U16;
                                    M = 2^quant_bits - 1                               */
    int32_t  inter_dtype;        /* storage of the splatted image between the splat and
                                    the epilogue: SYNTHPIX_F32 keeps it in on-chip
                                    memory (fused, no HBM intermediate); SYNTHPIX_F16 /
                                    SYNTHPIX_BF16 write it to the workspace in 16 bits
                                    (accumulation stays FP32 or wider)                 */
    int32_t  integrator;         /* SYNTHPIX_RK4 or SYNTHPIX_EULER                      */
    int32_t  n_substeps;         /* substeps over dt, 1..1024                          */
    float    dt;                 /* time between the frames, in frames (|dt| <= 64)    */
    int32_t  tile;               /* square screen tile edge of every pair: 16, 32, 64 or
                                    128; or 0: an edge per frame size class (frame area
                                    < 2^15, < 2^17, < 2^19 pixels, larger), from the
                                    autotuner's table where synthpix_autotune has an
                                    entry for the class, else 32, 64, 128, 128.  Tile
                                    128 fails with SYNTHPIX_EUNSUPPORTED when the
                                    largest blur radius needs more shared memory than a
                                    CTA has.                                           */
    int32_t  flags;              /* 0 or an OR of SYNTHPIX_FLAG_*.  By default a
                                    seeded render advects each particle where it is
                                    seeded, by flow-grid gathers that keep the last
                                    grid cell's nodes in registers, and places both
                                    frames' records into fixed-capacity bins in the
                                    same pass.  TILED_ADVECT advects tile by tile from
                                    flow windows staged on chip; GATHER_ADVECT bins by
                                    a counting sort.  Renders from given particles and
                                    the adjoint always gather per particle.  All give
                                    the same positions and images.                    */
    float    hide_prob;          /* probability, 0..1, that a particle is left out of a
                                    frame, independently per frame (Section 2,
                                    aggregation of the particle contributions)         */
    int32_t  reserved[5];        /* must be zero                                       */
} synthpix_batch_desc;

/*
 * Bytes of device workspace synthpix_render_pairs needs for this batch
 * (a 256-byte aligned region the caller allocates).  With batch->tile = 0 it
 * is an upper bound over every tuning the autotuners try or cache, so one
 * workspace serves every choice.  Returns 0 and sets the last error if the
 * descriptors are invalid.  Only the host arrays are read.
 */
size_t synthpix_workspace_bytes(const synthpix_batch_desc *batch,
                                const synthpix_pair_desc *pairs, int32_t n_pairs);

/*
 * Render n_pairs image pairs (paper Section 2; Eq. 1 integrated per pixel).
 *
 *   batch      host pointer, batch settings.
 *   pairs      host pointer, n_pairs descriptors; read during the call only.
 *   pairs_dev  NULL, or a 16-byte aligned device copy of the same n_pairs
 *              descriptors.  With
 *              NULL the library copies `pairs` into the workspace with
 *              cudaMemcpyAsync on `stream` (keep `pairs` unchanged until the
 *              stream reaches the copy if it is pinned memory).  Passing a
 *              device copy makes the call free of host-to-device copies, as a
 *              CUDA-graph capture needs.
 *   n_pairs    0 .. 1<<20 (0 returns SYNTHPIX_OK and does nothing).
 *   flows      device pointer, float32; each pair reads
 *              flows[flow_offset .. flow_offset + flow_h*flow_w*2).
 *   images     device pointer to the output buffer of element type
 *              batch->out_dtype; pair b writes elements
 *              [image_offset, image_offset + 2*H*W) once each (frame 1, then 2).
 *   workspace  device pointer, 256-byte aligned, at least
 *              synthpix_workspace_bytes(...) bytes; contents on entry ignored.
 *   stream     cudaStream_t.
 *
 * Launches: the render's kernels (plan, seeding and binning, splat) run in
 * stream order on `stream`.  Unless the stream is being captured, the
 * library submits them as one CUDA graph from the second render of the same
 * launch shapes on a device on (the first render of a shape launches kernel
 * by kernel; the second instantiates the graph, which may allocate device
 * memory; later renders set its arguments and launch it).  Graph launches of
 * one shape are ordered behind one another even on different streams.  The
 * cached graphs belong to the device's context: a cudaDeviceReset after such
 * a render is not supported.
 *
 * Returns SYNTHPIX_OK or a negative status (nothing is launched on error).
 */
int synthpix_render_pairs(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                          const synthpix_pair_desc *pairs_dev, int32_t n_pairs,
                          const float *flows, void *images,
                          void *workspace, size_t workspace_bytes, void *stream);

/*
 * synthpix_render_pairs with given particles instead of the seeded ones:
 * particles_in is a device array [sum of n_particles][3] of FP32 (x0, y0, d)
 * (frame-1 position in pixels and diameter), pairs in order; NULL means the
 * seeded values (then identical to synthpix_render_pairs).  Intensities and
 * out-of-plane positions still come from the seeded streams.  Used for
 * differentiation (finite differences, optimisation over positions).
 * Round particles only: a batch with hide_prob or any general-shape or
 * variation field set fails with SYNTHPIX_EUNSUPPORTED.
 */
int synthpix_render_pairs_from(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                               const synthpix_pair_desc *pairs_dev, int32_t n_pairs,
                               const float *particles_in, const float *flows, void *images,
                               void *workspace, size_t workspace_bytes, void *stream);

/*
 * The seeded particles: writes particles_out [sum of n_particles][3] (FP32
 * x0, y0, d of each particle; device pointer), the values
 * synthpix_render_pairs draws (Section 2, "Sampling the particles").  flows
 * and images are not needed.  Same workspace as synthpix_render_pairs.
 */
int synthpix_seed_particles(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                            const synthpix_pair_desc *pairs_dev, int32_t n_pairs, float *particles_out,
                            void *workspace, size_t workspace_bytes, void *stream);

/*
 * Particle reuse across consecutive frames (the paper's Conclusions list it
 * as planned work: the flow applied for a second, possibly different, dt' to
 * the frame-2 positions gives the frame-1 positions of the next batch).
 * Writes [sum of n_particles][3] (x, y, d) to particles_out (device, 4-byte
 * aligned, caller-owned): each particle advected from its frame-1 position
 * over batch->dt exactly as synthpix_render_pairs advects it, rounded once to
 * FP32, and its diameter.  particles_in (nullable) as in
 * synthpix_render_pairs_from: the frame-1 (x0, y0, d); NULL takes the seeded
 * ones.  A sequence: advect a batch's particles over dt' (this call, with
 * particles_in = its frame-2 positions, themselves from this call over dt),
 * then render the next batch with synthpix_render_pairs_from and the same
 * pair_id, which keeps each particle's intensity and depth (drawn from the
 * same Philox counters).  Same workspace as synthpix_render_pairs; images
 * are not needed.
 */
int synthpix_advect_particles(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                              const synthpix_pair_desc *pairs_dev, int32_t n_pairs, const float *particles_in,
                              const float *flows, float *particles_out, void *workspace, size_t workspace_bytes,
                              void *stream);

/*
 * Adjoint of the render (not in the paper; its differentiable use): given
 * grad_images = dL/d(images) (FP32, same packing as the images), computes
 *   grad_flows      dL/d(flows), ADDED to the caller's array (same layout as
 *                   flows, 8-byte aligned; several pairs sharing a grid sum
 *                   into it), or NULL;
 *   grad_particles  [sum of n_particles][3] dL/d(x0, y0, d), overwritten, or NULL;
 * for the frames B = L * S + noise (the splat of Eq. 1 integrated per pixel,
 * times the illumination field).  Requires out_dtype F32 (quantisation has no
 * gradient), blur_sigma = 0 for every pair, at most 64 substeps and round
 * particles without hiding or variation (SYNTHPIX_EUNSUPPORTED otherwise).  particles_in as in
 * synthpix_render_pairs_from.  Positions and bins are recomputed, not taken
 * from a forward call.  The splat gradient is a per-particle reduction over
 * its window; flow gradients are accumulated with atomics, so their last bits
 * may vary from run to run.  Same workspace as synthpix_render_pairs.
 */
int synthpix_render_backward(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                             const synthpix_pair_desc *pairs_dev, int32_t n_pairs,
                             const float *particles_in, const float *flows,
                             const float *grad_images, float *grad_flows, float *grad_particles,
                             void *workspace, size_t workspace_bytes, void *stream);

/*
 * synthpix_render_pairs plus per-stage timing: stage_events holds 6 CUDA
 * events (cudaEvent_t, created by the caller; NULL entries are skipped) that
 * are recorded on `stream` at the stage boundaries, so the caller can time
 * each kernel with cudaEventElapsedTime after synchronising:
 *   [0] before the plan kernel, [1] after the plan and the bin reset,
 *   [2] after everything up to the advection: seeding and advection, and
 *       the binning done with them.  Seeded renders of round particles bin
 *       the records into fixed-capacity bins while seeding (frame 1) and
 *       advecting (frame 2); renders from given particles or with
 *       per-frame shapes only seed and advect here,
 *   [3] after the scan of the bin counts (renders from given particles or
 *       with per-frame shapes; nothing for seeded renders),
 *   [4] after the scatter of the records into the bins (seeded renders:
 *       the exact rebinning of frame 2, which does work only if a bin
 *       overflowed, and is not launched when no pair's bins can overflow),
 *   [5] after the splat + epilogue kernel.
 * The paper has no counterpart; it exists for measurement.  Same arguments,
 * errors and asynchrony as synthpix_render_pairs; no synchronisation.
 */
int synthpix_render_pairs_staged(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                                 const synthpix_pair_desc *pairs_dev, int32_t n_pairs,
                                 const float *flows, void *images,
                                 void *workspace, size_t workspace_bytes, void *stream,
                                 void *const *stage_events);

/*
 * synthpix_render_pairs for callers that cannot allocate device memory: host
 * applications that own all device memory through their own allocator and
 * do not let libraries call cudaMalloc (plugin hosts, embedded runtimes with
 * a fixed memory budget), and loops that cannot afford the device
 * synchronisation cudaMalloc may imply.  The paper has no counterpart.
 *
 * The caller passes inputs and outputs only.  The scratch memory lives in a
 * static __device__ array of SYNTHPIX_NOALLOC_SCRATCH_BYTES (32 MiB) compiled
 * into the library; every GPU that loads the library holds it until the
 * process exits.  This call allocates nothing (no cudaMalloc / cudaFree, no
 * allocating library routine); its kernels are launched one by one, never
 * submitted as a CUDA graph (graph instantiation may allocate).
 *  - A batch that needs more scratch than the array holds (compare
 *    synthpix_workspace_bytes) is rejected with SYNTHPIX_EWORKSPACE and a
 *    message, before anything is launched.
 *  - The scratch needed is that of the plan the render runs: the tile edge
 *    batch->tile, or for 0 the edges the render picks (the autotuner's table
 *    or the defaults), so a batch can fit here although
 *    synthpix_workspace_bytes, which for tile 0 covers every tuning, reports
 *    more.
 *  - The first call on a device looks up the array's device address on that
 *    device (cudaGetSymbolAddress with the device current) and caches it;
 *    make that first call on each device before any stream capture.
 *  - The cached address belongs to the device's context at the time of the
 *    first call.  A device reset (cudaDeviceReset) after that call is not
 *    supported: the next call would use a stale address.  Reset devices only
 *    before the first call, or not at all in a process that uses this entry
 *    point.
 *  - All calls share the one array, which keeps the last call's contents;
 *    the call clears what must start at zero itself.  Calls whose work
 *    overlaps on the GPU (other streams, other host threads) race on the
 *    array: the caller must order them.
 * Other arguments, errors and asynchrony are those of synthpix_render_pairs.
 */
#define SYNTHPIX_NOALLOC_SCRATCH_BYTES (32u << 20)
int synthpix_render_pairs_noalloc(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                                  const synthpix_pair_desc *pairs_dev, int32_t n_pairs,
                                  const float *flows, void *images, void *stream);

/*
 * Autotuner of one screen tile edge for the whole batch (a scheduling
 * parameter; the paper has no counterpart; synthpix_autotune below tunes an
 * edge per frame size class and more, and caches the result).  Renders the
 * batch with each candidate edge (16, 32, 64, 128; edges whose shared memory
 * does not fit the blur radius are skipped):
 * once to warm up, then `reps` (1..1000) timed times on `stream`, timed with
 * CUDA events, and returns the fastest edge in *best_tile and its mean time
 * per render in *best_ms (nullable).  The images are overwritten.  The
 * workspace must hold synthpix_workspace_bytes for batch->tile = 0.  Unlike
 * the other entry points this call BLOCKS the host until the timings are
 * done.  Results never depend on the tile edge (exact accumulation), only
 * the speed does.
 */
int synthpix_autotune_tile(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                           const synthpix_pair_desc *pairs_dev, int32_t n_pairs,
                           const float *flows, void *images,
                           void *workspace, size_t workspace_bytes, void *stream,
                           int32_t reps, int32_t *best_tile, float *best_ms);

/*
 * Launch parameters of a render (a scheduling choice; the paper has no
 * counterpart beyond batching, Section 2 "Configuration file").  Results
 * never depend on them (exact fixed-point sums; every finishing path has the
 * same arithmetic), only the speed does.
 */
typedef struct synthpix_tuning {
    int32_t tile[4];            /* screen tile edge per frame size class, by frame area:
                                   < 2^15 pixels, < 2^17, < 2^19, larger; 16, 32, 64 or
                                   128, or 0 for a class the batch does not have          */
    int32_t records_per_stage;  /* round-particle records staged on chip per chunk of a tile */
    int32_t register_epilogue;  /* 1: full 128 x 128 tiles finish with the blur in
                                   registers; 0: with the shared-memory passes            */
    float   ms;                 /* mean time of one render (synthpix_autotune), else 0    */
    int32_t reserved[2];
} synthpix_tuning;

/*
 * Autotuner of the launch parameters (Section 2 / 3.3: batching amortises
 * overhead; the tile edges, records per stage and blur path are this
 * library's).  The batch must have tile = 0.  Starting from the default edges
 * (32, 64, 128, 128 by size class), it renders the batch with each candidate
 * edge of each size class present (the class with the most pixels first,
 * the others' best edges kept), then with each records-per-stage candidate,
 * then with the other epilogue path: once to warm up, then `reps` (1..1000)
 * timed times each on `stream` with CUDA events.  Candidates that do not fit
 * on chip (shared memory for the blur radius) are skipped.  The best
 * parameters are written to *out (nullable) and kept in a process-wide table
 * keyed by (frame size class, largest particle diameter in quarter pixels,
 * blur radius, general-shape splat, fused epilogue); every later render of a
 * batch with tile = 0 whose classes have entries uses them, with no timing.
 * The table is guarded by a mutex: renders, lookups and autotune calls may
 * come from any host thread.  The images are overwritten.  The workspace must
 * hold synthpix_workspace_bytes for the batch (tile = 0).  Unlike the render
 * entry points this call BLOCKS the host until its timings are done.
 */
int synthpix_autotune(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                      const synthpix_pair_desc *pairs_dev, int32_t n_pairs, const float *flows, void *images,
                      void *workspace, size_t workspace_bytes, void *stream, int32_t reps, synthpix_tuning *out);

/* The parameters a render of this batch runs with now (batch->tile, or the
   table's entries and the defaults for tile = 0); ms = 0.  No device call. */
int synthpix_tuning_lookup(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs, int32_t n_pairs,
                           synthpix_tuning *out);

/*
 * Writes parameters into the autotuner's table for this batch's classes
 * (tile = 0 batches), e.g. ones saved from an earlier process: the tile
 * edges of the classes present (others ignored), records_per_stage
 * (1..4096; more than the splat's staged-record region holds for the
 * largest edge, 1078 records at edge 128 and 822 below, gives
 * SYNTHPIX_EUNSUPPORTED) and register_epilogue (0 or 1); ms is ignored.  No
 * device call.
 */
int synthpix_tuning_set(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs, int32_t n_pairs,
                        const synthpix_tuning *tuning);

/* Empties the autotuner's table (renders fall back to the defaults). */
void synthpix_tuning_clear(void);

/* Message of the last failing call on this host thread ("" if none). */
const char *synthpix_last_error(void);

/*
 * Procedural flow fields on the device, for streaming renders (Section 2,
 * "Data loaders": flows may be supplied procedurally).  Writes n_flows
 * divergence-free fields to flows (device, float32 [n_flows][flow_h][flow_w]
 * [2], 8-byte aligned, caller-owned): field f is the curl of the stream
 * function psi = sum_m a_m sin(kx_m x + ky_m y + phi_m), u = d psi / dy,
 * v = -d psi / dx, at the cell-centred nodes ((l + 1/2) width / flow_w,
 * (k + 1/2) height / flow_h) of a height x width image, scaled so that
 * sqrt(mean(u^2 + v^2)) = rms (rms = 0 leaves the field unscaled).
 *   modes      device, 8-byte aligned, float64 [n_flows][n_modes][4]:
 *              (kx, ky, phi, a) per mode, k in radians per pixel;
 *   n_flows    1..65535; n_modes 1..256; sizes 1..32768;
 *   workspace  device, 256-byte aligned, at least
 *              synthpix_fourier_flows_workspace_bytes(...) bytes (per-mode
 *              cos / sin tables of the grid's columns and rows).
 * Angles are formed and reduced in FP64, their cos / sin tabulated in FP32;
 * the sums over the modes are FP32, the normalisation FP64.  Asynchronous on stream;
 * SYNTHPIX_EINVAL / SYNTHPIX_EWORKSPACE before any launch on bad arguments.
 */
size_t synthpix_fourier_flows_workspace_bytes(int32_t n_flows, int32_t n_modes, int32_t flow_h, int32_t flow_w);
int synthpix_fourier_flows(int32_t n_flows, int32_t n_modes, int32_t flow_h, int32_t flow_w, int32_t height,
                           int32_t width, const double *modes, float rms, float *flows, void *workspace,
                           size_t workspace_bytes, void *stream);

/*
 * Intensity-histogram matching of rendered frames (Section 2: generated
 * images are optionally adjusted to a user-specified intensity histogram).
 * Acts in place on quantised outputs (batch->out_dtype U8 or U16 with
 * quant_bits b, n_codes = 2^b codes); every frame of the n_pairs pairs (two
 * per pair, at image_offset and image_offset + H W, as rendered) is matched
 * to the same target by histogram specification: with the frame's code
 * counts (N pixels) and the target counts (T in all, 0 < T < 2^64), code c
 * becomes the smallest t with C_t(t) N >= C_s(c) T (cumulative counts,
 * compared exactly); the mapping is monotone.
 *   images     device, the render's output buffer (element type out_dtype);
 *   target     device, 8-byte aligned, uint64 [n_codes] counts per code;
 *   workspace  device, 256-byte aligned, at least
 *              synthpix_match_histogram_workspace_bytes(...) bytes.
 * SYNTHPIX_EUNSUPPORTED for float outputs; asynchronous on stream (five
 * launches; the frame table is copied from host memory with
 * cudaMemcpyAsync).
 */
size_t synthpix_match_histogram_workspace_bytes(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                                                int32_t n_pairs);
int synthpix_match_histogram(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs, int32_t n_pairs,
                             void *images, const uint64_t *target, void *workspace, size_t workspace_bytes,
                             void *stream);

/* SYNTHPIX_ABI_VERSION of the loaded library. */
int synthpix_version(void);

/*
 * Kernel launches the library has issued in this process so far (all
 * threads and devices; a launch that returned an error is not counted).  For
 * measurement: the difference around a loop of calls is the number of the
 * library's kernels those calls launched.  The paper has no counterpart.
 */
uint64_t synthpix_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* SYNTHPIX_H */
