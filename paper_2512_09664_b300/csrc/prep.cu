// sm_103a kernels of the PIV image-pair renderer (SynthPix, arXiv 2512.09664,
// Section 2) that prepare the splat.  One batch is rendered by a fixed
// sequence of launches.  Seeded renders of round particles, with
// fixed-capacity bins:
//
//   k_plan         per-pair prefix sums of particles, tiles and bin slots,
//                  blur taps, the work-queue ticket; clears the bin counters
//   k_seed_place   Philox attributes of every particle, split positions, the
//                  per-particle advection, and both frames' records placed
//                  into the fixed bins
//   k_rebin        a CTA per (pair, frame); only after a bin of that frame
//                  overflowed: the exact binning
//   k_splat        (splat.cuh) persistent CTAs over the work items
//
// With SYNTHPIX_FLAG_TILED_ADVECT, k_seed_place places frame 1 only, then
// k_rebin (frame 1), k_advect (advects each frame-1 tile's home particles
// from a flow window in shared memory and places the frame-2 records) and
// k_rebin (frame 2).
//
// Renders that need each particle's index when its frame-2 record is made
// (given particles, per-frame shapes) advect per particle and bin both frames
// by a counting sort: k_plan, k_seed_advect (attributes, advection, counts),
// k_scan (offsets and work items), k_scatter, k_splat.
//
// No kernel waits on another CTA, spins, traps or asserts.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "particle.cuh"

namespace spx {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// k_plan: per-pair prefix sums (CTA 0, 1024 threads); the next CTAs clear
// the bin counts of a render; then CTAs that form the FP64 blur taps, four
// pairs each, a tap per lane (FP64 is slow on this part: spread over SMs and
// lanes, off CTA 0's path); the last ones, when the batch's flow grids are
// small enough to stay in L2 (single pairs, small batches), ask the L2 to
// fetch them with bulk prefetches, so that the dependent flow gathers of the
// per-particle advection that follows hit L2 instead of waiting on DRAM.
// ---------------------------------------------------------------------------
constexpr int kPlanZeroWords = 16384;
constexpr int kTapLanes = 8;                  // lanes per pair of the blur-tap CTAs
constexpr int kPlanTapPairs = 32 / kTapLanes;  // pairs per blur-tap CTA (one warp each: FP64 spread over SMs)

__global__ void __launch_bounds__(1024) k_plan(const synthpix_pair_desc *__restrict__ descs, int32_t n_pairs,
                                               TileRule rule, int32_t fused, PairPlan *__restrict__ plan,
                                               int64_t want_part, int64_t want_tiles, int64_t want_list,
                                               int64_t want_inter, int64_t want_chunks, int32_t *__restrict__ check,
                                               float *__restrict__ blur_w, uint32_t *__restrict__ ticket,
                                               uint32_t *__restrict__ count, int64_t n_count, int32_t zero_ctas,
                                               const float *__restrict__ pf_flows, int32_t pf_planes) {
    const int tap_ctas = (n_pairs + kPlanTapPairs - 1) / kPlanTapPairs;
    if ((int)blockIdx.x > zero_ctas + tap_ctas) {  // L2 prefetch of pair b's flow grid
        const int b = (int)blockIdx.x - 1 - zero_ctas - tap_ctas;
        const synthpix_pair_desc &d = descs[b];
        // the grid's bytes from its first 16-byte boundary to its last one
        const uintptr_t p0 = ((uintptr_t)(pf_flows + d.flow_offset) + 15) & ~(uintptr_t)15;
        const uintptr_t p1 = (uintptr_t)(pf_flows + d.flow_offset + (int64_t)pf_planes * d.flow_h * d.flow_w) &
                             ~(uintptr_t)15;
        for (uintptr_t p = p0 + (uintptr_t)threadIdx.x * kPrefetchPieceBytes; p < p1;
             p += (uintptr_t)blockDim.x * kPrefetchPieceBytes) {
            const uint32_t n = (uint32_t)min((uintptr_t)kPrefetchPieceBytes, p1 - p);  // a multiple of 16
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(n) : "memory");
        }
        return;
    }
    if (blockIdx.x > 0 && (int)blockIdx.x <= zero_ctas) {  // clear the bin counts, 16 Ki words per CTA
        const int64_t k0 = ((int64_t)blockIdx.x - 1) * kPlanZeroWords;
        const int64_t n = min((int64_t)kPlanZeroWords, n_count - k0);
        for (int64_t k = threadIdx.x; k < n; k += blockDim.x) count[k0 + k] = 0u;
        return;
    }
    if (blockIdx.x > 0) {  // normalised blur taps w[|k|], k = -R..R (FP64, stored FP32)
        // kPlanTapPairs pairs per CTA, a group of kTapLanes lanes of warp 0 per pair: lane k
        // evaluates w[k] (R < kTapLanes; larger radii: the group's first lane evaluates them in
        // turn), every lane of the group sums them in the order k = 0..R
        if (threadIdx.x >= 32) return;
        const int q = (int)threadIdx.x / kTapLanes, k = (int)threadIdx.x % kTapLanes;
        const int b = ((int)blockIdx.x - 1 - zero_ctas) * kPlanTapPairs + q;
        const int32_t R = b < n_pairs ? blur_radius_of(descs[b].blur_sigma) : 0;
        const unsigned grp = ((1u << kTapLanes) - 1u) << (q * kTapLanes);
        if (R == 0) return;  // the whole group
        const double sb = (double)descs[b].blur_sigma;
        if (R < kTapLanes) {
            const double wk = k <= R ? exp(-(double)(k * k) / (2.0 * sb * sb)) : 0.0;
            double sum = 0.0;
            for (int j = 0; j <= R; ++j) {
                const double v = __shfl_sync(grp, wk, q * kTapLanes + j);
                sum += j ? 2.0 * v : v;
            }
            if (k <= R) blur_w[b * kBlurStride + k] = (float)(wk / sum);
        } else if (k == 0) {
            double w[kMaxBlurRadius + 1], sum = 0.0;
            for (int j = 0; j <= R; ++j) {
                w[j] = exp(-(double)(j * j) / (2.0 * sb * sb));
                sum += j ? 2.0 * w[j] : w[j];
            }
            for (int j = 0; j <= R; ++j) blur_w[b * kBlurStride + j] = (float)(w[j] / sum);
        }
        return;
    }
    // block scan of five per-thread sums: inclusive scans within each warp by
    // shuffles, the warps' totals scanned by warp 0, two barriers in all
    __shared__ long long s_w[5][32];
    __shared__ long long s_tot[5];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int per = (n_pairs + 1023) / 1024;
    const int b0 = min(t * per, n_pairs), b1 = min(b0 + per, n_pairs);
    long long v[5] = {0, 0, 0, 0, 0};  // particles, tiles, bin slots, intermediate elements, chunks
    for (int b = b0; b < b1; ++b) {
        const synthpix_pair_desc d = descs[b];
        const PairGeom g = pair_geom(d, rule_tile(rule, d), fused != 0);
        v[0] += d.n_particles;
        v[1] += 2LL * g.ntiles;
        v[2] += 2LL * g.list_cap;
        v[3] += fused ? 0LL : 2LL * d.height * d.width;
        v[4] += g.chunks;
    }
    long long inc[5];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        inc[j] = v[j];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const long long o = __shfl_up_sync(0xffffffffu, inc[j], d);
            if (lane >= d) inc[j] += o;
        }
        if (lane == 31) s_w[j][warp] = inc[j];
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int j = 0; j < 5; ++j) {
            long long x = s_w[j][lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const long long o = __shfl_up_sync(0xffffffffu, x, d);
                if (lane >= d) x += o;
            }
            s_w[j][lane] = x - s_w[j][lane];  // exclusive offset of each warp
            if (lane == 31) s_tot[j] = x;
        }
    }
    __syncthreads();
    long long bp = s_w[0][warp] + inc[0] - v[0], bt = s_w[1][warp] + inc[1] - v[1];
    long long bl = s_w[2][warp] + inc[2] - v[2], bi = s_w[3][warp] + inc[3] - v[3];
    long long bc = s_w[4][warp] + inc[4] - v[4];
    for (int b = b0; b < b1; ++b) {
        const synthpix_pair_desc d = descs[b];
        const int32_t tile = rule_tile(rule, d);
        const PairGeom g = pair_geom(d, tile, fused != 0);
        PairPlan p;
        p.part_base = bp;
        p.list_base = bl;
        p.list_cap = g.list_cap;
        p.inter_base = bi;
        p.tile_base = (int32_t)bt;
        p.tiles_x = g.tiles_x;
        p.tiles_y = g.tiles_y;
        p.ntiles = g.ntiles;
        p.blur_r = g.blur_r;
        p.halo = g.halo;
        p.chunk_base = (int32_t)bc;
        p.tile = tile;
        plan[b] = p;
        bp += d.n_particles;
        bt += 2LL * g.ntiles;
        bl += 2LL * g.list_cap;
        bi += fused ? 0LL : 2LL * d.height * d.width;
        bc += g.chunks;
    }
    if (t == 1023) {
        ticket[0] = 0u;  // the splat's work queue
        ticket[1] = 0u;  // overflow flags of the fixed bins (frames 1, 2)
        ticket[2] = 0u;
        const bool ok = s_tot[0] == want_part && s_tot[1] == want_tiles && s_tot[2] == want_list &&
                        s_tot[3] == want_inter && s_tot[4] == want_chunks;
        *check = ok ? 1 : 0;
    }
}

// ---------------------------------------------------------------------------
// One CTA per chunk of kChunk consecutive particles of one pair (seeding and
// binning): the pair's descriptor and plan are read once into shared memory,
// and per-(frame, tile) counts are aggregated in shared memory, so each CTA
// makes one global atomic per tile it touches instead of one per particle.
// ---------------------------------------------------------------------------
constexpr int kPrepThreads = 256;
constexpr int kHistMax = 2048;  // (frame, tile) counters of a pair held on chip; larger pairs count in global

struct ChunkCtx {
    synthpix_pair_desc d;
    PairPlan pl;
    int32_t pair;
    int32_t first;  // first particle of the chunk within the pair
    int32_t n;      // particles in the chunk
};

// The chunk of this CTA: pair (largest b with chunk_base(b) <= blockIdx.x),
// descriptor and plan in shared memory.  Ends with a barrier.
__device__ __forceinline__ void load_chunk(const KernelArgs &a, ChunkCtx &c) {
    const int b = block_upper_find(a.n_pairs, (int64_t)blockIdx.x, [&](int m) { return (int64_t)a.plan[m].chunk_base; });
    constexpr int kD = sizeof(synthpix_pair_desc) / 16, kP = sizeof(PairPlan) / 16;
    if (threadIdx.x < kD)
        reinterpret_cast<int4 *>(&c.d)[threadIdx.x] = reinterpret_cast<const int4 *>(a.descs + b)[threadIdx.x];
    else if (threadIdx.x < kD + kP)
        reinterpret_cast<int4 *>(&c.pl)[threadIdx.x - kD] = reinterpret_cast<const int4 *>(a.plan + b)[threadIdx.x - kD];
    __syncthreads();
    if (threadIdx.x == 0) {
        c.pair = b;
        c.first = (int32_t)(((int64_t)blockIdx.x - c.pl.chunk_base) * kChunk);
        c.n = (int32_t)min((int64_t)kChunk, (int64_t)c.d.n_particles - c.first);
    }
    __syncthreads();
}

// Bin counts of one frame's window: into the on-chip histogram, or global.
__device__ __forceinline__ void count_window(const KernelArgs &a, const ChunkCtx &c, const Window &w, int f,
                                             uint32_t *hist) {
    if (w.j0 > w.j1 || w.i0 > w.i1) return;
    int32_t tx0, tx1, ty0, ty1;
    window_tiles(w, c.pl.halo, c.pl.tile, c.d.width, c.d.height, tx0, tx1, ty0, ty1);
    const int32_t k0 = f * c.pl.ntiles;
    for (int32_t ty = ty0; ty <= ty1; ++ty)
        for (int32_t tx = tx0; tx <= tx1; ++tx) {
            const int32_t k = k0 + ty * c.pl.tiles_x + tx;
            if (hist) atomicAdd(hist + k, 1u);
            else atomicAdd(a.count + c.pl.tile_base + k, 1u);
        }
}

// ---------------------------------------------------------------------------
// k_seed_advect: Philox attributes, frame-1 position, advection to frame 2,
// split positions and bin counts (export only: writes (x, y, d) of frame 1
// or, advected, of frame 2)
// ---------------------------------------------------------------------------
// CACHE: the flow lookups of the per-particle advection keep the last grid
// cell's nodes in registers (GridVelocity), with the register room of three
// CTAs per SM (at five per SM the cache spilled).  Used by the renders that
// advect per particle and by the adjoint's positions; the export of
// particle positions keeps the five-CTA variant.
template <bool CACHE>
__global__ void __launch_bounds__(kPrepThreads, CACHE ? 3 : 5) k_seed_advect(KernelArgs a) {
    if (*a.check != 1) return;
    __shared__ __align__(16) ChunkCtx c;
    __shared__ uint32_t hist[kHistMax];
    load_chunk(a, c);
    const int nk = 2 * c.pl.ntiles;
    const bool counting = a.count != nullptr && !a.particles_out;
    const bool local = counting && nk <= kHistMax;
    if (local) {
        for (int k = threadIdx.x; k < nk; k += kPrepThreads) hist[k] = 0u;
        __syncthreads();
    }
    const Flow F = pair_flow(a, c.d);
    for (int q = threadIdx.x; q < c.n; q += kPrepThreads) {
        const uint32_t i = (uint32_t)(c.first + q);
        const int64_t g = c.pl.part_base + i;
        const Seeded P = seed_particle(a, c.d, i, g);
        a.sa[g] = make_float2(P.sigma, P.amp);
        a.pos0[g] = make_float4(P.fx, P.fy, __int_as_float(P.ix), __int_as_float(P.iy));
        if (a.particles_out) {
            int32_t jx = P.ix, jy = P.iy;
            float gx = P.fx, gy = P.fy;
            if (a.export_frame) advect_split(F, a.dt, a.n_substeps, a.integrator, jx, gx, jy, gy);
            // the split position rounded once to FP32; d = 4 sigma exactly
            a.particles_out[3 * g] = (float)jx + gx;
            a.particles_out[3 * g + 1] = (float)jy + gy;
            a.particles_out[3 * g + 2] = 4.0f * P.sigma;
            continue;
        }
        // frame 2 here unless the tiled advection (k_advect) makes it
        int32_t jx = P.ix, jy = P.iy;
        float gx = P.fx, gy = P.fy, z2 = P.z;
        if (!a.tiled) {
            if (a.out_of_plane)
                advect_split_z(F, a.flows + c.d.flow_offset + 2LL * c.d.flow_h * c.d.flow_w, a.dt, a.n_substeps,
                               a.integrator, jx, gx, jy, gy, z2);
            else if (a.states) {  // each substep's start kept for the adjoint (the same arithmetic)
                float4 *sp = a.states + g * a.n_substeps;
                const float h = a.dt / (float)a.n_substeps;
                if constexpr (CACHE) {
                    GridVelocity vel(F);  // its cached cell carries over the substeps
                    for (int s = 0; s < a.n_substeps; ++s) {
                        sp[s] = make_float4(gx, gy, __int_as_float(jx), __int_as_float(jy));
                        advect_split_with(vel, h, 1, a.integrator, jx, gx, jy, gy);
                    }
                } else {
                    for (int s = 0; s < a.n_substeps; ++s) {
                        sp[s] = make_float4(gx, gy, __int_as_float(jx), __int_as_float(jy));
                        advect_split(F, h, 1, a.integrator, jx, gx, jy, gy);
                    }
                }
            } else {
                if constexpr (CACHE) advect_split_with(GridVelocity(F), a.dt, a.n_substeps, a.integrator, jx, gx, jy, gy);
                else advect_split(F, a.dt, a.n_substeps, a.integrator, jx, gx, jy, gy);
            }
            a.pos1[g] = make_float4(gx, gy, __int_as_float(jx), __int_as_float(jy));
        }
        // window half-extents 1.5 d (x) and 1.5 d_y (y) of each frame; < 0: hidden
        float r1x = 6.0f * P.sigma, r1y = r1x, r2x = r1x, r2y = r1x;
        if (a.ext) {
            float4 s1, s2;
            frame_shapes(a, c.d, i, P, a.out_of_plane ? sheet_gain(c.d, z2) : P.gain, s1, s2);
            a.shape[g] = s1;
            a.shape[a.n_part + g] = s2;
            r1x = 6.0f * s1.x;
            r1y = 6.0f * s1.y;
            r2x = 6.0f * s2.x;
            r2y = 6.0f * s2.y;
        }
        if (counting && r1x >= 0.0f)
            count_window(a, c, particle_window2(P.ix, P.fx, P.iy, P.fy, r1x, r1y, c.d.width, c.d.height), 0,
                         local ? hist : nullptr);
        if (!a.tiled && counting && r2x >= 0.0f)
            count_window(a, c, particle_window2(jx, gx, jy, gy, r2x, r2y, c.d.width, c.d.height), 1,
                         local ? hist : nullptr);
    }
    if (local) {
        __syncthreads();
        for (int k = threadIdx.x; k < nk; k += kPrepThreads)
            if (hist[k]) atomicAdd(a.count + c.pl.tile_base + k, hist[k]);
    }
}

// ---------------------------------------------------------------------------
// k_seed_place (seeded renders with fixed bins): k_seed_advect's seeding
// with the records binned in the same pass (frame 1, or both frames with the
// advection).  A CTA counts its chunk's records per tile on chip, reserves
// each tile's range of the tile's fixed bin with one global atomic (the bin
// counters count every record), and places its records.  Records past a bin's capacity are dropped and
// flag the frame for k_rebin.  The split positions and sigma / amplitude
// are still written (k_rebin's input).  The first chunk of each pair writes
// the pair's work items of the fixed layout.
// ---------------------------------------------------------------------------
// Record r at slot `slot` of the fixed bin of tile k of frame f of a pair
// (bin capacity cap), or the frame's overflow flag.
__device__ __forceinline__ void place_fixed(const KernelArgs &a, const PairPlan &pl, int f, int32_t k, int64_t cap,
                                            uint32_t slot, const Record &r) {
    if ((int64_t)slot >= cap) {
        a.ovf[f] = 1u;
        return;
    }
    float2 *o = reinterpret_cast<float2 *>(a.rec + pl.list_base + (int64_t)f * pl.list_cap + (int64_t)k * cap + slot);
    o[0] = make_float2(r.fx, r.fy);
    o[1] = make_float2(__int_as_float(r.ix), __int_as_float(r.iy));
    o[2] = make_float2(r.sigma, r.amp);
}

// ADV (a.tiled == 2): each particle is also advected here, through the
// flow grid with the last cell's nodes in registers (GridVelocity), and
// both frames' records are placed: frame 2 follows frame 1 on the counters
// and bins; the frame-2 positions go to pos1 (the exact rebinning's input).
// The advection waits on flow gathers.  NT = 256 (two particles a thread,
// four CTAs per SM) for batches of more chunks than fill the GPU in one
// wave (measured: 100 us for the 64-pair 512 x 512 batch, against 117 us at
// three CTAs per SM and 114 us with NT = 512; five and six CTAs per SM
// gained nothing); NT = 512 (a particle a thread: half the dependent lookups
// of a lane) for smaller batches (the single 256 x 256 pair 45.1 -> 37.1 us).
template <bool ADV, int NT>
__global__ void __launch_bounds__(NT, NT == 512 ? 2 : 4) k_seed_place(KernelArgs a) {
    static_assert(kChunk % NT == 0, "whole particles per thread");
    if (*a.check != 1) return;
    __shared__ __align__(16) ChunkCtx c;
    __shared__ uint32_t cnt[kHistMax], base[kHistMax];
    load_chunk(a, c);
    const int nk = c.pl.ntiles;
    constexpr int NF = ADV ? 2 : 1;  // frames placed here
    const bool local = NF * nk <= kHistMax;
    int64_t cap1, cap2;
    fixed_caps(c.d, c.pl.tile, c.pl.halo, cap1, cap2);
    if ((int64_t)blockIdx.x == c.pl.chunk_base) {  // the pair's work items (fixed layout)
        for (int k = threadIdx.x; k < 2 * nk; k += NT) {
            ItemInfo it;
            it.pair = c.pair;
            it.frame = k >= nk ? 1 : 0;
            it.tile = k - it.frame * nk;
            const int64_t cap = it.frame ? cap2 : cap1;
            it.count = (uint32_t)cap;
            it.rec0 = c.pl.list_base + (int64_t)it.frame * c.pl.list_cap + (int64_t)it.tile * cap;
            a.items[c.pl.tile_base + k] = it;
        }
    }
    if (local) {
        for (int k = threadIdx.x; k < NF * nk; k += NT) cnt[k] = 0u;
        __syncthreads();
    }
    uint32_t *cnt1 = a.count + c.pl.tile_base;  // frame f's counter of tile k at f nk + k
    const int W = c.d.width, H = c.d.height;
    auto tiles_of = [&](const Record &r, int32_t &tx0, int32_t &tx1, int32_t &ty0, int32_t &ty1) {
        const Window w = particle_window(r.ix, r.fx, r.iy, r.fy, 6.0f * r.sigma, W, H);
        if (w.j0 > w.j1 || w.i0 > w.i1) return false;
        window_tiles(w, c.pl.halo, c.pl.tile, W, H, tx0, tx1, ty0, ty1);
        return true;
    };
    constexpr int U = kChunk / NT;
    // without the advection the records stay in registers between the count
    // and the placement; with it they are read back from pos0 / pos1 / sa
    // (written just before by the same thread), which frees the registers
    // across the advection for more resident CTAs
    constexpr int UK = ADV ? 1 : U;
    Record rk[UK];
    const Flow F = pair_flow(a, c.d);
    auto count_or_place = [&](int f, const Record &r, bool place, const uint32_t *at) {
        int32_t tx0, tx1, ty0, ty1;
        if (!tiles_of(r, tx0, tx1, ty0, ty1)) return;
        for (int32_t ty = ty0; ty <= ty1; ++ty)
            for (int32_t tx = tx0; tx <= tx1; ++tx) {
                const int32_t k = f * nk + ty * c.pl.tiles_x + tx;
                if (!place) atomicAdd(cnt + k, 1u);
                else place_fixed(a, c.pl, f, k - f * nk, f ? cap2 : cap1,
                                 (at ? at[k] + atomicAdd(cnt + k, 1u) : atomicAdd(cnt1 + k, 1u)), r);
            }
    };
#pragma unroll (ADV ? 1 : U)
    for (int u = 0; u < U; ++u) {
        const int q = threadIdx.x + u * NT;
        if constexpr (!ADV) rk[u].sigma = -1.0f;
        if (q >= c.n) continue;
        const uint32_t i = (uint32_t)(c.first + q);
        const int64_t g = c.pl.part_base + i;
        const Seeded P = seed_particle(a, c.d, i, g);
        a.sa[g] = make_float2(P.sigma, P.amp);
        a.pos0[g] = make_float4(P.fx, P.fy, __int_as_float(P.ix), __int_as_float(P.iy));
        const Record r0{P.fx, P.fy, P.ix, P.iy, P.sigma, P.amp};
        if constexpr (!ADV) rk[u] = r0;
        count_or_place(0, r0, !local, nullptr);
        if constexpr (ADV) {
            int32_t jx = P.ix, jy = P.iy;
            float gx = P.fx, gy = P.fy;
            advect_split_with(GridVelocity(F), a.dt, a.n_substeps, a.integrator, jx, gx, jy, gy);
            a.pos1[g] = make_float4(gx, gy, __int_as_float(jx), __int_as_float(jy));
            count_or_place(1, Record{gx, gy, jx, jy, P.sigma, P.amp}, !local, nullptr);
        }
    }
    if (!local) return;
    __syncthreads();
    for (int k = threadIdx.x; k < NF * nk; k += NT) {
        const uint32_t n = cnt[k];
        base[k] = n ? atomicAdd(cnt1 + k, n) : 0u;
        cnt[k] = 0u;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if constexpr (ADV) {
            const int q = threadIdx.x + u * NT;
            if (q >= c.n) continue;
            const int64_t g = c.pl.part_base + (uint32_t)(c.first + q);
            const float2 sa = a.sa[g];
            const float4 p0 = a.pos0[g], p1 = a.pos1[g];
            count_or_place(0, Record{p0.x, p0.y, __float_as_int(p0.z), __float_as_int(p0.w), sa.x, sa.y}, true, base);
            count_or_place(1, Record{p1.x, p1.y, __float_as_int(p1.z), __float_as_int(p1.w), sa.x, sa.y}, true, base);
        } else {
            if (rk[u].sigma < 0.0f) continue;
            count_or_place(0, rk[u], true, base);
        }
    }
}

// ---------------------------------------------------------------------------
// k_scan: exclusive scan of the bin counts of one (pair, frame) per CTA
// ---------------------------------------------------------------------------
// Offsets, cursors and work items of the bins of pair b, frame f, by the
// 1024 threads of a CTA.  Contains barriers.
__device__ __forceinline__ void scan_pair(const KernelArgs &a, int b, int f) {
    __shared__ uint32_t s[1024];
    __shared__ uint32_t carry;
    const PairPlan pl = a.plan[b];
    const int64_t base = pl.tile_base + (int64_t)f * pl.ntiles;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int32_t c0 = 0; c0 < pl.ntiles; c0 += 1024) {
        const int32_t t = c0 + threadIdx.x;
        const uint32_t v = t < pl.ntiles ? a.count[base + t] : 0u;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            const uint32_t add = threadIdx.x >= off ? s[threadIdx.x - off] : 0u;
            __syncthreads();
            s[threadIdx.x] += add;
            __syncthreads();
        }
        const uint32_t excl = carry + s[threadIdx.x] - v;
        if (t < pl.ntiles) {
            a.off[base + t] = excl;
            a.cursor[base + t] = excl;
            ItemInfo it;
            it.pair = b;
            it.frame = f;
            it.tile = t;
            // a bin never exceeds its segment; clamped for memory safety
            const int64_t room = pl.list_cap - (int64_t)excl;
            it.count = (uint32_t)max((int64_t)0, min((int64_t)v, room));
            it.rec0 = pl.list_base + (int64_t)f * pl.list_cap + excl;
            a.items[base + t] = it;
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_scan(KernelArgs a, int frame) {
    if (*a.check != 1) return;
    const int b = frame < 0 ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;
    const int f = frame < 0 ? (int)(blockIdx.x & 1) : frame;
    scan_pair(a, b, f);
}

// ---------------------------------------------------------------------------
// k_scatter: particle records into their tiles' bins (order within a bin is
// free: the splat accumulates in exact fixed point, so sums are
// order-independent).  On chip: count the chunk's records per tile, reserve
// each tile's range with one global atomic, then place the records.
// ---------------------------------------------------------------------------
// put(f, k, p, sh) for each bin k of frame f a particle's window meets; sh =
// (sigma_x, sigma_y, rho, amplitude) of the frame (hidden particles skipped).
template <typename Put>
__device__ __forceinline__ void chunk_windows(const KernelArgs &a, const ChunkCtx &c, int nf, Put put) {
    constexpr int U = kChunk / kPrepThreads;  // particles of the chunk per thread
    static_assert(U * kPrepThreads == kChunk, "whole particles per thread");
    // every particle's loads are issued before any is binned (U requests in flight)
    int64_t g[U];
    bool v[U];
    float4 sh[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        g[u] = c.pl.part_base + c.first + threadIdx.x + u * kPrepThreads;
        v[u] = (int)threadIdx.x + u * kPrepThreads < c.n;
        sh[u] = make_float4(-1.0f, 0.0f, 0.0f, 0.0f);
        if (!a.ext && v[u]) {
            const float2 sa = a.sa[g[u]];
            sh[u] = make_float4(sa.x, sa.x, 0.0f, sa.y);
        }
    }
    for (int f = 0; f < nf; ++f) {
        const float4 *pos = f ? a.pos1 : a.pos0;
        float4 p[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (a.ext) {
                sh[u].x = -1.0f;
                if (v[u]) sh[u] = a.shape[f * a.n_part + g[u]];
            }
            p[u] = v[u] ? pos[g[u]] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (sh[u].x < 0.0f) continue;  // outside the chunk, or hidden from this frame
            const Window w = particle_window2(__float_as_int(p[u].z), p[u].x, __float_as_int(p[u].w), p[u].y,
                                              6.0f * sh[u].x, 6.0f * sh[u].y, c.d.width, c.d.height);
            if (w.j0 > w.j1 || w.i0 > w.i1) continue;
            int32_t tx0, tx1, ty0, ty1;
            window_tiles(w, c.pl.halo, c.pl.tile, c.d.width, c.d.height, tx0, tx1, ty0, ty1);
            for (int32_t ty = ty0; ty <= ty1; ++ty)
                for (int32_t tx = tx0; tx <= tx1; ++tx)
                    put(f, f * c.pl.ntiles + ty * c.pl.tiles_x + tx, p[u], sh[u]);
        }
    }
}

// One bin record: 24 bytes (Record) for round particles, 32 (RecordG) for
// the general-shape splat.
__device__ __forceinline__ void put_record(const KernelArgs &a, const ChunkCtx &c, int f, uint32_t slot,
                                           const float4 &p, const float4 &sh) {
    if ((int64_t)slot < c.pl.list_cap) {
        const int64_t k = c.pl.list_base + (int64_t)f * c.pl.list_cap + slot;
        if (a.general) {
            float4 *r = reinterpret_cast<float4 *>(reinterpret_cast<RecordG *>(a.rec) + k);
            r[0] = p;
            r[1] = sh;
        } else {
            float2 *r = reinterpret_cast<float2 *>(a.rec + k);
            r[0] = make_float2(p.x, p.y);
            r[1] = make_float2(p.z, p.w);
            r[2] = make_float2(sh.x, sh.w);
        }
    }
}

__global__ void __launch_bounds__(kPrepThreads) k_scatter(KernelArgs a) {
    if (*a.check != 1) return;
    __shared__ __align__(16) ChunkCtx c;
    __shared__ uint32_t cnt[kHistMax], base[kHistMax];
    load_chunk(a, c);
    const int nf = 2;  // (renders without the tiled advection) both frames
    const int nk = nf * c.pl.ntiles;
    uint32_t *cursor = a.cursor + c.pl.tile_base;
    if (nk > kHistMax) {
        chunk_windows(a, c, nf, [&](int f, int k, const float4 &p, const float4 &sh) {
            put_record(a, c, f, atomicAdd(cursor + k, 1u), p, sh);
        });
        return;
    }
    for (int k = threadIdx.x; k < nk; k += kPrepThreads) cnt[k] = 0u;
    __syncthreads();
    chunk_windows(a, c, nf, [&](int, int k, const float4 &, const float4 &) { atomicAdd(cnt + k, 1u); });
    __syncthreads();
    for (int k = threadIdx.x; k < nk; k += kPrepThreads) {
        const uint32_t n = cnt[k];
        base[k] = n ? atomicAdd(cursor + k, n) : 0u;
        cnt[k] = 0u;
    }
    __syncthreads();
    chunk_windows(a, c, nf, [&](int f, int k, const float4 &p, const float4 &sh) {
        put_record(a, c, f, base[k] + atomicAdd(cnt + k, 1u), p, sh);
    });
}

// ---------------------------------------------------------------------------
// Tiled advection (seeded renders): one CTA per frame-1 tile.  The flow-grid
// nodes under the tile and a margin are staged into shared memory with
// coalesced 8-byte loads; the tile's home particles (integer position inside
// the tile, so each particle once) are advected from it, lookups that leave
// the window read global memory.  Frame-2 records go to adv (by frame-1 bin
// slot: k_rebin's input after an overflow) and, counted on chip for the tiles
// near the home tile, into those tiles' fixed frame-2 bins.
// ---------------------------------------------------------------------------
constexpr int kAdvMargin = 2;  // image pixels of flow staged beyond the tile on each side (measured best)
constexpr int kNbr = 3;        // on-chip counters for frame-2 tiles within +-kNbr of the home tile
constexpr int kNbrSide = 2 * kNbr + 1;
constexpr int kAdvBatch = 2048;  // records of a bin examined per pass (home list in shared memory)

// A tile's advection is split into adv_bands(tile) row bands, one CTA each
// (two at tile 128, so that two CTAs with their flow windows fit on an SM).
__host__ __device__ inline int adv_bands(int tile) { return tile >= 128 ? 2 : 1; }
__host__ __device__ inline int adv_window_nodes(int tile) {
    const int band = (tile + adv_bands(tile) - 1) / adv_bands(tile);
    return (tile + 2 * kAdvMargin + 2) * (band + 2 * kAdvMargin + 2);
}

struct TileCtx {
    int32_t b, t, tx, ty, x0, x1, y0, y1;
    ItemInfo it;
    int64_t adv0;  // first adv slot of the tile's frame-1 bin
};

// Frame-1 tile gt (over all pairs' frame-1 tiles) of pair b.
__device__ __forceinline__ TileCtx frame1_tile(const KernelArgs &a, const PairPlan &pl, int b, int W, int H,
                                               int64_t gt) {
    TileCtx c;
    c.b = b;
    c.t = (int32_t)(gt - (pl.tile_base >> 1));
    c.ty = c.t / pl.tiles_x;
    c.tx = c.t - c.ty * pl.tiles_x;
    c.x0 = c.tx * pl.tile;
    c.y0 = c.ty * pl.tile;
    c.x1 = min(c.x0 + pl.tile, W);
    c.y1 = min(c.y0 + pl.tile, H);
    c.it = work_item(a, pl.tile_base + c.t);  // the fixed layout's count, or the exact item
    c.adv0 = c.it.rec0 - (pl.list_base >> 1);
    return c;
}

__device__ __forceinline__ int frame1_pair(const KernelArgs &a, int64_t gt) {
    return block_upper_find(a.n_pairs, gt, [&](int m) { return (int64_t)(a.plan[m].tile_base >> 1); });
}

// Calls put(k, tile) for each frame-2 tile of advected record r; k = index of
// the on-chip counter, or -1 for a tile beyond the neighbourhood.
template <typename Put>
__device__ __forceinline__ void frame2_tiles(const KernelArgs &a, const PairPlan &pl, const TileCtx &c, const Record &r,
                                             int W, int H, Put put) {
    const Window w = particle_window(r.ix, r.fx, r.iy, r.fy, 6.0f * r.sigma, W, H);
    if (w.j0 > w.j1 || w.i0 > w.i1) return;
    int32_t tx0, tx1, ty0, ty1;
    window_tiles(w, pl.halo, pl.tile, W, H, tx0, tx1, ty0, ty1);
    for (int32_t ty = ty0; ty <= ty1; ++ty)
        for (int32_t tx = tx0; tx <= tx1; ++tx) {
            const int32_t dy = ty - c.ty + kNbr, dx = tx - c.tx + kNbr;
            const int k = ((unsigned)dy < (unsigned)kNbrSide && (unsigned)dx < (unsigned)kNbrSide) ? dy * kNbrSide + dx : -1;
            put(k, ty * pl.tiles_x + tx);
        }
}

// NT threads per CTA (256, or 512 at tile 128 with two 64-row bands: two CTAs
// per SM, the launch bounds keeping 64 registers), NB row bands per tile
// (blockIdx.x = NB tile + band).
template <int NT, int NB>
__global__ void __launch_bounds__(NT, 1024 / NT) k_advect(KernelArgs a) {
    if (*a.check != 1) return;
    extern __shared__ __align__(16) float2 s_flow[];
    __shared__ uint32_t s_nb[kNbrSide * kNbrSide], s_base[kNbrSide * kNbrSide];
    __shared__ uint16_t s_home[kAdvBatch];
    __shared__ uint32_t s_nhome;
    const int64_t gt = (int64_t)(blockIdx.x / NB);
    const int band = (int)(blockIdx.x - gt * NB);
    const int b = frame1_pair(a, gt);
    const PairPlan pl = a.plan[b];
    const synthpix_pair_desc &D = a.descs[b];
    const int W = D.width, H = D.height;
    const TileCtx c = frame1_tile(a, pl, b, W, H, gt);
    // this CTA's home rows [hy0, hy1): its band of the tile
    const int bh = (pl.tile + NB - 1) / NB;
    const int hy0 = min(c.y0 + band * bh, c.y1), hy1 = min(hy0 + bh, c.y1);
    const Flow F = pair_flow(a, D);
    // grid nodes under [x0 - M, x1 + M) x [hy0 - M, hy1 + M), bilinear neighbours included
    int32_t l0, l1, k0, k1;
    float t_;
    grid_coord(c.x0 - kAdvMargin, 0.0f, F.gw, F.W, l0, t_);
    grid_coord(c.x1 + kAdvMargin, 0.0f, F.gw, F.W, l1, t_);
    grid_coord(hy0 - kAdvMargin, 0.0f, F.gh, F.H, k0, t_);
    grid_coord(hy1 + kAdvMargin, 0.0f, F.gh, F.H, k1, t_);
    FlowWindow Wn;
    Wn.s = s_flow;
    Wn.sa = (uint32_t)__cvta_generic_to_shared(s_flow);
    Wn.gx0 = min(max(l0, 0), F.gw - 1);
    Wn.gy0 = min(max(k0, 0), F.gh - 1);
    Wn.nw = min(max(l1 + 1, 0), F.gw - 1) - Wn.gx0 + 1;
    Wn.nh = min(max(k1 + 1, 0), F.gh - 1) - Wn.gy0 + 1;
    if (Wn.nw * Wn.nh > adv_window_nodes(a.tile)) Wn.nw = Wn.nh = 0;  // finer grid than fits: all lookups global
    for (int i = threadIdx.x; i < kNbrSide * kNbrSide; i += NT) s_nb[i] = 0u;
    // a warp per row: consecutive lanes copy consecutive nodes (coalesced 8-byte
    // asynchronous copies, all in flight at once; waited for before the barrier below)
    for (int r = threadIdx.x >> 5; r < Wn.nh; r += NT / 32) {
        const float2 *src = F.f + (size_t)(Wn.gy0 + r) * F.gw + Wn.gx0;
        for (int q = threadIdx.x & 31; q < Wn.nw; q += 32) {
            const unsigned d = (unsigned)__cvta_generic_to_shared(s_flow + r * Wn.nw + q);
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src + q) : "memory");
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    uint32_t *cnt2 = a.count + pl.tile_base + pl.ntiles;
    const bool same_res = F.gw == F.W && F.gh == F.H;
    // fixed bins: each batch's frame-2 records are placed here (ranges of the
    // neighbourhood's bins reserved per batch, farther bins record by record)
    int64_t cap1, cap2;  // frame 1's capacity is not needed here
    fixed_caps(D, pl.tile, pl.halo, cap1, cap2);
    auto nb_tile = [&](int i) { return (c.ty + i / kNbrSide - kNbr) * pl.tiles_x + (c.tx + i % kNbrSide - kNbr); };
    for (uint32_t base = 0; base < c.it.count; base += kAdvBatch) {
        // compact this batch's home particles (integer position inside the band); particles
        // outside the tile are advected by their own home tile and marked here (by every
        // band, with the same value); those of the tile's other bands are left to them
        if (threadIdx.x == 0) s_nhome = 0u;
        __syncthreads();
        for (uint32_t k = base + threadIdx.x; k < min(c.it.count, base + kAdvBatch); k += NT) {
            const int2 ip = reinterpret_cast<const int2 *>(a.rec + c.it.rec0 + k)[1];
            if (ip.x < c.x0 || ip.x >= c.x1 || ip.y < c.y0 || ip.y >= c.y1)
                reinterpret_cast<float2 *>(a.adv + c.adv0 + k)[2] = make_float2(-1.0f, 0.0f);
            else if (ip.y >= hy0 && ip.y < hy1)
                s_home[atomicAdd(&s_nhome, 1u)] = (uint16_t)(k - base);
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");  // the flow window (overlapped with the compaction)
        __syncthreads();
        for (uint32_t h = threadIdx.x; h < s_nhome; h += NT) {
            const uint32_t k = base + s_home[h];
            const float2 *rp = reinterpret_cast<const float2 *>(a.rec + c.it.rec0 + k);
            const float2 p0 = rp[0], p1 = rp[1], p2 = rp[2];
            float2 *o = reinterpret_cast<float2 *>(a.adv + c.adv0 + k);
            Record r;
            r.fx = p0.x;
            r.fy = p0.y;
            r.ix = __float_as_int(p1.x);
            r.iy = __float_as_int(p1.y);
            r.sigma = p2.x;
            r.amp = p2.y;
            if (same_res)
                advect_split_with(TileVelocity(F, Wn), a.dt, a.n_substeps, a.integrator, r.ix, r.fx, r.iy, r.fy);
            else
                advect_split_with(
                    [&](int32_t ix, float fx, int32_t iy, float fy) { return velocity_windowed(F, Wn, ix, fx, iy, fy); },
                    a.dt, a.n_substeps, a.integrator, r.ix, r.fx, r.iy, r.fy);
            o[0] = make_float2(r.fx, r.fy);
            o[1] = make_float2(__int_as_float(r.ix), __int_as_float(r.iy));
            o[2] = make_float2(r.sigma, r.amp);
            frame2_tiles(a, pl, c, r, W, H, [&](int kk, int32_t tile) {
                if (kk >= 0) atomicAdd(s_nb + kk, 1u);
                else place_fixed(a, pl, 1, tile, cap2, atomicAdd(cnt2 + tile, 1u), r);
            });
        }
        __syncthreads();
        {  // reserve the neighbourhood's ranges, then place this batch's records there
            for (int i = threadIdx.x; i < kNbrSide * kNbrSide; i += NT) {
                const uint32_t n = s_nb[i];
                s_base[i] = n ? atomicAdd(cnt2 + nb_tile(i), n) : 0u;
                s_nb[i] = 0u;
            }
            __syncthreads();
            for (uint32_t h = threadIdx.x; h < s_nhome; h += NT) {
                // the record this thread advected above (read back: fewer registers across the integration)
                const uint32_t k = base + s_home[h];
                const float2 *rp = reinterpret_cast<const float2 *>(a.adv + c.adv0 + k);
                const float2 p0 = rp[0], p1 = rp[1], p2 = rp[2];
                Record r;
                r.fx = p0.x;
                r.fy = p0.y;
                r.ix = __float_as_int(p1.x);
                r.iy = __float_as_int(p1.y);
                r.sigma = p2.x;
                r.amp = p2.y;
                frame2_tiles(a, pl, c, r, W, H, [&](int kk, int32_t tile) {
                    if (kk >= 0) place_fixed(a, pl, 1, tile, cap2, s_base[kk] + atomicAdd(s_nb + kk, 1u), r);
                });
            }
            __syncthreads();
            // the next batch counts from zero (the barrier after its compaction orders this first)
            for (int i = threadIdx.x; i < kNbrSide * kNbrSide; i += NT) s_nb[i] = 0u;
        }
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");  // an empty bin never waited for the window
}

// ---------------------------------------------------------------------------
// k_rebin: after an overflow of a fixed bin of frame f (a.ovf[f]), the
// frame's bins are rebuilt in the exact layout, one CTA per pair: the scan
// of the bin counters (which counted every record), then every record placed
// at its bin's cursor.  Frame 1 from the seeded positions, frame 2 from the
// advected records of the frame-1 bins (tiled advection) or from the
// advected positions (advection in k_seed_place).  Without an overflow every
// CTA returns at once.
// ---------------------------------------------------------------------------
// f < 0: both frames in one launch, CTA f n_pairs + b (frame 2 independent
// of frame 1's bins: the advection inside the seeding kernel).
__global__ void __launch_bounds__(1024) k_rebin(KernelArgs a, int f) {
    int b = (int)blockIdx.x;
    if (f < 0) {
        f = b >= a.n_pairs ? 1 : 0;
        b -= f * a.n_pairs;
    }
    if (*a.check != 1 || a.ovf[f] == 0u) return;
    scan_pair(a, b, f);
    __syncthreads();  // the cursors written by this CTA
    const PairPlan pl = a.plan[b];
    const synthpix_pair_desc &D = a.descs[b];
    const int W = D.width, H = D.height;
    uint32_t *cursor = a.cursor + pl.tile_base + (int64_t)f * pl.ntiles;
    Record *seg = a.rec + pl.list_base + (int64_t)f * pl.list_cap;
    auto place = [&](int32_t tile, const Record &r) {
        const uint32_t slot = atomicAdd(cursor + tile, 1u);
        if ((int64_t)slot < pl.list_cap) {
            float2 *o = reinterpret_cast<float2 *>(seg + slot);
            o[0] = make_float2(r.fx, r.fy);
            o[1] = make_float2(__int_as_float(r.ix), __int_as_float(r.iy));
            o[2] = make_float2(r.sigma, r.amp);
        }
    };
    auto place_all = [&](const Record &r) {
        const Window w = particle_window(r.ix, r.fx, r.iy, r.fy, 6.0f * r.sigma, W, H);
        if (w.j0 > w.j1 || w.i0 > w.i1) return;
        int32_t tx0, tx1, ty0, ty1;
        window_tiles(w, pl.halo, pl.tile, W, H, tx0, tx1, ty0, ty1);
        for (int32_t ty = ty0; ty <= ty1; ++ty)
            for (int32_t tx = tx0; tx <= tx1; ++tx) place(ty * pl.tiles_x + tx, r);
    };
    if (f == 0 || a.tiled == 2) {
        const float4 *pos = f ? a.pos1 : a.pos0;
        for (uint32_t q = threadIdx.x; q < D.n_particles; q += blockDim.x) {
            const int64_t g = pl.part_base + q;
            const float4 p = pos[g];
            const float2 sa = a.sa[g];
            Record r;
            r.fx = p.x;
            r.fy = p.y;
            r.ix = __float_as_int(p.z);
            r.iy = __float_as_int(p.w);
            r.sigma = sa.x;
            r.amp = sa.y;
            place_all(r);
        }
        return;
    }
    for (int32_t t = 0; t < pl.ntiles; ++t) {  // the advected records of each frame-1 bin
        const ItemInfo it = work_item(a, pl.tile_base + t);
        const Record *adv = a.adv + (it.rec0 - (pl.list_base >> 1));
        for (uint32_t k = threadIdx.x; k < it.count; k += blockDim.x) {
            const float2 *rp = reinterpret_cast<const float2 *>(adv + k);
            const float2 p0 = rp[0], p1 = rp[1], p2 = rp[2];
            if (p2.x < 0.0f) continue;  // advected by another tile
            Record r;
            r.fx = p0.x;
            r.fy = p0.y;
            r.ix = __float_as_int(p1.x);
            r.iy = __float_as_int(p1.y);
            r.sigma = p2.x;
            r.amp = p2.y;
            place_all(r);
        }
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
cudaError_t launch_plan(const synthpix_pair_desc *descs, int32_t n_pairs, const TileRule &rule, int32_t fused,
                        PairPlan *plan, const Layout &L, int32_t *check, float *blur_w, uint32_t *ticket,
                        uint32_t *count, const float *pf_flows, int32_t pf_planes, cudaStream_t st) {
    const int64_t n_count = count ? L.n_tiles : 0;
    const int32_t zero_ctas = (int32_t)((n_count + kPlanZeroWords - 1) / kPlanZeroWords);
    const int32_t tap_ctas = (n_pairs + kPlanTapPairs - 1) / kPlanTapPairs;
    const int32_t pf_ctas = pf_flows ? n_pairs : 0;
    const unsigned grid = 1u + (unsigned)zero_ctas + (unsigned)tap_ctas + (unsigned)pf_ctas;
    return launch_kernel(k_plan, grid, 1024, 0, st, descs, n_pairs, rule, fused, plan, L.n_part, L.n_tiles, L.n_list,
                          L.n_inter, L.n_chunks, check, blur_w, ticket, count, n_count, zero_ctas, pf_flows, pf_planes);
}

cudaError_t launch_prep(const KernelArgs &a, cudaStream_t st, cudaEvent_t const *ev) {
    auto mark = [&](int k) {
        if (ev && ev[k]) cudaEventRecord(ev[k], st);
    };
    const unsigned nb = (unsigned)a.n_chunks;
    cudaError_t e = cudaSuccess;
    auto ok = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    if (!a.tiled) {
        if (nb > 0) ok(launch_kernel(k_seed_advect<true>, nb, kPrepThreads, 0, st, a));
        mark(2);
        ok(launch_kernel(k_scan, 2u * (unsigned)a.n_pairs, 1024, 0, st, a, -1));
        mark(3);
        if (nb > 0) ok(launch_kernel(k_scatter, nb, kPrepThreads, 0, st, a));
        mark(4);
        return e;
    }
    if (a.tiled == 2) {  // seeded render: seeding, advection and both frames' placement in one pass
        int dev = 0, nsm = 0;
        ok(cudaGetDevice(&dev));
        ok(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        if (e != cudaSuccess) return e;
        if (nb > 2u * (unsigned)nsm) ok(launch_kernel(k_seed_place<true, 256>, nb, 256, 0, st, a));
        else if (nb > 0) ok(launch_kernel(k_seed_place<true, 512>, nb, 512, 0, st, a));
        mark(2);
        // both frames' checks in one launch (each CTA returns at once unless its frame overflowed)
        if (a.rebin) ok(launch_kernel(k_rebin, 2u * (unsigned)a.n_pairs, 1024, 0, st, a, -1));
        mark(3);
        mark(4);
        return e;
    }
    // seeded render: seeding with the frame-1 placement, tiled advection with the frame-2 placement
    const unsigned nt1 = (unsigned)(a.n_tiles / 2);
    const size_t adv_smem = (size_t)adv_window_nodes(a.tile) * sizeof(float2);
    const bool big = a.tile >= 128;  // two row bands per tile, 512 threads each
    ok(big ? cudaFuncSetAttribute(k_advect<512, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adv_smem)
           : cudaFuncSetAttribute(k_advect<256, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)adv_smem));
    if (e != cudaSuccess) return e;
    if (nb > 0) ok(launch_kernel(k_seed_place<false, kPrepThreads>, nb, kPrepThreads, 0, st, a));
    if (a.rebin) ok(launch_kernel(k_rebin, (unsigned)a.n_pairs, 1024, 0, st, a, 0));  // at once unless overflowed
    if (nt1 > 0) {
        if (big) ok(launch_kernel(k_advect<512, 2>, 2 * nt1, 512, adv_smem, st, a));
        else ok(launch_kernel(k_advect<256, 1>, nt1, 256, adv_smem, st, a));
    }
    mark(2);
    mark(3);
    if (a.rebin) ok(launch_kernel(k_rebin, (unsigned)a.n_pairs, 1024, 0, st, a, 1));
    mark(4);
    return e;
}

}  // namespace spx

namespace spx {

cudaError_t launch_seed_only(const KernelArgs &a, cudaStream_t st) {
    if (a.n_chunks > 0) {
        if (a.states) return launch_kernel(k_seed_advect<true>, (unsigned)a.n_chunks, kPrepThreads, 0, st, a);
        return launch_kernel(k_seed_advect<false>, (unsigned)a.n_chunks, kPrepThreads, 0, st, a);
    }
    return cudaGetLastError();
}

}  // namespace spx
