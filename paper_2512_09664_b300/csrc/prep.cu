// sm_103a kernels of the PIV image-pair renderer (SynthPix, arXiv 2512.09664,
// Section 2) that prepare the splat.  One batch is rendered by a fixed
// sequence of launches:
//
//   k_plan         per-pair prefix sums of particles, tiles and bin slots,
//                  blur taps, the work-queue ticket
//   k_seed_advect  Philox attributes of every particle, advection through the
//                  flow grid (RK4 / Euler substeps), split positions and
//                  per-(frame, tile) counts
//   k_scan         exclusive scan of the counts of each (pair, frame), and the
//                  splat's work items
//   k_scatter      particle records into the bins of every tile their (halo-
//                  widened) window meets
//   k_splat        (splat.cu) persistent CTAs over the work items
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
// k_plan: per-pair prefix sums (one CTA of 1024 threads)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_plan(const synthpix_pair_desc *__restrict__ descs, int32_t n_pairs,
                                               int32_t tile, int32_t fused, PairPlan *__restrict__ plan,
                                               int64_t want_part, int64_t want_tiles, int64_t want_list,
                                               int64_t want_inter, int32_t *__restrict__ check,
                                               float *__restrict__ blur_w, uint32_t *__restrict__ ticket) {
    __shared__ long long s_part[1024], s_tile[1024], s_list[1024], s_inter[1024];
    const int t = threadIdx.x;
    const int per = (n_pairs + 1023) / 1024;
    const int b0 = min(t * per, n_pairs), b1 = min(b0 + per, n_pairs);
    long long np = 0, nt = 0, nl = 0, ni = 0;
    for (int b = b0; b < b1; ++b) {
        const synthpix_pair_desc d = descs[b];
        const PairGeom g = pair_geom(d, tile, fused != 0);
        np += d.n_particles;
        nt += 2LL * g.ntiles;
        nl += 2LL * g.list_cap;
        ni += fused ? 0LL : 2LL * d.height * d.width;
    }
    s_part[t] = np; s_tile[t] = nt; s_list[t] = nl; s_inter[t] = ni;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // inclusive Hillis-Steele scan
        long long a = 0, bq = 0, c = 0, e = 0;
        if (t >= off) { a = s_part[t - off]; bq = s_tile[t - off]; c = s_list[t - off]; e = s_inter[t - off]; }
        __syncthreads();
        s_part[t] += a; s_tile[t] += bq; s_list[t] += c; s_inter[t] += e;
        __syncthreads();
    }
    long long bp = s_part[t] - np, bt = s_tile[t] - nt, bl = s_list[t] - nl, bi = s_inter[t] - ni;
    for (int b = b0; b < b1; ++b) {
        const synthpix_pair_desc d = descs[b];
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
        p.pad[0] = p.pad[1] = 0;
        plan[b] = p;
        // normalised blur taps w[|k|], k = -R..R (FP64, stored FP32)
        if (g.blur_r > 0) {
            double w[kMaxBlurRadius + 1], sum = 0.0;
            const double sb = (double)d.blur_sigma;
            for (int k = 0; k <= g.blur_r; ++k) {
                w[k] = exp(-(double)(k * k) / (2.0 * sb * sb));
                sum += k ? 2.0 * w[k] : w[k];
            }
            for (int k = 0; k <= g.blur_r; ++k) blur_w[b * kBlurStride + k] = (float)(w[k] / sum);
        }
        bp += d.n_particles;
        bt += 2LL * g.ntiles;
        bl += 2LL * g.list_cap;
        bi += fused ? 0LL : 2LL * d.height * d.width;
    }
    if (t == 1023) {
        *ticket = 0u;
        const bool ok = s_part[1023] == want_part && s_tile[1023] == want_tiles && s_list[1023] == want_list &&
                        s_inter[1023] == want_inter;
        *check = ok ? 1 : 0;
    }
}

// ---------------------------------------------------------------------------
// k_seed_advect: one thread per particle
// ---------------------------------------------------------------------------
// One particle of k_seed_advect: attributes, frame-1 record, and what the
// advection needs.
struct SeedState {
    int64_t g;
    int b;
    Seeded P;
    Flow F;
    int32_t jx, jy;
    float gx, gy;
};

__device__ __forceinline__ bool seed_one(const KernelArgs &a, int64_t g, SeedState &S) {
    S.g = g;
    if (g >= a.n_part) return false;
    S.b = upper_find(a.n_pairs, g, [&](int m) { return a.plan[m].part_base; });
    const synthpix_pair_desc &D = a.descs[S.b];
    S.P = seed_particle(a, D, (uint32_t)(g - a.plan[S.b].part_base), g);
    a.sa[g] = make_float2(S.P.sigma, S.P.amp);
    a.pos0[g] = make_float4(S.P.fx, S.P.fy, __int_as_float(S.P.ix), __int_as_float(S.P.iy));
    if (a.particles_out) {
        a.particles_out[3 * g] = (float)S.P.ix + S.P.fx;
        a.particles_out[3 * g + 1] = (float)S.P.iy + S.P.fy;
        a.particles_out[3 * g + 2] = 4.0f * S.P.sigma;
    }
    S.F = pair_flow(a, D);
    S.jx = S.P.ix;
    S.jy = S.P.iy;
    S.gx = S.P.fx;
    S.gy = S.P.fy;
    return true;
}

// Frame-2 record and bin counts of both frames.
__device__ __forceinline__ void finish_one(const KernelArgs &a, const SeedState &S) {
    a.pos1[S.g] = make_float4(S.gx, S.gy, __int_as_float(S.jx), __int_as_float(S.jy));
    if (!a.count) return;
    const PairPlan pl = a.plan[S.b];
    const int32_t H = a.descs[S.b].height, W = a.descs[S.b].width;
    const float r15 = 6.0f * S.P.sigma;  // 1.5 d
    for (int f = 0; f < 2; ++f) {
        const Window w = f ? particle_window(S.jx, S.gx, S.jy, S.gy, r15, W, H)
                           : particle_window(S.P.ix, S.P.fx, S.P.iy, S.P.fy, r15, W, H);
        if (w.j0 > w.j1 || w.i0 > w.i1) continue;
        int32_t tx0, tx1, ty0, ty1;
        window_tiles(w, pl.halo, a.tile, W, H, tx0, tx1, ty0, ty1);
        uint32_t *cnt = a.count + pl.tile_base + (int64_t)f * pl.ntiles;
        for (int32_t ty = ty0; ty <= ty1; ++ty)
            for (int32_t tx = tx0; tx <= tx1; ++tx) atomicAdd(cnt + ty * pl.tiles_x + tx, 1u);
    }
}

// One thread per particle.  (Two particles per thread in lockstep needs 80
// registers and lost more occupancy than it gained in overlap.)
__global__ void __launch_bounds__(256) k_seed_advect(KernelArgs a) {
    if (*a.check != 1) return;
    SeedState A;
    if (!seed_one(a, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, A) || a.particles_out) return;
    // frame-2 position: displacement over dt through the bilinear flow
    advect_split(A.F, a.dt, a.n_substeps, a.integrator, A.jx, A.gx, A.jy, A.gy);
    finish_one(a, A);
}

// ---------------------------------------------------------------------------
// k_scan: exclusive scan of the bin counts of one (pair, frame) per CTA
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_scan(KernelArgs a) {
    if (*a.check != 1) return;
    __shared__ uint32_t s[1024];
    __shared__ uint32_t carry;
    const int b = blockIdx.x >> 1, f = blockIdx.x & 1;
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

// ---------------------------------------------------------------------------
// k_scatter: particle records into their tiles' bins (order within a bin is
// free: the splat accumulates in exact fixed point, so sums are
// order-independent)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_scatter(KernelArgs a) {
    if (*a.check != 1) return;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n_part) return;
    const int b = upper_find(a.n_pairs, g, [&](int m) { return a.plan[m].part_base; });
    const PairPlan pl = a.plan[b];
    const int32_t H = a.descs[b].height, W = a.descs[b].width;
    const float2 q = a.sa[g];
    const float r15 = 6.0f * q.x;
    for (int f = 0; f < 2; ++f) {
        const float4 p = f ? a.pos1[g] : a.pos0[g];
        const Window w = particle_window(__float_as_int(p.z), p.x, __float_as_int(p.w), p.y, r15, W, H);
        if (w.j0 > w.j1 || w.i0 > w.i1) continue;
        int32_t tx0, tx1, ty0, ty1;
        window_tiles(w, pl.halo, a.tile, W, H, tx0, tx1, ty0, ty1);
        const int64_t tb = pl.tile_base + (int64_t)f * pl.ntiles;
        Record *seg = a.rec + pl.list_base + (int64_t)f * pl.list_cap;
        for (int32_t ty = ty0; ty <= ty1; ++ty)
            for (int32_t tx = tx0; tx <= tx1; ++tx) {
                const uint32_t slot = atomicAdd(a.cursor + tb + ty * pl.tiles_x + tx, 1u);
                if ((int64_t)slot < pl.list_cap) {
                    float2 *r = reinterpret_cast<float2 *>(seg + slot);
                    r[0] = make_float2(p.x, p.y);
                    r[1] = make_float2(p.z, p.w);
                    r[2] = q;
                }
            }
    }
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
cudaError_t launch_plan(const synthpix_pair_desc *descs, int32_t n_pairs, int32_t tile, int32_t fused,
                        PairPlan *plan, const Layout &L, int32_t *check, float *blur_w, uint32_t *ticket,
                        cudaStream_t st) {
    k_plan<<<1, 1024, 0, st>>>(descs, n_pairs, tile, fused, plan, L.n_part, L.n_tiles, L.n_list, L.n_inter, check,
                               blur_w, ticket);
    return cudaGetLastError();
}

cudaError_t launch_prep(const KernelArgs &a, cudaStream_t st, cudaEvent_t const *ev) {
    auto mark = [&](int k) {
        if (ev && ev[k]) cudaEventRecord(ev[k], st);
    };
    const unsigned nb = (unsigned)((a.n_part + 255) / 256);
    if (a.n_part > 0) k_seed_advect<<<(unsigned)((a.n_part + 255) / 256), 256, 0, st>>>(a);
    mark(2);
    k_scan<<<2 * a.n_pairs, 1024, 0, st>>>(a);
    mark(3);
    if (a.n_part > 0) k_scatter<<<nb, 256, 0, st>>>(a);
    mark(4);
    return cudaGetLastError();
}

}  // namespace spx

namespace spx {

cudaError_t launch_seed_only(const KernelArgs &a, cudaStream_t st) {
    if (a.n_part > 0) k_seed_advect<<<(unsigned)((a.n_part + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace spx
