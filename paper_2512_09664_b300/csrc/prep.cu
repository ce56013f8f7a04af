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

namespace spx {

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

// Largest b with base(b) <= key (bases non-decreasing, base(0) = 0).
template <typename F>
__device__ __forceinline__ int upper_find(int n, int64_t key, F base) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (base(mid) <= key) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct Flow {
    const float2 *f;
    int32_t gh, gw, H, W;
};

// Grid coordinate of an image coordinate i + f along one axis:
// g = (i + f) * gn / n - 1/2 = cell + frac, computed without rounding the
// integer part (integer division when the grid and image sizes differ).
__device__ __forceinline__ void grid_coord(int32_t i, float f, int32_t gn, int32_t n, int32_t &cell, float &t) {
    float g;
    int32_t base;
    if (gn == n) {
        base = i;
        g = f - 0.5f;
    } else {
        const long long num = (long long)i * gn;
        long long q = num / n;
        long long r = num - q * n;
        if (r < 0) { r += n; q -= 1; }
        base = (int32_t)q;
        g = fmaf(f, (float)gn, (float)r) / (float)n - 0.5f;
    }
    const float fl = floorf(g);
    cell = base + (int32_t)fl;
    t = g - fl;
}

// Bilinear velocity on the cell-centred grid, indices clamped (border).
__device__ __forceinline__ float2 velocity(const Flow &F, int32_t ix, float fx, int32_t iy, float fy) {
    int32_t l, k;
    float tx, ty;
    grid_coord(ix, fx, F.gw, F.W, l, tx);
    grid_coord(iy, fy, F.gh, F.H, k, ty);
    const int32_t l0 = min(max(l, 0), F.gw - 1), l1 = min(max(l + 1, 0), F.gw - 1);
    const int32_t k0 = min(max(k, 0), F.gh - 1), k1 = min(max(k + 1, 0), F.gh - 1);
    const float2 a = __ldg(F.f + (size_t)k0 * F.gw + l0);
    const float2 b = __ldg(F.f + (size_t)k0 * F.gw + l1);
    const float2 c = __ldg(F.f + (size_t)k1 * F.gw + l0);
    const float2 d = __ldg(F.f + (size_t)k1 * F.gw + l1);
    const float tu = fmaf(tx, b.x - a.x, a.x), tv = fmaf(tx, b.y - a.y, a.y);
    const float bu = fmaf(tx, d.x - c.x, c.x), bv = fmaf(tx, d.y - c.y, c.y);
    return make_float2(fmaf(ty, bu - tu, tu), fmaf(ty, bv - tv, tv));
}

// Clipped pixel window [j0, j1] x [i0, i1] of a particle (empty: j0 > j1).
struct Window {
    int32_t j0, j1, i0, i1;
};

__device__ __forceinline__ Window particle_window(int32_t ix, float fx, int32_t iy, float fy, float r15,
                                                  int32_t W, int32_t H) {
    Window w;
    w.j0 = max(ix + (int32_t)floorf(fx - r15), 0);
    w.j1 = min(ix + (int32_t)floorf(fx + r15), W - 1);
    w.i0 = max(iy + (int32_t)floorf(fy - r15), 0);
    w.i1 = min(iy + (int32_t)floorf(fy + r15), H - 1);
    return w;
}

// Tiles whose halo-widened rectangle meets the window.
__device__ __forceinline__ void window_tiles(const Window &w, int32_t halo, int32_t tile, int32_t W, int32_t H,
                                             int32_t &tx0, int32_t &tx1, int32_t &ty0, int32_t &ty1) {
    tx0 = max(w.j0 - halo, 0) / tile;
    tx1 = min(w.j1 + halo, W - 1) / tile;
    ty0 = max(w.i0 - halo, 0) / tile;
    ty1 = min(w.i1 + halo, H - 1) / tile;
}

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
__global__ void __launch_bounds__(256) k_seed_advect(KernelArgs a) {
    if (*a.check != 1) return;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n_part) return;
    const int b = upper_find(a.n_pairs, g, [&](int m) { return a.plan[m].part_base; });
    const PairPlan pl = a.plan[b];
    const synthpix_pair_desc &D = a.descs[b];
    const int32_t H = D.height, W = D.width;
    const uint32_t i = (uint32_t)(g - pl.part_base);

    // attributes (Section 2: uniform position over the image, parameters from
    // their intervals; clipped-normal diameter via Box-Muller)
    const uint4 wa = stream_words(a.seed, D.pair_id, i, kTagAttrA);
    const uint4 wb = stream_words(a.seed, D.pair_id, i, kTagAttrB);
    const unsigned long long px = (unsigned long long)(wa.x >> 8) * (uint32_t)W;
    const unsigned long long py = (unsigned long long)(wa.y >> 8) * (uint32_t)H;
    int32_t ix = (int32_t)(px >> 24), iy = (int32_t)(py >> 24);
    float fx = (float)(uint32_t)(px & 0xFFFFFFu) * (1.0f / 16777216.0f);  // exact
    float fy = (float)(uint32_t)(py & 0xFFFFFFu) * (1.0f / 16777216.0f);
    float d;
    if (D.d_dist == 0) {
        d = fminf(fmaf(u24f(wa.z), D.d_max - D.d_min, D.d_min), D.d_max);
    } else {
        float s, c;
        sincospif(2.0f * u24f(wb.y), &s, &c);
        const float r = sqrtf(-2.0f * logf(uo24f(wa.z)));
        d = fminf(fmaxf(fmaf(D.d_sigma, r * c, D.d_mu), D.d_min), D.d_max);
    }
    const float I0 = fmaf(u24f(wa.w), D.i_max - D.i_min, D.i_min);
    const float z = fmaf(u24f(wb.x), D.z_max - D.z_min, D.z_min);
    float gain = 1.0f;
    if (D.sheet_sigma > 0.0f) gain = expf(-(z * z) / (2.0f * D.sheet_sigma * D.sheet_sigma));
    const float sigma = 0.25f * d;
    const float amp = (I0 * gain) * (6.28318530717958647692f * sigma * sigma);  // Ieff * 2 pi sigma^2
    a.sa[g] = make_float2(sigma, amp);
    a.pos0[g] = make_float4(fx, fy, __int_as_float(ix), __int_as_float(iy));

    // frame-2 position: displacement over dt through the bilinear flow
    Flow F;
    F.f = reinterpret_cast<const float2 *>(a.flows + D.flow_offset);
    F.gh = D.flow_h; F.gw = D.flow_w; F.H = H; F.W = W;
    const float h = a.dt / (float)a.n_substeps;
    const float hh = 0.5f * h, h6 = h / 6.0f;
    int32_t jx = ix, jy = iy;
    float gx = fx, gy = fy;
    for (int s = 0; s < a.n_substeps; ++s) {
        const float2 k1 = velocity(F, jx, gx, jy, gy);
        if (a.integrator == SYNTHPIX_EULER) {
            split_add(jx, gx, __fmul_rn(h, k1.x));
            split_add(jy, gy, __fmul_rn(h, k1.y));
            continue;
        }
        const float2 k2 = velocity(F, jx, fmaf(hh, k1.x, gx), jy, fmaf(hh, k1.y, gy));
        const float2 k3 = velocity(F, jx, fmaf(hh, k2.x, gx), jy, fmaf(hh, k2.y, gy));
        const float2 k4 = velocity(F, jx, fmaf(h, k3.x, gx), jy, fmaf(h, k3.y, gy));
        split_add(jx, gx, __fmul_rn(h6, (k1.x + k4.x) + 2.0f * (k2.x + k3.x)));
        split_add(jy, gy, __fmul_rn(h6, (k1.y + k4.y) + 2.0f * (k2.y + k3.y)));
    }
    a.pos1[g] = make_float4(gx, gy, __int_as_float(jx), __int_as_float(jy));

    // bin counts of both frames
    const float r15 = 6.0f * sigma;  // 1.5 d
    for (int f = 0; f < 2; ++f) {
        const Window w = f ? particle_window(jx, gx, jy, gy, r15, W, H) : particle_window(ix, fx, iy, fy, r15, W, H);
        if (w.j0 > w.j1 || w.i0 > w.i1) continue;
        int32_t tx0, tx1, ty0, ty1;
        window_tiles(w, pl.halo, a.tile, W, H, tx0, tx1, ty0, ty1);
        uint32_t *cnt = a.count + pl.tile_base + (int64_t)f * pl.ntiles;
        for (int32_t ty = ty0; ty <= ty1; ++ty)
            for (int32_t tx = tx0; tx <= tx1; ++tx) atomicAdd(cnt + ty * pl.tiles_x + tx, 1u);
    }
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
    if (a.n_part > 0) k_seed_advect<<<nb, 256, 0, st>>>(a);
    mark(2);
    k_scan<<<2 * a.n_pairs, 1024, 0, st>>>(a);
    mark(3);
    if (a.n_part > 0) k_scatter<<<nb, 256, 0, st>>>(a);
    mark(4);
    return cudaGetLastError();
}

}  // namespace spx
