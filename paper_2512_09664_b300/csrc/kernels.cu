// sm_103a kernels of the PIV image-pair renderer (SynthPix, arXiv 2512.09664,
// Section 2).  One batch is rendered by a fixed sequence of launches:
//
//   k_plan         per-pair prefix sums of particles, tiles and bin-list slots
//   k_seed_advect  Philox attributes of every particle, advection through the
//                  flow grid (RK4 / Euler substeps), split-position records and
//                  per-(frame, tile) counts
//   k_scan         exclusive scan of the counts of each (pair, frame)
//   k_scatter      particle ids into the bins of every tile their (halo-
//                  widened) window meets
//   k_splat_fused  one CTA per (pair, frame, tile): pixel-integrated Gaussian
//                  splat into an on-chip fixed-point tile, then illumination,
//                  noise, separable blur and quantisation; every output pixel
//                  written once
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
                                               float *__restrict__ blur_w) {
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
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// k_scatter: particle ids into their tiles' bins (order within a bin is free:
// the splat accumulates in exact fixed point, so the sum is order-independent)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_scatter(KernelArgs a) {
    if (*a.check != 1) return;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n_part) return;
    const int b = upper_find(a.n_pairs, g, [&](int m) { return a.plan[m].part_base; });
    const PairPlan pl = a.plan[b];
    const int32_t H = a.descs[b].height, W = a.descs[b].width;
    const uint32_t i = (uint32_t)(g - pl.part_base);
    const float r15 = 6.0f * a.sa[g].x;
    for (int f = 0; f < 2; ++f) {
        const float4 p = f ? a.pos1[g] : a.pos0[g];
        const Window w = particle_window(__float_as_int(p.z), p.x, __float_as_int(p.w), p.y, r15, W, H);
        if (w.j0 > w.j1 || w.i0 > w.i1) continue;
        int32_t tx0, tx1, ty0, ty1;
        window_tiles(w, pl.halo, a.tile, W, H, tx0, tx1, ty0, ty1);
        const int64_t tb = pl.tile_base + (int64_t)f * pl.ntiles;
        uint32_t *lst = a.list + pl.list_base + (int64_t)f * pl.list_cap;
        for (int32_t ty = ty0; ty <= ty1; ++ty)
            for (int32_t tx = tx0; tx <= tx1; ++tx) {
                const uint32_t slot = atomicAdd(a.cursor + tb + ty * pl.tiles_x + tx, 1u);
                if ((int64_t)slot < pl.list_cap) lst[slot] = i;
            }
    }
}

// ---------------------------------------------------------------------------
// splat + epilogue
// ---------------------------------------------------------------------------

// Lower-tail mass Phi(t) for t <= 0, minus the upper-tail mass 1 - Phi(t)
// for t > 0 (both from erfc, so tails keep their relative accuracy).
__device__ __forceinline__ float edge_value(float t) {
    const float q = 0.5f * erfcf(fabsf(t) * 0.70710678118654752440f);
    return t > 0.0f ? -q : q;
}

// Mass of the unit Gaussian between two pixel edges from their edge values:
// Phi(b) - Phi(a) = sb - sa, plus 1 when a <= 0 < b.
__device__ __forceinline__ float pixel_mass(float sa, float sb, bool a_pos, bool b_pos) {
    if (b_pos && !a_pos) return (1.0f - sa) + sb;
    return fmaxf(sb - sa, 0.0f);
}

template <typename T>
__device__ __forceinline__ void store_out(T *p, float v);
template <>
__device__ __forceinline__ void store_out<float>(float *p, float v) { *p = v; }
template <>
__device__ __forceinline__ void store_out<__half>(__half *p, float v) { *p = __float2half_rn(v); }
template <>
__device__ __forceinline__ void store_out<__nv_bfloat16>(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ void store_out<uint8_t>(uint8_t *p, float v) { *p = (uint8_t)v; }
template <>
__device__ __forceinline__ void store_out<uint16_t>(uint16_t *p, float v) { *p = (uint16_t)v; }

constexpr int kSplatThreads = 256;
constexpr int kSplatWarps = kSplatThreads / 32;

struct TileCtx {
    int b, f, tx, ty;
    int32_t H, W;
    int32_t x0, x1, y0, y1;  // tile pixels [x0, x1) x [y0, y1)
    int32_t ex0, ex1, ey0, ey1;  // halo-widened rectangle, clipped to the frame
    int32_t EW;              // row pitch of the on-chip tile
};

__device__ __forceinline__ TileCtx tile_ctx(const KernelArgs &a, int64_t gt, PairPlan &pl) {
    TileCtx c;
    c.b = upper_find(a.n_pairs, gt, [&](int m) { return (int64_t)a.plan[m].tile_base; });
    pl = a.plan[c.b];
    const int32_t local = (int32_t)(gt - pl.tile_base);
    c.f = local >= pl.ntiles ? 1 : 0;
    const int32_t t = local - c.f * pl.ntiles;
    c.ty = t / pl.tiles_x;
    c.tx = t - c.ty * pl.tiles_x;
    c.H = a.descs[c.b].height;
    c.W = a.descs[c.b].width;
    c.x0 = c.tx * a.tile;
    c.x1 = min(c.x0 + a.tile, c.W);
    c.y0 = c.ty * a.tile;
    c.y1 = min(c.y0 + a.tile, c.H);
    c.ex0 = max(c.x0 - pl.halo, 0);
    c.ex1 = min(c.x1 + pl.halo, c.W);
    c.ey0 = max(c.y0 - pl.halo, 0);
    c.ey1 = min(c.y1 + pl.halo, c.H);
    c.EW = c.ex1 - c.ex0;
    return c;
}

// Exact fixed-point accumulation without 64-bit conversions.  A contribution
// v in [0, i_max] is scaled to u = v * 1024 / i_max and split into
// hi = rint(u) and lo = rint((u - hi) * 2^22), both found with the FP32
// round-to-integer identity (x + 1.5 * 2^23 leaves rint(x) in the low
// mantissa bits for |x| < 2^22).  The tile keeps int32 sums of hi and lo:
// integer addition is associative, so a pixel's value does not depend on the
// order of its contributions, the tile size or the batch it is rendered in.
// lo sums stay inside int32 for kChunk contributions; between chunks the
// multiples of 2^22 in lo are carried into hi.  Resolution: 2^-32 i_max.
constexpr uint32_t kChunk = 1016;      // particles per carry; 1016 * 2^21 < 2^31
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr int32_t kMagicBits = 0x4B400000;

__device__ __forceinline__ void add_fixed(int32_t *hi, int32_t *lo, int idx, float u) {
    const float t = u + kMagic;
    const int32_t h = __float_as_int(t) - kMagicBits;
    const float r = u - (t - kMagic);  // exact, |r| <= 1/2
    const int32_t l = __float_as_int(fmaf(r, 4194304.0f, kMagic)) - kMagicBits;
    atomicAdd(hi + idx, h);
    atomicAdd(lo + idx, l);
}

__device__ __forceinline__ void carry_fixed(int32_t *hi, int32_t *lo, int n) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int32_t l = lo[k];
        const int32_t c = l >> 22;  // floor(l / 2^22)
        hi[k] += c;
        lo[k] = l - (c << 22);
    }
}

// Splat every particle of the tile's bin into hi/lo[(i - ey0) * EW + (j - ex0)]
// over the halo-widened rectangle.  Warp per particle: each lane evaluates
// one erfc edge value of the window (x edges then y edges), neighbouring
// lanes give the per-pixel masses Ex(j), Ey(i), and the warp sweeps the
// window's pixels adding amp * Ex(j) * Ey(i).  Windows with more than 30
// edges go through per-warp shared scratch instead of lanes.
__device__ __forceinline__ void splat_particle_wide(const TileCtx &c, int32_t *hi, int32_t *lo, float px, float py,
                                                    int32_t ix, int32_t iy, float inv, float amps, int32_t j0,
                                                    int32_t i0, int nx, int ny, float *scr, int wq) {
    const int lane = threadIdx.x & 31;
    float *exe = scr, *eye = scr + wq, *ex = scr + 2 * wq, *ey = scr + 3 * wq;
    for (int e = lane; e <= nx; e += 32) exe[e] = edge_value(((float)(j0 + e - ix) - px) * inv);
    for (int e = lane; e <= ny; e += 32) eye[e] = edge_value(((float)(i0 + e - iy) - py) * inv);
    __syncwarp();
    for (int e = lane; e < nx; e += 32)
        ex[e] = pixel_mass(exe[e], exe[e + 1], (float)(j0 + e - ix) > px, (float)(j0 + e + 1 - ix) > px);
    for (int e = lane; e < ny; e += 32)
        ey[e] = amps * pixel_mass(eye[e], eye[e + 1], (float)(i0 + e - iy) > py, (float)(i0 + e + 1 - iy) > py);
    __syncwarp();
    const int n = nx * ny;
    const float invx = 1.0f / (float)nx;
    for (int m = lane; m < n; m += 32) {
        const int r = min((int)(((float)m + 0.5f) * invx), ny - 1);
        const int cc = m - r * nx;
        if ((unsigned)cc >= (unsigned)nx) continue;
        add_fixed(hi, lo, (i0 - c.ey0 + r) * c.EW + (j0 - c.ex0 + cc), __fmul_rn(ex[cc], ey[r]));
    }
    __syncwarp();
}

__device__ __forceinline__ void splat_tile(const KernelArgs &a, const PairPlan &pl, const TileCtx &c, int32_t *hi,
                                           int32_t *lo, float *wscr, int wstride) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned FULL = 0xffffffffu;
    const int64_t tb = pl.tile_base + (int64_t)c.f * pl.ntiles + c.ty * pl.tiles_x + c.tx;
    const uint32_t beg = a.off[tb];
    const int64_t room = pl.list_cap - (int64_t)beg;
    const uint32_t cnt = (uint32_t)max((int64_t)0, min((int64_t)a.count[tb], room));
    const synthpix_pair_desc &D = a.descs[c.b];
    const uint32_t n_here = D.n_particles;
    const float imax = D.i_max > 0.0f ? D.i_max : 1.0f;
    const float scale = 1024.0f / imax;
    const uint32_t *lst = a.list + pl.list_base + (int64_t)c.f * pl.list_cap + beg;
    const float4 *pos = c.f ? a.pos1 : a.pos0;
    float *scr = wscr + warp * wstride;
    const int wq = wstride >> 2;
    const int npix = (c.ey1 - c.ey0) * c.EW;
    for (uint32_t c0 = 0; c0 < cnt; c0 += kChunk) {
        const uint32_t c1 = min(cnt, c0 + kChunk);
        for (uint32_t base = c0 + warp; base < c1; base += kSplatWarps * 32) {
            // prefetch this warp's next 32 particles (one per lane)
            const uint32_t k = base + kSplatWarps * lane;
            float4 P = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 Q = make_float2(0.f, 0.f);
            int ok = 0;
            if (k < c1) {
                const uint32_t li = lst[k];
                if (li < n_here) {
                    const int64_t g = pl.part_base + li;
                    P = pos[g];
                    Q = a.sa[g];
                    ok = 1;
                }
            }
            const int nb = min(32u, (c1 - base + kSplatWarps - 1) / kSplatWarps);
            for (int t = 0; t < nb; ++t) {
                if (!__shfl_sync(FULL, ok, t)) continue;  // warp-uniform
                const float px = __shfl_sync(FULL, P.x, t), py = __shfl_sync(FULL, P.y, t);
                const int32_t ix = __shfl_sync(FULL, __float_as_int(P.z), t);
                const int32_t iy = __shfl_sync(FULL, __float_as_int(P.w), t);
                const float sig = __shfl_sync(FULL, Q.x, t), amp = __shfl_sync(FULL, Q.y, t);
                const float r15 = 6.0f * sig;
                const int32_t j0 = max(ix + (int32_t)floorf(px - r15), c.ex0);
                const int32_t j1 = min(ix + (int32_t)floorf(px + r15), c.ex1 - 1);
                const int32_t i0 = max(iy + (int32_t)floorf(py - r15), c.ey0);
                const int32_t i1 = min(iy + (int32_t)floorf(py + r15), c.ey1 - 1);
                if (j0 > j1 || i0 > i1) continue;  // warp-uniform
                const int nx = j1 - j0 + 1, ny = i1 - i0 + 1;
                const float inv = __frcp_rn(sig);
                const float amps = amp * scale;
                if (nx + ny + 2 > 32) {
                    splat_particle_wide(c, hi, lo, px, py, ix, iy, inv, amps, j0, i0, nx, ny, scr, wq);
                    continue;
                }
                // lanes [0, nx]: x edges j0 + e; lanes [nx+1, nx+ny+1]: y edges i0 + e
                const int nxe = nx + 1;
                const bool isx = lane < nxe;
                const int e = isx ? lane : lane - nxe;
                const float dd = isx ? (float)(j0 + e - ix) - px : (float)(i0 + e - iy) - py;
                const bool dpos = dd > 0.0f;
                const float ev = lane < nxe + ny + 1 ? edge_value(dd * inv) : 0.0f;
                const float evn = __shfl_down_sync(FULL, ev, 1);
                const bool dposn = __shfl_down_sync(FULL, (int)dpos, 1) != 0;
                float m = pixel_mass(ev, evn, dpos, dposn);
                if (!isx) m *= amps;
                const int n = nx * ny;
                const float invx = 1.0f / (float)nx;
                for (int m0 = 0; m0 < n; m0 += 32) {
                    const int mm = m0 + lane;
                    const int r = min((int)(((float)mm + 0.5f) * invx), ny - 1);
                    const int cc = min(max(mm - r * nx, 0), nx - 1);
                    const float exv = __shfl_sync(FULL, m, cc);
                    const float eyv = __shfl_sync(FULL, m, nxe + r);
                    if (mm < n)
                        add_fixed(hi, lo, (i0 - c.ey0 + r) * c.EW + (j0 - c.ex0 + cc), __fmul_rn(exv, eyv));
                }
            }
        }
        __syncthreads();
        carry_fixed(hi, lo, npix);
        __syncthreads();
    }
}

// The per-frame finishing steps on the tile: A = L * S + sigma_n * n,
// separable Gaussian blur (horizontal pass, then vertical), quantisation.
template <typename T>
__device__ __forceinline__ void epilogue_tile(const KernelArgs &a, const PairPlan &pl, const TileCtx &c,
                                              const synthpix_pair_desc &D, float *A, float *Bh, float *sx2,
                                              float *sy2, float *wts) {
    const int EH = c.ey1 - c.ey0, EW = c.EW;
    const int R = pl.blur_r;
    // separable illumination factors
    const bool illum = D.illum_min != 1.0f || D.illum_max != 1.0f;
    for (int k = threadIdx.x; k < EW + EH; k += blockDim.x) {
        if (k < EW) {
            const float s = sinpif(((float)(c.ex0 + k) + 0.5f) / (float)c.W);
            sx2[k] = s * s;
        } else {
            const float s = sinpif(((float)(c.ey0 + k - EW) + 0.5f) / (float)c.H);
            sy2[k - EW] = s * s;
        }
    }
    for (int k = threadIdx.x; k <= 2 * R; k += blockDim.x) wts[k] = a.blur_w[c.b * kBlurStride + abs(k - R)];
    __syncthreads();
    // A = L * S (+ noise): S was converted from fixed point in place of A
    const float dl = D.illum_max - D.illum_min;
    if (D.noise_sigma != 0.0f) {
        // one Philox call per 4 consecutive pixels of the row-major frame
        const int64_t HW = (int64_t)c.H * c.W;
        const int nq = (EW + 6) / 4 + 1;
        for (int item = threadIdx.x; item < EH * nq; item += blockDim.x) {
            const int r = item / nq, qi = item - r * nq;
            const int64_t rowlin = (int64_t)(c.ey0 + r) * c.W;
            const int64_t q = ((rowlin + c.ex0) >> 2) + qi;
            if (4 * q > rowlin + c.ex1 - 1) continue;
            const uint4 w = stream_words(a.seed, D.pair_id, (uint32_t)q, kTagNoise + (uint32_t)c.f);
            float s0, c0, s1, c1;
            sincospif(2.0f * u24f(w.y), &s0, &c0);
            sincospif(2.0f * u24f(w.w), &s1, &c1);
            const float r0 = sqrtf(-2.0f * logf(uo24f(w.x)));
            const float r1 = sqrtf(-2.0f * logf(uo24f(w.z)));
            const float nv[4] = {r0 * c0, r0 * s0, r1 * c1, r1 * s1};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int64_t pix = 4 * q + k;
                const int64_t col = pix - rowlin;
                if (pix < HW && col >= c.ex0 && col < c.ex1) {
                    const int idx = r * EW + (int)(col - c.ex0);
                    const float L = illum ? fmaf(dl, sx2[idx - r * EW] * sy2[r], D.illum_min) : 1.0f;
                    A[idx] = fmaf(L, A[idx], D.noise_sigma * nv[k]);
                }
            }
        }
    } else if (illum) {
        for (int idx = threadIdx.x; idx < EH * EW; idx += blockDim.x) {
            const int r = idx / EW, cc = idx - r * EW;
            A[idx] = fmaf(dl, sx2[cc] * sy2[r], D.illum_min) * A[idx];
        }
    }
    __syncthreads();
    const int TW = c.x1 - c.x0, TH = c.y1 - c.y0;
    const float *src = A;
    int srow0 = c.ey0, scol0 = c.ex0, spitch = EW;
    if (R > 0) {
        // horizontal pass over the halo rows, tile columns, replicate border
        for (int idx = threadIdx.x; idx < EH * TW; idx += blockDim.x) {
            const int r = idx / TW, cc = idx - r * TW;
            const int j = c.x0 + cc;
            float acc = 0.0f;
            for (int k = -R; k <= R; ++k) {
                const int jj = min(max(j + k, 0), c.W - 1);
                acc = fmaf(wts[k + R], A[r * EW + (jj - c.ex0)], acc);
            }
            Bh[idx] = acc;
        }
        __syncthreads();
        src = Bh;
        scol0 = c.x0;
        spitch = TW;
    }
    // vertical pass (or identity) and store
    const int64_t HW = (int64_t)c.H * c.W;
    T *out = reinterpret_cast<T *>(a.images) + a.descs[c.b].image_offset + (int64_t)c.f * HW;
    const float M = a.quant_bits > 0 ? (float)((1u << a.quant_bits) - 1u) : 0.0f;
    for (int idx = threadIdx.x; idx < TH * TW; idx += blockDim.x) {
        const int r = idx / TW, cc = idx - r * TW;
        const int i = c.y0 + r, j = c.x0 + cc;
        float v;
        if (R > 0) {
            v = 0.0f;
            for (int k = -R; k <= R; ++k) {
                const int ii = min(max(i + k, 0), c.H - 1);
                v = fmaf(wts[k + R], src[(ii - srow0) * spitch + (j - scol0)], v);
            }
        } else {
            v = src[(i - srow0) * spitch + (j - scol0)];
        }
        if (a.quant_bits > 0) v = fminf(fmaxf(rintf(v * M), 0.0f), M);
        store_out<T>(out + (int64_t)i * c.W + j, v);
    }
}

template <typename T>
__global__ void __launch_bounds__(kSplatThreads) k_splat_fused(KernelArgs a) {
    if (*a.check != 1) return;
    extern __shared__ __align__(16) unsigned char smem[];
    PairPlan pl;
    const TileCtx c = tile_ctx(a, blockIdx.x, pl);
    const synthpix_pair_desc &D = a.descs[c.b];
    const int E = a.smem_edge;  // capacity edge of the on-chip tile
    int32_t *hi = reinterpret_cast<int32_t *>(smem);
    int32_t *lo = hi + E * E;
    float *A = reinterpret_cast<float *>(lo + E * E);
    float *Bh = A + E * E;
    float *sx2 = Bh + E * a.tile;
    float *sy2 = sx2 + E;
    float *wts = sy2 + E;
    float *wscr = wts + (2 * kMaxBlurRadius + 1 + 3);
    const int npix = (c.ey1 - c.ey0) * c.EW;
    for (int k = threadIdx.x; k < npix; k += blockDim.x) {
        hi[k] = 0;
        lo[k] = 0;
    }
    __syncthreads();
    splat_tile(a, pl, c, hi, lo, wscr, a.warp_scratch);  // ends with carried lo in [0, 2^22)
    const float imax = D.i_max > 0.0f ? D.i_max : 1.0f;
    const float unit = imax * (1.0f / 1024.0f);
    for (int k = threadIdx.x; k < npix; k += blockDim.x)
        A[k] = fmaf((float)lo[k], 1.0f / 4194304.0f, (float)hi[k]) * unit;
    __syncthreads();
    epilogue_tile<T>(a, pl, c, D, A, Bh, sx2, sy2, wts);
}

size_t splat_smem_bytes(int edge, int tile, int warp_scratch) {
    return (size_t)edge * edge * 8 + (size_t)edge * edge * 4 + (size_t)edge * tile * 4 + 2 * (size_t)edge * 4 +
           (2 * kMaxBlurRadius + 1 + 3) * 4 + (size_t)kSplatWarps * warp_scratch * 4;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
cudaError_t launch_plan(const synthpix_pair_desc *descs, int32_t n_pairs, int32_t tile, int32_t fused,
                        PairPlan *plan, const Layout &L, int32_t *check, float *blur_w, cudaStream_t st) {
    k_plan<<<1, 1024, 0, st>>>(descs, n_pairs, tile, fused, plan, L.n_part, L.n_tiles, L.n_list, L.n_inter, check,
                               blur_w);
    return cudaGetLastError();
}

cudaError_t launch_render(const KernelArgs &a, int32_t out_dtype, cudaStream_t st, cudaEvent_t const *ev) {
    auto mark = [&](int k) {
        if (ev && ev[k]) cudaEventRecord(ev[k], st);
    };
    if (a.n_part > 0) {
        const unsigned nb = (unsigned)((a.n_part + 255) / 256);
        k_seed_advect<<<nb, 256, 0, st>>>(a);
        mark(2);
        k_scan<<<2 * a.n_pairs, 1024, 0, st>>>(a);
        mark(3);
        k_scatter<<<nb, 256, 0, st>>>(a);
        mark(4);
    } else {
        mark(2);
        k_scan<<<2 * a.n_pairs, 1024, 0, st>>>(a);
        mark(3);
        mark(4);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = splat_smem_bytes(a.smem_edge, a.tile, a.warp_scratch);
    const unsigned grid = (unsigned)a.n_tiles;
#define SPX_LAUNCH(T)                                                                                     \
    do {                                                                                                  \
        e = cudaFuncSetAttribute(k_splat_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                                   \
        k_splat_fused<T><<<grid, kSplatThreads, smem, st>>>(a);                                           \
    } while (0)
    switch (out_dtype) {
    case SYNTHPIX_F32: SPX_LAUNCH(float); break;
    case SYNTHPIX_F16: SPX_LAUNCH(__half); break;
    case SYNTHPIX_BF16: SPX_LAUNCH(__nv_bfloat16); break;
    case SYNTHPIX_U8: SPX_LAUNCH(uint8_t); break;
    default: SPX_LAUNCH(uint16_t); break;
    }
#undef SPX_LAUNCH
    mark(5);
    return cudaGetLastError();
}

}  // namespace spx
