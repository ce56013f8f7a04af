// The splat + epilogue of the PIV image-pair renderer (SynthPix, arXiv
// 2512.09664, Section 2): Eq. 1 integrated over each pixel and summed over
// the particles ("aggregation of the particle contributions"), then the
// imaging steps named in the Abstract (illumination non-uniformity, noise,
// blur) and quantisation.
//
// k_splat is persistent: each CTA takes (pair, frame, tile) work items from a
// ticket counter (atomicAdd, no waiting on other CTAs) and, while it renders
// one item, stages the next item's descriptor, plan, blur taps and binned
// particle records into shared memory with cp.async.  An item renders the
// tile plus the blur halo into an on-chip fixed-point accumulator, finishes
// it, and writes every output pixel of the tile once.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "particle.cuh"
#include "phi_table.cuh"

namespace spx {

// ---------------------------------------------------------------------------
// asynchronous copies into shared memory
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// descriptor (128 B), plan (64 B), blur taps (128 B) of a pair
__device__ __forceinline__ void stage_header(const KernelArgs &a, int pair, unsigned char *buf) {
    const int t = threadIdx.x;
    if (t < 20) {
        const unsigned char *src;
        if (t < 8) src = reinterpret_cast<const unsigned char *>(a.descs + pair) + 16 * t;
        else if (t < 12) src = reinterpret_cast<const unsigned char *>(a.plan + pair) + 16 * (t - 8);
        else src = reinterpret_cast<const unsigned char *>(a.blur_w + (int64_t)pair * kBlurStride) + 16 * (t - 12);
        cp_async16(buf + 16 * t, src);
    }
}

// records [first, first + n) of the bins, copied in 16-byte chunks from the
// 16-byte boundary at or below the first record: record k of the span lands
// at dst + lead + 24 k with lead = (24 first) mod 16.
__device__ __forceinline__ void stage_records(const KernelArgs &a, int64_t first, uint32_t n, unsigned char *dst) {
    const int64_t start = first * (int64_t)sizeof(Record);
    const int64_t astart = start & ~(int64_t)15;
    const int64_t nbytes = (start - astart) + (int64_t)n * (int64_t)sizeof(Record);
    const int nchunks = (int)((nbytes + 15) >> 4);
    const unsigned char *base = reinterpret_cast<const unsigned char *>(a.rec) + astart;
    for (int c = threadIdx.x; c < nchunks; c += blockDim.x) cp_async16(dst + 16 * c, base + 16 * c);
}

__device__ __forceinline__ int record_lead(int64_t first) { return (int)((first * (int64_t)sizeof(Record)) & 15); }

// ---------------------------------------------------------------------------
// pixel integration of Eq. 1
// ---------------------------------------------------------------------------

// ---------------------------------------------------------------------------
// exact fixed-point accumulation
// ---------------------------------------------------------------------------
// A contribution v in [0, i_max] is scaled to u = v * 1024 / i_max and split
// into hi = rint(u) and lo = rint((u - hi) * 2^22), both found with the FP32
// round-to-integer identity (x + 1.5 * 2^23 leaves rint(x) in the low
// mantissa bits for |x| < 2^22).  The tile keeps int32 sums of hi and lo:
// integer addition is associative, so a pixel's value does not depend on the
// order of its contributions, the tile size or the batch it is rendered in.
// lo sums stay inside int32 for up to 1016 contributions; after every staged
// chunk of records (at most 1016) the multiples of 2^22 in lo are carried
// into hi.  Resolution 2^-32 i_max; pixel sums must stay below 2^21 i_max.
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr int32_t kMagicBits = 0x4B400000;

__device__ __forceinline__ void add_fixed(int32_t *hi, int32_t *lo, int idx, float u) {
    const float t = __fadd_rn(u, kMagic);
    const int32_t h = __float_as_int(t) - kMagicBits;
    const float r = __fsub_rn(u, __fsub_rn(t, kMagic));  // exact, |r| <= 1/2
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

struct Geo {
    int32_t W, H;
    int32_t x0, x1, y0, y1;      // tile pixels [x0, x1) x [y0, y1)
    int32_t ex0, ex1, ey0, ey1;  // halo-widened rectangle clipped to the frame
    int32_t EW, EH;              // its width and height (accumulator pitch EW)
    int32_t R;                   // blur radius = halo
    int32_t FW, FH;              // full halo rectangle (replicated outside the frame)
};

// Upper normal tail Q(t) = erfc(t / sqrt 2) / 2 for t >= 0 from the
// piecewise polynomial table (staged in shared memory as [coef][piece]).
__device__ __forceinline__ float phi_tail(float t, const float *tab) {
    const int k = min((int)(t * kPhiWidthInv), kPhiPieces - 1);
    const float s = t - fmaf((float)k, 1.0f / kPhiWidthInv, 0.5f / kPhiWidthInv);
    float acc = tab[kPhiDegree * kPhiPieces + k];
#pragma unroll
    for (int j = kPhiDegree - 1; j >= 0; --j) acc = fmaf(acc, s, tab[j * kPhiPieces + k]);
    return t < 8.0f ? acc : 0.0f;
}

// edge_value() evaluated from the table: Phi(t) for t <= 0, -(1 - Phi(t)) for t > 0.
__device__ __forceinline__ float edge_value_tab(float t, const float *tab) {
    const float q = phi_tail(fabsf(t), tab);
    return t > 0.0f ? -q : q;
}

// Large windows (more than 30 edges): per-warp scratch in shared memory.
__device__ __noinline__ void splat_particle_wide(const Geo &g, int32_t *hi, int32_t *lo, float px, float py,
                                                 int32_t ix, int32_t iy, float inv, float amps, int32_t j0,
                                                 int32_t i0, int nx, int ny, float *scr, int wq, const float *tab) {
    const int lane = threadIdx.x & 31;
    float *exe = scr, *eye = scr + wq, *ex = scr + 2 * wq, *ey = scr + 3 * wq;
    for (int e = lane; e <= nx; e += 32) exe[e] = edge_value_tab(((float)(j0 + e - ix) - px) * inv, tab);
    for (int e = lane; e <= ny; e += 32) eye[e] = edge_value_tab(((float)(i0 + e - iy) - py) * inv, tab);
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
        add_fixed(hi, lo, (i0 - g.ey0 + r) * g.EW + (j0 - g.ex0 + cc), __fmul_rn(ex[cc], ey[r]));
    }
    __syncwarp();
}

// Quotient of small non-negative integers a / b (a < 2^20, 1 <= b <= 2^10)
// from b's reciprocal: (a + 1/2) / b is at least 1/(2b) away from an integer,
// far more than the rounding error of the product.
__device__ __forceinline__ int small_div(int a, float inv_b) { return (int)(((float)a + 0.5f) * inv_b); }

// Splat n staged records.  A warp takes up to 32 records at a time (record
// warp + 8 l for lane l), sets each one up lane-parallel (window clipped to
// the halo rectangle, reciprocals), then renders them one after another:
// lanes [0, nx] evaluate the x edges, lanes [nx+1, nx+ny+1] the y edges;
// each lane then takes one column and every rpr-th row of the window.
__device__ __forceinline__ void splat_records(const unsigned char *recs, uint32_t n, const Geo &g, float scale,
                                              int32_t *hi, int32_t *lo, float *scr, int wq, const float *tab) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned FULL = 0xffffffffu;
    const uint32_t nw = blockDim.x >> 5;
    for (uint32_t k0 = warp; k0 < n; k0 += nw * 32) {
        const uint32_t k = k0 + nw * lane;
        float px = 0.f, py = 0.f, inv = 0.f, amps = 0.f, invn = 0.f;
        int32_t ix = 0, iy = 0, j0 = 0, i0 = 0, nx = 0, ny = 0;
        if (k < n) {
            const unsigned char *rp = recs + (size_t)k * sizeof(Record);
            const float2 pf = *reinterpret_cast<const float2 *>(rp);
            const int2 pi = *reinterpret_cast<const int2 *>(rp + 8);
            const float2 ps = *reinterpret_cast<const float2 *>(rp + 16);
            px = pf.x;
            py = pf.y;
            ix = pi.x;
            iy = pi.y;
            const float r15 = 6.0f * ps.x;  // 1.5 d
            j0 = max(ix + (int32_t)floorf(px - r15), g.ex0);
            const int32_t j1 = min(ix + (int32_t)floorf(px + r15), g.ex1 - 1);
            i0 = max(iy + (int32_t)floorf(py - r15), g.ey0);
            const int32_t i1 = min(iy + (int32_t)floorf(py + r15), g.ey1 - 1);
            if (j0 <= j1 && i0 <= i1) {
                nx = j1 - j0 + 1;
                ny = i1 - i0 + 1;
                inv = __frcp_rn(ps.x);
                amps = ps.y * scale;
                invn = __frcp_rn((float)nx);
            }
        }
        uint32_t todo = __ballot_sync(FULL, nx > 0);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int bnx = __shfl_sync(FULL, nx, src), bny = __shfl_sync(FULL, ny, src);
            const float bpx = __shfl_sync(FULL, px, src), bpy = __shfl_sync(FULL, py, src);
            const int32_t bix = __shfl_sync(FULL, ix, src), biy = __shfl_sync(FULL, iy, src);
            const int32_t bj0 = __shfl_sync(FULL, j0, src), bi0 = __shfl_sync(FULL, i0, src);
            const float binv = __shfl_sync(FULL, inv, src), bamps = __shfl_sync(FULL, amps, src);
            if (bnx + bny + 2 > 32) {
                splat_particle_wide(g, hi, lo, bpx, bpy, bix, biy, binv, bamps, bj0, bi0, bnx, bny, scr, wq, tab);
                continue;
            }
            const float binvn = __shfl_sync(FULL, invn, src);
            const int nxe = bnx + 1;
            const bool isx = lane < nxe;
            const int e = isx ? lane : lane - nxe;
            const float dd = isx ? (float)(bj0 + e - bix) - bpx : (float)(bi0 + e - biy) - bpy;
            const bool dpos = dd > 0.0f;
            const float ev = lane < nxe + bny + 1 ? edge_value_tab(dd * binv, tab) : 0.0f;
            const float evn = __shfl_down_sync(FULL, ev, 1);
            const bool dposn = __shfl_down_sync(FULL, (int)dpos, 1) != 0;
            float m = pixel_mass(ev, evn, dpos, dposn);
            if (!isx) m *= bamps;
            // lane -> (row offset lr, column lc); rpr rows per round
            const int rpr = small_div(32, binvn);
            const int lr = small_div(lane, binvn);
            const int lc = lane - lr * bnx;
            const float exv = __shfl_sync(FULL, m, lc);
            const bool act = lr < rpr;
            const int base = (bi0 - g.ey0 + lr) * g.EW + (bj0 - g.ex0 + lc);
            for (int r0 = 0; r0 < bny; r0 += rpr) {
                const int r = r0 + lr;
                const float eyv = __shfl_sync(FULL, m, nxe + min(r, bny - 1));
                if (act && r < bny) add_fixed(hi, lo, base + r0 * g.EW, __fmul_rn(exv, eyv));
            }
        }
    }
}

// ---------------------------------------------------------------------------
// epilogue helpers
// ---------------------------------------------------------------------------

// Box-Muller pair from two Philox words: r = sqrt(-2 ln u), theta = 2 pi v,
// evaluated as -r (cos, sin)(theta - pi) so the fast sine and cosine work on
// [-pi, pi).
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float &n0, float &n1) {
    const float x = -2.0f * logf(uo24f(wa));
    const float r = x > 0.0f ? x * rsqrtf(x) : 0.0f;
    float s, c;
    __sincosf(6.28318530717958647692f * (u24f(wb) - 0.5f), &s, &c);
    n0 = -r * c;
    n1 = -r * s;
}

template <typename T>
struct Out;
template <>
struct Out<float> {
    static __device__ __forceinline__ float cvt(float v) { return v; }
    static __device__ __forceinline__ void store4(float *p, const float *v) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <>
struct Out<__half> {
    static __device__ __forceinline__ __half cvt(float v) { return __float2half_rn(v); }
    static __device__ __forceinline__ void store4(__half *p, const float *v) {
        __half2 a = __floats2half2_rn(v[0], v[1]), b = __floats2half2_rn(v[2], v[3]);
        uint2 u;
        u.x = *reinterpret_cast<unsigned *>(&a);
        u.y = *reinterpret_cast<unsigned *>(&b);
        *reinterpret_cast<uint2 *>(p) = u;
    }
};
template <>
struct Out<__nv_bfloat16> {
    static __device__ __forceinline__ __nv_bfloat16 cvt(float v) { return __float2bfloat16_rn(v); }
    static __device__ __forceinline__ void store4(__nv_bfloat16 *p, const float *v) {
        __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]), b = __floats2bfloat162_rn(v[2], v[3]);
        uint2 u;
        u.x = *reinterpret_cast<unsigned *>(&a);
        u.y = *reinterpret_cast<unsigned *>(&b);
        *reinterpret_cast<uint2 *>(p) = u;
    }
};
template <>
struct Out<uint8_t> {
    static __device__ __forceinline__ uint8_t cvt(float v) { return (uint8_t)v; }
    static __device__ __forceinline__ void store4(uint8_t *p, const float *v) {
        *reinterpret_cast<uchar4 *>(p) = make_uchar4((uint8_t)v[0], (uint8_t)v[1], (uint8_t)v[2], (uint8_t)v[3]);
    }
};
template <>
struct Out<uint16_t> {
    static __device__ __forceinline__ uint16_t cvt(float v) { return (uint16_t)v; }
    static __device__ __forceinline__ void store4(uint16_t *p, const float *v) {
        *reinterpret_cast<ushort4 *>(p) =
            make_ushort4((uint16_t)v[0], (uint16_t)v[1], (uint16_t)v[2], (uint16_t)v[3]);
    }
};

// Store up to 4 consecutive outputs of a row (quantised when M > 0).
template <typename T>
__device__ __forceinline__ void store_group(T *o, float *v, int nvalid, float M) {
    if (M > 0.0f) {
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = fminf(fmaxf(rintf(v[j] * M), 0.0f), M);
    }
    if (nvalid == 4 && (reinterpret_cast<uintptr_t>(o) % (4 * sizeof(T))) == 0) {
        Out<T>::store4(o, v);
    } else {
        for (int j = 0; j < nvalid; ++j) o[j] = Out<T>::cvt(v[j]);
    }
}

// Horizontal pass (rows of the full halo rectangle, tile columns) and
// vertical pass with store; taps w[|k|], k = -R..R, replicate border already
// materialised in A.  R is a compile-time radius (0 < R <= 6).
template <typename T, int R>
__device__ __forceinline__ void blur_store(const Geo &g, const float *A, float *Bh, int BP, const float *w, T *out,
                                           float M) {
    const int TW = g.x1 - g.x0, TH = g.y1 - g.y0;
    const int G = (TW + 3) >> 2;
    const float iG = 1.0f / (float)G;
    float wr[R + 1];
#pragma unroll
    for (int k = 0; k <= R; ++k) wr[k] = w[k];
    for (int it = threadIdx.x; it < g.FH * G; it += blockDim.x) {
        const int r = small_div(it, iG), c0 = (it - r * G) * 4;
        const float *row = A + r * g.FW;
        float v[4 + 2 * R];
#pragma unroll
        for (int k = 0; k < 4 + 2 * R; ++k) v[k] = row[min(c0 + k, g.FW - 1)];
        float4 o;
        float *op = &o.x;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float acc = wr[0] * v[j + R];
#pragma unroll
            for (int k = 1; k <= R; ++k) acc = fmaf(wr[k], v[j + R - k] + v[j + R + k], acc);
            op[j] = acc;
        }
        *reinterpret_cast<float4 *>(Bh + r * BP + c0) = o;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < TH * G; it += blockDim.x) {
        const int r = small_div(it, iG), c0 = (it - r * G) * 4;
        const float4 *col = reinterpret_cast<const float4 *>(Bh + c0);
        const int p4 = BP >> 2;
        const float4 m0 = col[(r + R) * p4];
        float v[4] = {wr[0] * m0.x, wr[0] * m0.y, wr[0] * m0.z, wr[0] * m0.w};
#pragma unroll
        for (int k = 1; k <= R; ++k) {
            const float4 a = col[(r + R - k) * p4], b = col[(r + R + k) * p4];
            v[0] = fmaf(wr[k], a.x + b.x, v[0]);
            v[1] = fmaf(wr[k], a.y + b.y, v[1]);
            v[2] = fmaf(wr[k], a.z + b.z, v[2]);
            v[3] = fmaf(wr[k], a.w + b.w, v[3]);
        }
        store_group<T>(out + r * g.W + c0, v, min(4, TW - c0), M);
    }
}

// Any radius (slow path for R > 6), same arithmetic.
template <typename T>
__device__ __noinline__ void blur_store_any(const Geo &g, const float *A, float *Bh, int BP, const float *w, T *out,
                                            float M) {
    const int R = g.R, TW = g.x1 - g.x0, TH = g.y1 - g.y0;
    for (int it = threadIdx.x; it < g.FH * TW; it += blockDim.x) {
        const int r = it / TW, c = it - r * TW;
        const float *row = A + r * g.FW + c + R;
        float acc = w[0] * row[0];
        for (int k = 1; k <= R; ++k) acc = fmaf(w[k], row[-k] + row[k], acc);
        Bh[r * BP + c] = acc;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < TH * TW; it += blockDim.x) {
        const int r = it / TW, c = it - r * TW;
        const float *col = Bh + (r + R) * BP + c;
        float acc = w[0] * col[0];
        for (int k = 1; k <= R; ++k) acc = fmaf(w[k], col[-k * BP] + col[k * BP], acc);
        float v[4] = {acc, 0.f, 0.f, 0.f};
        store_group<T>(out + r * g.W + c, v, 1, M);
    }
}

template <typename T>
__device__ __forceinline__ void store_unblurred(const Geo &g, const float *A, T *out, float M) {
    const int TW = g.x1 - g.x0, TH = g.y1 - g.y0;
    const int G = (TW + 3) >> 2;
    for (int it = threadIdx.x; it < TH * G; it += blockDim.x) {
        const int r = it / G, c0 = (it - r * G) * 4;
        float v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = A[r * g.FW + min(c0 + j, g.FW - 1)];
        store_group<T>(out + r * g.W + c0, v, min(4, TW - c0), M);
    }
}

// ---------------------------------------------------------------------------
// one work item
// ---------------------------------------------------------------------------
struct Smem {
    int32_t *hi, *lo;
    float *A, *Bh, *sx2, *sy2, *scr, *phi;
    int BP;
};

__device__ __forceinline__ Geo make_geo(const synthpix_pair_desc &D, const PairPlan &pl, int tile_edge, int tile,
                                        int halo) {
    Geo g;
    g.W = D.width;
    g.H = D.height;
    const int ty = tile / pl.tiles_x, tx = tile - ty * pl.tiles_x;
    g.R = pl.blur_r;
    g.x0 = tx * tile_edge;
    g.x1 = min(g.x0 + tile_edge, g.W);
    g.y0 = ty * tile_edge;
    g.y1 = min(g.y0 + tile_edge, g.H);
    g.ex0 = max(g.x0 - halo, 0);
    g.ex1 = min(g.x1 + halo, g.W);
    g.ey0 = max(g.y0 - halo, 0);
    g.ey1 = min(g.y1 + halo, g.H);
    g.EW = g.ex1 - g.ex0;
    g.EH = g.ey1 - g.ey0;
    g.FW = (g.x1 - g.x0) + 2 * g.R;
    g.FH = (g.y1 - g.y0) + 2 * g.R;
    return g;
}

// separable illumination factors sin^2 of the clipped halo rectangle
__device__ __forceinline__ bool illum_factors(const Geo &g, const synthpix_pair_desc &D, const Smem &s) {
    const bool illum = D.illum_min != 1.0f || D.illum_max != 1.0f;
    if (illum) {
        for (int k = threadIdx.x; k < g.EW + g.EH; k += blockDim.x) {
            if (k < g.EW) {
                const float sv = sinpif(((float)(g.ex0 + k) + 0.5f) / (float)g.W);
                s.sx2[k] = sv * sv;
            } else {
                const float sv = sinpif(((float)(g.ey0 + k - g.EW) + 0.5f) / (float)g.H);
                s.sy2[k - g.EW] = sv * sv;
            }
        }
    }
    return illum;
}

// The finishing steps of one tile of one frame: A = L * S + sigma_n * n over
// the clipped halo rectangle, border replication, separable blur, store.
// src(idx, r, c) gives S at row r, column c of the clipped halo rectangle
// (idx = r * EW + c).  The illumination factors must be in s.sx2 / s.sy2 and
// visible (a barrier after illum_factors).
template <typename T, typename Src>
__device__ __forceinline__ void finish_tile(const KernelArgs &a, const Geo &g, const synthpix_pair_desc &D,
                                            const float *wtab, int frame, bool illum, const Smem &s, Src src) {
    const float dl = D.illum_max - D.illum_min;
    const int fx0 = g.x0 - g.R, fy0 = g.y0 - g.R;
    if (D.noise_sigma != 0.0f) {
        // 32-bit pixel indices: frames hold at most 32768^2 = 2^30 pixels
        const int nq = (g.EW + 6) / 4 + 1;
        const float inq = 1.0f / (float)nq;
        const uint32_t tag = kTagNoise + (uint32_t)frame;
        const int fpitch = g.FW;
        float *Abase = s.A + (g.ey0 - fy0) * fpitch + (g.ex0 - fx0);
        for (int item = threadIdx.x; item < g.EH * nq; item += blockDim.x) {
            const int r = small_div(item, inq), qi = item - r * nq;
            const int rowlin = (g.ey0 + r) * g.W;
            const int p0 = (((rowlin + g.ex0) >> 2) + qi) << 2;
            if (p0 > rowlin + g.ex1 - 1) continue;
            const uint4 w = stream_words(a.seed, D.pair_id, (uint32_t)(p0 >> 2), tag);
            float nv[4];
            box_muller(w.x, w.y, nv[0], nv[1]);
            box_muller(w.z, w.w, nv[2], nv[3]);
            const int c0 = p0 - rowlin - g.ex0;  // column of the quad's first pixel in the halo rectangle
            const float ly = illum ? s.sy2[r] : 0.0f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = c0 + k;
                if (c >= 0 && c < g.EW) {
                    const float S = src(r * g.EW + c, r, c);
                    const float L = illum ? fmaf(dl, s.sx2[c] * ly, D.illum_min) : 1.0f;
                    Abase[r * fpitch + c] = fmaf(L, S, D.noise_sigma * nv[k]);
                }
            }
        }
    } else {
        const float iew = 1.0f / (float)g.EW;
        for (int idx = threadIdx.x; idx < g.EH * g.EW; idx += blockDim.x) {
            const int r = small_div(idx, iew), c = idx - r * g.EW;
            const float S = src(idx, r, c);
            const float L = illum ? fmaf(dl, s.sx2[c] * s.sy2[r], D.illum_min) : 1.0f;
            s.A[(g.ey0 + r - fy0) * g.FW + (g.ex0 + c - fx0)] = L * S;
        }
    }
    __syncthreads();
    // replicate the border into the halo outside the frame
    if (g.R > 0 && (fx0 < 0 || fy0 < 0 || g.x1 + g.R > g.W || g.y1 + g.R > g.H)) {
        const float ifw = 1.0f / (float)g.FW;
        for (int k = threadIdx.x; k < g.FH * g.FW; k += blockDim.x) {
            const int r = small_div(k, ifw), c = k - r * g.FW;
            const int gi = fy0 + r, gj = fx0 + c;
            if (gi < 0 || gi >= g.H || gj < 0 || gj >= g.W) {
                const int ci = min(max(gi, 0), g.H - 1) - fy0, cj = min(max(gj, 0), g.W - 1) - fx0;
                s.A[k] = s.A[ci * g.FW + cj];
            }
        }
    }
    __syncthreads();
    const int64_t HW = (int64_t)g.H * g.W;
    // the tile's first output pixel; stores add 32-bit row / column offsets
    T *out = reinterpret_cast<T *>(a.images) + D.image_offset + (int64_t)frame * HW + (int64_t)g.y0 * g.W + g.x0;
    const float M = a.quant_bits > 0 ? (float)((1u << a.quant_bits) - 1u) : 0.0f;
    switch (g.R) {
    case 0: store_unblurred<T>(g, s.A, out, M); break;
    case 1: blur_store<T, 1>(g, s.A, s.Bh, s.BP, wtab, out, M); break;
    case 2: blur_store<T, 2>(g, s.A, s.Bh, s.BP, wtab, out, M); break;
    case 3: blur_store<T, 3>(g, s.A, s.Bh, s.BP, wtab, out, M); break;
    case 4: blur_store<T, 4>(g, s.A, s.Bh, s.BP, wtab, out, M); break;
    case 5: blur_store<T, 5>(g, s.A, s.Bh, s.BP, wtab, out, M); break;
    case 6: blur_store<T, 6>(g, s.A, s.Bh, s.BP, wtab, out, M); break;
    default: blur_store_any<T>(g, s.A, s.Bh, s.BP, wtab, out, M); break;
    }
}

template <typename I>
__device__ __forceinline__ I to_inter(float v);
template <>
__device__ __forceinline__ __half to_inter<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 to_inter<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// One work item of k_splat.  Fused (inter_dtype F32): splat the tile plus
// its blur halo and finish it on chip.  Otherwise splat the tile alone and
// store S in 16 bits to the intermediate frames; k_finish does the rest.
template <typename T>
__device__ __forceinline__ void process_item(const KernelArgs &a, const ItemInfo &it, unsigned char *buf,
                                             uint32_t cap, const Smem &s) {
    const synthpix_pair_desc &D = *reinterpret_cast<const synthpix_pair_desc *>(buf);
    const PairPlan &pl = *reinterpret_cast<const PairPlan *>(buf + 128);
    const float *wtab = reinterpret_cast<const float *>(buf + 192);
    const Geo g = make_geo(D, pl, a.tile, it.tile, pl.halo);
    const bool fused = a.inter_dtype == SYNTHPIX_F32;
    const bool illum = fused ? illum_factors(g, D, s) : false;

    // splat, chunk by chunk of staged records
    const float imax = D.i_max > 0.0f ? D.i_max : 1.0f;
    const float scale = 1024.0f / imax;
    uint32_t done = 0;
    while (done < it.count) {
        const uint32_t n = min(it.count - done, cap);
        splat_records(buf + kStageHeader + record_lead(it.rec0 + done), n, g, scale, s.hi, s.lo,
                      s.scr + (threadIdx.x >> 5) * a.warp_scratch, a.warp_scratch >> 2, s.phi);
        done += n;
        __syncthreads();
        if (done < it.count) {  // more records: carry lo before the next chunk (the last carry is in pass 1)
            carry_fixed(s.hi, s.lo, g.EH * g.EW);
            stage_records(a, it.rec0 + done, min(it.count - done, cap), buf + kStageHeader);
            cp_async_commit();
            cp_async_wait_all();
            __syncthreads();
        }
    }
    if (it.count == 0) __syncthreads();  // illumination factors

    const float unit = imax * (1.0f / 1024.0f);
    int32_t *hi = s.hi, *lo = s.lo;
    // S from the fixed-point sums, carrying lo into hi on the fly; each pixel
    // is read once, and its accumulator cleared for the next item
    auto fixed_src = [hi, lo, unit](int idx, int, int) {
        const int32_t l = lo[idx], c = l >> 22;
        const float v = fmaf((float)(l - (c << 22)), 1.0f / 4194304.0f, (float)(hi[idx] + c)) * unit;
        hi[idx] = 0;
        lo[idx] = 0;
        return v;
    };
    if (!fused) {
        // halo 0: the clipped rectangle is the tile
        const int64_t HW = (int64_t)g.H * g.W;
        const int64_t base = pl.inter_base + (int64_t)it.frame * HW;
        const float iew = 1.0f / (float)g.EW;
        for (int idx = threadIdx.x; idx < g.EH * g.EW; idx += blockDim.x) {
            const int r = small_div(idx, iew), c = idx - r * g.EW;
            const float S = fixed_src(idx, r, c);
            const int64_t o = base + (int64_t)(g.ey0 + r) * g.W + (g.ex0 + c);
            if (a.inter_dtype == SYNTHPIX_F16) reinterpret_cast<__half *>(a.inter)[o] = to_inter<__half>(S);
            else reinterpret_cast<__nv_bfloat16 *>(a.inter)[o] = to_inter<__nv_bfloat16>(S);
        }
        return;  // the caller's loop ends with a barrier
    }
    finish_tile<T>(a, g, D, wtab, it.frame, illum, s, fixed_src);
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
struct SmemLayout {
    size_t hi, lo, A, Bh, sx2, sy2, scr, phi, bufs, total;
};

__host__ __device__ inline SmemLayout smem_layout(int E, int tile, int warp_scratch, int rec_buf_bytes) {
    SmemLayout L;
    const int BP = (tile + 3) & ~3;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = (o + bytes + 15) & ~(size_t)15;
        return at;
    };
    L.hi = take((size_t)E * E * 4);
    L.lo = take((size_t)E * E * 4);
    L.A = take((size_t)E * E * 4);
    L.Bh = take((size_t)E * BP * 4);
    L.sx2 = take((size_t)E * 4);
    L.sy2 = take((size_t)E * 4);
    L.scr = take((size_t)(kSplatMaxThreads / 32) * warp_scratch * 4);
    L.phi = take((size_t)(kPhiDegree + 1) * kPhiPieces * 4);
    L.bufs = take(2 * (size_t)rec_buf_bytes);
    L.total = o;
    return L;
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) k_splat(KernelArgs a) {
    if (*a.check != 1) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ItemInfo s_item[2];
    const SmemLayout L = smem_layout(a.smem_edge, a.tile, a.warp_scratch, a.rec_buf_bytes);
    Smem s;
    s.hi = reinterpret_cast<int32_t *>(smem + L.hi);
    s.lo = reinterpret_cast<int32_t *>(smem + L.lo);
    s.A = reinterpret_cast<float *>(smem + L.A);
    s.Bh = reinterpret_cast<float *>(smem + L.Bh);
    s.sx2 = reinterpret_cast<float *>(smem + L.sx2);
    s.sy2 = reinterpret_cast<float *>(smem + L.sy2);
    s.scr = reinterpret_cast<float *>(smem + L.scr);
    s.phi = reinterpret_cast<float *>(smem + L.phi);
    for (int k = threadIdx.x; k < (kPhiDegree + 1) * kPhiPieces; k += blockDim.x) s.phi[k] = kPhiTable[k];
    s.BP = (a.tile + 3) & ~3;
    unsigned char *bufs = smem + L.bufs;
    const uint32_t cap = (uint32_t)((a.rec_buf_bytes - kStageHeader - 32) / (int)sizeof(Record));
    const int E2 = a.smem_edge * a.smem_edge;
    for (int k = threadIdx.x; k < E2; k += blockDim.x) {
        s.hi[k] = 0;
        s.lo[k] = 0;
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < 2; ++q) {
            const uint32_t t = atomicAdd(a.ticket, 1u);
            ItemInfo it;
            if ((int64_t)t < a.n_tiles) it = a.items[t];
            else it.pair = -1;
            s_item[q] = it;
        }
    }
    __syncthreads();
    if (s_item[0].pair < 0) return;
    stage_header(a, s_item[0].pair, bufs);
    stage_records(a, s_item[0].rec0, min(s_item[0].count, cap), bufs + kStageHeader);
    cp_async_commit();
    int cur = 0;
    for (;;) {
        const ItemInfo it = s_item[cur];
        const ItemInfo nx = s_item[cur ^ 1];
        cp_async_wait_all();
        __syncthreads();  // staged data of `it` visible; the other buffer is free
        if (it.pair < 0) break;
        unsigned char *bnext = bufs + (cur ^ 1) * a.rec_buf_bytes;
        if (nx.pair >= 0) {
            stage_header(a, nx.pair, bnext);
            stage_records(a, nx.rec0, min(nx.count, cap), bnext + kStageHeader);
        }
        cp_async_commit();
        uint32_t t2 = 0;
        if (threadIdx.x == 0) t2 = atomicAdd(a.ticket, 1u);
        process_item<T>(a, it, bufs + cur * a.rec_buf_bytes, cap, s);
        if (threadIdx.x == 0) {
            ItemInfo after;
            if ((int64_t)t2 < a.n_tiles) after = a.items[t2];
            else after.pair = -1;
            s_item[cur] = after;
        }
        cur ^= 1;
        __syncthreads();
    }
    cp_async_wait_all();
}

// ---------------------------------------------------------------------------
// k_finish: the epilogue of the 16-bit intermediate path, one CTA per item
// (pair, frame, tile).  S of the tile and its blur halo is read from the
// intermediate frames written by k_splat; every output pixel written once.
// ---------------------------------------------------------------------------
struct FinishLayout {
    size_t A, Bh, sx2, sy2, total;
};

__host__ __device__ inline FinishLayout finish_layout(int E, int tile) {
    FinishLayout L;
    const int BP = (tile + 3) & ~3;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = (o + bytes + 15) & ~(size_t)15;
        return at;
    };
    L.A = take((size_t)E * E * 4);
    L.Bh = take((size_t)E * BP * 4);
    L.sx2 = take((size_t)E * 4);
    L.sy2 = take((size_t)E * 4);
    L.total = o;
    return L;
}

template <typename T, typename I>
__global__ void __launch_bounds__(kSplatThreads) k_finish(KernelArgs a) {
    if (*a.check != 1) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float wtab[kBlurStride];
    const FinishLayout FL = finish_layout(a.smem_edge, a.tile);
    Smem s;
    s.hi = s.lo = nullptr;
    s.A = reinterpret_cast<float *>(smem + FL.A);
    s.Bh = reinterpret_cast<float *>(smem + FL.Bh);
    s.sx2 = reinterpret_cast<float *>(smem + FL.sx2);
    s.sy2 = reinterpret_cast<float *>(smem + FL.sy2);
    s.scr = nullptr;
    s.phi = nullptr;
    s.BP = (a.tile + 3) & ~3;
    const ItemInfo it = a.items[blockIdx.x];
    const synthpix_pair_desc &D = a.descs[it.pair];
    const PairPlan pl = a.plan[it.pair];
    if (threadIdx.x < kBlurStride) wtab[threadIdx.x] = a.blur_w[(int64_t)it.pair * kBlurStride + threadIdx.x];
    const Geo g = make_geo(D, pl, a.tile, it.tile, pl.blur_r);
    const bool illum = illum_factors(g, D, s);
    __syncthreads();
    const I *S16 = reinterpret_cast<const I *>(a.inter) + pl.inter_base + (int64_t)it.frame * g.H * g.W;
    const int W = g.W, ex0 = g.ex0, ey0 = g.ey0;
    auto src = [S16, W, ex0, ey0](int, int r, int c) {
        return (float)S16[(int64_t)(ey0 + r) * W + (ex0 + c)];
    };
    finish_tile<T>(a, g, D, wtab, it.frame, illum, s, src);
}

size_t splat_smem_bytes(int edge, int tile, int warp_scratch, int rec_buf_bytes) {
    return smem_layout(edge, tile, warp_scratch, rec_buf_bytes).total;
}

cudaError_t launch_splat(const KernelArgs &a, int32_t out_dtype, cudaStream_t st, cudaEvent_t const *ev) {
    const size_t smem = splat_smem_bytes(a.smem_edge, a.tile, a.warp_scratch, a.rec_buf_bytes);
    int dev = 0, nsm = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
#define SPX_LAUNCH(T)                                                                                        \
    do {                                                                                                     \
        if (a.tile >= 64) {                                                                                  \
            e = cudaFuncSetAttribute(k_splat<T, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);\
            if (e != cudaSuccess) return e;                                                                  \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_splat<T, 512>, 512, smem);             \
            if (e != cudaSuccess) return e;                                                                  \
            const int64_t want = (int64_t)nsm * (occ > 0 ? occ : 1);                                         \
            k_splat<T, 512><<<(unsigned)(a.n_tiles < want ? a.n_tiles : want), 512, smem, st>>>(a);          \
        } else {                                                                                             \
            e = cudaFuncSetAttribute(k_splat<T, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);\
            if (e != cudaSuccess) return e;                                                                  \
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_splat<T, 256>, 256, smem);             \
            if (e != cudaSuccess) return e;                                                                  \
            const int64_t want = (int64_t)nsm * (occ > 0 ? occ : 1);                                         \
            k_splat<T, 256><<<(unsigned)(a.n_tiles < want ? a.n_tiles : want), 256, smem, st>>>(a);          \
        }                                                                                                    \
    } while (0)
    switch (out_dtype) {
    case SYNTHPIX_F32: SPX_LAUNCH(float); break;
    case SYNTHPIX_F16: SPX_LAUNCH(__half); break;
    case SYNTHPIX_BF16: SPX_LAUNCH(__nv_bfloat16); break;
    case SYNTHPIX_U8: SPX_LAUNCH(uint8_t); break;
    default: SPX_LAUNCH(uint16_t); break;
    }
#undef SPX_LAUNCH
    if (a.inter_dtype != SYNTHPIX_F32) {
        const size_t fsm = finish_layout(a.smem_edge, a.tile).total;
        const unsigned grid = (unsigned)a.n_tiles;
#define SPX_FINISH(T, I)                                                                                     \
    do {                                                                                                     \
        e = cudaFuncSetAttribute(k_finish<T, I>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);     \
        if (e != cudaSuccess) return e;                                                                      \
        k_finish<T, I><<<grid, kSplatThreads, fsm, st>>>(a);                                                 \
    } while (0)
#define SPX_FINISH_I(I)                                                                                      \
    switch (out_dtype) {                                                                                     \
    case SYNTHPIX_F32: SPX_FINISH(float, I); break;                                                          \
    case SYNTHPIX_F16: SPX_FINISH(__half, I); break;                                                         \
    case SYNTHPIX_BF16: SPX_FINISH(__nv_bfloat16, I); break;                                                 \
    case SYNTHPIX_U8: SPX_FINISH(uint8_t, I); break;                                                         \
    default: SPX_FINISH(uint16_t, I); break;                                                                 \
    }
        if (a.inter_dtype == SYNTHPIX_F16) {
            SPX_FINISH_I(__half)
        } else {
            SPX_FINISH_I(__nv_bfloat16)
        }
#undef SPX_FINISH_I
#undef SPX_FINISH
    }
    if (ev && ev[5]) cudaEventRecord(ev[5], st);
    return cudaGetLastError();
}

}  // namespace spx
