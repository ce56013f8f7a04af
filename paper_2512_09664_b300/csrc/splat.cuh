// The splat + epilogue of the PIV image-pair renderer (SynthPix, arXiv
// 2512.09664, Section 2): Eq. 1 integrated over each pixel and summed over
// the particles ("aggregation of the particle contributions"), then the
// imaging steps named in the Abstract (illumination non-uniformity, noise,
// blur) and quantisation.
//
// k_splat is persistent: each CTA takes (pair, frame, tile) work items from a
// ticket counter (atomicAdd, no waiting on other CTAs) and stages the next
// item's descriptor, plan and blur taps while it renders one item, and the
// next item's binned particle records while it finishes one (they take the
// record region the splatted records leave), into shared memory with
// cp.async.  An item renders the
// tile plus the blur halo into an on-chip fixed-point accumulator, finishes
// it, and writes every output pixel of the tile once.
//
// This header holds the device code; splat_<type>.cu instantiate the kernels
// of one output type each (compiled in parallel) and splat.cu dispatches.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "particle.cuh"
#include "phi.cuh"

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

// descriptor, plan and blur taps (128 B) of a pair, in 16-byte copies
__device__ __forceinline__ void stage_header(const KernelArgs &a, int pair, unsigned char *buf) {
    constexpr int kD = kStageDesc / 16, kP = kStagePlan / 16, kH = kStageHeader / 16;
    const int t = threadIdx.x;
    if (t < kH) {
        const unsigned char *src;
        if (t < kD) src = reinterpret_cast<const unsigned char *>(a.descs + pair) + 16 * t;
        else if (t < kP) src = reinterpret_cast<const unsigned char *>(a.plan + pair) + 16 * (t - kD);
        else src = reinterpret_cast<const unsigned char *>(a.blur_w + (int64_t)pair * kBlurStride) + 16 * (t - kP);
        cp_async16(buf + 16 * t, src);
    }
}

// records [first, first + n) of the bins (RS bytes each), copied in 16-byte
// chunks from the 16-byte boundary at or below the first record: record k of
// the span lands at dst + lead + RS k with lead = (RS first) mod 16.
template <int RS>
__device__ __forceinline__ void stage_records(const KernelArgs &a, int64_t first, uint32_t n, unsigned char *dst) {
    const int64_t start = first * (int64_t)RS;
    const int64_t astart = start & ~(int64_t)15;
    const int64_t nbytes = (start - astart) + (int64_t)n * (int64_t)RS;
    const int nchunks = (int)((nbytes + 15) >> 4);
    const unsigned char *base = reinterpret_cast<const unsigned char *>(a.rec) + astart;
    for (int c = threadIdx.x; c < nchunks; c += blockDim.x) cp_async16(dst + 16 * c, base + 16 * c);
}

template <int RS>
__device__ __forceinline__ int record_lead(int64_t first) { return (int)((first * (int64_t)RS) & 15); }

// ---------------------------------------------------------------------------
// exact fixed-point accumulation
// ---------------------------------------------------------------------------
// A pixel sums integer contributions in units q = i_max 2^-26 in a 32-bit
// word of shared memory.  Integer addition is associative: a pixel's value
// does not depend on the order of its contributions, the tile size or the
// batch it is rendered in.
//
// Round particles: the x mass of a window column (at most 1) is held as
// mq = rint(m 2^31) and the row mass times the amplitude as
// yq = rint(m_y amp 2^27 / i_max); the contribution is the high word of
// their 64-bit product, mq yq 2^-32 = m_x m_y amp / q, truncated (error
// below 1.3 q; one integer multiply per pixel, no float-to-integer
// conversion).  General particles round their FP32 pixel value once.  A
// contribution is at most i_max (the pixel mass of a unit Gaussian is at
// most 1 / (sqrt(2 pi) sigma) per axis), i.e. at most 2^26 units.
//
// A word holds 64 i_max.  Before a chunk of visits is splatted, the visits
// of the item so far are counted per 8 x 8 block of the accumulator; while
// no block is met by more than 63 visits, no pixel sum can reach 2^32 units
// and the adds go unchecked.  Otherwise the chunk takes the checked path:
// the thread whose add wraps a word adds 1 to the pixel's carry word (worth
// 2^32 units), so no sum is ever lost.
constexpr float kFixedScale = 67108864.0f;      // 2^26 units per i_max
constexpr float kFixedUnit = 1.0f / 67108864.0f;
constexpr float kWrapValue = 4294967296.0f;     // 2^32: the weight of a carry
constexpr float kMassScale = 2147483648.0f;     // 2^31: x masses as integers
constexpr uint32_t kSafeVisits = 63;            // visits per block that cannot wrap a word
constexpr int kBlkShift = 3;                    // 8 x 8 pixel blocks
constexpr int kBlkSide = 24;                    // blocks per side of the counter grid (row pitch <= 192)
constexpr int kBlkPitch = kBlkSide + 1;         // counter rows padded: a lane per row hits its own bank

// Tile geometry of one work item.  The accumulator and the finishing buffer A
// share memory: the full halo rectangle [x0 - R, x1 + R) x [y0 - R, y1 + R)
// from column afx0 (x0 - R rounded down to a multiple of 4) with row pitch AP,
// so quads of 4 pixels are 16-byte aligned.  Particles are splatted into its
// part inside the frame, the halo-widened rectangle clipped to the frame
// (from column ax0, ex0 rounded down to a multiple of 4, P columns); the first
// finishing pass turns those words into A in place, and the pixels outside
// the frame take replicated border values.
struct Geo {
    int32_t W, H;
    int32_t x0, x1, y0, y1;      // tile pixels [x0, x1) x [y0, y1)
    int32_t ex0, ex1, ey0, ey1;  // halo-widened rectangle clipped to the frame
    int32_t EW, EH;              // its width and height
    int32_t R;                   // blur radius
    int32_t ax0, P;              // accumulator: first column, row pitch
    int32_t fx0, fy0, FW, FH;    // full halo rectangle (may leave the frame)
    int32_t afx0, AP;            // accumulator = finishing buffer: first column, row pitch
    int32_t aoff;                // index of (ey0, ax0) in it (rows from fy0, columns from afx0)
};

// Visit classes of the splat's sort (see splat_chunk): windows of at most
// 2 (c + 1) pixels a side for c < kWideClass, wider ones in kWideClass;
// 32 accumulator-bank buckets per class.
constexpr int kNarrowMax = 16;
constexpr int kWideClass = kNarrowMax / 2;
constexpr int kBuckets = (kWideClass + 1) * 32;

// Sort and work-queue state of a k_splat CTA (static shared memory).
static __shared__ uint32_t sh_cnt[kBuckets];              // visits of the chunk per (class, bank) key
static __shared__ uint32_t sh_off[kBuckets + 1];          // their exclusive offsets
static __shared__ uint32_t sh_next;                       // warp-slot ticket of the chunk's render
static __shared__ uint32_t sh_slot_end[kWideClass + 1];   // slots of the classes, widest first: cumulative ends
// The visits of the item so far per 8 x 8 block, as a difference array
// along each block row: a visit whose window meets blocks [bx0, bx1] of rows
// [by0, by1] adds +1 at bx0 and -1 at bx1 + 1 of each of those rows (two
// adds per row, at most three rows for windows up to 17 px); the counts are
// the rows' prefix sums (blocks_checked).  Column kBlkSide holds the end
// marks of windows reaching the last block.
static __shared__ uint32_t sh_blk[kBlkPitch * kBlkSide];
static __shared__ int sh_checked;                         // the chunk takes the checked path
static __shared__ int sh_carry_clean;                     // the item's carry words are zero
static __shared__ int sh_wrap;                            // a checked add wrapped a word in this item
// The next work item's raw fields, copied in by cp.async while the current
// item renders: ItemInfo (24 bytes), the bin's counter, the overflow flags.
static __shared__ __align__(16) uint32_t sh_raw[10];
static __shared__ uint32_t sh_tk;  // its ticket

__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async8(void *smem_dst, const void *gsrc) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
// Thread 0: copy the fields of work item t into sh_raw (nothing past the queue).
__device__ __forceinline__ void fetch_item(const KernelArgs &a, uint32_t t) {
    sh_tk = t;
    if ((int64_t)t >= a.n_tiles) return;
    const uint32_t *src = reinterpret_cast<const uint32_t *>(a.items + t);
    for (int k = 0; k < 3; ++k) cp_async8(sh_raw + 2 * k, src + 2 * k);
    if (a.tiled) {
        cp_async4(sh_raw + 6, a.count + t);
        cp_async4(sh_raw + 7, a.ovf);
        cp_async4(sh_raw + 8, a.ovf + 1);
    }
    cp_async_commit();
}
// Thread 0, once its copies are complete: the fetched work item (work_item's rule).
__device__ __forceinline__ ItemInfo fetched_item(const KernelArgs &a) {
    const uint32_t t = sh_tk;
    ItemInfo it;
    if ((int64_t)t >= a.n_tiles) {
        it.pair = -1;
        return it;
    }
    it = *reinterpret_cast<const ItemInfo *>(sh_raw);
    if (a.tiled && (it.frame ? sh_raw[8] : sh_raw[7]) == 0u) it.count = min(it.count, sh_raw[6]);
    return it;
}

// Count a visit whose clipped window is [j0, j1] x [i0, i1] (frame pixels)
// in the blocks it meets.
__device__ __forceinline__ void count_blocks(const Geo &g, int32_t j0, int32_t j1, int32_t i0, int32_t i1) {
    const int bx0 = (j0 - g.afx0) >> kBlkShift, bx1 = ((j1 - g.afx0) >> kBlkShift) + 1;
    const int by0 = (i0 - g.fy0) >> kBlkShift, by1 = (i1 - g.fy0) >> kBlkShift;
    for (int by = by0; by <= by1; ++by) {
        atomicAdd(sh_blk + by * kBlkPitch + bx0, 1u);
        atomicAdd(sh_blk + by * kBlkPitch + bx1, 0xFFFFFFFFu);
    }
}

// Warp 0, after the counts of a chunk: true when some block has been met by
// more than kSafeVisits visits of the item (a lane per block row sums its
// row's differences).
__device__ __forceinline__ bool blocks_checked() {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    uint32_t mx = 0;
    if (lane < kBlkSide) {
        uint32_t run = 0;
#pragma unroll 8
        for (int c = 0; c < kBlkSide; ++c) {
            run += sh_blk[lane * kBlkPitch + c];
            mx = max(mx, run);
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) mx = max(mx, __shfl_xor_sync(FULL, mx, d));
    return mx > kSafeVisits;
}

// The tile's accumulator as the splat sees it.
struct Acc {
    uint32_t acc;     // .shared address of word 0 ([rows][P] words)
    uint32_t *carry;  // the CTA's carry words in global memory, same indices
    int P;
};

// x mass (in [0, 1]) as an integer of 2^-31; row mass times the doubled
// amplitude (amps2 = 2 amp 2^26 / i_max) as an integer
__device__ __forceinline__ uint32_t mass_q31(float m) { return __float2uint_rn(__fmul_rn(m, kMassScale)); }
__device__ __forceinline__ uint32_t row_q(float m, float amps2) { return __float2uint_rn(__fmul_rn(m, amps2)); }

// Add u units to the word at .shared address w.
template <bool CHECKED>
__device__ __forceinline__ void add_units(uint32_t w, const Acc &A, uint32_t u) {
    if (!CHECKED) {
        sh_red_add<0>(w, u);
        return;
    }
    const uint32_t old = sh_atom_add(w, u);
    if (old + u < old) {
        atomicAdd(A.carry + ((w - A.acc) >> 2), 1u);
        sh_wrap = 1;
    }
}

// Adds of one window row: column C gets hi(mx[C] my) at byte offset 4 C.
template <int C, int N>
struct RowAdds {
    static __device__ __forceinline__ void run(uint32_t row, const uint32_t (&mx)[N], uint32_t my) {
        sh_red_add<4 * C>(row, __umulhi(mx[C], my));
        RowAdds<C + 1, N>::run(row, mx, my);
    }
};
template <int N>
struct RowAdds<N, N> {
    static __device__ __forceinline__ void run(uint32_t, const uint32_t (&)[N], uint32_t) {}
};

// One particle's visit of a tile, set up for the splat (same size as a
// Record, written over the staged records it comes from).
struct Visit {
    float px, py;    // fractions of the split position
    float inv;       // 1 / sigma
    float amps;      // 2 * amplitude * 2^26 / i_max (row masses times it give yq)
    int32_t base;    // accumulator index of the clipped window's first pixel
    uint32_t shape;  // bx | by << 8 (int8: window start - integer position) | nx << 16 | ny << 24
};
static_assert(sizeof(Visit) == sizeof(Record), "Visit layout");

__device__ __forceinline__ int visit_bx(uint32_t s) { return (int)(int8_t)(s & 0xFFu); }
__device__ __forceinline__ int visit_by(uint32_t s) { return (int)(int8_t)((s >> 8) & 0xFFu); }
__device__ __forceinline__ int visit_nx(uint32_t s) { return (int)((s >> 16) & 0xFFu); }
__device__ __forceinline__ int visit_ny(uint32_t s) { return (int)(s >> 24); }

// Visits are sorted by (class, accumulator bank) before the splat.  Class
// c < 8 holds windows of at most N = 2 (c + 1) pixels a side; each is
// rendered by a group of U = class_lanes(c) adjacent lanes (splat_group):
// the lanes share the N + 1 x edges and take RG = class_rows(c) rows each.
// Class 8 holds the wider windows, rendered by a whole warp per visit, four
// visits per warp slot (more slots spread the long wide visits over the
// warps: with 32 per slot a few warps held them all while the rest waited
// at the chunk's barrier); its slots come first and are rendered by a loop of
// their own, so the narrow classes' loop keeps its registers.  The visits of one warp are spread over the bank
// order, so their accumulator addresses fall in different banks.
__host__ __device__ constexpr int class_lanes(int c) { return c < 2 ? 1 : 2; }
// log2 of the visits one warp slot of class c renders (32 / lanes per visit; 4 for the wide class)
__host__ __device__ constexpr int class_slot_shift(int c) { return c >= 8 ? 2 : (c < 2 ? 5 : 4); }
__host__ __device__ constexpr int class_rows(int c) { return c == 0 ? 2 : (c == 1 ? 4 : c + 1); }

// Quotient of small non-negative integers a / b (a < 2^20, 1 <= b <= 2^10)
// from b's reciprocal: (a + 1/2) / b is at least 1/(2b) away from an integer,
// far more than the rounding error of the product.
__device__ __forceinline__ int small_div(int a, float inv_b) { return (int)(((float)a + 0.5f) * inv_b); }

// One visit per group of U lanes, window at most N x N.  Lane j of the group
// evaluates the x edges e = j + U k and the masses that start there; the
// group exchanges them (as integers) by shuffles, then lane j renders rows
// [j RG, j RG + RG) of the window.  Columns past the window's nx get mass 0:
// their adds land inside the accumulator (its rows are at least 16 words
// apart from the window's right edge or end in its padding) and add nothing,
// so the row needs no per-column test.  All lanes of the warp take part (the
// shuffles); lanes of an empty visit add nothing.
template <int N, int U, int RG>
__device__ __forceinline__ void splat_group(const Visit &v, const Acc &A, uint32_t tab) {
    static_assert(U * RG >= N, "rows of a window");
    constexpr int EPL = (N + U) / U;  // ceil((N + 1) / U) x edges per lane
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, j = lane & (U - 1), gbase = lane & ~(U - 1);
    const int nx = visit_nx(v.shape), ny = visit_ny(v.shape);
    const float fbx = (float)(visit_bx(v.shape) + j);
    float ev[EPL];
#pragma unroll
    for (int k = 0; k < EPL; ++k) ev[k] = edge_value_tab(__fsub_rn(__fadd_rn(fbx, (float)(U * k)), v.px), v.inv, tab);
    uint32_t mq[EPL];
#pragma unroll
    for (int k = 0; k < EPL; ++k) {
        float nb;
        if (U == 1) {
            nb = ev[k + 1 < EPL ? k + 1 : k];
        } else {
            const float a = __shfl_sync(FULL, ev[k], lane + 1);                  // edge e + 1 of lanes j < U - 1
            const float b = __shfl_sync(FULL, ev[k + 1 < EPL ? k + 1 : k], gbase);  // of lane U - 1
            nb = j == U - 1 ? b : a;
        }
        mq[k] = mass_q31(edge_mass(ev[k], nb));
    }
    uint32_t mx[N];
#pragma unroll
    for (int e = 0; e < N; ++e) {
        const uint32_t m = U == 1 ? mq[e] : __shfl_sync(FULL, mq[e / U], gbase + e % U);
        mx[e] = e < nx ? m : 0u;
    }
    const int r0 = j * RG;
    const int rows = min(max(ny - r0, 0), RG);
    const float fby = (float)(visit_by(v.shape) + r0);
    float ey = edge_value_tab(__fsub_rn(fby, v.py), v.inv, tab);
    uint32_t row = A.acc + 4u * (uint32_t)(v.base + r0 * A.P);
    const uint32_t pitch = 4u * (uint32_t)A.P;
#pragma unroll 1  // a rolled row loop keeps the class templates small enough for the instruction cache
    for (int q = 0; q < rows; ++q) {
        const float en = edge_value_tab(__fsub_rn(__fadd_rn(fby, (float)(q + 1)), v.py), v.inv, tab);
        const uint32_t my = row_q(edge_mass(ey, en), v.amps);
        ey = en;
        RowAdds<0, N>::run(row, mx, my);
        row += pitch;
    }
}

// Windows with more edges than lanes (out of line: the inlined renders keep
// their registers).  Up to 64 edges: two per lane, entries k = lane and
// k = lane + 32 of the x edges 0..nx followed by the y edges 0..ny; lane c
// owns columns c and c + 32 and walks the rows, each row's mass broadcast by
// one shuffle.  Wider windows: per-warp scratch in shared memory.
template <bool CHECKED>
__device__ __noinline__ void splat_particle_wide(const Acc A, float px, float py, float inv,
                                                 float amps, int32_t base, int bx, int by, int nx, int ny,
                                                 float *scr, int wq, uint32_t tab) {
    const int lane = threadIdx.x & 31;
    if (nx + ny + 2 <= 64) {
        const unsigned FULL = 0xffffffffu;
        auto edge = [&](int k) {
            const float dd = k <= nx ? __fsub_rn((float)(bx + k), px) : __fsub_rn((float)(by + k - nx - 1), py);
            return k < nx + ny + 2 ? edge_value_tab(dd, inv, tab) : 0.0f;
        };
        const float e0 = edge(lane), e1 = edge(lane + 32);
        const float e1l0 = __shfl_sync(FULL, e1, 0);
        float n0 = __shfl_down_sync(FULL, e0, 1);
        if (lane == 31) n0 = e1l0;
        const float n1 = __shfl_down_sync(FULL, e1, 1);
        const float m0 = edge_mass(e0, n0), m1 = edge_mass(e1, n1);
        // x masses as q31, row masses (entries past nx) times the amplitude
        const uint32_t q0 = lane > nx ? row_q(m0, amps) : mass_q31(m0);
        const uint32_t q1 = lane + 32 > nx ? row_q(m1, amps) : mass_q31(m1);
        const uint32_t col = A.acc + 4u * (uint32_t)(base + lane);
        for (int r = 0; r < ny; ++r) {
            const int k = nx + 1 + r;  // uniform across the warp
            const uint32_t my = k < 32 ? __shfl_sync(FULL, q0, k) : __shfl_sync(FULL, q1, k - 32);
            const uint32_t w = col + 4u * (uint32_t)(r * A.P);
            if (lane < nx) add_units<CHECKED>(w, A, __umulhi(q0, my));
            if (lane + 32 < nx) add_units<CHECKED>(w + 128u, A, __umulhi(q1, my));
        }
        return;
    }
    uint32_t *exe = reinterpret_cast<uint32_t *>(scr), *eye = exe + wq, *ex = exe + 2 * wq, *ey = exe + 3 * wq;
    for (int e = lane; e <= nx; e += 32)
        exe[e] = __float_as_uint(edge_value_tab(__fsub_rn((float)(bx + e), px), inv, tab));
    for (int e = lane; e <= ny; e += 32)
        eye[e] = __float_as_uint(edge_value_tab(__fsub_rn((float)(by + e), py), inv, tab));
    __syncwarp();
    for (int e = lane; e < nx; e += 32) ex[e] = mass_q31(edge_mass(__uint_as_float(exe[e]), __uint_as_float(exe[e + 1])));
    for (int e = lane; e < ny; e += 32) ey[e] = row_q(edge_mass(__uint_as_float(eye[e]), __uint_as_float(eye[e + 1])), amps);
    __syncwarp();
    const int n = nx * ny;
    const float invx = 1.0f / (float)nx;
    for (int m = lane; m < n; m += 32) {
        const int r = min((int)(((float)m + 0.5f) * invx), ny - 1);
        const int cc = m - r * nx;
        if ((unsigned)cc >= (unsigned)nx) continue;
        add_units<CHECKED>(A.acc + 4u * (uint32_t)(base + r * A.P + cc), A, __umulhi(ex[cc], ey[r]));
    }
    __syncwarp();
}

// Wide visits, a warp per visit: lanes [0, nx] evaluate the x edges, lanes
// [nx+1, nx+ny+1] the y edges; each lane then takes one column and every
// rpr-th row of the window.  Windows with more edges than lanes go through
// splat_particle_wide.
template <bool CHECKED>
__device__ __forceinline__ void splat_coop(const Visit &v, bool valid, const Acc &A, float *scr,
                                           int wq, uint32_t tab) {
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    uint32_t todo = __ballot_sync(FULL, valid);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const float px = __shfl_sync(FULL, v.px, src), py = __shfl_sync(FULL, v.py, src);
        const float inv = __shfl_sync(FULL, v.inv, src), amps = __shfl_sync(FULL, v.amps, src);
        const int32_t base = __shfl_sync(FULL, v.base, src);
        const uint32_t shape = __shfl_sync(FULL, v.shape, src);
        const int nx = visit_nx(shape), ny = visit_ny(shape), bx = visit_bx(shape), by = visit_by(shape);
        if (nx + ny + 2 > 32) {
            splat_particle_wide<CHECKED>(A, px, py, inv, amps, base, bx, by, nx, ny, scr, wq, tab);
            continue;
        }
        const int nxe = nx + 1;
        const bool isx = lane < nxe;
        const int e = isx ? lane : lane - nxe;
        const float dd = __fsub_rn((float)((isx ? bx : by) + e), isx ? px : py);
        const float ev = lane < nxe + ny + 1 ? edge_value_tab(dd, inv, tab) : 0.0f;
        const float evn = __shfl_down_sync(FULL, ev, 1);
        const float m = edge_mass(ev, evn);
        const uint32_t q = isx ? mass_q31(m) : row_q(m, amps);
        // lane -> (row offset lr, column lc); rpr rows per round
        const float invn = __frcp_rn((float)nx);
        const int rpr = small_div(32, invn);
        const int lr = small_div(lane, invn);
        const int lc = lane - lr * nx;
        const uint32_t exq = __shfl_sync(FULL, q, lc);
        const bool act = lr < rpr;
        const uint32_t dst = A.acc + 4u * (uint32_t)(base + lr * A.P + lc);
        const uint32_t step = 4u * (uint32_t)(rpr * A.P);
        uint32_t w = dst;
        for (int r0 = 0; r0 < ny; r0 += rpr) {
            const int r = r0 + lr;
            const uint32_t eyq = __shfl_sync(FULL, q, nxe + min(r, ny - 1));
            if (act && r < ny) add_units<CHECKED>(w, A, __umulhi(exq, eyq));
            w += step;
        }
    }
}


// Splat n staged records (at recs) into the tile's accumulator:
//   A. each thread sets up its records' visits (window clipped to the halo
//      rectangle), takes a slot in its (class, bank) bucket and counts the
//      visit in the 8 x 8 blocks its window meets;
//   B. warp 0 scans the bucket counts, and warp 1 decides from the block
//      counts whether the chunk's adds must be checked for wrapping;
//   C. the visits are written in key order over the staged records (out);
//   D. warps claim slots of 32 visits, widest class first, and render them
//      (checked: every visit by a whole warp, with checked adds).
// fetch_t: thread 0 starts the copy of work item fetch_t (fetch_item) after
// the first barrier (~0u: none).
template <int NT>
__device__ __forceinline__ void splat_chunk(const unsigned char *recs, unsigned char *out, uint32_t n, const Geo &g,
                                            float scale, const Acc &acc, float *scr,
                                            int wq, uint32_t tab, const KernelArgs &a, uint32_t fetch_t) {
    constexpr int RPT = kSplatRpt;  // n <= RPT NT (k_splat caps its chunks)
    const int lane = threadIdx.x & 31;
    const unsigned FULL = 0xffffffffu;
    Visit v[RPT];
    int key[RPT];
    uint32_t slot[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        const uint32_t k = threadIdx.x + (uint32_t)q * NT;
        key[q] = -1;
        slot[q] = 0;
        if (k < n) {
            const unsigned char *rp = recs + (size_t)k * sizeof(Record);
            const float2 pf = *reinterpret_cast<const float2 *>(rp);
            const int2 pi = *reinterpret_cast<const int2 *>(rp + 8);
            const float2 ps = *reinterpret_cast<const float2 *>(rp + 16);
            const float r15 = 6.0f * ps.x;  // 1.5 d
            const int32_t j0 = max(pi.x + (int32_t)floorf(pf.x - r15), g.ex0);
            const int32_t j1 = min(pi.x + (int32_t)floorf(pf.x + r15), g.ex1 - 1);
            const int32_t i0 = max(pi.y + (int32_t)floorf(pf.y - r15), g.ey0);
            const int32_t i1 = min(pi.y + (int32_t)floorf(pf.y + r15), g.ey1 - 1);
            if (j0 <= j1 && i0 <= i1) {
                const int nx = j1 - j0 + 1, ny = i1 - i0 + 1;
                v[q].px = pf.x;
                v[q].py = pf.y;
                v[q].inv = __frcp_rn(ps.x);
                v[q].amps = ps.y * (2.0f * scale);  // doubled amplitude units (row_q)
                v[q].base = (i0 - g.fy0) * g.AP + (j0 - g.afx0);
                v[q].shape = ((uint32_t)(j0 - pi.x) & 0xFFu) | (((uint32_t)(i0 - pi.y) & 0xFFu) << 8) |
                             ((uint32_t)nx << 16) | ((uint32_t)ny << 24);
                const int m = max(nx, ny);
                const int cls = m > kNarrowMax ? kWideClass : (m - 1) >> 1;
                key[q] = cls * 32 + (v[q].base & 31);
                slot[q] = atomicAdd(sh_cnt + key[q], 1u);
                count_blocks(g, j0, j1, i0, i1);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && fetch_t != ~0u) fetch_item(a, fetch_t);
    if (threadIdx.x < 32) {
        constexpr int PER = kBuckets / 32;
        uint32_t c[PER], sum = 0;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            c[j] = sh_cnt[lane * PER + j];
            sh_cnt[lane * PER + j] = 0;
            sum += c[j];
        }
        uint32_t incl = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, incl, d);
            if (lane >= d) incl += t;
        }
        uint32_t run = incl - sum;
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            sh_off[lane * PER + j] = run;
            run += c[j];
        }
        if (lane == 31) sh_off[kBuckets] = incl;
        if (lane == 0) sh_next = 0;
        __syncwarp();
        // warp slots per class (widest first) and their cumulative ends
        uint32_t nsl = 0;
        if (lane <= kWideClass) {
            const int cc = kWideClass - lane;
            const uint32_t G = sh_off[32 * cc + 32] - sh_off[32 * cc];
            const int sh = class_slot_shift(cc);
            nsl = (G + (1u << sh) - 1u) >> sh;
        }
#pragma unroll
        for (int d = 1; d < 16; d <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, nsl, d);
            if (lane >= d) nsl += t;
        }
        if (lane <= kWideClass) sh_slot_end[lane] = nsl;
    } else if (threadIdx.x < 64) {  // warp 1: the wrap guard's block counts, beside warp 0's scan
        const bool ck = blocks_checked();
        if (lane == 0) sh_checked = ck ? 1 : 0;
    }
    __syncthreads();
    float2 *o8 = reinterpret_cast<float2 *>(out);  // 16-byte aligned; a Visit is three 8-byte words
    const bool chk = sh_checked != 0;
    if (chk && !sh_carry_clean) {  // the item's first checked chunk: clear the CTA's carry words
        uint4 *cw = reinterpret_cast<uint4 *>(acc.carry);
        for (int k = threadIdx.x; k < (g.FH * g.AP) >> 2; k += blockDim.x) cw[k] = make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
        if (key[q] >= 0) {
            const uint32_t p = sh_off[key[q]] + slot[q];
            o8[3 * p] = make_float2(v[q].px, v[q].py);
            o8[3 * p + 1] = make_float2(v[q].inv, v[q].amps);
            o8[3 * p + 2] = make_float2(__int_as_float(v[q].base), __uint_as_float(v[q].shape));
        }
    }
    __syncthreads();
    if (chk) {  // dense item: a warp per visit, adds checked for wrapping
        if (threadIdx.x == 0) sh_carry_clean = 1;  // read again after this chunk's last barrier
        const uint32_t total = sh_off[kBuckets];
        for (;;) {
            uint32_t sl = 0;
            if (lane == 0) sl = atomicAdd(&sh_next, 1u);
            sl = __shfl_sync(FULL, sl, 0);
            if (sl * 32 >= total) break;
            const uint32_t idx = sl * 32 + lane;
            const bool valid = idx < total;
            Visit e;
            e.px = e.py = e.inv = e.amps = 0.0f;
            e.base = 0;
            e.shape = 0;
            if (valid) {
                const float2 a = o8[3 * idx], b = o8[3 * idx + 1], d = o8[3 * idx + 2];
                e.px = a.x;
                e.py = a.y;
                e.inv = b.x;
                e.amps = b.y;
                e.base = __float_as_int(d.x);
                e.shape = __float_as_uint(d.y);
            }
            splat_coop<true>(e, valid, acc, scr, wq, tab);
        }
        return;
    }
    const uint32_t total_slots = sh_slot_end[kWideClass];
    const uint32_t my_end = lane <= kWideClass ? sh_slot_end[lane] : 0xffffffffu;
    const uint32_t wide_end = sh_slot_end[0];  // the wide class's slots come first
    auto claim = [&]() {
        uint32_t t = 0;
        if (lane == 0) t = atomicAdd(&sh_next, 1u);
        return __shfl_sync(FULL, t, 0);
    };
    uint32_t sl = claim();
    {  // the wide class: a warp per visit, four visits per slot
        const uint32_t g0 = sh_off[32 * kWideClass], G = sh_off[32 * kWideClass + 32] - g0;
        for (; sl < wide_end; sl = claim()) {
            const uint32_t idx = (sl << class_slot_shift(kWideClass)) + lane;
            const bool valid = lane < (1 << class_slot_shift(kWideClass)) && idx < G;
            Visit e;
            e.px = e.py = e.inv = e.amps = 0.0f;
            e.base = 0;
            e.shape = 0;
            if (valid) {
                const float2 a = o8[3 * (g0 + idx)], b = o8[3 * (g0 + idx) + 1], d = o8[3 * (g0 + idx) + 2];
                e.px = a.x;
                e.py = a.y;
                e.inv = b.x;
                e.amps = b.y;
                e.base = __float_as_int(d.x);
                e.shape = __float_as_uint(d.y);
            }
            splat_coop<false>(e, valid, acc, scr, wq, tab);
        }
    }
    for (; sl < total_slots; sl = claim()) {
        // the slot's class: the first (widest-first) class whose slots end beyond sl
        const int o = __ffs(__ballot_sync(FULL, sl < my_end)) - 1;
        const int c = kWideClass - o;
        const uint32_t sc = sl - (o ? __shfl_sync(FULL, my_end, o - 1) : 0u);  // slot within the class
        const uint32_t g0 = sh_off[32 * c], G = sh_off[32 * c + 32] - g0;
        const int csh = class_slot_shift(c);
        const uint32_t nw = (G + (1u << csh) - 1u) >> csh;  // slots of the class
        // group q of U lanes takes visit sc + q nw (spread over the bank order)
        const uint32_t idx = sc + (uint32_t)(lane >> (5 - csh)) * nw;
        const bool valid = idx < G;
        Visit e;
        if (valid) {
            const float2 a = o8[3 * (g0 + idx)], b = o8[3 * (g0 + idx) + 1], d = o8[3 * (g0 + idx) + 2];
            e.px = a.x;
            e.py = a.y;
            e.inv = b.x;
            e.amps = b.y;
            e.base = __float_as_int(d.x);
            e.shape = __float_as_uint(d.y);
        } else {
            e.px = e.py = e.inv = e.amps = 0.0f;
            e.base = 0;
            e.shape = 0;
        }
        switch (c) {
        case 0: splat_group<2, class_lanes(0), class_rows(0)>(e, acc, tab); break;
        case 1: splat_group<4, class_lanes(1), class_rows(1)>(e, acc, tab); break;
        case 2: splat_group<6, class_lanes(2), class_rows(2)>(e, acc, tab); break;
        case 3: splat_group<8, class_lanes(3), class_rows(3)>(e, acc, tab); break;
        case 4: splat_group<10, class_lanes(4), class_rows(4)>(e, acc, tab); break;
        case 5: splat_group<12, class_lanes(5), class_rows(5)>(e, acc, tab); break;
        case 6: splat_group<14, class_lanes(6), class_rows(6)>(e, acc, tab); break;
        default: splat_group<16, class_lanes(7), class_rows(7)>(e, acc, tab); break;
        }
    }
}

// ---------------------------------------------------------------------------
// general particle shapes (Eq. 1 with sigma_x != sigma_y or rho != 0)
// ---------------------------------------------------------------------------
// The 4-node Gauss-Legendre rule on [-1, 1]: nodes +-0.8611363115940526 and
// +-0.3399810435848563 (the roots of P_4), weights 0.3478548451374538 and
// 0.6521451548625461.

// rho = 0 (axis-aligned ellipse), a warp per visit: lanes [0, nx] evaluate
// the x edges (1 / sigma_x), lanes [nx + 1, nx + ny + 1] the y edges
// (1 / sigma_y), then the lanes take the window's pixels 32 at a time and
// fetch their column and row masses by shuffles.  Windows with more edges
// than lanes evaluate both masses per pixel.
template <bool CHECKED>
__device__ __forceinline__ void splat_general_sep(const RecordG &r, int32_t j0, int32_t i0, int nx, int ny,
                                                  float amps, uint32_t w0, const Acc &acc, uint32_t tab) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const float isx = 1.0f / r.sx, isy = 1.0f / r.sy;
    const int npx = nx * ny;
    const float invn = __frcp_rn((float)nx);
    // an edge's offset from the centre: (edge - integer part) - fraction, one rounding, so the
    // values do not depend on where the tile clips the window
    if (nx + ny + 2 <= 32) {
        const bool isx_lane = lane <= nx;
        const int e = isx_lane ? lane : lane - (nx + 1);
        const float dd = isx_lane ? __fsub_rn((float)(j0 + e - r.ix), r.fx) : __fsub_rn((float)(i0 + e - r.iy), r.fy);
        const float ev = lane <= nx + ny + 1 ? edge_value_tab(dd, isx_lane ? isx : isy, tab) : 0.0f;
        float m = edge_mass(ev, __shfl_down_sync(FULL, ev, 1));
        if (!isx_lane) m = __fmul_rn(m, amps);
        for (int b = 0; b < npx; b += 32) {
            const int p = min(b + lane, npx - 1);
            const int rr = small_div(p, invn), cc = p - rr * nx;
            const float mx = __shfl_sync(FULL, m, cc), my = __shfl_sync(FULL, m, nx + 1 + rr);
            if (b + lane < npx)
                add_units<CHECKED>(w0 + 4u * (uint32_t)(rr * acc.P + cc), acc, __float2uint_rn(__fmul_rn(mx, my)));
        }
        return;
    }
    for (int p = lane; p < npx; p += 32) {
        const int rr = small_div(p, invn), cc = p - rr * nx;
        const int jc = j0 + cc - r.ix, ir = i0 + rr - r.iy;
        const float mx = edge_mass(edge_value_tab(__fsub_rn((float)jc, r.fx), isx, tab),
                                   edge_value_tab(__fsub_rn((float)(jc + 1), r.fx), isx, tab));
        const float my = edge_mass(edge_value_tab(__fsub_rn((float)ir, r.fy), isy, tab),
                                   edge_value_tab(__fsub_rn((float)(ir + 1), r.fy), isy, tab));
        add_units<CHECKED>(w0 + 4u * (uint32_t)(rr * acc.P + cc), acc, __float2uint_rn(__fmul_rn(mx, __fmul_rn(my, amps))));
    }
}

// rho != 0, a warp per visit.  The pixel's probability is the x-marginal
// times the conditional mass of y (normal, mean rho sigma_y u / sigma_x at
// offset u, std sigma_y sqrt(1 - rho^2)), exact in y and integrated in x by
// the 4-node Gauss-Legendre rule on M equal sub-intervals of the pixel.  The
// Q = 4 M nodes of a window column go to a group of G = min(Q, 32) lanes
// (Q / G nodes each); walking down the column, each lane carries its nodes'
// last edge value to the next row, and the group sums the row's node masses
// by shuffles.
template <int M, bool CHECKED>
__device__ __forceinline__ void splat_general_corr(const RecordG &r, int32_t j0, int32_t i0, int nx, int ny,
                                                   float amps, uint32_t w0, const Acc &acc, uint32_t tab) {
    constexpr int Q = 4 * M, G = Q < 32 ? Q : 32, L = Q / G, CPP = 32 / G;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, gl = lane & (G - 1), gc = lane / G;
    const float c = sqrtf(1.0f - r.rho * r.rho);
    const float isx = 1.0f / r.sx, is = 1.0f / (r.sy * c), k = r.rho * r.sy * isx;
    constexpr float h = 1.0f / (float)M;
    const float wscale = 0.5f * h * isx * 0.39894228040143267794f * amps;  // h/2, 1/(sqrt(2 pi) sigma_x), units
    // this lane's nodes: offsets within the pixel and weights (same for every column)
    float du[L], wq[L];
#pragma unroll
    for (int t = 0; t < L; ++t) {
        const int n = gl + G * t, g4 = n & 3;
        const float xg = g4 == 0 ? -0.8611363115940526f : g4 == 1 ? -0.3399810435848563f
                       : g4 == 2 ? 0.3399810435848563f : 0.8611363115940526f;
        du[t] = h * ((float)(n >> 2) + 0.5f * (xg + 1.0f));
        wq[t] = (g4 == 0 || g4 == 3) ? 0.3478548451374538f : 0.6521451548625461f;
    }
    for (int c0 = 0; c0 < nx; c0 += CPP) {
        const int col = c0 + gc;
        const bool live = col < nx;
        // offsets from the centre formed from exact integers (one rounding each), so the
        // values do not depend on where the tile clips the window
        const float ul = __fsub_rn((float)(j0 + col - r.ix), r.fx);  // the column's left edge
        const float fy = r.fy;
        float wn[L], mu[L], ev[L];
#pragma unroll
        for (int t = 0; t < L; ++t) {
            const float u = __fadd_rn(ul, du[t]);
            const float tt = u * isx;
            wn[t] = live ? wq[t] * __expf(-0.5f * tt * tt) * wscale : 0.0f;
            mu[t] = k * u;  // conditional mean of y at this node
            ev[t] = edge_value_tab(__fsub_rn(__fsub_rn((float)(i0 - r.iy), fy), mu[t]), is, tab);
        }
        const uint32_t wc = w0 + 4u * (uint32_t)col;
#pragma unroll 1
        for (int rr = 0; rr < ny; ++rr) {
            float v = 0.0f;
            const float ye = __fsub_rn((float)(i0 + rr + 1 - r.iy), fy);  // the row's lower edge
#pragma unroll
            for (int t = 0; t < L; ++t) {
                const float en = edge_value_tab(__fsub_rn(ye, mu[t]), is, tab);
                v = fmaf(wn[t], edge_mass(ev[t], en), v);
                ev[t] = en;
            }
#pragma unroll
            for (int o = G >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
            if (gl == 0 && live) add_units<CHECKED>(wc + 4u * (uint32_t)(rr * acc.P), acc, __float2uint_rn(v));
        }
    }
}

// rho != 0 with windows at most 32 / S columns wide: the same quadrature,
// S lanes per (column, chunk of rows), each lane summing Q / S <= 8 of the
// Q = 4 M nodes (consecutive ones, in node order).  The window's columns
// repeat floor(32 / (S nx)) times across the warp, each copy taking its own
// chunk of rows; walking down its rows a lane carries its nodes' last edge
// values, the S partial sums meet by butterfly shuffles, and the column's
// first lane adds the pixel.  A pixel's value depends only on its offset
// from the particle, not on the tile's clipping of the window nor on the
// lanes that compute it.
template <int M, int S, bool CHECKED>
__device__ __forceinline__ void splat_general_corr_cols(const RecordG &r, int32_t j0, int32_t i0, int nx, int ny,
                                                        float amps, uint32_t w0, const Acc &acc,
                                                        uint32_t tab) {
    constexpr int Q = 4 * M, QL = Q / S;
    static_assert(QL >= 1 && QL <= 8 && (S & (S - 1)) == 0, "at most 8 nodes per lane");
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int span = S * nx;       // lanes of one copy of the window's columns (<= 32)
    const int nch = 32 / span;     // copies across the warp, each with its chunk of rows
    const int chunk = lane / span, within = lane - chunk * span;
    const int col = within / S, sub = within & (S - 1);
    const int rpc = (ny + nch - 1) / nch;  // rows per chunk (the loop below is warp-uniform)
    const bool live = chunk < nch;
    const int r0 = chunk * rpc;
    const float c = sqrtf(1.0f - r.rho * r.rho);
    const float isx = 1.0f / r.sx, is = 1.0f / (r.sy * c), k = r.rho * r.sy * isx;
    constexpr float h = 1.0f / (float)M;
    const float wscale = 0.5f * h * isx * 0.39894228040143267794f * amps;  // h/2, 1/(sqrt(2 pi) sigma_x), units
    // offsets from the centre formed from exact integers (one rounding each)
    const float ul = __fsub_rn((float)(j0 + col - r.ix), r.fx);  // the column's left edge
    const float yt = __fsub_rn((float)(i0 + r0 - r.iy), r.fy);   // the top edge of the chunk's first row
    float wn[QL], mu[QL], ev[QL];
#pragma unroll
    for (int q = 0; q < QL; ++q) {
        const int t = sub * QL + q, g4 = t & 3;
        const float xg = g4 == 0 ? -0.8611363115940526f : g4 == 1 ? -0.3399810435848563f
                       : g4 == 2 ? 0.3399810435848563f : 0.8611363115940526f;
        const float wgt = (g4 == 0 || g4 == 3) ? 0.3478548451374538f : 0.6521451548625461f;
        const float u = __fadd_rn(ul, h * ((float)(t >> 2) + 0.5f * (xg + 1.0f)));
        const float tt = u * isx;
        wn[q] = wgt * __expf(-0.5f * tt * tt) * wscale;
        mu[q] = k * u;  // conditional mean of y at this node
        ev[q] = edge_value_tab(__fsub_rn(yt, mu[q]), is, tab);
    }
    const uint32_t wc = w0 + 4u * (uint32_t)col;
#pragma unroll 1
    for (int i = 0; i < rpc; ++i) {
        const int rr = r0 + i;
        const float ye = __fsub_rn((float)(i0 + rr + 1 - r.iy), r.fy);  // the row's lower edge
        float v = 0.0f;
#pragma unroll
        for (int q = 0; q < QL; ++q) {
            const float en = edge_value_tab(__fsub_rn(ye, mu[q]), is, tab);
            v = fmaf(wn[q], edge_mass(ev[q], en), v);
            ev[q] = en;
        }
#pragma unroll
        for (int o = S >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        if (live && sub == 0 && rr < ny) add_units<CHECKED>(wc + 4u * (uint32_t)(rr * acc.P), acc, __float2uint_rn(v));
    }
}

// Sub-intervals of the x quadrature of a correlated particle: a power of two
// no smaller than 1 / min(sigma_x, sigma_x sqrt(1 - rho^2) / |rho|) (the
// integrand's shortest x-scale; quadrature error below 1e-7 of I0), at most 64.
__device__ __forceinline__ int corr_subintervals(float sx, float rho) {
    const float c = sqrtf(1.0f - rho * rho);
    const float ell = fabsf(rho) > c ? sx * c / fabsf(rho) : sx;
    const int m = min(max((int)ceilf(1.0f / ell), 1), 64);
    return 1 << (32 - __clz(m - 1));  // next power of two (1 stays 1)
}

template <bool CHECKED>
__device__ __forceinline__ void splat_general_visit(const RecordG &r, int32_t j0, int32_t i0, int nx, int ny,
                                                    float amps, uint32_t w0, const Acc &acc, uint32_t tab) {
    if (r.rho == 0.0f) {
        splat_general_sep<CHECKED>(r, j0, i0, nx, ny, amps, w0, acc, tab);
        return;
    }
    const int m = corr_subintervals(r.sx, r.rho);
    if (m <= 8) {
        // lanes per column: at most 8 nodes per lane; the particle's unclipped window
        // width (not the tile's clipping of it) decides, so every tile renders it the same way
        const int lpc = m <= 2 ? 1 : m / 2;
        const float r15x = 6.0f * r.sx;
        const int width = (int)floorf(r.fx + r15x) - (int)floorf(r.fx - r15x) + 1;
        if (width * lpc <= 32) {
            switch (m) {
            case 1: splat_general_corr_cols<1, 1, CHECKED>(r, j0, i0, nx, ny, amps, w0, acc, tab); break;
            case 2: splat_general_corr_cols<2, 1, CHECKED>(r, j0, i0, nx, ny, amps, w0, acc, tab); break;
            case 4: splat_general_corr_cols<4, 2, CHECKED>(r, j0, i0, nx, ny, amps, w0, acc, tab); break;
            default: splat_general_corr_cols<8, 4, CHECKED>(r, j0, i0, nx, ny, amps, w0, acc, tab); break;
            }
            return;
        }
    }
    switch (m) {
    case 1: splat_general_corr<1, CHECKED>(r, j0, i0, nx, ny, amps, w0, acc, tab); break;
    case 2: splat_general_corr<2, CHECKED>(r, j0, i0, nx, ny, amps, w0, acc, tab); break;
    case 4: splat_general_corr<4, CHECKED>(r, j0, i0, nx, ny, amps, w0, acc, tab); break;
    case 8: splat_general_corr<8, CHECKED>(r, j0, i0, nx, ny, amps, w0, acc, tab); break;
    case 16: splat_general_corr<16, CHECKED>(r, j0, i0, nx, ny, amps, w0, acc, tab); break;
    case 32: splat_general_corr<32, CHECKED>(r, j0, i0, nx, ny, amps, w0, acc, tab); break;
    default: splat_general_corr<64, CHECKED>(r, j0, i0, nx, ny, amps, w0, acc, tab); break;
    }
}

// A general record's window clipped to the tile's halo rectangle (empty: j0 > j1).
__device__ __forceinline__ void general_window(const RecordG &r, const Geo &g, int32_t &j0, int32_t &j1, int32_t &i0,
                                               int32_t &i1) {
    const float r15x = 6.0f * r.sx, r15y = 6.0f * r.sy;  // 1.5 d, 1.5 d_y
    j0 = max(r.ix + (int32_t)floorf(r.fx - r15x), g.ex0);
    j1 = min(r.ix + (int32_t)floorf(r.fx + r15x), g.ex1 - 1);
    i0 = max(r.iy + (int32_t)floorf(r.fy - r15y), g.ey0);
    i1 = min(r.iy + (int32_t)floorf(r.fy + r15y), g.ey1 - 1);
}

// Splat n staged general records:
//   A. each thread counts its records' windows in the 8 x 8 blocks they meet
//      (the item's counts so far, as in splat_chunk);
//   B. warp 0 decides whether the chunk's adds must be checked for wrapping;
//   C. warps take records from a shared counter, a warp per record.
__device__ __forceinline__ void splat_chunk_general(const unsigned char *recs, uint32_t n, const Geo &g, float scale,
                                                    const Acc &acc, uint32_t tab, const KernelArgs &a,
                                                    uint32_t fetch_t) {
    const RecordG *R = reinterpret_cast<const RecordG *>(recs);
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) {
        int32_t j0, j1, i0, i1;
        general_window(R[k], g, j0, j1, i0, i1);
        if (j0 > j1 || i0 > i1) continue;
        count_blocks(g, j0, j1, i0, i1);
    }
    __syncthreads();
    if (threadIdx.x == 0 && fetch_t != ~0u) fetch_item(a, fetch_t);
    if (threadIdx.x < 32) {
        const bool ck = blocks_checked();
        if (lane == 0) {
            sh_checked = ck ? 1 : 0;
            sh_next = 0;
        }
    }
    __syncthreads();
    const bool chk = sh_checked != 0;
    if (chk) {
        if (!sh_carry_clean) {  // the item's first checked chunk: clear the CTA's carry words
            uint4 *cw = reinterpret_cast<uint4 *>(acc.carry);
            for (int k = threadIdx.x; k < (g.FH * g.AP) >> 2; k += blockDim.x) cw[k] = make_uint4(0u, 0u, 0u, 0u);
        }
        __syncthreads();
        if (threadIdx.x == 0) sh_carry_clean = 1;  // read again only after the chunk's last barrier
    }
    for (;;) {
        uint32_t k = 0;
        if (lane == 0) k = atomicAdd(&sh_next, 1u);
        k = __shfl_sync(FULL, k, 0);
        if (k >= n) break;
        const RecordG r = R[k];
        int32_t j0, j1, i0, i1;
        general_window(r, g, j0, j1, i0, i1);
        if (j0 > j1 || i0 > i1) continue;
        const uint32_t w0 = acc.acc + 4u * (uint32_t)((i0 - g.fy0) * acc.P + (j0 - g.afx0));
        const float amps = r.amp * scale;
        if (chk) splat_general_visit<true>(r, j0, i0, j1 - j0 + 1, i1 - i0 + 1, amps, w0, acc, tab);
        else splat_general_visit<false>(r, j0, i0, j1 - j0 + 1, i1 - i0 + 1, amps, w0, acc, tab);
    }
}

// ---------------------------------------------------------------------------
// epilogue helpers
// ---------------------------------------------------------------------------

// -2 ln u for u = uo24(w) = ((w >> 8) + 1) 2^-24 in (0, 1].  With x = 1 - u
// (exact in FP32): for x < 2^-8 the series -ln(1 - x) = x + x^2/2 + x^3/3 +
// x^4/4 (truncation below 1e-10 relative); otherwise -2 ln 2 log2(u) from
// the hardware base-2 logarithm, whose absolute error (about 2^-22 on
// log2) is then at most 3e-5 of the result, i.e. below 2e-6 on the normal
// deviate (and below 5e-8 of full scale at a noise sigma of 0.02).
__device__ __forceinline__ float neg2_log_uo24(uint32_t w) {
    const float u = uo24f(w);
    const float x = 1.0f - u;
    const float series = 2.0f * x * fmaf(x, fmaf(x, fmaf(x, 0.25f, 1.0f / 3.0f), 0.5f), 1.0f);
    const float viaLog2 = -1.38629436111989061883f * __log2f(u);  // -2 ln 2 log2(u)
    return x < 0.00390625f ? series : viaLog2;
}

// Box-Muller pair from two Philox words, times the noise sigma sn:
// r = sqrt(-2 ln u), theta = 2 pi v, evaluated as -(sn r) (cos, sin)(theta - pi)
// so the fast sine and cosine work on [-pi, pi).  sqrt(x) = x rsqrt(x), with
// x raised to at least 1e-30 inside the rsqrt so that x = 0 (u = 1) gives 0
// (the smallest positive x, -2 ln(1 - 2^-24), is far above it).
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float sn, float &n0, float &n1) {
    const float x = neg2_log_uo24(wa);
    const float r = sn * (x * rsqrtf(fmaxf(x, 1e-30f)));
    float s, c;
    __sincosf(6.28318530717958647692f * (u24f(wb) - 0.5f), &s, &c);
    n0 = -r * c;
    n1 = -r * s;
}

// Quantised code clamp(rint(v M), 0, M): v saturated to [0, 1] first (NaN
// gives 0), then the product rounded half to even by one FMA with 1.5 2^23
// (exact for products below 2^22; M <= 65535).  quant_raw returns the bit
// pattern of that sum, 0x4B400000 + code: its low 16 bits are the code.
__device__ __forceinline__ uint32_t quant_raw(float v, float M) {
    return __float_as_uint(fmaf(__saturatef(v), M, kMagic));
}
__device__ __forceinline__ uint32_t quant_code(float v, float M) { return quant_raw(v, M) - (uint32_t)kMagicBits; }

// Four codes packed from their raw patterns: bytes (8-bit codes) or 16-bit halves.
__device__ __forceinline__ uint32_t pack_u8(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3) {
    return __byte_perm(__byte_perm(r0, r1, 0x0040), __byte_perm(r2, r3, 0x0040), 0x5410);
}
__device__ __forceinline__ uint2 pack_u16(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3) {
    return make_uint2(__byte_perm(r0, r1, 0x5410), __byte_perm(r2, r3, 0x5410));
}

// Packed FP32 pairs (two lanes of one 64-bit register; each lane rounds as
// the scalar instruction would, so results equal the scalar arithmetic).
__device__ __forceinline__ unsigned long long f2_pack(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
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
struct IsCode {
    static constexpr bool value = false;
};
template <>
struct IsCode<uint8_t> {
    static constexpr bool value = true;
};
template <>
struct IsCode<uint16_t> {
    static constexpr bool value = true;
};

template <typename T>
__device__ __forceinline__ void store_group(T *o, float *v, int nvalid, float M) {
    if constexpr (IsCode<T>::value) {
        if (M > 0.0f) {
            // Q = clamp(rint(B M), 0, M)
            uint32_t q[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) q[j] = quant_raw(v[j], M);
            if (nvalid == 4 && (reinterpret_cast<uintptr_t>(o) % (4 * sizeof(T))) == 0) {
                if (sizeof(T) == 1) *reinterpret_cast<uint32_t *>(o) = pack_u8(q[0], q[1], q[2], q[3]);
                else *reinterpret_cast<uint2 *>(o) = pack_u16(q[0], q[1], q[2], q[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (j < nvalid) o[j] = (T)(q[j] - (uint32_t)kMagicBits);
            }
            return;
        }
    }
    if (M > 0.0f) {
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = (float)quant_code(v[j], M);
    }
    if (nvalid == 4 && (reinterpret_cast<uintptr_t>(o) % (4 * sizeof(T))) == 0) {
        Out<T>::store4(o, v);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j < nvalid) o[j] = Out<T>::cvt(v[j]);
    }
}

// Store 4 consecutive outputs of a row at a 4-element aligned address
// (quantised when M > 0): the store_group arithmetic without its checks.
template <typename T>
__device__ __forceinline__ void store_quad(T *o, const float *v, float M) {
    if constexpr (IsCode<T>::value) {
        uint32_t q[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) q[j] = quant_raw(v[j], M);
        if (sizeof(T) == 1) *reinterpret_cast<uint32_t *>(o) = pack_u8(q[0], q[1], q[2], q[3]);
        else *reinterpret_cast<uint2 *>(o) = pack_u16(q[0], q[1], q[2], q[3]);
    } else {
        Out<T>::store4(o, v);
    }
}

// Horizontal pass (rows of the full halo rectangle, tile columns) and
// vertical pass with store; taps w[|k|], k = -R..R, replicate border already
// materialised in A.  R is a compile-time radius (0 < R <= 6).  Tiles start
// on multiples of 4, so the tile's first input column x0 - R sits
// OFF = (-R) mod 4 columns into A's 16-byte aligned rows, and its first
// output column at CB = OFF + R, a multiple of 4.
//
// The horizontal pass works in place: a warp takes whole rows (32 / G rows
// of G output quads per pass), its lanes read their inputs, the warp
// synchronises, and the lanes write their outputs over the row at CB.  No
// other warp reads those rows in that pass except past the row's end, which
// feeds only outputs beyond the tile.
template <typename T, int R>
__device__ __forceinline__ void blur_store(const Geo &g, float *A, const float *w, T *out, float M) {
    constexpr int OFF = (4 - R % 4) % 4;
    constexpr int CB = OFF + R;
    const int TW = g.x1 - g.x0, TH = g.y1 - g.y0;
    const int G = (TW + 3) >> 2;  // output quads per row (<= 32: tiles are at most 128 wide)
    float wr[R + 1];
#pragma unroll
    for (int k = 0; k <= R; ++k) wr[k] = w[k];
    constexpr int NV = (OFF + 4 + 2 * R + 3) / 4;  // float4 loads covering the 4 + 2R inputs
    const int lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int rpp = 32 / G;                       // rows per warp pass
    const int lr = small_div(lane, 1.0f / (float)G), lg = lane - lr * G;
    for (int rb = (threadIdx.x >> 5) * rpp; rb < g.FH; rb += nwarps * rpp) {
        const int r = rb + lr;
        const bool on = lr < rpp && r < g.FH;
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (on) {
            const float4 *row = reinterpret_cast<const float4 *>(A + r * g.AP + 4 * lg);
            float v[4 * NV];
#pragma unroll
            for (int q = 0; q < NV; ++q) {
                const float4 t = row[q];
                v[4 * q] = t.x;
                v[4 * q + 1] = t.y;
                v[4 * q + 2] = t.z;
                v[4 * q + 3] = t.w;
            }
            float *op = &o.x;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float acc = wr[0] * v[OFF + j + R];
#pragma unroll
                for (int k = 1; k <= R; ++k) acc = fmaf(wr[k], v[OFF + j + R - k] + v[OFF + j + R + k], acc);
                op[j] = acc;
            }
        }
        __syncwarp();  // the warp's rows are read before they are overwritten
        if (on) *reinterpret_cast<float4 *>(A + r * g.AP + CB + 4 * lg) = o;
    }
    __syncthreads();
    const float iG = 1.0f / (float)G;
    const int p4 = g.AP >> 2;
    for (int it = threadIdx.x; it < TH * G; it += blockDim.x) {
        const int r = small_div(it, iG), c0 = (it - r * G) * 4;
        const float4 *col = reinterpret_cast<const float4 *>(A + CB + c0);
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
    const int cx = g.fx0 - g.afx0 + R;  // A column of the tile's first column
    for (int it = threadIdx.x; it < g.FH * TW; it += blockDim.x) {
        const int r = it / TW, c = it - r * TW;
        const float *row = A + r * g.AP + cx + c;
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

// R = 0: A's first column is the tile's first column (x0 is a multiple of 4).
template <typename T>
__device__ __forceinline__ void store_unblurred(const Geo &g, const float *A, T *out, float M) {
    const int TW = g.x1 - g.x0, TH = g.y1 - g.y0;
    const int G = (TW + 3) >> 2;
    const float iG = 1.0f / (float)G;
    for (int it = threadIdx.x; it < TH * G; it += blockDim.x) {
        const int r = small_div(it, iG), c0 = (it - r * G) * 4;
        const float4 t = *reinterpret_cast<const float4 *>(A + r * g.AP + c0);
        float v[4] = {t.x, t.y, t.z, t.w};
        store_group<T>(out + r * g.W + c0, v, min(4, TW - c0), M);
    }
}

// ---------------------------------------------------------------------------
// one work item
// ---------------------------------------------------------------------------
struct Smem {
    uint32_t *acc;    // accumulator words; A (floats) in the same memory after the first finishing pass
    uint32_t *carry;  // the CTA's carry words (global memory)
    float *A, *Bh, *sx2, *sy2, *scr;
    uint32_t phi;     // .shared address of the normal-tail table
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
    g.ax0 = g.ex0 & ~3;
    g.P = (g.ex1 - g.ax0 + 3) & ~3;
    g.fx0 = g.x0 - g.R;
    g.fy0 = g.y0 - g.R;
    g.FW = (g.x1 - g.x0) + 2 * g.R;
    g.FH = (g.y1 - g.y0) + 2 * g.R;
    g.afx0 = g.fx0 & ~3;  // rounds down for negative columns too (two's complement)
    g.AP = (g.x1 + g.R - g.afx0 + 3) & ~3;
    g.aoff = (g.ey0 - g.fy0) * g.AP + (g.ax0 - g.afx0);
    return g;
}

// Constants of an item's finishing steps, A = Lu S + sigma_n n: S is in units
// of `unit` (accumulator units on the fused path, full scale on the 16-bit
// path), Lu = (lmin + dl sx^2 sy^2) unit, with s.sx2[k] = dl sx^2 unit per
// column and s.sy2[r] = sy^2 per row (illum_factors).
struct EpiK {
    float lminu;       // lmin unit
    float unit;        // value of one unit of S
    float sn;          // noise sigma
    bool illum, noise;
    uint32_t tag;      // noise stream of the frame
    uint64_t pair_id;
};

__device__ __forceinline__ EpiK epi_consts(const synthpix_pair_desc &D, int frame, float unit) {
    EpiK K;
    K.illum = D.illum_min != 1.0f || D.illum_max != 1.0f;
    K.lminu = D.illum_min * unit;
    K.unit = unit;
    K.sn = D.noise_sigma;
    K.noise = D.noise_sigma != 0.0f;
    K.tag = kTagNoise + (uint32_t)frame;
    K.pair_id = D.pair_id;
    return K;
}

// separable illumination factors: dl sin^2 unit for columns [ax0, ax0 + P)
// and sin^2 for rows [ey0, ey1) of the accumulator rectangle
__device__ __forceinline__ void illum_factors(const Geo &g, const synthpix_pair_desc &D, const EpiK &K, const Smem &s) {
    if (!K.illum) return;
    const float dl = D.illum_max - D.illum_min;
    for (int k = threadIdx.x; k < g.P + g.EH; k += blockDim.x) {
        if (k < g.P) {
            const float sv = sinpif(((float)(g.ax0 + k) + 0.5f) / (float)g.W);
            s.sx2[k] = (dl * (sv * sv)) * K.unit;
        } else {
            const float sv = sinpif(((float)(g.ey0 + k - g.P) + 0.5f) / (float)g.H);
            s.sy2[k - g.P] = sv * sv;
        }
    }
}

// Lu of 4 pixels of a row from their column factors (16-byte aligned) and the row factor
__device__ __forceinline__ float4 lu_quad(const EpiK &K, const float *sx, float ly) {
    if (!K.illum) return make_float4(K.unit, K.unit, K.unit, K.unit);
    const float4 c = *reinterpret_cast<const float4 *>(sx);
    return make_float4(fmaf(c.x, ly, K.lminu), fmaf(c.y, ly, K.lminu), fmaf(c.z, ly, K.lminu),
                       fmaf(c.w, ly, K.lminu));
}

// A = Lu S + sigma_n n of one aligned quad (q: its call of the noise stream)
__device__ __forceinline__ float4 a_quad(const KernelArgs &a, const EpiK &K, const float4 &S, const float4 &Lu,
                                         uint32_t q) {
    if (!K.noise) return make_float4(Lu.x * S.x, Lu.y * S.y, Lu.z * S.z, Lu.w * S.w);
    const uint4 w = stream_words(a.keys, K.pair_id, q, K.tag);
    float n0, n1, n2, n3;
    box_muller(w.x, w.y, K.sn, n0, n1);
    box_muller(w.z, w.w, K.sn, n2, n3);
    return make_float4(fmaf(Lu.x, S.x, n0), fmaf(Lu.y, S.y, n1), fmaf(Lu.z, S.z, n2), fmaf(Lu.w, S.w, n3));
}

// S of the fused path in accumulator units: the accumulator words.  r:
// accumulator row, c: column from ax0 (a multiple of 4 for quad()).  quad()
// leaves the words (the finishing buffer is written over them and cleared
// after the blur); pixel() clears each word as it is read (the 16-bit path,
// which leaves the accumulator to the next item).  When an add wrapped a word,
// the words were first converted to S in place (float bits), carries
// included (wrapped_to_float).
struct AccSource {
    uint32_t *acc;
    int P;
    bool floats;  // the words hold S as float bits
    __device__ __forceinline__ float value(uint32_t v) const { return floats ? __uint_as_float(v) : (float)v; }
    __device__ __forceinline__ float4 quad(int r, int c) const {
        const uint4 v = *reinterpret_cast<const uint4 *>(acc + r * P + c);
        return make_float4(value(v.x), value(v.y), value(v.z), value(v.w));
    }
    __device__ __forceinline__ float pixel(int r, int c) const {
        uint32_t *p = acc + r * P + c;
        const uint32_t v = *p;
        *p = 0u;
        return value(v);
    }
};

// A wrapped item: S = word + carry 2^32 (units) written over the words as
// floats, before the finishing buffer (which holds the carry words) is
// written.  Ends with a barrier.
__device__ __forceinline__ void wrapped_to_float(const Smem &s, const Geo &g) {
    const float ip = 1.0f / (float)g.P;
    for (int k = threadIdx.x; k < g.EH * g.P; k += blockDim.x) {
        const int r = small_div(k, ip), i = g.aoff + r * g.AP + (k - r * g.P);
        s.acc[i] = __float_as_uint(fmaf((float)s.carry[i], kWrapValue, (float)s.acc[i]));
    }
    __syncthreads();
}

template <typename I>
__device__ __forceinline__ float4 load4_inter(const I *p);
template <>
__device__ __forceinline__ float4 load4_inter<__half>(const __half *p) {
    const uint2 u = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
template <>
__device__ __forceinline__ float4 load4_inter<__nv_bfloat16>(const __nv_bfloat16 *p) {
    const uint2 u = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

// S of the 16-bit path: the intermediate frame (frame row ey0 + r, column ax0 + c).
template <typename I>
struct InterSource {
    const I *S;  // the frame
    int W, ey0, ax0;
    bool vec;    // 8-byte aligned quads
    __device__ __forceinline__ float4 quad(int r, int c) const {
        const I *p = S + (ey0 + r) * W + ax0 + c;
        if (vec) return load4_inter<I>(p);
        // W not a multiple of 4: the quad may run past the row (and the frame)
        const int n = W - (ax0 + c);
        return make_float4(n > 0 ? (float)p[0] : 0.0f, n > 1 ? (float)p[1] : 0.0f, n > 2 ? (float)p[2] : 0.0f,
                           n > 3 ? (float)p[3] : 0.0f);
    }
    __device__ __forceinline__ float pixel(int r, int c) const { return (float)S[(ey0 + r) * W + ax0 + c]; }
};

// First pass of the finishing steps of one tile of one frame, over the
// accumulator rectangle: A = Lu S + sigma_n n.  The illumination factors
// must be in s.sx2 / s.sy2 and visible (a barrier after illum_factors).
// With W a multiple of 4 (or without noise) a thread takes a 16-byte
// aligned quad of a row, which is then also one Philox call of the noise
// stream (pixels 4q..4q+3 of the frame's row-major order); otherwise noise
// quads straddle rows and pixels are taken one by one.
template <typename Src>
__device__ __forceinline__ void finish_pass1(const KernelArgs &a, const Geo &g, const EpiK &K, const Smem &s,
                                             const Src &src) {
    float *A0 = s.A + g.aoff;  // A at (ey0, ax0): in place over the accumulator words it is made from
    if (!K.noise || (g.W & 3) == 0) {
        const int nq = g.P >> 2;
        const float inq = 1.0f / (float)nq;
        for (int item = threadIdx.x; item < g.EH * nq; item += blockDim.x) {
            const int r = small_div(item, inq), c = 4 * (item - r * nq);
            const float4 S = src.quad(r, c);
            const float4 Lu = lu_quad(K, s.sx2 + c, K.illum ? s.sy2[r] : 0.0f);
            // 32-bit pixel indices: frames hold at most 32768^2 = 2^30 pixels
            const uint32_t q = (uint32_t)(((g.ey0 + r) * g.W + g.ax0 + c) >> 2);
            *reinterpret_cast<float4 *>(A0 + r * g.AP + c) = a_quad(a, K, S, Lu, q);
        }
    } else {
        const int nq = (g.EW + 6) / 4 + 1;
        const float inq = 1.0f / (float)nq;
        const int cx = g.ex0 - g.ax0;  // accumulator column of ex0
        for (int item = threadIdx.x; item < g.EH * nq; item += blockDim.x) {
            const int r = small_div(item, inq), qi = item - r * nq;
            const int rowlin = (g.ey0 + r) * g.W;
            const int p0 = (((rowlin + g.ex0) >> 2) + qi) << 2;
            if (p0 > rowlin + g.ex1 - 1) continue;
            const uint4 w = stream_words(a.keys, K.pair_id, (uint32_t)(p0 >> 2), K.tag);
            float nv[4];
            box_muller(w.x, w.y, K.sn, nv[0], nv[1]);
            box_muller(w.z, w.w, K.sn, nv[2], nv[3]);
            const int c0 = p0 - rowlin - g.ex0;  // column of the quad's first pixel from ex0
            const float ly = K.illum ? s.sy2[r] : 0.0f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = c0 + k;
                if (c >= 0 && c < g.EW) {
                    const float S = src.pixel(r, cx + c);
                    const float Lu = K.illum ? fmaf(s.sx2[cx + c], ly, K.lminu) : K.unit;
                    A0[r * g.AP + cx + c] = fmaf(Lu, S, nv[k]);
                }
            }
        }
    }
}

// The rest of the finishing steps once A is complete over the accumulator
// rectangle (a barrier after finish_pass1): border replication into the halo
// outside the frame, separable blur, quantisation, one store per pixel.
// clear_after: clear A (the accumulator's memory) for the next item.
template <typename T>
__device__ __forceinline__ void finish_rest(const KernelArgs &a, const Geo &g, const synthpix_pair_desc &D,
                                            const float *wtab, int frame, const Smem &s, bool clear_after) {
    if (g.R > 0 && (g.fx0 < 0 || g.fy0 < 0 || g.x1 + g.R > g.W || g.y1 + g.R > g.H)) {  // uniform
        // only the pixels of the full halo rectangle outside the frame: whole rows
        // above and below it, then the columns left and right of it in the rows
        // between; each copies an in-frame pixel, so the order does not matter
        const int cx = g.fx0 - g.afx0;  // A column of frame column fx0
        const int top = max(-g.fy0, 0), bot = max(g.fy0 + g.FH - g.H, 0);
        const int left = max(-g.fx0, 0), right = max(g.fx0 + g.FW - g.W, 0);
        const int nband = (top + bot) * g.FW, nside = left + right;
        const int n = nband + (g.FH - top - bot) * nside;
        const float ifw = 1.0f / (float)g.FW, ins = 1.0f / (float)max(nside, 1);
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            int r, c;
            if (k < nband) {
                const int q = small_div(k, ifw);
                r = q < top ? q : g.FH - bot + (q - top);
                c = k - q * g.FW;
            } else {
                const int q = small_div(k - nband, ins), e = k - nband - q * nside;
                r = top + q;
                c = e < left ? e : g.FW - right + (e - left);
            }
            const int gi = g.fy0 + r, gj = g.fx0 + c;
            const int ci = min(max(gi, 0), g.H - 1) - g.fy0, cj = min(max(gj, 0), g.W - 1) - g.fx0;
            s.A[r * g.AP + cx + c] = s.A[ci * g.AP + cx + cj];
        }
        __syncthreads();
    }
    const int64_t HW = (int64_t)g.H * g.W;
    // the tile's first output pixel; stores add 32-bit row / column offsets
    T *out = reinterpret_cast<T *>(a.images) + D.image_offset + (int64_t)frame * HW + (int64_t)g.y0 * g.W + g.x0;
    const float M = a.quant_bits > 0 ? (float)((1u << a.quant_bits) - 1u) : 0.0f;
    switch (g.R) {
    case 0: store_unblurred<T>(g, s.A, out, M); break;
    case 1: blur_store<T, 1>(g, s.A, wtab, out, M); break;
    case 2: blur_store<T, 2>(g, s.A, wtab, out, M); break;
    case 3: blur_store<T, 3>(g, s.A, wtab, out, M); break;
    case 4: blur_store<T, 4>(g, s.A, wtab, out, M); break;
    case 5: blur_store<T, 5>(g, s.A, wtab, out, M); break;
    case 6: blur_store<T, 6>(g, s.A, wtab, out, M); break;
    default: blur_store_any<T>(g, s.A, s.Bh, s.BP, wtab, out, M); break;
    }
    if (clear_after) {  // A is the next item's accumulator: zero once every pass has read it
        __syncthreads();
        float4 *a4 = reinterpret_cast<float4 *>(s.A);
        for (int k = threadIdx.x; k < (g.FH * g.AP) >> 2; k += blockDim.x) a4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// The finishing steps of a full 128 x 128 tile (fused path, 16 warps, W a
// multiple of 4, blur radius R <= 4), with the blur in registers:
//   1. the quads just left and right of the tile (columns x0 - 4 .. x0 - 1
//      and x1 .. x1 + 3, where inside the frame) of every row of the
//      accumulator rectangle: A written in place;
//   2. a warp per row, lane l on the tile's quad l: A of the quad, then the
//      horizontal blur of its 4 pixels from its own values and those of its
//      neighbours (shuffles; the quads of step 1 from shared memory; the
//      pixel at the frame's edge repeated past it), written in place;
//   3. a warp per 8 output rows, lane l on quad l: the vertical blur over the
//      8 + 2R rows it needs (row indices clamped into the frame: replicated
//      border), in packed FP32 pairs, then quantisation and the stores.
// The arithmetic (a_quad, the tap order of both passes, quant_code) is that
// of finish_pass1 / blur_store, so a pixel's value does not depend on the
// tile edge that renders it.  R = 0: step 2 stores the quantised A directly.
template <typename T, int R>
__device__ __forceinline__ void finish_fast(const KernelArgs &a, const Geo &g, const synthpix_pair_desc &D,
                                            const float *wtab, int frame, const EpiK &K, const Smem &s,
                                            const AccSource &src) {
    static_assert(R >= 0 && R <= 4, "halo of at most one quad");
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int AP = g.AP;
    const int cx = g.x0 - g.afx0;       // accumulator column of the tile's first column
    const int sc = g.ax0 - g.afx0;      // src columns count from ax0
    float *A = s.A;                     // accumulator rows from fy0, columns from afx0
    const int rlo = g.ey0 - g.fy0, rhi = g.ey1 - g.fy0;  // accumulator rows inside the frame
    const float M = a.quant_bits > 0 ? (float)((1u << a.quant_bits) - 1u) : 0.0f;
    T *out = reinterpret_cast<T *>(a.images) + D.image_offset + (int64_t)frame * ((int64_t)g.H * g.W) +
             (int64_t)g.y0 * g.W + g.x0;
    float w[R + 1];
#pragma unroll
    for (int k = 0; k <= R; ++k) w[k] = wtab[k];
    const bool left = g.x0 > 0, right = g.x1 < g.W;  // the side quads lie inside the frame
    if constexpr (R > 0) {  // 1. side quads
        for (int k = threadIdx.x; k < 2 * (rhi - rlo); k += blockDim.x) {
            const int r = rlo + (k >> 1);
            const bool rt = (k & 1) != 0;
            if (rt ? !right : !left) continue;
            const int c = rt ? cx + 128 : cx - 4;
            const float4 S = src.quad(r - rlo, c - sc);
            const float4 Lu = lu_quad(K, s.sx2 + (c - sc), K.illum ? s.sy2[r - rlo] : 0.0f);
            const uint32_t q = (uint32_t)(((g.fy0 + r) * g.W + g.afx0 + c) >> 2);
            *reinterpret_cast<float4 *>(A + r * AP + c) = a_quad(a, K, S, Lu, q);
        }
        __syncthreads();
    }
    // 2. A and the horizontal blur, a warp per row
    const int cl = cx + 4 * lane;  // this lane's accumulator column
    for (int r = rlo + warp; r < rhi; r += 16) {
        const float4 S = src.quad(r - rlo, cl - sc);
        const float4 Lu = lu_quad(K, s.sx2 + (cl - sc), K.illum ? s.sy2[r - rlo] : 0.0f);
        const float4 v4 = a_quad(a, K, S, Lu, (uint32_t)(((g.fy0 + r) * g.W + g.afx0 + cl) >> 2));
        const float v[4] = {v4.x, v4.y, v4.z, v4.w};
        if constexpr (R == 0) {
            store_quad<T>(out + (r - rlo) * g.W + 4 * lane, v, M);
        } else {
            // x[m], m = -R .. 3 + R: the row's A around this lane's 4 pixels
            float x[4 + 2 * R];
    #pragma unroll
            for (int j = 0; j < 4; ++j) x[R + j] = v[j];
    #pragma unroll
            for (int k = 1; k <= R; ++k) {
                x[R - k] = __shfl_up_sync(FULL, v[4 - k], 1);       // column 4l - k, lane l - 1
                x[R + 3 + k] = __shfl_down_sync(FULL, v[k - 1], 1);  // column 4l + 3 + k, lane l + 1
            }
            if (lane == 0) {
    #pragma unroll
                for (int k = 1; k <= R; ++k) x[R - k] = left ? A[r * AP + cx - k] : v[0];
            }
            if (lane == 31) {
    #pragma unroll
                for (int k = 1; k <= R; ++k) x[R + 3 + k] = right ? A[r * AP + cx + 127 + k] : v[3];
            }
            float h[4];
    #pragma unroll
            for (int j = 0; j < 4; ++j) {
                float acc = w[0] * x[R + j];
    #pragma unroll
                for (int k = 1; k <= R; ++k) acc = fmaf(w[k], x[R + j - k] + x[R + j + k], acc);
                h[j] = acc;
            }
            *reinterpret_cast<float4 *>(A + r * AP + cl) = make_float4(h[0], h[1], h[2], h[3]);
        }
    }
    if constexpr (R > 0) {
        __syncthreads();
        // 3. the vertical blur of output rows [8 warp, 8 warp + 8), quantisation, stores
        unsigned long long wp[R + 1];
#pragma unroll
        for (int k = 0; k <= R; ++k) wp[k] = f2_pack(w[k], w[k]);
        const int t0 = 8 * warp;  // first output row (tile row); its accumulator row is t0 + R
        unsigned long long hv[8 + 2 * R][2];
#pragma unroll
        for (int i = 0; i < 8 + 2 * R; ++i) {
            const int ra = min(max(t0 + i, rlo), rhi - 1);  // tile row t0 + i - R
            const float4 t = *reinterpret_cast<const float4 *>(A + ra * AP + cl);
            hv[i][0] = f2_pack(t.x, t.y);
            hv[i][1] = f2_pack(t.z, t.w);
        }
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            unsigned long long p0 = f2_mul(wp[0], hv[o + R][0]), p1 = f2_mul(wp[0], hv[o + R][1]);
#pragma unroll
            for (int k = 1; k <= R; ++k) {
                p0 = f2_fma(wp[k], f2_add(hv[o + R - k][0], hv[o + R + k][0]), p0);
                p1 = f2_fma(wp[k], f2_add(hv[o + R - k][1], hv[o + R + k][1]), p1);
            }
            const float2 a0 = f2_unpack(p0), a1 = f2_unpack(p1);
            const float ov[4] = {a0.x, a0.y, a1.x, a1.y};
            store_quad<T>(out + (t0 + o) * g.W + 4 * lane, ov, M);
        }
    }
    __syncthreads();
    // the accumulator's rows inside the frame start the next item at zero
    float4 *a4 = reinterpret_cast<float4 *>(A + rlo * AP);
    for (int k = threadIdx.x; k < ((rhi - rlo) * AP) >> 2; k += blockDim.x) a4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// The fast finishing path applies: a full 128 x 128 tile, W a multiple of 4
// (aligned noise quads), blur radius at most 4, outputs of the pair starting
// on a 4-element boundary of a 16-byte aligned buffer (aligned quad stores).
__device__ __forceinline__ bool fast_finish_ok(const Geo &g, const synthpix_pair_desc &D, const void *images) {
    return g.x1 - g.x0 == 128 && g.y1 - g.y0 == 128 && (g.W & 3) == 0 && g.R <= 4 && (D.image_offset & 3) == 0 &&
           (reinterpret_cast<uintptr_t>(images) & 15) == 0;
}

template <typename T>
__device__ __forceinline__ void finish_fast_r(const KernelArgs &a, const Geo &g, const synthpix_pair_desc &D,
                                              const float *wtab, int frame, const EpiK &K, const Smem &s,
                                              const AccSource &src) {
    switch (g.R) {
    case 0: finish_fast<T, 0>(a, g, D, wtab, frame, K, s, src); break;
    case 1: finish_fast<T, 1>(a, g, D, wtab, frame, K, s, src); break;
    case 2: finish_fast<T, 2>(a, g, D, wtab, frame, K, s, src); break;
    case 3: finish_fast<T, 3>(a, g, D, wtab, frame, K, s, src); break;
    default: finish_fast<T, 4>(a, g, D, wtab, frame, K, s, src); break;
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
// The next work item is ticket tk (taken during the previous item): thread
// 0 copies its fields in while the first chunk renders (fetch_item) and
// publishes it in *next at the last chunk's barrier.  hdr: the item's staged
// header; hdr_next: the next item's header slot; rec: the record region,
// which receives the next item's header and first chunk as soon as the
// item's own records are splatted (the copies run behind the finishing).
template <typename T, int NT, int RS>
__device__ __forceinline__ void process_item(const KernelArgs &a, const ItemInfo &it, uint32_t &tk,
                                             const unsigned char *hdr, unsigned char *hdr_next, unsigned char *rec,
                                             uint32_t cap, const Smem &s, ItemInfo *next) {
    const synthpix_pair_desc &D = *reinterpret_cast<const synthpix_pair_desc *>(hdr);
    const PairPlan &pl = *reinterpret_cast<const PairPlan *>(hdr + kStageDesc);
    const float *wtab = reinterpret_cast<const float *>(hdr + kStagePlan);
    const Geo g = make_geo(D, pl, pl.tile, it.tile, pl.halo);
    const bool fused = a.inter_dtype == SYNTHPIX_F32;
    const float imax = D.i_max > 0.0f ? D.i_max : 1.0f;
    const float unit = imax * kFixedUnit;
    const EpiK K = epi_consts(D, it.frame, unit);
    if (fused) illum_factors(g, D, K, s);

    // splat, chunk by chunk of staged records
    const float scale = kFixedScale / imax;
    const Acc acc{sh_addr(s.acc), s.carry, g.AP};
    if (it.count == 0 && threadIdx.x == 0) fetch_item(a, tk);  // no chunk to start the copy in
    uint32_t done = 0;
    while (done < it.count) {
        const uint32_t n = min(it.count - done, cap);
        const uint32_t ft = done == 0 ? tk : ~0u;
        if constexpr (RS == (int)sizeof(RecordG))
            splat_chunk_general(rec + record_lead<RS>(it.rec0 + done), n, g, scale, acc, s.phi, a, ft);
        else
            splat_chunk<NT>(rec + record_lead<RS>(it.rec0 + done), rec, n, g, scale, acc,
                            s.scr + (threadIdx.x >> 5) * a.warp_scratch, a.warp_scratch >> 2, s.phi, a, ft);
        done += n;
        if (done >= it.count && threadIdx.x == 0) {
            cp_async_wait_all();  // the next item's fields (copied while this item rendered)
            *next = fetched_item(a);
        }
        __syncthreads();
        if (done < it.count) {  // more records: stage the next chunk
            stage_records<RS>(a, it.rec0 + done, min(it.count - done, cap), rec);
            cp_async_commit();
            cp_async_wait_all();
            __syncthreads();
        }
    }
    if (it.count == 0) {  // no records: the barrier also shows the illumination factors
        if (threadIdx.x == 0) {
            cp_async_wait_all();
            *next = fetched_item(a);
        }
        __syncthreads();
    }
    // every warp is past the last chunk: the next item's header and first chunk are staged
    const ItemInfo nx = *next;
    if (nx.pair >= 0) {
        stage_header(a, nx.pair, hdr_next);
        stage_records<RS>(a, nx.rec0, min(nx.count, cap), rec);
    }
    cp_async_commit();
    // the ticket of the item after the next (thread 0 alone uses tk): taken
    // here, ahead of the finishing, so that the atomic's round trip overlaps
    // the finishing instead of holding the item-end barrier
    if (threadIdx.x == 0) tk = 2u * gridDim.x + atomicAdd(a.ticket, 1u);
    // block counts of the next item start from zero (its first count comes after a barrier)
    for (int k = threadIdx.x; k < kBlkPitch * kBlkSide; k += blockDim.x) sh_blk[k] = 0u;

    const bool wrapped = sh_wrap != 0;
    if (wrapped) wrapped_to_float(s, g);
    const AccSource src{s.acc + g.aoff, g.AP, wrapped};
    if (!fused) {
        // halo 0: the accumulator rectangle is the tile (ax0 = ex0 = x0)
        const int64_t HW = (int64_t)g.H * g.W;
        const int64_t base = pl.inter_base + (int64_t)it.frame * HW;
        const float iew = 1.0f / (float)g.EW;
        for (int idx = threadIdx.x; idx < g.EH * g.EW; idx += blockDim.x) {
            const int r = small_div(idx, iew), c = idx - r * g.EW;
            const float S = src.pixel(r, c) * unit;  // full scale
            const int64_t o = base + (int64_t)(g.ey0 + r) * g.W + (g.ex0 + c);
            if (a.inter_dtype == SYNTHPIX_F16) reinterpret_cast<__half *>(a.inter)[o] = to_inter<__half>(S);
            else reinterpret_cast<__nv_bfloat16 *>(a.inter)[o] = to_inter<__nv_bfloat16>(S);
        }
        return;  // the caller's loop ends with a barrier
    }
    if (NT == 512 && a.reg_epilogue && fast_finish_ok(g, D, a.images)) {
        finish_fast_r<T>(a, g, D, wtab, it.frame, K, s, src);
        return;
    }
    finish_pass1(a, g, K, s, src);
    __syncthreads();
    finish_rest<T>(a, g, D, wtab, it.frame, s, true);
}

// ---------------------------------------------------------------------------
// the persistent kernel
// ---------------------------------------------------------------------------
struct SmemLayout {
    size_t acc, Bh, sx2, sy2, scr, phi, bufs, total;
};

// The accumulator words, which hold the finishing buffer A after the first
// finishing pass (+ padding read by the last row's blur loads); illumination
// factors; per-warp window scratch; the normal-tail table; two staged
// headers and the staged-record region; the horizontal-blur buffer Bh of the
// blur for radii above 6 (the others blur rows in place).
__host__ __device__ inline SmemLayout smem_layout(int E, int tile, int warp_scratch, int rec_buf_bytes) {
    SmemLayout L;
    const int BP = (tile + 3) & ~3;
    const size_t PC = (size_t)pitch_cap(E);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = (o + bytes + 15) & ~(size_t)15;
        return at;
    };
    L.acc = take(((size_t)E * PC + 32) * 4);
    L.sx2 = take(PC * 4);
    L.sy2 = take((size_t)E * 4);
    L.scr = take((size_t)(splat_threads(tile) / 32) * warp_scratch * 4);
    L.phi = take((size_t)(kPhiDegree + 1) * kPhiPieces * 4);
    L.bufs = take(2 * (size_t)kStageHeader + (size_t)rec_buf_bytes);  // two headers, one record region
    const bool need_bh = (E - tile) / 2 > 6;  // only the blur of radii above 6 uses Bh
    L.Bh = need_bh ? take((size_t)E * BP * 4) : L.acc;
    L.total = o;
    return L;
}

// RS: bytes of a bin record (24: Record, round particles; 32: RecordG, general shapes).
template <typename T, int NT, int RS>
__global__ void __launch_bounds__(NT, 1024 / NT) k_splat(KernelArgs a) {
    if (*a.check != 1) return;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ItemInfo s_item[2];
    const SmemLayout L = smem_layout(a.smem_edge, a.tile, a.warp_scratch, a.rec_buf_bytes);
    const int words = a.smem_edge * pitch_cap(a.smem_edge);
    Smem s;
    s.acc = reinterpret_cast<uint32_t *>(smem + L.acc);
    s.carry = a.carry + (int64_t)blockIdx.x * a.carry_stride;
    s.A = reinterpret_cast<float *>(smem + L.acc);
    s.Bh = reinterpret_cast<float *>(smem + L.Bh);
    s.sx2 = reinterpret_cast<float *>(smem + L.sx2);
    s.sy2 = reinterpret_cast<float *>(smem + L.sy2);
    s.scr = reinterpret_cast<float *>(smem + L.scr);
    float *phi = reinterpret_cast<float *>(smem + L.phi);
    for (int k = threadIdx.x; k < (kPhiDegree + 1) * kPhiPieces; k += blockDim.x) phi[k] = kPhiTable[k];
    s.phi = sh_addr(phi);
    for (int k = threadIdx.x; k < kBuckets; k += blockDim.x) sh_cnt[k] = 0;
    for (int k = threadIdx.x; k < kBlkPitch * kBlkSide; k += blockDim.x) sh_blk[k] = 0;
    s.BP = (a.tile + 3) & ~3;
    unsigned char *bufs = smem + L.bufs;  // headers [0, 2 kStageHeader), then the record region
    unsigned char *rec = bufs + 2 * kStageHeader;
    const uint32_t cap = (uint32_t)(RS == (int)sizeof(RecordG) ? rec_cap(a.rec_buf_bytes, RS)
                                                               : min(rec_cap(a.rec_buf_bytes, RS), kSplatRpt * NT));
    for (int k = threadIdx.x; k < (words >> 2); k += blockDim.x)
        reinterpret_cast<uint4 *>(s.acc)[k] = make_uint4(0u, 0u, 0u, 0u);
    // work queue: the current item and the ticket tk of the next one, whose
    // fields are copied in while the current item renders (process_item).  A
    // CTA holds one ticket beyond the item it renders (two while it finishes
    // one), so when the queue runs dry the CTAs stop within about one item of
    // each other.  Tickets
    // only grow, so a CTA never drops a valid one.  The first two tickets of
    // CTA b are b and grid + b; the counter hands out the rest from 2 grid,
    // each taken once an item's records are splatted, ahead of its finishing.
    uint32_t tk = gridDim.x + blockIdx.x;
    if (threadIdx.x == 0) {
        sh_wrap = 0;
        ItemInfo it;
        if ((int64_t)blockIdx.x < a.n_tiles) it = work_item(a, blockIdx.x);
        else it.pair = -1;
        s_item[0] = it;
    }
    __syncthreads();
    if (s_item[0].pair < 0) return;
    stage_header(a, s_item[0].pair, bufs);
    stage_records<RS>(a, s_item[0].rec0, min(s_item[0].count, cap), rec);
    cp_async_commit();
    int cur = 0;
    for (;;) {
        const ItemInfo it = s_item[cur];
        cp_async_wait_all();
        __syncthreads();  // staged header and records of `it` visible; the other header slot is free; the wrap flag is read
        if (it.pair < 0) break;
        // the splat's first add comes after a barrier inside splat_chunk
        if (threadIdx.x == 0) {
            sh_wrap = 0;
            sh_carry_clean = 0;
        }
        process_item<T, NT, RS>(a, it, tk, bufs + cur * kStageHeader, bufs + (cur ^ 1) * kStageHeader, rec, cap, s,
                                &s_item[cur ^ 1]);  // takes the ticket of the item after the next
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
    const size_t PC = (size_t)pitch_cap(E);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = (o + bytes + 15) & ~(size_t)15;
        return at;
    };
    L.A = take(((size_t)E * PC + 32) * 4);
    L.Bh = take((E - tile) / 2 > 6 ? (size_t)E * BP * 4 : 0);  // only radii above 6 use Bh
    L.sx2 = take(PC * 4);
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
    s.acc = nullptr;
    s.carry = nullptr;
    s.A = reinterpret_cast<float *>(smem + FL.A);
    s.Bh = reinterpret_cast<float *>(smem + FL.Bh);
    s.sx2 = reinterpret_cast<float *>(smem + FL.sx2);
    s.sy2 = reinterpret_cast<float *>(smem + FL.sy2);
    s.scr = nullptr;
    s.phi = 0u;
    s.BP = (a.tile + 3) & ~3;
    const ItemInfo it = a.items[blockIdx.x];
    const synthpix_pair_desc &D = a.descs[it.pair];
    const PairPlan pl = a.plan[it.pair];
    if (threadIdx.x < kBlurStride) wtab[threadIdx.x] = a.blur_w[(int64_t)it.pair * kBlurStride + threadIdx.x];
    const Geo g = make_geo(D, pl, pl.tile, it.tile, pl.blur_r);
    const EpiK K = epi_consts(D, it.frame, 1.0f);  // the intermediate frames hold S at full scale
    illum_factors(g, D, K, s);
    __syncthreads();
    const I *S16 = reinterpret_cast<const I *>(a.inter) + pl.inter_base + (int64_t)it.frame * g.H * g.W;
    const bool vec = (g.W & 3) == 0 && (reinterpret_cast<uintptr_t>(S16) & 7) == 0;
    const InterSource<I> src{S16, g.W, g.ey0, g.ax0, vec};
    finish_pass1(a, g, K, s, src);
    __syncthreads();
    finish_rest<T>(a, g, D, wtab, it.frame, s, false);
}

// Launch of the persistent splat (and, on the 16-bit intermediate path, of
// k_finish) for output type T.
template <typename T>
cudaError_t launch_splat_t(const KernelArgs &a, cudaStream_t st) {
    const size_t smem = smem_layout(a.smem_edge, a.tile, a.warp_scratch, a.rec_buf_bytes).total;
    int dev = 0, nsm = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    auto go = [&](auto kern, int nt) -> cudaError_t {
        cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (r != cudaSuccess) return r;
        r = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, nt, smem);
        if (r != cudaSuccess) return r;
        int64_t want = (int64_t)nsm * (occ > 0 ? occ : 1);
        if (want > splat_max_ctas(a.tile, a.n_tiles)) want = splat_max_ctas(a.tile, a.n_tiles);  // carries
        return launch_kernel(kern, (unsigned)(a.n_tiles < want ? a.n_tiles : want), nt, smem, st, a);
    };
    const int nt = splat_threads(a.tile);
    if (a.general) e = nt == 512 ? go(k_splat<T, 512, 32>, 512) : go(k_splat<T, 256, 32>, 256);
    else e = nt == 512 ? go(k_splat<T, 512, 24>, 512) : go(k_splat<T, 256, 24>, 256);
    if (e != cudaSuccess) return e;
    if (a.inter_dtype != SYNTHPIX_F32) {
        const size_t fsm = finish_layout(a.smem_edge, a.tile).total;
        auto fin = [&](auto kern) -> cudaError_t {
            cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
            if (r != cudaSuccess) return r;
            return launch_kernel(kern, (unsigned)a.n_tiles, kSplatThreads, fsm, st, a);
        };
        e = a.inter_dtype == SYNTHPIX_F16 ? fin(k_finish<T, __half>) : fin(k_finish<T, __nv_bfloat16>);
    }
    return e;
}

}  // namespace spx
