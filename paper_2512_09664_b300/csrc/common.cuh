// Shared declarations of the sm_103a PIV renderer: per-pair plan, workspace
// layout, Philox4x32-10 and the split (integer + fraction) particle position.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "synthpix.h"

namespace spx {

constexpr int kMaxBlurRadius = 24;  // ceil(3 * 8)
constexpr int kChunk = 512;         // particles of one pair per CTA of the seeding and binning kernels
constexpr int kBlurStride = 32;     // floats per pair in the blur-tap table

// Derived per-pair geometry (device table built by k_plan, mirrored on the host).
struct PairPlan {
    int64_t part_base;   // first global particle index of the pair
    int64_t list_base;   // first bin-list slot of the frame-1 segment
    int64_t list_cap;    // slots of one frame segment (frame 2 at list_base + list_cap)
    int64_t inter_base;  // first element of the pair's 16-bit intermediate frames
    int32_t tile_base;   // first global tile id of frame 1 (frame 2 at + ntiles)
    int32_t tiles_x, tiles_y, ntiles;
    int32_t blur_r;      // ceil(3 * blur_sigma), 0 without blur
    int32_t halo;        // pixels a tile's bins extend beyond the tile (blur_r or 0)
    int32_t chunk_base;  // first particle chunk (kChunk particles) of the pair
    int32_t tile;        // screen tile edge of the pair (16, 32, 64 or 128)
};
static_assert(sizeof(PairPlan) == 64, "PairPlan layout");

// Screen tile edges by frame size class: a batch may render its small and
// large frames with different tile edges in one launch sequence.  The class
// of a pair is that of its frame area: < 2^15 pixels (up to about 181^2),
// < 2^17 (362^2), < 2^19 (724^2), larger.  Host and device resolve a pair's
// edge from the same rule (passed by value to the plan kernel).
constexpr int kSizeClasses = 4;
struct TileRule {
    int32_t edge[kSizeClasses];
};
__host__ __device__ inline int size_class(int32_t height, int32_t width) {
    const int64_t a = (int64_t)height * width;
    return a < (1 << 15) ? 0 : (a < (1 << 17) ? 1 : (a < (1 << 19) ? 2 : 3));
}
__host__ __device__ inline int32_t rule_tile(const TileRule &r, const synthpix_pair_desc &d) {
    return r.edge[size_class(d.height, d.width)];
}

// Screen tile edge and per-pair quantities shared by host and device.
struct PairGeom {
    int32_t tiles_x, tiles_y, ntiles, blur_r, halo, span;
    int64_t list_cap;
    int64_t chunks;  // ceil(n_particles / kChunk), at least 1 (the first chunk of a pair writes its work items)
};

__host__ __device__ inline int32_t blur_radius_of(float blur_sigma) {
    if (!(blur_sigma > 0.0f)) return 0;
    return (int32_t)ceil(3.0 * (double)blur_sigma);  // exact product of an FP32 value
}

// Upper bound of the pixels along one axis of a particle window [floor(x-1.5d), floor(x+1.5d)].
__host__ __device__ inline int32_t window_max(float d_max) { return (int32_t)floor(3.0 * (double)d_max) + 5; }

// Largest particle diameter of a pair along either axis.
__host__ __device__ inline float pair_max_diameter(const synthpix_pair_desc &d) {
    return d.dy_max > d.d_max ? d.dy_max : d.d_max;
}

// The pair draws general shapes (d_y or rho intervals set).
__host__ __device__ inline bool pair_general_shape(const synthpix_pair_desc &d) {
    return d.dy_min != 0.0f || d.dy_max != 0.0f || d.rho_min != 0.0f || d.rho_max != 0.0f;
}

constexpr int64_t kExactBinRecords = 1 << 16;  // see fixed_caps

// Records per bin of the fixed bin layout of seeded renders (each producer
// places its records directly, without a counting pass).  A bin of an
// interior tile collects the particles whose centres lie within the tile
// widened by the halo and a window on each side: E = N side_x side_y / (W H)
// expected for uniform positions.  Frame 1 gets E + E/4 + 64 (more than 9
// standard deviations of the binomial count for E >= 100), frame 2, whose
// density the flow changes, E + E/2 + 64; both at most N (a bin receives a
// particle at most once, so a frame of one tile never overflows), and N for
// pairs whose N x tiles is at most kExactBinRecords (no overflow, and a
// render of such pairs alone needs no rebinning launch).  A bin that
// overflows sets a flag and the frame is binned again exactly (k_rebin).
// Integer arithmetic, so host and device agree.
__host__ __device__ inline void fixed_caps(const synthpix_pair_desc &d, int32_t tile, int32_t halo, int64_t &cap1,
                                           int64_t &cap2) {
    const int64_t W = d.width, H = d.height;
    const int64_t reach = (int64_t)tile + 2LL * halo + window_max(pair_max_diameter(d));
    const int64_t sx = reach < W ? reach : W, sy = reach < H ? reach : H;
    const int64_t e = ((int64_t)d.n_particles * sx * sy + W * H - 1) / (W * H);
#ifdef SPX_SMALL_FIXED_BINS  // the overflow test library: nearly every bin overflows (k_rebin rebins)
    cap1 = e / 2 + 1;
    cap2 = e / 2 + 1;
#else
    // a bin receives each particle at most once: N records always fit; small pairs (at most
    // kExactBinRecords records over all their bins of a frame) take N, so they never overflow
    const int64_t n = (int64_t)d.n_particles;
    const int64_t ntiles = ((W + tile - 1) / tile) * ((H + tile - 1) / tile);
    cap1 = e + e / 4 + 64;
    cap2 = e + e / 2 + 64;
    if (cap1 > n || n * ntiles <= kExactBinRecords) cap1 = n;
    if (cap2 > n || n * ntiles <= kExactBinRecords) cap2 = n;
#endif
}
// The pair's fixed bins cannot overflow (both capacities are N).
__host__ __device__ inline bool fixed_exact(const synthpix_pair_desc &d, int32_t tile, int32_t halo) {
    int64_t cap1, cap2;
    fixed_caps(d, tile, halo, cap1, cap2);
    return cap1 == (int64_t)d.n_particles && cap2 == (int64_t)d.n_particles;
}

__host__ __device__ inline PairGeom pair_geom(const synthpix_pair_desc &d, int tile, bool fused) {
    PairGeom g;
    g.tiles_x = (d.width + tile - 1) / tile;
    g.tiles_y = (d.height + tile - 1) / tile;
    g.ntiles = g.tiles_x * g.tiles_y;
    g.blur_r = blur_radius_of(d.blur_sigma);
    g.halo = fused ? g.blur_r : 0;
    // pixels of a clipped particle window: <= floor(3 d_max) + 2, plus margin
    // for FP32 rounding of d and x +- 1.5 d; widened by the halo on both sides
    int32_t ext = window_max(pair_max_diameter(d)) + 2 * g.halo;
    g.span = (ext - 1) / tile + 2;
    int32_t sx = g.span < g.tiles_x ? g.span : g.tiles_x;
    int32_t sy = g.span < g.tiles_y ? g.span : g.tiles_y;
    g.list_cap = (int64_t)d.n_particles * (int64_t)sx * (int64_t)sy;
    // room for the fixed bins too (sparse pairs of many tiles need more than the bound above)
    int64_t cap1, cap2;
    fixed_caps(d, tile, g.halo, cap1, cap2);
    const int64_t fixed = (int64_t)g.ntiles * (cap1 > cap2 ? cap1 : cap2);
    if (fixed > g.list_cap) g.list_cap = fixed;
    g.chunks = max((int64_t)1, ((int64_t)d.n_particles + kChunk - 1) / kChunk);  // an empty pair: one empty chunk
    return g;
}

// A particle as binned for one frame: split position, sigma, amplitude.
struct Record {
    float fx, fy;      // fractions of the split position
    int32_t ix, iy;    // integer parts
    float sigma, amp;  // d / 4 and Ieff * 2 pi sigma^2
};
static_assert(sizeof(Record) == 24, "Record layout");

// A particle of general shape as binned for one frame (Eq. 1 with
// sigma_x != sigma_y or rho != 0).
struct RecordG {
    float fx, fy;      // fractions of the split position
    int32_t ix, iy;    // integer parts
    float sx, sy;      // d / 4 and d_y / 4
    float rho;         // correlation
    float amp;         // Ieff * 2 pi sigma_x sigma_y sqrt(1 - rho^2)
};
static_assert(sizeof(RecordG) == 32, "RecordG layout");

// One work item of the splat: the bin of one (pair, frame, tile).
struct ItemInfo {
    int32_t pair, frame, tile;
    uint32_t count;  // records in the bin
    int64_t rec0;    // first record of the bin
};
static_assert(sizeof(ItemInfo) == 24, "ItemInfo layout");

// Workspace layout (byte offsets, 256-aligned), computed on the host.
struct Layout {
    size_t plan, desc, check, blur, count, off, cursor, items, pos, sa, shape, rec, adv, inter, gfr, carry, total;
    int64_t n_part, n_tiles, n_list, n_inter, n_chunks;
    int64_t carry_stride;  // carry words per k_splat CTA
};

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }


// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies of counter words 0 and 2, mixing the high halves with
// the other counter words and the key, the key advanced by the Weyl
// increments between rounds.
// ---------------------------------------------------------------------------
// Stream layout: counter = (index, tag, pair_id lo, pair_id hi), key = seed.
constexpr uint32_t kTagAttrA = 0u;      // (x, y, d, I)
constexpr uint32_t kTagAttrB = 1u;      // (z, d2, -, -)
constexpr uint32_t kTagShapeA = 2u;     // (hide 1, hide 2, normals of the frame-2 d and I0 changes)
constexpr uint32_t kTagShapeB = 3u;     // (d_y, rho, normals of the frame-2 d_y and rho changes)
constexpr uint32_t kTagNoise = 0x100u;  // + frame; index = pixel / 4

// The ten round keys (key + r * Weyl increments) are computed once per
// launch: kernels read them from the launch parameters instead of advancing
// the key in every call.
struct PhiloxKeys {
    uint32_t x[10], y[10];
};

__host__ __device__ inline PhiloxKeys philox_round_keys(uint64_t seed) {
    PhiloxKeys K;
    uint32_t kx = (uint32_t)seed, ky = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        K.x[r] = kx;
        K.y[r] = ky;
        kx += 0x9E3779B9u;
        ky += 0xBB67AE85u;
    }
    return K;
}

__device__ __forceinline__ uint4 stream_words(const PhiloxKeys &K, uint64_t pair_id, uint32_t idx, uint32_t tag) {
    uint4 c = make_uint4(idx, tag, (uint32_t)pair_id, (uint32_t)(pair_id >> 32));
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // one 32 x 32 -> 64-bit multiply per word gives both halves
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c = make_uint4(hi1 ^ c.y ^ K.x[r], lo1, hi0 ^ c.w ^ K.y[r], lo0);
    }
    return c;
}

__device__ __forceinline__ float u24f(uint32_t w) { return (float)(w >> 8) * (1.0f / 16777216.0f); }
__device__ __forceinline__ float uo24f(uint32_t w) { return (float)((w >> 8) + 1u) * (1.0f / 16777216.0f); }

// ---------------------------------------------------------------------------
// Split particle coordinate: value = i + f with integer i and FP32 f (|f| <= ~1
// after renormalisation), keeping ~2^-24 px absolute resolution anywhere in
// a 32768 px frame (a plain FP32 coordinate has 2^-9 px at 16384).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void split_add(int32_t &i, float &f, float d) {
    // TwoSum with non-contractible intrinsics (an FMA fused into f + d would
    // break the exact error term)
    const float s = __fadd_rn(f, d);
    const float bb = __fsub_rn(s, f);
    const float e = __fadd_rn(__fsub_rn(f, __fsub_rn(s, bb)), __fsub_rn(d, bb));
    const float n = floorf(s);
    float r = __fadd_rn(__fsub_rn(s, n), e);  // s - n is exact
    int32_t ni = (int32_t)fminf(fmaxf(n, -1.0e9f), 1.0e9f);
    if (r >= 1.0f) { r = __fsub_rn(r, 1.0f); ni += 1; }
    else if (r < 0.0f) { r = __fadd_rn(r, 1.0f); ni -= 1; }
    // |i|, |ni| <= 1e9: the sum fits in int32
    i = min(max(i + ni, -1000000000), 1000000000);
    f = r;
}

}  // namespace spx
