// Intensity-histogram matching of rendered, quantised frames (the paper's
// optional adjustment of generated images to a user-specified intensity
// histogram, end of Section 2 "Mathematical model").  Histogram
// specification on the codes: with a frame's code counts (N pixels) and the
// target counts (T in all), code c becomes the smallest t with
// C_t(t) / T >= C_s(c) / N, compared exactly in 128-bit integers as
// C_t(t) N >= C_s(c) T.  Every frame of a batch (two per pair) is matched
// to the same target.
//
//   k_hist_target  the target's cumulative counts (one CTA, tiled block scan)
//   k_hist_prep    zero the frames' counts
//   k_hist_count   per (frame, chunk of pixels): counts in shared memory
//                  (codes up to 13 bits) or global atomics, added to the
//                  frame's counts
//   k_hist_map     per frame: cumulative counts in place, then the code
//                  mapping (a binary search of the target's cumulative
//                  counts per code)
//   k_hist_apply   per (frame, chunk): code -> mapped code, in place
#include <cstdio>
#include <vector>

#include "synthpix.h"

namespace spx {
void count_launch();  // api.cu: the library's launch counter
}

namespace spx {
int set_error(int code, const char *msg);
}

namespace {

constexpr int kHistThreads = 256;
constexpr int64_t kChunkPx = 65536;       // pixels per CTA of the count and apply kernels
constexpr int kSharedCodesMax = 8192;     // codes counted in shared memory (32 KB)

struct Frame {
    int64_t offset;  // first element of the frame in the images
    int64_t npx;     // its pixels
    int64_t chunk0;  // first chunk of the frame over all frames
};

struct HistArgs {
    const Frame *frames;
    int32_t n_frames;
    int32_t n_codes;
    const uint64_t *target;  // [n_codes]
    uint64_t *ct;            // [n_codes] cumulative target counts
    uint32_t *hist;          // [n_frames][n_codes] counts, then cumulative counts
    uint16_t *lut;           // [n_frames][n_codes] mapped codes
};

struct HistLayout {
    size_t frames, ct, hist, lut, total;
};

HistLayout hist_layout(int n_frames, int n_codes) {
    HistLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = (o + bytes + 255) & ~(size_t)255;
        return at;
    };
    L.frames = take((size_t)n_frames * sizeof(Frame));
    L.ct = take((size_t)n_codes * sizeof(uint64_t));
    L.hist = take((size_t)n_frames * n_codes * sizeof(uint32_t));
    L.lut = take((size_t)n_frames * n_codes * sizeof(uint16_t));
    L.total = o;
    return L;
}

// The frame of chunk q: largest f with frames[f].chunk0 <= q.
__device__ __forceinline__ int frame_of_chunk(const HistArgs &h, int64_t q) {
    int lo = 0, hi = h.n_frames - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (h.frames[mid].chunk0 <= q) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(1024) k_hist_target(HistArgs h) {
    __shared__ uint64_t s[1024];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < h.n_codes; c0 += 1024) {
        const int c = c0 + threadIdx.x;
        s[threadIdx.x] = c < h.n_codes ? h.target[c] : 0ull;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            const uint64_t add = threadIdx.x >= off ? s[threadIdx.x - off] : 0ull;
            __syncthreads();
            s[threadIdx.x] += add;
            __syncthreads();
        }
        if (c < h.n_codes) h.ct[c] = carry + s[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
}

__global__ void k_hist_prep(HistArgs h) {
    const int64_t n = (int64_t)h.n_frames * h.n_codes;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        h.hist[k] = 0u;
}

// A chunk's element range [e0, e1) of the images split into a scalar head
// [e0, a0), 16-byte vectors [a0, a1) and a scalar tail [a1, e1) (all scalar
// when the images are not 16-byte aligned).
template <typename T>
__device__ __forceinline__ void vector_span(const void *img, int64_t e0, int64_t e1, int64_t &a0, int64_t &a1) {
    constexpr int64_t V = 16 / sizeof(T);
    if ((reinterpret_cast<uintptr_t>(img) & 15) != 0) {
        a0 = a1 = e1;
        return;
    }
    a0 = min(e1, (e0 + V - 1) / V * V);
    a1 = max(a0, e1 / V * V);
}

template <typename T>
__device__ __forceinline__ uint32_t lane_code(const uint4 &x, int j) {
    const uint32_t w = j < 16 / (int)sizeof(T) / 4 ? x.x : j < 2 * (16 / (int)sizeof(T) / 4) ? x.y
                     : j < 3 * (16 / (int)sizeof(T) / 4) ? x.z : x.w;
    constexpr int per = 4 / (int)sizeof(T);
    return (w >> (8 * sizeof(T) * (j % per))) & (sizeof(T) == 1 ? 0xFFu : 0xFFFFu);
}

template <typename T>
__global__ void __launch_bounds__(kHistThreads) k_hist_count(HistArgs h, const T *__restrict__ img) {
    __shared__ uint32_t s_h[kSharedCodesMax];
    constexpr int V = 16 / sizeof(T);
    const int64_t q = blockIdx.x;
    const int f = frame_of_chunk(h, q);
    const Frame fr = h.frames[f];
    const int64_t p0 = (q - fr.chunk0) * kChunkPx, p1 = min(p0 + kChunkPx, fr.npx);
    const int64_t e0 = fr.offset + p0, e1 = fr.offset + p1;
    uint32_t *gh = h.hist + (size_t)f * h.n_codes;
    const bool local = h.n_codes <= kSharedCodesMax;
    // one copy of the counts per warp when they fit (frames are mostly background, so a
    // few codes take most pixels: private copies spread those atomics)
    constexpr int kWarps = kHistThreads / 32;
    const int copies = h.n_codes * kWarps <= kSharedCodesMax ? kWarps : 1;
    uint32_t *mine = s_h + (copies > 1 ? (threadIdx.x >> 5) * h.n_codes : 0);
    const uint32_t cmax = (uint32_t)(h.n_codes - 1);
    if (local) {
        for (int c = threadIdx.x; c < h.n_codes * copies; c += kHistThreads) s_h[c] = 0u;
        __syncthreads();
    }
    auto count = [&](uint32_t c) {
        c = min(c, cmax);
        if (local) atomicAdd(mine + c, 1u);
        else atomicAdd(gh + c, 1u);
    };
    int64_t a0, a1;
    vector_span<T>(img, e0, e1, a0, a1);
    for (int64_t e = e0 + threadIdx.x; e < a0; e += kHistThreads) count((uint32_t)img[e]);
    for (int64_t e = a1 + threadIdx.x; e < e1; e += kHistThreads) count((uint32_t)img[e]);
    const uint4 *vec = reinterpret_cast<const uint4 *>(img + a0);
    const int64_t nv = (a1 - a0) / V;
    constexpr int kU = 4;  // vectors loaded before they are counted (loads in flight)
    for (int64_t k0 = threadIdx.x; k0 < nv; k0 += kU * kHistThreads) {
        uint4 x[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const int64_t k = k0 + (int64_t)u * kHistThreads;
            x[u] = k < nv ? vec[k] : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (k0 + (int64_t)u * kHistThreads >= nv) break;
#pragma unroll
            for (int j = 0; j < V; ++j) count(lane_code<T>(x[u], j));
        }
    }
    if (local) {
        __syncthreads();
        for (int c = threadIdx.x; c < h.n_codes; c += kHistThreads) {
            uint32_t n = 0;
            for (int w = 0; w < copies; ++w) n += s_h[w * h.n_codes + c];
            if (n) atomicAdd(gh + c, n);
        }
    }
}

// a * b as a 128-bit (hi, lo) pair
__device__ __forceinline__ void mul128(uint64_t a, uint64_t b, uint64_t &hi, uint64_t &lo) {
    lo = a * b;
    hi = __umul64hi(a, b);
}

__device__ __forceinline__ bool ge128(uint64_t ah, uint64_t al, uint64_t bh, uint64_t bl) {
    return ah > bh || (ah == bh && al >= bl);
}

// One CTA (1024 threads) per frame.
__global__ void __launch_bounds__(1024) k_hist_map(HistArgs h) {
    __shared__ uint32_t s[1024];
    __shared__ uint32_t carry;
    const int f = blockIdx.x;
    uint32_t *cs = h.hist + (size_t)f * h.n_codes;
    const uint64_t N = (uint64_t)h.frames[f].npx;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int c0 = 0; c0 < h.n_codes; c0 += 1024) {  // cumulative counts in place (block scan per tile)
        const int c = c0 + threadIdx.x;
        const uint32_t v = c < h.n_codes ? cs[c] : 0u;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            const uint32_t add = threadIdx.x >= off ? s[threadIdx.x - off] : 0u;
            __syncthreads();
            s[threadIdx.x] += add;
            __syncthreads();
        }
        if (c < h.n_codes) cs[c] = carry + s[threadIdx.x];
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
    const uint64_t T = h.ct[h.n_codes - 1];
    for (int c = threadIdx.x; c < h.n_codes; c += blockDim.x) {
        uint64_t rh, rl;
        mul128((uint64_t)cs[c], T, rh, rl);  // C_s(c) T
        int lo = 0, hi = h.n_codes - 1;      // smallest t with C_t(t) N >= C_s(c) T (the last code if none)
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            uint64_t mh, ml;
            mul128(h.ct[mid], N, mh, ml);
            if (ge128(mh, ml, rh, rl)) hi = mid;
            else lo = mid + 1;
        }
        h.lut[(size_t)f * h.n_codes + c] = (uint16_t)lo;
    }
}

template <typename T>
__global__ void __launch_bounds__(kHistThreads) k_hist_apply(HistArgs h, T *__restrict__ img) {
    __shared__ uint16_t s_lut[kSharedCodesMax];
    constexpr int V = 16 / sizeof(T);
    const int64_t q = blockIdx.x;
    const int f = frame_of_chunk(h, q);
    const Frame fr = h.frames[f];
    const int64_t p0 = (q - fr.chunk0) * kChunkPx, p1 = min(p0 + kChunkPx, fr.npx);
    const int64_t e0 = fr.offset + p0, e1 = fr.offset + p1;
    const uint16_t *glut = h.lut + (size_t)f * h.n_codes;
    const bool local = h.n_codes <= kSharedCodesMax;  // the frame's map staged in shared memory
    if (local) {
        for (int c = threadIdx.x; c < h.n_codes; c += kHistThreads) s_lut[c] = glut[c];
        __syncthreads();
    }
    const uint32_t cmax = (uint32_t)(h.n_codes - 1);
    auto map = [&](uint32_t c) -> uint32_t {
        c = min(c, cmax);
        return local ? s_lut[c] : glut[c];
    };
    int64_t a0, a1;
    vector_span<T>(img, e0, e1, a0, a1);
    for (int64_t e = e0 + threadIdx.x; e < a0; e += kHistThreads) img[e] = (T)map((uint32_t)img[e]);
    for (int64_t e = a1 + threadIdx.x; e < e1; e += kHistThreads) img[e] = (T)map((uint32_t)img[e]);
    uint4 *vec = reinterpret_cast<uint4 *>(img + a0);
    for (int64_t k = threadIdx.x; k < (a1 - a0) / V; k += kHistThreads) {
        const uint4 x = vec[k];
        uint32_t o[4] = {0u, 0u, 0u, 0u};
        constexpr int per = 4 / (int)sizeof(T);
#pragma unroll
        for (int j = 0; j < V; ++j) o[j / per] |= map(lane_code<T>(x, j)) << (8 * sizeof(T) * (j % per));
        vec[k] = make_uint4(o[0], o[1], o[2], o[3]);
    }
}

int fail(int code, const char *msg) { return spx::set_error(code, msg); }

// Validates the call and returns the codes per frame (0 on error, the message set).
int codes_of(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs, int32_t n_pairs) {
    if (!batch || (n_pairs > 0 && !pairs) || n_pairs < 0 || n_pairs > (1 << 20)) {
        fail(SYNTHPIX_EINVAL, "histogram matching: batch / pairs invalid");
        return 0;
    }
    if (batch->out_dtype != SYNTHPIX_U8 && batch->out_dtype != SYNTHPIX_U16) {
        fail(SYNTHPIX_EUNSUPPORTED, "histogram matching acts on quantised (U8 / U16) frames");
        return 0;
    }
    const int bits = batch->quant_bits;
    if (bits < 1 || bits > (batch->out_dtype == SYNTHPIX_U8 ? 8 : 16)) {
        fail(SYNTHPIX_EINVAL, "histogram matching: quant_bits out of range for the output type");
        return 0;
    }
    for (int32_t b = 0; b < n_pairs; ++b)
        if (pairs[b].height < 1 || pairs[b].width < 1 || pairs[b].height > 32768 || pairs[b].width > 32768 ||
            pairs[b].image_offset < 0) {
            fail(SYNTHPIX_EINVAL, "histogram matching: a pair's frame size or offset is invalid");
            return 0;
        }
    return 1 << bits;
}

}  // namespace

extern "C" {

size_t synthpix_match_histogram_workspace_bytes(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                                                int32_t n_pairs) {
    const int n_codes = codes_of(batch, pairs, n_pairs);
    if (!n_codes) return 0;
    return hist_layout(2 * n_pairs, n_codes).total;
}

int synthpix_match_histogram(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs, int32_t n_pairs,
                             void *images, const uint64_t *target, void *workspace, size_t workspace_bytes,
                             void *stream) {
    const int n_codes = codes_of(batch, pairs, n_pairs);
    if (!n_codes) return batch && batch->out_dtype != SYNTHPIX_U8 && batch->out_dtype != SYNTHPIX_U16
                             ? SYNTHPIX_EUNSUPPORTED : SYNTHPIX_EINVAL;
    if (n_pairs == 0) return spx::set_error(SYNTHPIX_OK, "");
    const size_t esz = batch->out_dtype == SYNTHPIX_U8 ? 1 : 2;
    if (!images || ((uintptr_t)images % esz)) return fail(SYNTHPIX_EINVAL, "histogram matching: images NULL or misaligned");
    if (!target || ((uintptr_t)target & 7)) return fail(SYNTHPIX_EINVAL, "histogram matching: target NULL or misaligned");
    const int n_frames = 2 * n_pairs;
    const HistLayout L = hist_layout(n_frames, n_codes);
    if (!workspace || ((uintptr_t)workspace & 255) || workspace_bytes < L.total)
        return fail(SYNTHPIX_EWORKSPACE, "histogram matching: workspace NULL, unaligned or too small");
    std::vector<Frame> fr((size_t)n_frames);
    int64_t chunks = 0;
    for (int32_t b = 0; b < n_pairs; ++b)
        for (int f = 0; f < 2; ++f) {
            Frame &x = fr[2 * b + f];
            x.npx = (int64_t)pairs[b].height * pairs[b].width;
            x.offset = pairs[b].image_offset + f * x.npx;
            x.chunk0 = chunks;
            chunks += (x.npx + kChunkPx - 1) / kChunkPx;
        }
    if (chunks > 0x7FFFFFFF) return fail(SYNTHPIX_EINVAL, "histogram matching: batch too large");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    cudaError_t e = cudaMemcpyAsync(ws + L.frames, fr.data(), fr.size() * sizeof(Frame), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(SYNTHPIX_ECUDA, "histogram matching: frame table copy failed");
    HistArgs h;
    h.frames = reinterpret_cast<const Frame *>(ws + L.frames);
    h.n_frames = n_frames;
    h.n_codes = n_codes;
    h.target = target;
    h.ct = reinterpret_cast<uint64_t *>(ws + L.ct);
    h.hist = reinterpret_cast<uint32_t *>(ws + L.hist);
    h.lut = reinterpret_cast<uint16_t *>(ws + L.lut);
    const int64_t nz = (int64_t)n_frames * n_codes;
    k_hist_target<<<1, 1024, 0, st>>>(h);
    k_hist_prep<<<(unsigned)std::min<int64_t>((nz + 255) / 256, 4096), 256, 0, st>>>(h);
    if (esz == 1) k_hist_count<uint8_t><<<(unsigned)chunks, kHistThreads, 0, st>>>(h, static_cast<const uint8_t *>(images));
    else k_hist_count<uint16_t><<<(unsigned)chunks, kHistThreads, 0, st>>>(h, static_cast<const uint16_t *>(images));
    k_hist_map<<<(unsigned)n_frames, 1024, 0, st>>>(h);
    if (esz == 1) k_hist_apply<uint8_t><<<(unsigned)chunks, kHistThreads, 0, st>>>(h, static_cast<uint8_t *>(images));
    else k_hist_apply<uint16_t><<<(unsigned)chunks, kHistThreads, 0, st>>>(h, static_cast<uint16_t *>(images));
    e = cudaGetLastError();
    if (e == cudaSuccess)
        for (int k = 0; k < 5; ++k) spx::count_launch();
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof(msg), "histogram matching launch: %s", cudaGetErrorString(e));
        return fail(SYNTHPIX_ECUDA, msg);
    }
    return spx::set_error(SYNTHPIX_OK, "");
}

}  // extern "C"
