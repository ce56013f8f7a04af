// Host entry points of the C ABI declared in include/synthpix.h: argument
// validation, workspace layout and the launch sequence.  Nothing here touches
// the device before every argument has been checked.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

bool finite(float v) { return std::isfinite(v); }

// Launch parameters a render runs with (a scheduling choice: results do not
// depend on them).
struct Tuning {
    spx::TileRule rule;  // tile edge per frame size class
    int32_t rec_buf;     // bytes of the splat's staged-record region
    int32_t reg_epi;     // 1: full 128 x 128 tiles finish with the register blur
};

struct Plan {
    spx::Layout L;
    Tuning T;
    int32_t tile;     // largest tile edge of the batch's pairs
    int32_t fused;
    int32_t max_halo;
    int32_t max_r;
    float max_d;
    int32_t ext;      // per-frame shapes: general shapes, frame-2 variation or hiding
    int32_t general;  // general-shape splat (32-byte records)
    int32_t rebin;    // some pair's fixed bins could overflow: the rebinning launches are needed
};

int check_batch(const synthpix_batch_desc *b) {
    if (!b) return fail(SYNTHPIX_EINVAL, "batch descriptor is NULL");
    if (b->out_dtype < SYNTHPIX_F32 || b->out_dtype > SYNTHPIX_U16)
        return fail(SYNTHPIX_EINVAL, "out_dtype %d is not one of F32/F16/BF16/U8/U16", b->out_dtype);
    if (b->out_dtype == SYNTHPIX_U8 && (b->quant_bits < 1 || b->quant_bits > 8))
        return fail(SYNTHPIX_EINVAL, "U8 output needs quant_bits in 1..8 (got %d)", b->quant_bits);
    if (b->out_dtype == SYNTHPIX_U16 && (b->quant_bits < 1 || b->quant_bits > 16))
        return fail(SYNTHPIX_EINVAL, "U16 output needs quant_bits in 1..16 (got %d)", b->quant_bits);
    if (b->out_dtype <= SYNTHPIX_BF16 && b->quant_bits != 0)
        return fail(SYNTHPIX_EINVAL, "float outputs need quant_bits = 0 (got %d)", b->quant_bits);
    if (b->inter_dtype < SYNTHPIX_F32 || b->inter_dtype > SYNTHPIX_BF16)
        return fail(SYNTHPIX_EINVAL, "inter_dtype %d is not one of F32/F16/BF16", b->inter_dtype);
    if (b->integrator != SYNTHPIX_RK4 && b->integrator != SYNTHPIX_EULER)
        return fail(SYNTHPIX_EINVAL, "integrator %d is not RK4 (0) or Euler (1)", b->integrator);
    if (b->n_substeps < 1 || b->n_substeps > 1024)
        return fail(SYNTHPIX_EINVAL, "n_substeps %d outside 1..1024", b->n_substeps);
    if (!finite(b->dt) || std::fabs(b->dt) > 64.0f) return fail(SYNTHPIX_EINVAL, "dt must be finite with |dt| <= 64");
    if (b->tile != 0 && b->tile != 16 && b->tile != 32 && b->tile != 64 && b->tile != 128)
        return fail(SYNTHPIX_EINVAL, "tile %d is not 0, 16, 32, 64 or 128", b->tile);
    if (b->flags & ~(SYNTHPIX_FLAG_GATHER_ADVECT | SYNTHPIX_FLAG_OUT_OF_PLANE | SYNTHPIX_FLAG_TILED_ADVECT))
        return fail(SYNTHPIX_EUNSUPPORTED, "unknown flags 0x%x", b->flags);
    if ((b->flags & SYNTHPIX_FLAG_GATHER_ADVECT) && (b->flags & SYNTHPIX_FLAG_TILED_ADVECT))
        return fail(SYNTHPIX_EINVAL, "flags GATHER_ADVECT and TILED_ADVECT exclude each other");
    if (!finite(b->hide_prob) || b->hide_prob < 0.0f || b->hide_prob > 1.0f)
        return fail(SYNTHPIX_EINVAL, "hide_prob must lie in [0, 1]");
    for (int k = 0; k < 5; ++k)
        if (b->reserved[k] != 0) return fail(SYNTHPIX_EUNSUPPORTED, "batch reserved[%d] is not zero", k);
    return SYNTHPIX_OK;
}

int check_pair(const synthpix_pair_desc &d, int b) {
    if (d.height < 1 || d.height > 32768 || d.width < 1 || d.width > 32768)
        return fail(SYNTHPIX_EINVAL, "pair %d: frame %dx%d outside 1..32768", b, d.height, d.width);
    if (d.flow_h < 1 || d.flow_h > 32768 || d.flow_w < 1 || d.flow_w > 32768)
        return fail(SYNTHPIX_EINVAL, "pair %d: flow grid %dx%d outside 1..32768", b, d.flow_h, d.flow_w);
    if (d.flow_offset < 0 || (d.flow_offset & 1))
        return fail(SYNTHPIX_EINVAL, "pair %d: flow_offset must be even and >= 0", b);
    if (d.image_offset < 0 || d.image_offset > (int64_t(1) << 60))
        return fail(SYNTHPIX_EINVAL, "pair %d: image_offset out of range", b);
    if (d.d_dist != 0 && d.d_dist != 1) return fail(SYNTHPIX_EINVAL, "pair %d: d_dist must be 0 or 1", b);
    const float fs[] = {d.d_min, d.d_max, d.d_mu, d.d_sigma, d.i_min, d.i_max, d.z_min, d.z_max,
                        d.sheet_sigma, d.illum_min, d.illum_max, d.noise_sigma, d.blur_sigma,
                        d.dy_min, d.dy_max, d.rho_min, d.rho_max, d.jitter_d, d.jitter_i, d.jitter_rho};
    for (float v : fs)
        if (!finite(v)) return fail(SYNTHPIX_EINVAL, "pair %d: non-finite parameter", b);
    if (!(d.d_min > 0.0f) || d.d_max < d.d_min || d.d_max > 32.0f)
        return fail(SYNTHPIX_EINVAL, "pair %d: need 0 < d_min <= d_max <= 32", b);
    if (d.d_sigma < 0.0f) return fail(SYNTHPIX_EINVAL, "pair %d: d_sigma < 0", b);
    if (d.i_min < 0.0f || d.i_max < d.i_min || d.i_max > 1e6f)
        return fail(SYNTHPIX_EINVAL, "pair %d: need 0 <= i_min <= i_max <= 1e6", b);
    if (d.z_max < d.z_min) return fail(SYNTHPIX_EINVAL, "pair %d: z_max < z_min", b);
    if (d.illum_max < d.illum_min || std::fabs(d.illum_min) > 1e6f || std::fabs(d.illum_max) > 1e6f)
        return fail(SYNTHPIX_EINVAL, "pair %d: need illum_min <= illum_max within +-1e6", b);
    if (d.noise_sigma < 0.0f || d.noise_sigma > 1e6f) return fail(SYNTHPIX_EINVAL, "pair %d: noise_sigma < 0", b);
    if (d.blur_sigma < 0.0f || d.blur_sigma > 8.0f) return fail(SYNTHPIX_EINVAL, "pair %d: blur_sigma outside 0..8", b);
    if (!(d.dy_min == 0.0f && d.dy_max == 0.0f) && !(d.dy_min > 0.0f && d.dy_max >= d.dy_min && d.dy_max <= 32.0f))
        return fail(SYNTHPIX_EINVAL, "pair %d: need dy_min = dy_max = 0 or 0 < dy_min <= dy_max <= 32", b);
    if (d.rho_min < -0.95f || d.rho_max < d.rho_min || d.rho_max > 0.95f)
        return fail(SYNTHPIX_EINVAL, "pair %d: need -0.95 <= rho_min <= rho_max <= 0.95", b);
    if (d.jitter_d < 0.0f || d.jitter_i < 0.0f || d.jitter_rho < 0.0f || d.jitter_d > 1e6f || d.jitter_i > 1e6f ||
        d.jitter_rho > 1e6f)
        return fail(SYNTHPIX_EINVAL, "pair %d: jitter stds must lie in [0, 1e6]", b);
    if (d.sheet_model != SYNTHPIX_SHEET_GAUSSIAN && d.sheet_model != SYNTHPIX_SHEET_REMARK)
        return fail(SYNTHPIX_EINVAL, "pair %d: sheet_model must be 0 (Gaussian) or 1 (Remark form)", b);
    if (d.sheet_model == SYNTHPIX_SHEET_REMARK && !(d.sheet_shape > 0.0f && d.sheet_shape <= 16.0f))
        return fail(SYNTHPIX_EINVAL, "pair %d: the Remark form needs 0 < sheet_shape <= 16", b);
    if (!finite(d.sheet_shape)) return fail(SYNTHPIX_EINVAL, "pair %d: non-finite sheet_shape", b);
    for (int k = 0; k < 6; ++k)
        if (d.reserved[k] != 0) return fail(SYNTHPIX_EUNSUPPORTED, "pair %d: reserved[%d] is not zero", b, k);
    return SYNTHPIX_OK;
}

// Tile edges used when batch->tile is 0 and no tuned entry exists, by frame
// size class: 32 below 2^15 pixels (enough work items for small frames), 64
// below 2^17, 128 from there (fewer particles rendered twice at tile
// borders, fewer work items).
constexpr spx::TileRule kDefaultRule = {{32, 64, 128, 128}};
constexpr int kTileCandidates[4] = {16, 32, 64, 128};
constexpr int kRecBufCandidates[3] = {2 * 8192 - 2 * spx::kStageHeader, spx::kRecBufBytes, spx::kRecBufBytesLarge};

spx::TileRule uniform_rule(int t) { return spx::TileRule{{t, t, t, t}}; }

Tuning default_tuning(const spx::TileRule &rule) {
    Tuning T;
    T.rule = rule;
    T.rec_buf = 0;  // resolved from the largest edge by make_plan_tuned
    T.reg_epi = 1;
    return T;
}

// The autotuner's cache: per (frame size class, largest diameter in quarter
// pixels, blur radius, general-shape splat, fused epilogue) the tuned tile
// edge, and the batch-level choices (records per stage, register epilogue)
// of the batch that was tuned.  Guarded by a mutex; renders with tile 0 read
// it, synthpix_autotune writes it (after its timed renders, never while
// holding the lock).
struct TuneKey {
    int32_t cls, dq, r, general, fused;
    bool operator<(const TuneKey &o) const {
        if (cls != o.cls) return cls < o.cls;
        if (dq != o.dq) return dq < o.dq;
        if (r != o.r) return r < o.r;
        if (general != o.general) return general < o.general;
        return fused < o.fused;
    }
};
struct TuneEntry {
    int32_t tile, rec_buf, reg_epi;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneEntry> g_tune;

// Per size class of the batch: present, its key, and its pixels (work).
struct ClassInfo {
    bool present[spx::kSizeClasses];
    TuneKey key[spx::kSizeClasses];
    double pixels[spx::kSizeClasses];
    int largest;  // the class with the most pixels
};

ClassInfo batch_classes(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs, int32_t n_pairs) {
    ClassInfo c;
    float dmax[spx::kSizeClasses] = {0.f, 0.f, 0.f, 0.f};
    int32_t rmax[spx::kSizeClasses] = {0, 0, 0, 0};
    bool general = false;
    for (int k = 0; k < spx::kSizeClasses; ++k) {
        c.present[k] = false;
        c.pixels[k] = 0.0;
    }
    for (int32_t b = 0; b < n_pairs; ++b) {
        const int k = spx::size_class(pairs[b].height, pairs[b].width);
        c.present[k] = true;
        c.pixels[k] += (double)pairs[b].height * pairs[b].width;
        dmax[k] = std::max(dmax[k], spx::pair_max_diameter(pairs[b]));
        rmax[k] = std::max(rmax[k], spx::blur_radius_of(pairs[b].blur_sigma));
        general = general || spx::pair_general_shape(pairs[b]);
    }
    c.largest = 0;
    for (int k = 0; k < spx::kSizeClasses; ++k) {
        c.key[k] = TuneKey{k, (int32_t)std::ceil(4.0f * dmax[k]), rmax[k], general ? 1 : 0,
                           batch->inter_dtype == SYNTHPIX_F32 ? 1 : 0};
        if (c.pixels[k] > c.pixels[c.largest]) c.largest = k;
    }
    return c;
}

// The tuning a render runs with: batch->tile for every class when it is
// set; otherwise the cached entries of the batch's classes, default edges
// where none is cached.  A cached record-buffer size was tuned with the
// largest edge of the tuned batch; it is clamped to what this batch's
// largest edge allows (the chunking changes, the rendered bits do not).
Tuning resolve_tuning(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs, int32_t n_pairs) {
    if (batch->tile != 0) return default_tuning(uniform_rule(batch->tile));
    Tuning T = default_tuning(kDefaultRule);
    if (n_pairs <= 0 || !pairs) return T;
    const ClassInfo c = batch_classes(batch, pairs, n_pairs);
    std::lock_guard<std::mutex> lock(g_tune_mu);
    int32_t emax = 0;
    for (int k = 0; k < spx::kSizeClasses; ++k) {
        if (!c.present[k]) continue;
        const auto it = g_tune.find(c.key[k]);
        if (it != g_tune.end()) {
            T.rule.edge[k] = it->second.tile;
            if (k == c.largest) {
                T.rec_buf = it->second.rec_buf;
                T.reg_epi = it->second.reg_epi;
            }
        }
        emax = std::max(emax, T.rule.edge[k]);
    }
    if (T.rec_buf > spx::rec_buf_bytes_for(emax)) T.rec_buf = spx::rec_buf_bytes_for(emax);
    return T;
}

int make_plan_tuned(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs, int32_t n_pairs,
                    const Tuning &T, Plan &P);

int check_counts(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs, int32_t n_pairs) {
    int rc = check_batch(batch);
    if (rc) return rc;
    if (n_pairs < 0 || n_pairs > (1 << 20)) return fail(SYNTHPIX_EINVAL, "n_pairs %d outside 0..2^20", n_pairs);
    if (n_pairs > 0 && !pairs) return fail(SYNTHPIX_EINVAL, "pairs is NULL");
    return SYNTHPIX_OK;
}

int make_plan(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs, int32_t n_pairs, Plan &P) {
    const int rc = check_counts(batch, pairs, n_pairs);
    if (rc) return rc;
    return make_plan_tuned(batch, pairs, n_pairs, resolve_tuning(batch, pairs, n_pairs), P);
}

// The workspace plan of a batch under tuning T.  With worst = true, every
// pair takes the largest of its per-tile sizes over all candidate edges and
// the carry words those of the largest edge: an upper bound for any tuning.
int make_plan_any(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs, int32_t n_pairs,
                  const Tuning &T, bool worst, Plan &P) {
    int rc;
    P.T = T;
    P.tile = 0;
    P.fused = batch->inter_dtype == SYNTHPIX_F32 ? 1 : 0;
    P.max_halo = 0;
    P.max_r = 0;
    P.max_d = 0.0f;
    P.ext = (batch->hide_prob > 0.0f || (batch->flags & SYNTHPIX_FLAG_OUT_OF_PLANE)) ? 1 : 0;
    P.general = 0;
    P.rebin = 0;
    spx::Layout &L = P.L;
    L.n_part = L.n_tiles = L.n_list = L.n_inter = L.n_chunks = 0;
    for (int32_t b = 0; b < n_pairs; ++b) {
        rc = check_pair(pairs[b], b);
        if (rc) return rc;
        const int32_t t = worst ? 128 : spx::rule_tile(T.rule, pairs[b]);
        if (t != 16 && t != 32 && t != 64 && t != 128)
            return fail(SYNTHPIX_EINVAL, "pair %d: tile edge %d is not 16, 32, 64 or 128", b, t);
        P.tile = std::max(P.tile, t);
        spx::PairGeom g = spx::pair_geom(pairs[b], t, P.fused != 0);
        if (worst)
            for (int c : kTileCandidates) {
                const spx::PairGeom h = spx::pair_geom(pairs[b], c, P.fused != 0);
                g.ntiles = std::max(g.ntiles, h.ntiles);
                g.list_cap = std::max(g.list_cap, h.list_cap);
            }
        if (!spx::fixed_exact(pairs[b], t, g.halo)) P.rebin = 1;
        L.n_part += pairs[b].n_particles;
        L.n_tiles += 2LL * g.ntiles;
        L.n_list += 2LL * g.list_cap;
        L.n_chunks += g.chunks;
        if (!P.fused) L.n_inter += 2LL * pairs[b].height * pairs[b].width;
        if (g.halo > P.max_halo) P.max_halo = g.halo;
        if (g.blur_r > P.max_r) P.max_r = g.blur_r;
        const float dmax = spx::pair_max_diameter(pairs[b]);
        if (dmax > P.max_d) P.max_d = dmax;
        if (spx::pair_general_shape(pairs[b])) P.general = P.ext = 1;
        if (pairs[b].jitter_d != 0.0f || pairs[b].jitter_i != 0.0f || pairs[b].jitter_rho != 0.0f) P.ext = 1;
    }
    if (L.n_tiles > 0x7FFFFFFFLL) return fail(SYNTHPIX_EINVAL, "batch has more than 2^31-1 tiles");
    if (L.n_chunks > 0x7FFFFFFFLL) return fail(SYNTHPIX_EINVAL, "batch has more than 2^40 particles");
    if (L.n_list > (int64_t(1) << 40)) return fail(SYNTHPIX_EINVAL, "batch bin lists too large");
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = spx::align256(o + bytes);
        return at;
    };
    L.plan = take((size_t)n_pairs * sizeof(spx::PairPlan));
    L.desc = take((size_t)n_pairs * sizeof(synthpix_pair_desc));
    L.check = take(256);
    L.blur = take((size_t)n_pairs * spx::kBlurStride * sizeof(float));
    L.count = take((size_t)L.n_tiles * 4);
    L.off = take((size_t)L.n_tiles * 4);
    L.cursor = take((size_t)L.n_tiles * 4);
    L.items = take((size_t)L.n_tiles * sizeof(spx::ItemInfo));
    L.pos = take((size_t)L.n_part * 32);
    L.sa = take((size_t)L.n_part * 8);
    L.shape = take(P.ext ? (size_t)L.n_part * 2 * sizeof(float4) : 0);
    const size_t rec_bytes = P.general ? sizeof(spx::RecordG) : sizeof(spx::Record);
    L.rec = take((size_t)L.n_list * rec_bytes + 64);  // + read-over of 16-byte staging
    L.adv = take((size_t)(L.n_list / 2) * sizeof(spx::Record));  // frame-1 segments only
    L.inter = take((size_t)L.n_inter * 2);
    if (P.tile == 0) P.tile = 16;  // no pairs: nothing is launched
    {  // carry words of the splat's CTAs: one accumulator's worth each
        const int E = P.tile + 2 * P.max_r;
        L.carry_stride = (int64_t)E * spx::pitch_cap(E);
        size_t cw = (size_t)spx::splat_max_ctas(P.tile, L.n_tiles) * (size_t)L.carry_stride;
        if (worst)  // the largest over every edge the pairs could take
            for (int c : kTileCandidates) {
                const int Ec = c + 2 * P.max_r;
                cw = std::max(cw, (size_t)spx::splat_max_ctas(c, L.n_tiles) * (size_t)Ec * spx::pitch_cap(Ec));
            }
        L.carry = take(cw * 4);
    }
    if (P.T.rec_buf == 0) P.T.rec_buf = spx::rec_buf_bytes_for(P.tile);
    // at least one record of either size; at most what the splat's per-thread slots cover
    if (P.T.rec_buf < 32 + (int)sizeof(spx::RecordG) ||
        P.T.rec_buf > spx::rec_buf_bytes_for(P.tile) || (P.T.rec_buf & 15))
        return fail(SYNTHPIX_EUNSUPPORTED, "%d-byte record buffers do not fit tile edge %d", P.T.rec_buf, P.tile);
    L.gfr = take((size_t)L.n_part * 2 * sizeof(float4));
    L.total = o;
    return SYNTHPIX_OK;
}

int make_plan_tuned(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs, int32_t n_pairs,
                    const Tuning &T, Plan &P) {
    return make_plan_any(batch, pairs, n_pairs, T, false, P);
}

size_t elem_size(int32_t dt) {
    switch (dt) {
    case SYNTHPIX_F32: return 4;
    case SYNTHPIX_U8: return 1;
    default: return 2;
    }
}

}  // namespace

namespace spx {
static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
uint64_t launch_total() { return g_launches.load(std::memory_order_relaxed); }
thread_local std::vector<RecordedLaunch> *t_recording = nullptr;
}  // namespace spx

namespace {

// A render's launch sequence (plan, seeding and binning, splat) submitted as
// one CUDA graph: the GPU starts each kernel of a graph sooner after the
// previous one than it starts stream launches.  Sequences are keyed by the
// device and by each launch's kernel and shape; a sequence met for the first
// time is launched kernel by kernel, the second time it is instantiated as a
// graph (a chain of kernel nodes), and from then on each render sets the
// nodes' arguments and launches the graph.  Graph launches of one sequence
// are ordered behind one another, whatever their streams.  Not used while
// the stream is being captured (the caller's graph records the kernels
// themselves), for staged renders (events between the stages), or where the
// library must not allocate (t_direct).
struct SeqKey {
    int device;
    std::vector<std::tuple<const void *, unsigned, unsigned, size_t>> shape;
    bool operator<(const SeqKey &o) const { return std::tie(device, shape) < std::tie(o.device, o.shape); }
};
struct SeqGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaGraphNode_t> nodes;
};
constexpr size_t kMaxSeqGraphs = 32;  // instantiated sequences kept (then new ones run kernel by kernel)
constexpr size_t kMaxSeqSeen = 1024;  // sequences remembered as met once
std::mutex g_seq_mu;
std::map<SeqKey, SeqGraph> g_seq_graphs;
std::map<SeqKey, int> g_seq_seen;
thread_local bool t_direct = false;

cudaKernelNodeParams node_params(const spx::RecordedLaunch &r) {
    cudaKernelNodeParams p{};
    p.func = const_cast<void *>(r.func);
    p.gridDim = dim3(r.grid);
    p.blockDim = dim3(r.block);
    p.sharedMemBytes = (unsigned)r.smem;
    p.kernelParams = const_cast<void **>(r.params.data());
    p.extra = nullptr;
    return p;
}

cudaError_t launch_direct(const std::vector<spx::RecordedLaunch> &seq, cudaStream_t st) {
    for (const spx::RecordedLaunch &r : seq) {
        const cudaError_t e = cudaLaunchKernel(r.func, dim3(r.grid), dim3(r.block),
                                               const_cast<void **>(r.params.data()), r.smem, st);
        if (e != cudaSuccess) return e;
        spx::count_launch();
    }
    return cudaSuccess;
}

void destroy(SeqGraph &g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g = SeqGraph();
}

cudaError_t build(const std::vector<spx::RecordedLaunch> &seq, SeqGraph &g) {
    cudaError_t e = cudaGraphCreate(&g.graph, 0);
    for (size_t i = 0; e == cudaSuccess && i < seq.size(); ++i) {
        const cudaKernelNodeParams p = node_params(seq[i]);
        cudaGraphNode_t n = nullptr;
        e = cudaGraphAddKernelNode(&n, g.graph, i ? &g.nodes.back() : nullptr, i ? 1 : 0, &p);
        if (e == cudaSuccess) g.nodes.push_back(n);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, g.graph, 0);
    if (e != cudaSuccess) destroy(g);
    return e;
}

cudaError_t submit(const std::vector<spx::RecordedLaunch> &seq, cudaStream_t st) {
    if (seq.empty()) return cudaSuccess;
    SeqKey key;
    cudaError_t e = cudaGetDevice(&key.device);
    if (e != cudaSuccess) return e;
    for (const spx::RecordedLaunch &r : seq) key.shape.emplace_back(r.func, r.grid, r.block, r.smem);
    std::lock_guard<std::mutex> lock(g_seq_mu);
    auto it = g_seq_graphs.find(key);
    if (it == g_seq_graphs.end()) {
        if (g_seq_graphs.size() >= kMaxSeqGraphs) return launch_direct(seq, st);
        if (g_seq_seen.size() >= kMaxSeqSeen) g_seq_seen.clear();
        if (g_seq_seen[key]++ == 0) return launch_direct(seq, st);
        SeqGraph g;
        if (build(seq, g) != cudaSuccess) {
            cudaGetLastError();  // the sequence still runs, kernel by kernel
            return launch_direct(seq, st);
        }
        g_seq_seen.erase(key);
        it = g_seq_graphs.emplace(std::move(key), g).first;
    } else {
        for (size_t i = 0; i < seq.size(); ++i) {
            const cudaKernelNodeParams p = node_params(seq[i]);
            e = cudaGraphExecKernelNodeSetParams(it->second.exec, it->second.nodes[i], &p);
            if (e != cudaSuccess) return e;
        }
    }
    e = cudaGraphLaunch(it->second.exec, st);
    if (e == cudaSuccess)
        for (size_t i = 0; i < seq.size(); ++i) spx::count_launch();
    return e;
}

// Records the launches of its scope on this thread (see launch_kernel).
struct Recording {
    std::vector<spx::RecordedLaunch> seq;
    bool on;
    explicit Recording(bool enable) : on(enable) {
        if (on) spx::t_recording = &seq;
    }
    ~Recording() {
        if (on) spx::t_recording = nullptr;
    }
};

bool stream_capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
        cudaGetLastError();
        return true;  // unknown: launch kernel by kernel
    }
    return cs != cudaStreamCaptureStatusNone;
}

}  // namespace

static_assert(sizeof(synthpix_pair_desc) == 160, "pair descriptor ABI");
static_assert(sizeof(synthpix_batch_desc) == 64, "batch descriptor ABI");

extern "C" {

const char *synthpix_last_error(void) { return g_err; }

int synthpix_version(void) { return SYNTHPIX_ABI_VERSION; }

uint64_t synthpix_launch_count(void) { return spx::launch_total(); }

size_t synthpix_workspace_bytes(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                                int32_t n_pairs) {
    Plan P;
    if (make_plan(batch, pairs, n_pairs, P) != SYNTHPIX_OK) return 0;
    size_t need = P.L.total;
    if (batch->tile == 0) {  // large enough for every tuning the autotuner may try or cache
        Plan Q;
        if (make_plan_any(batch, pairs, n_pairs, default_tuning(kDefaultRule), true, Q) != SYNTHPIX_OK) return 0;
        need = std::max(need, Q.L.total);
    }
    g_err[0] = 0;
    return need;
}

}  // extern "C"

enum class Mode { Render, Seed, Advect, Backward };

// Optional arguments of the seeding and adjoint entry points.
struct Extra {
    const float *particles_in = nullptr;
    float *particles_out = nullptr;
    const float *grad_images = nullptr;
    float *grad_flows = nullptr;
    float *grad_particles = nullptr;
};

static int run(Mode mode, const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
               const synthpix_pair_desc *pairs_dev, int32_t n_pairs, const float *flows, void *images,
               void *workspace, size_t workspace_bytes, void *stream, cudaEvent_t const *ev, const Extra &x,
               const Tuning *tuning = nullptr) {
    Plan P;
    int rc = check_counts(batch, pairs, n_pairs);
    if (rc) return rc;
    rc = make_plan_tuned(batch, pairs, n_pairs, tuning ? *tuning : resolve_tuning(batch, pairs, n_pairs), P);
    if (rc) return rc;
    if (n_pairs == 0) {
        g_err[0] = 0;
        return SYNTHPIX_OK;
    }
    const bool exporting = mode == Mode::Seed || mode == Mode::Advect;
    if (mode != Mode::Seed && (!flows || ((uintptr_t)flows & 7)))
        return fail(SYNTHPIX_EINVAL, "flows is NULL or not 8-byte aligned");
    if (mode == Mode::Render && (!images || ((uintptr_t)images % elem_size(batch->out_dtype))))
        return fail(SYNTHPIX_EINVAL, "images is NULL or misaligned for its element type");
    if (exporting && (!x.particles_out || ((uintptr_t)x.particles_out & 3)))
        return fail(SYNTHPIX_EINVAL, "particles_out is NULL or not 4-byte aligned");
    if (x.particles_in && ((uintptr_t)x.particles_in & 3))
        return fail(SYNTHPIX_EINVAL, "particles_in is not 4-byte aligned");
    if ((x.particles_in || mode == Mode::Backward) && P.ext)
        return fail(SYNTHPIX_EUNSUPPORTED,
                    "given particles and the adjoint need round particles without hiding or frame-2 variation");
    if (mode == Mode::Backward) {
        if (!x.grad_images || ((uintptr_t)x.grad_images & 3))
            return fail(SYNTHPIX_EINVAL, "grad_images is NULL or not 4-byte aligned");
        if ((x.grad_flows && ((uintptr_t)x.grad_flows & 7)) || (x.grad_particles && ((uintptr_t)x.grad_particles & 3)))
            return fail(SYNTHPIX_EINVAL, "grad_flows must be 8-byte and grad_particles 4-byte aligned");
        if (batch->out_dtype != SYNTHPIX_F32)
            return fail(SYNTHPIX_EUNSUPPORTED, "the adjoint needs out_dtype F32 (quantisation has no gradient)");
        if (batch->n_substeps > spx::kMaxAdjointSubsteps)
            return fail(SYNTHPIX_EUNSUPPORTED, "the adjoint supports at most %d substeps", spx::kMaxAdjointSubsteps);
        for (int32_t b = 0; b < n_pairs; ++b)
            if (pairs[b].blur_sigma != 0.0f)
                return fail(SYNTHPIX_EUNSUPPORTED, "pair %d: the adjoint does not support blur", b);
    }
    if (!workspace || ((uintptr_t)workspace & 255))
        return fail(SYNTHPIX_EWORKSPACE, "workspace is NULL or not 256-byte aligned");
    if (workspace_bytes < P.L.total)
        return fail(SYNTHPIX_EWORKSPACE, "workspace has %zu bytes, %zu needed", workspace_bytes, P.L.total);
    if (pairs_dev && ((uintptr_t)pairs_dev & 15)) return fail(SYNTHPIX_EINVAL, "pairs_dev is not 16-byte aligned");

    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    const spx::Layout &L = P.L;
    const synthpix_pair_desc *descs = pairs_dev;
    cudaError_t e;
    if (!descs) {
        e = cudaMemcpyAsync(ws + L.desc, pairs, (size_t)n_pairs * sizeof(synthpix_pair_desc),
                            cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return fail(SYNTHPIX_ECUDA, "descriptor copy: %s", cudaGetErrorString(e));
        descs = reinterpret_cast<const synthpix_pair_desc *>(ws + L.desc);
    }
    spx::PairPlan *plan = reinterpret_cast<spx::PairPlan *>(ws + L.plan);
    int32_t *check = reinterpret_cast<int32_t *>(ws + L.check);
    uint32_t *ticket = reinterpret_cast<uint32_t *>(ws + L.check + 16);
    float *blur_w = reinterpret_cast<float *>(ws + L.blur);
    // flow grids of at most a quarter of L2 in all: the plan launch has them
    // fetched into L2 ahead of the advection's dependent gathers
    const int32_t planes = (batch->flags & SYNTHPIX_FLAG_OUT_OF_PLANE) ? 3 : 2;
    int64_t flow_bytes = 0;
    for (int32_t b = 0; b < n_pairs; ++b) flow_bytes += 4LL * planes * pairs[b].flow_h * pairs[b].flow_w;
    const float *pf_flows = mode != Mode::Seed && flow_bytes <= spx::kPrefetchMaxBytes ? flows : nullptr;
    // renders without stage events: the launch sequence goes to the GPU as one graph
    Recording rec(mode == Mode::Render && !ev && !t_direct && !stream_capturing(st));
    if (ev && ev[0]) cudaEventRecord(ev[0], st);
    e = spx::launch_plan(descs, n_pairs, P.T.rule, P.fused, plan, L, check, blur_w, ticket,
                         mode == Mode::Render ? reinterpret_cast<uint32_t *>(ws + L.count) : nullptr, pf_flows,
                         planes, st);
    if (e != cudaSuccess) return fail(SYNTHPIX_ECUDA, "plan launch: %s", cudaGetErrorString(e));
    if (ev && ev[1]) cudaEventRecord(ev[1], st);

    spx::KernelArgs a;
    a.descs = descs;
    a.plan = plan;
    a.check = check;
    a.n_pairs = n_pairs;
    a.tile = P.tile;
    a.n_part = L.n_part;
    a.n_tiles = L.n_tiles;
    a.n_chunks = L.n_chunks;
    a.seed = batch->seed;
    a.keys = spx::philox_round_keys(batch->seed);
    a.dt = batch->dt;
    a.n_substeps = batch->n_substeps;
    a.integrator = batch->integrator;
    a.quant_bits = batch->quant_bits;
    a.flows = flows;
    a.images = images;
    a.pos0 = reinterpret_cast<float4 *>(ws + L.pos);
    a.pos1 = a.pos0 + L.n_part;
    a.sa = reinterpret_cast<float2 *>(ws + L.sa);
    a.shape = reinterpret_cast<float4 *>(ws + L.shape);
    a.ext = P.ext;
    a.general = P.general;
    a.hide_prob = batch->hide_prob;
    a.out_of_plane = (batch->flags & SYNTHPIX_FLAG_OUT_OF_PLANE) ? 1 : 0;
    a.count = mode == Mode::Render ? reinterpret_cast<uint32_t *>(ws + L.count) : nullptr;
    a.off = reinterpret_cast<uint32_t *>(ws + L.off);
    a.cursor = reinterpret_cast<uint32_t *>(ws + L.cursor);
    a.items = reinterpret_cast<spx::ItemInfo *>(ws + L.items);
    a.rec = reinterpret_cast<spx::Record *>(ws + L.rec);
    a.adv = reinterpret_cast<spx::Record *>(ws + L.adv);
    // per-frame shapes need each particle's index: those renders advect per particle
    if (mode == Mode::Render && !x.particles_in && !P.ext && !(batch->flags & SYNTHPIX_FLAG_GATHER_ADVECT))
        a.tiled = (batch->flags & SYNTHPIX_FLAG_TILED_ADVECT) ? 1 : 2;
    else
        a.tiled = 0;
    a.ticket = ticket;
    a.ovf = ticket + 1;
    a.rebin = P.rebin;
    a.rec_buf_bytes = P.T.rec_buf;
    a.reg_epilogue = P.T.reg_epi;
    a.blur_w = blur_w;
    a.inter_dtype = batch->inter_dtype;
    a.inter = ws + L.inter;
    a.particles_in = x.particles_in;
    a.particles_out = exporting ? x.particles_out : nullptr;
    a.export_frame = mode == Mode::Advect ? 1 : 0;
    a.grad_images = x.grad_images;
    a.grad_flows = x.grad_flows;
    a.grad_particles = x.grad_particles;
    a.grad_frames = reinterpret_cast<float4 *>(ws + L.gfr);
    a.states = nullptr;
    a.carry = reinterpret_cast<uint32_t *>(ws + L.carry);
    a.carry_stride = L.carry_stride;
    a.smem_edge = P.tile + 2 * P.max_r;
    const int wmax = std::min(spx::window_max(P.max_d), a.smem_edge);
    a.warp_scratch = 4 * (wmax + 2);
    if (exporting) {
        e = spx::launch_seed_only(a, st);
        if (e != cudaSuccess) return fail(SYNTHPIX_ECUDA, "seeding launch: %s", cudaGetErrorString(e));
    } else if (mode == Mode::Backward) {
        a.warp_scratch = spx::window_max(P.max_d) + 2;  // floats per scratch array of the adjoint splat
        // the substep starts of the advection go to the bin records' region (no bins in the adjoint)
        // when they fit there; otherwise the adjoint recomputes them
        const size_t states = (size_t)L.n_part * (size_t)batch->n_substeps * sizeof(float4);
        if (states <= (size_t)L.n_list * (P.general ? sizeof(spx::RecordG) : sizeof(spx::Record)))
            a.states = reinterpret_cast<float4 *>(ws + L.rec);
        e = spx::launch_seed_only(a, st);                // positions of both frames
        if (e == cudaSuccess) e = spx::launch_adjoint(a, st);
        if (e != cudaSuccess) return fail(SYNTHPIX_ECUDA, "adjoint launch: %s", cudaGetErrorString(e));
    } else {
        if (spx::splat_smem_bytes(a.smem_edge, a.tile, a.warp_scratch, a.rec_buf_bytes) > spx::kMaxSmemBytes)
            return fail(SYNTHPIX_EUNSUPPORTED, "tile %d with blur radius %d needs too much shared memory", P.tile,
                        P.max_r);
        e = spx::launch_prep(a, st, ev);
        if (e != cudaSuccess) return fail(SYNTHPIX_ECUDA, "seeding/binning launch: %s", cudaGetErrorString(e));
        e = spx::launch_splat(a, batch->out_dtype, st, ev);
        if (e != cudaSuccess) return fail(SYNTHPIX_ECUDA, "splat launch: %s", cudaGetErrorString(e));
        if (rec.on) {
            spx::t_recording = nullptr;
            e = submit(rec.seq, st);
            if (e != cudaSuccess) return fail(SYNTHPIX_ECUDA, "render launch: %s", cudaGetErrorString(e));
        }
    }
    g_err[0] = 0;
    return SYNTHPIX_OK;
}

static int render_impl(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                       const synthpix_pair_desc *pairs_dev, int32_t n_pairs, const float *flows, void *images,
                       void *workspace, size_t workspace_bytes, void *stream, cudaEvent_t const *ev,
                       const Tuning *tuning = nullptr) {
    return run(Mode::Render, batch, pairs, pairs_dev, n_pairs, flows, images, workspace, workspace_bytes, stream, ev,
               Extra(), tuning);
}

// Mean time (ms) of `reps` renders with tuning T after one warm-up render, on
// `stream` (blocks the host).  SYNTHPIX_EUNSUPPORTED: the tuning does not fit
// the batch (shared memory); other errors as the render's.
static int time_renders(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                        const synthpix_pair_desc *pairs_dev, int32_t n_pairs, const float *flows, void *images,
                        void *workspace, size_t workspace_bytes, void *stream, int32_t reps, const Tuning &T,
                        cudaEvent_t e0, cudaEvent_t e1, float *ms) {
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int rc = render_impl(batch, pairs, pairs_dev, n_pairs, flows, images, workspace, workspace_bytes, stream, nullptr,
                         &T);
    if (rc) return rc;
    cudaEventRecord(e0, st);
    for (int k = 0; k < reps && !rc; ++k)
        rc = render_impl(batch, pairs, pairs_dev, n_pairs, flows, images, workspace, workspace_bytes, stream, nullptr,
                         &T);
    cudaEventRecord(e1, st);
    if (rc) return rc;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
        return fail(SYNTHPIX_ECUDA, "autotune: event timing failed");
    *ms /= (float)reps;
    return SYNTHPIX_OK;
}

extern "C" {

int synthpix_render_pairs(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                          const synthpix_pair_desc *pairs_dev, int32_t n_pairs, const float *flows, void *images,
                          void *workspace, size_t workspace_bytes, void *stream) {
    return render_impl(batch, pairs, pairs_dev, n_pairs, flows, images, workspace, workspace_bytes, stream, nullptr);
}

int synthpix_autotune_tile(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                           const synthpix_pair_desc *pairs_dev, int32_t n_pairs, const float *flows, void *images,
                           void *workspace, size_t workspace_bytes, void *stream, int32_t reps, int32_t *best_tile,
                           float *best_ms) {
    if (!batch || !best_tile) return fail(SYNTHPIX_EINVAL, "batch and best_tile must not be NULL");
    if (reps < 1 || reps > 1000) return fail(SYNTHPIX_EINVAL, "reps %d outside 1..1000", reps);
    Plan P;
    int rc = make_plan(batch, pairs, n_pairs, P);
    if (rc) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail(SYNTHPIX_ECUDA, "autotune: cudaEventCreate failed");
    }
    float best = -1.0f;
    int best_t = 0;
    for (int t : kTileCandidates) {
        float ms = 0.0f;
        rc = time_renders(batch, pairs, pairs_dev, n_pairs, flows, images, workspace, workspace_bytes, stream, reps,
                          default_tuning(uniform_rule(t)), e0, e1, &ms);
        if (rc == SYNTHPIX_EUNSUPPORTED) {  // this edge does not fit the blur radius on chip: try the others
            rc = SYNTHPIX_OK;
            continue;
        }
        if (rc) break;
        if (best < 0.0f || ms < best) {
            best = ms;
            best_t = t;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (best < 0.0f) return fail(SYNTHPIX_EUNSUPPORTED, "autotune: no tile edge fits the batch's blur radius on chip");
    *best_tile = best_t;
    if (best_ms) *best_ms = best;
    g_err[0] = 0;
    return SYNTHPIX_OK;
}

static void to_public(const Tuning &T, const ClassInfo &c, float ms, synthpix_tuning *out) {
    for (int k = 0; k < spx::kSizeClasses; ++k) out->tile[k] = c.present[k] ? T.rule.edge[k] : 0;
    out->records_per_stage = spx::rec_cap(T.rec_buf);
    out->register_epilogue = T.reg_epi;
    out->ms = ms;
    out->reserved[0] = out->reserved[1] = 0;
}

int synthpix_autotune(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                      const synthpix_pair_desc *pairs_dev, int32_t n_pairs, const float *flows, void *images,
                      void *workspace, size_t workspace_bytes, void *stream, int32_t reps, synthpix_tuning *out) {
    if (!batch) return fail(SYNTHPIX_EINVAL, "batch is NULL");
    if (batch->tile != 0) return fail(SYNTHPIX_EINVAL, "autotune needs batch->tile = 0");
    if (reps < 1 || reps > 1000) return fail(SYNTHPIX_EINVAL, "reps %d outside 1..1000", reps);
    Plan P;
    int rc = make_plan(batch, pairs, n_pairs, P);
    if (rc) return rc;
    if (n_pairs == 0) return fail(SYNTHPIX_EINVAL, "autotune needs at least one pair");
    const ClassInfo c = batch_classes(batch, pairs, n_pairs);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail(SYNTHPIX_ECUDA, "autotune: cudaEventCreate failed");
    }
    // coordinate descent from the defaults: each class's edge (largest class
    // first), then the records per stage, then the epilogue variant
    Tuning best = default_tuning(kDefaultRule);
    float best_ms = -1.0f;
    auto trial = [&](Tuning T) -> int {
        float ms = 0.0f;
        const int r = time_renders(batch, pairs, pairs_dev, n_pairs, flows, images, workspace, workspace_bytes,
                                   stream, reps, T, e0, e1, &ms);
        if (r == SYNTHPIX_EUNSUPPORTED) return SYNTHPIX_OK;  // does not fit on chip: not a candidate
        if (r) return r;
        if (best_ms < 0.0f || ms < best_ms) {
            best_ms = ms;
            best = T;
        }
        return SYNTHPIX_OK;
    };
    int order[spx::kSizeClasses], n_order = 0;
    order[n_order++] = c.largest;
    for (int k = spx::kSizeClasses - 1; k >= 0; --k)
        if (c.present[k] && k != c.largest) order[n_order++] = k;
    rc = trial(best);
    for (int q = 0; q < n_order && !rc; ++q) {
        const Tuning base = best;
        for (int t : kTileCandidates) {
            if (t == base.rule.edge[order[q]]) continue;
            Tuning T = base;
            T.rule.edge[order[q]] = t;
            rc = trial(T);
            if (rc) break;
        }
    }
    if (!rc) {
        const Tuning base = best;
        for (int rb : kRecBufCandidates) {
            Plan Q;
            if (make_plan_tuned(batch, pairs, n_pairs, base, Q) != SYNTHPIX_OK) break;
            if (rb == Q.T.rec_buf) continue;
            Tuning T = base;
            T.rec_buf = rb;
            rc = trial(T);
            if (rc) break;
        }
    }
    if (!rc) {
        Tuning T = best;
        T.reg_epi = 1 - best.reg_epi;
        rc = trial(T);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if (best_ms < 0.0f) return fail(SYNTHPIX_EUNSUPPORTED, "autotune: no tuning fits the batch on chip");
    {
        Plan Q;
        if (make_plan_tuned(batch, pairs, n_pairs, best, Q) == SYNTHPIX_OK) best.rec_buf = Q.T.rec_buf;
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (int k = 0; k < spx::kSizeClasses; ++k)
            if (c.present[k]) g_tune[c.key[k]] = TuneEntry{best.rule.edge[k], best.rec_buf, best.reg_epi};
    }
    if (out) to_public(best, c, best_ms, out);
    g_err[0] = 0;
    return SYNTHPIX_OK;
}

int synthpix_tuning_lookup(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs, int32_t n_pairs,
                           synthpix_tuning *out) {
    if (!out) return fail(SYNTHPIX_EINVAL, "out is NULL");
    Plan P;
    const int rc = make_plan(batch, pairs, n_pairs, P);
    if (rc) return rc;
    to_public(P.T, batch_classes(batch, pairs, n_pairs), 0.0f, out);
    g_err[0] = 0;
    return SYNTHPIX_OK;
}

int synthpix_tuning_set(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs, int32_t n_pairs,
                        const synthpix_tuning *t) {
    if (!t) return fail(SYNTHPIX_EINVAL, "tuning is NULL");
    if (!batch) return fail(SYNTHPIX_EINVAL, "batch is NULL");
    if (batch->tile != 0) return fail(SYNTHPIX_EINVAL, "the table serves batches with tile = 0");
    int rc = check_counts(batch, pairs, n_pairs);
    if (rc) return rc;
    if (t->register_epilogue != 0 && t->register_epilogue != 1)
        return fail(SYNTHPIX_EINVAL, "register_epilogue must be 0 or 1");
    if (t->records_per_stage < 1 || t->records_per_stage > 4096)
        return fail(SYNTHPIX_EINVAL, "records_per_stage %d outside 1..4096", t->records_per_stage);
    const ClassInfo c = batch_classes(batch, pairs, n_pairs);
    Tuning T = default_tuning(kDefaultRule);
    for (int k = 0; k < spx::kSizeClasses; ++k) {
        if (!c.present[k]) continue;
        const int e = t->tile[k];
        if (e != 16 && e != 32 && e != 64 && e != 128)
            return fail(SYNTHPIX_EINVAL, "tile[%d] = %d is not 16, 32, 64 or 128", k, e);
        T.rule.edge[k] = e;
    }
    // the staged-record region that holds records_per_stage 24-byte records
    T.rec_buf = (32 + 24 * t->records_per_stage + 15) & ~15;
    T.reg_epi = t->register_epilogue;
    Plan P;
    rc = make_plan_tuned(batch, pairs, n_pairs, T, P);  // validates the buffer against the largest edge
    if (rc) return rc;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    for (int k = 0; k < spx::kSizeClasses; ++k)
        if (c.present[k]) g_tune[c.key[k]] = TuneEntry{T.rule.edge[k], T.rec_buf, T.reg_epi};
    g_err[0] = 0;
    return SYNTHPIX_OK;
}

void synthpix_tuning_clear(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune.clear();
}

int synthpix_render_pairs_from(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                               const synthpix_pair_desc *pairs_dev, int32_t n_pairs, const float *particles_in,
                               const float *flows, void *images, void *workspace, size_t workspace_bytes,
                               void *stream) {
    Extra x;
    x.particles_in = particles_in;
    return run(Mode::Render, batch, pairs, pairs_dev, n_pairs, flows, images, workspace, workspace_bytes, stream,
               nullptr, x);
}

int synthpix_seed_particles(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                            const synthpix_pair_desc *pairs_dev, int32_t n_pairs, float *particles_out,
                            void *workspace, size_t workspace_bytes, void *stream) {
    Extra x;
    x.particles_out = particles_out;
    return run(Mode::Seed, batch, pairs, pairs_dev, n_pairs, nullptr, nullptr, workspace, workspace_bytes, stream,
               nullptr, x);
}

int synthpix_advect_particles(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                              const synthpix_pair_desc *pairs_dev, int32_t n_pairs, const float *particles_in,
                              const float *flows, float *particles_out, void *workspace, size_t workspace_bytes,
                              void *stream) {
    Extra x;
    x.particles_in = particles_in;
    x.particles_out = particles_out;
    return run(Mode::Advect, batch, pairs, pairs_dev, n_pairs, flows, nullptr, workspace, workspace_bytes, stream,
               nullptr, x);
}

int synthpix_render_backward(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                             const synthpix_pair_desc *pairs_dev, int32_t n_pairs, const float *particles_in,
                             const float *flows, const float *grad_images, float *grad_flows, float *grad_particles,
                             void *workspace, size_t workspace_bytes, void *stream) {
    Extra x;
    x.particles_in = particles_in;
    x.grad_images = grad_images;
    x.grad_flows = grad_flows;
    x.grad_particles = grad_particles;
    return run(Mode::Backward, batch, pairs, pairs_dev, n_pairs, flows, nullptr, workspace, workspace_bytes, stream,
               nullptr, x);
}

int synthpix_render_pairs_staged(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                                 const synthpix_pair_desc *pairs_dev, int32_t n_pairs, const float *flows,
                                 void *images, void *workspace, size_t workspace_bytes, void *stream,
                                 void *const *stage_events) {
    return render_impl(batch, pairs, pairs_dev, n_pairs, flows, images, workspace, workspace_bytes, stream,
                       reinterpret_cast<cudaEvent_t const *>(stage_events));
}

}  // extern "C"

namespace spx {

// Sets the thread's last-error message (used by entry points in other files).
int set_error(int code, const char *msg) {
    snprintf(g_err, sizeof(g_err), "%s", msg);
    return code;
}

// Workspace bytes of the plan synthpix_render_pairs runs for this batch, with
// the tile edge it resolves (batch->tile, or the default edge for 0), in
// *need; SYNTHPIX_OK, or the plan's error status with its message set.
int render_workspace_need(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs, int32_t n_pairs,
                          size_t *need) {
    Plan P;
    const int rc = make_plan(batch, pairs, n_pairs, P);
    if (rc) return rc;
    *need = n_pairs > 0 ? P.L.total : 0;
    return SYNTHPIX_OK;
}

}  // namespace spx

namespace spx {

// synthpix_render_pairs with its kernels launched one by one: no CUDA graph
// is instantiated (which may allocate), for callers that cannot have the
// library allocate device memory.
int render_pairs_direct(const synthpix_batch_desc *batch, const synthpix_pair_desc *pairs,
                        const synthpix_pair_desc *pairs_dev, int32_t n_pairs, const float *flows, void *images,
                        void *workspace, size_t workspace_bytes, void *stream) {
    t_direct = true;
    const int rc =
        synthpix_render_pairs(batch, pairs, pairs_dev, n_pairs, flows, images, workspace, workspace_bytes, stream);
    t_direct = false;
    return rc;
}

}  // namespace spx
