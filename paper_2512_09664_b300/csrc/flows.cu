// Procedural flow fields on the device for streaming renders (paper Section
// 2, "Data loaders": flow fields may be supplied procedurally).  Each field
// is the curl of a stream function psi = sum_m a_m sin(k_m . x + phi_m)
// sampled at the cell-centred nodes of the flow grid: u = d psi / dy =
// sum_m a_m ky_m cos(arg_m), v = -d psi / dx = -sum_m a_m kx_m cos(arg_m),
// then scaled to a target RMS speed.
//
//   k_flow_tables  cos / sin of kx x_l + phi (per grid column) and of ky y_k
//                  (per grid row) for every mode: the angle formed and reduced
//                  to [-pi, pi] in FP64, its cos / sin in FP32
//   k_flow_sum     cos(a + b) = cos a cos b - sin a sin b summed over the
//                  modes per node (FP32 FMAs on tables staged in shared
//                  memory, 2 rows x 4 columns of nodes per thread); per-field
//                  sum of u^2 + v^2 in FP64
//   k_flow_scale   multiply each field by rms / sqrt(mean(u^2 + v^2))
#include <cmath>
#include <cstdio>

#include "synthpix.h"

namespace spx {
void count_launch();  // api.cu: the library's launch counter
}

namespace spx {
int set_error(int code, const char *msg);
}

namespace {

constexpr int kMaxModes = 256;
constexpr int kSumThreads = 256;            // k_flow_sum: 32 lanes x 8 warps
constexpr int kColsPer = 4, kRowsPer = 2;   // nodes per thread
constexpr int kTileX = 32 * kColsPer;       // 128 columns per block
constexpr int kTileY = 8 * kRowsPer;        // 16 rows per block
constexpr int kModeChunk = 32;              // modes staged per pass

struct FlowTables {
    float *cx, *sx;  // [n_flows][M][gw]
    float *cy, *sy;  // [n_flows][M][gh]
    double *ss;      // [n_flows] sum of u^2 + v^2
};

size_t tables_bytes(int n_flows, int n_modes, int gh, int gw) {
    const size_t col = (size_t)n_flows * gw * n_modes * sizeof(float);
    const size_t row = (size_t)n_flows * gh * n_modes * sizeof(float);
    return 2 * col + 2 * row + (size_t)n_flows * sizeof(double) + 5 * 256;
}

FlowTables carve(void *ws, int n_flows, int n_modes, int gh, int gw) {
    unsigned char *p = static_cast<unsigned char *>(ws);
    auto take = [&](size_t bytes) {
        unsigned char *at = p;
        p += (bytes + 255) & ~(size_t)255;
        return at;
    };
    FlowTables t;
    t.cx = reinterpret_cast<float *>(take((size_t)n_flows * gw * n_modes * sizeof(float)));
    t.sx = reinterpret_cast<float *>(take((size_t)n_flows * gw * n_modes * sizeof(float)));
    t.cy = reinterpret_cast<float *>(take((size_t)n_flows * gh * n_modes * sizeof(float)));
    t.sy = reinterpret_cast<float *>(take((size_t)n_flows * gh * n_modes * sizeof(float)));
    t.ss = reinterpret_cast<double *>(take((size_t)n_flows * sizeof(double)));
    return t;
}

// sin and cos of an angle given in FP64: reduced to r in [-pi, pi] in FP64
// (exact to ~1e-13 for the angles here, |a| < 1e6), then evaluated in FP32
// (abs error ~1e-7, the precision the tables are stored in).
__device__ __forceinline__ void sincos_reduced(double a, float *s, float *c) {
    const double n = rint(a * 0.15915494309189533577);          // a / (2 pi)
    const double r = fma(-n, 6.2831853071795864769, a);
    sincosf((float)r, s, c);
}

// Thread per (grid column or row, mode) of field blockIdx.y.  Node l of a
// grid of gw columns over an image of width W sits at x = (l + 1/2) dx with
// dx = W / gw (and likewise y; dx, dy computed on the host: FP64 division
// is slow on this part).
__global__ void k_flow_tables(const double *__restrict__ modes, int n_modes, int gh, int gw, double dx, double dy,
                              FlowTables t) {
    const int f = blockIdx.y;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx == 0) t.ss[f] = 0.0;
    const int ncol = gw * n_modes, nrow = gh * n_modes;
    if (idx >= ncol + nrow) return;
    const double *md = modes + (size_t)f * n_modes * 4;
    float s, c;
    if (idx < ncol) {  // mode-major: consecutive threads take consecutive columns
        const int m = idx / gw, l = idx - m * gw;
        const double x = ((double)l + 0.5) * dx;
        sincos_reduced(md[4 * m] * x + md[4 * m + 2], &s, &c);
        const size_t o = ((size_t)f * n_modes + m) * gw + l;
        t.cx[o] = c;
        t.sx[o] = s;
    } else {
        const int r = idx - ncol;
        const int m = r / gh, k = r - m * gh;
        const double y = ((double)k + 0.5) * dy;
        sincos_reduced(md[4 * m + 1] * y, &s, &c);
        const size_t o = ((size_t)f * n_modes + m) * gh + k;
        t.cy[o] = c;
        t.sy[o] = s;
    }
}

// Block of kTileX x kTileY nodes of field blockIdx.z: lane x of warp w
// computes columns 4x .. 4x + 3 of rows 2w, 2w + 1.  The tables of the
// block's columns and rows and the mode weights are staged in shared memory
// kModeChunk modes at a time; per mode a thread reads its four columns' cos
// and sin as two float4 and its two rows' values as broadcasts.
__global__ void __launch_bounds__(kSumThreads) k_flow_sum(const double *__restrict__ modes, int n_modes, int gh,
                                                          int gw, FlowTables t, float2 *__restrict__ out) {
    __shared__ __align__(16) float s_cx[kModeChunk][kTileX], s_sx[kModeChunk][kTileX];
    __shared__ float s_cy[kModeChunk][kTileY], s_sy[kModeChunk][kTileY];
    __shared__ float s_wu[kModeChunk], s_wv[kModeChunk];
    __shared__ double s_red[kSumThreads / 32];
    const int f = blockIdx.z;
    const int l0 = blockIdx.x * kTileX, k0 = blockIdx.y * kTileY;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const double *md = modes + (size_t)f * n_modes * 4;
    float u[kRowsPer][kColsPer] = {}, v[kRowsPer][kColsPer] = {};
    for (int m0 = 0; m0 < n_modes; m0 += kModeChunk) {
        const int mc = min(kModeChunk, n_modes - m0);
        __syncthreads();
        for (int i = threadIdx.x; i < kModeChunk * kTileX; i += kSumThreads) {
            const int m = i / kTileX, c = i % kTileX;
            const int lc = min(l0 + c, gw - 1);
            const size_t o = ((size_t)f * n_modes + m0 + min(m, mc - 1)) * gw + lc;
            s_cx[m][c] = m < mc ? t.cx[o] : 0.0f;
            s_sx[m][c] = m < mc ? t.sx[o] : 0.0f;
        }
        for (int i = threadIdx.x; i < kModeChunk * kTileY; i += kSumThreads) {
            const int m = i / kTileY, r = i % kTileY;
            const int kr = min(k0 + r, gh - 1);
            const size_t o = ((size_t)f * n_modes + m0 + min(m, mc - 1)) * gh + kr;
            s_cy[m][r] = m < mc ? t.cy[o] : 0.0f;
            s_sy[m][r] = m < mc ? t.sy[o] : 0.0f;
        }
        for (int m = threadIdx.x; m < kModeChunk; m += kSumThreads) {
            const double a = m < mc ? md[4 * (m0 + m) + 3] : 0.0;
            s_wu[m] = m < mc ? (float)(a * md[4 * (m0 + m) + 1]) : 0.0f;   //  a ky
            s_wv[m] = m < mc ? (float)(-a * md[4 * (m0 + m)]) : 0.0f;      // -a kx
        }
        __syncthreads();
#pragma unroll 4
        for (int m = 0; m < kModeChunk; ++m) {
            const float4 cx = *reinterpret_cast<const float4 *>(&s_cx[m][kColsPer * lane]);
            const float4 sx = *reinterpret_cast<const float4 *>(&s_sx[m][kColsPer * lane]);
            const float cxa[kColsPer] = {cx.x, cx.y, cx.z, cx.w}, sxa[kColsPer] = {sx.x, sx.y, sx.z, sx.w};
            const float wu = s_wu[m], wv = s_wv[m];
#pragma unroll
            for (int r = 0; r < kRowsPer; ++r) {
                const float cy = s_cy[m][kRowsPer * warp + r], sy = s_sy[m][kRowsPer * warp + r];
#pragma unroll
                for (int c = 0; c < kColsPer; ++c) {
                    const float cm = fmaf(cy, cxa[c], -sy * sxa[c]);  // cos(arg_m)
                    u[r][c] = fmaf(wu, cm, u[r][c]);
                    v[r][c] = fmaf(wv, cm, v[r][c]);
                }
            }
        }
    }
    float ef = 0.0f;  // this thread's 8 nodes in FP32, the block's sum in FP64 (FP64 is slow here)
#pragma unroll
    for (int r = 0; r < kRowsPer; ++r) {
        const int k = k0 + kRowsPer * warp + r;
#pragma unroll
        for (int c = 0; c < kColsPer; ++c) {
            const int l = l0 + kColsPer * lane + c;
            if (l < gw && k < gh) {
                out[((size_t)f * gh + k) * gw + l] = make_float2(u[r][c], v[r][c]);
                ef = fmaf(u[r][c], u[r][c], fmaf(v[r][c], v[r][c], ef));
            }
        }
    }
    double e = (double)ef;
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if (lane == 0) s_red[warp] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < kSumThreads / 32; ++w) sum += s_red[w];
        atomicAdd(t.ss + f, sum);
    }
}

// The field's scale is computed once per block (FP64 division and square
// root are slow on this part).
__global__ void k_flow_scale(int gh, int gw, float rms, const double *__restrict__ ss, float2 *__restrict__ out) {
    __shared__ float s_scale;
    const int f = blockIdx.y;
    const int64_t n = (int64_t)gh * gw;
    if (threadIdx.x == 0) {
        const double mean = ss[f] / (double)n;
        s_scale = mean > 0.0 ? (float)((double)rms / sqrt(mean)) : 0.0f;
    }
    __syncthreads();
    const float scale = s_scale;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float2 *p = out + (size_t)f * n + i;
        const float2 w = *p;
        *p = make_float2(w.x * scale, w.y * scale);
    }
}

int fail(int code, const char *what) { return spx::set_error(code, what); }

bool valid_sizes(int n_flows, int n_modes, int gh, int gw, int H, int W) {
    return n_flows >= 1 && n_flows <= 65535 && n_modes >= 1 && n_modes <= kMaxModes && gh >= 1 && gh <= 32768 &&
           gw >= 1 && gw <= 32768 && H >= 1 && H <= 32768 && W >= 1 && W <= 32768;
}

}  // namespace

extern "C" {

size_t synthpix_fourier_flows_workspace_bytes(int32_t n_flows, int32_t n_modes, int32_t flow_h, int32_t flow_w) {
    if (!valid_sizes(n_flows, n_modes, flow_h, flow_w, 1, 1)) {
        fail(SYNTHPIX_EINVAL, "fourier flows: n_flows 1..65535, n_modes 1..256, grid 1..32768 per side");
        return 0;
    }
    return tables_bytes(n_flows, n_modes, flow_h, flow_w);
}

int synthpix_fourier_flows(int32_t n_flows, int32_t n_modes, int32_t flow_h, int32_t flow_w, int32_t height,
                           int32_t width, const double *modes, float rms, float *flows, void *workspace,
                           size_t workspace_bytes, void *stream) {
    if (!valid_sizes(n_flows, n_modes, flow_h, flow_w, height, width))
        return fail(SYNTHPIX_EINVAL, "fourier flows: n_flows 1..65535, n_modes 1..256, sizes 1..32768");
    if (!modes || ((uintptr_t)modes & 7)) return fail(SYNTHPIX_EINVAL, "fourier flows: modes NULL or misaligned");
    if (!flows || ((uintptr_t)flows & 7)) return fail(SYNTHPIX_EINVAL, "fourier flows: flows NULL or misaligned");
    if (!(rms >= 0.0f) || !std::isfinite(rms)) return fail(SYNTHPIX_EINVAL, "fourier flows: rms must be >= 0");
    if (!workspace || ((uintptr_t)workspace & 255))
        return fail(SYNTHPIX_EWORKSPACE, "fourier flows: workspace NULL or not 256-byte aligned");
    if (workspace_bytes < tables_bytes(n_flows, n_modes, flow_h, flow_w))
        return fail(SYNTHPIX_EWORKSPACE, "fourier flows: workspace too small");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const FlowTables t = carve(workspace, n_flows, n_modes, flow_h, flow_w);
    const int64_t per_field = ((int64_t)flow_w + flow_h) * n_modes;
    dim3 g1((unsigned)((per_field + 255) / 256), (unsigned)n_flows);
    k_flow_tables<<<g1, 256, 0, st>>>(modes, n_modes, flow_h, flow_w, (double)width / (double)flow_w,
                                      (double)height / (double)flow_h, t);
    dim3 g2((unsigned)((flow_w + kTileX - 1) / kTileX), (unsigned)((flow_h + kTileY - 1) / kTileY), (unsigned)n_flows);
    float2 *out = reinterpret_cast<float2 *>(flows);
    k_flow_sum<<<g2, kSumThreads, 0, st>>>(modes, n_modes, flow_h, flow_w, t, out);
    if (rms > 0.0f) {
        dim3 g3((unsigned)std::min<int64_t>(((int64_t)flow_h * flow_w + 255) / 256, 1024), (unsigned)n_flows);
        k_flow_scale<<<g3, 256, 0, st>>>(flow_h, flow_w, rms, t.ss, out);
    }
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        for (int k = 0; k < (rms > 0.0f ? 3 : 2); ++k) spx::count_launch();
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof(msg), "fourier flows launch: %s", cudaGetErrorString(e));
        return fail(SYNTHPIX_ECUDA, msg);
    }
    return spx::set_error(SYNTHPIX_OK, "");
}

}  // extern "C"
