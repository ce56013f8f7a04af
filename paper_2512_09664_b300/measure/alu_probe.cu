// Throughput probes of the arithmetic the render is built from, for the
// ALU term of its roofline: FP32 FMA (the pixel-mass products and the blur),
// erfcf (the pixel edge values of Eq. 1), the SFU base-2 exponential and the
// 32-bit high multiply of the Philox rounds.  Each thread runs kChains
// independent dependency chains, so the probe measures throughput, not
// latency; the grid is one full wave (up to 2048 threads per SM, as the
// kernel's registers allow).  The caller times a
// launch with CUDA events and divides the operation count it is given.
//
// This is measurement support for the benchmark, built into a library of its
// own (libsynthpix_probe.so); it is no part of the rendering method nor of
// the renderer's C ABI.
#include <algorithm>
#include <cstdint>
#include <cstdio>

#include <cuda_runtime.h>

#include "alu_probe.h"

namespace {

thread_local char g_probe_error[256] = "";

int fail(int code, const char *what) {
    snprintf(g_probe_error, sizeof(g_probe_error), "%s", what);
    return code;
}

constexpr int kProbeThreads = 256;
constexpr int kProbeCtasPerSm = 8;  // 2048 resident threads per SM
constexpr int kChains = 8;
constexpr int kMaxIters = 1 << 16;

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm volatile("ex2.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) k_alu_probe(int32_t iters, float *sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    float x[kChains];
    uint32_t u[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        x[c] = 0.25f + 1e-3f * (float)((t + 7u * c) & 255u);
        u[c] = 0x9E3779B9u * (t + 1u) + 0x85EBCA6Bu * (uint32_t)c;
    }
    for (int32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if (KIND == SYNTHPIX_PROBE_FMA) x[c] = fmaf(x[c], 0.99999988f, 1.0e-7f);
            if (KIND == SYNTHPIX_PROBE_ERFC) x[c] = erfcf(x[c]);
            if (KIND == SYNTHPIX_PROBE_EX2) x[c] = ex2_approx(-x[c]);
            if (KIND == SYNTHPIX_PROBE_UMULHI) u[c] = __umulhi(u[c], 0xD2511F53u) + u[c];
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += KIND == SYNTHPIX_PROBE_UMULHI ? (float)(u[c] >> 8) : x[c];
    sink[t] = s;
}

int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) return -1;
    return sms;
}

int64_t probe_threads() {
    const int sms = sm_count();
    return sms < 0 ? -1 : (int64_t)sms * kProbeCtasPerSm * kProbeThreads;
}

// One full wave of kernel k: the SMs times the CTAs of k resident per SM
// (at most kProbeCtasPerSm; fewer where k's registers allow fewer).
template <typename K>
int64_t wave_ctas(K k) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kProbeThreads, 0) != cudaSuccess || occ <= 0) return -1;
    return (int64_t)sm_count() * std::min(occ, kProbeCtasPerSm);
}

template <int KIND>
int64_t launch_probe(int32_t iters, float *sink, cudaStream_t st) {
    const int64_t ctas = wave_ctas(k_alu_probe<KIND>);
    if (ctas <= 0) return -1;
    k_alu_probe<KIND><<<(unsigned)ctas, kProbeThreads, 0, st>>>(iters, sink);
    return ctas * kProbeThreads;
}

}  // namespace

extern "C" {

int64_t synthpix_alu_probe_threads(void) {
    const int64_t n = probe_threads();
    if (n < 0) {
        fail(SYNTHPIX_PROBE_ECUDA, "alu probe: no current CUDA device");
        return 0;
    }
    return n;
}

int synthpix_alu_probe(int32_t kind, int32_t iters, float *sink, int64_t sink_elems, int64_t *ops, void *stream) {
    if (kind < SYNTHPIX_PROBE_FMA || kind > SYNTHPIX_PROBE_UMULHI) return fail(SYNTHPIX_PROBE_EINVAL, "alu probe: unknown kind");
    if (iters < 1 || iters > kMaxIters) return fail(SYNTHPIX_PROBE_EINVAL, "alu probe: iters outside 1..65536");
    if (!ops) return fail(SYNTHPIX_PROBE_EINVAL, "alu probe: ops is NULL");
    if (!sink || ((uintptr_t)sink & 3)) return fail(SYNTHPIX_PROBE_EINVAL, "alu probe: sink NULL or misaligned");
    const int64_t n = probe_threads();
    if (n <= 0) return fail(SYNTHPIX_PROBE_ECUDA, "alu probe: no current CUDA device");
    if (sink_elems < n) return fail(SYNTHPIX_PROBE_EINVAL, "alu probe: sink smaller than synthpix_alu_probe_threads()");
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int64_t launched = -1;
    switch (kind) {
    case SYNTHPIX_PROBE_FMA: launched = launch_probe<SYNTHPIX_PROBE_FMA>(iters, sink, st); break;
    case SYNTHPIX_PROBE_ERFC: launched = launch_probe<SYNTHPIX_PROBE_ERFC>(iters, sink, st); break;
    case SYNTHPIX_PROBE_EX2: launched = launch_probe<SYNTHPIX_PROBE_EX2>(iters, sink, st); break;
    default: launched = launch_probe<SYNTHPIX_PROBE_UMULHI>(iters, sink, st); break;
    }
    if (launched <= 0) return fail(SYNTHPIX_PROBE_ECUDA, "alu probe: occupancy query failed");
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        char msg[256];
        snprintf(msg, sizeof(msg), "alu probe launch: %s", cudaGetErrorString(e));
        return fail(SYNTHPIX_PROBE_ECUDA, msg);
    }
    *ops = launched * (int64_t)iters * kChains;
    g_probe_error[0] = 0;
    return 0;
}

const char *synthpix_probe_last_error(void) { return g_probe_error; }

}  // extern "C"
