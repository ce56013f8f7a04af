/*
 * ALU throughput probes: measurement support for the benchmark's roofline
 * (the ALU term of the render), in a library of its own,
 * libsynthpix_probe.so.  No part of the rendering method or of the
 * renderer's C ABI (include/synthpix.h).
 *
 *   SYNTHPIX_PROBE_FMA     FP32 fused multiply-add
 *   SYNTHPIX_PROBE_ERFC    erfcf(), the pixel edge values of Eq. 1 in closed form
 *   SYNTHPIX_PROBE_EX2     the SFU base-2 exponential (ex2.approx.f32)
 *   SYNTHPIX_PROBE_UMULHI  32 x 32 -> high 32 multiply plus an add, as in the
 *                          Philox rounds that draw particles and noise
 *
 * synthpix_alu_probe_threads() is the probe's thread count on the current
 * device (8 CTAs of 256 threads per SM), 0 with an error message if there is
 * no device.  synthpix_alu_probe launches one full wave of CTAs (as many per
 * SM as the kind's kernel fits, at most 8) in which every thread runs 8
 * independent chains of `iters` operations of `kind` (iters 1..65536) and
 * writes one float to sink; *ops (host) receives the number of operations
 * the launch performs.  The caller times the launch with CUDA events on
 * `stream` (a cudaStream_t, NULL for the legacy stream) and divides.
 *   sink  device, 4-byte aligned, at least synthpix_alu_probe_threads()
 *         floats (values are meaningless; they keep the work alive).
 * Returns 0, or SYNTHPIX_PROBE_EINVAL for invalid arguments (before anything
 * is launched), SYNTHPIX_PROBE_ECUDA for a CUDA error; the message is in
 * synthpix_probe_last_error() (thread-local).
 */
#ifndef SYNTHPIX_ALU_PROBE_H
#define SYNTHPIX_ALU_PROBE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SYNTHPIX_PROBE_FMA 0
#define SYNTHPIX_PROBE_ERFC 1
#define SYNTHPIX_PROBE_EX2 2
#define SYNTHPIX_PROBE_UMULHI 3
#define SYNTHPIX_PROBE_EINVAL (-1)
#define SYNTHPIX_PROBE_ECUDA (-3)

int64_t synthpix_alu_probe_threads(void);
int synthpix_alu_probe(int32_t kind, int32_t iters, float *sink, int64_t sink_elems, int64_t *ops, void *stream);
const char *synthpix_probe_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SYNTHPIX_ALU_PROBE_H */
