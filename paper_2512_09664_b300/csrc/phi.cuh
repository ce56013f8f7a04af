// The tabulated normal tail and the pixel edge values and masses of Eq. 1
// integrated over a pixel (shared by the splat and its adjoint), with the
// 32-bit shared-memory access helpers they use.
#pragma once

#include <cstdint>

#include "phi_table.cuh"

namespace spx {

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: float-to-integer rounding by one addition
constexpr int32_t kMagicBits = 0x4B400000;

// ---------------------------------------------------------------------------
// shared-memory accesses by 32-bit .shared addresses: immediate offsets fold
// into the instruction and no access needs generic-address handling
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t sh_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
template <int OFF>
__device__ __forceinline__ void sh_red_add(uint32_t a, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0+%2], %1;" ::"r"(a), "r"(v), "n"(OFF));
}
__device__ __forceinline__ uint32_t sh_atom_add(uint32_t a, uint32_t v) {
    uint32_t old;
    asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(a), "r"(v));
    return old;
}
// a read of data that stays constant while the kernel runs (the tail table)
__device__ __forceinline__ float4 sh_ld_const4(uint32_t a) {
    float4 v;
    asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}

// ---------------------------------------------------------------------------
// pixel integration of Eq. 1
// ---------------------------------------------------------------------------
// Upper normal tail Q(a) = erfc(a / sqrt 2) / 2 for a >= 0 from the cubic
// table (one float4 per piece, staged in shared memory at .shared address
// tab).  a is clamped to the table's end (Q(8) = 6e-16); the piece is
// k = rint(16 a), so s = a - k / 16 is exact and |s| <= 1/32.
__device__ __forceinline__ float phi_tail(float a, uint32_t tab) {
    a = fminf(a, kPhiTMax);
    const float kf = fmaf(a, kPhiPerUnit, kMagic);
    const int k = __float_as_int(kf) - kMagicBits;
    const float s = fmaf(__fsub_rn(kf, kMagic), -1.0f / kPhiPerUnit, a);
    const float4 c = sh_ld_const4(tab + 16u * (uint32_t)k);
    return fmaf(fmaf(fmaf(c.w, s, c.z), s, c.y), s, c.x);
}

// Edge value of a pixel edge at offset dd = edge - particle centre (pixels):
// the lower tail Phi(t), t = dd / sigma, for dd < 0, and minus the upper tail
// -(1 - Phi(t)) for dd >= +0, so both tails keep their absolute accuracy.
// Q never reaches 0 on the table (Q(8) > 0), so the sign bit of the value
// tells the side of the centre.
__device__ __forceinline__ float edge_value_tab(float dd, float inv, uint32_t tab) {
    const float q = phi_tail(fabsf(__fmul_rn(dd, inv)), tab);
    return __int_as_float(__float_as_int(q) ^ (~__float_as_int(dd) & (int)0x80000000));
}

// Mass of the unit Gaussian between two pixel edges from their edge values:
// Phi(b) - Phi(a) = sb - sa, plus 1 when the centre lies between them (sa on
// the lower side, sb on the upper side).
__device__ __forceinline__ float edge_mass(float sa, float sb) {
    const int across = (__float_as_int(sb) & ~__float_as_int(sa)) >> 31;  // -1 or 0
    return fmaxf(__fadd_rn(__fsub_rn(sb, sa), __int_as_float(across & 0x3F800000)), 0.0f);
}

}  // namespace spx
