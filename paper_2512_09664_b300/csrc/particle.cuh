// Device functions shared by the forward kernels (prep.cu) and the adjoint
// (adjoint.cu): particle attributes from the Philox streams, the bilinear
// flow and the RK4 / Euler advection on split coordinates.
#pragma once

#include "common.cuh"
#include "kernels.cuh"

namespace spx {

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

// The same search by a whole block, for a key common to the block: thread
// t tests the bases m = t, t + blockDim, ... with independent loads (one
// memory round trip instead of log2(n) dependent ones); the one m with
// base(m) <= key < base(m + 1) is the answer.  Ends with a barrier.
template <typename F>
__device__ __forceinline__ int block_upper_find(int n, int64_t key, F base) {
    __shared__ int s_found;
    for (int m = threadIdx.x; m < n; m += blockDim.x) {
        const int64_t b0 = base(m);
        const int64_t b1 = m + 1 < n ? base(m + 1) : INT64_MAX;
        if (b0 <= key && key < b1) s_found = m;
    }
    __syncthreads();
    return s_found;
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

// velocity() with the four nodes of the last grid cell (l, k) kept in
// registers: consecutive RK4 stages mostly sample the same cell (the third
// stage that of the second, a substep's first that of the previous fourth),
// and a lane reloads the nodes from the grid only when its cell changes.
// Same nodes, same arithmetic: the result is identical.
struct GridVelocity {
    const Flow &F;
    int32_t cl, ck;  // the cached cell (l, k) before clamping; cl = INT32_MIN: none
    float2 a, b, c, d;
    __device__ explicit GridVelocity(const Flow &f) : F(f), cl(INT32_MIN), ck(0) {}
    __device__ __forceinline__ float2 operator()(int32_t ix, float fx, int32_t iy, float fy) {
        int32_t l, k;
        float tx, ty;
        grid_coord(ix, fx, F.gw, F.W, l, tx);
        grid_coord(iy, fy, F.gh, F.H, k, ty);
        if (l != cl || k != ck) {
            cl = l;
            ck = k;
            const int32_t l0 = min(max(l, 0), F.gw - 1), l1 = min(max(l + 1, 0), F.gw - 1);
            const int32_t k0 = min(max(k, 0), F.gh - 1), k1 = min(max(k + 1, 0), F.gh - 1);
            a = __ldg(F.f + (size_t)k0 * F.gw + l0);
            b = __ldg(F.f + (size_t)k0 * F.gw + l1);
            c = __ldg(F.f + (size_t)k1 * F.gw + l0);
            d = __ldg(F.f + (size_t)k1 * F.gw + l1);
        }
        const float tu = fmaf(tx, b.x - a.x, a.x), tv = fmaf(tx, b.y - a.y, a.y);
        const float bu = fmaf(tx, d.x - c.x, c.x), bv = fmaf(tx, d.y - c.y, c.y);
        return make_float2(fmaf(ty, bu - tu, tu), fmaf(ty, bv - tv, tv));
    }
};

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

// The same with half-extents r15x = 1.5 d along x and r15y = 1.5 d_y along y.
__device__ __forceinline__ Window particle_window2(int32_t ix, float fx, int32_t iy, float fy, float r15x,
                                                   float r15y, int32_t W, int32_t H) {
    Window w;
    w.j0 = max(ix + (int32_t)floorf(fx - r15x), 0);
    w.j1 = min(ix + (int32_t)floorf(fx + r15x), W - 1);
    w.i0 = max(iy + (int32_t)floorf(fy - r15y), 0);
    w.i1 = min(iy + (int32_t)floorf(fy + r15y), H - 1);
    return w;
}

// Tiles whose halo-widened rectangle meets the window.
__device__ __forceinline__ void window_tiles(const Window &w, int32_t halo, int32_t tile, int32_t W, int32_t H,
                                             int32_t &tx0, int32_t &tx1, int32_t &ty0, int32_t &ty1) {
    const int sh = __ffs(tile) - 1;  // tile edges are powers of two; the coordinates are non-negative
    tx0 = max(w.j0 - halo, 0) >> sh;
    tx1 = min(w.j1 + halo, W - 1) >> sh;
    ty0 = max(w.i0 - halo, 0) >> sh;
    ty1 = min(w.i1 + halo, H - 1) >> sh;
}


// ---------------------------------------------------------------------------
// pixel integration of Eq. 1 (separable erf differences)
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

// A particle of frame 1: split position, sigma = d / 4, amplitude Ieff 2 pi sigma^2;
// d, I0, the out-of-plane position z and its sheet gain for the per-frame shapes.
struct Seeded {
    int32_t ix, iy;
    float fx, fy;
    float sigma, amp;
    float d, i0, z, gain;
};

// Intensity factor at out-of-plane position z: the Gaussian sheet
// exp(-z^2 / (2 s^2)), or the out-of-focus form of the Remark
// exp(-|2 z^2 / dz0^2|^shape / sqrt(2 pi)) with dz0 = sheet_sigma.
__device__ __forceinline__ float sheet_gain(const synthpix_pair_desc &D, float z) {
    if (!(D.sheet_sigma > 0.0f)) return 1.0f;
    if (D.sheet_model == SYNTHPIX_SHEET_REMARK) {
        const float q = fabsf(2.0f * z * z / (D.sheet_sigma * D.sheet_sigma));
        return expf(-powf(q, D.sheet_shape) * 0.39894228040143267794f);
    }
    return expf(-(z * z) / (2.0f * D.sheet_sigma * D.sheet_sigma));
}

// Attributes of particle i of a pair (Section 2, "Sampling the particles":
// uniform position over the image, parameters from their intervals; the
// clipped-normal diameter via Box-Muller).  With a.particles_in, position and
// diameter are taken from it (FP32 x0, y0, d of global particle g) instead.
__device__ __forceinline__ Seeded seed_particle(const KernelArgs &a, const synthpix_pair_desc &D, uint32_t i,
                                                int64_t g) {
    Seeded P;
    const int32_t H = D.height, W = D.width;
    const uint4 wa = stream_words(a.keys, D.pair_id, i, kTagAttrA);
    const uint4 wb = stream_words(a.keys, D.pair_id, i, kTagAttrB);
    float d;
    if (a.particles_in) {
        const float x0 = a.particles_in[3 * g], y0 = a.particles_in[3 * g + 1];
        const float fl = floorf(x0), fk = floorf(y0);
        P.ix = (int32_t)fminf(fmaxf(fl, -1.0e9f), 1.0e9f);
        P.iy = (int32_t)fminf(fmaxf(fk, -1.0e9f), 1.0e9f);
        P.fx = x0 - fl;  // exact
        P.fy = y0 - fk;
        d = a.particles_in[3 * g + 2];
    } else {
        const unsigned long long px = (unsigned long long)(wa.x >> 8) * (uint32_t)W;
        const unsigned long long py = (unsigned long long)(wa.y >> 8) * (uint32_t)H;
        P.ix = (int32_t)(px >> 24);
        P.iy = (int32_t)(py >> 24);
        P.fx = (float)(uint32_t)(px & 0xFFFFFFu) * (1.0f / 16777216.0f);  // exact
        P.fy = (float)(uint32_t)(py & 0xFFFFFFu) * (1.0f / 16777216.0f);
        if (D.d_dist == 0) {
            d = fminf(fmaf(u24f(wa.z), D.d_max - D.d_min, D.d_min), D.d_max);
        } else {
            float s, c;
            sincospif(2.0f * u24f(wb.y), &s, &c);
            const float r = sqrtf(-2.0f * logf(uo24f(wa.z)));
            d = fminf(fmaxf(fmaf(D.d_sigma, r * c, D.d_mu), D.d_min), D.d_max);
        }
    }
    const float I0 = fmaf(u24f(wa.w), D.i_max - D.i_min, D.i_min);
    const float z = fmaf(u24f(wb.x), D.z_max - D.z_min, D.z_min);
    const float gain = sheet_gain(D, z);
    P.sigma = 0.25f * d;
    P.amp = (I0 * gain) * (6.28318530717958647692f * P.sigma * P.sigma);  // Ieff * 2 pi sigma^2
    P.d = d;
    P.i0 = I0;
    P.z = z;
    P.gain = gain;
    return P;
}

// Standard normals (cos and sin branches of Box-Muller) from two words.
__device__ __forceinline__ void normal_pair(uint32_t wa, uint32_t wb, float &n0, float &n1) {
    float s, c;
    sincospif(2.0f * u24f(wb), &s, &c);
    const float r = sqrtf(-2.0f * logf(uo24f(wa)));
    n0 = r * c;
    n1 = r * s;
}

__device__ __forceinline__ float clampf(float v, float lo, float hi) { return fminf(fmaxf(v, lo), hi); }

// (sigma_x, sigma_y, rho, Ieff 2 pi sigma_x sigma_y sqrt(1 - rho^2)) of a
// particle in one frame; sigma_x = -1 when it is hidden from the frame.
__device__ __forceinline__ float4 frame_shape(float dx, float dy, float rho, float ieff, bool hidden) {
    const float sx = 0.25f * dx, sy = 0.25f * dy;
    const float amp = ieff * (6.28318530717958647692f * sx * sy * sqrtf(1.0f - rho * rho));
    return make_float4(hidden ? -1.0f : sx, sy, rho, amp);
}

// Frame-1 and frame-2 shapes of particle i (Section 2, text after Eq. 1:
// sigma_x, sigma_y and rho drawn per particle from their intervals; every
// parameter of the second image is the first image's plus a zero-mean
// Gaussian change, clamped to the parameter's interval; aggregation
// paragraph: a particle hidden from each image with probability hide_prob).
// d_y = d when the d_y interval is [0, 0] (then one change for both axes).
// gain2: the sheet factor in frame 2 (P.gain unless the particle moved in z).
__device__ __forceinline__ void frame_shapes(const KernelArgs &a, const synthpix_pair_desc &D, uint32_t i,
                                             const Seeded &P, float gain2, float4 &s1, float4 &s2) {
    const uint4 w2 = stream_words(a.keys, D.pair_id, i, kTagShapeA);
    const uint4 w3 = stream_words(a.keys, D.pair_id, i, kTagShapeB);
    const bool same_d = D.dy_min == 0.0f && D.dy_max == 0.0f;
    const float dy = same_d ? P.d : fminf(fmaf(u24f(w3.x), D.dy_max - D.dy_min, D.dy_min), D.dy_max);
    const float rho = fminf(fmaf(u24f(w3.y), D.rho_max - D.rho_min, D.rho_min), D.rho_max);
    float nd, ni, ndy, nr;
    normal_pair(w2.z, w2.w, nd, ni);
    normal_pair(w3.z, w3.w, ndy, nr);
    const float dx2 = clampf(fmaf(D.jitter_d, nd, P.d), D.d_min, D.d_max);
    const float dy2 = same_d ? dx2 : clampf(fmaf(D.jitter_d, ndy, dy), D.dy_min, D.dy_max);
    const float rho2 = clampf(fmaf(D.jitter_rho, nr, rho), D.rho_min, D.rho_max);
    const float i2 = clampf(fmaf(D.jitter_i, ni, P.i0), D.i_min, D.i_max);
    s1 = frame_shape(P.d, dy, rho, P.i0 * P.gain, u24f(w2.x) < a.hide_prob);
    s2 = frame_shape(dx2, dy2, rho2, i2 * gain2, u24f(w2.y) < a.hide_prob);
}

__device__ __forceinline__ Flow pair_flow(const KernelArgs &a, const synthpix_pair_desc &D) {
    Flow F;
    F.f = reinterpret_cast<const float2 *>(a.flows + D.flow_offset);
    F.gh = D.flow_h;
    F.gw = D.flow_w;
    F.H = D.height;
    F.W = D.width;
    return F;
}

// Frame-2 position: n substeps of RK4 (or Euler) over dt, on split
// coordinates; vel(ix, fx, iy, fy) is the bilinear velocity.
template <typename Vel>
__device__ __forceinline__ void advect_split_with(Vel &&vel, float dt, int n_substeps, int integrator, int32_t &jx,
                                                  float &gx, int32_t &jy, float &gy) {
    const float h = dt / (float)n_substeps;
    const float hh = 0.5f * h, h6 = h / 6.0f;
    for (int s = 0; s < n_substeps; ++s) {
        const float2 k1 = vel(jx, gx, jy, gy);
        if (integrator == SYNTHPIX_EULER) {
            split_add(jx, gx, __fmul_rn(h, k1.x));
            split_add(jy, gy, __fmul_rn(h, k1.y));
            continue;
        }
        const float2 k2 = vel(jx, fmaf(hh, k1.x, gx), jy, fmaf(hh, k1.y, gy));
        const float2 k3 = vel(jx, fmaf(hh, k2.x, gx), jy, fmaf(hh, k2.y, gy));
        const float2 k4 = vel(jx, fmaf(h, k3.x, gx), jy, fmaf(h, k3.y, gy));
        split_add(jx, gx, __fmul_rn(h6, (k1.x + k4.x) + 2.0f * (k2.x + k3.x)));
        split_add(jy, gy, __fmul_rn(h6, (k1.y + k4.y) + 2.0f * (k2.y + k3.y)));
    }
}

__device__ __forceinline__ void advect_split(const Flow &F, float dt, int n_substeps, int integrator, int32_t &jx,
                                             float &gx, int32_t &jy, float &gy) {
    advect_split_with([&](int32_t ix, float fx, int32_t iy, float fy) { return velocity(F, ix, fx, iy, fy); }, dt,
                      n_substeps, integrator, jx, gx, jy, gy);
}

// The scalar grid w (same nodes as the flow) at a split position: the
// bilinear weights of velocity().
__device__ __forceinline__ float scalar_at(const Flow &F, const float *w, int32_t ix, float fx, int32_t iy, float fy) {
    int32_t l, k;
    float tx, ty;
    grid_coord(ix, fx, F.gw, F.W, l, tx);
    grid_coord(iy, fy, F.gh, F.H, k, ty);
    const int32_t l0 = min(max(l, 0), F.gw - 1), l1 = min(max(l + 1, 0), F.gw - 1);
    const int32_t k0 = min(max(k, 0), F.gh - 1), k1 = min(max(k + 1, 0), F.gh - 1);
    const float a = __ldg(w + (size_t)k0 * F.gw + l0), b = __ldg(w + (size_t)k0 * F.gw + l1);
    const float c = __ldg(w + (size_t)k1 * F.gw + l0), d = __ldg(w + (size_t)k1 * F.gw + l1);
    const float t = fmaf(tx, b - a, a), u = fmaf(tx, d - c, c);
    return fmaf(ty, u - t, t);
}

// advect_split with the out-of-plane position z moved by the scalar grid w
// along the path: the same stages (and the same position arithmetic) as
// advect_split_with, each also evaluating w.
__device__ __forceinline__ void advect_split_z(const Flow &F, const float *w, float dt, int n_substeps, int integrator,
                                               int32_t &jx, float &gx, int32_t &jy, float &gy, float &z) {
    const float h = dt / (float)n_substeps;
    const float hh = 0.5f * h, h6 = h / 6.0f;
    for (int s = 0; s < n_substeps; ++s) {
        const float2 k1 = velocity(F, jx, gx, jy, gy);
        const float w1 = scalar_at(F, w, jx, gx, jy, gy);
        if (integrator == SYNTHPIX_EULER) {
            split_add(jx, gx, __fmul_rn(h, k1.x));
            split_add(jy, gy, __fmul_rn(h, k1.y));
            z = fmaf(h, w1, z);
            continue;
        }
        const float x2 = fmaf(hh, k1.x, gx), y2 = fmaf(hh, k1.y, gy);
        const float2 k2 = velocity(F, jx, x2, jy, y2);
        const float w2 = scalar_at(F, w, jx, x2, jy, y2);
        const float x3 = fmaf(hh, k2.x, gx), y3 = fmaf(hh, k2.y, gy);
        const float2 k3 = velocity(F, jx, x3, jy, y3);
        const float w3 = scalar_at(F, w, jx, x3, jy, y3);
        const float x4 = fmaf(h, k3.x, gx), y4 = fmaf(h, k3.y, gy);
        const float2 k4 = velocity(F, jx, x4, jy, y4);
        const float w4 = scalar_at(F, w, jx, x4, jy, y4);
        split_add(jx, gx, __fmul_rn(h6, (k1.x + k4.x) + 2.0f * (k2.x + k3.x)));
        split_add(jy, gy, __fmul_rn(h6, (k1.y + k4.y) + 2.0f * (k2.y + k3.y)));
        z = fmaf(h6, (w1 + w4) + 2.0f * (w2 + w3), z);
    }
}

// A block of flow-grid nodes [gx0, gx0 + nw) x [gy0, gy0 + nh) staged in
// shared memory.  The bilinear velocity reads the four corners from it when
// all lie inside, else from global memory: the same nodes and arithmetic as
// velocity(), so the result is identical.
struct FlowWindow {
    const float2 *s;
    uint32_t sa;  // .shared address of s
    int32_t gx0, gy0, nw, nh;
};

// One node of the staged window by its .shared address (explicit state
// space: no generic-address handling per load).
__device__ __forceinline__ float2 window_node(uint32_t a) {
    float2 v;
    asm("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a));
    return v;
}

__device__ __forceinline__ float2 velocity_windowed(const Flow &F, const FlowWindow &Wn, int32_t ix, float fx,
                                                    int32_t iy, float fy) {
    int32_t l, k;
    float tx, ty;
    grid_coord(ix, fx, F.gw, F.W, l, tx);
    grid_coord(iy, fy, F.gh, F.H, k, ty);
    const int32_t l0 = min(max(l, 0), F.gw - 1), l1 = min(max(l + 1, 0), F.gw - 1);
    const int32_t k0 = min(max(k, 0), F.gh - 1), k1 = min(max(k + 1, 0), F.gh - 1);
    const int32_t u0 = l0 - Wn.gx0, u1 = l1 - Wn.gx0, v0 = k0 - Wn.gy0, v1 = k1 - Wn.gy0;
    const bool in = (unsigned)u0 < (unsigned)Wn.nw && (unsigned)u1 < (unsigned)Wn.nw &&
                    (unsigned)v0 < (unsigned)Wn.nh && (unsigned)v1 < (unsigned)Wn.nh;
    // per-lane generic pointers (shared window or global grid): no divergent branch
    const float2 *r0 = in ? Wn.s + v0 * Wn.nw : F.f + (size_t)k0 * F.gw;
    const float2 *r1 = in ? Wn.s + v1 * Wn.nw : F.f + (size_t)k1 * F.gw;
    const int32_t c0 = in ? u0 : l0, c1 = in ? u1 : l1;
    const float2 a = r0[c0], b = r0[c1], c = r1[c0], d = r1[c1];
    const float tu = fmaf(tx, b.x - a.x, a.x), tv = fmaf(tx, b.y - a.y, a.y);
    const float bu = fmaf(tx, d.x - c.x, c.x), bv = fmaf(tx, d.y - c.y, c.y);
    return make_float2(fmaf(ty, bu - tu, tu), fmaf(ty, bv - tv, tv));
}

// velocity() for a grid with the image's resolution (gw = W, gh = H), the
// common case: the node below the position is (ix + floor(fx - 1/2),
// iy + floor(fy - 1/2)).  When it and its three neighbours lie in the staged
// window, they are read from shared memory with one row offset; otherwise
// (window edge, grid border clamping) velocity() reads the grid.  The four
// nodes of the last cell are kept in registers: the stages of an RK4
// substep mostly sample the cell of the stage before (the third stage that
// of the second, the next substep's first that of the fourth), so a lane
// reloads the nodes only when its cell changes and the window's
// shared-memory loads (random gathers, bank-conflicted) are issued by fewer
// lanes.  The nodes and the arithmetic are those of velocity(), so the
// result is identical.
struct TileVelocity {
    const Flow &F;
    const FlowWindow &Wn;
    uint32_t p;  // .shared address of node (v, u) of the cached cell, ~0u: none
    float2 a, b, c, d;
    __device__ TileVelocity(const Flow &f, const FlowWindow &w) : F(f), Wn(w), p(~0u) {}
    __device__ __forceinline__ float2 operator()(int32_t ix, float fx, int32_t iy, float fy) {
        const float gx = fx - 0.5f, gy = fy - 0.5f;
        const float flx = floorf(gx), fly = floorf(gy);
        const float tx = gx - flx, ty = gy - fly;
        const int32_t u = ix - Wn.gx0 + (__float_as_int(flx + 12582912.0f) - 0x4B400000);
        const int32_t v = iy - Wn.gy0 + (__float_as_int(fly + 12582912.0f) - 0x4B400000);
        const unsigned lx = Wn.nw > 1 ? (unsigned)(Wn.nw - 1) : 0u, ly = Wn.nh > 1 ? (unsigned)(Wn.nh - 1) : 0u;
        if ((unsigned)u < lx && (unsigned)v < ly) {
            const uint32_t pp = Wn.sa + 8u * (uint32_t)(v * Wn.nw + u);
            if (pp != p) {
                p = pp;
                const uint32_t q = pp + 8u * (uint32_t)Wn.nw;
                a = window_node(pp);
                b = window_node(pp + 8u);
                c = window_node(q);
                d = window_node(q + 8u);
            }
            const float tu = fmaf(tx, b.x - a.x, a.x), tv = fmaf(tx, b.y - a.y, a.y);
            const float bu = fmaf(tx, d.x - c.x, c.x), bv = fmaf(tx, d.y - c.y, c.y);
            return make_float2(fmaf(ty, bu - tu, tu), fmaf(ty, bv - tv, tv));
        }
        return velocity(F, ix, fx, iy, fy);
    }
};

}  // namespace spx
