// The adjoint of the differentiable render (frames B_f = L * S_f with float
// output, no blur; noise is additive and does not depend on the inputs): the
// gradient of a loss with dL/dB given, with respect to the flow grids, the
// frame-1 particle positions and the particle diameters.
//
//   k_adj_splat   a group of 8, 16 or 32 lanes per (particle, frame): gathers
//                 sum_ij dL/dB(i,j) L(i,j) dS(i,j)/d(x, y, sigma) over the
//                 particle's window (a per-particle reduction, no pixel atomics)
//   k_adj_advect  one thread per particle: recomputes the RK4 / Euler
//                 substeps and sweeps them backwards with the bilinear
//                 Jacobians, adding dL/dflow at each stage's four stencil nodes
#include "common.cuh"
#include "kernels.cuh"
#include "particle.cuh"
#include "phi.cuh"

namespace spx {

// Standard normal density (the hardware exponential: relative error ~1e-7,
// far below the gradient's FP32 tolerance).
__device__ __forceinline__ float gauss_pdf(float t) { return 0.39894228040143267794f * __expf(-0.5f * t * t); }

// Pixel mass of column j for a particle at i + f (split), and its derivatives
// with respect to the centre and to sigma:
//   m = Phi(b) - Phi(a), dm/dc = (pdf(a) - pdf(b)) / sigma,
//   dm/dsigma = (a pdf(a) - b pdf(b)) / sigma,  a = (j - c)/sigma, b = (j + 1 - c)/sigma.
// The masses use the forward splat's tabulated tail (tab: the table in
// shared memory), so the gradient is that of the rendered values.
__device__ __forceinline__ void axis_terms(int32_t ic, float fc, int32_t j, float inv, uint32_t tab, float &m,
                                           float &dm, float &ds) {
    const float da = (float)(j - ic) - fc, db = (float)(j + 1 - ic) - fc;
    const float ta = da * inv, tb = db * inv;
    m = edge_mass(edge_value_tab(da, inv, tab), edge_value_tab(db, inv, tab));
    const float pa = gauss_pdf(ta), pb = gauss_pdf(tb);
    dm = (pa - pb) * inv;
    ds = (ta * pa - tb * pb) * inv;
}

// GS lanes per (particle, frame): 32 / GS of them per warp, so that lanes
// are not left idle on windows much narrower than a warp.
template <int GS>
__global__ void __launch_bounds__(256) k_adj_splat(KernelArgs a) {
    static_assert(GS == 8 || GS == 16 || GS == 32, "lane groups within a warp");
    if (*a.check != 1) return;
    extern __shared__ float scr[];
    __shared__ __align__(16) float s_phi[(kPhiDegree + 1) * kPhiPieces];
    for (int k = threadIdx.x; k < (kPhiDegree + 1) * kPhiPieces; k += blockDim.x) s_phi[k] = kPhiTable[k];
    __syncthreads();
    const uint32_t tab = sh_addr(s_phi);
    const int lane = threadIdx.x & 31, j = lane & (GS - 1);
    const int grp = (int)(threadIdx.x / GS);  // group of the CTA
    const int64_t wg = (int64_t)blockIdx.x * (256 / GS) + grp;
    const bool valid = wg < 2 * a.n_part;
    const int64_t g = valid ? wg >> 1 : 0;
    const int f = (int)(wg & 1);
    float sx = 0.f, sy = 0.f, ss = 0.f, sm = 0.f, amp = 0.f, inv = 0.f;
    // the group's particle and window (any: a non-empty window)
    bool any = false, illum = false;
    int32_t H = 0, W = 0, ix = 0, iy = 0, nx = 0, ny = 0;
    float px = 0.f, py = 0.f, dl = 0.f, lmin = 0.f;
    Window w;
    w.j0 = w.i0 = 0;
    int64_t img = 0;
    if (valid) {
        const int b = upper_find(a.n_pairs, g, [&](int m) { return a.plan[m].part_base; });
        const synthpix_pair_desc &D = a.descs[b];
        H = D.height;
        W = D.width;
        const float4 p = f ? a.pos1[g] : a.pos0[g];
        const float2 q = a.sa[g];
        ix = __float_as_int(p.z);
        iy = __float_as_int(p.w);
        px = p.x;
        py = p.y;
        const float sig = q.x;
        amp = q.y;
        inv = __frcp_rn(sig);
        w = particle_window(ix, px, iy, py, 6.0f * sig, W, H);
        any = w.j0 <= w.j1 && w.i0 <= w.i1;
        nx = w.j1 - w.j0 + 1;
        ny = w.i1 - w.i0 + 1;
        illum = D.illum_min != 1.0f || D.illum_max != 1.0f;
        dl = D.illum_max - D.illum_min;
        lmin = D.illum_min;
        img = D.image_offset + (int64_t)f * H * W;
    }
    const int wq = a.warp_scratch;  // floats per array
    float *ex = scr + grp * 8 * wq, *dex = ex + wq, *dsx = dex + wq, *lx = dsx + wq;
    float *ey = lx + wq, *dey = ey + wq, *dsy = dey + wq, *ly = dsy + wq;
    if (any) {
        for (int e = j; e < nx; e += GS) {
            axis_terms(ix, px, w.j0 + e, inv, tab, ex[e], dex[e], dsx[e]);
            if (illum) {
                const float sv = sinpif(((float)(w.j0 + e) + 0.5f) / (float)W);
                lx[e] = sv * sv;
            }
        }
        for (int e = j; e < ny; e += GS) {
            axis_terms(iy, py, w.i0 + e, inv, tab, ey[e], dey[e], dsy[e]);
            if (illum) {
                const float sv = sinpif(((float)(w.i0 + e) + 0.5f) / (float)H);
                ly[e] = sv * sv;
            }
        }
    }
    __syncwarp();  // every lane of the warp: the group's terms are visible to the group
    if (any) {
        // lane j walks the rows of columns j, j + GS, ...: the column terms stay in registers, the
        // row terms are read once per pixel (the same word for all lanes), dL/dB a row at a time
        const float *G = a.grad_images + img + (int64_t)w.i0 * W + w.j0;
        for (int c = j; c < nx; c += GS) {
            const float exc = ex[c], dexc = dex[c], dsxc = dsx[c], lxc = illum ? lx[c] : 0.0f;
            const float *gc = G + c;
            for (int r = 0; r < ny; ++r) {
                float gv = gc[(int64_t)r * W];
                const float eyr = ey[r];
                if (illum) gv *= fmaf(dl, lxc * ly[r], lmin);
                sx = fmaf(gv * dexc, eyr, sx);
                sy = fmaf(gv * exc, dey[r], sy);
                ss = fmaf(gv, fmaf(dsxc, eyr, exc * dsy[r]), ss);
                sm = fmaf(gv * exc, eyr, sm);
            }
        }
    }
#pragma unroll
    for (int o = GS / 2; o > 0; o >>= 1) {  // within the group (xor offsets below GS stay in it)
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        ss += __shfl_xor_sync(0xffffffffu, ss, o);
        sm += __shfl_xor_sync(0xffffffffu, sm, o);
    }
    // S = amp Ex Ey with amp = Ieff 2 pi sigma^2: d amp / d sigma = 2 amp / sigma
    if (valid && j == 0)
        a.grad_frames[2 * g + f] =
            any ? make_float4(amp * sx, amp * sy, amp * ss + 2.0f * amp * inv * sm, 0.f) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// The four nodes of the last grid cell (l, k) a thread's Jacobians read: the
// third stage of an RK4 substep nearly always samples the cell of the second,
// so its gathers (and their latency in the thread's dependent chain) are
// skipped.  Same nodes, same arithmetic.
struct CellCache {
    int32_t l, k;  // the cell before clamping; l = INT32_MIN: none
    float2 A, B, C, D;
};

// Velocity at i + f (split) with its Jacobian (J = du/dx, du/dy, dv/dx, dv/dy)
// and the four stencil nodes (flat index k * gw + l) with their weights.
__device__ __forceinline__ float2 velocity_jac(const Flow &F, int32_t ix, float fx, int32_t iy, float fy, float J[4],
                                               int node[4], float wgt[4], CellCache &cc) {
    int32_t l, k;
    float tx, ty;
    grid_coord(ix, fx, F.gw, F.W, l, tx);
    grid_coord(iy, fy, F.gh, F.H, k, ty);
    const int32_t l0 = min(max(l, 0), F.gw - 1), l1 = min(max(l + 1, 0), F.gw - 1);
    const int32_t k0 = min(max(k, 0), F.gh - 1), k1 = min(max(k + 1, 0), F.gh - 1);
    if (l != cc.l || k != cc.k) {
        cc.l = l;
        cc.k = k;
        cc.A = __ldg(F.f + (size_t)k0 * F.gw + l0);
        cc.B = __ldg(F.f + (size_t)k0 * F.gw + l1);
        cc.C = __ldg(F.f + (size_t)k1 * F.gw + l0);
        cc.D = __ldg(F.f + (size_t)k1 * F.gw + l1);
    }
    const float2 A = cc.A, B = cc.B, C = cc.C, D = cc.D;
    const float tu = fmaf(tx, B.x - A.x, A.x), tv = fmaf(tx, B.y - A.y, A.y);
    const float bu = fmaf(tx, D.x - C.x, C.x), bv = fmaf(tx, D.y - C.y, C.y);
    const float sxg = (float)F.gw / (float)F.W, syg = (float)F.gh / (float)F.H;
    J[0] = ((1.0f - ty) * (B.x - A.x) + ty * (D.x - C.x)) * sxg;
    J[1] = (bu - tu) * syg;
    J[2] = ((1.0f - ty) * (B.y - A.y) + ty * (D.y - C.y)) * sxg;
    J[3] = (bv - tv) * syg;
    node[0] = k0 * F.gw + l0; wgt[0] = (1.0f - tx) * (1.0f - ty);
    node[1] = k0 * F.gw + l1; wgt[1] = tx * (1.0f - ty);
    node[2] = k1 * F.gw + l0; wgt[2] = (1.0f - tx) * ty;
    node[3] = k1 * F.gw + l1; wgt[3] = tx * ty;
    return make_float2(fmaf(ty, bu - tu, tu), fmaf(ty, bv - tv, tv));
}

// dL/dflow of one stage at its four stencil nodes: one vector reduction per
// node adds (u, v) (each component atomically, as two atomicAdds would).
__device__ __forceinline__ void scatter_flow(float *gf, const int node[4], const float wgt[4], float lx, float ly) {
    if (!gf) return;
#pragma unroll
    for (int n = 0; n < 4; ++n)
        asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(gf + 2 * node[n]), "f"(wgt[n] * lx),
                     "f"(wgt[n] * ly) : "memory");
}

// NMAX: capacity of the substep arrays (n_substeps <= NMAX); with a small
// NMAX the loops unroll and the arrays live in registers.
template <int NMAX>
__global__ void __launch_bounds__(128) k_adj_advect(KernelArgs a) {
    if (*a.check != 1) return;
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= a.n_part) return;
    const int b = upper_find(a.n_pairs, g, [&](int m) { return a.plan[m].part_base; });
    const PairPlan pl = a.plan[b];
    const synthpix_pair_desc &D = a.descs[b];
    const uint32_t i = (uint32_t)(g - pl.part_base);
    const float4 g1 = a.grad_frames[2 * g], g2 = a.grad_frames[2 * g + 1];
    const Flow F = pair_flow(a, D);
    float *gf = a.grad_flows ? a.grad_flows + D.flow_offset : nullptr;
    const int n = a.n_substeps;
    const float h = a.dt / (float)n;
    const float hh = 0.5f * h, h6 = h / 6.0f;
    // the start of every substep (n <= NMAX): kept by the forward advection, or recomputed
    int32_t si[NMAX], sj[NMAX];
    float sfx[NMAX], sfy[NMAX];
    if (a.states) {
        const float4 *sp = a.states + g * n;
#pragma unroll(NMAX <= 8 ? NMAX : 1)
        for (int s = 0; s < NMAX; ++s) {
            if (s < n) {
                const float4 q = sp[s];
                sfx[s] = q.x; sfy[s] = q.y; si[s] = __float_as_int(q.z); sj[s] = __float_as_int(q.w);
            }
        }
    } else {
        const Seeded P = seed_particle(a, D, i, g);
        int32_t jx = P.ix, jy = P.iy;
        float fx = P.fx, fy = P.fy;
#pragma unroll(NMAX <= 8 ? NMAX : 1)
        for (int s = 0; s < NMAX; ++s) {
            if (s < n) {
                si[s] = jx; sj[s] = jy; sfx[s] = fx; sfy[s] = fy;
                advect_split(F, h, 1, a.integrator, jx, fx, jy, fy);
            }
        }
    }
    float lx = g2.x, ly = g2.y;  // dL / d(frame-2 position)
    CellCache cc;
    cc.l = INT32_MIN;
    cc.k = 0;
#pragma unroll(NMAX <= 8 ? NMAX : 1)
    for (int s = NMAX - 1; s >= 0; --s) {
        if (s >= n) continue;
        const int32_t px = si[s], py = sj[s];
        const float ux = sfx[s], uy = sfy[s];
        float J1[4], w1[4];
        int n1[4];
        const float2 k1 = velocity_jac(F, px, ux, py, uy, J1, n1, w1, cc);
        if (a.integrator == SYNTHPIX_EULER) {
            scatter_flow(gf, n1, w1, h * lx, h * ly);
            const float ax = lx + h * (J1[0] * lx + J1[2] * ly);
            const float ay = ly + h * (J1[1] * lx + J1[3] * ly);
            lx = ax;
            ly = ay;
            continue;
        }
        float J2[4], w2[4], J3[4], w3[4], J4[4], w4[4];
        int n2[4], n3[4], n4[4];
        const float2 k2 = velocity_jac(F, px, fmaf(hh, k1.x, ux), py, fmaf(hh, k1.y, uy), J2, n2, w2, cc);
        const float2 k3 = velocity_jac(F, px, fmaf(hh, k2.x, ux), py, fmaf(hh, k2.y, uy), J3, n3, w3, cc);
        velocity_jac(F, px, fmaf(h, k3.x, ux), py, fmaf(h, k3.y, uy), J4, n4, w4, cc);
        // p+ = p + h/6 (k1 + 2 k2 + 2 k3 + k4), k_m = U(q_m): adjoints of the stages
        const float k4x = h6 * lx, k4y = h6 * ly;
        const float k3x = 2.0f * h6 * lx + h * (J4[0] * k4x + J4[2] * k4y);
        const float k3y = 2.0f * h6 * ly + h * (J4[1] * k4x + J4[3] * k4y);
        const float k2x = 2.0f * h6 * lx + hh * (J3[0] * k3x + J3[2] * k3y);
        const float k2y = 2.0f * h6 * ly + hh * (J3[1] * k3x + J3[3] * k3y);
        const float k1x = h6 * lx + hh * (J2[0] * k2x + J2[2] * k2y);
        const float k1y = h6 * ly + hh * (J2[1] * k2x + J2[3] * k2y);
        scatter_flow(gf, n1, w1, k1x, k1y);
        scatter_flow(gf, n2, w2, k2x, k2y);
        scatter_flow(gf, n3, w3, k3x, k3y);
        scatter_flow(gf, n4, w4, k4x, k4y);
        const float ax = lx + (J1[0] * k1x + J1[2] * k1y) + (J2[0] * k2x + J2[2] * k2y) + (J3[0] * k3x + J3[2] * k3y) +
                         (J4[0] * k4x + J4[2] * k4y);
        const float ay = ly + (J1[1] * k1x + J1[3] * k1y) + (J2[1] * k2x + J2[3] * k2y) + (J3[1] * k3x + J3[3] * k3y) +
                         (J4[1] * k4x + J4[3] * k4y);
        lx = ax;
        ly = ay;
    }
    if (a.grad_particles) {
        a.grad_particles[3 * g] = g1.x + lx;
        a.grad_particles[3 * g + 1] = g1.y + ly;
        a.grad_particles[3 * g + 2] = 0.25f * (g1.z + g2.z);  // sigma = d / 4
    }
}

// Lanes per (particle, frame) of k_adj_splat for windows of at most wmax
// pixels a side: the narrowest group whose lanes take at most two columns
// (or rows) each.
__host__ __device__ inline int adj_group(int wmax) { return wmax <= 16 ? 8 : (wmax <= 32 ? 16 : 32); }

cudaError_t launch_adjoint(const KernelArgs &a, cudaStream_t st) {
    if (a.n_part == 0) return cudaGetLastError();
    const int gs = adj_group(a.warp_scratch - 2);
    const int per_cta = 256 / gs;  // (particle, frame) groups of a CTA
    const size_t smem = (size_t)per_cta * 8 * a.warp_scratch * sizeof(float);
    const unsigned grid = (unsigned)((2 * a.n_part + per_cta - 1) / per_cta);
    auto go = [&](auto kern) -> cudaError_t {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        return launch_kernel(kern, grid, 256, smem, st, a);
    };
    cudaError_t e = gs == 8 ? go(k_adj_splat<8>) : (gs == 16 ? go(k_adj_splat<16>) : go(k_adj_splat<32>));
    if (e != cudaSuccess) return e;
    const unsigned agrid = (unsigned)((a.n_part + 127) / 128);
    if (a.n_substeps <= 4) return launch_kernel(k_adj_advect<4>, agrid, 128, 0, st, a);
    if (a.n_substeps <= 8) return launch_kernel(k_adj_advect<8>, agrid, 128, 0, st, a);
    return launch_kernel(k_adj_advect<kMaxAdjointSubsteps>, agrid, 128, 0, st, a);
}

}  // namespace spx
