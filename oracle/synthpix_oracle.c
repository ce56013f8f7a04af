/*
 * FP64 CPU oracle for PIV image-pair rendering (SynthPix, arXiv 2512.09664).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, step-by-step
 * restatement of the rendering method, used to check the CUDA library.
 * It shares no code, header or constant table with the CUDA path and must
 * never be linked into it.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.
 *
 * The method (paper Section 2):
 *   - particles sampled uniformly over the image domain, parameters drawn
 *     uniformly from configured intervals            ("Sampling the particles",
 *                                                       text after Eq. 1)
 *   - image-2 positions from the displacement map (x, y) -> (x+u, y+v)
 *                                                     ("Sampling the particles")
 *   - single-particle image: the Gaussian of Eq. 1 (round by default; general
 *     sigma_x, sigma_y, rho under R8)
 *   - contributions summed (superposition)          ("aggregation of the
 *                                                       particle contributions")
 *   - each particle rendered on a patch of 3 max(d)+1 px ("Efficient rasterization")
 *   - illumination non-uniformity, noise and blur named among the imaging
 *     parameters (Abstract) with no formula given.
 *
 * Readings taken where the paper is silent:
 *   R1  sigma = d / 4 (e^-2 diameter), so the integrated particle image is
 *       pi d^2 / 8 * I0.
 *   R2  pixel (i, j) covers [j, j+1) x [i, i+1), x = column, y = row (down);
 *       the particle image is integrated over the pixel (100% fill factor,
 *       Remark "camera-model"), giving separable erf differences.
 *   R3  out-of-plane gain exp(-z^2 / (2 s^2)) (Gaussian laser sheet), z fixed
 *       between frames; the Remark "out-of-focus" form is deferred by the paper.
 *   R4  flow grid nodes at cell centres, bilinear interpolation in lerp form,
 *       indices clamped to the grid (border); displacement integrated with RK4
 *       (or Euler) in n substeps over dt.  Euler with n = 1 and dt = 1 is the
 *       paper's x + u(x).
 *   R5  window: per particle j in [floor(x - 1.5 d), floor(x + 1.5 d)] (the
 *       3 d + 1 patch), clipped to the image.
 *   R6  epilogue per frame: A = L * S + sigma_n * n, L a separable sin^2
 *       bump between illum_min and illum_max, n standard normal (Box-Muller on
 *       Philox words); separable normalised Gaussian blur, radius ceil(3 sigma_b),
 *       replicate border, horizontal pass first; quantisation
 *       clamp(rint(B * M), 0, M), M = 2^bits - 1, round-half-even, decided on
 *       the FP64 value B (codes are defined on the exact value; a renderer in
 *       lower precision can differ only within its error of a boundary).
 *   R7  random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the seed,
 *       counter (index, stream tag, pair id): tag 0 -> (x, y, d, I) words,
 *       tag 1 -> (z, d2) words, tag 2 -> (hide 1, hide 2, two normals for
 *       the frame-2 change of d and I0), tag 3 -> (d_y, rho, two normals for
 *       the frame-2 change of d_y and rho), tag 0x100 + f -> noise words of
 *       frame f.
 *   R9  out-of-focus intensity: the Gaussian sheet of R3, or the Remark
 *       "out-of-focus" form exp(-|2 z^2 / dz0^2|^s / sqrt(2 pi)) with the
 *       sheet thickness dz0 and shape factor s, the drawn I0 playing the
 *       scattering efficiency q.  Out-of-plane motion (the Remark's 3-D flow):
 *       an optional scalar grid w (same nodes as the flow) moves z along the
 *       particle's path, integrated with the same substeps and stages as x,
 *       y; frame 2's intensity then uses the moved z.
 *   R8  general particle shapes (Eq. 1 with sigma_x != sigma_y and rho != 0;
 *       text after Eq. 1): sigma_x = d / 4, sigma_y = d_y / 4 with d_y drawn
 *       from its own interval (d_y = d when that interval is [0, 0]), rho from
 *       its interval.  Frame-2 parameters are the frame-1 ones plus a zero-mean
 *       Gaussian change of the configured std, clamped to the parameter's
 *       interval (I0 to [i_min, i_max]).  A particle is hidden from each frame
 *       independently with probability hide_prob (aggregation paragraph).
 *       The pixel value is the integral of Eq. 1 over the pixel: the
 *       integrated image of a particle is I0 2 pi sigma_x sigma_y sqrt(1-rho^2)
 *       and its window is floor(x +- 1.5 d) by floor(y +- 1.5 d_y).
 *
 * Precision: FP64 everywhere, the quantisation decision included (R6).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846

typedef struct {
    int32_t height, width;      /* image size in pixels */
    int32_t flow_h, flow_w;     /* flow grid size in nodes */
    int64_t n_particles;        /* particles seeded in frame 1 */
    uint64_t seed, pair_id;     /* Philox key and counter words */
    int32_t d_dist;             /* 0 uniform diameter, 1 clipped normal */
    int32_t integrator;         /* 0 RK4, 1 Euler */
    int32_t n_substeps;         /* >= 1 */
    int32_t quant_bits;         /* 0: no quantisation */
    double d_min, d_max, d_mu, d_sigma;
    double i_min, i_max, z_min, z_max, sheet_sigma;
    double illum_min, illum_max, noise_sigma, blur_sigma;
    double dt;
    /* general shapes, frame-2 variation, hiding (R8); all 0: round particles */
    double dy_min, dy_max, rho_min, rho_max;
    double jitter_d, jitter_i, jitter_rho, hide_prob;
    /* out-of-focus model (R9): 0 Gaussian sheet, 1 Remark form with shape factor */
    int32_t sheet_model;
    double sheet_shape;
} oracle_pair;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As  */
/* Easy as 1, 2, 3", SC'11.  Round: two 32x32->64 products of counter words */
/* 0 and 2 with the multipliers, outputs mixed with the other counter words */
/* and the key; the key is bumped by the Weyl constants between rounds.     */
/* ------------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Words of stream `tag` at index `idx` for this pair (R7). */
void oracle_stream_words(uint64_t seed, uint64_t pair_id, uint32_t idx, uint32_t tag, uint32_t w[4])
{
    uint32_t ctr[4] = { idx, tag, (uint32_t)pair_id, (uint32_t)(pair_id >> 32) };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    oracle_philox4x32_10(ctr, key, w);
}

/* uniform in [0, 1) from the top 24 bits */
static double u24(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }
/* uniform in (0, 1] from the top 24 bits (safe for log) */
static double uo24(uint32_t w) { return (double)((w >> 8) + 1u) * (1.0 / 16777216.0); }

/* Box-Muller normal; second = 0 takes the cosine branch, 1 the sine branch */
static double box_muller(uint32_t wa, uint32_t wb, int second)
{
    double r = sqrt(-2.0 * log(uo24(wa)));
    double th = 2.0 * ORACLE_PI * u24(wb);
    return second ? r * sin(th) : r * cos(th);
}

/* ------------------------------------------------------------------------ */
/* particle attributes (paper Section 2, text after Eq. 1; R1, R3, R7)      */
/* ------------------------------------------------------------------------ */
typedef struct { double x0, y0, d, intensity, z, gain, ieff; } oracle_attr;

/* Intensity factor of a particle at out-of-plane position z (R3, R9). */
double oracle_sheet_gain(const oracle_pair *p, double z)
{
    if (!(p->sheet_sigma > 0.0)) return 1.0;
    if (p->sheet_model == 1) {
        double q = fabs(2.0 * z * z / (p->sheet_sigma * p->sheet_sigma));
        return exp(-pow(q, p->sheet_shape) / sqrt(2.0 * ORACLE_PI));
    }
    return exp(-(z * z) / (2.0 * p->sheet_sigma * p->sheet_sigma));
}

static void particle_attr(const oracle_pair *p, uint32_t i, oracle_attr *a)
{
    uint32_t w0[4], w1[4];
    oracle_stream_words(p->seed, p->pair_id, i, 0u, w0);
    oracle_stream_words(p->seed, p->pair_id, i, 1u, w1);
    a->x0 = u24(w0[0]) * (double)p->width;
    a->y0 = u24(w0[1]) * (double)p->height;
    if (p->d_dist == 0) {
        a->d = p->d_min + u24(w0[2]) * (p->d_max - p->d_min);
    } else {
        double n = box_muller(w0[2], w1[1], 0);
        double d = p->d_mu + p->d_sigma * n;
        a->d = d < p->d_min ? p->d_min : (d > p->d_max ? p->d_max : d);
    }
    a->intensity = p->i_min + u24(w0[3]) * (p->i_max - p->i_min);
    a->z = p->z_min + u24(w1[0]) * (p->z_max - p->z_min);
    a->gain = oracle_sheet_gain(p, a->z);
    a->ieff = a->intensity * a->gain;
}

static double clampd(double v, double lo, double hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* A particle as rendered in one frame (R8). */
typedef struct { double dx, dy, rho, ieff; int visible; } oracle_shape;

int oracle_round_particles(const oracle_pair *p)
{
    return p->dy_min == 0.0 && p->dy_max == 0.0 && p->rho_min == 0.0 && p->rho_max == 0.0;
}

/* Frame 1 and frame 2 shapes of particle i with attributes a (R8); gain2 is
 * the sheet factor in frame 2 (a->gain unless the particle moved in z, R9). */
static void particle_shapes(const oracle_pair *p, uint32_t i, const oracle_attr *a, double gain2, oracle_shape s[2])
{
    uint32_t w2[4], w3[4];
    oracle_stream_words(p->seed, p->pair_id, i, 2u, w2);
    oracle_stream_words(p->seed, p->pair_id, i, 3u, w3);
    const int same_d = p->dy_min == 0.0 && p->dy_max == 0.0;
    double dy = same_d ? a->d : p->dy_min + u24(w3[0]) * (p->dy_max - p->dy_min);
    double rho = p->rho_min + u24(w3[1]) * (p->rho_max - p->rho_min);
    s[0].dx = a->d;
    s[0].dy = dy;
    s[0].rho = rho;
    s[0].ieff = a->ieff;
    s[0].visible = !(u24(w2[0]) < p->hide_prob);
    double dx2 = clampd(a->d + p->jitter_d * box_muller(w2[2], w2[3], 0), p->d_min, p->d_max);
    double i2 = clampd(a->intensity + p->jitter_i * box_muller(w2[2], w2[3], 1), p->i_min, p->i_max);
    s[1].dx = dx2;
    s[1].dy = same_d ? dx2 : clampd(dy + p->jitter_d * box_muller(w3[2], w3[3], 0), p->dy_min, p->dy_max);
    s[1].rho = clampd(rho + p->jitter_rho * box_muller(w3[2], w3[3], 1), p->rho_min, p->rho_max);
    s[1].ieff = i2 * gain2;
    s[1].visible = !(u24(w2[1]) < p->hide_prob);
}

/*
 * Per-particle shape table, 10 doubles per particle: for frame 1 then
 * frame 2, (d_x, d_y, rho, Ieff, visible).
 */
int oracle_particle_shapes(const oracle_pair *p, double *out)
{
    for (int64_t i = 0; i < p->n_particles; ++i) {
        oracle_attr a;
        oracle_shape s[2];
        particle_attr(p, (uint32_t)i, &a);
        particle_shapes(p, (uint32_t)i, &a, a.gain, s);
        for (int f = 0; f < 2; ++f) {
            double *o = out + 10 * i + 5 * f;
            o[0] = s[f].dx; o[1] = s[f].dy; o[2] = s[f].rho; o[3] = s[f].ieff; o[4] = (double)s[f].visible;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* bilinear velocity on the cell-centred grid, border clamp (R4)            */
/* ------------------------------------------------------------------------ */
static long clampl(long v, long lo, long hi) { return v < lo ? lo : (v > hi ? hi : v); }

void oracle_velocity(const float *flow, int32_t gh, int32_t gw, int32_t height, int32_t width,
                     double x, double y, double *u, double *v)
{
    double gx = x * (double)gw / (double)width - 0.5;
    double gy = y * (double)gh / (double)height - 0.5;
    double fl = floor(gx), fk = floor(gy);
    double tx = gx - fl, ty = gy - fk;
    long l0 = clampl((long)fl, 0, gw - 1), l1 = clampl((long)fl + 1, 0, gw - 1);
    long k0 = clampl((long)fk, 0, gh - 1), k1 = clampl((long)fk + 1, 0, gh - 1);
    double out[2];
    for (int c = 0; c < 2; ++c) {
        double a = flow[(k0 * gw + l0) * 2 + c], b = flow[(k0 * gw + l1) * 2 + c];
        double e = flow[(k1 * gw + l0) * 2 + c], f = flow[(k1 * gw + l1) * 2 + c];
        double top = a + tx * (b - a);
        double bot = e + tx * (f - e);
        out[c] = top + ty * (bot - top);
    }
    *u = out[0];
    *v = out[1];
}

/* Position after dt (paper: displacement map; R4: RK4 / Euler substeps). */
void oracle_advect(const oracle_pair *p, const float *flow, double x, double y,
                   double *xo, double *yo)
{
    int n = p->n_substeps;
    double h = p->dt / (double)n;
    for (int s = 0; s < n; ++s) {
        double u1, v1;
        oracle_velocity(flow, p->flow_h, p->flow_w, p->height, p->width, x, y, &u1, &v1);
        if (p->integrator == 1) {
            x += h * u1;
            y += h * v1;
            continue;
        }
        double u2, v2, u3, v3, u4, v4;
        oracle_velocity(flow, p->flow_h, p->flow_w, p->height, p->width,
                        x + 0.5 * h * u1, y + 0.5 * h * v1, &u2, &v2);
        oracle_velocity(flow, p->flow_h, p->flow_w, p->height, p->width,
                        x + 0.5 * h * u2, y + 0.5 * h * v2, &u3, &v3);
        oracle_velocity(flow, p->flow_h, p->flow_w, p->height, p->width,
                        x + h * u3, y + h * v3, &u4, &v4);
        x += h / 6.0 * (u1 + 2.0 * u2 + 2.0 * u3 + u4);
        y += h / 6.0 * (v1 + 2.0 * v2 + 2.0 * v3 + v4);
    }
    *xo = x;
    *yo = y;
}

/* Scalar w (out-of-plane velocity) at (x, y): bilinear on the same nodes as the flow (R9). */
double oracle_scalar_at(const float *w, int32_t gh, int32_t gw, int32_t height, int32_t width, double x, double y)
{
    double gx = x * (double)gw / (double)width - 0.5;
    double gy = y * (double)gh / (double)height - 0.5;
    double fl = floor(gx), fk = floor(gy);
    double tx = gx - fl, ty = gy - fk;
    long l0 = clampl((long)fl, 0, gw - 1), l1 = clampl((long)fl + 1, 0, gw - 1);
    long k0 = clampl((long)fk, 0, gh - 1), k1 = clampl((long)fk + 1, 0, gh - 1);
    double a = w[k0 * gw + l0], b = w[k0 * gw + l1], e = w[k1 * gw + l0], f = w[k1 * gw + l1];
    double top = a + tx * (b - a), bot = e + tx * (f - e);
    return top + ty * (bot - top);
}

/* Position after dt and the out-of-plane position moved by w along the path
 * (R9): the stages of oracle_advect, each also evaluating w. */
void oracle_advect3(const oracle_pair *p, const float *flow, const float *w, double x, double y, double z,
                    double *xo, double *yo, double *zo)
{
    int n = p->n_substeps;
    double h = p->dt / (double)n;
    const int32_t gh = p->flow_h, gw = p->flow_w, H = p->height, W = p->width;
    for (int s = 0; s < n; ++s) {
        double u1, v1;
        oracle_velocity(flow, gh, gw, H, W, x, y, &u1, &v1);
        double w1 = oracle_scalar_at(w, gh, gw, H, W, x, y);
        if (p->integrator == 1) {
            x += h * u1;
            y += h * v1;
            z += h * w1;
            continue;
        }
        double u2, v2, u3, v3, u4, v4;
        double x2 = x + 0.5 * h * u1, y2 = y + 0.5 * h * v1;
        oracle_velocity(flow, gh, gw, H, W, x2, y2, &u2, &v2);
        double w2 = oracle_scalar_at(w, gh, gw, H, W, x2, y2);
        double x3 = x + 0.5 * h * u2, y3 = y + 0.5 * h * v2;
        oracle_velocity(flow, gh, gw, H, W, x3, y3, &u3, &v3);
        double w3 = oracle_scalar_at(w, gh, gw, H, W, x3, y3);
        double x4 = x + h * u3, y4 = y + h * v3;
        oracle_velocity(flow, gh, gw, H, W, x4, y4, &u4, &v4);
        double w4 = oracle_scalar_at(w, gh, gw, H, W, x4, y4);
        x += h / 6.0 * (u1 + 2.0 * u2 + 2.0 * u3 + u4);
        y += h / 6.0 * (v1 + 2.0 * v2 + 2.0 * v3 + v4);
        z += h / 6.0 * (w1 + 2.0 * w2 + 2.0 * w3 + w4);
    }
    *xo = x;
    *yo = y;
    *zo = z;
}

/*
 * Per-particle table, 8 doubles per particle:
 *   x0, y0 (frame 1), d, I, z, Ieff, x1, y1 (frame 2).
 */
int oracle_particles(const oracle_pair *p, const float *flow, double *out)
{
    for (int64_t i = 0; i < p->n_particles; ++i) {
        oracle_attr a;
        particle_attr(p, (uint32_t)i, &a);
        double x1, y1;
        oracle_advect(p, flow, a.x0, a.y0, &x1, &y1);
        double *o = out + 8 * i;
        o[0] = a.x0; o[1] = a.y0; o[2] = a.d; o[3] = a.intensity;
        o[4] = a.z; o[5] = a.ieff; o[6] = x1; o[7] = y1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* pixel integration of Eq. 1 (rho = 0): separable erf differences (R2)     */
/* ------------------------------------------------------------------------ */

/* Mass of a unit 1-D Gaussian (centre c, std sigma) over [j, j + 1). */
double oracle_pixel_mass(double c, double sigma, int64_t j)
{
    const double s2 = 1.4142135623730950488;
    double a = ((double)j - c) / sigma;
    double b = ((double)j + 1.0 - c) / sigma;
    /* Phi(t) = erfc(-t / sqrt 2) / 2; the tails use erfc differences */
    if (a >= 0.0)
        return 0.5 * (erfc(a / s2) - erfc(b / s2));
    if (b <= 0.0)
        return 0.5 * (erfc(-b / s2) - erfc(-a / s2));
    return 1.0 - 0.5 * erfc(-a / s2) - 0.5 * erfc(b / s2);
}

/*
 * Accumulate particles into one frame S[H][W] (not cleared here).
 * parts: n rows of (x, y, d, Ieff).  mode 0: windowed pixel-integrated
 * (the method); mode 1: pixel-integrated over every pixel (brute force, no
 * window); mode 2: Eq. 1 point-sampled at pixel centres inside the window.
 */
int oracle_splat(int32_t height, int32_t width, const double *parts, int64_t n, int32_t mode,
                 double *S)
{
    double *ex = (double *)malloc(sizeof(double) * (size_t)width);
    if (!ex) return -1;
    for (int64_t k = 0; k < n; ++k) {
        double x = parts[4 * k], y = parts[4 * k + 1], d = parts[4 * k + 2], ieff = parts[4 * k + 3];
        double sigma = d / 4.0;
        double amp = ieff * 2.0 * ORACLE_PI * sigma * sigma;
        long j0 = (long)floor(x - 1.5 * d), j1 = (long)floor(x + 1.5 * d);
        long i0 = (long)floor(y - 1.5 * d), i1 = (long)floor(y + 1.5 * d);
        if (mode == 1) {
            j0 = 0; j1 = width - 1; i0 = 0; i1 = height - 1;
        }
        if (j0 < 0) j0 = 0;
        if (i0 < 0) i0 = 0;
        if (j1 > width - 1) j1 = width - 1;
        if (i1 > height - 1) i1 = height - 1;
        if (j0 > j1 || i0 > i1) continue;
        if (mode == 2) {
            for (long i = i0; i <= i1; ++i)
                for (long j = j0; j <= j1; ++j) {
                    double dx = (double)j + 0.5 - x, dy = (double)i + 0.5 - y;
                    S[i * width + j] += ieff * exp(-(dx * dx + dy * dy) / (2.0 * sigma * sigma));
                }
            continue;
        }
        for (long j = j0; j <= j1; ++j) ex[j] = oracle_pixel_mass(x, sigma, j);
        for (long i = i0; i <= i1; ++i) {
            double ey = oracle_pixel_mass(y, sigma, i);
            for (long j = j0; j <= j1; ++j) S[i * width + j] += amp * ex[j] * ey;
        }
    }
    free(ex);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* pixel integration of Eq. 1 with sigma_x != sigma_y and rho != 0 (R8)     */
/* ------------------------------------------------------------------------ */

/* Gauss-Legendre rule on [-1, 1] with 16 nodes: the roots of the Legendre
 * polynomial P_16 by Newton's method (P_n from its three-term recurrence,
 * starting points cos(pi (k - 1/4) / (n + 1/2))); weight 2 / ((1 - t^2) P_n'(t)^2). */
#define ORACLE_GL 16
static double gl_x[ORACLE_GL], gl_w[ORACLE_GL];

static void legendre(int n, double t, double *pn, double *dpn)
{
    double p0 = 1.0, p1 = t;
    for (int m = 2; m <= n; ++m) {
        double p2 = ((2.0 * m - 1.0) * t * p1 - (m - 1.0) * p0) / (double)m;
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *dpn = (double)n * (t * p1 - p0) / (t * t - 1.0);
}

static void __attribute__((constructor)) gauss_legendre_init(void)
{
    const int n = ORACLE_GL;
    for (int k = 1; k <= n; ++k) {
        double t = cos(ORACLE_PI * ((double)k - 0.25) / ((double)n + 0.5)), pn, dpn;
        for (int it = 0; it < 100; ++it) {
            legendre(n, t, &pn, &dpn);
            double step = pn / dpn;
            t -= step;
            if (fabs(step) < 1e-16) break;
        }
        legendre(n, t, &pn, &dpn);
        gl_x[k - 1] = t;
        gl_w[k - 1] = 2.0 / ((1.0 - t * t) * dpn * dpn);
    }
}

/*
 * Probability of the pixel [j, j+1) x [i, i+1) under the normal density of
 * Eq. 1 centred at (x0, y0) with (sigma_x, sigma_y, rho).  rho = 0: the
 * product of the 1-D masses.  Otherwise the x-marginal N(x0, sigma_x^2)
 * times the conditional mass of y, which is normal with mean
 * y0 + rho sigma_y (x - x0) / sigma_x and std sigma_y sqrt(1 - rho^2): exact
 * in y (erfc), composite 16-node Gauss-Legendre in x over sub-intervals no
 * wider than half the shortest x-scale of the integrand,
 * min(sigma_x, sigma_x sqrt(1 - rho^2) / |rho|).
 */
double oracle_pixel_mass2(double x0, double y0, double sx, double sy, double rho, int64_t j, int64_t i)
{
    if (rho == 0.0) return oracle_pixel_mass(x0, sx, j) * oracle_pixel_mass(y0, sy, i);
    const double c = sqrt(1.0 - rho * rho);
    const double ell = fabs(rho) > c ? sx * c / fabs(rho) : sx;
    long nsub = (long)ceil(2.0 / ell);
    if (nsub < 1) nsub = 1;
    if (nsub > 4096) nsub = 4096;
    const double h = 1.0 / (double)nsub;
    double sum = 0.0;
    for (long q = 0; q < nsub; ++q) {
        const double a = (double)j + (double)q * h;
        for (int k = 0; k < ORACLE_GL; ++k) {
            const double x = a + 0.5 * h * (gl_x[k] + 1.0);
            const double t = (x - x0) / sx;
            const double px = exp(-0.5 * t * t) / (2.50662827463100050242 * sx);
            sum += 0.5 * h * gl_w[k] * px * oracle_pixel_mass(y0 + rho * sy * t, sy * c, i);
        }
    }
    return sum;
}

/*
 * Accumulate particles of general shape into one frame S[H][W] (R8; not
 * cleared here).  parts: n rows of (x, y, d_x, d_y, rho, Ieff).  mode 0:
 * windowed, pixel-integrated (the method); mode 1: pixel-integrated over
 * every pixel (brute force); mode 2: Eq. 1 point-sampled at pixel centres
 * inside the window.
 */
int oracle_splat_shapes(int32_t height, int32_t width, const double *parts, int64_t n, int32_t mode, double *S)
{
    for (int64_t k = 0; k < n; ++k) {
        const double *r = parts + 6 * k;
        double x = r[0], y = r[1], dx = r[2], dy = r[3], rho = r[4], ieff = r[5];
        double sx = dx / 4.0, sy = dy / 4.0, c = sqrt(1.0 - rho * rho);
        double amp = ieff * 2.0 * ORACLE_PI * sx * sy * c;
        long j0 = (long)floor(x - 1.5 * dx), j1 = (long)floor(x + 1.5 * dx);
        long i0 = (long)floor(y - 1.5 * dy), i1 = (long)floor(y + 1.5 * dy);
        if (mode == 1) {
            j0 = 0; j1 = width - 1; i0 = 0; i1 = height - 1;
        }
        if (j0 < 0) j0 = 0;
        if (i0 < 0) i0 = 0;
        if (j1 > width - 1) j1 = width - 1;
        if (i1 > height - 1) i1 = height - 1;
        for (long i = i0; i <= i1; ++i)
            for (long j = j0; j <= j1; ++j) {
                if (mode == 2) {
                    double tx = ((double)j + 0.5 - x) / sx, ty = ((double)i + 0.5 - y) / sy;
                    double e = (tx * tx - 2.0 * rho * tx * ty + ty * ty) / (2.0 * (1.0 - rho * rho));
                    S[i * width + j] += ieff * exp(-e);
                } else {
                    S[i * width + j] += amp * oracle_pixel_mass2(x, y, sx, sy, rho, j, i);
                }
            }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* epilogue (R6)                                                            */
/* ------------------------------------------------------------------------ */

/* Standard normal noise sample of pixel `pix` (row-major) in frame `frame`. */
double oracle_noise(uint64_t seed, uint64_t pair_id, int32_t frame, int64_t pix)
{
    uint32_t w[4];
    oracle_stream_words(seed, pair_id, (uint32_t)(pix >> 2), 0x100u + (uint32_t)frame, w);
    switch (pix & 3) {
    case 0: return box_muller(w[0], w[1], 0);
    case 1: return box_muller(w[0], w[1], 1);
    case 2: return box_muller(w[2], w[3], 0);
    default: return box_muller(w[2], w[3], 1);
    }
}

double oracle_illumination(const oracle_pair *p, int64_t i, int64_t j)
{
    double sx = sin(ORACLE_PI * ((double)j + 0.5) / (double)p->width);
    double sy = sin(ORACLE_PI * ((double)i + 0.5) / (double)p->height);
    return p->illum_min + (p->illum_max - p->illum_min) * (sx * sx) * (sy * sy);
}

int32_t oracle_blur_radius(double blur_sigma)
{
    if (!(blur_sigma > 0.0)) return 0;
    return (int32_t)ceil(3.0 * blur_sigma);
}

/* frame: 0 or 1.  S, B: [H][W] FP64.  Q: [H][W] codes or NULL. */
int oracle_epilogue(const oracle_pair *p, int32_t frame, const double *S, double *B, uint32_t *Q)
{
    const long H = p->height, W = p->width;
    double *A = (double *)malloc(sizeof(double) * (size_t)(H * W));
    if (!A) return -1;
    for (long i = 0; i < H; ++i)
        for (long j = 0; j < W; ++j) {
            double val = oracle_illumination(p, i, j) * S[i * W + j];
            if (p->noise_sigma != 0.0)
                val += p->noise_sigma * oracle_noise(p->seed, p->pair_id, frame, i * W + j);
            A[i * W + j] = val;
        }
    int32_t R = oracle_blur_radius(p->blur_sigma);
    if (R > 0) {
        double *w = (double *)malloc(sizeof(double) * (size_t)(2 * R + 1));
        double *T = (double *)malloc(sizeof(double) * (size_t)(H * W));
        if (!w || !T) { free(A); free(w); free(T); return -1; }
        double sum = 0.0;
        for (int k = -R; k <= R; ++k) {
            w[k + R] = exp(-(double)(k * k) / (2.0 * p->blur_sigma * p->blur_sigma));
            sum += w[k + R];
        }
        for (int k = 0; k <= 2 * R; ++k) w[k] /= sum;
        for (long i = 0; i < H; ++i)           /* horizontal pass */
            for (long j = 0; j < W; ++j) {
                double acc = 0.0;
                for (int k = -R; k <= R; ++k)
                    acc += w[k + R] * A[i * W + clampl(j + k, 0, W - 1)];
                T[i * W + j] = acc;
            }
        for (long i = 0; i < H; ++i)           /* vertical pass */
            for (long j = 0; j < W; ++j) {
                double acc = 0.0;
                for (int k = -R; k <= R; ++k)
                    acc += w[k + R] * T[clampl(i + k, 0, H - 1) * W + j];
                B[i * W + j] = acc;
            }
        free(w);
        free(T);
    } else {
        memcpy(B, A, sizeof(double) * (size_t)(H * W));
    }
    free(A);
    if (Q && p->quant_bits > 0) {
        /* Q = clamp(rint(B M), 0, M) on the FP64 value B: rint rounds half to
           even in the default rounding mode (reading C10) */
        double M = (double)((1u << p->quant_bits) - 1u);
        for (long k = 0; k < H * W; ++k) {
            double q = rint(B[k] * M);
            Q[k] = q < 0.0 ? 0u : (q > M ? (uint32_t)M : (uint32_t)q);
        }
    }
    return 0;
}

/*
 * Render one pair.  S (nullable) receives the splatted frames before the
 * epilogue, B the frames after it, Q (nullable) the quantised codes, parts
 * (nullable) the particle table of oracle_particles.  Frame f occupies
 * [f*H*W, (f+1)*H*W) of each output.
 */
int oracle_render_pair3(const oracle_pair *p, const float *flow, const float *wgrid, double *S, double *B,
                        uint32_t *Q, double *parts, int32_t splat_mode);

int oracle_render_pair(const oracle_pair *p, const float *flow, double *S, double *B, uint32_t *Q,
                       double *parts, int32_t splat_mode)
{
    return oracle_render_pair3(p, flow, NULL, S, B, Q, parts, splat_mode);
}

/* oracle_render_pair with out-of-plane motion: wgrid (nullable) [flow_h][flow_w] (R9). */
int oracle_render_pair3(const oracle_pair *p, const float *flow, const float *wgrid, double *S, double *B,
                        uint32_t *Q, double *parts, int32_t splat_mode)
{
    const int64_t HW = (int64_t)p->height * p->width;
    const int64_t n = p->n_particles;
    double *tab = (double *)malloc(sizeof(double) * (size_t)(8 * (n > 0 ? n : 1)));
    double *xy = (double *)malloc(sizeof(double) * (size_t)(4 * (n > 0 ? n : 1)));
    double *s = S ? S : (double *)malloc(sizeof(double) * (size_t)(2 * HW));
    if (!tab || !xy || !s) { free(tab); free(xy); if (!S) free(s); return -1; }
    oracle_particles(p, flow, tab);
    memset(s, 0, sizeof(double) * (size_t)(2 * HW));
    const int general = !oracle_round_particles(p) || p->jitter_d != 0.0 || p->jitter_i != 0.0 ||
                        p->jitter_rho != 0.0 || p->hide_prob > 0.0 || wgrid != NULL;
    if (general) {
        double *sh = (double *)malloc(sizeof(double) * (size_t)(10 * (n > 0 ? n : 1)));
        double *rows = (double *)malloc(sizeof(double) * (size_t)(6 * (n > 0 ? n : 1)));
        if (!sh || !rows) { free(sh); free(rows); free(tab); free(xy); if (!S) free(s); return -1; }
        for (int64_t i = 0; i < n; ++i) {
            oracle_attr a;
            oracle_shape sp[2];
            particle_attr(p, (uint32_t)i, &a);
            double gain2 = a.gain;
            if (wgrid) {  /* frame-2 position and depth moved together (R9) */
                double x1, y1, z1;
                oracle_advect3(p, flow, wgrid, a.x0, a.y0, a.z, &x1, &y1, &z1);
                tab[8 * i + 6] = x1;
                tab[8 * i + 7] = y1;
                gain2 = oracle_sheet_gain(p, z1);
            }
            particle_shapes(p, (uint32_t)i, &a, gain2, sp);
            for (int f = 0; f < 2; ++f) {
                double *o = sh + 10 * i + 5 * f;
                o[0] = sp[f].dx; o[1] = sp[f].dy; o[2] = sp[f].rho; o[3] = sp[f].ieff; o[4] = (double)sp[f].visible;
            }
        }
        for (int f = 0; f < 2; ++f) {
            int64_t m = 0;
            for (int64_t i = 0; i < n; ++i) {
                const double *q = sh + 10 * i + 5 * f;
                if (q[4] == 0.0) continue; /* hidden from this frame */
                double *r = rows + 6 * m++;
                r[0] = tab[8 * i + (f ? 6 : 0)];
                r[1] = tab[8 * i + (f ? 7 : 1)];
                r[2] = q[0]; r[3] = q[1]; r[4] = q[2]; r[5] = q[3];
            }
            oracle_splat_shapes(p->height, p->width, rows, m, splat_mode, s + f * HW);
            oracle_epilogue(p, f, s + f * HW, B + f * HW, Q ? Q + f * HW : NULL);
        }
        free(sh);
        free(rows);
        if (parts) memcpy(parts, tab, sizeof(double) * (size_t)(8 * n));
        free(tab);
        free(xy);
        if (!S) free(s);
        return 0;
    }
    for (int f = 0; f < 2; ++f) {
        for (int64_t i = 0; i < n; ++i) {
            xy[4 * i] = tab[8 * i + (f ? 6 : 0)];
            xy[4 * i + 1] = tab[8 * i + (f ? 7 : 1)];
            xy[4 * i + 2] = tab[8 * i + 2];
            xy[4 * i + 3] = tab[8 * i + 5];
        }
        oracle_splat(p->height, p->width, xy, n, splat_mode, s + f * HW);
        oracle_epilogue(p, f, s + f * HW, B + f * HW, Q ? Q + f * HW : NULL);
    }
    if (parts) memcpy(parts, tab, sizeof(double) * (size_t)(8 * n));
    free(tab);
    free(xy);
    if (!S) free(s);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* intensity-histogram matching of a quantised frame (R10)                  */
/* ------------------------------------------------------------------------ */
/*
 * R10: the paper adjusts generated images to a user-specified intensity
 * histogram (Section 2, end of "Mathematical model").  Reading: histogram
 * specification on the quantised codes.  With the frame's code counts h_s
 * (N pixels) and the target counts h_t (T in all), cumulative C_s, C_t, code
 * c becomes the smallest t with C_t(t) / T >= C_s(c) / N, compared exactly as
 * C_t(t) N >= C_s(c) T.  n_codes = M + 1.  codes: n pixels, rewritten in place.
 */
int oracle_match_histogram(uint32_t *codes, int64_t n, int32_t n_codes, const uint64_t *target)
{
    uint64_t *hs = (uint64_t *)calloc((size_t)n_codes, sizeof(uint64_t));
    uint32_t *map = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n_codes);
    if (!hs || !map) { free(hs); free(map); return -1; }
    for (int64_t k = 0; k < n; ++k) hs[codes[k]] += 1;
    uint64_t T = 0;
    for (int32_t t = 0; t < n_codes; ++t) T += target[t];
    uint64_t cs = 0;
    for (int32_t c = 0; c < n_codes; ++c) {
        cs += hs[c];
        uint64_t ct = 0;
        int32_t t = 0;
        for (; t < n_codes; ++t) {
            ct += target[t];
            if ((unsigned __int128)ct * (uint64_t)n >= (unsigned __int128)cs * T) break;
        }
        map[c] = (uint32_t)(t < n_codes ? t : n_codes - 1);
    }
    for (int64_t k = 0; k < n; ++k) codes[k] = map[codes[k]];
    free(hs);
    free(map);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* forward with given particles, and its adjoint (gradients)                */
/* ------------------------------------------------------------------------ */
/*
 * The differentiable form of the render: frames S_f = splat of the particles
 * at their frame-f positions, B_f = L * S_f (no noise, no blur).  parts_in
 * holds (x0, y0, d) per particle, or is NULL for the seeded values; the
 * intensities always come from the seeded streams.
 */
static void particle_inputs(const oracle_pair *p, const double *parts_in, int64_t i, double *x0, double *y0,
                            double *d, double *ieff)
{
    oracle_attr a;
    particle_attr(p, (uint32_t)i, &a);
    *x0 = parts_in ? parts_in[3 * i] : a.x0;
    *y0 = parts_in ? parts_in[3 * i + 1] : a.y0;
    *d = parts_in ? parts_in[3 * i + 2] : a.d;
    *ieff = a.ieff;
}

/* B[2][H][W] = L * S of both frames. */
int oracle_render_from(const oracle_pair *p, const float *flow, const double *parts_in, double *B)
{
    const int64_t HW = (int64_t)p->height * p->width, n = p->n_particles;
    double *xy = (double *)malloc(sizeof(double) * (size_t)(8 * (n > 0 ? n : 1)));
    if (!xy) return -1;
    for (int64_t i = 0; i < n; ++i) {
        double x0, y0, d, ie, x1, y1;
        particle_inputs(p, parts_in, i, &x0, &y0, &d, &ie);
        oracle_advect(p, flow, x0, y0, &x1, &y1);
        double *r = xy + 8 * i;
        r[0] = x0; r[1] = y0; r[2] = d; r[3] = ie; r[4] = x1; r[5] = y1; r[6] = d; r[7] = ie;
    }
    memset(B, 0, sizeof(double) * (size_t)(2 * HW));
    for (int f = 0; f < 2; ++f) {
        double *tmp = (double *)malloc(sizeof(double) * (size_t)(4 * (n > 0 ? n : 1)));
        if (!tmp) { free(xy); return -1; }
        for (int64_t i = 0; i < n; ++i) {
            tmp[4 * i] = xy[8 * i + (f ? 4 : 0)];
            tmp[4 * i + 1] = xy[8 * i + (f ? 5 : 1)];
            tmp[4 * i + 2] = xy[8 * i + 2];
            tmp[4 * i + 3] = xy[8 * i + 3];
        }
        oracle_splat(p->height, p->width, tmp, n, 0, B + f * HW);
        free(tmp);
        for (int64_t i = 0; i < p->height; ++i)
            for (int64_t j = 0; j < p->width; ++j) B[f * HW + i * p->width + j] *= oracle_illumination(p, i, j);
    }
    free(xy);
    return 0;
}

static double gauss_pdf(double t) { return exp(-0.5 * t * t) / 2.50662827463100050242; }

/* Velocity, its Jacobian dU/dp (J[0] = du/dx, J[1] = du/dy, J[2] = dv/dx,
 * J[3] = dv/dy) and the four (node, weight) pairs of the bilinear stencil. */
static void velocity_jac(const float *flow, int32_t gh, int32_t gw, int32_t height, int32_t width, double x,
                         double y, double *u, double *v, double J[4], long node[4], double wgt[4])
{
    double gx = x * (double)gw / (double)width - 0.5;
    double gy = y * (double)gh / (double)height - 0.5;
    double fl = floor(gx), fk = floor(gy);
    double tx = gx - fl, ty = gy - fk;
    long l0 = clampl((long)fl, 0, gw - 1), l1 = clampl((long)fl + 1, 0, gw - 1);
    long k0 = clampl((long)fk, 0, gh - 1), k1 = clampl((long)fk + 1, 0, gh - 1);
    double out[2];
    for (int c = 0; c < 2; ++c) {
        double a = flow[(k0 * gw + l0) * 2 + c], b = flow[(k0 * gw + l1) * 2 + c];
        double e = flow[(k1 * gw + l0) * 2 + c], f = flow[(k1 * gw + l1) * 2 + c];
        double top = a + tx * (b - a), bot = e + tx * (f - e);
        out[c] = top + ty * (bot - top);
        J[2 * c] = ((1.0 - ty) * (b - a) + ty * (f - e)) * (double)gw / (double)width;
        J[2 * c + 1] = (bot - top) * (double)gh / (double)height;
    }
    *u = out[0];
    *v = out[1];
    node[0] = k0 * gw + l0; wgt[0] = (1.0 - tx) * (1.0 - ty);
    node[1] = k0 * gw + l1; wgt[1] = tx * (1.0 - ty);
    node[2] = k1 * gw + l0; wgt[2] = (1.0 - tx) * ty;
    node[3] = k1 * gw + l1; wgt[3] = tx * ty;
}

/* Adds w * lam (per velocity component) to the stencil's nodes. */
static void scatter_flow(double *grad_flow, const long node[4], const double wgt[4], double lx, double ly)
{
    for (int n = 0; n < 4; ++n) {
        grad_flow[node[n] * 2] += wgt[n] * lx;
        grad_flow[node[n] * 2 + 1] += wgt[n] * ly;
    }
}

/* Reverse sweep of the advection: given dL/d(frame-2 position), returns
 * dL/d(start position) and adds dL/dflow (RK4 or Euler, as the forward). */
static void advect_adjoint(const oracle_pair *p, const float *flow, double x0, double y0, double lx, double ly,
                           double *gx0, double *gy0, double *grad_flow)
{
    const int n = p->n_substeps;
    const double h = p->dt / (double)n;
    double *xs = (double *)malloc(sizeof(double) * (size_t)(2 * (n + 1)));
    double x = x0, y = y0;
    for (int s = 0; s < n; ++s) {  /* forward, keeping the substep starts */
        xs[2 * s] = x;
        xs[2 * s + 1] = y;
        oracle_pair one = *p;
        one.n_substeps = 1;
        one.dt = h;
        oracle_advect(&one, flow, x, y, &x, &y);
    }
    for (int s = n - 1; s >= 0; --s) {
        const double px = xs[2 * s], py = xs[2 * s + 1];
        double u1, v1, J1[4], w1[4];
        long n1[4];
        velocity_jac(flow, p->flow_h, p->flow_w, p->height, p->width, px, py, &u1, &v1, J1, n1, w1);
        if (p->integrator == 1) {
            scatter_flow(grad_flow, n1, w1, h * lx, h * ly);
            const double ax = lx + h * (J1[0] * lx + J1[2] * ly);
            const double ay = ly + h * (J1[1] * lx + J1[3] * ly);
            lx = ax;
            ly = ay;
            continue;
        }
        double u2, v2, J2[4], w2[4], u3, v3, J3[4], w3[4], u4, v4, J4[4], w4[4];
        long n2[4], n3[4], n4[4];
        velocity_jac(flow, p->flow_h, p->flow_w, p->height, p->width, px + 0.5 * h * u1, py + 0.5 * h * v1, &u2,
                     &v2, J2, n2, w2);
        velocity_jac(flow, p->flow_h, p->flow_w, p->height, p->width, px + 0.5 * h * u2, py + 0.5 * h * v2, &u3,
                     &v3, J3, n3, w3);
        velocity_jac(flow, p->flow_h, p->flow_w, p->height, p->width, px + h * u3, py + h * v3, &u4, &v4, J4, n4,
                     w4);
        /* p+ = p + h/6 (k1 + 2 k2 + 2 k3 + k4), k_m = U(q_m) */
        const double k4x = h / 6.0 * lx, k4y = h / 6.0 * ly;
        const double k3x = h / 3.0 * lx + h * (J4[0] * k4x + J4[2] * k4y);
        const double k3y = h / 3.0 * ly + h * (J4[1] * k4x + J4[3] * k4y);
        const double k2x = h / 3.0 * lx + 0.5 * h * (J3[0] * k3x + J3[2] * k3y);
        const double k2y = h / 3.0 * ly + 0.5 * h * (J3[1] * k3x + J3[3] * k3y);
        const double k1x = h / 6.0 * lx + 0.5 * h * (J2[0] * k2x + J2[2] * k2y);
        const double k1y = h / 6.0 * ly + 0.5 * h * (J2[1] * k2x + J2[3] * k2y);
        scatter_flow(grad_flow, n1, w1, k1x, k1y);
        scatter_flow(grad_flow, n2, w2, k2x, k2y);
        scatter_flow(grad_flow, n3, w3, k3x, k3y);
        scatter_flow(grad_flow, n4, w4, k4x, k4y);
        const double ax = lx + (J1[0] * k1x + J1[2] * k1y) + (J2[0] * k2x + J2[2] * k2y) +
                          (J3[0] * k3x + J3[2] * k3y) + (J4[0] * k4x + J4[2] * k4y);
        const double ay = ly + (J1[1] * k1x + J1[3] * k1y) + (J2[1] * k2x + J2[3] * k2y) +
                          (J3[1] * k3x + J3[3] * k3y) + (J4[1] * k4x + J4[3] * k4y);
        lx = ax;
        ly = ay;
    }
    free(xs);
    *gx0 = lx;
    *gy0 = ly;
}

/* Per-axis pixel mass and its derivatives w.r.t. the centre and sigma. */
static void mass_derivs(double c, double sigma, int64_t j, double *m, double *dm_dc, double *dm_ds)
{
    const double a = ((double)j - c) / sigma, b = ((double)j + 1.0 - c) / sigma;
    *m = oracle_pixel_mass(c, sigma, j);
    *dm_dc = (gauss_pdf(a) - gauss_pdf(b)) / sigma;
    *dm_ds = (a * gauss_pdf(a) - b * gauss_pdf(b)) / sigma;
}

/* Gradient of one frame's splat against G at (x, y): (dL/dx, dL/dy, dL/dsigma). */
static void splat_adjoint(const oracle_pair *p, const double *G, double x, double y, double d, double ieff,
                          double g[3])
{
    const double sigma = d / 4.0, amp = ieff * 2.0 * ORACLE_PI * sigma * sigma;
    long j0 = (long)floor(x - 1.5 * d), j1 = (long)floor(x + 1.5 * d);
    long i0 = (long)floor(y - 1.5 * d), i1 = (long)floor(y + 1.5 * d);
    if (j0 < 0) j0 = 0;
    if (i0 < 0) i0 = 0;
    if (j1 > p->width - 1) j1 = p->width - 1;
    if (i1 > p->height - 1) i1 = p->height - 1;
    g[0] = g[1] = g[2] = 0.0;
    for (long i = i0; i <= i1; ++i) {
        double ey, dey, dsy;
        mass_derivs(y, sigma, i, &ey, &dey, &dsy);
        for (long j = j0; j <= j1; ++j) {
            double ex, dex, dsx;
            mass_derivs(x, sigma, j, &ex, &dex, &dsx);
            const double gl = G[i * p->width + j] * oracle_illumination(p, i, j);
            g[0] += gl * amp * dex * ey;
            g[1] += gl * amp * ex * dey;
            g[2] += gl * (amp * (dsx * ey + ex * dsy) + 2.0 * amp / sigma * ex * ey);
        }
    }
}

/*
 * Gradients of L = sum_f sum_ij G[f][i][j] * B_f(i, j) (B from
 * oracle_render_from): grad_flow [flow_h][flow_w][2] is added to, grad_parts
 * [N][3] = (dL/dx0, dL/dy0, dL/dd) is overwritten (either may be NULL).
 */
int oracle_backward(const oracle_pair *p, const float *flow, const double *parts_in, const double *G,
                    double *grad_flow, double *grad_parts)
{
    const int64_t HW = (int64_t)p->height * p->width;
    double *gf = grad_flow;
    if (!gf) {
        gf = (double *)calloc((size_t)(2 * p->flow_h * p->flow_w), sizeof(double));
        if (!gf) return -1;
    }
    for (int64_t i = 0; i < p->n_particles; ++i) {
        double x0, y0, d, ie, x1, y1, g1[3], g2[3], ax, ay;
        particle_inputs(p, parts_in, i, &x0, &y0, &d, &ie);
        oracle_advect(p, flow, x0, y0, &x1, &y1);
        splat_adjoint(p, G, x0, y0, d, ie, g1);
        splat_adjoint(p, G + HW, x1, y1, d, ie, g2);
        advect_adjoint(p, flow, x0, y0, g2[0], g2[1], &ax, &ay, gf);
        if (grad_parts) {
            grad_parts[3 * i] = g1[0] + ax;
            grad_parts[3 * i + 1] = g1[1] + ay;
            grad_parts[3 * i + 2] = (g1[2] + g2[2]) / 4.0; /* sigma = d / 4 */
        }
    }
    if (!grad_flow) free(gf);
    return 0;
}
