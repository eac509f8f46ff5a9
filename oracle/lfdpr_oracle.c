/*
 * CPU oracle for light field display point rendering (LFDPR).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or call
 * this file: only the tests, the package's smoke check and the benchmark's CPU
 * baseline do. It shares no code, header, table or constant generator with
 * the CUDA library; the two meet only through the seeded inputs.
 *
 * What it computes, step by step in the paper's order (Sec. 3 and Sec. 4):
 *   1. per-frame model transform (the scenes rotate every frame, Sec. 5.1);
 *   2. vertex visibility against every LFD view (Sec. 3, pipeline overview);
 *   3. the triangle's sampling frame aligned with the views' horizontal and
 *      vertical axes (Sec. 3.1, T_align);
 *   4. LFD-biased horizontal and vertical sample spacings from pixel edges
 *      reverse-projected at the closest point of the triangle (Sec. 3.1, Fig. 5);
 *   5. texture-based sampling, Eq. 1-3 (Sec. 3.1);
 *   6. multiview-mipmap setup, Eq. 4-7 (Sec. 3.3);
 *   7. one point per sampling-lattice cell overlapping the triangle;
 *   8. tv_min / tv_max fetched from the mip chain at LOD_min / LOD_max (Sec. 3.3);
 *   9. EPR splatting of every point into every view: the point's cell is
 *      projected and only pixels inside both the cell and the triangle are
 *      written, with a 64-bit depth|id minimum per view pixel (Sec. 3.2, Sec. 5.1);
 *  10. per-view, per-splat texture interpolation, Eq. 8-9 (Sec. 3.3);
 *  11. angular supersampling, reconstruction, crosstalk (Sec. 4);
 *  12. lenticular interleave into the elemental image array (Sec. 4).
 *
 * Floating point: IEEE binary32 throughout, every fused multiply-add written
 * as fmaf(), compiled with -ffp-contract=off so no other contraction happens.
 * Where the paper leaves a choice open, the reading taken is stated at the
 * step. The splat bounding box is computed in double with a one-pixel pad; it
 * only limits which pixels are tested and never decides one.
 *
 * Parity pins (tests, not this file): closed-form point counts, brute-force
 * ray casting (orc_raycast below, double precision), constant and
 * checkerboard textures, log2 against the C library, interleave histograms.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* -------------------------------------------------------------------------- */
/* Types                                                                       */
/* -------------------------------------------------------------------------- */

typedef struct {
    int32_t n_views, view_w, view_h;
    float cone_deg, view_dist, focal_w, focal_h, near_z, far_z, bias_h, bias_v;
    int32_t panel_w, panel_h;
    float lens_pitch_px, slant, phase_offset;
    int32_t recon;          /* 0 none, 1 2x angular + tent, 2 2x angular + Gaussian, 3 Gaussian */
    float crosstalk;
    const float *jitter;    /* NULL, or per rendered view u in [0, 1]: its place in its interval */
    const float *samples;   /* recon 2, 3: n_samples x (dx, dy in view pixels, dphi in display views) */
    int32_t n_samples;
    int32_t ss_level;       /* spatial supersampling: views rendered at 2^ss_level x the output size */
} orc_display;

/* Per-triangle record, written by orc_setup as ORC_TRI_FLOATS floats. */
enum {
    T_LIVE = 0,            /* 1 if the triangle emits points */
    T_P0 = 1,              /* 3: transformed first vertex */
    T_N = 4,               /* 3: unit normal */
    T_EU = 7,              /* 3: horizontal sampling axis u-hat */
    T_EV = 10,             /* 3: vertical sampling axis v-hat */
    T_UMIN = 13, T_VMIN = 14,
    T_A1 = 15, T_B1 = 16, T_A2 = 17, T_B2 = 18,   /* unshifted 2-D coords of v1, v2 */
    T_U = 19,              /* 3: shifted 2-D u of v0, v1, v2 */
    T_V = 22,              /* 3: shifted 2-D v */
    T_AWS = 25, T_ATS = 26, T_NTEX = 27, T_SIZE_UV = 28,
    T_DMIN = 29, T_DMAX = 30, T_SU = 31, T_SV = 32,
    T_VPUV_MIN = 33, T_VPUV_MAX = 34, T_SPL_UV = 35,
    T_LOD_MIN = 36, T_LOD_MAX = 37,
    T_S0 = 38, T_SGU = 39, T_SGV = 40, T_T0 = 41, T_TGU = 42, T_TGV = 43,
    T_TEX = 44, T_UMAX = 45, T_VMAX = 46,
    ORC_TRI_FLOATS = 48
};

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_EOVERFLOW = 4 };

/* Largest lattice index along either axis (cells are stored as u16 pairs). */
#define ORC_MAX_CELL 65535

/* -------------------------------------------------------------------------- */
/* Small float helpers (each is the plain formula with its rounding spelled out) */
/* -------------------------------------------------------------------------- */

static float dot3(const float *a, const float *b) {
    return fmaf(a[0], b[0], fmaf(a[1], b[1], a[2] * b[2]));
}

static void cross3(const float *a, const float *b, float *o) {
    o[0] = fmaf(a[1], b[2], -(a[2] * b[1]));
    o[1] = fmaf(a[2], b[0], -(a[0] * b[2]));
    o[2] = fmaf(a[0], b[1], -(a[1] * b[0]));
}

/* Signed doubled area of (p, r, q): the 2-D edge function of edge p->r at q. */
static float edge2(float px, float py, float rx, float ry, float qx, float qy) {
    return fmaf(rx - px, qy - py, -((ry - py) * (qx - px)));
}

/* Reciprocal squared length of segment p-r (0 for a zero-length segment). */
static float seg_inv_len2(float px, float py, float rx, float ry) {
    float ex = rx - px, ey = ry - py;
    float ee = fmaf(ex, ex, ey * ey);
    return ee > 0.0f ? 1.0f / ee : 0.0f;
}

/* Squared distance from q to segment p-r; inv_ee = seg_inv_len2(p, r). The
 * closest point's parameter along the segment is (q-p).(r-p) / |r-p|^2,
 * clamped to [0, 1]. */
static float segd2(float px, float py, float rx, float ry, float inv_ee, float qx, float qy) {
    float ex = rx - px, ey = ry - py, wx = qx - px, wy = qy - py;
    float t = fmaf(wx, ex, wy * ey) * inv_ee;
    t = fminf(fmaxf(t, 0.0f), 1.0f);
    float dx = fmaf(-t, ex, wx), dy = fmaf(-t, ey, wy);
    return fmaf(dx, dx, dy * dy);
}

static int inside3(float w0, float w1, float w2) {
    return (w0 >= 0.0f && w1 >= 0.0f && w2 >= 0.0f) ||
           (w0 <= 0.0f && w1 <= 0.0f && w2 <= 0.0f);
}

static uint32_t fbits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }
static float bitsf(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }

/*
 * log2 for Eq. 6-7. Neither side has a correctly rounded library log2, so both
 * write this one method: split x = m * 2^e from the bits, fold m into
 * [sqrt(1/2), sqrt(2)], and take ln m = 2 atanh(z), z = (m-1)/(m+1), from the
 * Taylor series of atanh truncated after z^9/9 (|z| < 0.172 so the first
 * dropped term is below 2^-28); log2 x = e + ln m / ln 2.
 */
float orc_log2f(float x) {
    if (isnan(x)) return x;
    if (x <= 0.0f) return -INFINITY;
    if (isinf(x)) return INFINITY;
    int e;
    uint32_t b = fbits(x);
    if ((b >> 23) == 0) {               /* subnormal: scale into the normal range */
        b = fbits(x * 16777216.0f);
        e = (int)(b >> 23) - 127 - 24;
    } else {
        e = (int)(b >> 23) - 127;
    }
    float m = bitsf((b & 0x007fffffu) | 0x3f800000u);
    if (m > 1.41421356f) { m = m * 0.5f; e += 1; }
    float z = (m - 1.0f) / (m + 1.0f);
    float z2 = z * z;
    float p = fmaf(z2, (float)(1.0 / 9.0), (float)(1.0 / 7.0));
    p = fmaf(z2, p, (float)(1.0 / 5.0));
    p = fmaf(z2, p, (float)(1.0 / 3.0));
    p = fmaf(z2, p, 1.0f);
    float ln_m = (2.0f * z) * p;
    return fmaf(ln_m, (float)(1.0 / 0.69314718055994530942), (float)e);
}

/* -------------------------------------------------------------------------- */
/* Views (Sec. 3: views defined by the LFD; Sec. 4: angular supersampling)      */
/* -------------------------------------------------------------------------- */

int orc_n_render_views(const orc_display *d) {
    return d->recon == 1 || d->recon == 2 ? 2 * d->n_views : d->n_views;
}

/*
 * Eye x positions. The N display views sit at the centres of N equal angular
 * intervals of the viewing cone, on the line y = 0, z = D. With angular
 * supersampling (recon 1 or 2) Sec. 4 projects the splats into twice as many
 * views, placed randomly inside their intervals: rendered view m sits at the
 * fraction u_m of the half-interval [(m + 1/2), (m + 3/2)] / 2N of the cone
 * (u_m = d->jitter[m], or 1/2 without jitter: then the even views fall on the
 * N display-view centres). Without supersampling view k sits at the
 * fraction u_k of its interval (1/2: the centre).
 */
static double jitter_of(const orc_display *d, int m) {
    return d->jitter ? (double)d->jitter[m] : 0.5;
}

void orc_eyes(const orc_display *d, float *ex) {
    int nr = orc_n_render_views(d);
    double cone = d->cone_deg, D = d->view_dist;
    for (int k = 0; k < nr; k++) {
        double deg = nr == 2 * d->n_views ? -cone / 2.0 + cone * (k + 0.5 + jitter_of(d, k)) / (2.0 * d->n_views)
                                          : -cone / 2.0 + cone * (k + jitter_of(d, k)) / d->n_views;
        ex[k] = (float)(D * tan(deg * M_PI / 180.0));
    }
}

/* Position of rendered view m on the display-view axis (display view k
 * covers [k, k+1), its centre k + 1/2), the reading of the angle above. */
float orc_view_pos(const orc_display *d, int m) {
    int nr = orc_n_render_views(d);
    return nr == 2 * d->n_views ? (float)((m + 0.5 + jitter_of(d, m)) / 2.0) : (float)(m + jitter_of(d, m));
}

/* -------------------------------------------------------------------------- */
/* Mip chain (Sec. 3.3 relies on the hardware mipmap; here: 2x2 box, rounded)   */
/* -------------------------------------------------------------------------- */

static int ilog2u(uint32_t v) { int l = 0; while ((1u << l) < v) l++; return l; }

int orc_mip_levels(uint32_t w, uint32_t h) {
    return ilog2u(w > h ? w : h) + 1;
}

size_t orc_mip_bytes(uint32_t w, uint32_t h) {
    size_t n = 0;
    int L = orc_mip_levels(w, h);
    for (int l = 0; l < L; l++) {
        uint32_t lw = w >> l ? w >> l : 1, lh = h >> l ? h >> l : 1;
        n += (size_t)lw * lh * 4;
    }
    return n;
}

/* chain = level 0 followed by every coarser level, each row-major RGBA8.
 * Texel (x, y) of level l+1 is the rounded mean (a+b+c+d+2)>>2 of texels
 * (2x..2x+1, 2y..2y+1) of level l, indices clamped to the level. */
void orc_build_mips(const uint8_t *level0, uint32_t w, uint32_t h, uint8_t *chain) {
    memcpy(chain, level0, (size_t)w * h * 4);
    int L = orc_mip_levels(w, h);
    const uint8_t *src = chain;
    uint32_t sw = w, sh = h;
    uint8_t *dst = chain + (size_t)w * h * 4;
    for (int l = 1; l < L; l++) {
        uint32_t dw = sw > 1 ? sw / 2 : 1, dh = sh > 1 ? sh / 2 : 1;
        for (uint32_t y = 0; y < dh; y++) {
            uint32_t y0 = 2 * y < sh ? 2 * y : sh - 1, y1 = 2 * y + 1 < sh ? 2 * y + 1 : sh - 1;
            for (uint32_t x = 0; x < dw; x++) {
                uint32_t x0 = 2 * x < sw ? 2 * x : sw - 1, x1 = 2 * x + 1 < sw ? 2 * x + 1 : sw - 1;
                for (int c = 0; c < 4; c++) {
                    unsigned s = src[((size_t)y0 * sw + x0) * 4 + c] + src[((size_t)y0 * sw + x1) * 4 + c] +
                                 src[((size_t)y1 * sw + x0) * 4 + c] + src[((size_t)y1 * sw + x1) * 4 + c];
                    dst[((size_t)y * dw + x) * 4 + c] = (uint8_t)((s + 2) >> 2);
                }
            }
        }
        src = dst;
        dst += (size_t)dw * dh * 4;
        sw = dw;
        sh = dh;
    }
}

/* Bilinear sample of one level with wrap addressing; texel centres at (k+1/2)/w. */
static void bilinear(const uint8_t *lvl, uint32_t w, uint32_t h, float s, float t, float out[4]) {
    if (!isfinite(s)) s = 0.0f;
    if (!isfinite(t)) t = 0.0f;
    float fs = s - floorf(s), ft = t - floorf(t);
    float x = fmaf(fs, (float)w, -0.5f), y = fmaf(ft, (float)h, -0.5f);
    float xf = floorf(x), yf = floorf(y);
    float fx = x - xf, fy = y - yf;
    uint32_t ix0 = (uint32_t)(int)xf & (w - 1), iy0 = (uint32_t)(int)yf & (h - 1);
    uint32_t ix1 = (ix0 + 1) & (w - 1), iy1 = (iy0 + 1) & (h - 1);
    const uint8_t *t00 = lvl + ((size_t)iy0 * w + ix0) * 4, *t10 = lvl + ((size_t)iy0 * w + ix1) * 4;
    const uint8_t *t01 = lvl + ((size_t)iy1 * w + ix0) * 4, *t11 = lvl + ((size_t)iy1 * w + ix1) * 4;
    for (int c = 0; c < 4; c++) {
        float a = t00[c], b = t10[c], cc = t01[c], dd = t11[c];
        float top = fmaf(fx, b - a, a);
        float bot = fmaf(fx, dd - cc, cc);
        out[c] = fmaf(fy, bot - top, top);
    }
}

static uint8_t to_u8(float v) {
    float r = rintf(v);
    if (!(r >= 0.0f)) r = 0.0f;
    if (r > 255.0f) r = 255.0f;
    return (uint8_t)r;
}

/* Trilinear fetch at a level of detail (Sec. 3.3, the tv_min / tv_max fetch):
 * LOD clamped to [0, L_max], level floor(LOD), blended to the next level by
 * the fraction, FP32 weights, then rounded half-to-even to RGBA8. */
void orc_trilinear(const uint8_t *chain, uint32_t w, uint32_t h, float s, float t,
                   float lod, uint8_t out[4]) {
    int L = orc_mip_levels(w, h) - 1;
    lod = fminf(fmaxf(lod, 0.0f), (float)L);
    int l = (int)floorf(lod);
    float f = lod - (float)l;
    const uint8_t *p = chain;
    for (int k = 0; k < l; k++) {
        uint32_t lw = w >> k ? w >> k : 1, lh = h >> k ? h >> k : 1;
        p += (size_t)lw * lh * 4;
    }
    uint32_t lw = w >> l ? w >> l : 1, lh = h >> l ? h >> l : 1;
    float c0[4], c1[4];
    bilinear(p, lw, lh, s, t, c0);
    if (f > 0.0f && l < L) {
        const uint8_t *q = p + (size_t)lw * lh * 4;
        uint32_t nw = lw > 1 ? lw / 2 : 1, nh = lh > 1 ? lh / 2 : 1;
        bilinear(q, nw, nh, s, t, c1);
        for (int c = 0; c < 4; c++) out[c] = to_u8(fmaf(f, c1[c] - c0[c], c0[c]));
    } else {
        for (int c = 0; c < 4; c++) out[c] = to_u8(c0[c]);
    }
}

/* -------------------------------------------------------------------------- */
/* Per-frame model transform                                                    */
/* -------------------------------------------------------------------------- */

void orc_transform(const float *m, const float *p, float *o) {
    o[0] = fmaf(m[0], p[0], fmaf(m[1], p[1], fmaf(m[2], p[2], m[3])));
    o[1] = fmaf(m[4], p[0], fmaf(m[5], p[1], fmaf(m[6], p[2], m[7])));
    o[2] = fmaf(m[8], p[0], fmaf(m[9], p[1], fmaf(m[10], p[2], m[11])));
}

/* -------------------------------------------------------------------------- */
/* Triangle setup: visibility, T_align frame, spacings, Eq. 1-7, point count    */
/* -------------------------------------------------------------------------- */

/*
 * Vertex visibility (Sec. 3): a triangle is dropped when, for every view, all
 * three vertices lie outside one common plane of that view's frustum. The
 * frustum of view k has apex E_k = (Ex_k, 0, D) and passes through the focal
 * rectangle [-fw/2, fw/2] x [-fh/2, fh/2] at z = 0; near and far bound the
 * depth D - z. Each plane is the linear form below, negative outside.
 */
static int culled(const orc_display *d, const float *ex, int nr, float P[3][3]) {
    float D = d->view_dist, fw2 = 0.5f * d->focal_w, fh2 = 0.5f * d->focal_h;
    int out_t = 1, out_b = 1, out_n = 1, out_f = 1;
    for (int k = 0; k < 3; k++) {
        float dep = D - P[k][2];
        float top = fmaf(fh2, dep, -(P[k][1] * D));
        float bot = fmaf(P[k][1], D, fh2 * dep);
        out_t &= top < 0.0f;
        out_b &= bot < 0.0f;
        out_n &= dep - d->near_z < 0.0f;
        out_f &= d->far_z - dep < 0.0f;
    }
    if (out_t || out_b || out_n || out_f) return 1;
    for (int v = 0; v < nr; v++) {
        float lx = -fw2 - ex[v], rx = fw2 - ex[v];
        int out_l = 1, out_r = 1;
        for (int k = 0; k < 3; k++) {
            float dep = D - P[k][2];
            float l = fmaf(P[k][0] - ex[v], D, -(lx * dep));
            float r = fmaf(rx, dep, -((P[k][0] - ex[v]) * D));
            out_l &= l < 0.0f;
            out_r &= r < 0.0f;
        }
        if (!(out_l || out_r)) return 0;   /* visible in view v */
    }
    return 1;
}

/*
 * Rows of lattice column i: the cells [i s_u, (i+1) s_u) x [j s_v, (j+1) s_v)
 * of the triangle's shifted 2-D frame whose open interior overlaps the open
 * triangle (reading of iVIR's rasterisation of the aligned triangle: the
 * conservative rule, which makes the splat union hole-free). The triangle's v
 * range over the column slab comes from the vertices inside the slab and the
 * edges' crossings of its two borders.
 */
static int column_rows(const float *T, int i, int *j0, int *j1) {
    float su = T[T_SU], sv = T[T_SV];
    const float *U = T + T_U, *V = T + T_V;
    float a = (float)i * su;
    float b = fminf((float)(i + 1) * su, T[T_UMAX]);
    float lo = INFINITY, hi = -INFINITY;
    for (int k = 0; k < 3; k++) {
        if (U[k] >= a && U[k] <= b) { lo = fminf(lo, V[k]); hi = fmaxf(hi, V[k]); }
    }
    static const int E[3][2] = {{0, 1}, {1, 2}, {2, 0}};
    for (int e = 0; e < 3; e++) {
        int p = E[e][0], r = E[e][1];
        if (U[p] == U[r]) continue;
        float xs[2] = {a, b};
        for (int q = 0; q < 2; q++) {
            float x = xs[q];
            if (x >= fminf(U[p], U[r]) && x <= fmaxf(U[p], U[r])) {
                float tt = (x - U[p]) / (U[r] - U[p]);
                float vx = fmaf(tt, V[r] - V[p], V[p]);
                lo = fminf(lo, vx);
                hi = fmaxf(hi, vx);
            }
        }
    }
    if (lo > hi) { *j0 = 0; *j1 = 0; return 0; }
    *j0 = (int)floorf(lo / sv);
    *j1 = (int)ceilf(hi / sv);
    if (*j1 < *j0) *j1 = *j0;
    return *j1 - *j0;
}

static int n_columns(const float *T) {
    return (int)ceilf(T[T_UMAX] / T[T_SU]);
}

/*
 * orc_setup: steps 1-7 for every triangle. tri_out receives ORC_TRI_FLOATS
 * floats per triangle, counts the number of points it emits. Returns ORC_OK,
 * or ORC_EOVERFLOW if some triangle needs more than ORC_MAX_CELL lattice
 * columns or rows (its count is then 0).
 */
/* mat_tex: NULL (tri_tex holds one texture per triangle), or a material
 * table of n_mat x 4 texture indices (albedo, normal, roughness, metallic;
 * tri_tex then holds material indices): Eq. 1 takes the largest texel count
 * over the material's four textures, and the record's LOD pair is the
 * albedo's (the other textures' pairs follow from Eq. 6-7 in the fetch). */
static int setup_impl(const orc_display *d, const float *xyz, const float *uvs,
                      const uint32_t *idx, const uint32_t *tri_tex, uint32_t n_tris,
                      const uint32_t *tex_wh, uint32_t n_tex, const uint32_t *mat_tex, uint32_t n_mat,
                      const float *model, float *tri_out, uint32_t *counts) {
    const uint32_t n_textures = n_tex;   /* the float n_tex below shadows the count */
    int nr = orc_n_render_views(d);
    float *ex = (float *)malloc(sizeof(float) * (size_t)nr);
    orc_eyes(d, ex);
    float D = d->view_dist;
    /* pixel footprint per unit distance, horizontal and vertical */
    float px = (float)((double)d->focal_w / ((double)d->view_dist * d->view_w));
    float py = (float)((double)d->focal_h / ((double)d->view_dist * d->view_h));
    int status = ORC_OK;
    for (uint32_t t = 0; t < n_tris; t++) {
        float *T = tri_out + (size_t)t * ORC_TRI_FLOATS;
        memset(T, 0, sizeof(float) * ORC_TRI_FLOATS);
        counts[t] = 0;
        float P[3][3], Q[3][2];
        for (int k = 0; k < 3; k++) {
            uint32_t vi = idx[3 * (size_t)t + k];
            orc_transform(model, xyz + 3 * (size_t)vi, P[k]);
            Q[k][0] = uvs[2 * (size_t)vi];
            Q[k][1] = uvs[2 * (size_t)vi + 1];
        }
        uint32_t tex, mat = 0;
        if (mat_tex) {
            mat = tri_tex[t] < n_mat ? tri_tex[t] : 0;
            tex = mat_tex[4 * (size_t)mat] < n_tex ? mat_tex[4 * (size_t)mat] : 0;
            T[T_TEX] = (float)mat;
        } else {
            tex = tri_tex[t] < n_tex ? tri_tex[t] : 0;
            T[T_TEX] = (float)tex;
        }
        memcpy(T + T_P0, P[0], sizeof(float) * 3);
        if (culled(d, ex, nr, P)) continue;

        /* world-space area and unit normal */
        float e1[3], e2[3], cr[3];
        for (int c = 0; c < 3; c++) { e1[c] = P[1][c] - P[0][c]; e2[c] = P[2][c] - P[0][c]; }
        cross3(e1, e2, cr);
        float len2 = dot3(cr, cr);
        float len = sqrtf(len2);
        /* zero area: no points. Collinear vertices can leave a cross product of
         * rounding size, so an area below 2^-20 |e1| |e2| / 2 (the sine of the
         * vertex angle below 2^-20) counts as zero. */
        if (!(len2 > 0x1p-40f * (dot3(e1, e1) * dot3(e2, e2))) || !isfinite(len)) continue;
        float n[3] = {cr[0] / len, cr[1] / len, cr[2] / len};
        float A_ws = 0.5f * len;

        /* T_align (Sec. 3.1): v-hat is world up projected into the plane (the
         * views' shared vertical), u-hat = v-hat x n the horizontal. When the
         * plane is nearly horizontal, world x projected gives u-hat instead. */
        float eu[3], ev[3];
        float vv[3] = {-(n[1] * n[0]), fmaf(-n[1], n[1], 1.0f), -(n[1] * n[2])};
        float l2 = dot3(vv, vv);
        if (l2 >= 1e-6f) {
            float l = sqrtf(l2);
            for (int c = 0; c < 3; c++) ev[c] = vv[c] / l;
            cross3(ev, n, eu);
        } else {
            float uu[3] = {fmaf(-n[0], n[0], 1.0f), -(n[0] * n[1]), -(n[0] * n[2])};
            float l = sqrtf(dot3(uu, uu));
            for (int c = 0; c < 3; c++) eu[c] = uu[c] / l;
            cross3(n, eu, ev);
        }
        memcpy(T + T_N, n, sizeof n);
        memcpy(T + T_EU, eu, sizeof eu);
        memcpy(T + T_EV, ev, sizeof ev);

        /* 2-D vertex coordinates relative to P0, then shifted to the bbox min */
        float a1 = dot3(e1, eu), b1 = dot3(e1, ev), a2 = dot3(e2, eu), b2 = dot3(e2, ev);
        float umin = fminf(fminf(0.0f, a1), a2), vmin = fminf(fminf(0.0f, b1), b2);
        float U[3] = {0.0f - umin, a1 - umin, a2 - umin};
        float V[3] = {0.0f - vmin, b1 - vmin, b2 - vmin};
        T[T_UMIN] = umin; T[T_VMIN] = vmin;
        T[T_A1] = a1; T[T_B1] = b1; T[T_A2] = a2; T[T_B2] = b2;
        memcpy(T + T_U, U, sizeof U);
        memcpy(T + T_V, V, sizeof V);
        T[T_UMAX] = fmaxf(fmaxf(U[0], U[1]), U[2]);
        T[T_VMAX] = fmaxf(fmaxf(V[0], V[1]), V[2]);

        /* closest and farthest eye over all views (Fig. 5: pixel edges are
         * reverse-projected around the point of the triangle closest to the
         * eye). The eye's distance to the triangle: its height over the plane
         * and its in-plane distance to the 2-D triangle. */
        float d2min = INFINITY, d2max = -INFINITY;
        float ie01 = seg_inv_len2(0.0f, 0.0f, a1, b1), ie12 = seg_inv_len2(a1, b1, a2, b2);
        float ie20 = seg_inv_len2(a2, b2, 0.0f, 0.0f);
        for (int v = 0; v < nr; v++) {
            float q[3] = {ex[v] - P[0][0], 0.0f - P[0][1], D - P[0][2]};
            float qu = dot3(q, eu), qv = dot3(q, ev), h = dot3(q, n);
            float w0 = edge2(a1, b1, a2, b2, qu, qv);
            float w1 = edge2(a2, b2, 0.0f, 0.0f, qu, qv);
            float w2 = edge2(0.0f, 0.0f, a1, b1, qu, qv);
            float d2 = 0.0f;
            if (!inside3(w0, w1, w2))
                d2 = fminf(fminf(segd2(0.0f, 0.0f, a1, b1, ie01, qu, qv), segd2(a1, b1, a2, b2, ie12, qu, qv)),
                           segd2(a2, b2, 0.0f, 0.0f, ie20, qu, qv));
            float dd = fmaf(h, h, d2);
            d2min = fminf(d2min, dd);
            d2max = fmaxf(d2max, dd);
        }
        /* the footprint is never taken closer than the near plane */
        float dmin = fmaxf(sqrtf(d2min), d->near_z), dmax = fmaxf(sqrtf(d2max), d->near_z);
        T[T_DMIN] = dmin; T[T_DMAX] = dmax;

        /* LFD-biased spacings (Sec. 3.1): horizontal and vertical pixel edges
         * reverse-projected at distance dmin, times the sampling bias. */
        float su0 = (d->bias_h * dmin) * px, sv0 = (d->bias_v * dmin) * py;
        float size_xy = su0 * sv0;

        /* Eq. 1-2: texels spanned and world area per texel */
        uint32_t X = tex_wh[2 * tex], Y = tex_wh[2 * tex + 1];
        float ds1 = Q[1][0] - Q[0][0], dt1 = Q[1][1] - Q[0][1];
        float ds2 = Q[2][0] - Q[0][0], dt2 = Q[2][1] - Q[0][1];
        float A_ts = 0.5f * fabsf(fmaf(ds1, dt2, -(dt1 * ds2)));
        float n_tex = (A_ts * (float)X) * (float)Y;
        if (mat_tex) {   /* Eq. 1: the maximum over the material's textures */
            for (int k = 1; k < 4; k++) {
                uint32_t tk = mat_tex[4 * (size_t)mat + k] < n_textures ? mat_tex[4 * (size_t)mat + k] : 0;
                n_tex = fmaxf(n_tex, (A_ts * (float)tex_wh[2 * tk]) * (float)tex_wh[2 * tk + 1]);
            }
        }
        if (n_tex < 1.0f) n_tex = 1.0f;   /* a triangle spans at least one texel */
        float size_uv = A_ws / n_tex;

        /* Eq. 3: sampling density lowered to the texel density (S_ortho is a
         * density, so spacings grow by sqrt(size_uv / size_xy)) */
        float su = su0, sv = sv0;
        if (size_uv > size_xy) {
            float f = sqrtf(size_uv / size_xy);
            su = su0 * f;
            sv = sv0 * f;
        }
        T[T_AWS] = A_ws; T[T_ATS] = A_ts; T[T_NTEX] = n_tex; T[T_SIZE_UV] = size_uv;
        T[T_SU] = su; T[T_SV] = sv;

        /* Eq. 4-5: pixel area in texture space, min and max over views; the
         * per-view pixel area is the reverse-projected (biased) pixel at d_v,
         * monotone in d_v, so the extremes sit at dmin and dmax. */
        float r = A_ts / A_ws;
        float size_xy_max = ((d->bias_h * dmax) * px) * ((d->bias_v * dmax) * py);
        float vpuv_min = size_xy * r, vpuv_max = size_xy_max * r;
        T[T_VPUV_MIN] = vpuv_min; T[T_VPUV_MAX] = vpuv_max;
        T[T_SPL_UV] = (su * sv) * r;   /* the splat's area in texture space (Eq. 8) */

        /* Eq. 6-7 */
        T[T_LOD_MIN] = 0.5f * orc_log2f((vpuv_min * (float)X) * (float)Y);
        T[T_LOD_MAX] = 0.5f * orc_log2f((vpuv_max * (float)X) * (float)Y);

        /* affine map from the shifted 2-D frame to texture coordinates */
        float det = fmaf(a1, b2, -(a2 * b1));
        float gsu = 0.0f, gsv = 0.0f, gtu = 0.0f, gtv = 0.0f;
        if (det != 0.0f) {
            gsu = fmaf(ds1, b2, -(ds2 * b1)) / det;
            gsv = fmaf(ds2, a1, -(ds1 * a2)) / det;
            gtu = fmaf(dt1, b2, -(dt2 * b1)) / det;
            gtv = fmaf(dt2, a1, -(dt1 * a2)) / det;
        }
        T[T_SGU] = gsu; T[T_SGV] = gsv; T[T_TGU] = gtu; T[T_TGV] = gtv;
        T[T_S0] = fmaf(gsu, umin, fmaf(gsv, vmin, Q[0][0]));
        T[T_T0] = fmaf(gtu, umin, fmaf(gtv, vmin, Q[0][1]));

        /* point count: one point per overlapped lattice cell */
        float ncol = ceilf(T[T_UMAX] / su);
        if (!(ncol <= (float)ORC_MAX_CELL)) { status = ORC_EOVERFLOW; continue; }
        T[T_LIVE] = 1.0f;
        int cols = (int)ncol;
        uint32_t cnt = 0;
        for (int i = 0; i < cols; i++) {
            int j0, j1;
            int rows = column_rows(T, i, &j0, &j1);
            if (j1 > ORC_MAX_CELL + 1) { status = ORC_EOVERFLOW; cnt = 0; T[T_LIVE] = 0.0f; break; }
            cnt += (uint32_t)rows;
        }
        counts[t] = cnt;
    }
    free(ex);
    return status;
}

int orc_setup(const orc_display *d, const float *xyz, const float *uvs,
              const uint32_t *idx, const uint32_t *tri_tex, uint32_t n_tris,
              const uint32_t *tex_wh, uint32_t n_tex, const float *model,
              float *tri_out, uint32_t *counts) {
    return setup_impl(d, xyz, uvs, idx, tri_tex, n_tris, tex_wh, n_tex, NULL, 0, model, tri_out, counts);
}

/* orc_setup_mat: orc_setup for a mesh of materials (tri_mat: material per
 * triangle, mat_tex: n_mat x 4 texture indices). */
int orc_setup_mat(const orc_display *d, const float *xyz, const float *uvs,
                  const uint32_t *idx, const uint32_t *tri_mat, uint32_t n_tris,
                  const uint32_t *tex_wh, uint32_t n_tex, const uint32_t *mat_tex, uint32_t n_mat,
                  const float *model, float *tri_out, uint32_t *counts) {
    if (!mat_tex || n_mat == 0) return ORC_EINVAL;
    return setup_impl(d, xyz, uvs, idx, tri_mat, n_tris, tex_wh, n_tex, mat_tex, n_mat, model, tri_out, counts);
}

/*
 * orc_emit: the point buffer. Points are numbered by triangle (exclusive
 * prefix sum of counts), then column i, then row j. Each point is four u32:
 * triangle id, i | j << 16, tv_min RGBA8, tv_max RGBA8 (the last two are
 * filled by orc_fetch). Returns the number of points, or -1 if it exceeds cap.
 */
int64_t orc_emit(const float *tri, const uint32_t *counts, uint32_t n_tris,
                 uint32_t *points, int64_t cap) {
    int64_t total = 0;
    for (uint32_t t = 0; t < n_tris; t++) total += counts[t];
    if (total > cap) return -1;
    int64_t p = 0;
    for (uint32_t t = 0; t < n_tris; t++) {
        if (counts[t] == 0) continue;
        const float *T = tri + (size_t)t * ORC_TRI_FLOATS;
        int cols = n_columns(T);
        for (int i = 0; i < cols; i++) {
            int j0, j1;
            column_rows(T, i, &j0, &j1);
            for (int j = j0; j < j1; j++) {
                uint32_t *o = points + 4 * p;
                o[0] = t;
                o[1] = (uint32_t)i | ((uint32_t)j << 16);
                o[2] = 0;
                o[3] = 0;
                p++;
            }
        }
    }
    return p;
}

/*
 * orc_fetch: tv_min and tv_max of every point (Sec. 3.3): the texture
 * coordinate of the cell centre, trilinear at LOD_min and at LOD_max.
 */
void orc_fetch(const float *tri, uint32_t *points, int64_t n_points,
               const uint8_t *const *chains, const uint32_t *tex_wh) {
    for (int64_t p = 0; p < n_points; p++) {
        uint32_t *o = points + 4 * p;
        const float *T = tri + (size_t)o[0] * ORC_TRI_FLOATS;
        uint32_t i = o[1] & 0xffffu, j = o[1] >> 16;
        float uc = ((float)i + 0.5f) * T[T_SU];
        float vc = ((float)j + 0.5f) * T[T_SV];
        float s = fmaf(T[T_SGU], uc, fmaf(T[T_SGV], vc, T[T_S0]));
        float t = fmaf(T[T_TGU], uc, fmaf(T[T_TGV], vc, T[T_T0]));
        uint32_t tex = (uint32_t)T[T_TEX];
        uint32_t w = tex_wh[2 * tex], h = tex_wh[2 * tex + 1];
        uint8_t a[4], b[4];
        orc_trilinear(chains[tex], w, h, s, t, T[T_LOD_MIN], a);
        orc_trilinear(chains[tex], w, h, s, t, T[T_LOD_MAX], b);
        memcpy(&o[2], a, 4);
        memcpy(&o[3], b, 4);
    }
}

/*
 * orc_fetch_mat: the fetch of a mesh of materials (Sec. 3.3 with several
 * textures): every texture of the point's material gets its own Eq. 6-7 LOD
 * pair from the record's size_vpuv bounds and its own resolution, and its
 * own tv_min / tv_max. The albedo's pair goes to the point (as orc_fetch);
 * the normal, roughness and metallic pairs to tvx[6 p .. 6 p + 5].
 */
void orc_fetch_mat(const float *tri, uint32_t *points, int64_t n_points,
                   const uint8_t *const *chains, const uint32_t *tex_wh,
                   const uint32_t *mat_tex, uint32_t *tvx) {
    for (int64_t p = 0; p < n_points; p++) {
        uint32_t *o = points + 4 * p;
        const float *T = tri + (size_t)o[0] * ORC_TRI_FLOATS;
        uint32_t i = o[1] & 0xffffu, j = o[1] >> 16;
        float uc = ((float)i + 0.5f) * T[T_SU];
        float vc = ((float)j + 0.5f) * T[T_SV];
        float s = fmaf(T[T_SGU], uc, fmaf(T[T_SGV], vc, T[T_S0]));
        float t = fmaf(T[T_TGU], uc, fmaf(T[T_TGV], vc, T[T_T0]));
        uint32_t mat = (uint32_t)T[T_TEX];
        for (int k = 0; k < 4; k++) {
            uint32_t tex = mat_tex[4 * (size_t)mat + k];
            uint32_t w = tex_wh[2 * tex], h = tex_wh[2 * tex + 1];
            float lo, hi;
            if (k == 0) {
                lo = T[T_LOD_MIN];
                hi = T[T_LOD_MAX];
            } else {
                lo = 0.5f * orc_log2f((T[T_VPUV_MIN] * (float)w) * (float)h);
                hi = 0.5f * orc_log2f((T[T_VPUV_MAX] * (float)w) * (float)h);
            }
            uint8_t a[4], b[4];
            orc_trilinear(chains[tex], w, h, s, t, lo, a);
            orc_trilinear(chains[tex], w, h, s, t, hi, b);
            uint32_t *dst = k == 0 ? &o[2] : &tvx[6 * (size_t)p + 2 * (size_t)(k - 1)];
            memcpy(&dst[0], a, 4);
            memcpy(&dst[1], b, 4);
        }
    }
}

/* -------------------------------------------------------------------------- */
/* Splatting (Sec. 3.2) and the per-view depth test (64-bit buffers, Sec. 5.1)  */
/* -------------------------------------------------------------------------- */

/* World position of lattice corner (a s_u, b s_v) of the triangle's frame. */
static void cell_corner(const float *T, int a, int b, float o[3]) {
    float cu = (float)a * T[T_SU] + T[T_UMIN];
    float cv = (float)b * T[T_SV] + T[T_VMIN];
    for (int c = 0; c < 3; c++)
        o[c] = fmaf(cu, T[T_EU + c], fmaf(cv, T[T_EV + c], T[T_P0 + c]));
}

/*
 * Eq. 8's size_ndc^vs x 0.25 X_v Y_v: the area, in view pixels, of the splat
 * (the point's cell) projected into the view of eye (Ex, 0, D). Each corner
 * C of the cell is projected through the focal plane z = 0 by the plain
 * perspective map, x_s = Ex + (C_x - Ex) D / (D - C_z), y_s = C_y D / (D - C_z),
 * then to pixel coordinates ((x_s + fw/2) W/fw, (fh/2 - y_s) H/fh); the area
 * is the shoelace sum of the projected corners taken relative to the first
 * one. A cell that reaches within near_z of the eyes' plane has no bounded
 * projection; its splat is the part that can be drawn, the cell clipped to
 * depth D - z >= near_z (a plane shared by every view, since all eyes lie at
 * z = D), which leaves every other cell as it is. Evaluated in double from
 * the binary32 corners: the area only weights a colour (Eq. 9), it decides
 * no integer.
 */
static float splat_area_px(const orc_display *d, const float *T, int i, int j, float Ex) {
    float Cf[4][3];
    cell_corner(T, i, j, Cf[0]);
    cell_corner(T, i + 1, j, Cf[1]);
    cell_corner(T, i + 1, j + 1, Cf[2]);
    cell_corner(T, i, j + 1, Cf[3]);
    double D = d->view_dist, E = Ex, fw = d->focal_w, fh = d->focal_h;
    double zc = D - (double)d->near_z;
    double P[5][3];
    int m = 0;
    for (int c = 0; c < 4; c++) {
        const float *p = Cf[c], *q = Cf[(c + 1) & 3];
        int pin = p[2] <= zc, qin = q[2] <= zc;
        if (pin) {
            for (int k = 0; k < 3; k++) P[m][k] = p[k];
            m++;
        }
        if (pin != qin) {
            double f = (zc - p[2]) / ((double)q[2] - p[2]);
            for (int k = 0; k < 3; k++) P[m][k] = p[k] + f * ((double)q[k] - p[k]);
            P[m][2] = zc;
            m++;
        }
    }
    if (m < 3) return 0.0f;
    double px[5], py[5];
    for (int c = 0; c < m; c++) {
        double k = D / (D - P[c][2]);
        double xs = E + (P[c][0] - E) * k, ys = P[c][1] * k;
        px[c] = (xs + 0.5 * fw) * d->view_w / fw;
        py[c] = (0.5 * fh - ys) * d->view_h / fh;
    }
    double twice = 0.0;
    for (int c = 1; c + 1 < m; c++) {
        double ax = px[c] - px[0], ay = py[c] - py[0];
        double bx = px[c + 1] - px[0], by = py[c + 1] - py[0];
        twice += ax * by - bx * ay;
    }
    return (float)(0.5 * fabs(twice));
}

/* orc_splat_area_px: splat_area_px of cell (i, j) of the record T (one
 * triangle's ORC_TRI_FLOATS floats) in the view of eye x Ex. */
float orc_splat_area_px(const orc_display *d, const float *T, int i, int j, float Ex) {
    return splat_area_px(d, T, i, j, Ex);
}

/*
 * orc_splat: for every point and every listed view, each pixel whose centre
 * ray hits the triangle's plane inside the point's cell and inside the
 * triangle (EPR's inside-triangle test), at a depth within [near, far], gets
 * key = float_bits(t) << 32 | point id, keeping the minimum. t is the ray
 * parameter from the eye through the pixel centre on the focal plane, so on
 * one pixel it orders hits like depth (= t D). keys holds n_list views of
 * view_h x view_w u64, initialised here to all ones (empty).
 */
void orc_splat(const orc_display *d, const float *tri, const uint32_t *points,
               int64_t n_points, const int32_t *views, int n_list, uint64_t *keys) {
    int nr = orc_n_render_views(d);
    float *ex = (float *)malloc(sizeof(float) * (size_t)nr);
    orc_eyes(d, ex);
    int W = d->view_w, H = d->view_h;
    float D = d->view_dist;
    float pw = (float)((double)d->focal_w / W), ph = (float)((double)d->focal_h / H);
    float x0 = -0.5f * d->focal_w, y0 = 0.5f * d->focal_h;
    size_t npix = (size_t)W * H;
    for (size_t k = 0; k < npix * (size_t)n_list; k++) keys[k] = ~0ull;
    for (int64_t p = 0; p < n_points; p++) {
        const uint32_t *pt = points + 4 * p;
        const float *T = tri + (size_t)pt[0] * ORC_TRI_FLOATS;
        int i = (int)(pt[1] & 0xffffu), j = (int)(pt[1] >> 16);
        float C[4][3];
        cell_corner(T, i, j, C[0]);
        cell_corner(T, i + 1, j, C[1]);
        cell_corner(T, i + 1, j + 1, C[2]);
        cell_corner(T, i, j + 1, C[3]);
        const float *n = T + T_N, *eu = T + T_EU, *ev = T + T_EV, *P0 = T + T_P0;
        float su = T[T_SU], sv = T[T_SV];
        float ulo = (float)i * su, uhi = (float)(i + 1) * su;
        float vlo = (float)j * sv, vhi = (float)(j + 1) * sv;
        float a1 = T[T_A1], b1 = T[T_B1], a2 = T[T_A2], b2 = T[T_B2];
        for (int li = 0; li < n_list; li++) {
            int v = views[li];
            float E[3] = {ex[v], 0.0f, D};
            /* conservative pixel box of the projected cell, in double */
            int bx0 = 0, bx1 = W - 1, by0 = 0, by1 = H - 1;
            int behind = 0;
            double mnx = 1e300, mxx = -1e300, mny = 1e300, mxy = -1e300;
            for (int c = 0; c < 4; c++) {
                double dep = (double)D - C[c][2];
                if (!(dep > 1e-9)) { behind = 1; break; }
                double sx = E[0] + (C[c][0] - (double)E[0]) * D / dep;
                double sy = C[c][1] * (double)D / dep;
                double qx = (sx + 0.5 * d->focal_w) * W / d->focal_w;
                double qy = (0.5 * d->focal_h - sy) * H / d->focal_h;
                mnx = fmin(mnx, qx); mxx = fmax(mxx, qx);
                mny = fmin(mny, qy); mxy = fmax(mxy, qy);
            }
            if (!behind) {
                double fx0 = floor(mnx - 0.5) - 1, fx1 = ceil(mxx - 0.5) + 1;
                double fy0 = floor(mny - 0.5) - 1, fy1 = ceil(mxy - 0.5) + 1;
                if (fx1 < 0 || fy1 < 0 || fx0 > W - 1 || fy0 > H - 1) continue;
                bx0 = fx0 < 0 ? 0 : (int)fx0;
                bx1 = fx1 > W - 1 ? W - 1 : (int)fx1;
                by0 = fy0 < 0 ? 0 : (int)fy0;
                by1 = fy1 > H - 1 ? H - 1 : (int)fy1;
            }
            float qE[3] = {E[0] - P0[0], E[1] - P0[1], E[2] - P0[2]};
            float num = -dot3(n, qE);
            uint64_t *kv = keys + (size_t)li * npix;
            for (int y = by0; y <= by1; y++) {
                float Fy = fmaf((float)y + 0.5f, -ph, y0);
                for (int x = bx0; x <= bx1; x++) {
                    float Fx = fmaf((float)x + 0.5f, pw, x0);
                    float dir[3] = {Fx - E[0], Fy - E[1], -D};
                    float den = dot3(n, dir);
                    if (den == 0.0f) continue;
                    float t = num / den;
                    float depth = t * D;
                    if (!(depth >= d->near_z && depth <= d->far_z)) continue;
                    float h[3] = {fmaf(t, dir[0], qE[0]), fmaf(t, dir[1], qE[1]), fmaf(t, dir[2], qE[2])};
                    float uq = dot3(h, eu), vq = dot3(h, ev);
                    float u = uq - T[T_UMIN], vv = vq - T[T_VMIN];
                    if (!(u >= ulo && u < uhi && vv >= vlo && vv < vhi)) continue;
                    float w0 = edge2(a1, b1, a2, b2, uq, vq);
                    float w1 = edge2(a2, b2, 0.0f, 0.0f, uq, vq);
                    float w2 = edge2(0.0f, 0.0f, a1, b1, uq, vq);
                    if (!inside3(w0, w1, w2)) continue;
                    uint64_t key = ((uint64_t)fbits(t) << 32) | (uint64_t)(uint32_t)p;
                    size_t o = (size_t)y * W + x;
                    if (key < kv[o]) kv[o] = key;
                }
            }
        }
    }
    free(ex);
}

/*
 * orc_splat_hits: how many (point) splats pass every test at each pixel of the
 * listed views, without the depth minimum. On a single-triangle scene this is
 * 1 on the triangle's pixels and 0 elsewhere when the lattice cells tile the
 * triangle exactly once (the half-open cells of the conservative rule).
 */
void orc_splat_hits(const orc_display *d, const float *tri, const uint32_t *points,
                    int64_t n_points, const int32_t *views, int n_list, uint32_t *hits) {
    int W = d->view_w, H = d->view_h;
    size_t npix = (size_t)W * H;
    uint64_t *one = (uint64_t *)malloc(sizeof(uint64_t) * npix);
    for (size_t k = 0; k < npix * (size_t)n_list; k++) hits[k] = 0;
    for (int64_t p = 0; p < n_points; p++) {
        for (int li = 0; li < n_list; li++) {
            orc_splat(d, tri, points + 4 * p, 1, views + li, 1, one);
            for (size_t o = 0; o < npix; o++) hits[(size_t)li * npix + o] += one[o] != ~0ull;
        }
    }
    free(one);
}

/* -------------------------------------------------------------------------- */
/* Per-view texture interpolation, Eq. 8-9, and shading (unlit: colour = tv)    */
/* -------------------------------------------------------------------------- */

/*
 * orc_resolve: per listed view and pixel, the winning point's colour. The
 * splat's pixel area is the shoelace area of its cell's four corners
 * projected into the view (= size_ndc * 0.25 * X_v * Y_v of Eq. 8,
 * splat_area_px). Eq. 8
 * grows the splat's texture area when it covers less than a pixel and clamps
 * it to [size_vpuv_min, size_vpuv_max]; Eq. 9 interpolates tv between tv_min
 * and tv_max per channel. Empty pixels are (0, 0, 0, 0).
 */
void orc_resolve(const orc_display *d, const float *tri, const uint32_t *points,
                 const uint64_t *keys, const int32_t *views, int n_list, uint8_t *rgba) {
    int nr = orc_n_render_views(d);
    float *ex = (float *)malloc(sizeof(float) * (size_t)nr);
    orc_eyes(d, ex);
    int W = d->view_w, H = d->view_h;
    size_t npix = (size_t)W * H;
    for (int li = 0; li < n_list; li++) {
        float Ex = ex[views[li]];
        for (size_t o = 0; o < npix; o++) {
            uint64_t key = keys[(size_t)li * npix + o];
            uint8_t *out = rgba + ((size_t)li * npix + o) * 4;
            if (key == ~0ull) { out[0] = out[1] = out[2] = out[3] = 0; continue; }
            const uint32_t *pt = points + 4 * (size_t)(uint32_t)key;
            const float *T = tri + (size_t)pt[0] * ORC_TRI_FLOATS;
            int i = (int)(pt[1] & 0xffffu), j = (int)(pt[1] >> 16);
            float area_px = splat_area_px(d, T, i, j, Ex);
            float vmin = T[T_VPUV_MIN], vmax = T[T_VPUV_MAX];
            float size_vse = T[T_SPL_UV] / fminf(1.0f, area_px);
            float size_vs = fminf(fmaxf(size_vse, vmin), vmax);
            float w = vmax > vmin ? (size_vs - vmin) / (vmax - vmin) : 0.0f;
            const uint8_t *tmin = (const uint8_t *)&pt[2], *tmax = (const uint8_t *)&pt[3];
            for (int c = 0; c < 4; c++) {
                float a = tmin[c], b = tmax[c];
                out[c] = to_u8(fmaf(w, b - a, a));
            }
        }
    }
    free(ex);
}

/* -------------------------------------------------------------------------- */
/* Physically based shading of a mesh of materials (Sec. 3.3 shades during     */
/* view generation; Sec. 5 names a PBR shader over albedo, roughness,          */
/* metallic and normal textures without defining it: this is the reading)      */
/* -------------------------------------------------------------------------- */

typedef struct {
    float light_dir[3];   /* toward the light (normalised here) */
    float light_rgb[3];   /* radiance of the directional light */
    float ambient[3];     /* constant ambient, times albedo */
} orc_shading;

static const double kPi = 3.14159265358979323846;

static void dnorm(double *v) {
    double l = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (l > 0.0) { v[0] /= l; v[1] /= l; v[2] /= l; }
}
static double ddot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/*
 * orc_pbr_shade: outgoing colour (linear, 0..1 before clamping) of one
 * surface sample: metallic-roughness microfacet BRDF with the GGX normal
 * distribution D = a^2 / (pi ((n.h)^2 (a^2 - 1) + 1)^2), a = r^2 (r >= 0.045),
 * Schlick-GGX visibility G = G1(n.l) G1(n.v), G1(x) = x / (x (1 - k) + k),
 * k = (r + 1)^2 / 8, Schlick Fresnel F = F0 + (1 - F0)(1 - v.h)^5 with
 * F0 = 0.04 (1 - m) + albedo m, diffuse (1 - F)(1 - m) albedo / pi:
 *   rgb = (diffuse + D G F / (4 n.l n.v)) light n.l + ambient albedo,
 * n.l clamped at 0, n.v at 1e-4. n, v, l are unit vectors.
 */
void orc_pbr_shade(const double *albedo, double rough, double metal, const double *n, const double *v,
                   const double *l, const float *light_rgb, const float *ambient, double *out) {
    double h[3] = {l[0] + v[0], l[1] + v[1], l[2] + v[2]};
    dnorm(h);
    double nl = ddot(n, l), nv = ddot(n, v), nh = ddot(n, h), vh = ddot(v, h);
    if (nl < 0.0) nl = 0.0;
    if (nv < 1e-4) nv = 1e-4;
    if (nh < 0.0) nh = 0.0;
    if (vh < 0.0) vh = 0.0;
    double r = rough < 0.045 ? 0.045 : rough;
    double a = r * r, a2 = a * a;
    double dn = nh * nh * (a2 - 1.0) + 1.0;
    double Dg = a2 / (kPi * dn * dn);
    double k = (r + 1.0) * (r + 1.0) / 8.0;
    double G = (nl / (nl * (1.0 - k) + k)) * (nv / (nv * (1.0 - k) + k));
    double f5 = (1.0 - vh) * (1.0 - vh);
    f5 = f5 * f5 * (1.0 - vh);
    double den = 4.0 * nl * nv;
    if (den < 1e-4) den = 1e-4;
    for (int c = 0; c < 3; c++) {
        double F0 = 0.04 * (1.0 - metal) + albedo[c] * metal;
        double F = F0 + (1.0 - F0) * f5;
        double diffuse = (1.0 - F) * (1.0 - metal) * albedo[c] / kPi;
        double spec = Dg * G * F / den;
        out[c] = (diffuse + spec) * light_rgb[c] * nl + ambient[c] * albedo[c];
    }
}

/*
 * Shading frame of a triangle from its record: N the unit normal; the
 * tangent and bitangent are the world directions of increasing texture s and
 * t (the inverse of the record's affine map over the lattice frame u-hat,
 * v-hat), the tangent made orthogonal to N and the bitangent N x T with the
 * sign of the t direction. A degenerate map gives u-hat and v-hat.
 */
static void shading_frame(const float *T, double *tg, double *bt, double *nn) {
    for (int c = 0; c < 3; c++) nn[c] = T[T_N + c];
    double gsu = T[T_SGU], gsv = T[T_SGV], gtu = T[T_TGU], gtv = T[T_TGV];
    double det = gsu * gtv - gsv * gtu;
    double dus = 1.0, dvs = 0.0, dut = 0.0, dvt = 1.0;   /* d(u, v) / d(s, t) */
    if (det != 0.0) {
        dus = gtv / det; dvs = -gtu / det;
        dut = -gsv / det; dvt = gsu / det;
    }
    double ts[3], tt[3];
    for (int c = 0; c < 3; c++) {
        ts[c] = T[T_EU + c] * dus + T[T_EV + c] * dvs;
        tt[c] = T[T_EU + c] * dut + T[T_EV + c] * dvt;
    }
    double dn = ddot(ts, nn);
    for (int c = 0; c < 3; c++) tg[c] = ts[c] - nn[c] * dn;
    dnorm(tg);
    double cb[3] = {nn[1] * tg[2] - nn[2] * tg[1], nn[2] * tg[0] - nn[0] * tg[2], nn[0] * tg[1] - nn[1] * tg[0]};
    double sg = ddot(cb, tt) < 0.0 ? -1.0 : 1.0;
    for (int c = 0; c < 3; c++) bt[c] = cb[c] * sg;
}

/*
 * orc_resolve_pbr: orc_resolve for a mesh of materials under one directional
 * light. Per pixel: Eq. 8's weight w as in orc_resolve; each texture's value
 * interpolated by Eq. 9 (unrounded); the surface point where the pixel
 * centre's ray meets the triangle (the depth key's t: P = E + t (F - E)); the
 * shading normal = the normal map's (2 c / 255 - 1) vector in the triangle's
 * frame, flipped with the frame when the triangle faces away from the eye;
 * colour = orc_pbr_shade, clamped to [0, 1], times 255, rounded half to even,
 * alpha 255. tvx as written by orc_fetch_mat.
 */
void orc_resolve_pbr(const orc_display *d, const float *tri, const uint32_t *points, const uint32_t *tvx,
                     const uint64_t *keys, const int32_t *views, int n_list, const orc_shading *sh,
                     uint8_t *rgba) {
    int nr = orc_n_render_views(d);
    float *ex = (float *)malloc(sizeof(float) * (size_t)nr);
    orc_eyes(d, ex);
    int W = d->view_w, H = d->view_h;
    float D = d->view_dist;
    float pw = (float)((double)d->focal_w / W), ph = (float)((double)d->focal_h / H);
    float x0 = -0.5f * d->focal_w, y0 = 0.5f * d->focal_h;
    double L[3] = {sh->light_dir[0], sh->light_dir[1], sh->light_dir[2]};
    dnorm(L);
    size_t npix = (size_t)W * H;
    for (int li = 0; li < n_list; li++) {
        float Ex = ex[views[li]];
        for (size_t o = 0; o < npix; o++) {
            uint64_t key = keys[(size_t)li * npix + o];
            uint8_t *out = rgba + ((size_t)li * npix + o) * 4;
            if (key == ~0ull) { out[0] = out[1] = out[2] = out[3] = 0; continue; }
            uint32_t p = (uint32_t)key;
            const uint32_t *pt = points + 4 * (size_t)p;
            const float *T = tri + (size_t)pt[0] * ORC_TRI_FLOATS;
            int i = (int)(pt[1] & 0xffffu), j = (int)(pt[1] >> 16);
            /* Eq. 8 weight, exactly as orc_resolve */
            float area_px = splat_area_px(d, T, i, j, Ex);
            float vmin = T[T_VPUV_MIN], vmax = T[T_VPUV_MAX];
            float size_vse = T[T_SPL_UV] / fminf(1.0f, area_px);
            float size_vs = fminf(fmaxf(size_vse, vmin), vmax);
            double w = vmax > vmin ? (double)((size_vs - vmin) / (vmax - vmin)) : 0.0;
            /* Eq. 9 per texture (unrounded) */
            const uint8_t *amin = (const uint8_t *)&pt[2], *amax = (const uint8_t *)&pt[3];
            const uint8_t *nmin = (const uint8_t *)&tvx[6 * (size_t)p], *nmax = (const uint8_t *)&tvx[6 * (size_t)p + 1];
            const uint8_t *rmin = (const uint8_t *)&tvx[6 * (size_t)p + 2], *rmax = (const uint8_t *)&tvx[6 * (size_t)p + 3];
            const uint8_t *mmin = (const uint8_t *)&tvx[6 * (size_t)p + 4], *mmax = (const uint8_t *)&tvx[6 * (size_t)p + 5];
            double alb[3], nt[3];
            for (int c = 0; c < 3; c++) {
                alb[c] = (amin[c] + w * ((double)amax[c] - amin[c])) / 255.0;
                nt[c] = 2.0 * (nmin[c] + w * ((double)nmax[c] - nmin[c])) / 255.0 - 1.0;
            }
            double rough = (rmin[0] + w * ((double)rmax[0] - rmin[0])) / 255.0;
            double metal = (mmin[0] + w * ((double)mmax[0] - mmin[0])) / 255.0;
            /* surface point and view direction */
            int px = (int)(o % (size_t)W), py = (int)(o / (size_t)W);
            double Fx = fmaf((float)px + 0.5f, pw, x0), Fy = fmaf((float)py + 0.5f, -ph, y0);
            double t = (double)bitsf((uint32_t)(key >> 32));
            double P[3] = {Ex + t * (Fx - Ex), t * Fy, D - t * D};
            double V[3] = {Ex - P[0], -P[1], D - P[2]};
            dnorm(V);
            double tg[3], bt[3], nn[3];
            shading_frame(T, tg, bt, nn);
            double n[3];
            for (int c = 0; c < 3; c++) n[c] = nt[0] * tg[c] + nt[1] * bt[c] + nt[2] * nn[c];
            if (ddot(n, n) == 0.0) memcpy(n, nn, sizeof n);
            dnorm(n);
            if (ddot(nn, V) < 0.0) for (int c = 0; c < 3; c++) n[c] = -n[c];
            double rgb[3];
            orc_pbr_shade(alb, rough, metal, n, V, L, sh->light_rgb, sh->ambient, rgb);
            for (int c = 0; c < 3; c++) {
                double v = rgb[c] < 0.0 ? 0.0 : rgb[c] > 1.0 ? 1.0 : rgb[c];
                out[c] = (uint8_t)nearbyint(v * 255.0);
            }
            out[3] = 255;
        }
    }
    free(ex);
}

/* -------------------------------------------------------------------------- */
/* Reconstruction, crosstalk and interleave (Sec. 4)                           */
/* -------------------------------------------------------------------------- */

/*
 * orc_display_views: the N views the panel shows, as floats (RGBA, 0..255).
 * With angular supersampling (recon = 1) view k is the [1/4, 1/2, 1/4] tent
 * over rendered views 2k-1, 2k, 2k+1, renormalised over the taps that exist.
 * With crosstalk x > 0 each view then becomes (1-2x) own + x each neighbour,
 * neighbour indices wrapping (the lens phase is cyclic).
 */
void orc_display_views(const orc_display *d, const uint8_t *rendered, float *out) {
    int N = d->n_views, nr = orc_n_render_views(d);
    size_t npix = (size_t)d->view_w * d->view_h;
    size_t nval = npix * 4;
    float *o = (float *)malloc(sizeof(float) * nval * (size_t)N);
    for (int k = 0; k < N; k++) {
        for (size_t e = 0; e < nval; e++) {
            if (d->recon == 1) {
                static const float w[3] = {0.25f, 0.5f, 0.25f};
                float acc = 0.0f, ws = 0.0f;
                for (int q = 0; q < 3; q++) {
                    int m = 2 * k - 1 + q;
                    if (m < 0 || m >= nr) continue;
                    acc = fmaf(w[q], (float)rendered[(size_t)m * nval + e], acc);
                    ws += w[q];
                }
                o[(size_t)k * nval + e] = acc / ws;
            } else {
                o[(size_t)k * nval + e] = (float)rendered[(size_t)k * nval + e];
            }
        }
    }
    if (d->crosstalk > 0.0f) {
        float x = d->crosstalk, c0 = (float)(1.0 - 2.0 * (double)d->crosstalk);
        for (int k = 0; k < N; k++) {
            int km = (k + N - 1) % N, kp = (k + 1) % N;
            for (size_t e = 0; e < nval; e++) {
                float acc = o[(size_t)k * nval + e] * c0;
                acc = fmaf(x, o[(size_t)km * nval + e], acc);
                acc = fmaf(x, o[(size_t)kp * nval + e], acc);
                out[(size_t)k * nval + e] = acc;
            }
        }
    } else {
        memcpy(out, o, sizeof(float) * nval * (size_t)N);
    }
    free(o);
}

/* Subpixel phase on the display-view axis under the slanted lenticular lens
 * (reading of the interleave of Sec. 4: a van Berkel-style slanted-lens phase
 * taken at the subpixel's centre, x + (c + 1/2)/3 for colour channel c of
 * pixel x): phi in [0, N). */
float orc_subpixel_phase(const orc_display *d, int x, int y, int c) {
    static const float third[3] = {(float)(1.0 / 6.0), 0.5f, (float)(5.0 / 6.0)};
    float inv_pitch = (float)(1.0 / (double)d->lens_pitch_px);
    float cx = (float)x + third[c];
    float a = fmaf(d->slant, (float)y, cx);
    float ph = fmaf(a, inv_pitch, d->phase_offset);
    float fr = ph - floorf(ph);
    return fr * (float)d->n_views;
}

int orc_view_of_subpixel(const orc_display *d, int x, int y, int c) {
    int k = (int)orc_subpixel_phase(d, x, y, c);
    if (k >= d->n_views) k = d->n_views - 1;
    if (k < 0) k = 0;
    return k;
}

/*
 * Gaussian reconstruction (recon 2 over the 2N supersampled views, recon 3
 * over the N views; Sec. 4: Gaussian filters in space and angle, integrated
 * with a few random samples). The display value at phase
 * phi, channel c, for panel pixel (x, y) is the mean over the samples s of
 * the rendered view nearest (on the display-view axis; on a tie the later
 * view) to phi + dphi_s, at the view pixel holding (vx + dx_s, vy + dy_s),
 * clamped to the view, where (vx, vy) = ((x + 1/2) W / Wp, (y + 1/2) H / Hp).
 * The samples (offsets drawn from the filters) are the caller's.
 */
float orc_gauss_value(const orc_display *d, const uint8_t *rendered, const float *pos, float phi, int x, int y,
                      int c) {
    int nr = orc_n_render_views(d), W = d->view_w, H = d->view_h;
    size_t npix = (size_t)W * H;
    float r = (float)(nr / d->n_views);
    float sxw = (float)W / (float)d->panel_w, syh = (float)H / (float)d->panel_h;
    float vx = ((float)x + 0.5f) * sxw, vy = ((float)y + 0.5f) * syh;
    float acc = 0.0f;
    for (int s = 0; s < d->n_samples; s++) {
        float a = phi + d->samples[3 * s + 2];
        int lo = (int)floorf(r * a) - 2;
        if (lo > nr - 4) lo = nr - 4;
        if (lo < 0) lo = 0;
        int hi = lo + 3 < nr - 1 ? lo + 3 : nr - 1;
        int m = lo;
        float best = fabsf(pos[lo] - a);
        for (int q = lo + 1; q <= hi; q++) {
            float dq = fabsf(pos[q] - a);
            if (dq <= best) {
                best = dq;
                m = q;
            }
        }
        int px = (int)floorf(vx + d->samples[3 * s]), py = (int)floorf(vy + d->samples[3 * s + 1]);
        px = px < 0 ? 0 : (px >= W ? W - 1 : px);
        py = py < 0 ? 0 : (py >= H ? H - 1 : py);
        acc += (float)rendered[((size_t)m * npix + (size_t)py * W + px) * 4 + c];
    }
    return acc / (float)d->n_samples;
}

/*
 * Mip level L of one rendered view (Sec. 5.1: with spatial supersampling a
 * mipmap of each light field view is built): L times the 2 x 2 box of the
 * level above, (a + b + c + d + 2) >> 2 per channel, as for the textures.
 * W and H must be multiples of 2^L; out holds (W >> L) x (H >> L) RGBA8.
 */
void orc_view_mip(const uint8_t *view, int W, int H, int L, uint8_t *out) {
    size_t n = (size_t)W * H * 4;
    uint8_t *cur = (uint8_t *)malloc(n), *nxt = (uint8_t *)malloc(n);
    memcpy(cur, view, n);
    int w = W, h = H;
    for (int l = 0; l < L; l++) {
        int nw = w / 2, nh = h / 2;
        for (int y = 0; y < nh; y++)
            for (int x = 0; x < nw; x++)
                for (int c = 0; c < 4; c++) {
                    unsigned s = cur[((size_t)(2 * y) * w + 2 * x) * 4 + c] + cur[((size_t)(2 * y) * w + 2 * x + 1) * 4 + c] +
                                 cur[((size_t)(2 * y + 1) * w + 2 * x) * 4 + c] +
                                 cur[((size_t)(2 * y + 1) * w + 2 * x + 1) * 4 + c];
                    nxt[((size_t)y * nw + x) * 4 + c] = (uint8_t)((s + 2) >> 2);
                }
        uint8_t *t = cur;
        cur = nxt;
        nxt = t;
        w = nw;
        h = nh;
    }
    memcpy(out, cur, (size_t)w * h * 4);
    free(cur);
    free(nxt);
}

static void interleave_views(const orc_display *d, const uint8_t *rendered, uint8_t *panel);

/*
 * orc_interleave: the elemental image array. With spatial supersampling
 * (ss_level L > 0) the views are first reduced to mip level L, whose texels
 * are output pixels, and the interleave below reads those. Panel subpixel (x, y, c) shows
 * channel c of display view orc_view_of_subpixel(x, y, c) at the nearest view
 * texel (floor((x+1/2) W / W_p), floor((y+1/2) H / H_p)); alpha is 255. With
 * Gaussian reconstruction (recon 2 or 3) it shows orc_gauss_value at the
 * subpixel's phase phi, with crosstalk x mixing in the values at phi - 1 and
 * phi + 1 (wrapping over the N views) at weight x each.
 */
void orc_interleave(const orc_display *d, const uint8_t *rendered, uint8_t *panel) {
    if (d->ss_level > 0) {
        int L = d->ss_level, nr = orc_n_render_views(d);
        orc_display dl = *d;
        dl.view_w = d->view_w >> L;
        dl.view_h = d->view_h >> L;
        dl.ss_level = 0;
        size_t per = (size_t)dl.view_w * dl.view_h * 4;
        uint8_t *lv = (uint8_t *)malloc(per * (size_t)nr);
        for (int m = 0; m < nr; m++)
            orc_view_mip(rendered + (size_t)m * d->view_w * d->view_h * 4, d->view_w, d->view_h, L, lv + per * m);
        interleave_views(&dl, lv, panel);
        free(lv);
        return;
    }
    interleave_views(d, rendered, panel);
}

static void interleave_views(const orc_display *d, const uint8_t *rendered, uint8_t *panel) {
    int N = d->n_views, W = d->view_w, H = d->view_h, Wp = d->panel_w, Hp = d->panel_h;
    size_t npix = (size_t)W * H;
    if (d->recon == 2 || d->recon == 3) {
        int nr = orc_n_render_views(d);
        float *pos = (float *)malloc(sizeof(float) * (size_t)nr);
        for (int m = 0; m < nr; m++) pos[m] = orc_view_pos(d, m);
        float x = d->crosstalk, c0 = (float)(1.0 - 2.0 * (double)d->crosstalk);
        for (int y = 0; y < Hp; y++)
            for (int xp = 0; xp < Wp; xp++) {
                uint8_t *o = panel + ((size_t)y * Wp + xp) * 4;
                for (int c = 0; c < 3; c++) {
                    float phi = orc_subpixel_phase(d, xp, y, c);
                    float v = orc_gauss_value(d, rendered, pos, phi, xp, y, c);
                    if (x > 0.0f) {
                        float pm = phi - 1.0f, pp = phi + 1.0f;
                        if (pm < 0.0f) pm += (float)N;
                        if (pp >= (float)N) pp -= (float)N;
                        float acc = v * c0;
                        acc = fmaf(x, orc_gauss_value(d, rendered, pos, pm, xp, y, c), acc);
                        acc = fmaf(x, orc_gauss_value(d, rendered, pos, pp, xp, y, c), acc);
                        v = acc;
                    }
                    o[c] = to_u8(v);
                }
                o[3] = 255;
            }
        free(pos);
        return;
    }
    float *dv = (float *)malloc(sizeof(float) * npix * 4 * (size_t)N);
    orc_display_views(d, rendered, dv);
    for (int y = 0; y < Hp; y++) {
        int sy = (int)(((int64_t)(2 * y + 1) * H) / (2 * (int64_t)Hp));
        for (int x = 0; x < Wp; x++) {
            int sx = (int)(((int64_t)(2 * x + 1) * W) / (2 * (int64_t)Wp));
            uint8_t *o = panel + ((size_t)y * Wp + x) * 4;
            for (int c = 0; c < 3; c++) {
                int k = orc_view_of_subpixel(d, x, y, c);
                o[c] = to_u8(dv[((size_t)k * npix + (size_t)sy * W + sx) * 4 + c]);
            }
            o[3] = 255;
        }
    }
    free(dv);
}

/* -------------------------------------------------------------------------- */
/* Brute-force ray caster (double precision): the pin for the splat step      */
/* -------------------------------------------------------------------------- */

/*
 * orc_raycast: the triangle nearest along the centre ray of pixel (x, y) of
 * rendered view v, over all triangles (transformed vertices txyz, 9 floats per
 * triangle), within [near, far] depth; Moller-Trumbore in double. Returns the
 * triangle id or -1, and the ray parameter in *t_out.
 */
int32_t orc_raycast(const orc_display *d, const float *txyz, uint32_t n_tris,
                    int v, int x, int y, double *t_out) {
    int nr = orc_n_render_views(d);
    float *ex = (float *)malloc(sizeof(float) * (size_t)nr);
    orc_eyes(d, ex);
    double D = d->view_dist;
    double E[3] = {ex[v], 0.0, D};
    free(ex);
    double Fx = -0.5 * d->focal_w + (x + 0.5) * d->focal_w / d->view_w;
    double Fy = 0.5 * d->focal_h - (y + 0.5) * d->focal_h / d->view_h;
    double dir[3] = {Fx - E[0], Fy - E[1], -D};
    double best = INFINITY;
    int32_t hit = -1;
    for (uint32_t t = 0; t < n_tris; t++) {
        const float *p = txyz + 9 * (size_t)t;
        double a[3] = {p[0], p[1], p[2]}, e1[3], e2[3], s[3], pv[3], qv[3];
        for (int c = 0; c < 3; c++) { e1[c] = p[3 + c] - a[c]; e2[c] = p[6 + c] - a[c]; s[c] = E[c] - a[c]; }
        pv[0] = dir[1] * e2[2] - dir[2] * e2[1];
        pv[1] = dir[2] * e2[0] - dir[0] * e2[2];
        pv[2] = dir[0] * e2[1] - dir[1] * e2[0];
        double det = e1[0] * pv[0] + e1[1] * pv[1] + e1[2] * pv[2];
        if (fabs(det) < 1e-30) continue;
        double inv = 1.0 / det;
        double bu = (s[0] * pv[0] + s[1] * pv[1] + s[2] * pv[2]) * inv;
        if (bu < 0.0 || bu > 1.0) continue;
        qv[0] = s[1] * e1[2] - s[2] * e1[1];
        qv[1] = s[2] * e1[0] - s[0] * e1[2];
        qv[2] = s[0] * e1[1] - s[1] * e1[0];
        double bv = (dir[0] * qv[0] + dir[1] * qv[1] + dir[2] * qv[2]) * inv;
        if (bv < 0.0 || bu + bv > 1.0) continue;
        double tt = (e2[0] * qv[0] + e2[1] * qv[1] + e2[2] * qv[2]) * inv;
        double depth = tt * D;
        if (depth < d->near_z || depth > d->far_z) continue;
        if (tt < best) { best = tt; hit = (int32_t)t; }
    }
    *t_out = best;
    return hit;
}
