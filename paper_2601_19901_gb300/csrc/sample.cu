// Triangle sampling (Sec. 3.1) and multiview-mip fetch (Sec. 3.3).
//
//   k_setup  one thread per triangle: model transform, visibility against every
//            view (Sec. 3), T_align frame, LFD-biased spacings from the closest
//            eye, Eq. 1-3 texture limit, Eq. 4-7 mip set-up, point count by the
//            lattice column walk (each column's first row and row count kept
//            for k_emit when there are at most four); block sums for the scan.
//   k_scan   one block: exclusive scan of the block sums -> block offsets,
//            total point count, overflow flag.
//   k_emit   one thread per triangle: warp-shuffle block scan of the counts
//            plus the block offset gives each triangle's first point id; the
//            column summary (or, for a wider triangle, the column walk again)
//            writes (triangle, cell) for each of its points (a warp per
//            triangle of more than kEmitBig points).
//   k_fetch  one thread per point: texture coordinate of the cell centre and
//            two trilinear fetches at LOD_min and LOD_max (Eq. 6-7); then the
//            point's splat record (its cell projected into the views) and, if
//            some view can hold a candidate pixel of it, its place in the
//            splat's work list; the pass ends with the frame's key reset.
//
// Every kernel after k_setup is launched as a programmatic dependent of the
// one before it and waits for it at its top (wait_previous_kernel).
//   k_near_work  one thread per point whose cell or triangle reaches within
//            near_z of the eyes' plane: the splat record of its cell and
//            triangle clipped to that limit.
//
// Every floating-point step here is bit-specified (binary32, explicit fmaf,
// IEEE division and square root) so the point set is identical to the CPU
// oracle's.
#include "lfdpr_internal.cuh"

namespace lfdpr {
namespace {

__device__ __forceinline__ void transform(const float* m, float x, float y, float z, float* o) {
    o[0] = fmaf(m[0], x, fmaf(m[1], y, fmaf(m[2], z, m[3])));
    o[1] = fmaf(m[4], x, fmaf(m[5], y, fmaf(m[6], z, m[7])));
    o[2] = fmaf(m[8], x, fmaf(m[9], y, fmaf(m[10], z, m[11])));
}

// Visibility (Sec. 3): dropped iff for every view all three vertices are on
// the outer side of one common frustum plane. Planes as linear forms,
// negative outside; top, bottom, near and far are shared by all views.
__device__ __forceinline__ bool seen_by(const DispConst& c, float e, const float P[3][3]) {
    const float lx = -c.fw2 - e, rx = c.fw2 - e;
    bool out_l = true, out_r = true;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float dep = c.D - P[k][2];
        const float l = fmaf(P[k][0] - e, c.D, -(lx * dep));
        const float r = fmaf(rx, dep, -((P[k][0] - e) * c.D));
        out_l &= l < 0.0f;
        out_r &= r < 0.0f;
    }
    return !(out_l || out_r);
}

// The eye whose x is nearest `target` (eyes ascending in x): binary search
// for the first eye at or beyond it, then the nearer of it and the one
// before (the earlier on a tie). Only a starting guess for the searches
// below: culling and the closest / farthest eye do not depend on it.
__device__ __forceinline__ int nearest_eye(const float* __restrict__ ex, int nr, float target) {
    int lo = 0, hi = nr;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ex[mid] < target) lo = mid + 1;
        else hi = mid;
    }
    if (lo == 0) return 0;
    if (lo == nr) return nr - 1;
    return fabsf(ex[lo] - target) < fabsf(ex[lo - 1] - target) ? lo : lo - 1;
}

__device__ bool culled(const DispConst& c, const float* __restrict__ ex, const float P[3][3]) {
    bool out_t = true, out_b = true, out_n = true, out_f = true;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const float dep = c.D - P[k][2];
        const float top = fmaf(c.fh2, dep, -(P[k][1] * c.D));
        const float bot = fmaf(P[k][1], c.D, c.fh2 * dep);
        out_t &= top < 0.0f;
        out_b &= bot < 0.0f;
        out_n &= (dep - c.near_z) < 0.0f;
        out_f &= (c.far_z - dep) < 0.0f;
    }
    if (out_t || out_b || out_n || out_f) return true;
    // Any one view that sees the triangle settles it. Try first the view
    // whose eye centres the centroid in the focal rectangle (the eye x at
    // which the centroid projects to x = 0 is x_c D / z_c), then all views.
    const float cx = (P[0][0] + P[1][0] + P[2][0]) * (1.0f / 3.0f);
    const float cz = (P[0][2] + P[1][2] + P[2][2]) * (1.0f / 3.0f);
    const float target = fabsf(cz) > 1e-6f ? __fdividef(cx * c.D, cz) : 0.0f;
    const int vb = nearest_eye(ex, c.nr, target);
    if (seen_by(c, ex[vb], P)) return false;
    for (int v = 0; v < c.nr; v++)
        if (seen_by(c, ex[v], P)) return false;
    return true;
}

// The lattice columns of a triangle, in order: rows [j0, j1) of column i
// overlapping it (conservative rule) span its v range over the column slab
// [i s_u, min((i+1) s_u, u_max)], from the vertices inside the slab and the
// edge crossings of the slab's two borders. For every column i < ceil(u_max /
// s_u), i s_u <= u_max, so a column's left border is exactly the right border
// of the one before: its crossings are carried over, not recomputed.
struct ColumnWalk {
    float U[3], V[3], su, sv, umax;
    float lo_b, hi_b;   // v range of the edge crossings of the last right border

    __device__ __forceinline__ void crossings(float x, float& lo, float& hi) const {
        lo = INFINITY;
        hi = -INFINITY;
#pragma unroll
        for (int e = 0; e < 3; e++) {
            const int p = e, r = e == 2 ? 0 : e + 1;
            if (U[p] == U[r]) continue;
            const float umn = fminf(U[p], U[r]), umx = fmaxf(U[p], U[r]);
            if (x >= umn && x <= umx) {
                const float vx = fmaf(__fdiv_rn(x - U[p], U[r] - U[p]), V[r] - V[p], V[p]);
                lo = fminf(lo, vx);
                hi = fmaxf(hi, vx);
            }
        }
    }
    __device__ __forceinline__ ColumnWalk(const float U_[3], const float V_[3], float su_, float sv_, float umax_)
        : su(su_), sv(sv_), umax(umax_) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            U[k] = U_[k];
            V[k] = V_[k];
        }
        crossings(float(0) * su, lo_b, hi_b);
    }
    // column i: call for i = 0, 1, 2, ... in turn
    __device__ __forceinline__ int rows(int i, int* j0, int* j1) {
        const float a = float(i) * su;
        const float b = fminf(float(i + 1) * su, umax);
        float lo = lo_b, hi = hi_b;
#pragma unroll
        for (int k = 0; k < 3; k++) {
            if (U[k] >= a && U[k] <= b) { lo = fminf(lo, V[k]); hi = fmaxf(hi, V[k]); }
        }
        crossings(b, lo_b, hi_b);
        lo = fminf(lo, lo_b);
        hi = fmaxf(hi, hi_b);
        if (lo > hi) { *j0 = 0; *j1 = 0; return 0; }
        *j0 = int(floorf(__fdiv_rn(lo, sv)));
        *j1 = int(ceilf(__fdiv_rn(hi, sv)));
        if (*j1 < *j0) *j1 = *j0;
        return *j1 - *j0;
    }
};

__device__ __forceinline__ void shifted_uv(const TriRec& r, float U[3], float V[3]) {
    const float umin = r.q[2].w, vmin = r.q[3].w;
    U[0] = 0.0f - umin; U[1] = r.q[4].x - umin; U[2] = r.q[4].z - umin;
    V[0] = 0.0f - vmin; V[1] = r.q[4].y - vmin; V[2] = r.q[4].w - vmin;
}

struct SetupOut {
    uint32_t count;
    bool live;
    bool cell_overflow;
};

// ex: the rendered views' eye x, ascending (a copy in shared memory)
__device__ SetupOut setup_triangle(const FrameArgs& a, const float* ex, uint32_t t, TriRec& r, TriProj& tp) {
    const DispConst& c = a.dc;
    SetupOut res{0u, false, false};
    float P[3][3], Q[3][2], M[12];
#pragma unroll
    for (int k = 0; k < 12; k++) M[k] = a.model_dev ? __ldg(a.model_dev + k) : a.model[k];
#pragma unroll
    for (int k = 0; k < 3; k++) {
        uint32_t vi = a.idx[3 * (size_t)t + k];
        if (!LFDPR_IN_BOUNDS(vi, a.n_verts, 1)) vi = 0;
        transform(M, a.xyz[3 * (size_t)vi], a.xyz[3 * (size_t)vi + 1], a.xyz[3 * (size_t)vi + 2], P[k]);
        Q[k][0] = a.uv[2 * (size_t)vi];
        Q[k][1] = a.uv[2 * (size_t)vi + 1];
    }
    // the texture's size (of a mesh of materials, the albedo's): loaded
    // before the cull so that its dependent loads overlap the frame arithmetic
    uint32_t tex = a.tri_tex[t];
    if (a.mat_tex) {
        if (!LFDPR_IN_BOUNDS(tex, a.n_mat, 3)) tex = 0;
        tex = a.mat_tex[tex].x;
    }
    if (!LFDPR_IN_BOUNDS(tex, a.n_tex, 2)) tex = 0;
    const uint32_t tex_w = a.tex[tex].w, tex_h = a.tex[tex].h;
#pragma unroll
    for (int k = 0; k < 8; k++) r.q[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    r.q[0] = make_float4(P[0][0], P[0][1], P[0][2], 0.0f);
    if (culled(c, ex, P)) return res;

    // area and unit normal
    float e1[3], e2[3];
#pragma unroll
    for (int k = 0; k < 3; k++) { e1[k] = P[1][k] - P[0][k]; e2[k] = P[2][k] - P[0][k]; }
    const float crx = fmaf(e1[1], e2[2], -(e1[2] * e2[1]));
    const float cry = fmaf(e1[2], e2[0], -(e1[0] * e2[2]));
    const float crz = fmaf(e1[0], e2[1], -(e1[1] * e2[0]));
    const float len2 = dot3(crx, cry, crz, crx, cry, crz);
    const float len = __fsqrt_rn(len2);
    // zero area (up to rounding: vertex-angle sine below 2^-20) emits no points
    const float e11 = dot3(e1[0], e1[1], e1[2], e1[0], e1[1], e1[2]);
    const float e22 = dot3(e2[0], e2[1], e2[2], e2[0], e2[1], e2[2]);
    if (!(len2 > 0x1p-40f * (e11 * e22)) || isinf(len)) return res;
    const float nx = __fdiv_rn(crx, len), ny = __fdiv_rn(cry, len), nz = __fdiv_rn(crz, len);
    const float A_ws = 0.5f * len;

    // T_align frame (Sec. 3.1): v-hat along the world vertical projected into
    // the plane, u-hat = v-hat x n; near-horizontal planes use world x instead.
    float ux, uy, uz, vx, vy, vz;
    {
        const float tx = -(ny * nx), ty = fmaf(-ny, ny, 1.0f), tz = -(ny * nz);
        const float l2 = dot3(tx, ty, tz, tx, ty, tz);
        if (l2 >= 1e-6f) {
            const float l = __fsqrt_rn(l2);
            vx = __fdiv_rn(tx, l); vy = __fdiv_rn(ty, l); vz = __fdiv_rn(tz, l);
            ux = fmaf(vy, nz, -(vz * ny));
            uy = fmaf(vz, nx, -(vx * nz));
            uz = fmaf(vx, ny, -(vy * nx));
        } else {
            const float sx = fmaf(-nx, nx, 1.0f), sy = -(nx * ny), sz = -(nx * nz);
            const float l = __fsqrt_rn(dot3(sx, sy, sz, sx, sy, sz));
            ux = __fdiv_rn(sx, l); uy = __fdiv_rn(sy, l); uz = __fdiv_rn(sz, l);
            vx = fmaf(ny, uz, -(nz * uy));
            vy = fmaf(nz, ux, -(nx * uz));
            vz = fmaf(nx, uy, -(ny * ux));
        }
    }

    // 2-D coordinates relative to P0 and the lattice origin (bbox min)
    const float a1 = dot3(e1[0], e1[1], e1[2], ux, uy, uz), b1 = dot3(e1[0], e1[1], e1[2], vx, vy, vz);
    const float a2 = dot3(e2[0], e2[1], e2[2], ux, uy, uz), b2 = dot3(e2[0], e2[1], e2[2], vx, vy, vz);
    const float umin = fminf(fminf(0.0f, a1), a2), vmin = fminf(fminf(0.0f, b1), b2);
    const float U[3] = {0.0f - umin, a1 - umin, a2 - umin};
    const float V[3] = {0.0f - vmin, b1 - vmin, b2 - vmin};
    const float umax = fmaxf(fmaxf(U[0], U[1]), U[2]);

    // closest and farthest eye (Fig. 5): height over the plane plus the
    // in-plane distance to the 2-D triangle; min and max over every rendered
    // view. exact_d2(v) is the defining formula for view v, and the result
    // equals its minimum and maximum over all views; views that cannot hold
    // either are ruled out without evaluating them:
    // - f(x), the exact squared distance from the eye at x to the triangle of
    //   this same binary32 frame, is convex in x: a squared distance to a
    //   convex set, taken along a line. exact_d2(v) is within E of f(x_v),
    //   E = 2^-18 (S + L)^2 = 64 u (S + L)^2 (u = 2^-24), S bounding |q|_1
    //   over the eyes and L the 2-D extent |a1| + |b1| + |a2| + |b2|: the
    //   rounding of the dot products, edge tests and segment distances stays
    //   below 30 u (S + L)^2, and the rest covers the tests' own rounding.
    // - Minimum: walking from a start view, once a view's value exceeds the
    //   one before it by 2E, f does not decrease from there on, so every later
    //   view computes at least that value - 2E, which is at least the value
    //   before it: no later view can lower the minimum. The same walking back.
    // - Maximum: between two evaluated views a < b, f lies under its chord,
    //   so the views strictly between compute at most the chord + 2E; the
    //   chord is largest at the view next to a or the one next to b.
    const float ie01 = seg_inv_len2(0.0f, 0.0f, a1, b1), ie12 = seg_inv_len2(a1, b1, a2, b2);
    const float ie20 = seg_inv_len2(a2, b2, 0.0f, 0.0f);
    const float qy = 0.0f - P[0][1], qz = c.D - P[0][2];
    auto exact_d2 = [&](int v) -> float {
        const float qx = ex[v] - P[0][0];
        const float qu = dot3(qx, qy, qz, ux, uy, uz);
        const float qv = dot3(qx, qy, qz, vx, vy, vz);
        const float h = dot3(qx, qy, qz, nx, ny, nz);
        const float w0 = edge_fn(a1, b1, a2, b2, qu, qv);
        const float w1 = edge_fn(a2, b2, 0.0f, 0.0f, qu, qv);
        const float w2 = edge_fn(0.0f, 0.0f, a1, b1, qu, qv);
        float d2 = 0.0f;
        if (!inside_either(w0, w1, w2))
            d2 = fminf(fminf(seg_dist2(0.0f, 0.0f, a1, b1, ie01, qu, qv), seg_dist2(a1, b1, a2, b2, ie12, qu, qv)),
                       seg_dist2(a2, b2, 0.0f, 0.0f, ie20, qu, qv));
        return fmaf(h, h, d2);
    };
    const int nr = c.nr;
    const float x_first = ex[0], x_last = ex[nr - 1];
    const float S = fmaxf(fabsf(x_first - P[0][0]), fabsf(x_last - P[0][0])) * 1.0001f + fabsf(qy) + fabsf(qz);
    const float SL = S + ((fabsf(a1) + fabsf(b1)) + (fabsf(a2) + fabsf(b2)));
    const float E2 = 0x1p-17f * (SL * SL);   // 2E
    const int g = nearest_eye(ex, nr, (P[0][0] + P[1][0] + P[2][0]) * (1.0f / 3.0f));
    const float fg = exact_d2(g);
    float d2min = fg, d2max = fg;
    int hi = g, lo = g;
    float f_at_hi = fg, f_at_lo = fg;   // the values of views hi and lo
    while (hi + 1 < nr) {
        const float f = exact_d2(++hi);
        d2min = fminf(d2min, f);
        d2max = fmaxf(d2max, f);
        const bool rising = f - f_at_hi >= E2;
        f_at_hi = f;
        if (rising) break;
    }
    while (lo > 0) {
        const float f = exact_d2(--lo);
        d2min = fminf(d2min, f);
        d2max = fmaxf(d2max, f);
        const bool rising = f - f_at_lo >= E2;
        f_at_lo = f;
        if (rising) break;
    }
    float f_first = 0.0f, f_last = 0.0f;
    if (lo > 0) {
        f_first = exact_d2(0);
        d2max = fmaxf(d2max, f_first);
    }
    if (hi < nr - 1) {
        f_last = exact_d2(nr - 1);
        d2max = fmaxf(d2max, f_last);
    }
    // the two gaps (0, lo) and (hi, nr - 1); d2max is final unless a gap
    // fails its chord test, and then that gap is evaluated view by view
    auto gap_clear = [&](int ga, int gb, float fa, float fb) -> bool {
        const float xa = ex[ga], span = ex[gb] - xa;
        if (!(span > 0.0f)) return false;
        const float t1 = (ex[ga + 1] - xa) / span, t2 = (ex[gb - 1] - xa) / span;
        const float cmax = fmaxf(fmaf(fb - fa, t1, fa), fmaf(fb - fa, t2, fa));
        return cmax + E2 <= d2max;
    };
    const bool clear_lo = lo < 2 || gap_clear(0, lo, f_first, f_at_lo);
    const bool clear_hi = hi > nr - 3 || gap_clear(hi, nr - 1, f_at_hi, f_last);
    if (!clear_lo)
        for (int v = 1; v < lo; v++) d2max = fmaxf(d2max, exact_d2(v));
    if (!clear_hi)
        for (int v = hi + 1; v < nr - 1; v++) d2max = fmaxf(d2max, exact_d2(v));
    const float dmin = fmaxf(__fsqrt_rn(d2min), c.near_z);
    const float dmax = fmaxf(__fsqrt_rn(d2max), c.near_z);

    // LFD-biased spacings and Eq. 1-3
    const float su0 = (c.bias_h * dmin) * c.px, sv0 = (c.bias_v * dmin) * c.py;
    const float size_xy = su0 * sv0;
    // a mesh of materials: the albedo sets the record's LOD pair, Eq. 1 takes
    // the largest texel count of the material's four textures
    const float X = float(tex_w), Y = float(tex_h);
    const float ds1 = Q[1][0] - Q[0][0], dt1 = Q[1][1] - Q[0][1];
    const float ds2 = Q[2][0] - Q[0][0], dt2 = Q[2][1] - Q[0][1];
    const float A_ts = 0.5f * fabsf(fmaf(ds1, dt2, -(dt1 * ds2)));
    float n_tex = (A_ts * X) * Y;
    if (a.mat_tex) {
        uint32_t m = a.tri_tex[t];
        if (!LFDPR_IN_BOUNDS(m, a.n_mat, 3)) m = 0;
        uint4 mt = a.mat_tex[m];
        if (!LFDPR_IN_BOUNDS(mt.y, a.n_tex, 2) || !LFDPR_IN_BOUNDS(mt.z, a.n_tex, 2) ||
            !LFDPR_IN_BOUNDS(mt.w, a.n_tex, 2))
            mt.y = mt.z = mt.w = 0;
        const uint32_t ids[3] = {mt.y, mt.z, mt.w};
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const TexDesc tk = a.tex[ids[k]];
            n_tex = fmaxf(n_tex, (A_ts * float(tk.w)) * float(tk.h));
        }
    }
    if (n_tex < 1.0f) n_tex = 1.0f;
    const float size_uv = __fdiv_rn(A_ws, n_tex);
    float su = su0, sv = sv0;
    if (size_uv > size_xy) {
        const float f = __fsqrt_rn(__fdiv_rn(size_uv, size_xy));
        su = su0 * f;
        sv = sv0 * f;
    }

    // Eq. 4-7
    const float ratio = __fdiv_rn(A_ts, A_ws);
    const float size_xy_max = ((c.bias_h * dmax) * c.px) * ((c.bias_v * dmax) * c.py);
    const float vpuv_min = size_xy * ratio, vpuv_max = size_xy_max * ratio;
    const float spl_uv = (su * sv) * ratio;
    const float lod_min = 0.5f * log2_series((vpuv_min * X) * Y);
    const float lod_max = 0.5f * log2_series((vpuv_max * X) * Y);

    // affine texture map over the lattice frame
    const float det = fmaf(a1, b2, -(a2 * b1));
    float gsu = 0.0f, gsv = 0.0f, gtu = 0.0f, gtv = 0.0f;
    if (det != 0.0f) {
        gsu = __fdiv_rn(fmaf(ds1, b2, -(ds2 * b1)), det);
        gsv = __fdiv_rn(fmaf(ds2, a1, -(ds1 * a2)), det);
        gtu = __fdiv_rn(fmaf(dt1, b2, -(dt2 * b1)), det);
        gtv = __fdiv_rn(fmaf(dt2, a1, -(dt1 * a2)), det);
    }
    const float s0 = fmaf(gsu, umin, fmaf(gsv, vmin, Q[0][0]));
    const float t0 = fmaf(gtu, umin, fmaf(gtv, vmin, Q[0][1]));

    r.q[0].w = su;
    r.q[1] = make_float4(ux, uy, uz, sv);
    r.q[2] = make_float4(vx, vy, vz, umin);
    r.q[3] = make_float4(nx, ny, nz, vmin);
    r.q[4] = make_float4(a1, b1, a2, b2);
    r.q[5] = make_float4(spl_uv, vpuv_min, vpuv_max, umax);
    r.q[6] = make_float4(s0, gsu, gsv, t0);
    r.q[7] = make_float4(gtu, gtv, lod_min, lod_max);

    // point count: one per lattice cell overlapping the triangle
    const float ncol = ceilf(__fdiv_rn(umax, su));
    if (!(ncol <= float(kMaxCell))) { res.cell_overflow = true; return res; }
    const int cols = int(ncol);
    uint32_t cnt = 0;
    // the column summary for k_emit, stored word by word as the columns are
    // found (a wider triangle, or a column of 2^16 rows, is marked for a walk)
    uint32_t* cs = a.colsum ? reinterpret_cast<uint32_t*>(a.colsum + t) : nullptr;
    bool summary = cols <= 4;
    ColumnWalk walk(U, V, su, sv, umax);
    for (int i = 0; i < cols; i++) {
        int j0, j1;
        const int rows = walk.rows(i, &j0, &j1);
        if (j1 > kMaxCell + 1) { res.cell_overflow = true; return res; }
        cnt += uint32_t(rows);
        summary &= rows <= 0xffff;
        if (cs && summary) cs[i] = uint32_t(j0) | (uint32_t(rows) << 16);
    }
    if (cs && !summary) cs[0] = kColSumWalk;
    res.count = cnt;
    res.live = true;
    // the splat's per-triangle projection constants
    float pA[3], pB[3], pY[3];
#pragma unroll
    for (int k = 0; k < 3; k++)
        project_point(c.D, c.x0, c.y0, c.ipw, c.iph, P[k][0], P[k][1], P[k][2], pA[k], pB[k], pY[k]);
    tp.a = make_float4(pA[0], pA[1], pA[2], fminf(fminf(P[0][2], P[1][2]), P[2][2]));
    tp.b = make_float4(pB[0], pB[1], pB[2], fmaxf(fmaxf(P[0][2], P[1][2]), P[2][2]));
    tp.y = make_float4(pY[0], pY[1], pY[2], 0.0f);
    return res;
}

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* smem) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    T tot = 0;
    if (threadIdx.x < 32) {
        tot = threadIdx.x < (blockDim.x >> 5) ? smem[threadIdx.x] : T(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    return tot;   // valid in thread 0
}

__global__ void __launch_bounds__(kSetupThreads, 4) k_setup(FrameArgs a) {
    wait_previous_kernel();
    allow_next_kernel();
    __shared__ uint32_t s_cnt[kSetupThreads / 32];
    __shared__ uint32_t s_live[kSetupThreads / 32];
    __shared__ float s_ex[kMaxRenderViews];
    for (int v = threadIdx.x; v < a.dc.nr; v += blockDim.x) s_ex[v] = a.ex[v];
    __syncthreads();
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t count = 0, live = 0;
    if (t < a.n_tris) {
        TriRec r;
        TriProj tp;
        const SetupOut o = setup_triangle(a, s_ex, t, r, tp);
        TriRec* dst = a.rec + t;
#pragma unroll
        for (int k = 0; k < 8; k++) dst->q[k] = r.q[k];
        if (o.live && a.tproj) a.tproj[t] = tp;
        count = o.count;
        live = o.live ? 1u : 0u;
        a.counts[t] = count;
        if (o.cell_overflow) atomicExch(&a.ctr->cell_overflow, 1u);
    }
    const uint32_t bs = block_sum(count, s_cnt);
    const uint32_t bl = block_sum(live, s_live);
    if (threadIdx.x == 0) {
        a.block_sums[blockIdx.x] = bs;
        if (bl) atomicAdd(&a.ctr->n_live, bl);
    }
}

// Exclusive scan of the per-block point counts in one block of 1024 threads:
// each thread sums a contiguous run of ceil(n / 1024) block sums, the block
// scans those 1024 sums, and each thread writes its run's prefixes; the
// total decides overflow. Prefixes saturate at 2^32 - 1.
__global__ void __launch_bounds__(1024) k_scan(FrameArgs a) {
    wait_previous_kernel();
    allow_next_kernel();
    __shared__ unsigned long long s_warp[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t n = a.n_blocks, per = (n + 1023u) / 1024u;
    const uint32_t lo = min(n, threadIdx.x * per), hi = min(n, lo + per);
    unsigned long long run = 0ull;
    for (uint32_t k = lo; k < hi; k++) run += a.block_sums[k];
    unsigned long long inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = s_warp[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        s_warp[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    unsigned long long excl = (warp > 0 ? s_warp[warp - 1] : 0ull) + inc - run;
    for (uint32_t k = lo; k < hi; k++) {
        const uint32_t v = a.block_sums[k];
        a.block_sums[k] = uint32_t(excl > 0xffffffffull ? 0xffffffffull : excl);
        excl += v;
    }
    if (threadIdx.x == 1023) {
        const unsigned long long total = s_warp[31];
        a.ctr->n_points = uint32_t(total > 0xffffffffull ? 0xffffffffull : total);
        a.ctr->overflow = total > (unsigned long long)a.max_points ? 1u : 0u;
    }
}

// The n points of triangle t from point id p on, in (column, row) order: a
// single thread (lanes = 1) or a warp's lanes side by side in each column.
__device__ __forceinline__ void emit_points(const FrameArgs& a, uint32_t t, uint32_t p, uint32_t n, int lane,
                                            int lanes) {
    if (a.colsum) {
        // the columns k_setup found, without walking them again; the words
        // past the last column are not written, and are not read: the
        // columns before them hold all n points
        const uint4 cs = a.colsum[t];
        if (cs.x != kColSumWalk) {
            const uint32_t w[4] = {cs.x, cs.y, cs.z, cs.w};
            const uint32_t end = p + n;
#pragma unroll
            for (int i = 0; i < 4; i++) {
                if (p == end) break;
                const uint32_t j0 = w[i] & 0xffffu, rows = w[i] >> 16;
                for (uint32_t r = uint32_t(lane); r < rows; r += uint32_t(lanes)) {
                    const uint32_t q = p + r;
                    if (LFDPR_IN_BOUNDS(q, a.max_points, 4))
                        *reinterpret_cast<uint2*>(a.points + q) = make_uint2(t, uint32_t(i) | ((j0 + r) << 16));
                }
                p += rows;
            }
            return;
        }
    }
    const TriRec* rp = a.rec + t;
    TriRec r;
    r.q[0] = rp->q[0]; r.q[1] = rp->q[1]; r.q[2] = rp->q[2]; r.q[3] = rp->q[3];
    r.q[4] = rp->q[4]; r.q[5] = rp->q[5];
    float U[3], V[3];
    shifted_uv(r, U, V);
    const float su = r.q[0].w, sv = r.q[1].w, umax = r.q[5].w;
    const int cols = int(ceilf(__fdiv_rn(umax, su)));
    ColumnWalk walk(U, V, su, sv, umax);
    for (int i = 0; i < cols; i++) {
        int j0, j1;
        walk.rows(i, &j0, &j1);
        for (int j = j0 + lane; j < j1; j += lanes) {
            const uint32_t q = p + uint32_t(j - j0);
            if (LFDPR_IN_BOUNDS(q, a.max_points, 4))
                *reinterpret_cast<uint2*>(a.points + q) = make_uint2(t, uint32_t(i) | (uint32_t(j) << 16));
        }
        p += uint32_t(j1 - j0);
    }
}

// Block-level exclusive scan of the counts (warp shuffles), plus the block's
// offset: each triangle's first point id. Then emit its points in (column,
// row) order; the block's triangles of more than kEmitBig points are listed
// in shared memory and emitted afterwards by the block's warps, a warp each,
// so that one thread does not walk tens of thousands of points.
__global__ void __launch_bounds__(kSetupThreads) k_emit(FrameArgs a) {
    wait_previous_kernel();
    allow_next_kernel();
    __shared__ uint32_t s_warp[kSetupThreads / 32];
    __shared__ uint32_t s_big[kSetupThreads], s_first[kSetupThreads];
    __shared__ uint32_t s_nbig;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t cnt = t < a.n_tris ? a.counts[t] : 0u;
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t n = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += n;
    }
    if (lane == 31) s_warp[warp] = inc;
    if (threadIdx.x == 0) s_nbig = 0u;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kSetupThreads / 32 ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t n = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += n;
        }
        if (lane < kSetupThreads / 32) s_warp[lane] = w;
    }
    __syncthreads();
    const bool overflow = a.ctr->overflow != 0u;
    if (t < a.n_tris) {
        const uint32_t first = a.block_sums[blockIdx.x] + (warp > 0 ? s_warp[warp - 1] : 0u) + inc - cnt;
        a.offsets[t] = first;
        if (cnt > kEmitBig && !overflow) {
            const uint32_t b = atomicAdd(&s_nbig, 1u);
            s_big[b] = t;
            s_first[b] = first;
        } else if (cnt > 0 && !overflow) {
            emit_points(a, t, first, cnt, 0, 1);
        }
    }
    __syncthreads();
    for (uint32_t b = uint32_t(warp); b < s_nbig; b += kSetupThreads / 32)
        emit_points(a, s_big[b], s_first[b], a.counts[s_big[b]], lane, 32);
}

// One mip level's bilinear sample at texture coordinates (fs, ft) in [0, 1):
// wrap addressing, texel centres at (k+1/2)/w. Loading the four texels and
// blending them are separate steps, so that every load of a point can be in
// flight before the first blend.
struct BilinearTap {
    uint32_t tex[4];
    float fx, fy;
};
__device__ __forceinline__ void bilinear_load(const uint8_t* __restrict__ pool, const uint64_t* __restrict__ loff,
                                              uint32_t w, uint32_t h, int l, float fs, float ft, BilinearTap& b) {
    const uint32_t lw = (w >> l) ? (w >> l) : 1u, lh = (h >> l) ? (h >> l) : 1u;
    const float x = fmaf(fs, float(lw), -0.5f), y = fmaf(ft, float(lh), -0.5f);
    const float xf = floorf(x), yf = floorf(y);
    b.fx = x - xf;
    b.fy = y - yf;
    const uint32_t ix0 = uint32_t(int(xf)) & (lw - 1), iy0 = uint32_t(int(yf)) & (lh - 1);
    const uint32_t ix1 = (ix0 + 1) & (lw - 1), iy1 = (iy0 + 1) & (lh - 1);
    const uint32_t* T = reinterpret_cast<const uint32_t*>(pool + __ldg(loff + l));
    b.tex[0] = __ldg(T + (size_t)iy0 * lw + ix0);
    b.tex[1] = __ldg(T + (size_t)iy0 * lw + ix1);
    b.tex[2] = __ldg(T + (size_t)iy1 * lw + ix0);
    b.tex[3] = __ldg(T + (size_t)iy1 * lw + ix1);
}
__device__ __forceinline__ float bilinear_channel(const BilinearTap& b, int ch) {
    const float va = float((b.tex[0] >> (8 * ch)) & 255u), vb = float((b.tex[1] >> (8 * ch)) & 255u);
    const float vc = float((b.tex[2] >> (8 * ch)) & 255u), vd = float((b.tex[3] >> (8 * ch)) & 255u);
    const float top = fmaf(b.fx, vb - va, va);
    const float bot = fmaf(b.fx, vd - vc, vc);
    return fmaf(b.fy, bot - top, top);
}

// The two trilinear fetches of a point (Sec. 3.3: tv_min at lod_a, tv_max at
// lod_b). Each: LOD clamped to [0, L_max], level floor(LOD) blended to the
// next by the fraction (FP32 weights), bilinear, rounded half-even to RGBA8.
// The levels are A = floor(lod_a), B = min(A + 1, L) and C = floor(lod_b),
// D = min(C + 1, L) with C >= A; when C is A (then D is B) or C is B, those
// levels' samples are shared instead of loaded and blended twice (the LOD
// pair of a triangle mostly lies within one level). loff[l] is the byte
// offset of level l in the pool.
__device__ __forceinline__ void trilinear_pair(const uint8_t* __restrict__ pool, const uint64_t* __restrict__ loff,
                                               uint32_t w, uint32_t h, int L, float s, float t, float lod_a,
                                               float lod_b, uint32_t& out_a, uint32_t& out_b) {
    if (!isfinite(s)) s = 0.0f;
    if (!isfinite(t)) t = 0.0f;
    const float fs = s - floorf(s), ft = t - floorf(t);
    float lods[2] = {lod_a, lod_b}, frac[2];
    int lev[2];
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const float lod = fminf(fmaxf(lods[q], 0.0f), float(L));
        lev[q] = int(floorf(lod));
        frac[q] = lod - float(lev[q]);
    }
    const int A = lev[0], B = A + 1 > L ? L : A + 1, C = lev[1], D = C + 1 > L ? L : C + 1;
    // C is A (then D is B) or B for almost every triangle: three taps, the
    // third at D; C beyond B takes its own tap in place of A's for the
    // second fetch
    const bool far_c = C != A && C != B;
    BilinearTap ta, tb, te;
    bilinear_load(pool, loff, w, h, A, fs, ft, ta);
    bilinear_load(pool, loff, w, h, B, fs, ft, tb);
    bilinear_load(pool, loff, w, h, D, fs, ft, te);
    uint32_t out[2] = {0u, 0u};
    const bool blend0 = frac[0] > 0.0f && lev[0] < L, blend1 = frac[1] > 0.0f && lev[1] < L;
#pragma unroll
    for (int ch = 0; ch < 4; ch++) {
        const float va = bilinear_channel(ta, ch), vb = bilinear_channel(tb, ch);
        const float v0 = blend0 ? fmaf(frac[0], vb - va, va) : va;
        out[0] |= uint32_t(round_u8(v0)) << (8 * ch);
        if (!far_c) {
            const float vc = C == A ? va : vb;
            const float vd = C == A ? vb : bilinear_channel(te, ch);
            const float v1 = blend1 ? fmaf(frac[1], vd - vc, vc) : vc;
            out[1] |= uint32_t(round_u8(v1)) << (8 * ch);
        }
    }
    if (far_c) {
        bilinear_load(pool, loff, w, h, C, fs, ft, ta);
#pragma unroll
        for (int ch = 0; ch < 4; ch++) {
            const float vc = bilinear_channel(ta, ch), vd = bilinear_channel(te, ch);
            const float v1 = blend1 ? fmaf(frac[1], vd - vc, vc) : vc;
            out[1] |= uint32_t(round_u8(v1)) << (8 * ch);
        }
    }
    out_a = out[0];
    out_b = out[1];
}

// Cell corner (a s_u + umin, b s_v + vmin) of the lattice frame in world space.
__device__ __forceinline__ void lattice_corner(const float4& q0, const float4& q1, const float4& q2,
                                               const float4& q3, int ia, int jb, float* o) {
    const float cu = float(ia) * q0.w + q2.w;
    const float cv = float(jb) * q1.w + q3.w;
    o[0] = fmaf(cu, q1.x, fmaf(cv, q2.x, q0.x));
    o[1] = fmaf(cu, q1.y, fmaf(cv, q2.y, q0.y));
    o[2] = fmaf(cu, q1.z, fmaf(cv, q2.z, q0.z));
}

// Bounds of a convex polygon's x-extent within the band of pixel rows
// ya <= y <= yb, for every eye in [-E, E] (projected vertices: pixel
// x = A + B Ex, y = Y): a lower and an upper line x = a + b Ex, as
// L = (lower a, b, upper a, b).
//
// The extent within the band is reached at the vertices inside it or where
// its two boundary rows cross the edges (half-open in y); each such point
// moves along a line in Ex. A crossing at fraction f along its edge is taken
// as the two lines at f -+ kCrossDy / |dy| (clamped to the edge's ends): the
// projected y carry errors of about 2e-4 pixel, so the true crossing lies
// between them, and a steep edge gives two nearly equal lines while a flat
// one gives its two ends. A band that misses the polygon (a margin row)
// takes every vertex. The lower bound is the chord, between the extreme eyes
// -E and +E, of the minimum of those lines: the minimum of lines is concave,
// so the chord lies below it, and it is the minimum itself where one line
// stays lowest. The upper bound likewise. Each point enters only through its
// x at the two extreme eyes, so the bounds need no branch per point.
constexpr float kCrossDy = 1e-3f;
template <int N>
__device__ __forceinline__ void band_bounds(const float* A, const float* B, const float* Y, float ya, float yb,
                                            float E, float cross_dy, float4& L) {
    float xm[N], xp[N];   // x at eye -E and at eye +E
#pragma unroll
    for (int k = 0; k < N; k++) {
        xm[k] = fmaf(-B[k], E, A[k]);
        xp[k] = fmaf(B[k], E, A[k]);
    }
    float lm = INFINITY, lp = INFINITY, um = -INFINITY, up = -INFINITY;
    auto fold = [&](bool on, float m, float p) {
        if (on) {
            lm = fminf(lm, m);
            lp = fminf(lp, p);
            um = fmaxf(um, m);
            up = fmaxf(up, p);
        }
    };
#pragma unroll
    for (int k = 0; k < N; k++) fold(Y[k] >= ya && Y[k] <= yb, xm[k], xp[k]);
    // an edge's reciprocal height is used only where a row crosses it (so
    // its height is not zero)
    float rdy[N];
#pragma unroll
    for (int e = 0; e < N; e++) rdy[e] = __fdividef(1.0f, Y[e + 1 == N ? 0 : e + 1] - Y[e]);
    auto row_crossings = [&](float yc) {
#pragma unroll
        for (int e = 0; e < N; e++) {
            const int p = e, q = e + 1 == N ? 0 : e + 1;
            const bool cross = (Y[p] <= yc && yc < Y[q]) || (Y[q] <= yc && yc < Y[p]);
            const float dxm = xm[q] - xm[p], dxp = xp[q] - xp[p];
            const float f = (yc - Y[p]) * rdy[e], d = cross_dy * fabsf(rdy[e]);
            const float f0 = fmaxf(f - d, 0.0f), f1 = fminf(f + d, 1.0f);
            fold(cross, fmaf(f0, dxm, xm[p]), fmaf(f0, dxp, xp[p]));
            fold(cross, fmaf(f1, dxm, xm[p]), fmaf(f1, dxp, xp[p]));
        }
    };
    row_crossings(ya);
    // a band of one row (most cells are at most a pixel high) has no second
    // boundary row
    if (yb > ya) row_crossings(yb);
    if (!(lm <= um)) {
#pragma unroll
        for (int k = 0; k < N; k++) fold(true, xm[k], xp[k]);
    }
    const float hE = E > 0.0f ? __fdividef(0.5f, E) : 0.0f;
    L = make_float4(0.5f * (lm + lp), (lp - lm) * hE, 0.5f * (um + up), (up - um) * hE);
}

// Points whose cell or triangle reaches within near_z of the eyes' plane are
// projected with up to D / near_z magnification and, past the plane, not at
// all. Their cell and triangle are clipped to depth D - z >= near_z first (a
// plane shared by every view: all eyes lie at z = D), which leaves bounded
// polygons whose vertices project affinely in Ex like any other; candidate
// bounds then come from band_bounds with a margin kNearPad (and crossing
// uncertainty kNearCrossDy) sized for that magnification. Hits nearer than
// near_z are rejected by the per-pixel test as everywhere.
constexpr float kNearPad = 1.0f / 16.0f;
constexpr float kNearCrossDy = 1.0f / 32.0f;

// Clip the convex polygon V (N world vertices) to z <= zc (Sutherland-
// Hodgman against one plane): at most N + 1 vertices, written to O and padded
// to N + 1 by repeating the last one (repeated vertices add no area and cross
// no row). Returns the vertex count (below 3: nothing left).
template <int N>
__device__ __forceinline__ int clip_below(const float (&V)[N][3], float zc, float (&O)[N + 1][3]) {
    int m = 0;
#pragma unroll
    for (int k = 0; k < N; k++) {
        const float* p = V[k];
        const float* q = V[k + 1 == N ? 0 : k + 1];
        const bool pin = p[2] <= zc, qin = q[2] <= zc;
        if (pin) {
            O[m][0] = p[0];
            O[m][1] = p[1];
            O[m][2] = p[2];
            m++;
        }
        if (pin != qin) {
            const float f = __fdiv_rn(zc - p[2], q[2] - p[2]);
            O[m][0] = fmaf(f, q[0] - p[0], p[0]);
            O[m][1] = fmaf(f, q[1] - p[1], p[1]);
            O[m][2] = zc;
            m++;
        }
    }
    for (int k = m; k < N + 1; k++) {
        O[k][0] = m ? O[m - 1][0] : 0.0f;
        O[k][1] = m ? O[m - 1][1] : 0.0f;
        O[k][2] = m ? O[m - 1][2] : zc;
    }
    return m;
}

// The splat record of such a point: candidate rows and column bounds of the
// clipped cell and triangle (L0, L1, not yet shifted to pixel columns), and
// Eq. 8's area coefficients of the clipped cell (its drawable part).
struct NearRec {
    uint32_t y0, ny;
    float4 L0, L1;
    float alpha, beta;
};
__device__ __forceinline__ NearRec near_record(const DispConst& c, const float4& q0, const float4& q1,
                                               const float4& q2, const float4& q3, const float4& q4, int i, int j,
                                               bool interior) {
    const float zc = c.D - c.near_z;
    NearRec o;
    o.y0 = 0;
    o.ny = 0;
    o.L0 = make_float4(-INFINITY, 0.0f, INFINITY, 0.0f);
    o.L1 = o.L0;
    o.alpha = 0.0f;
    o.beta = 0.0f;
    float Cw[4][3];
#pragma unroll
    for (int k = 0; k < 4; k++)
        lattice_corner(q0, q1, q2, q3, i + (k == 1 || k == 2), j + (k >= 2), Cw[k]);
    float P[5][3];
    const int m = clip_below<4>(Cw, zc, P);
    if (m < 3) return o;
    // the triangle's vertices from the lattice frame: P0 + a u-hat + b v-hat
    float Tw[3][3];
    Tw[0][0] = q0.x;
    Tw[0][1] = q0.y;
    Tw[0][2] = q0.z;
#pragma unroll
    for (int k = 0; k < 2; k++) {
        const float aa = k ? q4.z : q4.x, bb = k ? q4.w : q4.y;
        Tw[k + 1][0] = fmaf(aa, q1.x, fmaf(bb, q2.x, q0.x));
        Tw[k + 1][1] = fmaf(aa, q1.y, fmaf(bb, q2.y, q0.y));
        Tw[k + 1][2] = fmaf(aa, q1.z, fmaf(bb, q2.z, q0.z));
    }
    float Q[4][3];
    const int mt = clip_below<3>(Tw, zc, Q);
    float A[5], B[5], Y[5], s[5];
#pragma unroll
    for (int k = 0; k < 5; k++) {
        s[k] = __fdiv_rn(c.D, c.D - P[k][2]);
        project_point(c.D, c.x0, c.y0, c.ipw, c.iph, P[k][0], P[k][1], P[k][2], A[k], B[k], Y[k]);
    }
    // Eq. 8: the clipped cell's shoelace sum relative to its first vertex
    const float cx0 = P[0][0] * s[0], cy0 = P[0][1] * s[0];
    float da[4], db[4], dy[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        da[k] = fmaf(P[k + 1][0], s[k + 1], -cx0) * c.ipw;
        db[k] = (s[0] - s[k + 1]) * c.ipw;
        dy[k] = fmaf(-P[k + 1][1], s[k + 1], cy0) * c.iph;
    }
#pragma unroll
    for (int k = 0; k < 3; k++) {
        o.alpha = o.alpha + fmaf(da[k], dy[k + 1], -(da[k + 1] * dy[k]));
        o.beta = o.beta + fmaf(db[k], dy[k + 1], -(db[k + 1] * dy[k]));
    }
    if (mt < 3) return o;   // no part of the triangle can be drawn
    float tA[4], tB[4], tY[4];
#pragma unroll
    for (int k = 0; k < 4; k++)
        project_point(c.D, c.x0, c.y0, c.ipw, c.iph, Q[k][0], Q[k][1], Q[k][2], tA[k], tB[k], tY[k]);
    float cymn = Y[0], cymx = Y[0], tymn = tY[0], tymx = tY[0];
#pragma unroll
    for (int k = 1; k < 5; k++) {
        cymn = fminf(cymn, Y[k]);
        cymx = fmaxf(cymx, Y[k]);
    }
#pragma unroll
    for (int k = 1; k < 4; k++) {
        tymn = fminf(tymn, tY[k]);
        tymx = fmaxf(tymx, tY[k]);
    }
    const float fy0 = fmaxf(ceilf(fmaxf(cymn, tymn) - 0.5f - kNearPad), 0.0f);
    const float fy1 = fminf(floorf(fminf(cymx, tymx) - 0.5f + kNearPad), float(c.H - 1));
    if (!(fy0 <= fy1)) return o;
    o.y0 = uint32_t(int(fy0));
    o.ny = uint32_t(int(fy1) - int(fy0) + 1);
    const float ya = float(o.y0) + 0.5f, yb = float(o.y0 + o.ny - 1u) + 0.5f;
    band_bounds<5>(A, B, Y, ya, yb, c.ex_max, kNearCrossDy, o.L0);
    if (!interior) band_bounds<4>(tA, tB, tY, ya, yb, c.ex_max, kNearCrossDy, o.L1);
    return o;
}

// One thread per point: tv_min / tv_max (Sec. 3.3), then the point's splat
// record (its cell's projection into the views, candidate rows, flags), and
// the point joins the splat's work list if some view can hold a candidate
// pixel of it.
__global__ void __launch_bounds__(256, 4) k_fetch(FrameArgs a) {
    wait_previous_kernel();
    allow_next_kernel();
    const DispConst& c = a.dc;
    const uint32_t n = a.ctr->overflow ? 0u : a.ctr->n_points;
    const float H1 = float(c.H - 1);
    const int lane = threadIdx.x & 31;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        uint2 pt = *reinterpret_cast<const uint2*>(a.points + p);
        if (!LFDPR_IN_BOUNDS(pt.x, a.n_tris, 5)) pt.x = 0;
        const TriRec* r = a.rec + pt.x;
        // the thread's next point's triangle, read now: its record and
        // projection lines are asked of L1 while this point's texels load
        const uint32_t pnext = p + gridDim.x * blockDim.x;
        const uint32_t tnext = pnext < n ? a.points[pnext].x : 0xffffffffu;
        // the texture map and spacings first; the frame (the same 128-byte
        // line) after the fetch, so it does not stay live across the gathers
        const float su = __ldg(&r->q[0].w), sv = __ldg(&r->q[1].w);
        const float4 q6 = __ldg(&r->q[6]), q7 = __ldg(&r->q[7]);
        const uint32_t i = pt.y & 0xffffu, j = pt.y >> 16;
        const float uc = (float(i) + 0.5f) * su;
        const float vc = (float(j) + 0.5f) * sv;
        const float s = fmaf(q6.y, uc, fmaf(q6.z, vc, q6.x));
        const float t = fmaf(q7.x, uc, fmaf(q7.y, vc, q6.w));
        uint32_t texid = __ldg(a.tri_tex + pt.x);
        if (a.mat_tex) texid = __ldg(&a.mat_tex[texid].x);   // a material's albedo (k_fetch_mat: its other maps)
        const TexDesc td = a.tex[texid];
        uint32_t tmin, tmax;
        trilinear_pair(a.pool, a.lvl + (size_t)texid * kMaxLevels, td.w, td.h, int(td.levels) - 1, s, t, q7.z,
                       q7.w, tmin, tmax);
        *(reinterpret_cast<uint2*>(a.points + p) + 1) = make_uint2(tmin, tmax);
        if (tnext < a.n_tris) {
            prefetch_l1(a.rec + tnext);
            prefetch_l1(a.tproj + tnext);
        }
        const float4 q0 = __ldg(&r->q[0]), q1 = __ldg(&r->q[1]), q2 = __ldg(&r->q[2]);
        const float4 q3 = __ldg(&r->q[3]), q4 = __ldg(&r->q[4]), q5 = __ldg(&r->q[5]);

        // splat work record
        const TriProj tp = a.tproj[pt.x];
        float Cw[4][3];
        // the cell or its triangle reaches depth D - z < near_z: clipped path
        bool near = !((c.D - tp.b.w) >= c.near_z);
        bool interior = true;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int ia = int(i) + (k == 1 || k == 2), jb = int(j) + (k >= 2);
            lattice_corner(q0, q1, q2, q3, ia, jb, Cw[k]);
            near |= !((c.D - Cw[k][2]) >= c.near_z);
            const float uu = float(ia) * su + q2.w, vv = float(jb) * sv + q3.w;
            interior &= edge_fn(q4.x, q4.y, q4.z, q4.w, uu, vv) >= 0.0f &&
                        edge_fn(q4.z, q4.w, 0.0f, 0.0f, uu, vv) >= 0.0f &&
                        edge_fn(0.0f, 0.0f, q4.x, q4.y, uu, vv) >= 0.0f;
        }
        const bool depth_ok = !near && (c.D - tp.a.w) <= c.far_z;
        const uint32_t flags = (interior ? kFlagInterior : 0u) | (depth_ok ? kFlagDepthOk : 0u);
        uint32_t y0 = 0, ny = 0;
        float alpha, beta, pad;
        // candidate columns: lower and upper lines of the cell's and of the
        // triangle's x-extent within the band of candidate rows (none where
        // the triangle is one cell, or the cell lies inside its triangle)
        float4 L0 = make_float4(-INFINITY, 0.0f, INFINITY, 0.0f), L1 = L0;
        if (!near) {
            pad = kBoxPad;
            float A[4], B[4], Y[4], Cs[4];
#pragma unroll
            for (int k = 0; k < 4; k++) {
                Cs[k] = __fdiv_rn(c.D, c.D - Cw[k][2]);
                project_point(c.D, c.x0, c.y0, c.ipw, c.iph, Cw[k][0], Cw[k][1], Cw[k][2], A[k], B[k], Y[k]);
            }
            const float cymn = fminf(fminf(Y[0], Y[1]), fminf(Y[2], Y[3]));
            const float cymx = fmaxf(fmaxf(Y[0], Y[1]), fmaxf(Y[2], Y[3]));
            const float tymn = fminf(fminf(tp.y.x, tp.y.y), tp.y.z), tymx = fmaxf(fmaxf(tp.y.x, tp.y.y), tp.y.z);
            const float fy0 = fmaxf(ceilf(fmaxf(cymn, tymn) - 0.5f - kBoxPad), 0.0f);
            const float fy1 = fminf(floorf(fminf(cymx, tymx) - 0.5f + kBoxPad), H1);
            if (fy0 <= fy1) {
                y0 = uint32_t(int(fy0));
                ny = uint32_t(int(fy1) - int(fy0) + 1);
                const float ya = float(y0) + 0.5f, yb = float(y0 + ny - 1u) + 0.5f;
                const float tA3[3] = {tp.a.x, tp.a.y, tp.a.z}, tB3[3] = {tp.b.x, tp.b.y, tp.b.z};
                const float tY3[3] = {tp.y.x, tp.y.y, tp.y.z};
                if (__ldg(a.counts + pt.x) != 1u) band_bounds<4>(A, B, Y, ya, yb, c.ex_max, kCrossDy, L0);
                if (!interior) band_bounds<3>(tA3, tB3, tY3, ya, yb, c.ex_max, kCrossDy, L1);
            }
            // Eq. 8's projected cell area is |alpha + beta Ex| / 2: a corner's pixel
            // x is (x s - x0) W/fw + (1 - s) W/fw Ex (s = D / (D - z)), its pixel y
            // (y0 - y s) H/fh the same in every view, so the shoelace sum of the
            // corners taken relative to the first one is affine in Ex; the
            // differences are formed before scaling so that x0 and y0 cancel exactly
            float da[3], db[3], dy[3];
            const float cx0 = Cw[0][0] * Cs[0], cy0 = Cw[0][1] * Cs[0];
#pragma unroll
            for (int k = 0; k < 3; k++) {
                da[k] = fmaf(Cw[k + 1][0], Cs[k + 1], -cx0) * c.ipw;
                db[k] = (Cs[0] - Cs[k + 1]) * c.ipw;
                dy[k] = fmaf(-Cw[k + 1][1], Cs[k + 1], cy0) * c.iph;
            }
            alpha = fmaf(da[0], dy[1], -(da[1] * dy[0])) + fmaf(da[1], dy[2], -(da[2] * dy[1]));
            beta = fmaf(db[0], dy[1], -(db[1] * dy[0])) + fmaf(db[1], dy[2], -(db[2] * dy[1]));
        } else {
            // listed for k_near_work, which writes its record
            pad = kNearPad;
            alpha = 0.0f;
            beta = 0.0f;
        }
        if (ny > 0) {
            // shifted so the splat converts them straight to pixel columns:
            // pixel centres at x + 1/2, candidate margin `pad` on each side
            L0.x = L0.x - (0.5f + pad);
            L1.x = L1.x - (0.5f + pad);
            L0.z = L0.z - (0.5f - pad);
            L1.z = L1.z - (0.5f - pad);
            // No candidate column in any view: a correctly rounded fmaf is
            // monotone in Ex, so over eyes in [-E, E] the splat's lower
            // line stays above the larger of its two lines' smaller end
            // values and its upper line below the smaller of their larger
            // end values; no integer between those two leaves every view
            // empty and the point joins no work list.
            const float E = c.ex_max;
            const float l0m = fmaf(L0.y, -E, L0.x), l0p = fmaf(L0.y, E, L0.x);
            const float l1m = fmaf(L1.y, -E, L1.x), l1p = fmaf(L1.y, E, L1.x);
            const float h0m = fmaf(L0.w, -E, L0.z), h0p = fmaf(L0.w, E, L0.z);
            const float h1m = fmaf(L1.w, -E, L1.z), h1p = fmaf(L1.w, E, L1.z);
            const bool ordered = !(isnan(l0m) | isnan(l0p) | isnan(l1m) | isnan(l1p) | isnan(h0m) | isnan(h0p) |
                                   isnan(h1m) | isnan(h1p));
            const float xlo = fmaxf(ceilf(fmaxf(fminf(l0m, l0p), fminf(l1m, l1p))), 0.0f);
            const float xhi = fminf(floorf(fminf(fmaxf(h0m, h0p), fmaxf(h1m, h1p))), float(c.W - 1));
            if (ordered && xlo > xhi) ny = 0;
        }
        ResolveRec* rr = a.rrec + p;
        rr->a = make_float4(alpha, beta, q5.x, q5.y);
        rr->b = make_uint4(__float_as_uint(q5.z), tmin, tmax, 0u);

        // warp-aggregated appends: points with candidate rows to the work
        // list, points reaching within near_z of the eyes' plane to the near list
        const unsigned mask = __activemask();
        const int leader = __ffs(mask) - 1;
        const unsigned below = (1u << lane) - 1u;
        const unsigned bal = __ballot_sync(mask, ny > 0);
        const unsigned bnear = __ballot_sync(mask, near);
        uint32_t base = 0, nbase = 0;
        if (lane == leader) {
            if (bal) base = atomicAdd(&a.ctr->n_work, uint32_t(__popc(bal)));
            if (bnear) nbase = atomicAdd(&a.ctr->n_near, uint32_t(__popc(bnear)));
        }
        base = __shfl_sync(mask, base, leader);
        nbase = __shfl_sync(mask, nbase, leader);
        if (ny > 0 && LFDPR_IN_BOUNDS(base + __popc(bal & below), a.max_points, 6)) {
            WorkRec* w = a.work + base + __popc(bal & below);
            w->L0 = L0;
            w->L1 = L1;
            w->meta = make_uint4(y0 | (ny << 14) | (flags << 29), pt.y, pt.x, p);
        }
        if (near && LFDPR_IN_BOUNDS(nbase + __popc(bnear & below), a.max_points, 7))
            a.near[nbase + __popc(bnear & below)] = p;
    }
    // the splat's depth keys reset to empty (all ones) at the end of the
    // pass, so that they are still in L2 when the splat starts (the frame's
    // key clear, when clear_keys is set)
    if (a.clear_keys) {
        const uint64_t n8 = uint64_t(c.W) * uint64_t(c.H) * uint64_t(c.nr), n16 = n8 / 2u;
        uint4* k16 = reinterpret_cast<uint4*>(a.keys);
        const uint4 ones = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
        const uint64_t first = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
        for (uint64_t i = first; i < n16; i += uint64_t(gridDim.x) * blockDim.x) k16[i] = ones;
        if (first == 0 && (n8 & 1u)) a.keys[n8 - 1] = ~0ull;
    }
}

// The splat records of the near list (run after k_fetch): each point's cell
// and triangle clipped to depth >= near_z (near_record), its work record
// appended to the work list if some view can hold a candidate pixel, and
// Eq. 8's coefficients of the clipped cell in its resolve record.
__global__ void __launch_bounds__(256) k_near_work(FrameArgs a) {
    wait_previous_kernel();
    allow_next_kernel();
    if (a.ctr->overflow) return;
    const DispConst& c = a.dc;
    const uint32_t n = a.ctr->n_near;
    const int lane = threadIdx.x & 31;
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint32_t p = a.near[k];
        if (!LFDPR_IN_BOUNDS(p, a.max_points, 8)) continue;
        const uint2 pt = *reinterpret_cast<const uint2*>(a.points + p);
        const TriRec* r = a.rec + pt.x;
        const float4 q0 = __ldg(&r->q[0]), q1 = __ldg(&r->q[1]), q2 = __ldg(&r->q[2]);
        const float4 q3 = __ldg(&r->q[3]), q4 = __ldg(&r->q[4]);
        const int i = int(pt.y & 0xffffu), j = int(pt.y >> 16);
        bool interior = true;
#pragma unroll
        for (int m = 0; m < 4; m++) {
            const int ia = i + (m == 1 || m == 2), jb = j + (m >= 2);
            const float uu = float(ia) * q0.w + q2.w, vv = float(jb) * q1.w + q3.w;
            interior &= edge_fn(q4.x, q4.y, q4.z, q4.w, uu, vv) >= 0.0f &&
                        edge_fn(q4.z, q4.w, 0.0f, 0.0f, uu, vv) >= 0.0f &&
                        edge_fn(0.0f, 0.0f, q4.x, q4.y, uu, vv) >= 0.0f;
        }
        NearRec o = near_record(c, q0, q1, q2, q3, q4, i, j, interior);
        a.rrec[p].a.x = o.alpha;
        a.rrec[p].a.y = o.beta;
        if (o.ny > 0) {
            o.L0.x = o.L0.x - (0.5f + kNearPad);
            o.L1.x = o.L1.x - (0.5f + kNearPad);
            o.L0.z = o.L0.z - (0.5f - kNearPad);
            o.L1.z = o.L1.z - (0.5f - kNearPad);
        }
        const unsigned mask = __activemask();
        const int leader = __ffs(mask) - 1;
        const unsigned bal = __ballot_sync(mask, o.ny > 0);
        uint32_t base = 0;
        if (lane == leader && bal) base = atomicAdd(&a.ctr->n_work, uint32_t(__popc(bal)));
        base = __shfl_sync(mask, base, leader);
        if (o.ny > 0 && LFDPR_IN_BOUNDS(base + __popc(bal & ((1u << lane) - 1u)), a.max_points, 9)) {
            WorkRec* w = a.work + base + __popc(bal & ((1u << lane) - 1u));
            w->L0 = o.L0;
            w->L1 = o.L1;
            w->meta = make_uint4(o.y0 | (o.ny << 14) | ((interior ? kFlagInterior : 0u) << 29), pt.y, pt.x, p);
        }
    }
}

// The normal, roughness and metallic maps of every point of a mesh of
// materials (run after k_fetch): each texture at its own Eq. 6-7 LOD pair
// (the record's size_vpuv bounds and its resolution), at the cell centre's
// texture coordinate (as k_fetch); the normal map's two RGBA8 values go to
// rmat, the roughness and metallic R channels to the resolve record's b.w as
// bytes (min, max, min, max).
__global__ void __launch_bounds__(256) k_fetch_mat(FrameArgs a) {
    wait_previous_kernel();
    allow_next_kernel();
    if (a.ctr->overflow) return;
    const uint32_t n = a.ctr->n_points;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const uint2 pt = *reinterpret_cast<const uint2*>(a.points + p);
        const TriRec* r = a.rec + pt.x;
        const float4 q0 = __ldg(&r->q[0]), q1 = __ldg(&r->q[1]), q5 = __ldg(&r->q[5]);
        const float4 q6 = __ldg(&r->q[6]), q7 = __ldg(&r->q[7]);
        const uint32_t i = pt.y & 0xffffu, j = pt.y >> 16;
        const float uc = (float(i) + 0.5f) * q0.w;
        const float vc = (float(j) + 0.5f) * q1.w;
        const float s = fmaf(q6.y, uc, fmaf(q6.z, vc, q6.x));
        const float t = fmaf(q7.x, uc, fmaf(q7.y, vc, q6.w));
        const uint4 mt = __ldg(a.mat_tex + __ldg(a.tri_tex + pt.x));
        uint32_t lo[3], hi[3];
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const uint32_t id = k == 0 ? mt.y : k == 1 ? mt.z : mt.w;
            const TexDesc tk = a.tex[id];
            const float lod_lo = 0.5f * log2_series((q5.y * float(tk.w)) * float(tk.h));
            const float lod_hi = 0.5f * log2_series((q5.z * float(tk.w)) * float(tk.h));
            trilinear_pair(a.pool, a.lvl + (size_t)id * kMaxLevels, tk.w, tk.h, int(tk.levels) - 1, s, t, lod_lo,
                           lod_hi, lo[k], hi[k]);
        }
        a.rmat[p] = make_uint2(lo[0], hi[0]);
        a.rrec[p].b.w = (lo[1] & 255u) | ((hi[1] & 255u) << 8) | ((lo[2] & 255u) << 16) | ((hi[2] & 255u) << 24);
    }
}

}  // namespace

LFDPR_CHECK_READER(checks_sample)

cudaError_t launch_setup(const FrameArgs& a, cudaStream_t s) {
    k_setup<<<a.n_blocks, kSetupThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_scan(const FrameArgs& a, cudaStream_t s) {
    return launch_after_previous(k_scan, dim3(1), dim3(1024), 0, s, a);
}

cudaError_t launch_emit(const FrameArgs& a, cudaStream_t s) {
    return launch_after_previous(k_emit, dim3(a.n_blocks), dim3(kSetupThreads), 0, s, a);
}

cudaError_t launch_fetch_mat(const FrameArgs& a, cudaStream_t s) {
    return launch_after_previous(k_fetch_mat, dim3(a.sm_count * 8), dim3(256), 0, s, a);
}

cudaError_t launch_fetch(const FrameArgs& a, cudaStream_t s) {
    return launch_after_previous(k_fetch, dim3(a.sm_count * 8), dim3(256), 0, s, a);
}

cudaError_t launch_near_work(const FrameArgs& a, cudaStream_t s) {
    return launch_after_previous(k_near_work, dim3(a.sm_count), dim3(256), 0, s, a);
}

}  // namespace lfdpr
