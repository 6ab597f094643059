/*
 * FP64 collision oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, brute-force C used by tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py to check the CUDA library.  Nothing in the
 * library links, includes or calls this file.
 *
 * Contents (paper: "Efficient GPU Cloth Simulation with Non-distance
 * Barriers and Subspace Reuse", arXiv 2403.19272):
 *   - brute-force broad phase over all vertex-triangle (VT) and edge-edge
 *     (EE) primitive pairs (Sec. 4: candidate pairs for CCD; Sec. 8
 *     implementation details replace the paper's patch BVH by any exact
 *     culling, here the O(n*m + e^2) definition itself);
 *   - exact CCD: first time of impact in [0,1] under linear trajectories
 *     (Sec. 4, Eq. intersect), found as the first root of the coplanarity
 *     cubic at which the primitives touch;
 *   - partial CCD: the sign test of the query function Q (Sec. 4.1,
 *     Eq. collision_judge and Eq. query) at sample points;
 *   - closest points between primitives and triangle-triangle intersection
 *     (for the penetration-free invariant of Sec. 7).
 *
 * Every floating-point quantity is double; the FP32 box-overlap predicate of
 * the broad phase is evaluated on float inputs with the single rounding the
 * definition states (see bp_overlap).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct { double x, y, z; } v3;

static inline v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static inline v3 ld(const double *p) { return mk(p[0], p[1], p[2]); }
static inline v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static inline v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static inline v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static inline double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static inline v3 crs(v3 a, v3 b) { return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x); }
static inline double nrm(v3 a) { return sqrt(dot(a, a)); }
static inline v3 lerp(v3 a, v3 b, double t) { return add(a, scl(sub(b, a), t)); }
static inline double clamp01(double t) { return t < 0 ? 0 : (t > 1 ? 1 : t); }

/* ------------------------------------------------------------------------
 * Closest points.
 * ------------------------------------------------------------------------ */

/* Closest point of segment [a,b] to point p: parameter in [0,1]. */
static double seg_point_param(v3 a, v3 b, v3 p) {
    v3 ab = sub(b, a);
    double den = dot(ab, ab);
    if (den <= 0) return 0.0;
    return clamp01(dot(sub(p, a), ab) / den);
}

/* Closest point on triangle (a,b,c) to p, as barycentric weights w[3] of
 * (a,b,c).  Written as: project p to the plane; if the projection lies in
 * the triangle (all barycentrics >= 0) take it, otherwise the nearest of the
 * three edge closest points.  Degenerate (zero-area) triangles use the
 * edges only. */
static void closest_pt_tri(v3 p, v3 a, v3 b, v3 c, double w[3]) {
    v3 ab = sub(b, a), ac = sub(c, a), ap = sub(p, a);
    double d00 = dot(ab, ab), d01 = dot(ab, ac), d11 = dot(ac, ac);
    double d20 = dot(ap, ab), d21 = dot(ap, ac);
    double den = d00 * d11 - d01 * d01;
    if (den > 1e-300 * (d00 * d11 + 1e-300)) {
        double v = (d11 * d20 - d01 * d21) / den;
        double u = (d00 * d21 - d01 * d20) / den;
        if (v >= 0 && u >= 0 && v + u <= 1) {
            w[0] = 1 - v - u; w[1] = v; w[2] = u;
            return;
        }
    }
    /* edges: (a,b), (b,c), (c,a) */
    double best = INFINITY;
    v3 P[3] = {a, b, c};
    for (int e = 0; e < 3; ++e) {
        v3 s0 = P[e], s1 = P[(e + 1) % 3];
        double t = seg_point_param(s0, s1, p);
        v3 q = lerp(s0, s1, t);
        double d = dot(sub(p, q), sub(p, q));
        if (d < best) {
            best = d;
            w[0] = w[1] = w[2] = 0;
            w[e] = 1 - t;
            w[(e + 1) % 3] = t;
        }
    }
}

/* Closest points between segments [p1,q1], [p2,q2]: parameters s,t in [0,1].
 * Non-parallel segments: the unique minimiser of |p1(s) - p2(t)|^2 over the
 * unit square, i.e. the unconstrained minimiser if it is interior, else the
 * best of the four boundary problems (each a clamped 1-D projection).
 * Parallel segments (a e - b^2 <= 1e-6 a e) have a whole set of closest
 * pairs; the sample point is then taken at s = the midpoint of the clamped
 * projections of p2 and q2 onto segment 1, t = the clamped projection of
 * p1(s) onto segment 2 (a tie-break the paper does not fix).  Zero-length
 * segments project the other segment's start. */
static void closest_seg_seg(v3 p1, v3 q1, v3 p2, v3 q2, double *s_out, double *t_out) {
    v3 d1 = sub(q1, p1), d2 = sub(q2, p2), r = sub(p1, p2);
    double a = dot(d1, d1), e = dot(d2, d2), b = dot(d1, d2), c = dot(d1, r), f = dot(d2, r);
    if (a <= 0 && e <= 0) { *s_out = 0; *t_out = 0; return; }
    if (a <= 0) { *s_out = 0; *t_out = clamp01(f / e); return; }
    if (e <= 0) { *t_out = 0; *s_out = clamp01(-c / a); return; }
    double den = a * e - b * b;
    if (den <= 1e-6 * a * e) {
        double s = 0.5 * (clamp01(-c / a) + clamp01((b - c) / a));
        *s_out = s;
        *t_out = clamp01((b * s + f) / e);
        return;
    }
    {
        double s = (b * f - c * e) / den, t = (a * f - b * c) / den;
        if (s >= 0 && s <= 1 && t >= 0 && t <= 1) { *s_out = s; *t_out = t; return; }
    }
    double best = INFINITY, bs = 0, bt = 0;
    /* boundaries s=0, s=1: t = clamp(projection) ; t=0, t=1: s = clamp */
    for (int k = 0; k < 4; ++k) {
        double s, t;
        if (k < 2) { s = (double)k; v3 ps = lerp(p1, q1, s); t = seg_point_param(p2, q2, ps); }
        else { t = (double)(k - 2); v3 pt = lerp(p2, q2, t); s = seg_point_param(p1, q1, pt); }
        v3 dd = sub(lerp(p1, q1, s), lerp(p2, q2, t));
        double d = dot(dd, dd);
        if (d < best) { best = d; bs = s; bt = t; }
    }
    *s_out = bs; *t_out = bt;
}

static double dist_vt(v3 p, v3 a, v3 b, v3 c) {
    double w[3];
    closest_pt_tri(p, a, b, c, w);
    v3 q = add(add(scl(a, w[0]), scl(b, w[1])), scl(c, w[2]));
    return nrm(sub(p, q));
}

static double dist_ee(v3 a, v3 b, v3 c, v3 d) {
    double s, t;
    closest_seg_seg(a, b, c, d, &s, &t);
    return nrm(sub(lerp(a, b, s), lerp(c, d, t)));
}

/* ------------------------------------------------------------------------
 * Exact CCD (Sec. 4, Eq. intersect): four points moving linearly from x0 to
 * x1 over t in [0,1].  Contact of a VT or EE pair needs the four points to
 * be coplanar, i.e. f(t) = det[q1-q0, q2-q0, q3-q0] = 0, a cubic in t.  The
 * time of impact is the first coplanarity time (a root of f, or a critical
 * point of f, which also catches tangential grazing) at which the closest
 * distance between the primitives is <= eta.  If the cubic vanishes
 * identically (coplanar motion) the distance is checked on a uniform grid of
 * 1025 times instead.  Returns 2.0 when there is no impact in [0,1].
 * ------------------------------------------------------------------------ */

static double det3(v3 a, v3 b, v3 c) { return dot(a, crs(b, c)); }

static double cubic_eval(const double c[4], double t) { return ((c[3] * t + c[2]) * t + c[1]) * t + c[0]; }

typedef double (*distfn)(const v3 *q);

static double dvt(const v3 *q) { return dist_vt(q[0], q[1], q[2], q[3]); }
static double dee(const v3 *q) { return dist_ee(q[0], q[1], q[2], q[3]); }

static void pos_at(const v3 *q0, const v3 *q1, double t, v3 *q) {
    for (int i = 0; i < 4; ++i) q[i] = lerp(q0[i], q1[i], t);
}

static int dcmp(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

static double ccd_generic(const v3 *q0, const v3 *q1, double eta, distfn dist) {
    /* cubic coefficients of det[u(t), v(t), w(t)], u = q1-q0 etc. */
    v3 u0 = sub(q0[1], q0[0]), v0 = sub(q0[2], q0[0]), w0 = sub(q0[3], q0[0]);
    v3 du = sub(sub(q1[1], q1[0]), u0), dv = sub(sub(q1[2], q1[0]), v0), dw = sub(sub(q1[3], q1[0]), w0);
    double c[4];
    c[0] = det3(u0, v0, w0);
    c[1] = det3(du, v0, w0) + det3(u0, dv, w0) + det3(u0, v0, dw);
    c[2] = det3(du, dv, w0) + det3(du, v0, dw) + det3(u0, dv, dw);
    c[3] = det3(du, dv, dw);
    double scale = 0;
    v3 vs[6] = {u0, v0, w0, du, dv, dw};
    for (int i = 0; i < 6; ++i) { double m = nrm(vs[i]); if (m > scale) scale = m; }
    double s3 = scale * scale * scale;
    v3 q[4];
    if (fabs(c[0]) <= 1e-14 * s3 && fabs(c[1]) <= 1e-14 * s3 && fabs(c[2]) <= 1e-14 * s3 &&
        fabs(c[3]) <= 1e-14 * s3) {
        for (int k = 0; k <= 1024; ++k) {
            double t = k / 1024.0;
            pos_at(q0, q1, t, q);
            if (dist(q) <= eta) return t;
        }
        return 2.0;
    }
    /* candidate times: 0, critical points of f in (0,1), roots of f */
    double cand[8];
    int nc = 0;
    cand[nc++] = 0.0;
    double brk[4];
    int nb = 0;
    brk[nb++] = 0.0;
    {
        /* f'(t) = c1 + 2 c2 t + 3 c3 t^2 */
        double A = 3 * c[3], B = 2 * c[2], C = c[1];
        double r[2];
        int nr = 0;
        if (fabs(A) > 1e-300) {
            double disc = B * B - 4 * A * C;
            if (disc >= 0) {
                double sq = sqrt(disc);
                double qq = -0.5 * (B + (B >= 0 ? sq : -sq));
                if (qq != 0) { r[nr++] = qq / A; r[nr++] = C / qq; }
                else { r[nr++] = 0.0; }
            }
        } else if (fabs(B) > 1e-300) {
            r[nr++] = -C / B;
        }
        if (nr == 2 && r[0] > r[1]) { double tmp = r[0]; r[0] = r[1]; r[1] = tmp; }
        for (int i = 0; i < nr; ++i)
            if (r[i] > 0 && r[i] < 1) { brk[nb++] = r[i]; cand[nc++] = r[i]; }
    }
    brk[nb++] = 1.0;
    for (int i = 0; i + 1 < nb; ++i) {
        double lo = brk[i], hi = brk[i + 1];
        double flo = cubic_eval(c, lo), fhi = cubic_eval(c, hi);
        if (flo == 0) { cand[nc++] = lo; continue; }
        if (fhi == 0) { cand[nc++] = hi; continue; }
        if ((flo < 0) == (fhi < 0)) continue;
        for (int it = 0; it < 200 && hi - lo > 1e-17; ++it) {
            double mid = 0.5 * (lo + hi);
            double fm = cubic_eval(c, mid);
            if (fm == 0) { lo = hi = mid; break; }
            if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else { hi = mid; }
        }
        cand[nc++] = lo;
    }
    qsort(cand, nc, sizeof(double), dcmp);
    for (int i = 0; i < nc; ++i) {
        pos_at(q0, q1, cand[i], q);
        if (dist(q) <= eta) return cand[i];
    }
    return 2.0;
}

/* VT: q = {vertex, tri a, tri b, tri c}; EE: q = {e1 a, e1 b, e2 a, e2 b}. */
double oc_ccd_vt(const double *x0, const double *x1, double eta) {
    v3 q0[4], q1[4];
    for (int i = 0; i < 4; ++i) { q0[i] = ld(x0 + 3 * i); q1[i] = ld(x1 + 3 * i); }
    return ccd_generic(q0, q1, eta, dvt);
}

double oc_ccd_ee(const double *x0, const double *x1, double eta) {
    v3 q0[4], q1[4];
    for (int i = 0; i < 4; ++i) { q0[i] = ld(x0 + 3 * i); q1[i] = ld(x1 + 3 * i); }
    return ccd_generic(q0, q1, eta, dee);
}

/* Batched exact CCD over a pair list.  X0, X1: [nvert,3] float positions
 * (converted exactly to double).  pairs: [np,4] vertex ids in the order
 * documented above; kind[i] = 0 (VT) or 1 (EE).  out_toi[i] in [0,1] or 2. */
void oc_ccd_batch(const float *X0, const float *X1, int64_t np, const int32_t *pairs, const int32_t *kind,
                  double eta, double *out_toi) {
    for (int64_t i = 0; i < np; ++i) {
        double a[12], b[12];
        for (int k = 0; k < 4; ++k)
            for (int d = 0; d < 3; ++d) {
                a[3 * k + d] = (double)X0[3 * (int64_t)pairs[4 * i + k] + d];
                b[3 * k + d] = (double)X1[3 * (int64_t)pairs[4 * i + k] + d];
            }
        out_toi[i] = kind[i] ? oc_ccd_ee(a, b, eta) : oc_ccd_vt(a, b, eta);
    }
}

/* ------------------------------------------------------------------------
 * Closest-point coefficients at t = 0 (used by partial CCD sample points and
 * by the contact projection).  The gap vector p2 - p1 is sum_j c_j x_j:
 *   VT (v; a,b,c): p1 = x_v, p2 = closest point on the triangle,
 *                  c = (-1, w_a, w_b, w_c)
 *   EE (a,b; c,d): p1 = a + s(b-a), p2 = c + t(d-c),
 *                  c = (-(1-s), -s, 1-t, t)
 * ------------------------------------------------------------------------ */
void oc_closest_coef(const double *x, int kind, double *coef) {
    v3 q[4];
    for (int i = 0; i < 4; ++i) q[i] = ld(x + 3 * i);
    if (kind == 0) {
        double w[3];
        closest_pt_tri(q[0], q[1], q[2], q[3], w);
        coef[0] = -1; coef[1] = w[0]; coef[2] = w[1]; coef[3] = w[2];
    } else {
        double s, t;
        closest_seg_seg(q[0], q[1], q[2], q[3], &s, &t);
        coef[0] = -(1 - s); coef[1] = -s; coef[2] = 1 - t; coef[3] = t;
    }
}

/* Partial CCD (Sec. 4.1): Q(lambda) = (p2^1 - p1^1) . (p2^0 - p1^0) at each
 * sample lambda.  The pair is active when, at some sample,
 * Q <= dhat * |p2^0 - p1^0| (the end separation measured along the start
 * direction is below the gap dhat; with dhat = 0 this is exactly the
 * necessary collision condition Q <= 0 of Eq. collision_judge).
 * Samples: the closest point at t=0 plus a fixed pattern of nsamp points:
 *   VT: nsamp 1 -> centroid; 3 -> (1/6,1/6),(2/3,1/6),(1/6,2/3) as weights of
 *       (b, c) with a getting the remainder;
 *   EE: nsamp 1 -> (1/2,1/2); 4 -> {1/4,3/4}^2 as (s, t).
 * Also returns min over samples of Q - dhat*|d0| in *margin. */
int oc_partial_ccd(const double *x0, const double *x1, int kind, int nsamp, double dhat, double *margin) {
    double coef[4];
    oc_closest_coef(x0, kind, coef);
    double lam[5][2];
    int ns = 0;
    if (kind == 0) {
        lam[ns][0] = coef[2]; lam[ns][1] = coef[3]; ns++;
        if (nsamp == 1) { lam[ns][0] = 1.0 / 3; lam[ns][1] = 1.0 / 3; ns++; }
        if (nsamp == 3) {
            lam[ns][0] = 1.0 / 6; lam[ns][1] = 1.0 / 6; ns++;
            lam[ns][0] = 2.0 / 3; lam[ns][1] = 1.0 / 6; ns++;
            lam[ns][0] = 1.0 / 6; lam[ns][1] = 2.0 / 3; ns++;
        }
    } else {
        lam[ns][0] = -coef[1]; lam[ns][1] = coef[3]; ns++;
        if (nsamp == 1) { lam[ns][0] = 0.5; lam[ns][1] = 0.5; ns++; }
        if (nsamp == 4) {
            double v[2] = {0.25, 0.75};
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) { lam[ns][0] = v[i]; lam[ns][1] = v[j]; ns++; }
        }
    }
    v3 a0[4], a1[4];
    for (int i = 0; i < 4; ++i) { a0[i] = ld(x0 + 3 * i); a1[i] = ld(x1 + 3 * i); }
    double best = INFINITY;
    for (int s = 0; s < ns; ++s) {
        double l1 = lam[s][0], l2 = lam[s][1];
        v3 p10, p20, p11, p21;
        if (kind == 0) {
            p10 = a0[0]; p11 = a1[0];
            p20 = add(a0[1], add(scl(sub(a0[2], a0[1]), l1), scl(sub(a0[3], a0[1]), l2)));
            p21 = add(a1[1], add(scl(sub(a1[2], a1[1]), l1), scl(sub(a1[3], a1[1]), l2)));
        } else {
            p10 = lerp(a0[0], a0[1], l1); p11 = lerp(a1[0], a1[1], l1);
            p20 = lerp(a0[2], a0[3], l2); p21 = lerp(a1[2], a1[3], l2);
        }
        v3 d0 = sub(p20, p10), d1 = sub(p21, p11);
        double m = dot(d1, d0) - dhat * nrm(d0);
        if (m < best) best = m;
    }
    *margin = best;
    return best <= 0 ? 1 : 0;
}

void oc_partial_ccd_batch(const float *X0, const float *X1, int64_t np, const int32_t *pairs, const int32_t *kind,
                          int nsamp_vt, int nsamp_ee, double dhat, int32_t *out_active, double *out_margin) {
    for (int64_t i = 0; i < np; ++i) {
        double a[12], b[12];
        for (int k = 0; k < 4; ++k)
            for (int d = 0; d < 3; ++d) {
                a[3 * k + d] = (double)X0[3 * (int64_t)pairs[4 * i + k] + d];
                b[3 * k + d] = (double)X1[3 * (int64_t)pairs[4 * i + k] + d];
            }
        out_active[i] = oc_partial_ccd(a, b, kind[i], kind[i] ? nsamp_ee : nsamp_vt, dhat, &out_margin[i]);
    }
}

/* ------------------------------------------------------------------------
 * Brute-force broad phase.  The swept box of a primitive is the per-axis
 * min/max of its vertices' float coordinates at t=0 and t=1.  Boxes A and B
 * are candidates when, on every axis,
 *     lo_A <= fl32(hi_B + dhat)  and  lo_B <= fl32(hi_A + dhat),
 * fl32 being round-to-nearest float addition (computed here as the exact
 * double sum of two floats, then rounded to float).
 * VT: every (vertex v, triangle t) with v not in t and not both kinematic.
 * EE: every (edge e, edge f), e < f by edge index, sharing no vertex and not
 * both kinematic.  Vertices with id >= n_dyn are kinematic (obstacles).
 * Returns the pair count; writes at most cap pairs.
 * ------------------------------------------------------------------------ */

typedef struct { float lo[3], hi[3]; } box;

static box box_of(const float *X0, const float *X1, const int32_t *ids, int k) {
    box b;
    for (int d = 0; d < 3; ++d) { b.lo[d] = INFINITY; b.hi[d] = -INFINITY; }
    for (int i = 0; i < k; ++i)
        for (int d = 0; d < 3; ++d) {
            float u = X0[3 * (int64_t)ids[i] + d], v = X1[3 * (int64_t)ids[i] + d];
            float mn = u < v ? u : v, mx = u < v ? v : u;
            if (mn < b.lo[d]) b.lo[d] = mn;
            if (mx > b.hi[d]) b.hi[d] = mx;
        }
    return b;
}

static inline float f32add(float a, float b) { return (float)((double)a + (double)b); }

static int bp_overlap(const box *a, const box *b, float dhat) {
    for (int d = 0; d < 3; ++d) {
        if (!(a->lo[d] <= f32add(b->hi[d], dhat))) return 0;
        if (!(b->lo[d] <= f32add(a->hi[d], dhat))) return 0;
    }
    return 1;
}

int64_t oc_broadphase_vt(const float *X0, const float *X1, int32_t nv, int32_t n_dyn, const int32_t *tris,
                         int32_t nt, float dhat, int64_t cap, int32_t *out) {
    box *tb = (box *)malloc(sizeof(box) * (size_t)(nt > 0 ? nt : 1));
    for (int t = 0; t < nt; ++t) tb[t] = box_of(X0, X1, tris + 3 * t, 3);
    int64_t n = 0;
    for (int v = 0; v < nv; ++v) {
        box vb = box_of(X0, X1, &v, 1);
        for (int t = 0; t < nt; ++t) {
            const int32_t *T = tris + 3 * t;
            if (T[0] == v || T[1] == v || T[2] == v) continue;
            if (v >= n_dyn && T[0] >= n_dyn && T[1] >= n_dyn && T[2] >= n_dyn) continue;
            if (!bp_overlap(&vb, &tb[t], dhat)) continue;
            if (n < cap) { out[2 * n] = v; out[2 * n + 1] = t; }
            ++n;
        }
    }
    free(tb);
    return n;
}

int64_t oc_broadphase_ee(const float *X0, const float *X1, int32_t n_dyn, const int32_t *edges, int32_t ne,
                         float dhat, int64_t cap, int32_t *out) {
    box *eb = (box *)malloc(sizeof(box) * (size_t)(ne > 0 ? ne : 1));
    for (int e = 0; e < ne; ++e) eb[e] = box_of(X0, X1, edges + 2 * e, 2);
    int64_t n = 0;
    for (int e = 0; e < ne; ++e) {
        const int32_t *E = edges + 2 * e;
        for (int f = e + 1; f < ne; ++f) {
            const int32_t *F = edges + 2 * f;
            if (E[0] == F[0] || E[0] == F[1] || E[1] == F[0] || E[1] == F[1]) continue;
            if (E[0] >= n_dyn && E[1] >= n_dyn && F[0] >= n_dyn && F[1] >= n_dyn) continue;
            if (!bp_overlap(&eb[e], &eb[f], dhat)) continue;
            if (n < cap) { out[2 * n] = e; out[2 * n + 1] = f; }
            ++n;
        }
    }
    free(eb);
    return n;
}

/* Brute-force candidates of ONE query primitive against all others (for
 * sampled checks at sizes where the full O(n*m) sweep is too slow). */
int64_t oc_broadphase_vt_one(const float *X0, const float *X1, int32_t v, int32_t n_dyn, const int32_t *tris,
                             int32_t nt, float dhat, int64_t cap, int32_t *out_t) {
    box vb = box_of(X0, X1, &v, 1);
    int64_t n = 0;
    for (int t = 0; t < nt; ++t) {
        const int32_t *T = tris + 3 * t;
        if (T[0] == v || T[1] == v || T[2] == v) continue;
        if (v >= n_dyn && T[0] >= n_dyn && T[1] >= n_dyn && T[2] >= n_dyn) continue;
        box tb = box_of(X0, X1, T, 3);
        if (!bp_overlap(&vb, &tb, dhat)) continue;
        if (n < cap) out_t[n] = t;
        ++n;
    }
    return n;
}

int64_t oc_broadphase_ee_one(const float *X0, const float *X1, const int32_t *e2, int32_t n_dyn,
                             const int32_t *edges, int32_t ne, float dhat, int64_t cap, int32_t *out_f) {
    box qb = box_of(X0, X1, e2, 2);
    int64_t n = 0;
    for (int f = 0; f < ne; ++f) {
        const int32_t *F = edges + 2 * f;
        if (e2[0] == F[0] || e2[0] == F[1] || e2[1] == F[0] || e2[1] == F[1]) continue;
        if (e2[0] >= n_dyn && e2[1] >= n_dyn && F[0] >= n_dyn && F[1] >= n_dyn) continue;
        box fb = box_of(X0, X1, F, 2);
        if (!bp_overlap(&qb, &fb, dhat)) continue;
        if (n < cap) out_f[n] = f;
        ++n;
    }
    return n;
}

/* ------------------------------------------------------------------------
 * Triangle-triangle intersection (penetration-free invariant, Sec. 7).
 * Two triangles intersect iff an edge of one crosses the other (closed
 * segment-vs-triangle test, done with exact-sign-style orientation
 * predicates in double).  Pairs sharing a vertex test only the edges that
 * do not contain the shared vertex; pairs sharing an edge are skipped.
 * ------------------------------------------------------------------------ */

/* Exact sign of the orientation determinant det[b - a, c - a, d - a]
 * (Shewchuk, "Adaptive precision floating-point arithmetic and fast robust
 * geometric predicates", 1997): the double evaluation is kept when it
 * exceeds a bound on its rounding error; otherwise the determinant is
 * evaluated exactly in floating-point expansions (sums of nonoverlapping
 * doubles, increasing magnitude) built with Two-Sum, the FMA two-product
 * and Grow-/Scale-Expansion, whose largest component has the sign of the
 * exact value.  Returns a value with the exact sign (0 exactly when the
 * four points are coplanar). */
#define OC_EXP_MAX 1024
static void two_sum(double a, double b, double *x, double *y) {
    *x = a + b;
    double bv = *x - a, av = *x - bv;
    *y = (a - av) + (b - bv);
}
/* h = e + b (e nonoverlapping, increasing); returns the length, zeros dropped */
static int grow_exp(const double *e, int n, double b, double *h) {
    double q = b;
    int m = 0;
    for (int i = 0; i < n; ++i) {
        double x, y;
        two_sum(q, e[i], &x, &y);
        if (y != 0.0) h[m++] = y;
        q = x;
    }
    if (q != 0.0 || m == 0) h[m++] = q;
    return m;
}
static int sum_exp(const double *e, int n, const double *f, int m, double *h) {
    double t[OC_EXP_MAX];
    int k = n;
    memcpy(t, e, sizeof(double) * (size_t)n);
    for (int j = 0; j < m; ++j) {
        double u[OC_EXP_MAX];
        k = grow_exp(t, k, f[j], u);
        memcpy(t, u, sizeof(double) * (size_t)k);
    }
    memcpy(h, t, sizeof(double) * (size_t)k);
    return k;
}
/* h = e * b exactly */
static int scale_exp(const double *e, int n, double b, double *h) {
    double t[OC_EXP_MAX];
    int k = 1;
    t[0] = 0.0;
    for (int i = 0; i < n; ++i) {
        double p = e[i] * b, q = fma(e[i], b, -p);  /* e_i b = p + q exactly */
        double u[OC_EXP_MAX];
        k = grow_exp(t, k, q, u);
        k = grow_exp(u, k, p, t);
    }
    memcpy(h, t, sizeof(double) * (size_t)k);
    return k;
}
static int mul_exp(const double *e, int n, const double *f, int m, double *h) {
    double acc[OC_EXP_MAX], t[OC_EXP_MAX], u[OC_EXP_MAX];
    int k = 1;
    acc[0] = 0.0;
    for (int j = 0; j < m; ++j) {
        int kt = scale_exp(e, n, f[j], t);
        k = sum_exp(acc, k, t, kt, u);
        memcpy(acc, u, sizeof(double) * (size_t)k);
    }
    memcpy(h, acc, sizeof(double) * (size_t)k);
    return k;
}
static double exp_sign_value(const double *e, int n) {
    for (int i = n - 1; i >= 0; --i)
        if (e[i] != 0.0) return e[i];
    return 0.0;
}
/* b - a as an expansion of one or two components */
static int diff_exp(double b, double a, double *e) {
    double x, y;
    two_sum(b, -a, &x, &y);
    if (y == 0.0) {
        e[0] = x;
        return 1;
    }
    e[0] = y;
    e[1] = x;
    return 2;
}
static double orient_exact(v3 a, v3 b, v3 c, v3 d) {
    double U[3][2], V[3][2], W[3][2];
    int nu[3], nv[3], nw[3];
    const double A[3] = {a.x, a.y, a.z}, B[3] = {b.x, b.y, b.z}, C[3] = {c.x, c.y, c.z}, D[3] = {d.x, d.y, d.z};
    for (int k = 0; k < 3; ++k) {
        nu[k] = diff_exp(B[k], A[k], U[k]);
        nv[k] = diff_exp(C[k], A[k], V[k]);
        nw[k] = diff_exp(D[k], A[k], W[k]);
    }
    /* det = sum over (i, j, k) cyclic of U_i (V_j W_k - V_k W_j) */
    double det[OC_EXP_MAX];
    int nd = 1;
    det[0] = 0.0;
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3, k = (i + 2) % 3;
        double p1[OC_EXP_MAX], p2[OC_EXP_MAX], c1[OC_EXP_MAX], term[OC_EXP_MAX], nxt[OC_EXP_MAX];
        int n1 = mul_exp(V[j], nv[j], W[k], nw[k], p1);
        int n2 = mul_exp(V[k], nv[k], W[j], nw[j], p2);
        for (int q = 0; q < n2; ++q) p2[q] = -p2[q];
        int nc = sum_exp(p1, n1, p2, n2, c1);
        int nt = mul_exp(c1, nc, U[i], nu[i], term);
        nd = sum_exp(det, nd, term, nt, nxt);
        memcpy(det, nxt, sizeof(double) * (size_t)nd);
    }
    return exp_sign_value(det, nd);
}
static double orient(v3 a, v3 b, v3 c, v3 d) {
    v3 u = sub(b, a), v = sub(c, a), w = sub(d, a);
    double det = det3(u, v, w);
    /* the rounding error of the double evaluation (differences included) is
     * below (7 + 56 eps) eps of the permanent, eps = 2^-53 (Shewchuk's bound);
     * 2e-15 keeps a margin over it */
    double perm = fabs(u.x) * (fabs(v.y * w.z) + fabs(v.z * w.y)) + fabs(u.y) * (fabs(v.z * w.x) + fabs(v.x * w.z)) +
                  fabs(u.z) * (fabs(v.x * w.y) + fabs(v.y * w.x));
    if (fabs(det) > 2e-15 * perm) return det;
    return orient_exact(a, b, c, d);
}

/* does segment pq cross triangle abc (proper or touching)?  The
 * orientation signs are exact (orient), so a segment in the triangle's
 * plane is recognised as coplanar and a segment whose line runs nearly
 * parallel to the plane gets the signs of the exact geometry. */
static int seg_tri(v3 p, v3 q, v3 a, v3 b, v3 c) {
    double sp = orient(a, b, c, p), sq = orient(a, b, c, q);
    if ((sp > 0 && sq > 0) || (sp < 0 && sq < 0)) return 0;
    if (sp == 0 && sq == 0) return 0; /* coplanar: not counted as crossing */
    double s1 = orient(p, q, a, b), s2 = orient(p, q, b, c), s3 = orient(p, q, c, a);
    return ((s1 >= 0 && s2 >= 0 && s3 >= 0) || (s1 <= 0 && s2 <= 0 && s3 <= 0));
}

/* exact test of one pair (boxes already overlap or not checked) */
static int tri_pair_hits(const double *X, const int32_t *A, const int32_t *B) {
    int shared = 0, sa = -1, sb = -1;
    for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y)
            if (A[x] == B[y]) { shared++; sa = x; sb = y; }
    if (shared >= 2) return 0;
    v3 a[3] = {ld(X + 3 * A[0]), ld(X + 3 * A[1]), ld(X + 3 * A[2])};
    v3 b[3] = {ld(X + 3 * B[0]), ld(X + 3 * B[1]), ld(X + 3 * B[2])};
    int hit = 0;
    for (int e = 0; e < 3 && !hit; ++e) {
        int e0 = e, e1 = (e + 1) % 3;
        if (!(shared == 1 && (e0 == sa || e1 == sa))) hit |= seg_tri(a[e0], a[e1], b[0], b[1], b[2]);
        if (!(shared == 1 && (e0 == sb || e1 == sb))) hit |= seg_tri(b[e0], b[e1], a[0], a[1], a[2]);
    }
    return hit;
}

int64_t oc_count_tri_tri(const double *X, const int32_t *tris, int32_t nt, int64_t cap, int32_t *out) {
    int64_t n = 0;
    for (int i = 0; i < nt; ++i) {
        const int32_t *A = tris + 3 * i;
        v3 a[3] = {ld(X + 3 * A[0]), ld(X + 3 * A[1]), ld(X + 3 * A[2])};
        double lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
            double u = (&a[0].x)[d], v = (&a[1].x)[d], w = (&a[2].x)[d];
            lo[d] = fmin(u, fmin(v, w)); hi[d] = fmax(u, fmax(v, w));
        }
        for (int j = i + 1; j < nt; ++j) {
            const int32_t *B = tris + 3 * j;
            v3 b[3] = {ld(X + 3 * B[0]), ld(X + 3 * B[1]), ld(X + 3 * B[2])};
            int skip = 0;
            for (int d = 0; d < 3 && !skip; ++d) {
                double u = (&b[0].x)[d], v = (&b[1].x)[d], w = (&b[2].x)[d];
                if (fmax(u, fmax(v, w)) < lo[d] || fmin(u, fmin(v, w)) > hi[d]) skip = 1;
            }
            if (skip) continue;
            if (tri_pair_hits(X, A, B)) {
                if (n < cap) { out[2 * n] = i; out[2 * n + 1] = j; }
                ++n;
            }
        }
    }
    return n;
}

/* The same list of intersecting pairs, culled by a uniform grid instead of
 * the all-pairs sweep: every triangle is entered in each cell its box
 * touches (cell side `cell`), entries are sorted by cell, and a pair is
 * tested (with the same exact test) only in the lowest cell its two boxes
 * share, so each pair is seen once.  Pairs come out sorted (i < j, by i then
 * j).  Returns the count (-1 when an allocation fails or a box spans more
 * than 2^21 cells per axis). */
typedef struct { int64_t key; int32_t tri; } oc_ent;
/* closed boxes of the two triangles meet (no intersection otherwise) */
static int tri_boxes_meet(const double *X, const int32_t *A, const int32_t *B) {
    for (int d = 0; d < 3; ++d) {
        double a0 = X[3 * A[0] + d], a1 = X[3 * A[1] + d], a2 = X[3 * A[2] + d];
        double b0 = X[3 * B[0] + d], b1 = X[3 * B[1] + d], b2 = X[3 * B[2] + d];
        if (fmax(b0, fmax(b1, b2)) < fmin(a0, fmin(a1, a2)) || fmin(b0, fmin(b1, b2)) > fmax(a0, fmax(a1, a2)))
            return 0;
    }
    return 1;
}
static int oc_ent_cmp(const void *p, const void *q) {
    const oc_ent *a = (const oc_ent *)p, *b = (const oc_ent *)q;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->tri - b->tri;
}
static int oc_pair_cmp(const void *p, const void *q) {
    const int32_t *a = (const int32_t *)p, *b = (const int32_t *)q;
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
    return a[1] < b[1] ? -1 : (a[1] > b[1]);
}

int64_t oc_count_tri_tri_grid(const double *X, const int32_t *tris, int32_t nt, double cell, int64_t cap,
                              int32_t *out) {
    if (nt <= 1) return 0;
    const double inv = 1.0 / cell;
    int64_t *clo = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)nt);
    int64_t *chi = (int64_t *)malloc(sizeof(int64_t) * 3 * (size_t)nt);
    if (!clo || !chi) { free(clo); free(chi); return -1; }
    int64_t total = 0;
    for (int i = 0; i < nt; ++i) {
        const int32_t *A = tris + 3 * i;
        int64_t cnt = 1;
        for (int d = 0; d < 3; ++d) {
            double u = X[3 * A[0] + d], v = X[3 * A[1] + d], w = X[3 * A[2] + d];
            clo[3 * i + d] = (int64_t)floor(fmin(u, fmin(v, w)) * inv);
            chi[3 * i + d] = (int64_t)floor(fmax(u, fmax(v, w)) * inv);
            int64_t span = chi[3 * i + d] - clo[3 * i + d] + 1;
            if (span > (1 << 20) || clo[3 * i + d] < -(1 << 20) || chi[3 * i + d] >= (1 << 20)) {
                free(clo); free(chi); return -1;
            }
            cnt *= span;
        }
        total += cnt;
    }
    oc_ent *E = (oc_ent *)malloc(sizeof(oc_ent) * (size_t)total);
    if (!E) { free(clo); free(chi); return -1; }
    int64_t k = 0;
    for (int i = 0; i < nt; ++i)
        for (int64_t z = clo[3 * i + 2]; z <= chi[3 * i + 2]; ++z)
            for (int64_t y = clo[3 * i + 1]; y <= chi[3 * i + 1]; ++y)
                for (int64_t x = clo[3 * i]; x <= chi[3 * i]; ++x) {
                    E[k].key = ((x + (1 << 20)) << 42) | ((y + (1 << 20)) << 21) | (z + (1 << 20));
                    E[k].tri = i;
                    ++k;
                }
    qsort(E, (size_t)total, sizeof(oc_ent), oc_ent_cmp);
    int64_t n = 0;
    for (int64_t a0 = 0; a0 < total;) {
        int64_t a1 = a0;
        while (a1 < total && E[a1].key == E[a0].key) ++a1;
        const int64_t key = E[a0].key;
        const int64_t cx = (key >> 42) - (1 << 20), cy = ((key >> 21) & ((1 << 21) - 1)) - (1 << 20),
                      cz = (key & ((1 << 21) - 1)) - (1 << 20);
        for (int64_t p = a0; p < a1; ++p)
            for (int64_t q = p + 1; q < a1; ++q) {
                const int i = E[p].tri, j = E[q].tri;  /* i < j: sorted within the cell */
                /* the lowest cell both boxes touch (their ranges overlap here) */
                int64_t lx = clo[3 * i] > clo[3 * j] ? clo[3 * i] : clo[3 * j];
                int64_t ly = clo[3 * i + 1] > clo[3 * j + 1] ? clo[3 * i + 1] : clo[3 * j + 1];
                int64_t lz = clo[3 * i + 2] > clo[3 * j + 2] ? clo[3 * i + 2] : clo[3 * j + 2];
                if (lx != cx || ly != cy || lz != cz) continue;
                if (!tri_boxes_meet(X, tris + 3 * i, tris + 3 * j)) continue;
                if (!tri_pair_hits(X, tris + 3 * i, tris + 3 * j)) continue;
                if (n < cap) { out[2 * n] = i; out[2 * n + 1] = j; }
                ++n;
            }
        a0 = a1;
    }
    free(E);
    free(clo);
    free(chi);
    if (n <= cap) qsort(out, (size_t)n, 2 * sizeof(int32_t), oc_pair_cmp);
    return n;
}

/* ---------------------------------------------------------------------------
 * Grid-culled broad phase: the same VT and EE pairs as oc_broadphase_vt /
 * oc_broadphase_ee (the same bp_overlap predicate and exclusions), found by
 * binning every primitive into the cells of side `cell` that its box grown
 * by g = d_hat + 1e-5 (1 + |largest coordinate|) on every side touches, and
 * testing all pairs that share a cell.  If bp_overlap holds, lo_a <=
 * fl32(hi_b + d_hat) <= hi_b + g and likewise for b, so the grown boxes
 * overlap and share a cell.  A pair found in several cells is kept once
 * (sort, then drop repeats).  For lists too large for the brute force.
 * Returns 0, or -1 when memory or the cell range runs out; the pair counts
 * go to n_vt / n_ee, at most cap_* pairs to out_*, sorted.
 * ------------------------------------------------------------------------ */
typedef struct { int64_t key; int32_t id, kind; } oc_bent;  /* kind 0 vertex, 1 edge, 2 triangle */

static int oc_bent_cmp(const void *p, const void *q) {
    const oc_bent *a = (const oc_bent *)p, *b = (const oc_bent *)q;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->kind != b->kind) return a->kind - b->kind;
    return a->id - b->id;
}

/* sorts the n pairs of P and moves the distinct ones to its front; returns their count */
static int64_t oc_unique_count(int32_t *P, int64_t n) {
    qsort(P, (size_t)n, 2 * sizeof(int32_t), oc_pair_cmp);
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        if (m == 0 || P[2 * i] != P[2 * (m - 1)] || P[2 * i + 1] != P[2 * (m - 1) + 1]) {
            P[2 * m] = P[2 * i];
            P[2 * m + 1] = P[2 * i + 1];
            ++m;
        }
    return m;
}

int oc_broadphase_grid(const float *X0, const float *X1, int32_t nv, int32_t n_dyn, const int32_t *tris,
                       int32_t nt, const int32_t *edges, int32_t ne, float dhat, double cell, int64_t cap_vt,
                       int32_t *out_vt, int64_t cap_ee, int32_t *out_ee, int64_t *n_vt, int64_t *n_ee) {
    const int64_t np = (int64_t)nv + ne + nt;
    *n_vt = 0;
    *n_ee = 0;
    if (np == 0) return 0;
    box *B = (box *)malloc(sizeof(box) * (size_t)np);
    if (!B) return -1;
    double amax = 0.0;
    for (int64_t p = 0; p < np; ++p) {
        if (p < nv) { int32_t v = (int32_t)p; B[p] = box_of(X0, X1, &v, 1); }
        else if (p < nv + ne) B[p] = box_of(X0, X1, edges + 2 * (p - nv), 2);
        else B[p] = box_of(X0, X1, tris + 3 * (p - nv - ne), 3);
        for (int d = 0; d < 3; ++d) {
            if (fabs(B[p].lo[d]) > amax) amax = fabs(B[p].lo[d]);
            if (fabs(B[p].hi[d]) > amax) amax = fabs(B[p].hi[d]);
        }
    }
    const double g = (double)dhat + 1e-5 * (1.0 + amax), inv = 1.0 / cell;
    /* cell ranges of the grown boxes */
    int64_t total = 0;
    for (int64_t p = 0; p < np; ++p) {
        int64_t c = 1;
        for (int d = 0; d < 3; ++d) {
            double lo = floor(((double)B[p].lo[d] - g) * inv), hi = floor(((double)B[p].hi[d] + g) * inv);
            if (lo < -(double)(1 << 20) || hi >= (double)(1 << 20) || hi - lo > 4096) { free(B); return -1; }
            c *= (int64_t)(hi - lo) + 1;
        }
        total += c;
    }
    oc_bent *E = (oc_bent *)malloc(sizeof(oc_bent) * (size_t)total);
    if (!E) { free(B); return -1; }
    int64_t k = 0;
    for (int64_t p = 0; p < np; ++p) {
        int64_t lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
            lo[d] = (int64_t)floor(((double)B[p].lo[d] - g) * inv);
            hi[d] = (int64_t)floor(((double)B[p].hi[d] + g) * inv);
        }
        const int kind = p < nv ? 0 : (p < nv + ne ? 1 : 2);
        const int32_t id = (int32_t)(kind == 0 ? p : (kind == 1 ? p - nv : p - nv - ne));
        for (int64_t z = lo[2]; z <= hi[2]; ++z)
            for (int64_t y = lo[1]; y <= hi[1]; ++y)
                for (int64_t x = lo[0]; x <= hi[0]; ++x) {
                    E[k].key = ((x + (1 << 20)) << 42) | ((y + (1 << 20)) << 21) | (z + (1 << 20));
                    E[k].id = id;
                    E[k].kind = kind;
                    ++k;
                }
    }
    qsort(E, (size_t)total, sizeof(oc_bent), oc_bent_cmp);
    /* pairs of every cell, repeats included */
    int64_t cvt = 1024, cee = 1024, nvt = 0, nee = 0;
    int32_t *PV = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)cvt);
    int32_t *PE = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)cee);
    int fail = !PV || !PE;
    for (int64_t a0 = 0; a0 < total && !fail;) {
        int64_t a1 = a0;
        while (a1 < total && E[a1].key == E[a0].key) ++a1;
        /* the cell's entries are sorted by kind: vertices, edges, triangles */
        int64_t e0 = a0, t0;
        while (e0 < a1 && E[e0].kind == 0) ++e0;
        t0 = e0;
        while (t0 < a1 && E[t0].kind == 1) ++t0;
        for (int64_t i = a0; i < t0 && !fail; ++i)
            for (int64_t j = (i < e0 ? t0 : i + 1); j < (i < e0 ? a1 : t0) && !fail; ++j) {
                int32_t a = E[i].id, b = E[j].id;
                if (E[i].kind == 0 && E[j].kind == 2) {          /* (vertex a, triangle b) */
                    const int32_t *T = tris + 3 * b;
                    if (T[0] == a || T[1] == a || T[2] == a) continue;
                    if (a >= n_dyn && T[0] >= n_dyn && T[1] >= n_dyn && T[2] >= n_dyn) continue;
                    if (!bp_overlap(&B[a], &B[nv + ne + b], dhat)) continue;
                    if (nvt == cvt) {
                        cvt *= 2;
                        int32_t *t = (int32_t *)realloc(PV, sizeof(int32_t) * 2 * (size_t)cvt);
                        if (!t) { fail = 1; break; }
                        PV = t;
                    }
                    PV[2 * nvt] = a;
                    PV[2 * nvt + 1] = b;
                    ++nvt;
                } else if (E[i].kind == 1 && E[j].kind == 1 && a < b) {  /* (edge a, edge b), a < b */
                    const int32_t *Ea = edges + 2 * a, *Eb = edges + 2 * b;
                    if (Ea[0] == Eb[0] || Ea[0] == Eb[1] || Ea[1] == Eb[0] || Ea[1] == Eb[1]) continue;
                    if (Ea[0] >= n_dyn && Ea[1] >= n_dyn && Eb[0] >= n_dyn && Eb[1] >= n_dyn) continue;
                    if (!bp_overlap(&B[nv + a], &B[nv + b], dhat)) continue;
                    if (nee == cee) {
                        cee *= 2;
                        int32_t *t = (int32_t *)realloc(PE, sizeof(int32_t) * 2 * (size_t)cee);
                        if (!t) { fail = 1; break; }
                        PE = t;
                    }
                    PE[2 * nee] = a;
                    PE[2 * nee + 1] = b;
                    ++nee;
                }
            }
        a0 = a1;
    }
    free(E);
    free(B);
    if (fail) { free(PV); free(PE); return -1; }
    nvt = oc_unique_count(PV, nvt);
    nee = oc_unique_count(PE, nee);
    for (int64_t i = 0; i < nvt && i < cap_vt; ++i) { out_vt[2 * i] = PV[2 * i]; out_vt[2 * i + 1] = PV[2 * i + 1]; }
    for (int64_t i = 0; i < nee && i < cap_ee; ++i) { out_ee[2 * i] = PE[2 * i]; out_ee[2 * i + 1] = PE[2 * i + 1]; }
    free(PV);
    free(PE);
    *n_vt = nvt;
    *n_ee = nee;
    return 0;
}
