// Per-pair collision kernels: exact CCD, partial CCD + NDB counters,
// active-constraint collection, collision springs.
//
// Closest points (used for the partial-CCD sample at the t = 0 projection
// point, for the contact direction and for the CCD contact test):
//   VT: the closest point of a triangle to a point, by the Voronoi region of
//       the triangle that contains the point (vertex, edge or face region);
//   EE: the minimiser of |p1(s) - p2(t)|^2 over [0,1]^2, found by clamping the
//       unconstrained minimiser one parameter at a time; for parallel
//       segments (a e - b^2 <= 1e-6 a e) the parameter s is the midpoint of
//       the projections of segment 2's end points onto segment 1 (clamped),
//       t the clamped projection of p1(s) onto segment 2.
#include "pdc_collide.cuh"

namespace pdc {

namespace {

template <class T> struct V {
    T x, y, z;
};
// the float3 helpers of the enclosing namespace stay visible beside the V<T> ones
using pdc::operator+;
using pdc::operator-;
using pdc::operator*;
template <class T> __device__ inline V<T> mk(T x, T y, T z) { return V<T>{x, y, z}; }
template <class T> __device__ inline V<T> operator+(V<T> a, V<T> b) { return mk<T>(a.x + b.x, a.y + b.y, a.z + b.z); }
template <class T> __device__ inline V<T> operator-(V<T> a, V<T> b) { return mk<T>(a.x - b.x, a.y - b.y, a.z - b.z); }
template <class T> __device__ inline V<T> operator*(T s, V<T> a) { return mk<T>(s * a.x, s * a.y, s * a.z); }
template <class T> __device__ inline T dotv(V<T> a, V<T> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> __device__ inline V<T> crossv(V<T> a, V<T> b) {
    return mk<T>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
template <class T> __device__ inline V<T> ld(float4 a) { return mk<T>((T)a.x, (T)a.y, (T)a.z); }
template <class T> __device__ inline T clamp01(T v) { return v < T(0) ? T(0) : (v > T(1) ? T(1) : v); }

// Barycentric weights (wa, wb, wc) of the closest point of triangle abc to p.
template <class T> __device__ void closest_tri(V<T> p, V<T> a, V<T> b, V<T> c, T w[3]) {
    V<T> ab = b - a, ac = c - a, ap = p - a;
    T d1 = dotv(ab, ap), d2 = dotv(ac, ap);
    if (d1 <= T(0) && d2 <= T(0)) { w[0] = 1; w[1] = 0; w[2] = 0; return; }
    V<T> bp = p - b;
    T d3 = dotv(ab, bp), d4 = dotv(ac, bp);
    if (d3 >= T(0) && d4 <= d3) { w[0] = 0; w[1] = 1; w[2] = 0; return; }
    T vc = d1 * d4 - d3 * d2;
    if (vc <= T(0) && d1 >= T(0) && d3 <= T(0)) {
        T den = d1 - d3;
        T v = den > T(0) ? d1 / den : T(0);
        w[0] = 1 - v; w[1] = v; w[2] = 0;
        return;
    }
    V<T> cp = p - c;
    T d5 = dotv(ab, cp), d6 = dotv(ac, cp);
    if (d6 >= T(0) && d5 <= d6) { w[0] = 0; w[1] = 0; w[2] = 1; return; }
    T vb = d5 * d2 - d1 * d6;
    if (vb <= T(0) && d2 >= T(0) && d6 <= T(0)) {
        T den = d2 - d6;
        T u = den > T(0) ? d2 / den : T(0);
        w[0] = 1 - u; w[1] = 0; w[2] = u;
        return;
    }
    T va = d3 * d6 - d5 * d4;
    if (va <= T(0) && (d4 - d3) >= T(0) && (d5 - d6) >= T(0)) {
        T den = (d4 - d3) + (d5 - d6);
        T u = den > T(0) ? (d4 - d3) / den : T(0);
        w[0] = 0; w[1] = 1 - u; w[2] = u;
        return;
    }
    T sum = va + vb + vc;
    if (!(sum > T(0))) {  // degenerate triangle: nearest vertex
        T da = dotv(ap, ap), db = dotv(bp, bp), dc = dotv(cp, cp);
        w[0] = w[1] = w[2] = 0;
        if (da <= db && da <= dc) w[0] = 1; else if (db <= dc) w[1] = 1; else w[2] = 1;
        return;
    }
    T inv = T(1) / sum;
    T v = vb * inv, u = vc * inv;
    w[0] = 1 - v - u; w[1] = v; w[2] = u;
}

template <class T> __device__ void closest_seg(V<T> p1, V<T> q1, V<T> p2, V<T> q2, T &s, T &t) {
    V<T> d1 = q1 - p1, d2 = q2 - p2, r = p1 - p2;
    T a = dotv(d1, d1), e = dotv(d2, d2), f = dotv(d2, r);
    if (a <= T(0) && e <= T(0)) { s = 0; t = 0; return; }
    if (a <= T(0)) { s = 0; t = clamp01(f / e); return; }
    T c = dotv(d1, r);
    if (e <= T(0)) { t = 0; s = clamp01(-c / a); return; }
    T b = dotv(d1, d2);
    T den = a * e - b * b;
    if (den <= T(1e-6) * a * e) {
        // parallel: midpoint of the projections of p2, q2 onto segment 1
        T s0 = clamp01(-c / a), s1 = clamp01((b - c) / a);
        s = T(0.5) * (s0 + s1);
        t = clamp01((b * s + f) / e);
        return;
    }
    s = clamp01((b * f - c * e) / den);
    t = (b * s + f) / e;
    if (t < T(0)) { t = 0; s = clamp01(-c / a); }
    else if (t > T(1)) { t = 1; s = clamp01((b - c) / a); }
}

// Gap-vector coefficients c at the closest points of the 4 points q (kind 0:
// v, a, b, c; kind 1: a, b, c, d): p2 - p1 = sum_j c_j q_j.
template <class T> __device__ void closest_coef(int kind, const V<T> q[4], T c[4]) {
    if (kind == 0) {
        T w[3];
        closest_tri(q[0], q[1], q[2], q[3], w);
        c[0] = -1; c[1] = w[0]; c[2] = w[1]; c[3] = w[2];
    } else {
        T s, t;
        closest_seg(q[0], q[1], q[2], q[3], s, t);
        c[0] = -(1 - s); c[1] = -s; c[2] = 1 - t; c[3] = t;
    }
}

template <class T> __device__ inline T gap_dist(int kind, const V<T> q[4]) {
    T c[4];
    closest_coef(kind, q, c);
    V<T> d = c[0] * q[0] + c[1] * q[1] + c[2] * q[2] + c[3] * q[3];
    return sqrt(dotv(d, d));
}

__device__ inline double det3(V<double> a, V<double> b, V<double> c) { return dotv(a, crossv(b, c)); }
__device__ inline double cubic(const double c[4], double t) { return ((c[3] * t + c[2]) * t + c[1]) * t + c[0]; }

// Exact CCD (Sec. 4, Eq. intersect) of one pair moving linearly q0 -> q1.
// FP32 filter (ccd_may_hit): a Lipschitz bound of the distance over [0, 1]
// rejects pairs that stay apart.  Survivors (ccd_exact, FP64): the four points must become coplanar for
// contact, f(t) = det[q1-q0, q2-q0, q3-q0] = 0 (cubic); candidate times are
// 0, the critical points of f and its roots (bisection on monotone pieces),
// in increasing order; the first one at which the primitives are within eta
// is the time of impact.  Coplanar motion (f == 0): 1025 uniform samples.
// The FP32 part: false when no impact is possible (the pair is then done).
__device__ inline bool ccd_may_hit(int kind, const float4 a0[4], const float4 a1[4], double eta) {
    {
        V<float> q[4];
        float cmax = 0.f;
        V<float> dv[4];
        for (int i = 0; i < 4; ++i) {
            q[i] = ld<float>(a0[i]);
            V<float> e = ld<float>(a1[i]);
            dv[i] = e - q[i];
            cmax = fmaxf(cmax, fmaxf(fabsf(q[i].x), fmaxf(fabsf(q[i].y), fabsf(q[i].z))));
            cmax = fmaxf(cmax, fmaxf(fabsf(e.x), fmaxf(fabsf(e.y), fabsf(e.z))));
        }
        float maxrel = 0.f;
        if (kind == 0) {
            for (int j = 1; j < 4; ++j) { V<float> r = dv[j] - dv[0]; maxrel = fmaxf(maxrel, sqrtf(dotv(r, r))); }
        } else {
            for (int j = 0; j < 2; ++j)
                for (int k = 2; k < 4; ++k) { V<float> r = dv[k] - dv[j]; maxrel = fmaxf(maxrel, sqrtf(dotv(r, r))); }
        }
        float d0 = gap_dist<float>(kind, q);
        // The gap d(t) of linearly moving primitives changes by at most the
        // largest relative displacement L per unit t (for fixed closest-point
        // parameters the gap vector moves by a convex combination of relative
        // displacements), so on [t_a, t_b] it stays above
        // (d(t_a) + d(t_b) - L (t_b - t_a)) / 2.  No impact if that bound
        // clears eta (with the FP32 margin) on all of [0, 1]: first from d0
        // alone, then on [0, 1] and, where it does not, on its halves,
        // quarters and eighths (distances at t = k / 8, evaluated as needed).
        const float L = 1.001f * maxrel, mg = (float)eta + 4e-6f * cmax;
        if (d0 > L + mg) return false;
        float d[9];
        unsigned have = 1u | (1u << 8);
        d[0] = d0;
        auto at = [&](int k) {
            if (!(have >> k & 1u)) {
                const float t = 0.125f * (float)k;
                V<float> qt[4];
                for (int i = 0; i < 4; ++i) qt[i] = q[i] + t * dv[i];
                d[k] = gap_dist<float>(kind, qt);
                have |= 1u << k;
            }
            return d[k];
        };
        {
            V<float> q1[4];
            for (int i = 0; i < 4; ++i) q1[i] = q[i] + dv[i];
            d[8] = gap_dist<float>(kind, q1);
        }
        unsigned open = 1u;  // intervals of the current level not yet cleared
        for (int level = 0; level <= 3; ++level) {
            const int w = 8 >> level;  // interval width in eighths
            unsigned next = 0u;
            for (int i = 0; i < (1 << level); ++i) {
                if (!(open >> i & 1u)) continue;
                const int a = i * w, b = a + w;
                if (0.5f * (at(a) + at(b) - 0.125f * (float)w * L) > mg) continue;
                next |= 3u << (2 * i);  // both halves go on to the next level
            }
            if (!next) return false;
            open = next;
        }
        return true;
    }
}

// The FP64 part for pairs that passed ccd_may_hit.
__device__ double ccd_exact(int kind, const float4 a0[4], const float4 a1[4], double eta) {
    V<double> q0[4], q1[4];
    for (int i = 0; i < 4; ++i) { q0[i] = ld<double>(a0[i]); q1[i] = ld<double>(a1[i]); }
    V<double> u0 = q0[1] - q0[0], v0 = q0[2] - q0[0], w0 = q0[3] - q0[0];
    V<double> du = (q1[1] - q1[0]) - u0, dv = (q1[2] - q1[0]) - v0, dw = (q1[3] - q1[0]) - w0;
    double c[4];
    c[0] = det3(u0, v0, w0);
    c[1] = det3(du, v0, w0) + det3(u0, dv, w0) + det3(u0, v0, dw);
    c[2] = det3(du, dv, w0) + det3(du, v0, dw) + det3(u0, dv, dw);
    c[3] = det3(du, dv, dw);
    double sc = 0.0;
    {
        V<double> vs[6] = {u0, v0, w0, du, dv, dw};
        for (int i = 0; i < 6; ++i) sc = fmax(sc, sqrt(dotv(vs[i], vs[i])));
    }
    double s3 = sc * sc * sc;
    V<double> q[4];
    auto at = [&](double t) {
        for (int i = 0; i < 4; ++i) q[i] = q0[i] + t * (q1[i] - q0[i]);
        return gap_dist<double>(kind, q);
    };
    double lim = 1e-14 * s3;
    if (fabs(c[0]) <= lim && fabs(c[1]) <= lim && fabs(c[2]) <= lim && fabs(c[3]) <= lim) {
        for (int k = 0; k <= 1024; ++k) {
            double t = k / 1024.0;
            if (at(t) <= eta) return t;
        }
        return 2.0;
    }
    double cand[8];
    int nc = 0;
    cand[nc++] = 0.0;
    double brk[4];
    int nb = 0;
    brk[nb++] = 0.0;
    {
        double A = 3.0 * c[3], B = 2.0 * c[2], C = c[1];
        double r0 = 2.0, r1 = 2.0;
        if (fabs(A) > 1e-300) {
            double disc = B * B - 4.0 * A * C;
            if (disc >= 0.0) {
                double sq = sqrt(disc);
                double qq = -0.5 * (B + (B >= 0.0 ? sq : -sq));
                if (qq != 0.0) { r0 = qq / A; r1 = C / qq; }
                else { r0 = 0.0; }
            }
        } else if (fabs(B) > 1e-300) {
            r0 = -C / B;
        }
        if (r0 > r1) { double tmp = r0; r0 = r1; r1 = tmp; }
        if (r0 > 0.0 && r0 < 1.0) { brk[nb++] = r0; cand[nc++] = r0; }
        if (r1 > 0.0 && r1 < 1.0 && r1 != r0) { brk[nb++] = r1; cand[nc++] = r1; }
    }
    brk[nb++] = 1.0;
    for (int i = 0; i + 1 < nb; ++i) {
        double lo = brk[i], hi = brk[i + 1];
        double flo = cubic(c, lo), fhi = cubic(c, hi);
        if (flo == 0.0) { cand[nc++] = lo; continue; }
        if (fhi == 0.0) { cand[nc++] = hi; continue; }
        if ((flo < 0.0) == (fhi < 0.0)) continue;
        for (int it = 0; it < 200; ++it) {
            double mid = 0.5 * (lo + hi);
            if (!(mid > lo && mid < hi)) break;
            double fm = cubic(c, mid);
            if (fm == 0.0) { lo = hi = mid; break; }
            if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
        }
        cand[nc++] = lo;
    }
    // ascending order (at most 6 candidates)
    for (int i = 1; i < nc; ++i) {
        double v = cand[i];
        int j = i - 1;
        while (j >= 0 && cand[j] > v) { cand[j + 1] = cand[j]; --j; }
        cand[j + 1] = v;
    }
    for (int i = 0; i < nc; ++i)
        if (at(cand[i]) <= eta) return cand[i];
    return 2.0;
}

__device__ double ccd_pair(int kind, const float4 a0[4], const float4 a1[4], double eta) {
    return ccd_may_hit(kind, a0, a1, eta) ? ccd_exact(kind, a0, a1, eta) : 2.0;
}

// Partial CCD (Sec. 4.1): Q(lambda) = (p2^1 - p1^1).(p2^0 - p1^0) at the t=0
// closest point and the fixed sample pattern; active when some sample has
// Q <= dhat |p2^0 - p1^0|.  Returns the closest-point coefficients in c.
__device__ bool partial_pair(int kind, const float4 a0[4], const float4 a1[4], float dhat, int ns, float c[4]) {
    V<float> p[4], e[4];
    for (int i = 0; i < 4; ++i) { p[i] = ld<float>(a0[i]); e[i] = ld<float>(a1[i]); }
    closest_coef<float>(kind, p, c);
    float lam[5][2];
    int n = 0;
    if (kind == 0) {
        lam[n][0] = c[2]; lam[n][1] = c[3]; ++n;
        if (ns == 1) { lam[n][0] = 1.f / 3.f; lam[n][1] = 1.f / 3.f; ++n; }
        if (ns == 3) {
            lam[n][0] = 1.f / 6.f; lam[n][1] = 1.f / 6.f; ++n;
            lam[n][0] = 2.f / 3.f; lam[n][1] = 1.f / 6.f; ++n;
            lam[n][0] = 1.f / 6.f; lam[n][1] = 2.f / 3.f; ++n;
        }
    } else {
        lam[n][0] = -c[1]; lam[n][1] = c[3]; ++n;
        if (ns == 1) { lam[n][0] = 0.5f; lam[n][1] = 0.5f; ++n; }
        if (ns == 4) {
            const float v[2] = {0.25f, 0.75f};
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) { lam[n][0] = v[i]; lam[n][1] = v[j]; ++n; }
        }
    }
    for (int k = 0; k < n; ++k) {
        float l1 = lam[k][0], l2 = lam[k][1];
        V<float> p10, p20, p11, p21;
        if (kind == 0) {
            p10 = p[0]; p11 = e[0];
            p20 = p[1] + (l1 * (p[2] - p[1]) + l2 * (p[3] - p[1]));
            p21 = e[1] + (l1 * (e[2] - e[1]) + l2 * (e[3] - e[1]));
        } else {
            p10 = p[0] + l1 * (p[1] - p[0]); p11 = e[0] + l1 * (e[1] - e[0]);
            p20 = p[2] + l2 * (p[3] - p[2]); p21 = e[2] + l2 * (e[3] - e[2]);
        }
        V<float> d0 = p20 - p10, d1 = p21 - p11;
        if (dotv(d1, d0) - dhat * sqrtf(dotv(d0, d0)) <= 0.f) return true;
    }
    return false;
}

// Partial CCD with the sample density of Eq. (sample_bound) (Sec. 4.1): for
// a pair that collides before alpha of the step, Q < 0 on the disc of radius
//   rho* = (1/alpha - 1) (H^0)^2 / (2 sqrt(2) L (H^1 + 2L))
// around the contact parameters (H^0: closest distance at t = 0; H^1: the
// largest distance between a point of one primitive and one of the other at
// t = 0 or 1, which bounds their distance over the step; L: the longest edge
// of either primitive at t = 0 or 1).  A square lattice of spacing 1/m with
// 1/m <= sqrt(2) rho* puts a sample inside that disc: m = ceil(1 / (sqrt(2)
// rho*)), at least 1, capped at max_axis (H^0 = 0: max_axis).  The bound and
// m are taken in FP64 (so that the lattice is the same as an FP64 reference
// computes from these positions); the samples, the t = 0 closest point and
// the lattice {(i/m, j/m)} (VT: i + j <= m, barycentric weights of the
// triangle's second and third vertex; EE: the two edge parameters), are
// tested in FP32 as the fixed patterns are.
__device__ int adaptive_axis(int kind, const float4 a0[4], const float4 a1[4], double alpha, int max_axis) {
    V<double> p[4], e[4];
    for (int i = 0; i < 4; ++i) { p[i] = ld<double>(a0[i]); e[i] = ld<double>(a1[i]); }
    const double h0 = gap_dist<double>(kind, p);
    double h1 = 0.0, L = 0.0;
    const int n1 = kind == 0 ? 1 : 2;
    for (int t = 0; t < 2; ++t) {
        const V<double> *q = t == 0 ? p : e;
        for (int i = 0; i < n1; ++i)
            for (int j = n1; j < 4; ++j) { V<double> d = q[j] - q[i]; h1 = fmax(h1, sqrt(dotv(d, d))); }
        if (kind == 0) {
            const int ed[3][2] = {{1, 2}, {2, 3}, {3, 1}};
            for (int k = 0; k < 3; ++k) { V<double> d = q[ed[k][1]] - q[ed[k][0]]; L = fmax(L, sqrt(dotv(d, d))); }
        } else {
            V<double> d = q[1] - q[0];
            L = fmax(L, sqrt(dotv(d, d)));
            d = q[3] - q[2];
            L = fmax(L, sqrt(dotv(d, d)));
        }
    }
    if (!(L > 0.0)) return 1;  // rho* infinite
    const double rho = (1.0 / alpha - 1.0) * h0 * h0 / (2.0 * sqrt(2.0) * L * (h1 + 2.0 * L));
    if (!(rho > 0.0)) return max_axis;
    const double need = 1.0 / (sqrt(2.0) * rho);
    if (!(need < (double)max_axis)) return max_axis;
    return max(1, (int)ceil(need));
}

__device__ bool partial_pair_adaptive(int kind, const float4 a0[4], const float4 a1[4], float dhat, double alpha,
                                      int max_axis, float c[4]) {
    V<float> p[4], e[4];
    for (int i = 0; i < 4; ++i) { p[i] = ld<float>(a0[i]); e[i] = ld<float>(a1[i]); }
    closest_coef<float>(kind, p, c);
    auto test = [&](float l1, float l2) {
        V<float> p10, p20, p11, p21;
        if (kind == 0) {
            p10 = p[0]; p11 = e[0];
            p20 = p[1] + (l1 * (p[2] - p[1]) + l2 * (p[3] - p[1]));
            p21 = e[1] + (l1 * (e[2] - e[1]) + l2 * (e[3] - e[1]));
        } else {
            p10 = p[0] + l1 * (p[1] - p[0]); p11 = e[0] + l1 * (e[1] - e[0]);
            p20 = p[2] + l2 * (p[3] - p[2]); p21 = e[2] + l2 * (e[3] - e[2]);
        }
        V<float> d0 = p20 - p10, d1 = p21 - p11;
        return dotv(d1, d0) - dhat * sqrtf(dotv(d0, d0)) <= 0.f;
    };
    // the t = 0 closest point first (FP64 coefficients, as the bound's)
    {
        V<double> q[4];
        for (int i = 0; i < 4; ++i) q[i] = ld<double>(a0[i]);
        double cd[4];
        closest_coef<double>(kind, q, cd);
        if (kind == 0 ? test((float)cd[2], (float)cd[3]) : test((float)-cd[1], (float)cd[3])) return true;
    }
    const int m = adaptive_axis(kind, a0, a1, alpha, max_axis);
    const float inv = 1.f / (float)m;
    for (int i = 0; i <= m; ++i) {
        const int jm = kind == 0 ? m - i : m;
        for (int j = 0; j <= jm; ++j)
            if (test((float)i * inv, (float)j * inv)) return true;
    }
    return false;
}

__device__ inline bool partial_test(int kind, const float4 a0[4], const float4 a1[4], const CollParams &P, float c[4]) {
    if (P.adaptive) return partial_pair_adaptive(kind, a0, a1, P.dhat, P.alpha, P.max_axis, c);
    return partial_pair(kind, a0, a1, P.dhat, kind == 0 ? P.samples_vt : P.samples_ee, c);
}

// Unit start direction of the gap vector; falls back to the triangle normal
// (VT) or the edge cross product (EE) when the gap vanishes.
__device__ float3 start_dir(int kind, const float4 a0[4], const float c[4]) {
    float3 q[4];
    for (int i = 0; i < 4; ++i) q[i] = f3(a0[i]);
    float3 d = c[0] * q[0] + c[1] * q[1] + c[2] * q[2] + c[3] * q[3];
    float l = sqrtf(dot3(d, d));
    if (l > 1e-30f) return (1.f / l) * d;
    float3 nn = kind == 0 ? cross3(q[2] - q[1], q[3] - q[1]) : cross3(q[1] - q[0], q[3] - q[2]);
    l = sqrtf(dot3(nn, nn));
    return l > 1e-30f ? (1.f / l) * nn : make_float3(0.f, 0.f, 1.f);
}

// Index guard: an entry of a device-built list that lies outside the current
// topology sets a bit in the handle's guard word (CollView::guard) and is
// skipped (no access through it); the host reads the word after each step
// and fails the step.
enum GuardBits { GUARD_PAIR = 1, GUARD_WATCH = 2, GUARD_NEAR = 4, GUARD_ACTIVE = 8 };
__device__ inline void guard_raise(const CollView &cv, unsigned int bit) {
    if (cv.guard) atomicOr(cv.guard, bit);
}

__device__ inline bool pair_ids(const CollView &cv, const int2 *vt, const int2 *ee, long long nvt, long long idx,
                                int ids[4], int &kind) {
    ids[0] = ids[1] = ids[2] = ids[3] = 0;
    if (idx < nvt) {
        int2 p = vt[idx];
        kind = 0;
        if (p.x < 0 || p.x >= cv.nv || p.y < 0 || p.y >= cv.nt) {
            guard_raise(cv, GUARD_PAIR);
            return false;
        }
        int4 T = cv.tri[p.y];
        ids[0] = p.x; ids[1] = T.x; ids[2] = T.y; ids[3] = T.z;
    } else {
        int2 p = ee[idx - nvt];
        kind = 1;
        if (p.x < 0 || p.x >= cv.ne || p.y < 0 || p.y >= cv.ne) {
            guard_raise(cv, GUARD_PAIR);
            return false;
        }
        int2 E = cv.edge[p.x], F = cv.edge[p.y];
        ids[0] = E.x; ids[1] = E.y; ids[2] = F.x; ids[3] = F.y;
    }
    return true;
}

__device__ inline float ndb_weight(const CollParams &P, int a) {
    float w = P.k_ndb;
    for (int i = 0; i < a; ++i) w *= P.K_ndb;  // w = k K^a, Eq. (exp)
    return w;
}

// Warp-aggregated append (all 32 lanes must call it together).
__device__ inline void append_active(bool want, const ActivePair &ap, ActivePair *act, int cap, int *n_act,
                                     int *overflow) {
    unsigned m = __ballot_sync(0xffffffffu, want);
    if (!m) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(n_act, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (want) {
        int slot = base + __popc(m & ((1u << lane) - 1u));
        if (slot < cap) act[slot] = ap;
        else atomicOr(overflow, OVF_ACTIVE);
    }
}

__device__ inline long long find_pair(const int2 *list, long long n, int2 key) {
    long long lo = 0, hi = n;
    while (lo < hi) {
        long long mid = (lo + hi) >> 1;
        int2 v = list[mid];
        if (v.x < key.x || (v.x == key.x && v.y < key.y)) lo = mid + 1; else hi = mid;
    }
    if (lo < n) {
        int2 v = list[lo];
        if (v.x == key.x && v.y == key.y) return lo;
    }
    return -1;
}

// The same search within the segment of key.x when the list's per-primary
// offsets are known (off: np primaries, the last segment ends at n).
__device__ inline long long find_pair_seg(const int2 *list, long long n, const int *off, int np, int2 key) {
    if (key.x < 0 || key.x >= np) return -1;
    long long b = off[key.x], e = key.x + 1 < np ? (long long)off[key.x + 1] : n;
    b = max(b, 0ll);
    e = min(e, n);
    for (long long j = b; j < e; ++j) {
        const int2 v = list[j];
        if (v.x == key.x && v.y == key.y) return j;
        if (v.x != key.x || v.y > key.y) break;
    }
    return -1;
}

constexpr int PAIR_THREADS = 256;

// Full CCD in two kernels.  k_full_ccd_filter takes every pair: its NDB
// state carried from the previous list (merge), then the FP32 filter; a pair
// that cannot hit is done, the others are appended (warp-aggregated) to a
// survivor list.  k_full_ccd_exact runs the FP64 part on the survivors only,
// so the filter runs at full occupancy and the FP64 registers are paid only
// where needed.  An impact in [0, 1] makes the pair active.
__global__ void __launch_bounds__(PAIR_THREADS) k_full_ccd_filter(
    CollView cv, const int2 *__restrict__ vt, const int2 *__restrict__ ee, const long long *nvt_p,
    const long long *nee_p, unsigned char *__restrict__ st_vt, unsigned char *__restrict__ st_ee,
    const int2 *__restrict__ ovt, const int2 *__restrict__ oee, const long long *onvt_p, const long long *onee_p,
    const unsigned char *__restrict__ ost_vt, const unsigned char *__restrict__ ost_ee,
    const int *__restrict__ ooff_v, const int *__restrict__ ooff_e, const float4 *__restrict__ x0,
    const float4 *__restrict__ x1, double eta, int *__restrict__ surv, int *nsurv, long long cap) {
    const long long nvt = *nvt_p, n = nvt + *nee_p;
    const long long onvt = ovt ? *onvt_p : 0, onee = oee ? *onee_p : 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const unsigned lane = threadIdx.x & 31;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += stride) {  // warp-uniform trip count
        const long long idx = base + lane;
        bool hit = false;
        int ids[4], kind;
        if (idx < n && pair_ids(cv, vt, ee, nvt, idx, ids, kind)) {
            unsigned char st = 0;
            if (ovt) {
                long long j;
                if (kind == 0) {
                    j = ooff_v ? find_pair_seg(ovt, onvt, ooff_v, cv.nv, vt[idx]) : find_pair(ovt, onvt, vt[idx]);
                    if (j >= 0) st = ost_vt[j];
                } else {
                    j = ooff_e ? find_pair_seg(oee, onee, ooff_e, cv.ne, ee[idx - nvt])
                               : find_pair(oee, onee, ee[idx - nvt]);
                    if (j >= 0) st = ost_ee[j];
                }
                if (!(st & ST_ACTIVE)) st = 0;
            }
            if (kind == 0) st_vt[idx] = st;
            else st_ee[idx - nvt] = st;
            float4 a0[4], a1[4];
            for (int i = 0; i < 4; ++i) {
                a0[i] = x0[ids[i]];
                a1[i] = x1[ids[i]];
            }
            hit = ccd_may_hit(kind, a0, a1, eta);
        }
        const unsigned m = __ballot_sync(0xffffffffu, hit);
        if (m) {
            int b0 = 0;
            if (lane == 0) b0 = atomicAdd(nsurv, __popc(m));
            b0 = __shfl_sync(0xffffffffu, b0, 0);
            const long long pos = (long long)b0 + __popc(m & ((1u << lane) - 1u));
            if (hit && pos < cap) surv[pos] = (int)idx;
        }
    }
}

__global__ void __launch_bounds__(PAIR_THREADS) k_full_ccd_exact(CollView cv, const int2 *__restrict__ vt,
                                                                 const int2 *__restrict__ ee, const long long *nvt_p,
                                                                 unsigned char *__restrict__ st_vt,
                                                                 unsigned char *__restrict__ st_ee,
                                                                 const int *__restrict__ surv, const int *nsurv,
                                                                 long long cap, const float4 *__restrict__ x0,
                                                                 const float4 *__restrict__ x1, double eta,
                                                                 unsigned long long *toi_min) {
    const long long nvt = *nvt_p, ns = min((long long)*nsurv, cap);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < ns;
         k += (long long)gridDim.x * blockDim.x) {
        const long long idx = surv[k];
        int ids[4], kind;
        if (!pair_ids(cv, vt, ee, nvt, idx, ids, kind)) continue;
        float4 a0[4], a1[4];
        for (int i = 0; i < 4; ++i) {
            a0[i] = x0[ids[i]];
            a1[i] = x1[ids[i]];
        }
        const double t = ccd_exact(kind, a0, a1, eta);
        if (t <= 1.0) {
            if (kind == 0) st_vt[idx] |= ST_ACTIVE;
            else st_ee[idx - nvt] |= ST_ACTIVE;
            const unsigned long long tb = (unsigned long long)__double_as_longlong(t);
            atomicMin(toi_min, tb);
            if (cv.toi_inst)  // every instance the pair touches
                for (int j = 0; j < 4; ++j) {
                    const int kk = cv.vinst[ids[j]];
                    if (kk >= 0) atomicMin(&cv.toi_inst[kk], tb);
                }
        }
    }
}

// After a full CCD: store each pair's closest distance on x^- (the partial-CCD
// filter's d0; x^- is fixed for the step) and rebuild the active list from
// the pair states, with closest points and start directions on x^-.
__global__ void __launch_bounds__(PAIR_THREADS) k_pairs_collect(CollView cv, const int2 *__restrict__ vt,
                                                               const int2 *__restrict__ ee, const long long *nvt_p,
                                                               const long long *nee_p,
                                                               const unsigned char *__restrict__ st_vt,
                                                               const unsigned char *__restrict__ st_ee,
                                                               float *d0_vt, float *d0_ee,
                                                               const float4 *__restrict__ xm, CollParams P,
                                                               ActivePair *act, int cap, int *n_act, int *overflow) {
    long long nvt = *nvt_p, n = nvt + *nee_p;
    long long stride = (long long)gridDim.x * blockDim.x;
    long long start = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    for (long long base = start; base < n; base += stride) {  // warp-uniform trip count
        long long idx = base + (threadIdx.x & 31);
        bool want = false;
        ActivePair ap;
        int ids[4], kind;
        if (idx < n && pair_ids(cv, vt, ee, nvt, idx, ids, kind)) {
            unsigned char st = kind == 0 ? st_vt[idx] : st_ee[idx - nvt];
            float4 a0[4];
            for (int i = 0; i < 4; ++i) a0[i] = xm[ids[i]];
            V<float> q[4];
            for (int i = 0; i < 4; ++i) q[i] = ld<float>(a0[i]);
            float c[4];
            closest_coef<float>(kind, q, c);
            V<float> d = c[0] * q[0] + c[1] * q[1] + c[2] * q[2] + c[3] * q[3];
            float dist = sqrtf(dotv(d, d));
            if (kind == 0) d0_vt[idx] = dist;
            else d0_ee[idx - nvt] = dist;
            if (st & ST_ACTIVE) {
                want = true;
                float3 n0 = start_dir(kind, a0, c);
                ap.ids = make_int4(ids[0], ids[1], ids[2], ids[3]);
                ap.c = make_float4(c[0], c[1], c[2], c[3]);
                ap.n0w = make_float4(n0.x, n0.y, n0.z, ndb_weight(P, st & 0x7f));
            }
        }
        append_active(want, ap, act, cap, n_act, overflow);
    }
}


// ------------------------------------------------------------------ partial-CCD filter
// Pass structure (one partial CCD, Sec. 4.1): k_pccd_disp -> k_pccd_decide
// -> k_pccd_filter -> k_pccd_test.  The filter applies the displacement
// bound to every pair (full pass) or only to the watch list; the test runs
// the sampled activity test of Eq. (query) on the near pairs only.  Pairs the
// filter proves non-near are inactive, exactly as the test would find them.

__device__ inline void warp_max_atomic(float v, unsigned int *dst) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0.f) atomicMax(dst, __float_as_uint(v));
}

// disp = xp - xm; amax = max |disp - disp0| (disp0 := the previous disp when
// the previous pass was full, i.e. the reference moves to that pass).
__global__ void k_pccd_disp(int nv, const float4 *__restrict__ xm, const float4 *__restrict__ xp,
                            float4 *__restrict__ disp, float4 *__restrict__ disp0, PccdState *ps, const int *live) {
    if (loop_dead(live)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool moved_ref = ps->pass_full != 0;
    float m = 0.f;
    if (i < nv) {
        float3 ref;
        if (moved_ref) {
            float4 old = disp[i];
            disp0[i] = old;
            ref = f3(old);
        } else {
            ref = f3(disp0[i]);
        }
        float3 d = f3(xp[i]) - f3(xm[i]);
        disp[i] = f4(d);
        float3 e = d - ref;
        m = sqrtf(dot3(e, e));
    }
    warp_max_atomic(m, &ps->amax_bits);
}

// Finishes the previous pass (a full pass installs its watch list) and
// decides this one; resets the per-pass counters.
__global__ void k_pccd_decide(PccdState *ps, float tau, long long cap, const int *live, int *n_act) {
    if (loop_dead(live)) return;
    if (n_act) *n_act = 0;  // the active list is rebuilt by this pass
    PccdState p = *ps;
    if (p.pass_full) {
        p.cur ^= 1;
        p.n_watch = p.n_watch_new;
        p.watch_ok = p.n_watch_new <= cap;
    }
    float amax = __uint_as_float(p.amax_bits);
    // 1% slack over the bound 2 amax < tau keeps FP32 rounding on the safe side
    p.pass_full = (p.force_full || !p.watch_ok || !(2.f * amax < 0.99f * tau)) ? 1 : 0;
    p.force_full = 0;
    p.amax_bits = 0;
    p.n_near = 0;
    p.n_watch_new = 0;
    *ps = p;
}

__device__ inline void warp_append_idx(bool want, int idx, int *list, int *count, long long cap, int *flag,
                                       int flag_bit) {
    unsigned m = __ballot_sync(0xffffffffu, want);
    if (!m) return;
    int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (want) {
        long long slot = (long long)base + __popc(m & ((1u << lane) - 1u));
        if (slot < cap) list[slot] = idx;
        else if (flag) atomicOr(flag, flag_bit);
    }
}

__global__ void __launch_bounds__(256) k_pccd_filter(CollView cv, const int2 *__restrict__ vt,
                                                     const int2 *__restrict__ ee, const long long *nvt_p,
                                                     const long long *nee_p, unsigned char *st_vt,
                                                     unsigned char *st_ee, const float *__restrict__ d0_vt,
                                                     const float *__restrict__ d0_ee,
                                                     const float4 *__restrict__ disp4, float dhat, float tau,
                                                     PccdState *ps, int *watch0, int *watch1, int *near,
                                                     long long cap) {
    if (loop_dead(cv.live)) return;
    const bool full = ps->pass_full != 0;
    const int cur = ps->cur;
    const int *watch = cur ? watch1 : watch0;
    int *watch_new = cur ? watch0 : watch1;
    long long nvt = *nvt_p;
    long long n = full ? nvt + *nee_p : (long long)ps->n_watch;
    long long stride = (long long)gridDim.x * blockDim.x;
    long long start = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    for (long long base = start; base < n; base += stride) {  // warp-uniform trip count
        long long t = base + (threadIdx.x & 31);
        bool is_near = false, keep = false;
        int idx = 0;
        int ids[4], kind;
        if (t < n) idx = full ? (int)t : watch[t];
        bool valid = t < n && idx >= 0 && idx < nvt + *nee_p;
        if (t < n && !valid) guard_raise(cv, GUARD_WATCH);
        if (valid && pair_ids(cv, vt, ee, nvt, idx, ids, kind)) {
            float d0 = kind == 0 ? d0_vt[idx] : d0_ee[idx - nvt];
            // |d1 - d0| at any sample is at most the largest relative
            // displacement between a vertex of side 1 and one of side 2
            float4 D[4];
            for (int q = 0; q < 4; ++q) D[q] = disp4[ids[q]];
            float rel = 0.f;
            int n1 = kind == 0 ? 1 : 2;
            for (int a = 0; a < n1; ++a)
                for (int b = n1; b < 4; ++b) {
                    float3 dd = make_float3(D[b].x - D[a].x, D[b].y - D[a].y, D[b].z - D[a].z);
                    rel = fmaxf(rel, dot3(dd, dd));
                }
            float srel = sqrtf(rel);
            is_near = d0 <= (dhat + srel) * 1.001f + 1e-7f;
            if (!is_near) {
                unsigned char *stp = kind == 0 ? st_vt + idx : st_ee + (idx - nvt);
                if (*stp) *stp = 0;
            }
            if (full) keep = is_near || (d0 - 1e-7f) / 1.001f - dhat - srel < tau;
        }
        warp_append_idx(is_near, idx, near, &ps->n_near, cap, nullptr, 0);
        if (full) warp_append_idx(keep, idx, watch_new, &ps->n_watch_new, cap, nullptr, 0);
    }
}

// Sampled activity test on the near pairs: state update (a + 1 while active,
// reset when not) and the active list.
__global__ void __launch_bounds__(256) k_pccd_test(CollView cv, const int2 *__restrict__ vt,
                                                   const int2 *__restrict__ ee, const long long *nvt_p,
                                                   const long long *nee_p,
                                                   unsigned char *st_vt, unsigned char *st_ee,
                                                   const float4 *__restrict__ xm, const float4 *__restrict__ xp,
                                                   CollParams P, const int *__restrict__ near,
                                                   const PccdState *ps, long long cap, ActivePair *act,
                                                   int cap_act, int *n_act, int *overflow) {
    if (loop_dead(cv.live)) return;
    long long nvt = *nvt_p;
    long long n = min((long long)ps->n_near, cap);
    long long stride = (long long)gridDim.x * blockDim.x;
    long long start = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    for (long long base = start; base < n; base += stride) {
        long long t = base + (threadIdx.x & 31);
        bool want = false;
        ActivePair ap;
        int ids[4], kind;
        int idx = t < n ? near[t] : -1;
        bool valid = idx >= 0 && idx < nvt + *nee_p;
        if (t < n && !valid) guard_raise(cv, GUARD_NEAR);
        if (valid && pair_ids(cv, vt, ee, nvt, idx, ids, kind)) {
            unsigned char *stp = kind == 0 ? st_vt + idx : st_ee + (idx - nvt);
            unsigned char st = *stp;
            float4 a0[4], a1[4];
            for (int i = 0; i < 4; ++i) {
                a0[i] = xm[ids[i]];
                a1[i] = xp[ids[i]];
            }
            float c[4];
            bool flag = partial_test(kind, a0, a1, P, c);
            if (flag) {
                int a = (st & ST_ACTIVE) ? min((int)(st & 0x7f) + 1, P.a_max) : 0;
                st = ST_ACTIVE | (unsigned char)a;
            } else {
                st = 0;
            }
            *stp = st;
            if (flag) {
                want = true;
                float3 n0 = start_dir(kind, a0, c);
                ap.ids = make_int4(ids[0], ids[1], ids[2], ids[3]);
                ap.c = make_float4(c[0], c[1], c[2], c[3]);
                ap.n0w = make_float4(n0.x, n0.y, n0.z, ndb_weight(P, st & 0x7f));
            }
        }
        append_active(want, ap, act, cap_act, n_act, overflow);
    }
}

// Collision springs (Sec. 5.1, A_i = B_i = Id): constraint C(x) = d(x).n0 - dhat
// with d = sum_j c_j x_j; the least-norm displacement restoring C = 0 moves
// movable vertex j by -min(C,0) c_j n0 / sum_k c_k^2; every movable vertex
// of the pair gets weight w toward its target (held in place when c_j = 0).
__global__ void k_contact(CollView cv, const ActivePair *__restrict__ act, const int *n_act_p, int cap,
                          const float4 *__restrict__ x, float dhat, float *__restrict__ cw, float4 *__restrict__ cf) {
    if (loop_dead(cv.live)) return;
    int n = min(*n_act_p, cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        ActivePair ap = act[i];
        int ids[4] = {ap.ids.x, ap.ids.y, ap.ids.z, ap.ids.w};
        if (min(min(ids[0], ids[1]), min(ids[2], ids[3])) < 0 || max(max(ids[0], ids[1]), max(ids[2], ids[3])) >= cv.nv) {
            guard_raise(cv, GUARD_ACTIVE);
            continue;
        }
        float c[4] = {ap.c.x, ap.c.y, ap.c.z, ap.c.w};
        float3 n0 = make_float3(ap.n0w.x, ap.n0w.y, ap.n0w.z);
        float w = ap.n0w.w;
        float3 d = make_float3(0.f, 0.f, 0.f);
        float S = 0.f;
        bool mv[4];
        for (int j = 0; j < 4; ++j) {
            d = d + c[j] * f3(x[ids[j]]);
            mv[j] = !cv.vfixed[ids[j]];
            if (mv[j]) S += c[j] * c[j];
        }
        if (!(S > 0.f)) continue;
        float C = dot3(d, n0) - dhat;
        float k = -fminf(C, 0.f) / S;
        for (int j = 0; j < 4; ++j) {
            if (!mv[j]) continue;
            int v = ids[j];
            atomicAdd(&cw[v], w);
            float s = w * k * c[j];
            if (s != 0.f) {
                atomicAdd(&cf[v].x, s * n0.x);
                atomicAdd(&cf[v].y, s * n0.y);
                atomicAdd(&cf[v].z, s * n0.z);
            }
        }
    }
}

__global__ void k_contact_list(int n, const float *__restrict__ cw, int *__restrict__ list, int *count,
                               const int *live) {
    if (loop_dead(live)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool want = i < n && cw[i] > 0.f;
    unsigned m = __ballot_sync(0xffffffffu, want);
    if (!m) return;
    int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (want) list[base + __popc(m & ((1u << lane) - 1u))] = i;
}

// ----------------------------------------------------------------- stage helpers
__global__ void k_ccd_quads(const int4 *q, const int *kinds, long long np, const float4 *x0, const float4 *x1,
                            double eta, double *toi) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (long long)gridDim.x * blockDim.x) {
        int4 Q = q[i];
        int ids[4] = {Q.x, Q.y, Q.z, Q.w};
        float4 a0[4], a1[4];
        for (int k = 0; k < 4; ++k) { a0[k] = x0[ids[k]]; a1[k] = x1[ids[k]]; }
        toi[i] = ccd_pair(kinds[i], a0, a1, eta);
    }
}

__global__ void k_partial_quads(const int4 *q, const int *kinds, long long np, const float4 *x0, const float4 *x1,
                                CollParams P, int *active) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (long long)gridDim.x * blockDim.x) {
        int4 Q = q[i];
        int ids[4] = {Q.x, Q.y, Q.z, Q.w};
        float4 a0[4], a1[4];
        for (int k = 0; k < 4; ++k) { a0[k] = x0[ids[k]]; a1[k] = x1[ids[k]]; }
        float c[4];
        int kind = kinds[i];
        active[i] = partial_test(kind, a0, a1, P, c) ? 1 : 0;
    }
}

__global__ void k_activate_quads(const int4 *q, const int *kinds, const float *w, long long np, const float4 *xm,
                                 ActivePair *act, int *n_act) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (long long)gridDim.x * blockDim.x) {
        int4 Q = q[i];
        int ids[4] = {Q.x, Q.y, Q.z, Q.w};
        float4 a0[4];
        V<float> p[4];
        for (int k = 0; k < 4; ++k) { a0[k] = xm[ids[k]]; p[k] = ld<float>(a0[k]); }
        float c[4];
        int kind = kinds[i];
        closest_coef<float>(kind, p, c);
        float3 n0 = start_dir(kind, a0, c);
        ActivePair ap;
        ap.ids = Q;
        ap.c = make_float4(c[0], c[1], c[2], c[3]);
        ap.n0w = make_float4(n0.x, n0.y, n0.z, w[i]);
        act[i] = ap;
        if (i == 0) *n_act = (int)np;
    }
}

__global__ void k_pairs_to_quads(CollView cv, const int2 *ee, long long nee, int4 *out) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nee; i += (long long)gridDim.x * blockDim.x) {
        int2 p = ee[i];
        int2 E = cv.edge[p.x], F = cv.edge[p.y];
        out[i] = make_int4(E.x, E.y, F.x, F.y);
    }
}

inline int nblk(long long n, int b) { return (int)std::min<long long>((n + b - 1) / b, 152LL * 16); }

}  // namespace

unsigned int pair_guard_take(cudaStream_t s, unsigned int *guard) {
    unsigned int v = 0;
    PDC_CK(cudaMemcpyAsync(&v, guard, sizeof(v), cudaMemcpyDeviceToHost, s));
    PDC_CK(cudaStreamSynchronize(s));
    if (v) PDC_CK(cudaMemsetAsync(guard, 0, sizeof(v), s));
    return v;
}

void launch_full_ccd(cudaStream_t s, const CollView &cv, BroadPhase &bp, const float4 *x0, const float4 *x1,
                     const CollParams &P, bool merge, unsigned long long *toi_min) {
    int c = bp.cur, o = c ^ 1;
    // survivors of the filter go to the near list (free until the next partial CCD)
    bp.ccd_count.alloc(1);
    auto launch = [&](int blocks) {
        bp.ccd_count.zero(s);
        k_full_ccd_filter<<<blocks, PAIR_THREADS, 0, s>>>(
            cv, bp.vt[c], bp.ee[c], bp.cnt_vt_d[c], bp.cnt_ee_d[c], bp.st_vt[c], bp.st_ee[c],
            merge ? bp.vt[o].p : nullptr, merge ? bp.ee[o].p : nullptr, bp.cnt_vt_d[o], bp.cnt_ee_d[o], bp.st_vt[o],
            bp.st_ee[o], merge && bp.off_ok[o] ? bp.off_v[o].p : nullptr, merge && bp.off_ok[o] ? bp.off_e[o].p : nullptr,
            x0, x1, P.eta, bp.near, bp.ccd_count, bp.cap_pairs);
        k_full_ccd_exact<<<blocks, PAIR_THREADS, 0, s>>>(cv, bp.vt[c], bp.ee[c], bp.cnt_vt_d[c], bp.st_vt[c],
                                                         bp.st_ee[c], bp.near, bp.ccd_count, bp.cap_pairs, x0, x1,
                                                         P.eta, toi_min);
        PDC_LAUNCH_CK();
    };
    if (bp.tune_pairs) {
        // every candidate computes the same states and minimum (the kernel is
        // idempotent): time each on this list and keep the fastest grid
        bp.tune_pairs = false;
        const int cand[4] = {152 * 2, 152 * 4, 152 * 8, 152 * 16};
        cudaEvent_t e[5];
        for (auto &ev : e) PDC_CK(cudaEventCreate(&ev));
        launch(cand[2]);  // warm-up
        PDC_CK(cudaEventRecord(e[0], s));
        for (int k = 0; k < 4; ++k) {
            launch(cand[k]);
            PDC_CK(cudaEventRecord(e[k + 1], s));
        }
        PDC_CK(cudaEventSynchronize(e[4]));
        for (int k = 0; k < 4; ++k) PDC_CK(cudaEventElapsedTime(&bp.pair_ms[k], e[k], e[k + 1]));
        int best = 0;  // the fastest, once all are timed
        for (int k = 1; k < 4; ++k)
            if (bp.pair_ms[k] < bp.pair_ms[best]) best = k;
        for (auto &ev : e) cudaEventDestroy(ev);
        bp.pair_blocks = cand[best];
    }
    launch(bp.pair_blocks);
}

void launch_collect_active(cudaStream_t s, const CollView &cv, BroadPhase &bp, const float4 *xm,
                           const CollParams &P, ActivePair *act, int cap_act, int *n_act, int *overflow) {
    int c = bp.cur;
    PDC_CK(cudaMemsetAsync(n_act, 0, sizeof(int), s));
    k_pairs_collect<<<bp.pair_blocks, PAIR_THREADS, 0, s>>>(cv, bp.vt[c], bp.ee[c], bp.cnt_vt_d[c], bp.cnt_ee_d[c],
                                                         bp.st_vt[c], bp.st_ee[c], bp.d0_vt[c], bp.d0_ee[c], xm, P,
                                                         act, cap_act, n_act, overflow);
    PDC_LAUNCH_CK();
}

void launch_partial_ccd(cudaStream_t s, const CollView &cv, BroadPhase &bp, const float4 *xm, const float4 *xp,
                        const CollParams &P, ActivePair *act, int cap_act, int *n_act, int *overflow, float4 *disp) {
    int c = bp.cur;
    // watch gap: pairs within 2 d_hat of the near bound are re-tested every pass
    const float tau = 2.f * P.dhat;
    if (bp.prof) bp.prof->begin(s, "pccd_prep", 40.0 * cv.nv);
    if (cv.nv > 0) k_pccd_disp<<<(cv.nv + 255) / 256, 256, 0, s>>>(cv.nv, xm, xp, disp, bp.disp0, bp.pccd, cv.live);
    k_pccd_decide<<<1, 1, 0, s>>>(bp.pccd, tau, bp.cap_pairs, cv.live, n_act);
    PDC_LAUNCH_CK();
    if (bp.prof) bp.prof->end(s);
    // (full or watch-list pass is decided on the device: no byte model here)
    if (bp.prof) bp.prof->begin(s, "pccd_filter", 0.0);
    k_pccd_filter<<<bp.pair_blocks, PAIR_THREADS, 0, s>>>(cv, bp.vt[c], bp.ee[c], bp.cnt_vt_d[c], bp.cnt_ee_d[c],
                                                       bp.st_vt[c], bp.st_ee[c], bp.d0_vt[c], bp.d0_ee[c], disp,
                                                       P.dhat, tau, bp.pccd, bp.watch[0], bp.watch[1], bp.near,
                                                       bp.cap_pairs);
    PDC_LAUNCH_CK();
    if (bp.prof) bp.prof->end(s);
    if (bp.prof) bp.prof->begin(s, "pccd_test", 0.0);
    k_pccd_test<<<bp.pair_blocks, PAIR_THREADS, 0, s>>>(cv, bp.vt[c], bp.ee[c], bp.cnt_vt_d[c], bp.cnt_ee_d[c], bp.st_vt[c],
                                                     bp.st_ee[c], xm, xp, P, bp.near, bp.pccd, bp.cap_pairs, act,
                                                     cap_act, n_act, overflow);
    PDC_LAUNCH_CK();
    if (bp.prof) bp.prof->end(s);
}

// Residual forwarding: every active constraint at the base weight k (a = 0).
__global__ void k_rf_weights(ActivePair *act, const int *n_act, int cap, float k) {
    const int n = min(*n_act, cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) act[i].n0w.w = k;
}

void launch_rf_weights(cudaStream_t s, ActivePair *act, const int *n_act, int cap_act, float k) {
    k_rf_weights<<<152, 256, 0, s>>>(act, n_act, cap_act, k);
    PDC_LAUNCH_CK();
}

void launch_contact(cudaStream_t s, const CollView &cv, const ActivePair *act, const int *n_act, int cap_act,
                    const float4 *x, float dhat, float *cw, float4 *cf) {
    k_contact<<<152 * 4, 256, 0, s>>>(cv, act, n_act, cap_act, x, dhat, cw, cf);
    PDC_LAUNCH_CK();
}

void launch_contact_list(cudaStream_t s, int n, const float *cw, int *list, int *count, const int *live,
                         bool zero) {
    if (zero) launch_live_zero(s, live, count, sizeof(int));
    if (n > 0) k_contact_list<<<(n + 255) / 256, 256, 0, s>>>(n, cw, list, count, live);
    PDC_LAUNCH_CK();
}

void launch_ccd_quads(cudaStream_t s, const int4 *quads, const int *kinds, long long np, const float4 *x0,
                      const float4 *x1, double eta, double *toi) {
    if (np > 0) k_ccd_quads<<<nblk(np, 128), 128, 0, s>>>(quads, kinds, np, x0, x1, eta, toi);
    PDC_LAUNCH_CK();
}

void launch_partial_quads(cudaStream_t s, const int4 *quads, const int *kinds, long long np, const float4 *x0,
                          const float4 *x1, const CollParams &P, int *active) {
    if (np > 0) k_partial_quads<<<nblk(np, 128), 128, 0, s>>>(quads, kinds, np, x0, x1, P, active);
    PDC_LAUNCH_CK();
}

void launch_activate_quads(cudaStream_t s, const int4 *quads, const int *kinds, const float *w, long long np,
                           const float4 *xm, ActivePair *act, int *n_act) {
    PDC_CK(cudaMemsetAsync(n_act, 0, sizeof(int), s));
    if (np > 0) k_activate_quads<<<nblk(np, 128), 128, 0, s>>>(quads, kinds, w, np, xm, act, n_act);
    PDC_LAUNCH_CK();
}

void launch_pairs_to_quads(cudaStream_t s, const CollView &cv, const int2 *ee, long long nee, int4 *out) {
    if (nee > 0) k_pairs_to_quads<<<nblk(nee, 256), 256, 0, s>>>(cv, ee, nee, out);
    PDC_LAUNCH_CK();
}

}  // namespace pdc
