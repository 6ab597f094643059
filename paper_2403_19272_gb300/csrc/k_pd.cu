// Projective-dynamics kernels: inertial target, local projections fused with
// the residual of the global system, Jacobi sweeps, line search.
//
// All vertex streams are float4 (16 B); one thread per vertex.  The
// residual is formed in "force form": instead of assembling b and
// subtracting H x (two large, nearly cancelling vectors), every element adds
// its force w (target - current) directly, which is the same vector
// r = b - (H + dH) x of Eq. (global) without the cancellation error.
#include <algorithm>

#include "pdc_internal.cuh"
#include "pdc_async.cuh"

namespace pdc {

namespace {

__device__ inline float warp_sum(float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ inline float warp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum of one float, added (one atomic per block) into a double.
__device__ inline void block_add(float v, double *dst) {
    __shared__ float part[32];
    v = warp_sum(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) part[w] = v;
    __syncthreads();
    if (w == 0) {
        int nw = (blockDim.x + 31) >> 5;
        float t = lane < nw ? part[lane] : 0.f;
        t = warp_sum(t);
        if (lane == 0 && t != 0.f) atomicAdd(dst, (double)t);
    }
}

__device__ inline void block_max(float v, unsigned int *dst) {
    __shared__ float part[32];
    v = warp_max(v);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) part[w] = v;
    __syncthreads();
    if (w == 0) {
        int nw = (blockDim.x + 31) >> 5;
        float t = lane < nw ? part[lane] : 0.f;
        t = warp_max(t);
        if (lane == 0 && t > 0.f) atomicMax(dst, __float_as_uint(t));
    }
}

// Closest 3x2 matrix with orthonormal columns to F = [f1 f2] (polar factor).
// C = F^T F = [[a, b], [b, d]];  with s = sqrt(det C) and t = sqrt(tr C + 2s)
// the inverse square root is C^{-1/2} = [[d + s, -b], [-b, a + s]] / (s t),
// and R = F C^{-1/2}.  Nearly rank-deficient F: Gram-Schmidt of its columns.
__device__ inline void polar32(float3 f1, float3 f2, float3 &r1, float3 &r2) {
    float a = dot3(f1, f1), b = dot3(f1, f2), d = dot3(f2, f2);
    float det = fmaf(a, d, -b * b);
    float tr = a + d;
    if (det > 1e-10f * tr * tr) {
        float s = sqrtf(det);
        float t = sqrtf(tr + 2.f * s);
        float k = 1.f / (s * t);
        float m00 = (d + s) * k, m01 = -b * k, m11 = (a + s) * k;
        r1 = m00 * f1 + m01 * f2;
        r2 = m01 * f1 + m11 * f2;
        return;
    }
    float n1 = sqrtf(a);
    float3 c1 = n1 > 1e-30f ? (1.f / n1) * f1 : make_float3(1.f, 0.f, 0.f);
    float3 c2 = f2 - dot3(f2, c1) * c1;
    float n2 = sqrtf(dot3(c2, c2));
    if (n2 <= 1e-6f * fmaxf(n1, 1e-30f)) {
        float ax = fabsf(c1.x), ay = fabsf(c1.y), az = fabsf(c1.z);
        float3 e = (ax <= ay && ax <= az) ? make_float3(1, 0, 0) : (ay <= az ? make_float3(0, 1, 0) : make_float3(0, 0, 1));
        c2 = e - dot3(e, c1) * c1;
        n2 = sqrtf(dot3(c2, c2));
    }
    r1 = c1;
    r2 = (1.f / n2) * c2;
}

// Positions inside a step are carried as x = x* + u: x* (the step's start
// state, FP32) stays fixed and u is a small FP32 displacement.  Differences
// of neighbouring x* entries are exact in FP32, so element quantities keep
// the precision of u instead of the ulp of the absolute coordinates.

// Eq. (z): z - x* = h v* + h^2 g (f_ext = m g), plus 2 dx of the previous
// step's residual forwarding when given (Eq. z_rf: h^2 M^-1 df = 2 dx); the
// iterate starts at u = z - x*.
__global__ void k_prologue(int n, const float4 *__restrict__ xs, const float4 *__restrict__ vs, float h, float3 g,
                           const float4 *__restrict__ rf, float4 *__restrict__ zrel, float4 *__restrict__ u,
                           float4 *__restrict__ xabs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float3 v = f3(vs[i]);
    float3 d = h * v + (h * h) * g;
    if (rf) d = d + 2.f * f3(rf[i]);
    float4 o = f4(d);
    zrel[i] = o;
    u[i] = o;
    xabs[i] = f4(f3(xs[i]) + d);
}

// pinned rows: u = target - x*, absolute position = target (zrel too if given)
__global__ void k_set_pins(const int *__restrict__ pins, int np, const float4 *__restrict__ tgt,
                           const float4 *__restrict__ xs, float4 *__restrict__ zrel, float4 *__restrict__ u,
                           float4 *__restrict__ xabs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    int p = pins[i];
    float4 d = f4(f3(tgt[i]) - f3(xs[p]));
    if (zrel) zrel[p] = d;
    u[p] = d;
    xabs[p] = tgt[i];
}

// Residual forwarding starts from the filtered positions: the base becomes
// x_new (the caller has stored it in xs), z - x* becomes z - x_new (xold is
// the step's x*), the displacement restarts at 0 and xabs = x_new.
__global__ void k_rf_rebase(int n, const float4 *__restrict__ xs, const float4 *__restrict__ xold,
                            float4 *__restrict__ zrel, float4 *__restrict__ u, float4 *__restrict__ xabs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float3 xn = f3(xs[i]);
    zrel[i] = f4(f3(zrel[i]) - (xn - f3(xold[i])));
    u[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    xabs[i] = f4(xn);
}

// u = um (the displacement of x^-), xabs = x* + um
__global__ void k_restart(int n, const float4 *__restrict__ xs, const float4 *__restrict__ um, float4 *__restrict__ u,
                          float4 *__restrict__ xabs) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 d = um[i];
    u[i] = d;
    xabs[i] = f4(f3(xs[i]) + f3(d));
}

// um = s u (cloth part of the filtered x^-), xm = x* + um; s is the vertex's
// instance's fraction when vinst is given (per-instance line search)
__global__ void k_scale_disp(int n, const float4 *__restrict__ xs, const float4 *__restrict__ u, const double *s_frac,
                             float4 *__restrict__ um, float4 *__restrict__ xm, const int *__restrict__ vinst,
                             const double *__restrict__ s_inst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = (float)((vinst && vinst[i] >= 0) ? s_inst[vinst[i]] : *s_frac);
    float3 d = s * f3(u[i]);
    um[i] = f4(d);
    xm[i] = f4(f3(xs[i]) + d);
}

// r_i = m_i/h^2 (z_i - x_i) + sum_t w_t (R_t - F_t) g_{t,i} + sum_h w_h K_{h,i} (s_hat_h - s_h) + cf_i
// The residual in two stages.  Each element computes its projection once and
// writes its force on each of its vertices (stretch: w_t (g_k^T)(R - F) with F
// from exact differences of the rest part and of the displacements; bend:
// w_h K_j (s_hat - s)); each vertex then sums the forces of its incident
// elements in incidence order, adds inertia and contact, and reduces |r|^2.
// One launch for both element kinds: blocks [0, tri_blocks) take triangles,
// the rest hinges.
__device__ inline void tri_corner(const ClothView &c, int t, const float4 *__restrict__ xs,
                                  const float4 *__restrict__ u, float4 *__restrict__ ct) {
    int4 T = c.tri[t];
    float4 g = c.tri_g[t];
    float w = c.tri_w[t];
    float3 p0 = f3(xs[T.x]), p1 = f3(xs[T.y]), p2 = f3(xs[T.z]);
    float3 q0 = f3(u[T.x]), q1 = f3(u[T.y]), q2 = f3(u[T.z]);
    float3 e1 = (p1 - p0) + (q1 - q0), e2 = (p2 - p0) + (q2 - q0);  // (x*_a - x*_b) + (u_a - u_b)
    float3 F1 = g.x * e1 + g.z * e2;  // column 1 of F = [e1 e2] Dm^-1
    float3 F2 = g.y * e1 + g.w * e2;  // column 2
    float3 R1, R2;
    polar32(F1, F2, R1, R2);
    float3 d1 = R1 - F1, d2 = R2 - F2;
    ct[3 * (size_t)t + 0] = f4(w * (-(g.x + g.z) * d1 + -(g.y + g.w) * d2));
    ct[3 * (size_t)t + 1] = f4(w * (g.x * d1 + g.y * d2));
    ct[3 * (size_t)t + 2] = f4(w * (g.z * d1 + g.w * d2));
}

__device__ inline void hinge_corner(const ClothView &c, int h, const float4 *__restrict__ xs,
                                    const float4 *__restrict__ u, float4 *__restrict__ ch) {
    int4 H = c.hin[h];
    float4 K = c.hin_K[h];
    float sl = c.hin_slen[h], hw = c.hin_w[h];
    float3 p0 = f3(xs[H.x]), q0 = f3(u[H.x]);
    float3 d1 = (f3(xs[H.y]) - p0) + (f3(u[H.y]) - q0);
    float3 d2 = (f3(xs[H.z]) - p0) + (f3(u[H.z]) - q0);
    float3 d3 = (f3(xs[H.w]) - p0) + (f3(u[H.w]) - q0);
    float3 sv = K.y * d1 + K.z * d2 + K.w * d3;
    float3 sh;
    float ns = sqrtf(dot3(sv, sv));
    if (sl == 0.f) sh = make_float3(0.f, 0.f, 0.f);
    else if (ns > 1e-30f) sh = (sl / ns) * sv;
    else sh = f3(c.hin_srest[h]);
    float3 d = sh - sv;
    float4 *o = ch + 4 * (size_t)h;
    o[0] = f4((hw * K.x) * d);
    o[1] = f4((hw * K.y) * d);
    o[2] = f4((hw * K.z) * d);
    o[3] = f4((hw * K.w) * d);
}

__global__ void __launch_bounds__(256) k_elem_corner(const ClothView c, int tri_blocks, const float4 *__restrict__ xs,
                                                     const float4 *__restrict__ u, float4 *__restrict__ ct,
                                                     float4 *__restrict__ ch) {
    grid_dep_wait();
    grid_dep_release();
    if (loop_dead(c.live)) return;
    if ((int)blockIdx.x < tri_blocks) {
        int t = blockIdx.x * blockDim.x + threadIdx.x;
        if (t < c.m) tri_corner(c, t, xs, u, ct);
    } else {
        int h = (blockIdx.x - tri_blocks) * blockDim.x + threadIdx.x;
        if (h < c.nh) hinge_corner(c, h, xs, u, ch);
    }
}

__global__ void __launch_bounds__(256) k_residual(const ClothView c, const float4 *__restrict__ u,
                                                  const float4 *__restrict__ zrel, const float *__restrict__ cw,
                                                  const float4 *__restrict__ cf, const float4 *__restrict__ ct,
                                                  const float4 *__restrict__ ch, float4 *__restrict__ r, Scalars *sc,
                                                  float *__restrict__ r_soa, int soa_ld) {
    grid_dep_wait();
    grid_dep_release();
    if (loop_dead(c.live)) return;  // block-uniform: no thread reaches the block reduction
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float sq = 0.f;
    if (i < c.n) {
        float3 f = make_float3(0.f, 0.f, 0.f);
        if (c.is_free[i]) {
            f = c.mh2[i] * (f3(zrel[i]) - f3(u[i]));
            const int tb = c.vt_off[i], te = c.vt_off[i + 1];
#pragma unroll 4
            for (int e = tb; e < te; ++e) {
                int ent = __ldg(c.vt_list + e);
                f = f + f3(ct[3 * (size_t)(ent >> 2) + (ent & 3)]);
            }
            const int hb = c.vh_off[i], he = c.vh_off[i + 1];
#pragma unroll 4
            for (int e = hb; e < he; ++e) {
                int ent = __ldg(c.vh_list + e);
                f = f + f3(ch[4 * (size_t)(ent >> 2) + (ent & 3)]);
            }
            if (cf) f = f + f3(cf[i]);
            sq = dot3(f, f);
        }
        r[i] = f4(f);
        if (r_soa) {
            r_soa[i] = f.x;
            r_soa[soa_ld + i] = f.y;
            r_soa[2 * soa_ld + i] = f.z;
        }
    }
    if (sc) block_add(sq, &sc->rsq);
}

// Two Chebyshev steps in one launch over two-step patch tiles
// (ClothView::ell_halo2).  A block takes one patch; its rows are the patch's
// own vertices and their neighbours (the first ring), its vertices those rows
// and their neighbours.  After staging delta_k of all its vertices it forms
// delta_{k+1} of all its rows (the first-ring rows as their own patches form
// them), then delta_{k+2} of its own rows from those, and writes both for its
// own rows: the next launch reads delta_{k+2} and delta_{k+1}.  Each step is
// k_cheb_step's arithmetic in the same order, so the results are bitwise
// those of two single steps.
template <int W>
__global__ void __launch_bounds__(256) k_cheb_step2_halo(
    const ClothView c, const float *__restrict__ cw, const float4 *__restrict__ r, const float4 *__restrict__ din,
    const float4 *__restrict__ dprev, float4 *__restrict__ dmid, float4 *__restrict__ dout, float a1, float b1,
    float a2, float b2, const float4 *x, float4 *xout, float4 *xprev, float w_acc, const float4 *__restrict__ xs,
    float4 *__restrict__ xabs, Scalars *sc, int *err) {
    extern __shared__ __align__(128) unsigned char h2sm[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_dead;
    const int RW = c.h2_rows, VW = c.h2_verts;
    const uint32_t BYTES = (uint32_t)halo2_tile_bytes(W, RW, VW);
    unsigned char *tile = h2sm;
    float *dk = reinterpret_cast<float *>(h2sm + BYTES);  // [3 * VW] delta_k of the vertices
    float *d1 = dk + 3 * VW;                              // [3 * RW] delta_{k+1} of the rows
    const int t = threadIdx.x;
    if (t == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
        s_dead = loop_dead(c.live) ? 1 : 0;  // final once read as 0 (see k_cheb_step_tile)
    }
    __syncthreads();
    const bool dead_early = s_dead != 0;
    if (t == 0 && !dead_early) {
        mbar_expect_tx(&bar, BYTES);
        bulk_load(tile, c.ell_halo2 + (size_t)blockIdx.x * BYTES, BYTES, &bar);
    }
    grid_dep_wait();
    grid_dep_release();
    if (dead_early) return;  // no copy in flight
    const bool alive = !loop_dead(c.live);
    if (!__syncthreads_and(mbar_wait(&bar, 0))) {  // block-uniform
        if (t == 0) {
            atomicOr(err, PDC_DEVERR_COPY);
            mbar_wait(&bar, 0);  // let the copy land before the block's shared memory is released
        }
        return;
    }
    const int *hd = reinterpret_cast<const int *>(tile);
    const int nown = min(hd[0], ELL_TILE_ROWS), nrows = min(hd[1], RW), nverts = min(hd[2], VW);
    const float *sv = reinterpret_cast<const float *>(tile + 16);
    const short *sd = reinterpret_cast<const short *>(tile + 16 + (size_t)W * RW * 4);
    const int *gid = reinterpret_cast<const int *>(tile + 16 + (size_t)W * RW * 6);
    for (int j = t; j < nverts; j += blockDim.x) {
        const int g = gid[j];
        const float4 v = (alive && g >= 0 && g < c.n) ? din[g] : make_float4(0.f, 0.f, 0.f, 0.f);
        dk[3 * j] = v.x;
        dk[3 * j + 1] = v.y;
        dk[3 * j + 2] = v.z;
    }
    // the block's rows t and t + 256: right-hand side, delta_{k-1}, diagonal
    float3 rr[2], pp[2];
    float DD[2];
    bool fr[2];
    int gi[2];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int j = t + q * ELL_TILE_ROWS;
        gi[q] = j < nrows ? gid[j] : -1;
        fr[q] = alive && gi[q] >= 0 && gi[q] < c.n && c.is_free[gi[q]];
        rr[q] = pp[q] = make_float3(0.f, 0.f, 0.f);
        DD[q] = 1.f;
        if (fr[q]) {
            rr[q] = f3(r[gi[q]]);
            if (a1 != 0.f) pp[q] = f3(dprev[gi[q]]);
            DD[q] = c.hdiag[gi[q]] + (cw ? cw[gi[q]] : 0.f);
        }
    }
    __syncthreads();
    auto V3 = [](const float *a, int j) { return make_float3(a[3 * j], a[3 * j + 1], a[3 * j + 2]); };
    // step k -> k + 1 on every row
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int j = t + q * ELL_TILE_ROWS;
        if (j >= nrows) continue;
        float3 dn = make_float3(0.f, 0.f, 0.f);
        if (fr[q]) {
            const float3 di = V3(dk, j);
            float3 e = make_float3(0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < W; ++k)
                if (k < c.ell_w) e = e + sv[k * RW + j] * V3(dk, sd[k * RW + j]);
            float3 acc = rr[q] - DD[q] * di - e;
            float3 dd = (b1 / DD[q]) * acc;
            if (a1 != 0.f) dd = dd + a1 * (di - pp[q]);
            dn = di + dd;
        }
        d1[3 * j] = dn.x;
        d1[3 * j + 1] = dn.y;
        d1[3 * j + 2] = dn.z;
    }
    __syncthreads();
    // step k + 1 -> k + 2 on the own rows (row t, t < nown; their columns are rows)
    float mx = 0.f;
    if (alive && t < nown && gi[0] >= 0 && gi[0] < c.n) {
        const int i = gi[0];
        const float3 dm = V3(d1, t);
        float3 dn = make_float3(0.f, 0.f, 0.f);
        if (fr[0]) {
            const float3 di = dm, pi = V3(dk, t);
            float3 e = make_float3(0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < W; ++k)
                if (k < c.ell_w) e = e + sv[k * RW + t] * V3(d1, sd[k * RW + t]);
            float3 acc = rr[0] - DD[0] * di - e;
            float3 dd = (b2 / DD[0]) * acc;
            if (a2 != 0.f) dd = dd + a2 * (di - pi);
            dn = di + dd;
        }
        dmid[i] = f4(dm);
        dout[i] = f4(dn);
        if (xout) {
            float3 xo = f3(x[i]);
            float3 xn = xo + dn;
            if (xprev) {
                if (fr[0] && w_acc != 1.f) {
                    float3 xpv = f3(xprev[i]);
                    xn = xpv + w_acc * (xn - xpv);
                }
                xprev[i] = f4(xo);
            }
            xout[i] = f4(xn);
            if (xabs) xabs[i] = f4(f3(xs[i]) + xn);
            float3 d = xn - xo;
            mx = fmaxf(fabsf(d.x), fmaxf(fabsf(d.y), fabsf(d.z)));
        }
    }
    if (xout && sc) block_max(mx, &sc->dxmax);
}

// The same residual in one kernel per mesh patch (ClothView::rp_rec): a
// block stages x* and u of the vertices its patch touches in shared memory,
// computes the projections of the triangles and hinges at its rows once into
// shared memory (a triangle's three corner forces as tri_corner forms them; a
// hinge's vector s_hat - s and its four weights w K_j, whose products are
// hinge_corner's corner forces), and each of its rows then sums its corner
// forces in the order of its incidence lists, as k_residual does; the
// per-corner arrays never go through device memory.
// Elements at a patch border are computed by every patch they touch.  512
// threads a block, four blocks an SM at 54 KB of shared memory (512 x 512
// sheet): the element phase has about three elements per thread.
__device__ __forceinline__ const unsigned char *align16(const unsigned char *p, size_t bytes) {
    return p + ((bytes + 15) & ~(size_t)15);
}

__global__ void __launch_bounds__(512) k_residual_patch(const ClothView c, const float4 *__restrict__ xs,
                                                        const float4 *__restrict__ u,
                                                        const float4 *__restrict__ zrel,
                                                        const float *__restrict__ cw, const float4 *__restrict__ cf,
                                                        float4 *__restrict__ r, Scalars *sc,
                                                        float *__restrict__ r_soa, int soa_ld) {
    extern __shared__ float rp_sm[];
    grid_dep_wait();
    grid_dep_release();
    if (loop_dead(c.live)) return;  // block-uniform: no thread reaches the block reduction
    const int t = threadIdx.x;
    const unsigned char *p = c.rp_rec + c.rp_off[blockIdx.x];
    const int4 hd = *reinterpret_cast<const int4 *>(p);
    const int nloc = hd.x, ntri = hd.y, nhin = hd.z, nown = hd.w;
    const int *vid = reinterpret_cast<const int *>(align16(p, 16));
    const int *tg = reinterpret_cast<const int *>(align16(reinterpret_cast<const unsigned char *>(vid), 4 * (size_t)nloc));
    const int2 *tl = reinterpret_cast<const int2 *>(align16(reinterpret_cast<const unsigned char *>(tg), 4 * (size_t)ntri));
    const int *hg = reinterpret_cast<const int *>(align16(reinterpret_cast<const unsigned char *>(tl), 8 * (size_t)ntri));
    const int2 *hl = reinterpret_cast<const int2 *>(align16(reinterpret_cast<const unsigned char *>(hg), 4 * (size_t)nhin));
    const int *vto = reinterpret_cast<const int *>(align16(reinterpret_cast<const unsigned char *>(hl), 8 * (size_t)nhin));
    const int *vte = reinterpret_cast<const int *>(align16(reinterpret_cast<const unsigned char *>(vto), 4 * (size_t)(nown + 1)));
    const int *vho = reinterpret_cast<const int *>(align16(reinterpret_cast<const unsigned char *>(vte), 4 * (size_t)__ldg(vto + nown)));
    const int *vhe = reinterpret_cast<const int *>(align16(reinterpret_cast<const unsigned char *>(vho), 4 * (size_t)(nown + 1)));
    float *px = rp_sm;                     // [3 * rp_loc] x*
    float *pu = px + 3 * c.rp_loc;         // [3 * rp_loc] u
    float *td = pu + 3 * c.rp_loc;         // [9 * rp_tri] triangle corner forces
    float *hv = td + 9 * c.rp_tri;         // [7 * rp_hin] hinge: s_hat - s, then w K_j (j = 0..3)
    for (int j = t; j < nloc; j += blockDim.x) {
        const int g = __ldg(vid + j);
        const float4 a = xs[g], b = u[g];
        px[3 * j] = a.x;
        px[3 * j + 1] = a.y;
        px[3 * j + 2] = a.z;
        pu[3 * j] = b.x;
        pu[3 * j + 1] = b.y;
        pu[3 * j + 2] = b.z;
    }
    __syncthreads();
    auto P3 = [&](const float *q, int j) { return make_float3(q[3 * j], q[3 * j + 1], q[3 * j + 2]); };
    auto put3 = [&](float *o, float3 v) {
        o[0] = v.x;
        o[1] = v.y;
        o[2] = v.z;
    };
    for (int e = t; e < ntri; e += blockDim.x) {  // as tri_corner
        const float w = c.tri_w[__ldg(tg + e)];
        const int gt = __ldg(tg + e);
        const int2 L = __ldg(tl + e);
        const int a = L.x & 0xffff, b = L.x >> 16, cc = L.y;
        const float4 g = c.tri_g[gt];
        const float3 p0 = P3(px, a), p1 = P3(px, b), p2 = P3(px, cc);
        const float3 q0 = P3(pu, a), q1 = P3(pu, b), q2 = P3(pu, cc);
        float3 e1 = (p1 - p0) + (q1 - q0), e2 = (p2 - p0) + (q2 - q0);
        float3 F1 = g.x * e1 + g.z * e2;
        float3 F2 = g.y * e1 + g.w * e2;
        float3 R1, R2;
        polar32(F1, F2, R1, R2);
        const float3 d1 = R1 - F1, d2 = R2 - F2;
        float *o = td + 9 * e;
        put3(o, w * (-(g.x + g.z) * d1 + -(g.y + g.w) * d2));
        put3(o + 3, w * (g.x * d1 + g.y * d2));
        put3(o + 6, w * (g.z * d1 + g.w * d2));
    }
    for (int e = t; e < nhin; e += blockDim.x) {  // as hinge_corner
        const int gh = __ldg(hg + e);
        const int2 L = __ldg(hl + e);
        const int a = L.x & 0xffff, b = L.x >> 16, cc = L.y & 0xffff, dd = L.y >> 16;
        const float4 K = c.hin_K[gh];
        const float sl = c.hin_slen[gh];
        const float3 p0 = P3(px, a), q0 = P3(pu, a);
        const float3 d1 = (P3(px, b) - p0) + (P3(pu, b) - q0);
        const float3 d2 = (P3(px, cc) - p0) + (P3(pu, cc) - q0);
        const float3 d3 = (P3(px, dd) - p0) + (P3(pu, dd) - q0);
        const float3 sv = K.y * d1 + K.z * d2 + K.w * d3;
        float3 sh;
        const float ns = sqrtf(dot3(sv, sv));
        if (sl == 0.f) sh = make_float3(0.f, 0.f, 0.f);
        else if (ns > 1e-30f) sh = (sl / ns) * sv;
        else sh = f3(c.hin_srest[gh]);
        const float3 d = sh - sv;
        const float hw = c.hin_w[gh];
        float *o = hv + 7 * e;  // corner j = (w K_j) d, formed in the gather
        put3(o, d);
        o[3] = hw * K.x;
        o[4] = hw * K.y;
        o[5] = hw * K.z;
        o[6] = hw * K.w;
    }
    __syncthreads();
    float sq = 0.f;
    if (t < nown) {
        const int i = __ldg(vid + t);
        float3 f = make_float3(0.f, 0.f, 0.f);
        if (c.is_free[i]) {
            f = c.mh2[i] * (f3(zrel[i]) - P3(pu, t));
            const int tb = __ldg(vto + t), te = __ldg(vto + t + 1);
#pragma unroll 4
            for (int k = tb; k < te; ++k) {
                const int ent = __ldg(vte + k);
                f = f + P3(td, 3 * (ent >> 2) + (ent & 3));
            }
            const int hb = __ldg(vho + t), he = __ldg(vho + t + 1);
#pragma unroll 4
            for (int k = hb; k < he; ++k) {
                const int ent = __ldg(vhe + k);
                const float *o = hv + 7 * (ent >> 2);
                f = f + o[3 + (ent & 3)] * make_float3(o[0], o[1], o[2]);
            }
            if (cf) f = f + f3(cf[i]);
            sq = dot3(f, f);
        }
        r[i] = f4(f);
        if (r_soa) {
            r_soa[i] = f.x;
            r_soa[soa_ld + i] = f.y;
            r_soa[2 * soa_ld + i] = f.z;
        }
    }
    if (sc) block_add(sq, &sc->rsq);
}

// sum_k H_ik delta_k over the ELL off-diagonals of row i; with WMAX > 0 (a
// compile-time bound on the row width) the loop is unrolled so that the
// loads of all entries are in flight together.
template <int WMAX>
__device__ inline float3 ell_apply(const ClothView &c, int i, const float4 *__restrict__ v) {
    float3 acc = make_float3(0.f, 0.f, 0.f);
    const int *col = c.ell_col + i;
    const float *val = c.ell_val + i;
    if constexpr (WMAX > 0) {
        if (c.ell_dcol) {  // 16-bit offsets: 6 instead of 8 bytes per entry
            const short *dc = c.ell_dcol + i;
#pragma unroll
            for (int k = 0; k < WMAX; ++k)
                if (k < c.ell_w) acc = acc + __ldg(val + (size_t)k * c.n) * f3(v[i + (int)__ldg(dc + (size_t)k * c.n)]);
        } else {
#pragma unroll
            for (int k = 0; k < WMAX; ++k)
                if (k < c.ell_w) acc = acc + __ldg(val + (size_t)k * c.n) * f3(v[__ldg(col + (size_t)k * c.n)]);
        }
    } else {
        for (int k = 0; k < c.ell_w; ++k) acc = acc + val[(size_t)k * c.n] * f3(v[col[(size_t)k * c.n]]);
    }
    return acc;
}

// One damped Jacobi sweep on (H + diag(cw)) delta = r:
//   delta'_i = (1 - omega) delta_i + omega (r_i - sum_{j != i} H_ij delta_j) / (H_ii + cw_i)
// If xout is given, also writes the new iterate and reduces max |x_new - x|:
//   x_new = x + delta'                                   (xprev == NULL), or
//   x_new = w (x + delta' - xprev) + xprev, xprev <- x   (Chebyshev step, weight w)
template <int WMAX>
__global__ void __launch_bounds__(256) k_sweep(const ClothView c, const float *__restrict__ cw,
                                               const float4 *__restrict__ r, const float4 *__restrict__ din,
                                               float4 *__restrict__ dout, float omega,
                                               const float4 *x, float4 *xout, float4 *xprev, float w_acc,
                                               const float4 *__restrict__ xs, float4 *__restrict__ xabs,
                                               Scalars *sc) {
    if (loop_dead(c.live)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float mx = 0.f;
    if (i < c.n) {
        float3 dn = make_float3(0.f, 0.f, 0.f);
        if (c.is_free[i]) {
            float3 acc = f3(r[i]) - ell_apply<WMAX>(c, i, din);
            float D = c.hdiag[i] + (cw ? cw[i] : 0.f);
            float3 di = f3(din[i]);
            dn = (1.f - omega) * di + (omega / D) * acc;
        }
        dout[i] = f4(dn);
        if (xout) {
            float3 xo = f3(x[i]);
            float3 xn = xo + dn;
            if (xprev) {
                if (c.is_free[i] && w_acc != 1.f) {
                    float3 xp = f3(xprev[i]);
                    xn = xp + w_acc * (xn - xp);
                }
                xprev[i] = f4(xo);
            }
            xout[i] = f4(xn);
            if (xabs) xabs[i] = f4(f3(xs[i]) + xn);
            float3 d = xn - xo;
            mx = fmaxf(fabsf(d.x), fmaxf(fabsf(d.y), fabsf(d.z)));
        }
    }
    if (xout && sc) block_max(mx, &sc->dxmax);
}

// One step of the Jacobi-preconditioned Chebyshev iteration on
// (H + diag(cw)) delta = r:
//   d'     = alpha d + beta D^-1 (r - (H + diag(cw)) delta)
//   delta' = delta + d'
// (alpha, beta from the Chebyshev recurrence for the interval [a, b] of the
// spectrum of D^-1 (H + diag cw)).  The last step also writes the iterate as
// k_sweep does.
//
// Launched as a programmatic dependent (launch_overlap), a block may start
// while the previous kernel is still running: it waits for that kernel's
// completion (and memory) before its first load or store, then releases the
// next launch.  Launched plainly, the wait returns at once.
template <int WMAX>
__global__ void __launch_bounds__(256) k_cheb_step(const ClothView c, const float *__restrict__ cw,
                                                   const float4 *__restrict__ r, const float4 *__restrict__ din,
                                                   const float4 *__restrict__ dprev, float4 *__restrict__ dout,
                                                   float alpha, float beta,
                                                   const float4 *x, float4 *xout, float4 *xprev, float w_acc,
                                                   const float4 *__restrict__ xs, float4 *__restrict__ xabs,
                                                   Scalars *sc) {
    grid_dep_wait();
    grid_dep_release();
    if (loop_dead(c.live)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float mx = 0.f;
    if (i < c.n) {
        float3 dn = make_float3(0.f, 0.f, 0.f);
        if (c.is_free[i]) {
            float3 di = f3(din[i]);
            float D = c.hdiag[i] + (cw ? cw[i] : 0.f);
            float3 acc = f3(r[i]) - D * di - ell_apply<WMAX>(c, i, din);
            float3 dd = (beta / D) * acc;
            if (alpha != 0.f) dd = dd + alpha * (di - f3(dprev[i]));  // alpha (delta_k - delta_k-1)
            dn = di + dd;
        }
        dout[i] = f4(dn);
        if (xout) {
            float3 xo = f3(x[i]);
            float3 xn = xo + dn;
            if (xprev) {
                if (c.is_free[i] && w_acc != 1.f) {
                    float3 xp = f3(xprev[i]);
                    xn = xp + w_acc * (xn - xp);
                }
                xprev[i] = f4(xo);
            }
            xout[i] = f4(xn);
            if (xabs) xabs[i] = f4(f3(xs[i]) + xn);
            float3 d = xn - xo;
            mx = fmaxf(fabsf(d.x), fmaxf(fabsf(d.y), fabsf(d.z)));
        }
    }
    if (xout && sc) block_max(mx, &sc->dxmax);
}

// The Chebyshev step with the row's off-diagonals taken from its block's
// ELL tile, which one thread brings into shared memory with a bulk copy
// before the block waits on the previous kernel: the matrix never changes
// during a step, so its fetch overlaps the previous kernel's tail, and only
// the vertex streams are read after the wait.  Same arithmetic, in the same
// order, as k_cheb_step.
template <int W>
__global__ void __launch_bounds__(ELL_TILE_ROWS, 8) k_cheb_step_tile(
    const ClothView c, const float *__restrict__ cw, const float4 *__restrict__ r, const float4 *__restrict__ din,
    const float4 *__restrict__ dprev, float4 *__restrict__ dout, float alpha, float beta, const float4 *x,
    float4 *xout, float4 *xprev, float w_acc, const float4 *__restrict__ xs, float4 *__restrict__ xabs, Scalars *sc,
    int *err) {
    constexpr uint32_t BYTES = (uint32_t)W * ELL_TILE_ROWS * 6;
    __shared__ __align__(128) unsigned char tile[BYTES];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_dead;
    const int t = threadIdx.x;
    if (t == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
        // a device loop's flag only ever goes from 1 to 0 within the loop, so
        // an early read of 0 is final: the step of an iteration enqueued past
        // the loop's end issues no tile copy
        s_dead = loop_dead(c.live) ? 1 : 0;
    }
    __syncthreads();
    const bool dead_early = s_dead != 0;
    if (t == 0 && !dead_early) {
        mbar_expect_tx(&bar, BYTES);
        bulk_load(tile, c.ell_tile + (size_t)blockIdx.x * BYTES, BYTES, &bar);
    }
    grid_dep_wait();
    grid_dep_release();
    if (dead_early) return;  // no copy in flight
    const int i = blockIdx.x * ELL_TILE_ROWS + t;
    float mx = 0.f;
    // an ended device loop: no load or store, but the tile copy is still awaited
    const bool live = i < c.n && !loop_dead(c.live);
    const bool fr = live && c.is_free[i];
    float3 di = make_float3(0.f, 0.f, 0.f), ri = di, pi = di;
    float D = 1.f;
    if (fr) {
        di = f3(din[i]);
        ri = f3(r[i]);
        if (alpha != 0.f) pi = f3(dprev[i]);
        D = c.hdiag[i] + (cw ? cw[i] : 0.f);
    }
    if (!__syncthreads_and(mbar_wait(&bar, 0))) {  // block-uniform: the reduction below syncs
        if (t == 0) {
            atomicOr(err, PDC_DEVERR_COPY);
            mbar_wait(&bar, 0);  // let the copy land before the block's shared memory is released
        }
        return;
    }
    if (live) {
        float3 dn = make_float3(0.f, 0.f, 0.f);
        if (fr) {
            const float *sv = reinterpret_cast<const float *>(tile);
            const short *sd = reinterpret_cast<const short *>(tile + (size_t)W * ELL_TILE_ROWS * 4);
            float3 e = make_float3(0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < W; ++k)
                if (k < c.ell_w) e = e + sv[k * ELL_TILE_ROWS + t] * f3(din[i + (int)sd[k * ELL_TILE_ROWS + t]]);
            float3 acc = ri - D * di - e;
            float3 dd = (beta / D) * acc;
            if (alpha != 0.f) dd = dd + alpha * (di - pi);
            dn = di + dd;
        }
        dout[i] = f4(dn);
        if (xout) {
            float3 xo = f3(x[i]);
            float3 xn = xo + dn;
            if (xprev) {
                if (fr && w_acc != 1.f) {
                    float3 xp = f3(xprev[i]);
                    xn = xp + w_acc * (xn - xp);
                }
                xprev[i] = f4(xo);
            }
            xout[i] = f4(xn);
            if (xabs) xabs[i] = f4(f3(xs[i]) + xn);
            float3 d = xn - xo;
            mx = fmaxf(fabsf(d.x), fmaxf(fabsf(d.y), fabsf(d.z)));
        }
    }
    if (xout && sc) block_max(mx, &sc->dxmax);
}

// The Chebyshev step over patch tiles (ClothView::ell_halo): a block takes
// one patch of ELL_TILE_ROWS rows that are close on the rest mesh, so the
// vertices its rows reference are its own rows plus a thin halo.  One thread
// bulk-copies the patch's tile (values, local columns, vertex ids of rows and
// halo) before the dependency wait; after it the block stages delta of its
// rows and halo in shared memory once, and every neighbour term reads it from
// there instead of gathering from global memory.  Same arithmetic, in the
// same order, as k_cheb_step.
template <int W>
__global__ void __launch_bounds__(ELL_TILE_ROWS, 4) k_cheb_step_halo(
    const ClothView c, const float *__restrict__ cw, const float4 *__restrict__ r, const float4 *__restrict__ din,
    const float4 *__restrict__ dprev, float4 *__restrict__ dout, float alpha, float beta, const float4 *x,
    float4 *xout, float4 *xprev, float w_acc, const float4 *__restrict__ xs, float4 *__restrict__ xabs, Scalars *sc,
    int *err) {
    // the copy takes values, columns and row ids; the halo ids are read from
    // global memory by the threads that stage them
    constexpr uint32_t BYTES = (uint32_t)((size_t)W * ELL_TILE_ROWS * 6 + (size_t)ELL_TILE_ROWS * 4);
    constexpr int R = ELL_TILE_ROWS;
    __shared__ __align__(128) unsigned char tile[BYTES];
    __shared__ float dsh[3 * (R + HALO_MAX)];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_dead;
    const int t = threadIdx.x;
    if (t == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
        s_dead = loop_dead(c.live) ? 1 : 0;  // final once read as 0 (see k_cheb_step_tile)
    }
    __syncthreads();
    const bool dead_early = s_dead != 0;
    if (t == 0 && !dead_early) {
        mbar_expect_tx(&bar, BYTES);
        bulk_load(tile, c.ell_halo + (size_t)blockIdx.x * halo_tile_bytes(W), BYTES, &bar);
    }
    grid_dep_wait();
    grid_dep_release();
    if (dead_early) return;  // no copy in flight
    const bool alive = !loop_dead(c.live);
    if (!__syncthreads_and(mbar_wait(&bar, 0))) {  // block-uniform
        if (t == 0) {
            atomicOr(err, PDC_DEVERR_COPY);
            mbar_wait(&bar, 0);  // let the copy land before the block's shared memory is released
        }
        return;
    }
    const int *gid = reinterpret_cast<const int *>(tile + (size_t)W * R * 6);
    const int *hid = reinterpret_cast<const int *>(c.ell_halo + (size_t)blockIdx.x * halo_tile_bytes(W) +
                                                   (size_t)W * R * 6) + R;
    const int nh = min(__ldg(hid + HALO_MAX), HALO_MAX);
    const int i = gid[t];
    // delta of the rows and the halo, once per block
    for (int j = t; j < R + nh; j += R) {
        const int g = j < R ? gid[j] : __ldg(hid + (j - R));
        const float4 v = (alive && g >= 0 && g < c.n) ? din[g] : make_float4(0.f, 0.f, 0.f, 0.f);
        dsh[3 * j] = v.x;
        dsh[3 * j + 1] = v.y;
        dsh[3 * j + 2] = v.z;
    }
    const bool live = alive && i >= 0 && i < c.n;
    const bool fr = live && c.is_free[i];
    float3 ri = make_float3(0.f, 0.f, 0.f), pi = ri;
    float D = 1.f;
    if (fr) {
        ri = f3(r[i]);
        if (alpha != 0.f) pi = f3(dprev[i]);
        D = c.hdiag[i] + (cw ? cw[i] : 0.f);
    }
    __syncthreads();
    float mx = 0.f;
    if (live) {
        float3 dn = make_float3(0.f, 0.f, 0.f);
        if (fr) {
            const float *sv = reinterpret_cast<const float *>(tile);
            const short *sd = reinterpret_cast<const short *>(tile + (size_t)W * R * 4);
            const float3 di = make_float3(dsh[3 * t], dsh[3 * t + 1], dsh[3 * t + 2]);
            float3 e = make_float3(0.f, 0.f, 0.f);
#pragma unroll
            for (int k = 0; k < W; ++k)
                if (k < c.ell_w) {
                    const int j = sd[k * R + t];
                    e = e + sv[k * R + t] * make_float3(dsh[3 * j], dsh[3 * j + 1], dsh[3 * j + 2]);
                }
            float3 acc = ri - D * di - e;
            float3 dd = (beta / D) * acc;
            if (alpha != 0.f) dd = dd + alpha * (di - pi);
            dn = di + dd;
        }
        dout[i] = f4(dn);
        if (xout) {
            float3 xo = f3(x[i]);
            float3 xn = xo + dn;
            if (xprev) {
                if (fr && w_acc != 1.f) {
                    float3 xp = f3(xprev[i]);
                    xn = xp + w_acc * (xn - xp);
                }
                xprev[i] = f4(xo);
            }
            xout[i] = f4(xn);
            if (xabs) xabs[i] = f4(f3(xs[i]) + xn);
            float3 d = xn - xo;
            mx = fmaxf(fabsf(d.x), fmaxf(fabsf(d.y), fabsf(d.z)));
        }
    }
    if (xout && sc) block_max(mx, &sc->dxmax);
}

// Anderson mixing of the LG fixed-point map x -> G(x) = x + delta(x)
// (history of depth m): with f_k = delta_k, g_k = x_k + delta_k and the
// differences dF_j, dG_j of consecutive f and g, theta minimises
// |f_k - dF theta| and x_{k+1} = g_k - dG theta.
constexpr int AA_MAX = 8;

// Inserts the newest differences (if a previous iterate exists) into slot
// `slot`, stores f_k, g_k, and accumulates the normal equations
// G_jl = dF_j . dF_l, b_j = dF_j . f_k over the ncol valid columns.
__global__ void __launch_bounds__(256) k_aa_gram(int n, const unsigned char *__restrict__ is_free,
                                                 const float4 *__restrict__ delta, const float4 *__restrict__ xhat,
                                                 float4 *__restrict__ fprev, float4 *__restrict__ gprev,
                                                 float4 *__restrict__ dF, float4 *__restrict__ dG, int slot,
                                                 int have_prev, int ncol, double *__restrict__ Gb,
                                                 const LoopCtl *ctl) {
    __shared__ float red[AA_MAX * (AA_MAX + 3) / 2 + AA_MAX][8];
    grid_dep_wait();
    grid_dep_release();
    if (ctl && !ctl->go) return;  // the device loop has ended
    if (ctl) {  // bookkeeping taken on the device
        slot = ctl->aa_slot;
        have_prev = ctl->aa_prev;
        ncol = ctl->aa_ncol;
    }
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float3 col[AA_MAX];
    float3 fk = make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int j = 0; j < AA_MAX; ++j) col[j] = make_float3(0.f, 0.f, 0.f);
    if (i < n && is_free[i]) {
        fk = f3(delta[i]);
        float3 gk = f3(xhat[i]);
        float3 df = make_float3(0.f, 0.f, 0.f);
        if (have_prev) {
            df = fk - f3(fprev[i]);
            float3 dg = gk - f3(gprev[i]);
            dF[(size_t)slot * n + i] = f4(df);
            dG[(size_t)slot * n + i] = f4(dg);
        }
        fprev[i] = f4(fk);
        gprev[i] = f4(gk);
#pragma unroll
        for (int j = 0; j < AA_MAX; ++j)
            if (j < ncol) col[j] = (have_prev && j == slot) ? df : f3(dF[(size_t)j * n + i]);
    } else if (i < n) {
        fprev[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        gprev[i] = xhat[i];
    }
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int e = 0;
    for (int j = 0; j < ncol; ++j) {
        for (int l = j; l < ncol; ++l) {
            float v = dot3(col[j], col[l]);
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[e][w] = v;
            ++e;
        }
        float v = dot3(col[j], fk);
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[e][w] = v;
        ++e;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < e; q += blockDim.x) {
        float t = 0.f;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[q][k];
        if (t != 0.f) atomicAdd(&Gb[q], (double)t);
    }
}

// theta solving the (regularised) normal equations of the mixing
// least-squares problem by Cholesky (one thread, FP64); M (= the column
// count) is a template parameter so the tiny system lives in registers.
template <int M>
__device__ inline void aa_solve(const double *__restrict__ Gb, float *__restrict__ theta) {
    double A[M][M], b[M];
    int e = 0;
    double tr = 0.0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
#pragma unroll
        for (int l = j; l < M; ++l) A[j][l] = A[l][j] = Gb[e + l - j];
        e += M - j;
        b[j] = Gb[e++];
        tr += A[j][j];
    }
#pragma unroll
    for (int j = 0; j < M; ++j) A[j][j] += 1e-10 * tr + 1e-300;
    bool ok = tr > 0.0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        double d = A[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= A[j][k] * A[j][k];
        ok = ok && d > 0.0;
        d = sqrt(fmax(d, 1e-300));
        A[j][j] = d;
        double inv = 1.0 / d;
#pragma unroll
        for (int q = j + 1; q < M; ++q) {
            double v = A[q][j];
#pragma unroll
            for (int k = 0; k < j; ++k) v -= A[q][k] * A[j][k];
            A[q][j] = v * inv;
        }
    }
    double y[M], x[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        double v = b[j];
#pragma unroll
        for (int k = 0; k < j; ++k) v -= A[j][k] * y[k];
        y[j] = v / A[j][j];
    }
#pragma unroll
    for (int j = M - 1; j >= 0; --j) {
        double v = y[j];
#pragma unroll
        for (int k = j + 1; k < M; ++k) v -= A[k][j] * x[k];
        x[j] = v / A[j][j];
    }
#pragma unroll
    for (int j = 0; j < AA_MAX; ++j) theta[j] = (j < M && ok && isfinite(x[j < M ? j : 0])) ? (float)x[j < M ? j : 0] : 0.f;
}

// One thread solves the M x M system (a kernel of its own: inside the mixing
// kernel its FP64 registers would cut that kernel's occupancy).
template <int M> __global__ void k_aa_solve(const double *__restrict__ Gb, float *__restrict__ theta) {
    grid_dep_wait();
    grid_dep_release();
    if (threadIdx.x == 0 && blockIdx.x == 0) aa_solve<M>(Gb, theta);
}

// The same solve for a column count ncol <= M read on the device: the
// ncol x ncol system in the leading block of an M x M one whose other rows
// and columns are the identity (theta = 0 there).  The leading block's
// arithmetic is that of aa_solve<ncol> step for step, so theta is the same.
template <int M> __device__ inline void aa_solve_rt(const double *__restrict__ Gb, float *__restrict__ theta, int ncol) {
    double A[M][M], b[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        b[j] = 0.0;
#pragma unroll
        for (int l = 0; l < M; ++l) A[j][l] = j == l ? 1.0 : 0.0;
    }
    int e = 0;
    double tr = 0.0;
    for (int j = 0; j < ncol; ++j) {
        for (int l = j; l < ncol; ++l) A[j][l] = A[l][j] = Gb[e + l - j];
        e += ncol - j;
        b[j] = Gb[e++];
        tr += A[j][j];
    }
    for (int j = 0; j < ncol; ++j) A[j][j] += 1e-10 * tr + 1e-300;
    bool ok = tr > 0.0;
#pragma unroll
    for (int j = 0; j < M; ++j) {
        double d = A[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= A[j][k] * A[j][k];
        ok = ok && d > 0.0;
        d = sqrt(fmax(d, 1e-300));
        A[j][j] = d;
        double inv = 1.0 / d;
#pragma unroll
        for (int q = j + 1; q < M; ++q) {
            double v = A[q][j];
#pragma unroll
            for (int k = 0; k < j; ++k) v -= A[q][k] * A[j][k];
            A[q][j] = v * inv;
        }
    }
    double y[M], x[M];
#pragma unroll
    for (int j = 0; j < M; ++j) {
        double v = b[j];
#pragma unroll
        for (int k = 0; k < j; ++k) v -= A[j][k] * y[k];
        y[j] = v / A[j][j];
    }
#pragma unroll
    for (int j = M - 1; j >= 0; --j) {
        double v = y[j];
#pragma unroll
        for (int k = j + 1; k < M; ++k) v -= A[k][j] * x[k];
        x[j] = v / A[j][j];
    }
#pragma unroll
    for (int j = 0; j < AA_MAX; ++j)
        theta[j] = (j < ncol && j < M && ok && isfinite(x[j < M ? j : 0])) ? (float)x[j < M ? j : 0] : 0.f;
}

template <int M> __global__ void k_aa_solve_dev(const double *__restrict__ Gb, float *__restrict__ theta,
                                                const LoopCtl *ctl) {
    grid_dep_wait();
    grid_dep_release();
    if (!ctl->go) return;
    if (threadIdx.x == 0 && blockIdx.x == 0) aa_solve_rt<M>(Gb, theta, min(ctl->aa_ncol, M));
}

// x_{k+1} = g_k - sum_j theta_j dG_j over the ncol columns of the device state.
__global__ void __launch_bounds__(256) k_aa_mix_dev(int n, const unsigned char *__restrict__ is_free,
                                                    const float4 *__restrict__ xhat, const float4 *__restrict__ dG,
                                                    const float *__restrict__ theta, float4 *__restrict__ xout,
                                                    const float4 *__restrict__ xs, float4 *__restrict__ xabs,
                                                    const LoopCtl *ctl, int m) {
    grid_dep_wait();
    grid_dep_release();
    if (!ctl->go) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int ncol = min(ctl->aa_ncol, m);
    float3 x = f3(xhat[i]);
    if (is_free[i])
        for (int j = 0; j < ncol; ++j) x = x - theta[j] * f3(dG[(size_t)j * n + i]);
    xout[i] = f4(x);
    if (xabs) xabs[i] = f4(f3(xs[i]) + x);
}

// x_{k+1} = g_k - sum_j theta_j dG_j on free vertices.
template <int M>
__global__ void __launch_bounds__(256) k_aa_mix(int n, const unsigned char *__restrict__ is_free,
                                                const float4 *__restrict__ xhat, const float4 *__restrict__ dG,
                                                const float *__restrict__ theta, float4 *__restrict__ xout,
                                                const float4 *__restrict__ xs, float4 *__restrict__ xabs) {
    grid_dep_wait();
    grid_dep_release();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float3 x = f3(xhat[i]);
    if (is_free[i])
#pragma unroll
        for (int j = 0; j < M; ++j) x = x - theta[j] * f3(dG[(size_t)j * n + i]);
    xout[i] = f4(x);
    if (xabs) xabs[i] = f4(f3(xs[i]) + x);
}

__global__ void k_lerp(int nv, const float4 *__restrict__ a, const float4 *__restrict__ b, const double *s_frac,
                       float4 *__restrict__ out, const int *__restrict__ vinst, const double *__restrict__ s_inst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    float s = (float)((vinst && vinst[i] >= 0) ? s_inst[vinst[i]] : *s_frac);
    float3 p = f3(a[i]), q = f3(b[i]);
    out[i] = f4(p + s * (q - p));
}


inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

}  // namespace

void launch_prologue(cudaStream_t s, int n, const float4 *xs, const float4 *vs, const int *pins, const float4 *pin_tgt,
                     int npins, float h, float3 g, float4 *zrel, float4 *u, float4 *xabs, const float4 *rf) {
    if (n > 0) k_prologue<<<nblk(n, 256), 256, 0, s>>>(n, xs, vs, h, g, rf, zrel, u, xabs);
    PDC_LAUNCH_CK();
    if (npins > 0) {
        k_set_pins<<<nblk(npins, 256), 256, 0, s>>>(pins, npins, pin_tgt, xs, zrel, u, xabs);
        PDC_LAUNCH_CK();
    }
}

void launch_rf_rebase(cudaStream_t s, int n, const float4 *xs, const float4 *xold, float4 *zrel, float4 *u,
                      float4 *xabs) {
    if (n > 0) k_rf_rebase<<<nblk(n, 256), 256, 0, s>>>(n, xs, xold, zrel, u, xabs);
    PDC_LAUNCH_CK();
}

void launch_set_pins(cudaStream_t s, const int *pins, int npins, const float4 *tgt, const float4 *xs, float4 *u,
                     float4 *xabs) {
    if (npins > 0) k_set_pins<<<nblk(npins, 256), 256, 0, s>>>(pins, npins, tgt, xs, nullptr, u, xabs);
    PDC_LAUNCH_CK();
}

void launch_restart(cudaStream_t s, int n, const float4 *xs, const float4 *um, float4 *u, float4 *xabs) {
    if (n > 0) k_restart<<<nblk(n, 256), 256, 0, s>>>(n, xs, um, u, xabs);
    PDC_LAUNCH_CK();
}

void launch_scale_disp(cudaStream_t s, int n, const float4 *xs, const float4 *u, const double *s_frac, float4 *um,
                       float4 *xm, const int *vinst, const double *s_inst) {
    if (n > 0) k_scale_disp<<<nblk(n, 256), 256, 0, s>>>(n, xs, u, s_frac, um, xm, vinst, s_inst);
    PDC_LAUNCH_CK();
}

void launch_residual(cudaStream_t s, const ClothView &c, const float4 *xs, const float4 *u, const float4 *zrel,
                     const float *cw, const float4 *cf, float4 *r, Scalars *sc, float *r_soa, int soa_ld) {
    if (c.rp_rec && c.n > 0) {
        const size_t smem = 4 * (6 * (size_t)c.rp_loc + 9 * (size_t)c.rp_tri + 7 * (size_t)c.rp_hin);
        static unsigned long long attr = 0;  // per-device bits: the shared-memory limit raised
        int dev = 0;
        PDC_CK(cudaGetDevice(&dev));
        if (!(attr >> (dev & 63) & 1ull)) {
            PDC_CK(cudaFuncSetAttribute(k_residual_patch, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
            attr |= 1ull << (dev & 63);
        }
        launch_dependent(c.overlap != 0, k_residual_patch, nblk(c.n, ELL_TILE_ROWS), 512, smem, s, c, xs, u, zrel, cw,
                         cf, r, sc, r_soa, soa_ld);
        PDC_LAUNCH_CK();
        return;
    }
    float4 *ct = c.corner, *ch = c.corner + 3 * (size_t)c.m;
    const int bs = (c.res_block == 64 || c.res_block == 128) ? c.res_block : 256;
    const int tb = nblk(c.m, bs), hb = nblk(c.nh, bs);
    if (tb + hb > 0) launch_dependent(c.overlap != 0, k_elem_corner, tb + hb, bs, 0, s, c, tb, xs, u, ct, ch);
    if (c.n > 0)
        launch_dependent(c.overlap != 0, k_residual, nblk(c.n, bs), bs, 0, s, c, u, zrel, cw, cf, ct, ch, r, sc,
                         r_soa, soa_ld);
    PDC_LAUNCH_CK();
}

void launch_sweep(cudaStream_t s, const ClothView &c, const float *cw, const float4 *r, const float4 *din,
                  float4 *dout, float omega, const float4 *x, float4 *xout, Scalars *sc, float4 *xprev,
                  float w_acc, const float4 *xs, float4 *xabs) {
    if (c.n > 0) {
        int b = nblk(c.n, 256);
        if (c.ell_w <= 8) k_sweep<8><<<b, 256, 0, s>>>(c, cw, r, din, dout, omega, x, xout, xprev, w_acc, xs, xabs, sc);
        else if (c.ell_w <= 12)
            k_sweep<12><<<b, 256, 0, s>>>(c, cw, r, din, dout, omega, x, xout, xprev, w_acc, xs, xabs, sc);
        else if (c.ell_w <= 16)
            k_sweep<16><<<b, 256, 0, s>>>(c, cw, r, din, dout, omega, x, xout, xprev, w_acc, xs, xabs, sc);
        else k_sweep<0><<<b, 256, 0, s>>>(c, cw, r, din, dout, omega, x, xout, xprev, w_acc, xs, xabs, sc);
    }
    PDC_LAUNCH_CK();
}

void launch_cheb_step(cudaStream_t s, const ClothView &c, const float *cw, const float4 *r, const float4 *din,
                      const float4 *dprev, float4 *dout, float alpha, float beta, const float4 *x,
                      float4 *xout, Scalars *sc, float4 *xprev, float w_acc, const float4 *xs, float4 *xabs,
                      bool overlap, int *err) {
    if (c.n > 0 && c.ell_halo && err && c.cheb_mode == 2) {
        int b = nblk(c.n, ELL_TILE_ROWS);
        // all of the shared memory for the blocks (29 KB each at width 12)
        static unsigned long long carve_h[3] = {0, 0, 0};  // per-device bits
        int ci = c.ell_tw == 8 ? 0 : c.ell_tw == 12 ? 1 : 2, dev = 0;
        PDC_CK(cudaGetDevice(&dev));
        if (!(carve_h[ci] >> (dev & 63) & 1ull)) {
            const int pct = 100;
            cudaError_t e = ci == 0 ? cudaFuncSetAttribute(k_cheb_step_halo<8>, cudaFuncAttributePreferredSharedMemoryCarveout, pct)
                          : ci == 1 ? cudaFuncSetAttribute(k_cheb_step_halo<12>, cudaFuncAttributePreferredSharedMemoryCarveout, pct)
                                    : cudaFuncSetAttribute(k_cheb_step_halo<16>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
            PDC_CK(e);
            carve_h[ci] |= 1ull << (dev & 63);
        }
#define PDC_CHEB_H(W)                                                                                       \
    launch_dependent(overlap, k_cheb_step_halo<W>, b, ELL_TILE_ROWS, 0, s, c, cw, r, din, dprev, dout, alpha, beta, x, \
                     xout, xprev, w_acc, xs, xabs, sc, err)
        if (c.ell_tw == 8) PDC_CHEB_H(8);
        else if (c.ell_tw == 12) PDC_CHEB_H(12);
        else PDC_CHEB_H(16);
#undef PDC_CHEB_H
        PDC_LAUNCH_CK();
        return;
    }
    if (c.n > 0 && c.ell_tile && err && c.cheb_mode != 0) {
        int b = nblk(c.n, ELL_TILE_ROWS);
        // shared-memory carveout for 8 resident blocks (the register limit)
        static unsigned long long carve[3] = {0, 0, 0};  // per-device bits
        int ci = c.ell_tw == 8 ? 0 : c.ell_tw == 12 ? 1 : 2, dev = 0;
        PDC_CK(cudaGetDevice(&dev));
        if (!(carve[ci] >> (dev & 63) & 1ull)) {
            size_t need = 8 * (ell_tile_bytes(c.ell_tw) + 2048);
            int pct = (int)std::min<size_t>(100, (need * 100 + 228 * 1024 - 1) / (228 * 1024));
            cudaError_t e = ci == 0 ? cudaFuncSetAttribute(k_cheb_step_tile<8>, cudaFuncAttributePreferredSharedMemoryCarveout, pct)
                          : ci == 1 ? cudaFuncSetAttribute(k_cheb_step_tile<12>, cudaFuncAttributePreferredSharedMemoryCarveout, pct)
                                    : cudaFuncSetAttribute(k_cheb_step_tile<16>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
            PDC_CK(e);
            carve[ci] |= 1ull << (dev & 63);
        }
#define PDC_CHEB_T(W)                                                                                       \
    launch_dependent(overlap, k_cheb_step_tile<W>, b, ELL_TILE_ROWS, 0, s, c, cw, r, din, dprev, dout, alpha, beta, x, \
                     xout, xprev, w_acc, xs, xabs, sc, err)
        if (c.ell_tw == 8) PDC_CHEB_T(8);
        else if (c.ell_tw == 12) PDC_CHEB_T(12);
        else PDC_CHEB_T(16);
#undef PDC_CHEB_T
        PDC_LAUNCH_CK();
        return;
    }
    if (c.n > 0) {
        int b = nblk(c.n, 256);
#define PDC_CHEB(W)                                                                                         \
    launch_dependent(overlap, k_cheb_step<W>, b, 256, 0, s, c, cw, r, din, dprev, dout, alpha, beta, x, xout, xprev, \
                     w_acc, xs, xabs, sc)
        if (c.ell_w <= 8) PDC_CHEB(8);
        else if (c.ell_w <= 12) PDC_CHEB(12);
        else if (c.ell_w <= 16) PDC_CHEB(16);
        else PDC_CHEB(0);
#undef PDC_CHEB
    }
    PDC_LAUNCH_CK();
}

bool cheb_two_steps(const ClothView &c) { return c.n > 0 && c.ell_halo2 && c.cheb_mode == 3; }

void launch_cheb_step2(cudaStream_t s, const ClothView &c, const float *cw, const float4 *r, const float4 *din,
                       const float4 *dprev, float4 *dmid, float4 *dout, float a1, float b1, float a2, float b2,
                       const float4 *x, float4 *xout, Scalars *sc, float4 *xprev, float w_acc, const float4 *xs,
                       float4 *xabs, bool overlap, int *err) {
    if (!cheb_two_steps(c) || !err) throw Error(PDC_ERR_STATE, "two-step Chebyshev tiles not built");
    const size_t smem = halo2_tile_bytes(c.ell_tw, c.h2_rows, c.h2_verts) + 12 * (size_t)(c.h2_rows + c.h2_verts);
    static unsigned long long attr[3] = {0, 0, 0};  // per-device bits: the shared-memory limit raised
    int ci = c.ell_tw == 8 ? 0 : c.ell_tw == 12 ? 1 : 2, dev = 0;
    PDC_CK(cudaGetDevice(&dev));
    if (!(attr[ci] >> (dev & 63) & 1ull)) {
        const int lim = 160 * 1024;
        cudaError_t e = ci == 0 ? cudaFuncSetAttribute(k_cheb_step2_halo<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)
                      : ci == 1 ? cudaFuncSetAttribute(k_cheb_step2_halo<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)
                                : cudaFuncSetAttribute(k_cheb_step2_halo<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        PDC_CK(e);
        attr[ci] |= 1ull << (dev & 63);
    }
    const int b = nblk(c.n, ELL_TILE_ROWS);
#define PDC_CHEB2(W)                                                                                          \
    launch_dependent(overlap, k_cheb_step2_halo<W>, b, 256, smem, s, c, cw, r, din, dprev, dmid, dout, a1, b1, a2, b2, \
                     x, xout, xprev, w_acc, xs, xabs, sc, err)
    if (c.ell_tw == 8) PDC_CHEB2(8);
    else if (c.ell_tw == 12) PDC_CHEB2(12);
    else PDC_CHEB2(16);
#undef PDC_CHEB2
    PDC_LAUNCH_CK();
}

void launch_aa(cudaStream_t s, int n, const unsigned char *is_free, const float4 *delta, float4 *x, float4 *fprev,
               float4 *gprev, float4 *dF, float4 *dG, int slot, int have_prev, int ncol, double *Gb, float *theta,
               const float4 *xs, float4 *xabs, bool overlap) {
    if (n <= 0) return;
    // Gb is zeroed by the caller (aa_clear) before the kernels of this LG
    // iteration, so that the gram kernel can follow the last sweep directly
    const int b = nblk(n, 256);
    launch_dependent(overlap, k_aa_gram, b, 256, 0, s, n, is_free, delta, (const float4 *)x, fprev, gprev, dF, dG,
                     slot, have_prev, ncol, Gb, (const LoopCtl *)nullptr);
    if (ncol > 0) {
#define PDC_AA(M)                                                                                             \
    launch_dependent(overlap, k_aa_solve<M>, 1, 32, 0, s, (const double *)Gb, theta);                          \
    launch_dependent(overlap, k_aa_mix<M>, b, 256, 0, s, n, is_free, (const float4 *)x, (const float4 *)dG,   \
                     (const float *)theta, x, xs, xabs)
        switch (ncol) {
            case 1: PDC_AA(1); break;
            case 2: PDC_AA(2); break;
            case 3: PDC_AA(3); break;
            case 4: PDC_AA(4); break;
            case 5: PDC_AA(5); break;
            case 6: PDC_AA(6); break;
            case 7: PDC_AA(7); break;
            default: PDC_AA(8); break;
        }
#undef PDC_AA
    }
    PDC_LAUNCH_CK();
}

void launch_aa_device(cudaStream_t s, int n, const unsigned char *is_free, const float4 *delta, float4 *x,
                      float4 *fprev, float4 *gprev, float4 *dF, float4 *dG, int m, const LoopCtl *ctl, double *Gb,
                      float *theta, const float4 *xs, float4 *xabs, bool overlap) {
    if (n <= 0) return;
    const int b = nblk(n, 256);
    launch_dependent(overlap, k_aa_gram, b, 256, 0, s, n, is_free, delta, (const float4 *)x, fprev, gprev, dF, dG, 0,
                     0, 0, Gb, ctl);
#define PDC_AAD(M) launch_dependent(overlap, k_aa_solve_dev<M>, 1, 32, 0, s, (const double *)Gb, theta, ctl)
    switch (std::min(std::max(m, 1), AA_MAX)) {
        case 1: PDC_AAD(1); break;
        case 2: PDC_AAD(2); break;
        case 3: PDC_AAD(3); break;
        case 4: PDC_AAD(4); break;
        case 5: PDC_AAD(5); break;
        case 6: PDC_AAD(6); break;
        case 7: PDC_AAD(7); break;
        default: PDC_AAD(8); break;
    }
#undef PDC_AAD
    launch_dependent(overlap, k_aa_mix_dev, b, 256, 0, s, n, is_free, (const float4 *)x, (const float4 *)dG,
                     (const float *)theta, x, xs, xabs, ctl, m);
    PDC_LAUNCH_CK();
}

__global__ void k_live_zero(const int *live, unsigned int *p, size_t words) {
    if (loop_dead(live)) return;
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < words; k += (size_t)gridDim.x * blockDim.x)
        p[k] = 0u;
}

void launch_live_zero(cudaStream_t s, const int *live, void *p, size_t bytes) {
    if (!bytes) return;
    if (!live) {
        PDC_CK(cudaMemsetAsync(p, 0, bytes, s));
        return;
    }
    const size_t words = bytes / 4;
    const int blocks = (int)std::min<size_t>((words + 255) / 256, 152 * 8);
    k_live_zero<<<blocks, 256, 0, s>>>(live, (unsigned int *)p, words);
    PDC_LAUNCH_CK();
}

int aa_gram_doubles() { return AA_MAX * (AA_MAX + 3) / 2 + AA_MAX; }

void aa_clear(cudaStream_t s, double *Gb, const int *live) {
    launch_live_zero(s, live, Gb, sizeof(double) * (AA_MAX * (AA_MAX + 3) / 2 + AA_MAX));
}

void launch_lerp(cudaStream_t s, int nv, const float4 *a, const float4 *b, const double *s_frac, float4 *out,
                 const int *vinst, const double *s_inst) {
    if (nv > 0) k_lerp<<<nblk(nv, 256), 256, 0, s>>>(nv, a, b, s_frac, out, vinst, s_inst);
    PDC_LAUNCH_CK();
}


}  // namespace pdc
