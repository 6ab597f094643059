// C-ABI of the pdcloth library: context set-up (rest model of Sec. 3,
// basis of Sec. 5/7) and the per-step pipeline of Alg. 1 / Sec. 7.
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <unordered_map>

#include "pdc_collide.cuh"
#include "pdc_prof.cuh"
#include "pdc_subspace.cuh"
#include "pdc_umma.cuh"

namespace pdc {
void set_chol_smem_limits();

namespace {

__global__ void k_f3_to_f4(int n, const float *__restrict__ a, float4 *__restrict__ b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_float4(a[3 * i], a[3 * i + 1], a[3 * i + 2], 0.f);
}
__global__ void k_f4_to_f3(int n, const float4 *__restrict__ a, float *__restrict__ b) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        float4 v = a[i];
        b[3 * i] = v.x;
        b[3 * i + 1] = v.y;
        b[3 * i + 2] = v.z;
    }
}
// x_i <- rest_i transformed by the 3x4 affine m (row major)
__global__ void k_transform(int n, const float4 *__restrict__ rest, const float *__restrict__ m, float4 *__restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 p = rest[i];
    out[i] = make_float4(m[0] * p.x + m[1] * p.y + m[2] * p.z + m[3], m[4] * p.x + m[5] * p.y + m[6] * p.z + m[7],
                         m[8] * p.x + m[9] * p.y + m[10] * p.z + m[11], 0.f);
}
// s = alpha * t if an impact was found (t <= 1), else 1
__global__ void k_step_fraction(const unsigned long long *toi_bits, double alpha, double *s_out, double *t_out) {
    double t = __longlong_as_double((long long)*toi_bits);
    *t_out = t;
    *s_out = (t <= 1.0) ? alpha * t : 1.0;
}
// the same per instance (per-instance line search)
__global__ void k_instance_fractions(int count, const unsigned long long *toi_bits, double alpha, double *s_out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    double t = __longlong_as_double((long long)toi_bits[k]);
    s_out[k] = (t <= 1.0) ? alpha * t : 1.0;
}
__global__ void k_fill_u64(unsigned long long *p, int count, unsigned long long v) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < count) p[k] = v;
}
// final state (exit line search of Alg. 1): cloth u = um + s (up - um) (or up),
// x = x* + u, v = u / h, and u itself in ulast; obstacle vertices lerp
// between their absolute x^- and x^+.  s: the union's fraction, or with
// vinst the fraction of the vertex's instance.
__global__ void k_finish(int nv, int n, const float4 *__restrict__ um, const float4 *__restrict__ up,
                         const float4 *__restrict__ xm, const float4 *__restrict__ xp, const double *s_frac,
                         int use_lerp, float inv_h, float4 *__restrict__ xs, float4 *__restrict__ vs,
                         float4 *__restrict__ ulast, const int *__restrict__ vinst, const double *__restrict__ s_inst) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    float s = use_lerp ? (float)((vinst && vinst[i] >= 0) ? s_inst[vinst[i]] : *s_frac) : 1.f;
    if (i < n) {
        float3 d = f3(up[i]);
        if (use_lerp) {
            float3 a = f3(um[i]);
            d = a + s * (d - a);
        }
        vs[i] = f4(inv_h * d);
        ulast[i] = f4(d);
        xs[i] = f4(f3(xs[i]) + d);
    } else {
        float3 b = f3(xp[i]);
        if (use_lerp) {
            float3 a = f3(xm[i]);
            b = a + s * (b - a);
        }
        xs[i] = f4(b);
    }
}
__global__ void k_maxdiff(int n, const float4 *__restrict__ a, const float4 *__restrict__ b, unsigned int *out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    float m = 0.f;
    if (i < n) {
        float4 p = a[i], q = b[i];
        m = fmaxf(fabsf(p.x - q.x), fmaxf(fabsf(p.y - q.y), fabsf(p.z - q.z)));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(out, __float_as_uint(m));
}
__global__ void k_finite(int n, const float4 *__restrict__ a, int *bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        float4 p = a[i];
        if (!isfinite(p.x) || !isfinite(p.y) || !isfinite(p.z)) atomicOr(bad, 1);
    }
}

// `passes` copies between the halves a and b of a working set (a -> b on
// even passes, b -> a on odd ones) in one launch, 4 float4 per thread in
// flight, loads and stores that bypass L1 (cache-global), and the element
// each thread handles shifted every pass, so that no thread reads back what
// it has just written.  Timing it gives the copy bandwidth of the level of
// the memory hierarchy the working set lives in.
__global__ void __launch_bounds__(512) k_copy_passes(float4 *a, float4 *b, long long n, int passes) {
    const long long nthr = (long long)gridDim.x * blockDim.x;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (int p = 0; p < passes; ++p) {
        const float4 *src = (p & 1) ? b : a;
        float4 *dst = (p & 1) ? a : b;
        const long long shift = ((long long)p * 4099) % nthr;
        const long long me = (t + shift) % nthr;
        for (long long i0 = me; i0 < n; i0 += 4 * nthr) {
            float4 v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                long long i = i0 + k * nthr;
                if (i < n) v[k] = __ldcg(src + i);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                long long i = i0 + k * nthr;
                if (i < n) __stcg(dst + i, v[k]);
            }
        }
    }
}

// ---- device-side control of an LG loop (loops run as CUDA graphs)
// Settings of one loop for its stopping tests (same tests, in the same order,
// as the host-driven loop of pdc_ctx::step).
struct LoopCfg {
    int kind;                // 0: warm start (counts into warm_iters), 1: inner loop
    int max_iters;           // iteration cap of the loop
    int check_rel;           // relative-residual test and stagnation stop before each solve
    int dx_inner;            // after each solve: stop when max |dx| <= tolx_in
    int dx_springs;          // after a solve with collision springs: stop when max |dx| <= tolx_out
    int aa_m;                // Anderson history depth (0: no mixing)
    int stag_n;              // iterations without 1 % progress that stop the loop
    int use_cond;            // set the graph's while condition
    double tol_rel;
    double tolx_in, tolx_out;
    cudaGraphConditionalHandle cond;
};

// Everything an LG iteration accumulates into, zeroed in one launch at the
// start of its residual part: the residual norm, the contact-vertex count,
// the collision springs (cw, cf), the Anderson normal equations, the
// collision update of the reduced matrix and (host-driven loops; device
// decisions zero it after reading it) the step-change maximum.
struct IterZero {
    double *rsq;
    unsigned int *dxmax;  // NULL: left to the decision kernel
    int *ncv;
    float *cw;
    float4 *cf;
    int n;                // entries of cw / cf (0: no collision springs this loop)
    double *gb;
    int ngb;
    double *da;
    int nda;
};
__global__ void k_iter_begin(IterZero z, const int *live) {
    grid_dep_wait();
    grid_dep_release();
    if (loop_dead(live)) return;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x, nt = (long long)gridDim.x * blockDim.x;
    if (t == 0) {
        *z.rsq = 0.0;
        if (z.dxmax) *z.dxmax = 0u;
        *z.ncv = 0;
    }
    for (long long k = t; k < z.ngb; k += nt) z.gb[k] = 0.0;
    for (long long k = t; k < z.nda; k += nt) z.da[k] = 0.0;
    for (long long i = t; i < z.n; i += nt) {
        z.cw[i] = 0.f;
        z.cf[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// At the start of a step: the reference residual (its squared norm is in
// sc->rsq) and the step's counters.
__global__ void k_loop_step_init(LoopCtl *c, const Scalars *sc) {
    c->rho0 = sqrt(sc->rsq);
    c->rel = 0.0;
    c->warm_iters = c->inner_iters = c->contact_iters = 0;
    c->device_loops = 0;
}

// At the start of a loop (the host-driven loop resets its Accel state here).
__global__ void k_loop_begin(LoopCtl *c, int graph, Scalars *sc) {
    sc->dxmax = 0u;  // the loop's first solve reduces into zero
    c->iters = 0;
    c->go = 1;
    c->springs = 0;
    c->stag_best = 0.0;
    c->stag_count = 0;
    c->aa_hist_min = 0.0;
    c->aa_hist_n = 0;
    c->aa_count = c->aa_widx = c->aa_have_prev = 0;
    c->aa_slot = c->aa_prev = c->aa_ncol = 0;
    if (graph) c->device_loops++;
}

// The loop's decision after the residual of the current iterate (and, with
// after_solve, after the solve that produced it): the step-change tests of
// that solve, the iteration cap, then the relative-residual and stagnation
// tests; when the loop goes on, the iteration is counted and its
// Anderson-mixing slot assigned.  One thread.  Every path sets go (and the
// graph's condition), and go = 1 only while iters < max_iters, so a graph
// loop ends after at most max_iters iterations; a device error bit (a
// bounded wait that ran out) ends it at once.
__device__ int loop_decide(LoopCtl *c, const LoopCfg &f, const Scalars *sc, const int *n_cv, const int *dev_err,
                           int after_solve) {
    if (after_solve && !c->go) return 0;  // an earlier iteration of this pass ended the loop
    int go = (*dev_err & (PDC_DEVERR_UMMA | PDC_DEVERR_COPY)) ? 0 : 1;
    const double dx = (double)__uint_as_float(sc->dxmax);
    const_cast<Scalars *>(sc)->dxmax = 0u;  // consumed: the next solve reduces into zero
    if (go && after_solve) {
        if (f.dx_inner && dx <= f.tolx_in) go = 0;
        else if (f.dx_springs && c->springs && dx <= f.tolx_out) go = 0;
    }
    if (go && c->iters >= f.max_iters) go = 0;
    if (go) {
        const int springs = (n_cv && *n_cv > 0) ? 1 : 0;
        const double rho = sqrt(sc->rsq);
        if (f.check_rel) {
            c->rel = rho / fmax(c->rho0, 1e-300);
            if (rho <= f.tol_rel * c->rho0) {
                go = 0;
            } else if (springs || c->stag_best == 0.0 || rho < 0.99 * c->stag_best) {
                c->stag_best = (springs || c->stag_best == 0.0) ? rho : fmin(c->stag_best, rho);
                c->stag_count = 0;
            } else if (++c->stag_count >= f.stag_n) {
                go = 0;
            }
        }
        if (go) {
            if (springs) c->contact_iters++;
            if (f.aa_m > 0) {
                // restart the history when the residual jumps above twice its
                // smallest value since the last restart
                if (c->aa_hist_n > 0 && rho > 2.0 * c->aa_hist_min) {
                    c->aa_hist_n = 0;
                    c->aa_count = c->aa_widx = c->aa_have_prev = 0;
                }
                c->aa_hist_min = c->aa_hist_n > 0 ? fmin(c->aa_hist_min, rho) : rho;
                c->aa_hist_n++;
                c->aa_prev = c->aa_have_prev;
                c->aa_slot = 0;
                if (c->aa_have_prev) {
                    c->aa_slot = c->aa_widx % f.aa_m;
                    c->aa_widx++;
                    c->aa_count = min(c->aa_count + 1, f.aa_m);
                }
                c->aa_ncol = c->aa_count;
                c->aa_have_prev = 1;
            }
            c->springs = springs;
            c->iters++;
            if (f.kind == 0) c->warm_iters++;
            else c->inner_iters++;
        }
    }
    c->go = go;
    return go;
}

// Two kernels: only the decision that ends a pass of the while node sets its
// condition (a kernel that calls into the device runtime costs more to
// complete, so the other decisions of an unrolled pass do without).
__global__ void k_loop_decide(LoopCtl *c, LoopCfg f, const Scalars *sc, const int *n_cv, const int *dev_err,
                              int after_solve) {
    if (threadIdx.x == 0 && blockIdx.x == 0) loop_decide(c, f, sc, n_cv, dev_err, after_solve);
}
// The decision of a loop whose iterations the host enqueues ahead: go and
// the number of decisions taken so far go to host-mapped memory (read there
// without a stream synchronisation).
__global__ void k_loop_decide_host(LoopCtl *c, LoopCfg f, const Scalars *sc, const int *n_cv, const int *dev_err,
                                   int after_solve, volatile int *host) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int go = loop_decide(c, f, sc, n_cv, dev_err, after_solve);
    host[0] = go;
    __threadfence_system();
    host[1] = host[1] + 1;
    __threadfence_system();
}
__global__ void k_loop_decide_cond(LoopCtl *c, LoopCfg f, const Scalars *sc, const int *n_cv, const int *dev_err,
                                   int after_solve) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int go = loop_decide(c, f, sc, n_cv, dev_err, after_solve);
    cudaGraphSetConditional(f.cond, go ? 1u : 0u);
}



inline int nb(long long n) { return (int)((n + 255) / 256); }
inline float bits_to_float(unsigned int u) {
    float f;
    std::memcpy(&f, &u, sizeof(f));
    return f;
}

struct Obstacle {
    std::vector<float> V;  // rest verts
    std::vector<int> T;
    int off;               // first collision-vertex id
};

// Chebyshev semi-iterative acceleration of the LG iterates (Wang 2015, a
// Jacobi-type PD accelerator the paper cites): after S plain iterations of a
// pass, x_{k+1} = w_{k+1} (x_hat_{k+1} - x_{k-1}) + x_{k-1} with
// w = 2 / (2 - rho^2) first and w_{k+1} = 4 / (4 - rho^2 w_k) after; rho is
// the spectral radius of the plain iteration, estimated from the decay of the
// measured residual over the plain iterations.  A residual jump restarts it.
struct Accel {
    bool on = false;
    double rho_fixed = 0.0, rho = 0.0, w = 1.0;
    int k = 0;
    std::vector<double> hist;
    static constexpr int S = 5;
    void reset() {
        k = 0;
        w = 1.0;
        hist.clear();
        aa_reset();
        stag_best = 0.0;
        stag_count = 0;
    }
    // residual-stagnation stop of the relative-residual mode: without
    // collision springs, STAG_N iterations that do not lower the best
    // residual of the pass by 1% end the inner loop (the FP32 floor of a
    // nearly unstrained cloth, e.g. in free fall, lies above small targets)
    static constexpr int STAG_N = 32;
    double stag_best = 0.0;
    int stag_count = 0;
    bool stagnated(double rho, bool springs) {
        if (springs || stag_best == 0.0 || rho < 0.99 * stag_best) {
            stag_best = (springs || stag_best == 0.0) ? rho : std::min(stag_best, rho);
            stag_count = 0;
            return false;
        }
        return ++stag_count >= STAG_N;
    }
    double rho_carry = 0.0;  // estimate carried from earlier passes
    // Anderson mixing history (accel = 2)
    int aa_count = 0, aa_widx = 0;
    bool aa_have_prev = false;
    void aa_reset() {
        aa_count = 0;
        aa_widx = 0;
        aa_have_prev = false;
    }
    // Anderson: restart the history when the residual jumps above twice the
    // smallest residual of the current history
    void aa_observe(double meas) {
        if (!hist.empty() && meas > 2.0 * *std::min_element(hist.begin(), hist.end())) {
            hist.clear();
            aa_reset();
        }
        hist.push_back(meas);
    }
    double next(double meas) {
        if (!on) return 1.0;
        if (!hist.empty() && meas > 2.0 * *std::min_element(hist.begin(), hist.end())) reset();
        hist.push_back(meas);
        if (k < S) {
            ++k;
            w = 1.0;
            return 1.0;
        }
        if (k == S) {
            if (rho_fixed > 0) {
                rho = rho_fixed;
            } else {
                size_t n = hist.size();
                double ratio = hist[n - 1] / std::max(hist[n - 4], 1e-300);
                rho = std::pow(std::max(ratio, 1e-12), 1.0 / 3.0);
                // the first iterations of a pass decay faster than the asymptotic
                // rate: keep the largest estimate seen so far
                if (!std::isfinite(rho)) rho = 0.3;
                rho = std::max(rho, rho_carry);
                rho = std::min(std::max(rho, 0.3), 0.99);
                rho_carry = rho;
            }
            w = 2.0 / (2.0 - rho * rho);
        } else {
            w = 4.0 / (4.0 - rho * rho * w);
        }
        ++k;
        return w;
    }
};

}  // namespace
}  // namespace pdc

using namespace pdc;

#define PROF(name, bytes, ...)                                                                        \
    do {                                                                                               \
        if (prof.on) prof.begin(s, name, (double)(bytes));                                              \
        __VA_ARGS__;                                                                                   \
        if (prof.on) prof.end(s);                                                                      \
        if (sync_check) check_region(name);                                                            \
    } while (0)

struct pdc_ctx {
    std::string err;
    cudaStream_t s = nullptr;
    pdc_params P;
    pdc_material M;
    // batched form: material of each instance and the instance of each triangle
    // (empty: one cloth with material M)
    std::vector<pdc_material> mats;
    std::vector<int> tri_inst;
    const pdc_material &mat(int t) const { return tri_inst.empty() ? M : mats[tri_inst[t]]; }
    int n = 0, m = 0, nh = 0, npins = 0;
    std::vector<float> X;
    std::vector<int> T, pins;
    std::vector<unsigned char> freev;
    double L = 1.0, k_ndb = 1.0, omega = 1.0;
    float dhat = 1e-3f;
    // rest model
    DevBuf<int4> tri, hin;
    DevBuf<float4> tri_g, hin_K, hin_srest;
    DevBuf<float> tri_w, hin_w, hin_slen, mh2, hdiag, ell_val;
    DevBuf<int> vt_off, vt_list, vh_off, vh_list, ell_col, pins_d;
    DevBuf<short> ell_dcol;
    DevBuf<unsigned char> ell_tile;
    int ell_tw = 0;
    DevBuf<unsigned char> ell_halo;  // patch tiles (ClothView::ell_halo)
    DevBuf<unsigned char> ell_halo2; // two-step patch tiles (ClothView::ell_halo2)
    int h2_rows = 0, h2_verts = 0;
    void build_patch_tiles2(const std::vector<int> &ecol, const std::vector<float> &evalv);
    std::vector<int> morton_order() const;
    void build_patch_tiles(const std::vector<int> &ecol, const std::vector<float> &evalv);
    // element forces and residual per mesh patch (ClothView::rp_*)
    DevBuf<unsigned char> rp_rec;
    DevBuf<long long> rp_off;
    int rp_loc = 0, rp_tri = 0, rp_hin = 0;  // largest counts over the patches
    // shared memory of k_residual_patch: positions x*, u of the touched
    // vertices (6 floats), corner forces of the triangles (9), per hinge its
    // vector s_hat - s and the four weights w K_j (7)
    size_t residual_patch_smem() const {
        return 4 * (6 * (size_t)rp_loc + 9 * (size_t)rp_tri + 7 * (size_t)rp_hin);
    }
    void build_residual_patches(const std::vector<int> &vto, const std::vector<int> &vtl, const std::vector<int> &vho,
                                const std::vector<int> &vhl, const std::vector<int4> &tri_h,
                                const std::vector<int4> &hin_h);
    DevBuf<unsigned char> is_free;
    int ell_w = 0;
    // pins
    DevBuf<float4> pin_tgt;
    // state (collision-vertex arrays: cloth first, obstacles after)
    DevBuf<float4> Xs, Vs, Z, Xp, Xm, Xbak, Vbak, Xprev;
    DevBuf<float4> R, RL, D0, D1, CF;
    DevBuf<float4> Ucur, Um;  // iterate and x^- as displacements from x* (cloth vertices)
    DevBuf<float4> Ulast;     // displacement x_new - x* of the last step, before rounding x_new
    DevBuf<float> CW;
    DevBuf<float> stage3;  // staging for float[3] transfers
    // obstacles
    std::vector<Obstacle> obs;
    DevBuf<float4> obs_rest, obs_tgt;  // [nv_obs]
    int nv_all = 0, nt_all = 0, ne_all = 0;
    bool topo_dirty = true;
    std::vector<int> ctri_h, cedge_h;
    DevBuf<int4> ctri;
    DevBuf<int2> cedge;
    DevBuf<unsigned char> vfixed;
    DevBuf<unsigned int> guard_d;  // index-guard word of this handle's pair kernels
    // batched form: first vertex of each instance (count + 1 entries), the
    // instance each obstacle is attached to (-1: none), and for the
    // per-instance line search the instance of every collision vertex and
    // each instance's time of impact and step fraction
    std::vector<int> inst_off;
    std::vector<int> obs_inst;
    DevBuf<int> vinst;
    DevBuf<unsigned long long> toi_inst;
    DevBuf<double> sfrac_inst;
    int ninst() const { return inst_off.empty() ? 1 : (int)inst_off.size() - 1; }
    // one step fraction per instance: asked for, batched, every obstacle attached
    bool per_instance() const {
        if (!P.instance_line_search || ninst() < 2) return false;
        for (int k : obs_inst)
            if (k < 0) return false;
        return vinst.p != nullptr;
    }
    void upload_vinst();
    BroadPhase bp;
    DevBuf<ActivePair> act;
    int cap_act = 0;
    DevBuf<int> contact_list;
    // subspace
    int r_warm = 0, r_reuse = 0, ld = 0;
    DevBuf<float> U32, A0inv32, proj_partial, qbuf;
    DevBuf<double> dA;
    DevBuf<uint16_t> U16bits;    // 16-bit basis [n][ld] (BF16 or scaled FP16 bits)
    DevBuf<uint16_t> Ut16;       // its transpose [ld][n_pad] (tensor-core projection)
    int n_pad = 0;
    UmmaMaps umma;
    DevBuf<float> umma_partial;
    int ldc = 0;                 // width of the compact copy of the leading r_reuse columns
    DevBuf<float> Uc32;
    DevBuf<uint16_t> Uc16bits;
    DevBuf<double> A0, A0inv, gbuf;
    DevBuf<int> sflag;
    // scalars
    DevBuf<Scalars> sc;
    Scalars *hsc = nullptr;
    DevBuf<double> sfrac, ttoi;
    DevBuf<unsigned long long> toi_bits;
    DevBuf<int> n_act_d, n_cv_d, bad_d, bp_ovf;
    DevBuf<unsigned int> umax_d;
    pdc_stats st;
    bool stepped = false;
    Profiler prof;
    Accel accel;
    float last_dx = 0.f;
    DevBuf<float4> Xacc;  // previous iterate for the accelerated update
    DevBuf<float4> disp;  // x^+ - x^- per collision vertex
    DevBuf<float4> CD0;  // third Chebyshev iterate (delta_{k-1})
    DevBuf<float4> CD1;  // fourth, for two steps a launch
    DevBuf<float4> corner;  // per-element corner forces of the residual [3m + 4nh]
    DevBuf<float4> aa_dF, aa_dG, aa_f, aa_g;  // Anderson history
    DevBuf<double> aa_Gb;
    DevBuf<float4> RFd;        // residual-forwarding dx carried to the next step
    bool rf_pending = false;
    DevBuf<float> aa_theta;
    double gersh = 1.0;       // Gershgorin bound of D^-1 H
    long long nnz_off = 0;  // off-diagonal entries of H over free rows
    bool log = std::getenv("PDC_LOG") != nullptr;  // per-iteration residuals to stderr
    // initial candidate-list capacity (pairs of each kind) when set: small
    // values exercise the regrowth of the broad-phase buffers
    long long bp_cap0 = std::getenv("PDC_BP_CAPACITY") ? std::atoll(std::getenv("PDC_BP_CAPACITY")) : 0;
    // diagnostics: synchronise after every profiled region and name the
    // region in the error of a failed kernel
    bool sync_check = std::getenv("PDC_SYNC_CHECK") != nullptr;
    bool last_springs = false;  // the last LG iteration had collision springs
    void check_region(const char *name) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess)
            throw Error(PDC_ERR_CUDA, std::string("after ") + name + ": " + cudaGetErrorString(e));
    }

    ~pdc_ctx() {
        if (hsc) cudaFreeHost(hsc);
        if (hmap) cudaFreeHost((void *)hmap);
        for (auto &G : gl) free_graph(G);
        for (auto &G : gb) free_body(G);
        if (gs) cudaStreamDestroy(gs);
    }

    ClothView cloth() const {
        ClothView c;
        c.n = n;
        c.m = m;
        c.nh = nh;
        c.tri = tri;
        c.tri_g = tri_g;
        c.tri_w = tri_w;
        c.hin = hin;
        c.hin_K = hin_K;
        c.hin_w = hin_w;
        c.hin_slen = hin_slen;
        c.hin_srest = hin_srest;
        c.vt_off = vt_off;
        c.vt_list = vt_list;
        c.vh_off = vh_off;
        c.vh_list = vh_list;
        c.mh2 = mh2;
        c.hdiag = hdiag;
        c.is_free = is_free;
        c.ell_w = ell_w;
        c.ell_col = ell_col;
        c.ell_dcol = ell_dcol.p;
        c.ell_val = ell_val;
        c.overlap = P.launch_overlap != 0;
        c.ell_tile = ell_tile.p;
        c.ell_tw = ell_tw;
        c.ell_halo = ell_halo.p;
        c.ell_halo2 = ell_halo2.p;
        c.h2_rows = h2_rows;
        c.h2_verts = h2_verts;
        const bool rp = P.residual_patch != 0 && rp_rec.p;
        c.rp_rec = rp ? rp_rec.p : nullptr;
        c.rp_off = rp ? rp_off.p : nullptr;
        c.rp_loc = rp_loc;
        c.rp_tri = rp_tri;
        c.rp_hin = rp_hin;
        c.corner = corner;
        c.res_block = tune.residual_block;
        {
            int want = P.cheb_source >= 0 ? P.cheb_source : tune.cheb_tile;
            if (want == 3 && !ell_halo2.p) want = 2;
            if (want == 2 && !ell_halo.p) want = 1;
            c.cheb_mode = want;
        }
        c.live = live_ptr;
        return c;
    }
    CollView coll() const {
        CollView v;
        v.nv = nv_all;
        v.nc = n;
        v.nt = nt_all;
        v.ne = ne_all;
        v.tri = ctri;
        v.edge = cedge;
        v.vfixed = vfixed;
        v.guard = guard_d;
        v.live = live_ptr;
        const bool pi = per_instance();
        v.vinst = pi ? vinst.p : nullptr;
        v.toi_inst = pi ? toi_inst.p : nullptr;
        return v;
    }
    SubspaceView sub(int r_nc, int r_c) const {
        SubspaceView S;
        S.n = n;
        S.ld = ld;
        S.r_nc = r_nc;
        S.r_c = r_c;
        S.U32 = U32;
        S.U16 = P.precision == 1 ? reinterpret_cast<const __nv_bfloat16 *>(U16bits.p) : nullptr;
        S.Uh = P.precision == 2 ? reinterpret_cast<const __half *>(U16bits.p) : nullptr;
        S.A0 = A0;
        S.A0inv = A0inv;
        S.A0inv32 = A0inv32;
        S.precision = P.precision;
        S.ldc = ldc;
        S.Uc32 = Uc32;
        S.Uc16 = P.precision == 1 ? reinterpret_cast<const __nv_bfloat16 *>(Uc16bits.p) : nullptr;
        S.Uch = P.precision == 2 ? reinterpret_cast<const __half *>(Uc16bits.p) : nullptr;
        S.umma = (umma.ok && P.precision != 0 && P.tensor_cores) ? &umma : nullptr;
        S.umma_partial = umma_partial;
        S.dev_err = sflag;
        S.overlap = P.launch_overlap != 0;
        S.live = live_ptr;
        return S;
    }
    SubspaceWork work() {
        SubspaceWork W;
        W.partial = proj_partial;
        W.g = gbuf;
        W.q = qbuf;
        W.dA = dA;
        W.flag = sflag;
        return W;
    }
    CollParams cparams() const {
        CollParams C;
        C.dhat = dhat;
        C.eta = P.eta_ccd;
        C.k_ndb = (float)k_ndb;
        C.K_ndb = (float)P.K_ndb;
        C.a_max = P.a_max;
        C.samples_vt = P.samples_vt;
        C.samples_ee = P.samples_ee;
        C.adaptive = P.pccd_adaptive;
        C.max_axis = P.pccd_max_axis;
        C.alpha = P.alpha_ls;
        return C;
    }

    void setup(const pdc_mesh_desc *mesh);
    void setup_basis();
    void install_basis(const std::vector<float> &U, int r);
    void ensure_topology();
    void read_scalars() {
        sc.download(hsc, 1, s);
        PDC_CK(cudaStreamSynchronize(s));
    }
    // algorithmic bytes per launch (FP32 values, 4-byte indices)
    double bytes_residual(bool contacts) const {
        return (double)m * 32 + (double)nh * 40 + (double)n * (12 + 12 + 12 + 4 + 1 + 8) +
               (double)(3LL * m + 4LL * nh) * 4 + (contacts ? (double)n * 16 : 0.0);
    }
    double bytes_sweep(bool contacts, bool writes_x) const {
        return (double)nnz_off * (ell_dcol.p ? 6 : 8) + (double)n * (12 + 12 + 4 + 1 + 12) + (contacts ? 4.0 * n : 0.0) +
               (writes_x ? 24.0 * n : 0.0);
    }
    double bytes_basis(int r) const { return (double)n * r * (P.precision != 0 ? 2 : 4) + (double)n * 12; }
    void lg_iteration(bool contacts, bool check_rel, double rho0, bool &converged, int r_nc, int r_c, int cycles,
                      int sweeps, bool pccd = true);
    void enqueue_residual(bool contacts);
    void enqueue_solve(bool contacts, bool springs, bool device, float w_acc, int r_nc, int r_c, int cycles,
                       int sweeps, bool pccd);
    // device-driven LG loops (CUDA graphs with a conditional while node)
    struct GraphLoop {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t e = nullptr;
        unsigned gen = 0;
    };
    GraphLoop gl[4];             // warm start, inner loop without collisions, inner loop with bp.cur = 0 / 1
    // loop_control = 3: one iteration of the same four loops, instantiated
    // MAX_AHEAD + 1 times and launched in turn, so that no instance is
    // launched again while its previous launch is in flight (such a launch
    // starts late, by about the time the device takes to relaunch it)
    static constexpr int MAX_AHEAD = 2;  // largest loop_ahead
    struct BodyGraph {
        cudaGraph_t g = nullptr;
        cudaGraphExec_t e[MAX_AHEAD + 1] = {};
        unsigned gen = 0;
    };
    BodyGraph gb[4];
    bool bodies_failed = false;  // an iteration graph could not be built: stream launches
    cudaStream_t gs = nullptr;   // capture stream
    unsigned graph_gen = 1;      // bumped when a buffer a graph captures is reallocated
    bool graphs_failed = false;  // a graph could not be built: host-driven loops from then on
    bool graph_overlap = true;   // programmatic dependent launches inside the graphs
    // while a device-driven loop is captured: the loop's go flag, which every
    // kernel of its iterations reads (they do nothing once the loop has ended)
    const int *live_ptr = nullptr;
    DevBuf<LoopCtl> ctl;
    LoopCtl hctl;
    bool device_decides = false;  // the loop being enqueued takes its tests on the device
    pdc_tuning tune = {0, 256, 2, 152 * 8, 8, {0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0}, 1.f, {0, 0, 0}};
    void autotune_vertex_kernels();
    bool device_loops_ok() const;
    void free_graph(GraphLoop &G);
    LoopCfg loop_cfg(int kind, int max_iters, bool relmode, bool contacts) const;
    bool build_loop(GraphLoop &G, const LoopCfg &cfg, bool contacts, int r_nc, int r_c, int cycles, int sweeps,
                    bool pccd);
    bool run_loop(int gi, const LoopCfg &cfg, bool contacts, int r_nc, int r_c, int cycles, int sweeps, bool pccd);
    // loop_control = 2, 3: host-mapped {go, decisions} of the loop being run
    volatile int *hmap = nullptr;
    int *hmap_dev = nullptr;
    void enqueue_iteration(const LoopCfg &cfg, bool contacts, int r_nc, int r_c, int cycles, int sweeps, bool pccd);
    void free_body(BodyGraph &G);
    bool build_body(BodyGraph &G, const LoopCfg &cfg, bool contacts, int r_nc, int r_c, int cycles, int sweeps,
                    bool pccd);
    void run_loop_ahead(int gi, const LoopCfg &cfg, bool contacts, int r_nc, int r_c, int cycles, int sweeps,
                        bool pccd);
    void residual_forwarding();
    void full_ccd(const float4 *x0, const float4 *x1, bool merge);
    void broad_phase_pass(const float4 *x0, const float4 *x1, bool super);
    void step();
};

// ============================================================================ set-up
void pdc_ctx::setup(const pdc_mesh_desc *mesh) {
    n = mesh->nv;
    m = mesh->nt;
    npins = mesh->npins;
    X.assign(mesh->verts, mesh->verts + 3 * (size_t)n);
    T.assign(mesh->tris, mesh->tris + 3 * (size_t)m);
    pins.assign(mesh->pins, mesh->pins + npins);
    freev.assign(n, 1);
    for (int p : pins) {
        if (p < 0 || p >= n) throw Error(PDC_ERR_ARG, "pin index out of range");
        freev[p] = 0;
    }
    for (int t = 0; t < m; ++t)
        for (int k = 0; k < 3; ++k)
            if (T[3 * t + k] < 0 || T[3 * t + k] >= n) throw Error(PDC_ERR_ARG, "triangle index out of range");
    const double h = P.dt;
    auto Xd = [&](int i, int k) { return (double)X[3 * (size_t)i + k]; };
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], Xd(i, k));
            hi[k] = std::max(hi[k], Xd(i, k));
        }
    L = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                  (hi[2] - lo[2]) * (hi[2] - lo[2]));
    if (!(L > 0)) L = 1.0;

    // ---- triangles: rest frame, Dm^-1 rows, area, weight, lumped mass
    std::vector<int4> tri_h(m);
    std::vector<float4> trig_h(m);
    std::vector<float> triw_h(m);
    std::vector<double> area(m), mass(n, 0.0);
    std::vector<std::array<double, 6>> G(m);  // g0, g1, g2 (2 each)
    for (int t = 0; t < m; ++t) {
        int a = T[3 * t], b = T[3 * t + 1], c = T[3 * t + 2];
        double e1[3], e2[3];
        for (int k = 0; k < 3; ++k) {
            e1[k] = Xd(b, k) - Xd(a, k);
            e2[k] = Xd(c, k) - Xd(a, k);
        }
        double nr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double nn = std::sqrt(nr[0] * nr[0] + nr[1] * nr[1] + nr[2] * nr[2]);
        double l1 = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        if (!(nn > 1e-14 * L * L) || !(l1 > 0)) throw Error(PDC_ERR_DEGENERATE, "zero-area rest triangle " + std::to_string(t));
        area[t] = 0.5 * nn;
        // orthonormal frame (t1 along e1, t2 = n x t1 / |..|) -> Dm = [[|e1|, e2.t1], [0, e2.t2]]
        double t1[3] = {e1[0] / l1, e1[1] / l1, e1[2] / l1};
        double e2t1 = e2[0] * t1[0] + e2[1] * t1[1] + e2[2] * t1[2];
        double e2t2 = nn / l1;  // |e1 x e2| / |e1|
        // Dm^-1 = [[1/l1, -e2t1/(l1 e2t2)], [0, 1/e2t2]]
        double i00 = 1.0 / l1, i01 = -e2t1 / (l1 * e2t2), i10 = 0.0, i11 = 1.0 / e2t2;
        // g1 = row 0, g2 = row 1, g0 = -g1 - g2
        G[t] = {-(i00 + i10), -(i01 + i11), i00, i01, i10, i11};
        tri_h[t] = make_int4(a, b, c, 0);
        trig_h[t] = make_float4((float)i00, (float)i01, (float)i10, (float)i11);
        triw_h[t] = (float)(mat(t).k_stretch * area[t]);
        for (int k = 0; k < 3; ++k) mass[T[3 * t + k]] += mat(t).density * area[t] / 3.0;
    }

    // ---- edges -> hinges
    std::map<std::pair<int, int>, std::vector<std::pair<int, int>>> emap;  // edge -> (tri, opposite)
    for (int t = 0; t < m; ++t)
        for (int k = 0; k < 3; ++k) {
            int u = T[3 * t + k], v = T[3 * t + (k + 1) % 3], o = T[3 * t + (k + 2) % 3];
            emap[{std::min(u, v), std::max(u, v)}].push_back({t, o});
        }
    std::vector<int4> hin_h;
    std::vector<float4> hK_h, hsr_h;
    std::vector<float> hw_h, hsl_h;
    std::vector<std::array<double, 4>> Kd;
    std::vector<double> wd;
    for (auto &kv : emap) {
        if (kv.second.size() > 2) throw Error(PDC_ERR_DEGENERATE, "edge shared by more than two triangles");
        if (kv.second.size() != 2) continue;
        int x0 = kv.first.first, x1 = kv.first.second, x2 = kv.second[0].second, x3 = kv.second[1].second;
        auto cotv = [&](int o, int p, int q) {  // cot of the angle at o between (p - o) and (q - o)
            double u[3], w[3];
            for (int k = 0; k < 3; ++k) {
                u[k] = Xd(p, k) - Xd(o, k);
                w[k] = Xd(q, k) - Xd(o, k);
            }
            double d = u[0] * w[0] + u[1] * w[1] + u[2] * w[2];
            double cx = u[1] * w[2] - u[2] * w[1], cy = u[2] * w[0] - u[0] * w[2], cz = u[0] * w[1] - u[1] * w[0];
            return d / std::sqrt(cx * cx + cy * cy + cz * cz);
        };
        double cA0 = cotv(x0, x1, x2), cA1 = cotv(x1, x0, x2), cB0 = cotv(x0, x1, x3), cB1 = cotv(x1, x0, x3);
        std::array<double, 4> K = {cA1 + cB1, cA0 + cB0, -cA0 - cA1, -cB0 - cB1};
        double w = 3.0 * mat(kv.second[0].first).k_bend / (area[kv.second[0].first] + area[kv.second[1].first]);
        int ids[4] = {x0, x1, x2, x3};
        double s[3] = {0, 0, 0};
        for (int j = 0; j < 4; ++j)
            for (int k = 0; k < 3; ++k) s[k] += K[j] * Xd(ids[j], k);
        double sl = std::sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
        hin_h.push_back(make_int4(x0, x1, x2, x3));
        hK_h.push_back(make_float4((float)K[0], (float)K[1], (float)K[2], (float)K[3]));
        hw_h.push_back((float)w);
        hsl_h.push_back((float)sl);
        hsr_h.push_back(make_float4((float)s[0], (float)s[1], (float)s[2], 0.f));
        Kd.push_back(K);
        wd.push_back(w);
    }
    nh = (int)hin_h.size();
    corner.alloc(std::max<size_t>(3 * (size_t)m + 4 * (size_t)nh, 1));

    // ---- H = M/h^2 + sum_t w_t G G^T + sum_h w_h K K^T  (scalar, per vertex pair)
    std::vector<std::unordered_map<int, double>> rows(n);
    for (int i = 0; i < n; ++i) rows[i][i] += mass[i] / (h * h);
    for (int t = 0; t < m; ++t) {
        double w = mat(t).k_stretch * area[t];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double v = w * (G[t][2 * a] * G[t][2 * b] + G[t][2 * a + 1] * G[t][2 * b + 1]);
                rows[T[3 * t + a]][T[3 * t + b]] += v;
            }
    }
    for (int hh = 0; hh < nh; ++hh) {
        int ids[4] = {hin_h[hh].x, hin_h[hh].y, hin_h[hh].z, hin_h[hh].w};
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) rows[ids[a]][ids[b]] += wd[hh] * Kd[hh][a] * Kd[hh][b];
    }
    std::vector<float> hdiag_h(n), mh2_h(n);
    ell_w = 0;
    for (int i = 0; i < n; ++i) {
        hdiag_h[i] = (float)rows[i][i];
        mh2_h[i] = (float)(mass[i] / (h * h));
        if (!freev[i]) continue;
        int cnt = 0;
        for (auto &kv : rows[i])
            if (kv.first != i && freev[kv.first]) ++cnt;
        ell_w = std::max(ell_w, cnt);
    }
    nnz_off = 0;
    for (int i = 0; i < n; ++i)
        if (freev[i])
            for (auto &kv : rows[i])
                if (kv.first != i && freev[kv.first]) ++nnz_off;
    std::vector<int> ecol((size_t)ell_w * n);
    std::vector<float> evalv((size_t)ell_w * n, 0.f);
    for (int i = 0; i < n; ++i) {
        std::vector<std::pair<int, double>> ent;
        if (freev[i])
            for (auto &kv : rows[i])
                if (kv.first != i && freev[kv.first]) ent.push_back(kv);
        std::sort(ent.begin(), ent.end());
        for (int k = 0; k < ell_w; ++k) {
            ecol[(size_t)k * n + i] = k < (int)ent.size() ? ent[k].first : i;
            evalv[(size_t)k * n + i] = k < (int)ent.size() ? (float)ent[k].second : 0.f;
        }
    }
    double dsum = 0;
    int nf = 0;
    for (int i = 0; i < n; ++i)
        if (freev[i]) {
            dsum += rows[i][i];
            ++nf;
        }
    k_ndb = P.k_ndb_scale * (nf ? dsum / nf : 1.0);

    // Jacobi damping: omega < 2 / lambda_max(D^-1 H) keeps the sweep
    // convergent; the Gershgorin bound max_i sum_j |H_ij| / H_ii bounds
    // lambda_max from above (bending makes H far from diagonally dominant:
    // lambda_max(D^-1 H) is about 3.5 on a 512 x 512 sheet).
    if (P.jacobi_omega > 0) {
        omega = P.jacobi_omega;
    } else {
        double gmax = 1.0;
        for (int i = 0; i < n; ++i) {
            if (!freev[i]) continue;
            double sum = 0;
            for (auto &kv : rows[i])
                if (freev[kv.first]) sum += std::fabs(kv.second);
            gmax = std::max(gmax, sum / rows[i][i]);
        }
        omega = std::min(1.0, 1.8 / gmax);
    }
    {
        double gmax = 1.0;
        for (int i = 0; i < n; ++i) {
            if (!freev[i]) continue;
            double sum = 0;
            for (auto &kv : rows[i])
                if (freev[kv.first]) sum += std::fabs(kv.second);
            gmax = std::max(gmax, sum / rows[i][i]);
        }
        gersh = gmax;
    }
    // gap
    if (P.d_hat > 0) {
        dhat = (float)P.d_hat;
    } else {
        double es = 0;
        for (auto &kv : emap) {
            double d2 = 0;
            for (int k = 0; k < 3; ++k) {
                double dd = Xd(kv.first.first, k) - Xd(kv.first.second, k);
                d2 += dd * dd;
            }
            es += std::sqrt(d2);
        }
        double me = emap.empty() ? 1.0 : es / emap.size();
        dhat = (float)std::min(1e-3, 0.2 * me);
    }

    // ---- incidence lists
    std::vector<int> vto(n + 1, 0), vho(n + 1, 0);
    for (int t = 0; t < m; ++t)
        for (int k = 0; k < 3; ++k) vto[T[3 * t + k] + 1]++;
    for (int hh = 0; hh < nh; ++hh) {
        vho[hin_h[hh].x + 1]++;
        vho[hin_h[hh].y + 1]++;
        vho[hin_h[hh].z + 1]++;
        vho[hin_h[hh].w + 1]++;
    }
    for (int i = 0; i < n; ++i) {
        vto[i + 1] += vto[i];
        vho[i + 1] += vho[i];
    }
    std::vector<int> vtl(vto[n]), vhl(vho[n]), ft(vto.begin(), vto.end() - 1), fh(vho.begin(), vho.end() - 1);
    for (int t = 0; t < m; ++t)
        for (int k = 0; k < 3; ++k) vtl[ft[T[3 * t + k]]++] = (t << 2) | k;
    for (int hh = 0; hh < nh; ++hh) {
        int ids[4] = {hin_h[hh].x, hin_h[hh].y, hin_h[hh].z, hin_h[hh].w};
        for (int k = 0; k < 4; ++k) vhl[fh[ids[k]]++] = (hh << 2) | k;
    }
    build_residual_patches(vto, vtl, vho, vhl, tri_h, hin_h);

    // ---- upload
    tri.upload(tri_h, s);
    tri_g.upload(trig_h, s);
    tri_w.upload(triw_h, s);
    hin.upload(hin_h, s);
    hin_K.upload(hK_h, s);
    hin_w.upload(hw_h, s);
    hin_slen.upload(hsl_h, s);
    hin_srest.upload(hsr_h, s);
    vt_off.upload(vto, s);
    vt_list.upload(vtl, s);
    vh_off.upload(vho, s);
    vh_list.upload(vhl, s);
    mh2.upload(mh2_h, s);
    hdiag.upload(hdiag_h, s);
    is_free.upload(freev, s);
    ell_col.upload(ecol, s);
    {  // 16-bit column offsets for the sweeps when the matrix bandwidth allows
        std::vector<short> dcol(ecol.size());
        bool fits = true;
        for (size_t k = 0; k < ecol.size() && fits; ++k) {
            long long d = (long long)ecol[k] - (long long)(k % (size_t)n);
            fits = d >= -32768 && d <= 32767;
            dcol[k] = (short)d;
        }
        if (fits && !dcol.empty()) ell_dcol.upload(dcol, s);
        else ell_dcol.release();
        // per-block tiles of the same entries for the Chebyshev steps
        ell_tw = ell_w <= 8 ? 8 : ell_w <= 12 ? 12 : 16;
        if (fits && ell_w > 0 && ell_w <= 16) {
            const size_t nb = ((size_t)n + ELL_TILE_ROWS - 1) / ELL_TILE_ROWS, tb = ell_tile_bytes(ell_tw);
            std::vector<unsigned char> tiles(nb * tb, 0);
            for (size_t b = 0; b < nb; ++b) {
                float *tv = reinterpret_cast<float *>(tiles.data() + b * tb);
                short *td = reinterpret_cast<short *>(tiles.data() + b * tb + (size_t)ell_tw * ELL_TILE_ROWS * 4);
                for (int k = 0; k < ell_w; ++k)
                    for (int t = 0; t < ELL_TILE_ROWS; ++t) {
                        size_t i = b * ELL_TILE_ROWS + t;
                        if (i >= (size_t)n) break;
                        tv[k * ELL_TILE_ROWS + t] = evalv[(size_t)k * n + i];
                        td[k * ELL_TILE_ROWS + t] = dcol[(size_t)k * n + i];
                    }
            }
            ell_tile.upload(tiles, s);
            build_patch_tiles(ecol, evalv);
            build_patch_tiles2(ecol, evalv);
        } else {
            ell_tile.release();
            ell_halo.release();
            ell_halo2.release();
        }
    }
    ell_val.upload(evalv, s);
    pins_d.upload(pins, s);
    std::vector<float4> pt(npins);
    for (int k = 0; k < npins; ++k) pt[k] = make_float4(X[3 * pins[k]], X[3 * pins[k] + 1], X[3 * pins[k] + 2], 0.f);
    pin_tgt.upload(pt, s);
    if (npins == 0) pin_tgt.alloc(1);

    R.alloc(n);
    RL.alloc(n);
    Xacc.alloc(n);
    Ucur.alloc(n);
    Um.alloc(n);
    Ulast.alloc(n);
    Ulast.zero(s);
    if (P.sweep_kind == 1) {
        CD0.alloc(n);
        CD1.alloc(n);

    }
    if (P.accel == 2) {
        int m = std::min(std::max(P.aa_depth, 1), 8);
        aa_dF.alloc((size_t)m * n);
        aa_dG.alloc((size_t)m * n);
        aa_f.alloc(n);
        aa_g.alloc(n);
        aa_Gb.alloc(64);
        aa_theta.alloc(8);
    }
    D0.alloc(n);
    D1.alloc(n);
    CF.alloc(n);
    CW.alloc(n);
    Z.alloc(n);
    Vs.alloc(n);
    Vs.zero(s);
    stage3.alloc(3 * (size_t)std::max(n, 1));
    sc.alloc(1);
    PDC_CK(cudaHostAlloc((void **)&hsc, sizeof(Scalars), cudaHostAllocDefault));
    sfrac.alloc(1);
    ttoi.alloc(1);
    toi_bits.alloc(1);
    n_act_d.alloc(1);
    bp_ovf.alloc(1);
    n_cv_d.alloc(1);
    bad_d.alloc(1);
    umax_d.alloc(1);
    sflag.alloc(1);
    sflag.zero(s);
    ctl.alloc(1);
    ctl.zero(s);
    n_cv_d.zero(s);
    n_act_d.zero(s);
    contact_list.alloc(std::max(n, 1));
    // cloth-only collision arrays until obstacles are added
    ensure_topology();
    std::vector<float4> x4(n);
    for (int i = 0; i < n; ++i) x4[i] = make_float4(X[3 * i], X[3 * i + 1], X[3 * i + 2], 0.f);
    PDC_CK(cudaMemcpyAsync(Xs.p, x4.data(), sizeof(float4) * n, cudaMemcpyHostToDevice, s));
    PDC_CK(cudaStreamSynchronize(s));
}

void pdc_ctx::install_basis(const std::vector<float> &U, int r) {
    ++graph_gen;  // new basis buffers
    r_warm = r;
    r_reuse = std::min(std::max(P.r_reuse, 0), r);
    if (r_reuse > R_REUSE_MAX) throw Error(PDC_ERR_ARG, "r_reuse must be <= 512");
    if (r > 1024) throw Error(PDC_ERR_ARG, "basis size must be <= 1024");
    // rows padded to a multiple of 8 columns: 16-byte aligned vector loads
    ld = (r + 7) / 8 * 8;
    std::vector<float> Uz((size_t)n * ld, 0.f);
    for (int i = 0; i < n; ++i)
        if (freev[i])
            for (int j = 0; j < r; ++j) Uz[(size_t)i * ld + j] = U[(size_t)i * r + j];
    // mixed forms: round to 16 bits; everything downstream (reduced matrix,
    // SYRK, projections) uses the rounded basis.  BF16 as is; FP16 after
    // scaling by the power of two that puts the largest entry in [2^13, 2^14)
    // (the scale cancels: U^T H U scales by s^2, U^T r by s, q by 1/s).
    const bool half16 = P.precision == 2;
    std::vector<uint16_t> ub;
    if (P.precision != 0) {
        float scale = 1.f;
        if (half16) {
            float mx = 0.f;
            for (float v : Uz) mx = std::max(mx, std::fabs(v));
            int e = 0;
            if (mx > 0.f) std::frexp(mx, &e);
            scale = std::ldexp(1.f, 14 - e);
        }
        ub.resize(Uz.size());
        for (size_t k = 0; k < Uz.size(); ++k) {
            float v = Uz[k] * scale;
            if (half16) {
                __half h = __float2half_rn(v);
                std::memcpy(&ub[k], &h, 2);
                Uz[k] = __half2float(h);
            } else {
                __nv_bfloat16 h = __float2bfloat16_rn(v);
                std::memcpy(&ub[k], &h, 2);
                Uz[k] = __bfloat162float(h);
            }
        }
        U16bits.upload(ub, s);
        // transposed copy and TMA descriptors for the tensor-core kernels
        umma.ok = false;
        if (umma_supported(ld, n)) {
            n_pad = (n + 63) / 64 * 64;
            std::vector<uint16_t> ut((size_t)ld * n_pad, 0);
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < ld; ++j) ut[(size_t)j * n_pad + i] = ub[(size_t)i * ld + j];
            Ut16.upload(ut, s);
            umma_setup(umma, U16bits, Ut16, half16, n, n_pad, ld);
            umma_partial.alloc((size_t)umma_project_blocks(n) * ld * 3);
        } else {
            Ut16.release();
        }
    } else {
        U16bits.release();
        Ut16.release();
        umma.ok = false;
    }
    U32.upload(Uz, s);
    // compact copy of the leading columns for the solves with collision
    // springs: width a power of two in [8, 128] holding r_reuse columns
    // (wider reuse bases stream the full basis)
    ldc = 0;
    Uc32.release();
    Uc16bits.release();
    if (r_reuse > 0 && r_reuse <= CHOL_ONE_CTA) {
        ldc = 8;
        while (ldc < r_reuse) ldc *= 2;
        if (P.precision != 0) {
            std::vector<uint16_t> uc((size_t)n * ldc, 0);
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < std::min(ldc, ld); ++j) uc[(size_t)i * ldc + j] = ub[(size_t)i * ld + j];
            Uc16bits.upload(uc, s);
        } else {
            std::vector<float> Uc((size_t)n * ldc, 0.f);
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < std::min(ldc, ld); ++j) Uc[(size_t)i * ldc + j] = Uz[(size_t)i * ld + j];
            Uc32.upload(Uc, s);
        }
    }
    std::vector<double> A0h;  // [ld][ld], zero padding rows / columns
    reduced_matrix(s, cloth(), U32, ld, A0h);
    std::vector<double> A0r((size_t)r * r), Ainv;
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < r; ++j) A0r[(size_t)i * r + j] = A0h[(size_t)i * ld + j];
    spd_inverse(A0r, r, Ainv);
    A0.upload(A0h, s);
    A0inv.upload(Ainv, s);
    std::vector<float> Ainv32(Ainv.begin(), Ainv.end());
    A0inv32.upload(Ainv32, s);
    proj_partial.alloc((size_t)PROJ_BLOCKS * ld * 3);
    gbuf.alloc((size_t)ld * 3);
    qbuf.alloc((size_t)ld * 3);
    dA.alloc(dA_elems(r_reuse));
    PDC_CK(cudaStreamSynchronize(s));
}

void pdc_ctx::setup_basis() {
    int r = std::min(P.r_warm, (int)std::count(freev.begin(), freev.end(), 1));
    if (r <= 0) {
        r_warm = r_reuse = 0;
        return;
    }
    std::vector<float> U;
    std::vector<double> ritz;
    build_basis(s, cloth(), r, std::max(P.eig_iters, 0), P.seed, U, ritz);
    install_basis(U, (int)(U.size() / n));
}

void pdc_ctx::ensure_topology() {
    if (!topo_dirty) return;
    ++graph_gen;  // collision-set buffers reallocated
    int nvo = 0, nto = 0;
    for (auto &o : obs) {
        nvo += (int)o.V.size() / 3;
        nto += (int)o.T.size() / 3;
    }
    int nv_new = n + nvo;
    // grow the collision-vertex state arrays, keeping the cloth part
    auto grow = [&](DevBuf<float4> &b) {
        DevBuf<float4> nbuf;
        nbuf.alloc(nv_new);
        nbuf.zero(s);
        if (b.p) PDC_CK(cudaMemcpyAsync(nbuf.p, b.p, sizeof(float4) * std::min<size_t>(b.n, n), cudaMemcpyDeviceToDevice, s));
        std::swap(b.p, nbuf.p);
        std::swap(b.n, nbuf.n);
    };
    grow(Xs);
    grow(Xp);
    grow(Xm);
    grow(Xbak);
    grow(Xprev);
    Vbak.alloc(n);
    nv_all = nv_new;
    // obstacle rest / current / target positions
    std::vector<float4> orest;
    for (auto &o : obs)
        for (size_t k = 0; k < o.V.size() / 3; ++k) orest.push_back(make_float4(o.V[3 * k], o.V[3 * k + 1], o.V[3 * k + 2], 0.f));
    if (!orest.empty()) {
        obs_rest.upload(orest, s);
        if (obs_tgt.n != orest.size()) obs_tgt.upload(orest, s);
        PDC_CK(cudaMemcpyAsync(Xs.p + n, orest.data(), sizeof(float4) * nvo, cudaMemcpyHostToDevice, s));
    }
    // triangles and edges of the collision set
    ctri_h.clear();
    std::vector<int4> ct;
    for (int t = 0; t < m; ++t) ct.push_back(make_int4(T[3 * t], T[3 * t + 1], T[3 * t + 2], 0));
    for (auto &o : obs)
        for (size_t t = 0; t < o.T.size() / 3; ++t)
            ct.push_back(make_int4(o.T[3 * t] + o.off, o.T[3 * t + 1] + o.off, o.T[3 * t + 2] + o.off, 0));
    nt_all = (int)ct.size();
    std::vector<std::pair<int, int>> ed;
    ed.reserve(ct.size() * 3);
    for (auto &q : ct) {
        int v[3] = {q.x, q.y, q.z};
        for (int k = 0; k < 3; ++k) ed.push_back({std::min(v[k], v[(k + 1) % 3]), std::max(v[k], v[(k + 1) % 3])});
    }
    std::sort(ed.begin(), ed.end());
    ed.erase(std::unique(ed.begin(), ed.end()), ed.end());
    std::vector<int2> ce(ed.size());
    for (size_t k = 0; k < ed.size(); ++k) ce[k] = make_int2(ed[k].first, ed[k].second);
    ne_all = (int)ce.size();
    ctri.upload(ct, s);
    cedge.upload(ce, s);
    std::vector<unsigned char> vf(nv_all, 1);
    for (int i = 0; i < n; ++i) vf[i] = freev[i] ? 0 : 1;
    vfixed.upload(vf, s);
    long long cvt = std::max<long long>(1024, 16LL * nv_all), cee = std::max<long long>(1024, 24LL * ne_all);
    long long cent = std::max<long long>(4096, 8LL * ((long long)nv_all + nt_all + ne_all));
    if (bp_cap0 > 0) cvt = cee = bp_cap0;
    if (!guard_d.p) {
        guard_d.alloc(1);
        guard_d.zero(s);
    }
    bp.reserve(coll(), cvt, cee, cent, s);
    cap_act = (int)std::max<long long>(1024, 4LL * nv_all);
    disp.alloc(nv_all);
    act.alloc(cap_act);
    obs_inst.resize(obs.size(), -1);
    upload_vinst();
    PDC_CK(cudaStreamSynchronize(s));
    topo_dirty = false;
}

void pdc_ctx::upload_vinst() {
    if (ninst() < 2) return;
    std::vector<int> vi(std::max(nv_all, 1), -1);
    for (int k = 0; k < ninst(); ++k)
        for (int v = inst_off[k]; v < inst_off[k + 1]; ++v) vi[v] = k;
    for (size_t j = 0; j < obs.size(); ++j) {
        const int nvo = (int)obs[j].V.size() / 3;
        for (int v = 0; v < nvo; ++v) vi[obs[j].off + v] = obs_inst[j];
    }
    vinst.upload(vi, s);
    toi_inst.alloc(ninst());
    sfrac_inst.alloc(ninst());
    PDC_CK(cudaStreamSynchronize(s));
}

// ============================================================================ autotuning
// Launch shapes of the hot kernels picked at the first step (autotune = 1):
// each candidate runs on this handle's own data and its time is taken with
// CUDA events; the fastest is kept.  Every candidate computes the same
// values (up to the order of float atomics), so the choice changes speed
// only.  Here: the block size of the element-force and residual kernels and
// the Chebyshev step's matrix source; the pair kernels' grid and the VT
// query's lanes per vertex are tuned at the first full CCD / broad phase.
// Patch tiles for the Chebyshev step: the rows are cut into the mesh patches
// (morton_order), ids ascending within a patch; each patch lists the other
// vertices its rows reference (its halo) and stores its rows' off-diagonals,
// in the order of the ELL arrays, with columns local to rows + halo.  Not
// built (the row tiles serve) when some patch's halo exceeds HALO_MAX.
// Vertices in the Morton order of their rest positions (10 bits per axis, one
// scale for all three axes, so a flat sheet's jitter does not decide the
// order); consecutive runs of ELL_TILE_ROWS are the mesh patches.
std::vector<int> pdc_ctx::morton_order() const {
    std::vector<int> order(n);
    if (n == 0) return order;
    float lo[3] = {X[0], X[1], X[2]}, hi[3] = {X[0], X[1], X[2]};
    for (int i = 0; i < n; ++i)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], X[3 * (size_t)i + d]);
            hi[d] = std::max(hi[d], X[3 * (size_t)i + d]);
        }
    double ext = std::max({(double)hi[0] - lo[0], (double)hi[1] - lo[1], (double)hi[2] - lo[2], 1e-30});
    std::vector<std::pair<unsigned long long, int>> key(n);
    for (int i = 0; i < n; ++i) {
        unsigned long long code = 0;
        unsigned q[3];
        for (int d = 0; d < 3; ++d)
            q[d] = (unsigned)std::min(1023.0, std::max(0.0, ((double)X[3 * (size_t)i + d] - lo[d]) / ext * 1023.0));
        for (int b = 0; b < 10; ++b)
            for (int d = 0; d < 3; ++d) code |= (unsigned long long)((q[d] >> b) & 1u) << (3 * b + d);
        key[i] = {code, i};
    }
    std::sort(key.begin(), key.end());
    for (int i = 0; i < n; ++i) order[i] = key[i].second;
    return order;
}

// Records for the one-kernel residual: per mesh patch, the vertices it
// touches (its own rows first, then the other vertices of the elements at
// them), the triangles and hinges at its rows with their vertices as local
// indices, and each row's incidences as local element indices in the order
// of the global incidence lists (so the residual sums the same terms in the
// same order as the two-kernel form).  Sections 16-byte aligned:
// int4 {n_loc, n_tri, n_hin, n_own}; int vid[n_loc]; int tri[n_tri];
// int2 tri_loc[n_tri] (a | b << 16, c); int hin[n_hin]; int2 hin_loc[n_hin]
// (a | b << 16, c | d << 16); int vt_off[n_own + 1], vt_ent[]; int
// vh_off[n_own + 1], vh_ent[] (entries: local element << 2 | corner).  Not
// built when a patch would need more than 96 KB of shared memory.
void pdc_ctx::build_residual_patches(const std::vector<int> &vto, const std::vector<int> &vtl,
                                     const std::vector<int> &vho, const std::vector<int> &vhl,
                                     const std::vector<int4> &tri_h, const std::vector<int4> &hin_h) {
    rp_rec.release();
    rp_off.release();
    rp_loc = rp_tri = rp_hin = 0;
    if (n == 0) return;
    const std::vector<int> order = morton_order();
    const int R = ELL_TILE_ROWS;
    const size_t nb = ((size_t)n + R - 1) / R;
    std::vector<unsigned char> rec;
    std::vector<long long> off(nb + 1, 0);
    std::vector<int> vloc(n, -1), tloc(m, -1), hloc(nh, -1);
    std::vector<int> own, verts, tris, hins;
    auto put = [&](const void *p, size_t bytes) {
        const unsigned char *q = static_cast<const unsigned char *>(p);
        rec.insert(rec.end(), q, q + bytes);
        while (rec.size() % 16) rec.push_back(0);
    };
    for (size_t b = 0; b < nb; ++b) {
        off[b] = (long long)rec.size();
        own.assign(order.begin() + b * R, order.begin() + std::min((size_t)n, (b + 1) * R));
        std::sort(own.begin(), own.end());
        verts = own;
        for (int k = 0; k < (int)own.size(); ++k) vloc[own[k]] = k;
        tris.clear();
        hins.clear();
        for (int v : own) {
            for (int e = vto[v]; e < vto[v + 1]; ++e)
                if (tloc[vtl[e] >> 2] < 0) {
                    tloc[vtl[e] >> 2] = (int)tris.size();
                    tris.push_back(vtl[e] >> 2);
                }
            for (int e = vho[v]; e < vho[v + 1]; ++e)
                if (hloc[vhl[e] >> 2] < 0) {
                    hloc[vhl[e] >> 2] = (int)hins.size();
                    hins.push_back(vhl[e] >> 2);
                }
        }
        auto local = [&](int g) {
            if (vloc[g] < 0) {
                vloc[g] = (int)verts.size();
                verts.push_back(g);
            }
            return vloc[g];
        };
        std::vector<int2> tl(tris.size()), hl(hins.size());
        for (size_t k = 0; k < tris.size(); ++k) {
            const int4 T = tri_h[tris[k]];
            const int a = local(T.x), bb = local(T.y), cc = local(T.z);
            tl[k] = make_int2(a | (bb << 16), cc);
        }
        for (size_t k = 0; k < hins.size(); ++k) {
            const int4 Hh = hin_h[hins[k]];
            const int a = local(Hh.x), bb = local(Hh.y), cc = local(Hh.z), dd = local(Hh.w);
            hl[k] = make_int2(a | (bb << 16), cc | (dd << 16));
        }
        std::vector<int> vt_o(own.size() + 1, 0), vt_e, vh_o(own.size() + 1, 0), vh_e;
        for (size_t k = 0; k < own.size(); ++k) {
            const int v = own[k];
            for (int e = vto[v]; e < vto[v + 1]; ++e) vt_e.push_back((tloc[vtl[e] >> 2] << 2) | (vtl[e] & 3));
            for (int e = vho[v]; e < vho[v + 1]; ++e) vh_e.push_back((hloc[vhl[e] >> 2] << 2) | (vhl[e] & 3));
            vt_o[k + 1] = (int)vt_e.size();
            vh_o[k + 1] = (int)vh_e.size();
        }
        const bool fits = verts.size() < 65536;
        const int hd[4] = {(int)verts.size(), (int)tris.size(), (int)hins.size(), (int)own.size()};
        put(hd, sizeof(hd));
        put(verts.data(), 4 * verts.size());
        put(tris.data(), 4 * tris.size());
        put(tl.data(), 8 * tl.size());
        put(hins.data(), 4 * hins.size());
        put(hl.data(), 8 * hl.size());
        put(vt_o.data(), 4 * vt_o.size());
        put(vt_e.data(), 4 * vt_e.size());
        put(vh_o.data(), 4 * vh_o.size());
        put(vh_e.data(), 4 * vh_e.size());
        rp_loc = std::max(rp_loc, hd[0]);
        rp_tri = std::max(rp_tri, hd[1]);
        rp_hin = std::max(rp_hin, hd[2]);
        for (int v : verts) vloc[v] = -1;
        for (int t : tris) tloc[t] = -1;
        for (int h : hins) hloc[h] = -1;
        if (!fits) {
            rp_loc = rp_tri = rp_hin = 0;
            return;
        }
    }
    off[nb] = (long long)rec.size();
    if (residual_patch_smem() > 96 * 1024) {
        rp_loc = rp_tri = rp_hin = 0;
        return;
    }
    rp_rec.upload(rec, s);
    rp_off.upload(off, s);
}

// Records for the two-step Chebyshev kernel: per mesh patch, its rows are the
// patch's own vertices and their ELL neighbours (first ring), its vertices
// those rows and their neighbours (second ring); columns local to the
// vertices, entries in the order of the ELL arrays.  Not built when a patch
// exceeds 512 rows or 1024 vertices.
void pdc_ctx::build_patch_tiles2(const std::vector<int> &ecol, const std::vector<float> &evalv) {
    ell_halo2.release();
    h2_rows = h2_verts = 0;
    if (n == 0 || ell_w == 0) return;
    const std::vector<int> order = morton_order();
    const int R = ELL_TILE_ROWS, tw = ell_tw;
    const size_t nb = ((size_t)n + R - 1) / R;
    std::vector<int> loc(n, -1);
    std::vector<std::vector<int>> verts(nb);
    std::vector<int> nown(nb), nrows(nb);
    for (size_t b = 0; b < nb; ++b) {
        std::vector<int> &V = verts[b];
        V.assign(order.begin() + b * R, order.begin() + std::min((size_t)n, (b + 1) * R));
        std::sort(V.begin(), V.end());
        nown[b] = (int)V.size();
        for (int k = 0; k < (int)V.size(); ++k) loc[V[k]] = k;
        auto ring = [&](int from, int to) {  // neighbours of V[from, to) not yet listed
            for (int r = from; r < to; ++r)
                for (int k = 0; k < ell_w; ++k) {
                    const int col = ecol[(size_t)k * n + V[r]];
                    if (loc[col] < 0) {
                        loc[col] = (int)V.size();
                        V.push_back(col);
                    }
                }
        };
        ring(0, nown[b]);
        nrows[b] = (int)V.size();
        ring(nown[b], nrows[b]);
        for (int v : V) loc[v] = -1;
        h2_rows = std::max(h2_rows, nrows[b]);
        h2_verts = std::max(h2_verts, (int)V.size());
    }
    h2_rows = (h2_rows + 31) & ~31;
    h2_verts = (h2_verts + 31) & ~31;
    if (h2_rows > 512 || h2_verts > 1024) {
        h2_rows = h2_verts = 0;
        return;
    }
    const size_t rb = halo2_tile_bytes(tw, h2_rows, h2_verts);
    std::vector<unsigned char> rec(nb * rb, 0);
    for (size_t b = 0; b < nb; ++b) {
        const std::vector<int> &V = verts[b];
        for (int k = 0; k < (int)V.size(); ++k) loc[V[k]] = k;
        unsigned char *p = rec.data() + b * rb;
        int *hd = reinterpret_cast<int *>(p);
        hd[0] = nown[b];
        hd[1] = nrows[b];
        hd[2] = (int)V.size();
        float *tv = reinterpret_cast<float *>(p + 16);
        short *tc = reinterpret_cast<short *>(p + 16 + (size_t)tw * h2_rows * 4);
        int *gid = reinterpret_cast<int *>(p + 16 + (size_t)tw * h2_rows * 6);
        for (int r = 0; r < nrows[b]; ++r)
            for (int k = 0; k < ell_w; ++k) {
                tv[k * h2_rows + r] = evalv[(size_t)k * n + V[r]];
                tc[k * h2_rows + r] = (short)loc[ecol[(size_t)k * n + V[r]]];
            }
        for (int k = 0; k < h2_verts; ++k) gid[k] = k < (int)V.size() ? V[k] : -1;
        for (int v : V) loc[v] = -1;
    }
    ell_halo2.upload(rec, s);
}

void pdc_ctx::build_patch_tiles(const std::vector<int> &ecol, const std::vector<float> &evalv) {
    ell_halo.release();
    if (n == 0 || ell_w == 0) return;
    const std::vector<int> order = morton_order();
    const int R = ELL_TILE_ROWS, tw = ell_tw;
    const size_t nb = ((size_t)n + R - 1) / R, rb = halo_tile_bytes(tw);
    std::vector<unsigned char> rec(nb * rb, 0);
    std::vector<int> loc(n, -1), own, halo;
    for (size_t b = 0; b < nb; ++b) {
        own.clear();
        halo.clear();
        for (size_t j = b * R; j < std::min((size_t)n, (b + 1) * R); ++j) own.push_back(order[j]);
        std::sort(own.begin(), own.end());
        for (int t = 0; t < (int)own.size(); ++t) loc[own[t]] = t;
        bool ok = true;
        for (int t = 0; t < (int)own.size() && ok; ++t)
            for (int k = 0; k < ell_w && ok; ++k) {
                const int col = ecol[(size_t)k * n + own[t]];
                if (loc[col] >= 0) continue;
                if ((int)halo.size() == HALO_MAX) ok = false;
                else {
                    loc[col] = R + (int)halo.size();
                    halo.push_back(col);
                }
            }
        if (ok) {
            unsigned char *p = rec.data() + b * rb;
            float *tv = reinterpret_cast<float *>(p);
            short *tc = reinterpret_cast<short *>(p + (size_t)tw * R * 4);
            int *gid = reinterpret_cast<int *>(p + (size_t)tw * R * 6);
            int *hid = gid + R;
            for (int t = 0; t < R; ++t) gid[t] = t < (int)own.size() ? own[t] : -1;
            for (int t = 0; t < (int)own.size(); ++t)
                for (int k = 0; k < ell_w; ++k) {
                    tv[k * R + t] = evalv[(size_t)k * n + own[t]];
                    tc[k * R + t] = (short)loc[ecol[(size_t)k * n + own[t]]];
                }
            for (int h = 0; h < (int)halo.size(); ++h) hid[h] = halo[h];
            hid[HALO_MAX] = (int)halo.size();
        }
        for (int v : own) loc[v] = -1;
        for (int v : halo) loc[v] = -1;
        if (!ok) return;
    }
    ell_halo.upload(rec, s);
}

void pdc_ctx::autotune_vertex_kernels() {
    cudaEvent_t e0, e1;
    PDC_CK(cudaEventCreate(&e0));
    PDC_CK(cudaEventCreate(&e1));
    auto timed = [&](auto &&f) {
        f();  // warm-up
        PDC_CK(cudaEventRecord(e0, s));
        for (int k = 0; k < 3; ++k) f();
        PDC_CK(cudaEventRecord(e1, s));
        PDC_CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        PDC_CK(cudaEventElapsedTime(&ms, e0, e1));
        return ms / 3.f;
    };
    const int bsz[3] = {64, 128, 256};
    for (int k = 0; k < 3; ++k) {
        tune.residual_block = bsz[k];
        ClothView c = cloth();
        tune.residual_ms[k] = timed([&] { launch_residual(s, c, Xs, Ucur, Z, nullptr, nullptr, R, nullptr, nullptr, 0); });
    }
    int best = 0;  // the fastest, once all are timed
    for (int k = 1; k < 3; ++k)
        if (tune.residual_ms[k] < tune.residual_ms[best]) best = k;
    tune.residual_block = bsz[best];
    if (P.sweep_kind == 1 && ell_tile.p && P.cheb_source < 0) {
        // Chebyshev steps from delta = 0 on the residual just formed (scratch outputs)
        PDC_CK(cudaMemsetAsync(D0.p, 0, sizeof(float4) * n, s));
        double b = std::max(gersh, 1.0) * 1.02, a = b / std::max(P.cheb_ratio, 1.0001);
        const float beta = (float)(2.0 / (b + a));
        const int modes[4] = {1, 0, 2, 3};  // row tiles, ELL arrays, patch tiles, two-step patch tiles
        const int nm = ell_halo2.p ? 4 : ell_halo.p ? 3 : 2;
        for (int k = 0; k < nm; ++k) {
            tune.cheb_tile = modes[k];
            ClothView c = cloth();
            // eight steps back to back, launched as in the LG iteration
            tune.cheb_ms[k] = timed([&] {
                if (modes[k] == 3)
                    for (int rep = 0; rep < 4; ++rep)
                        launch_cheb_step2(s, c, nullptr, R, D0, CD0, D1, CD1, 0.f, beta, 0.f, beta, nullptr, nullptr,
                                          nullptr, nullptr, 1.f, Xs, nullptr, P.launch_overlap != 0, sflag.p);
                else
                    for (int rep = 0; rep < 8; ++rep)
                        launch_cheb_step(s, c, nullptr, R, D0, CD0, D1, 0.f, beta, nullptr, nullptr, nullptr, nullptr,
                                         1.f, Xs, nullptr, P.launch_overlap != 0, sflag.p);
            }) / 8.f;
        }
        int best = 0;  // the fastest, once all are timed
        for (int k = 1; k < nm; ++k)
            if (tune.cheb_ms[k] < tune.cheb_ms[best]) best = k;
        tune.cheb_tile = modes[best];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    bp.tune_pairs = bp.tune_cells = P.collisions != 0;
    ++graph_gen;  // graphs capture launch shapes
}

// ============================================================================ the step (Alg. 1)
// An LG iteration in two parts, enqueued on s: the residual part (contact
// springs of the active pairs and the local projections + residual at the
// iterate, Eq. local / Eq. global), and the solve part (`cycles` x {subspace
// correction, `sweeps` Jacobi or Chebyshev steps}, the iterate += delta, LG
// acceleration, then with contacts the partial CCD of Sec. 4.1 on (Xm, Xp)).
// The host-driven loop (lg_iteration) takes its stopping tests between the
// two on the host; the device-driven loop (run_loop) in k_loop_decide.
void pdc_ctx::enqueue_residual(bool contacts) {
    ClothView c = cloth();
    {
        IterZero z;
        z.rsq = &sc.p->rsq;
        z.dxmax = device_decides ? nullptr : &sc.p->dxmax;
        z.ncv = n_cv_d.p;
        z.cw = CW.p;
        z.cf = CF.p;
        z.n = contacts ? n : 0;
        const bool aa = accel.on && P.fixed_iters == 0 && P.accel == 2;
        z.gb = aa_Gb.p;
        z.ngb = aa ? aa_gram_doubles() : 0;
        z.da = dA.p;
        z.nda = contacts ? (int)dA_zero_elems(r_reuse) : 0;
        const int blocks = contacts ? std::min(nb(n), 152 * 4) : 1;
        launch_dependent(P.launch_overlap != 0, k_iter_begin, blocks, 256, 0, s, z, live_ptr);
    }
    const float *cw = nullptr;
    const float4 *cf = nullptr;
    if (contacts) {
        PROF("contact_springs", 0, launch_contact(s, coll(), act, n_act_d, cap_act, Xp, dhat, CW, CF));
        launch_contact_list(s, n, CW, contact_list, n_cv_d, live_ptr, false);
        cw = CW;
        cf = CF;
    }
    PROF("local_residual", bytes_residual(contacts), launch_residual(s, c, Xs, Ucur, Z, cw, cf, R, sc, nullptr, 0));
}

// springs: whether the iteration has collision springs when the host knows
// it (host-driven loop); device: the device decides (the tensor-core /
// compact path, the Anderson bookkeeping) and the host knows only whether
// springs are possible (contacts).
void pdc_ctx::enqueue_solve(bool contacts, bool springs, bool device, float w_acc, int r_nc, int r_c, int cycles,
                            int sweeps, bool pccd) {
    ClothView c = cloth();
    const float *cw = contacts ? CW.p : nullptr;
    // the accumulators of this solve (step-change maximum, Anderson normal
    // equations, reduced-matrix update) were zeroed by the residual part
    const bool acc = accel.on && P.fixed_iters == 0;
    const bool aa = acc && P.accel == 2;
    float4 *xprev = (acc && !aa && !device) ? Xacc.p : nullptr;
    const bool sp = device ? contacts : springs;  // springs possible on this path
    SubspaceView S = sub(r_nc, r_c);
    SubspaceWork W = work();
    float4 *din = D0, *dout = D1;
    bool have_delta = false;
    for (int cyc = 0; cyc < cycles; ++cyc) {
        const float4 *rl = R;
        if (have_delta) {
            PROF("linear_residual", bytes_sweep(contacts, false), launch_linear_residual(s, c, cw, R, din, RL));
            rl = RL;
        }
        if (r_warm > 0 && (r_nc > 0 || r_c > 0)) {
            PROF("subspace_project", bytes_basis(springs ? r_c : r_nc),
                 launch_project(s, S, rl, n_cv_d, W, sp, device));
            // the spring weights and the basis are fixed within a solve: the
            // reduced matrix is updated (and factored) in its first cycle
            if (sp && r_c > 0 && cyc == 0)
                PROF("subspace_syrk", 0, launch_syrk(s, S, contact_list, n_cv_d, cw, W, false));
            PROF("reduced_solve", 0, launch_reduced_solve(s, S, n_cv_d, W, cyc == 0));
            PROF("subspace_lift", bytes_basis(springs ? r_c : r_nc) + 12.0 * n,
                 launch_lift(s, S, n_cv_d, W, have_delta ? din : nullptr, dout, sp, device));
            std::swap(din, dout);
            have_delta = true;
        }
        if (!have_delta) {
            launch_live_zero(s, live_ptr, din, sizeof(float4) * n);
            have_delta = true;
        }
        if (P.sweep_kind == 1) {
            // Chebyshev iteration on the interval [b / ratio, b] of the spectrum of D^-1 A
            double b = std::max(gersh, 1.0) * 1.02, a = b / std::max(P.cheb_ratio, 1.0001);
            double theta = 0.5 * (b + a), dl = 0.5 * (b - a), sig = theta / dl;
            double rho_prev = 1.0 / sig;
            // delta_{k-1}: the one of the three buffers that is neither din nor dout
            float4 *dp = (CD0.p != din && CD0.p != dout) ? CD0.p : (D0.p != din && D0.p != dout) ? D0.p : D1.p;
            auto coef = [&](int k, double &alpha, double &beta) {  // in step order
                if (k == 0) {
                    alpha = 0.0;
                    beta = 1.0 / theta;
                } else {
                    double rk = 1.0 / (2.0 * sig - rho_prev);
                    alpha = rk * rho_prev;
                    beta = 2.0 * rk / dl;
                    rho_prev = rk;
                }
            };
            // the steps run back to back (each a programmatic dependent of the
            // one before) and are timed as one run between two events
            if (prof.on && sweeps > 0)
                prof.begin(s, "cheb_sweep",
                           (sweeps - 1) * bytes_sweep(contacts, false) + bytes_sweep(contacts, cyc == cycles - 1) +
                               12.0 * n * sweeps,
                           sweeps);
            int k0 = 0;
            if (cheb_two_steps(c) && sweeps >= 2) {
                // pairs of steps: delta_k, delta_{k-1} in, delta_{k+1}, delta_{k+2}
                // out (a fourth buffer, since other blocks still read the
                // inputs while the outputs are written)
                float4 *q = nullptr;  // the buffer that is none of din, dp, dout
                for (float4 *cand : {D0.p, D1.p, CD0.p, CD1.p})
                    if (cand != din && cand != dp && cand != dout) q = cand;
                for (; k0 + 1 < sweeps; k0 += 2) {
                    const bool last = (cyc == cycles - 1) && (k0 + 1 == sweeps - 1);
                    double a1, b1, a2, b2;
                    coef(k0, a1, b1);
                    coef(k0 + 1, a2, b2);
                    launch_cheb_step2(s, c, cw, R, din, dp, dout, q, (float)a1, (float)b1, (float)a2, (float)b2, Ucur,
                                      last ? Ucur.p : nullptr, last ? sc.p : nullptr, last ? xprev : nullptr, w_acc,
                                      Xs, last ? Xp.p : nullptr, P.launch_overlap != 0, sflag.p);
                    float4 *a = din, *b = dp;  // delta_{k+2}, delta_{k+1} become the inputs
                    din = q;
                    dp = dout;
                    dout = a;
                    q = b;
                }
            }
            for (int k = k0; k < sweeps; ++k) {
                bool last = (cyc == cycles - 1) && (k == sweeps - 1);
                double alpha, beta;
                coef(k, alpha, beta);
                launch_cheb_step(s, c, cw, R, din, dp, dout, (float)alpha, (float)beta, Ucur, last ? Ucur.p : nullptr,
                                 last ? sc.p : nullptr, last ? xprev : nullptr, w_acc, Xs, last ? Xp.p : nullptr,
                                 P.launch_overlap != 0, sflag.p);
                float4 *t = dp;  // rotate: delta_{k-1} <- delta_k <- delta_{k+1}
                dp = din;
                din = dout;
                dout = t;
            }
            if (prof.on && sweeps > 0) prof.end(s);
            if (sync_check && sweeps > 0) check_region("cheb_sweep");
        } else {
            for (int k = 0; k < sweeps; ++k) {
                bool last = (cyc == cycles - 1) && (k == sweeps - 1);
                PROF("jacobi_sweep", bytes_sweep(contacts, last),
                     launch_sweep(s, c, cw, R, din, dout, (float)omega, Ucur, last ? Ucur.p : nullptr,
                                  last ? sc.p : nullptr, last ? xprev : nullptr, w_acc, Xs, last ? Xp.p : nullptr));
                std::swap(din, dout);
            }
        }
        if (sweeps == 0 && cyc == cycles - 1) {
            // no sweep: apply the correction directly
            launch_sweep(s, c, cw, R, din, dout, 0.f, Ucur, Ucur.p, sc.p, xprev, w_acc, Xs, Xp.p);
        }
    }
    if (aa) {
        const int m = std::min(std::max(P.aa_depth, 1), 8);
        if (device) {
            PROF("anderson_mix", 0,
                 launch_aa_device(s, n, is_free, din, Ucur, aa_f, aa_g, aa_dF, aa_dG, m, ctl.p, aa_Gb, aa_theta, Xs,
                                  Xp, P.launch_overlap != 0));
        } else {
            int slot = 0;
            if (accel.aa_have_prev) {
                slot = accel.aa_widx % m;
                accel.aa_widx++;
                accel.aa_count = std::min(accel.aa_count + 1, m);
            }
            PROF("anderson_mix", 0,
                 launch_aa(s, n, is_free, din, Ucur, aa_f, aa_g, aa_dF, aa_dG, slot, accel.aa_have_prev ? 1 : 0,
                           accel.aa_count, aa_Gb, aa_theta, Xs, Xp, P.launch_overlap != 0));
            accel.aa_have_prev = true;
        }
    }
    if (contacts && P.collisions && pccd) {
        bp.prof = prof.on ? &prof : nullptr;
        PROF("partial_ccd", 0,
             launch_partial_ccd(s, coll(), bp, Xm, Xp, cparams(), act, cap_act, n_act_d, &sc.p->overflow, disp));
        if (log) {
            long long cnt[2] = {0, 0};
            PccdState ps;
            bp.cnt_vt_d[bp.cur].download(&cnt[0], 1, s);
            bp.cnt_ee_d[bp.cur].download(&cnt[1], 1, s);
            bp.pccd.download(&ps, 1, s);
            PDC_CK(cudaStreamSynchronize(s));
            std::fprintf(stderr, "[pdc] partial ccd: pairs vt=%lld ee=%lld, %s pass, watch %d, near %d\n", cnt[0],
                         cnt[1], ps.pass_full ? "full" : "watch-list", ps.n_watch, ps.n_near);
        }
    }
}

// One LG iteration driven by the host: the residual part, the stopping tests
// on the host (residual read back), then the solve part.
void pdc_ctx::lg_iteration(bool contacts, bool check_rel, double rho0, bool &converged, int r_nc, int r_c, int cycles,
                           int sweeps, bool pccd) {
    converged = false;
    enqueue_residual(contacts);
    bool acc = accel.on && !(P.fixed_iters != 0);
    bool aa = acc && P.accel == 2;
    // whether collision springs exist this iteration (device count); known on
    // the host when the residual is read back anyway
    bool springs = contacts;
    last_springs = contacts;
    if (check_rel || log || acc) {
        if (contacts) PDC_CK(cudaMemcpyAsync(&sc.p->n_contact_v, n_cv_d.p, sizeof(int), cudaMemcpyDeviceToDevice, s));
        read_scalars();
        if (contacts) springs = hsc->n_contact_v > 0;
        last_springs = springs;
        double rho = std::sqrt(hsc->rsq);
        if (log) {
            int na = 0, ncv = 0;
            n_act_d.download(&na, 1, s);
            n_cv_d.download(&ncv, 1, s);
            PDC_CK(cudaStreamSynchronize(s));
            std::fprintf(stderr, "[pdc] lg contacts=%d rho=%.6g rel=%.6g active=%d contact_v=%d\n", (int)contacts, rho,
                         rho / std::max(rho0, 1e-300), na, ncv);
        }
    }
    if (check_rel) {
        double rho = std::sqrt(hsc->rsq);
        st.rel_residual = rho / std::max(rho0, 1e-300);
        if (rho <= P.tol_rel_residual * rho0 || accel.stagnated(rho, springs)) {
            converged = true;
            return;
        }
    }
    if (springs) st.contact_iters++;
    float w_acc = 1.f;
    if (aa) accel.aa_observe(std::sqrt(hsc->rsq));
    else if (acc) w_acc = (float)accel.next(std::sqrt(hsc->rsq));
    if (log && acc && !aa) std::fprintf(stderr, "[pdc]    accel k=%d w=%.4f rho=%.4f\n", accel.k, w_acc, accel.rho);
    enqueue_solve(contacts, springs, false, w_acc, r_nc, r_c, cycles, sweeps, pccd);
}

// ---------------------------------------------------------------------------- LG loops as CUDA graphs
// A loop as one graph: k_loop_begin, the residual part and k_loop_decide,
// then a conditional while node whose body is {solve part, residual part,
// k_loop_decide}; k_loop_decide sets the while condition, so the loop runs
// on the device with no host round trip per iteration.  The graph captures
// buffer addresses and the list index bp.cur, so it is rebuilt when either
// changes (graph_gen counts reallocations).
bool pdc_ctx::device_loops_ok() const {
    if (P.loop_control == 0 || prof.on || log || sync_check) return false;
    if (P.loop_control == 1 && graphs_failed) return false;
    if (P.accel == 1 && P.fixed_iters == 0) return false;  // Chebyshev acceleration: host-side weights
    // a spring iteration of the mixed form chooses between the tensor-core and
    // the compact path on the device only when the compact copy covers r_reuse
    SubspaceView S = sub(r_warm, r_reuse);
    if (P.collisions && S.umma && r_warm > 0 && !device_path_choice(S)) return false;
    return true;
}

void pdc_ctx::free_graph(GraphLoop &G) {
    if (G.e) cudaGraphExecDestroy(G.e);
    if (G.g) cudaGraphDestroy(G.g);
    G.e = nullptr;
    G.g = nullptr;
}

LoopCfg pdc_ctx::loop_cfg(int kind, int max_iters, bool relmode, bool contacts) const {
    LoopCfg f;
    std::memset(&f, 0, sizeof(f));
    const bool fixed = P.fixed_iters != 0;
    f.kind = kind;
    f.max_iters = max_iters;
    f.check_rel = relmode ? 1 : 0;
    f.dx_inner = (!fixed && !relmode) ? 1 : 0;
    f.dx_springs = (contacts && relmode) ? 1 : 0;
    f.aa_m = (P.accel == 2 && !fixed) ? std::min(std::max(P.aa_depth, 1), 8) : 0;
    f.stag_n = Accel::STAG_N;
    f.tol_rel = P.tol_rel_residual;
    f.tolx_in = P.tol_inner * L;
    f.tolx_out = P.tol_outer * L;
    return f;
}

bool pdc_ctx::build_loop(GraphLoop &G, const LoopCfg &cfg0, bool contacts, int r_nc, int r_c, int cycles, int sweeps,
                         bool pccd) {
    free_graph(G);
    if (!gs) PDC_CK(cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking));
    cudaStream_t saved = s;
    s = gs;  // everything below is captured from the capture stream
    // unrolled: the captured iterations do nothing once the loop has ended (a
    // single iteration per pass always runs: the while node checked go)
    const int unroll = std::min(std::max(P.graph_unroll, 1), 8);
    live_ptr = unroll > 1 ? &ctl.p->go : nullptr;
    device_decides = true;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t e = nullptr;
    bool capturing = false;
    try {
        PDC_CK(cudaStreamBeginCapture(gs, cudaStreamCaptureModeRelaxed));
        capturing = true;
        cudaStreamCaptureStatus cst;
        cudaGraph_t cg = nullptr;
        PDC_CK(cudaStreamGetCaptureInfo(gs, &cst, nullptr, &cg, nullptr, nullptr, nullptr));
        cudaGraphConditionalHandle h;
        PDC_CK(cudaGraphConditionalHandleCreate(&h, cg, 0, cudaGraphCondAssignDefault));
        LoopCfg cfg = cfg0;
        cfg.cond = h;
        cfg.use_cond = 1;
        k_loop_begin<<<1, 1, 0, s>>>(ctl, 1, sc);
        PDC_LAUNCH_CK();
        enqueue_residual(contacts);
        k_loop_decide_cond<<<1, 1, 0, s>>>(ctl, cfg, sc, n_cv_d, sflag, 0);
        PDC_LAUNCH_CK();
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        PDC_CK(cudaStreamGetCaptureInfo(gs, &cst, nullptr, nullptr, &deps, nullptr, &nd));
        // (the parameter union has no default constructor: zeroed storage)
        alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
        std::memset(cp_raw, 0, sizeof(cp_raw));
        cudaGraphNodeParams &cp = *reinterpret_cast<cudaGraphNodeParams *>(cp_raw);
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cn;
        PDC_CK(cudaGraphAddNode(&cn, cg, deps, nullptr, nd, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        PDC_CK(cudaStreamUpdateCaptureDependencies(gs, &cn, nullptr, 1, cudaStreamSetCaptureDependencies));
        capturing = false;
        PDC_CK(cudaStreamEndCapture(gs, &g));
        PDC_CK(cudaStreamBeginCaptureToGraph(gs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        capturing = true;
        // graph_unroll iterations per pass of the while node (each pass costs a
        // relaunch of the body on the device): the kernels of an iteration that
        // follows the end of the loop read go = 0 and return at once, and only
        // the last decision of the pass sets the while condition
        for (int u = 0; u < unroll; ++u) {
            LoopCfg cu = cfg;
            cu.use_cond = u == unroll - 1 ? 1 : 0;
            enqueue_solve(contacts, contacts, true, 1.f, r_nc, r_c, cycles, sweeps, pccd);
            enqueue_residual(contacts);
            if (cu.use_cond) k_loop_decide_cond<<<1, 1, 0, s>>>(ctl, cu, sc, n_cv_d, sflag, 1);
            else k_loop_decide<<<1, 1, 0, s>>>(ctl, cu, sc, n_cv_d, sflag, 1);
            PDC_LAUNCH_CK();
        }
        cudaGraph_t b2 = nullptr;
        capturing = false;
        PDC_CK(cudaStreamEndCapture(gs, &b2));
        PDC_CK(cudaGraphInstantiate(&e, g, 0));
    } catch (const std::exception &ex) {
        if (capturing) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(gs, &junk);
            if (junk && junk != g) cudaGraphDestroy(junk);
        }
        if (g) cudaGraphDestroy(g);
        (void)cudaGetLastError();  // clear the failed capture's error
        s = saved;
        live_ptr = nullptr;
        device_decides = false;
        if (log) std::fprintf(stderr, "[pdc] LG loop graph not built (%s): host-driven loops\n", ex.what());
        return false;
    }
    s = saved;
    live_ptr = nullptr;
    device_decides = false;
    G.g = g;
    G.e = e;
    G.gen = graph_gen + bp.gen;
    return true;
}

// Runs one LG loop with its tests on the device: enqueued ahead of the
// device's decisions (loop_control 2), or as a graph launch on s (1; the
// graph is built or rebuilt when needed).  False when the graph cannot be
// built: the caller then runs the host-driven loop.
bool pdc_ctx::run_loop(int gi, const LoopCfg &cfg, bool contacts, int r_nc, int r_c, int cycles, int sweeps,
                       bool pccd) {
    if (P.loop_control >= 2) {
        run_loop_ahead(gi, cfg, contacts, r_nc, r_c, cycles, sweeps, pccd);
        return true;
    }
    GraphLoop &G = gl[gi];
    if (!G.e || G.gen != graph_gen + bp.gen) {
        // programmatic dependent launches inside the graph when the driver
        // takes them, else plain kernel nodes
        const int ov = P.launch_overlap;
        if (!graph_overlap) P.launch_overlap = 0;
        bool ok = build_loop(G, cfg, contacts, r_nc, r_c, cycles, sweeps, pccd);
        if (!ok && P.launch_overlap) {
            graph_overlap = false;
            P.launch_overlap = 0;
            ok = build_loop(G, cfg, contacts, r_nc, r_c, cycles, sweeps, pccd);
        }
        P.launch_overlap = ov;
        if (!ok) {
            graphs_failed = true;
            return false;
        }
    }
    PDC_CK(cudaGraphLaunch(G.e, s));
    return true;
}

// One iteration of a device-decided loop after its first decision: the solve
// part, the residual part and the decision, which it writes to host memory.
void pdc_ctx::enqueue_iteration(const LoopCfg &cfg, bool contacts, int r_nc, int r_c, int cycles, int sweeps,
                                bool pccd) {
    enqueue_solve(contacts, contacts, true, 1.f, r_nc, r_c, cycles, sweeps, pccd);
    enqueue_residual(contacts);
    k_loop_decide_host<<<1, 1, 0, s>>>(ctl, cfg, sc, n_cv_d, sflag, 1, hmap_dev);
    PDC_LAUNCH_CK();
}

// enqueue_iteration captured as a graph (loop_control = 3), with programmatic
// dependent launches inside when the driver takes them; false if it cannot be
// built.  Called with the loop's go flag set (live_ptr, device_decides).
void pdc_ctx::free_body(BodyGraph &G) {
    for (auto &e : G.e) {
        if (e) cudaGraphExecDestroy(e);
        e = nullptr;
    }
    if (G.g) cudaGraphDestroy(G.g);
    G.g = nullptr;
}

bool pdc_ctx::build_body(BodyGraph &G, const LoopCfg &cfg, bool contacts, int r_nc, int r_c, int cycles, int sweeps,
                         bool pccd) {
    free_body(G);
    if (!gs) PDC_CK(cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking));
    const int ov = P.launch_overlap;
    for (int attempt = 0; attempt < 2; ++attempt) {
        if (!graph_overlap) P.launch_overlap = 0;
        cudaStream_t saved = s;
        s = gs;
        bool capturing = false;
        try {
            PDC_CK(cudaStreamBeginCapture(gs, cudaStreamCaptureModeRelaxed));
            capturing = true;
            enqueue_iteration(cfg, contacts, r_nc, r_c, cycles, sweeps, pccd);
            capturing = false;
            PDC_CK(cudaStreamEndCapture(gs, &G.g));
            for (auto &e : G.e) PDC_CK(cudaGraphInstantiate(&e, G.g, 0));
            s = saved;
            P.launch_overlap = ov;
            G.gen = graph_gen + bp.gen;
            return true;
        } catch (const std::exception &ex) {
            if (capturing) {
                cudaGraph_t junk = nullptr;
                cudaStreamEndCapture(gs, &junk);
                if (junk) cudaGraphDestroy(junk);
            }
            free_body(G);
            (void)cudaGetLastError();
            s = saved;
            P.launch_overlap = ov;
            if (log) std::fprintf(stderr, "[pdc] iteration graph not built (%s)\n", ex.what());
            if (!graph_overlap || !ov) return false;
            graph_overlap = false;  // once more without programmatic launches
        }
    }
    return false;
}

// loop_control = 2, 3: the host enqueues the loop's iterations (residual
// part, device decision, solve part) on s, each kernel returning at once
// after the loop's end, and keeps loop_ahead iterations enqueued beyond the
// last one whose decision it has read from host-mapped memory: with
// loop_ahead >= 1 the device does not wait for the host between iterations,
// and no stream synchronisation is needed.  With 3 an iteration is one launch
// of its graph gb[gi] (stream launches if the graph cannot be built).  The
// wait for the device is bounded (a stream synchronisation after
// AHEAD_TIMEOUT_S, then the decisions are read from device memory).
void pdc_ctx::run_loop_ahead(int gi, const LoopCfg &cfg, bool contacts, int r_nc, int r_c, int cycles, int sweeps,
                             bool pccd) {
    constexpr double AHEAD_TIMEOUT_S = 30.0;
    if (!hmap) {
        void *p = nullptr;
        PDC_CK(cudaHostAlloc(&p, 2 * sizeof(int), cudaHostAllocMapped));
        hmap = (volatile int *)p;
        PDC_CK(cudaHostGetDevicePointer((void **)&hmap_dev, p, 0));
    }
    // the previous loop's kernels must be done before the flags are reset
    PDC_CK(cudaStreamSynchronize(s));
    hmap[0] = 1;
    hmap[1] = 0;
    live_ptr = &ctl.p->go;
    device_decides = true;
    struct Reset {  // the flags belong to this loop only, whatever happens
        pdc_ctx *c;
        ~Reset() {
            c->live_ptr = nullptr;
            c->device_decides = false;
        }
    } reset{this};
    BodyGraph &G = gb[gi];
    bool graph = P.loop_control == 3 && !bodies_failed;
    if (graph && (!G.e[0] || G.gen != graph_gen + bp.gen)) {
        if (!build_body(G, cfg, contacts, r_nc, r_c, cycles, sweeps, pccd)) {
            bodies_failed = true;
            graph = false;
        }
    }
    k_loop_begin<<<1, 1, 0, s>>>(ctl, 1, sc);
    PDC_LAUNCH_CK();
    enqueue_residual(contacts);
    k_loop_decide_host<<<1, 1, 0, s>>>(ctl, cfg, sc, n_cv_d, sflag, 0, hmap_dev);
    PDC_LAUNCH_CK();
    int enq = 0;  // iterations enqueued after the first decision
    auto t0 = std::chrono::steady_clock::now();
    while (enq < cfg.max_iters) {
        // wait until at most loop_ahead iterations are enqueued beyond the
        // last one decided (enq + 1 decisions enqueued, hmap[1] taken)
        bool timed_out = false;
        while (hmap[0] && enq - hmap[1] >= P.loop_ahead) {
            if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > AHEAD_TIMEOUT_S) {
                timed_out = true;
                break;
            }
        }
        if (timed_out) {
            PDC_CK(cudaStreamSynchronize(s));
            if (!hmap[0]) break;
        }
        if (!hmap[0]) break;  // the loop has ended; anything enqueued after its end does nothing
        if (graph) PDC_CK(cudaGraphLaunch(G.e[enq % (MAX_AHEAD + 1)], s));
        else enqueue_iteration(cfg, contacts, r_nc, r_c, cycles, sweeps, pccd);
        ++enq;
    }
}

void pdc_ctx::full_ccd(const float4 *x0, const float4 *x1, bool merge) {
    bp.prof = prof.on ? &prof : nullptr;
    const bool reuse = P.bp_reuse > 0;
    if (reuse && merge && bp.can_reuse(s, coll(), x0, x1)) {
        PROF("broad_phase", 0, bp.filter(s, coll(), x0, x1, dhat));
        st.bp_reused++;
    } else
        broad_phase_pass(x0, x1, reuse);
    if (prof.on) {  // list size for the byte models of the pair kernels
        long long cnt[2] = {0, 0};
        bp.cnt_vt_d[bp.cur].download(&cnt[0], 1, s);
        bp.cnt_ee_d[bp.cur].download(&cnt[1], 1, s);
        PDC_CK(cudaStreamSynchronize(s));
        bp.h_pairs = cnt[0] + cnt[1];
    }
    unsigned long long inf = 0x7ff0000000000000ULL;  // +inf
    PDC_CK(cudaMemcpyAsync(toi_bits.p, &inf, sizeof(inf), cudaMemcpyHostToDevice, s));
    if (per_instance()) {
        k_fill_u64<<<(ninst() + 255) / 256, 256, 0, s>>>(toi_inst, ninst(), inf);
        PDC_LAUNCH_CK();
    }
    // algorithmic bytes: both position sets once, per pair its key and state
    // (plus the previous list's key and state read by the merge)
    PROF("full_ccd", 32.0 * nv_all + (merge ? 18.0 : 9.0) * (double)bp.h_pairs,
         launch_full_ccd(s, coll(), bp, x0, x1, cparams(), merge, toi_bits));
    k_step_fraction<<<1, 1, 0, s>>>(toi_bits, P.alpha_ls, sfrac, ttoi);
    if (per_instance()) k_instance_fractions<<<(ninst() + 255) / 256, 256, 0, s>>>(ninst(), toi_inst, P.alpha_ls, sfrac_inst);
    PDC_LAUNCH_CK();
}

void pdc_ctx::broad_phase_pass(const float4 *x0, const float4 *x1, bool super) {
    // broad phase; a list or table that overflows is regrown and rebuilt here
    // (candidate sets spike while the iterate is far from converged), so the
    // step itself need not be redone
    for (int tries = 0;; ++tries) {
        int cur0 = bp.cur;
        bp_ovf.zero(s);
        if (super)
            PROF("broad_phase", 0, bp.run_super(s, coll(), x0, x1, dhat, (float)(P.bp_reuse * dhat), bp_ovf));
        else
            PROF("broad_phase", 0, bp.run(s, coll(), x0, x1, dhat, bp_ovf));
        int ovf = 0;
        bp_ovf.download(&ovf, 1, s);
        PDC_CK(cudaStreamSynchronize(s));
        if (!ovf) break;
        if (tries >= 6) throw Error(PDC_ERR_CAPACITY, "broad phase buffers could not be grown enough");
        bp.cur = cur0;  // the previous lists stay the merge source of the rebuilt ones
        long long cvt = bp.cap_vt * ((ovf & OVF_VT) ? 2 : 1), cee = bp.cap_ee * ((ovf & OVF_EE) ? 2 : 1),
                  cent = bp.cap_ent * ((ovf & OVF_HASH) ? 2 : 1);
        if (ovf & OVF_CELLS) bp.cell_scale *= 4.f;
        if (ovf & OVF_SLOTS) bp.grow_slots(coll(), true, true);
        bp.grow(coll(), cvt, cee, cent, s);  // keeps the current lists (NDB states merge from them)
        st.overflow_retries++;
        if (log) std::fprintf(stderr, "[pdc] broad phase regrown after overflow 0x%x\n", ovf);
    }
}

void pdc_ctx::step() {
    ensure_topology();
    ClothView c = cloth();
    const float h = (float)P.dt;
    const bool fixed = P.fixed_iters != 0;
    const bool relmode = P.tol_rel_residual > 0 && !fixed;
    const int cycles = std::max(P.solve_cycles, 1), sweeps = std::max(P.jacobi_sweeps, 0);
    st = pdc_stats();
    sflag.zero(s);  // status bits of this step (factorisation, tensor-core waits)
    st.t_toi = 2.0;
    st.s_line_search = 1.0;
    auto t0 = std::chrono::steady_clock::now();
    PDC_CK(cudaMemcpyAsync(Xbak.p, Xs.p, sizeof(float4) * nv_all, cudaMemcpyDeviceToDevice, s));
    PDC_CK(cudaMemcpyAsync(Vbak.p, Vs.p, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s));
    PDC_CK(cudaMemsetAsync(sc.p, 0, sizeof(Scalars), s));

    // Eq. (z) and x <- z (Alg. 1); obstacles move to their targets in x^+
    float3 g = make_float3((float)P.gravity[0], (float)P.gravity[1], (float)P.gravity[2]);
    launch_prologue(s, n, Xs, Vs, pins_d, pin_tgt, npins, h, g, Z, Ucur, Xp, rf_pending ? RFd.p : nullptr);
    if (nv_all > n)
        PDC_CK(cudaMemcpyAsync(Xp.p + n, obs_tgt.p, sizeof(float4) * (nv_all - n), cudaMemcpyDeviceToDevice, s));
    if (P.autotune && !tune.tuned) {
        autotune_vertex_kernels();
        tune.tuned = 1;
        c = cloth();
    }
    // rho0 = residual at z (no collision springs)
    PDC_CK(cudaMemsetAsync(&sc.p->rsq, 0, sizeof(double), s));
    launch_residual(s, c, Xs, Ucur, Z, nullptr, nullptr, R, sc, nullptr, 0);
    k_loop_step_init<<<1, 1, 0, s>>>(ctl, sc);
    PDC_LAUNCH_CK();
    std::memset(&hctl, 0, sizeof(hctl));
    // device-driven loops need no residual on the host; the host-driven ones read it here
    const bool dev = device_loops_ok();
    double rho0 = 0.0;
    bool have_rho0 = false;
    auto host_rho0 = [&]() {
        if (!have_rho0) {
            read_scalars();
            rho0 = std::sqrt(hsc->rsq);
            st.rho0 = rho0;
            have_rho0 = true;
        }
        return rho0;
    };
    if (!dev) host_rho0();
    if (log) std::fprintf(stderr, "[pdc] step n=%d omega=%.4f rho0=%.6g dhat=%.3g k=%.4g\n", n, omega, rho0, dhat, k_ndb);
    const double tolx_in = P.tol_inner * L, tolx_out = P.tol_outer * L;
    bool dev_used = false;  // some loop ran on the device: its counters are in ctl
    bool last_dev = false;  // the last loop ran on the device: the last residual is in ctl

    // ---- warm start: LG iterations of I + Psi in span(U) + sweeps
    accel.on = P.accel != 0 && !fixed;
    accel.rho_fixed = P.accel_rho;
    accel.reset();
    if (dev && run_loop(0, loop_cfg(0, P.warm_iters, relmode, false), false, r_warm, 0, cycles, sweeps, true)) {
        dev_used = last_dev = true;
    } else {
        last_dev = false;
        host_rho0();
        for (int it = 0; it < P.warm_iters; ++it) {
            bool conv = false;
            lg_iteration(false, relmode, rho0, conv, r_warm, 0, cycles, sweeps);
            if (conv) break;
            st.warm_iters++;
            if (!fixed && !relmode) {
                read_scalars();
                if (bits_to_float(hsc->dxmax) <= tolx_in) break;
            }
        }
    }

    bool use_lerp = false;
    if (!P.collisions) {
        // no collision handling: the inner LG loop without springs or CCD
        accel.reset();
        if (dev && !graphs_failed &&
            run_loop(1, loop_cfg(1, P.max_inner, relmode, false), false, r_warm, 0, cycles, sweeps, true)) {
            dev_used = last_dev = true;
        } else {
            last_dev = false;
            host_rho0();
            for (int it = 0; it < P.max_inner; ++it) {
                bool conv = false;
                lg_iteration(false, relmode, rho0, conv, r_warm, 0, cycles, sweeps);
                if (conv) break;
                st.inner_iters++;
                if (!fixed && !relmode) {
                    read_scalars();
                    if (bits_to_float(hsc->dxmax) <= tolx_in) break;
                }
            }
        }
    } else {
        use_lerp = true;
        // initial full CCD from x* to the warm start, filter -> x^- (Alg. 1)
        full_ccd(Xs, Xp, false);
        if (log) {
            double t0v = 0, s0v = 0;
            ttoi.download(&t0v, 1, s);
            sfrac.download(&s0v, 1, s);
            PDC_CK(cudaStreamSynchronize(s));
            std::fprintf(stderr, "[pdc] initial full CCD: t_toi=%.6g s=%.6g\n", t0v, s0v);
        }
        const int *vi = per_instance() ? vinst.p : nullptr;      // per-instance fractions
        launch_lerp(s, nv_all, Xs, Xp, sfrac, Xm, vi, sfrac_inst);        // obstacles (and cloth, overwritten next)
        launch_scale_disp(s, n, Xs, Ucur, sfrac, Um, Xm, vi, sfrac_inst); // cloth x^- = x* + s u
        // the iterate restarts at x^- with pins at their targets
        launch_restart(s, n, Xs, Um, Ucur, Xp);
        launch_set_pins(s, pins_d, npins, pin_tgt, Xs, Ucur, Xp);
        launch_collect_active(s, coll(), bp, Xm, cparams(), act, cap_act, n_act_d, &sc.p->overflow);
        PDC_CK(cudaMemcpyAsync(Xprev.p, Um.p, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s));
        unsigned long long none = 0x4000000000000000ULL;  // 2.0: no impact yet
        PDC_CK(cudaMemcpyAsync(toi_bits.p, &none, sizeof(none), cudaMemcpyHostToDevice, s));
        k_step_fraction<<<1, 1, 0, s>>>(toi_bits, P.alpha_ls, sfrac, ttoi);
        if (vi) {
            k_fill_u64<<<(ninst() + 255) / 256, 256, 0, s>>>(toi_inst, ninst(), none);
            k_instance_fractions<<<(ninst() + 255) / 256, 256, 0, s>>>(ninst(), toi_inst, P.alpha_ls, sfrac_inst);
        }
        PDC_LAUNCH_CK();
        for (int o = 0; o < P.max_outer; ++o) {
            st.outer_iters++;
            accel.reset();  // the constraint set changed (full CCD)
            int inner = 0;
            const int inner0 = hctl.inner_iters;
            bool ran_dev = dev && !graphs_failed &&
                           run_loop(2 + bp.cur, loop_cfg(1, P.max_inner, relmode, true), true, r_warm, r_reuse, cycles,
                                    sweeps, true);
            if (ran_dev) {
                dev_used = last_dev = true;
            } else {
                last_dev = false;
                host_rho0();
                for (int it = 0; it < P.max_inner; ++it) {
                    bool conv = false;
                    lg_iteration(true, relmode, rho0, conv, r_warm, r_reuse, cycles, sweeps);
                    if (conv) break;
                    ++inner;
                    st.inner_iters++;
                    if (!fixed && !relmode) {
                        read_scalars();
                        if (bits_to_float(hsc->dxmax) <= tolx_in) break;
                    } else if (relmode && last_springs) {
                        // with collision springs the residual carries barrier
                        // terms whose weights change every iteration: the inner
                        // loop also ends once the iterate has settled to the
                        // outer tolerance
                        read_scalars();
                        if (bits_to_float(hsc->dxmax) <= tolx_out) break;
                    }
                }
            }
            // change of the iterate over this pass (the full CCD below leaves it alone)
            if (!fixed) {
                umax_d.zero(s);
                k_maxdiff<<<nb(n), 256, 0, s>>>(n, Ucur, Xprev, umax_d);
                PDC_LAUNCH_CK();
            }
            unsigned int um = 0;
            if (ran_dev) {  // one read-back for the pass: its iteration count and change
                ctl.download(&hctl, 1, s);
                if (!fixed) umax_d.download(&um, 1, s);
                PDC_CK(cudaStreamSynchronize(s));
                inner = hctl.inner_iters - inner0;
            }
            if (inner > 0 || o == 0) {
                full_ccd(Xm, Xp, true);
                launch_collect_active(s, coll(), bp, Xm, cparams(), act, cap_act, n_act_d, &sc.p->overflow);
            }
            if (!fixed) {
                if (!ran_dev) {
                    umax_d.download(&um, 1, s);
                    PDC_CK(cudaStreamSynchronize(s));
                }
                PDC_CK(cudaMemcpyAsync(Xprev.p, Ucur.p, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s));
                if (bits_to_float(um) <= tolx_out) break;
            }
        }
    }
    // exit line search and velocities (Alg. 1; v = (x - x*)/h)
    k_finish<<<nb(nv_all), 256, 0, s>>>(nv_all, n, Um, Ucur, Xm, Xp, sfrac, use_lerp ? 1 : 0, 1.f / h, Xs, Vs, Ulast,
                                        per_instance() ? vinst.p : nullptr, sfrac_inst.p);
    PDC_LAUNCH_CK();
    bad_d.zero(s);
    k_finite<<<nb(n), 256, 0, s>>>(n, Xs, bad_d);
    PDC_LAUNCH_CK();
    int bad = 0, sflag_h = 0;
    long long counts[2] = {0, 0};
    int nact = 0, ncv = 0;
    double tt = 2.0, sf = 1.0;
    bad_d.download(&bad, 1, s);
    sflag.download(&sflag_h, 1, s);
    PDC_CK(cudaStreamSynchronize(s));
    if (sflag_h & (PDC_DEVERR_UMMA | PDC_DEVERR_COPY)) {
        PDC_CK(cudaMemcpyAsync(Xs.p, Xbak.p, sizeof(float4) * nv_all, cudaMemcpyDeviceToDevice, s));
        PDC_CK(cudaMemcpyAsync(Vs.p, Vbak.p, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s));
        sflag.zero(s);
        PDC_CK(cudaStreamSynchronize(s));
        throw Error(PDC_ERR_TIMEOUT, (sflag_h & PDC_DEVERR_UMMA)
                                         ? "a tensor-core subspace kernel timed out waiting on its copies; state rolled back"
                                         : "a Chebyshev step timed out waiting on its matrix tile; state rolled back");
    }
    if (P.collisions) {
        bp.cnt_vt_d[bp.cur].download(&counts[0], 1, s);
        bp.cnt_ee_d[bp.cur].download(&counts[1], 1, s);
    }
    n_act_d.download(&nact, 1, s);
    n_cv_d.download(&ncv, 1, s);
    ttoi.download(&tt, 1, s);
    sfrac.download(&sf, 1, s);
    if (dev_used) ctl.download(&hctl, 1, s);
    read_scalars();
    if (dev_used) {  // counters of the loops that ran on the device
        st.warm_iters += hctl.warm_iters;
        st.inner_iters += hctl.inner_iters;
        st.contact_iters += hctl.contact_iters;
        st.device_loops = hctl.device_loops;
        if (relmode && last_dev) st.rel_residual = hctl.rel;
        if (!have_rho0) st.rho0 = hctl.rho0;
    }
    st.n_candidates = counts[0] + counts[1];
    st.n_active = nact;
    st.n_contact_vertices = ncv;
    if (P.collisions) {
        st.t_toi = tt <= 1.0 ? tt : 2.0;
        st.s_line_search = sf;
    }
    if (hsc->overflow) {
        // roll back; the caller (pdc_step) grows the buffers and retries
        PDC_CK(cudaMemcpyAsync(Xs.p, Xbak.p, sizeof(float4) * nv_all, cudaMemcpyDeviceToDevice, s));
        PDC_CK(cudaMemcpyAsync(Vs.p, Vbak.p, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s));
        PDC_CK(cudaStreamSynchronize(s));
        throw Error(PDC_ERR_CAPACITY, "overflow:" + std::to_string(hsc->overflow));
    }
    if (bad) {
        PDC_CK(cudaMemcpyAsync(Xs.p, Xbak.p, sizeof(float4) * nv_all, cudaMemcpyDeviceToDevice, s));
        PDC_CK(cudaMemcpyAsync(Vs.p, Vbak.p, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s));
        PDC_CK(cudaStreamSynchronize(s));
        throw Error(PDC_ERR_NUMERIC, "non-finite positions; state rolled back");
    }
    if (unsigned int guard = P.collisions ? pair_guard_take(s, guard_d) : 0u) {
        PDC_CK(cudaMemcpyAsync(Xs.p, Xbak.p, sizeof(float4) * nv_all, cudaMemcpyDeviceToDevice, s));
        PDC_CK(cudaMemcpyAsync(Vs.p, Vbak.p, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s));
        PDC_CK(cudaStreamSynchronize(s));
        throw Error(PDC_ERR_STATE, "collision list index outside the topology (guard 0x" + std::to_string(guard) +
                                       "); state rolled back");
    }
    rf_pending = false;  // the previous step's forwarded displacement is used up
    if (P.collisions && P.rf_toi > 0 && st.t_toi < P.rf_toi) residual_forwarding();
    st.ms_step = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (prof.on) prof.flush();
    stepped = true;
}

// Residual forwarding (Sec. 6, end of Alg. 1).  The step has ended at x_new
// (in Xs); more LG iterations of the same problem (same z) run from x_new
// with every active constraint at weight k (a = 0) and no partial or full
// CCD, and their total change dx (pinned rows 0) is kept for the next
// step's z.  The step's statistics other than rf_iters are left as they
// were; a non-finite dx is dropped.
void pdc_ctx::residual_forwarding() {
    const bool fixed = P.fixed_iters != 0;
    const int cycles = std::max(P.solve_cycles, 1), sweeps = std::max(P.jacobi_sweeps, 0);
    const double tolx_in = P.tol_inner * L;
    launch_rf_rebase(s, n, Xs, Xbak, Z, Ucur, Xp);
    if (nv_all > n)
        PDC_CK(cudaMemcpyAsync(Xp.p + n, Xs.p + n, sizeof(float4) * (nv_all - n), cudaMemcpyDeviceToDevice, s));
    launch_rf_weights(s, act, n_act_d, cap_act, (float)k_ndb);
    const bool acc_on = accel.on;
    const double rel = st.rel_residual;
    const int citers = st.contact_iters;
    accel.on = false;
    for (int it = 0; it < std::max(P.rf_iters, 0); ++it) {
        bool conv = false;
        lg_iteration(true, false, st.rho0, conv, r_warm, r_reuse, cycles, sweeps, false);
        st.rf_iters++;
        if (!fixed) {
            read_scalars();
            if (bits_to_float(hsc->dxmax) <= tolx_in) break;
        }
    }
    accel.on = acc_on;
    st.rel_residual = rel;
    st.contact_iters = citers;
    RFd.alloc(n);
    PDC_CK(cudaMemcpyAsync(RFd.p, Ucur.p, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s));
    bad_d.zero(s);
    k_finite<<<nb(n), 256, 0, s>>>(n, RFd, bad_d);
    PDC_LAUNCH_CK();
    int bad = 0;
    bad_d.download(&bad, 1, s);
    PDC_CK(cudaStreamSynchronize(s));
    rf_pending = bad == 0;
}

// ============================================================================ C ABI
static std::string g_create_error = "no error";

#define API_BEGIN(h)                                                                                  \
    if (!(h)) return PDC_ERR_ARG;                                                                      \
    try {
#define API_END(h)                                                                                    \
    }                                                                                                  \
    catch (const Error &e) {                                                                           \
        (h)->err = e.what();                                                                           \
        return e.code;                                                                                 \
    }                                                                                                  \
    catch (const std::exception &e) {                                                                  \
        (h)->err = e.what();                                                                           \
        return PDC_ERR_CUDA;                                                                           \
    }                                                                                                  \
    return PDC_OK;

extern "C" {

void pdc_default_params(pdc_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->dt = 1.0 / 200.0;
    p->gravity[2] = -9.8;
    p->k_ndb_scale = 1.0;
    p->K_ndb = 2.0;
    p->a_max = 20;
    p->alpha_ls = 0.8;
    p->d_hat = 0.0;
    p->eta_ccd = 1e-9;
    p->tol_outer = 1e-3;
    p->tol_inner = 5e-2;
    p->tol_rel_residual = 0.0;
    p->max_outer = 4;
    p->max_inner = 32;
    p->warm_iters = 5;
    p->jacobi_sweeps = 4;
    p->jacobi_omega = 0.0;
    p->solve_cycles = 1;
    p->r_warm = 0;
    p->r_reuse = 0;
    p->precision = 0;
    p->samples_vt = 3;
    p->samples_ee = 4;
    p->collisions = 1;
    p->fixed_iters = 0;
    p->eig_iters = 12;
    p->seed = 12345;
    p->accel = 0;
    p->accel_rho = 0.0;
    p->sweep_kind = 0;
    p->cheb_ratio = 100.0;
    p->aa_depth = 6;
    p->tensor_cores = 1;
    p->bp_reuse = 0.0;
    p->launch_overlap = 1;
    p->rf_toi = 0.0;
    p->rf_iters = 8;
    p->loop_control = 1;
    p->pccd_adaptive = 0;
    p->pccd_max_axis = 64;
    p->instance_line_search = 0;
    p->autotune = 0;
    p->graph_unroll = 1;
    p->loop_ahead = 1;
    p->cheb_source = -1;
    p->residual_patch = 1;
}

static bool params_valid(const pdc_params *params) {
    return params->dt > 0 && params->precision >= 0 && params->precision <= 2 && params->r_warm >= 0 &&
           params->r_reuse >= 0 && params->r_reuse <= R_REUSE_MAX && params->max_outer >= 0 && params->max_inner >= 0 &&
           params->warm_iters >= 0 && params->a_max >= 0 && params->a_max <= 127 &&
           (params->samples_vt == 0 || params->samples_vt == 1 || params->samples_vt == 3) &&
           (params->samples_ee == 0 || params->samples_ee == 1 || params->samples_ee == 4) &&
           params->sweep_kind >= 0 && params->sweep_kind <= 1 && (params->sweep_kind != 1 || params->cheb_ratio > 1.0) &&
           params->accel >= 0 && params->accel <= 2 && (params->accel != 2 || (params->aa_depth >= 1 && params->aa_depth <= 8)) &&
           params->loop_control >= 0 && params->loop_control <= 3 && params->loop_ahead >= 0 &&
           params->loop_ahead <= 2 && params->cheb_source >= -1 && params->cheb_source <= 3 &&
           (params->residual_patch == 0 || params->residual_patch == 1) &&
           (params->pccd_adaptive == 0 || (params->pccd_adaptive == 1 && params->pccd_max_axis >= 1 &&
                                           params->pccd_max_axis <= 256 && params->alpha_ls > 0 && params->alpha_ls < 1));
}

static bool mesh_valid(const pdc_mesh_desc *mesh) {
    return mesh->nv > 0 && mesh->nt > 0 && mesh->verts && mesh->tris && mesh->npins >= 0 &&
           (mesh->npins == 0 || mesh->pins);
}

// Builds the context for one mesh; batch material tables are filled by the caller.
static pdc_status create_ctx(std::unique_ptr<pdc_ctx> &c, const pdc_mesh_desc *mesh, const pdc_params *params,
                             void *stream, pdc_handle *out) {
    c->P = *params;
    c->s = (cudaStream_t)stream;
    try {
        set_chol_smem_limits();
        c->setup(mesh);
        c->setup_basis();
    } catch (const Error &e) {
        g_create_error = e.what();
        return e.code;
    } catch (const std::exception &e) {
        g_create_error = e.what();
        return PDC_ERR_CUDA;
    }
    *out = c.release();
    return PDC_OK;
}

pdc_status pdc_create(const pdc_mesh_desc *mesh, const pdc_material *mat, const pdc_params *params, void *stream,
                      pdc_handle *out) {
    if (!out || !mesh || !mat || !params) {
        g_create_error = "pdc_create: NULL argument";
        return PDC_ERR_ARG;
    }
    *out = nullptr;
    if (!mesh_valid(mesh)) {
        g_create_error = "pdc_create: empty or inconsistent mesh";
        return PDC_ERR_ARG;
    }
    if (!params_valid(params)) {
        g_create_error = "pdc_create: invalid parameters";
        return PDC_ERR_ARG;
    }
    std::unique_ptr<pdc_ctx> c(new pdc_ctx());
    c->M = *mat;
    return create_ctx(c, mesh, params, stream, out);
}

pdc_status pdc_create_batch(int32_t count, const pdc_mesh_desc *meshes, const pdc_material *materials,
                            const pdc_params *params, void *stream, pdc_handle *out) {
    if (!out || !meshes || !materials || !params || count <= 0) {
        g_create_error = "pdc_create_batch: NULL argument or empty batch";
        return PDC_ERR_ARG;
    }
    *out = nullptr;
    if (!params_valid(params)) {
        g_create_error = "pdc_create_batch: invalid parameters";
        return PDC_ERR_ARG;
    }
    // the union mesh: instance k's vertices, triangles and pins follow those of
    // instances 0..k-1, its ids shifted by their vertex count
    std::vector<float> V;
    std::vector<int32_t> Tr, Pn;
    std::unique_ptr<pdc_ctx> c(new pdc_ctx());
    long long nv = 0;
    for (int k = 0; k < count; ++k) {
        const pdc_mesh_desc &m = meshes[k];
        if (!mesh_valid(&m)) {
            g_create_error = "pdc_create_batch: empty or inconsistent mesh " + std::to_string(k);
            return PDC_ERR_ARG;
        }
        if (nv + m.nv > (1LL << 30)) {
            g_create_error = "pdc_create_batch: too many vertices";
            return PDC_ERR_ARG;
        }
        V.insert(V.end(), m.verts, m.verts + 3 * (size_t)m.nv);
        for (int t = 0; t < 3 * m.nt; ++t) {
            if (m.tris[t] < 0 || m.tris[t] >= m.nv) {
                g_create_error = "pdc_create_batch: triangle index out of range in mesh " + std::to_string(k);
                return PDC_ERR_ARG;
            }
            Tr.push_back((int32_t)(m.tris[t] + nv));
        }
        for (int p = 0; p < m.npins; ++p) {
            if (m.pins[p] < 0 || m.pins[p] >= m.nv) {
                g_create_error = "pdc_create_batch: pin index out of range in mesh " + std::to_string(k);
                return PDC_ERR_ARG;
            }
            Pn.push_back((int32_t)(m.pins[p] + nv));
        }
        c->mats.push_back(materials[k]);
        c->tri_inst.insert(c->tri_inst.end(), (size_t)m.nt, k);
        nv += m.nv;
    }
    c->M = materials[0];
    c->inst_off.push_back(0);
    {
        long long acc = 0;
        for (int k = 0; k < count; ++k) {
            acc += meshes[k].nv;
            c->inst_off.push_back((int)acc);
        }
    }
    pdc_mesh_desc u;
    u.verts = V.data();
    u.nv = (int32_t)nv;
    u.tris = Tr.data();
    u.nt = (int32_t)(Tr.size() / 3);
    u.pins = Pn.empty() ? nullptr : Pn.data();
    u.npins = (int32_t)Pn.size();
    return create_ctx(c, &u, params, stream, out);
}

pdc_status pdc_measure_copy_bandwidth(int64_t bytes, int32_t passes, void *stream, double *gbs) {
    if (!gbs || bytes < 1024 || passes < 1 || bytes > ((int64_t)1 << 36)) {
        g_create_error = "pdc_measure_copy_bandwidth: bytes must be in [1 KiB, 64 GiB], passes >= 1, gbs not NULL";
        return PDC_ERR_ARG;
    }
    try {
        cudaStream_t s = (cudaStream_t)stream;
        const long long n = bytes / 2 / (long long)sizeof(float4);
        DevBuf<float4> a, b;
        a.alloc(n);
        b.alloc(n);
        a.zero(s);
        b.zero(s);
        int dev = 0, sms = 1;
        PDC_CK(cudaGetDevice(&dev));
        PDC_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int grid = sms * 4;
        k_copy_passes<<<grid, 512, 0, s>>>(a, b, n, 2);  // warm the working set into the cache
        PDC_LAUNCH_CK();
        cudaEvent_t e0, e1;
        PDC_CK(cudaEventCreate(&e0));
        PDC_CK(cudaEventCreate(&e1));
        PDC_CK(cudaEventRecord(e0, s));
        k_copy_passes<<<grid, 512, 0, s>>>(a, b, n, passes);
        PDC_CK(cudaEventRecord(e1, s));
        cudaError_t le = cudaGetLastError();
        cudaError_t se = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (le == cudaSuccess && se == cudaSuccess) PDC_CK(cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        PDC_CK(le);
        PDC_CK(se);
        *gbs = ms > 0.f ? 2.0 * (double)n * sizeof(float4) * passes / (ms * 1e-3) / 1e9 : 0.0;
    } catch (const Error &e) {
        g_create_error = e.what();
        return e.code;
    } catch (const std::exception &e) {
        g_create_error = e.what();
        return PDC_ERR_CUDA;
    }
    return PDC_OK;
}

void pdc_destroy(pdc_handle h) {
    if (!h) return;
    if (h->s) cudaStreamSynchronize(h->s);
    else cudaDeviceSynchronize();
    delete h;
}

const char *pdc_last_error(pdc_handle h) { return h ? h->err.c_str() : g_create_error.c_str(); }

pdc_status pdc_add_obstacle(pdc_handle h, const float *verts, int32_t nv, const int32_t *tris, int32_t nt,
                            int32_t *out_id) {
    API_BEGIN(h)
    if (!verts || !tris || nv <= 0 || nt <= 0) throw Error(PDC_ERR_ARG, "pdc_add_obstacle: empty mesh");
    if (h->stepped) throw Error(PDC_ERR_STATE, "pdc_add_obstacle: obstacles must be added before the first step");
    for (int k = 0; k < 3 * nt; ++k)
        if (tris[k] < 0 || tris[k] >= nv) throw Error(PDC_ERR_ARG, "pdc_add_obstacle: triangle index out of range");
    Obstacle o;
    o.V.assign(verts, verts + 3 * (size_t)nv);
    o.T.assign(tris, tris + 3 * (size_t)nt);
    o.off = h->nv_all;
    for (auto &q : h->obs) (void)q;
    int id = (int)h->obs.size();
    h->obs.push_back(o);
    h->topo_dirty = true;
    h->obs_tgt.release();
    h->ensure_topology();
    if (out_id) *out_id = id;
    API_END(h)
}

pdc_status pdc_set_obstacle_instance(pdc_handle h, int32_t id, int32_t instance) {
    API_BEGIN(h)
    if (id < 0 || id >= (int)h->obs.size()) throw Error(PDC_ERR_ARG, "pdc_set_obstacle_instance: bad obstacle id");
    if (instance < -1 || instance >= h->ninst() || h->ninst() < 2)
        throw Error(PDC_ERR_ARG, "pdc_set_obstacle_instance: instance out of range (or not a batched handle)");
    h->ensure_topology();
    h->obs_inst[id] = instance;
    h->upload_vinst();
    API_END(h)
}

pdc_status pdc_set_obstacle_transform(pdc_handle h, int32_t id, const float *m4x4) {
    API_BEGIN(h)
    if (id < 0 || id >= (int)h->obs.size() || !m4x4) throw Error(PDC_ERR_ARG, "pdc_set_obstacle_transform: bad id");
    h->ensure_topology();
    const Obstacle &o = h->obs[id];
    int base = o.off - h->n, cnt = (int)o.V.size() / 3;
    DevBuf<float> md;
    std::vector<float> m(m4x4, m4x4 + 12);
    md.upload(m, h->s);
    k_transform<<<nb(cnt), 256, 0, h->s>>>(cnt, h->obs_rest.p + base, md, h->obs_tgt.p + base);
    PDC_LAUNCH_CK();
    PDC_CK(cudaStreamSynchronize(h->s));
    API_END(h)
}

pdc_status pdc_set_pin_targets(pdc_handle h, const float *xyz, int32_t on_device) {
    API_BEGIN(h)
    if (h->npins == 0) return PDC_OK;
    if (!xyz) throw Error(PDC_ERR_ARG, "pdc_set_pin_targets: NULL");
    if (on_device) {
        k_f3_to_f4<<<nb(h->npins), 256, 0, h->s>>>(h->npins, xyz, h->pin_tgt);
    } else {
        PDC_CK(cudaMemcpyAsync(h->stage3.p, xyz, sizeof(float) * 3 * h->npins, cudaMemcpyHostToDevice, h->s));
        k_f3_to_f4<<<nb(h->npins), 256, 0, h->s>>>(h->npins, h->stage3, h->pin_tgt);
    }
    PDC_LAUNCH_CK();
    PDC_CK(cudaStreamSynchronize(h->s));
    API_END(h)
}

pdc_status pdc_set_state(pdc_handle h, const float *x, const float *v, int32_t on_device) {
    API_BEGIN(h)
    if (!x) throw Error(PDC_ERR_ARG, "pdc_set_state: NULL positions");
    int n = h->n;
    const float *src = x;
    if (!on_device) {
        PDC_CK(cudaMemcpyAsync(h->stage3.p, x, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, h->s));
        src = h->stage3;
    }
    k_f3_to_f4<<<nb(n), 256, 0, h->s>>>(n, src, h->Xs);
    PDC_LAUNCH_CK();
    if (v) {
        const float *vs = v;
        if (!on_device) {
            PDC_CK(cudaMemcpyAsync(h->stage3.p, v, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, h->s));
            vs = h->stage3;
        }
        k_f3_to_f4<<<nb(n), 256, 0, h->s>>>(n, vs, h->Vs);
        PDC_LAUNCH_CK();
    } else {
        h->Vs.zero(h->s);
    }
    h->rf_pending = false;  // a forwarded residual belongs to the replaced state
    h->Ulast.zero(h->s);
    PDC_CK(cudaStreamSynchronize(h->s));
    API_END(h)
}

static void get_f4(pdc_handle h, const float4 *src, float *out, int on_device) {
    int n = h->n;
    float *dst = on_device ? out : h->stage3.p;
    k_f4_to_f3<<<nb(n), 256, 0, h->s>>>(n, src, dst);
    PDC_LAUNCH_CK();
    if (!on_device) PDC_CK(cudaMemcpyAsync(out, h->stage3.p, sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, h->s));
    PDC_CK(cudaStreamSynchronize(h->s));
}

pdc_status pdc_get_state(pdc_handle h, float *x, float *v, int32_t on_device) {
    API_BEGIN(h)
    if (x) get_f4(h, h->Xs, x, on_device);
    if (v) get_f4(h, h->Vs, v, on_device);
    API_END(h)
}

pdc_status pdc_get_positions(pdc_handle h, float *out, int32_t on_device) {
    API_BEGIN(h)
    if (!out) throw Error(PDC_ERR_ARG, "pdc_get_positions: NULL");
    get_f4(h, h->Xs, out, on_device);
    API_END(h)
}

pdc_status pdc_get_displacement(pdc_handle h, float *u, int32_t on_device) {
    API_BEGIN(h)
    if (!u) throw Error(PDC_ERR_ARG, "pdc_get_displacement: NULL");
    get_f4(h, h->Ulast, u, on_device);
    API_END(h)
}

pdc_status pdc_set_basis(pdc_handle h, const float *U, int32_t r) {
    API_BEGIN(h)
    if (!U || r <= 0) throw Error(PDC_ERR_ARG, "pdc_set_basis: empty basis");
    std::vector<float> Uh(U, U + (size_t)h->n * r);
    h->install_basis(Uh, r);
    API_END(h)
}

pdc_status pdc_get_basis(pdc_handle h, float *U, double *A0) {
    API_BEGIN(h)
    if (h->r_warm == 0) throw Error(PDC_ERR_STATE, "pdc_get_basis: no basis");
    int r = h->r_warm, ld = h->ld;
    std::vector<float> Uh((size_t)h->n * ld);
    std::vector<double> Ah((size_t)ld * ld);
    h->U32.download(Uh.data(), Uh.size(), h->s);
    h->A0.download(Ah.data(), Ah.size(), h->s);
    PDC_CK(cudaStreamSynchronize(h->s));
    for (int i = 0; i < h->n && U; ++i)
        for (int j = 0; j < r; ++j) U[(size_t)i * r + j] = Uh[(size_t)i * ld + j];
    for (int i = 0; i < r && A0; ++i)
        for (int j = 0; j < r; ++j) A0[(size_t)i * r + j] = Ah[(size_t)i * ld + j];
    API_END(h)
}

pdc_status pdc_step(pdc_handle h, double dt) {
    API_BEGIN(h)
    if (std::fabs(dt - h->P.dt) > 1e-12 * h->P.dt) throw Error(PDC_ERR_ARG, "pdc_step: dt differs from params.dt");
    int retries = 0;
    for (;;) {
        try {
            h->step();
            break;
        } catch (const Error &e) {
            if (e.code != PDC_ERR_CAPACITY || retries >= 6) throw;
            int ovf = h->hsc->overflow;
            ++retries;
            BroadPhase &bp = h->bp;
            CollView cv = h->coll();
            long long cvt = bp.cap_vt, cee = bp.cap_ee, cent = bp.cap_ent;
            if (ovf & OVF_VT) cvt *= 2;
            if (ovf & OVF_EE) cee *= 2;
            if (ovf & OVF_HASH) cent *= 2;
            if (ovf & OVF_CELLS) bp.cell_scale *= 4.f;
            if (ovf & OVF_SLOTS) bp.grow_slots(cv, true, true);
            if (ovf & (OVF_VT | OVF_EE | OVF_HASH)) bp.reserve(cv, cvt, cee, cent, h->s);
            if (ovf & OVF_ACTIVE) {
                h->cap_act *= 2;
                h->act.alloc(h->cap_act);
                ++h->graph_gen;
            }
            h->accel.rho_carry = 0.0;
            if (h->log) std::fprintf(stderr, "[pdc] step retried after overflow 0x%x\n", ovf);
        }
    }
    h->st.overflow_retries += retries;  // regrowths inside the step plus whole-step retries
    API_END(h)
}

pdc_status pdc_set_profiling(pdc_handle h, int32_t enable) {
    API_BEGIN(h)
    h->prof.reset();
    h->prof.on = enable != 0;
    API_END(h)
}

pdc_status pdc_get_kernel_times(pdc_handle h, pdc_kernel_time *out, int32_t cap, int32_t *count) {
    API_BEGIN(h)
    int k = (int)h->prof.acc.size();
    if (count) *count = k;
    if (out)
        for (int i = 0; i < std::min(k, (int)cap); ++i) out[i] = h->prof.acc[i];
    API_END(h)
}

pdc_status pdc_get_pairs(pdc_handle h, int32_t *prim, int32_t *kinds, uint8_t *state, int64_t cap, int64_t *count) {
    API_BEGIN(h)
    if (!count || cap < 0 || (cap > 0 && (!prim || !kinds || !state))) throw Error(PDC_ERR_ARG, "pdc_get_pairs: NULL");
    *count = 0;
    if (!h->P.collisions || !h->stepped) return PDC_OK;
    BroadPhase &bp = h->bp;
    long long nvt = 0, nee = 0;
    bp.cnt_vt_d[bp.cur].download(&nvt, 1, h->s);
    bp.cnt_ee_d[bp.cur].download(&nee, 1, h->s);
    PDC_CK(cudaStreamSynchronize(h->s));
    *count = nvt + nee;
    const long long kv = std::min<long long>(nvt, cap), ke = std::min<long long>(nee, cap - kv);
    std::vector<int2> pv(std::max<long long>(kv, 1)), pe(std::max<long long>(ke, 1));
    std::vector<unsigned char> sv(std::max<long long>(kv, 1)), se(std::max<long long>(ke, 1));
    if (kv > 0) {
        bp.vt[bp.cur].download(pv.data(), kv, h->s);
        bp.st_vt[bp.cur].download(sv.data(), kv, h->s);
    }
    if (ke > 0) {
        bp.ee[bp.cur].download(pe.data(), ke, h->s);
        bp.st_ee[bp.cur].download(se.data(), ke, h->s);
    }
    PDC_CK(cudaStreamSynchronize(h->s));
    for (long long i = 0; i < kv; ++i) {
        prim[2 * i] = pv[i].x;
        prim[2 * i + 1] = pv[i].y;
        kinds[i] = 0;
        state[i] = sv[i];
    }
    for (long long i = 0; i < ke; ++i) {
        prim[2 * (kv + i)] = pe[i].x;
        prim[2 * (kv + i) + 1] = pe[i].y;
        kinds[kv + i] = 1;
        state[kv + i] = se[i];
    }
    API_END(h)
}

pdc_status pdc_get_tuning(pdc_handle h, pdc_tuning *out) {
    API_BEGIN(h)
    if (!out) throw Error(PDC_ERR_ARG, "pdc_get_tuning: NULL");
    *out = h->tune;
    out->pair_blocks = h->bp.pair_blocks;
    out->cell_warps = h->bp.cell_warps;
    out->cheb_tile = h->cloth().cheb_mode;  // the source in use
    for (int k = 0; k < 4; ++k) out->pair_ms[k] = h->bp.pair_ms[k];
    for (int k = 0; k < 3; ++k) out->cell_ms[k] = h->bp.cell_ms[k];
    out->cell_grid = h->bp.cell_grid;
    for (int k = 0; k < 3; ++k) out->grid_ms[k] = h->bp.grid_ms[k];
    API_END(h)
}

pdc_status pdc_get_stats(pdc_handle h, pdc_stats *out) {
    API_BEGIN(h)
    if (!out) throw Error(PDC_ERR_ARG, "pdc_get_stats: NULL");
    *out = h->st;
    API_END(h)
}

// ----------------------------------------------------------------------------- stage entry points
static void upload_f4(pdc_handle h, const float *x, int count, DevBuf<float4> &dst) {
    DevBuf<float> tmp;
    tmp.upload(x, 3 * (size_t)count, h->s);
    dst.alloc(count);
    k_f3_to_f4<<<nb(count), 256, 0, h->s>>>(count, tmp, dst);
    PDC_LAUNCH_CK();
    PDC_CK(cudaStreamSynchronize(h->s));
}

pdc_status pdc_op_broadphase(pdc_handle h, const float *x0, const float *x1, int32_t *vt, int64_t cap_vt,
                             int64_t *n_vt, int32_t *ee, int64_t cap_ee, int64_t *n_ee) {
    API_BEGIN(h)
    if (!x0 || !x1) throw Error(PDC_ERR_ARG, "pdc_op_broadphase: NULL positions");
    h->ensure_topology();
    DevBuf<float4> a, b;
    upload_f4(h, x0, h->nv_all, a);
    upload_f4(h, x1, h->nv_all, b);
    for (int tries = 0;; ++tries) {
        PDC_CK(cudaMemsetAsync(h->sc.p, 0, sizeof(Scalars), h->s));
        h->bp.run(h->s, h->coll(), a, b, h->dhat, &h->sc.p->overflow);
        h->read_scalars();
        int ovf = h->hsc->overflow;
        if (!ovf) break;
        if (tries > 6) throw Error(PDC_ERR_CAPACITY, "broad phase capacity");
        BroadPhase &bp = h->bp;
        long long cvt = bp.cap_vt * ((ovf & OVF_VT) ? 2 : 1), cee = bp.cap_ee * ((ovf & OVF_EE) ? 2 : 1),
                  cent = bp.cap_ent * ((ovf & OVF_HASH) ? 2 : 1);
        if (ovf & OVF_CELLS) bp.cell_scale *= 4.f;
        if (ovf & OVF_SLOTS) bp.grow_slots(h->coll(), true, true);
        bp.reserve(h->coll(), cvt, cee, cent, h->s);
    }
    BroadPhase &bp = h->bp;
    long long nv_ = 0, ne_ = 0;
    bp.cnt_vt_d[bp.cur].download(&nv_, 1, h->s);
    bp.cnt_ee_d[bp.cur].download(&ne_, 1, h->s);
    PDC_CK(cudaStreamSynchronize(h->s));
    if (n_vt) *n_vt = nv_;
    if (n_ee) *n_ee = ne_;
    if (vt && cap_vt > 0) {
        long long k = std::min<long long>(cap_vt, nv_);
        if (k) PDC_CK(cudaMemcpyAsync(vt, bp.vt[bp.cur].p, sizeof(int2) * k, cudaMemcpyDeviceToHost, h->s));
    }
    if (ee && cap_ee > 0) {
        long long k = std::min<long long>(cap_ee, ne_);
        if (k) {
            DevBuf<int4> q;
            q.alloc(k);
            launch_pairs_to_quads(h->s, h->coll(), bp.ee[bp.cur], k, q);
            PDC_CK(cudaMemcpyAsync(ee, q.p, sizeof(int4) * k, cudaMemcpyDeviceToHost, h->s));
        }
    }
    PDC_CK(cudaStreamSynchronize(h->s));
    API_END(h)
}

static void upload_quads(pdc_handle h, const int32_t *quads, const int32_t *kinds, int64_t np, DevBuf<int4> &q,
                         DevBuf<int> &k) {
    std::vector<int4> qh(np);
    for (int64_t i = 0; i < np; ++i) {
        qh[i] = make_int4(quads[4 * i], quads[4 * i + 1], quads[4 * i + 2], quads[4 * i + 3]);
        for (int j = 0; j < 4; ++j)
            if (quads[4 * i + j] < 0 || quads[4 * i + j] >= h->nv_all) throw Error(PDC_ERR_ARG, "vertex id out of range");
        if (kinds[i] != 0 && kinds[i] != 1) throw Error(PDC_ERR_ARG, "kind must be 0 or 1");
    }
    q.upload(qh, h->s);
    k.upload(kinds, np, h->s);
}

pdc_status pdc_op_ccd(pdc_handle h, const float *x0, const float *x1, const int32_t *quads, const int32_t *kinds,
                      int64_t np, double *toi) {
    API_BEGIN(h)
    if (np < 0 || (np > 0 && (!x0 || !x1 || !quads || !kinds || !toi))) throw Error(PDC_ERR_ARG, "pdc_op_ccd: NULL");
    if (np == 0) return PDC_OK;
    h->ensure_topology();
    DevBuf<float4> a, b;
    upload_f4(h, x0, h->nv_all, a);
    upload_f4(h, x1, h->nv_all, b);
    DevBuf<int4> q;
    DevBuf<int> k;
    upload_quads(h, quads, kinds, np, q, k);
    DevBuf<double> t;
    t.alloc(np);
    launch_ccd_quads(h->s, q, k, np, a, b, h->P.eta_ccd, t);
    t.download(toi, np, h->s);
    PDC_CK(cudaStreamSynchronize(h->s));
    API_END(h)
}

pdc_status pdc_op_partial_ccd(pdc_handle h, const float *x0, const float *x1, const int32_t *quads,
                              const int32_t *kinds, int64_t np, int32_t *active) {
    API_BEGIN(h)
    if (np < 0 || (np > 0 && (!x0 || !x1 || !quads || !kinds || !active)))
        throw Error(PDC_ERR_ARG, "pdc_op_partial_ccd: NULL");
    if (np == 0) return PDC_OK;
    h->ensure_topology();
    DevBuf<float4> a, b;
    upload_f4(h, x0, h->nv_all, a);
    upload_f4(h, x1, h->nv_all, b);
    DevBuf<int4> q;
    DevBuf<int> k;
    upload_quads(h, quads, kinds, np, q, k);
    DevBuf<int> out;
    out.alloc(np);
    launch_partial_quads(h->s, q, k, np, a, b, h->cparams(), out);
    out.download(active, np, h->s);
    PDC_CK(cudaStreamSynchronize(h->s));
    API_END(h)
}

pdc_status pdc_op_contact(pdc_handle h, const float *x0, const float *x, const int32_t *quads, const int32_t *kinds,
                          const float *w, int64_t np, float *cw, float *cf) {
    API_BEGIN(h)
    if (!x0 || !x || !cw || !cf || np < 0 || (np > 0 && (!quads || !kinds || !w)))
        throw Error(PDC_ERR_ARG, "pdc_op_contact: NULL");
    h->ensure_topology();
    DevBuf<float4> a, b;
    upload_f4(h, x0, h->nv_all, a);
    upload_f4(h, x, h->nv_all, b);
    DevBuf<int4> q;
    DevBuf<int> k;
    DevBuf<float> wd;
    DevBuf<ActivePair> ap;
    DevBuf<int> na;
    na.alloc(1);
    ap.alloc(std::max<int64_t>(np, 1));
    if (np > 0) {
        upload_quads(h, quads, kinds, np, q, k);
        wd.upload(w, np, h->s);
    }
    launch_activate_quads(h->s, q, k, wd, np, a, ap, na);
    h->CW.zero(h->s);
    h->CF.zero(h->s);
    launch_contact(h->s, h->coll(), ap, na, (int)std::max<int64_t>(np, 1), b, h->dhat, h->CW, h->CF);
    h->CW.download(cw, h->n, h->s);
    get_f4(h, h->CF, cf, 0);
    API_END(h)
}

static void upload_contact(pdc_handle h, const float *cw, const float *cf) {
    if (cw) {
        h->CW.upload(cw, h->n, h->s);
    } else {
        h->CW.zero(h->s);
    }
    if (cf) {
        PDC_CK(cudaMemcpyAsync(h->stage3.p, cf, sizeof(float) * 3 * h->n, cudaMemcpyHostToDevice, h->s));
        k_f3_to_f4<<<nb(h->n), 256, 0, h->s>>>(h->n, h->stage3, h->CF);
        PDC_LAUNCH_CK();
    } else {
        h->CF.zero(h->s);
    }
}

pdc_status pdc_op_residual(pdc_handle h, const float *x, const float *z, const float *cw, const float *cf, float *r) {
    API_BEGIN(h)
    if (!x || !z || !r) throw Error(PDC_ERR_ARG, "pdc_op_residual: NULL");
    // reference x* = x, displacement u = 0, z - x* = z - x (differences in double)
    DevBuf<float4> a, u0, zr;
    upload_f4(h, x, h->n, a);
    std::vector<float> d(3 * (size_t)h->n);
    for (size_t k = 0; k < d.size(); ++k) d[k] = (float)((double)z[k] - (double)x[k]);
    upload_f4(h, d.data(), h->n, zr);
    u0.alloc(h->n);
    u0.zero(h->s);
    upload_contact(h, cw, cf);
    launch_residual(h->s, h->cloth(), a, u0, zr, h->CW, h->CF, h->R, nullptr, nullptr, 0);
    get_f4(h, h->R, r, 0);
    API_END(h)
}

pdc_status pdc_op_global_solve(pdc_handle h, const float *x, const float *z, const float *cw, const float *cf,
                               int32_t r, int32_t cycles, int32_t sweeps, float *x_out) {
    API_BEGIN(h)
    if (!x || !z || !x_out || cycles < 1 || sweeps < 0) throw Error(PDC_ERR_ARG, "pdc_op_global_solve: bad arguments");
    if (r < 0 || r > h->r_warm) throw Error(PDC_ERR_ARG, "pdc_op_global_solve: r exceeds the basis size");
    if (r > R_REUSE_MAX) throw Error(PDC_ERR_ARG, "pdc_op_global_solve: r must be <= 512");
    cudaStream_t s = h->s;
    int n = h->n;
    DevBuf<float4> xa, za, ua, xo;
    upload_f4(h, x, n, xa);
    std::vector<float> dz(3 * (size_t)n);
    for (size_t k = 0; k < dz.size(); ++k) dz[k] = (float)((double)z[k] - (double)x[k]);
    upload_f4(h, dz.data(), n, za);
    ua.alloc(n);
    ua.zero(s);
    xo.alloc(n);
    upload_contact(h, cw, cf);
    ClothView c = h->cloth();
    if (h->dA.n < dA_elems(r)) h->dA.alloc(dA_elems(r));
    // the factorised path with the leading r columns: reduced matrix U^T (H + diag(cw)) U
    SubspaceView S = h->sub(0, r);
    SubspaceWork W = h->work();
    DevBuf<int> one, ncv;
    int o1 = 1;
    one.upload(&o1, 1, s);
    ncv.alloc(1);
    launch_contact_list(s, n, h->CW, h->contact_list, ncv);
    launch_residual(s, c, xa, ua, za, h->CW, h->CF, h->R, nullptr, nullptr, 0);
    float4 *din = h->D0, *dout = h->D1;
    bool have = false;
    for (int cyc = 0; cyc < cycles; ++cyc) {
        const float4 *rl = h->R;
        if (have) {
            launch_linear_residual(s, c, h->CW, h->R, din, h->RL);
            rl = h->RL;
        }
        if (r > 0) {
            launch_project(s, S, rl, one, W);
            PDC_CK(cudaMemsetAsync(W.dA, 0, sizeof(double) * dA_zero_elems(r), s));
            launch_syrk(s, S, h->contact_list, ncv, h->CW, W);
            launch_reduced_solve(s, S, one, W);
            launch_lift(s, S, one, W, have ? din : nullptr, dout);
            std::swap(din, dout);
            have = true;
        }
        if (!have) {
            PDC_CK(cudaMemsetAsync(din, 0, sizeof(float4) * n, s));
            have = true;
        }
        for (int k = 0; k < sweeps; ++k) {
            launch_sweep(s, c, h->CW, h->R, din, dout, (float)h->omega, nullptr, nullptr, nullptr);
            std::swap(din, dout);
        }
    }
    launch_sweep(s, c, h->CW, h->R, din, dout, 0.f, ua, ua.p, nullptr, nullptr, 1.f, xa, xo.p);  // x + delta
    get_f4(h, xo, x_out, 0);
    API_END(h)
}

pdc_status pdc_op_project(pdc_handle h, const float *v, int32_t r, double *g) {
    API_BEGIN(h)
    if (!v || !g) throw Error(PDC_ERR_ARG, "pdc_op_project: NULL");
    if (r <= 0 || r > h->r_warm) throw Error(PDC_ERR_ARG, "pdc_op_project: r must be in [1, r_warm]");
    DevBuf<float4> va;
    upload_f4(h, v, h->n, va);
    DevBuf<int> zero;
    zero.alloc(1);
    zero.zero(h->s);
    SubspaceView S = h->sub(r, 0);
    SubspaceWork W = h->work();
    launch_project(h->s, S, va, zero, W, false);
    PDC_CK(cudaMemcpyAsync(g, W.g, sizeof(double) * 3 * r, cudaMemcpyDeviceToHost, h->s));
    int fl = 0;
    h->sflag.download(&fl, 1, h->s);
    PDC_CK(cudaStreamSynchronize(h->s));
    if (fl & PDC_DEVERR_UMMA) {
        h->sflag.zero(h->s);
        throw Error(PDC_ERR_TIMEOUT, "pdc_op_project: tensor-core kernel timed out");
    }
    API_END(h)
}

pdc_status pdc_op_lift(pdc_handle h, const double *q, int32_t r, float *out) {
    API_BEGIN(h)
    if (!q || !out) throw Error(PDC_ERR_ARG, "pdc_op_lift: NULL");
    if (r <= 0 || r > h->r_warm) throw Error(PDC_ERR_ARG, "pdc_op_lift: r must be in [1, r_warm]");
    std::vector<float> qf(3 * (size_t)r);
    for (size_t k = 0; k < qf.size(); ++k) qf[k] = (float)q[k];
    SubspaceView S = h->sub(r, 0);
    SubspaceWork W = h->work();
    PDC_CK(cudaMemcpyAsync(W.q, qf.data(), sizeof(float) * qf.size(), cudaMemcpyHostToDevice, h->s));
    DevBuf<int> zero;
    zero.alloc(1);
    zero.zero(h->s);
    DevBuf<float4> o;
    o.alloc(h->n);
    launch_lift(h->s, S, zero, W, nullptr, o, false);
    int fl = 0;
    h->sflag.download(&fl, 1, h->s);
    PDC_CK(cudaStreamSynchronize(h->s));
    if (fl & PDC_DEVERR_UMMA) {
        h->sflag.zero(h->s);
        throw Error(PDC_ERR_TIMEOUT, "pdc_op_lift: tensor-core kernel timed out");
    }
    get_f4(h, o, out, 0);
    API_END(h)
}

}  // extern "C"

// ============================================================================ allocation-free contact springs
// Library-integration entry point with no counterpart in the paper: the
// collision springs of pdc_op_contact computed without allocating device
// memory.  Callers that need it: a process whose caching allocator already
// holds nearly all free device memory (a cudaMalloc inside the call would
// fail or force the allocator to release memory), and latency-bound loops,
// because cudaFree synchronises the whole device and stalls other streams.
// All temporaries live in this one statically sized device array; calls that
// overlap in time on one device share it and therefore race.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PDC_NOALLOC_SCRATCH_BYTES];

namespace pdc {
namespace {

// bad += number of quads with a vertex id outside [0, nv) or a kind not 0/1
__global__ void k_check_quads(long long np, const int4 *__restrict__ q, const int *__restrict__ kinds, int nv,
                              int *bad) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < np;
         i += (long long)gridDim.x * blockDim.x) {
        int4 v = q[i];
        int k = kinds[i];
        bool ok = v.x >= 0 && v.x < nv && v.y >= 0 && v.y < nv && v.z >= 0 && v.z < nv && v.w >= 0 && v.w < nv &&
                  (k == 0 || k == 1);
        if (!ok) atomicAdd(bad, 1);
    }
}

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_base[NOALLOC_MAX_DEVICES];

// Device address of the static scratch on the current device, looked up
// once per device (the lookup can load the module, so it must not happen
// for the first time inside a stream capture).
unsigned char *noalloc_scratch() {
    int dev = -1;
    PDC_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) throw Error(PDC_ERR_CUDA, "noalloc scratch: device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_base[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            throw Error(PDC_ERR_CUDA, std::string("cudaGetSymbolAddress(noalloc scratch): ") + cudaGetErrorString(e));
        g_noalloc_base[dev] = p;
    }
    return (unsigned char *)g_noalloc_base[dev];
}

inline size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace
}  // namespace pdc

extern "C" pdc_status pdc_op_contact_noalloc(pdc_handle h, const float *x0, const float *x, const int32_t *quads,
                                             const int32_t *kinds, const float *w, int64_t np, float *cw, float *cf,
                                             void *stream) {
    API_BEGIN(h)
    if (!x0 || !x || !cw || !cf || np < 0 || (np > 0 && (!quads || !kinds || !w)))
        throw Error(PDC_ERR_ARG, "pdc_op_contact_noalloc: NULL pointer or negative np");
    if (((uintptr_t)quads & 15) != 0) throw Error(PDC_ERR_ARG, "pdc_op_contact_noalloc: quads must be 16-byte aligned");
    if (h->topo_dirty) throw Error(PDC_ERR_STATE, "pdc_op_contact_noalloc: collision topology not built");
    const size_t nv = (size_t)h->nv_all, n = (size_t)h->n;
    // scratch layout: X0 | X1 | CF | active pairs | counters (n_act, bad)
    const size_t off_x1 = round256(sizeof(float4) * nv);
    const size_t off_cf = off_x1 + round256(sizeof(float4) * nv);
    const size_t off_act = off_cf + round256(sizeof(float4) * n);
    // room for the pair list: what is left after the counters, in whole
    // 256-byte units so that the rounded-up list still fits; np is compared
    // against it before a byte count is formed from it
    const size_t act_room =
        PDC_NOALLOC_SCRATCH_BYTES > off_act + 256 ? ((PDC_NOALLOC_SCRATCH_BYTES - off_act - 256) & ~(size_t)255) : 0;
    const size_t np_max = act_room / sizeof(ActivePair);
    if (act_room < 256 || (uint64_t)np > np_max)
        throw Error(PDC_ERR_CAPACITY,
                    "pdc_op_contact_noalloc: np=" + std::to_string(np) + " pairs with " + std::to_string(nv) +
                        " collision vertices exceed the static scratch of " +
                        std::to_string((size_t)PDC_NOALLOC_SCRATCH_BYTES) + " bytes (at most " +
                        std::to_string(np_max) + " pairs here); use pdc_op_contact");
    const size_t off_cnt = off_act + round256(sizeof(ActivePair) * (size_t)std::max<int64_t>(np, 1));
    unsigned char *base = noalloc_scratch();
    cudaStream_t s = stream ? (cudaStream_t)stream : h->s;
    float4 *X0 = (float4 *)base, *X1 = (float4 *)(base + off_x1), *CFa = (float4 *)(base + off_cf);
    ActivePair *AP = (ActivePair *)(base + off_act);
    int *n_act = (int *)(base + off_cnt), *bad = n_act + 1;
    const int4 *q = (const int4 *)quads;
    if (np > 0) {
        PDC_CK(cudaMemsetAsync(bad, 0, sizeof(int), s));
        k_check_quads<<<(int)std::min<long long>((np + 255) / 256, 152LL * 8), 256, 0, s>>>(np, q, kinds, (int)nv, bad);
        PDC_LAUNCH_CK();
        int nbad = 0;
        PDC_CK(cudaMemcpyAsync(&nbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
        PDC_CK(cudaStreamSynchronize(s));
        if (nbad)
            throw Error(PDC_ERR_ARG, "pdc_op_contact_noalloc: " + std::to_string(nbad) +
                                         " pairs with a vertex id out of range or a kind other than 0/1");
    }
    if (nv) {
        k_f3_to_f4<<<nb((long long)nv), 256, 0, s>>>((int)nv, x0, X0);
        k_f3_to_f4<<<nb((long long)nv), 256, 0, s>>>((int)nv, x, X1);
        PDC_LAUNCH_CK();
    }
    launch_activate_quads(s, q, kinds, w, np, X0, AP, n_act);
    PDC_CK(cudaMemsetAsync(cw, 0, sizeof(float) * n, s));
    PDC_CK(cudaMemsetAsync(CFa, 0, sizeof(float4) * n, s));
    launch_contact(s, h->coll(), AP, n_act, (int)std::max<int64_t>(np, 1), X1, h->dhat, cw, CFa);
    if (n) {
        k_f4_to_f3<<<nb((long long)n), 256, 0, s>>>((int)n, CFa, cf);
        PDC_LAUNCH_CK();
    }
    API_END(h)
}
