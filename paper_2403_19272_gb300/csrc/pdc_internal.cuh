// Internal declarations of the pdcloth CUDA library (sm_103a).
//
// Layout in HBM (one cloth of n vertices, m triangles, nh hinges):
//   vertex streams   float4 (x, y, z, 0), 16 B per vertex: x*, v*, z, x,
//                    x^-, residual r, Jacobi increments, contact force
//   per-triangle     int4 ids, float4 (g1, g2) rows of Dm^-1, float weight
//   per-hinge        int4 ids, float4 cotangent stencil K, weight, rest |s|
//   vertex incidence CSR of (element << 2 | corner) for the gather residual
//   rest matrix H    diagonal + ELL off-diagonals (column-major, width W)
//   basis U          row-major [n][r_warm] (FP32 or BF16) + column-major copy
//   collision set    cloth vertices then obstacle vertices; triangles and
//                    edges likewise; broad-phase hash and pair lists
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "../../include/pdcloth.h"

namespace pdc {

// ---------------------------------------------------------------- errors
struct Error : std::runtime_error {
    pdc_status code;
    Error(pdc_status c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define PDC_CK(call)                                                                                   \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess)                                                                         \
            throw ::pdc::Error(PDC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_) +       \
                                                 " (" __FILE__ ":" + std::to_string(__LINE__) + ")");   \
    } while (0)

#define PDC_LAUNCH_CK() PDC_CK(cudaGetLastError())

// ---------------------------------------------------------------- device buffer
template <class T> struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    void alloc(size_t count) {
        if (count == n && p) return;
        release();
        if (count == 0) return;
        PDC_CK(cudaMalloc((void **)&p, count * sizeof(T)));
        n = count;
    }
    void zero(cudaStream_t s) {
        if (p) PDC_CK(cudaMemsetAsync(p, 0, n * sizeof(T), s));
    }
    void upload(const T *h, size_t count, cudaStream_t s) {
        alloc(count);
        if (count) PDC_CK(cudaMemcpyAsync(p, h, count * sizeof(T), cudaMemcpyHostToDevice, s));
    }
    void upload(const std::vector<T> &h, cudaStream_t s) { upload(h.data(), h.size(), s); }
    void download(T *h, size_t count, cudaStream_t s) const {
        if (count) PDC_CK(cudaMemcpyAsync(h, p, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    }
    operator T *() const { return p; }
};

// ---------------------------------------------------------------- small vector math
__host__ __device__ inline float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__host__ __device__ inline float4 f4(float3 a) { return make_float4(a.x, a.y, a.z, 0.f); }
__host__ __device__ inline float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__host__ __device__ inline float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__host__ __device__ inline float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__host__ __device__ inline float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ inline float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// ---------------------------------------------------------------- dependent launches
// A kernel launched by launch_dependent(true, ...) may begin while the kernel
// before it in the stream is still running.  It must call grid_dep_wait()
// before touching any memory that an earlier kernel writes or reads (the wait
// returns once the previous grid has completed and its writes are visible;
// with a plain launch it returns at once), and every thread calls it before
// exiting, so that this grid's completion implies its predecessor's.
// grid_dep_release() lets the next dependent launch begin.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_dependent(bool overlap, void (*kernel)(KArgs...), int grid, int block, size_t smem,
                             cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = overlap ? 1 : 0;
    PDC_CK(cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...));
}

// ---------------------------------------------------------------- device views
// Rest model of the cloth (read-only in the step kernels).
struct ClothView {
    int n, m, nh;
    const int4 *tri;       // [m] (i0, i1, i2, 0)
    const float4 *tri_g;   // [m] (g1.x, g1.y, g2.x, g2.y); g0 = -g1 - g2
    const float *tri_w;    // [m] k_stretch * area
    const int4 *hin;       // [nh] (x0, x1 | x2, x3)
    const float4 *hin_K;   // [nh] cotangent stencil
    const float *hin_w;    // [nh] 3 k_bend / (A_A + A_B)
    const float *hin_slen; // [nh] |sum_j K_j X_j| at rest
    const float4 *hin_srest; // [nh] rest stencil vector (fallback direction)
    const int *vt_off;     // [n+1] triangle incidence
    const int *vt_list;    // (t << 2) | corner
    const int *vh_off;     // [n+1] hinge incidence
    const int *vh_list;    // (h << 2) | slot
    const float *mh2;      // [n] m / h^2
    const float *hdiag;    // [n] diag(H)
    const unsigned char *is_free; // [n]
    int ell_w;
    const int *ell_col;    // [ell_w][n]
    const short *ell_dcol; // [ell_w][n] column minus row when every offset fits 16 bits (else NULL)
    int overlap;           // launch the step kernels as programmatic dependents
    const float *ell_val;  // [ell_w][n]
    // the same off-diagonals in blocks of ELL_TILE_ROWS rows, one contiguous
    // tile per block: [ell_tw][ELL_TILE_ROWS] float values, then
    // [ell_tw][ELL_TILE_ROWS] 16-bit offsets, zero-padded (NULL when the
    // offsets do not fit 16 bits or the width exceeds 16)
    const unsigned char *ell_tile;
    int ell_tw;            // tile width: 8, 12 or 16 (>= ell_w)
    // the same off-diagonals per patch of ELL_TILE_ROWS rows (vertices
    // consecutive in the Morton order of the rest positions), with columns
    // local to the patch and its halo (see halo_tile_bytes; NULL when some
    // patch's halo exceeds HALO_MAX or the tiles above are absent)
    const unsigned char *ell_halo;
    // two-step patch tiles (see k_cheb_step2_halo): rows = the patch and its
    // first halo ring, columns local to rows + second ring; fixed stride
    const unsigned char *ell_halo2;
    int h2_rows, h2_verts;  // largest row and vertex counts over the patches (multiples of 32)
    float4 *corner;        // scratch [3m + 4nh]: per-element corner forces of the residual
    // one-kernel residual per mesh patch (NULL when not built or not used):
    // records and their byte offsets, the largest counts over the patches
    const unsigned char *rp_rec;
    const long long *rp_off;
    int rp_loc, rp_tri, rp_hin;
    int res_block;         // threads per block of the residual kernels (64, 128 or 256)
    int cheb_mode;         // Chebyshev step reads: 0 the ELL arrays, 1 the row tiles, 2 the patch tiles,
                           // 3 the two-step patch tiles (two steps a launch)
    const int *live;       // device loop flag: the kernels do nothing when *live == 0 (NULL: always run)
};

// A kernel of an LG iteration of a device-driven loop does nothing once the
// loop has ended (*live == 0); read after grid_dep_wait().
__device__ __forceinline__ bool loop_dead(const int *live) { return live && *(const volatile int *)live == 0; }

constexpr int ELL_TILE_ROWS = 256;
inline size_t ell_tile_bytes(int tw) { return (size_t)tw * ELL_TILE_ROWS * 6; }
// Patch tile: [tw][ELL_TILE_ROWS] float values, [tw][ELL_TILE_ROWS] int16
// columns local to the patch (rows at 0..255, halo vertices from 256 on),
// [ELL_TILE_ROWS] int32 vertex ids of the rows (-1 past the last), [HALO_MAX]
// int32 vertex ids of the halo, int32 halo count, 12 bytes of padding.
constexpr int HALO_MAX = 512;
// Two-step patch tile, per patch: int4 {n_own, n_rows, n_verts, 0};
// [tw][rows] float values, [tw][rows] int16 columns local to the vertices,
// [verts] int32 vertex ids (rows first, own rows first among them; -1 past
// the counts); rows and verts are the largest counts over the patches.
__host__ __device__ constexpr size_t halo2_tile_bytes(int tw, int rows, int verts) {
    return 16 + (size_t)tw * rows * 6 + (size_t)verts * 4;
}
__host__ __device__ constexpr size_t halo_tile_bytes(int tw) {
    return (size_t)tw * ELL_TILE_ROWS * 6 + (size_t)ELL_TILE_ROWS * 4 + (size_t)HALO_MAX * 4 + 16;
}

// Device error bit set in the status word when a bounded wait for a bulk
// copy into shared memory ran out.
constexpr int PDC_DEVERR_COPY = 4;

// Collision-set topology (cloth + obstacles).
struct CollView {
    int nv, nc;            // all vertices, cloth vertices
    int nt, ne;            // all triangles, all edges
    const int4 *tri;       // [nt]
    const int2 *edge;      // [ne] (a < b)
    const unsigned char *vfixed; // [nv] 1: infinite mass (obstacle or pinned)
    unsigned int *guard;   // the handle's index-guard word (GuardBits), or NULL
    const int *live;       // device loop flag (see loop_dead), or NULL
    // per-instance line search (batched form): instance of each collision
    // vertex (-1: none) and per-instance minimum time of impact (double bits);
    // NULL when the union takes one step fraction
    const int *vinst;
    unsigned long long *toi_inst;
};

// Scalars written by reductions (device).
struct Scalars {
    double rsq;            // sum of squared residual entries
    unsigned int dxmax;    // max |delta| (float bits)
    unsigned int pad0;
    unsigned long long toi_min; // min time of impact (double bits, >= 0)
    int n_active;          // active pairs appended this pass
    int n_contact_v;       // contact vertices
    int overflow;          // buffer overflow flags (bit mask)
    int pad1;
    long long n_vt, n_ee;  // candidate counts
    long long n_hash;      // hash insertions
};

// ---------------------------------------------------------------- device-side loop control
// State of the LG loop that is running when its stopping tests are taken on
// the device (loops run as CUDA graphs): the tests of the host-driven loop
// (relative residual, stagnation, step change, iteration cap) and the
// Anderson-mixing bookkeeping, in one struct that one thread updates.
struct LoopCtl {
    double rho0;          // PD residual at z (set at the start of the step)
    double rel;           // last relative residual the stopping test saw
    double stag_best;     // best residual of the loop (stagnation test)
    double aa_hist_min;   // smallest residual since the last history restart
    int aa_hist_n;        // residuals seen since that restart
    int iters;            // iterations of this loop that ran their solve
    int go;               // 1 while the loop continues
    int springs;          // the current iteration has collision springs
    int stag_count;       // iterations without 1 % progress
    int aa_count, aa_widx, aa_have_prev;
    int aa_slot, aa_prev, aa_ncol;  // the mixing step of the current iteration
    int warm_iters, inner_iters, contact_iters;  // totals of the step
    int device_loops;     // loops of the step whose tests ran on the device
};

// ---------------------------------------------------------------- kernels (k_pd.cu)
// Inside a step positions are x = x* + u (x* = xs fixed, u a small FP32
// displacement); zrel = z - x*; xabs receives absolute positions for the
// collision kernels.
void launch_prologue(cudaStream_t s, int n, const float4 *xs, const float4 *vs, const int *pins, const float4 *pin_tgt,
                     int npins, float h, float3 g, float4 *zrel, float4 *u, float4 *xabs, const float4 *rf = nullptr);
// residual forwarding: rebase the displacement representation on x_new (in xs)
void launch_rf_rebase(cudaStream_t s, int n, const float4 *xs, const float4 *xold, float4 *zrel, float4 *u,
                      float4 *xabs);
void launch_residual(cudaStream_t s, const ClothView &c, const float4 *xs, const float4 *u, const float4 *zrel,
                     const float *cw, const float4 *cf, float4 *r, Scalars *sc, float *r_soa, int soa_ld);
void launch_sweep(cudaStream_t s, const ClothView &c, const float *cw, const float4 *r, const float4 *din,
                  float4 *dout, float omega, const float4 *x, float4 *xout, Scalars *sc, float4 *xprev = nullptr,
                  float w_acc = 1.f, const float4 *xs = nullptr, float4 *xabs = nullptr);
// One Chebyshev step in three-term form: dout = din + alpha (din - dprev)
// + beta D^-1 (r - (H + diag cw) din) (dprev unused when alpha = 0).
void launch_cheb_step(cudaStream_t s, const ClothView &c, const float *cw, const float4 *r, const float4 *din,
                      const float4 *dprev, float4 *dout, float alpha, float beta, const float4 *x,
                      float4 *xout, Scalars *sc, float4 *xprev, float w_acc, const float4 *xs, float4 *xabs,
                      bool overlap = false, int *err = nullptr);
// Two Chebyshev steps in one launch over the two-step patch tiles
// (cheb_mode 3): dmid = the first step's result, dout = the second's
// (coefficients a1, b1 then a2, b2); the iterate outputs as the second step
// of launch_cheb_step.  cheb_two_steps: whether the view selects it.
bool cheb_two_steps(const ClothView &c);
void launch_cheb_step2(cudaStream_t s, const ClothView &c, const float *cw, const float4 *r, const float4 *din,
                       const float4 *dprev, float4 *dmid, float4 *dout, float a1, float b1, float a2, float b2,
                       const float4 *x, float4 *xout, Scalars *sc, float4 *xprev, float w_acc, const float4 *xs,
                       float4 *xabs, bool overlap, int *err);
// Anderson mixing step on the iterate u (= u_k + delta_k on entry, u_{k+1} on exit).
// Gb must have been zeroed (aa_clear) after the previous mixing step.
void launch_aa(cudaStream_t s, int n, const unsigned char *is_free, const float4 *delta, float4 *x, float4 *fprev,
               float4 *gprev, float4 *dF, float4 *dG, int slot, int have_prev, int ncol, double *Gb, float *theta,
               const float4 *xs, float4 *xabs, bool overlap);
// The same step with slot, have_prev and the column count read from the
// loop state on the device (aa_slot, aa_prev, aa_ncol; at most m columns).
void launch_aa_device(cudaStream_t s, int n, const unsigned char *is_free, const float4 *delta, float4 *x,
                      float4 *fprev, float4 *gprev, float4 *dF, float4 *dG, int m, const LoopCtl *ctl, double *Gb,
                      float *theta, const float4 *xs, float4 *xabs, bool overlap);
void aa_clear(cudaStream_t s, double *Gb, const int *live = nullptr);
int aa_gram_doubles();  // entries of the Anderson normal-equation buffer
// Zeroes `bytes` (a multiple of 4) at p unless *live == 0; with live NULL a
// plain stream memset.
void launch_live_zero(cudaStream_t s, const int *live, void *p, size_t bytes);
// out = a + s (b - a) with s = *s_frac, or with vinst (per-instance line
// search) s_inst[vinst[i]] for vertices of an instance (vinst[i] >= 0)
void launch_lerp(cudaStream_t s, int nv, const float4 *a, const float4 *b, const double *s_frac, float4 *out,
                 const int *vinst = nullptr, const double *s_inst = nullptr);
void launch_set_pins(cudaStream_t s, const int *pins, int npins, const float4 *tgt, const float4 *xs, float4 *u,
                     float4 *xabs);
void launch_restart(cudaStream_t s, int n, const float4 *xs, const float4 *um, float4 *u, float4 *xabs);
void launch_scale_disp(cudaStream_t s, int n, const float4 *xs, const float4 *u, const double *s_frac, float4 *um,
                       float4 *xm, const int *vinst = nullptr, const double *s_inst = nullptr);

}  // namespace pdc
