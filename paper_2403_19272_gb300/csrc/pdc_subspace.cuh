// Subspace-reuse kernels (Sec. 5) and basis construction.
#pragma once
#include <algorithm>

#include "pdc_internal.cuh"
#include "pdc_umma.cuh"

namespace pdc {

// Which of the two bases a solve uses: with no collision spring the full
// basis of r_nc columns and the precomputed inverse of U^T H U; with springs
// the leading r_c columns and a per-iteration factorisation of
// U^T (H + dH) U (Eq. subspace_collision, Eq. uu).
struct SubspaceView {
    int n;
    int ld;                    // row stride of U (r_warm)
    int r_nc, r_c;             // columns used without / with collision springs
    const float *U32;          // [n][ld] FP32 basis (plain form)
    const __nv_bfloat16 *U16;  // [n][ld] BF16 basis (mixed form, precision 1)
    const __half *Uh;          // [n][ld] FP16 basis, power-of-two scaled (mixed form, precision 2)
    const double *A0;          // [ld][ld] U^T H U of the stored basis
    const double *A0inv;       // [r_nc][r_nc] inverse (FP64)
    const float *A0inv32;      // [r_nc][r_nc] inverse (FP32)
    int precision;             // 0 plain FP32, 1 mixed BF16, 2 mixed FP16
    // compact copy of the leading ldc columns ([n][ldc], same values as U):
    // the solves with collision springs stream only these
    int ldc;                   // 0: no compact copy
    const float *Uc32;
    const __nv_bfloat16 *Uc16;
    const __half *Uch;
    // tensor-core path of the full-basis solves (host pointer; NULL: off)
    const UmmaMaps *umma;
    float *umma_partial;       // [tiles][ld][3]
    int *dev_err;              // status word receiving PDC_DEVERR_UMMA
    int overlap;               // tensor-core path: launch as programmatic dependents
    const int *live;           // device loop flag (see loop_dead), or NULL
};

struct SubspaceWork {
    float *partial;    // [blocks][ld][3]
    double *g;         // [ld][3]
    float *q;          // [ld][3]
    double *dA;        // collision update of the reduced matrix (FP64), see dA_elems
    int *flag;         // factorisation status
};

// Solves with collision springs on up to CHOL_ONE_CTA columns factor the
// reduced matrix in one CTA's shared memory, dA holding [r_c][r_c].  Wider
// ones pad r_c to R = a multiple of CHOL_B and factor by blocks over many
// CTAs: dA then holds the [R][R] matrix (lower triangle used), the factors
// of its diagonal blocks ([R/CHOL_B][CHOL_B][CHOL_B]), the right-hand side
// b, the forward solution y and the solution q (each [R][3]) and a
// failed-pivot marker.
constexpr int CHOL_ONE_CTA = 128;
constexpr int CHOL_B = 32;
constexpr int R_REUSE_MAX = 512;
__host__ __device__ inline int chol_pad(int r) { return (r + CHOL_B - 1) / CHOL_B * CHOL_B; }
// doubles of dA a solve on r_c columns uses / that must be zero before the update
inline size_t dA_elems(int r) {
    if (r <= CHOL_ONE_CTA) return (size_t)std::max(r * r, 1);
    size_t R = (size_t)chol_pad(r);
    return R * R + (size_t)(CHOL_B + 9) * R + 1;
}
inline size_t dA_zero_elems(int r) {
    if (r <= CHOL_ONE_CTA) return (size_t)r * r;
    size_t R = (size_t)chol_pad(r);
    return R * R;
}

constexpr int PROJ_BLOCKS = 608;

// g = U[:, :r]^T rl  (r = r_c if *n_cv > 0 else r_nc).  maybe_contacts =
// false promises *n_cv == 0 (only the full-basis kernel is launched).  With
// device_choice (and device_path_choice(S)) an iteration that may have
// springs launches both the tensor-core full-basis kernels and the compact
// ones, and *n_cv (read on the device) decides which of them work, so that
// the host need not read the count back.
void launch_project(cudaStream_t s, const SubspaceView &S, const float4 *rl, const int *n_cv, SubspaceWork &W,
                    bool maybe_contacts = true, bool device_choice = false);
// whether the tensor-core / compact choice of a spring iteration can be left to the device
bool device_path_choice(const SubspaceView &S);
// dA = sum over listed vertices of cw_v U_v U_v^T (leading r_c columns;
// above CHOL_ONE_CTA columns only the lower block triangle of the padded
// matrix); zero = false: dA has been zeroed already.
void launch_syrk(cudaStream_t s, const SubspaceView &S, const int *list, const int *n_cv, const float *cw,
                 SubspaceWork &W, bool zero = true);
// q = (reduced matrix)^-1 g.  factor = false: the reduced matrix with
// springs is the one the previous call factored (only the blocked path above
// CHOL_ONE_CTA columns keeps its factor; the one-CTA path refactors).
void launch_reduced_solve(cudaStream_t s, const SubspaceView &S, const int *n_cv, SubspaceWork &W,
                          bool factor = true);
// dout = din + U q (din may be NULL: zero).
void launch_lift(cudaStream_t s, const SubspaceView &S, const int *n_cv, const SubspaceWork &W, const float4 *din,
                 float4 *dout, bool maybe_contacts = true, bool device_choice = false);
// rl = r - (H + diag(cw)) delta (linear residual of the global system).
void launch_linear_residual(cudaStream_t s, const ClothView &c, const float *cw, const float4 *r,
                            const float4 *delta, float4 *rl);

// Basis construction (eigen.cu): the r lowest eigenvectors of the rest
// matrix restricted to free vertices, by Chebyshev-filtered subspace
// iteration with Rayleigh-Ritz; returns U [n][r] (pinned rows 0) and the
// Ritz values.
void build_basis(cudaStream_t s, const ClothView &c, int r, int iters, uint64_t seed, std::vector<float> &U,
                 std::vector<double> &ritz);
// A = U^T H U (FP64) for a basis stored on the device [n][ld] (FP32).
void reduced_matrix(cudaStream_t s, const ClothView &c, const float *U, int ld, std::vector<double> &A);

// Host dense helpers (FP64).
bool cholesky_inplace(std::vector<double> &A, int n);          // lower factor in place
void spd_inverse(const std::vector<double> &A, int n, std::vector<double> &Ainv);
void sym_eig(std::vector<double> A, int n, std::vector<double> &w, std::vector<double> &V);  // A = V diag(w) V^T, ascending

}  // namespace pdc
