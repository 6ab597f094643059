// Subspace-reuse kernels (Sec. 5) and basis construction.
#pragma once
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
    double *dA;        // [r_c][r_c] collision update of the reduced matrix (FP64)
    int *flag;         // factorisation status
};

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
// dA = sum over listed vertices of cw_v U_v U_v^T (leading r_c columns);
// zero = false: dA has been zeroed already.
void launch_syrk(cudaStream_t s, const SubspaceView &S, const int *list, const int *n_cv, const float *cw,
                 SubspaceWork &W, bool zero = true);
// q = (reduced matrix)^-1 g.
void launch_reduced_solve(cudaStream_t s, const SubspaceView &S, const int *n_cv, SubspaceWork &W);
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
