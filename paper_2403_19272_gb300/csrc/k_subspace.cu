// Subspace-reuse kernels (Sec. 5): projection g = U^T r, the collision
// update of the reduced matrix (Eq. uu), the reduced solve and the lift
// delta = U q (Eq. subspace_collision), plus the linear residual used when a
// global solve runs several correction cycles.
//
// Reduced solves: without collision springs the reduced matrix U^T H U is
// fixed and its inverse is precomputed (the explicit-inverse idea of the
// paper's implementation section), so the solve is a matrix-vector product;
// with springs the leading r_c x r_c block plus the SYRK update is factored
// by Cholesky in FP64 (in one CTA up to 128 columns, by blocks over many
// CTAs above).  The inverse is FP64 in the mixed forms and FP32 in the
// plain form.
#include <algorithm>
#include <type_traits>

#include "pdc_subspace.cuh"

namespace pdc {

namespace {

__device__ inline int active_r(const SubspaceView &S, const int *n_cv) {
    return (n_cv && *n_cv > 0) ? S.r_c : S.r_nc;
}

// The compact copy serves the solves with collision springs when it holds
// their r_c columns.
__host__ __device__ inline bool compact_covers(const SubspaceView &S) { return S.ldc > 0 && S.r_c > 0 && S.r_c <= S.ldc; }
__device__ inline bool compact_active(const SubspaceView &S, const int *n_cv) {
    return compact_covers(S) && n_cv && *n_cv > 0;
}

template <class TU> __device__ inline float tofloat(TU v);
template <> __device__ inline float tofloat<float>(float v) { return v; }
template <> __device__ inline float tofloat<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ inline float tofloat<__half>(__half v) { return __half2float(v); }

constexpr int PROJ_T = 256;
constexpr int PROJ_W = PROJ_T / 32;  // warps per block

// 8 consecutive basis entries of one row as floats (one 16-byte load for
// BF16, two for FP32).  Requires 16-byte aligned rows (ld % 8 == 0).
__device__ inline void load8(const __nv_bfloat16 *p, float u[8]) {
    uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float2 f = __bfloat1622float2(h[k]);
        u[2 * k] = f.x;
        u[2 * k + 1] = f.y;
    }
}
__device__ inline void load8(const __half *p, float u[8]) {
    uint4 v = __ldg(reinterpret_cast<const uint4 *>(p));
    const __half2 *h = reinterpret_cast<const __half2 *>(&v);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float2 f = __half22float2(h[k]);
        u[2 * k] = f.x;
        u[2 * k + 1] = f.y;
    }
}
__device__ inline void load8(const float *p, float u[8]) {
    float4 a = __ldg(reinterpret_cast<const float4 *>(p));
    float4 b = __ldg(reinterpret_cast<const float4 *>(p) + 1);
    u[0] = a.x; u[1] = a.y; u[2] = a.z; u[3] = a.w;
    u[4] = b.x; u[5] = b.y; u[6] = b.z; u[7] = b.w;
}

// Partial projection partial[b][j][c] = sum_{rows i of block b} U[i][j] rl_i[c].
// One warp per row, lane l owns columns 8l..8l+7 of each 256-column chunk;
// NCH chunks cover r <= 256*NCH.  The warps of a block reduce in shared memory.
template <class TU, int NCH>
__global__ void __launch_bounds__(PROJ_T) k_project(SubspaceView S, const TU *__restrict__ U,
                                                    const float4 *__restrict__ rl, const int *n_cv,
                                                    float *__restrict__ partial) {
    __shared__ float s_acc[PROJ_W][256 * 3];
    if (loop_dead(S.live)) return;
    if (compact_active(S, n_cv)) return;
    int r = active_r(S, n_cv);
    if (r == 0) return;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float acc[NCH][8][3];
#pragma unroll
    for (int c = 0; c < NCH; ++c)
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[c][k][0] = acc[c][k][1] = acc[c][k][2] = 0.f;
    long long gw = (long long)blockIdx.x * PROJ_W + w, nw = (long long)gridDim.x * PROJ_W;
    constexpr int UR = NCH == 1 ? 4 : 2;  // rows in flight per warp
    for (long long i0 = gw; i0 < S.n; i0 += nw * UR) {
        float4 rv[UR];
        float u[UR][NCH][8];
#pragma unroll
        for (int q = 0; q < UR; ++q) {
            long long i = i0 + q * nw;
            bool ok = i < S.n;
            rv[q] = ok ? __ldg(rl + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            const TU *row = U + (ok ? i : 0) * S.ld;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                int j0 = c * 256 + lane * 8;
                if (ok && j0 < r) load8(row + j0, u[q][c]);
                else
#pragma unroll
                    for (int k = 0; k < 8; ++k) u[q][c][k] = 0.f;
            }
        }
#pragma unroll
        for (int q = 0; q < UR; ++q)
#pragma unroll
            for (int c = 0; c < NCH; ++c)
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    acc[c][k][0] = fmaf(u[q][c][k], rv[q].x, acc[c][k][0]);
                    acc[c][k][1] = fmaf(u[q][c][k], rv[q].y, acc[c][k][1]);
                    acc[c][k][2] = fmaf(u[q][c][k], rv[q].z, acc[c][k][2]);
                }
    }
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            int j = lane * 8 + k;
            s_acc[w][j * 3 + 0] = acc[c][k][0];
            s_acc[w][j * 3 + 1] = acc[c][k][1];
            s_acc[w][j * 3 + 2] = acc[c][k][2];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 256 * 3; e += PROJ_T) {
            int j = c * 256 + e / 3;
            if (j < r) {
                float v = 0.f;
#pragma unroll
                for (int q = 0; q < PROJ_W; ++q) v += s_acc[q][e];
                partial[((long long)blockIdx.x * S.ld + j) * 3 + e % 3] = v;
            }
        }
    }
}


// Projection and lift over the compact copy [n][ldc] (ldc <= 128): LPR =
// ldc/8 lanes share a row (8 columns each), so a warp covers 32/LPR
// consecutive rows with one contiguous 512-byte (BF16) or 1 KB (FP32) load.
template <class TU, int LPR>
__global__ void __launch_bounds__(PROJ_T) k_project_compact(SubspaceView S, const TU *__restrict__ U,
                                                            const float4 *__restrict__ rl, const int *n_cv,
                                                            float *__restrict__ partial) {
    __shared__ float s_acc[PROJ_W][128 * 3];
    if (loop_dead(S.live)) return;
    if (!compact_active(S, n_cv)) return;
    constexpr int RPW = 32 / LPR;  // rows per warp and pass
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int slot = lane / LPR, cg = lane % LPR;
    float acc[8][3];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k][0] = acc[k][1] = acc[k][2] = 0.f;
    long long gw = (long long)blockIdx.x * PROJ_W + w, nw = (long long)gridDim.x * PROJ_W;
    constexpr int UR = 4;  // passes in flight per warp
    for (long long p0 = gw; p0 * RPW < S.n; p0 += nw * UR) {
        float4 rv[UR];
        float u[UR][8];
#pragma unroll
        for (int q = 0; q < UR; ++q) {
            long long i = (p0 + q * nw) * RPW + slot;
            bool ok = i < S.n;
            rv[q] = ok ? __ldg(rl + i) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (ok) load8(U + i * S.ldc + cg * 8, u[q]);
            else
#pragma unroll
                for (int k = 0; k < 8; ++k) u[q][k] = 0.f;
        }
#pragma unroll
        for (int q = 0; q < UR; ++q)
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                acc[k][0] = fmaf(u[q][k], rv[q].x, acc[k][0]);
                acc[k][1] = fmaf(u[q][k], rv[q].y, acc[k][1]);
                acc[k][2] = fmaf(u[q][k], rv[q].z, acc[k][2]);
            }
    }
    // sum the row slots of each column group
#pragma unroll
    for (int o = LPR; o < 32; o <<= 1)
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int d = 0; d < 3; ++d) acc[k][d] += __shfl_xor_sync(0xffffffffu, acc[k][d], o);
    if (slot == 0)
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int d = 0; d < 3; ++d) s_acc[w][(cg * 8 + k) * 3 + d] = acc[k][d];
    __syncthreads();
    int r = S.r_c;
    for (int e = threadIdx.x; e < r * 3; e += PROJ_T) {
        float v = 0.f;
#pragma unroll
        for (int q = 0; q < PROJ_W; ++q) v += s_acc[q][e];
        partial[(long long)blockIdx.x * S.ld * 3 + e] = v;
    }
}

template <class TU, int LPR>
__global__ void __launch_bounds__(256) k_lift_compact(SubspaceView S, const TU *__restrict__ U, const int *n_cv,
                                                      const float *__restrict__ q, const float4 *__restrict__ din,
                                                      float4 *__restrict__ dout) {
    if (loop_dead(S.live)) return;
    if (!compact_active(S, n_cv)) return;
    constexpr int RPW = 32 / LPR;
    int lane = threadIdx.x & 31;
    int slot = lane / LPR, cg = lane % LPR;
    int r = S.r_c;
    float ql[8][3];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        int j = cg * 8 + k;
#pragma unroll
        for (int d = 0; d < 3; ++d) ql[k][d] = j < r ? q[j * 3 + d] : 0.f;
    }
    int wpb = blockDim.x >> 5;
    long long nw = (long long)gridDim.x * wpb;
    constexpr int UR = 4;
    for (long long p0 = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); p0 * RPW < S.n; p0 += nw * UR) {
        float u[UR][8];
#pragma unroll
        for (int t = 0; t < UR; ++t) {
            long long i = (p0 + t * nw) * RPW + slot;
            if (i < S.n) load8(U + i * S.ldc + cg * 8, u[t]);
            else
#pragma unroll
                for (int k = 0; k < 8; ++k) u[t][k] = 0.f;
        }
#pragma unroll
        for (int t = 0; t < UR; ++t) {
            float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                a0 = fmaf(u[t][k], ql[k][0], a0);
                a1 = fmaf(u[t][k], ql[k][1], a1);
                a2 = fmaf(u[t][k], ql[k][2], a2);
            }
#pragma unroll
            for (int o = 1; o < LPR; o <<= 1) {
                a0 += __shfl_xor_sync(0xffffffffu, a0, o);
                a1 += __shfl_xor_sync(0xffffffffu, a1, o);
                a2 += __shfl_xor_sync(0xffffffffu, a2, o);
            }
            long long i = (p0 + t * nw) * RPW + slot;
            if (cg == 0 && i < S.n) {
                float4 d = din ? din[i] : make_float4(0.f, 0.f, 0.f, 0.f);
                dout[i] = make_float4(d.x + a0, d.y + a1, d.z + a2, 0.f);
            }
        }
    }
}

// g[e] = sum over blocks of partial[b][e] (e = 3 j + c): one warp per output,
// lanes stride over the blocks, shuffle reduction in double.
__global__ void k_project_reduce(SubspaceView S, const int *n_cv, int nblocks, const float *__restrict__ partial,
                                 double *__restrict__ g, int only_with_contacts) {
    if (loop_dead(S.live)) return;
    if (only_with_contacts && !(n_cv && *n_cv > 0)) return;  // the tensor-core reduction wrote g
    int r = active_r(S, n_cv);
    int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (e >= r * 3) return;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += (double)partial[(long long)b * S.ld * 3 + e];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) g[e] = s;
}

// q = A0^-1 g without collision springs (one warp per row of the inverse).
template <class T>
__global__ void k_apply_inverse(SubspaceView S, const int *n_cv, const T *__restrict__ Ainv, const double *__restrict__ g,
                                float *__restrict__ q) {
    grid_dep_wait();
    grid_dep_release();
    if (loop_dead(S.live)) return;
    if (n_cv && *n_cv > 0) return;
    int r = S.r_nc;
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (w >= r) return;
    T a0 = 0, a1 = 0, a2 = 0;
    for (int k = lane; k < r; k += 32) {
        T m = Ainv[(long long)w * r + k];
        a0 += m * (T)g[k * 3 + 0];
        a1 += m * (T)g[k * 3 + 1];
        a2 += m * (T)g[k * 3 + 2];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if (lane == 0) {
        q[w * 3 + 0] = (float)a0;
        q[w * 3 + 1] = (float)a1;
        q[w * 3 + 2] = (float)a2;
    }
}

// dA = sum_v cw_v U_v U_v^T over the contact list (leading r_c columns), in
// FP64: NDB weights reach 2^a_max k, and single-precision sums of those terms
// would bury the elastic part A0 of the reduced matrix in rounding noise.
constexpr int SYRK_T = 256;
template <class TU, int E>  // E entries per thread: r_c^2 <= 256 E
__global__ void __launch_bounds__(SYRK_T) k_syrk(SubspaceView S, const TU *__restrict__ U, const int *__restrict__ list,
                                                 const int *n_cv, const float *__restrict__ cw, double *__restrict__ dA) {
    __shared__ double s_u[128];
    __shared__ double s_w;
    if (loop_dead(S.live)) return;
    int nc = n_cv ? *n_cv : 0;
    int r = S.r_c;
    if (nc == 0 || r == 0) return;
    int ne = r * r;
    double acc[E];
#pragma unroll
    for (int p = 0; p < E; ++p) acc[p] = 0.0;
    for (int c = blockIdx.x; c < nc; c += gridDim.x) {
        int v = list[c];
        __syncthreads();
        if (threadIdx.x < r) s_u[threadIdx.x] = (double)tofloat<TU>(U[(long long)v * S.ld + threadIdx.x]);
        if (threadIdx.x == 0) s_w = (double)cw[v];
        __syncthreads();
        double w = s_w;
#pragma unroll
        for (int p = 0; p < E; ++p) {
            int e = threadIdx.x + p * SYRK_T;
            if (e < ne) {
                int i = e / r, j = e % r;
                acc[p] = fma(w * s_u[i], s_u[j], acc[p]);
            }
        }
    }
#pragma unroll
    for (int p = 0; p < E; ++p) {
        int e = threadIdx.x + p * SYRK_T;
        if (e < ne && acc[p] != 0.0) atomicAdd(&dA[e], acc[p]);
    }
}

// Cholesky factorisation and solve of (A0[:r,:r] + dA) q = g in one CTA, in
// FP64.  A non-positive pivot sets the flag and the correction is dropped
// (q = 0: the sweeps still run) instead of dividing by a tiny pivot.
__global__ void __launch_bounds__(256) k_chol_solve(SubspaceView S, const int *n_cv, const double *__restrict__ dA,
                                                    const double *__restrict__ g, float *__restrict__ q, int *flag) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ int s_bad;
    if (loop_dead(S.live)) return;
    if (!(n_cv && *n_cv > 0)) return;
    int r = S.r_c;
    if (r == 0) return;
    double *A = reinterpret_cast<double *>(smem_raw);  // [r][r]
    double *b = A + r * r;                              // [r][3]
    int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) s_bad = 0;
    for (int e = tid; e < r * r; e += nt) {
        int i = e / r, j = e % r;
        A[e] = S.A0[(long long)i * S.ld + j] + dA[e];
    }
    for (int e = tid; e < r * 3; e += nt) b[e] = g[e];
    __syncthreads();
    for (int k = 0; k < r; ++k) {
        if (tid == 0) {
            double d = A[k * r + k];
            if (!(d > 0.0) || !isfinite(d)) {
                s_bad = 1;
                d = 1.0;
            }
            A[k * r + k] = sqrt(d);
        }
        __syncthreads();
        double dk = A[k * r + k];
        for (int i = k + 1 + tid; i < r; i += nt) A[i * r + k] /= dk;
        __syncthreads();
        for (int i = k + 1 + tid; i < r; i += nt) {
            double lik = A[i * r + k];
            for (int j = k + 1; j <= i; ++j) A[i * r + j] -= lik * A[j * r + k];
        }
        __syncthreads();
    }
    // forward: L y = b
    for (int k = 0; k < r; ++k) {
        if (tid < 3) b[k * 3 + tid] /= A[k * r + k];
        __syncthreads();
        for (int e = tid; e < (r - k - 1) * 3; e += nt) {
            int i = k + 1 + e / 3, c = e % 3;
            b[i * 3 + c] -= A[i * r + k] * b[k * 3 + c];
        }
        __syncthreads();
    }
    // backward: L^T q = y
    for (int k = r - 1; k >= 0; --k) {
        if (tid < 3) b[k * 3 + tid] /= A[k * r + k];
        __syncthreads();
        for (int e = tid; e < k * 3; e += nt) {
            int i = e / 3, c = e % 3;
            b[i * 3 + c] -= A[k * r + i] * b[k * 3 + c];
        }
        __syncthreads();
    }
    if (s_bad && tid == 0) atomicOr(flag, 1);
    for (int e = tid; e < r * 3; e += nt) q[e] = s_bad ? 0.f : (float)b[e];
}

// ---------------------------------------------------------------- blocked factorisation (r_c > CHOL_ONE_CTA)
// The same solve as k_chol_solve for wider reuse bases: r_c is padded to
// R = nb * CHOL_B (identity on the padding, zero right-hand side there) and
// the lower Cholesky factor is formed by block columns (a panel launch, then
// a launch updating the trailing block triangle), followed by forward and
// backward substitution by blocks.  Every step is FP64.  A CTA that needs a
// diagonal block's factor or a block of the solution computes it itself from
// data the previous launches finished, in the same order as the CTA that
// stores it, so no CTA waits on another.

// Block (bi, bj), bj <= bi, of a lower block triangle numbered row by row.
__device__ inline void tri_tile(int t, int &bi, int &bj) {
    int i = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
    while ((i + 1) * (i + 2) / 2 <= t) ++i;
    while (i > 0 && i * (i + 1) / 2 > t) --i;
    bi = i;
    bj = t - i * (i + 1) / 2;
}

// Regions of dA on the blocked path (see dA_elems).
struct BlkLayout {
    double *A, *Dg, *b, *y, *q, *bad;
};
__device__ inline BlkLayout blk_layout(double *dA, int R) {
    BlkLayout L;
    L.A = dA;
    L.Dg = dA + (long long)R * R;
    L.b = L.Dg + (long long)CHOL_B * R;
    L.y = L.b + 3LL * R;
    L.q = L.y + 3LL * R;
    L.bad = L.q + 3LL * R;
    return L;
}

__device__ inline bool blk_skip(const SubspaceView &S, const int *n_cv) {
    return loop_dead(S.live) || !(n_cv && *n_cv > 0) || S.r_c <= CHOL_ONE_CTA;
}

constexpr int SYRKB_C = 32;  // contact vertices staged per round

// Lower block tiles of dA = sum_v cw_v U_v U_v^T (leading r_c columns, rows
// and columns padded to R with zeros); blockIdx.y splits the contact list.
template <class TU>
__global__ void __launch_bounds__(256) k_syrk_blocks(SubspaceView S, const TU *__restrict__ U,
                                                     const int *__restrict__ list, const int *n_cv,
                                                     const float *__restrict__ cw, double *__restrict__ dA) {
    __shared__ double s_a[SYRKB_C][CHOL_B + 1], s_b[SYRKB_C][CHOL_B + 1];
    __shared__ double s_w[SYRKB_C];
    if (blk_skip(S, n_cv)) return;
    const int nc = *n_cv, r = S.r_c, R = chol_pad(r);
    int bi, bj;
    tri_tile(blockIdx.x, bi, bj);
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
    const int nchunk = (nc + SYRKB_C - 1) / SYRKB_C;
    for (int ch = blockIdx.y; ch < nchunk; ch += gridDim.y) {
        __syncthreads();
        for (int e = tid; e < SYRKB_C * CHOL_B; e += blockDim.x) {
            const int c = e / CHOL_B, k = e % CHOL_B, ci = ch * SYRKB_C + c;
            double a = 0.0, b = 0.0;
            if (ci < nc) {
                const TU *row = U + (long long)list[ci] * S.ld;
                const int ja = bi * CHOL_B + k, jb = bj * CHOL_B + k;
                if (ja < r) a = (double)tofloat<TU>(row[ja]);
                if (jb < r) b = (double)tofloat<TU>(row[jb]);
            }
            s_a[c][k] = a;
            s_b[c][k] = b;
        }
        if (tid < SYRKB_C) {
            const int ci = ch * SYRKB_C + tid;
            s_w[tid] = ci < nc ? (double)cw[list[ci]] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int c = 0; c < SYRKB_C; ++c) {
            const double w = s_w[c];
            const double a0 = w * s_a[c][2 * ty], a1 = w * s_a[c][2 * ty + 1];
            const double b0 = s_b[c][2 * tx], b1 = s_b[c][2 * tx + 1];
            acc[0][0] = fma(a0, b0, acc[0][0]);
            acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][0] = fma(a1, b0, acc[1][0]);
            acc[1][1] = fma(a1, b1, acc[1][1]);
        }
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
            if (acc[a][b] != 0.0)
                atomicAdd(&dA[(long long)(bi * CHOL_B + 2 * ty + a) * R + bj * CHOL_B + 2 * tx + b], acc[a][b]);
}

// b = g (zero on the padding); with `matrix`, also the lower triangle of
// A = A0[:r, :r] + dA (identity on the padding) and the failed-pivot marker
// cleared.
__global__ void k_chol_blk_init(SubspaceView S, const int *n_cv, double *__restrict__ dA,
                                const double *__restrict__ g, int matrix) {
    if (blk_skip(S, n_cv)) return;
    const int r = S.r_c, R = chol_pad(r);
    const BlkLayout L = blk_layout(dA, R);
    const long long nm = (long long)R * R, tot = nm + 3LL * R + (matrix ? 1 : 0);
    for (long long e = (matrix ? 0 : nm) + (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        if (e < nm) {
            const int i = (int)(e / R), j = (int)(e % R);
            if (j > i) continue;
            dA[e] = i < r ? S.A0[(long long)i * S.ld + j] + dA[e] : (i == j ? 1.0 : 0.0);
        } else if (e < nm + 3LL * R) {
            const int k = (int)(e - nm);
            L.b[k] = k < 3 * r ? g[k] : 0.0;
        } else {
            *L.bad = 0.0;
        }
    }
}

// Cholesky factor of diagonal block k (lower, in place in shared memory),
// one warp; lane i owns row i.  A non-positive pivot is replaced by 1 and
// reported.
__device__ inline bool factor_diag_block(double (*D)[CHOL_B + 1], int lane) {
    bool bad = false;
    for (int c = 0; c < CHOL_B; ++c) {
        double p = D[c][c];
        if (!(p > 0.0) || !isfinite(p)) {
            bad = true;
            p = 1.0;
        }
        const double d = sqrt(p);
        __syncwarp();
        if (lane == c) D[c][c] = d;
        if (lane > c) D[lane][c] /= d;
        __syncwarp();
        if (lane > c) {
            const double l = D[lane][c];
            for (int j = c + 1; j <= lane; ++j) D[lane][j] -= l * D[j][c];
        }
        __syncwarp();
    }
    return bad;
}

// Panel k: every CTA factors diagonal block k of A; CTA 0 stores the factor
// L_kk in the diagonal-factor region, CTA c >= 1 forms block (k + c, k) of
// the factor in place, L_ik = A_ik L_kk^-T.
__global__ void __launch_bounds__(32) k_chol_blk_panel(SubspaceView S, const int *n_cv, double *__restrict__ dA,
                                                       int k, int *flag) {
    __shared__ double D[CHOL_B][CHOL_B + 1];
    __shared__ double X[CHOL_B][CHOL_B + 1];
    if (blk_skip(S, n_cv)) return;
    const int R = chol_pad(S.r_c), lane = threadIdx.x;
    const long long k0 = (long long)k * CHOL_B;
    for (int i = 0; i < CHOL_B; ++i) D[i][lane] = dA[(k0 + i) * R + k0 + lane];
    __syncwarp();
    const bool bad = factor_diag_block(D, lane);
    if (blockIdx.x == 0) {  // to its own region: the other CTAs read block (k, k) of A
        const BlkLayout L = blk_layout(dA, R);
        for (int i = 0; i < CHOL_B; ++i) L.Dg[(k0 + i) * CHOL_B + lane] = D[i][lane];
        if (bad && lane == 0) {
            *L.bad = 1.0;
            atomicOr(flag, 1);
        }
        return;
    }
    const long long i0 = (long long)(k + blockIdx.x) * CHOL_B;
    for (int i = 0; i < CHOL_B; ++i) X[i][lane] = dA[(i0 + i) * R + k0 + lane];
    __syncwarp();
    // row `lane` of X L_kk^T = A_ik, column by column
    for (int c = 0; c < CHOL_B; ++c) {
        double x = X[lane][c];
        for (int m = 0; m < c; ++m) x -= X[lane][m] * D[c][m];
        X[lane][c] = x / D[c][c];
    }
    __syncwarp();
    for (int i = 0; i < CHOL_B; ++i) dA[(i0 + i) * R + k0 + lane] = X[i][lane];
}

// Trailing update after panel k: A_ij -= L_ik L_jk^T for the lower block
// tiles k < j <= i < nb (diagonal tiles in full; their upper half is never read).
__global__ void __launch_bounds__(256) k_chol_blk_update(SubspaceView S, const int *n_cv, double *__restrict__ dA,
                                                         int k) {
    __shared__ double Li[CHOL_B][CHOL_B + 1], Lj[CHOL_B][CHOL_B + 1];
    if (blk_skip(S, n_cv)) return;
    const int R = chol_pad(S.r_c);
    int ti, tj;
    tri_tile(blockIdx.x, ti, tj);
    const long long k0 = (long long)k * CHOL_B, i0 = (long long)(k + 1 + ti) * CHOL_B,
                    j0 = (long long)(k + 1 + tj) * CHOL_B;
    const int tid = threadIdx.x;
    for (int e = tid; e < CHOL_B * CHOL_B; e += blockDim.x) {
        const int row = e / CHOL_B, col = e % CHOL_B;
        Li[row][col] = dA[(i0 + row) * R + k0 + col];
        Lj[row][col] = dA[(j0 + row) * R + k0 + col];
    }
    __syncthreads();
    const int ty = tid >> 4, tx = tid & 15;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int row = 2 * ty + a, col = 2 * tx + b;
            double acc = 0.0;
#pragma unroll 8
            for (int m = 0; m < CHOL_B; ++m) acc = fma(Li[row][m], Lj[col][m], acc);
            dA[(i0 + row) * R + j0 + col] -= acc;
        }
}

// Forward substitution, block column k: every CTA forms y_k = L_kk^-1 b_k
// (lane i owns row i); CTA 0 stores it, CTA c >= 1 updates
// b_{k+c} -= L_{k+c,k} y_k.
__global__ void __launch_bounds__(32) k_chol_blk_fwd(SubspaceView S, const int *n_cv, double *__restrict__ dA,
                                                     int k) {
    __shared__ double D[CHOL_B][CHOL_B + 1];
    __shared__ double Y[CHOL_B][3];
    if (blk_skip(S, n_cv)) return;
    const int R = chol_pad(S.r_c), lane = threadIdx.x;
    const long long k0 = (long long)k * CHOL_B;
    const BlkLayout L = blk_layout(dA, R);
    double *b = L.b, *y = L.y;
    for (int i = 0; i < CHOL_B; ++i) D[i][lane] = L.Dg[(k0 + i) * CHOL_B + lane];
    double v[3];
    for (int d = 0; d < 3; ++d) v[d] = b[(k0 + lane) * 3 + d];
    __syncwarp();
    for (int c = 0; c < CHOL_B; ++c) {
        const double dcc = D[c][c];
        for (int d = 0; d < 3; ++d) {
            if (lane == c) v[d] /= dcc;
            const double yc = __shfl_sync(0xffffffffu, v[d], c);
            if (lane > c) v[d] -= D[lane][c] * yc;
        }
    }
    if (blockIdx.x == 0) {
        for (int d = 0; d < 3; ++d) y[(k0 + lane) * 3 + d] = v[d];
        return;
    }
    for (int d = 0; d < 3; ++d) Y[lane][d] = v[d];
    const long long i0 = (long long)(k + blockIdx.x) * CHOL_B;
    __syncwarp();
    for (int i = 0; i < CHOL_B; ++i) D[i][lane] = dA[(i0 + i) * R + k0 + lane];
    __syncwarp();
    double acc[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < CHOL_B; ++c) {
        const double l = D[lane][c];
        for (int d = 0; d < 3; ++d) acc[d] = fma(l, Y[c][d], acc[d]);
    }
    for (int d = 0; d < 3; ++d) b[(i0 + lane) * 3 + d] -= acc[d];
}

// Backward substitution L^T q = y, block row k (launched for k = nb-1 .. 0):
// every CTA forms q_k = L_kk^-T y_k; CTA 0 stores it (and, at k = 0, writes
// the FP32 solution, zero after a failed pivot), CTA c >= 1 updates
// y_{k-c} -= L_{k,k-c}^T q_k.
__global__ void __launch_bounds__(32) k_chol_blk_bwd(SubspaceView S, const int *n_cv, double *__restrict__ dA,
                                                     int k, float *__restrict__ q_out) {
    __shared__ double D[CHOL_B][CHOL_B + 1];
    __shared__ double Q[CHOL_B][3];
    if (blk_skip(S, n_cv)) return;
    const int r = S.r_c, R = chol_pad(r), lane = threadIdx.x;
    const long long k0 = (long long)k * CHOL_B;
    const BlkLayout L = blk_layout(dA, R);
    double *y = L.y, *q = L.q;
    for (int i = 0; i < CHOL_B; ++i) D[i][lane] = L.Dg[(k0 + i) * CHOL_B + lane];
    double v[3];
    for (int d = 0; d < 3; ++d) v[d] = y[(k0 + lane) * 3 + d];
    __syncwarp();
    for (int c = CHOL_B - 1; c >= 0; --c) {
        const double dcc = D[c][c];
        for (int d = 0; d < 3; ++d) {
            if (lane == c) v[d] /= dcc;
            const double qc = __shfl_sync(0xffffffffu, v[d], c);
            if (lane < c) v[d] -= D[c][lane] * qc;
        }
    }
    if (blockIdx.x == 0) {
        for (int d = 0; d < 3; ++d) q[(k0 + lane) * 3 + d] = v[d];
        if (k == 0) {
            __syncwarp();  // this warp's stores of block 0 are visible to its lanes
            const bool bad = *L.bad != 0.0;
            for (int e = lane; e < 3 * r; e += 32) q_out[e] = bad ? 0.f : (float)q[e];
        }
        return;
    }
    for (int d = 0; d < 3; ++d) Q[lane][d] = v[d];
    __syncwarp();
    const long long i0 = (long long)(k - blockIdx.x) * CHOL_B;
    double acc[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < CHOL_B; ++c) {
        const double l = dA[(k0 + c) * R + i0 + lane];  // L[k0 + c][i0 + lane]
        for (int d = 0; d < 3; ++d) acc[d] = fma(l, Q[c][d], acc[d]);
    }
    for (int d = 0; d < 3; ++d) y[(i0 + lane) * 3 + d] -= acc[d];
}

// dout_i = din_i + sum_j U[i][j] q_j: one warp per row, lane l owns columns
// 8l..8l+7 of each 256-column chunk, warp-shuffle reduction of the 3 sums.
template <class TU, int NCH>
__global__ void __launch_bounds__(256) k_lift(SubspaceView S, const TU *__restrict__ U, const int *n_cv,
                                              const float *__restrict__ q, const float4 *__restrict__ din,
                                              float4 *__restrict__ dout) {
    __shared__ float s_q[256 * NCH * 3];
    if (loop_dead(S.live)) return;
    if (compact_active(S, n_cv)) return;
    int r = active_r(S, n_cv);
    for (int e = threadIdx.x; e < 256 * NCH * 3; e += blockDim.x) s_q[e] = e < r * 3 ? q[e] : 0.f;
    __syncthreads();
    int lane = threadIdx.x & 31;
    int wpb = blockDim.x >> 5;
    // this lane's q entries stay in registers
    float ql[NCH][8][3];
#pragma unroll
    for (int c = 0; c < NCH; ++c)
#pragma unroll
        for (int k = 0; k < 8; ++k)
#pragma unroll
            for (int d = 0; d < 3; ++d) ql[c][k][d] = s_q[(c * 256 + lane * 8 + k) * 3 + d];
    constexpr int UR = NCH == 1 ? 4 : 2;  // rows in flight per warp
    long long nwarp = (long long)gridDim.x * wpb;
    for (long long i0 = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); i0 < S.n; i0 += nwarp * UR) {
        float u[UR][NCH][8];
#pragma unroll
        for (int q = 0; q < UR; ++q) {
            long long i = i0 + q * nwarp;
            bool ok = i < S.n;
            const TU *row = U + (ok ? i : 0) * S.ld;
#pragma unroll
            for (int c = 0; c < NCH; ++c) {
                int j0 = c * 256 + lane * 8;
                if (ok && j0 < r) load8(row + j0, u[q][c]);
                else
#pragma unroll
                    for (int k = 0; k < 8; ++k) u[q][c][k] = 0.f;
            }
        }
#pragma unroll
        for (int q = 0; q < UR; ++q) {
            float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
            for (int c = 0; c < NCH; ++c)
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    a0 = fmaf(u[q][c][k], ql[c][k][0], a0);
                    a1 = fmaf(u[q][c][k], ql[c][k][1], a1);
                    a2 = fmaf(u[q][c][k], ql[c][k][2], a2);
                }
            for (int o = 16; o > 0; o >>= 1) {
                a0 += __shfl_xor_sync(0xffffffffu, a0, o);
                a1 += __shfl_xor_sync(0xffffffffu, a1, o);
                a2 += __shfl_xor_sync(0xffffffffu, a2, o);
            }
            long long i = i0 + q * nwarp;
            if (lane == 0 && i < S.n) {
                float4 d = din ? din[i] : make_float4(0.f, 0.f, 0.f, 0.f);
                dout[i] = make_float4(d.x + a0, d.y + a1, d.z + a2, 0.f);
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_linear_residual(ClothView c, const float *__restrict__ cw,
                                                         const float4 *__restrict__ r, const float4 *__restrict__ d,
                                                         float4 *__restrict__ rl) {
    if (loop_dead(c.live)) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= c.n) return;
    float3 acc = make_float3(0.f, 0.f, 0.f);
    if (c.is_free[i]) {
        acc = f3(r[i]);
        for (int k = 0; k < c.ell_w; ++k) {
            float v = c.ell_val[(size_t)k * c.n + i];
            int j = c.ell_col[(size_t)k * c.n + i];
            acc = acc - v * f3(d[j]);
        }
        float D = c.hdiag[i] + (cw ? cw[i] : 0.f);
        acc = acc - D * f3(d[i]);
    }
    rl[i] = f4(acc);
}

}  // namespace

template <class TU> static void project_t(cudaStream_t s, const SubspaceView &S, const TU *U, const float4 *rl,
                                          const int *n_cv, float *partial) {
    int rmax = std::max(S.r_nc, S.r_c);
    if (rmax <= 256) k_project<TU, 1><<<PROJ_BLOCKS, PROJ_T, 0, s>>>(S, U, rl, n_cv, partial);
    else if (rmax <= 512) k_project<TU, 2><<<PROJ_BLOCKS, PROJ_T, 0, s>>>(S, U, rl, n_cv, partial);
    else k_project<TU, 4><<<PROJ_BLOCKS, PROJ_T, 0, s>>>(S, U, rl, n_cv, partial);
}

template <class TU> static void project_compact_t(cudaStream_t s, const SubspaceView &S, const TU *U,
                                                  const float4 *rl, const int *n_cv, float *partial) {
    switch (S.ldc) {
        case 8: k_project_compact<TU, 1><<<PROJ_BLOCKS, PROJ_T, 0, s>>>(S, U, rl, n_cv, partial); break;
        case 16: k_project_compact<TU, 2><<<PROJ_BLOCKS, PROJ_T, 0, s>>>(S, U, rl, n_cv, partial); break;
        case 32: k_project_compact<TU, 4><<<PROJ_BLOCKS, PROJ_T, 0, s>>>(S, U, rl, n_cv, partial); break;
        case 64: k_project_compact<TU, 8><<<PROJ_BLOCKS, PROJ_T, 0, s>>>(S, U, rl, n_cv, partial); break;
        case 128: k_project_compact<TU, 16><<<PROJ_BLOCKS, PROJ_T, 0, s>>>(S, U, rl, n_cv, partial); break;
        default: throw Error(PDC_ERR_ARG, "compact basis width must be 8, 16, 32, 64 or 128");
    }
}

template <class TU> static void lift_compact_t(cudaStream_t s, const SubspaceView &S, const TU *U, const int *n_cv,
                                               const float *q, const float4 *din, float4 *dout) {
    int blocks = std::min((S.n + 63) / 64, 152 * 8);
    switch (S.ldc) {
        case 8: k_lift_compact<TU, 1><<<blocks, 256, 0, s>>>(S, U, n_cv, q, din, dout); break;
        case 16: k_lift_compact<TU, 2><<<blocks, 256, 0, s>>>(S, U, n_cv, q, din, dout); break;
        case 32: k_lift_compact<TU, 4><<<blocks, 256, 0, s>>>(S, U, n_cv, q, din, dout); break;
        case 64: k_lift_compact<TU, 8><<<blocks, 256, 0, s>>>(S, U, n_cv, q, din, dout); break;
        case 128: k_lift_compact<TU, 16><<<blocks, 256, 0, s>>>(S, U, n_cv, q, din, dout); break;
        default: throw Error(PDC_ERR_ARG, "compact basis width must be 8, 16, 32, 64 or 128");
    }
}

// Calls f with the basis of the view's element type (full or compact copy).
template <class F> static void with_basis(const SubspaceView &S, bool compact, F f) {
    if (S.precision == 1) f(compact ? S.Uc16 : S.U16);
    else if (S.precision == 2) f(compact ? S.Uch : S.Uh);
    else f(compact ? S.Uc32 : S.U32);
}

bool device_path_choice(const SubspaceView &S) {
    return S.umma && S.r_nc > 0 && S.r_nc <= S.ld && compact_covers(S);
}

void launch_project(cudaStream_t s, const SubspaceView &S, const float4 *rl, const int *n_cv, SubspaceWork &W,
                    bool maybe_contacts, bool device_choice) {
    if (!maybe_contacts && S.umma && S.r_nc > 0 && S.r_nc <= S.ld) {
        launch_project_umma(s, *S.umma, S.r_nc, rl, S.umma_partial, W.g, S.dev_err, S.overlap != 0, nullptr, S.live);
        return;
    }
    int mx = S.ld * 3 * 32;
    if (maybe_contacts && device_choice && device_path_choice(S)) {
        // the iteration's contact-vertex count (device) picks the path: the
        // full basis on the tensor cores without springs, the compact basis
        // on the CUDA cores with them; each kernel of the other path returns
        launch_project_umma(s, *S.umma, S.r_nc, rl, S.umma_partial, W.g, S.dev_err, S.overlap != 0, n_cv, S.live);
        with_basis(S, true, [&](auto *U) { project_compact_t(s, S, U, rl, n_cv, W.partial); });
        k_project_reduce<<<(mx + 255) / 256, 256, 0, s>>>(S, n_cv, PROJ_BLOCKS, W.partial, W.g, 1);
        PDC_LAUNCH_CK();
        return;
    }
    with_basis(S, false, [&](auto *U) { project_t(s, S, U, rl, n_cv, W.partial); });
    if (maybe_contacts && compact_covers(S))
        with_basis(S, true, [&](auto *U) { project_compact_t(s, S, U, rl, n_cv, W.partial); });
    k_project_reduce<<<(mx + 255) / 256, 256, 0, s>>>(S, n_cv, PROJ_BLOCKS, W.partial, W.g, 0);
    PDC_LAUNCH_CK();
}

void launch_syrk(cudaStream_t s, const SubspaceView &S, const int *list, const int *n_cv, const float *cw,
                 SubspaceWork &W, bool zero) {
    if (S.r_c == 0) return;
    if (zero) launch_live_zero(s, S.live, W.dA, sizeof(double) * dA_zero_elems(S.r_c));
    if (S.r_c > CHOL_ONE_CTA) {
        const int nb = chol_pad(S.r_c) / CHOL_B, ntile = nb * (nb + 1) / 2;
        const dim3 grid(ntile, std::max(1, 4 * 152 / ntile));
        with_basis(S, false, [&](auto *U) {
            using TU = std::remove_const_t<std::remove_pointer_t<decltype(U)>>;
            k_syrk_blocks<TU><<<grid, 256, 0, s>>>(S, U, list, n_cv, cw, W.dA);
        });
        PDC_LAUNCH_CK();
        return;
    }
    with_basis(S, false, [&](auto *U) {
        using TU = std::remove_const_t<std::remove_pointer_t<decltype(U)>>;
        int ne = S.r_c * S.r_c;
        if (ne <= 4 * SYRK_T) k_syrk<TU, 4><<<152, SYRK_T, 0, s>>>(S, U, list, n_cv, cw, W.dA);
        else if (ne <= 16 * SYRK_T) k_syrk<TU, 16><<<152, SYRK_T, 0, s>>>(S, U, list, n_cv, cw, W.dA);
        else k_syrk<TU, 64><<<152, SYRK_T, 0, s>>>(S, U, list, n_cv, cw, W.dA);
    });
    PDC_LAUNCH_CK();
}

void launch_reduced_solve(cudaStream_t s, const SubspaceView &S, const int *n_cv, SubspaceWork &W, bool factor) {
    const bool mixed = S.precision != 0;  // mixed forms: FP64 reduced solves
    if (S.r_nc > 0) {
        int thr = S.r_nc * 32;
        if (mixed)
            launch_dependent(S.overlap != 0, k_apply_inverse<double>, (thr + 255) / 256, 256, 0, s, S, n_cv,
                             (const double *)S.A0inv, (const double *)W.g, W.q);
        else
            k_apply_inverse<float><<<(thr + 255) / 256, 256, 0, s>>>(S, n_cv, S.A0inv32, W.g, W.q);
    }
    if (S.r_c > 0 && S.r_c <= CHOL_ONE_CTA) {  // FP64 in both forms (see k_syrk)
        size_t sm = sizeof(double) * (S.r_c * S.r_c + S.r_c * 3);
        k_chol_solve<<<1, 256, sm, s>>>(S, n_cv, W.dA, W.g, W.q, W.flag);
    } else if (S.r_c > CHOL_ONE_CTA) {
        const int R = chol_pad(S.r_c), nb = R / CHOL_B;
        const long long tot = factor ? (long long)R * R + 3LL * R + 1 : 3LL * R;
        k_chol_blk_init<<<(int)std::min<long long>((tot + 255) / 256, 152 * 8), 256, 0, s>>>(S, n_cv, W.dA, W.g,
                                                                                          factor ? 1 : 0);
        for (int k = 0; factor && k < nb; ++k) {
            k_chol_blk_panel<<<nb - k, 32, 0, s>>>(S, n_cv, W.dA, k, W.flag);
            const int m = nb - k - 1;
            if (m > 0) k_chol_blk_update<<<m * (m + 1) / 2, 256, 0, s>>>(S, n_cv, W.dA, k);
        }
        for (int k = 0; k < nb; ++k) k_chol_blk_fwd<<<nb - k, 32, 0, s>>>(S, n_cv, W.dA, k);
        for (int k = nb - 1; k >= 0; --k) k_chol_blk_bwd<<<k + 1, 32, 0, s>>>(S, n_cv, W.dA, k, W.q);
    }
    PDC_LAUNCH_CK();
}

template <class TU> static void lift_t(cudaStream_t s, const SubspaceView &S, const TU *U, const int *n_cv,
                                       const float *q, const float4 *din, float4 *dout) {
    int blocks = std::min((S.n + 7) / 8, 152 * 16);
    if (blocks < 1) return;
    int rmax = std::max(S.r_nc, S.r_c);
    if (rmax <= 256) k_lift<TU, 1><<<blocks, 256, 0, s>>>(S, U, n_cv, q, din, dout);
    else if (rmax <= 512) k_lift<TU, 2><<<blocks, 256, 0, s>>>(S, U, n_cv, q, din, dout);
    else k_lift<TU, 4><<<blocks, 256, 0, s>>>(S, U, n_cv, q, din, dout);
}

void launch_lift(cudaStream_t s, const SubspaceView &S, const int *n_cv, const SubspaceWork &W, const float4 *din,
                 float4 *dout, bool maybe_contacts, bool device_choice) {
    if (!maybe_contacts && S.umma && S.r_nc > 0 && S.r_nc <= S.ld) {
        launch_lift_umma(s, *S.umma, S.r_nc, W.q, din, dout, S.dev_err, S.overlap != 0, nullptr, S.live);
        return;
    }
    if (maybe_contacts && device_choice && device_path_choice(S)) {  // as in launch_project
        launch_lift_umma(s, *S.umma, S.r_nc, W.q, din, dout, S.dev_err, S.overlap != 0, n_cv, S.live);
        if (S.n > 0) with_basis(S, true, [&](auto *U) { lift_compact_t(s, S, U, n_cv, W.q, din, dout); });
        PDC_LAUNCH_CK();
        return;
    }
    if (maybe_contacts && compact_covers(S) && S.n > 0)
        with_basis(S, true, [&](auto *U) { lift_compact_t(s, S, U, n_cv, W.q, din, dout); });
    with_basis(S, false, [&](auto *U) { lift_t(s, S, U, n_cv, W.q, din, dout); });
    PDC_LAUNCH_CK();
}

void launch_linear_residual(cudaStream_t s, const ClothView &c, const float *cw, const float4 *r,
                            const float4 *delta, float4 *rl) {
    if (c.n > 0) k_linear_residual<<<(c.n + 255) / 256, 256, 0, s>>>(c, cw, r, delta, rl);
    PDC_LAUNCH_CK();
}

void set_chol_smem_limits() {
    size_t mx = sizeof(double) * (128 * 128 + 128 * 3);
    PDC_CK(cudaFuncSetAttribute(k_chol_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mx));
}

}  // namespace pdc
