// Basis precomputation (Sec. 5 / Sec. 7): the r eigenvectors of the rest
// global matrix H (Eq. global without collisions, pinned rows removed) with
// the smallest eigenvalues.  Chebyshev-filtered subspace iteration: a block
// of r + oversampling vectors is repeatedly multiplied by a Chebyshev
// polynomial of H that damps the interval [a, b] above the wanted modes,
// orthonormalised (Cholesky QR, twice) and rotated by a Rayleigh-Ritz step.
// b is the Gershgorin bound of H, a the largest current Ritz value.
//
// Device work: sparse H times block (ELL), block Gram matrices X^T Y with
// FP64 accumulation, block times small matrix.  Host work (FP64): Cholesky,
// triangular inverse and the symmetric eigenproblem of the small Rayleigh
// matrix (cyclic Jacobi rotations).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "pdc_subspace.cuh"

namespace pdc {

namespace {

__device__ inline unsigned long long mix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

__global__ void k_randn(int n, int m, const unsigned char *__restrict__ is_free, unsigned long long seed,
                        float *__restrict__ X) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n * m) return;
    int i = (int)(idx / m);
    if (!is_free[i]) {
        X[idx] = 0.f;
        return;
    }
    unsigned long long h1 = mix64(seed ^ (2 * (unsigned long long)idx));
    unsigned long long h2 = mix64(seed ^ (2 * (unsigned long long)idx + 1));
    double u1 = ((h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);
    X[idx] = (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
}

// Y = alpha (H X - shift X) + beta Z   (Z may alias nothing; beta = 0 skips it)
__global__ void k_spmm(ClothView c, int m, const float *__restrict__ X, float *__restrict__ Y, float alpha, float shift,
                       float beta, const float *__restrict__ Z) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)c.n * m) return;
    int i = (int)(idx / m), j = (int)(idx % m);
    if (!c.is_free[i]) {
        Y[idx] = 0.f;
        return;
    }
    float xi = X[idx];
    float acc = c.hdiag[i] * xi;
    for (int k = 0; k < c.ell_w; ++k) {
        float v = c.ell_val[(size_t)k * c.n + i];
        int col = c.ell_col[(size_t)k * c.n + i];
        acc = fmaf(v, X[(long long)col * m + j], acc);
    }
    float y = alpha * (acc - shift * xi);
    if (beta != 0.f) y = fmaf(beta, Z[idx], y);
    Y[idx] = y;
}

// G += A^T B over a chunk of rows; 32x32 tile per block, FP32 within the
// chunk, FP64 across chunks.
constexpr int GCH = 1024;
__global__ void __launch_bounds__(256) k_gram(const float *__restrict__ A, const float *__restrict__ B, int n, int m,
                                              double *__restrict__ G) {
    __shared__ float sa[32][33], sb[32][33];
    int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    long long r0 = (long long)blockIdx.z * GCH, r1 = min(r0 + GCH, (long long)n);
    int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (long long t = r0; t < r1; t += 32) {
        for (int k = ty; k < 32; k += 8) {
            long long row = t + k;
            sa[k][tx] = (row < r1 && i0 + tx < m) ? A[row * m + i0 + tx] : 0.f;
            sb[k][tx] = (row < r1 && j0 + tx < m) ? B[row * m + j0 + tx] : 0.f;
        }
        __syncthreads();
        for (int k = 0; k < 32; ++k) {
            float b = sb[k][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fmaf(sa[k][ty + 8 * q], b, acc[q]);
        }
        __syncthreads();
    }
    for (int q = 0; q < 4; ++q) {
        int i = i0 + ty + 8 * q, j = j0 + tx;
        if (i < m && j < m && acc[q] != 0.f) atomicAdd(&G[(long long)i * m + j], (double)acc[q]);
    }
}

// Y[n][m2] = X[n][m] C[m][m2]
__global__ void __launch_bounds__(256) k_apply(const float *__restrict__ X, int n, int m, const float *__restrict__ C,
                                               int m2, float *__restrict__ Y) {
    __shared__ float sx[32][33], sc[32][65];
    long long r0 = (long long)blockIdx.x * 32;
    int c0 = blockIdx.y * 64;
    int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;  // 64 x 4
    float acc[8];
    for (int q = 0; q < 8; ++q) acc[q] = 0.f;
    for (int k0 = 0; k0 < m; k0 += 32) {
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
            int rr = e / 32, kk = e % 32;
            long long row = r0 + rr;
            sx[rr][kk] = (row < n && k0 + kk < m) ? X[row * m + k0 + kk] : 0.f;
        }
        for (int e = threadIdx.x; e < 32 * 64; e += 256) {
            int kk = e / 64, cc = e % 64;
            sc[kk][cc] = (k0 + kk < m && c0 + cc < m2) ? C[(long long)(k0 + kk) * m2 + c0 + cc] : 0.f;
        }
        __syncthreads();
        for (int kk = 0; kk < 32; ++kk) {
            float cv = sc[kk][tx];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = fmaf(sx[ty + 4 * q][kk], cv, acc[q]);
        }
        __syncthreads();
    }
    for (int q = 0; q < 8; ++q) {
        long long row = r0 + ty + 4 * q;
        int col = c0 + tx;
        if (row < n && col < m2) Y[row * m2 + col] = acc[q];
    }
}

struct Ctx {
    cudaStream_t s;
    const ClothView &c;
    int n, m;
    DevBuf<double> G;
    DevBuf<float> C;
    Ctx(cudaStream_t s_, const ClothView &c_, int m_) : s(s_), c(c_), n(c_.n), m(m_) {
        G.alloc((size_t)m * m);
        C.alloc((size_t)m * m);
    }
    void spmm(const float *X, float *Y, float alpha, float shift, float beta, const float *Z) {
        long long tot = (long long)n * m;
        k_spmm<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(c, m, X, Y, alpha, shift, beta, Z);
        PDC_LAUNCH_CK();
    }
    std::vector<double> gram(const float *A, const float *B) {
        G.zero(s);
        dim3 grid((m + 31) / 32, (m + 31) / 32, (n + GCH - 1) / GCH);
        k_gram<<<grid, 256, 0, s>>>(A, B, n, m, G);
        PDC_LAUNCH_CK();
        std::vector<double> h((size_t)m * m);
        G.download(h.data(), h.size(), s);
        PDC_CK(cudaStreamSynchronize(s));
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < i; ++j) {
                double v = 0.5 * (h[(size_t)i * m + j] + h[(size_t)j * m + i]);
                h[(size_t)i * m + j] = h[(size_t)j * m + i] = v;
            }
        return h;
    }
    void apply(const float *X, const std::vector<double> &Cm, int m2, float *Y) {
        std::vector<float> cf(Cm.begin(), Cm.end());
        C.upload(cf, s);
        dim3 grid((unsigned)((n + 31) / 32), (m2 + 63) / 64);
        k_apply<<<grid, 256, 0, s>>>(X, n, m, C, m2, Y);
        PDC_LAUNCH_CK();
    }
};

// X <- X L^-T with L L^T = X^T X (twice); tmp is scratch of the same size.
void orthonormalize(Ctx &cx, float *X, float *tmp) {
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<double> G = cx.gram(X, X);
        int m = cx.m;
        double tr = 0;
        for (int i = 0; i < m; ++i) tr += G[(size_t)i * m + i];
        double shift = 0;
        std::vector<double> L;
        for (int tries = 0; tries < 8; ++tries) {
            L = G;
            for (int i = 0; i < m; ++i) L[(size_t)i * m + i] += shift;
            if (cholesky_inplace(L, m)) break;
            shift = shift == 0 ? 1e-12 * tr / m : shift * 100;
        }
        // C = L^-T (upper triangular): solve L^T C = I column by column
        std::vector<double> Ci((size_t)m * m, 0.0);
        for (int col = 0; col < m; ++col) {
            // forward solve L y = e_col gives column of L^-1; C = (L^-1)^T
            std::vector<double> y(m, 0.0);
            for (int i = 0; i < m; ++i) {
                double v = (i == col) ? 1.0 : 0.0;
                for (int k = 0; k < i; ++k) v -= L[(size_t)i * m + k] * y[k];
                y[i] = v / L[(size_t)i * m + i];
            }
            for (int i = 0; i < m; ++i) Ci[(size_t)col * m + i] = y[i];  // C[col][i] = Linv[i][col]
        }
        cx.apply(X, Ci, m, tmp);
        PDC_CK(cudaMemcpyAsync(X, tmp, sizeof(float) * (size_t)cx.n * m, cudaMemcpyDeviceToDevice, cx.s));
    }
}

// Rayleigh-Ritz: X <- X W, returns Ritz values (ascending).
std::vector<double> rayleigh_ritz(Ctx &cx, float *X, float *HX, float *tmp) {
    cx.spmm(X, HX, 1.f, 0.f, 0.f, nullptr);
    std::vector<double> T = cx.gram(X, HX);
    std::vector<double> w, V;
    sym_eig(T, cx.m, w, V);
    cx.apply(X, V, cx.m, tmp);
    PDC_CK(cudaMemcpyAsync(X, tmp, sizeof(float) * (size_t)cx.n * cx.m, cudaMemcpyDeviceToDevice, cx.s));
    return w;
}

}  // namespace

// ----------------------------------------------------------------- host dense helpers
bool cholesky_inplace(std::vector<double> &A, int n) {
    for (int j = 0; j < n; ++j) {
        double d = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(d > 0)) return false;
        d = std::sqrt(d);
        A[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double v = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) v -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = v / d;
        }
        for (int i = 0; i < j; ++i) A[(size_t)i * n + j] = 0.0;
    }
    return true;
}

void spd_inverse(const std::vector<double> &A, int n, std::vector<double> &Ainv) {
    std::vector<double> L = A;
    if (!cholesky_inplace(L, n)) throw Error(PDC_ERR_NUMERIC, "reduced matrix U^T H U is not positive definite");
    Ainv.assign((size_t)n * n, 0.0);
    std::vector<double> y(n), x(n);
    for (int col = 0; col < n; ++col) {
        for (int i = 0; i < n; ++i) {
            double v = (i == col) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) v -= L[(size_t)i * n + k] * y[k];
            y[i] = v / L[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double v = y[i];
            for (int k = i + 1; k < n; ++k) v -= L[(size_t)k * n + i] * x[k];
            x[i] = v / L[(size_t)i * n + i];
        }
        for (int i = 0; i < n; ++i) Ainv[(size_t)i * n + col] = x[i];
    }
}

// Cyclic Jacobi rotations on a symmetric matrix: A = V diag(w) V^T.
void sym_eig(std::vector<double> A, int n, std::vector<double> &w, std::vector<double> &V) {
    V.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0, tot = 0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double v = A[(size_t)i * n + j] * A[(size_t)i * n + j];
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-30 * tot || off == 0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double apq = A[(size_t)p * n + q];
                if (std::fabs(apq) < 1e-300) continue;
                double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < n; ++k) {  // columns p, q
                    double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - s * akq;
                    A[(size_t)k * n + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {  // rows p, q
                    double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - s * aqk;
                    A[(size_t)q * n + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - s * vkq;
                    V[(size_t)k * n + q] = s * vkp + c * vkq;
                }
            }
    }
    std::vector<int> idx(n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return A[(size_t)a * n + a] < A[(size_t)b * n + b]; });
    w.resize(n);
    std::vector<double> Vs((size_t)n * n);
    for (int c2 = 0; c2 < n; ++c2) {
        w[c2] = A[(size_t)idx[c2] * n + idx[c2]];
        for (int k = 0; k < n; ++k) Vs[(size_t)k * n + c2] = V[(size_t)k * n + idx[c2]];
    }
    V.swap(Vs);
}

void reduced_matrix(cudaStream_t s, const ClothView &c, const float *U, int ld, std::vector<double> &A) {
    Ctx cx(s, c, ld);
    DevBuf<float> HU;
    HU.alloc((size_t)c.n * ld);
    cx.spmm(U, HU, 1.f, 0.f, 0.f, nullptr);
    A = cx.gram(U, HU);
}

void build_basis(cudaStream_t s, const ClothView &c, int r, int iters, uint64_t seed, std::vector<float> &U,
                 std::vector<double> &ritz) {
    int n = c.n;
    std::vector<unsigned char> fr0(n);
    PDC_CK(cudaMemcpyAsync(fr0.data(), c.is_free, n, cudaMemcpyDeviceToHost, s));
    PDC_CK(cudaStreamSynchronize(s));
    int nfree = (int)std::count(fr0.begin(), fr0.end(), 1);
    int m = ((r + std::max(16, r / 4)) + 31) / 32 * 32;
    m = std::min(m, nfree);
    if (r > m) r = m;
    Ctx cx(s, c, m);
    DevBuf<float> X, Y, Z, HX;
    size_t nm = (size_t)n * m;
    X.alloc(nm);
    Y.alloc(nm);
    Z.alloc(nm);
    HX.alloc(nm);
    k_randn<<<(unsigned)((nm + 255) / 256), 256, 0, s>>>(n, m, c.is_free, (unsigned long long)seed, X);
    PDC_LAUNCH_CK();

    // Gershgorin upper bound of the spectrum (host, from the ELL rows)
    std::vector<float> hd(n), ev((size_t)c.ell_w * n);
    std::vector<unsigned char> fr(n);
    PDC_CK(cudaMemcpyAsync(hd.data(), c.hdiag, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
    if (c.ell_w)
        PDC_CK(cudaMemcpyAsync(ev.data(), c.ell_val, sizeof(float) * ev.size(), cudaMemcpyDeviceToHost, s));
    PDC_CK(cudaMemcpyAsync(fr.data(), c.is_free, n, cudaMemcpyDeviceToHost, s));
    PDC_CK(cudaStreamSynchronize(s));
    double bmax = 0;
    for (int i = 0; i < n; ++i) {
        if (!fr[i]) continue;
        double sr = std::fabs(hd[i]);
        for (int k = 0; k < c.ell_w; ++k) sr += std::fabs(ev[(size_t)k * n + i]);
        bmax = std::max(bmax, sr);
    }

    orthonormalize(cx, X, Y);
    // Initial filter bound from the eigenvalue count of a 2-D operator (Weyl:
    // lambda_m / lambda_max ~ m / n); later bounds are the largest Ritz value.
    // Rayleigh-Ritz (host eigenproblem of the m x m Rayleigh matrix) runs every
    // third pass and at the end.
    double a_bound = bmax * std::min(0.5, 2.0 * m / std::max(nfree, 1));
    double a_low = 0.0;
    ritz.assign(m, 0.0);
    for (int it = 0; it < iters; ++it) {
        double a = a_bound, b = bmax * 1.01, aL = a_low;
        if (!(a < b)) break;
        double e = 0.5 * (b - a), cc = 0.5 * (b + a);
        // degree: enough to damp [a, b] relative to the low end, bounded growth
        double x = (cc - aL) / e;  // > 1
        int deg = (int)std::ceil(std::acosh(1e3) / std::acosh(std::max(x, 1.0 + 1e-12)));
        deg = std::min(std::max(deg, 8), 400);
        // scaled Chebyshev recurrence (values ~ 1 at aL)
        double sigma = e / (aL - cc);
        double sigma1 = sigma, tau = 2.0 / sigma1;
        float *P = X.p, *Q = Y.p, *R = Z.p;
        cx.spmm(P, Q, (float)(sigma1 / e), (float)cc, 0.f, nullptr);
        for (int k = 2; k <= deg; ++k) {
            double sn = 1.0 / (tau - sigma);
            cx.spmm(Q, R, (float)(2.0 * sn / e), (float)cc, (float)(-sigma * sn), P);
            float *t = P;
            P = Q;
            Q = R;
            R = t;
            sigma = sn;
        }
        if (Q != X.p) PDC_CK(cudaMemcpyAsync(X.p, Q, sizeof(float) * nm, cudaMemcpyDeviceToDevice, s));
        orthonormalize(cx, X, Y);
        if (it % 3 == 2 || it == iters - 1) {
            ritz = rayleigh_ritz(cx, X, HX, Y);
            a_bound = std::min(a_bound, ritz[m - 1]);
            a_low = std::max(ritz[0], 0.0);
            if (std::getenv("PDC_LOG"))
                std::fprintf(stderr, "[pdc] basis pass %d deg %d ritz[0]=%.5g ritz[r-1]=%.5g ritz[m-1]=%.5g bmax=%.5g\n", it,
                             deg, ritz[0], ritz[r - 1], ritz[m - 1], bmax);
        }
    }
    if (iters <= 0) ritz = rayleigh_ritz(cx, X, HX, Y);
    // first r Ritz vectors
    std::vector<float> hX(nm);
    X.download(hX.data(), nm, s);
    PDC_CK(cudaStreamSynchronize(s));
    U.assign((size_t)n * r, 0.f);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < r; ++j) U[(size_t)i * r + j] = hX[(size_t)i * m + j];
    ritz.resize(r);
}

}  // namespace pdc
