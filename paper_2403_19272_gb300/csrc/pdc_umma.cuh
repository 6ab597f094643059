// Tensor-core (tcgen05) subspace kernels of the mixed form (k_umma.cu).
#pragma once
#include <cuda.h>

#include "pdc_internal.cuh"

namespace pdc {

// Largest basis row stride served by the tensor-core kernels (shared-memory
// budget: the lift stages a [128][UMMA_MAX_LD] BF16 tile per CTA).
constexpr int UMMA_MAX_LD = 256;

// Device error bit set in the factorisation/status word when a bounded wait
// of a tensor-core kernel ran out.
constexpr int PDC_DEVERR_UMMA = 2;

// TMA descriptors of the 16-bit basis U [n][ld] (BF16 or FP16) and of its
// transpose Ut [ld][n_pad].
struct UmmaMaps {
    CUtensorMap mapU;
    CUtensorMap mapUt;
    int n = 0, ld = 0;
    bool f16 = false;  // FP16 (scaled) basis instead of BF16
    int sms = 1;
    bool ok = false;
};

bool umma_supported(int ld, int n);
void umma_setup(UmmaMaps &M, const void *U, const void *Ut, bool f16, int n, int n_pad, int ld);
int umma_project_blocks(int n);
// g = U[:, :r]^T rl via per-tile partial sums [blocks][ld][3] and an FP64 reduction.
// With overlap, the kernels are launched as programmatic dependents of the
// kernel before them (barrier setup and TMEM allocation overlap its tail).
// skip_if (device, may be NULL): the kernels do nothing when *skip_if > 0
// (an iteration whose collision springs use the compact basis instead);
// live (may be NULL): nor once a device-driven loop has ended (*live == 0).
void launch_project_umma(cudaStream_t s, const UmmaMaps &M, int r, const float4 *rl, float *partial, double *g,
                         int *err, bool overlap = false, const int *skip_if = nullptr, const int *live = nullptr);
// dout = din + U[:, :r] q (din may be NULL).
void launch_lift_umma(cudaStream_t s, const UmmaMaps &M, int r, const float *q, const float4 *din, float4 *dout,
                      int *err, bool overlap = false, const int *skip_if = nullptr, const int *live = nullptr);

}  // namespace pdc
