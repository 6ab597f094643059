// Tensor-core (tcgen05) kernels for the BF16 subspace contractions of the
// mixed form (Sec. 5: g = U^T r of Eq. subspace_global and the lift
// delta = U q of Eq. subspace_collision), without collision springs.
//
// Both products are tall-skinny: U is n x r (BF16, or FP16 scaled by a power
// of two), the other operand n x 3 or r x 3 (FP32).  The FP32 operand is
// split into two parts of U's type, v = hi + lo with hi = rn(v) and
// lo = rn(v - hi), so that the tensor cores see a 6-column operand (padded to
// N = 16) and the FP32 accumulator receives U^T hi + U^T lo: the product
// with a 16-bit (BF16) or 22-bit (FP16) significand of v.  For FP16 each CTA
// first scales its part of v by a power of two that puts its largest entry
// in [2^13, 2^14), and divides the result by it (both exact).  The kernels
// stream U once; they are bound by that HBM stream, not by the tensor pipe.
//
// Layout (both operands K-major, 128-byte swizzle):
//   lift:       A = U tile [128 rows][r] from U   [n][ld]        (TMA)
//               B = q hi/lo [16][r]                (written by the CTA)
//   projection: A = U^T tile [128 j][128 i] from Ut [ld][n_pad]  (TMA)
//               B = r hi/lo [16][128 i]            (written by the CTA)
// Persistent kernels: one CTA per SM loops over its 128-row tiles through a
// ring of shared-memory stages (6 warps: 0-3 write the split operand and read
// the accumulator, warp w reading TMEM lanes 32w..32w+31; warp 4 issues the
// TMA loads; warp 5 owns the 32 TMEM columns and issues the MMAs).  Every
// wait on an mbarrier is bounded by the global timer; on expiry the CTA
// records an error bit, waits (bounded) for its copies, frees its TMEM and
// returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "pdc_subspace.cuh"
#include "pdc_umma.cuh"
#include "pdc_async.cuh"

namespace pdc {

namespace {

constexpr int TILE = 128;            // rows of U per CTA (lift) / U^T rows per MMA (projection)
constexpr int KBOX = 64;             // BF16 elements per 128-byte swizzle row
constexpr int ABOX_BYTES = TILE * 128;  // one [128][64] BF16 box
constexpr int BBOX_BYTES = 16 * 128;    // one [16][64] BF16 box
constexpr uint32_t NCOLS = 32;       // TMEM columns per CTA

__device__ inline void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

__device__ inline void tmem_alloc(uint32_t *dst) {  // whole warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ inline void tmem_dealloc(uint32_t taddr) {  // whole warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(NCOLS) : "memory");
}
__device__ inline void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ inline void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 B apart (SBO), version 1; the leading offset is unused for this layout.
__device__ inline uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, A and B both BF16
// (format 1) or both FP16 (format 0), both K-major, M = 128, N = 16.
template <bool F16>
constexpr uint32_t IDESC = (1u << 4) | ((F16 ? 0u : 1u) << 7) | ((F16 ? 0u : 1u) << 10) | ((16u >> 3) << 17) |
                           ((128u >> 4) << 24);

template <bool F16> __device__ inline void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(IDESC<F16>), "r"(accumulate)
        : "memory");
}
__device__ inline void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ inline void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

// Byte offset of element (row, k) inside a [rows][64] BF16 box written in the
// 128-byte-swizzled K-major layout (16-byte chunk index XOR row mod 8).
__device__ inline uint32_t sw128_offset(int row, int k) {
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((k >> 3) ^ (row & 7)) & 7) << 4) + (k & 7) * 2);
}

// Pack 8 values of the split operand row `nn` (0-2 hi of x,y,z, 3-5 lo,
// rest 0) for the 8 consecutive k whose FP32 vectors are given (times scale).
template <bool F16> __device__ inline uint4 split_chunk(int nn, const float3 *v, float scale) {
    uint16_t h[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        float x = 0.f;
        if (nn < 6) {
            int c = nn % 3;
            float a = scale * (c == 0 ? v[t].x : (c == 1 ? v[t].y : v[t].z));
            float hi = F16 ? __half2float(__float2half_rn(a)) : __bfloat162float(__float2bfloat16_rn(a));
            x = nn < 3 ? hi : a - hi;
        }
        if (F16) {
            __half e = __float2half_rn(x);
            memcpy(&h[t], &e, 2);
        } else {
            __nv_bfloat16 e = __float2bfloat16_rn(x);
            memcpy(&h[t], &e, 2);
        }
    }
    uint4 out;
    memcpy(&out, h, 16);
    return out;
}

// Power of two putting the block's largest |value| in [2^13, 2^14) (1 for
// BF16, whose exponent range is FP32's).  All threads of the block call it.
__device__ inline float block_scale_f16(float local_max, float *red) {
    for (int o = 16; o > 0; o >>= 1) local_max = fmaxf(local_max, __shfl_xor_sync(0xffffffffu, local_max, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = local_max;
    __syncthreads();
    float m = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
    __syncthreads();
    if (!(m > 0.f) || !isfinite(m)) return 1.f;
    int e;
    frexpf(m, &e);  // m in [2^(e-1), 2^e)
    return ldexpf(1.f, 14 - e);
}

template <bool F16> __device__ inline float block_scale(float local_max, float *red) {
    if constexpr (!F16) {
        return 1.f;
    } else {
        return block_scale_f16(local_max, red);
    }
}

template <class Smem> __device__ inline Smem &smem_1024() {
    extern __shared__ unsigned char smem_raw[];
    uintptr_t p = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023;
    return *reinterpret_cast<Smem *>(p);
}


// ------------------------------------------------------------------ persistent, pipelined versions
// One CTA per SM loops over its tiles with a ring of LSTAGES shared-memory
// stages, so the TMA stream of U never waits for an MMA or an epilogue.
// Warp roles: warps 0-3 write the split operand and read the accumulator
// (TMEM lane quadrant = warp), warp 4 issues the TMA loads, warp 5 owns TMEM
// and issues the MMAs.  Barrier phases: the i-th use of a barrier completes
// phase i, awaited with parity i & 1.
constexpr int PSTAGES = 3;
constexpr int PTHREADS = 192;

struct alignas(1024) LiftPSmem {
    unsigned char A[PSTAGES][UMMA_MAX_LD / KBOX][ABOX_BYTES];
    unsigned char B[UMMA_MAX_LD / KBOX][BBOX_BYTES];
    uint64_t full[PSTAGES], empty[PSTAGES], accfull[2], accempty[2];
    uint32_t taddr;
    int fail;
    float red[8];
};

struct alignas(1024) ProjPSmem {
    unsigned char A[PSTAGES][UMMA_MAX_LD / TILE][TILE / KBOX][ABOX_BYTES];
    unsigned char B[PSTAGES][TILE / KBOX][BBOX_BYTES];
    uint64_t afull[PSTAGES], bfull[PSTAGES], empty[PSTAGES], accdone;
    uint32_t taddr;
    int fail;
    float red[8];
};

__device__ inline bool failed(const int *f) { return *(const volatile int *)f != 0; }

// Producer tail after a failure: wait (bounded) for the copies this thread
// issued into the stages that were not consumed, so none lands after exit.
__device__ inline void drain_copies(uint64_t *full, int issued) {
    for (int k = issued - 1; k >= 0 && k >= issued - PSTAGES; --k) mbar_wait(&full[k % PSTAGES], (k / PSTAGES) & 1);
}

template <bool F16>
__global__ void __launch_bounds__(PTHREADS, 1) k_lift_umma_p(const __grid_constant__ CUtensorMap mapU, int n, int ld,
                                                            int r, const float *__restrict__ q,
                                                            const float4 *__restrict__ din, float4 *__restrict__ dout,
                                                            int *err, const int *skip_if, const int *live) {
    LiftPSmem &S = smem_1024<LiftPSmem>();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nkb = ld / KBOX;
    const int ntiles = (n + TILE - 1) / TILE;
    int mine = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (tid == 0) {
        S.fail = 0;
        for (int s = 0; s < PSTAGES; ++s) {
            mbar_init(&S.full[s], 1);
            mbar_init(&S.empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&S.accfull[a], 1);
            mbar_init(&S.accempty[a], 128);
        }
        mbar_fence_init();
    }
    if (warp == 5) {
        __syncwarp();
        tmem_alloc(&S.taddr);
    }
    // launched as a programmatic dependent: everything above overlapped the
    // previous kernel; q, din and dout are touched only after this wait
    grid_dep_wait();
    grid_dep_release();
    // the lift of an iteration with collision springs runs on the compact
    // basis instead (skip_if: that iteration's contact-vertex count)
    if ((skip_if && *skip_if > 0) || loop_dead(live)) mine = 0;
    // B = q split into hi / lo parts, [16][ld], fixed for all tiles
    float qmax = 0.f;
    for (int e = tid; e < 3 * r; e += blockDim.x) qmax = fmaxf(qmax, fabsf(q[e]));
    const float scale = block_scale<F16>(qmax, S.red);
    for (int c = tid; c < 16 * (ld / 8); c += blockDim.x) {
        int nn = c / (ld / 8), k0 = (c % (ld / 8)) * 8;
        float3 v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            int k = k0 + t;
            v[t] = k < r ? make_float3(q[k * 3 + 0], q[k * 3 + 1], q[k * 3 + 2]) : make_float3(0.f, 0.f, 0.f);
        }
        *reinterpret_cast<uint4 *>(S.B[k0 / KBOX] + sw128_offset(nn, k0 % KBOX)) = split_chunk<F16>(nn, v, scale);
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.taddr;
    int issued = 0;
    if (warp == 4) {
        if (lane == 0) {
            for (int k = 0; k < mine; ++k) {
                const int s = k % PSTAGES;
                if (k >= PSTAGES && !mbar_wait(&S.empty[s], ((k / PSTAGES) - 1) & 1)) {
                    atomicOr(&S.fail, 1);
                    break;
                }
                if (failed(&S.fail)) break;
                mbar_expect_tx(&S.full[s], (uint32_t)(nkb * ABOX_BYTES));
                const int row0 = ((int)blockIdx.x + k * (int)gridDim.x) * TILE;
                for (int kb = 0; kb < nkb; ++kb) tma_load_2d(S.A[s][kb], &mapU, &S.full[s], kb * KBOX, row0);
                issued = k + 1;
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            for (int k = 0; k < mine; ++k) {
                const int s = k % PSTAGES, a = k & 1;
                if (failed(&S.fail)) break;
                if (!mbar_wait(&S.full[s], (k / PSTAGES) & 1) ||
                    (k >= 2 && !mbar_wait(&S.accempty[a], ((k >> 1) - 1) & 1))) {
                    atomicOr(&S.fail, 1);
                    break;
                }
                tc_fence_after();
                for (int kb = 0; kb < nkb; ++kb)
#pragma unroll
                    for (int kk = 0; kk < KBOX / 16; ++kk)
                        umma<F16>(tmem + 16 * a, desc_sw128(smem_u32(S.A[s][kb]) + kk * 32),
                                  desc_sw128(smem_u32(S.B[kb]) + kk * 32), (kb | kk) != 0);
                umma_commit(&S.empty[s]);
                umma_commit(&S.accfull[a]);
            }
        }
    } else {
        const float inv = 1.f / scale;  // exact: a power of two
        for (int k = 0; k < mine; ++k) {
            const int a = k & 1;
            bool ok = mbar_wait(&S.accfull[a], (k >> 1) & 1);
            if (!__all_sync(0xffffffffu, ok)) {
                atomicOr(&S.fail, 1);
                break;
            }
            tc_fence_after();
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + 16 * a, v);
            tc_fence_before();
            mbar_arrive(&S.accempty[a]);
            const int i = ((int)blockIdx.x + k * (int)gridDim.x) * TILE + warp * 32 + lane;
            if (i < n) {
                float4 d = din ? din[i] : make_float4(0.f, 0.f, 0.f, 0.f);
                dout[i] = make_float4(d.x + inv * (v[0] + v[3]), d.y + inv * (v[1] + v[4]),
                                      d.z + inv * (v[2] + v[5]), 0.f);
            }
        }
    }
    __syncthreads();
    if (S.fail) {
        if (tid == 0) atomicOr(err, PDC_DEVERR_UMMA);
        if (warp == 4 && lane == 0) drain_copies(S.full, issued);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 5) {
        __syncwarp();
        tmem_dealloc(tmem);
    }
}

template <bool F16>
__global__ void __launch_bounds__(PTHREADS, 1) k_project_umma_p(const __grid_constant__ CUtensorMap mapUt, int n,
                                                               int ld, int r, const float4 *__restrict__ rl,
                                                               float *__restrict__ partial, int *err,
                                                               const int *skip_if, const int *live) {
    ProjPSmem &S = smem_1024<ProjPSmem>();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nh = ld / TILE;
    const int nchunks = (n + TILE - 1) / TILE;
    int mine = (int)blockIdx.x < nchunks ? (nchunks - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    if (tid == 0) {
        S.fail = 0;
        for (int s = 0; s < PSTAGES; ++s) {
            mbar_init(&S.afull[s], 1);
            mbar_init(&S.bfull[s], 128);
            mbar_init(&S.empty[s], 1);
        }
        mbar_init(&S.accdone, 1);
        mbar_fence_init();
    }
    if (warp == 5) {
        __syncwarp();
        tmem_alloc(&S.taddr);
    }
    // launched as a programmatic dependent: everything above overlapped the
    // previous kernel; rl and partial are touched only after this wait
    grid_dep_wait();
    grid_dep_release();
    // an iteration with collision springs projects on the compact basis instead
    if ((skip_if && *skip_if > 0) || loop_dead(live)) mine = 0;
    // one scale for all of this CTA's rows (its accumulator sums them all)
    float vmax = 0.f;
    for (int k = 0; k < mine; ++k) {
        const int i = ((int)blockIdx.x + k * (int)gridDim.x) * TILE + tid;
        if (tid < TILE && i < n) {
            float3 a = f3(rl[i]);
            vmax = fmaxf(vmax, fmaxf(fabsf(a.x), fmaxf(fabsf(a.y), fabsf(a.z))));
        }
    }
    const float scale = block_scale<F16>(vmax, S.red);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.taddr;
    int issued = 0;
    if (warp == 4) {
        if (lane == 0) {
            for (int k = 0; k < mine; ++k) {
                const int s = k % PSTAGES;
                if (k >= PSTAGES && !mbar_wait(&S.empty[s], ((k / PSTAGES) - 1) & 1)) {
                    atomicOr(&S.fail, 1);
                    break;
                }
                if (failed(&S.fail)) break;
                mbar_expect_tx(&S.afull[s], (uint32_t)(nh * (TILE / KBOX) * ABOX_BYTES));
                const int i0 = ((int)blockIdx.x + k * (int)gridDim.x) * TILE;
                for (int h = 0; h < nh; ++h)
                    for (int kb = 0; kb < TILE / KBOX; ++kb)
                        tma_load_2d(S.A[s][h][kb], &mapUt, &S.afull[s], i0 + kb * KBOX, h * TILE);
                issued = k + 1;
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            int k = 0;
            for (; k < mine; ++k) {
                const int s = k % PSTAGES;
                if (failed(&S.fail)) break;
                if (!mbar_wait(&S.afull[s], (k / PSTAGES) & 1) || !mbar_wait(&S.bfull[s], (k / PSTAGES) & 1)) {
                    atomicOr(&S.fail, 1);
                    break;
                }
                tc_fence_after();
                for (int h = 0; h < nh; ++h)
                    for (int kb = 0; kb < TILE / KBOX; ++kb)
#pragma unroll
                        for (int kk = 0; kk < KBOX / 16; ++kk)
                            umma<F16>(tmem + 16 * h, desc_sw128(smem_u32(S.A[s][h][kb]) + kk * 32),
                                      desc_sw128(smem_u32(S.B[s][kb]) + kk * 32), (k | kb | kk) != 0);
                umma_commit(&S.empty[s]);
            }
            if (k == mine && mine > 0) umma_commit(&S.accdone);
            else mbar_arrive(&S.accdone);  // nothing accumulated, or given up: release the readers
        }
    } else {
        // write B = rl split into hi / lo parts, [16][128] per chunk
        for (int k = 0; k < mine; ++k) {
            const int s = k % PSTAGES;
            if (failed(&S.fail)) break;
            bool ok = k < PSTAGES || mbar_wait(&S.empty[s], ((k / PSTAGES) - 1) & 1);
            if (!ok) {
                atomicOr(&S.fail, 1);
                break;
            }
            const int i0 = ((int)blockIdx.x + k * (int)gridDim.x) * TILE;
            for (int c = tid; c < 16 * (TILE / 8); c += 128) {
                int nn = c / (TILE / 8), k0 = (c % (TILE / 8)) * 8;
                float3 v[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    int i = i0 + k0 + t;
                    v[t] = i < n ? f3(rl[i]) : make_float3(0.f, 0.f, 0.f);
                }
                *reinterpret_cast<uint4 *>(S.B[s][k0 / KBOX] + sw128_offset(nn, k0 % KBOX)) =
                    split_chunk<F16>(nn, v, scale);
            }
            fence_async_smem();
            mbar_arrive(&S.bfull[s]);
        }
        bool ok = mbar_wait(&S.accdone, 0);
        if (!__all_sync(0xffffffffu, ok)) atomicOr(&S.fail, 1);
    }
    __syncthreads();  // S.fail is final and uniform from here on
    if (!S.fail && warp < 4 && mine > 0) {
        tc_fence_after();
        const float inv = 1.f / scale;  // exact: a power of two
        for (int h = 0; h < nh; ++h) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + 16 * h, v);
            const int j = h * TILE + warp * 32 + lane;
            if (j < r) {
                float *p = partial + ((long long)blockIdx.x * ld + j) * 3;
                p[0] = inv * (v[0] + v[3]);
                p[1] = inv * (v[1] + v[4]);
                p[2] = inv * (v[2] + v[5]);
            }
        }
    } else if (!S.fail && warp < 4) {
        for (int h = 0; h < nh; ++h) {
            const int j = h * TILE + warp * 32 + lane;
            if (j < r) {
                float *p = partial + ((long long)blockIdx.x * ld + j) * 3;
                p[0] = p[1] = p[2] = 0.f;
            }
        }
    }
    if (S.fail) {
        if (tid == 0) atomicOr(err, PDC_DEVERR_UMMA);
        if (warp == 4 && lane == 0) drain_copies(S.afull, issued);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 5) {
        __syncwarp();
        tmem_dealloc(tmem);
    }
}

__global__ void k_umma_reduce(int r, int ld, int nblocks, const float *__restrict__ partial, double *__restrict__ g,
                              const int *skip_if, const int *live) {
    grid_dep_wait();
    grid_dep_release();
    if ((skip_if && *skip_if > 0) || loop_dead(live)) return;
    int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (e >= r * 3) return;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += (double)partial[(long long)b * ld * 3 + e];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) g[e] = s;
}

size_t lift_p_smem() { return sizeof(LiftPSmem) + 1024; }
size_t proj_p_smem() { return sizeof(ProjPSmem) + 1024; }

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        PDC_CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !p) throw Error(PDC_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D BF16 tensor map over a row-major [rows][cols] array with row stride
// `stride` elements; boxes of 64 columns x 128 rows, 128-byte swizzle.
void encode_map(CUtensorMap *m, const void *base, uint64_t cols, uint64_t rows, uint64_t stride, bool f16) {
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (stride * 2) % 16)
        throw Error(PDC_ERR_ARG, "tensor map: base and row stride must be 16-byte aligned");
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {stride * 2};
    cuuint32_t box[2] = {KBOX, TILE};
    cuuint32_t es[2] = {1, 1};
    CUresult rc = encode_fn()(m, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                              const_cast<void *>(base), dims, strides, box,
                              es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (rc != CUDA_SUCCESS) throw Error(PDC_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)rc));
}

}  // namespace

bool umma_supported(int ld, int n) { return ld > 0 && ld % TILE == 0 && ld <= UMMA_MAX_LD && n > 0; }

void umma_setup(UmmaMaps &M, const void *U, const void *Ut, bool f16, int n, int n_pad, int ld) {
    M.ok = false;
    if (!umma_supported(ld, n) || !U || !Ut) return;
    encode_map(&M.mapU, U, (uint64_t)ld, (uint64_t)n, (uint64_t)ld, f16);
    encode_map(&M.mapUt, Ut, (uint64_t)n, (uint64_t)ld, (uint64_t)n_pad, f16);
    PDC_CK(cudaFuncSetAttribute(k_lift_umma_p<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lift_p_smem()));
    PDC_CK(cudaFuncSetAttribute(k_lift_umma_p<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lift_p_smem()));
    PDC_CK(cudaFuncSetAttribute(k_project_umma_p<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)proj_p_smem()));
    PDC_CK(cudaFuncSetAttribute(k_project_umma_p<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)proj_p_smem()));
    int dev = 0;
    PDC_CK(cudaGetDevice(&dev));
    PDC_CK(cudaDeviceGetAttribute(&M.sms, cudaDevAttrMultiProcessorCount, dev));
    M.n = n;
    M.ld = ld;
    M.f16 = f16;
    M.ok = true;
}

int umma_project_blocks(int n) { return (n + TILE - 1) / TILE; }

void launch_project_umma(cudaStream_t s, const UmmaMaps &M, int r, const float4 *rl, float *partial, double *g,
                         int *err, bool overlap, const int *skip_if, const int *live) {
    const int nb = std::max(1, std::min(M.sms, umma_project_blocks(M.n)));
    if (M.f16)
        launch_dependent(overlap, k_project_umma_p<true>, nb, PTHREADS, proj_p_smem(), s, M.mapUt, M.n, M.ld, r, rl,
                         partial, err, skip_if, live);
    else
        launch_dependent(overlap, k_project_umma_p<false>, nb, PTHREADS, proj_p_smem(), s, M.mapUt, M.n, M.ld, r, rl,
                         partial, err, skip_if, live);
    PDC_LAUNCH_CK();
    int thr = r * 3 * 32;
    launch_dependent(overlap, k_umma_reduce, (thr + 255) / 256, 256, 0, s, r, M.ld, nb, (const float *)partial, g,
                     skip_if, live);
    PDC_LAUNCH_CK();
}

void launch_lift_umma(cudaStream_t s, const UmmaMaps &M, int r, const float *q, const float4 *din, float4 *dout,
                      int *err, bool overlap, const int *skip_if, const int *live) {
    const int nt = (M.n + TILE - 1) / TILE;
    const int nb = std::max(1, std::min(M.sms, nt));
    if (M.f16)
        launch_dependent(overlap, k_lift_umma_p<true>, nb, PTHREADS, lift_p_smem(), s, M.mapU, M.n, M.ld, r, q, din,
                         dout, err, skip_if, live);
    else
        launch_dependent(overlap, k_lift_umma_p<false>, nb, PTHREADS, lift_p_smem(), s, M.mapU, M.n, M.ld, r, q, din,
                         dout, err, skip_if, live);
    PDC_LAUNCH_CK();
}

}  // namespace pdc
