// Tensor-core (tcgen05) kernels for the BF16 subspace contractions of the
// mixed form (Sec. 5: g = U^T r of Eq. subspace_global and the lift
// delta = U q of Eq. subspace_collision), without collision springs.
//
// Both products are tall-skinny: U is n x r (BF16), the other operand n x 3
// or r x 3 (FP32).  The FP32 operand is split into two BF16 parts,
// v = hi + lo with hi = bf16(v) and lo = bf16(v - hi), so that the tensor
// cores see a 6-column BF16 operand (padded to N = 16) and the FP32
// accumulator receives U^T hi + U^T lo, i.e. the product with a 16-bit
// significand instead of BF16's 8.  The kernels stream U once; they are
// bound by that HBM stream, not by the tensor pipe.
//
// Layout (both operands K-major, 128-byte swizzle):
//   lift:       A = U tile [128 rows][r] from U   [n][ld]        (TMA)
//               B = q hi/lo [16][r]                (written by the CTA)
//   projection: A = U^T tile [128 j][128 i] from Ut [ld][n_pad]  (TMA)
//               B = r hi/lo [16][128 i]            (written by the CTA)
// One CTA per 128-row tile, 4 warps: thread 0 issues the TMA loads and the
// MMAs, warp 0 owns the 32 TMEM columns, all four warps read the
// accumulator (warp w: TMEM lanes 32w..32w+31).  Every wait on an mbarrier
// is bounded by the global timer; on expiry the CTA records an error bit,
// waits (bounded) for its copies, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "pdc_subspace.cuh"
#include "pdc_umma.cuh"

namespace pdc {

namespace {

constexpr int TILE = 128;            // rows of U per CTA (lift) / U^T rows per MMA (projection)
constexpr int KBOX = 64;             // BF16 elements per 128-byte swizzle row
constexpr int ABOX_BYTES = TILE * 128;  // one [128][64] BF16 box
constexpr int BBOX_BYTES = 16 * 128;    // one [16][64] BF16 box
constexpr uint32_t NCOLS = 32;       // TMEM columns per CTA
constexpr unsigned long long WAIT_NS = 1000000000ull;  // 1 s

__device__ inline uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ inline void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ inline void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ inline void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ inline void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ inline bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
// Wait for phase `parity` of the barrier, giving up after WAIT_NS.
__device__ inline bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_test(bar, parity)) return true;
    unsigned long long t0 = global_ns();
    while (!mbar_test(bar, parity)) {
        if (global_ns() - t0 > WAIT_NS) return false;
        __nanosleep(64);
    }
    return true;
}

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

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, M = 128, N = 16.
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ inline void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(IDESC), "r"(accumulate)
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

// Pack 8 BF16 values of the split operand row `nn` (0-2 hi of x,y,z, 3-5 lo,
// rest 0) for the 8 consecutive k whose FP32 vectors are given.
__device__ inline uint4 split_chunk(int nn, const float3 *v) {
    __nv_bfloat16 h[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        float x = 0.f;
        if (nn < 6) {
            int c = nn % 3;
            float a = c == 0 ? v[t].x : (c == 1 ? v[t].y : v[t].z);
            __nv_bfloat16 hi = __float2bfloat16_rn(a);
            x = nn < 3 ? __bfloat162float(hi) : a - __bfloat162float(hi);
        }
        h[t] = __float2bfloat16_rn(x);
    }
    uint4 out;
    memcpy(&out, h, 16);
    return out;
}

struct alignas(1024) LiftSmem {
    unsigned char A[UMMA_MAX_LD / KBOX][ABOX_BYTES];
    unsigned char B[UMMA_MAX_LD / KBOX][BBOX_BYTES];
    uint64_t bar_tma, bar_mma;
    uint32_t taddr;
    int fail;
};

struct alignas(1024) ProjSmem {
    unsigned char A[UMMA_MAX_LD / TILE][TILE / KBOX][ABOX_BYTES];
    unsigned char B[TILE / KBOX][BBOX_BYTES];
    uint64_t bar_tma, bar_mma;
    uint32_t taddr;
    int fail;
};

template <class Smem> __device__ inline Smem &smem_1024() {
    extern __shared__ unsigned char smem_raw[];
    uintptr_t p = (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023;
    return *reinterpret_cast<Smem *>(p);
}

// Wait for the MMAs; on expiry mark the CTA failed (no TMEM reads follow).
__device__ inline void wait_or_flag(uint64_t *bar, uint32_t parity, int *fail) {
    if (!mbar_wait(bar, parity)) atomicOr(fail, 1);
}

// dout_i = din_i + sum_j U[i][j] q_j for the 128 rows of this CTA's tile.
__global__ void __launch_bounds__(128, 1) k_lift_umma(const __grid_constant__ CUtensorMap mapU, int n, int ld, int r,
                                                      const float *__restrict__ q, const float4 *__restrict__ din,
                                                      float4 *__restrict__ dout, int *err) {
    LiftSmem &S = smem_1024<LiftSmem>();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nkb = ld / KBOX;
    const int row0 = blockIdx.x * TILE;
    if (tid == 0) {
        S.fail = 0;
        mbar_init(&S.bar_tma, 1);
        mbar_init(&S.bar_mma, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(&S.bar_tma, (uint32_t)(nkb * ABOX_BYTES));
        for (int kb = 0; kb < nkb; ++kb) tma_load_2d(S.A[kb], &mapU, &S.bar_tma, kb * KBOX, row0);
    }
    if (warp == 0) {
        __syncwarp();
        tmem_alloc(&S.taddr);
    }
    // B = q split into hi / lo parts: [16][ld] in swizzled 64-column boxes
    for (int c = tid; c < 16 * (ld / 8); c += blockDim.x) {
        int nn = c / (ld / 8), k0 = (c % (ld / 8)) * 8;
        float3 v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            int k = k0 + t;
            v[t] = k < r ? make_float3(q[k * 3 + 0], q[k * 3 + 1], q[k * 3 + 2]) : make_float3(0.f, 0.f, 0.f);
        }
        uint4 val = split_chunk(nn, v);
        *reinterpret_cast<uint4 *>(S.B[k0 / KBOX] + sw128_offset(nn, k0 % KBOX)) = val;
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.taddr;
    if (tid == 0) {
        if (mbar_wait(&S.bar_tma, 0)) {
            tc_fence_after();
            for (int kb = 0; kb < nkb; ++kb)
#pragma unroll
                for (int k = 0; k < KBOX / 16; ++k)
                    umma(tmem, desc_sw128(smem_u32(S.A[kb]) + k * 32), desc_sw128(smem_u32(S.B[kb]) + k * 32),
                         (kb | k) != 0);
            umma_commit(&S.bar_mma);
        } else {
            S.fail = 1;
            mbar_arrive(&S.bar_mma);
        }
    }
    __syncwarp();
    wait_or_flag(&S.bar_mma, 0, &S.fail);
    tc_fence_after();
    __syncthreads();  // S.fail is uniform from here on
    if (S.fail) {
        if (tid == 0) {
            atomicOr(err, PDC_DEVERR_UMMA);
            mbar_wait(&S.bar_tma, 0);  // let the copies land before the CTA exits
        }
    } else {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), v);
        int i = row0 + warp * 32 + lane;
        if (i < n) {
            float4 d = din ? din[i] : make_float4(0.f, 0.f, 0.f, 0.f);
            dout[i] = make_float4(d.x + (v[0] + v[3]), d.y + (v[1] + v[4]), d.z + (v[2] + v[5]), 0.f);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tmem_dealloc(tmem);
    }
}

// partial[b][j][c] = sum over the 128 rows i of tile b of U[i][j] rl_i[c].
__global__ void __launch_bounds__(128, 1) k_project_umma(const __grid_constant__ CUtensorMap mapUt, int n, int ld,
                                                         int r, const float4 *__restrict__ rl,
                                                         float *__restrict__ partial, int *err) {
    ProjSmem &S = smem_1024<ProjSmem>();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nh = ld / TILE;
    const int i0 = blockIdx.x * TILE;
    if (tid == 0) {
        S.fail = 0;
        mbar_init(&S.bar_tma, 1);
        mbar_init(&S.bar_mma, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (tid == 0) {
        mbar_expect_tx(&S.bar_tma, (uint32_t)(nh * (TILE / KBOX) * ABOX_BYTES));
        for (int h = 0; h < nh; ++h)
            for (int kb = 0; kb < TILE / KBOX; ++kb) tma_load_2d(S.A[h][kb], &mapUt, &S.bar_tma, i0 + kb * KBOX, h * TILE);
    }
    if (warp == 0) {
        __syncwarp();
        tmem_alloc(&S.taddr);
    }
    // B = r split into hi / lo parts: [16][128] for rows i0 .. i0+127
    for (int c = tid; c < 16 * (TILE / 8); c += blockDim.x) {
        int nn = c / (TILE / 8), k0 = (c % (TILE / 8)) * 8;
        float3 v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            int i = i0 + k0 + t;
            v[t] = i < n ? f3(rl[i]) : make_float3(0.f, 0.f, 0.f);
        }
        uint4 val = split_chunk(nn, v);
        *reinterpret_cast<uint4 *>(S.B[k0 / KBOX] + sw128_offset(nn, k0 % KBOX)) = val;
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.taddr;
    if (tid == 0) {
        if (mbar_wait(&S.bar_tma, 0)) {
            tc_fence_after();
            for (int h = 0; h < nh; ++h)
                for (int kb = 0; kb < TILE / KBOX; ++kb)
#pragma unroll
                    for (int k = 0; k < KBOX / 16; ++k)
                        umma(tmem + 16 * h, desc_sw128(smem_u32(S.A[h][kb]) + k * 32),
                             desc_sw128(smem_u32(S.B[kb]) + k * 32), (kb | k) != 0);
            umma_commit(&S.bar_mma);
        } else {
            S.fail = 1;
            mbar_arrive(&S.bar_mma);
        }
    }
    __syncwarp();
    wait_or_flag(&S.bar_mma, 0, &S.fail);
    tc_fence_after();
    __syncthreads();  // S.fail is uniform from here on
    if (S.fail) {
        if (tid == 0) {
            atomicOr(err, PDC_DEVERR_UMMA);
            mbar_wait(&S.bar_tma, 0);
        }
    } else {
        for (int h = 0; h < nh; ++h) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + 16 * h, v);
            int j = h * TILE + warp * 32 + lane;
            if (j < r) {
                float *p = partial + ((long long)blockIdx.x * ld + j) * 3;
                p[0] = v[0] + v[3];
                p[1] = v[1] + v[4];
                p[2] = v[2] + v[5];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tmem_dealloc(tmem);
    }
}

__global__ void k_umma_reduce(int r, int ld, int nblocks, const float *__restrict__ partial, double *__restrict__ g) {
    int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (e >= r * 3) return;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += (double)partial[(long long)b * ld * 3 + e];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) g[e] = s;
}

size_t lift_smem() { return sizeof(LiftSmem) + 1024; }
size_t proj_smem() { return sizeof(ProjSmem) + 1024; }

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
void encode_map(CUtensorMap *m, const void *base, uint64_t cols, uint64_t rows, uint64_t stride) {
    if ((reinterpret_cast<uintptr_t>(base) & 15) || (stride * 2) % 16)
        throw Error(PDC_ERR_ARG, "tensor map: base and row stride must be 16-byte aligned");
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {stride * 2};
    cuuint32_t box[2] = {KBOX, TILE};
    cuuint32_t es[2] = {1, 1};
    CUresult rc = encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box,
                              es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (rc != CUDA_SUCCESS) throw Error(PDC_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)rc));
}

}  // namespace

bool umma_supported(int ld, int n) { return ld > 0 && ld % TILE == 0 && ld <= UMMA_MAX_LD && n > 0; }

void umma_setup(UmmaMaps &M, const __nv_bfloat16 *U, const __nv_bfloat16 *Ut, int n, int n_pad, int ld) {
    M.ok = false;
    if (!umma_supported(ld, n) || !U || !Ut) return;
    encode_map(&M.mapU, U, (uint64_t)ld, (uint64_t)n, (uint64_t)ld);
    encode_map(&M.mapUt, Ut, (uint64_t)n, (uint64_t)ld, (uint64_t)n_pad);
    PDC_CK(cudaFuncSetAttribute(k_lift_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lift_smem()));
    PDC_CK(cudaFuncSetAttribute(k_project_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)proj_smem()));
    M.n = n;
    M.ld = ld;
    M.ok = true;
}

int umma_project_blocks(int n) { return (n + TILE - 1) / TILE; }

void launch_project_umma(cudaStream_t s, const UmmaMaps &M, int r, const float4 *rl, float *partial, double *g,
                         int *err) {
    int nb = umma_project_blocks(M.n);
    k_project_umma<<<nb, 128, proj_smem(), s>>>(M.mapUt, M.n, M.ld, r, rl, partial, err);
    PDC_LAUNCH_CK();
    int thr = r * 3 * 32;
    k_umma_reduce<<<(thr + 255) / 256, 256, 0, s>>>(r, M.ld, nb, partial, g);
    PDC_LAUNCH_CK();
}

void launch_lift_umma(cudaStream_t s, const UmmaMaps &M, int r, const float *q, const float4 *din, float4 *dout,
                      int *err) {
    int nb = (M.n + TILE - 1) / TILE;
    k_lift_umma<<<nb, 128, lift_smem(), s>>>(M.mapU, M.n, M.ld, r, q, din, dout, err);
    PDC_LAUNCH_CK();
}

}  // namespace pdc
