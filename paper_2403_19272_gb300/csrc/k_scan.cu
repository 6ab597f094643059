// Device-wide exclusive prefix sum of int32 counts (three passes:
// per-block scan, scan of block sums in one block, add offsets).
// Used for hash-bucket offsets and candidate-pair offsets.
#include "pdc_scan.cuh"

namespace pdc {

namespace {

constexpr int SCAN_T = 1024;           // threads per block
constexpr int SCAN_E = 4;              // elements per thread
constexpr int SCAN_B = SCAN_T * SCAN_E; // elements per block

__device__ inline int block_excl_scan(int v, int *sh, int &total) {
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int nw = blockDim.x >> 5;
        int s = lane < nw ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sh[lane] = s;
    }
    __syncthreads();
    int base = w > 0 ? sh[w - 1] : 0;
    total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return base + x - v;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_local(const int *__restrict__ in, int n, int *__restrict__ out,
                                                       int *__restrict__ bsum) {
    __shared__ int sh[32];
    long long base = (long long)blockIdx.x * SCAN_B + (long long)threadIdx.x * SCAN_E;
    int v[SCAN_E];
    int s = 0;
    for (int k = 0; k < SCAN_E; ++k) {
        long long i = base + k;
        v[k] = i < n ? in[i] : 0;
        s += v[k];
    }
    int tot;
    int ex = block_excl_scan(s, sh, tot);
    for (int k = 0; k < SCAN_E; ++k) {
        long long i = base + k;
        if (i < n) out[i] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_sums(int *__restrict__ bsum, int nb, long long *__restrict__ total) {
    __shared__ int sh[32];
    int v[SCAN_E];
    int s = 0;
    // nb <= SCAN_B (checked on the host)
    for (int k = 0; k < SCAN_E; ++k) {
        int i = threadIdx.x * SCAN_E + k;
        v[k] = i < nb ? bsum[i] : 0;
        s += v[k];
    }
    int tot;
    int ex = block_excl_scan(s, sh, tot);
    for (int k = 0; k < SCAN_E; ++k) {
        int i = threadIdx.x * SCAN_E + k;
        if (i < nb) bsum[i] = ex;
        ex += v[k];
    }
    if (threadIdx.x == 0 && total) *total = (long long)tot;
}

__global__ void k_scan_add(int *__restrict__ out, int n, const int *__restrict__ bsum) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += bsum[i / SCAN_B];
}

}  // namespace

size_t scan_scratch_ints(int n) { return (size_t)((n + SCAN_B - 1) / SCAN_B) + 1; }
long long scan_capacity() { return (long long)SCAN_B * SCAN_B; }

void exclusive_scan(cudaStream_t s, const int *in, int *out, int n, int *scratch, long long *total) {
    if (n <= 0) {
        if (total) PDC_CK(cudaMemsetAsync(total, 0, sizeof(long long), s));
        return;
    }
    int nb = (n + SCAN_B - 1) / SCAN_B;
    if (nb > SCAN_B) throw Error(PDC_ERR_CAPACITY, "exclusive_scan: too many elements");
    k_scan_local<<<nb, SCAN_T, 0, s>>>(in, n, out, scratch);
    k_scan_sums<<<1, SCAN_T, 0, s>>>(scratch, nb, total);
    k_scan_add<<<(n + 255) / 256, 256, 0, s>>>(out, n, scratch);
    PDC_LAUNCH_CK();
}

}  // namespace pdc
