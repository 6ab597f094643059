// Device-wide exclusive scan of int32 counts.
#pragma once
#include "pdc_internal.cuh"

namespace pdc {
// Number of int32 scratch entries exclusive_scan needs for n elements.
size_t scan_scratch_ints(int n);
long long scan_capacity();  // largest n exclusive_scan accepts
// out[i] = sum_{j<i} in[j]; *total (device, may be NULL) = sum of all.
// in and out may alias.  n <= 16,777,216.
void exclusive_scan(cudaStream_t s, const int *in, int *out, int n, int *scratch, long long *total);
}  // namespace pdc
