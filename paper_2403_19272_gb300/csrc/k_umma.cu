// Tensor-core (tcgen05) kernels for the BF16 subspace contractions.
#include "pdc_subspace.cuh"
