// Sampling kernels for float recursion/FFT/output and float step tables, p = 1.
#include "smerf_sample_impl.cuh"

SMERF_INSTANTIATE(float, float, ff, 1)
