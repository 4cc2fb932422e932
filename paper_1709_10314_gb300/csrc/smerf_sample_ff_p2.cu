// Sampling kernels for float recursion/FFT/output and float step tables, p = 2.
#include "smerf_sample_impl.cuh"

SMERF_INSTANTIATE(float, float, ff, 2)
