// Sampling kernels for double recursion/FFT/output and float step tables, p = 1.
#include "smerf_sample_impl.cuh"

SMERF_INSTANTIATE(double, float, df, 1)
