// Sampling kernels for double recursion/FFT/output and float step tables, p = 3.
#include "smerf_sample_impl.cuh"

SMERF_INSTANTIATE(double, float, df, 3)
