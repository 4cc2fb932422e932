// Sampling kernels for double recursion/FFT/output and double step tables, p = 3.
#include "smerf_sample_impl.cuh"

SMERF_INSTANTIATE(double, double, dd, 3)
