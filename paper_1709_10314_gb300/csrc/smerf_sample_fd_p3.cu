// Sampling kernels for float recursion/FFT/output and double step tables, p = 3.
#include "smerf_sample_impl.cuh"

SMERF_INSTANTIATE(float, double, fd, 3)
