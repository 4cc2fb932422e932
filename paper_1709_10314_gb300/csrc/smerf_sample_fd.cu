// Sampling entry points for float recursion/FFT/output and double step tables.
#include "smerf_sample_impl.cuh"

SMERF_PRECISION_PAIR(float, double, fd)
