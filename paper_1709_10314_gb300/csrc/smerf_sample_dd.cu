// Sampling entry points for double recursion/FFT/output and double step tables.
#include "smerf_sample_impl.cuh"

SMERF_PRECISION_PAIR(double, double, dd)
