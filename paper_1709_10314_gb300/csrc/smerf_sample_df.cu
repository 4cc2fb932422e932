// Sampling entry points for double recursion/FFT/output and float step tables.
#include "smerf_sample_impl.cuh"

SMERF_PRECISION_PAIR(double, float, df)
