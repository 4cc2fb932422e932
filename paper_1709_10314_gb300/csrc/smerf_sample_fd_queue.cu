// The persistent single batch launch for float recursion and double step tables.
#include "smerf_sample_impl.cuh"

SMERF_QUEUE(float, double, fd)
