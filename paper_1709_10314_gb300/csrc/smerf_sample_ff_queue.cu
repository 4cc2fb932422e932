// The persistent single batch launch for float recursion and float step tables.
#include "smerf_sample_impl.cuh"

SMERF_QUEUE(float, float, ff)
