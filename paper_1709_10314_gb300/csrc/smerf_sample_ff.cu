// Sampling kernels with float recursion/FFT/output and float step tables.
#include "smerf_sample_impl.cuh"

int smerf_launch_sample_ff(const smerf_plan* pl, uint64_t seed, int n, void* out, void* scratch, cudaStream_t st,
                          cudaEvent_t ev0, cudaEvent_t ev1)
{
    return smerf::launch_sample_t<float, float>(pl, seed, n, out, scratch, st, ev0, ev1);
}
