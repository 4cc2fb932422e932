// Sampling kernels for float recursion/FFT/output and float step tables, p = 3.
#include "smerf_sample_impl.cuh"

SMERF_INSTANTIATE(float, float, ff, 3)

// FP64 tables staged as FP32 per call, FP32 recursion (float-table kernels)
int smerf_launch_sample_staged_p3(const smerf_plan* sh, const StageSmall& S, const StageJob& J, uint64_t seed,
                                  int n, void* out, void* scratch, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1)
{
    return smerf::launch_sample_staged_m<3>(sh, S, J, seed, n, out, scratch, st, ev0, ev1);
}
