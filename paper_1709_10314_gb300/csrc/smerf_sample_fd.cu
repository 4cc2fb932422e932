// Sampling entry points for float recursion/FFT/output and double step tables.
#include "smerf_sample_impl.cuh"

SMERF_PRECISION_PAIR(float, double, fd)

// FP64 tables converted once per call to the FP32 values the float-recursion kernels use
// (the same conversion the kernels apply when they read FP64 rows themselves).
namespace {
__global__ void stage_tables_kernel(const double* __restrict__ src, float* __restrict__ dst, size_t n)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = smerf::tabcvt<float, double>(src[i]);
}
}  // namespace

int smerf_stage_tables(const double* src, float* dst, size_t n, cudaStream_t st)
{
    if (n == 0) return SMERF_OK;
    const size_t blocks = (n + 255) / 256;
    stage_tables_kernel<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError() == cudaSuccess ? SMERF_OK : SMERF_ECUDA;
}
