// Sampling kernels with double recursion/FFT/output and float step tables.
#include "smerf_sample_impl.cuh"

int smerf_launch_sample_df(const smerf_plan* pl, uint64_t seed, int n, void* out, void* scratch, cudaStream_t st,
                          cudaEvent_t ev0, cudaEvent_t ev1)
{
    return smerf::launch_sample_t<double, float>(pl, seed, n, out, scratch, st, ev0, ev1);
}

int smerf_fill_params_df(const smerf_plan* pl, uint64_t seed, int n, void* out, void* scratch,
                         smerf::SampleParams* P, int* batchable, int* rmax)
{
    return smerf::fill_params_c<double, float>(pl, seed, n, out, scratch, P, batchable, rmax);
}

int smerf_launch_group_df(const smerf_plan* rep, const smerf::SampleParams* d_descs, const int4* anc_items,
                          int n_anc, const int4* seg_items, int n_seg, cudaStream_t st)
{
    return smerf::launch_group_t<double, float>(rep, d_descs, anc_items, n_anc, seg_items, n_seg, st);
}

int smerf_tune_candidates_df(const smerf_plan* pl, int* cand, int max_n)
{
    return smerf::tune_candidates<double>(pl, cand, max_n);
}
