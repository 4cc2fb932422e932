// smerf_setup.h -- the set-up entry point (smerf_setup.cu) used by smerf_api.cu.
#pragma once
#include <cuda_runtime.h>

struct smerf_plan;

// Set-up of a plan's tables (Alg. 1), every device step ordered on `st`.  sync: wait for it
// and record setup_ms; otherwise the caller synchronises `st` before the plan is used.
int smerf_setup_tables(smerf_plan* plan, cudaStream_t st, bool sync);
