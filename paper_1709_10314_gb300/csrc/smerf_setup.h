// smerf_setup.h -- the set-up entry point (smerf_setup.cu) used by smerf_api.cu.
#pragma once
#include <cuda_runtime.h>

struct smerf_plan;

// Set-up of a plan's tables (Alg. 1), every device step ordered on `st`.  sync: wait for it
// and record setup_ms; otherwise the caller synchronises `st` before the plan is used.
int smerf_setup_tables(smerf_plan* plan, cudaStream_t st, bool sync);

// Whether the ring colatitudes (n_theta values, increasing) are symmetric about the equator,
// theta_k + theta_{n_theta-1-k} = pi within 1e-12 pi; NULL (the equiangular grid) is.  On a
// symmetric grid the southern chain's steps are the northern ones mirrored and the start ring is
// n_theta / 2; otherwise the start ring is the ring nearest the equator and the southern chain's
// steps are computed on their own.
bool smerf_grid_symmetric(const double* theta, int n_theta);

// The start ring k0 of both chains (Alg. 2 starts at the equator): n_theta / 2 on a symmetric
// grid (the equator ring for odd n_theta, the first ring south of it for even n_theta), else the
// ring whose colatitude is nearest pi / 2, the southern one of two at the same distance.
int smerf_start_ring(const double* theta, int n_theta);
