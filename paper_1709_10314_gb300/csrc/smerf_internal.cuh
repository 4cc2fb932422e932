// smerf_internal.cuh -- shared device helpers and the plan structure of the GB300
// sphere-GMRF sampler (Creasey & Lang, arXiv 1709.10314).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include "../../include/smerf.h"

#ifndef SMERF_PI
#define SMERF_PI 3.14159265358979323846
#endif

namespace smerf {

constexpr int kMaxP = 3;             // spectrum factors supported by the kernels
constexpr int kDefaultAnchor = 16;   // default anchor spacing H

// ------------------------------------------------------------------ plan
struct Chain {
    int len;          // positions 1..len after the start ring
    int n_anchors;    // anchors at positions H, 2H, ... <= len
};

struct Segment {      // one independently sampled run of rings
    int chain;        // 0 north, 1 south
    int p0;           // left anchor position (0 = start ring)
    int p1;           // one past the last position sampled here
    int left;         // anchor index of p0 (0 = start)
    int right;        // anchor index of p1 if p1 is an anchor, else -1
};

}  // namespace smerf

struct smerf_plan {
    int p;                 // M
    double kappa[smerf::kMaxP];   // real spectra: kappa_i (kappa-hat_i = kappa_i^2)
    double khat_re[smerf::kMaxP], khat_im[smerf::kMaxP];  // kappa-hat_i
    int complex_spec;              // some kappa-hat_i is complex (a conjugate pair)
    double A;
    int n_theta, n_phi, n_modes, n_modes_pad, n_slots;
    // ring colatitudes of an iso-latitude grid other than the equiangular one (host and device
    // copies, symmetric about the equator; null: theta_k = pi (k + 1/2) / n_theta)
    double* theta_host;
    double* theta_dev;
    int k0;
    unsigned flags;
    int H;                 // effective anchor spacing (0 = none)
    bool recur64, tab64;
    // p = 1 FP32 step tables of plans run by the ring kernel are stored packed: per position
    // three rows A, C, B of n_modes_pad values (12 bytes per (mode, ring)) instead of one
    // 16-byte row per mode
    bool packed;
    smerf::Chain chain[2];
    int n_segments;
    smerf::Segment* segs_host;
    smerf::Segment* segs_dev;
    // tables (TabT = double if tab64 else float)
    void* beq;             // [tri][n_modes_pad]
    void* steps[2];        // [len+1][n_modes_pad][step_row]
    void* coarse[2];       // [n_anchors+1][Ec][n_modes_pad] (row 0 unused)
    // FFT tables in the recursion precision: per-pass twiddles, pre[Nc] = e^{2 pi i s / n_phi}
    void* tw;
    void* pre;
    // per-pass twiddles of the high-radix plans (hr_* below, MB = 4 and 3), recursion precision
    void* tw2;
    void* tw3;
    size_t table_bytes;
    size_t step_table_bytes;  // the two step tables' part of table_bytes
    double setup_ms;
    int dev;
    // ring-dependent longitudes (smerf_plan_set_rings; rings_total = 0: none)
    int* rings_n_dev;
    double* rings_h_dev;
    long long* rings_off_dev;
    long long rings_total;
    // launch parameters chosen by smerf_plan_autotune (valid = 0: built-in heuristic)
    struct { int valid, upt, rmax, np, nf, minb, radix; float ms; } tune;
};

namespace smerf {

constexpr int kLaunchInts = SMERF_LAUNCH_INTS;  // integers per launch configuration

__host__ __device__ constexpr int tri(int M) { return M * (M + 1) / 2; }
__host__ __device__ constexpr int step_elems(int M) { return 2 * M * M + tri(M); }
// step tables are stored mode-major, one row of step_row(M) values (padded to 16 bytes in
// FP32 and 32 bytes in FP64) per (ring, mode)
__host__ __device__ constexpr int step_row(int M) { return (step_elems(M) + 3) & ~3; }
__host__ __device__ constexpr int coarse_elems(int M) { return M * M + tri(M); }

// Everything a sampling kernel needs about one request (plan tables, grid, seed, output,
// scratch); passed by value to single-request kernels and through device memory to batched
// ones.
struct SampleParams {
    const Segment* segs;
    const void* steps[2];
    const void* coarse[2];
    const void* beq;
    const void* tw;   // per-pass complex twiddle tables (see pass_radix)
    const void* pre;  // complex e^{2 pi i s / n_phi}, s < Nc
    const void* tw2;  // per-pass complex twiddles of the high-radix plan, MB = 4 (hr_off)
    const void* tw3;  // the same for MB = 3
    void* anc;        // anchor states [c][r][j][2M][n_slots]
    void* out;
    uint64_t seed;
    int n_samples, n_theta, n_phi, Nc, n_units, n_modes_pad, k0, H, na_max;
    int n_anchors[2];
    int pingpong;     // 1: two FFT buffers + right anchors on chip; 0: one buffer, in place
    int np;           // warp-specialised kernel: producer threads
    int lgNc;
    int fft_r4;       // warp-specialised kernel, FP32: 1 = radix-4 FFT passes, 0 = the high-radix plan
    // iso-latitude grid with ring-dependent longitudes (null: the full n_theta x n_phi grid):
    // ring k holds ring_n[k] points from phi0 = ring_h[k] pi, at ring_off[k] within a
    // realisation of ring_total points
    const int* ring_n;
    const double* ring_h;
    const long long* ring_off;
    long long ring_total;
};

// High-radix pass plan of the Nc = 2^L point inverse FFT with passes of at most 2^MB points:
// ceil(L / MB) Stockham passes whose radices 2^bits split L as evenly as possible, largest
// first (L = 10, MB = 4: 16, 8, 8).  Pass i runs with stride Ns = 2^hr_lgns(L, i); its
// twiddles e^{2 pi i a kk / (Ns RP)}, a in [1, RP), kk < Ns, sit at
// tw[hr_off(L, i) + (a - 1) Ns + kk] (pass 0 has none).  The warp-specialised kernel uses
// MB = 4 (table tw2), the in-place kernel MB = SMERF_INPLACE_MB (table tw3).
#ifndef SMERF_INPLACE_MB
#define SMERF_INPLACE_MB 3
#endif
__host__ __device__ constexpr int hr_passes(int L, int MB = 4) { return (L + MB - 1) / MB; }
__host__ __device__ constexpr int hr_bits(int L, int i, int MB = 4)
{
    return L / hr_passes(L, MB) + (i < L % hr_passes(L, MB) ? 1 : 0);
}
__host__ __device__ constexpr int hr_lgns(int L, int i, int MB = 4)
{
    int s = 0;
    for (int p = 0; p < i; ++p) s += hr_bits(L, p, MB);
    return s;
}
__host__ __device__ constexpr int hr_off(int L, int i, int MB = 4)
{
    int o = 0;
    for (int p = 1; p < i; ++p) o += ((1 << hr_bits(L, p, MB)) - 1) << hr_lgns(L, p, MB);
    return o;
}

// The batch's persistent launch: kQueueThreads threads per CTA, two CTAs per SM; a
// request runs with np = ceil32(units / upt) <= 256 producer threads (upt the smallest of 1, 2,
// 4, 8 that allows it), the rest FFT threads, and 4, 2, 2, 1 realisations per CTA for upt = 1,
// 2, 4, 8.  Its shape, shape = (p - 1) * kQueueBuilds + build, selects that build.
constexpr int kQueueThreads = 384;   // 320 x 3 and 512 x 2 per SM measured slower
constexpr int kQueueMinBlocks = 2;
constexpr int kQueueBuilds = 4;  // (upt, rmax): (1,4) (2,2) (4,2) (8,1)
__host__ __device__ constexpr int queue_upt(int b) { return 1 << b; }
__host__ __device__ constexpr int queue_rmax(int b) { return b == 0 ? 4 : b <= 2 ? 2 : 1; }
// the build of a request with n_units units (-1: more than 8 x 256 units)
inline int queue_build(int n_units)
{
    for (int b = 0; b < kQueueBuilds; ++b)
        if ((n_units + queue_upt(b) - 1) / queue_upt(b) <= 256) return b;
    return -1;
}

// units: the fewest slots whose 2p normals each fill whole Philox calls (4 normals per call).
// p = 1: 2 slots per call; p = 2: 1 slot per call; p = 3: 2 slots per 3 calls.  A unit holds
// unit_vals(p) state values and draws the normals of calls [unit_calls u, unit_calls (u + 1)).
__host__ __device__ constexpr int unit_slots(int M) { return M == 2 ? 1 : 2; }
__host__ __device__ constexpr int unit_vals(int M) { return 2 * M * unit_slots(M); }
__host__ __device__ constexpr int unit_calls(int M) { return unit_vals(M) / 4; }

// ----------------------------------------------------------------- Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11.
struct PhiloxKey { uint32_t k0, k1; };

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, PhiloxKey key)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        const uint64_t p0 = (uint64_t)M0 * c.x;  // one 32x32->64 multiply each
        const uint64_t p1 = (uint64_t)M1 * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
    }
    return c;
}

// ------------------------------------------------------------------ Box-Muller
// Normals (r cos t, r sin t) with r = sqrt(-2 ln u0), t = 2 pi u1, u = (x + 1/2) 2^-32.
// FP32: ln u0 from the hardware log2 except when 1 - u0 < 2^-10, where the log2 of a
// rounded u0 would lose the small radius; there -ln(1 - v) = v + v^2/2 + v^3/3 + O(v^4)
// with v = (~x + 1/2) 2^-32 exact.
__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, float& n0, float& n1)
{
    float r2;
    const uint32_t na = ~a;
    if (na < (1u << 22)) {
        const float v = fmaf((float)na, 0x1p-32f, 0x1p-33f);
        r2 = 2.0f * v * fmaf(v, fmaf(v, 0.33333334f, 0.5f), 1.0f);
    } else {
        const float u = fmaf((float)a, 0x1p-32f, 0x1p-33f);
        r2 = -1.3862944f * __log2f(u);  // -2 ln 2 * log2(u)
    }
    const float r = r2 * rsqrtf(r2);  // r2 > 0: u0 < 1 and v > 0
    const float t = fmaf((float)b, 0x1p-32f, 0x1p-33f) * 6.2831855f;
    float s, c;
    __sincosf(t, &s, &c);
    n0 = r * c;
    n1 = r * s;
}

__device__ __forceinline__ void box_muller(uint32_t a, uint32_t b, double& n0, double& n1)
{
    const double u0 = ((double)a + 0.5) * 0x1p-32;
    const double u1 = ((double)b + 0.5) * 0x1p-32;
    const double r = sqrt(-2.0 * log(u0));
    double s, c;
    sincospi(2.0 * u1, &s, &c);
    n0 = r * c;
    n1 = r * s;
}

// ------------------------------------------------------------------ complex helpers
template <class R> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <class R> using cplx = typename cplx_t<R>::type;

template <class C> __device__ __forceinline__ C cmk(decltype(C::x) a, decltype(C::x) b) { C c; c.x = a; c.y = b; return c; }
template <class C> __device__ __forceinline__ C cadd(C a, C b) { return cmk<C>(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return cmk<C>(a.x - b.x, a.y - b.y); }
template <class C> __device__ __forceinline__ C cmul(C a, C b) { return cmk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <class C> __device__ __forceinline__ C cconj(C a) { return cmk<C>(a.x, -a.y); }
template <class C> __device__ __forceinline__ C cmuli(C a) { return cmk<C>(-a.y, a.x); }  // i * a


}  // namespace smerf

namespace smerf {
// Every device or page-locked allocation the library makes goes through these wrappers, so that
// a test can make one of them fail as if memory were exhausted (smerf_debug_fail_alloc).
bool alloc_fail_now();  // smerf_api.cu
inline cudaError_t dev_malloc(void** p, size_t n)
{
    return alloc_fail_now() ? cudaErrorMemoryAllocation : cudaMalloc(p, n);
}
inline cudaError_t dev_malloc_async(void** p, size_t n, cudaStream_t st)
{
    return alloc_fail_now() ? cudaErrorMemoryAllocation : cudaMallocAsync(p, n, st);
}
inline cudaError_t dev_malloc_pool(void** p, size_t n, cudaMemPool_t pool, cudaStream_t st)
{
    return alloc_fail_now() ? cudaErrorMemoryAllocation : cudaMallocFromPoolAsync(p, n, pool, st);
}
inline cudaError_t host_malloc(void** p, size_t n)
{
    return alloc_fail_now() ? cudaErrorMemoryAllocation : cudaMallocHost(p, n);
}
}  // namespace smerf

// sampling entry points used by smerf_api.cu (the set-up's are in smerf_setup.h)
int smerf_launch_sample(const smerf_plan* plan, uint64_t seed, int n_samples, void* out,
                        void* scratch, cudaStream_t stream, cudaEvent_t ev0 = nullptr,
                        cudaEvent_t ev1 = nullptr);
size_t smerf_scratch_bytes(const smerf_plan* plan, int n_samples);
// batched launches (smerf_batch.cu): per precision pair XX in {ff, fd, dd, df}
//   smerf_fill_params_XX: the request's SampleParams and whether it can join a batched group
//   smerf_launch_group_XX: one anchor and one segment launch over a group's work items
#define SMERF_DECLARE_GROUP(XX)                                                                   \
    int smerf_fill_params_##XX(const smerf_plan* pl, uint64_t seed, int n, void* out, void* scratch, \
                               smerf::SampleParams* P, int* batchable, int* rmax);                 \
    int smerf_launch_group_##XX(const smerf_plan* rep, const smerf::SampleParams* d_descs,          \
                                const int4* anc_items, int n_anc, const int4* seg_items, int n_seg,  \
                                cudaStream_t st);
SMERF_DECLARE_GROUP(ff)
SMERF_DECLARE_GROUP(fd)
SMERF_DECLARE_GROUP(dd)
SMERF_DECLARE_GROUP(df)
// shared memory of the warp-specialised kernel for a request and realisations per CTA
#define SMERF_DECLARE_GROUP_CONFIG(XX) size_t smerf_ws_smem_##XX(const smerf_plan* pl, int rmax);
SMERF_DECLARE_GROUP_CONFIG(ff)
SMERF_DECLARE_GROUP_CONFIG(fd)
SMERF_DECLARE_GROUP_CONFIG(dd)
SMERF_DECLARE_GROUP_CONFIG(df)
// the persistent work of a batch for FP32 recursion (FP32 or FP64 tables): `ctas` CTAs pulling
// anchor items, then segment items, from a device queue in one launch (single), or an anchor
// launch over anc128 and a persistent launch over the segment items; ctl = head, status, anchor
// counters
#define SMERF_DECLARE_QUEUE(XX)                                                                          \
    int smerf_launch_queue_##XX(const smerf::SampleParams* d, const int4* items, int n_items, int n_anc,  \
                                const int4* anc128, int n_anc128, int* ctl, int n_req, int single,         \
                                int fail_waits, size_t smem, int ctas, cudaStream_t st);                   \
    int smerf_queue_ctas_##XX(size_t smem);
SMERF_DECLARE_QUEUE(ff)
SMERF_DECLARE_QUEUE(fd)

// launch-configuration candidates of a plan for the autotuner (per precision pair XX):
// writes up to max_n (upt, rmax, np, nf, minb) tuples of kLaunchInts, returns how many
#define SMERF_DECLARE_TUNE(XX) int smerf_tune_candidates_##XX(const smerf_plan* pl, int* cand, int max_n);
SMERF_DECLARE_TUNE(ff)
SMERF_DECLARE_TUNE(fd)
SMERF_DECLARE_TUNE(dd)
SMERF_DECLARE_TUNE(df)

// FP64 tables with FP32 recursion: the plan's two FP64 step tables (one per chain; the
// tables the segment kernels read) converted to FP32 by the threads of the call's anchor
// launch (smerf_sample_impl.cuh, anchor_stage_kernel).  The work is groups of eight elements,
// taken in rounds of one group per thread: rounds [0, rounds0) cover table 0, [rounds0,
// rounds) table 1; every anchor thread converts k_loop groups during its anchors, one every
// `every` anchors, and the rest after them.
constexpr int kStageParts = 2;
struct StageJob {
    const double* src[kStageParts];
    float* dst[kStageParts];
    unsigned long long n[kStageParts];  // elements
    unsigned rounds0, rounds;           // set by the launch (they depend on its thread count)
    int every, k_loop;                  // a round every `every` anchors, k_loop rounds in all
};
// the coarse and start tables (small: one row per anchor, one for the start ring) are staged
// by a short launch ahead of the anchor launch, which reads them in FP32
struct StageSmall {
    const double* src[3];
    float* dst[3];
    unsigned end[3];  // cumulative element counts of coarse[0], coarse[1], beq
};
// the staged call for p = 1, 2, 3 (smerf_sample_ff_pM.cu): plan `sh` reads the FP32 copies
// S.dst and J.dst
#define SMERF_DECLARE_STAGED(M)                                                                     \
    int smerf_launch_sample_staged_p##M(const smerf_plan* sh, const StageSmall& S, const StageJob& J,      \
                                        uint64_t seed, int n, void* out, void* scratch, cudaStream_t st,    \
                                        cudaEvent_t ev0, cudaEvent_t ev1);
SMERF_DECLARE_STAGED(1)
SMERF_DECLARE_STAGED(2)
SMERF_DECLARE_STAGED(3)

// dynamic shared-memory attribute bookkeeping (smerf_api.cu)
int smerf_smem_attr_done(const void* kern, int dev, size_t smem, bool record);
int smerf_launch_philox(uint64_t key64, uint32_t ring, int64_t ncalls, uint32_t* out, cudaStream_t s);
int smerf_launch_normals(uint64_t key64, uint32_t ring, int64_t n, int fp64, void* out, cudaStream_t s);
