// smerf_api.cu -- the C ABI of the GB300 sphere-GMRF sampler (declared in include/smerf.h).
// Validation, plan layout (chains, anchors, segments), scratch management and the
// noise test hooks.  No entry point aborts, exits or throws.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "smerf_internal.cuh"
#include "smerf_setup.h"

int smerf_launch_sample_ff(const smerf_plan*, uint64_t, int, void*, void*, cudaStream_t, cudaEvent_t, cudaEvent_t);
int smerf_launch_sample_fd(const smerf_plan*, uint64_t, int, void*, void*, cudaStream_t, cudaEvent_t, cudaEvent_t);
int smerf_launch_sample_dd(const smerf_plan*, uint64_t, int, void*, void*, cudaStream_t, cudaEvent_t, cudaEvent_t);
int smerf_launch_sample_df(const smerf_plan*, uint64_t, int, void*, void*, cudaStream_t, cudaEvent_t, cudaEvent_t);

using namespace smerf;

namespace {

void free_plan_memory(smerf_plan* pl)
{
    if (!pl) return;
    cudaFree(pl->beq);
    for (int c = 0; c < 2; ++c) {
        cudaFree(pl->steps[c]);
        cudaFree(pl->coarse[c]);
    }
    cudaFree(pl->tw);
    cudaFree(pl->pre);
    cudaFree(pl->tw2);
    cudaFree(pl->tw3);
    cudaFree(pl->segs_dev);
    free(pl->segs_host);
    cudaFree(pl->rings_n_dev);
    cudaFree(pl->rings_h_dev);
    cudaFree(pl->rings_off_dev);
    free(pl->theta_host);
    cudaFree(pl->theta_dev);
}

void free_rings(smerf_plan* pl)
{
    cudaFree(pl->rings_n_dev);
    cudaFree(pl->rings_h_dev);
    cudaFree(pl->rings_off_dev);
    pl->rings_n_dev = nullptr;
    pl->rings_h_dev = nullptr;
    pl->rings_off_dev = nullptr;
    pl->rings_total = 0;
}

// output values of one realisation
size_t plan_points(const smerf_plan* pl)
{
    return pl->rings_total ? (size_t)pl->rings_total : (size_t)pl->n_theta * pl->n_phi;
}

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

__global__ void philox_kernel(uint64_t key64, uint32_t ring, int64_t ncalls, uint32_t* out)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ncalls) return;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)j, ring, 0u, 0u), PhiloxKey{(uint32_t)key64, (uint32_t)(key64 >> 32)});
    out[4 * j + 0] = w.x;
    out[4 * j + 1] = w.y;
    out[4 * j + 2] = w.z;
    out[4 * j + 3] = w.w;
}

template <class Real>
__global__ void normals_kernel(uint64_t key64, uint32_t ring, int64_t n, Real* out)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (4 * j >= n) return;
    const uint4 w = philox4x32_10(make_uint4((uint32_t)j, ring, 0u, 0u), PhiloxKey{(uint32_t)key64, (uint32_t)(key64 >> 32)});
    Real v[4];
    box_muller(w.x, w.y, v[0], v[1]);
    box_muller(w.z, w.w, v[2], v[3]);
    for (int i = 0; i < 4 && 4 * j + i < n; ++i) out[4 * j + i] = v[i];
}

}  // namespace

// Largest dynamic shared memory already granted to each (kernel, device): the attribute is
// set once, so that later launches (e.g. under stream capture) make no attribute calls.
int smerf_smem_attr_done(const void* kern, int dev, size_t smem, bool record)
{
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, size_t> granted;
    std::lock_guard<std::mutex> lock(mu);
    size_t& g = granted[std::make_pair(kern, dev)];
    if (record) {
        if (smem > g) g = smem;
        return 1;
    }
    return smem <= g ? 1 : 0;
}

size_t smerf_scratch_bytes(const smerf_plan* pl, int n_samples)
{
    const int na = pl->chain[0].n_anchors > pl->chain[1].n_anchors ? pl->chain[0].n_anchors : pl->chain[1].n_anchors;
    const size_t rs = pl->recur64 ? 8 : 4;
    return (size_t)2 * n_samples * (na + 1) * 2 * pl->p * (size_t)(pl->n_phi / 2) * rs;
}

// ---- FP64 tables with FP32 recursion: the tables the float kernels read are staged once per
// call as FP32 (the kernels' own truncating conversion, so the field is bit-identical) instead
// of being converted by every realisation group's CTAs: the coarse and start tables by a short
// launch, the step tables by the anchor launch's threads beside their anchors.
namespace {
struct StageLayout {
    size_t steps[2], coarse[2], beq, total;  // element counts; total in bytes (256-aligned parts)
};

StageLayout stage_layout(const smerf_plan* pl)
{
    StageLayout L;
    const size_t mp = pl->n_modes_pad;
    size_t off = 0;
    auto add = [&](size_t elems) { off += ((elems * sizeof(float) + 255) / 256) * 256; return elems; };
    for (int c = 0; c < 2; ++c) L.steps[c] = add((size_t)(pl->chain[c].len + 1) * step_row(pl->p) * mp);
    for (int c = 0; c < 2; ++c) L.coarse[c] = add((size_t)(pl->chain[c].n_anchors + 1) * coarse_elems(pl->p) * mp);
    L.beq = add((size_t)tri(pl->p) * mp);
    L.total = off;
    return L;
}
}  // namespace

// whether a call stages its tables (FP64 tables, FP32 recursion, enough realisations to share them)
static bool use_stage(const smerf_plan* pl, int n) { return !pl->recur64 && pl->tab64 && n >= 4; }

size_t smerf_stage_bytes(const smerf_plan* pl, int n) { return use_stage(pl, n) ? stage_layout(pl).total : 0; }

// smerf_launch_sample with the tables staged in `stage` (smerf_stage_bytes bytes) when the call
// qualifies, else the plain launch
int smerf_launch_sample_staged(const smerf_plan* pl, uint64_t seed, int n, void* out, void* scratch, void* stage,
                               cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1)
{
    if (!use_stage(pl, n) || !stage) return smerf_launch_sample(pl, seed, n, out, scratch, st, ev0, ev1);
    const StageLayout L = stage_layout(pl);
    // the anchor threads index groups of eight elements and themselves in 32 bits (no index
    // reaches 2^31 while both counts are below 2^30), the short launch elements; larger tables
    // are converted by the segment kernels instead
    const unsigned long long groups = (L.steps[0] + 7) / 8 + (L.steps[1] + 7) / 8;
    const unsigned long long small = (unsigned long long)L.coarse[0] + L.coarse[1] + L.beq;
    const unsigned long long threads = 2ull * n * ((pl->n_phi / 2 / unit_slots(pl->p) + 127) / 128) * 128;
    if (groups >= (1ull << 30) || threads >= (1ull << 30) || small >= (1ull << 31))
        return smerf_launch_sample(pl, seed, n, out, scratch, st, ev0, ev1);
    smerf_plan sh = *pl;  // shallow copy: the same plan reading FP32 copies of its tables
    unsigned char* p = (unsigned char*)stage;
    auto take = [&](size_t elems) {
        float* d = (float*)p;
        p += ((elems * sizeof(float) + 255) / 256) * 256;
        return d;
    };
    StageJob job;
    for (int c = 0; c < 2; ++c) {
        job.src[c] = (const double*)pl->steps[c];
        job.dst[c] = take(L.steps[c]);
        job.n[c] = L.steps[c];
        sh.steps[c] = job.dst[c];
    }
    job.rounds0 = job.rounds = 0;  // set by the launch
    job.every = 1;
    job.k_loop = 0;
    StageSmall sm;
    const void* ssrc[3] = {pl->coarse[0], pl->coarse[1], pl->beq};
    const size_t sel[3] = {L.coarse[0], L.coarse[1], L.beq};
    unsigned end = 0;
    for (int q = 0; q < 3; ++q) {
        sm.src[q] = (const double*)ssrc[q];
        sm.dst[q] = take(sel[q]);
        end += (unsigned)sel[q];
        sm.end[q] = end;
    }
    sh.coarse[0] = sm.dst[0];
    sh.coarse[1] = sm.dst[1];
    sh.beq = sm.dst[2];
    sh.tab64 = false;
    switch (pl->p) {
        case 1: return smerf_launch_sample_staged_p1(&sh, sm, job, seed, n, out, scratch, st, ev0, ev1);
        case 2: return smerf_launch_sample_staged_p2(&sh, sm, job, seed, n, out, scratch, st, ev0, ev1);
        default: return smerf_launch_sample_staged_p3(&sh, sm, job, seed, n, out, scratch, st, ev0, ev1);
    }
}

int smerf_launch_sample(const smerf_plan* pl, uint64_t seed, int n, void* out, void* scratch, cudaStream_t st,
                        cudaEvent_t ev0, cudaEvent_t ev1)
{
    if (pl->recur64) return pl->tab64 ? smerf_launch_sample_dd(pl, seed, n, out, scratch, st, ev0, ev1)
                                      : smerf_launch_sample_df(pl, seed, n, out, scratch, st, ev0, ev1);
    return pl->tab64 ? smerf_launch_sample_fd(pl, seed, n, out, scratch, st, ev0, ev1)
                     : smerf_launch_sample_ff(pl, seed, n, out, scratch, st, ev0, ev1);
}

int smerf_launch_philox(uint64_t key64, uint32_t ring, int64_t ncalls, uint32_t* out, cudaStream_t s)
{
    if (ncalls <= 0) return SMERF_OK;
    philox_kernel<<<(unsigned)((ncalls + 255) / 256), 256, 0, s>>>(key64, ring, ncalls, out);
    return cudaGetLastError() == cudaSuccess ? SMERF_OK : SMERF_ECUDA;
}

int smerf_launch_normals(uint64_t key64, uint32_t ring, int64_t n, int fp64, void* out, cudaStream_t s)
{
    if (n <= 0) return SMERF_OK;
    const int64_t calls = (n + 3) / 4;
    if (fp64) normals_kernel<double><<<(unsigned)((calls + 255) / 256), 256, 0, s>>>(key64, ring, n, (double*)out);
    else normals_kernel<float><<<(unsigned)((calls + 255) / 256), 256, 0, s>>>(key64, ring, n, (float*)out);
    return cudaGetLastError() == cudaSuccess ? SMERF_OK : SMERF_ECUDA;
}

// ---- per-call scratch (anchor states, staged tables, host-path field) comes from a memory
// pool the library owns, one per device, that keeps its memory between calls: the default
// pool returns its memory at every synchronisation, after which the next call's allocation
// maps fresh memory on the stream.  smerf_scratch_trim returns what is not in use.
namespace {
std::mutex g_pool_mu;
std::map<int, cudaMemPool_t> g_pools;

cudaMemPool_t scratch_pool(int dev, bool create)
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) return it->second;
    if (!create) return nullptr;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t keep = UINT64_MAX;
    if (cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
        cudaMemPoolDestroy(pool);
        return nullptr;
    }
    g_pools[dev] = pool;
    return pool;
}

// stream-ordered scratch from the device's pool; under stream capture (a graph records the
// allocation as its own node) and if the pool cannot be made, the stream's default pool
cudaError_t scratch_alloc(void** p, size_t bytes, int dev, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return cudaGetLastError();
    cudaMemPool_t pool = cs == cudaStreamCaptureStatusNone ? scratch_pool(dev, true) : nullptr;
    return pool ? smerf::dev_malloc_pool(p, bytes, pool, st) : smerf::dev_malloc_async(p, bytes, st);
}
}  // namespace

// allocation-failure injection (smerf_debug_fail_alloc): -1 = off, k >= 0 = the allocation
// after k more succeeds fails
static std::atomic<long> g_alloc_countdown(-1);

bool smerf::alloc_fail_now()
{
    long v = g_alloc_countdown.load();
    while (v >= 0) {
        if (g_alloc_countdown.compare_exchange_weak(v, v - 1)) return v == 0;
    }
    return false;
}

extern "C" {

int smerf_debug_fail_alloc(int k)
{
    g_alloc_countdown.store(k < 0 ? -1 : (long)k);
    return SMERF_OK;
}

const char* smerf_status_string(int status)
{
    switch (status) {
        case SMERF_OK: return "ok";
        case SMERF_EINVAL: return "invalid argument";
        case SMERF_EILLCOND: return "kappa values too close (ill-conditioned partial fractions)";
        case SMERF_ENOMEM: return "out of memory";
        case SMERF_ECUDA: return "CUDA error";
        case SMERF_EUNSUPPORTED: return "unsupported configuration";
        case SMERF_ESCRATCH: return "request exceeds the fixed scratch of smerf_sample_noalloc";
        case SMERF_ETIMEOUT: return "a device wait ran out";
        default: return "unknown status";
    }
}

static int check_grid(int p, double A, int n_theta, int n_phi, unsigned flags, int anchor_spacing)
{
    if (p < 1 || p > 3) return SMERF_EINVAL;
    if (!(A > 0.0) || !isfinite(A)) return SMERF_EINVAL;
    if (n_theta < 2 || n_theta > 65536) return SMERF_EINVAL;
    if (n_phi < 2 || (n_phi & 1)) return SMERF_EINVAL;
    if ((flags & ~0xFu) != 0) return SMERF_EINVAL;
    if ((flags & SMERF_TABLES_FP64) && (flags & SMERF_TABLES_FP32)) return SMERF_EINVAL;
    if (anchor_spacing < 0) return SMERF_EINVAL;
    return SMERF_OK;
}

static int create_plan(const double* kappa, const double* kh_re, const double* kh_im, int complex_spec, int p,
                       double A, int n_theta, int n_phi, unsigned flags, int anchor_spacing, smerf_plan** out_plan,
                       cudaStream_t st = 0, bool sync = true, const double* theta = nullptr);

// ring colatitudes of an iso-latitude grid: finite, strictly increasing inside (0, pi) (any such
// set of rings: the Markov property along the colatitude holds on every iso-latitude grid, Sec. 2)
static int check_colatitudes(const double* theta, int n_theta)
{
    for (int k = 0; k < n_theta; ++k) {
        if (!isfinite(theta[k]) || !(theta[k] > 0.0) || !(theta[k] < SMERF_PI)) return SMERF_EINVAL;
        if (k > 0 && !(theta[k] > theta[k - 1])) return SMERF_EINVAL;
    }
    return SMERF_OK;
}

// smerf_plan_create_ex with the set-up ordered on `st` (sync: wait for it)
static int create_ex_on(const double* kappa, int p, double A, int n_theta, int n_phi, unsigned flags,
                        int anchor_spacing, smerf_plan** out_plan, cudaStream_t st, bool sync)
{
    if (!out_plan) return SMERF_EINVAL;
    *out_plan = nullptr;
    if (!kappa) return SMERF_EINVAL;
    int rc = check_grid(p, A, n_theta, n_phi, flags, anchor_spacing);
    if (rc != SMERF_OK) return rc;
    for (int i = 0; i < p; ++i)
        if (!(kappa[i] > 0.0) || !isfinite(kappa[i])) return SMERF_EINVAL;
    for (int i = 0; i < p; ++i)
        for (int j = i + 1; j < p; ++j) {
            const double a = kappa[i] * kappa[i], b = kappa[j] * kappa[j];
            if (fabs(a - b) < 1e-6 * fmax(a, b)) return SMERF_EILLCOND;
        }
    double kr[kMaxP + 1] = {0}, ki[kMaxP + 1] = {0};
    for (int i = 0; i < p && i <= kMaxP; ++i) kr[i] = kappa[i] * kappa[i];
    return create_plan(kappa, kr, ki, 0, p, A, n_theta, n_phi, flags, anchor_spacing, out_plan, st, sync);
}

int smerf_plan_create_ex(const double* kappa, int p, double A, int n_theta, int n_phi,
                         unsigned flags, int anchor_spacing, smerf_plan** out_plan)
{
    return create_ex_on(kappa, p, A, n_theta, n_phi, flags, anchor_spacing, out_plan, 0, true);
}

int smerf_plan_create_many(const smerf_plan_spec* specs, int n, smerf_plan** out_plans)
{
    if (n < 0 || (n > 0 && (!specs || !out_plans))) return SMERF_EINVAL;
    for (int i = 0; i < n; ++i) out_plans[i] = nullptr;
    if (n == 0) return SMERF_OK;
    // the set-ups go round-robin onto a few non-blocking streams and overlap on the GPU
    const int ns = n < 16 ? n : 16;
    std::vector<cudaStream_t> streams((size_t)ns, nullptr);
    int rc = SMERF_OK;
    for (int k = 0; k < ns && rc == SMERF_OK; ++k)
        if (cudaStreamCreateWithFlags(&streams[k], cudaStreamNonBlocking) != cudaSuccess) rc = SMERF_ECUDA;
    const auto t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < n && rc == SMERF_OK; ++i) {
        const smerf_plan_spec& q = specs[i];
        rc = create_ex_on(q.kappa, q.p, q.A, q.n_theta, q.n_phi, q.flags, q.anchor_spacing, &out_plans[i],
                          streams[i % ns], false);
    }
    for (int k = 0; k < ns; ++k) {
        if (!streams[k]) continue;
        if (cudaStreamSynchronize(streams[k]) != cudaSuccess && rc == SMERF_OK) rc = SMERF_ECUDA;
        cudaStreamDestroy(streams[k]);
    }
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    for (int i = 0; i < n; ++i) {
        if (!out_plans[i]) continue;
        if (rc != SMERF_OK) {
            smerf_plan_destroy(out_plans[i]);
            out_plans[i] = nullptr;
        } else {
            out_plans[i]->setup_ms = ms;
        }
    }
    return rc;
}

// smerf_plan_create_khat on the equiangular grid (theta = NULL) or at the given colatitudes
static int create_khat(const double* khat_re, const double* khat_im, int p, double A, int n_theta,
                       const double* theta, int n_phi, unsigned flags, int anchor_spacing, smerf_plan** out_plan)
{
    if (!out_plan) return SMERF_EINVAL;
    *out_plan = nullptr;
    if (!khat_re || !khat_im) return SMERF_EINVAL;
    int rc = check_grid(p, A, n_theta, n_phi, flags, anchor_spacing);
    if (rc != SMERF_OK) return rc;
    if (theta && check_colatitudes(theta, n_theta) != SMERF_OK) return SMERF_EINVAL;
    if (p > kMaxP) return SMERF_EUNSUPPORTED;
    int complex_spec = 0;
    for (int i = 0; i < p; ++i) {
        if (!isfinite(khat_re[i]) || !isfinite(khat_im[i])) return SMERF_EINVAL;
        if (khat_im[i] != 0.0) complex_spec = 1;
    }
    if (!complex_spec) {
        // real kappa-hat: the real construction with kappa_i = sqrt(kappa-hat_i)
        double kappa[kMaxP];
        for (int i = 0; i < p; ++i) {
            if (!(khat_re[i] > 0.0)) return SMERF_EINVAL;
            kappa[i] = sqrt(khat_re[i]);
        }
        return theta ? smerf_plan_create_theta(kappa, p, A, n_theta, theta, n_phi, flags, anchor_spacing, out_plan)
                     : smerf_plan_create_ex(kappa, p, A, n_theta, n_phi, flags, anchor_spacing, out_plan);
    }
    // complex kappa-hat: every non-real value directly followed by its conjugate, the real values
    // positive, so that C_l = A / prod_i (l(l+1) + kappa-hat_i) is real and positive for every l
    for (int i = 0; i < p; ++i) {
        if (khat_im[i] == 0.0) {
            if (!(khat_re[i] > 0.0)) return SMERF_EINVAL;
            continue;
        }
        if (i + 1 >= p || khat_re[i + 1] != khat_re[i] || khat_im[i + 1] != -khat_im[i]) return SMERF_EINVAL;
        ++i;
    }
    // distinct values (the partial fractions of Eq. (C_ell_efficient) divide by their differences)
    for (int i = 0; i < p; ++i)
        for (int j = i + 1; j < p; ++j) {
            const double d = hypot(khat_re[i] - khat_re[j], khat_im[i] - khat_im[j]);
            const double s = fmax(hypot(khat_re[i], khat_im[i]), hypot(khat_re[j], khat_im[j]));
            if (d < 1e-6 * s) return SMERF_EILLCOND;
        }
    return create_plan(nullptr, khat_re, khat_im, 1, p, A, n_theta, n_phi, flags, anchor_spacing, out_plan, 0, true,
                       theta);
}

int smerf_plan_create_khat(const double* khat_re, const double* khat_im, int p, double A, int n_theta, int n_phi,
                           unsigned flags, int anchor_spacing, smerf_plan** out_plan)
{
    return create_khat(khat_re, khat_im, p, A, n_theta, nullptr, n_phi, flags, anchor_spacing, out_plan);
}

int smerf_plan_create_khat_theta(const double* khat_re, const double* khat_im, int p, double A, int n_theta,
                                 const double* theta, int n_phi, unsigned flags, int anchor_spacing,
                                 smerf_plan** out_plan)
{
    if (!out_plan) return SMERF_EINVAL;
    *out_plan = nullptr;
    if (!theta) return SMERF_EINVAL;
    return create_khat(khat_re, khat_im, p, A, n_theta, theta, n_phi, flags, anchor_spacing, out_plan);
}

static int create_plan(const double* kappa, const double* kh_re, const double* kh_im, int complex_spec, int p,
                       double A, int n_theta, int n_phi, unsigned flags, int anchor_spacing, smerf_plan** out_plan,
                       cudaStream_t st, bool sync, const double* theta)
{
    if (p > kMaxP) return SMERF_EUNSUPPORTED;
    if (!is_pow2(n_phi) || n_phi < 8 || n_phi > 32768) return SMERF_EUNSUPPORTED;
    // p = 3 runs on the warp-specialised kernels, whose ring buffers and right-anchor states must
    // fit in one SM's shared memory: rings up to 4096 complex points in FP32, 2048 in FP64
    if (p == 3 && n_phi > ((flags & SMERF_RECUR_FP64) ? 4096 : 8192)) return SMERF_EUNSUPPORTED;

    smerf_plan* pl = new (std::nothrow) smerf_plan;
    if (!pl) return SMERF_ENOMEM;
    memset(pl, 0, sizeof(*pl));
    pl->p = p;
    for (int i = 0; i < p; ++i) {
        if (kappa) pl->kappa[i] = kappa[i];
        pl->khat_re[i] = kh_re[i];
        pl->khat_im[i] = kh_im[i];
    }
    pl->complex_spec = complex_spec;
    pl->A = A;
    pl->n_theta = n_theta;
    pl->n_phi = n_phi;
    pl->n_slots = n_phi / 2;
    pl->n_modes = n_phi / 2 + 1;
    pl->n_modes_pad = ((pl->n_modes + 31) / 32) * 32;
    pl->k0 = smerf_start_ring(theta, n_theta);
    pl->flags = flags;
    pl->recur64 = (flags & SMERF_RECUR_FP64) != 0;
    pl->tab64 = (flags & SMERF_TABLES_FP64) ? true : ((flags & SMERF_TABLES_FP32) ? false : pl->recur64);
    pl->packed = p == 1 && !pl->recur64 && !pl->tab64 && (n_phi == 16384 || n_phi == 32768);
    int H = anchor_spacing == 0 ? kDefaultAnchor : anchor_spacing;
    if ((flags & SMERF_ORDER_PAPER) || H >= n_theta) H = 0;
    pl->H = H;
    pl->chain[0].len = pl->k0;
    pl->chain[1].len = n_theta - 1 - pl->k0;
    for (int c = 0; c < 2; ++c) pl->chain[c].n_anchors = H > 0 ? pl->chain[c].len / H : 0;
    cudaGetDevice(&pl->dev);

    std::vector<Segment> segs;
    for (int c = 0; c < 2; ++c) {
        const int len = pl->chain[c].len;
        const int nseg = H > 0 ? pl->chain[c].n_anchors + 1 : 1;
        for (int j = 0; j < nseg; ++j) {
            Segment s;
            s.chain = c;
            s.p0 = H > 0 ? j * H : 0;
            const bool right = H > 0 && s.p0 + H <= len;
            s.p1 = right ? s.p0 + H : len + 1;
            s.left = j;
            s.right = right ? j + 1 : -1;
            if (c == 1 && s.p0 == 0 && s.p1 == 1) continue;  // nothing to write: k0 belongs to the north
            segs.push_back(s);
        }
    }
    pl->n_segments = (int)segs.size();
    pl->segs_host = (Segment*)malloc(sizeof(Segment) * segs.size());
    if (!pl->segs_host) { delete pl; return SMERF_ENOMEM; }
    memcpy(pl->segs_host, segs.data(), sizeof(Segment) * segs.size());
    int rc = SMERF_OK;
    if (smerf::dev_malloc((void**)&pl->segs_dev, sizeof(Segment) * segs.size()) != cudaSuccess) rc = SMERF_ENOMEM;
    else if (cudaMemcpy(pl->segs_dev, segs.data(), sizeof(Segment) * segs.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = SMERF_ECUDA;
    if (rc == SMERF_OK && theta) {
        // the grid's own ring colatitudes; on the device followed by those of the mirrored grid,
        // pi - theta_{n_theta-1-j}, whose northern chain is the southern chain of a grid that is
        // not symmetric about the equator (the set-up computes its steps there)
        const size_t tb = sizeof(double) * (size_t)n_theta;
        pl->theta_host = (double*)malloc(tb);
        std::vector<double> both(2 * (size_t)n_theta);
        for (int j = 0; j < n_theta; ++j) {
            both[j] = theta[j];
            both[n_theta + j] = SMERF_PI - theta[n_theta - 1 - j];
        }
        if (!pl->theta_host || smerf::dev_malloc((void**)&pl->theta_dev, 2 * tb) != cudaSuccess) rc = SMERF_ENOMEM;
        else {
            memcpy(pl->theta_host, theta, tb);
            if (cudaMemcpy(pl->theta_dev, both.data(), 2 * tb, cudaMemcpyHostToDevice) != cudaSuccess) rc = SMERF_ECUDA;
        }
    }
    if (rc == SMERF_OK) rc = smerf_setup_tables(pl, st, sync);
    if (rc != SMERF_OK) {
        free_plan_memory(pl);
        delete pl;
        return rc;
    }
    *out_plan = pl;
    return SMERF_OK;
}

int smerf_plan_create_theta(const double* kappa, int p, double A, int n_theta, const double* theta, int n_phi,
                            unsigned flags, int anchor_spacing, smerf_plan** out_plan)
{
    if (!out_plan) return SMERF_EINVAL;
    *out_plan = nullptr;
    if (!kappa || !theta) return SMERF_EINVAL;
    int rc = check_grid(p, A, n_theta, n_phi, flags, anchor_spacing);
    if (rc != SMERF_OK) return rc;
    if (check_colatitudes(theta, n_theta) != SMERF_OK) return SMERF_EINVAL;
    for (int i = 0; i < p; ++i)
        if (!(kappa[i] > 0.0) || !isfinite(kappa[i])) return SMERF_EINVAL;
    for (int i = 0; i < p; ++i)
        for (int j = i + 1; j < p; ++j) {
            const double a = kappa[i] * kappa[i], b = kappa[j] * kappa[j];
            if (fabs(a - b) < 1e-6 * fmax(a, b)) return SMERF_EILLCOND;
        }
    double kr[kMaxP + 1] = {0}, ki[kMaxP + 1] = {0};
    for (int i = 0; i < p && i <= kMaxP; ++i) kr[i] = kappa[i] * kappa[i];
    return create_plan(kappa, kr, ki, 0, p, A, n_theta, n_phi, flags, anchor_spacing, out_plan, 0, true, theta);
}

int smerf_plan_create(const double* kappa, int p, double A, int n_theta, int n_phi, unsigned flags,
                      smerf_plan** out_plan)
{
    return smerf_plan_create_ex(kappa, p, A, n_theta, n_phi, flags, 0, out_plan);
}

int smerf_plan_destroy(smerf_plan* plan)
{
    if (!plan) return SMERF_OK;
    free_plan_memory(plan);
    delete plan;
    return SMERF_OK;
}

int smerf_sample(const smerf_plan* plan, uint64_t seed, int n_samples, void* out, void* stream)
{
    return smerf_sample_timed(plan, seed, n_samples, out, stream, nullptr, nullptr);
}

int smerf_sample_timed(const smerf_plan* plan, uint64_t seed, int n_samples, void* out, void* stream,
                       void* event_before_segments, void* event_after_segments)
{
    if (!plan || n_samples < 0 || n_samples > 65535) return SMERF_EINVAL;
    if (n_samples == 0) return SMERF_OK;
    if (!out || ((uintptr_t)out & 15u)) return SMERF_EINVAL;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != plan->dev) return SMERF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    void* scratch = nullptr;
    const size_t sb = (smerf_scratch_bytes(plan, n_samples) + 255) / 256 * 256;
    const size_t tb = smerf_stage_bytes(plan, n_samples);
    cudaError_t e = scratch_alloc(&scratch, sb + tb, dev, st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? SMERF_ENOMEM : SMERF_ECUDA;
    const int rc = smerf_launch_sample_staged(plan, seed, n_samples, out, scratch,
                                              tb ? (void*)((unsigned char*)scratch + sb) : nullptr, st,
                                              (cudaEvent_t)event_before_segments, (cudaEvent_t)event_after_segments);
    cudaFreeAsync(scratch, st);
    return rc;
}

int smerf_last_device_status(void* stream)
{
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return SMERF_ECUDA;
    }
    return SMERF_OK;
}

int smerf_scratch_trim(void)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SMERF_ECUDA;
    cudaMemPool_t pool = scratch_pool(dev, false);
    if (pool && cudaMemPoolTrimTo(pool, 0) != cudaSuccess) return SMERF_ECUDA;
    return SMERF_OK;
}

int smerf_sample_launches(const smerf_plan* plan, int n_samples)
{
    if (!plan || n_samples < 0) return SMERF_EINVAL;
    if (n_samples == 0) return 0;
    // anchor and segment launches, and ahead of them the short conversion of the coarse and
    // start tables when the call stages FP64 tables (the anchor launch converts the step tables)
    return use_stage(plan, n_samples) ? 3 : 2;
}

int smerf_sample_host(const smerf_plan* plan, uint64_t seed, int n_samples, void* host_out, void* stream)
{
    if (!plan || n_samples < 0 || (n_samples > 0 && !host_out)) return SMERF_EINVAL;
    if (n_samples == 0) return SMERF_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // Page-locked host memory the GPU can address: the last FFT pass streams the field into it
    // directly over the CPU-GPU link (no device copy of the output, no separate transfer).
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, host_out) == cudaSuccess && at.type == cudaMemoryTypeHost &&
        at.devicePointer && !((uintptr_t)at.devicePointer & 15u)) {
        int rc = smerf_sample(plan, seed, n_samples, at.devicePointer, stream);
        if (cudaStreamSynchronize(st) != cudaSuccess && rc == SMERF_OK) rc = SMERF_ECUDA;
        return rc;
    }
    cudaGetLastError();  // an unregistered pointer is not an error here
    const size_t bytes = (size_t)n_samples * plan_points(plan) * (plan->recur64 ? 8 : 4);
    void* dout = nullptr;
    cudaError_t e = scratch_alloc(&dout, bytes, plan->dev, st);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? SMERF_ENOMEM : SMERF_ECUDA;
    int rc = smerf_sample(plan, seed, n_samples, dout, stream);
    if (rc == SMERF_OK && cudaMemcpyAsync(host_out, dout, bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = SMERF_ECUDA;
    cudaFreeAsync(dout, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == SMERF_OK) rc = SMERF_ECUDA;
    return rc;
}

int smerf_plan_info(const smerf_plan* plan, smerf_plan_info_t* info)
{
    if (!plan || !info) return SMERF_EINVAL;
    memset(info, 0, sizeof(*info));
    info->p = plan->p;
    info->n_theta = plan->n_theta;
    info->n_phi = plan->n_phi;
    info->n_modes = plan->n_modes;
    info->start_ring = plan->k0;
    for (int c = 0; c < 2; ++c) {
        info->chain_len[c] = plan->chain[c].len;
        info->n_anchors[c] = plan->chain[c].n_anchors;
    }
    info->anchor_spacing = plan->H;
    info->n_segments = plan->n_segments;
    info->flags = plan->flags;
    info->table_bytes = plan->table_bytes;
    info->step_table_bytes = plan->step_table_bytes;
    info->scratch_bytes_per_sample = smerf_scratch_bytes(plan, 1);
    info->setup_ms = plan->setup_ms;
    info->points_per_sample = plan_points(plan);
    return SMERF_OK;
}

static int tune_candidates(const smerf_plan* plan, int* cand, int max_n);
constexpr int kMaxCand = 128;  // launch candidates a plan can have (the tuner's buffers)

int smerf_plan_set_rings(smerf_plan* plan, const int* n_phi_ring, const double* phi0_ring)
{
    if (!plan) return SMERF_EINVAL;
    if (!n_phi_ring) {
        free_rings(plan);
        return SMERF_OK;
    }
    std::vector<int> n(plan->n_theta);
    std::vector<double> h(plan->n_theta);
    std::vector<long long> off(plan->n_theta);
    long long total = 0;
    for (int k = 0; k < plan->n_theta; ++k) {
        const int nk = n_phi_ring[k];
        const double p0 = phi0_ring ? phi0_ring[k] : 0.0;
        if ((nk & 1) || nk < 4 || nk > plan->n_phi || !isfinite(p0)) return SMERF_EINVAL;
        n[k] = nk;
        h[k] = fmod(p0 / SMERF_PI, 2.0);
        off[k] = total;
        total += nk;
    }
    int cand[smerf::kLaunchInts * kMaxCand];
    if (tune_candidates(plan, cand, kMaxCand) == 0) return SMERF_EUNSUPPORTED;  // not a warp-specialised plan
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != plan->dev) return SMERF_EINVAL;
    free_rings(plan);
    int rc = SMERF_OK;
    if (smerf::dev_malloc((void**)&plan->rings_n_dev, sizeof(int) * n.size()) != cudaSuccess ||
        smerf::dev_malloc((void**)&plan->rings_h_dev, sizeof(double) * h.size()) != cudaSuccess ||
        smerf::dev_malloc((void**)&plan->rings_off_dev, sizeof(long long) * off.size()) != cudaSuccess)
        rc = SMERF_ENOMEM;
    if (rc == SMERF_OK &&
        (cudaMemcpy(plan->rings_n_dev, n.data(), sizeof(int) * n.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(plan->rings_h_dev, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
         cudaMemcpy(plan->rings_off_dev, off.data(), sizeof(long long) * off.size(), cudaMemcpyHostToDevice) != cudaSuccess))
        rc = SMERF_ECUDA;
    if (rc != SMERF_OK) {
        free_rings(plan);
        return rc;
    }
    plan->rings_total = total;
    return SMERF_OK;
}

int smerf_plan_copy_tables(const smerf_plan* plan, int which, int chain, int pos, double* host_out)
{
    if (!plan || !host_out || chain < 0 || chain > 1) return SMERF_EINVAL;
    const int M = plan->p;
    const size_t mp = plan->n_modes_pad;
    const size_t es = plan->tab64 ? 8 : 4;
    const unsigned char* base;
    int rows;
    bool mode_major = false;
    if (which == 0) {
        base = (const unsigned char*)plan->beq;
        rows = tri(M);
    } else if (which == 1) {
        if (pos < 1 || pos > plan->chain[chain].len) return SMERF_EINVAL;
        rows = step_elems(M);
        mode_major = !plan->packed;
        base = (const unsigned char*)plan->steps[chain] + (size_t)pos * (plan->packed ? rows : step_row(M)) * mp * es;
    } else if (which == 2) {
        if (pos < 1 || pos > plan->chain[chain].n_anchors) return SMERF_EINVAL;
        rows = coarse_elems(M);
        base = (const unsigned char*)plan->coarse[chain] + (size_t)pos * rows * mp * es;
    } else {
        return SMERF_EINVAL;
    }
    std::vector<unsigned char> tmp((size_t)(mode_major ? step_row(M) : rows) * mp * es);
    if (cudaMemcpy(tmp.data(), base, tmp.size(), cudaMemcpyDeviceToHost) != cudaSuccess) return SMERF_ECUDA;
    for (int r = 0; r < rows; ++r)
        for (int m = 0; m < plan->n_modes; ++m) {
            const size_t i = mode_major ? (size_t)m * step_row(M) + r : (size_t)r * mp + m;
            host_out[(size_t)r * plan->n_modes + m] = plan->tab64 ? ((const double*)tmp.data())[i]
                                                                  : (double)((const float*)tmp.data())[i];
        }
    return SMERF_OK;
}

static int tune_candidates(const smerf_plan* plan, int* cand, int max_n)
{
    return plan->recur64 ? (plan->tab64 ? smerf_tune_candidates_dd(plan, cand, max_n) : smerf_tune_candidates_df(plan, cand, max_n))
                         : (plan->tab64 ? smerf_tune_candidates_fd(plan, cand, max_n) : smerf_tune_candidates_ff(plan, cand, max_n));
}

int smerf_plan_launch_candidates(const smerf_plan* plan, int* cand, int max_n)
{
    if (!plan || max_n < 0 || (max_n > 0 && !cand)) return SMERF_EINVAL;
    int tmp[smerf::kLaunchInts * kMaxCand];
    const int n = tune_candidates(plan, tmp, kMaxCand);
    for (int i = 0; i < n && i < max_n; ++i)
        for (int k = 0; k < smerf::kLaunchInts; ++k) cand[smerf::kLaunchInts * i + k] = tmp[smerf::kLaunchInts * i + k];
    return n;
}

// a plan's fixed launch configuration from kLaunchInts integers (a candidate)
static void set_tune(smerf_plan* plan, const int* c)
{
    plan->tune.valid = 1;
    plan->tune.upt = c[0];
    plan->tune.rmax = c[1];
    plan->tune.np = c[2];
    plan->tune.nf = c[3];
    plan->tune.minb = c[4];
    plan->tune.radix = c[5];
}

int smerf_plan_set_launch(smerf_plan* plan, const int* config)
{
    if (!plan) return SMERF_EINVAL;
    if (!config) {
        plan->tune.valid = 0;
        return SMERF_OK;
    }
    int cand[smerf::kLaunchInts * kMaxCand];
    const int n = tune_candidates(plan, cand, kMaxCand);
    for (int i = 0; i < n; ++i) {
        const int* c = cand + smerf::kLaunchInts * i;
        bool same = true;
        for (int k = 0; k < smerf::kLaunchInts; ++k) same = same && c[k] == config[k];
        if (same) {
            set_tune(plan, c);
            plan->tune.ms = 0.0f;
            return SMERF_OK;
        }
    }
    return SMERF_EINVAL;
}

int smerf_plan_autotune(smerf_plan* plan, int n_samples, void* stream, int* chosen)
{
    if (!plan || n_samples < 1 || n_samples > 65535) return SMERF_EINVAL;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != plan->dev) return SMERF_EINVAL;
    int cand[smerf::kLaunchInts * kMaxCand];
    const int nc = tune_candidates(plan, cand, kMaxCand);
    plan->tune.valid = 0;
    if (nc == 0) {
        if (chosen)
            for (int k = 0; k < smerf::kLaunchInts; ++k) chosen[k] = 0;
        return SMERF_OK;  // no warp-specialised configuration: the built-in choice stays
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t ob = (size_t)n_samples * plan_points(plan) * (plan->recur64 ? 8 : 4);
    void* out = nullptr;
    void* scratch = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = SMERF_OK;
    const size_t sb = (smerf_scratch_bytes(plan, n_samples) + 255) / 256 * 256;
    const size_t tb = smerf_stage_bytes(plan, n_samples);
    if (smerf::dev_malloc((void**)&out, ob) != cudaSuccess || smerf::dev_malloc((void**)&scratch, sb + tb) != cudaSuccess)
        rc = SMERF_ENOMEM;
    if (rc == SMERF_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = SMERF_ECUDA;
    float best = 1e30f;
    int bi = -1;
    for (int i = 0; rc == SMERF_OK && i < nc; ++i) {
        set_tune(plan, cand + smerf::kLaunchInts * i);
        float tot = 0.0f;
        for (int it = 0; rc == SMERF_OK && it < 4; ++it) {
            rc = smerf_launch_sample_staged(plan, 1 + it, n_samples, out, scratch,
                                            tb ? (void*)((unsigned char*)scratch + sb) : nullptr, st, e0, e1);
            if (rc == SMERF_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = SMERF_ECUDA;
            float ms = 0.0f;
            if (rc == SMERF_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = SMERF_ECUDA;
            if (it > 0) tot += ms;  // first launch is a warm-up
        }
        if (rc == SMERF_OK && tot < best) {
            best = tot;
            bi = i;
        }
    }
    plan->tune.valid = 0;
    if (rc == SMERF_OK && bi >= 0) {
        const int* cb = cand + smerf::kLaunchInts * bi;
        set_tune(plan, cb);
        plan->tune.ms = best / 3.0f;
        if (chosen)
            for (int k = 0; k < smerf::kLaunchInts; ++k) chosen[k] = cb[k];
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    cudaFree(scratch);
    return rc;
}

int smerf_plan_autotune_anchor(smerf_plan* plan, int n_samples, const int* candidates, int n_cand, void* stream,
                               int* chosen)
{
    if (chosen) *chosen = 0;
    if (!plan || n_samples < 1 || n_samples > 65535 || n_cand < 1 || n_cand > 16 || !candidates) return SMERF_EINVAL;
    for (int i = 0; i < n_cand; ++i)
        if (candidates[i] < 1) return SMERF_EINVAL;
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != plan->dev) return SMERF_EINVAL;
    if (plan->flags & SMERF_ORDER_PAPER) return SMERF_OK;  // Alg. 2's order: no anchors to space
    cudaStream_t st = (cudaStream_t)stream;
    const size_t ob = (size_t)n_samples * plan->n_theta * plan->n_phi * (plan->recur64 ? 8 : 4);
    void* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = SMERF_OK;
    if (smerf::dev_malloc(&out, ob) != cudaSuccess) rc = SMERF_ENOMEM;
    if (rc == SMERF_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) rc = SMERF_ECUDA;
    smerf_plan* best = nullptr;
    float best_ms = 1e30f;
    for (int i = 0; rc == SMERF_OK && i < n_cand; ++i) {
        smerf_plan* cp = nullptr;
        rc = create_plan(plan->p > 0 ? plan->kappa : nullptr, plan->khat_re, plan->khat_im, plan->complex_spec, plan->p,
                         plan->A, plan->n_theta, plan->n_phi, plan->flags, candidates[i], &cp, 0, true, plan->theta_host);
        if (rc != SMERF_OK) break;
        cp->tune = plan->tune;  // the plan's launch configuration, if it fixed one
        const size_t sb = (smerf_scratch_bytes(cp, n_samples) + 255) / 256 * 256;
        const size_t tb = smerf_stage_bytes(cp, n_samples);
        void* scratch = nullptr;
        if (smerf::dev_malloc(&scratch, sb + tb) != cudaSuccess) rc = SMERF_ENOMEM;
        float tot = 0.0f;
        for (int it = 0; rc == SMERF_OK && it < 4; ++it) {
            if (cudaEventRecord(e0, st) != cudaSuccess) rc = SMERF_ECUDA;
            if (rc == SMERF_OK)
                rc = smerf_launch_sample_staged(cp, 1 + it, n_samples, out, scratch,
                                                tb ? (void*)((unsigned char*)scratch + sb) : nullptr, st, nullptr, nullptr);
            if (rc == SMERF_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
                rc = SMERF_ECUDA;
            float ms = 0.0f;
            if (rc == SMERF_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = SMERF_ECUDA;
            if (it > 0) tot += ms;  // the first call is a warm-up
        }
        cudaFree(scratch);
        if (rc == SMERF_OK && tot < best_ms) {
            best_ms = tot;
            std::swap(best, cp);
        }
        if (cp) smerf_plan_destroy(cp);
    }
    if (rc == SMERF_OK && best) {
        // the caller's handle takes the fastest plan's tables (keeping its ring layout); its old
        // tables go with `best`
        std::swap(*plan, *best);
        std::swap(plan->rings_n_dev, best->rings_n_dev);
        std::swap(plan->rings_h_dev, best->rings_h_dev);
        std::swap(plan->rings_off_dev, best->rings_off_dev);
        std::swap(plan->rings_total, best->rings_total);
        if (chosen) *chosen = plan->H;
    }
    if (best) smerf_plan_destroy(best);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
    return rc;
}

int smerf_philox_uint32(uint64_t key64, uint32_t ring, int64_t ncalls, uint32_t* out, void* stream)
{
    if (ncalls < 0 || (ncalls > 0 && !out)) return SMERF_EINVAL;
    return smerf_launch_philox(key64, ring, ncalls, out, (cudaStream_t)stream);
}

int smerf_ring_normals(uint64_t key64, uint32_t ring, int64_t n, int fp64, void* out, void* stream)
{
    if (n < 0 || (n > 0 && !out)) return SMERF_EINVAL;
    return smerf_launch_normals(key64, ring, n, fp64, out, (cudaStream_t)stream);
}

}  // extern "C"
