/*
 * smerf.h -- C ABI of the GB300 sampler for isotropic Gaussian Markov random fields on
 * the sphere (Creasey & Lang, "Fast generation of isotropic Gaussian random fields on the
 * sphere", arXiv 1709.10314).
 *
 * Field model.  Angular power spectrum C_l = A / prod_{i<p} (l(l+1) + kappa_i^2)
 * (Eq. (Cl) with kappa-hat_i = kappa_i^2, times an amplitude A).  The field T on an
 * equiangular grid of n_theta rings theta_k = pi (k + 1/2) / n_theta (k = 0 north) and
 * n_phi longitudes phi_j = 2 pi j / n_phi is the sum of azimuthal modes
 * g_m, m = 0..n_phi/2 (Sec. 2), each a Gaussian Markov process in z = cos(theta) whose
 * p-dimensional state (the U-basis "derivatives", Eq. (Jmatrix_more_efficient)) is
 * sampled ring by ring outward from the equator (Eqs. (state_space), (state_initial),
 * Alg. 2) and synthesised per ring by a real inverse DFT with prefactor 1:
 *     T(theta_k, phi_j) = g_0 + 2 sum_{0<m<n_phi/2} Re(g_m e^{i m phi_j}) + Re(g_{n_phi/2}) (-1)^j.
 * Other iso-latitude grids: rings at given colatitudes (smerf_plan_create_theta,
 * smerf_plan_create_khat_theta; HEALPix rings, latitude bands) and ring-dependent longitudes
 * (smerf_plan_set_rings).
 *
 * Conventions shared by every entry point
 *  - All calls return an int status (SMERF_OK or a negative SMERF_E* code); none aborts,
 *    exits or throws.  Asynchronous calls report launch errors only; kernel faults surface
 *    at the caller's next synchronisation.
 *  - Device pointers are plain CUDA device addresses of the current device; `stream` is a
 *    cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Output layout: out[r][k][j], r = realisation, k = ring (north to south), j = longitude,
 *    row-major and dense; float, or double for plans made with SMERF_RECUR_FP64.
 *  - Realisation r of a call draws Philox4x32-10 noise under the 64-bit key seed + r;
 *    call c of ring k uses counter (c, k, 0, 0) (Salmon et al., SC'11).
 */
#ifndef SMERF_H
#define SMERF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct smerf_plan smerf_plan;

/* status codes */
#define SMERF_OK 0
#define SMERF_EINVAL (-1)      /* bad argument (p, kappa, sizes, pointers, flags)              */
#define SMERF_EILLCOND (-2)    /* kappa_i^2 closer than 1e-6 relative: partial fractions cancel */
#define SMERF_ENOMEM (-3)      /* device or host allocation failed                              */
#define SMERF_ECUDA (-4)       /* a CUDA runtime call or kernel launch failed                    */
#define SMERF_EUNSUPPORTED (-5) /* valid but not built (e.g. n_phi not a power of two)          */
#define SMERF_ESCRATCH (-6)    /* smerf_sample_noalloc: request exceeds its fixed 16 MiB scratch */
#define SMERF_ETIMEOUT (-7)    /* a device wait ran out (the persistent batch launch's wait for
                                  a request's anchors: smerf_batch_status)                      */

/* plan flags */
#define SMERF_RECUR_FP64 0x1u    /* recursion, FFT and output in FP64 (default FP32, float out)   */
#define SMERF_TABLES_FP64 0x2u   /* store the step tables in FP64 (default: recursion precision)  */
#define SMERF_TABLES_FP32 0x4u   /* store the step tables in FP32 (default: recursion precision)  */
#define SMERF_ORDER_PAPER 0x8u   /* no anchor rings: every ring conditions on its inner neighbour
                                    only, exactly Alg. 2's order (less parallelism)              */

/*
 * smerf_plan_create_ex -- build the conditional-covariance tables for one grid and spectrum
 * (Alg. 1 and its equator-symmetric layout, Sec. 4; Sec. 3 "efficient covariance
 * computation").  Synchronous: returns after the FP64 set-up kernels finished.
 *
 *   kappa[p]       p distinct values kappa_i > 0 (host pointer, read during the call)
 *   p              number of spectrum factors, 1 <= p <= 3 (state dimension p per real chain;
 *                  p = 3 is built for n_phi <= 8192, or <= 4096 with SMERF_RECUR_FP64)
 *   A              amplitude > 0
 *   n_theta        rings, 2 <= n_theta <= 65536
 *   n_phi          longitudes, a power of two, 8 <= n_phi <= 32768
 *   flags          SMERF_* plan flags
 *   anchor_spacing H: every H-th ring of each chain is sampled first (an "anchor"); the
 *                  rings between two anchors are then sampled conditionally on both ends,
 *                  independently of other segments.  0 selects the default (16), and any
 *                  H >= n_theta (or SMERF_ORDER_PAPER) means no anchors.  The anchor order
 *                  changes the map from noise to field, not the field's law.
 *   out_plan       receives the plan (host pointer to a pointer)
 *
 * The plan owns its device tables; it is immutable after creation and may be used by
 * concurrent smerf_sample calls on different streams.  Errors: SMERF_EINVAL,
 * SMERF_EILLCOND, SMERF_ENOMEM, SMERF_ECUDA, SMERF_EUNSUPPORTED; *out_plan is NULL then.
 */
int smerf_plan_create_ex(const double* kappa, int p, double A, int n_theta, int n_phi,
                         unsigned flags, int anchor_spacing, smerf_plan** out_plan);

/*
 * smerf_plan_create_khat -- smerf_plan_create_ex with the spectrum given by kappa-hat_i
 * directly (Eq. (Cl): C_l = A / prod_i (l(l+1) + kappa-hat_i)), which may be complex as in the
 * paper's Sec. 5 example C_l = (10 + l^2 (l+1)^2)^-1, kappa-hat = +-i sqrt(10).
 *   khat_re, khat_im  host arrays of p doubles: real and imaginary parts of kappa-hat_i.
 *                     All real and > 0: the same plan as smerf_plan_create_ex with
 *                     kappa_i = sqrt(kappa-hat_i).  Otherwise every non-real value is directly
 *                     followed by its conjugate (a + ib, a - ib), b != 0, and the real values
 *                     are > 0 (p = 2: one pair; p = 3: one pair and one real value, either
 *                     order), so that C_l > 0 at every l.
 * The set-up runs the same construction in complex arithmetic (l_i, 2F1, the solution
 * matrices, the partial-fraction weights and Gamma factors complex); the tables are real.
 * Other arguments, ownership and errors as for smerf_plan_create_ex (SMERF_EINVAL for other
 * complex patterns, SMERF_EILLCOND when two kappa-hat_i lie closer than 1e-6 of the larger).
 */
int smerf_plan_create_khat(const double* khat_re, const double* khat_im, int p, double A, int n_theta, int n_phi,
                           unsigned flags, int anchor_spacing, smerf_plan** out_plan);

/*
 * smerf_plan_create_theta -- smerf_plan_create_ex on an iso-latitude grid whose rings sit at
 * the given colatitudes instead of the equiangular theta_k = pi (k + 1/2) / n_theta (the paper's
 * Sec. 1 remark: the method needs only rings of constant latitude; e.g. HEALPix, whose ring
 * point counts and offsets smerf_plan_set_rings then sets).
 *   theta[n_theta]  host array (read during the call): ring colatitudes in radians, strictly
 *                   increasing inside (0, pi).  They need not cover the sphere nor be symmetric
 *                   about the equator (a band of latitudes serves).  On a symmetric grid,
 *                   |theta[k] + theta[n_theta - 1 - k] - pi| <= 1e-12 pi for every k, both chains
 *                   start at ring n_theta / 2 and the southern chain's steps are the northern
 *                   ones mirrored (Alg. 1); on any other grid they start at the ring nearest the
 *                   equator (the southern one of two at the same distance) and the set-up
 *                   computes the southern chain's steps on their own (Alg. 2 starts at the
 *                   equator; a chain may then hold no ring).
 * Every other argument, the ownership and the errors as for smerf_plan_create_ex (SMERF_EINVAL
 * for colatitudes that break these rules).
 */
int smerf_plan_create_theta(const double* kappa, int p, double A, int n_theta, const double* theta, int n_phi,
                            unsigned flags, int anchor_spacing, smerf_plan** out_plan);

/*
 * smerf_plan_create_khat_theta -- smerf_plan_create_khat (the spectrum by its kappa-hat values,
 * complex-conjugate pairs allowed) at the ring colatitudes theta[n_theta] of
 * smerf_plan_create_theta, with the same rules for them.  theta = NULL is SMERF_EINVAL (use
 * smerf_plan_create_khat for the equiangular grid).  Every other argument, the ownership and the
 * errors as for smerf_plan_create_khat.
 */
int smerf_plan_create_khat_theta(const double* khat_re, const double* khat_im, int p, double A, int n_theta,
                                 const double* theta, int n_phi, unsigned flags, int anchor_spacing,
                                 smerf_plan** out_plan);

/* smerf_plan_create -- smerf_plan_create_ex with the default anchor spacing. */
int smerf_plan_create(const double* kappa, int p, double A, int n_theta, int n_phi,
                      unsigned flags, smerf_plan** out_plan);

/* smerf_plan_destroy -- frees the plan and its device memory.  The caller must have
 * synchronised every stream that still uses it.  NULL is accepted. */
int smerf_plan_destroy(smerf_plan* plan);

/*
 * smerf_sample -- draw n_samples realisations into caller-owned device memory
 * (Alg. 2: start state at the equator ring, Markov recursion outward along both chains,
 * per-ring real DFT).  Asynchronous on `stream`.
 *
 *   plan       a plan from smerf_plan_create*
 *   seed       Philox key of realisation 0; realisation r uses seed + r
 *   n_samples  >= 0 (0 is a no-op)
 *   out        device pointer to n_samples * n_theta * n_phi floats (doubles with
 *              SMERF_RECUR_FP64), 16-byte aligned (n_samples * points_per_sample for a plan
 *              with ring-dependent longitudes, smerf_plan_set_rings)
 *   stream     cudaStream_t as void*
 *
 * Scratch (the anchor states, 2 * n_samples * (anchors + 1) * 2p * n_phi/2 values) is
 * taken from the stream-ordered allocator and released on the same stream.
 */
int smerf_sample(const smerf_plan* plan, uint64_t seed, int n_samples, void* out, void* stream);

/*
 * smerf_sample_timed -- smerf_sample that also records two caller-owned CUDA events
 * (cudaEvent_t as void*, may be NULL) on `stream` immediately before and after the
 * segment kernel, the kernel that synthesises and writes the field.  For measuring that
 * kernel's duration on the stream it runs on; otherwise identical to smerf_sample.
 */
int smerf_sample_timed(const smerf_plan* plan, uint64_t seed, int n_samples, void* out, void* stream,
                       void* event_before_segments, void* event_after_segments);

/*
 * smerf_last_device_status -- synchronises `stream` (cudaStream_t as void*, NULL = legacy
 * default stream) and reports how the work queued on it ended: SMERF_OK, or SMERF_ECUDA if a
 * kernel or copy on it failed (a non-sticky CUDA error is cleared).  The single-request
 * kernels keep no device error word: none waits on a flag or on another CTA (the
 * producer/FFT hand-off uses the CTA's own named barriers, the table staging cp.async
 * groups, both complete by construction).  The one device wait of the library, in the
 * persistent batch launch, reports through smerf_batch_status.
 */
int smerf_last_device_status(void* stream);

/*
 * smerf_scratch_trim -- return to the device the memory that the library's per-call scratch
 * pool on the current device holds and no call is using.  smerf_sample and smerf_sample_host
 * take their temporary device memory (anchor states, FP32 copies of FP64 tables, the field on
 * the host path) stream-ordered from that pool, which keeps it between calls so that a call
 * after a synchronisation maps no new memory; the pool holds at most the largest amount that
 * calls in flight used together.  SMERF_OK, or SMERF_ECUDA.
 */
int smerf_scratch_trim(void);

/*
 * smerf_sample_launches -- how many kernels one smerf_sample(plan, ., n_samples, ...) call
 * launches on its stream: the anchor kernel and the segment kernel, and, when the plan keeps
 * FP64 tables, recurses in FP32 and n_samples >= 4, one short conversion of the coarse and
 * start tables to FP32 ahead of them (the anchor kernel's threads convert the step tables).
 * 0 for n_samples == 0; SMERF_EINVAL (negative) for a NULL plan or a negative count.
 */
int smerf_sample_launches(const smerf_plan* plan, int n_samples);

/*
 * smerf_sample_host -- smerf_sample into HOST memory `host_out` (n_samples * n_theta * n_phi
 * elements), synchronising the stream before returning.  For callers without device buffers.
 * Page-locked host memory (cudaHostAlloc, cudaHostRegister, pinned torch tensors) is written
 * directly by the kernels over the CPU-GPU link; other host memory gets a stream-ordered
 * device buffer and one device-to-host copy.
 */
int smerf_sample_host(const smerf_plan* plan, uint64_t seed, int n_samples, void* host_out,
                      void* stream);

/*
 * smerf_sample_batched -- n_req independent requests (plans may differ in grid, spectrum
 * and precision) in one call; request i produces exactly what
 * smerf_sample(plans[i], seeds[i], n_samples[i], outs[i], stream) produces.  Requests of
 * the same kernel shape (precision, p, n_phi, anchored or not) run as one anchor launch and
 * one segment launch over a device work list.  Host arrays of length n_req; outs[i] are
 * device pointers.  Builds a temporary smerf_batch and synchronises `stream` before
 * returning.
 */
int smerf_sample_batched(const smerf_plan* const* plans, const uint64_t* seeds,
                         const int* n_samples, void* const* outs, int n_req, void* stream);

/*
 * Reusable batches (for repeated sampling and CUDA graphs).
 *
 * smerf_batch_create: groups the requests (plans[i], n_samples[i]) by kernel shape, builds
 *   the device work lists and allocates all scratch.  Synchronous.  The plans must outlive
 *   the batch.
 * smerf_batch_set: stores seeds[i] and outputs outs[i] (16-byte aligned; device memory, or
 *   page-locked host memory that the GPU addresses with the same pointer, such as
 *   cudaHostAlloc memory or pinned torch tensors, which the kernels then write over the
 *   CPU-GPU link) in the batch's pinned staging memory.  Host-only; the previous launch's
 *   copy of the staging memory must have completed (synchronise its stream first).
 * smerf_batch_launch: copies the staging memory to the device and launches the batch on
 *   `stream` (asynchronous).  FP32 recursion with p <= 2, by default: one launch over every
 *   request's anchor items (Alg. 2's first step: start ring and anchors), a reset of the work
 *   queue, and one launch of persistent CTAs that take the segment items of every shape (the
 *   rings between anchors) from that queue; stream order puts the anchors first.  With
 *   smerf_batch_set_single_launch(batch, 1): a reset of the queue and one launch of persistent
 *   CTAs that take every anchor item and then every segment item from it; a segment item
 *   first waits, on the device, until every anchor item of its request has finished.  That
 *   wait is bounded (about one second): when it runs out the item is skipped and the launch
 *   records it, which smerf_batch_status reports.  FP64 recursion or p = 3: an anchor and a
 *   segment launch per kernel shape.  Capturable into a CUDA graph: a replay re-reads the staging
 *   memory, so smerf_batch_set between replays changes seeds and outputs.  Requests whose
 *   shape has no batched kernel (n_phi = 32768 in FP32), and requests whose plan has
 *   ring-dependent longitudes (smerf_plan_set_rings), are launched individually, with their
 *   seed and output passed by value; a batch that holds such requests returns
 *   SMERF_EUNSUPPORTED when `stream` is capturing (a replay could not see later seeds and
 *   outputs) and launches normally otherwise.
 * smerf_batch_sample: smerf_batch_set + smerf_batch_launch.
 * smerf_batch_info: number of kernel shapes among the batched requests (groups) and of
 *   individually launched requests.
 * smerf_batch_set_single_launch: 1 selects the one-launch form of the FP32-recursion work
 *   above, 0 (the default) the two-launch form, for the following launches.  Both give the
 *   same fields; the two-launch form is the faster of the two on GB300 (its persistent kernel
 *   carries no anchor code).  SMERF_EINVAL for other values.
 * smerf_batch_launch_count: kernels one smerf_batch_launch starts (requests with FP32
 *   recursion and p <= 2: two per table precision, or one with the single-launch form, every
 *   shape together; FP64 recursion or p = 3: two per shape; plus the individually launched
 *   requests').
 * smerf_batch_status: synchronises `stream` and reports how the batch's last persistent
 *   launches ended: SMERF_OK, SMERF_ETIMEOUT if a segment item's wait for its anchors ran out
 *   (its rings were not written), or SMERF_ECUDA.
 * smerf_debug_batch_fail_waits: test hook; the batch's next single launch starts its anchor
 *   counters one below zero, so that no segment item's wait can be met and smerf_batch_status
 *   then returns SMERF_ETIMEOUT.  The launch after that is normal again.
 * smerf_batch_destroy: frees the batch; synchronise its streams first.  NULL is accepted.
 */
typedef struct smerf_batch smerf_batch;
int smerf_batch_create(const smerf_plan* const* plans, const int* n_samples, int n_req, smerf_batch** out);
int smerf_batch_set(smerf_batch* batch, const uint64_t* seeds, void* const* outs);
int smerf_batch_launch(smerf_batch* batch, void* stream);
int smerf_batch_sample(smerf_batch* batch, const uint64_t* seeds, void* const* outs, void* stream);
int smerf_batch_info(const smerf_batch* batch, int* n_groups, int* n_singles);
int smerf_batch_launch_count(const smerf_batch* batch);
int smerf_batch_status(const smerf_batch* batch, void* stream);
int smerf_batch_set_single_launch(smerf_batch* batch, int single);
int smerf_debug_batch_fail_waits(smerf_batch* batch);
int smerf_batch_destroy(smerf_batch* batch);

/*
 * smerf_sample_noalloc -- smerf_sample without any device allocation.  The paper has no
 * counterpart; this exists for callers that cannot let a library allocate device memory:
 * real-time or embedded hosts whose device memory is carved out once at start-up, and
 * frameworks that own all device memory through their own pool and forbid other
 * allocations (a cudaMalloc there can fail, or synchronise the device mid-frame).
 *
 * Same arguments, output and noise as smerf_sample; `out` is still caller-owned device
 * memory.  The anchor-state scratch is a fixed 16 MiB array inside the library's device
 * image (present on every GPU that loads the library until the process exits).  A request
 * needs 2 * n_samples * (anchors + 1) * 2p * (n_phi/2) * (4 or 8 with SMERF_RECUR_FP64)
 * bytes of it (smerf_plan_info: scratch_bytes_per_sample * n_samples); larger requests
 * return SMERF_ESCRATCH and launch nothing.
 *
 * Each call made outside stream capture looks up the array's device address
 * (cudaGetSymbolAddress) with the plan's device current, so a context that was reset and
 * reloaded the library's device image is followed; a call made while `stream` is capturing
 * reuses the address found by the last call outside capture on that device (SMERF_EUNSUPPORTED
 * if there was none), so make one call before any capture.  All calls share the one array and it keeps the last call's contents: two calls
 * whose kernels overlap on the GPU (different streams, no ordering between them) race on
 * it, so serialise them.  Calls no cudaMalloc, cudaFree or other allocating routine.
 */
int smerf_sample_noalloc(const smerf_plan* plan, uint64_t seed, int n_samples, void* out, void* stream);

/*
 * smerf_plan_create_many -- n plans at once, each as smerf_plan_create_ex would make it from
 * specs[i] (the same tables, bit for bit), with the n set-ups overlapping on the GPU (they go
 * round-robin onto up to 16 internal streams; one synchronisation at the end).  For many
 * small plans, whose set-up kernels alone occupy a fraction of the GPU.  out_plans[i]
 * receives plan i; each plan's setup_ms (smerf_plan_info) is the wall time of the whole call.
 * Errors as for smerf_plan_create_ex; on any error every plan made is destroyed, all
 * out_plans[i] are NULL and the first error is returned.  Synchronous.
 */
typedef struct smerf_plan_spec {
    const double* kappa;  /* p values, as for smerf_plan_create_ex */
    int p;
    double A;
    int n_theta, n_phi;
    unsigned flags;
    int anchor_spacing;
} smerf_plan_spec;
int smerf_plan_create_many(const smerf_plan_spec* specs, int n, smerf_plan** out_plans);

/* Plan description, filled by smerf_plan_info. */
typedef struct smerf_plan_info_t {
    int p, n_theta, n_phi, n_modes;       /* n_modes = n_phi/2 + 1                              */
    int start_ring;                        /* k0 = n_theta/2                                     */
    int chain_len[2];                      /* rings after the start ring: [0] north, [1] south   */
    int anchor_spacing;                    /* effective H (0 = none)                             */
    int n_anchors[2];                      /* anchors per chain                                  */
    int n_segments;                        /* independent segments over both chains             */
    unsigned flags;
    size_t table_bytes;                    /* device bytes of step + coarse + start tables      */
    size_t scratch_bytes_per_sample;       /* anchor-state scratch per realisation              */
    double setup_ms;                       /* wall time of the set-up kernels                   */
    size_t step_table_bytes;               /* the step tables' part of table_bytes (the tables  */
                                           /* the segment kernel reads)                         */
    size_t points_per_sample;              /* output values of one realisation                  */
} smerf_plan_info_t;

int smerf_plan_info(const smerf_plan* plan, smerf_plan_info_t* info);

/*
 * smerf_plan_set_rings -- iso-latitude grid with ring-dependent longitudes (the paper's Sec. 1
 * remark that the method holds on any iso-latitude grid; HEALPix rings with the colatitudes of
 * smerf_plan_create_theta).  Ring k keeps its colatitude theta_k and holds n_phi_ring[k] points
 * phi = phi0_ring[k] + 2 pi j / n_phi_ring[k], j < n_phi_ring[k]; each n_phi_ring[k] even with
 * 4 <= n_phi_ring[k] <= n_phi of the plan (a power of two takes a radix-4 FFT, other counts a
 * direct synthesis, O(n_phi_ring[k]^2) per ring); phi0_ring may be NULL (no offsets).  Host
 * arrays of n_theta values.  The modes
 * m = 0..n_phi/2, their recursion and noise stay those of the plan; each ring's values are the
 * m-truncated field evaluated at its points: T(phi) = g_0 + 2 sum_{0<m<n_phi/2} Re(g_m e^{i m phi})
 * + Re(g_{n_phi/2}) cos(n_phi phi / 2), so modes above the ring's own Nyquist alias onto it.
 * Output of a sample call: realisation r's rings back to back, ring k at
 * r * P + sum_{k'<k} n_phi_ring[k'] (P = smerf_plan_info's points_per_sample).  Only plans run by
 * the warp-specialised kernels (n_phi <= 8192 with FP32 recursion, <= 4096 with FP64) take rings
 * (else SMERF_EUNSUPPORTED); in a batch such a plan's request is launched individually.
 * n_phi_ring = NULL restores the full grid.  Host only, synchronous; must not run while other
 * calls use the plan, nor while a batch made with the plan exists (a batch takes each plan's
 * ring layout when it is created).
 */
int smerf_plan_set_rings(smerf_plan* plan, const int* n_phi_ring, const double* phi0_ring);

/*
 * smerf_plan_autotune -- time every built launch configuration of the segment kernel that
 * fits this plan on n_samples realisations and keep the fastest for later calls.  A launch
 * configuration is SMERF_LAUNCH_INTS integers: (units per producer thread, realisations per
 * CTA, producer threads, FFT threads, CTAs per SM the kernel is built for, FFT radix plan).
 * The radix plan is 16 (the ring's C2R FFT in Stockham passes of up to 16 points, a
 * fixed-size plan per ring length: 1024 points as 16, 8, 8) or 4 (radix-4 passes for any
 * length); FP64 recursion offers 4 only.  The first five integers change launch parameters
 * only; the radix plan changes the FFT's rounding (FP32: ~1e-7 of the field std), so configurations
 * with the same radix plan give identical output.  Synchronous; allocates a temporary output;
 * must not run while other calls use the plan.  chosen (may be NULL) receives the chosen
 * configuration, all 0 when the plan's shape has no tunable kernel.
 */
#define SMERF_LAUNCH_INTS 6
int smerf_plan_autotune(smerf_plan* plan, int n_samples, void* stream, int* chosen);

/*
 * smerf_plan_autotune_anchor -- choose the anchor spacing H (the band of rings one segment CTA
 * samples between two anchors) by timing: for each of the n_cand (1..16) spacings in
 * candidates[] (each >= 1) the plan's tables are built again with that spacing and whole
 * smerf_sample calls of n_samples realisations are timed on `stream`; the plan keeps the
 * fastest spacing's tables (the same handle; its launch configuration, if fixed, is kept).  H
 * changes the order in which rings are conditioned, hence the map from noise to field, not the
 * field's law (Markov property, Sec. 2).  Synchronous; allocates a temporary output; must not
 * run while other calls use the plan.  *chosen (may be NULL) receives the chosen H, or 0 for a
 * plan in Alg. 2's order (SMERF_ORDER_PAPER), which has no anchors and is left unchanged.
 * Errors as for smerf_plan_create_ex, plus SMERF_EINVAL for bad candidates.
 */
int smerf_plan_autotune_anchor(smerf_plan* plan, int n_samples, const int* candidates, int n_cand, void* stream,
                               int* chosen);

/*
 * smerf_plan_launch_candidates -- the launch configurations smerf_plan_autotune chooses from,
 * SMERF_LAUNCH_INTS integers each, in cand[SMERF_LAUNCH_INTS * i ...] for
 * i < min(count, max_n).  Returns the count (0: no tunable kernel) or SMERF_EINVAL.  Host
 * only.
 */
int smerf_plan_launch_candidates(const smerf_plan* plan, int* cand, int max_n);

/*
 * smerf_plan_set_launch -- fix the segment-kernel launch configuration (SMERF_LAUNCH_INTS
 * integers) to one of the candidates (e.g. a choice smerf_plan_autotune made in an earlier
 * process), or with config == NULL return to the built-in choice (radix plan 16 in FP32).
 * SMERF_EINVAL if config is not a candidate.  Host only.
 */
int smerf_plan_set_launch(smerf_plan* plan, const int* config);

/*
 * smerf_plan_copy_tables -- copy one table block to host memory as FP64, for inspection.
 *   which = 0: start factor B_eq, [p(p+1)/2][n_modes]       (chain ignored)
 *   which = 1: step tables of chain c at position pos (1..chain_len[c]),
 *              [2p^2 + p(p+1)/2][n_modes]: A (p x p), C (p x p), B (lower, row-major)
 *   which = 2: coarse (anchor) tables of chain c, anchor pos (1..n_anchors[c]),
 *              [p^2 + p(p+1)/2][n_modes]: A, B
 * Chain 1 (south) tables act on the mirrored state S x, S = diag((-1)^q), and their B
 * factors have S folded into the columns (the chain is driven by S xi).  B factors of
 * modes m >= 1 carry the 1/sqrt(2) of the Re and Im chains.  FP64 tables hold no entry
 * of magnitude below 2^-120 (smaller values are stored as +-2^-120).  host_out holds
 * rows * n_modes doubles.  Synchronous.
 */
int smerf_plan_copy_tables(const smerf_plan* plan, int which, int chain, int pos, double* host_out);

/* Test hooks (device noise, bit-exact against any Philox4x32-10 implementation).
 * smerf_philox_uint32: out[4*c + i] = word i of call c = 0..ncalls-1 of ring `ring` under
 *   key64 (device pointer, 4*ncalls uint32).
 * smerf_ring_normals: the first n normals of that ring, Box-Muller of words (0,1), (2,3),
 *   in FP32 (fp64 = 0, float out) or FP64 (fp64 = 1, double out).  Asynchronous. */
int smerf_philox_uint32(uint64_t key64, uint32_t ring, int64_t ncalls, uint32_t* out, void* stream);
int smerf_ring_normals(uint64_t key64, uint32_t ring, int64_t n, int fp64, void* out, void* stream);

/* Test hook: the device or page-locked allocation that the library makes after k more from now
 * (k = 0: the next one) fails as if memory were exhausted; k < 0 turns the injection off.  The
 * failing call returns SMERF_ENOMEM and releases what it had allocated.  Process-wide; returns
 * SMERF_OK. */
int smerf_debug_fail_alloc(int k);

/* Human-readable name of a status code. */
const char* smerf_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* SMERF_H */
