// smerf_sample_impl.cuh -- the sampling kernels of the GB300 sphere-GMRF sampler
// (Alg. 2 of Creasey & Lang, arXiv 1709.10314), templated on precision, state size and
// per-thread work.  Included by one translation unit per (recursion, table) precision.
//
// Work decomposition.  Each chain (north, south) starts at ring k0.  Every H-th ring of
// a chain is an anchor; anchor_kernel samples the start state (Eq. (state_initial)) and
// the anchors along the chain (Eq. (state_space) between anchors), one thread per
// (chain, realisation, unit of slots), and keeps them in scratch memory.  segment_kernel
// then samples every segment between two anchors independently: one CTA per (segment,
// group of realisations), threads over azimuthal slots.  Per ring it draws Philox4x32-10
// noise, steps x = A x + C x_right + B xi for every slot, writes g_m into shared memory,
// runs the C2R FFT there and streams the ring to HBM with 16-byte stores.  The
// coefficients never touch HBM.
//
// Slots: slot s in [1, n_phi/2) is mode m = s (Re and Im chains); slot 0 holds the real
// chain of m = 0 and the Re chain of the Nyquist mode m = n_phi/2.  A "unit" is the set
// of slots whose 2p normals fill whole Philox calls (p = 1: two slots per call, p = 2: one slot
// per call, p = 3: two slots per three calls); it holds unit_vals(p) state values.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "smerf_internal.cuh"

// Thread limit of the warp-specialised kernels (producer + FFT threads per CTA); it also
// bounds their registers per thread (65536 / limit).
#ifndef SMERF_WS_MAXT
#define SMERF_WS_MAXT 768
#endif
// Resident 128-thread blocks per SM the FP32 anchor kernels are compiled for (7 x 152 SMs covers
// the 1024 blocks of a 64-realisation, 1024-unit request in one wave).
#ifndef SMERF_ANCHOR_MINB
#define SMERF_ANCHOR_MINB 7
#endif
// Realisations per interleaved group of Philox generators in the producer loop.
#ifndef SMERF_RB
#define SMERF_RB 1
#endif
// Thread limit of the p = 3 warp-specialised kernels (one CTA per SM)
#ifndef SMERF_P3_MAXT
#define SMERF_P3_MAXT 512
#endif

namespace smerf {

constexpr int kWsMaxThreads = SMERF_WS_MAXT;
// Thread limit of the warp-specialised kernels built for MINB resident CTAs per SM: one CTA
// gets 65536 / SMERF_WS_MAXT registers per thread, two get 64 (512 threads each).
// p = 3 (12 state values and two 24-value table rows per unit) is built for at most 512 threads
// (128 registers) with one CTA per SM.
__host__ __device__ constexpr int ws_max_threads(int minb, int M = 1) { return minb == 1 && M != 3 ? kWsMaxThreads : SMERF_P3_MAXT; }

template <int M> constexpr int kG = unit_slots(M);

// the 4 NC normals of unit u of ring `ring` for realisation key `key64`: Philox calls
// [NC u, NC (u + 1)), four normals each
template <class Real, int NC = 1>
__device__ __forceinline__ void unit_normals(uint64_t key64, uint32_t u, uint32_t ring, Real (&n)[4 * NC])
{
    const PhiloxKey key{(uint32_t)key64, (uint32_t)(key64 >> 32)};
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const uint4 w = philox4x32_10(make_uint4(u * NC + j, ring, 0u, 0u), key);
        box_muller(w.x, w.y, n[4 * j], n[4 * j + 1]);
        box_muller(w.z, w.w, n[4 * j + 2], n[4 * j + 3]);
    }
}

template <class Real, class TabT>
__device__ __forceinline__ Real tabcvt(TabT v) { return (Real)v; }
template <class Real, class TabT>
__device__ __forceinline__ Real tabld(const TabT* p) { return tabcvt<Real, TabT>(__ldg(p)); }

// FP64 table value -> FP32 with three integer instructions (GB300 runs FP64 conversions on
// its narrow FP64 pipe): shift the exponent and top mantissa bits into place, rebias the
// exponent by 896, restore the sign.  Truncates the mantissa.  Valid because FP64 tables
// hold no magnitude below 2^-120 (set-up clamps them) and none above the FP32 range.
template <>
__device__ __forceinline__ float tabcvt<float, double>(double v)
{
    const uint32_t hi = (uint32_t)(__double_as_longlong(v) >> 32);
    const uint32_t lo = (uint32_t)__double_as_longlong(v);
    const uint32_t t = __funnelshift_l(lo, hi, 3) - (128u << 23);
    return __uint_as_float((t & 0x7FFFFFFFu) | (hi & 0x80000000u));
}

// anchor scratch offset: [c][r][j][slot][f], f = part * M + q (a unit's unit_vals(M) values
// are contiguous: 16 bytes for p = 1, 2 and 48 for p = 3 in FP32)
template <int M>
__device__ __forceinline__ size_t aoff(const SampleParams& P, int c, int r, int j, int f, int slot)
{
    return ((((size_t)c * P.n_samples + r) * (P.na_max + 1) + j) * (size_t)P.Nc + slot) * (2 * M) + f;
}

// four consecutive values (16 bytes in FP32, 32 in FP64) as one or two vector accesses
template <class Real> struct Vec4;
template <> struct Vec4<float> {
    static __device__ __forceinline__ void ld(const float* p, float (&v)[4]) { const float4 a = *reinterpret_cast<const float4*>(p); v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; }
    static __device__ __forceinline__ void ldcg(const float* p, float (&v)[4]) { const float4 a = __ldcg(reinterpret_cast<const float4*>(p)); v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; }
    static __device__ __forceinline__ void ldg(const float* p, float (&v)[4]) { const float4 a = __ldg(reinterpret_cast<const float4*>(p)); v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; }
    static __device__ __forceinline__ void st(float* p, const float (&v)[4]) { *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]); }
};
template <> struct Vec4<double> {
    static __device__ __forceinline__ void ld(const double* p, double (&v)[4]) { const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1]; v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; }
    static __device__ __forceinline__ void ldcg(const double* p, double (&v)[4]) { const double2 a = __ldcg(reinterpret_cast<const double2*>(p)), b = __ldcg(reinterpret_cast<const double2*>(p) + 1); v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; }
    static __device__ __forceinline__ void ldg(const double* p, double (&v)[4]) { const double2 a = __ldg(reinterpret_cast<const double2*>(p)), b = __ldg(reinterpret_cast<const double2*>(p) + 1); v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y; }
    static __device__ __forceinline__ void st(double* p, const double (&v)[4]) { reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]); reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]); }
};

// a unit's NV state values (NV a multiple of 4; 16-byte aligned) as NV / 4 Vec4 accesses
template <class Real, int NV> struct VecN {
    static_assert(NV % 4 == 0, "whole Vec4 groups");
    using Q = Real[4];
    static __device__ __forceinline__ void ld(const Real* p, Real (&v)[NV])
    {
#pragma unroll
        for (int k = 0; k < NV; k += 4) Vec4<Real>::ld(p + k, *reinterpret_cast<Q*>(&v[k]));
    }
    static __device__ __forceinline__ void ldg(const Real* p, Real (&v)[NV])
    {
#pragma unroll
        for (int k = 0; k < NV; k += 4) Vec4<Real>::ldg(p + k, *reinterpret_cast<Q*>(&v[k]));
    }
    static __device__ __forceinline__ void ldcg(const Real* p, Real (&v)[NV])
    {
#pragma unroll
        for (int k = 0; k < NV; k += 4) Vec4<Real>::ldcg(p + k, *reinterpret_cast<Q*>(&v[k]));
    }
    // anchor states: through the read-only path when an earlier launch wrote them, through L2
    // only (CG) when the same launch did (the persistent batch kernel)
    template <bool CG> static __device__ __forceinline__ void ld_anchor(const Real* p, Real (&v)[NV])
    {
        if constexpr (CG) ldcg(p, v);
        else ldg(p, v);
    }
    static __device__ __forceinline__ void st(Real* p, const Real (&v)[NV])
    {
#pragma unroll
        for (int k = 0; k < NV; k += 4) Vec4<Real>::st(p + k, *reinterpret_cast<const Q*>(&v[k]));
    }
};

// a unit's coefficients g_m into the ring buffer (slot 0's imaginary part carries the Nyquist
// chain): p = 1 as one vector store of (Re, Im, Re, Im), else one complex value per slot
template <class C, class Real, int M>
__device__ __forceinline__ void put_unit(C* ring, int u, const Real (&x)[unit_vals(M)])
{
    constexpr int G = unit_slots(M);
    if constexpr (M == 1) {
        Vec4<Real>::st(reinterpret_cast<Real*>(ring + 2 * u), x);
    } else {
#pragma unroll
        for (int g = 0; g < G; ++g) ring[G * u + g] = cmk<C>(x[g * 2 * M], x[g * 2 * M + M]);
    }
}

// one step-table row (step_row(M) values, 16-byte aligned) converted to the recursion precision
template <class Real, class TabT, int ROW>
__device__ __forceinline__ void load_row(const TabT* p, Real (&t)[ROW])
{
#pragma unroll
    for (int k = 0; k < ROW; k += 4) {
        TabT v[4];
        Vec4<TabT>::ldg(p + k, v);
#pragma unroll
        for (int i = 0; i < 4; ++i) t[k + i] = tabcvt<Real, TabT>(v[i]);
    }
}

// ------------------------------------------------------------------ anchors
// anchors whose table values and normals are fetched ahead of the one being stepped
__host__ __device__ constexpr int anchor_ahead(int M) { return M == 1 ? 4 : M == 2 ? 2 : 1; }
// resident 128-thread blocks per SM the anchor kernels are built for: FP64 and p = 3 (whose
// fetched-ahead tables are 60 values) with the registers of four, FP32 p <= 2 seven
__host__ __device__ constexpr int anchor_minb(int real_bytes, int M) { return real_bytes == 8 || M == 3 ? 4 : SMERF_ANCHOR_MINB; }

// Work an anchor thread carries out beside its anchors: prologue() before the first anchor,
// step(j, d) at the end of anchor j's step (d = (j - 1) mod anchor_ahead(M)).  NoStage: none.
struct NoStage {
    __device__ __forceinline__ void prologue() {}
    __device__ __forceinline__ void step(int, int) {}
};

// FP64 -> FP32 conversion of a plan's step tables carried by the anchor threads (StageJob),
// so that the copies overlap the anchors' arithmetic instead of taking a launch of their own.
// In round k thread g of T converts group l = (k - k_0) T + g (kStageGroup elements) of table
// q (k_0 = 0 for q = 0, rounds0 for q = 1).  Rounds k < k_loop run during the thread's
// anchors: the group is copied asynchronously into one of the thread's two shared-memory
// slots (its destination noted beside the slot), then converted (tabcvt, the kernels' own
// conversion) and stored at the end of anchor (k + 1) every, two rounds after its copy
// started.  rest() runs the thread's remaining rounds one at a time (all of them if it had no
// anchors to step).
constexpr int kStageGroup = 8;      // elements per group: 64 bytes of FP64, 32 of FP32
constexpr int kStageSlots = 2;      // groups in flight per thread
struct StageCarrier {
    const StageJob& J;
    unsigned g, T;  // thread index and thread count of the launch (the host keeps both < 2^30)
    unsigned sa;    // shared address of the thread's data slot 0 (slot s at + s * kDataStride)
    unsigned sm;    // shared address of the thread's destination note 0 (+ s * kMetaStride)
    int k = 0;          // next round to convert during the anchors
    int countdown = 0;  // anchors until the next conversion

    static constexpr unsigned kDataStride = 128 * 8 * kStageGroup;  // 128 threads x 64 bytes
    static constexpr unsigned kMetaStride = 128 * 8;                // 128 threads x 8 bytes

    // start round k's copy into slot s and note its destination (null: nothing to store; a
    // group at a table's ragged end is converted at once); commits one copy group in every
    // case, so that the counts of committed groups stay uniform
    __device__ __forceinline__ void issue(int k, unsigned s) const
    {
        float* note = nullptr;
        if ((unsigned)k < J.rounds) {
            const bool q1 = (unsigned)k >= J.rounds0;
            const unsigned l = ((unsigned)k - (q1 ? J.rounds0 : 0u)) * T + g;
            const unsigned long long n = q1 ? J.n[1] : J.n[0];
            const unsigned long long i = (unsigned long long)kStageGroup * l;
            if (i < n) {
                const double* src = (q1 ? J.src[1] : J.src[0]) + i;
                float* dst = (q1 ? J.dst[1] : J.dst[0]) + i;
                if (n - i >= kStageGroup) {
                    const unsigned a = sa + s * kDataStride;
#pragma unroll
                    for (int e = 0; e < kStageGroup / 2; ++e)
                        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a + 16u * e), "l"(src + 2 * e));
                    note = dst;
                } else {
                    for (int e = 0; e < (int)(n - i); ++e) dst[e] = tabcvt<float, double>(src[e]);
                }
            }
        }
        asm volatile("st.shared.u64 [%0], %1;\n" ::"r"(sm + s * kMetaStride), "l"(note));
        asm volatile("cp.async.commit_group;\n" ::);
    }
    // convert and store the group in slot s (its copy has landed)
    __device__ __forceinline__ void finish(unsigned s) const
    {
        float* dst;
        asm volatile("ld.shared.u64 %0, [%1];\n" : "=l"(dst) : "r"(sm + s * kMetaStride));
        if (!dst) return;
        const unsigned a = sa + s * kDataStride;
#pragma unroll
        for (int e = 0; e < kStageGroup / 4; ++e) {
            double x0, x1, x2, x3;
            asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];\n" : "=d"(x0), "=d"(x1) : "r"(a + 32u * e));
            asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];\n" : "=d"(x2), "=d"(x3) : "r"(a + 32u * e + 16u));
            reinterpret_cast<float4*>(dst)[e] = make_float4(tabcvt<float, double>(x0), tabcvt<float, double>(x1),
                                                            tabcvt<float, double>(x2), tabcvt<float, double>(x3));
        }
    }
    __device__ __forceinline__ void issue_loop(int k, unsigned s) const
    {
        if (k < J.k_loop) {
            issue(k, s);
        } else {
            asm volatile("cp.async.commit_group;\n" ::);
        }
    }
    __device__ __forceinline__ void prologue()
    {
#pragma unroll
        for (int s = 0; s < kStageSlots; ++s) issue_loop(s, s);
        k = 0;
        countdown = J.every;
    }
    // end of an anchor: every J.every anchors, round k (copied kStageSlots rounds ago) is
    // converted and round k + kStageSlots started in its slot, spreading the copies over the
    // anchors instead of crowding them into the first ones
    __device__ __forceinline__ void step(int, int)
    {
        if (--countdown > 0) return;
        countdown = J.every;
        const unsigned s = (unsigned)k % kStageSlots;
        asm volatile("cp.async.wait_group %0;\n" ::"n"(kStageSlots - 1));  // round k has landed
        if (k < J.k_loop) finish(s);
        issue_loop(k + kStageSlots, s);
        ++k;
    }
    __device__ __forceinline__ void rest(bool stepped) const
    {
        asm volatile("cp.async.wait_all;\n" ::);
        for (int k = stepped ? J.k_loop : 0; (unsigned)k < J.rounds; ++k) {
            issue(k, 0);
            asm volatile("cp.async.wait_all;\n" ::);
            finish(0);
        }
    }
};

template <class Real, class TabT, int M, class Hook>
__device__ __forceinline__ void anchor_body(const SampleParams& P, int u, int r, int c, Hook& hook)
{
    constexpr int G = kG<M>;
    constexpr int T = tri(M);
    constexpr int Ec = coarse_elems(M);
    if (u >= P.n_units || r >= P.n_samples) return;
    const size_t mp = P.n_modes_pad;
    const uint64_t key = P.seed + (uint64_t)r;
    Real* anc = (Real*)P.anc;
    constexpr int NU = unit_vals(M), NC = unit_calls(M);
    Real x[G][2][M];
    Real nr[NU];
    // start ring: x = B_eq xi (x basis); the southern chain keeps S x
    unit_normals<Real, NC>(key, (uint32_t)u, (uint32_t)P.k0, nr);
    const TabT* beq = (const TabT*)P.beq;
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int part = 0; part < 2; ++part) {
            const int s = G * u + g;
            const int mode = (part == 1 && s == 0) ? P.Nc : s;
            int e = 0;
#pragma unroll
            for (int p = 0; p < M; ++p) {
                Real acc = 0;
#pragma unroll
                for (int q = 0; q <= p; ++q, ++e) acc += tabld<Real, TabT>(beq + (size_t)e * mp + mode) * nr[g * 2 * M + part * M + q];
                x[g][part][p] = (c == 1 && (p & 1)) ? -acc : acc;
            }
        }
    {
        Real v[NU];
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int part = 0; part < 2; ++part)
#pragma unroll
                for (int q = 0; q < M; ++q) v[g * 2 * M + part * M + q] = x[g][part][q];
        VecN<Real, NU>::st(anc + aoff<M>(P, c, r, 0, 0, G * u), v);
    }
    // anchors: x_j = Phi x_{j-1} + chol(S) xi.  The table values and normals of the next AD
    // anchors are fetched ahead of the matrix-vector products (they do not depend on the
    // state), so the load latencies of consecutive anchors overlap.
    // (selects, not P.x[c]: indexing a kernel parameter's array with a runtime index copies
    // the whole parameter block to local memory)
    const TabT* cs = (const TabT*)(c == 0 ? P.coarse[0] : P.coarse[1]);
    const int na = c == 0 ? P.n_anchors[0] : P.n_anchors[1];
    constexpr int AD = anchor_ahead(M);  // anchors prefetched ahead (the loads come from L2 or HBM)
    Real tq[AD][G][2][Ec];
    Real nq[AD][NU];
    const int k0 = P.k0, H = P.H, Ncm = P.Nc;  // copies: the lambda must not take P's address
    // table values of anchor j, converted; both chains of a slot share its mode's values except
    // slot 0, whose second chain is the Nyquist mode
    auto fetch = [=](int j, Real (&t)[G][2][Ec], Real (&xi)[NU]) {
        const int ring = c == 0 ? k0 - j * H : k0 + j * H;
        unit_normals<Real, NC>(key, (uint32_t)u, (uint32_t)ring, xi);
        const TabT* tb = cs + (size_t)j * Ec * mp;
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int s = G * u + g;
#pragma unroll
            for (int e = 0; e < Ec; ++e) t[g][0][e] = tabcvt<Real, TabT>(__ldg(tb + (size_t)e * mp + s));
            if (s == 0) {
#pragma unroll
                for (int e = 0; e < Ec; ++e) t[g][1][e] = tabcvt<Real, TabT>(__ldg(tb + (size_t)e * mp + Ncm));
            } else {
#pragma unroll
                for (int e = 0; e < Ec; ++e) t[g][1][e] = t[g][0][e];
            }
        }
    };
    // a ring of D prefetched anchors: slot d holds anchor j's tables and normals for j = d mod D
#pragma unroll
    for (int d = 0; d < AD; ++d)
        if (1 + d <= na) fetch(1 + d, tq[d], nq[d]);
    hook.prologue();
    for (int j0 = 1; j0 <= na; j0 += AD) {
#pragma unroll
        for (int d = 0; d < AD; ++d) {
            const int j = j0 + d;
            if (j > na) break;
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int part = 0; part < 2; ++part) {
                    Real xn[M];
#pragma unroll
                    for (int p = 0; p < M; ++p) {
                        Real acc = 0;
#pragma unroll
                        for (int q = 0; q < M; ++q) acc += tq[d][g][part][p * M + q] * x[g][part][q];
                        int e = M * M + p * (p + 1) / 2;
#pragma unroll
                        for (int q = 0; q <= p; ++q, ++e) acc += tq[d][g][part][e] * nq[d][g * 2 * M + part * M + q];
                        xn[p] = acc;
                    }
#pragma unroll
                    for (int q = 0; q < M; ++q) x[g][part][q] = xn[q];
                }
            Real v[NU];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int part = 0; part < 2; ++part)
#pragma unroll
                    for (int q = 0; q < M; ++q) v[g * 2 * M + part * M + q] = x[g][part][q];
            VecN<Real, NU>::st(anc + aoff<M>(P, c, r, j, 0, G * u), v);
            if (j + AD <= na) fetch(j + AD, tq[d], nq[d]);
            hook.step(j, d);
        }
    }
    (void)T;
}

// one thread per (chain c, realisation r, unit u)
template <class Real, class TabT, int M>
__global__ void __launch_bounds__(128, anchor_minb(sizeof(Real), M)) anchor_kernel(SampleParams P)
{
    NoStage h;
    anchor_body<Real, TabT, M>(P, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y, blockIdx.z, h);
}

// anchor_kernel that also converts the plan's FP64 step tables to FP32 (StageCarrier); its
// anchors read the coarse and start tables already staged as FP32
template <class Real, class TabT, int M>
__global__ void __launch_bounds__(128, anchor_minb(4, M)) anchor_stage_kernel(SampleParams P, StageJob J)
{
    static_assert(sizeof(Real) == 4 && sizeof(TabT) == 4, "staging converts FP64 tables for FP32 recursion");
    __shared__ __align__(16) double slots[kStageSlots * 128 * kStageGroup];  // [slot][thread][group]
    __shared__ __align__(8) unsigned long long notes[kStageSlots * 128];      // [slot][thread]
    const unsigned T = gridDim.x * blockDim.x * gridDim.y * gridDim.z;
    const unsigned g = ((blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x;
    StageCarrier h{J, g, T, (unsigned)__cvta_generic_to_shared(slots + kStageGroup * threadIdx.x),
                   (unsigned)__cvta_generic_to_shared(notes + threadIdx.x), 0, 0};
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const bool stepped = u < P.n_units && (int)blockIdx.y < P.n_samples;  // anchor_body's own test
    if (stepped) anchor_body<Real, TabT, M>(P, u, blockIdx.y, blockIdx.z, h);
    h.rest(stepped);
}

// batched: item = (request, block of 128 units, realisation, chain)
template <class Real, class TabT, int M>
__global__ void __launch_bounds__(128, anchor_minb(sizeof(Real), M)) anchor_batched_kernel(const SampleParams* __restrict__ descs,
                                                             const int4* __restrict__ items)
{
    const int4 it = items[blockIdx.x];
    const SampleParams P = descs[it.x];
    NoStage h;
    anchor_body<Real, TabT, M>(P, it.y * blockDim.x + threadIdx.x, it.z, it.w, h);
}

// ------------------------------------------------------------------ FFT
// Output rows of ring `ring` for the realisations of a CTA: gout[r] = base + r * stride
// (complex elements; stride = one realisation, n_theta x n_phi / 2).
template <class C> struct RingOut {
    C* base;
    size_t stride;
    __device__ __forceinline__ C* operator[](int r) const { return base + (size_t)r * stride; }
};

template <class C>
__device__ __forceinline__ void dft2(C& a, C& b) { const C t = a; a = cadd(t, b); b = csub(t, b); }

template <class C>
__device__ __forceinline__ void dft4(C* v)  // inverse (positive exponent), in place, natural order
{
    const C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    const C t2 = cadd(v[1], v[3]), t3 = cmuli(csub(v[1], v[3]));
    v[0] = cadd(t0, t2); v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3); v[3] = csub(t1, t3);
}

template <class C>
__device__ __forceinline__ void dft8(C* v)
{
    using R = decltype(C::x);
    C e[4] = {v[0], v[2], v[4], v[6]};
    C o[4] = {v[1], v[3], v[5], v[7]};
    dft4(e);
    dft4(o);
    const R h = (R)0.70710678118654752440;
    // w^a O_a, w = e^{i pi/4}
    const C o1 = cmk<C>(h * (o[1].x - o[1].y), h * (o[1].x + o[1].y));
    const C o2 = cmuli(o[2]);
    const C o3 = cmk<C>(-h * (o[3].x + o[3].y), h * (o[3].x - o[3].y));
    v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);   v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);   v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);   v[7] = csub(e[3], o3);
}

// 16 points as 4 x 4: DFT-4 over n1 of x[4 n1 + n2], twiddles w16^(n2 k1), DFT-4 over n2
template <class C>
__device__ __forceinline__ void dft16(C* v)
{
    using R = decltype(C::x);
    const R c1 = (R)0.92387953251128675613, s1 = (R)0.38268343236508977173, h = (R)0.70710678118654752440;
    C y[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
        y[n2][0] = v[n2];
        y[n2][1] = v[4 + n2];
        y[n2][2] = v[8 + n2];
        y[n2][3] = v[12 + n2];
        dft4(y[n2]);
    }
    y[1][1] = cmul(y[1][1], cmk<C>(c1, s1));
    y[1][2] = cmk<C>(h * (y[1][2].x - y[1][2].y), h * (y[1][2].x + y[1][2].y));
    y[1][3] = cmul(y[1][3], cmk<C>(s1, c1));
    y[2][1] = cmk<C>(h * (y[2][1].x - y[2][1].y), h * (y[2][1].x + y[2][1].y));
    y[2][2] = cmuli(y[2][2]);
    y[2][3] = cmk<C>(-h * (y[2][3].x + y[2][3].y), h * (y[2][3].x - y[2][3].y));
    y[3][1] = cmul(y[3][1], cmk<C>(s1, c1));
    y[3][2] = cmk<C>(-h * (y[3][2].x + y[3][2].y), h * (y[3][2].x - y[3][2].y));
    y[3][3] = cmul(y[3][3], cmk<C>(-c1, -s1));
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
        C t[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
        dft4(t);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = t[k2];
    }
}

template <class C, int RP>
__device__ __forceinline__ void dft(C* v)
{
    if constexpr (RP == 2) dft2(v[0], v[1]);
    else if constexpr (RP == 4) dft4(v);
    else if constexpr (RP == 8) dft8(v);
    else dft16(v);
}

// Z_s of the C2R packing (s < Nc): Z_0 = (X_0 + X_Nc) + i (X_0 - X_Nc) from slot 0 = (X_0, X_Nc);
// Z_s = (X_s + conj X_{Nc-s}) + i e^{2 pi i s / n_phi} (X_s - conj X_{Nc-s}).  The Nc-point
// inverse FFT of Z gives z_n = x_{2n} + i x_{2n+1}.
template <class C>
__device__ __forceinline__ C c2r_pack(const C* X, int s, int Nc, const C* pre)
{
    if (s == 0) {
        const C x = X[0];
        return cmk<C>(x.x + x.y, x.x - x.y);
    }
    const C a = X[s], b = cconj(X[Nc - s]);
    return cadd(cadd(a, b), cmuli(cmul(pre[s], csub(a, b))));
}

// Pass plan of the Nc-point FFT: radix 4 while at least 4 points remain per group, then
// radix 2.  Pass p with Ns > 1 reads its twiddles e^{2 pi i i kk / (Ns RP)} from
// twp[off + (i-1) Ns + kk] (laid out so that neighbouring butterflies read neighbouring
// entries); the tables are built with the plan (smerf_setup.cu, pass_twiddle_kernel).
__host__ __device__ inline int pass_radix(int lgNc, int Ns) { return (1 << lgNc) / Ns >= 4 ? 4 : 2; }

// In-place variant: every thread reads all its butterflies before a barrier and writes after
// it (BPT butterflies per thread at most).
template <class C, int RP, int BPT, bool FIRST>
__device__ __forceinline__ void fft_pass_inplace(C* buf, int R, int lgNc, int Ns, const C* twp, const C* pre)
{
    const int Nc = 1 << lgNc;
    const int lgnb = lgNc - (RP == 4 ? 2 : 1);
    const int nb = 1 << lgnb;
    const int total = R << lgnb;
    C v[BPT][RP];
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
        const int b = threadIdx.x + k * blockDim.x;
        if (b < total) {
            const int r = b >> lgnb, j = b & (nb - 1);
            const C* S = buf + ((size_t)r << lgNc);
#pragma unroll
            for (int i = 0; i < RP; ++i) v[k][i] = FIRST ? c2r_pack(S, j + i * nb, Nc, pre) : S[j + i * nb];
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BPT; ++k) {
        const int b = threadIdx.x + k * blockDim.x;
        if (b < total) {
            const int r = b >> lgnb, j = b & (nb - 1);
            const int kk = FIRST ? 0 : (j & (Ns - 1));
            if (!FIRST) {
#pragma unroll
                for (int i = 1; i < RP; ++i) v[k][i] = cmul(v[k][i], __ldg(twp + (i - 1) * Ns + kk));
            }
            dft<C, RP>(v[k]);
            C* D = buf + ((size_t)r << lgNc) + (j - kk) * RP + kk;
#pragma unroll
            for (int a = 0; a < RP; ++a) D[a * Ns] = v[k][a];
        }
    }
    __syncthreads();
}

template <class C, int EPT>
__device__ __forceinline__ void c2r_rings_inplace(C* buf, int R, int lgNc, const C* twp, const C* pre)
{
    const int Nc = 1 << lgNc;
    int Ns = 1, off = 0;
    bool first = true;
    while (Ns < Nc) {
        const int RP = pass_radix(lgNc, Ns);
        if (RP == 4) {
            if (first) fft_pass_inplace<C, 4, (EPT + 3) / 4, true>(buf, R, lgNc, Ns, twp + off, pre);
            else fft_pass_inplace<C, 4, (EPT + 3) / 4, false>(buf, R, lgNc, Ns, twp + off, pre);
        } else {
            if (first) fft_pass_inplace<C, 2, (EPT + 1) / 2, true>(buf, R, lgNc, Ns, twp + off, pre);
            else fft_pass_inplace<C, 2, (EPT + 1) / 2, false>(buf, R, lgNc, Ns, twp + off, pre);
        }
        if (!first) off += (RP - 1) * Ns;
        Ns *= RP;
        first = false;
    }
}

// XOR swizzle of the high-radix plan's shared layout between passes: element e of a ring
// sits at e ^ ((e >> 4) & 15).
__device__ __forceinline__ int hr_swz(int e) { return e ^ ((e >> 4) & 15); }

// In-place high-radix C2R (plan MB = 3: passes of at most 8 points) of one ring held in
// `buf` (natural order in, swizzled between passes), last pass straight to HBM (gout).  Each thread keeps its butterflies' inputs in
// registers across the barrier that separates a pass's reads from its writes; it holds at
// most EPT points (EPT x threads >= Nc).
template <class C, int LGNC, int EPT, int PASS = 0>
__device__ __forceinline__ void hr_c2r_inplace(C* buf, const C* __restrict__ tw3, const C* __restrict__ pre, C* gout)
{
    constexpr int MB = SMERF_INPLACE_MB;
    constexpr int Nc = 1 << LGNC;
    constexpr int LR = hr_bits(LGNC, PASS, MB), RP = 1 << LR;
    constexpr int Ns = 1 << hr_lgns(LGNC, PASS, MB);
    constexpr bool FIRST = PASS == 0, LAST = PASS == hr_passes(LGNC, MB) - 1;
    constexpr int LGNB = LGNC - LR, nb = 1 << LGNB;
    constexpr int KB = (EPT + RP - 1) / RP;  // butterflies per thread
    const C* twp = tw3 + hr_off(LGNC, PASS, MB);
    const int nt = blockDim.x;
    C v[KB][RP];
#pragma unroll
    for (int k = 0; k < KB; ++k) {
        const int j = threadIdx.x + k * nt;
        if (j < nb) {
            if constexpr (FIRST) {
                {
                    const C a = buf[j], bb = cconj(buf[(Nc - j) & (Nc - 1)]);
                    const C g = cadd(cadd(a, bb), cmuli(cmul(__ldg(pre + j), csub(a, bb))));
                    v[k][0] = j == 0 ? cmk<C>(a.x + a.y, a.x - a.y) : g;
                }
#pragma unroll
                for (int i = 1; i < RP; ++i) {
                    const int sidx = j + i * nb;
                    const C a = buf[sidx], bb = cconj(buf[Nc - sidx]);
                    v[k][i] = cadd(cadd(a, bb), cmuli(cmul(__ldg(pre + sidx), csub(a, bb))));
                }
            } else {
#pragma unroll
                for (int i = 0; i < RP; ++i) v[k][i] = buf[hr_swz(j + i * nb)];
                const int kk = j & (Ns - 1);
#pragma unroll
                for (int i = 1; i < RP; ++i) v[k][i] = cmul(v[k][i], __ldg(twp + (i - 1) * Ns + kk));
            }
            dft<C, RP>(v[k]);  // before the barrier: only results stay live across it
        }
        asm volatile("" ::: "memory");  // one butterfly's twiddles at a time
    }
    if constexpr (!LAST) __syncthreads();  // every read of this pass before any write
#pragma unroll
    for (int k = 0; k < KB; ++k) {
        const int j = threadIdx.x + k * nt;
        if (j < nb) {
            const int kk = FIRST ? 0 : (j & (Ns - 1));
            const int idx = ((j - kk) << LR) + kk;
            if constexpr (LAST) {
#pragma unroll
                for (int a = 0; a < RP; ++a) __stcs(gout + idx + a * Ns, v[k][a]);
            } else {
#pragma unroll
                for (int a = 0; a < RP; ++a) buf[hr_swz(idx + a * Ns)] = v[k][a];
            }
        }
    }
    if constexpr (!LAST) {
        __syncthreads();  // this pass's writes before the next pass's reads
        hr_c2r_inplace<C, LGNC, EPT, PASS + 1>(buf, tw3, pre, gout);
    }
}

// ------------------------------------------------------------------ segments
template <class Real>
__device__ __forceinline__ void store_ring(Real* dst, const cplx<Real>* src, int Nc, int tid, int nt);

template <>
__device__ __forceinline__ void store_ring<float>(float* dst, const float2* src, int Nc, int tid, int nt)
{
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int j = tid; j < Nc / 2; j += nt) __stcs(d4 + j, s4[j]);
}

template <>
__device__ __forceinline__ void store_ring<double>(double* dst, const double2* src, int Nc, int tid, int nt)
{
    double2* d2 = reinterpret_cast<double2*>(dst);
    for (int j = tid; j < Nc; j += nt) __stcs(d2 + j, src[j]);
}

// x <- A x + C x_right + B xi for one real chain (tables t = [A | C | B], B lower).
template <class Real, int M, bool RIGHT>
__device__ __forceinline__ void step_state(const Real* t, Real (&x)[M], const Real* xi, const Real* xr)
{
    Real xn[M];
#pragma unroll
    for (int p = 0; p < M; ++p) {
        Real acc = 0;
#pragma unroll
        for (int q = 0; q < M; ++q) acc = fma(t[p * M + q], x[q], acc);
        if (RIGHT) {
#pragma unroll
            for (int q = 0; q < M; ++q) acc = fma(t[M * M + p * M + q], xr[q], acc);
        }
        int e = 2 * M * M + p * (p + 1) / 2;
#pragma unroll
        for (int q = 0; q <= p; ++q, ++e) acc = fma(t[e], xi[q], acc);
        xn[p] = acc;
    }
#pragma unroll
    for (int q = 0; q < M; ++q) x[q] = xn[q];
}

// Philox4x32-10 with precomputed round keys rk[i] = (k0 + i W0, k1 + i W1), i < 10
__device__ __forceinline__ uint4 philox_rk(uint4 c, const uint2* rk)
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint2 k = rk[r];
        const uint64_t p0 = (uint64_t)M0 * c.x;
        const uint64_t p1 = (uint64_t)M1 * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k.x, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k.y, (uint32_t)p0);
    }
    return c;
}

// The normals of one Philox call for NB realisations at once (round keys rk[0..NB)): the NB
// generator chains are independent and run interleaved; the first round's products, which
// depend on the counter only, are shared.
template <class Real, int NB, int NC = 1>
__device__ __forceinline__ void unit_normals_multi(const uint2 (*rk)[10], uint32_t u, uint32_t ring, Real (&n)[NB][4 * NC])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
#pragma unroll
    for (int j = 0; j < NC; ++j) {  // the unit's Philox calls NC u + j
        uint4 c[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) c[b] = make_uint4(u * NC + j, ring, 0u, 0u);
#pragma unroll
        for (int r = 0; r < 10; ++r) {
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const uint2 k = rk[b][r];
                const uint64_t p0 = (uint64_t)M0 * c[b].x;
                const uint64_t p1 = (uint64_t)M1 * c[b].z;
                c[b] = make_uint4((uint32_t)(p1 >> 32) ^ c[b].y ^ k.x, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c[b].w ^ k.y,
                                  (uint32_t)p0);
            }
        }
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            box_muller(c[b].x, c[b].y, n[b][4 * j], n[b][4 * j + 1]);
            box_muller(c[b].z, c[b].w, n[b][4 * j + 2], n[b][4 * j + 3]);
        }
    }
}

template <class Real, int NC = 1>
__device__ __forceinline__ void unit_normals_rk(const uint2* rk, uint32_t u, uint32_t ring, Real (&n)[4 * NC])
{
#pragma unroll
    for (int j = 0; j < NC; ++j) {
        const uint4 w = philox_rk(make_uint4(u * NC + j, ring, 0u, 0u), rk);
        box_muller(w.x, w.y, n[4 * j], n[4 * j + 1]);
        box_muller(w.z, w.w, n[4 * j + 2], n[4 * j + 3]);
    }
}

// In-place segment kernel, for rings too long for the warp-specialised kernel's three
// buffers (one realisation per CTA, one ring buffer).  Every ring of one segment of one
// chain: the recursion for the thread's units (tables read once per unit), the coefficients
// into shared memory, the C2R FFT in place, the ring to HBM.  The states of all but UPT - PARK
// of each thread's units live in shared memory (loaded for their step, stored after it),
// which keeps the registers of the recursion and of the FFT free of spills.  LG = log2 Nc of a fixed-size high-radix
// FFT, or 0 for the runtime-size radix-4 one; PARK = units per thread parked (the last ones).
template <class Real, class TabT, int M, int UPT, int LG, int PARK>
__global__ void __launch_bounds__(1024, 1) segment_kernel(SampleParams P)
{
    using C = cplx<Real>;
    constexpr int G = kG<M>;
    constexpr int ROW = step_row(M);
    constexpr int EPT = UPT * G;          // complex FFT points per thread
    constexpr int UP = UPT - PARK;        // units whose state stays in registers during the FFT
    constexpr int NU = unit_vals(M), NC = unit_calls(M);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint2 rk[10];              // Philox round keys of the CTA's realisation

    const Segment sg = P.segs[blockIdx.y];
    const int r0 = blockIdx.x;
    const int c = sg.chain;
    const int nt = blockDim.x, tid = threadIdx.x;
    const int Nc = P.Nc;
    const int n_units = P.n_units;
    const size_t mp = P.n_modes_pad;
    const Real* anc = (const Real*)P.anc;
    const bool has_right = sg.right >= 0;

    // shared memory: the ring buffer, then the parked states [PARK][nt][NU]
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    Real* park = reinterpret_cast<Real*>(buf0 + Nc);
    const C* twp = (const C*)P.tw;
    const C* pre = (const C*)P.pre;
    if (tid < 10) {
        const uint64_t key = P.seed + (uint64_t)r0;
        rk[tid] = make_uint2((uint32_t)key + (uint32_t)tid * 0x9E3779B9u, (uint32_t)(key >> 32) + (uint32_t)tid * 0xBB67AE85u);
    }
    // right-anchor states are read from the scratch ([slot][2M])
    const Real* xrg = anc + aoff<M>(P, c, r0, has_right ? sg.right : 0, 0, 0);

    // states: units i < UP in registers, the others in the park area ([PARK][nt][NU]) between
    // their steps
    Real xreg[UP > 0 ? UP : 1][NU];
#pragma unroll
    for (int i = 0; i < UPT; ++i) {
        const int u = tid + i * nt;
        Real v[NU];
#pragma unroll
        for (int k = 0; k < NU; ++k) v[k] = 0;
        if (u < n_units) VecN<Real, NU>::ldg(anc + aoff<M>(P, c, r0, sg.left, 0, G * u), v);
        if (i < UP) {
#pragma unroll
            for (int k = 0; k < NU; ++k) xreg[i < UP ? i : 0][k] = v[k];
        } else {
            VecN<Real, NU>::st(park + ((size_t)(i - UP) * nt + tid) * NU, v);
        }
    }
    __syncthreads();

    const TabT* steps = (const TabT*)(c == 0 ? P.steps[0] : P.steps[1]);
    for (int pos = sg.p0; pos < sg.p1; ++pos) {
        const int ring = c == 0 ? P.k0 - pos : P.k0 + pos;
        const TabT* tb = steps + (size_t)pos * mp * ROW;
#pragma unroll
        for (int i = 0; i < UPT; ++i) {
            const int u = tid + i * nt;
            if (u >= n_units) continue;
            Real x[NU];
            Real* pk = park + ((size_t)(i - UP) * nt + tid) * NU;
            if (i < UP) {
#pragma unroll
                for (int k = 0; k < NU; ++k) x[k] = xreg[i < UP ? i : 0][k];
            } else {
                VecN<Real, NU>::ld(pk, x);
            }
            if (pos > sg.p0) {
                Real ta[G][ROW];
#pragma unroll
                for (int g = 0; g < G; ++g) load_row<Real, TabT, ROW>(tb + (size_t)(G * u + g) * ROW, ta[g]);
                Real nr[NU];
                unit_normals_rk<Real, NC>(rk, (uint32_t)u, (uint32_t)ring, nr);
                Real xr[NU];
                if (has_right) VecN<Real, NU>::ldg(xrg + (size_t)G * u * 2 * M, xr);
#pragma unroll
                for (int g = 0; g < G; ++g)
#pragma unroll
                    for (int part = 0; part < 2; ++part) {
                        Real(&xs)[M] = *reinterpret_cast<Real(*)[M]>(&x[g * 2 * M + part * M]);
                        const Real* xi = nr + g * 2 * M + part * M;
                        if (g == 0 && part == 1 && u == 0) {
                            // slot 0, second part: the Nyquist chain (mode Nc, own table row)
                            Real tn[ROW];
                            load_row<Real, TabT, ROW>(tb + (size_t)Nc * ROW, tn);
                            if (has_right) step_state<Real, M, true>(tn, xs, xi, xr + M);
                            else step_state<Real, M, false>(tn, xs, xi, nullptr);
                        } else if (has_right) {
                            step_state<Real, M, true>(ta[g], xs, xi, xr + g * 2 * M + part * M);
                        } else {
                            step_state<Real, M, false>(ta[g], xs, xi, nullptr);
                        }
                    }
                if (i < UP) {
#pragma unroll
                    for (int k = 0; k < NU; ++k) xreg[i < UP ? i : 0][k] = x[k];
                } else {
                    VecN<Real, NU>::st(pk, x);
                }
            }
            // the unit's coefficients of this ring (slot 0's imaginary part = Nyquist)
            put_unit<C, Real, M>(buf0, u, x);
        }
        __syncthreads();
        if (!(c == 1 && pos == 0)) {  // the start ring is written by the northern chain
            Real* dst = (Real*)P.out + ((size_t)r0 * P.n_theta + ring) * (size_t)P.n_phi;
            if constexpr (LG > 0) {
                hr_c2r_inplace<C, LG, EPT>(buf0, (const C*)P.tw3, pre, reinterpret_cast<C*>(dst));
            } else {
                c2r_rings_inplace<C, EPT>(buf0, 1, P.lgNc, twp, pre);
                store_ring<Real>(dst, buf0, Nc, tid, nt);
            }
        }
        __syncthreads();  // the buffer is rewritten by the next ring
    }
}

// ------------------------------------------------------------------ warp-specialised
// Named hardware barriers (bar.sync waits, bar.arrive does not); counts are thread counts,
// multiples of 32, and every participating thread executes the same sequence.
__device__ __forceinline__ void bar_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void bar_arrive(int id, int n) { asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory"); }

constexpr int kBarFull = 1;   // + buffer index: coefficients of a ring are ready
constexpr int kBarEmpty = 3;  // + buffer index: the FFT group is done with a buffer
constexpr int kBarFft = 5;    // FFT group internal

// general size (runtime log2 Nc)
template <class C, int RP, bool FIRST, bool LAST>
__device__ __forceinline__ void grp_pass_rt(const C* __restrict__ src, C* __restrict__ dst, int R, int lgNc, int Ns,
                                            const C* __restrict__ twp, const C* __restrict__ pre, RingOut<C> gout,
                                            int ftid, int nf)
{
    const int Nc = 1 << lgNc;
    constexpr int LR = RP == 4 ? 2 : 1;
    const int lgnb = lgNc - LR;
    const int nb = 1 << lgnb;
    const int total = R << lgnb;
    for (int b = ftid; b < total; b += nf) {
        const int r = b >> lgnb, j = b & (nb - 1);
        const C* S = src + (r << lgNc);
        C v[RP];
        int kk = 0;
        if (FIRST) {
#pragma unroll
            for (int i = 0; i < RP; ++i) v[i] = c2r_pack(S, j + i * nb, Nc, pre);
        } else {
            kk = j & (Ns - 1);
#pragma unroll
            for (int i = 0; i < RP; ++i) v[i] = S[j + i * nb];
#pragma unroll
            for (int i = 1; i < RP; ++i) v[i] = cmul(v[i], __ldg(twp + (i - 1) * Ns + kk));
        }
        dft<C, RP>(v);
        const int idx = ((j - kk) << LR) + kk;
        if (LAST) {
            C* D = gout[r] + idx;
#pragma unroll
            for (int a = 0; a < RP; ++a) __stcs(D + a * Ns, v[a]);
        } else {
            C* D = dst + (r << lgNc) + idx;
#pragma unroll
            for (int a = 0; a < RP; ++a) D[a * Ns] = v[a];
        }
    }
}

template <class C>
__device__ __forceinline__ void grp_c2r_rt(C* buf0, C* buf1, int R, int lgNc, const C* twp, const C* pre,
                                           RingOut<C> gout, int ftid, int nf)
{
    const int Nc = 1 << lgNc;
    C* src = buf0;
    C* dst = buf1;
    int Ns = 1, off = 0;
    bool first = true;
    while (Ns < Nc) {
        const int RP = pass_radix(lgNc, Ns);
        const bool last = Ns * RP == Nc;
        if (RP == 4) {
            if (first) {
                if (last) grp_pass_rt<C, 4, true, true>(src, dst, R, lgNc, Ns, twp + off, pre, gout, ftid, nf);
                else grp_pass_rt<C, 4, true, false>(src, dst, R, lgNc, Ns, twp + off, pre, gout, ftid, nf);
            } else {
                if (last) grp_pass_rt<C, 4, false, true>(src, dst, R, lgNc, Ns, twp + off, pre, gout, ftid, nf);
                else grp_pass_rt<C, 4, false, false>(src, dst, R, lgNc, Ns, twp + off, pre, gout, ftid, nf);
            }
        } else {
            if (first) {
                if (last) grp_pass_rt<C, 2, true, true>(src, dst, R, lgNc, Ns, twp + off, pre, gout, ftid, nf);
                else grp_pass_rt<C, 2, true, false>(src, dst, R, lgNc, Ns, twp + off, pre, gout, ftid, nf);
            } else {
                if (last) grp_pass_rt<C, 2, false, true>(src, dst, R, lgNc, Ns, twp + off, pre, gout, ftid, nf);
                else grp_pass_rt<C, 2, false, false>(src, dst, R, lgNc, Ns, twp + off, pre, gout, ftid, nf);
            }
        }
        if (!first) off += (RP - 1) * Ns;
        Ns *= RP;
        first = false;
        if (!last) bar_sync(kBarFft, nf);
        C* t = src;
        src = dst;
        dst = t;
    }
}

// ---- high-radix plan (hr_passes / hr_bits): passes of radix up to 16 held in registers.
// Between passes the rings sit in shared memory in an XOR-swizzled order, element e at
// e ^ ((e >> 4) & 15), so that the strided stores of the early passes and the unit-stride
// loads of the next pass are both free of bank conflicts (hr_swz).  The coefficient buffer
// the producer fills (first pass input) is in natural order; the last pass writes HBM.
// PAIR: FP32 passes of radix up to 8 take two neighbouring butterflies per thread (below); the
// persistent batch kernel, whose register budget is tighter, keeps one
template <class C, int LGNC, int PASS, bool PAIR = true>
__device__ __forceinline__ void hr_pass(const C* __restrict__ src, C* __restrict__ dst, int R,
                                        const C* __restrict__ tw2, const C* __restrict__ pre, RingOut<C> gout,
                                        int ftid, int nf)
{
    constexpr int Nc = 1 << LGNC;
    constexpr int LR = hr_bits(LGNC, PASS), RP = 1 << LR;
    constexpr int Ns = 1 << hr_lgns(LGNC, PASS);
    constexpr bool FIRST = PASS == 0, LAST = PASS == hr_passes(LGNC) - 1;
    constexpr int LGNB = LGNC - LR, nb = 1 << LGNB;
    const C* twp = tw2 + hr_off(LGNC, PASS);
    const int total = R << LGNB;
    if constexpr (PAIR && !FIRST && sizeof(C) == 8 && RP <= 8) {
        // FP32 last pass of radix up to 8 (two radix-16 butterflies would not fit the register
        // budget: 4096-point rings measured 12 % slower): a thread takes butterflies j and j + 1
        // (j even), whose swizzled inputs share one 16-byte pair (hr_swz(j + 1) = hr_swz(j) ^ 1)
        // and whose twiddles and outputs are neighbours (Ns >= 2): 16-byte shared loads,
        // twiddle loads and streaming HBM stores
        static_assert(Ns >= 2 && nb >= 2, "neighbouring butterflies share a block");
        for (int b = 2 * ftid; b < total; b += 2 * nf) {
            const int r = b >> LGNB, j = b & (nb - 1);
            const C* S = src + (r << LGNC);
            const int kk = j & (Ns - 1);
            C v0[RP], v1[RP];
#pragma unroll
            for (int i = 0; i < RP; ++i) {
                const int f = hr_swz(j + i * nb);
                const float4 w = reinterpret_cast<const float4*>(S)[f >> 1];
                const C lo = cmk<C>(w.x, w.y), hi = cmk<C>(w.z, w.w);
                v0[i] = (f & 1) ? hi : lo;
                v1[i] = (f & 1) ? lo : hi;
            }
#pragma unroll
            for (int i = 1; i < RP; ++i) {
                const float4 t = __ldg(reinterpret_cast<const float4*>(twp + (i - 1) * Ns + kk));
                v0[i] = cmul(v0[i], cmk<C>(t.x, t.y));
                v1[i] = cmul(v1[i], cmk<C>(t.z, t.w));
            }
            dft<C, RP>(v0);
            dft<C, RP>(v1);
            const int idx = ((j - kk) << LR) + kk;
            if constexpr (LAST) {
                C* D = gout[r] + idx;
#pragma unroll
                for (int a = 0; a < RP; ++a)
                    __stcs(reinterpret_cast<float4*>(D + a * Ns), make_float4(v0[a].x, v0[a].y, v1[a].x, v1[a].y));
            } else {
                // hr_swz(idx + a Ns + 1) = hr_swz(idx + a Ns) ^ 1 (idx + a Ns even)
                float4* D = reinterpret_cast<float4*>(dst + (r << LGNC));
#pragma unroll
                for (int a = 0; a < RP; ++a) {
                    const int f = hr_swz(idx + a * Ns);
                    D[f >> 1] = (f & 1) ? make_float4(v1[a].x, v1[a].y, v0[a].x, v0[a].y)
                                        : make_float4(v0[a].x, v0[a].y, v1[a].x, v1[a].y);
                }
            }
        }
        return;
    }
    for (int b = ftid; b < total; b += nf) {
        const int r = b >> LGNB, j = b & (nb - 1);
        const C* S = src + (r << LGNC);
        C v[RP];
        int kk = 0;
        if constexpr (FIRST) {
            // C2R packing on load: element i is slot s = j + i nb (slot 0 = (X_0, X_Nc))
            {
                const C a = S[j], bb = cconj(S[(Nc - j) & (Nc - 1)]);
                const C g = cadd(cadd(a, bb), cmuli(cmul(__ldg(pre + j), csub(a, bb))));
                const C z0 = cmk<C>(a.x + a.y, a.x - a.y);
                v[0] = j == 0 ? z0 : g;
            }
#pragma unroll
            for (int i = 1; i < RP; ++i) {
                const int sidx = j + i * nb;
                const C a = S[sidx], bb = cconj(S[Nc - sidx]);
                v[i] = cadd(cadd(a, bb), cmuli(cmul(__ldg(pre + sidx), csub(a, bb))));
            }
        } else {
            kk = j & (Ns - 1);
#pragma unroll
            for (int i = 0; i < RP; ++i) v[i] = S[hr_swz(j + i * nb)];
#pragma unroll
            for (int i = 1; i < RP; ++i) v[i] = cmul(v[i], __ldg(twp + (i - 1) * Ns + kk));
        }
        dft<C, RP>(v);
        const int idx = ((j - kk) << LR) + kk;
        if constexpr (LAST) {
            C* D = gout[r] + idx;
#pragma unroll
            for (int a = 0; a < RP; ++a) __stcs(D + a * Ns, v[a]);
        } else {
            C* D = dst + (r << LGNC);
#pragma unroll
            for (int a = 0; a < RP; ++a) D[hr_swz(idx + a * Ns)] = v[a];
        }
    }
}

template <class C, int LGNC, int PASS = 0, bool PAIR = true>
__device__ __forceinline__ void hr_c2r_fixed(C* src, C* dst, int R, const C* tw2, const C* pre, RingOut<C> gout,
                                             int ftid, int nf)
{
    hr_pass<C, LGNC, PASS, PAIR>(src, dst, R, tw2, pre, gout, ftid, nf);
    if constexpr (PASS + 1 < hr_passes(LGNC)) {
        bar_sync(kBarFft, nf);
        hr_c2r_fixed<C, LGNC, PASS + 1, PAIR>(dst, src, R, tw2, pre, gout, ftid, nf);
    }
}

// high-radix fixed-size FFTs for log2 Nc in [LO, HI], the runtime-size radix-4 one otherwise
template <class C, int LO, int HI, bool PAIR = true>
__device__ __forceinline__ void hr_c2r(int lgNc, C* b0, C* b1, int R, const C* twp, const C* tw2, const C* pre,
                                       RingOut<C> gout, int ftid, int nf)
{
    if constexpr (LO <= HI) {
        if (lgNc == LO) {
            hr_c2r_fixed<C, LO, 0, PAIR>(b0, b1, R, tw2, pre, gout, ftid, nf);
            return;
        }
        hr_c2r<C, LO + 1, HI, PAIR>(lgNc, b0, b1, R, twp, tw2, pre, gout, ftid, nf);
    } else {
        grp_c2r_rt<C>(b0, b1, R, lgNc, twp, pre, gout, ftid, nf);
    }
}

// log2 Nc range the warp-specialised kernel with UPT units per producer thread meets: the
// launch configurations use UPT only while 16 UPT < units <= 512 UPT (units = Nc / unit_slots)
__host__ __device__ constexpr int ws_lg_lo(int UPT, int M)
{
    return UPT == 1 ? 2 : (UPT == 2 ? 6 : UPT == 4 ? 7 : 8) + (unit_slots(M) == 2);
}
__host__ __device__ constexpr int ws_lg_hi(int UPT, int M)
{
    return ((UPT == 1 ? 9 : UPT == 2 ? 10 : UPT == 4 ? 11 : 12) + (unit_slots(M) == 2)) < 12
               ? ((UPT == 1 ? 9 : UPT == 2 ? 10 : UPT == 4 ? 11 : 12) + (unit_slots(M) == 2))
               : 12;
}

// ---- iso-latitude grids with ring-dependent longitudes (the paper's Sec. 1 remark)
// e^{i pi x} for a real x given in half-turns, reduced to [-1, 1) in FP64 first so that the
// phase of a large multiple of a small offset keeps full accuracy
template <class Real> __device__ __forceinline__ cplx<Real> cis_halfturns(double x)
{
    x -= 2.0 * floor(0.5 * x + 0.5);
    Real sn, cs;
    if constexpr (sizeof(Real) == 4) sincospif((float)x, &sn, &cs);
    else sincospi(x, &sn, &cs);
    return cmk<cplx<Real>>(cs, sn);
}

// e^{2 pi i a / n} for integers 0 <= a < n: the fraction 2a / n in the recursion precision (exact
// for a power-of-two n, within half an ulp otherwise), then sincospi
template <class Real> __device__ __forceinline__ cplx<Real> ring_phase(int a, int n)
{
    Real sn, cs;
    if constexpr (sizeof(Real) == 4) sincospif(2.0f * (float)a / (float)n, &sn, &cs);
    else sincospi(2.0 * (double)a / (double)n, &sn, &cs);
    return cmk<cplx<Real>>(cs, sn);
}

// Ring `ring` of n = 2 Ncp points from phi0 = h pi: the C2R input X' (slot 0 = (Y_0, Y_Ncp),
// slot q = Y_q) of the real field T(phi) = sum_{|m| <= M} c_m e^{i m phi} at its points, where
// c_0 = g_0, c_{+-m} = g_m, conj g_m (0 < m < M) and c_{+-M} = Re g_M / 2 (the Nyquist mode's real
// part); Y_q = sum over m = q (mod n) of c_m e^{i m phi0} (modes above the ring's own Nyquist
// alias onto it).  B: the ring's coefficients (slot 0 = (g_0, Re g_M), slot m = g_m) at stride
// Nc per realisation; W: the folded rings at stride Ncp.
template <class Real>
__device__ __forceinline__ void ring_fold(const cplx<Real>* B, cplx<Real>* W, int R, int Nc, int n, double h, int ftid,
                                          int nf)
{
    using C = cplx<Real>;
    const int Ncp = n / 2, M = Nc;
    // e^{i m phi0} along m = m0 + k n: exact (FP64-reduced) every 16 terms, products by
    // e^{i n phi0} between, so that rounding grows over at most 16 products
    const C step = cis_halfturns<Real>(h * n);
    for (int idx = ftid; idx < R * (Ncp + 1); idx += nf) {
        const int r = idx / (Ncp + 1), q = idx - r * (Ncp + 1);
        const C* X = B + (size_t)r * Nc;
        C acc = cmk<C>(0, 0);
        C e = cmk<C>(1, 0);
        int k = 0;
        for (int m = q; m <= M; m += n, ++k) {  // m >= 0
            e = (k & 15) == 0 ? cis_halfturns<Real>(h * m) : cmul(e, step);
            const C g = m == 0 ? cmk<C>(X[0].x, 0) : (m == M ? cmk<C>((Real)0.5 * X[0].y, 0) : X[m]);
            acc = cadd(acc, m == 0 ? g : cmul(g, e));
        }
        k = 0;
        for (int m = q == 0 ? n : n - q; m <= M; m += n, ++k) {  // the conjugate terms, -m < 0
            e = (k & 15) == 0 ? cis_halfturns<Real>(h * m) : cmul(e, step);
            const C g = m == M ? cmk<C>((Real)0.5 * X[0].y, 0) : X[m];
            acc = cadd(acc, cconj(cmul(g, e)));
        }
        C* Y = W + (size_t)r * Ncp;
        if (q == 0) Y[0].x = acc.x;
        else if (q == Ncp) Y[0].y = acc.x;
        else Y[q] = acc;
    }
}

// C2R of R rings of n = 2 Ncp points (Ncp = 2^lg >= 2) from their folded input in src (stride
// Ncp), ping-ponging with dst, last pass to gout: radix-4 Stockham passes (radix 2 last when lg
// is odd) with the twiddles computed, the packing factors e^{2 pi i s / n} = pre[s pstride] from
// the plan's table of its full ring.
template <class C>
__device__ __forceinline__ void ragged_c2r(C* src, C* dst, int R, int lg, const C* __restrict__ pre, int pstride,
                                           RingOut<C> gout, int ftid, int nf)
{
    using Real = decltype(C::x);
    const int Nc = 1 << lg;
    int Ns = 1;
    bool first = true;
    while (Ns < Nc) {
        const int RP = Nc / Ns >= 4 ? 4 : 2, LR = RP == 4 ? 2 : 1;
        const bool last = Ns * RP == Nc;
        const int lgnb = lg - LR, nb = 1 << lgnb, total = R << lgnb;
        for (int b = ftid; b < total; b += nf) {
            const int r = b >> lgnb, j = b & (nb - 1);
            const C* S = src + ((size_t)r << lg);
            C v[4];
            int kk = 0;
            if (first) {
                for (int i = 0; i < RP; ++i) {
                    const int sidx = j + i * nb;
                    if (sidx == 0) {
                        v[i] = cmk<C>(S[0].x + S[0].y, S[0].x - S[0].y);
                    } else {
                        const C a = S[sidx], bb = cconj(S[Nc - sidx]);
                        v[i] = cadd(cadd(a, bb), cmuli(cmul(__ldg(pre + (size_t)sidx * pstride), csub(a, bb))));
                    }
                }
            } else {
                kk = j & (Ns - 1);
                for (int i = 0; i < RP; ++i) v[i] = S[j + i * nb];
                for (int i = 1; i < RP; ++i) v[i] = cmul(v[i], ring_phase<Real>(i * kk, Ns * RP));
            }
            if (RP == 4) dft4(v);
            else dft2(v[0], v[1]);
            const int idx = ((j - kk) << LR) + kk;
            if (last) {
                C* D = gout[r] + idx;
                for (int a = 0; a < RP; ++a) __stcs(D + a * Ns, v[a]);
            } else {
                C* D = dst + ((size_t)r << lg) + idx;
                for (int a = 0; a < RP; ++a) D[a * Ns] = v[a];
            }
        }
        Ns *= RP;
        first = false;
        if (!last) bar_sync(kBarFft, nf);
        C* t = src;
        src = dst;
        dst = t;
    }
}

// Rings of an even point count n that is not a power of two (HEALPix polar caps): the real
// synthesis T_j = Y_0 + (-1)^j Y_{n/2} + 2 sum_{0<q<n/2} Re(Y_q e^{2 pi i q j / n}) of the folded
// input directly, O(n^2) per ring; the phases e^{2 pi i q j / n} exact (integer reduction of
// q j mod n) every 16 terms and products by e^{2 pi i j / n} between.
template <class Real>
__device__ __forceinline__ void ring_direct(const cplx<Real>* W, int R, int n, cplx<Real>* gbase, size_t gstride,
                                            int ftid, int nf)
{
    using C = cplx<Real>;
    const int Ncp = n / 2;
    for (int idx = ftid; idx < R * n; idx += nf) {
        const int r = idx / n, j = idx - r * n;
        const C* Y = W + (size_t)r * Ncp;
        Real t = Y[0].x + ((j & 1) ? -Y[0].y : Y[0].y);
        const C w = ring_phase<Real>(j, n);
        C e = w;
        for (int q = 1; q < Ncp; ++q) {
            if ((q & 15) == 0) e = ring_phase<Real>((int)(((long long)q * j) % n), n);
            t += (Real)2 * (Y[q].x * e.x - Y[q].y * e.y);
            e = cmul(e, w);
        }
        reinterpret_cast<Real*>(gbase + (size_t)r * gstride)[j] = t;
    }
}

// A ring whose point count or offset differs from the plan's full ring: fold, then the
// runtime-size C2R (n a power of two) or the direct synthesis (other even n).  Not inlined, so
// that the warp-specialised bodies keep their register allocation for the full-ring path.
template <class Real>
__device__ __noinline__ void ragged_ring(cplx<Real>* B, cplx<Real>* W, int R, int Nc, int n, double h,
                                         const cplx<Real>* pre, int n_phi, cplx<Real>* gbase, size_t gstride,
                                         int ftid, int nf)
{
    ring_fold<Real>(B, W, R, Nc, n, h, ftid, nf);
    bar_sync(kBarFft, nf);
    if (n & (n - 1)) {
        ring_direct<Real>(W, R, n, gbase, gstride, ftid, nf);
        return;
    }
    int lg = 0;
    while ((2 << lg) < n) ++lg;
    ragged_c2r<cplx<Real>>(W, B, R, lg, pre, n_phi / n, RingOut<cplx<Real>>{gbase, gstride}, ftid, nf);
}

// Warp-specialised segment kernel.  Threads [0, NP) are the producer group: the recursion of
// ring k (state in registers, units tid, tid + NP, ...) into coefficient buffer B[k & 1].
// Threads [NP, NP + NF) are the FFT group: the C2R FFT of ring k from B[k & 1] (with W as
// the second ping-pong buffer), last pass straight to HBM.  Handoff per ring:
//   producer: (k >= 2: sync EMPTY[k&1]) produce; arrive FULL[k&1]; after the last ring it
//             syncs the two outstanding EMPTY barriers
//   FFT:      sync FULL[k&1]; FFT; arrive EMPTY[k&1]
// Every FULL/EMPTY barrier counts NP + NF threads; the FFT passes use a group barrier.
// RINGS: the request may have ring-dependent longitudes (single-request launches; batches never do).
// CG: the anchor states were written by the same launch (read through L2, not the read-only path).
// PAIR: see hr_pass (false in the persistent batch kernels).
template <class Real, class TabT, int M, int UPT, int RMAX, bool RINGS = true, bool CG = false, bool PAIR = true>
__device__ __forceinline__ void ws_body(const SampleParams& P, int seg_index, int group)
{
    using C = cplx<Real>;
    constexpr int G = kG<M>;
    constexpr int ROW = step_row(M);
    constexpr int RB = RMAX < SMERF_RB ? RMAX : SMERF_RB;  // realisations whose noise is drawn together
    constexpr int NU = unit_vals(M), NC = unit_calls(M);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint2 rk[RMAX][10];

    const Segment sg = P.segs[seg_index];
    const int r0 = group * RMAX;
    const int R = min(RMAX, P.n_samples - r0);
    const int c = sg.chain;
    const int nt = blockDim.x, tid = threadIdx.x;
    const int NP = P.np, NF = nt - P.np;
    const int Nc = P.Nc;
    const int n_units = P.n_units;
    const size_t mp = P.n_modes_pad;
    const Real* anc = (const Real*)P.anc;
    const bool has_right = sg.right >= 0;
    const int nrings = sg.p1 - sg.p0;

    C* bufs = reinterpret_cast<C*>(smem_raw);  // B0, B1, W: RMAX * Nc each
    C* W = bufs + (size_t)2 * RMAX * Nc;
    Real* xRs = reinterpret_cast<Real*>(bufs + (size_t)3 * RMAX * Nc);
    const C* twp = (const C*)P.tw;
    const C* pre = (const C*)P.pre;
    if (tid < RMAX * 10) {
        const int r = tid / 10, i = tid % 10;
        const uint64_t key = P.seed + (uint64_t)(r0 + r);
        rk[r][i] = make_uint2((uint32_t)key + (uint32_t)i * 0x9E3779B9u, (uint32_t)(key >> 32) + (uint32_t)i * 0xBB67AE85u);
    }
    if (has_right) {
        const int per = 2 * M * Nc;
        for (int idx = 4 * tid; idx < R * per; idx += 4 * nt) {
            const int r = idx / per, rest = idx - r * per;
            Real v[4];
            VecN<Real, 4>::template ld_anchor<CG>(anc + aoff<M>(P, c, r0 + r, sg.right, 0, 0) + rest, v);
            Vec4<Real>::st(xRs + idx, v);
        }
    }
    __syncthreads();

    if (tid < NP) {
        // ------------------------------------------------ producer group
        Real x[UPT][RMAX][NU];
#pragma unroll
        for (int i = 0; i < UPT; ++i) {
            const int u = tid + i * NP;
#pragma unroll
            for (int r = 0; r < RMAX; ++r) {
                if (u < n_units && r < R) {
                    VecN<Real, NU>::template ld_anchor<CG>(anc + aoff<M>(P, c, r0 + r, sg.left, 0, G * u), x[i][r]);
                } else {
#pragma unroll
                    for (int k = 0; k < NU; ++k) x[i][r][k] = 0;
                }
            }
        }
        const TabT* steps = (const TabT*)(c == 0 ? P.steps[0] : P.steps[1]);
        for (int k = 0; k < nrings + 2; ++k) {
            if (k >= 2) bar_sync(kBarEmpty + (k & 1), nt);
            if (k >= nrings) continue;
            const int pos = sg.p0 + k;
            const int ring = c == 0 ? P.k0 - pos : P.k0 + pos;
            C* B = bufs + (size_t)(k & 1) * RMAX * Nc;
            if (k > 0) {
                const TabT* tb = steps + (size_t)pos * mp * ROW;
#pragma unroll
                for (int i = 0; i < UPT; ++i) {
                    const int u = tid + i * NP;
                    if (u >= n_units) continue;
                    if constexpr (M == 3) {
                        // p = 3 (one realisation per CTA): the unit's normals first, then one
                        // 24-value table row at a time, so that two rows are never live together
                        static_assert(RMAX == 1, "p = 3 builds hold one realisation per CTA");
                        Real nr[NU];
                        unit_normals_multi<Real, 1, NC>(rk, (uint32_t)u, (uint32_t)ring, *reinterpret_cast<Real(*)[1][NU]>(nr));
#pragma unroll
                        for (int g = 0; g < G; ++g) {
                            Real tg[ROW];
                            load_row<Real, TabT, ROW>(tb + (size_t)(G * u + g) * ROW, tg);
#pragma unroll
                            for (int part = 0; part < 2; ++part) {
                                Real(&xs)[M] = *reinterpret_cast<Real(*)[M]>(&x[i][0][g * 2 * M + part * M]);
                                const Real* xi = nr + g * 2 * M + part * M;
                                Real xr[M];
                                if (has_right) {
#pragma unroll
                                    for (int q = 0; q < M; ++q) xr[q] = xRs[(size_t)(G * u + g) * 2 * M + part * M + q];
                                }
                                if (g == 0 && part == 1 && u == 0) {
                                    // slot 0, second part: the Nyquist chain (mode Nc, own table row)
                                    Real tn[ROW];
                                    load_row<Real, TabT, ROW>(tb + (size_t)Nc * ROW, tn);
                                    if (has_right) step_state<Real, M, true>(tn, xs, xi, xr);
                                    else step_state<Real, M, false>(tn, xs, xi, nullptr);
                                } else if (has_right) {
                                    step_state<Real, M, true>(tg, xs, xi, xr);
                                } else {
                                    step_state<Real, M, false>(tg, xs, xi, nullptr);
                                }
                            }
                        }
                        continue;
                    }
                    Real ta[G][ROW];
#pragma unroll
                    for (int g = 0; g < G; ++g) load_row<Real, TabT, ROW>(tb + (size_t)(G * u + g) * ROW, ta[g]);
#pragma unroll
                    for (int rb = 0; rb < RMAX; rb += RB) {
                        if (rb >= R) continue;
                        // normals of realisations rb .. rb + RB - 1 (those past R are not used)
                        Real nrb[RB][NU];
                        unit_normals_multi<Real, RB, NC>(rk + rb, (uint32_t)u, (uint32_t)ring, nrb);
#pragma unroll
                    for (int r = rb; r < rb + RB; ++r) {
                        if (r >= R) continue;
                        const Real* nr = nrb[r - rb];
                        Real xr[NU];
                        if (has_right) VecN<Real, NU>::ld(xRs + ((size_t)r * Nc + G * u) * 2 * M, xr);
#pragma unroll
                        for (int g = 0; g < G; ++g)
#pragma unroll
                            for (int part = 0; part < 2; ++part) {
                                Real(&xs)[M] = *reinterpret_cast<Real(*)[M]>(&x[i][r][g * 2 * M + part * M]);
                                const Real* xi = nr + g * 2 * M + part * M;
                                if (g == 0 && part == 1 && u == 0) {
                                    // slot 0, second part: the Nyquist chain (mode Nc, own table row)
                                    Real tn[ROW];
                                    load_row<Real, TabT, ROW>(tb + (size_t)Nc * ROW, tn);
                                    if (has_right) step_state<Real, M, true>(tn, xs, xi, xr + M);
                                    else step_state<Real, M, false>(tn, xs, xi, nullptr);
                                } else if (has_right) {
                                    step_state<Real, M, true>(ta[g], xs, xi, xr + g * 2 * M + part * M);
                                } else {
                                    step_state<Real, M, false>(ta[g], xs, xi, nullptr);
                                }
                            }
                    }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < UPT; ++i) {
                const int u = tid + i * NP;
                if (u >= n_units) continue;
#pragma unroll
                for (int r = 0; r < RMAX; ++r) {
                    if (r >= R) continue;
                    put_unit<C, Real, M>(B + (size_t)r * Nc, u, x[i][r]);
                }
            }
            __threadfence_block();
            bar_arrive(kBarFull + (k & 1), nt);
        }
    } else {
        // ------------------------------------------------ FFT group
        const int ftid = tid - NP;
        for (int k = 0; k < nrings; ++k) {
            bar_sync(kBarFull + (k & 1), nt);
            const int pos = sg.p0 + k;
            const int ring = c == 0 ? P.k0 - pos : P.k0 + pos;
            C* B = bufs + (size_t)(k & 1) * RMAX * Nc;
            if (!(c == 1 && pos == 0)) {  // the start ring is written by the northern chain
                RingOut<C> gout{(C*)((Real*)P.out + ((size_t)r0 * P.n_theta + ring) * (size_t)P.n_phi),
                                (size_t)P.n_theta * (size_t)(P.n_phi / 2)};
                int n_ring = P.n_phi;
                double h_ring = 0.0;
                if (RINGS && P.ring_n) {  // ring-dependent longitudes: the rings lie back to back
                    n_ring = P.ring_n[ring];
                    h_ring = P.ring_h[ring];
                    gout = RingOut<C>{(C*)((Real*)P.out + (size_t)r0 * P.ring_total + P.ring_off[ring]),
                                      (size_t)(P.ring_total / 2)};
                }
                if (RINGS && (n_ring != P.n_phi || h_ring != 0.0)) {
                    ragged_ring<Real>(B, W, R, Nc, n_ring, h_ring, pre, P.n_phi, gout.base, gout.stride, ftid, NF);
                } else if (sizeof(Real) == 4 && !P.fft_r4) {
                    if constexpr (sizeof(Real) == 4)
                        hr_c2r<C, ws_lg_lo(UPT, M), ws_lg_hi(UPT, M), PAIR>(P.lgNc, B, W, R, twp, (const C*)P.tw2, pre, gout,
                                                                       ftid, NF);
                } else {
                    grp_c2r_rt<C>(B, W, R, P.lgNc, twp, pre, gout, ftid, NF);
                }
            }
            bar_arrive(kBarEmpty + (k & 1), nt);
        }
    }
}

template <class Real, class TabT, int M, int UPT, int RMAX, int MINB>
__global__ void __launch_bounds__(ws_max_threads(MINB, M), MINB) segment_ws_kernel(SampleParams P)
{
    ws_body<Real, TabT, M, UPT, RMAX>(P, blockIdx.y, blockIdx.x);
}

// batched: item = (request, segment, realisation group); all requests of a launch share the
// kernel shape (precision, p, n_phi, anchors or not) and hence the launch configuration
template <class Real, class TabT, int M, int UPT, int RMAX, int MINB>
__global__ void __launch_bounds__(ws_max_threads(MINB, M), MINB) segment_ws_batched_kernel(const SampleParams* __restrict__ descs,
                                                                 const int4* __restrict__ items)
{
    const int4 it = items[blockIdx.x];
    const SampleParams P = descs[it.x];
    ws_body<Real, TabT, M, UPT, RMAX, false>(P, it.y, it.z);
}

// ---- uneven batches: one persistent launch, or an anchor launch and a persistent launch
// Persistent CTAs (kQueueThreads threads, two per SM, as many as are resident) take items from
// a device queue -- an atomic counter reset before each launch.  The queue holds every
// request's anchor items first (request, block of kQueueThreads units, realisation, and
// w = -1 - (p << 4 | chain)), then the segment items (request, segment, realisation group,
// shape w >= 0), each list largest request first.  An anchor item walks its units' start
// states and anchors (anchor_body) and then adds one to its request's counter of finished
// anchor items; a segment item first waits until that counter shows all of its request's
// anchor items, then runs the warp-specialised body of its shape (p and the build: units per
// producer thread, realisations per CTA, queue_build), so requests of different grids, spectra
// and p share the launch and the anchors of later requests overlap the segments of earlier
// ones.  Every anchor item is claimed before any segment item and runs without waiting, so a
// waiting CTA only waits for items that resident CTAs are running; the wait is still bounded
// (about a second, kQueueWaitNs), after which it records SMERF_ETIMEOUT's cause in the
// launch's status word, skips the item, and makes every later wait give up at once.
//
// ctl[0]: queue head; ctl[1]: status (0, or 1 once a wait ran out); ctl[2 + i]: finished
// anchor items of request i.

constexpr unsigned long long kQueueWaitNs = 1000000000ull;  // a wait's limit in wall time
constexpr unsigned kQueueWaitPolls = 1u << 22;              // and in polls

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// anchor items of a request: both chains, every realisation, blocks of kQueueThreads units
__host__ __device__ inline int queue_anchor_items(int n_samples, int n_units)
{
    return 2 * n_samples * ((n_units + kQueueThreads - 1) / kQueueThreads);
}

// one thread: wait until *done >= need (bounded); false if the wait ran out or another did
__device__ inline bool wait_anchors(const int* done, int need, int* status)
{
    unsigned long long t0 = 0;
    for (unsigned i = 0; i < kQueueWaitPolls; ++i) {
        if (ld_acquire(done) >= need) return true;
        if (ld_acquire(status) != 0) return false;
        const unsigned long long t = global_ns();
        if (i == 0) t0 = t;
        else if (t - t0 > kQueueWaitNs) break;
        __nanosleep(128);
    }
    atomicCAS(status, 0, 1);
    return false;
}

// an anchor item of the persistent launch (called out of line: its registers stay apart from
// the segment bodies')
template <class Real, class TabT>
__device__ __noinline__ void queue_anchor(const SampleParams* __restrict__ desc, int code, int ub, int r)
{
    const SampleParams P = *desc;
    NoStage h;
    const int u = ub * kQueueThreads + threadIdx.x;
    if ((code >> 4) == 1) anchor_body<Real, TabT, 1>(P, u, r, code & 15, h);
    else anchor_body<Real, TabT, 2>(P, u, r, code & 15, h);
}

template <class Real, class TabT, int SH>
__device__ __forceinline__ void queue_segment(const SampleParams& P, int seg, int grp)
{
    constexpr int M = SH / kQueueBuilds + 1, B = SH % kQueueBuilds;
    ws_body<Real, TabT, M, queue_upt(B), queue_rmax(B), false, true, false>(P, seg, grp);
}

template <class Real, class TabT>
__global__ void __launch_bounds__(kQueueThreads, kQueueMinBlocks) queue_kernel(const SampleParams* __restrict__ descs,
                                                                 const int4* __restrict__ items, int n_items,
                                                                 int* __restrict__ ctl)
{
    // the next item is claimed while the current one runs (s_k[b ^ 1]), hiding the atomic
    __shared__ int s_k[2];
    __shared__ int s_go;
    if (threadIdx.x == 0) s_k[0] = atomicAdd(ctl, 1);
    __syncthreads();
    for (int b = 0;; b ^= 1) {
        const int k = s_k[b];
        if (k >= n_items) return;
        if (threadIdx.x == 0) s_k[b ^ 1] = atomicAdd(ctl, 1);
        const int4 it = items[k];
        if (it.w < 0) {
            queue_anchor<Real, TabT>(descs + it.x, -1 - it.w, it.y, it.z);
            __syncthreads();  // every anchor state of the item is written
            if (threadIdx.x == 0) {
                __threadfence();
                atomicAdd(ctl + 2 + it.x, 1);
            }
        } else {
            const SampleParams P = descs[it.x];
            if (threadIdx.x == 0)
                s_go = wait_anchors(ctl + 2 + it.x, queue_anchor_items(P.n_samples, P.n_units), ctl + 1);
            __syncthreads();
            if (s_go) {
                switch (it.w) {
                    case 0: queue_segment<Real, TabT, 0>(P, it.y, it.z); break;
                    case 1: queue_segment<Real, TabT, 1>(P, it.y, it.z); break;
                    case 2: queue_segment<Real, TabT, 2>(P, it.y, it.z); break;
                    case 3: queue_segment<Real, TabT, 3>(P, it.y, it.z); break;
                    case 4: queue_segment<Real, TabT, 4>(P, it.y, it.z); break;
                    case 5: queue_segment<Real, TabT, 5>(P, it.y, it.z); break;
                    case 6: queue_segment<Real, TabT, 6>(P, it.y, it.z); break;
                    default: queue_segment<Real, TabT, 7>(P, it.y, it.z); break;
                }
            }
        }
        __syncthreads();  // the item's shared buffers and s_go are free again, s_k[b ^ 1] is visible
    }
}

// The same work in two launches (the default; measured faster, since the persistent kernel then
// carries no anchor code and keeps the register allocation of the segment bodies): every
// anchor item in one launch of 128-thread blocks (item: request, block of 128 units,
// realisation, p << 4 | chain), then the persistent CTAs over the segment items alone, which
// need no wait: stream order puts every anchor before them.
template <class Real, class TabT>
__global__ void __launch_bounds__(128, SMERF_ANCHOR_MINB) anchor_queue_kernel(const SampleParams* __restrict__ descs,
                                                                               const int4* __restrict__ items)
{
    const int4 it = items[blockIdx.x];
    const SampleParams P = descs[it.x];
    NoStage h;
    const int u = it.y * blockDim.x + threadIdx.x;
    if ((it.w >> 4) == 1) anchor_body<Real, TabT, 1>(P, u, it.z, it.w & 15, h);
    else anchor_body<Real, TabT, 2>(P, u, it.z, it.w & 15, h);
}

template <class Real, class TabT, int SH>
__device__ __forceinline__ void queue_segment_after(const SampleParams& P, int seg, int grp)
{
    constexpr int M = SH / kQueueBuilds + 1, B = SH % kQueueBuilds;
    ws_body<Real, TabT, M, queue_upt(B), queue_rmax(B), false, false, false>(P, seg, grp);
}

template <class Real, class TabT>
__global__ void __launch_bounds__(kQueueThreads, kQueueMinBlocks) segment_queue_kernel(const SampleParams* __restrict__ descs,
                                                                         const int4* __restrict__ items, int n_items,
                                                                         int* __restrict__ head)
{
    __shared__ int s_k[2];  // the next item is claimed while the current one runs
    if (threadIdx.x == 0) s_k[0] = atomicAdd(head, 1);
    __syncthreads();
    for (int b = 0;; b ^= 1) {
        const int k = s_k[b];
        if (k >= n_items) return;
        if (threadIdx.x == 0) s_k[b ^ 1] = atomicAdd(head, 1);
        const int4 it = items[k];
        const SampleParams P = descs[it.x];
        switch (it.w) {
            case 0: queue_segment_after<Real, TabT, 0>(P, it.y, it.z); break;
            case 1: queue_segment_after<Real, TabT, 1>(P, it.y, it.z); break;
            case 2: queue_segment_after<Real, TabT, 2>(P, it.y, it.z); break;
            case 3: queue_segment_after<Real, TabT, 3>(P, it.y, it.z); break;
            case 4: queue_segment_after<Real, TabT, 4>(P, it.y, it.z); break;
            case 5: queue_segment_after<Real, TabT, 5>(P, it.y, it.z); break;
            case 6: queue_segment_after<Real, TabT, 6>(P, it.y, it.z); break;
            default: queue_segment_after<Real, TabT, 7>(P, it.y, it.z); break;
        }
        __syncthreads();  // the item's shared buffers are free again and s_k[b ^ 1] is visible
    }
}

}  // namespace smerf

#include "smerf_ring.cuh"

namespace smerf {

// ------------------------------------------------------------------ launch
// Raise a kernel's dynamic shared-memory limit to what it needs, once per kernel and size
// (so that later launches, e.g. under stream capture, make no attribute calls).
template <class K>
inline cudaError_t set_smem_attr(K kern, size_t smem)
{
    // the 48 KiB default covers dynamic plus static shared memory; the sampling kernels'
    // static arrays (round keys) take well under 1 KiB
    if (smem + 1024 <= 48 * 1024) return cudaSuccess;
    int dev = 0;
    cudaGetDevice(&dev);
    if (::smerf_smem_attr_done((const void*)kern, dev, smem, false)) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) ::smerf_smem_attr_done((const void*)kern, dev, smem, true);
    return e;
}

constexpr int kMaxThreads = 1024;
constexpr size_t kMaxSmem = 226 * 1024;  // leaves room for the static shared arrays

template <class Real, class TabT, int M, int UPT, int RMAX, int MINB = 1>
int launch_ws(const SampleParams& P, int n_segments, int nt, size_t smem, cudaStream_t st)
{
    auto kern = segment_ws_kernel<Real, TabT, M, UPT, RMAX, MINB>;
    if (set_smem_attr(kern, smem) != cudaSuccess) return SMERF_ECUDA;
    dim3 grid((P.n_samples + RMAX - 1) / RMAX, n_segments);
    kern<<<grid, nt, smem, st>>>(P);
    return cudaGetLastError() == cudaSuccess ? SMERF_OK : SMERF_ECUDA;
}

template <class Real, class TabT, int M, int UPT, int PARK>
auto pick_inplace(int lgNc)
{
    return lgNc == 14 ? segment_kernel<Real, TabT, M, UPT, 14, PARK>
         : lgNc == 13 ? segment_kernel<Real, TabT, M, UPT, 13, PARK>
         : lgNc == 12 ? segment_kernel<Real, TabT, M, UPT, 12, PARK>
                      : segment_kernel<Real, TabT, M, UPT, 0, PARK>;
}

template <class TabT, int LG, int PARK, int MINB, bool PACKED>
int launch_ring(const SampleParams& P, int n_segments, size_t smem, cudaStream_t st)
{
    auto kern = ring_kernel<TabT, LG, PARK, MINB, PACKED>;
    if (set_smem_attr(kern, smem) != cudaSuccess) return SMERF_ECUDA;
    dim3 grid(P.n_samples, n_segments);
    kern<<<grid, RingPass<LG>::NT, smem, st>>>(P);
    return cudaGetLastError() == cudaSuccess ? SMERF_OK : SMERF_ECUDA;
}

template <class Real, class TabT, int M, int UPT, int PARK>
int launch_inplace(const SampleParams& P, int n_segments, int nt, size_t smem, cudaStream_t st)
{
    auto kern = pick_inplace<Real, TabT, M, UPT, PARK>(P.lgNc);
    if (set_smem_attr(kern, smem) != cudaSuccess) return SMERF_ECUDA;
    dim3 grid(P.n_samples, n_segments);
    kern<<<grid, nt, smem, st>>>(P);
    return cudaGetLastError() == cudaSuccess ? SMERF_OK : SMERF_ECUDA;
}

// Launch configuration of the segment kernels for a plan.  Warp-specialised kernel when its
// three FFT buffers and the right-anchor states fit on chip: producer threads np = units /
// upt (<= 512), FFT threads np/2, rmax realisations per CTA (as many as registers and shared
// memory allow).  Otherwise the in-place kernel (one FFT buffer, anchors read from the
// scratch, one realisation per CTA, up to 1024 threads).
struct SegConfig { int ws, upt, nt, np, rmax, park, minb; size_t smem; int ring; int radix; };

// Long rings with p = 1 in FP32 (Nc = 8192 or 16384): the ring kernel (smerf_ring.cuh), NT =
// Nc / 16 threads, 8 units per thread of which 6 are parked in shared memory; at Nc = 8192 two
// CTAs fit on an SM.
#ifndef SMERF_RING_KERNEL
#define SMERF_RING_KERNEL 1
#endif
template <class Real>
inline bool ring_config(const smerf_plan* pl, SegConfig& cfg)
{
    const int Nc = pl->n_phi / 2;
    if (!SMERF_RING_KERNEL || sizeof(Real) != 4 || pl->p != 1 || (Nc != 8192 && Nc != 16384)) return false;
    cfg = SegConfig{};
    cfg.ring = pl->packed ? 2 : 1;
    cfg.nt = Nc / 16;
    cfg.upt = 8;
    cfg.rmax = 1;
    cfg.park = 6;
    cfg.minb = Nc == 8192 ? 2 : 1;
    cfg.smem = (size_t)Nc * 8 + (size_t)cfg.park * cfg.nt * 16;
    return true;
}

template <class Real> constexpr int ws_rmax_cap(int upt, int M)
{
    return sizeof(Real) == 8 || M == 3 ? 1 : (upt <= 2 ? 4 : (upt == 4 ? 2 : 1));
}

template <class Real>
inline size_t ws_smem(const smerf_plan* pl, int rmax)
{
    const int Nc = pl->n_phi / 2;
    return (size_t)3 * rmax * Nc * 2 * sizeof(Real) + (pl->H > 0 ? (size_t)rmax * Nc * 2 * pl->p * sizeof(Real) : 0);
}

// (units per thread, realisations per CTA, CTAs per SM) with a built warp-specialised kernel
// for state size M (p = 3, whose units hold 12 state values: one realisation per CTA, one
// CTA per SM)
template <class Real> inline bool ws_built(int upt, int rmax, int minb, int M)
{
    if (M == 3) return minb == 1 && rmax == 1 && (upt == 1 || upt == 2 || upt == 4 || upt == 8);
    if (minb == 2) return sizeof(Real) == 4 && ((upt == 4 && (rmax == 1 || rmax == 2)) || (upt == 8 && rmax == 1));
    if (minb != 1) return false;
    if (sizeof(Real) == 8) return rmax == 1 && (upt == 1 || upt == 2 || upt == 4 || upt == 8);
    return (upt == 1 && rmax == 4) || (upt == 2 && (rmax == 4 || rmax == 2)) || (upt == 4 && (rmax == 2 || rmax == 1)) ||
           (upt == 8 && rmax == 1);
}

// Every warp-specialised configuration that fits the plan, as kLaunchInts integers (units per
// producer thread, realisations per CTA, producer threads np = units / upt (<= 512, multiple
// of 32), FFT threads nf in {np/2, np, np/4}, CTAs per SM the kernel is built for, FFT radix
// plan; np + nf within that build's thread limit).  Radix plan 16 (the fixed high-radix plan)
// where the build has one for this ring length (FP32), and 4 (radix-4 passes) always.
template <class Real>
inline int tune_candidates(const smerf_plan* pl, int* cand, int max_n)
{
    const int n_units = pl->n_slots / unit_slots(pl->p);
    int n = 0;
    const int rm[3] = {4, 2, 1};
    for (int minb = 1; minb <= 2; ++minb)
        for (int upt = 1; upt <= 8; upt *= 2) {
            int np = (n_units + upt - 1) / upt;
            np = ((np + 31) / 32) * 32;
            if (np > 512 || (upt > 1 && (n_units + upt / 2 - 1) / (upt / 2) <= 32)) continue;
            for (int k = 0; k < 3; ++k) {
                const int rmax = rm[k];
                if (!ws_built<Real>(upt, rmax, minb, pl->p) || ws_smem<Real>(pl, rmax) > 226 * 1024) continue;
                const int div[3] = {2, 1, 4};
                for (int d = 0; d < 3; ++d) {
                    int nf = ((np / div[d] + 31) / 32) * 32;
                    if (nf < 32) nf = 32;
                    if (np + nf > ws_max_threads(minb, pl->p)) continue;
                    int lg = 0;
                    while ((2 << lg) < pl->n_phi) ++lg;
                    const int lo = ws_lg_lo(upt, pl->p), hi = ws_lg_hi(upt, pl->p);
                    const bool hr = sizeof(Real) == 4 && lg >= lo && lg <= hi;
                    for (int radix : {16, 4}) {
                        if (radix == 16 && !hr) continue;
                        if (n < max_n) {
                            int* c = cand + kLaunchInts * n;
                            c[0] = upt;
                            c[1] = rmax;
                            c[2] = np;
                            c[3] = nf;
                            c[4] = minb;
                            c[5] = radix;
                        }
                        ++n;
                    }
                }
            }
        }
    return n < max_n ? n : max_n;
}

template <class Real>
inline SegConfig seg_config(const smerf_plan* pl)
{
    SegConfig cfg{};
    const int M = pl->p;
    const int n_units = pl->n_slots / unit_slots(M);
    const int Nc = pl->n_phi / 2;
    if (pl->tune.valid && ws_built<Real>(pl->tune.upt, pl->tune.rmax, pl->tune.minb, M) &&
        ws_smem<Real>(pl, pl->tune.rmax) <= 226 * 1024 &&
        (n_units + pl->tune.upt - 1) / pl->tune.upt <= pl->tune.np &&
        pl->tune.np + pl->tune.nf <= ws_max_threads(pl->tune.minb, M)) {
        cfg.ws = 1;
        cfg.upt = pl->tune.upt;
        cfg.rmax = pl->tune.rmax;
        cfg.minb = pl->tune.minb;
        cfg.np = pl->tune.np;
        cfg.nt = pl->tune.np + pl->tune.nf;
        cfg.smem = ws_smem<Real>(pl, cfg.rmax);
        cfg.radix = pl->tune.radix;
        return cfg;
    }
    auto np_of = [&](int u) { return (((n_units + u - 1) / u + 31) / 32) * 32; };
    auto nf_of = [](int np) { return np / 2 > 32 ? ((np / 2 + 31) / 32) * 32 : 32; };
    auto fits = [&](int u) { return np_of(u) <= 512 && np_of(u) + nf_of(np_of(u)) <= ws_max_threads(1, M); };
    int upt = 1;
    while (upt < 8 && !fits(upt)) upt *= 2;
    if (fits(upt)) {
        const int np = np_of(upt), nf = nf_of(np);
        for (int rmax = ws_rmax_cap<Real>(upt, M); rmax >= 1; rmax /= 2) {
            const size_t smem = (size_t)3 * rmax * Nc * 2 * sizeof(Real) +
                                (pl->H > 0 ? (size_t)rmax * Nc * 2 * M * sizeof(Real) : 0);
            if (smem <= kMaxSmem) {
                cfg.ws = 1;
                cfg.upt = upt;
                cfg.np = np;
                cfg.nt = np + nf;
                cfg.rmax = rmax;
                cfg.minb = 1;
                cfg.smem = smem;
                cfg.radix = sizeof(Real) == 4 ? 16 : 4;
                return cfg;
            }
        }
    }
    if (ring_config<Real>(pl, cfg)) return cfg;
    upt = 1;
    while (upt < 8 && (n_units + upt - 1) / upt > kMaxThreads) upt *= 2;
    if (upt < 4) upt = 4;

    int nt = (n_units + upt - 1) / upt;
    nt = ((nt + 31) / 32) * 32;
    if (nt < 64) nt = 64;
    cfg.ws = 0;
    cfg.upt = upt;
    cfg.nt = nt;
    cfg.rmax = 1;
    // park all but two units' states during the FFT if shared memory allows, else half, else none
    const size_t ring = (size_t)Nc * 2 * sizeof(Real), per_unit = (size_t)nt * unit_vals(M) * sizeof(Real);
    cfg.park = ring + (upt - 2) * per_unit <= kMaxSmem ? upt - 2 : ring + (upt / 2) * per_unit <= kMaxSmem ? upt / 2 : 0;
    cfg.smem = ring + cfg.park * per_unit;
    return cfg;
}

template <class Real, class TabT, int M>
int dispatch_segments(const SampleParams& P, int n_segments, const SegConfig& cfg, cudaStream_t st)
{
    if (cfg.ws) {
        if constexpr (sizeof(Real) == 8 || M == 3) {
            if (cfg.rmax != 1 || cfg.minb != 1) return SMERF_EUNSUPPORTED;
            switch (cfg.upt) {
                case 1: return launch_ws<Real, TabT, M, 1, 1>(P, n_segments, cfg.nt, cfg.smem, st);
                case 2: return launch_ws<Real, TabT, M, 2, 1>(P, n_segments, cfg.nt, cfg.smem, st);
                case 4: return launch_ws<Real, TabT, M, 4, 1>(P, n_segments, cfg.nt, cfg.smem, st);
                case 8: return launch_ws<Real, TabT, M, 8, 1>(P, n_segments, cfg.nt, cfg.smem, st);
                default: return SMERF_EUNSUPPORTED;
            }
        } else {
        if (cfg.minb == 2) {
            switch (cfg.upt * 8 + cfg.rmax) {
                case 4 * 8 + 2: return launch_ws<Real, TabT, M, 4, 2, 2>(P, n_segments, cfg.nt, cfg.smem, st);
                case 4 * 8 + 1: return launch_ws<Real, TabT, M, 4, 1, 2>(P, n_segments, cfg.nt, cfg.smem, st);
                case 8 * 8 + 1: return launch_ws<Real, TabT, M, 8, 1, 2>(P, n_segments, cfg.nt, cfg.smem, st);
                default: return SMERF_EUNSUPPORTED;
            }
        }
        const int key = cfg.upt * 8 + cfg.rmax;
        switch (key) {
            case 1 * 8 + 4: return launch_ws<Real, TabT, M, 1, 4>(P, n_segments, cfg.nt, cfg.smem, st);
            case 2 * 8 + 4: return launch_ws<Real, TabT, M, 2, 4>(P, n_segments, cfg.nt, cfg.smem, st);
            case 2 * 8 + 2: return launch_ws<Real, TabT, M, 2, 2>(P, n_segments, cfg.nt, cfg.smem, st);
            case 4 * 8 + 2: return launch_ws<Real, TabT, M, 4, 2>(P, n_segments, cfg.nt, cfg.smem, st);
            case 4 * 8 + 1: return launch_ws<Real, TabT, M, 4, 1>(P, n_segments, cfg.nt, cfg.smem, st);
            case 8 * 8 + 1: return launch_ws<Real, TabT, M, 8, 1>(P, n_segments, cfg.nt, cfg.smem, st);
            default: return SMERF_EUNSUPPORTED;
        }
        }
    }
    if (cfg.ring) {
        if constexpr (sizeof(Real) == 4 && M == 1) {
            if constexpr (sizeof(TabT) == 4) {
                if (cfg.ring == 2) {
                    if (P.lgNc == 14) return launch_ring<TabT, 14, 6, 1, true>(P, n_segments, cfg.smem, st);
                    if (P.lgNc == 13) return launch_ring<TabT, 13, 6, 2, true>(P, n_segments, cfg.smem, st);
                    return SMERF_EUNSUPPORTED;
                }
            }
            if (P.lgNc == 14) return launch_ring<TabT, 14, 6, 1, false>(P, n_segments, cfg.smem, st);
            if (P.lgNc == 13) return launch_ring<TabT, 13, 6, 2, false>(P, n_segments, cfg.smem, st);
        }
        return SMERF_EUNSUPPORTED;
    }
    if constexpr (M == 3) {
        return SMERF_EUNSUPPORTED;  // p = 3 runs on the warp-specialised kernels only
    } else {
        switch (cfg.upt * 16 + cfg.park) {
            case 4 * 16 + 2: return launch_inplace<Real, TabT, M, 4, 2>(P, n_segments, cfg.nt, cfg.smem, st);
            case 4 * 16 + 0: return launch_inplace<Real, TabT, M, 4, 0>(P, n_segments, cfg.nt, cfg.smem, st);
            case 8 * 16 + 6: return launch_inplace<Real, TabT, M, 8, 6>(P, n_segments, cfg.nt, cfg.smem, st);
            case 8 * 16 + 4: return launch_inplace<Real, TabT, M, 8, 4>(P, n_segments, cfg.nt, cfg.smem, st);
            case 8 * 16 + 0: return launch_inplace<Real, TabT, M, 8, 0>(P, n_segments, cfg.nt, cfg.smem, st);
            default: return SMERF_EUNSUPPORTED;
        }
    }
}

// The request's kernel parameters and launch configuration.
template <class Real, class TabT>
int fill_params(const smerf_plan* pl, uint64_t seed, int n, void* out, void* scratch, SampleParams& P, SegConfig& cfg)
{
    P.segs = pl->segs_dev;
    P.steps[0] = pl->steps[0];
    P.steps[1] = pl->steps[1];
    P.coarse[0] = pl->coarse[0];
    P.coarse[1] = pl->coarse[1];
    P.beq = pl->beq;
    P.tw = pl->tw;
    P.pre = pl->pre;
    P.tw2 = pl->tw2;
    P.tw3 = pl->tw3;
    P.anc = scratch;
    P.out = out;
    P.seed = seed;
    P.n_samples = n;
    P.n_theta = pl->n_theta;
    P.n_phi = pl->n_phi;
    P.Nc = pl->n_phi / 2;
    P.n_units = P.Nc / unit_slots(pl->p);
    P.n_modes_pad = pl->n_modes_pad;
    P.k0 = pl->k0;
    P.H = pl->H;
    P.n_anchors[0] = pl->chain[0].n_anchors;
    P.n_anchors[1] = pl->chain[1].n_anchors;
    P.na_max = P.n_anchors[0] > P.n_anchors[1] ? P.n_anchors[0] : P.n_anchors[1];
    cfg = seg_config<Real>(pl);
    if (cfg.smem > kMaxSmem) return SMERF_EUNSUPPORTED;  // one ring per realisation must fit on chip
    if (!cfg.ws && (pl->n_slots / unit_slots(pl->p) + cfg.upt - 1) / cfg.upt > kMaxThreads) return SMERF_EUNSUPPORTED;
    if (pl->n_segments > 65535) return SMERF_EUNSUPPORTED;
    P.pingpong = cfg.ws;
    P.np = cfg.np;
    P.fft_r4 = cfg.ws && cfg.radix == 4;
    int lg = 0;
    while ((1 << lg) < P.Nc) ++lg;
    P.lgNc = lg;
    P.ring_n = pl->rings_total ? pl->rings_n_dev : nullptr;
    P.ring_h = pl->rings_total ? pl->rings_h_dev : nullptr;
    P.ring_off = pl->rings_total ? pl->rings_off_dev : nullptr;
    P.ring_total = pl->rings_total;
    // ring-dependent longitudes are synthesised by the warp-specialised kernels' FFT group only,
    // and p = 3 is built for those kernels only (rings up to 4096 complex points in FP32, 2048
    // in FP64)
    if ((pl->rings_total || pl->p == 3) && !cfg.ws) return SMERF_EUNSUPPORTED;
    return SMERF_OK;
}

// Anchor and segment launches of one request (state size M = p).
template <class Real, class TabT, int M>
int launch_sample_m(const smerf_plan* pl, uint64_t seed, int n, void* out, void* scratch, cudaStream_t st,
                    cudaEvent_t ev0, cudaEvent_t ev1)
{
    SampleParams P;
    SegConfig cfg;
    int rc = fill_params<Real, TabT>(pl, seed, n, out, scratch, P, cfg);
    if (rc != SMERF_OK) return rc;
    {
        dim3 ga((P.n_units + 127) / 128, n, 2);
        anchor_kernel<Real, TabT, M><<<ga, 128, 0, st>>>(P);
        if (cudaGetLastError() != cudaSuccess) return SMERF_ECUDA;
    }
    if (ev0 && cudaEventRecord(ev0, st) != cudaSuccess) return SMERF_ECUDA;
    rc = dispatch_segments<Real, TabT, M>(P, pl->n_segments, cfg, st);
    if (rc == SMERF_OK && ev1 && cudaEventRecord(ev1, st) != cudaSuccess) return SMERF_ECUDA;
    return rc;
}

// FP64 coarse and start tables -> FP32 (a few rows per mode; one element per thread)
static __global__ void __launch_bounds__(256) stage_small_kernel(StageSmall S)
{
    const unsigned total = S.end[2];
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int q = (i >= S.end[0]) + (i >= S.end[1]);
        const unsigned i0 = q == 0 ? 0u : q == 1 ? S.end[0] : S.end[1];
        const double* src = q == 0 ? S.src[0] : q == 1 ? S.src[1] : S.src[2];
        float* dst = q == 0 ? S.dst[0] : q == 1 ? S.dst[1] : S.dst[2];
        dst[i - i0] = tabcvt<float, double>(src[i - i0]);
    }
}

// FP64 tables, FP32 recursion, tables staged: a short launch converting the coarse and start
// tables, the anchor launch (FP32 tables) that also converts the step tables, then the segment
// launch of the plan `sh`, whose table pointers are the FP32 copies.
template <int M>
int launch_sample_staged_m(const smerf_plan* sh, const StageSmall& S, StageJob J, uint64_t seed, int n, void* out,
                           void* scratch, cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1)
{
    SampleParams P;
    SegConfig cfg;
    int rc = fill_params<float, float>(sh, seed, n, out, scratch, P, cfg);
    if (rc != SMERF_OK) return rc;
    if (S.end[2] > 0) {
        const unsigned blocks = (S.end[2] + 255) / 256;
        stage_small_kernel<<<blocks < 152 * 8 ? blocks : 152 * 8, 256, 0, st>>>(S);
        if (cudaGetLastError() != cudaSuccess) return SMERF_ECUDA;
    }
    {
        dim3 ga((P.n_units + 127) / 128, n, 2);
        // rounds per step table, and the rounds run during the anchors: one per anchor that
        // every thread steps, no more than there are
        const unsigned long long T = (unsigned long long)ga.x * 128 * ga.y * ga.z;
        const unsigned long long r0 = ((J.n[0] + kStageGroup - 1) / kStageGroup + T - 1) / T;
        const unsigned long long r1 = ((J.n[1] + kStageGroup - 1) / kStageGroup + T - 1) / T;
        J.rounds0 = (unsigned)r0;
        J.rounds = (unsigned)(r0 + r1);
        // rounds converted during the anchors, one every `every` anchors, spread over the
        // anchors that every thread steps
        const int na_min = P.n_anchors[0] < P.n_anchors[1] ? P.n_anchors[0] : P.n_anchors[1];
        J.every = J.rounds > 0 && (unsigned)na_min > J.rounds ? na_min / (int)J.rounds : 1;
        J.k_loop = na_min / J.every < (int)J.rounds ? na_min / J.every : (int)J.rounds;
        anchor_stage_kernel<float, float, M><<<ga, 128, 0, st>>>(P, J);
        if (cudaGetLastError() != cudaSuccess) return SMERF_ECUDA;
    }
    if (ev0 && cudaEventRecord(ev0, st) != cudaSuccess) return SMERF_ECUDA;
    rc = dispatch_segments<float, float, M>(P, sh->n_segments, cfg, st);
    if (rc == SMERF_OK && ev1 && cudaEventRecord(ev1, st) != cudaSuccess) return SMERF_ECUDA;
    return rc;
}

// ---- batched groups: requests of one shape share one anchor and one segment launch
template <class Real, class TabT, int M, int UPT, int RMAX, int MINB = 1>
int launch_ws_batched(const SampleParams* d, const int4* items, int n_items, int nt, size_t smem, cudaStream_t st)
{
    auto kern = segment_ws_batched_kernel<Real, TabT, M, UPT, RMAX, MINB>;
    if (set_smem_attr(kern, smem) != cudaSuccess) return SMERF_ECUDA;
    kern<<<n_items, nt, smem, st>>>(d, items);
    return cudaGetLastError() == cudaSuccess ? SMERF_OK : SMERF_ECUDA;
}

template <class Real, class TabT, int M>
int group_segments(const SegConfig& cfg, const SampleParams* d, const int4* items, int n_items, cudaStream_t st)
{
    if constexpr (sizeof(Real) == 8 || M == 3) {
        if (cfg.rmax != 1 || cfg.minb != 1) return SMERF_EUNSUPPORTED;
        switch (cfg.upt) {
            case 1: return launch_ws_batched<Real, TabT, M, 1, 1>(d, items, n_items, cfg.nt, cfg.smem, st);
            case 2: return launch_ws_batched<Real, TabT, M, 2, 1>(d, items, n_items, cfg.nt, cfg.smem, st);
            case 4: return launch_ws_batched<Real, TabT, M, 4, 1>(d, items, n_items, cfg.nt, cfg.smem, st);
            case 8: return launch_ws_batched<Real, TabT, M, 8, 1>(d, items, n_items, cfg.nt, cfg.smem, st);
            default: return SMERF_EUNSUPPORTED;
        }
    } else {
        if (cfg.minb == 2) {
            switch (cfg.upt * 8 + cfg.rmax) {
                case 4 * 8 + 2: return launch_ws_batched<Real, TabT, M, 4, 2, 2>(d, items, n_items, cfg.nt, cfg.smem, st);
                case 4 * 8 + 1: return launch_ws_batched<Real, TabT, M, 4, 1, 2>(d, items, n_items, cfg.nt, cfg.smem, st);
                case 8 * 8 + 1: return launch_ws_batched<Real, TabT, M, 8, 1, 2>(d, items, n_items, cfg.nt, cfg.smem, st);
                default: return SMERF_EUNSUPPORTED;
            }
        }
        switch (cfg.upt * 8 + cfg.rmax) {
            case 1 * 8 + 4: return launch_ws_batched<Real, TabT, M, 1, 4>(d, items, n_items, cfg.nt, cfg.smem, st);
            case 2 * 8 + 4: return launch_ws_batched<Real, TabT, M, 2, 4>(d, items, n_items, cfg.nt, cfg.smem, st);
            case 2 * 8 + 2: return launch_ws_batched<Real, TabT, M, 2, 2>(d, items, n_items, cfg.nt, cfg.smem, st);
            case 4 * 8 + 2: return launch_ws_batched<Real, TabT, M, 4, 2>(d, items, n_items, cfg.nt, cfg.smem, st);
            case 4 * 8 + 1: return launch_ws_batched<Real, TabT, M, 4, 1>(d, items, n_items, cfg.nt, cfg.smem, st);
            case 8 * 8 + 1: return launch_ws_batched<Real, TabT, M, 8, 1>(d, items, n_items, cfg.nt, cfg.smem, st);
            default: return SMERF_EUNSUPPORTED;
        }
    }
}

// A batch's persistent work (FP32 recursion).  One launch (single): `ctas` CTAs of queue_kernel
// over the n_items items (the anchor items first); ctl holds 2 + n_req integers (head, status,
// per-request anchor counters), set here before the launch; fail_waits (a test hook) starts the
// anchor counters at -1 instead of 0, so that no segment item's wait can be met: the waits run
// out and the status word records it.  Two launches (otherwise): anchor_queue_kernel over the
// n_anc128 items of anc128, then `ctas` CTAs of segment_queue_kernel over the segment items
// (items + n_anc, n_items - n_anc of them), ctl[0] their queue head.
template <class Real, class TabT>
int launch_queue(const SampleParams* d, const int4* items, int n_items, int n_anc, const int4* anc128, int n_anc128,
                 int* ctl, int n_req, int single, int fail_waits, size_t smem, int ctas, cudaStream_t st)
{
    if (n_items == 0) return SMERF_OK;
    if (single) {
        auto kern = queue_kernel<Real, TabT>;
        if (set_smem_attr(kern, smem) != cudaSuccess) return SMERF_ECUDA;
        if (cudaMemsetAsync(ctl, 0, sizeof(int) * 2, st) != cudaSuccess) return SMERF_ECUDA;
        if (n_req > 0 && cudaMemsetAsync(ctl + 2, fail_waits ? 0xFF : 0, sizeof(int) * n_req, st) != cudaSuccess)
            return SMERF_ECUDA;
        kern<<<ctas, kQueueThreads, smem, st>>>(d, items, n_items, ctl);
        return cudaGetLastError() == cudaSuccess ? SMERF_OK : SMERF_ECUDA;
    }
    if (n_anc128 > 0) {
        anchor_queue_kernel<Real, TabT><<<n_anc128, 128, 0, st>>>(d, anc128);
        if (cudaGetLastError() != cudaSuccess) return SMERF_ECUDA;
    }
    if (n_items == n_anc) return SMERF_OK;
    auto kern = segment_queue_kernel<Real, TabT>;
    if (set_smem_attr(kern, smem) != cudaSuccess) return SMERF_ECUDA;
    if (cudaMemsetAsync(ctl, 0, sizeof(int) * 2, st) != cudaSuccess) return SMERF_ECUDA;
    kern<<<ctas, kQueueThreads, smem, st>>>(d, items + n_anc, n_items - n_anc, ctl);
    return cudaGetLastError() == cudaSuccess ? SMERF_OK : SMERF_ECUDA;
}

// resident CTAs of the persistent launch (kQueueThreads threads, smem bytes) on this device:
// the smaller of the two persistent kernels' counts, so that either mode may use it
template <class Real, class TabT>
int queue_ctas(size_t smem)
{
    auto k1 = queue_kernel<Real, TabT>;
    auto k2 = segment_queue_kernel<Real, TabT>;
    if (set_smem_attr(k1, smem) != cudaSuccess || set_smem_attr(k2, smem) != cudaSuccess) return -1;
    int per1 = 0, per2 = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per1, k1, kQueueThreads, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k2, kQueueThreads, smem) != cudaSuccess)
        return -1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1;
    return (per1 < per2 ? per1 : per2) * sms;
}

template <class Real, class TabT>
int fill_params_c(const smerf_plan* pl, uint64_t seed, int n, void* out, void* scratch, SampleParams* P,
                  int* batchable, int* rmax)
{
    SegConfig cfg;
    const int rc = fill_params<Real, TabT>(pl, seed, n, out, scratch, *P, cfg);
    *batchable = rc == SMERF_OK && cfg.ws;
    *rmax = cfg.rmax;
    return rc;
}

// One anchor and one segment launch over a batched group's work items (state size M = p).
template <class Real, class TabT, int M>
int launch_group_m(const smerf_plan* rep, const SampleParams* d, const int4* anc_items, int n_anc,
                   const int4* seg_items, int n_seg, cudaStream_t st)
{
    const SegConfig cfg = seg_config<Real>(rep);
    if (!cfg.ws) return SMERF_EUNSUPPORTED;
    if (n_anc > 0) {
        anchor_batched_kernel<Real, TabT, M><<<n_anc, 128, 0, st>>>(d, anc_items);
        if (cudaGetLastError() != cudaSuccess) return SMERF_ECUDA;
    }
    if (n_seg == 0) return SMERF_OK;
    return group_segments<Real, TabT, M>(cfg, d, seg_items, n_seg, st);
}

}  // namespace smerf

// Kernel instantiations of one (recursion, table) precision pair XX and state size M, one
// translation unit each (smerf_sample_XX_pM.cu).
#define SMERF_INSTANTIATE(REAL, TABT, XX, M)                                                             \
    int smerf_launch_sample_##XX##_p##M(const smerf_plan* pl, uint64_t seed, int n, void* out, void* scratch, \
                                        cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1)                \
    {                                                                                                     \
        return smerf::launch_sample_m<REAL, TABT, M>(pl, seed, n, out, scratch, st, ev0, ev1);           \
    }                                                                                                     \
    int smerf_launch_group_##XX##_p##M(const smerf_plan* rep, const smerf::SampleParams* d,               \
                                       const int4* anc_items, int n_anc, const int4* seg_items, int n_seg, \
                                       cudaStream_t st)                                                   \
    {                                                                                                     \
        return smerf::launch_group_m<REAL, TABT, M>(rep, d, anc_items, n_anc, seg_items, n_seg, st);     \
    }

// The precision pair's entry points (smerf_sample_XX.cu): dispatch on p to the instantiations.
#define SMERF_PRECISION_PAIR(REAL, TABT, XX)                                                                \
    int smerf_launch_sample_##XX##_p1(const smerf_plan*, uint64_t, int, void*, void*, cudaStream_t, cudaEvent_t, \
                                      cudaEvent_t);                                                         \
    int smerf_launch_sample_##XX##_p2(const smerf_plan*, uint64_t, int, void*, void*, cudaStream_t, cudaEvent_t, \
                                      cudaEvent_t);                                                         \
    int smerf_launch_sample_##XX##_p3(const smerf_plan*, uint64_t, int, void*, void*, cudaStream_t, cudaEvent_t, \
                                      cudaEvent_t);                                                         \
    int smerf_launch_group_##XX##_p1(const smerf_plan*, const smerf::SampleParams*, const int4*, int,       \
                                     const int4*, int, cudaStream_t);                                       \
    int smerf_launch_group_##XX##_p2(const smerf_plan*, const smerf::SampleParams*, const int4*, int,       \
                                     const int4*, int, cudaStream_t);                                       \
    int smerf_launch_group_##XX##_p3(const smerf_plan*, const smerf::SampleParams*, const int4*, int,       \
                                     const int4*, int, cudaStream_t);                                       \
    int smerf_launch_sample_##XX(const smerf_plan* pl, uint64_t seed, int n, void* out, void* scratch,      \
                                 cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1)                         \
    {                                                                                                       \
        return pl->p == 1   ? smerf_launch_sample_##XX##_p1(pl, seed, n, out, scratch, st, ev0, ev1)        \
               : pl->p == 2 ? smerf_launch_sample_##XX##_p2(pl, seed, n, out, scratch, st, ev0, ev1)        \
                            : smerf_launch_sample_##XX##_p3(pl, seed, n, out, scratch, st, ev0, ev1);       \
    }                                                                                                       \
    int smerf_fill_params_##XX(const smerf_plan* pl, uint64_t seed, int n, void* out, void* scratch,        \
                               smerf::SampleParams* P, int* batchable, int* rmax)                           \
    {                                                                                                       \
        return smerf::fill_params_c<REAL, TABT>(pl, seed, n, out, scratch, P, batchable, rmax);             \
    }                                                                                                       \
    int smerf_launch_group_##XX(const smerf_plan* rep, const smerf::SampleParams* d_descs,                  \
                                const int4* anc_items, int n_anc, const int4* seg_items, int n_seg,         \
                                cudaStream_t st)                                                            \
    {                                                                                                       \
        return rep->p == 1   ? smerf_launch_group_##XX##_p1(rep, d_descs, anc_items, n_anc, seg_items, n_seg, st) \
               : rep->p == 2 ? smerf_launch_group_##XX##_p2(rep, d_descs, anc_items, n_anc, seg_items, n_seg, st) \
                             : smerf_launch_group_##XX##_p3(rep, d_descs, anc_items, n_anc, seg_items, n_seg, st); \
    }                                                                                                       \
    int smerf_tune_candidates_##XX(const smerf_plan* pl, int* cand, int max_n)                              \
    {                                                                                                       \
        return smerf::tune_candidates<REAL>(pl, cand, max_n);                                               \
    }                                                                                                            \
    size_t smerf_ws_smem_##XX(const smerf_plan* pl, int rmax) { return smerf::ws_smem<REAL>(pl, rmax); }

// The persistent batch launch of an FP32-recursion precision pair (its own translation unit,
// smerf_sample_XX_queue.cu, since it instantiates every shape of p = 1 and 2).
#define SMERF_QUEUE(REAL, TABT, XX)                                                                       \
    int smerf_launch_queue_##XX(const smerf::SampleParams* d, const int4* items, int n_items, int n_anc,   \
                                const int4* anc128, int n_anc128, int* ctl, int n_req, int single,          \
                                int fail_waits, size_t smem, int ctas, cudaStream_t st)                     \
    {                                                                                                     \
        return smerf::launch_queue<REAL, TABT>(d, items, n_items, n_anc, anc128, n_anc128, ctl, n_req,      \
                                               single, fail_waits, smem, ctas, st);                         \
    }                                                                                                     \
    int smerf_queue_ctas_##XX(size_t smem) { return smerf::queue_ctas<REAL, TABT>(smem); }
