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
// of slots whose 2p normals fill one Philox call (p = 1: two slots, p = 2: one slot).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "smerf_internal.cuh"

namespace smerf {

struct SampleParams {
    const Segment* segs;
    const void* steps[2];
    const void* coarse[2];
    const void* beq;
    const void* tw;   // per-pass complex twiddle tables (see pass_radix)
    const void* pre;  // complex e^{2 pi i s / n_phi}, s < Nc
    void* anc;        // anchor states [c][r][j][2M][n_slots]
    void* out;
    uint64_t seed;
    int n_samples, n_theta, n_phi, Nc, n_units, n_modes_pad, k0, H, na_max;
    int n_anchors[2];
    int pingpong;     // 1: two FFT buffers + right anchors on chip; 0: one buffer, in place
    int lgNc;
};

template <int M> constexpr int kG = unit_slots(M);

// the 4 normals of Philox call `call` of ring `ring` for realisation key `key64`
template <class Real>
__device__ __forceinline__ void unit_normals(uint64_t key64, uint32_t call, uint32_t ring, Real (&n)[4])
{
    const PhiloxKey key{(uint32_t)key64, (uint32_t)(key64 >> 32)};
    const uint4 w = philox4x32_10(make_uint4(call, ring, 0u, 0u), key);
    box_muller(w.x, w.y, n[0], n[1]);
    box_muller(w.z, w.w, n[2], n[3]);
}

template <class Real, class TabT>
__device__ __forceinline__ Real tabld(const TabT* p) { return (Real)__ldg(p); }

// FP64 table value -> FP32 with integer instructions only (GB300 runs FP64 conversions on
// its narrow FP64 pipe).  Truncates the mantissa; values below the FP32 normal range
// become 0 (tables hold no values above it).
template <>
__device__ __forceinline__ float tabld<float, double>(const double* p)
{
    const double v = __ldg(p);
    const uint32_t hi = (uint32_t)(__double_as_longlong(v) >> 32);
    const uint32_t lo = (uint32_t)__double_as_longlong(v);
    const uint32_t e11 = (hi >> 20) & 0x7FFu;
    uint32_t t = __funnelshift_l(lo, hi, 3) - (128u << 23);
    t = (t & 0x7FFFFFFFu) | (hi & 0x80000000u);
    return e11 > 896u ? __uint_as_float(t) : 0.0f;
}

// anchor scratch offset: [c][r][j][f][slot], f = part * M + q
template <int M>
__device__ __forceinline__ size_t aoff(const SampleParams& P, int c, int r, int j, int f, int slot)
{
    return ((((size_t)c * P.n_samples + r) * (P.na_max + 1) + j) * (2 * M) + f) * (size_t)P.Nc + slot;
}

// ------------------------------------------------------------------ anchors
template <class Real, class TabT, int M>
__global__ void __launch_bounds__(128) anchor_kernel(SampleParams P)
{
    constexpr int G = kG<M>;
    constexpr int T = tri(M);
    constexpr int Ec = coarse_elems(M);
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    const int c = blockIdx.z;
    if (u >= P.n_units) return;
    const size_t mp = P.n_modes_pad;
    const uint64_t key = P.seed + (uint64_t)r;
    Real* anc = (Real*)P.anc;
    Real x[G][2][M];
    Real nr[4];
    // start ring: x = B_eq xi (x basis); the southern chain keeps S x
    unit_normals<Real>(key, (uint32_t)u, (uint32_t)P.k0, nr);
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
#pragma unroll
    for (int g = 0; g < G; ++g)
#pragma unroll
        for (int part = 0; part < 2; ++part)
#pragma unroll
            for (int q = 0; q < M; ++q) anc[aoff<M>(P, c, r, 0, part * M + q, G * u + g)] = x[g][part][q];
    const TabT* cs = (const TabT*)P.coarse[c];
    for (int j = 1; j <= P.n_anchors[c]; ++j) {
        const int pos = j * P.H;
        const int ring = c == 0 ? P.k0 - pos : P.k0 + pos;
        unit_normals<Real>(key, (uint32_t)u, (uint32_t)ring, nr);
        const TabT* tb = cs + (size_t)j * Ec * mp;
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                const int s = G * u + g;
                const int mode = (part == 1 && s == 0) ? P.Nc : s;
                Real xi[M], xn[M];
#pragma unroll
                for (int q = 0; q < M; ++q) {
                    const Real v = nr[g * 2 * M + part * M + q];
                    xi[q] = (c == 1 && (q & 1)) ? -v : v;
                }
#pragma unroll
                for (int p = 0; p < M; ++p) {
                    Real acc = 0;
#pragma unroll
                    for (int q = 0; q < M; ++q) acc += tabld<Real, TabT>(tb + (size_t)(p * M + q) * mp + mode) * x[g][part][q];
                    int e = M * M + p * (p + 1) / 2;
#pragma unroll
                    for (int q = 0; q <= p; ++q, ++e) acc += tabld<Real, TabT>(tb + (size_t)e * mp + mode) * xi[q];
                    xn[p] = acc;
                }
#pragma unroll
                for (int q = 0; q < M; ++q) x[g][part][q] = xn[q];
            }
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int part = 0; part < 2; ++part)
#pragma unroll
                for (int q = 0; q < M; ++q) anc[aoff<M>(P, c, r, j, part * M + q, G * u + g)] = x[g][part][q];
    }
    (void)T;
}

// ------------------------------------------------------------------ FFT
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

template <class C, int RP>
__device__ __forceinline__ void dft(C* v)
{
    if (RP == 2) dft2(v[0], v[1]);
    else if (RP == 4) dft4(v);
    else dft8(v);
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

// One radix-RP Stockham pass over R rings of Nc points, src -> dst (distinct shared
// buffers), or, for the last pass, straight to the rings' rows in global memory (gout[r]).
// The first pass (Ns = 1) has unit twiddles and applies the C2R packing as it loads.
template <class C, int RP, bool FIRST, bool LAST>
__device__ __forceinline__ void fft_pass(const C* __restrict__ src, C* __restrict__ dst, int R, int lgNc,
                                         int Ns, const C* __restrict__ twp, const C* __restrict__ pre,
                                         C* const* gout)
{
    const int Nc = 1 << lgNc;
    constexpr int LR = RP == 4 ? 2 : 1;
    const int lgnb = lgNc - LR;
    const int nb = 1 << lgnb;
    const int total = R << lgnb;
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
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
__device__ __forceinline__ C c2r_pack_g(const C* X, int s, int Nc, const C* pre) { return c2r_pack(X, s, Nc, pre); }

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

// Real inverse DFT (prefactor 1) of R rings straight into their output rows gout[r]:
// buf0 holds the packed coefficients (slot 0 = (X_0, X_Nc), slot s = X_s); buf1 is the
// second ping-pong buffer.  The last pass writes global memory (rows of n_phi reals viewed
// as Nc complex (x_{2n}, x_{2n+1})).  One barrier per shared-memory pass; on return both
// buffers may be reused after the caller's next barrier.
template <class C>
__device__ __forceinline__ void c2r_rings_to_global(C* buf0, C* buf1, int R, int lgNc, const C* twp,
                                                    const C* pre, C* const* gout)
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
                if (last) fft_pass<C, 4, true, true>(src, dst, R, lgNc, Ns, twp + off, pre, gout);
                else fft_pass<C, 4, true, false>(src, dst, R, lgNc, Ns, twp + off, pre, gout);
            } else {
                if (last) fft_pass<C, 4, false, true>(src, dst, R, lgNc, Ns, twp + off, pre, gout);
                else fft_pass<C, 4, false, false>(src, dst, R, lgNc, Ns, twp + off, pre, gout);
            }
        } else {
            if (first) {
                if (last) fft_pass<C, 2, true, true>(src, dst, R, lgNc, Ns, twp + off, pre, gout);
                else fft_pass<C, 2, true, false>(src, dst, R, lgNc, Ns, twp + off, pre, gout);
            } else {
                if (last) fft_pass<C, 2, false, true>(src, dst, R, lgNc, Ns, twp + off, pre, gout);
                else fft_pass<C, 2, false, false>(src, dst, R, lgNc, Ns, twp + off, pre, gout);
            }
        }
        if (!first) off += (RP - 1) * Ns;
        Ns *= RP;
        first = false;
        if (!last) __syncthreads();
        C* t = src;
        src = dst;
        dst = t;
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

// x <- A x + C x_right + B xi for one real chain (tables t = [A | C | B], B lower); x_right
// is read at xr[q * Nc] (null when the segment has no right anchor).
template <class Real, int M>
__device__ __forceinline__ void step_state(const Real* t, Real (&x)[M], const Real (&xi)[M], const Real* xr, int Nc)
{
    Real xn[M];
#pragma unroll
    for (int p = 0; p < M; ++p) {
        Real acc = 0;
#pragma unroll
        for (int q = 0; q < M; ++q) acc = fma(t[p * M + q], x[q], acc);
        if (xr) {
#pragma unroll
            for (int q = 0; q < M; ++q) acc = fma(t[M * M + p * M + q], xr[(size_t)q * Nc], acc);
        }
        int e = 2 * M * M + p * (p + 1) / 2;
#pragma unroll
        for (int q = 0; q <= p; ++q, ++e) acc = fma(t[e], xi[q], acc);
        xn[p] = acc;
    }
#pragma unroll
    for (int q = 0; q < M; ++q) x[q] = xn[q];
}

template <class Real, class TabT, int M, int UPT, int RMAX, bool INPLACE>
__global__ void __launch_bounds__(1024) segment_kernel(SampleParams P)
{
    using C = cplx<Real>;
    constexpr int G = kG<M>;
    constexpr int E = step_elems(M);
    constexpr int EPT = RMAX * UPT * G;   // complex FFT points per thread (in-place mode)
    extern __shared__ __align__(16) unsigned char smem_raw[];

    const Segment sg = P.segs[blockIdx.x];
    const int r0 = blockIdx.y * RMAX;
    const int R = min(RMAX, P.n_samples - r0);
    const int c = sg.chain;
    const int nt = blockDim.x, tid = threadIdx.x;
    const int Nc = P.Nc;
    const size_t mp = P.n_modes_pad;
    const Real* anc = (const Real*)P.anc;
    const bool has_right = sg.right >= 0;

    // shared memory: FFT buffer(s), then (ping-pong mode) the right-anchor states
    C* buf0 = reinterpret_cast<C*>(smem_raw);
    C* buf1 = buf0 + (size_t)RMAX * Nc;
    Real* xRs = reinterpret_cast<Real*>(buf0 + (size_t)RMAX * Nc * (INPLACE ? 1 : 2));
    const C* twp = (const C*)P.tw;
    const C* pre = (const C*)P.pre;
    // right-anchor states: shared memory in ping-pong mode, the scratch itself in place mode;
    // layout [f][slot] per realisation in both
    const Real* xrg[RMAX];
#pragma unroll
    for (int r = 0; r < RMAX; ++r)
        xrg[r] = anc + aoff<M>(P, c, min(r0 + r, P.n_samples - 1), has_right ? sg.right : 0, 0, 0);
    if (!INPLACE && has_right) {
        const int per = 2 * M * Nc;
        for (int idx = tid; idx < R * per; idx += nt) {
            const int r = idx / per, rest = idx - r * per;
            xRs[idx] = anc[aoff<M>(P, c, r0 + r, sg.right, 0, 0) + rest];
        }
    }

    Real x[UPT][RMAX][G][2][M];
#pragma unroll
    for (int i = 0; i < UPT; ++i) {
        const int u = tid + i * nt;
#pragma unroll
        for (int r = 0; r < RMAX; ++r)
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int part = 0; part < 2; ++part)
#pragma unroll
                    for (int q = 0; q < M; ++q)
                        x[i][r][g][part][q] = (u < P.n_units && r < R)
                                                  ? anc[aoff<M>(P, c, r0 + r, sg.left, part * M + q, G * u + g)]
                                                  : (Real)0;
    }
    __syncthreads();

    const TabT* steps = (const TabT*)P.steps[c];
    for (int pos = sg.p0; pos < sg.p1; ++pos) {
        const int ring = c == 0 ? P.k0 - pos : P.k0 + pos;
        if (pos > sg.p0) {
            const TabT* tb = steps + (size_t)pos * E * mp;
#pragma unroll
            for (int i = 0; i < UPT; ++i) {
                const int u = tid + i * nt;
                if (u >= P.n_units) continue;
                // tables of the unit's slots (mode = slot); slot 0's second chain is the
                // Nyquist mode, stepped on a separate path that only unit 0 takes
                Real ta[G][E];
#pragma unroll
                for (int g = 0; g < G; ++g)
#pragma unroll
                    for (int e = 0; e < E; ++e) ta[g][e] = tabld<Real, TabT>(tb + (size_t)e * mp + G * u + g);
#pragma unroll
                for (int r = 0; r < RMAX; ++r) {
                    if (r >= R) continue;
                    Real nr[4];
                    unit_normals<Real>(P.seed + (uint64_t)(r0 + r), (uint32_t)u, (uint32_t)ring, nr);
#pragma unroll
                    for (int g = 0; g < G; ++g) {
                        const int s = G * u + g;
#pragma unroll
                        for (int part = 0; part < 2; ++part) {
                            Real xi[M];
#pragma unroll
                            for (int q = 0; q < M; ++q) {
                                const Real v = nr[g * 2 * M + part * M + q];
                                xi[q] = (c == 1 && (q & 1)) ? -v : v;
                            }
                            const Real* xr = INPLACE ? xrg[r] + (size_t)part * M * Nc + s
                                                     : xRs + ((size_t)r * 2 * M + part * M) * Nc + s;
                            if (part == 1 && s == 0) {
                                Real tn[E];
#pragma unroll
                                for (int e = 0; e < E; ++e) tn[e] = tabld<Real, TabT>(tb + (size_t)e * mp + Nc);
                                step_state<Real, M>(tn, x[i][r][g][part], xi, has_right ? xr : nullptr, Nc);
                            } else {
                                step_state<Real, M>(ta[g], x[i][r][g][part], xi, has_right ? xr : nullptr, Nc);
                            }
                        }
                    }
                }
            }
        }
        // coefficients of this ring into shared memory
#pragma unroll
        for (int i = 0; i < UPT; ++i) {
            const int u = tid + i * nt;
            if (u >= P.n_units) continue;
#pragma unroll
            for (int r = 0; r < RMAX; ++r) {
                if (r >= R) continue;
#pragma unroll
                for (int g = 0; g < G; ++g)
                    buf0[(size_t)r * Nc + G * u + g] = cmk<C>(x[i][r][g][0][0], x[i][r][g][1][0]);
            }
        }
        __syncthreads();
        if (!(c == 1 && pos == 0)) {  // the start ring is written by the northern chain
            if (INPLACE) {
                c2r_rings_inplace<C, EPT>(buf0, R, P.lgNc, twp, pre);
                for (int r = 0; r < R; ++r) {
                    Real* dst = (Real*)P.out + ((size_t)(r0 + r) * P.n_theta + ring) * (size_t)P.n_phi;
                    store_ring<Real>(dst, buf0 + (size_t)r * Nc, Nc, tid, nt);
                }
            } else {
                C* gout[RMAX];
#pragma unroll
                for (int r = 0; r < RMAX; ++r)
                    gout[r] = (C*)((Real*)P.out + ((size_t)min(r0 + r, P.n_samples - 1) * P.n_theta + ring) * (size_t)P.n_phi);
                c2r_rings_to_global<C>(buf0, buf1, R, P.lgNc, twp, pre, gout);
            }
        }
        __syncthreads();  // buffers are rewritten by the next ring
    }
}

// ------------------------------------------------------------------ launch
template <class Real, class TabT, int M, int UPT, int RMAX, bool INPLACE = false>
int launch_segments(const SampleParams& P, int n_segments, int nt, size_t smem, cudaStream_t st)
{
    auto kern = segment_kernel<Real, TabT, M, UPT, RMAX, INPLACE>;
    if (smem > 48 * 1024) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return SMERF_ECUDA;
    }
    dim3 grid(n_segments, (P.n_samples + RMAX - 1) / RMAX);
    kern<<<grid, nt, smem, st>>>(P);
    return cudaGetLastError() == cudaSuccess ? SMERF_OK : SMERF_ECUDA;
}

// (units per thread, realisations per CTA) pairs that are built: four realisations per CTA
// share each table load while the state fits in 64 registers, fewer for wide grids;
// FP64 recursion keeps one.
template <class Real> constexpr int rmax_for(int upt)
{
    return sizeof(Real) == 8 ? 1 : (upt == 1 ? 4 : (upt == 2 ? 2 : 1));
}

template <class Real, class TabT, int M>
int dispatch_upt(const SampleParams& P, int n_segments, int upt, int nt, size_t smem, cudaStream_t st)
{
    switch (upt) {
        case 1: return launch_segments<Real, TabT, M, 1, rmax_for<Real>(1)>(P, n_segments, nt, smem, st);
        case 2: return launch_segments<Real, TabT, M, 2, rmax_for<Real>(2)>(P, n_segments, nt, smem, st);
        case 4:
            return P.pingpong ? launch_segments<Real, TabT, M, 4, rmax_for<Real>(4)>(P, n_segments, nt, smem, st)
                              : launch_segments<Real, TabT, M, 4, rmax_for<Real>(4), true>(P, n_segments, nt, smem, st);
        case 8:
            return P.pingpong ? launch_segments<Real, TabT, M, 8, rmax_for<Real>(8)>(P, n_segments, nt, smem, st)
                              : launch_segments<Real, TabT, M, 8, rmax_for<Real>(8), true>(P, n_segments, nt, smem, st);
        default: return SMERF_EUNSUPPORTED;
    }
}

constexpr int kMaxThreads = 1024;
constexpr size_t kMaxSmem = 227 * 1024;

// Launch configuration of the segment kernel for a plan: units per thread, threads,
// realisations per CTA and the optional shared-memory parts.
struct SegConfig { int upt, nt, rmax; size_t smem; int pingpong; };

template <class Real>
inline SegConfig seg_config(const smerf_plan* pl)
{
    SegConfig cfg{};
    const int M = pl->p;
    const int n_units = pl->n_slots / unit_slots(M);
    int upt = 1;
    while (upt < 8 && (n_units + upt - 1) / upt > kMaxThreads) upt *= 2;
    int nt = (n_units + upt - 1) / upt;
    nt = ((nt + 31) / 32) * 32;
    if (nt < 64) nt = 64;
    const int rmax = rmax_for<Real>(upt);
    const int Nc = pl->n_phi / 2;
    const size_t one = (size_t)rmax * Nc * 2 * sizeof(Real);
    const size_t xr = pl->H > 0 ? (size_t)rmax * 2 * M * Nc * sizeof(Real) : 0;
    cfg.upt = upt;
    cfg.nt = nt;
    cfg.rmax = rmax;
    // ping-pong: two FFT buffers and the right-anchor states on chip; otherwise one buffer
    cfg.pingpong = (2 * one + xr <= kMaxSmem) ? 1 : 0;
    cfg.smem = cfg.pingpong ? 2 * one + xr : one;
    return cfg;
}

template <class Real, class TabT>
int launch_sample_t(const smerf_plan* pl, uint64_t seed, int n, void* out, void* scratch, cudaStream_t st,
                    cudaEvent_t ev0, cudaEvent_t ev1)
{
    SampleParams P;
    P.segs = pl->segs_dev;
    P.steps[0] = pl->steps[0];
    P.steps[1] = pl->steps[1];
    P.coarse[0] = pl->coarse[0];
    P.coarse[1] = pl->coarse[1];
    P.beq = pl->beq;
    P.tw = pl->tw;
    P.pre = pl->pre;
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
    const SegConfig cfg = seg_config<Real>(pl);
    if (cfg.smem > kMaxSmem) return SMERF_EUNSUPPORTED;  // one ring per realisation must fit on chip
    if ((pl->n_slots / unit_slots(pl->p) + cfg.upt - 1) / cfg.upt > kMaxThreads) return SMERF_EUNSUPPORTED;
    if (!cfg.pingpong && cfg.upt < 4) return SMERF_EUNSUPPORTED;
    P.pingpong = cfg.pingpong;
    int lg = 0;
    while ((1 << lg) < P.Nc) ++lg;
    P.lgNc = lg;
    {
        dim3 ga((P.n_units + 127) / 128, n, 2);
        if (pl->p == 1) anchor_kernel<Real, TabT, 1><<<ga, 128, 0, st>>>(P);
        else anchor_kernel<Real, TabT, 2><<<ga, 128, 0, st>>>(P);
        if (cudaGetLastError() != cudaSuccess) return SMERF_ECUDA;
    }
    if (ev0 && cudaEventRecord(ev0, st) != cudaSuccess) return SMERF_ECUDA;
    const int rc = pl->p == 1 ? dispatch_upt<Real, TabT, 1>(P, pl->n_segments, cfg.upt, cfg.nt, cfg.smem, st)
                              : dispatch_upt<Real, TabT, 2>(P, pl->n_segments, cfg.upt, cfg.nt, cfg.smem, st);
    if (rc == SMERF_OK && ev1 && cudaEventRecord(ev1, st) != cudaSuccess) return SMERF_ECUDA;
    return rc;
}

}  // namespace smerf
