// smerf_ring.cuh -- the segment kernel for long rings with one real state per chain (p = 1,
// FP32 recursion and FFT, n_phi = 2 Nc with Nc = 2^LG complex points, LG = 13 or 14): one CTA
// of NT = Nc / 16 threads per (segment, realisation).  Included by smerf_sample_impl.cuh.
//
// Per ring: every thread steps its units (Eq. (state_space), two slots per Philox call) and
// writes their coefficients into the ring buffer; then the ring's C2R FFT runs in place in
// four Stockham passes of radix 16, 16 (or 8), 8, 8 with every thread holding 16 points, and
// the last pass streams the ring to HBM.  Pass 0 fuses the C2R packing: its packing factors
// e^{2 pi i s / n_phi} for s = j + NT i are pre[j] times the constants e^{2 pi i i / 32}.
// Later passes load one twiddle e^{2 pi i kk / (Ns R)} per butterfly (the first row of the
// per-pass table) and form its powers by repeated products, so the tables a CTA reads stay
// small enough for L1.  While a ring's FFT runs, the next ring's step rows are prefetched into
// L2 (cp.async.bulk.prefetch), so the recursion's table loads hit L2.  Only pass 0's stride-16
// stores need a swizzle for conflict-free shared memory: its 16-byte chunk q of row r is stored
// at chunk q ^ (r & 7).  In the 16384-point
// ring's two radix-8 passes a thread takes two neighbouring butterflies, so that its shared
// accesses, twiddle loads and the last pass's stores to HBM are 16-byte vector accesses.
#pragma once

namespace smerf {

// e^{2 pi i t / 32}, t < 16
__device__ __forceinline__ float2 e32(int t)
{
    constexpr float c[16] = {1.000000000e+00f, 9.807852804e-01f, 9.238795325e-01f, 8.314696123e-01f,
                             7.071067812e-01f, 5.555702330e-01f, 3.826834324e-01f, 1.950903220e-01f,
                             0.0f, -1.950903220e-01f, -3.826834324e-01f, -5.555702330e-01f,
                             -7.071067812e-01f, -8.314696123e-01f, -9.238795325e-01f, -9.807852804e-01f};
    constexpr float s[16] = {0.0f, 1.950903220e-01f, 3.826834324e-01f, 5.555702330e-01f,
                             7.071067812e-01f, 8.314696123e-01f, 9.238795325e-01f, 9.807852804e-01f,
                             1.000000000e+00f, 9.807852804e-01f, 9.238795325e-01f, 8.314696123e-01f,
                             7.071067812e-01f, 5.555702330e-01f, 3.826834324e-01f, 1.950903220e-01f};
    return make_float2(c[t], s[t]);
}

template <int LG>
struct RingPass {
    template <int PI>
    struct P {
        static constexpr int B = hr_bits(LG, PI, 4);
        static constexpr int R = 1 << B;
        static constexpr int Ns = 1 << hr_lgns(LG, PI, 4);
        static constexpr int NB = (1 << LG) >> B;        // butterflies
        static constexpr int KB = 16 / R;                // butterflies per thread
        static constexpr bool LAST = PI == hr_passes(LG, 4) - 1;
        static constexpr int TW = hr_off(LG, PI, 4);     // first twiddle row of the pass in tw2
    };
    static constexpr int Nc = 1 << LG;
    static constexpr int NT = Nc / 16;
};

// element e of pass 0's output (rows of 16 complex values, 16-byte chunks swizzled)
__device__ __forceinline__ int ring_swz(int e)
{
    const int r = e >> 4, c = e & 15;
    return (r << 4) + ((((c >> 1) ^ (r & 7))) << 1) + (c & 1);
}

// v[a] *= w^a, a = 1..R-1 (powers by repeated products)
template <int R>
__device__ __forceinline__ void ring_twiddle(float2* v, float2 w)
{
    float2 t = w;
    v[1] = cmul(v[1], t);
#pragma unroll
    for (int a = 2; a < R; ++a) {
        t = cmul(t, w);
        v[a] = cmul(v[a], t);
    }
}

// pass 0: C2R packing + radix 16 (Ns = 1), swizzled stores
template <int LG>
__device__ __forceinline__ void ring_pass0(float2* X, const float2* __restrict__ pre, int tid)
{
    constexpr int Nc = RingPass<LG>::Nc, NT = RingPass<LG>::NT;
    float2 v[16];
    const float2 pj = __ldg(pre + tid);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int s = tid + NT * i;
        const float2 a = X[s];
        const float2 bb = cconj(X[(Nc - s) & (Nc - 1)]);
        const float2 ps = i == 0 ? pj : cmul(pj, e32(i));
        const float2 g = cadd(cadd(a, bb), cmuli(cmul(ps, csub(a, bb))));
        v[i] = (i == 0 && tid == 0) ? make_float2(a.x + a.y, a.x - a.y) : g;
    }
    dft16(v);
    __syncthreads();  // every read of the coefficients before any write
    float4* row = reinterpret_cast<float4*>(X + 16 * tid);
#pragma unroll
    for (int q = 0; q < 8; ++q) row[q ^ (tid & 7)] = make_float4(v[2 * q].x, v[2 * q].y, v[2 * q + 1].x, v[2 * q + 1].y);
    __syncthreads();
}

// pass PI >= 1: KB butterflies of radix R per thread (j = tid + q NT), in place; the last pass
// writes the ring's complex points z_n = x_{2n} + i x_{2n+1} to HBM
template <int LG, int PI>
__device__ __forceinline__ void ring_pass(float2* X, const float2* __restrict__ tw2, float2* __restrict__ gout, int tid)
{
    using PP = typename RingPass<LG>::template P<PI>;
    constexpr int R = PP::R, Ns = PP::Ns, NB = PP::NB, KB = PP::KB, NT = RingPass<LG>::NT;
    if constexpr (LG == 14 && KB == 2 && PI >= 2) {
        // the radix-8 passes of the 16384-point ring: butterflies j = 2 tid and 2 tid + 1, whose
        // points, twiddles and outputs are adjacent, so that every shared, twiddle and output
        // access is one 16-byte vector access for both (j < NB = 2 NT; Ns >= 256, so both share
        // one block of Ns and their outputs are neighbours)
        static_assert(2 * NT == NB && Ns >= 64 && Ns % 2 == 0, "two neighbouring butterflies per thread");
        float2 v[2][R];
        const int j = 2 * tid;
        const int kk = j & (Ns - 1);
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const float4 w = reinterpret_cast<const float4*>(X)[(j + i * NB) >> 1];
            v[0][i] = make_float2(w.x, w.y);
            v[1][i] = make_float2(w.z, w.w);
        }
        const float4 t = __ldg(reinterpret_cast<const float4*>(tw2 + PP::TW + kk));
        ring_twiddle<R>(v[0], make_float2(t.x, t.y));
        dft<float2, R>(v[0]);
        ring_twiddle<R>(v[1], make_float2(t.z, t.w));
        dft<float2, R>(v[1]);
        if constexpr (!PP::LAST) __syncthreads();  // every read of this pass before any write
        const int idx = (j - kk) * R + kk;
#pragma unroll
        for (int a = 0; a < R; ++a) {
            const float4 w = make_float4(v[0][a].x, v[0][a].y, v[1][a].x, v[1][a].y);
            if constexpr (PP::LAST) __stcs(reinterpret_cast<float4*>(gout + idx + a * Ns), w);
            else reinterpret_cast<float4*>(X)[(idx + a * Ns) >> 1] = w;
        }
        if constexpr (!PP::LAST) {
            __syncthreads();
            ring_pass<LG, PI + 1>(X, tw2, gout, tid);
        }
        return;
    }
    float2 v[KB][R];
#pragma unroll
    for (int q = 0; q < KB; ++q) {
        const int j = tid + q * NT;
        const int kk = j & (Ns - 1);
#pragma unroll
        for (int i = 0; i < R; ++i) v[q][i] = PI == 1 ? X[ring_swz(j + i * NB)] : X[j + i * NB];
        ring_twiddle<R>(v[q], __ldg(tw2 + PP::TW + kk));
        dft<float2, R>(v[q]);
    }
    if constexpr (!PP::LAST) __syncthreads();  // every read of this pass before any write
#pragma unroll
    for (int q = 0; q < KB; ++q) {
        const int j = tid + q * NT;
        const int kk = j & (Ns - 1);
        const int idx = (j - kk) * R + kk;
        if constexpr (PP::LAST) {
#pragma unroll
            for (int a = 0; a < R; ++a) __stcs(gout + idx + a * Ns, v[q][a]);
        } else {
#pragma unroll
            for (int a = 0; a < R; ++a) X[idx + a * Ns] = v[q][a];
        }
    }
    if constexpr (!PP::LAST) {
        __syncthreads();
        ring_pass<LG, PI + 1>(X, tw2, gout, tid);
    }
}

// Asynchronous prefetch of [p, p + bytes) into L2 by the CTA's first 16 threads (p and bytes
// multiples of 16): the next ring's step rows are fetched while this ring's FFT runs
__device__ __forceinline__ void ring_l2_prefetch(const void* p, size_t bytes, int tid)
{
    constexpr int kParts = 16;
    const size_t chunk = ((bytes / kParts + 15) / 16) * 16;
    const size_t off = (size_t)tid * chunk;
    if (tid < kParts && off < bytes) {
        const size_t n = bytes - off < chunk ? bytes - off : chunk;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"((const char*)p + off), "r"((unsigned)n) : "memory");
    }
}

// One CTA per (segment, realisation r = blockIdx.x); NT threads, thread t owns units
// u = t + i NT (slots 2u, 2u + 1), i < 8; the states of units i >= 8 - PARK live in shared
// memory between their steps.
// PACKED: FP32 tables stored as three rows A, C, B per position, mode fastest (smerf_plan.packed)
template <class TabT, int LG, int PARK, int MINB, bool PACKED>
__global__ void __launch_bounds__(RingPass<LG>::NT, MINB) ring_kernel(SampleParams P)
{
    constexpr int Nc = RingPass<LG>::Nc, NT = RingPass<LG>::NT;
    constexpr int U = 8, UP = U - PARK;
    constexpr int ROW = PACKED ? 3 : step_row(1);  // values per (mode, ring) as stored
    static_assert(!PACKED || sizeof(TabT) == 4, "packed tables are FP32");
    static_assert(Nc / 2 == U * NT, "8 units of two slots per thread");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint2 rk[10];  // Philox round keys of the CTA's realisation

    const Segment sg = P.segs[blockIdx.y];
    const int r0 = blockIdx.x;
    const int c = sg.chain;
    const int tid = threadIdx.x;
    const size_t mp = P.n_modes_pad;
    const float* anc = (const float*)P.anc;
    const bool has_right = sg.right >= 0;

    float2* X = reinterpret_cast<float2*>(smem_raw);                 // the ring, Nc complex
    float4* park = reinterpret_cast<float4*>(smem_raw + (size_t)Nc * sizeof(float2));  // [PARK][NT]
    if (tid < 10) {
        const uint64_t key = P.seed + (uint64_t)r0;
        rk[tid] = make_uint2((uint32_t)key + (uint32_t)tid * 0x9E3779B9u, (uint32_t)(key >> 32) + (uint32_t)tid * 0xBB67AE85u);
    }
    const float* xrg = anc + aoff<1>(P, c, r0, has_right ? sg.right : 0, 0, 0);

    float4 xreg[UP > 0 ? UP : 1];
#pragma unroll
    for (int i = 0; i < U; ++i) {
        const int u = tid + i * NT;
        const float4 v = __ldg(reinterpret_cast<const float4*>(anc + aoff<1>(P, c, r0, sg.left, 0, 2 * u)));
        if (i < UP) xreg[i < UP ? i : 0] = v;
        else park[(i - UP) * NT + tid] = v;
    }
    __syncthreads();

    const TabT* steps = (const TabT*)(c == 0 ? P.steps[0] : P.steps[1]);
    const size_t ring_tab_bytes = mp * ROW * sizeof(TabT);  // one ring's step rows, a multiple of 16
    if (sg.p0 + 1 < sg.p1) ring_l2_prefetch(steps + (size_t)(sg.p0 + 1) * mp * ROW, ring_tab_bytes, tid);
    for (int pos = sg.p0; pos < sg.p1; ++pos) {
        const int ring = c == 0 ? P.k0 - pos : P.k0 + pos;
        const TabT* tb = steps + (size_t)pos * mp * ROW;
#pragma unroll
        for (int i = 0; i < U; ++i) {
            const int u = tid + i * NT;
            float4 x = i < UP ? xreg[i < UP ? i : 0] : park[(i - UP) * NT + tid];
            if (pos > sg.p0) {
                float t0[4], t1[4];
                if constexpr (PACKED) {
                    const float* ta = (const float*)tb;
                    const float2 a = __ldg(reinterpret_cast<const float2*>(ta + 2 * u));
                    const float2 cc = __ldg(reinterpret_cast<const float2*>(ta + mp + 2 * u));
                    const float2 bb = __ldg(reinterpret_cast<const float2*>(ta + 2 * mp + 2 * u));
                    t0[0] = a.x, t0[1] = cc.x, t0[2] = bb.x;
                    t1[0] = a.y, t1[1] = cc.y, t1[2] = bb.y;
                } else {
                    load_row<float, TabT, 4>(tb + (size_t)(2 * u) * ROW, t0);
                    load_row<float, TabT, 4>(tb + (size_t)(2 * u + 1) * ROW, t1);
                }
                float nr[4];
                unit_normals_rk<float>(rk, (uint32_t)u, (uint32_t)ring, nr);
                float4 xr = make_float4(0.f, 0.f, 0.f, 0.f);
                if (has_right) xr = __ldg(reinterpret_cast<const float4*>(xrg + 4 * u));
                // slot 2u: (x.x Re, x.y Im); slot 2u + 1: (x.z, x.w).  Row: A, C, B.
                float tn0 = t0[0], tn1 = t0[1], tn2 = t0[2];
                if (i == 0 && u == 0) {  // slot 0's second chain is the Nyquist mode (own row)
                    if constexpr (PACKED) {
                        const float* ta = (const float*)tb;
                        tn0 = ta[Nc];
                        tn1 = ta[mp + Nc];
                        tn2 = ta[2 * mp + Nc];
                    } else {
                        float tn[4];
                        load_row<float, TabT, 4>(tb + (size_t)Nc * ROW, tn);
                        tn0 = tn[0];
                        tn1 = tn[1];
                        tn2 = tn[2];
                    }
                }
                // x = A x + C x_right + B xi, accumulated in that order (C x_right = 0 exactly
                // without a right anchor)
                x.x = fmaf(t0[2], nr[0], fmaf(t0[1], xr.x, t0[0] * x.x));
                x.y = fmaf(tn2, nr[1], fmaf(tn1, xr.y, tn0 * x.y));
                x.z = fmaf(t1[2], nr[2], fmaf(t1[1], xr.z, t1[0] * x.z));
                x.w = fmaf(t1[2], nr[3], fmaf(t1[1], xr.w, t1[0] * x.w));
                if (i < UP) xreg[i < UP ? i : 0] = x;
                else park[(i - UP) * NT + tid] = x;
            }
            reinterpret_cast<float4*>(X)[u] = x;  // the unit's two coefficients
        }
        if (pos + 1 < sg.p1) ring_l2_prefetch(tb + mp * ROW, ring_tab_bytes, tid);
        __syncthreads();
        if (!(c == 1 && pos == 0)) {  // the start ring is written by the northern chain
            float2* dst = reinterpret_cast<float2*>((float*)P.out + ((size_t)r0 * P.n_theta + ring) * (size_t)P.n_phi);
            ring_pass0<LG>(X, (const float2*)P.pre, tid);
            ring_pass<LG, 1>(X, (const float2*)P.tw2, dst, tid);
        }
        __syncthreads();  // the buffer is rewritten by the next ring
    }
}

}  // namespace smerf
