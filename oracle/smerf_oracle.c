/*
 * smerf_oracle.c -- the oracle: a plain, slow FP64 CPU restatement of the sampler of
 * Creasey & Lang, "Fast generation of isotropic Gaussian random fields on the sphere"
 * (arXiv 1709.10314).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call this
 * file: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * arm use it.  It shares no source with the CUDA path.
 *
 * What lives here (the heavy loops); the Python side (oracle/oracle.py) does the dense
 * Cholesky (LAPACK), the ordering and the assembly.
 *
 *  - Philox4x32-10 counter-based generator, from its published definition
 *    (Salmon, Moraes, Dror, Shaw, SC'11 "Parallel random numbers: as easy as 1, 2, 3").
 *  - Box-Muller transform (u = (x + 1/2) 2^-32).
 *  - Normalised associated Legendre functions L_lm (Sec. 2, definition of L_lm; with the
 *    Condon-Shortley phase of P_lm) by the standard three-term recurrence in l, with an
 *    extended exponent so that seeds sin(theta)^m never underflow.
 *  - The per-mode cross covariance of the U-basis state (Lemma 2.1 and the U-basis,
 *    Eq. (Jmatrix_more_efficient)):
 *        J^m_pq(z,z') = sum_{l>=m} C_l N_lm^2 P_l^{m+p}(z) P_l^{m+q}(z'),
 *    where N_lm P_l^{m+q} = s_lmq L_{l,m+q}, s_lmq^2 = prod_{j<q} (l-m-j)(l+m+1+j),
 *    and C_l = A / prod_i (l(l+1) + kappa-hat_i) (Eq. (Cl)); every function takes the
 *    kappa-hat_i as (re, im) pairs ("khat"), kappa-hat_i = kappa_i^2 for a real kappa.
 *    The series is summed with a smooth cut-off window w((l+1/2)/L) and, on the
 *    same-ring blocks (whose tail does not oscillate), Richardson-extrapolated in 1/L
 *    over K levels L, 2L, ..., 2^(K-1) L.
 *  - The naive O(n_phi^2) real DFT of one ring (Alg. 2, last step; prefactor 1), and the
 *    same synthesis through a textbook radix-2 FFT.
 *  - Alg. 2's per-sample recursion with tables given (the oracle derives them by Gaussian
 *    conditioning of its spectral-sum covariance): the CPU baseline of the sampler.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ---------------------------------------------------------------- Philox4x32-10 */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u; /* round multipliers */
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u; /* Weyl key increments */
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        if (r > 0) { k0 += W0; k1 += W1; }
        mulhilo32(M0, x0, &hi0, &lo0);
        mulhilo32(M1, x2, &hi1, &lo1);
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Box-Muller on two 32-bit words: u = (x + 1/2) 2^-32 lies in (0,1) and is exact in FP64. */
static void box_muller(uint32_t a, uint32_t b, double *n0, double *n1)
{
    double u0 = ((double)a + 0.5) * 2.3283064365386962890625e-10;
    double u1 = ((double)b + 0.5) * 2.3283064365386962890625e-10;
    double r = sqrt(-2.0 * log(u0));
    double t = 2.0 * M_PI * u1;
    *n0 = r * cos(t);
    *n1 = r * sin(t);
}

/* The first n standard normals of ring `ring` of the realisation whose 64-bit Philox key
 * is key64: call j uses counter (j, ring, 0, 0) and yields normals 4j..4j+3. */
void oracle_ring_normals(uint64_t key64, uint32_t ring, int64_t n, double *out)
{
    uint32_t key[2] = {(uint32_t)key64, (uint32_t)(key64 >> 32)};
    for (int64_t j = 0; 4 * j < n; ++j) {
        uint32_t ctr[4] = {(uint32_t)j, ring, 0u, 0u}, w[4];
        double v[4];
        oracle_philox4x32_10(ctr, key, w);
        box_muller(w[0], w[1], &v[0], &v[1]);
        box_muller(w[2], w[3], &v[2], &v[3]);
        for (int i = 0; i < 4 && 4 * j + i < n; ++i) out[4 * j + i] = v[i];
    }
}

void oracle_raw_uint32(uint64_t key64, uint32_t ring, int64_t ncalls, uint32_t *out)
{
    uint32_t key[2] = {(uint32_t)key64, (uint32_t)(key64 >> 32)};
    for (int64_t j = 0; j < ncalls; ++j) {
        uint32_t ctr[4] = {(uint32_t)j, ring, 0u, 0u};
        oracle_philox4x32_10(ctr, key, out + 4 * j);
    }
}

/* ------------------------------------------------------ spectrum and the window */
/* khat: kappa-hat_i as (re, im) pairs.  The product prod_i (l(l+1) + kappa-hat_i) is real
   when the kappa-hat are real or come in complex-conjugate pairs (Eq. (Cl); Sec. 5 uses the
   pair +-i sqrt(10)); its real part is taken. */
double oracle_Cl(int l, int M, const double *khat, double A)
{
    double dr = 1.0, di = 0.0, ll = (double)l * (double)(l + 1);
    for (int i = 0; i < M; ++i) {
        const double ar = ll + khat[2 * i], ai = khat[2 * i + 1];
        const double nr = dr * ar - di * ai, ni = dr * ai + di * ar;
        dr = nr;
        di = ni;
    }
    return A / dr;
}

/* Smooth cut-off: 1 on [0,1/2], 0 on [1,inf), C-infinity in between. */
static double window(double t)
{
    if (t <= 0.5) return 1.0;
    if (t >= 1.0) return 0.0;
    double u = (t - 0.5) / 0.5;
    double a = exp(-1.0 / u), b = exp(-1.0 / (1.0 - u));
    return 1.0 - a / (a + b);
}

/* ------------------------------------------ normalised Legendre recurrence in l
 * State of the recurrence for one (z, order mu): the two latest values scaled by
 * 2^e.  L_{mu,mu}(z) = (-1)^mu sqrt((2mu+1)/(4pi) prod_{i<=mu} (2i-1)/(2i)) (1-z^2)^{mu/2},
 * L_{mu+1,mu} = z sqrt(2mu+3) L_{mu,mu},
 * L_{l,mu} = a_l (z L_{l-1,mu} - b_l L_{l-2,mu}),
 * a_l = sqrt((4l^2-1)/(l^2-mu^2)), b_l = sqrt(((l-1)^2-mu^2)/(4(l-1)^2-1)).          */
typedef struct { double z, prev, cur; int e; int l; int mu; } legrec;

static void legrec_init(legrec *r, int mu, double z)
{
    double s = sqrt((1.0 - z) * (1.0 + z));
    double lg = 0.0; /* log2 of |seed| */
    lg += 0.5 * log2(1.0 / (4.0 * M_PI));
    for (int i = 1; i <= mu; ++i) lg += 0.5 * log2((2.0 * i + 1.0) / (2.0 * i)) + log2(s);
    int e = (int)floor(lg);
    r->z = z; r->mu = mu; r->l = mu; r->e = e;
    r->prev = 0.0;
    r->cur = ((mu & 1) ? -1.0 : 1.0) * exp2(lg - e);
}

/* advance to l+1 */
static void legrec_step(legrec *r)
{
    int l = r->l + 1, mu = r->mu;
    double nxt;
    if (l == mu + 1) {
        nxt = r->z * sqrt(2.0 * mu + 3.0) * r->cur;
    } else {
        double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)mu * mu));
        double b = sqrt((((double)(l - 1) * (l - 1)) - (double)mu * mu) / (4.0 * (l - 1) * (l - 1) - 1.0));
        nxt = a * (r->z * r->cur - b * r->prev);
    }
    r->prev = r->cur; r->cur = nxt; r->l = l;
    double m = fabs(nxt) > fabs(r->prev) ? fabs(nxt) : fabs(r->prev);
    if (m > 0x1p200 && r->e < 0) { /* values grow from tiny seeds: renormalise */
        r->prev *= 0x1p-200; r->cur *= 0x1p-200; r->e += 200;
    }
}

/* true value of the current L_{l,mu}, or 0 if below 2^-1000 */
static double legrec_value(const legrec *r)
{
    if (r->e < -1000) return 0.0;
    return ldexp(r->cur, r->e);
}

/* s_lmq = sqrt(prod_{j<q} (l-m-j)(l+m+1+j)); zero when l < m+q */
static double s_factor(int l, int m, int q)
{
    if (l < m + q) return 0.0;
    double p = 1.0;
    for (int j = 0; j < q; ++j) p *= (double)(l - m - j) * (double)(l + m + 1 + j);
    return sqrt(p);
}

/*
 * Cross covariance blocks of the U-basis state of mode m at n points z[0..n-1]
 * (Lemma 2.1 with the U-basis of Eq. (Jmatrix_more_efficient)).
 * Output Sigma is (n*M) x (n*M), row-major, index (k*M+p, k2*M+q).
 *
 * Off-diagonal blocks (k != k2): one windowed sum with cut-off Loff.
 * Same-point blocks (k == k2): windowed sums at Ld[k] * 2^i, i < K, Richardson-
 * extrapolated in 1/L.
 * Returns 0 on success, -1 on bad arguments.
 */
int oracle_cov_m(int m, int M, const double *khat, double A, int n, const double *z,
                 long Loff, const long *Ld, int K, double *Sigma)
{
    if (M < 1 || M > 4 || n < 1 || m < 0 || K < 1 || K > 8) return -1;
    int nM = n * M;
    memset(Sigma, 0, sizeof(double) * (size_t)nM * nM);

    /* ---- off-diagonal blocks: windowed single-level sum */
    if (n > 1) {
        legrec *rec = (legrec *)malloc(sizeof(legrec) * (size_t)nM);
        double *v = (double *)malloc(sizeof(double) * (size_t)nM);
        for (int k = 0; k < n; ++k)
            for (int q = 0; q < M; ++q) legrec_init(&rec[k * M + q], m + q, z[k]);
        for (long l = m; l <= Loff; ++l) {
            double w = window((l + 0.5) / (double)Loff);
            if (w == 0.0) break;
            double c = oracle_Cl((int)l, M, khat, A) * w;
            for (int k = 0; k < n; ++k)
                for (int q = 0; q < M; ++q) {
                    legrec *r = &rec[k * M + q];
                    while (r->l < l) legrec_step(r);
                    v[k * M + q] = (r->l == l) ? s_factor((int)l, m, q) * legrec_value(r) : 0.0;
                }
            for (int i = 0; i < nM; ++i) {
                double ci = c * v[i];
                if (ci == 0.0) continue;
                int ki = i / M;
                double *row = Sigma + (size_t)i * nM;
                for (int j = 0; j < i; ++j)
                    if (j / M != ki) row[j] += ci * v[j];
            }
        }
        for (int i = 0; i < nM; ++i)
            for (int j = 0; j < i; ++j)
                if (j / M != i / M) Sigma[(size_t)j * nM + i] = Sigma[(size_t)i * nM + j];
        free(rec); free(v);
    }

    /* ---- same-point blocks: windowed sums at K levels + Richardson */
    double *lev = (double *)malloc(sizeof(double) * (size_t)K * M * M);
    legrec *rr = (legrec *)malloc(sizeof(legrec) * (size_t)M);
    double *vv = (double *)malloc(sizeof(double) * (size_t)M);
    for (int k = 0; k < n; ++k) {
        for (int lv = 0; lv < K; ++lv) {
            long L = Ld[k] << lv;
            double *S = lev + (size_t)lv * M * M;
            memset(S, 0, sizeof(double) * M * M);
            for (int q = 0; q < M; ++q) legrec_init(&rr[q], m + q, z[k]);
            for (long l = m; l <= L; ++l) {
                double w = window((l + 0.5) / (double)L);
                if (w == 0.0) break;
                double c = oracle_Cl((int)l, M, khat, A) * w;
                for (int q = 0; q < M; ++q) {
                    while (rr[q].l < l) legrec_step(&rr[q]);
                    vv[q] = (rr[q].l == l) ? s_factor((int)l, m, q) * legrec_value(&rr[q]) : 0.0;
                }
                for (int p = 0; p < M; ++p)
                    for (int q = 0; q <= p; ++q) S[p * M + q] += c * vv[p] * vv[q];
            }
        }
        /* Richardson in 1/L: R_i <- (2^j R_{i+1} - R_i) / (2^j - 1) */
        for (int j = 1; j < K; ++j) {
            double f = (double)(1L << j);
            for (int i = 0; i + j < K; ++i) {
                double *a = lev + (size_t)i * M * M, *b = lev + (size_t)(i + 1) * M * M;
                for (int e = 0; e < M * M; ++e) a[e] = (f * b[e] - a[e]) / (f - 1.0);
            }
        }
        for (int p = 0; p < M; ++p)
            for (int q = 0; q <= p; ++q) {
                double val = lev[p * M + q];
                Sigma[(size_t)(k * M + p) * nM + (k * M + q)] = val;
                Sigma[(size_t)(k * M + q) * nM + (k * M + p)] = val;
            }
    }
    free(lev); free(rr); free(vv);
    return 0;
}

/* Plain (no window, no extrapolation) partial sum up to lmax of the same cross
 * covariance between two points; used by tests to show the tail behaviour. */
double oracle_cov_partial(int m, int M, const double *khat, double A, double z1, double z2,
                          int p, int q, long lmax)
{
    legrec r1, r2;
    legrec_init(&r1, m + p, z1);
    legrec_init(&r2, m + q, z2);
    double s = 0.0;
    for (long l = m; l <= lmax; ++l) {
        while (r1.l < l) legrec_step(&r1);
        while (r2.l < l) legrec_step(&r2);
        double a = (r1.l == l) ? s_factor((int)l, m, p) * legrec_value(&r1) : 0.0;
        double b = (r2.l == l) ? s_factor((int)l, m, q) * legrec_value(&r2) : 0.0;
        s += oracle_Cl((int)l, M, khat, A) * a * b;
    }
    return s;
}

/* Normalised L_{l,mu}(z) for l = mu..lmax (tests compare with library routines). */
void oracle_legendre_row(int mu, double z, int lmax, double *out)
{
    legrec r;
    legrec_init(&r, mu, z);
    for (int l = mu; l <= lmax; ++l) {
        while (r.l < l) legrec_step(&r);
        out[l - mu] = legrec_value(&r);
    }
}

/* Naive real DFT of one ring (Alg. 2 last step, prefactor 1, C2R convention):
 * T_j = X_0 + 2 sum_{m=1}^{N/2-1} Re(X_m e^{2 pi i m j / N}) + X_{N/2} (-1)^j,
 * X given as re[0..N/2], im[0..N/2] (im[0], im[N/2] ignored). */
void oracle_dft_ring(int N, const double *re, const double *im, double *out)
{
    int H = N / 2;
    for (int j = 0; j < N; ++j) {
        double s = re[0] + ((j & 1) ? -re[H] : re[H]);
        for (int m = 1; m < H; ++m) {
            long mj = ((long)m * j) % N;
            double ang = 2.0 * M_PI * (double)mj / (double)N;
            s += 2.0 * (re[m] * cos(ang) - im[m] * sin(ang));
        }
        out[j] = s;
    }
}

/* The same cross covariance for several modes at once (independent problems, run in
 * parallel over modes).  ms[i] is the mode of problem i; Loff[i] and Ld[i*n..] its
 * cut-offs; Sigma receives nmodes blocks of (n*M)^2 doubles.  Returns 0 or -1. */
int oracle_cov_modes(int nmodes, const int *ms, int M, const double *khat, double A, int n,
                     const double *z, const long *Loff, const long *Ld, int K, double *Sigma)
{
    int bad = 0;
    size_t blk = (size_t)n * M * n * M;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : bad)
    for (int i = 0; i < nmodes; ++i)
        bad |= oracle_cov_m(ms[i], M, khat, A, n, z, Loff[i], Ld + (size_t)i * n, K,
                            Sigma + blk * (size_t)i) != 0;
    return bad ? -1 : 0;
}

/* ------------------------------------------- plain FFT for the ring synthesis
 * The same real synthesis as oracle_dft_ring, through a textbook iterative radix-2
 * complex FFT (bit reversal, then log2 N butterfly stages with e^{+2 pi i k / len}):
 * the Hermitian spectrum Y_0 = Re X_0, Y_m = X_m, Y_{N-m} = conj X_m (0 < m < N/2),
 * Y_{N/2} = Re X_{N/2} is transformed and the real part kept.  N a power of two. */
static int ilog2_exact(int N)
{
    int L = 0;
    while ((1 << L) < N) ++L;
    return (1 << L) == N ? L : -1;
}

int oracle_fft_ring(int N, const double *re, const double *im, double *out)
{
    const int L = ilog2_exact(N);
    if (L < 1) return -1;
    const int H = N / 2;
    double *yr = (double *)malloc(sizeof(double) * (size_t)N);
    double *yi = (double *)malloc(sizeof(double) * (size_t)N);
    if (!yr || !yi) { free(yr); free(yi); return -1; }
    for (int k = 0; k < N; ++k) {
        double a, b;
        if (k == 0) { a = re[0]; b = 0.0; }
        else if (k < H) { a = re[k]; b = im[k]; }
        else if (k == H) { a = re[H]; b = 0.0; }
        else { a = re[N - k]; b = -im[N - k]; }
        /* bit-reversed position of k */
        int r = 0;
        for (int t = 0; t < L; ++t) r |= ((k >> t) & 1) << (L - 1 - t);
        yr[r] = a;
        yi[r] = b;
    }
    for (int len = 2; len <= N; len <<= 1) {
        const int half = len / 2;
        for (int j = 0; j < half; ++j) {
            const double ang = 2.0 * M_PI * (double)j / (double)len;
            const double wr = cos(ang), wi = sin(ang);
            for (int s = 0; s < N; s += len) {
                const int a = s + j, b = s + j + half;
                const double tr = wr * yr[b] - wi * yi[b];
                const double ti = wr * yi[b] + wi * yr[b];
                yr[b] = yr[a] - tr;
                yi[b] = yi[a] - ti;
                yr[a] += tr;
                yi[a] += ti;
            }
        }
    }
    memcpy(out, yr, sizeof(double) * (size_t)N);
    free(yr);
    free(yi);
    return 0;
}

/* ------------------------------------------- Alg. 2: the per-sample recursion
 * Given tables for every mode m = 0..N/2 and every position i of a conditioning order
 * (the start ring first), draw each realisation's states position by position,
 *     x_{m,i} = sum_{j < npar[i]} T_{m,i,j} x_{m,par[i][j]} + B_{m,i} xi_{m,i}
 * (Eq. (state_space); with no parent it is the start state B_eq xi of Eq. (state_initial)),
 * for the Re and Im chains of each mode, then synthesise each position's ring
 * (Alg. 2, last step; prefactor 1).  The tables come from the oracle's Gaussian conditioning
 * of its spectral-sum covariance: T the transition of Eq. (trans_matrix) onto each parent,
 * B the lower factor of the conditional covariance of Eq. (innov_matrix).
 *
 *   M, N               state size p and ring length n_phi (power of two)
 *   n_pos, ring[n_pos] positions of the order and their ring indices (noise counters)
 *   npar[n_pos], par[n_pos][2]  parents (earlier positions, at most two)
 *   T[m][i][j][M][M]   transition onto parent j (row-major M x M), j < 2
 *   B[m][i][M][M]      lower factor (row-major; upper part ignored)
 *   seed, n_samples    realisation r uses the Philox key seed + r (noise layout of the
 *                      sampler: slot s in [1, N/2) takes normals [2Ms, 2Ms+2M), Re then Im;
 *                      slot 0 the real m = 0 chain [0, M) and the Nyquist Re chain [M, 2M))
 *   nthreads           OpenMP threads over modes (and over rings for the synthesis)
 *   use_fft            1: oracle_fft_ring, 0: the naive oracle_dft_ring
 *   out[r][i][N]       the field on each position's ring
 * Modes m >= 1 carry the complex normal's 1/sqrt(2) (Re and Im parts each N(0, 1/2)).
 * Returns 0, or -1 on bad arguments or allocation failure. */
int oracle_recursion_sample(int M, int N, int n_pos, const int *ring, const int *npar, const int *par,
                            const double *T, const double *B, uint64_t seed, int n_samples, int nthreads,
                            int use_fft, double *out)
{
    if (M < 1 || M > 4 || N < 4 || n_pos < 1 || n_samples < 0 || nthreads < 1) return -1;
    if (use_fft && ilog2_exact(N) < 1) return -1;
    const int H = N / 2, nm = H + 1;
    const size_t tstride = (size_t)2 * M * M, bstride = (size_t)M * M;
    /* states [position][mode][part][M] and complex coefficients [position][mode] */
    double *x = (double *)malloc(sizeof(double) * (size_t)n_pos * nm * 2 * M);
    double *cre = (double *)malloc(sizeof(double) * (size_t)n_pos * nm);
    double *cim = (double *)malloc(sizeof(double) * (size_t)n_pos * nm);
    double *nrm = (double *)malloc(sizeof(double) * (size_t)M * N);
    if (!x || !cre || !cim || !nrm) { free(x); free(cre); free(cim); free(nrm); return -1; }
    const double half = sqrt(0.5);
    int bad = 0;
    for (int r = 0; r < n_samples && !bad; ++r) {
        const uint64_t key64 = seed + (uint64_t)r;
        const uint32_t key[2] = {(uint32_t)key64, (uint32_t)(key64 >> 32)};
        for (int i = 0; i < n_pos; ++i) {
            const int ncalls = (M * N + 3) / 4;
#pragma omp parallel for num_threads(nthreads) schedule(static)
            for (int c = 0; c < ncalls; ++c) {
                uint32_t ctr[4] = {(uint32_t)c, (uint32_t)ring[i], 0u, 0u}, w[4];
                double v[4];
                oracle_philox4x32_10(ctr, key, w);
                box_muller(w[0], w[1], &v[0], &v[1]);
                box_muller(w[2], w[3], &v[2], &v[3]);
                for (int e = 0; e < 4 && 4 * c + e < M * N; ++e) nrm[4 * c + e] = v[e];
            }
#pragma omp parallel for num_threads(nthreads) schedule(static)
            for (int m = 0; m < nm; ++m) {
                const double *Tm = T + ((size_t)m * n_pos + i) * tstride;
                const double *Bm = B + ((size_t)m * n_pos + i) * bstride;
                const int nparts = (m == 0 || m == H) ? 1 : 2;
                double g[2] = {0.0, 0.0};
                for (int part = 0; part < nparts; ++part) {
                    /* the normals driving this chain */
                    const double *xi = m == 0 ? nrm : (m == H ? nrm + M : nrm + 2 * M * m + M * part);
                    double *xs = x + (((size_t)i * nm + m) * 2 + part) * M;
                    for (int p = 0; p < M; ++p) {
                        double acc = 0.0;
                        for (int j = 0; j < npar[i]; ++j) {
                            const double *xp = x + (((size_t)par[2 * i + j] * nm + m) * 2 + part) * M;
                            for (int q = 0; q < M; ++q) acc += Tm[j * bstride + p * M + q] * xp[q];
                        }
                        for (int q = 0; q <= p; ++q) acc += Bm[p * M + q] * xi[q];
                        xs[p] = acc;
                    }
                    g[part] = xs[0];
                }
                const double s = m == 0 ? 1.0 : half;
                cre[(size_t)i * nm + m] = s * g[0];
                cim[(size_t)i * nm + m] = s * g[1];
            }
        }
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 1) reduction(| : bad)
        for (int i = 0; i < n_pos; ++i) {
            double *dst = out + ((size_t)r * n_pos + i) * N;
            if (use_fft)
                bad |= oracle_fft_ring(N, cre + (size_t)i * nm, cim + (size_t)i * nm, dst) != 0;
            else
                oracle_dft_ring(N, cre + (size_t)i * nm, cim + (size_t)i * nm, dst);
        }
    }
    free(x);
    free(cre);
    free(cim);
    free(nrm);
    return bad ? -1 : 0;
}
