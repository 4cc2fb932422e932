// smerf_setup.cu -- FP64 set-up of the conditional-covariance tables on the GPU
// (Alg. 1 of Creasey & Lang, arXiv 1709.10314, with the efficient covariance of Sec. 3).
//
// Everything lives in the "northern frame": a chain runs from its start angle toward the
// north pole (theta decreasing).  The southern chain is the mirror image z -> -z of the
// northern problem (Sec. 4 obtains the southern rings from the mirror symmetry); its tables act
// on the mirrored state S x, S = diag((-1)^q).
//
// Notation (Sec. 3).  kappa-hat_i = kappa_i^2 = -l_i (l_i + 1).  For integer order mu,
//   P^mu_l(z)  = (Q_mu / mu!) t^mu F_mu(x),   P^mu_l(-z) = (Q_mu / mu!) t^-mu F_mu(1-x),
//   t = tan(theta/2), x = sin^2(theta/2) = (1-z)/2,
//   Q_mu = prod_{j<mu} (j(j+1) + kappa^2) = (-l)_mu (1+l)_mu,
//   F_mu(x) = 2F1(-l, l+1; 1+mu; x)          (Eq. (Legendre_hypergeometric)),
// whose series has positive terms with ratio (n(n+1) + kappa^2) x / ((n+1+mu)(n+1)).
//
// U-basis state x_q = U^q_m g_m (Eq. (Jmatrix_more_efficient)), q < p.  The solution
// matrix regular at the north pole is U(z)_{q,i} = P^{m+q}_{l_i}(z).  Gaussian
// conditioning (Eqs. (trans_matrix), (innov_matrix)) with the product form of the
// cross covariance (Eq. (Jmatrix_efficient)) gives, for a northward step z1 -> z2:
//   A = U(z2) U(z1)^{-1}                                               (transition)
//   Q = Cov(x(z2) | x(z1)) = (A_amp / 2 pi) int_{z1}^{z2} phi phi^T ds / (1 - s^2),
//       phi(s) = U(z2) U(s)^{-1} e_{p-1}.
// The second form follows from the state-space model of the process: its covariance
// operator is (2 pi D_m)^{-1} (Lemma 2.1 and the orthonormality of sqrt(2 pi) L_lm in
// dz), D_m has leading coefficient (-1)^p (1-z^2)^p, so only the last U-component is
// driven, with intensity A_amp / (2 pi (1 - s^2)).  It needs only the regular solution,
// i.e. 2F1 at x <= 1/2, and has no cancellation when z1 and z2 are close.
// The start covariance J(z0, z0) uses Eq. (Jmatrix_efficient) directly (both solutions
// at |z0| ~ 0, where both series converge fast).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <vector>

#include <cuda/std/complex>

#include "smerf_internal.cuh"
#include "smerf_setup.h"

using namespace smerf;

namespace {

struct Spec {
    int M;
    double k2[kMaxP];     // kappa_i^2
    double b[kMaxP];      // partial-fraction weights (Eq. (C_ell_efficient))
    double lG0[kMaxP];    // log Gamma(1+l_i) Gamma(-l_i)
    double A;
    double kmax;
    int n_theta, k0, n_modes, n_modes_pad;
    const double* theta;  // device: ring colatitudes (null: equiangular, pi (k + 1/2) / n_theta)
};

// colatitude of ring k (the plan's table, or the equiangular grid)
__device__ __host__ inline double ring_colat(const double* theta, int n_theta, int k)
{
    return theta ? theta[k] : SMERF_PI * ((double)k + 0.5) / (double)n_theta;
}

// 2F1(-l, l+1; 1+mu; x) for kappa^2 = k2 (a positive series) as S * 1e250^E.  Terms are
// taken two at a time with one division: r0 = a0/d0 and r1 = a1/d1 from 1/(d0 d1).
__device__ void hyp_scaled(double k2, int mu, double x, double& S, int& E)
{
    double s = 1.0, t = 1.0;
    int e = 0;
    const double m1 = (double)mu + 1.0;
    for (int n = 0; n < 1000000; n += 2) {
        const double dn = (double)n;
        const double a0 = (dn * (dn + 1.0) + k2) * x, d0 = (dn + m1) * (dn + 1.0);
        const double a1 = ((dn + 1.0) * (dn + 2.0) + k2) * x, d1 = (dn + 1.0 + m1) * (dn + 2.0);
        const double inv = 1.0 / (d0 * d1);
        const double r0 = a0 * d1 * inv, r1 = a1 * d0 * inv;
        t *= r0;
        s += t;
        if (t < 1e-17 * s && r0 < 0.9) break;
        t *= r1;
        s += t;
        if (t < 1e-17 * s && r1 < 0.9) break;
        if (s > 1e250) { s *= 1e-250; t *= 1e-250; ++e; }
    }
    S = s;
    E = e;
}

// log of the same series
__device__ double log_hyp(double k2, int mu, double x)
{
    double s;
    int e;
    hyp_scaled(k2, mu, x, s, e);
    return log(s) + e * 575.64627324851142;
}

// the series relative to a reference value sref * 1e250^eref (given as 1/sref and eref)
__device__ inline double hyp_rel(double k2, int mu, double x, double sref_inv, int eref)
{
    double s;
    int e;
    hyp_scaled(k2, mu, x, s, e);
    double v = s * sref_inv;
    for (int d = e - eref; d > 0; --d) v *= 1e250;
    for (int d = e - eref; d < 0; ++d) v *= 1e-250;
    return v;
}

// ring angle of position pos in chain c, in the northern frame
__device__ __host__ inline double chain_theta(const Spec& sp, int c, int pos)
{
    const int k = (c == 0) ? sp.k0 - pos : sp.n_theta - 1 - sp.k0 - pos;
    return ring_colat(sp.theta, sp.n_theta, k);
}

// ---------------------------------------------------------------- small matrices
template <int M> struct Mat { double a[M][M]; };

template <int M> __device__ inline Mat<M> mzero() { Mat<M> r; for (int i = 0; i < M; ++i) for (int j = 0; j < M; ++j) r.a[i][j] = 0.0; return r; }
template <int M> __device__ inline Mat<M> meye() { Mat<M> r = mzero<M>(); for (int i = 0; i < M; ++i) r.a[i][i] = 1.0; return r; }
template <int M> __device__ inline Mat<M> mmul(const Mat<M>& x, const Mat<M>& y)
{
    Mat<M> r;
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            double s = 0.0;
            for (int k = 0; k < M; ++k) s += x.a[i][k] * y.a[k][j];
            r.a[i][j] = s;
        }
    return r;
}
template <int M> __device__ inline Mat<M> mT(const Mat<M>& x) { Mat<M> r; for (int i = 0; i < M; ++i) for (int j = 0; j < M; ++j) r.a[i][j] = x.a[j][i]; return r; }
template <int M> __device__ inline Mat<M> madd(const Mat<M>& x, const Mat<M>& y) { Mat<M> r; for (int i = 0; i < M; ++i) for (int j = 0; j < M; ++j) r.a[i][j] = x.a[i][j] + y.a[i][j]; return r; }
template <int M> __device__ inline Mat<M> msym(const Mat<M>& x) { Mat<M> r; for (int i = 0; i < M; ++i) for (int j = 0; j < M; ++j) r.a[i][j] = 0.5 * (x.a[i][j] + x.a[j][i]); return r; }

// inverse of a 3 x 3 matrix by its adjugate (cofactors, the transposed minors) over the
// determinant; T is a real or complex matrix type, S its scalar
template <class T, class S> __device__ inline T inv3(const T& x)
{
    const auto& a = x.a;
    T r;
    r.a[0][0] = a[1][1] * a[2][2] - a[1][2] * a[2][1];
    r.a[0][1] = a[0][2] * a[2][1] - a[0][1] * a[2][2];
    r.a[0][2] = a[0][1] * a[1][2] - a[0][2] * a[1][1];
    r.a[1][0] = a[1][2] * a[2][0] - a[1][0] * a[2][2];
    r.a[1][1] = a[0][0] * a[2][2] - a[0][2] * a[2][0];
    r.a[1][2] = a[0][2] * a[1][0] - a[0][0] * a[1][2];
    r.a[2][0] = a[1][0] * a[2][1] - a[1][1] * a[2][0];
    r.a[2][1] = a[0][1] * a[2][0] - a[0][0] * a[2][1];
    r.a[2][2] = a[0][0] * a[1][1] - a[0][1] * a[1][0];
    const S d = a[0][0] * r.a[0][0] + a[0][1] * r.a[1][0] + a[0][2] * r.a[2][0];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) r.a[i][j] = r.a[i][j] / d;
    return r;
}

// inverse of a general M x M matrix (M <= 3)
template <int M> __device__ inline Mat<M> minv(const Mat<M>& x);
template <> __device__ inline Mat<1> minv<1>(const Mat<1>& x) { Mat<1> r; r.a[0][0] = 1.0 / x.a[0][0]; return r; }
template <> __device__ inline Mat<2> minv<2>(const Mat<2>& x)
{
    const double d = x.a[0][0] * x.a[1][1] - x.a[0][1] * x.a[1][0];
    Mat<2> r;
    r.a[0][0] = x.a[1][1] / d; r.a[0][1] = -x.a[0][1] / d;
    r.a[1][0] = -x.a[1][0] / d; r.a[1][1] = x.a[0][0] / d;
    return r;
}
template <> __device__ inline Mat<3> minv<3>(const Mat<3>& x) { return inv3<Mat<3>, double>(x); }

// lower Cholesky factor of a symmetric positive semi-definite matrix (0 where it degenerates)
template <int M> __device__ inline Mat<M> mchol(const Mat<M>& x)
{
    Mat<M> L = mzero<M>();
    for (int j = 0; j < M; ++j) {
        double d = x.a[j][j];
        for (int k = 0; k < j; ++k) d -= L.a[j][k] * L.a[j][k];
        const double ljj = d > 0.0 ? sqrt(d) : 0.0;
        L.a[j][j] = ljj;
        for (int i = j + 1; i < M; ++i) {
            double s = x.a[i][j];
            for (int k = 0; k < j; ++k) s -= L.a[i][k] * L.a[j][k];
            L.a[i][j] = ljj > 0.0 ? s / ljj : 0.0;
        }
    }
    return L;
}

// inverse of a symmetric positive definite matrix through its Cholesky factor
template <int M> __device__ inline Mat<M> mspd_inv(const Mat<M>& x)
{
    if (M == 1) { Mat<M> r; r.a[0][0] = 1.0 / x.a[0][0]; return r; }
    Mat<M> L = mchol<M>(x);
    Mat<M> Li = mzero<M>();  // L^{-1}, lower
    for (int i = 0; i < M; ++i) {
        Li.a[i][i] = 1.0 / L.a[i][i];
        for (int j = 0; j < i; ++j) {
            double s = 0.0;
            for (int k = j; k < i; ++k) s += L.a[i][k] * Li.a[k][j];
            Li.a[i][j] = -s / L.a[i][i];
        }
    }
    return mmul<M>(mT<M>(Li), Li);
}

// H_{q,i}(x) = r_{q,i} F^i_{m+q}(x) / F^i_m(x_ref); r_{q,i} = prod_{j=m}^{m+q-1} (j(j+1)+kappa_i^2)/(j+1)
// (the reference series value F^i_m(x_ref) = sref * 1e250^eref, given as 1/sref and eref)
template <int M> __device__ inline Mat<M> hmat(const Spec& sp, int m, double x, const double* sinv, const int* eref)
{
    Mat<M> H;
    for (int i = 0; i < M; ++i) {
        double r = 1.0;
        for (int q = 0; q < M; ++q) {
            if (q > 0) {
                const double j = (double)(m + q - 1);
                r *= (j * (j + 1.0) + sp.k2[i]) / (j + 1.0);
            }
            H.a[q][i] = r * hyp_rel(sp.k2[i], m + q, x, sinv[i], eref[i]);
        }
    }
    return H;
}

__constant__ double kGL8x[8] = {-0.9602898564975363, -0.7966664774136267, -0.5255324099163290, -0.1834346424956498,
                                 0.1834346424956498,  0.5255324099163290,  0.7966664774136267,  0.9602898564975363};
__constant__ double kGL8w[8] = {0.1012285362903763, 0.2223810344533745, 0.3137066458778873, 0.3626837833783620,
                                0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};

// Transition Phi and conditional covariance Q of every northward step, one thread per
// (chain, position, mode).  phi/q: [c][pos][m][M*M] doubles (pos 1..len).
template <int M>
__global__ void step_kernel(Spec sp, int c, int len, double* phi, double* qout)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int pos = blockIdx.y + 1;
    if (m >= sp.n_modes || pos > len) return;
    const double th1 = chain_theta(sp, c, pos - 1), th2 = chain_theta(sp, c, pos);
    const double t1 = tan(0.5 * th1), t2 = tan(0.5 * th2);
    const double u1 = log(t1), u2 = log(t2);
    const double s1 = sin(0.5 * th1), s2 = sin(0.5 * th2);
    const double x1 = s1 * s1, x2 = s2 * s2;
    double sinv[M];
    int eref[M];
    for (int i = 0; i < M; ++i) {
        double sr;
        hyp_scaled(sp.k2[i], m, x2, sr, eref[i]);
        sinv[i] = 1.0 / sr;
    }
    const Mat<M> H2 = hmat<M>(sp, m, x2, sinv, eref);
    const Mat<M> H1 = hmat<M>(sp, m, x1, sinv, eref);
    // A = (t2/t1)^m diag(t2^q) H2 H1^{-1} diag(t1^-q)
    Mat<M> A = mmul<M>(H2, minv<M>(H1));
    const double g = exp((double)m * (u2 - u1));
    for (int p = 0; p < M; ++p)
        for (int q = 0; q < M; ++q) A.a[p][q] *= g * pow(t2, (double)p) / pow(t1, (double)q);
    // W = diag(t2^(q-M+1)) H2
    Mat<M> W = H2;
    for (int p = 0; p < M; ++p)
        for (int q = 0; q < M; ++q) W.a[p][q] *= pow(t2, (double)(p - M + 1));
    // Q = A_amp/(2 pi) int_0^{du} e^{-c v} (W h)(W h)^T dv, h = H(x(u2+v))^{-1} e_{M-1}
    const double cexp = 2.0 * (double)(m + M - 1);
    const double du = u1 - u2;
    const double vmax = cexp > 0.0 ? fmin(du, 46.0 / cexp) : du;
    const double sinmax = th1 > 0.5 * SMERF_PI ? 1.0 : sin(th1);
    const double rho = cexp + 2.0 * sp.kmax * sinmax + 1.0;
    int nsub = (int)ceil(0.25 * rho * vmax);  // one 8-point panel per 4 / rho (twice finer agrees to rounding)
    nsub = nsub < 1 ? 1 : (nsub > 256 ? 256 : nsub);
    const double h = vmax / nsub;
    Mat<M> acc = mzero<M>();
    for (int j = 0; j < nsub; ++j)
        for (int n = 0; n < 8; ++n) {
            const double v = (j + 0.5 * (kGL8x[n] + 1.0)) * h;
            const double w = 0.5 * h * kGL8w[n] * exp(-cexp * v);
            const double u = u2 + v;
            const double x = 1.0 / (1.0 + exp(-2.0 * u));   // sin^2(theta/2), tan(theta/2) = e^u
            const Mat<M> Hs = hmat<M>(sp, m, x, sinv, eref);
            const Mat<M> Hi = minv<M>(Hs);
            double ph[M];
            for (int p = 0; p < M; ++p) {
                double s = 0.0;
                for (int k = 0; k < M; ++k) s += W.a[p][k] * Hi.a[k][M - 1];
                ph[p] = s;
            }
            for (int p = 0; p < M; ++p)
                for (int q = 0; q < M; ++q) acc.a[p][q] += w * ph[p] * ph[q];
        }
    const double f = sp.A / (2.0 * SMERF_PI);
    const size_t o = (((size_t)pos) * sp.n_modes + m) * (M * M);
    for (int p = 0; p < M; ++p)
        for (int q = 0; q < M; ++q) {
            phi[o + p * M + q] = A.a[p][q];
            qout[o + p * M + q] = f * acc.a[p][q];
        }
}

// ---- p = 1 with a real spectrum: the step tables by a recurrence in m (Alg. 1 sets up the
// hypergeometric functions of every order m).  For fixed x the series of
// Eq. (Legendre_hypergeometric), F_m(x) = 2F1(-lambda, lambda+1; 1+m; x) with
// (-lambda)(lambda+1) = kappa^2, satisfy Gauss's contiguous relation in the third parameter,
//   F_{m-1} = [(1-2x) F_m + (1 + kappa^2/(m(m+1))) x F_{m+1}] / (1-x),   m >= 1.
// For large m its solutions behave like 1 (F_m itself) and like (-(1-x)/x)^m, so for x < 1/2
// F_m is the minimal solution and the relation taken downward from two series values is
// stable (relative error of order m eps; ratios of F at nearby x, which is what the tables
// use, to a few 1e-13 over 16384 orders).  For x > 1/2 the error grows by x/(1-x) per order:
// only the first step's equatorward ring can have x > 1/2 (south of the equator, even n_theta);
// that step keeps step_kernel's per-mode series unless the growth over all orders,
// (x/(1-x))^m_max, stays below 1e3 (it is about e^pi = 23 when n_phi = 2 n_theta).  Per step the
// construction is step_kernel's for M = 1: A = (t2/t1)^m F_m(x2)/F_m(x1) and
// Q = (A_amp/2 pi) int_0^du e^{-2 m v} (F_m(x2)/F_m(x(v)))^2 dv, on one node set for all m:
// composite 8-point Gauss-Legendre panels no wider than 4/rho(m) for every m whose weight
// e^{-2 m v} at the panel's start is above e^-46 (the same panel rule as step_kernel).
constexpr int kRecWarps = 4;         // warps per block, one step each
constexpr int kRecMaxPanels = 8192;  // node-set cap (reached only by grids far beyond 16384 rings)

// the series F_mu(x) as S * 2^(250 E)
__device__ void hyp_scaled2(double k2, int mu, double x, double& S, int& E)
{
    double s = 1.0, t = 1.0;
    int e = 0;
    const double m1 = (double)mu + 1.0;
    for (int n = 0; n < 1000000; n += 2) {
        const double dn = (double)n;
        const double a0 = (dn * (dn + 1.0) + k2) * x, d0 = (dn + m1) * (dn + 1.0);
        const double a1 = ((dn + 1.0) * (dn + 2.0) + k2) * x, d1 = (dn + 1.0 + m1) * (dn + 2.0);
        const double inv = 1.0 / (d0 * d1);
        const double r0 = a0 * d1 * inv, r1 = a1 * d0 * inv;
        t *= r0;
        s += t;
        if (t < 1e-17 * s && r0 < 0.9) break;
        t *= r1;
        s += t;
        if (t < 1e-17 * s && r1 < 0.9) break;
        if (s > 0x1p250) { s *= 0x1p-250; t *= 0x1p-250; ++e; }
    }
    S = s;
    E = e;
}

// width of the panel that starts at v: 4/rho(m*), m* the largest order whose weight e^{-2 m v}
// is above e^-46 at v, rho(m) = 2m + kap
__device__ inline double rec_panel_width(double v, int mtop, double kap)
{
    const double ms = v > 0.0 ? fmin((double)mtop, floor(23.0 / v)) : (double)mtop;
    return 4.0 / (2.0 * ms + kap);
}

// One warp per step of the northern chain (pos = first..len).  Lane 0 holds x2 (the step's
// poleward ring), lane 1 x1, lanes 2..31 up to 30 quadrature nodes (further nodes in further
// passes, which start at the highest order whose weight at their nodes is above e^-46).  The
// lanes run the recurrence downward in m together; per block of 32 orders they leave
// w_j e^{-2 m v_j} / F_m(x_j)^2 in shared memory, and lane l then sums order m_l's row in a
// fixed order, so that Q_m = (A_amp/2 pi) F_m(x2)^2 sum_j ... (the common scale of the F's
// cancels).
__global__ void __launch_bounds__(32 * kRecWarps) step_kernel_rec(Spec sp, int first, int len, double* phi, double* qout)
{
    __shared__ double tile[kRecWarps][32][33];  // [order in block][lane]
    __shared__ double fr2[kRecWarps][32], fr1[kRecWarps][32], alph[kRecWarps][32];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int pos = blockIdx.x * kRecWarps + wib + first;
    if (pos > len) return;  // whole warps
    const unsigned full = 0xffffffffu;
    const double th1 = chain_theta(sp, 0, pos - 1), th2 = chain_theta(sp, 0, pos);
    const double u1 = log(tan(0.5 * th1)), u2 = log(tan(0.5 * th2));
    const double du = u1 - u2;
    const double sa = sin(0.5 * th1), sb = sin(0.5 * th2);
    const double x1r = sa * sa, x2r = sb * sb;
    const double sinmax = th1 > 0.5 * SMERF_PI ? 1.0 : sin(th1);
    const double kap = 2.0 * sp.kmax * sinmax + 1.0;
    const double k2 = sp.k2[0];
    const double f = sp.A / (2.0 * SMERF_PI);
    const int mtop = sp.n_modes - 1;
    int np = 0;
    for (double v = 0.0; v < du && np < kRecMaxPanels; ++np) v += rec_panel_width(v, mtop, kap);
    const int K = 8 * np;
    const int passes = (K + 29) / 30;
    const size_t base = (size_t)pos * sp.n_modes;
    for (int ch = 0; ch < passes; ++ch) {
        // this lane's point: x, quadrature weight, v
        double x = x2r, wt = 0.0, v = 0.0;
        if (lane == 1) {
            x = x1r;
            v = du;
        } else if (lane >= 2 && 30 * ch + lane - 2 < K) {
            const int i = 30 * ch + lane - 2, j = i >> 3, n = i & 7;
            double b = 0.0;
            for (int q = 0; q < j; ++q) b += rec_panel_width(b, mtop, kap);
            const double h = (j == np - 1 || b + rec_panel_width(b, mtop, kap) > du) ? du - b
                                                                                       : rec_panel_width(b, mtop, kap);
            v = b + 0.5 * (kGL8x[n] + 1.0) * h;
            wt = 0.5 * h * kGL8w[n];
            x = 1.0 / (1.0 + exp(-2.0 * (u2 + v)));
        }
        // highest order of the pass: every order for the first (it also gives A), else the
        // last whose weight at the pass's first node is above e^-46
        int mstart = mtop;
        if (ch > 0) {
            const double vmin = __shfl_sync(full, v, 2);
            mstart = vmin > 0.0 ? (int)fmin((double)mtop, floor(23.0 / vmin)) : mtop;
        }
        double S0, S1;
        int E0, E1;
        hyp_scaled2(k2, mstart, x, S0, E0);
        hyp_scaled2(k2, mstart + 1, x, S1, E1);
        int W = E0;  // common scale of the lanes' values
        for (int o = 16; o > 0; o >>= 1) W = max(W, __shfl_xor_sync(full, W, o));
        double F = ldexp(S0, 250 * (E0 - W)), Fp = ldexp(S1, 250 * (E1 - W));
        const double beta = (1.0 - 2.0 * x) / (1.0 - x), gam = x / (1.0 - x);
        const double e2v = exp(2.0 * v);
        for (int mb = mstart; mb >= 0; mb -= 32) {
            {
                const int ml = mb - lane;
                alph[wib][lane] = ml >= 1 ? k2 / ((double)ml * (double)(ml + 1)) : 0.0;
            }
            __syncwarp();
            double Ew = exp(-2.0 * (double)mb * v);  // e^{-2 m v}, exact at the block's first order
            for (int k = 0; k < 32; ++k) {
                const int m = mb - k;
                if (m < 0) break;
                const double r = 1.0 / F;
                tile[wib][k][lane] = wt * Ew * r * r;
                if (lane == 0) fr2[wib][k] = F;
                if (lane == 1) fr1[wib][k] = F;
                if (m >= 1) {
                    const double t = gam + gam * alph[wib][k];
                    const double Fn = beta * F + t * Fp;
                    Fp = F;
                    F = Fn;
                    // a common rescale keeps the values, their squares and the squares of their
                    // reciprocals in range (ratios are unchanged)
                    if (__any_sync(full, (__double2hiint(F) & 0x7ff00000) > ((1023 + 250) << 20))) {
                        F *= 0x1p-250;
                        Fp *= 0x1p-250;
                    }
                }
                Ew *= e2v;
            }
            __syncwarp();
            const int m = mb - lane;
            if (m >= 0) {
                double sum = 0.0;
                for (int j = 2; j < 32; ++j) sum += tile[wib][lane][j];
                const double F2 = fr2[wib][lane];
                const double q = f * F2 * F2 * sum;
                if (ch == 0) {
                    qout[base + m] = q;
                    phi[base + m] = exp(-(double)m * du) * F2 / fr1[wib][lane];
                } else {
                    qout[base + m] += q;
                }
            }
            __syncwarp();
        }
    }
}

// p = 2 with a real spectrum: the same recurrence for both kappa_i.  Per order m a lane's
// point x has H(x) = [[F^1_m, F^2_m], [r_1 F^1_{m+1}, r_2 F^2_{m+1}]], r_i = (m(m+1)+kappa_i^2)/(m+1)
// (step_kernel's H up to a scale per column, which cancels in A = H2 H1^-1 and in
// phi = W H^-1 e_1), each column with its own common rescale.  A node's
// phi = diag(t2^-1, 1) H2 H(x)^-1 e_1 is formed from H2's entries (broadcast from lane 0) and
// the node's own before squaring (no cancellation); its three products go through shared
// memory as in step_kernel_rec.  One warp per block (three transposition tiles).
__global__ void __launch_bounds__(32) step_kernel_rec2(Spec sp, int first, int len, double* phi, double* qout)
{
    constexpr int M = 2;
    __shared__ double tile[3][32][33];  // [product][order in block][lane]
    __shared__ double h2[4][32], h1[4][32], alph[2][32], rr[2][32];
    const int lane = threadIdx.x & 31;
    const int pos = blockIdx.x + first;
    if (pos > len) return;
    const unsigned full = 0xffffffffu;
    const double th1 = chain_theta(sp, 0, pos - 1), th2 = chain_theta(sp, 0, pos);
    const double t1 = tan(0.5 * th1), t2 = tan(0.5 * th2);
    const double u1 = log(t1), u2 = log(t2);
    const double du = u1 - u2;
    const double sa = sin(0.5 * th1), sb = sin(0.5 * th2);
    const double x1r = sa * sa, x2r = sb * sb;
    const double sinmax = th1 > 0.5 * SMERF_PI ? 1.0 : sin(th1);
    const double kap = 2.0 * sp.kmax * sinmax + 1.0;
    const double f = sp.A / (2.0 * SMERF_PI);
    const int mtop = sp.n_modes - 1;
    // panel width at v: 4/rho(m*), rho(m) = 2(m + M - 1) + kap, m* the largest order whose
    // weight e^{-2(m+M-1)v} is above e^-46 at v
    auto width = [&](double v) {
        const double ms = v > 0.0 ? fmax(0.0, fmin((double)mtop, floor(23.0 / v) - (M - 1))) : (double)mtop;
        return 4.0 / (2.0 * (ms + M - 1) + kap);
    };
    int np = 0;
    for (double v = 0.0; v < du && np < kRecMaxPanels; ++np) v += width(v);
    const int K = 8 * np;
    const int passes = (K + 29) / 30;
    const size_t base = (size_t)pos * sp.n_modes;
    for (int ch = 0; ch < passes; ++ch) {
        double x = x2r, wt = 0.0, v = 0.0;
        if (lane == 1) {
            x = x1r;
            v = du;
        } else if (lane >= 2 && 30 * ch + lane - 2 < K) {
            const int i = 30 * ch + lane - 2, j = i >> 3, n = i & 7;
            double b = 0.0;
            for (int q = 0; q < j; ++q) b += width(b);
            const double h = (j == np - 1 || b + width(b) > du) ? du - b : width(b);
            v = b + 0.5 * (kGL8x[n] + 1.0) * h;
            wt = 0.5 * h * kGL8w[n];
            x = 1.0 / (1.0 + exp(-2.0 * (u2 + v)));
        }
        int mstart = mtop;
        if (ch > 0) {
            const double vmin = __shfl_sync(full, v, 2);
            mstart = vmin > 0.0 ? (int)fmax(0.0, fmin((double)mtop, floor(23.0 / vmin) - (M - 1))) : mtop;
        }
        double F[2], Fp[2];
        for (int c = 0; c < 2; ++c) {
            double S0, S1;
            int E0, E1;
            hyp_scaled2(sp.k2[c], mstart, x, S0, E0);
            hyp_scaled2(sp.k2[c], mstart + 1, x, S1, E1);
            int W = E0;
            for (int o = 16; o > 0; o >>= 1) W = max(W, __shfl_xor_sync(full, W, o));
            F[c] = ldexp(S0, 250 * (E0 - W));
            Fp[c] = ldexp(S1, 250 * (E1 - W));
        }
        const double beta = (1.0 - 2.0 * x) / (1.0 - x), gam = x / (1.0 - x);
        const double e2v = exp(2.0 * v);
        for (int mb = mstart; mb >= 0; mb -= 32) {
            {
                const int ml = mb - lane;
                for (int c = 0; c < 2; ++c) {
                    alph[c][lane] = ml >= 1 ? sp.k2[c] / ((double)ml * (double)(ml + 1)) : 0.0;
                    rr[c][lane] = ml >= 0 ? ((double)ml * (double)(ml + 1) + sp.k2[c]) / (double)(ml + 1) : 0.0;
                }
            }
            __syncwarp();
            double Ew = exp(-2.0 * (double)(mb + M - 1) * v);
            for (int k = 0; k < 32; ++k) {
                const int m = mb - k;
                if (m < 0) break;
                const double a = F[0], b = F[1], c = rr[0][k] * Fp[0], d = rr[1][k] * Fp[1];
                const double a2 = __shfl_sync(full, a, 0), b2 = __shfl_sync(full, b, 0);
                const double c2 = __shfl_sync(full, c, 0), d2 = __shfl_sync(full, d, 0);
                const double rdet = 1.0 / (a * d - b * c);
                const double p0 = (b2 * a - a2 * b) * rdet, p1 = (d2 * a - c2 * b) * rdet;
                const double we = wt * Ew;
                tile[0][k][lane] = we * p0 * p0;
                tile[1][k][lane] = we * p0 * p1;
                tile[2][k][lane] = we * p1 * p1;
                if (lane == 0) { h2[0][k] = a; h2[1][k] = b; h2[2][k] = c; h2[3][k] = d; }
                if (lane == 1) { h1[0][k] = a; h1[1][k] = b; h1[2][k] = c; h1[3][k] = d; }
                if (m >= 1) {
                    for (int cc = 0; cc < 2; ++cc) {
                        const double t = gam + gam * alph[cc][k];
                        const double Fn = beta * F[cc] + t * Fp[cc];
                        Fp[cc] = F[cc];
                        F[cc] = Fn;
                        if (__any_sync(full, (__double2hiint(F[cc]) & 0x7ff00000) > ((1023 + 250) << 20))) {
                            F[cc] *= 0x1p-250;
                            Fp[cc] *= 0x1p-250;
                        }
                    }
                }
                Ew *= e2v;
            }
            __syncwarp();
            const int m = mb - lane;
            if (m >= 0) {
                double s00 = 0.0, s01 = 0.0, s11 = 0.0;
                for (int j = 2; j < 32; ++j) {
                    s00 += tile[0][lane][j];
                    s01 += tile[1][lane][j];
                    s11 += tile[2][lane][j];
                }
                const size_t o = (base + m) * (M * M);
                const double q00 = f * s00 / (t2 * t2), q01 = f * s01 / t2, q11 = f * s11;
                if (ch == 0) {
                    qout[o + 0] = q00;
                    qout[o + 1] = q01;
                    qout[o + 2] = q01;
                    qout[o + 3] = q11;
                    // A = (t2/t1)^m diag(t2^p) H2 H1^-1 diag(t1^-q)
                    const double a2 = h2[0][lane], b2 = h2[1][lane], c2 = h2[2][lane], d2 = h2[3][lane];
                    const double a1 = h1[0][lane], b1 = h1[1][lane], c1 = h1[2][lane], d1 = h1[3][lane];
                    const double g = exp(-(double)m * du) / (a1 * d1 - b1 * c1);
                    phi[o + 0] = g * (a2 * d1 - b2 * c1);
                    phi[o + 1] = g * (b2 * a1 - a2 * b1) / t1;
                    phi[o + 2] = g * t2 * (c2 * d1 - d2 * c1);
                    phi[o + 3] = g * t2 * (d2 * a1 - c2 * b1) / t1;
                } else {
                    qout[o + 0] += q00;
                    qout[o + 1] += q01;
                    qout[o + 2] += q01;
                    qout[o + 3] += q11;
                }
            }
            __syncwarp();
        }
    }
}

// Table store.  FP64 tables keep every entry at magnitude >= 2^-120 (zeros and smaller
// values become +-2^-120, a change far below any effect on the field): FP32-recursion
// kernels then convert them to FP32 with three integer instructions and no range check.
template <class T>
__device__ inline void put(void* base, bool is64, size_t idx, double v)
{
    if (is64) {
        const double tiny = 0x1p-120;
        ((double*)base)[idx] = fabs(v) < tiny ? (v < 0.0 ? -tiny : tiny) : v;
    } else {
        ((float*)base)[idx] = (float)v;
    }
}

// The start ring's Pochhammer factors, log[(-l_i)_m (l_i+1)_m / (m!)^2]
// = sum_{j<m} log((j(j+1) + kappa_i^2) / (j+1)^2) (Eq. (Legendre_hypergeometric)), for every m at
// once: one block sums contiguous chunks of the terms, scans the chunk sums and writes each
// chunk's prefixes (a fixed order; start_kernel reads lq[i * n_modes + m]).
__global__ void __launch_bounds__(1024) lq_prefix_kernel(Spec sp, double* lq)
{
    __shared__ double part[1024];
    const int n = sp.n_modes, t = threadIdx.x, nt = blockDim.x;
    const int chunk = (n + nt - 1) / nt;
    const int j0 = min(n, t * chunk), j1 = min(n, j0 + chunk);
    for (int i = 0; i < sp.M; ++i) {
        const double k2 = sp.k2[i];
        double s = 0.0;
        for (int j = j0; j < j1; ++j) s += log((j * (j + 1.0) + k2) / ((j + 1.0) * (j + 1.0)));
        part[t] = s;
        __syncthreads();
        for (int o = 1; o < nt; o <<= 1) {  // inclusive scan of the chunk sums
            const double v = t >= o ? part[t - o] : 0.0;
            __syncthreads();
            part[t] += v;
            __syncthreads();
        }
        double acc = t > 0 ? part[t - 1] : 0.0;  // the terms j < j0
        for (int j = j0; j < j1; ++j) {
            lq[(size_t)i * n + j] = acc;
            acc += log((j * (j + 1.0) + k2) / ((j + 1.0) * (j + 1.0)));
        }
        __syncthreads();
    }
}

// Start factor B_eq = chol J(z0, z0) (Eq. (state_initial)), one thread per mode.
template <int M>
__global__ void start_kernel(Spec sp, const double* lqa, void* beq, bool tab64)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= sp.n_modes) return;
    const double th0 = ring_colat(sp.theta, sp.n_theta, sp.k0);
    const double t0 = tan(0.5 * th0);
    const double sx = sin(0.5 * th0), cx = cos(0.5 * th0);
    const double x0 = sx * sx, xb0 = cx * cx;
    Mat<M> J = mzero<M>();
    for (int i = 0; i < M; ++i) {
        const double k2 = sp.k2[i];
        const double lq = lqa[(size_t)i * sp.n_modes + m];  // log Q_m / (m!)^2
        double lF0[M], lF1[M], r[M];
        double rr = 1.0;
        for (int q = 0; q < M; ++q) {
            if (q > 0) {
                const double j = (double)(m + q - 1);
                rr *= (j * (j + 1.0) + k2) / (j + 1.0);
            }
            r[q] = rr;
            lF0[q] = log_hyp(k2, m + q, x0);
            lF1[q] = log_hyp(k2, m + q, xb0);
        }
        const double sb = sp.b[i] > 0.0 ? 1.0 : -1.0;
        const double lb = log(fabs(sp.b[i])) + sp.lG0[i] - log(4.0 * SMERF_PI) + lq;
        for (int p = 0; p < M; ++p)
            for (int q = 0; q < M; ++q) {
                const double v = exp(lb + lF1[p] + lF0[q]) * r[p] * r[q] * pow(t0, (double)(q - p));
                J.a[p][q] += sb * ((p & 1) ? -v : v);
            }
    }
    const Mat<M> L = mchol<M>(msym<M>(J));
    const double sc = m > 0 ? 0.70710678118654752440 : 1.0;
    int e = 0;
    for (int p = 0; p < M; ++p)
        for (int q = 0; q <= p; ++q, ++e)
            put<double>(beq, tab64, (size_t)e * sp.n_modes_pad + m, L.a[p][q] * sc);
}

// Bridge, forward and coarse tables of one segment, one thread per (segment, mode).
// Segment [pa, pb] with right anchor pb: for pa < pos < pb, condition x_pos on x_{pos-1}
// (prior N(Phi x, Q)) and on x_pb = Psi x_pos + N(0, S) (Psi, S accumulated backward):
//   P = (Q^{-1} + Psi^T S^{-1} Psi)^{-1},  Abar = P Q^{-1} Phi,  C = P Psi^T S^{-1},  B = chol P.
// The coarse step pa -> pb is (Psi_pa, chol S_pa).  Without a right anchor the tables are
// the plain forward step (Phi, 0, chol Q).
template <int M>
__global__ void segment_tables_kernel(Spec sp, int c, int len, int H, const double* phi,
                                      const double* qv, void* steps, void* coarse, bool tab64)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int seg = blockIdx.y;
    if (m >= sp.n_modes) return;
    const int Ec = coarse_elems(M);
    const size_t mp = sp.n_modes_pad;
    const double sc = m > 0 ? 0.70710678118654752440 : 1.0;
    // the southern chain runs in the mirrored state S x and is driven by S xi; its B
    // factors are stored with S folded into their columns so that the kernels use xi as is
    auto colsign = [&](int q) { return (c == 1 && (q & 1)) ? -1.0 : 1.0; };
    const int pa = H > 0 ? seg * H : 0;
    const int pb = (H > 0 && pa + H <= len) ? pa + H : -1;
    auto load = [&](const double* base, int pos) {
        Mat<M> r;
        const size_t o = (((size_t)pos) * sp.n_modes + m) * (M * M);
        for (int p = 0; p < M; ++p)
            for (int q = 0; q < M; ++q) r.a[p][q] = base[o + p * M + q];
        return r;
    };
    auto store_step = [&](int pos, const Mat<M>& A, const Mat<M>& C, const Mat<M>& B) {
        const size_t base = ((size_t)pos * mp + m) * step_row(M);
        int e = 0;
        for (int p = 0; p < M; ++p)
            for (int q = 0; q < M; ++q, ++e) put<double>(steps, tab64, base + e, A.a[p][q]);
        for (int p = 0; p < M; ++p)
            for (int q = 0; q < M; ++q, ++e) put<double>(steps, tab64, base + e, C.a[p][q]);
        for (int p = 0; p < M; ++p)
            for (int q = 0; q <= p; ++q, ++e) put<double>(steps, tab64, base + e, B.a[p][q] * sc * colsign(q));
        for (; e < step_row(M); ++e) put<double>(steps, tab64, base + e, 0.0);
    };
    if (pb < 0) {
        const int end = len;
        for (int pos = pa + 1; pos <= end; ++pos) {
            const Mat<M> Ph = load(phi, pos), Q = load(qv, pos);
            store_step(pos, Ph, mzero<M>(), mchol<M>(msym<M>(Q)));
        }
        return;
    }
    Mat<M> Psi = meye<M>(), S = mzero<M>();
    for (int pos = pb; pos > pa; --pos) {
        const Mat<M> Ph = load(phi, pos), Q = msym<M>(load(qv, pos));
        if (pos < pb) {
            const Mat<M> Qi = mspd_inv<M>(Q);
            const Mat<M> Si = mspd_inv<M>(msym<M>(S));
            const Mat<M> PsT = mT<M>(Psi);
            const Mat<M> P = msym<M>(mspd_inv<M>(msym<M>(madd<M>(Qi, mmul<M>(mmul<M>(PsT, Si), Psi)))));
            const Mat<M> Ab = mmul<M>(mmul<M>(P, Qi), Ph);
            const Mat<M> C = mmul<M>(mmul<M>(P, PsT), Si);
            store_step(pos, Ab, C, mchol<M>(P));
        }
        // move to pos-1: S_{pos-1} = Psi Q Psi^T + S, Psi_{pos-1} = Psi Phi
        S = madd<M>(mmul<M>(mmul<M>(Psi, Q), mT<M>(Psi)), S);
        Psi = mmul<M>(Psi, Ph);
    }
    const Mat<M> Bc = mchol<M>(msym<M>(S));
    const int j = pb / H;
    const size_t base = (size_t)j * Ec * mp + m;
    int e = 0;
    for (int p = 0; p < M; ++p)
        for (int q = 0; q < M; ++q, ++e) put<double>(coarse, tab64, base + (size_t)e * mp, Psi.a[p][q]);
    for (int p = 0; p < M; ++p)
        for (int q = 0; q <= p; ++q, ++e) put<double>(coarse, tab64, base + (size_t)e * mp, Bc.a[p][q] * sc * colsign(q));
}

// FFT tables, in FP64 on the host then rounded to the recursion precision:
//   pre[s] = e^{2 pi i s / n_phi}, s < Nc (C2R packing), and for every radix-RP pass with
//   Ns > 1 (pass plan: radix 4 while Nc/Ns >= 4, then 2) the block
//   tw[off + (i-1) Ns + kk] = e^{2 pi i i kk / (Ns RP)}, i = 1..RP-1, kk < Ns.
template <class R>
static int upload_fft_tables(int n_phi, void** tw, void** pre, void** tw2, void** tw3)
{
    const int Nc = n_phi / 2;
    std::vector<R> p(2 * (size_t)Nc), t;
    for (int s = 0; s < Nc; ++s) {
        p[2 * s] = (R)cos(2.0 * SMERF_PI * s / n_phi);
        p[2 * s + 1] = (R)sin(2.0 * SMERF_PI * s / n_phi);
    }
    int Ns = 1;
    while (Ns < Nc) {
        const int RP = (Nc / Ns >= 4) ? 4 : 2;
        if (Ns > 1)
            for (int i = 1; i < RP; ++i)
                for (int kk = 0; kk < Ns; ++kk) {
                    const double a = 2.0 * SMERF_PI * (double)i * kk / ((double)Ns * RP);
                    t.push_back((R)cos(a));
                    t.push_back((R)sin(a));
                }
        Ns *= RP;
    }
    if (t.empty()) t.assign(2, (R)0);
    // high-radix plans (passes of at most 16 and at most 8 points)
    int L = 0;
    while ((1 << L) < Nc) ++L;
    for (int t = 0; t < 2; ++t) {
        const int MB = t == 0 ? 4 : SMERF_INPLACE_MB;
        std::vector<R> t2;
        for (int ps = 1; ps < smerf::hr_passes(L, MB); ++ps) {
            const int RP = 1 << smerf::hr_bits(L, ps, MB), Ns2 = 1 << smerf::hr_lgns(L, ps, MB);
            for (int i = 1; i < RP; ++i)
                for (int kk = 0; kk < Ns2; ++kk) {
                    const double a = 2.0 * SMERF_PI * (double)i * kk / ((double)Ns2 * RP);
                    t2.push_back((R)cos(a));
                    t2.push_back((R)sin(a));
                }
        }
        if (t2.empty()) t2.assign(2, (R)0);
        void** dst = t == 0 ? tw2 : tw3;
        if (smerf::dev_malloc(dst, t2.size() * sizeof(R)) != cudaSuccess) return SMERF_ENOMEM;
        if (cudaMemcpy(*dst, t2.data(), t2.size() * sizeof(R), cudaMemcpyHostToDevice) != cudaSuccess) return SMERF_ECUDA;
    }
    if (smerf::dev_malloc(tw, t.size() * sizeof(R)) != cudaSuccess) return SMERF_ENOMEM;
    if (smerf::dev_malloc(pre, p.size() * sizeof(R)) != cudaSuccess) return SMERF_ENOMEM;
    if (cudaMemcpy(*tw, t.data(), t.size() * sizeof(R), cudaMemcpyHostToDevice) != cudaSuccess) return SMERF_ECUDA;
    if (cudaMemcpy(*pre, p.data(), p.size() * sizeof(R), cudaMemcpyHostToDevice) != cudaSuccess) return SMERF_ECUDA;
    return SMERF_OK;
}

// ---------------------------------------------------------------- complex kappa-hat
// Spectra with complex kappa-hat (Eq. (Cl) with complex-conjugate pairs, as in the paper's
// Sec. 5 example (10 + l^2 (l+1)^2)^-1, kappa-hat = +-i sqrt(10)).  The same construction in
// complex arithmetic: l_i, 2F1, U, the partial-fraction weights b_i and the Gamma factors are
// complex; A, Q and J(z0, z0) are real (the two columns of U of a conjugate pair are complex
// conjugates) and their real parts are kept.
using cdbl = cuda::std::complex<double>;

struct SpecC {
    cdbl k2[kMaxP], b[kMaxP], lG0[kMaxP];  // kappa-hat_i, b_i, log(Gamma(1+l_i) Gamma(-l_i))
    double A, kmax;
    int n_theta, k0, n_modes, n_modes_pad;
    const double* theta;  // device: ring colatitudes (null: equiangular)
};

template <int M> struct MatC { cdbl a[M][M]; };

template <int M> __device__ inline MatC<M> cmmul(const MatC<M>& x, const MatC<M>& y)
{
    MatC<M> r;
    for (int i = 0; i < M; ++i)
        for (int j = 0; j < M; ++j) {
            cdbl s = 0.0;
            for (int k = 0; k < M; ++k) s += x.a[i][k] * y.a[k][j];
            r.a[i][j] = s;
        }
    return r;
}
template <int M> __device__ inline MatC<M> cminv(const MatC<M>& x);
template <> __device__ inline MatC<1> cminv<1>(const MatC<1>& x) { MatC<1> r; r.a[0][0] = 1.0 / x.a[0][0]; return r; }
template <> __device__ inline MatC<2> cminv<2>(const MatC<2>& x)
{
    const cdbl d = x.a[0][0] * x.a[1][1] - x.a[0][1] * x.a[1][0];
    MatC<2> r;
    r.a[0][0] = x.a[1][1] / d; r.a[0][1] = -x.a[0][1] / d;
    r.a[1][0] = -x.a[1][0] / d; r.a[1][1] = x.a[0][0] / d;
    return r;
}
template <> __device__ inline MatC<3> cminv<3>(const MatC<3>& x) { return inv3<MatC<3>, cdbl>(x); }

// 2F1(-l, l+1; 1+mu; x) with kappa-hat = k2 complex, as S * 1e250^E (terms two per division)
__device__ void hyp_scaled_c(cdbl k2, int mu, double x, cdbl& S, int& E)
{
    cdbl s = 1.0, t = 1.0;
    int e = 0;
    const double m1 = (double)mu + 1.0;
    for (int n = 0; n < 1000000; n += 2) {
        const double dn = (double)n;
        const cdbl a0 = (dn * (dn + 1.0) + k2) * x, a1 = ((dn + 1.0) * (dn + 2.0) + k2) * x;
        const double d0 = (dn + m1) * (dn + 1.0), d1 = (dn + 1.0 + m1) * (dn + 2.0);
        const double inv = 1.0 / (d0 * d1);
        const cdbl r0 = a0 * (d1 * inv), r1 = a1 * (d0 * inv);
        t *= r0;
        s += t;
        if (cuda::std::abs(t) < 1e-17 * cuda::std::abs(s) && cuda::std::abs(r0) < 0.9) break;
        t *= r1;
        s += t;
        if (cuda::std::abs(t) < 1e-17 * cuda::std::abs(s) && cuda::std::abs(r1) < 0.9) break;
        if (cuda::std::abs(s) > 1e250) { s *= 1e-250; t *= 1e-250; ++e; }
    }
    S = s;
    E = e;
}

__device__ inline cdbl log_hyp_c(cdbl k2, int mu, double x)
{
    cdbl s;
    int e;
    hyp_scaled_c(k2, mu, x, s, e);
    return cuda::std::log(s) + e * 575.64627324851142;
}

__device__ inline cdbl hyp_rel_c(cdbl k2, int mu, double x, cdbl sref_inv, int eref)
{
    cdbl s;
    int e;
    hyp_scaled_c(k2, mu, x, s, e);
    cdbl v = s * sref_inv;
    for (int d = e - eref; d > 0; --d) v *= 1e250;
    for (int d = e - eref; d < 0; ++d) v *= 1e-250;
    return v;
}

template <int M> __device__ inline MatC<M> hmat_c(const SpecC& sp, int m, double x, const cdbl* sinv, const int* eref)
{
    MatC<M> H;
    for (int i = 0; i < M; ++i) {
        cdbl r = 1.0;
        for (int q = 0; q < M; ++q) {
            if (q > 0) {
                const double j = (double)(m + q - 1);
                r *= (j * (j + 1.0) + sp.k2[i]) / (j + 1.0);
            }
            H.a[q][i] = r * hyp_rel_c(sp.k2[i], m + q, x, sinv[i], eref[i]);
        }
    }
    return H;
}

// step_kernel in complex arithmetic (same construction, real parts stored)
template <int M>
__global__ void step_kernel_c(SpecC sp, int len, double* phi, double* qout)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const int pos = blockIdx.y + 1;
    if (m >= sp.n_modes || pos > len) return;
    const double th1 = ring_colat(sp.theta, sp.n_theta, sp.k0 - pos + 1);
    const double th2 = ring_colat(sp.theta, sp.n_theta, sp.k0 - pos);
    const double t1 = tan(0.5 * th1), t2 = tan(0.5 * th2);
    const double u1 = log(t1), u2 = log(t2);
    const double s1 = sin(0.5 * th1), s2 = sin(0.5 * th2);
    const double x1 = s1 * s1, x2 = s2 * s2;
    cdbl sinv[M];
    int eref[M];
    for (int i = 0; i < M; ++i) {
        cdbl sr;
        hyp_scaled_c(sp.k2[i], m, x2, sr, eref[i]);
        sinv[i] = 1.0 / sr;
    }
    const MatC<M> H2 = hmat_c<M>(sp, m, x2, sinv, eref);
    const MatC<M> H1 = hmat_c<M>(sp, m, x1, sinv, eref);
    MatC<M> A = cmmul<M>(H2, cminv<M>(H1));
    const double g = exp((double)m * (u2 - u1));
    for (int p = 0; p < M; ++p)
        for (int q = 0; q < M; ++q) A.a[p][q] *= g * pow(t2, (double)p) / pow(t1, (double)q);
    MatC<M> W = H2;
    for (int p = 0; p < M; ++p)
        for (int q = 0; q < M; ++q) W.a[p][q] *= pow(t2, (double)(p - M + 1));
    const double cexp = 2.0 * (double)(m + M - 1);
    const double du = u1 - u2;
    const double vmax = cexp > 0.0 ? fmin(du, 46.0 / cexp) : du;
    const double sinmax = th1 > 0.5 * SMERF_PI ? 1.0 : sin(th1);
    const double rho = cexp + 2.0 * sp.kmax * sinmax + 1.0;
    int nsub = (int)ceil(0.25 * rho * vmax);
    nsub = nsub < 1 ? 1 : (nsub > 256 ? 256 : nsub);
    const double h = vmax / nsub;
    double acc[M][M];
    for (int p = 0; p < M; ++p)
        for (int q = 0; q < M; ++q) acc[p][q] = 0.0;
    for (int j = 0; j < nsub; ++j)
        for (int n = 0; n < 8; ++n) {
            const double v = (j + 0.5 * (kGL8x[n] + 1.0)) * h;
            const double w = 0.5 * h * kGL8w[n] * exp(-cexp * v);
            const double u = u2 + v;
            const double x = 1.0 / (1.0 + exp(-2.0 * u));
            const MatC<M> Hi = cminv<M>(hmat_c<M>(sp, m, x, sinv, eref));
            double ph[M];
            for (int p = 0; p < M; ++p) {
                cdbl s = 0.0;
                for (int k = 0; k < M; ++k) s += W.a[p][k] * Hi.a[k][M - 1];
                ph[p] = s.real();  // phi is real (conjugate columns)
            }
            for (int p = 0; p < M; ++p)
                for (int q = 0; q < M; ++q) acc[p][q] += w * ph[p] * ph[q];
        }
    const double f = sp.A / (2.0 * SMERF_PI);
    const size_t o = (((size_t)pos) * sp.n_modes + m) * (M * M);
    for (int p = 0; p < M; ++p)
        for (int q = 0; q < M; ++q) {
            phi[o + p * M + q] = A.a[p][q].real();
            qout[o + p * M + q] = f * acc[p][q];
        }
}

// start_kernel in complex arithmetic
template <int M>
__global__ void start_kernel_c(SpecC sp, void* beq, bool tab64)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= sp.n_modes) return;
    const double th0 = ring_colat(sp.theta, sp.n_theta, sp.k0);
    const double t0 = tan(0.5 * th0);
    const double sx = sin(0.5 * th0), cx = cos(0.5 * th0);
    const double x0 = sx * sx, xb0 = cx * cx;
    Mat<M> J = mzero<M>();
    for (int i = 0; i < M; ++i) {
        const cdbl k2 = sp.k2[i];
        cdbl lq = 0.0;  // log Q_m / (m!)^2
        for (int j = 0; j < m; ++j) lq += cuda::std::log((j * (j + 1.0) + k2) / ((j + 1.0) * (j + 1.0)));
        cdbl lF0[M], lF1[M], r[M];
        cdbl rr = 1.0;
        for (int q = 0; q < M; ++q) {
            if (q > 0) {
                const double j = (double)(m + q - 1);
                rr *= (j * (j + 1.0) + k2) / (j + 1.0);
            }
            r[q] = rr;
            lF0[q] = log_hyp_c(k2, m + q, x0);
            lF1[q] = log_hyp_c(k2, m + q, xb0);
        }
        const cdbl lb = cuda::std::log(sp.b[i]) + sp.lG0[i] - log(4.0 * SMERF_PI) + lq;
        for (int p = 0; p < M; ++p)
            for (int q = 0; q < M; ++q) {
                const cdbl v = cuda::std::exp(lb + lF1[p] + lF0[q]) * r[p] * r[q] * pow(t0, (double)(q - p));
                J.a[p][q] += ((p & 1) ? -v : v).real();
            }
    }
    const Mat<M> L = mchol<M>(msym<M>(J));
    const double sc = m > 0 ? 0.70710678118654752440 : 1.0;
    int e = 0;
    for (int p = 0; p < M; ++p)
        for (int q = 0; q <= p; ++q, ++e)
            put<double>(beq, tab64, (size_t)e * sp.n_modes_pad + m, L.a[p][q] * sc);
}

// host: the complex spectrum's constants
static SpecC make_spec_c(const smerf_plan* pl)
{
    SpecC sc = SpecC();  // value-initialised: every member zero
    const int M = pl->p;
    sc.A = pl->A;
    sc.kmax = 0.0;
    for (int i = 0; i < M; ++i) {
        const cdbl kh(pl->khat_re[i], pl->khat_im[i]);
        sc.k2[i] = kh;
        sc.kmax = fmax(sc.kmax, sqrt(cuda::std::abs(kh)));
        cdbl b = pl->A;
        for (int j = 0; j < M; ++j)
            if (j != i) b /= cdbl(pl->khat_re[j], pl->khat_im[j]) - kh;
        sc.b[i] = b;
        // l = -1/2 + sqrt(1/4 - kappa-hat); Gamma(1+l) Gamma(-l) = -pi / sin(pi l)
        const cdbl lam = -0.5 + cuda::std::sqrt(0.25 - kh);
        const cdbl I(0.0, 1.0), z = SMERF_PI * lam;
        const cdbl ls = z.imag() > 0.0 ? -I * z + cuda::std::log(I * 0.5) + cuda::std::log(1.0 - cuda::std::exp(2.0 * I * z))
                                       : I * z + cuda::std::log(-I * 0.5) + cuda::std::log(1.0 - cuda::std::exp(-2.0 * I * z));
        sc.lG0[i] = cuda::std::log(cdbl(-SMERF_PI, 0.0)) - ls;
    }
    sc.n_theta = pl->n_theta;
    sc.k0 = pl->k0;
    sc.n_modes = pl->n_modes;
    sc.n_modes_pad = pl->n_modes_pad;
    sc.theta = pl->theta_dev;
    return sc;
}

#define CK(x)                                                                     \
    do {                                                                          \
        cudaError_t e_ = (x);                                                     \
        if (e_ != cudaSuccess) {                                                  \
            fprintf(stderr, "smerf setup: %s at %s:%d\n", cudaGetErrorString(e_), \
                    __FILE__, __LINE__);                                          \
            rc = (e_ == cudaErrorMemoryAllocation) ? SMERF_ENOMEM : SMERF_ECUDA;  \
            goto done;                                                            \
        }                                                                         \
    } while (0)

// p = 1 FP32 step rows [position][mode][A, C, B, pad] -> [position][A, C, B][mode]
__global__ void repack_rows_kernel(const float* __restrict__ rows, float* __restrict__ packed, int mp)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    const size_t pos = blockIdx.y;
    if (m >= mp) return;
    const float4 r = reinterpret_cast<const float4*>(rows)[pos * mp + m];
    packed[(pos * 3 + 0) * mp + m] = r.x;
    packed[(pos * 3 + 1) * mp + m] = r.y;
    packed[(pos * 3 + 2) * mp + m] = r.z;
}

template <int M>
int setup_impl(smerf_plan* pl, cudaStream_t st, bool sync)
{
    int rc = SMERF_OK;
    Spec sp;
    memset(&sp, 0, sizeof(sp));
    sp.M = M;
    sp.A = pl->A;
    sp.kmax = 0.0;
    for (int i = 0; i < M && !pl->complex_spec; ++i) {
        const double k = pl->kappa[i];
        sp.k2[i] = k * k;
        sp.kmax = fmax(sp.kmax, k);
        double b = pl->A;
        for (int j = 0; j < M; ++j)
            if (j != i) b /= pl->kappa[j] * pl->kappa[j] - k * k;
        sp.b[i] = b;
        if (k * k > 0.25) {
            const double nu = sqrt(k * k - 0.25);
            sp.lG0[i] = log(SMERF_PI) - SMERF_PI * nu - log(0.5 * (1.0 + exp(-2.0 * SMERF_PI * nu)));
        } else {
            const double lam = -0.5 + sqrt(0.25 - k * k);
            sp.lG0[i] = log(-SMERF_PI / sin(SMERF_PI * lam));
        }
    }
    sp.n_theta = pl->n_theta;
    sp.k0 = pl->k0;
    sp.n_modes = pl->n_modes;
    sp.n_modes_pad = pl->n_modes_pad;
    sp.theta = pl->theta_dev;

    const bool t64 = pl->tab64;
    const size_t es = t64 ? 8 : 4;
    const size_t mp = pl->n_modes_pad;
    double* phi = nullptr;
    double* qv = nullptr;
    double* lqa = nullptr;
    const int threads = 128;
    const int gm = (pl->n_modes + threads - 1) / threads;
    auto t_start = std::chrono::steady_clock::now();

    pl->table_bytes = 0;
    pl->step_table_bytes = 0;
    CK(smerf::dev_malloc((void**)&pl->beq, (size_t)tri(M) * mp * es));
    CK(cudaMemsetAsync(pl->beq, 0, (size_t)tri(M) * mp * es, st));
    pl->table_bytes += (size_t)tri(M) * mp * es;
    for (int c = 0; c < 2; ++c) {
        const int len = pl->chain[c].len;
        const size_t sb = (size_t)(len + 1) * step_row(M) * mp * es;
        const size_t cb = (size_t)(pl->chain[c].n_anchors + 1) * coarse_elems(M) * mp * es;
        CK(smerf::dev_malloc((void**)&pl->steps[c], sb > 0 ? sb : 16));
        CK(cudaMemsetAsync(pl->steps[c], 0, sb > 0 ? sb : 16, st));
        CK(smerf::dev_malloc((void**)&pl->coarse[c], cb > 0 ? cb : 16));
        CK(cudaMemsetAsync(pl->coarse[c], 0, cb > 0 ? cb : 16, st));
        pl->table_bytes += sb + cb;
        pl->step_table_bytes += sb;
    }
    rc = pl->recur64 ? upload_fft_tables<double>(pl->n_phi, &pl->tw, &pl->pre, &pl->tw2, &pl->tw3)
                     : upload_fft_tables<float>(pl->n_phi, &pl->tw, &pl->pre, &pl->tw2, &pl->tw3);
    if (rc != SMERF_OK) goto done;
    if (pl->complex_spec) start_kernel_c<M><<<gm, threads, 0, st>>>(make_spec_c(pl), pl->beq, t64);
    else {
        CK(smerf::dev_malloc_async((void**)&lqa, (size_t)M * pl->n_modes * sizeof(double), st));
        lq_prefix_kernel<<<1, 1024, 0, st>>>(sp, lqa);
        start_kernel<M><<<gm, threads, 0, st>>>(sp, lqa, pl->beq, t64);
        CK(cudaFreeAsync(lqa, st));
        lqa = nullptr;
    }
    CK(cudaGetLastError());
    {
        // Step transitions and covariances of the northern chain.  On a grid symmetric about the
        // equator the southern chain's steps are their mirror images (z -> -z): in the northern
        // frame its step pos is the northern step pos + shift, shift = 1 for even n_theta (start
        // ring south of the equator) and 0 for odd n_theta, so one computation serves both
        // chains.  On any other grid a second pass computes them as the northern chain of the
        // mirrored grid theta'_j = pi - theta_{n_theta-1-j} (stored after the grid's own
        // colatitudes) from its start ring n_theta - 1 - k0, whose ring k0' - pos is the southern
        // chain's ring k0 + pos.
        const int len0 = pl->chain[0].len, len1 = pl->chain[1].len;
        const bool sym = smerf_grid_symmetric(pl->theta_host, pl->n_theta);
        const int shift = (pl->n_theta % 2 == 0) ? 1 : 0;
        if (sym && len1 + shift > len0) { rc = SMERF_EUNSUPPORTED; goto done; }
        for (int pass = 0; pass < (sym ? 1 : 2); ++pass) {
            const int len = pass == 0 ? len0 : len1;
            Spec s = sp;
            SpecC sc = pl->complex_spec ? make_spec_c(pl) : SpecC();
            // colatitude of the pass's start ring in its own frame
            double th = ring_colat(pl->theta_host, pl->n_theta, pl->k0);
            if (pass == 1) {
                s.theta = sc.theta = pl->theta_dev + pl->n_theta;
                s.k0 = sc.k0 = pl->n_theta - 1 - pl->k0;
                th = SMERF_PI - th;
            }
            if (len > 0) {
                const size_t nb = (size_t)(len + 1) * pl->n_modes * M * M * sizeof(double);
                CK(smerf::dev_malloc_async((void**)&phi, nb, st));
                CK(smerf::dev_malloc_async((void**)&qv, nb, st));
                if (len > 65535) { rc = SMERF_EUNSUPPORTED; goto done; }
                dim3 grid(gm, len);
                if (pl->complex_spec) step_kernel_c<M><<<grid, threads, 0, st>>>(sc, len, phi, qv);
                else if (M == 3) step_kernel<M><<<grid, threads, 0, st>>>(s, 0, len, phi, qv);  // per-mode series
                else {
                    // the recurrence in m, but for a first step whose equatorward ring (x > 1/2)
                    // would amplify rounding errors by more than 1e3 over the orders: that one by
                    // the per-mode series (the start ring is the ring nearest the equator, so no
                    // later step starts south of it)
                    const double x1 = sin(0.5 * th) * sin(0.5 * th);
                    const bool first_series = x1 > 0.5 && (double)(pl->n_modes - 1) * log(x1 / (1.0 - x1)) > log(1e3);
                    const int first = first_series ? 2 : 1;
                    if (first_series) step_kernel<M><<<dim3(gm, 1), threads, 0, st>>>(s, 0, 1, phi, qv);
                    if (len >= first) {
                        const int n = len - first + 1;
                        if (M == 1) step_kernel_rec<<<(n + kRecWarps - 1) / kRecWarps, 32 * kRecWarps, 0, st>>>(s, first, len, phi, qv);
                        else step_kernel_rec2<<<n, 32, 0, st>>>(s, first, len, phi, qv);
                    }
                }
                CK(cudaGetLastError());
            }
            // the chains whose tables this pass's steps give: both (symmetric grid), or one
            for (int c = sym ? 0 : pass; c < (sym ? 2 : pass + 1); ++c) {
                const int lc = pl->chain[c].len;
                if (lc == 0) continue;
                const size_t off = (sym && c == 1) ? (size_t)shift * pl->n_modes * M * M : 0;
                const int H = pl->H;
                const int nseg = H > 0 ? (lc / H + 1) : 1;
                dim3 grid(gm, nseg);
                segment_tables_kernel<M><<<grid, threads, 0, st>>>(sp, c, lc, H, phi + off, qv + off, pl->steps[c],
                                                             pl->coarse[c], t64);
                CK(cudaGetLastError());
            }
            if (phi) CK(cudaFreeAsync(phi, st));
            if (qv) CK(cudaFreeAsync(qv, st));
            phi = qv = nullptr;
        }
    }
    if (M == 1 && pl->packed) {
        // the ring kernel's packed p = 1 layout: [position][A, C, B][mode]
        for (int c = 0; c < 2; ++c) {
            const int len = pl->chain[c].len;
            const size_t rb = (size_t)(len + 1) * step_row(M) * mp * es;
            const size_t pb = (size_t)(len + 1) * 3 * mp * es;
            void* packed = nullptr;
            CK(smerf::dev_malloc(&packed, pb > 0 ? pb : 16));
            repack_rows_kernel<<<dim3((unsigned)((mp + 255) / 256), (unsigned)(len + 1)), 256, 0, st>>>(
                (const float*)pl->steps[c], (float*)packed, (int)mp);
            CK(cudaGetLastError());
            CK(cudaStreamSynchronize(st));
            cudaFree(pl->steps[c]);
            pl->steps[c] = packed;
            pl->table_bytes = pl->table_bytes - rb + pb;
            pl->step_table_bytes = pl->step_table_bytes - rb + pb;
        }
    }
    if (sync) {
        CK(cudaStreamSynchronize(st));
        pl->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    }
done:
    if (phi || qv || lqa) {
        cudaStreamSynchronize(st);
        if (phi) cudaFree(phi);
        if (qv) cudaFree(qv);
        if (lqa) cudaFree(lqa);
    }
    return rc;
}

}  // namespace

bool smerf_grid_symmetric(const double* theta, int n_theta)
{
    if (!theta) return true;
    for (int k = 0; k < n_theta; ++k)
        if (fabs(theta[k] + theta[n_theta - 1 - k] - SMERF_PI) > 1e-12 * SMERF_PI) return false;
    return true;
}

int smerf_start_ring(const double* theta, int n_theta)
{
    if (smerf_grid_symmetric(theta, n_theta)) return n_theta / 2;
    int k0 = 0;
    for (int k = 1; k < n_theta; ++k)
        if (fabs(theta[k] - 0.5 * SMERF_PI) <= fabs(theta[k0] - 0.5 * SMERF_PI)) k0 = k;
    return k0;
}

int smerf_setup_tables(smerf_plan* pl, cudaStream_t st, bool sync)
{
    switch (pl->p) {
        case 1: return setup_impl<1>(pl, st, sync);
        case 2: return setup_impl<2>(pl, st, sync);
        case 3: return setup_impl<3>(pl, st, sync);
        default: return SMERF_EUNSUPPORTED;
    }
}
