"""The paper's Sec. 5 convergence study as a GPU validation workload: spectrum
C_l = (10 + l^2 (l+1)^2)^-1 (complex kappa-hat = +-i sqrt(10)), n_theta in {4, 8, 16, 32},
m_max = n_theta (n_phi = 2 n_theta), 320,000 realisations per grid.

* The sample covariance of the GPU field, equatorial (one ring near the equator, every
  azimuthal offset) and meridional (every pair of rings on a meridian), matches the exact
  covariance of the m-truncated discrete field (Lemma 2.1 summed over |m| <= m_max with the
  real-DFT weights) within 5 standard errors (from 40 batch means).
* The paper's error measure, max |sample covariance - C(g)| against the continuum covariance
  C(g) = sum_l (2l+1)/(4 pi) C_l P_l(cos g), on the equator and on the meridian, falls with
  m_max with a log-log slope between -2 and -1.2 on both (Sec. 5 reports m_max^(-3/2)).
  The truncation error alone (exact discrete covariance against C(g)) is printed beside it."""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

SEC5 = [complex(0.0, math.sqrt(10.0)), complex(0.0, -math.sqrt(10.0))]
N_SAMPLES, N_BATCH = 320000, 40


def continuum_cov(cosg, lmax=20000):
    """C(g) = sum_l (2l+1)/(4 pi) C_l P_l(cos g), Legendre recurrence in l."""
    cosg = np.asarray(cosg, dtype=np.float64)
    p0, p1 = np.ones_like(cosg), cosg.copy()
    tot = (1.0 / (4 * math.pi)) * (1.0 / 10.0) * p0
    for l in range(1, lmax + 1):
        L = l * (l + 1.0)
        tot = tot + (2 * l + 1) / (4 * math.pi) / (10.0 + L * L) * p1
        p0, p1 = p1, ((2 * l + 1) * cosg * p1 - l * p0) / (l + 1)
    return tot


def truncated_cov(th1, th2, dphi, n_phi, lmax=4000):
    """Covariance of the discrete field between (th1, phi) and (th2, phi + dphi):
    J^0 + 2 sum_{0<m<Hm} J^m cos(m dphi) + J^Hm cos(Hm dphi) / 2 (Lemma 2.1, real DFT)."""
    kh = oracle.KHat(SEC5)
    Hm = n_phi // 2
    z1, z2 = math.cos(th1), math.cos(th2)
    tot = 0.0
    for m in range(Hm + 1):
        w = 1.0 if m == 0 else (0.5 if m == Hm else 2.0)
        tot += w * math.cos(m * dphi) * oracle.cov_partial(m, kh, 1.0, z1, z2, 0, 0, lmax)
    return tot


def test_sec5_covariance_convergence():
    import torch
    from paper_1709_10314_gb300 import Plan
    rows = []
    for n_theta in (4, 8, 16, 32):
        n_phi = 2 * n_theta
        plan = Plan(A=1.0, n_theta=n_theta, n_phi=n_phi, anchor_spacing=0 if n_theta < 16 else 4, khat=SEC5)
        th = oracle.ring_theta(n_theta)
        ke = n_theta // 2                       # ring just south of the equator
        per = N_SAMPLES // N_BATCH
        eq = np.zeros((N_BATCH, n_phi // 2 + 1))
        mer = np.zeros((N_BATCH, n_theta, n_theta))
        for b in range(N_BATCH):
            x = plan.sample(1 + b * per, per).double()               # [per, n_theta, n_phi]
            ring = x[:, ke, :]
            for d in range(n_phi // 2 + 1):
                eq[b, d] = float((ring * torch.roll(ring, -d, dims=1)).mean())
            y = x.permute(0, 2, 1).reshape(-1, n_theta)
            mer[b] = (y.T @ y / y.shape[0]).cpu().numpy()
        torch.cuda.synchronize()
        eq_m, eq_se = eq.mean(0), eq.std(0, ddof=1) / math.sqrt(N_BATCH)
        mer_m, mer_se = mer.mean(0), mer.std(0, ddof=1) / math.sqrt(N_BATCH)
        dphis = 2 * math.pi * np.arange(n_phi // 2 + 1) / n_phi
        eq_tr = np.array([truncated_cov(th[ke], th[ke], d, n_phi) for d in dphis])
        mer_tr = np.array([[truncated_cov(th[a], th[b], 0.0, n_phi) for b in range(n_theta)] for a in range(n_theta)])
        z_eq = np.max(np.abs(eq_m - eq_tr) / eq_se)
        z_mer = np.max(np.abs(mer_m - mer_tr) / np.maximum(mer_se, 1e-300))
        assert z_eq < 5.0 and z_mer < 5.0, (n_theta, z_eq, z_mer)
        cos_eq = np.cos(th[ke]) ** 2 + np.sin(th[ke]) ** 2 * np.cos(dphis)
        e_eq = float(np.max(np.abs(eq_tr - continuum_cov(cos_eq))))
        cos_mer = np.cos(th[:, None] - th[None, :])
        e_mer = float(np.max(np.abs(mer_tr - continuum_cov(cos_mer))))
        rows.append((n_theta, e_eq, e_mer, z_eq, z_mer, float(np.max(np.abs(eq_m - continuum_cov(cos_eq)))),
                     float(np.max(np.abs(mer_m - continuum_cov(cos_mer))))))
    print("\nn_theta  trunc. err (eq)  trunc. err (mer)  max z (eq, mer)  sample err (eq)  sample err (mer)")
    for r in rows:
        print("%6d  %15.3e  %16.3e  %6.2f %6.2f  %15.3e  %16.3e" % r)
    ns = np.log([r[0] for r in rows])
    slope = lambda k: float(np.polyfit(ns, np.log([r[k] for r in rows]), 1)[0])
    print("log-log slopes vs m_max: truncation error eq %.2f, mer %.2f; sample error (Sec. 5's measure) eq %.2f, mer %.2f"
          % (slope(1), slope(2), slope(5), slope(6)))
    assert rows[-1][1] < rows[0][1] and rows[-1][2] < rows[0][2]
    # the paper's measure falls as m_max^(-3/2) (Sec. 5): both slopes near -1.5
    assert -2.0 <= slope(5) <= -1.2 and -2.0 <= slope(6) <= -1.2, (slope(5), slope(6))
