"""FP32 error bounds for Gibbs chain states, propagated along the FP64 path.

The GPU runs the Gibbs sweeps in FP32 while the oracle runs them in FP64 from
the same Philox bits, so the two chains see the same draws and differ only by
rounding.  Each sweep adds a per-draw error no larger than ``rtol`` times the
magnitude the FP32 arithmetic works at (the per-draw bar of the parity tests),
and carries the error already in the state through the sweep map.  To first
order in the errors (they are ~1e-6 relative, so second-order terms are
~1e-12), the carried error is the state error times the map's partial
derivative along the oracle's trajectory.  For the normal-gamma model
(tau | mu, then mu | tau, Sec. 1 Fig. 1's alternating-conditional loop):

    tau_t = G_t / r_t,     r_t = b0 + (S + n (xbar - mu_{t-1})^2) / 2
    mu_t  = m_t + z_t / sqrt(P_t),   P_t = prec0 + n tau_t,
    m_t   = (prec0 mu0 + tau_t n xbar) / P_t

    d tau_t / d mu_{t-1} = tau_t n (xbar - mu_{t-1}) / r_t
    d mu_t  / d tau_t    = n (xbar - m_t) / P_t - z_t n / (2 P_t^(3/2))

    E^tau_t = |d tau_t / d mu_{t-1}| E^mu_{t-1} + rtol |tau_t| (1 + kappa_t)
    E^mu_t  = |d mu_t / d tau_t| E^tau_t + rtol (|m_t| + |z_t| / sqrt(P_t))

with kappa_t the conditioning of the Gamma draw (3|cz|/t, plus |ln U_b / a|
when the shape is boosted), E^mu_0 the error of the start state (0 when both
sides start from the same FP32 value).  When the chain contracts
(|d mu_t/d mu_{t-1}| < 1, as it does strongly for informative data) the bound
settles at the per-draw error / (1 - contraction); nothing grows with the
number of sweeps.

The sweep moments are FP32 sums on the GPU: plain sums over groups of at most
8 consecutive sweeps, whose results go into compensated (Kahan) sums.  Their
error is the sum of the per-sweep state errors plus the summation's own error:
a plain sum of m terms errs by at most (m - 1) u sum |x_i| and a compensated
one by (2u + O(N u^2)) sum |x_i| for the unit roundoff u = 2^-24 (Higham,
Accuracy and Stability of Numerical Algorithms, 2nd ed., Secs. 4.2-4.3), so
(7 + 2 + 1) u covers both levels and the final FP64 fold.  (The LDA sums are
compensated per sweep, well inside the same bound.)  A square adds 2|x| E + E^2
plus the product's rounding u x^2.
"""
import numpy as np

U32 = 2.0 ** -24  # FP32 unit roundoff
SUM_ERR = 10.0 * U32  # groups of 8 plain (7u), compensated across groups (2u), FP64 fold


def ng_sweep_terms(nobs, xbar, sc, prior, mu_prev, G, z):
    """The sweep map's intermediate values and partial derivatives in FP64."""
    a0, b0, mu0, prec0 = (float(p) for p in prior)
    n = np.asarray(nobs, np.float64)
    xb = np.asarray(xbar, np.float64)
    S = np.asarray(sc, np.float64)
    dm = xb - mu_prev
    r = b0 + 0.5 * (S + n * dm * dm)
    tau = G / r
    P = prec0 + n * tau
    m = (prec0 * mu0 + tau * n * xb) / P
    dtau_dmu = tau * n * dm / r
    dmu_dtau = n * (xb - m) / P - z * n / (2.0 * P ** 1.5)
    return dict(tau=tau, P=P, m=m, dtau_dmu=dtau_dmu, dmu_dtau=dmu_dtau)


def ng_bounds(nobs, xbar, sc, prior, mu_start, trace, rtol, e_mu_start=0.0):
    """Bounds on |GPU - oracle| for the normal-gamma chains after the traced
    sweeps.  trace: the oracle's [n_chains, T, 5] (G, kappa, z, tau, mu);
    mu_start: the state mu before the first traced sweep.  Returns dict with
    per-chain bounds "mu", "tau" (final state) and "mom" [n_chains, 4] for the
    increments of (sum mu, sum tau, sum mu^2, sum tau^2) over the sweeps."""
    n_chains, T, _ = trace.shape
    mu_prev = np.asarray(mu_start, np.float64) * np.ones(n_chains)
    e_mu = np.asarray(e_mu_start, np.float64) * np.ones(n_chains)
    e_tau = np.zeros(n_chains)
    mom = np.zeros((n_chains, 4))
    abs_sums = np.zeros((n_chains, 4))
    for t in range(T):
        G, kappa, z, tau, mu = (trace[:, t, i] for i in range(5))
        w = ng_sweep_terms(nobs, xbar, sc, prior, mu_prev, G, z)
        e_tau = np.abs(w["dtau_dmu"]) * e_mu + rtol * np.abs(tau) * (1.0 + kappa)
        e_mu = np.abs(w["dmu_dtau"]) * e_tau + rtol * (np.abs(w["m"]) + np.abs(z) / np.sqrt(w["P"]))
        mom[:, 0] += e_mu
        mom[:, 1] += e_tau
        mom[:, 2] += (2.0 * np.abs(mu) + e_mu) * e_mu + U32 * mu * mu
        mom[:, 3] += (2.0 * np.abs(tau) + e_tau) * e_tau + U32 * tau * tau
        abs_sums += np.stack([np.abs(mu), np.abs(tau), mu * mu, tau * tau], axis=1)
        mu_prev = mu
    mom += SUM_ERR * abs_sums
    return dict(mu=e_mu, tau=e_tau, mom=mom)


def dirichlet_scale(logs, cond):
    """Magnitude the FP32 arithmetic of one Dirichlet row works at, per
    component: theta_k = exp(l_k - M) / sum_j exp(l_j - M) with M = max l,
    so the log-Gammas enter through exponentials (absolute error of l_k and of
    M become relative errors of theta), each log-Gamma l carrying its own
    conditioning.  logs, cond: [..., K]."""
    th = np.exp(logs - np.nanmax(logs, axis=-1, keepdims=True))
    th = th / th.sum(axis=-1, keepdims=True)
    mag = np.abs(logs) + np.nanmax(np.abs(logs), axis=-1, keepdims=True)
    kap = cond + np.nanmax(cond, axis=-1, keepdims=True)
    return th, np.abs(th) * (1.0 + mag + kap)


def lda_mom_bound(trace, rtol):
    """Bound on |GPU - oracle| of the LDA sweep sums of theta (every sweep is
    an independent Dirichlet draw from fixed counts, so errors do not
    propagate): the per-draw bounds summed, plus the compensated sum's own
    error.  trace: the oracle's [n_docs, T, K, 2] (log-Gamma, conditioning)."""
    th, scale = dirichlet_scale(trace[..., 0], trace[..., 1])
    return rtol * scale.sum(axis=1) + SUM_ERR * np.abs(th).sum(axis=1)
