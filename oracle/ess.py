"""Effective sample size and Monte-Carlo standard error of posterior means.

Test infrastructure only (see ``oracle/__init__.py``).

ESS uses Geyer's initial monotone sequence estimator (Geyer 1992, "Practical
Markov chain Monte Carlo"): with rho_k the lag-k autocorrelation, the sums of
adjacent pairs Gamma_m = rho_2m + rho_2m+1 are taken while positive, forced
non-increasing, and tau = -1 + 2 sum_m Gamma_m; ESS = N / tau.  Several
independent chains add their ESS.  The autocovariance is computed with an FFT
(a library primitive); the rest is written out.
"""
import numpy as np


def autocorrelation(x):
    """rho_k for k = 0..N-1 of a 1-D series (biased autocovariance / variance)."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    xc = x - x.mean()
    nfft = 1
    while nfft < 2 * n:
        nfft *= 2
    f = np.fft.rfft(xc, nfft)
    acov = np.fft.irfft(f * np.conj(f), nfft)[:n] / n
    if acov[0] <= 0.0:
        return np.concatenate([[1.0], np.zeros(n - 1)])
    return acov / acov[0]


def ess_geyer(x):
    """ESS of one chain by the initial monotone sequence estimator."""
    x = np.asarray(x, dtype=np.float64)
    n = x.shape[0]
    if n < 4:
        return float(n)
    rho = autocorrelation(x)
    if not np.isfinite(rho).all() or np.var(x) == 0.0:
        return float(n)
    tau_sum = 0.0
    prev = np.inf
    m = 0
    while 2 * m + 1 < n:
        gam = rho[2 * m] + rho[2 * m + 1]
        if gam <= 0.0:
            break
        gam = min(gam, prev)
        tau_sum += gam
        prev = gam
        m += 1
    tau = -1.0 + 2.0 * tau_sum
    tau = max(tau, 1.0 / np.log10(max(n, 10)))  # guard against tau ~ 0 on anticorrelated series
    return float(n / tau)


def ess_chains(draws):
    """ESS of one coordinate over independent chains: draws shape (chains, N)."""
    draws = np.asarray(draws, dtype=np.float64)
    return float(sum(ess_geyer(d) for d in draws))


def mcse_mean(draws):
    """Monte-Carlo standard error of the pooled mean: sd / sqrt(ESS)."""
    draws = np.asarray(draws, dtype=np.float64)
    ess = ess_chains(draws)
    return float(np.std(draws) / np.sqrt(ess)), ess
