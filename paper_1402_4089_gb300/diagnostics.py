"""Effective sample size of sampler output, for the throughput report (ESS/s).

Host-side numpy, applied to samples copied back from the device; not part of
the sampling path.  The estimator is Geyer's initial monotone sequence (Geyer,
"Practical Markov chain Monte Carlo", Statistical Science 1992), vectorised
over coordinates: with rho_t the lag-t autocorrelation of a coordinate's
chain, the adjacent-pair sums G_m = rho_2m + rho_2m+1 are kept while they stay
positive and are made non-increasing; the integrated autocorrelation time is
tau = 2 sum_m G_m - 1 and ESS = N / tau.  Independent chains add their ESS.
"""
import numpy as np


def _acf(x):
    """Autocorrelations along axis 0 of x [N, M] (biased autocovariance / variance)."""
    n = x.shape[0]
    xc = x - x.mean(axis=0, keepdims=True)
    nfft = 1 << int(np.ceil(np.log2(2 * n)))
    f = np.fft.rfft(xc, n=nfft, axis=0)
    acov = np.fft.irfft(f * np.conj(f), n=nfft, axis=0)[:n] / n
    var = acov[0]
    safe = np.where(var > 0, var, 1.0)
    rho = acov / safe
    rho[:, var <= 0] = 0.0
    rho[0, var <= 0] = 1.0
    return rho


def ess(samples):
    """ESS per coordinate of draws [N, chains, ...] (or [N, ...] for one chain)."""
    x = np.asarray(samples, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
    n = x.shape[0]
    if x.ndim == 2:
        x = x[:, None, :]
    flat = x.reshape(n, x.shape[1], -1)
    total = np.zeros(flat.shape[2])
    for c in range(flat.shape[1]):
        rho = _acf(flat[:, c, :])
        m = n // 2
        pairs = rho[0:2 * m:2] + rho[1:2 * m:2]                  # G_0 .. G_{m-1}
        pos = pairs > 0
        # initial positive sequence: stop at the first non-positive pair
        keep = np.cumprod(pos, axis=0).astype(bool)
        mono = np.minimum.accumulate(np.where(keep, pairs, 0.0), axis=0)
        tau = 2.0 * np.where(keep, mono, 0.0).sum(axis=0) - 1.0
        tau = np.maximum(tau, 1.0 / n)
        total += n / tau
    return total.reshape(x.shape[2:]) if x.ndim > 2 else total
