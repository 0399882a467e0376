"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds no arithmetic of the solver; it only draws permeability
fields and sources.  The paper's own fields (Model 1 channels and inclusions,
Model 2, SPE10) exist only as figures, so seeded stand-ins of the same
structure are used:

* channel field: horizontal bands two cells wide at non-overlapping rows,
  about n/16 of them, each covering a random x-extent of length in
  [n/2, n] at a random start; kappa = ``contrast`` in the bands and the
  background elsewhere (channels plus isolated inclusions where bands end);
* Gaussian field: log kappa with variance 4 and squared-exponential
  covariance exp(-r^2 / (2 l^2)), l = 0.05, sampled by FFT on the 2n x 2n
  periodic embedding of the unit square;
* sources: quarter five-spot (+1 in cell (0, 0), -1 in cell (n-1, n-1)) or
  random point source/sink pairs, as cell-average densities.

All generators use numpy's PCG64 stream (``default_rng``) with explicit seeds.
Arrays are (n, n) float64 indexed [j, i] (x fastest when flattened).
"""

import numpy as np


def channel_mask(n, seed, count=None, width=2):
    rng = np.random.default_rng(seed)
    count = max(1, n // 16) if count is None else count
    mask = np.zeros((n, n), dtype=bool)
    taken = np.zeros(n + 2, dtype=bool)
    placed, tries = 0, 0
    while placed < count and tries < 100 * count:
        tries += 1
        r = int(rng.integers(0, n - width + 1))
        # keep one free row between bands so that bands never merge
        if taken[max(0, r - 1): r + width + 1].any():
            continue
        length = int(rng.integers(n // 2, n + 1))
        x0 = int(rng.integers(0, n - length + 1))
        mask[r: r + width, x0: x0 + length] = True
        taken[r: r + width] = True
        placed += 1
    return mask


def gaussian_log_field(n, seed, variance=4.0, corr_len=0.05):
    """Stationary Gaussian field on the n x n cell centres of the unit square
    by circulant embedding on a 2n x 2n torus of side 2."""
    rng = np.random.default_rng(seed)
    m = 2 * n
    d = np.minimum(np.arange(m), m - np.arange(m)) / n
    r2 = d[:, None] ** 2 + d[None, :] ** 2
    cov = variance * np.exp(-r2 / (2.0 * corr_len ** 2))
    lam = np.real(np.fft.fft2(cov))
    lam = np.maximum(lam, 0.0)
    xi = rng.standard_normal((m, m)) + 1j * rng.standard_normal((m, m))
    field = np.fft.fft2(np.sqrt(lam / (m * m)) * xi)
    return np.real(field)[:n, :n].copy()


def channel_field(n, contrast, seed, background=None):
    """kappa = contrast in the channels, ``background`` (default 1) elsewhere."""
    kappa = np.ones((n, n)) if background is None else np.array(background, dtype=np.float64)
    kappa = kappa.copy()
    kappa[channel_mask(n, seed)] = contrast
    return kappa


def grf_channel_field(n, contrast, seed):
    """exp(Gaussian field) background with channels at ``contrast``."""
    return channel_field(n, contrast, seed + 1, background=np.exp(gaussian_log_field(n, seed)))


def quarter_five_spot(n):
    f = np.zeros((n, n))
    f[0, 0] = 1.0
    f[n - 1, n - 1] = -1.0
    return f


def random_pairs(n, npairs, seed):
    """npairs point source/sink pairs at distinct cells, +1 / -1 densities."""
    rng = np.random.default_rng(seed)
    cells = rng.choice(n * n, size=2 * npairs, replace=False)
    f = np.zeros(n * n)
    f[cells[:npairs]] = 1.0
    f[cells[npairs:]] = -1.0
    return f.reshape(n, n)


def lognormal_field(n, seed, sigma=1.0):
    """Cell-wise independent log-normal permeability (for small parity cases)."""
    rng = np.random.default_rng(seed)
    return np.exp(sigma * rng.standard_normal((n, n)))


def mlp_init_params(din, dout, hidden, seed):
    """Initial weights of the three-layer perceptron as one flat float32
    vector in the layout W1 (hidden x din), b1, W2 (hidden x hidden), b2,
    W3 (dout x hidden), b3: He-normal weights (std sqrt(2 / fan_in)), zero
    biases, the output layer scaled by 1/2."""
    rng = np.random.default_rng(seed)
    parts = [rng.standard_normal(hidden * din) * np.sqrt(2.0 / din), np.zeros(hidden),
             rng.standard_normal(hidden * hidden) * np.sqrt(2.0 / hidden), np.zeros(hidden),
             0.5 * rng.standard_normal(dout * hidden) * np.sqrt(2.0 / hidden), np.zeros(dout)]
    return np.concatenate(parts).astype(np.float32)


def sample_order(nsamples, nsteps, batch, seed):
    """Row indices of the training batches: consecutive random permutations of
    range(nsamples), cut into nsteps batches of ``batch`` (int32)."""
    rng = np.random.default_rng(seed)
    need = nsteps * batch
    reps = -(-need // max(nsamples, 1))
    return np.concatenate([rng.permutation(nsamples) for _ in range(reps)])[:need].astype(np.int32)
