"""Seeded synthetic inputs for the FFA period search.

This module only draws random numbers and lays out test series; it holds none
of the search's arithmetic (no folding, detrending or scoring), so both the
CUDA path and the CPU oracle can be fed from it.

Recipes (all float32, seeded with numpy's PCG64):

* white noise N(0, 1);
* red noise: a stationary AR(1) process r_t = a r_{t-1} + e_t with marginal
  standard deviation ``red_std`` (so e_t has std red_std * sqrt(1 - a^2));
* a pulsar: a train of Gaussian pulses whose FWHM is a fraction of the period
  (Eq. 12 relates the FWHM to the Gaussian's c), with a uniformly drawn phase,
  scaled so that the pulse train's L2 norm equals the requested matched-filter
  S/N in unit white noise.

The named workloads mirror the shapes of the paper's survey data (HTRU-S
LowLat style 64 us sampling, Section 4) and its Fig. 1 style synthetic
pulsars; the real survey data is not available, so these stand in for it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "gaussian_pulse_train",
    "red_noise",
    "make_series",
    "SeriesSpec",
    "plain_series",
    "survey_series",
    "batch_specs",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian_pulse_train(n: int, period: float, fwhm_frac: float, phase_frac: float,
                         snr_l2: float) -> np.ndarray:
    """Pulse train in samples: Gaussian pulses at t0 + j*period, FWHM = fwhm_frac*period.

    Only the nearest pulse to each sample is evaluated (the pulses are far
    narrower than the period).  Returned as float64, L2 norm = snr_l2.
    """
    if n <= 0:
        return np.zeros(0)
    c = fwhm_frac * period / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    t = np.arange(n, dtype=np.float64)
    t0 = phase_frac * period
    d = np.mod(t - t0, period)
    d = np.minimum(d, period - d)
    s = np.exp(-0.5 * (d / c) ** 2)
    norm = float(np.sqrt(np.sum(s * s)))
    if norm > 0:
        s *= snr_l2 / norm
    return s


def red_noise(rng: np.random.Generator, n: int, coef: float, std: float) -> np.ndarray:
    """Stationary AR(1) series with lag-1 coefficient ``coef`` and marginal std ``std``."""
    from scipy.signal import lfilter

    e = rng.standard_normal(n) * (std * math.sqrt(1.0 - coef * coef))
    r_prev = rng.standard_normal() * std
    out, _ = lfilter([1.0], [1.0, -coef], e, zi=[coef * r_prev])
    return out


@dataclass
class SeriesSpec:
    """One synthetic series: length, noise and an optional pulsar."""

    n: int
    seed: int
    red_coef: float = 0.0
    red_std: float = 0.0
    pulsar_period: float | None = None    # samples
    pulsar_fwhm_frac: float = 0.03
    pulsar_snr: float = 0.0
    pulsar_phase: float | None = None     # drawn from the seed when None
    extras: dict = field(default_factory=dict)


def make_series(spec: SeriesSpec) -> np.ndarray:
    """Materialise a SeriesSpec as a float32 array."""
    rng = _rng(spec.seed)
    x = rng.standard_normal(spec.n)
    if spec.red_std > 0.0:
        x += red_noise(rng, spec.n, spec.red_coef, spec.red_std)
    if spec.pulsar_period is not None and spec.pulsar_snr > 0.0:
        phase = spec.pulsar_phase if spec.pulsar_phase is not None else float(rng.random())
        x += gaussian_pulse_train(spec.n, spec.pulsar_period, spec.pulsar_fwhm_frac, phase,
                                  spec.pulsar_snr)
    return x.astype(np.float32)


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------

PLAIN = dict(n=65536, tsamp=2.048e-3, p0_min=256, p0_max=512, widths=(1, 2, 4, 8, 16),
             pulsar_period_s=0.8, fwhm_frac=0.03, snr=15.0, seed=1)

SURVEY = dict(n=1 << 26, tsamp=64e-6, period_min_s=1.0, period_max_s=30.0, duty=0.1,
              red_coef=0.999, red_std=0.3, pulsar_period_s=7.3, fwhm_frac=0.02, snr=12.0,
              seed=2)


# False-alarm statistics (Section 4.3): 26 white-noise series of the survey's
# shape searched from 1 to 20 s at D0 = 32, about 10^8 trials in all.
NOISE = dict(n=1 << 26, tsamp=64e-6, downsample0=32, period_min_s=1.0, period_max_s=20.0,
             n_series=26, seed=100)


def white_series(seed: int, n: int = NOISE["n"]) -> np.ndarray:
    """N(0, 1) float32 samples (the noise-only series of the false-alarm workload)."""
    return make_series(SeriesSpec(n=n, seed=seed))


def plain_series(seed: int = PLAIN["seed"], n: int = PLAIN["n"]) -> np.ndarray:
    """White noise + 0.8 s Gaussian pulsar (3 % FWHM, S/N 15) sampled at 2.048 ms."""
    p = PLAIN["pulsar_period_s"] / PLAIN["tsamp"]
    return make_series(SeriesSpec(n=n, seed=seed, pulsar_period=p,
                                  pulsar_fwhm_frac=PLAIN["fwhm_frac"],
                                  pulsar_snr=PLAIN["snr"]))


def survey_series(seed: int = SURVEY["seed"], n: int = SURVEY["n"]) -> np.ndarray:
    """White + AR(1) red noise + 7.3 s pulsar (2 % FWHM, S/N 12) at 64 us."""
    p = SURVEY["pulsar_period_s"] / SURVEY["tsamp"]
    return make_series(SeriesSpec(n=n, seed=seed, red_coef=SURVEY["red_coef"],
                                  red_std=SURVEY["red_std"], pulsar_period=p,
                                  pulsar_fwhm_frac=SURVEY["fwhm_frac"],
                                  pulsar_snr=SURVEY["snr"]))


def batch_specs(count: int, n_lo: int, n_hi: int, seed: int, tsamp: float = 512e-6,
                pulsar_frac: float = 0.05, period_range_s=(0.5, 20.0),
                red_coef: float = 0.999, red_std: float = 0.3) -> list[SeriesSpec]:
    """Uneven-length DM-trial batch: lengths uniform in [n_lo, n_hi], a fraction with pulsars."""
    rng = _rng(seed)
    lengths = rng.integers(n_lo, n_hi + 1, size=count)
    n_psr = int(round(pulsar_frac * count))
    with_psr = set(rng.choice(count, size=n_psr, replace=False).tolist()) if n_psr else set()
    specs = []
    for i in range(count):
        spec = SeriesSpec(n=int(lengths[i]), seed=seed * 100003 + i, red_coef=red_coef,
                          red_std=red_std)
        if i in with_psr:
            spec.pulsar_period = float(rng.uniform(*period_range_s)) / tsamp
            spec.pulsar_fwhm_frac = float(rng.uniform(0.01, 0.05))
            spec.pulsar_snr = float(rng.uniform(8.0, 20.0))
        specs.append(spec)
    return specs
