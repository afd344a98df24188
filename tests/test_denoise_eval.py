"""The growth-rate estimator used to compare runs (CPU): on synthetic histories
with a noise floor, exponential growth and saturation it recovers the rate."""
import numpy as np

from paper_2501_14795_gb300 import denoise as dn


def _history(gamma, floor, sat, steps, dt, seed, noise=0.3):
    rng = np.random.Generator(np.random.PCG64(seed))
    t = (np.arange(steps) + 1) * dt
    amp = np.minimum(1e-6 * np.exp(gamma * t), sat)          # growth, then saturation
    amp = np.sqrt(amp ** 2 + floor ** 2)                       # on top of a noise floor
    amp = amp * np.exp(noise * rng.standard_normal(steps) * (amp < 10 * floor))
    return amp ** 2


def test_mode_growth_rate_recovers_the_rate():
    dt, steps = 0.05, 600
    for gamma, floor, sat, seed in ((0.3, 1e-5, 1.0, 1), (0.25, 1e-4, 1e-1, 2),
                                    (0.34, 3e-6, 1.0, 3)):
        p1 = _history(gamma, floor, sat, steps, dt, seed)
        power = np.stack([np.full(steps, 1e-12), p1, 0.5 * p1, 1e-12 * np.ones(steps)], axis=1)
        g, (j0, j1) = dn.mode_growth_rate(power, dt, 1, band=0)
        assert abs(g - gamma) < 0.05 * gamma, (gamma, g, j0, j1)


def test_kinetic_rate_of_the_tabulated_case():
    # warm beams vd = +-0.2, vt = 0.1 in a box of 6.4: fastest mode (m = 3) rate 0.163
    assert abs(dn.kinetic_growth_rate(0.2, 0.1, 6.4, m_max=5) - 0.1634) < 2e-3
